// One step of the pivoted Hessenberg process with its sketch (Sec. 3.1 Eq.
// Hessenberg_s; Algorithm 1 lines 10-19 in the square form, A in place of
// the A^T the listing prints on line 9):
//
//   k_pivot_solve   append row p_j of L_p; h = L_p^{-1} u(p_1..p_j) in FP64
//                   (the sequential elimination H(i,j) = u(p_i),
//                   u -= H(i,j) v_i is this forward substitution because
//                   v_c(p_i) = 0 for c > i and v_i(p_i) = 1)
//   k_update        u -= V_j h, u(p_i) = 0, argmax |u| over the rest
//   k_normalize     H(j+1,j) = u(p_{j+1}); v_{j+1} = u / H(j+1,j) rounded to
//                   the storage type; S v_{j+1} (and S of the unrounded
//                   vector) accumulated exactly in 64-bit fixed point.
//
// Every kernel reads the step index j from device memory, so one captured
// step can be replayed for any j; the last CTA of k_normalize advances it.
#include "ipf_internal.cuh"

namespace ipf {

namespace {

template <class T> struct Vec16 { static constexpr int n = 16 / sizeof(T); };

// ------------------------------------------------------------------------
// b (nrhs x n, RHS-major) -> interleaved work vector w (element i*B + r)
// ------------------------------------------------------------------------
template <class Acc>
__global__ void k_load_rhs(const float* __restrict__ b, Acc* __restrict__ w, long long n, int B) {
    const long long N = n * B;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N;
         e += (long long)gridDim.x * blockDim.x) {
        const long long i = e / B;
        const int r = (int)(e - i * B);
        w[e] = (Acc)b[(long long)r * n + i];
    }
}

// ------------------------------------------------------------------------
// pivot-block forward substitution, one CTA per RHS
// ------------------------------------------------------------------------
template <class T, class Acc>
__global__ void __launch_bounds__(256) k_pivot_solve(Geom g, Bufs bf) {
    extern __shared__ unsigned char smem_raw[];
    const int r = blockIdx.x;
    DevState* st = bf.st;
    if (st->status[r] != IPF_OK) return;
    const int j = st->j;
    if (j < 0 || j >= g.k_max) return;
    const int K1 = g.k_max + 1;
    const int B = g.B;
    const T* V = (const T*)bf.V;
    const Acc* w = (const Acc*)bf.w;
    Acc* LpT = (Acc*)bf.LpT + (size_t)r * K1 * K1;
    const int* piv = bf.piv + (size_t)r * K1;

    // smem: x[0..j] (double), then L strictly-lower packed by column (Acc)
    double* s_x = (double*)smem_raw;
    Acc* s_L = (Acc*)(s_x + ((K1 + 1) & ~1));

    // row j of L_p: v_c(p_j), c < j (exact copies of the stored values)
    const long long pj = (long long)piv[j] * B + r;
    for (int c = threadIdx.x; c < j; c += blockDim.x) {
        const Acc val = to_acc(V[(size_t)c * g.ldv + pj]);
        LpT[(size_t)c * K1 + j] = val;
    }
    if (threadIdx.x == 0) LpT[(size_t)j * K1 + j] = (Acc)1;
    __syncthreads();
    // packed column c holds rows c+1..j at offset c*j - c*(c-1)/2
    for (int c = 0; c < j; ++c) {
        const int off = c * j - (c * (c - 1)) / 2;
        for (int i = c + 1 + threadIdx.x; i <= j; i += blockDim.x)
            s_L[off + (i - c - 1)] = LpT[(size_t)c * K1 + i];
    }
    for (int i = threadIdx.x; i <= j; i += blockDim.x)
        s_x[i] = (double)w[(long long)piv[i] * B + r];
    // forward substitution, column oriented: x_i -= L(i,c) x_c for i > c
    for (int c = 0; c < j; ++c) {
        __syncthreads();
        const double xc = s_x[c];
        const int off = c * j - (c * (c - 1)) / 2;
        for (int i = c + 1 + threadIdx.x; i <= j; i += blockDim.x)
            s_x[i] = fma(-(double)s_L[off + (i - c - 1)], xc, s_x[i]);
    }
    __syncthreads();
    double* Hc = bf.H + (size_t)r * K1 * g.k_max + (size_t)K1 * j;
    Acc* coef = (Acc*)bf.coef;
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
        Hc[i] = s_x[i];
        coef[(size_t)i * B + r] = (Acc)s_x[i];
    }
}

// ------------------------------------------------------------------------
// u -= V_j h ; u(pivots) = 0 ; argmax keys.  Acc = float.
// With g.want_z (nrhs <= 4) the incoming u = A v_j is also sketched,
// z_j = S u (Algorithm 1 line 11), exactly, while the V_j loads are in
// flight: shared split counters [B][m_s], folded every kFoldEvery elements.
// ------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(256) k_update_f(Geom g, Bufs bf, SketchParams sp) {
    constexpr int VEC = Vec16<T>::n;
    extern __shared__ unsigned char smem_raw[];
    const int B = g.B;
    const int K1 = g.k_max + 1;
    // smem: wide [B*m] int64, hi [B*m], lo [B*m] int32 (only with z), coefficients
    const int zc = g.want_z ? B * g.m_s : 0;
    long long* s_wide = (long long*)smem_raw;
    int* s_hi = (int*)(s_wide + zc);
    int* s_lo = s_hi + zc;
    float* s_coef = (float*)(s_lo + zc);
    __shared__ unsigned long long s_key[kMaxRhs];
    __shared__ int s_ok[kMaxRhs];
    DevState* st = bf.st;
    const int j = st->j;
    if (j >= g.k_max) return;            // never past the last basis column
    const int nc = j + 1;               // coefficients h_0..h_j (none during init)
    const bool do_z = g.want_z && j >= 0;
    const float* coef = (const float*)bf.coef;
    for (int t = threadIdx.x; t < nc * B; t += blockDim.x) s_coef[t] = coef[t];
    if (do_z)
        for (int t = threadIdx.x; t < zc; t += blockDim.x) { s_wide[t] = 0; s_hi[t] = 0; s_lo[t] = 0; }
    if (threadIdx.x < B) {
        s_key[threadIdx.x] = 0ull;
        s_ok[threadIdx.x] = st->status[threadIdx.x] == IPF_OK;
    }
    __syncthreads();
    if (B == 1 && !s_ok[0]) return;

    const T* V = (const T*)bf.V;
    float* w = (float*)bf.w;
    unsigned long long best[VEC];
#pragma unroll
    for (int q = 0; q < VEC; ++q) best[q] = 0ull;

    const long long stride = (long long)gridDim.x * blockDim.x * VEC;
    const long long base0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * VEC;
    const int fold_rounds = kFoldEvery / (256 * VEC);
    int round = 0;
    for (long long bstart = (long long)blockIdx.x * blockDim.x * VEC; bstart < g.N; bstart += stride) {
        const long long base = bstart + (long long)threadIdx.x * VEC;
        const bool live = base < g.N;
        float acc[VEC];
#pragma unroll
        for (int q = 0; q < VEC; ++q) acc[q] = 0.f;
        int c = 0;
        uint4 raw[4];
        if (live) {
            const float4* wp = (const float4*)(w + base);
#pragma unroll
            for (int q = 0; q < VEC / 4; ++q) {
                const float4 t4 = wp[q];
                acc[4 * q] = t4.x; acc[4 * q + 1] = t4.y; acc[4 * q + 2] = t4.z; acc[4 * q + 3] = t4.w;
            }
            if (nc >= 4) {
#pragma unroll
                for (int u = 0; u < 4; ++u) raw[u] = __ldcs((const uint4*)(V + (size_t)u * g.ldv + base));
            }
            if (do_z) {
                // z_j = S u for the incoming u = A v_j
#pragma unroll
                for (int q = 0; q < VEC; ++q) {
                    const long long e = base + q;
                    const long long i = (B == 1) ? e : e / B;
                    const int rr = (B == 1) ? 0 : (int)(e & (B - 1));
                    if (e < g.N && s_ok[rr]) {
                        const long long f = fixed_from(acc[q], g.Fz);
                        if (f) {
                            int rows[16];
                            unsigned neg;
                            if (sp.zeta == 8) sketch_column8(sp, i, rows, &neg);
                            else sketch_column(sp, i, rows, &neg);
#pragma unroll
                            for (int t = 0; t < 16; ++t)
                                if (t < sp.zeta)
                                    split_add(s_hi + rr * g.m_s, s_lo + rr * g.m_s, rows[t], ((neg >> t) & 1u) ? -f : f);
                        }
                    }
                }
            }
            for (; c + 4 <= nc; c += 4) {
                uint4 nxt[4];
                const bool more = c + 8 <= nc;
                if (more) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) nxt[u] = __ldcs((const uint4*)(V + (size_t)(c + 4 + u) * g.ldv + base));
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const T* vv = (const T*)&raw[u];
#pragma unroll
                    for (int q = 0; q < VEC; ++q) {
                        const int rr = (B == 1) ? 0 : (int)((base + q) & (B - 1));
                        acc[q] = fmaf(-s_coef[(c + u) * B + rr], to_acc(vv[q]), acc[q]);
                    }
                }
                if (more) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) raw[u] = nxt[u];
                }
            }
            for (; c < nc; ++c) {
                const uint4 r1 = __ldcs((const uint4*)(V + (size_t)c * g.ldv + base));
                const T* vv = (const T*)&r1;
#pragma unroll
                for (int q = 0; q < VEC; ++q) {
                    const int rr = (B == 1) ? 0 : (int)((base + q) & (B - 1));
                    acc[q] = fmaf(-s_coef[c * B + rr], to_acc(vv[q]), acc[q]);
                }
            }
            const unsigned bits = bf.ispiv[base >> 5] >> (unsigned)(base & 31);
#pragma unroll
            for (int q = 0; q < VEC; ++q) {
                if ((bits >> q) & 1u) acc[q] = 0.f;
                const long long e = base + q;
                const int rr = (B == 1) ? 0 : (int)(e & (B - 1));
                if (e < g.N && s_ok[rr]) {
                    const unsigned long long k = argmax_key(acc[q], (unsigned)(e / B));
                    best[q] = k > best[q] ? k : best[q];
                }
            }
            float4* wo = (float4*)(w + base);
#pragma unroll
            for (int q = 0; q < VEC / 4; ++q)
                wo[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
        }
        if (do_z && ++round == fold_rounds) {
            __syncthreads();
            split_fold(s_hi, s_lo, s_wide, zc);
            __syncthreads();
            round = 0;
        }
    }
    if (do_z) {
        __syncthreads();
        split_fold(s_hi, s_lo, s_wide, zc);
        __syncthreads();
        for (int t = threadIdx.x; t < zc; t += blockDim.x) {
            const int rr = t / g.m_s, row = t - rr * g.m_s;
            if (s_wide[t] && s_ok[rr])
                atomicAdd((unsigned long long*)&bf.accSZ[((size_t)rr * g.k_max + j) * g.m_s + row],
                          (unsigned long long)s_wide[t]);
        }
    }
    // reduce keys: per RHS rr = (base0 + q) mod B (same for every grid-stride pass)
    if (B == 1) {
        unsigned long long k = best[0];
#pragma unroll
        for (int q = 1; q < VEC; ++q) k = best[q] > k ? best[q] : k;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, k, off);
            k = o > k ? o : k;
        }
        if ((threadIdx.x & 31) == 0 && k) atomicMax(&s_key[0], k);
    } else {
#pragma unroll
        for (int q = 0; q < VEC; ++q)
            if (best[q]) atomicMax(&s_key[(int)((base0 + q) & (B - 1))], best[q]);
    }
    __syncthreads();
    if (threadIdx.x < B && s_key[threadIdx.x])
        atomicMax(&st->key[(j + 1) & 1][threadIdx.x], s_key[threadIdx.x]);
    (void)K1;
}

// ------------------------------------------------------------------------
// F64 storage (nrhs == 1): u -= V_j h in double; max |u| bits, then the
// lowest row attaining it in a second pass.
// ------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_update_d(Geom g, Bufs bf) {
    extern __shared__ unsigned char smem_raw[];
    double* s_coef = (double*)smem_raw;
    __shared__ unsigned long long s_max;
    DevState* st = bf.st;
    if (st->status[0] != IPF_OK) return;
    const int j = st->j;
    if (j >= g.k_max) return;
    const int nc = j + 1;
    const double* coef = (const double*)bf.coef;
    for (int t = threadIdx.x; t < nc; t += blockDim.x) s_coef[t] = coef[t];
    if (threadIdx.x == 0) s_max = 0ull;
    __syncthreads();
    const double* V = (const double*)bf.V;
    double* w = (double*)bf.w;
    unsigned long long best = 0ull;
    const long long stride = (long long)gridDim.x * blockDim.x * 2;
    for (long long base = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * 2; base < g.N; base += stride) {
        double2 a = *(const double2*)(w + base);
        for (int c = 0; c < nc; ++c) {
            const double2 v = __ldcs((const double2*)(V + (size_t)c * g.ldv + base));
            a.x = fma(-s_coef[c], v.x, a.x);
            a.y = fma(-s_coef[c], v.y, a.y);
        }
        const unsigned bits = bf.ispiv[base >> 5] >> (unsigned)(base & 31);
        if (bits & 1u) a.x = 0.0;
        if (bits & 2u) a.y = 0.0;
        *(double2*)(w + base) = a;
        const unsigned long long bx = (unsigned long long)__double_as_longlong(fabs(a.x));
        const unsigned long long by = (unsigned long long)__double_as_longlong(fabs(a.y));
        if (base < g.N && bx > best) best = bx;
        if (base + 1 < g.N && by > best) best = by;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, best, off);
        best = o > best ? o : best;
    }
    if ((threadIdx.x & 31) == 0 && best) atomicMax(&s_max, best);
    __syncthreads();
    if (threadIdx.x == 0 && s_max) atomicMax(&st->maxbits[(j + 1) & 1], s_max);
}

__global__ void k_argmin_d(Geom g, Bufs bf) {
    DevState* st = bf.st;
    if (st->status[0] != IPF_OK) return;
    const int kb = (st->j + 1) & 1;
    const unsigned long long mb = st->maxbits[kb];
    const double* w = (const double*)bf.w;
    unsigned long long lo = ~0ull;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < g.N;
         e += (long long)gridDim.x * blockDim.x) {
        if ((unsigned long long)__double_as_longlong(fabs(w[e])) == mb) { lo = (unsigned long long)e; break; }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, lo, off);
        lo = o < lo ? o : lo;
    }
    if ((threadIdx.x & 31) == 0 && lo != ~0ull) atomicMin(&st->minidx[kb], lo);
}

// ------------------------------------------------------------------------
// normalise + store + sketch.  Bg RHS per CTA (grid.y = B / Bg).  want_sw
// (initialisation only) also sketches the unrounded v_1 = b / beta, which
// gives c = S b = beta * S v_1.  Float modes use split int32 counters
// (2^-34 quantum); F64 storage uses int64 shared atomics with 2^-F,
// F = 61 - ceil(log2(n+1)).
// ------------------------------------------------------------------------
template <class T, class Acc>
__global__ void __launch_bounds__(256) k_normalize(Geom g, Bufs bf, SketchParams sp, int want_sw, int Bg) {
    extern __shared__ unsigned char smem_raw[];
    constexpr bool f64 = sizeof(Acc) == 8;
    const int nacc = want_sw ? 2 : 1;
    const int cnt = nacc * Bg * sp.m_s;          // counters: [acc][rl][row]
    long long* s_wide = (long long*)smem_raw;
    int* s_hi = (int*)(s_wide + cnt);
    int* s_lo = s_hi + cnt;
    __shared__ long long s_prow[kMaxRhs];
    __shared__ Acc s_hval[kMaxRhs];
    __shared__ int s_ok[kMaxRhs];
    __shared__ int s_code[kMaxRhs];
    __shared__ bool s_last;
    DevState* st = bf.st;
    const int j = st->j;
    const int jn = j + 1;                 // index of the new basis vector
    if (jn > g.k_max) return;             // a step past k_max writes nothing
    const int kb = jn & 1;
    const int B = g.B;
    const int r0 = blockIdx.y * Bg;
    const Acc* w = (const Acc*)bf.w;

    if (threadIdx.x < Bg) {
        const int r = r0 + threadIdx.x;
        int ok = st->status[r] == IPF_OK;
        int code = IPF_OK;
        long long row = 0;
        Acc hv = (Acc)0;
        if (ok) {
            bool zero;
            if (f64) {
                zero = st->maxbits[kb] == 0ull;
                row = zero ? 0 : (long long)st->minidx[kb];
            } else {
                const unsigned long long key = st->key[kb][r];
                zero = key == 0ull || key_absval(key) == 0.f;
                row = zero ? 0 : (long long)key_row(key);
            }
            if (zero) {
                ok = 0; code = IPF_BREAKDOWN;
            } else {
                hv = w[row * B + r];
                if (!isfinite((double)hv)) { ok = 0; code = IPF_ERR_NONFINITE; }
                else if (hv == (Acc)0) { ok = 0; code = IPF_BREAKDOWN; }
            }
        } else {
            code = st->status[r];
        }
        s_prow[threadIdx.x] = row;
        s_hval[threadIdx.x] = hv;
        s_ok[threadIdx.x] = ok;
        s_code[threadIdx.x] = code;
    }
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
        s_wide[t] = 0;
        if (!f64) { s_hi[t] = 0; s_lo[t] = 0; }
    }
    __syncthreads();

    bool any_ok = false;
    for (int q = 0; q < Bg; ++q) any_ok |= s_ok[q] != 0;
    const int F = g.F;
    if (any_ok) {
        T* vout = (T*)bf.V + (size_t)jn * g.ldv;
        const long long total = g.n * Bg;      // (i, rl) pairs this CTA's group covers
        const long long stride = (long long)gridDim.x * blockDim.x;
        const int fold_rounds = kFoldEvery / 256;
        int round = 0;
        for (long long t0 = blockIdx.x * (long long)blockDim.x; t0 < total; t0 += stride) {
            const long long t = t0 + threadIdx.x;
            const long long i = t / Bg;
            const int rl = (int)(t - i * Bg);
            if (t < total && s_ok[rl]) {
                const long long e = i * B + r0 + rl;
                const Acc v = (i == s_prow[rl]) ? (Acc)1 : w[e] / s_hval[rl];
                const T vs = from_acc<T>(v);
                vout[e] = vs;
                const long long fv = fixed_from(to_acc(vs), F);
                const long long fw = want_sw ? fixed_from(v, F) : 0;
                if (fv || fw) {
                    int rows[16];
                    unsigned neg;
                    if (sp.zeta == 8) sketch_column8(sp, i, rows, &neg);
                    else sketch_column(sp, i, rows, &neg);
                    const int o1 = rl * sp.m_s, o2 = (Bg + rl) * sp.m_s;
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        if (q < sp.zeta) {
                            const bool ng = (neg >> q) & 1u;
                            if (f64) {
                                if (fv) atomicAdd((unsigned long long*)&s_wide[o1 + rows[q]], (unsigned long long)(ng ? -fv : fv));
                                if (fw) atomicAdd((unsigned long long*)&s_wide[o2 + rows[q]], (unsigned long long)(ng ? -fw : fw));
                            } else {
                                if (fv) split_add(s_hi, s_lo, o1 + rows[q], ng ? -fv : fv);
                                if (fw) split_add(s_hi, s_lo, o2 + rows[q], ng ? -fw : fw);
                            }
                        }
                    }
                }
            }
            if (!f64 && ++round == fold_rounds) {
                __syncthreads();
                split_fold(s_hi, s_lo, s_wide, cnt);
                __syncthreads();
                round = 0;
            }
        }
    }
    __syncthreads();
    if (!f64) {
        split_fold(s_hi, s_lo, s_wide, cnt);
        __syncthreads();
    }
    const int K1 = g.k_max + 1;
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
        const int a = t / (Bg * sp.m_s);
        const int rem = t - a * Bg * sp.m_s;
        const int rl = rem / sp.m_s, row = rem - rl * sp.m_s;
        if (!s_ok[rl] || !s_wide[t]) continue;
        const size_t dst = ((size_t)(r0 + rl) * K1 + jn) * sp.m_s + row;
        atomicAdd((unsigned long long*)&((a == 0) ? bf.accSV : bf.accSW)[dst], (unsigned long long)s_wide[t]);
    }
    // bookkeeping for this CTA's RHS group (one CTA per group)
    if (blockIdx.x == 0 && threadIdx.x < Bg) {
        const int rl = threadIdx.x, r = r0 + rl;
        if (s_ok[rl]) {
            const long long row = s_prow[rl];
            bf.piv[(size_t)r * K1 + jn] = (int)row;
            if (jn == 0) st->beta[r] = (double)s_hval[rl];
            else bf.H[(size_t)r * K1 * g.k_max + (size_t)K1 * j + jn] = (double)s_hval[rl];
            const long long e = row * B + r;
            atomicOr(&bf.ispiv[e >> 5], 1u << (unsigned)(e & 31));
            st->kdone[r] = jn;
        } else if (st->status[r] == IPF_OK) {
            st->status[r] = s_code[rl];
            st->kdone[r] = (s_code[rl] == IPF_BREAKDOWN) ? jn : (jn > 0 ? jn - 1 : 0);
            if (jn == 0) st->beta[r] = 0.0;
        }
        st->key[kb ^ 1][r] = 0ull;
        if (f64 && rl == 0) { st->maxbits[kb ^ 1] = 0ull; st->minidx[kb ^ 1] = ~0ull; }
    }
    // last CTA advances the step counter
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned total = gridDim.x * gridDim.y;
        s_last = atomicAdd(&st->ctr, 1u) == total - 1;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        st->j = jn;
        st->ctr = 0u;
        __threadfence();
    }
}

// ------------------------------------------------------------------------
// standalone sketch y = S x (one RHS, FP32 input): max |x| then exact sums
// ------------------------------------------------------------------------
__global__ void k_absmax(const float* __restrict__ x, long long n, unsigned* out) {
    unsigned m = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const unsigned u = __float_as_uint(fabsf(x[i]));
        m = u > m ? u : m;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned o = __shfl_xor_sync(0xffffffffu, m, off);
        m = o > m ? o : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

__device__ __forceinline__ int sketch_F_from_absmax(unsigned absbits, long long n) {
    // |x| <= 2^e_max with e_max = unbiased exponent + 1
    const int eb = (int)((absbits >> 23) & 0xFFu);
    const int e_max = eb == 0 ? -126 : eb - 127 + 1;
    int lg = 0;
    while ((1ll << lg) < n + 1) ++lg;
    int F = 61 - lg - e_max;
    return F > 150 ? 150 : F;
}

__global__ void __launch_bounds__(256) k_sketch_vec(const float* __restrict__ x, long long n, SketchParams sp,
                                                    const unsigned* absmax, long long* acc) {
    extern __shared__ unsigned char smem_raw[];
    long long* s = (long long*)smem_raw;
    for (int t = threadIdx.x; t < sp.m_s; t += blockDim.x) s[t] = 0;
    __syncthreads();
    const int F = sketch_F_from_absmax(*absmax, n);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long f = fixed_from(x[i], F);
        if (!f) continue;
        int rows[16];
        unsigned neg;
        if (sp.zeta == 8) sketch_column8(sp, i, rows, &neg);
        else sketch_column(sp, i, rows, &neg);
#pragma unroll
        for (int q = 0; q < 16; ++q)
            if (q < sp.zeta)
                atomicAdd((unsigned long long*)&s[rows[q]], (unsigned long long)(((neg >> q) & 1u) ? -f : f));
    }
    __syncthreads();
    for (int t = threadIdx.x; t < sp.m_s; t += blockDim.x)
        if (s[t]) atomicAdd((unsigned long long*)&acc[t], (unsigned long long)s[t]);
}

__global__ void k_sketch_finish(const long long* acc, int m, long long n, int zeta, const unsigned* absmax,
                                double* y) {
    const int F = sketch_F_from_absmax(*absmax, n);
    const double scale = ldexp(1.0, -F) / sqrt((double)zeta);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m; t += gridDim.x * blockDim.x)
        y[t] = (double)acc[t] * scale;
}

// fresh DevState for a new solve (j = -1, all RHS OK, keys cleared)
__global__ void k_reset_state(DevState* st) {
    const int t = threadIdx.x;
    if (t < kMaxRhs) {
        st->status[t] = IPF_OK;
        st->kdone[t] = 0;
        st->beta[t] = 0.0;
        st->key[0][t] = 0ull;
        st->key[1][t] = 0ull;
    }
    if (t == 0) {
        st->j = -1;
        st->ctr = 0u;
        st->maxbits[0] = st->maxbits[1] = 0ull;
        st->minidx[0] = st->minidx[1] = ~0ull;
    }
}

}  // namespace

cudaError_t launch_reset_state(DevState* st, cudaStream_t s) {
    k_reset_state<<<1, 64, 0, s>>>(st);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------
#define IPF_DISPATCH_STORAGE(storage, ...)                                         \
    switch (storage) {                                                              \
        case IPF_STORE_F64: { using T = double; __VA_ARGS__; } break;              \
        case IPF_STORE_F32: { using T = float; __VA_ARGS__; } break;               \
        case IPF_STORE_BF16: { using T = __nv_bfloat16; __VA_ARGS__; } break;      \
        case IPF_STORE_F16: { using T = __half; __VA_ARGS__; } break;              \
        default: return cudaErrorInvalidValue;                                      \
    }

cudaError_t launch_load_rhs(int storage, const float* b, const Geom& g, const Bufs& bf, cudaStream_t s) {
    const long long N = g.N;
    const int blocks = (int)((N + 255) / 256 < 4096 ? (N + 255) / 256 : 4096);
    if (storage == IPF_STORE_F64) k_load_rhs<double><<<blocks, 256, 0, s>>>(b, (double*)bf.w, g.n, g.B);
    else k_load_rhs<float><<<blocks, 256, 0, s>>>(b, (float*)bf.w, g.n, g.B);
    return cudaGetLastError();
}

cudaError_t launch_pivot_solve(int storage, const Geom& g, const Bufs& bf, cudaStream_t s) {
    const int K1 = g.k_max + 1;
    IPF_DISPATCH_STORAGE(storage, {
        using Acc = typename AccOf<T>::type;
        const size_t smem = (size_t)((K1 + 1) & ~1) * sizeof(double) +
                            (size_t)g.k_max * (g.k_max + 1) / 2 * sizeof(Acc);
        auto fn = k_pivot_solve<T, Acc>;
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        fn<<<g.B, 256, smem, s>>>(g, bf);
    });
    return cudaGetLastError();
}

cudaError_t launch_update(int storage, const Geom& g, const Bufs& bf, const SketchParams& sp, int num_sms,
                          cudaStream_t s) {
    const int K1 = g.k_max + 1;
    int per_thread = 0;
    IPF_DISPATCH_STORAGE(storage, { per_thread = 16 / (int)sizeof(T); });
    const long long chunks = (g.N + (long long)256 * per_thread - 1) / ((long long)256 * per_thread);
    long long blocks = (long long)num_sms * 4;
    if (blocks > chunks) blocks = chunks < 1 ? 1 : chunks;
    if (storage == IPF_STORE_F64) {
        const size_t smem = (size_t)K1 * sizeof(double);
        k_update_d<<<(int)blocks, 256, smem, s>>>(g, bf);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        long long b2 = (g.N + 255) / 256;
        if (b2 > (long long)num_sms * 8) b2 = (long long)num_sms * 8;
        k_argmin_d<<<(int)b2, 256, 0, s>>>(g, bf);
        return cudaGetLastError();
    }
    const size_t zc = g.want_z ? (size_t)g.B * g.m_s : 0;
    const size_t smem = zc * 16 + (size_t)K1 * g.B * sizeof(float);
    auto go = [&](auto fn) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        fn<<<(int)blocks, 256, smem, s>>>(g, bf, sp);
        return cudaGetLastError();
    };
    switch (storage) {
        case IPF_STORE_F32: return go(k_update_f<float>);
        case IPF_STORE_BF16: return go(k_update_f<__nv_bfloat16>);
        case IPF_STORE_F16: return go(k_update_f<__half>);
        default: return cudaErrorInvalidValue;
    }
}

static int pick_group(int B, int m_s, int nacc) {
    int Bg = B;
    while (Bg > 1 && (size_t)Bg * m_s * 16 * nacc > 96 * 1024) Bg >>= 1;
    return Bg;
}

cudaError_t launch_normalize(int storage, const Geom& g, const Bufs& bf, const SketchParams& sp, bool want_sw,
                             int num_sms, cudaStream_t s) {
    const int nacc = want_sw ? 2 : 1;
    const int Bg = pick_group(g.B, g.m_s, nacc);
    const size_t smem = (size_t)Bg * g.m_s * 16 * nacc;
    const long long work = g.n * Bg;
    long long bx = (work + 255) / 256;
    const int groups = g.B / Bg;
    long long cap = (long long)num_sms * 2 / groups;
    if (cap < 1) cap = 1;
    if (bx > cap) bx = cap;
    dim3 grid((unsigned)bx, (unsigned)groups);
    IPF_DISPATCH_STORAGE(storage, {
        using Acc = typename AccOf<T>::type;
        auto fn = k_normalize<T, Acc>;
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        fn<<<grid, 256, smem, s>>>(g, bf, sp, want_sw ? 1 : 0, Bg);
    });
    return cudaGetLastError();
}

cudaError_t launch_sketch_vector(const float* x, long long n, const SketchParams& sp, int /*F*/, long long* acc,
                                 float* absmax_out, cudaStream_t s, int num_sms, bool /*find_max*/) {
    unsigned* amax = (unsigned*)absmax_out;
    long long blocks = (n + 255) / 256;
    if (blocks > (long long)num_sms * 4) blocks = (long long)num_sms * 4;
    if (blocks < 1) blocks = 1;
    k_absmax<<<(int)blocks, 256, 0, s>>>(x, n, amax);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = (size_t)sp.m_s * 8;
    e = cudaFuncSetAttribute(k_sketch_vec, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_sketch_vec<<<(int)blocks, 256, smem, s>>>(x, n, sp, amax, acc);
    return cudaGetLastError();
}

cudaError_t launch_sketch_finish(const long long* acc, int m, long long n, int zeta, const unsigned* absmax,
                                 double* y, cudaStream_t s) {
    k_sketch_finish<<<(m + 255) / 256, 256, 0, s>>>(acc, m, n, zeta, absmax, y);
    return cudaGetLastError();
}

}  // namespace ipf
