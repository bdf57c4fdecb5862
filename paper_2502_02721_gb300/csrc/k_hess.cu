// One step of the pivoted Hessenberg process with its sketch (Sec. 3.1 Eq.
// Hessenberg_s; the loop of Algorithm 1 in the square form, applying A where
// the algorithm, written for the generalized process, applies A^T):
//
//   k_pivot_minv    append row p_j of L_p and the matching row of L_p^{-1}
//   k_pivot_apply   h = L_p^{-1} u(p_1..p_j) in FP64 (the sequential
//                   elimination H(i,j) = u(p_i), u -= H(i,j) v_i is this
//                   triangular solve because v_c(p_i) = 0 for c > i and
//                   v_i(p_i) = 1)
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
// The FP64 pivot-block solve h = L_p^{-1} u(p_1..p_{j+1}) of step j.  L_p is
// unit lower triangular, L(i, c) = v_c(p_i) for c < i (the stored basis
// values at the pivot rows), so the sequential elimination H(i,j) = u(p_i),
// u -= H(i,j) v_i of Algorithm 1 is this triangular solve (v_c(p_i) = 0 for
// c > i and v_i(p_i) = 1).  Both L_p and M = L_p^{-1} are kept packed
// row-major, strictly lower (row i, entries c < i, at offset i(i-1)/2; the
// unit diagonal is implicit), each step appending one row.
//
// Inverse form (default).  The block inverse of [L 0; l^T 1] is
// [M 0; -l^T M 1], so appending row j of L_p (l = L(j, 0..j-1)) appends
//     M(j, c) = -( l_c + sum_{c < i < j} l_i M(i, c) ),   c < j,
// which needs only the pivots and the stored basis (k_pivot_minv: a warp
// per column, lanes over the rows, a fixed shuffle tree), and then h(i) = u(p_i) + sum_{c < i} M(i, c) u(p_c), i <= j, is a
// product with independent rows (k_pivot_apply: a warp per row, lanes over
// c, a fixed shuffle tree).  Forward substitution is a chain of j dependent
// columns on one SM; GB300's FP64 rate per SM (about two FMAs per clock)
// makes that chain the longest part of a step at large j, where the inverse
// form spreads the same j^2 FMAs over many SMs.
// Growth: with max-|.| pivots |L| <= 1; a row of M larger than kMinvGrowth
// in magnitude (or not finite) sets DevState::fwd and the RHS continues by
// forward substitution (k_pivot_apply runs pivot_fwd_body in one CTA); the
// configuration can also ask for forward substitution throughout.
//
// Forward substitution (pivot_fwd_body): warp 0..3 (one per SM partition)
// hold the rows in registers, four row groups of 32 per warp (j < 512);
// column blocks of 32 are solved by the warp holding their rows and applied
// by all four, each row's updates in column order; L_p is read from global
// memory (L2).
// ------------------------------------------------------------------------
// doubles per RHS for the packed L_p (and M), rounded up to whole 16-byte chunks
__host__ __device__ constexpr size_t lp_stride(int k_max) { return ((size_t)(k_max + 1) * k_max / 2 + 2) & ~(size_t)1; }

constexpr double kMinvGrowth = 1048576.0;      // 2^20
constexpr int kMinvCols = 8;                   // columns of M per CTA of k_pivot_minv (a warp each)
constexpr int kApplyRows = 8;                  // rows of h per CTA of k_pivot_apply
constexpr int kFwdNG = 4;                      // row groups of 32 per warp in pivot_fwd_body

template <class T, class Acc>
__device__ __forceinline__ void pivot_fwd_body(const Geom& g, const Bufs& bf, int r) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DevState* st = bf.st;
    if (st->status[r] != IPF_OK) return;
    const int j = st->j;
    if (j < 0 || j >= g.k_max || j >= 128 * kFwdNG) return;
    const int K1 = g.k_max + 1;
    const int B = g.B;
    const T* V = (const T*)bf.V;
    const Acc* w = (const Acc*)bf.w;
    double* Lp = (double*)bf.LpT + (size_t)r * lp_stride(g.k_max);
    const int* piv = bf.piv + (size_t)r * K1;
    double* s_g = (double*)smem_raw;                      // u(p), K1 rounded to even, then x_c
    const size_t rowj = (size_t)j * (j - 1) / 2;          // doubles in rows 1..j-1
    // row j (exact copies of the stored values) and u at the pivot rows
    const size_t pj = (size_t)piv[j] * B + r;
    for (int c = threadIdx.x; c < j; c += blockDim.x) Lp[rowj + c] = (double)to_acc(V[(size_t)c * g.ldv + pj]);
    if (bf.gpiv) {
        for (int i = threadIdx.x; i <= j; i += blockDim.x) s_g[i] = (double)bf.gpiv[(size_t)r * K1 + i];
    } else {
        for (int i = threadIdx.x; i <= j; i += blockDim.x) s_g[i] = (double)w[(size_t)piv[i] * B + r];
    }
    __syncthreads();
    if (threadIdx.x >= 128) return;
    const double* Lr = Lp;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int qmax = j >> 5;                               // last row group holding a row <= j
    double* s_x = s_g + ((j + 2) & ~1);                    // x_c per column, after g
    double x[kFwdNG];
    int off[kFwdNG];
#pragma unroll
    for (int h = 0; h < kFwdNG; ++h) {
        const int i = (warp + 4 * h) * 32 + lane;
        x[h] = (i <= j) ? s_g[i] : 0.0;
        off[h] = i * (i - 1) / 2;
    }
    for (int cb = 0; cb <= qmax; ++cb) {
        const int c0 = cb * 32;
        const int cend = j - c0 < 32 ? j - c0 : 32;            // columns c = c0 + cc < j
        if (warp == (cb & 3)) {
            const int oh = cb >> 2;
            double xv = x[0];
            int offr = off[0];
#pragma unroll
            for (int h = 1; h < kFwdNG; ++h)
                if (h == oh) { xv = x[h]; offr = off[h]; }
            const bool row_ok = c0 + lane <= j;
#pragma unroll 1
            for (int cc = 0; cc < cend; ++cc) {
                const double xc = __shfl_sync(0xffffffffu, xv, cc);
                if (row_ok && lane > cc) xv = fma(-Lr[offr + c0 + cc], xc, xv);
            }
#pragma unroll
            for (int h = 0; h < kFwdNG; ++h)
                if (h == oh) x[h] = xv;
            if (c0 + lane < j) s_x[c0 + lane] = xv;
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
#pragma unroll
        for (int h = 0; h < kFwdNG; ++h) {
            const int q = warp + 4 * h;
            // rows i > c with i <= j only: L_p holds rows 1..j and nothing beyond
            if (q > cb && q <= qmax && q * 32 + lane <= j) {
                double xv = x[h];
#pragma unroll 4
                for (int cc = 0; cc < cend; ++cc) xv = fma(-Lr[off[h] + c0 + cc], s_x[c0 + cc], xv);
                x[h] = xv;
            }
        }
    }
    double* Hc = bf.H + (size_t)r * K1 * g.k_max + (size_t)K1 * j;
    Acc* coef = (Acc*)bf.coef;
#pragma unroll
    for (int h = 0; h < kFwdNG; ++h) {
        const int i = (warp + 4 * h) * 32 + lane;
        if (i <= j) {
            Hc[i] = x[h];
            coef[(size_t)i * B + r] = (Acc)x[h];
        }
    }
}

// the dynamic shared memory of k_pivot_apply (pivot_fwd_body's u(p) and x_c)
__host__ __device__ constexpr size_t pivot_apply_smem(int k_max) {
    return (size_t)(((k_max + 2) & ~1) + k_max + 2) * sizeof(double);
}

// row j of L_p and of M = L_p^{-1}, columns 8 cb .. 8 cb + 7 (256 threads, a
// warp per column, lanes over the rows i = c + 1 + lane, c + 33 + lane, ...
// (at most (j - 1) / 32 + 1 dependent FMAs per lane), a fixed shuffle tree)
template <class T>
__device__ __forceinline__ void pivot_minv_body(const Geom& g, const Bufs& bf, int r, int cb) {
    __shared__ double s_l[kMaxK];
    DevState* st = bf.st;
    if (st->status[r] != IPF_OK) return;
    const int j = st->j;
    if (j < 1 || j >= g.k_max) return;
    const int c0 = cb * kMinvCols;
    if (c0 >= j) return;
    const int K1 = g.k_max + 1;
    const T* V = (const T*)bf.V;
    const size_t ls = lp_stride(g.k_max);
    double* Lp = (double*)bf.LpT + (size_t)r * ls;
    double* M = bf.Minv + (size_t)r * ls;
    const size_t rowj = (size_t)j * (j - 1) / 2;
    // l: the stored values at the pivot row p_j (exact copies) of the columns
    // this CTA reads (c0 .. j - 1); the first column block also appends all
    // of them to L_p (read by forward substitution)
    const size_t pj = (size_t)bf.piv[(size_t)r * K1 + j] * g.B + r;
    for (int c = (cb == 0 ? 0 : c0) + threadIdx.x; c < j; c += blockDim.x) {
        const double v = (double)to_acc(V[(size_t)c * g.ldv + pj]);
        s_l[c] = v;
        if (cb == 0) Lp[rowj + c] = v;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = c0 + warp;
    if (c >= j) return;
    double acc = 0.0;
#pragma unroll 4
    for (int i = c + 1 + lane; i < j; i += 32) acc = fma(s_l[i], M[(size_t)i * (i - 1) / 2 + c], acc);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) {
        const double m = -(s_l[c] + acc);
        M[rowj + c] = m;
        if (!(fabs(m) <= kMinvGrowth)) st->fwd[r] = 1;
    }
}

// h(i) = u(p_i) + sum_{c < i} M(i, c) u(p_c) for the rows i = 8 rb .. 8 rb + 7
// (<= j), a warp per row; writes column j of H and the update's coefficients
template <class T, class Acc>
__device__ __forceinline__ void pivot_apply_body(const Geom& g, const Bufs& bf, int r, int rb) {
    __shared__ double s_u[kMaxK + 1];
    const DevState* st = bf.st;
    if (st->status[r] != IPF_OK) return;
    const int j = st->j;
    if (j < 0 || j >= g.k_max) return;
    const int i0 = rb * kApplyRows;
    if (i0 > j) return;
    const int K1 = g.k_max + 1;
    const int* piv = bf.piv + (size_t)r * K1;
    const int cmax = min(j, i0 + kApplyRows - 1);        // the entries of u(p) these rows read
    if (bf.gpiv) {
        for (int c = threadIdx.x; c <= cmax; c += blockDim.x) s_u[c] = (double)bf.gpiv[(size_t)r * K1 + c];
    } else {
        const Acc* w = (const Acc*)bf.w;
        for (int c = threadIdx.x; c <= cmax; c += blockDim.x) s_u[c] = (double)w[(size_t)piv[c] * g.B + r];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = i0 + warp;
    if (i > j) return;
    const double* Mi = bf.Minv + (size_t)r * lp_stride(g.k_max) + (size_t)i * (i - 1) / 2;
    double acc = 0.0;
    for (int c = lane; c < i; c += 32) acc = fma(Mi[c], s_u[c], acc);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) {
        const double x = s_u[i] + acc;
        bf.H[(size_t)r * K1 * g.k_max + (size_t)K1 * j + i] = x;
        ((Acc*)bf.coef)[(size_t)i * g.B + r] = (Acc)x;
    }
}

// grid (column blocks, RHS)
template <class T>
__global__ void __launch_bounds__(256) k_pivot_minv(Geom g, Bufs bf) {
    pivot_minv_body<T>(g, bf, blockIdx.y, blockIdx.x);
}

// grid (row blocks, RHS); dynamic shared memory pivot_apply_smem(k_max)
template <class T, class Acc>
__global__ void __launch_bounds__(256) k_pivot_apply(Geom g, Bufs bf) {
    const int r = blockIdx.y;
    if (bf.st->fwd[r]) {
        if (blockIdx.x == 0) pivot_fwd_body<T, Acc>(g, bf, r);
        return;
    }
    pivot_apply_body<T, Acc>(g, bf, r, blockIdx.x);
}

// ------------------------------------------------------------------------
// the zeta = 8 sketch of one element: q (its fixed-point value) added with
// the element's signs to its 8 rows, decoded from the table entry (byte t =
// row offset in block t | sign << 7) into the split int32 counters; a
// counter word that is zero is not added (for BF16 values of magnitude at
// least 2^(e-10) the low word is zero)
// ------------------------------------------------------------------------
__device__ __forceinline__ void scatter8(int* s_hi, int* s_lo, const SketchParams& sp, long long qv, uint2 ent) {
    const int hp = (int)(qv >> 17), lp = (int)(qv & 0x1FFFFll);
    const long long qn = -qv;
    const int hn = (int)(qn >> 17), ln = (int)(qn & 0x1FFFFll);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const unsigned byte = ((q < 4 ? ent.x : ent.y) >> (8 * (q & 3))) & 0xFFu;
        const int row = sp.lo[q] + (int)(byte & 0x7Fu);
        const bool ng = (byte & 0x80u) != 0;
        const int h = ng ? hn : hp, l = ng ? ln : lp;
        if (h) atomicAdd(&s_hi[row], h);
        if (l) atomicAdd(&s_lo[row], l);
    }
}

// ------------------------------------------------------------------------
// u -= V_j h ; u(pivots) = 0 ; argmax keys.  Acc = float, B RHS interleaved
// (compile-time, so element -> (row, RHS) is a shift and a mask).  Each
// thread owns 16 bytes of every basis column per grid-stride pass and keeps
// two groups of four 128-bit loads in flight (evict-first: V_j is streamed
// once, u stays in L2 for the normaliser).
// ------------------------------------------------------------------------
template <class T, int B>
__global__ void __launch_bounds__(256, 4) k_update_f(Geom g, Bufs bf, SketchParams sp) {
    // the normaliser that follows may be placed as these CTAs finish; it
    // waits for the whole grid (griddepcontrol.wait) before it reads anything
    asm volatile("griddepcontrol.launch_dependents;");
    constexpr int VEC = Vec16<T>::n;
    constexpr int LB = (B == 1) ? 0 : (B == 2) ? 1 : (B == 4) ? 2 : (B == 8) ? 3 : (B == 16) ? 4 : 5;
    constexpr int NK = (B == 1) ? 1 : VEC;           // argmax keys kept per thread
    extern __shared__ unsigned char smem_raw[];
    float* s_coef = (float*)smem_raw;
    __shared__ unsigned long long s_key[kMaxRhs];
    __shared__ int s_ok[kMaxRhs];
    DevState* st = bf.st;
    const int j = st->j;
    if (j >= g.k_max) return;                       // never past the last basis column
    const int nc = j + 1;                           // coefficients h_0..h_j (none during init)
    const float* coef = (const float*)bf.coef;
    for (int t = threadIdx.x; t < nc * B; t += blockDim.x) s_coef[t] = coef[t];
    if (threadIdx.x < B) {
        s_key[threadIdx.x] = 0ull;
        s_ok[threadIdx.x] = st->status[threadIdx.x] == IPF_OK;
    }
    // deferred sketch (one RHS): the newest column v_j, left pending by the
    // previous normalisation, is sketched here from the same loads, into
    // split counters after the coefficients (at most kFoldEvery elements per
    // CTA, so no fold is needed before the flush)
    const int csk = (B == 1 && g.sketch_defer && st->sk_pending == j) ? j : -1;
    int* s_hi = (int*)(s_coef + ((nc * B + 3) & ~3));
    int* s_lo = s_hi + sp.m_s;
    if (csk >= 0)
        for (int t = threadIdx.x; t < 2 * sp.m_s; t += blockDim.x) s_hi[t] = 0;
    __syncthreads();
    if (B == 1 && !s_ok[0]) return;
    const int Ssk = csk >= 0 ? kSplitS - bf.colE[csk] : 0;
    const uint2* tab = (const uint2*)bf.sktab;

    const T* V = (const T*)bf.V;
    float* w = (float*)bf.w;
    const unsigned N = (unsigned)g.N;
    unsigned long long best[NK];
#pragma unroll
    for (int q = 0; q < NK; ++q) best[q] = 0ull;
    const size_t ldv = (size_t)g.ldv;
    const unsigned stride = gridDim.x * blockDim.x * VEC;
    const unsigned base0 = (blockIdx.x * blockDim.x + threadIdx.x) * VEC;
    for (unsigned base = base0; base < N; base += stride) {
        float acc[VEC];
        {
            const float4* wp = (const float4*)(w + base);
#pragma unroll
            for (int q = 0; q < VEC / 4; ++q) {
                const float4 t4 = wp[q];
                acc[4 * q] = t4.x; acc[4 * q + 1] = t4.y; acc[4 * q + 2] = t4.z; acc[4 * q + 3] = t4.w;
            }
        }
        const T* vb = V + base;
        if (csk >= 0) {
            const uint4 rv = *(const uint4*)(vb + (size_t)csk * ldv);
            const T* vv = (const T*)&rv;
#pragma unroll
            for (int q = 0; q < VEC; q += 2) {
                const uint4 te = *(const uint4*)(tab + base + q);
                if (base + q < N) {
                    const long long qv = fixed_from(to_acc(vv[q]), Ssk);
                    if (qv) scatter8(s_hi, s_lo, sp, qv, make_uint2(te.x, te.y));
                }
                if (base + q + 1 < N) {
                    const long long qv = fixed_from(to_acc(vv[q + 1]), Ssk);
                    if (qv) scatter8(s_hi, s_lo, sp, qv, make_uint2(te.z, te.w));
                }
            }
        }
        int c = 0;
        for (; c + 8 <= nc; c += 8) {
            uint4 raw[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) raw[u] = __ldcs((const uint4*)(vb + (size_t)(c + u) * ldv));
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const T* vv = (const T*)&raw[u];
#pragma unroll
                for (int q = 0; q < VEC; ++q)
                    acc[q] = fmaf(-s_coef[(c + u) * B + ((base + q) & (B - 1))], to_acc(vv[q]), acc[q]);
            }
        }
        for (; c < nc; ++c) {
            const uint4 r1 = __ldcs((const uint4*)(vb + (size_t)c * ldv));
            const T* vv = (const T*)&r1;
#pragma unroll
            for (int q = 0; q < VEC; ++q)
                acc[q] = fmaf(-s_coef[c * B + ((base + q) & (B - 1))], to_acc(vv[q]), acc[q]);
        }
        const unsigned bits = bf.ispiv[base >> 5] >> (base & 31);
#pragma unroll
        for (int q = 0; q < VEC; ++q) {
            if ((bits >> q) & 1u) acc[q] = 0.f;
            const unsigned e = base + q;
            const int rr = (int)(e & (B - 1));
            if (e < N && s_ok[rr]) {
                const unsigned long long k = argmax_key(acc[q], e >> LB);
                const int slot = (B == 1) ? 0 : q;
                best[slot] = k > best[slot] ? k : best[slot];
            }
        }
        float4* wo = (float4*)(w + base);
#pragma unroll
        for (int q = 0; q < VEC / 4; ++q)
            wo[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
    }
    // reduce keys: the RHS of slot q is (base0 + q) mod B on every pass
    if (B == 1) {
        unsigned long long k = best[0];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, k, off);
            k = o > k ? o : k;
        }
        if ((threadIdx.x & 31) == 0 && k) atomicMax(&s_key[0], k);
    } else {
#pragma unroll
        for (int q = 0; q < NK; ++q)
            if (best[q]) atomicMax(&s_key[(int)((base0 + q) & (B - 1))], best[q]);
    }
    __syncthreads();
    if (threadIdx.x < B && s_key[threadIdx.x])
        atomicMax(&st->key[(j + 1) & 1][threadIdx.x], s_key[threadIdx.x]);
    if (csk >= 0) {
        long long* dst = bf.accSV + (size_t)csk * sp.m_s;
        for (int t = threadIdx.x; t < sp.m_s; t += blockDim.x) {
            const long long v = ((long long)s_hi[t] << 17) + (long long)s_lo[t];
            if (v) atomicAdd((unsigned long long*)&dst[t], (unsigned long long)v);
        }
    }
}

// ------------------------------------------------------------------------
// split step, part 1: t = V_j h (the HBM stream), independent of A v_j
// except through h.  Same load scheme as k_update_f.
// ------------------------------------------------------------------------
template <class T, int B>
__global__ void __launch_bounds__(512, 2) k_gemv(Geom g, Bufs bf) {
    constexpr int VEC = Vec16<T>::n;
    extern __shared__ unsigned char smem_raw[];
    float* s_coef = (float*)smem_raw;
    DevState* st = bf.st;
    const int j = st->j;
    if (j < 0 || j >= g.k_max) return;
    if (B == 1 && st->status[0] != IPF_OK) return;
    const int nc = j + 1;
    const float* coef = (const float*)bf.coef;
    for (int t = threadIdx.x; t < nc * B; t += blockDim.x) s_coef[t] = coef[t];
    __syncthreads();
    const T* V = (const T*)bf.V;
    float* tout = bf.t;
    const unsigned N = (unsigned)g.N;
    const size_t ldv = (size_t)g.ldv;
    const unsigned stride = gridDim.x * blockDim.x * VEC;
    for (unsigned base = (blockIdx.x * blockDim.x + threadIdx.x) * VEC; base < N; base += stride) {
        float acc[VEC];
#pragma unroll
        for (int q = 0; q < VEC; ++q) acc[q] = 0.f;
        const T* vb = V + base;
        int c = 0;
        for (; c + 8 <= nc; c += 8) {
            uint4 raw[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) raw[u] = __ldcs((const uint4*)(vb + (size_t)(c + u) * ldv));
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const T* vv = (const T*)&raw[u];
#pragma unroll
                for (int q = 0; q < VEC; ++q)
                    acc[q] = fmaf(s_coef[(c + u) * B + ((base + q) & (B - 1))], to_acc(vv[q]), acc[q]);
            }
        }
        for (; c < nc; ++c) {
            const uint4 r1 = __ldcs((const uint4*)(vb + (size_t)c * ldv));
            const T* vv = (const T*)&r1;
#pragma unroll
            for (int q = 0; q < VEC; ++q)
                acc[q] = fmaf(s_coef[c * B + ((base + q) & (B - 1))], to_acc(vv[q]), acc[q]);
        }
        float4* to = (float4*)(tout + base);
#pragma unroll
        for (int q = 0; q < VEC / 4; ++q)
            to[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
    }
}

// ------------------------------------------------------------------------
// split step, part 2: u = w - t, u(pivots) = 0, argmax keys
// ------------------------------------------------------------------------
template <int B>
__global__ void __launch_bounds__(256) k_combine(Geom g, Bufs bf) {
    constexpr int LB = (B == 1) ? 0 : (B == 2) ? 1 : (B == 4) ? 2 : (B == 8) ? 3 : (B == 16) ? 4 : 5;
    __shared__ unsigned long long s_key[kMaxRhs];
    __shared__ int s_ok[kMaxRhs];
    DevState* st = bf.st;
    const int j = st->j;
    if (j < 0 || j >= g.k_max) return;
    if (threadIdx.x < B) {
        s_key[threadIdx.x] = 0ull;
        s_ok[threadIdx.x] = st->status[threadIdx.x] == IPF_OK;
    }
    __syncthreads();
    if (B == 1 && !s_ok[0]) return;
    float* w = (float*)bf.w;
    const float* t = bf.t;
    const unsigned N = (unsigned)g.N;
    unsigned long long best[(B == 1) ? 1 : 4];
#pragma unroll
    for (int q = 0; q < ((B == 1) ? 1 : 4); ++q) best[q] = 0ull;
    const unsigned stride = gridDim.x * blockDim.x * 4;
    const unsigned base0 = (blockIdx.x * blockDim.x + threadIdx.x) * 4;
    for (unsigned base = base0; base < N; base += stride) {
        const float4 a = *(const float4*)(w + base);
        const float4 b = *(const float4*)(t + base);
        float u[4] = {a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w};
        const unsigned bits = bf.ispiv[base >> 5] >> (base & 31);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if ((bits >> q) & 1u) u[q] = 0.f;
            const unsigned e = base + q;
            const int rr = (int)(e & (B - 1));
            if (e < N && s_ok[rr]) {
                const unsigned long long k = argmax_key(u[q], e >> LB);
                const int slot = (B == 1) ? 0 : q;
                best[slot] = k > best[slot] ? k : best[slot];
            }
        }
        *(float4*)(w + base) = make_float4(u[0], u[1], u[2], u[3]);
    }
    if (B == 1) {
        unsigned long long k = best[0];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, k, off);
            k = o > k ? o : k;
        }
        if ((threadIdx.x & 31) == 0 && k) atomicMax(&s_key[0], k);
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (best[q]) atomicMax(&s_key[(int)((base0 + q) & (B - 1))], best[q]);
    }
    __syncthreads();
    if (threadIdx.x < B && s_key[threadIdx.x])
        atomicMax(&st->key[(j + 1) & 1][threadIdx.x], s_key[threadIdx.x]);
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
__global__ void __launch_bounds__(256) k_normalize(Geom g, Bufs bf, SketchParams sp, int want_sw, int Bg, int lbg,
                                                   int lb) {
    // launched as a programmatic dependent of the update: its CTAs may be
    // placed while the update's last CTAs finish, and wait here until the
    // update has completed and its writes are visible (a no-op otherwise)
    asm volatile("griddepcontrol.wait;" ::: "memory");
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
    __shared__ int s_e[kMaxRhs];
    __shared__ bool s_last;
    DevState* st = bf.st;
    const int j = st->j;
    const int jn = j + 1;                 // index of the new basis vector
    if (jn > g.k_max) return;             // a step past k_max writes nothing
    const int kb = jn & 1;
    const int B = g.B;
    const int r0 = blockIdx.y * Bg;
    const Acc* w = (const Acc*)bf.w;
    const bool skip_sketch = g.sketch_off || g.sketch_defer;   // no counters at all then

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
        // column exponent: smallest e >= 0 with max |w| <= 2^e |H(j+1,j)|, so
        // every |v_{j+1}| (also after rounding) is at most 2^e
        int ex = 0;
        if (ok && bf.sampled) {
            const double a = fabs((double)hv), wm = st->wmax[r];
            while (ex < 60 && wm > ldexp(a, ex)) ++ex;
        }
        s_prow[threadIdx.x] = row;
        s_hval[threadIdx.x] = hv;
        s_ok[threadIdx.x] = ok;
        s_code[threadIdx.x] = code;
        s_e[threadIdx.x] = ex;
    }
    if (!skip_sketch)
        for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
            s_wide[t] = 0;
            if (!f64) { s_hi[t] = 0; s_lo[t] = 0; }
        }
    __syncthreads();

    bool any_ok = false;
    for (int q = 0; q < Bg; ++q) any_ok |= s_ok[q] != 0;
    const int F = g.F;
    // common case (float storage, one right-hand side, zeta = 8 with the
    // sketch table, no second sketch): the same integer sums with the
    // counter words of +q and -q formed once per element instead of once per
    // sketch row, and the table bytes decoded in 32-bit halves
    const bool fast = !f64 && Bg == 1 && g.B == 1 && (bf.sktab || skip_sketch) && sp.zeta == 8 && !want_sw &&
                      (((uintptr_t)bf.w | (uintptr_t)bf.V | (uintptr_t)bf.sktab) & 15u) == 0 && (g.ldv & 7) == 0;
    if (fast && any_ok) {
        // four consecutive elements per thread: one 16-byte load of w, one
        // store of the four rounded values, two 16-byte table loads
        T* vout = (T*)bf.V + (size_t)jn * g.ldv;
        const unsigned n = (unsigned)g.n;
        const unsigned n4 = n >> 2;
        const unsigned stride = gridDim.x * blockDim.x;
        const long long prow = s_prow[0];
        const Acc hval = s_hval[0];
        const int S = kSplitS - s_e[0];
        const uint2* tab = (const uint2*)bf.sktab;
        const bool sk = !skip_sketch;
        const int fold_rounds = kFoldEvery / (256 * 4);
        int round = 0;
        // v = u / H(j+1, j) (1 at the pivot) rounded to the storage type, four
        // elements from i0 on
        auto emit = [&](unsigned i0, const float4 w4, T* vs) {
            const float wv[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const Acc v = ((long long)(i0 + e) == prow) ? (Acc)1 : wv[e] / hval;
                vs[e] = from_acc<T>(v);
            }
            if constexpr (sizeof(T) == 2) {
                union { uint2 u; T t[4]; } pk;
#pragma unroll
                for (int e = 0; e < 4; ++e) pk.t[e] = vs[e];
                *reinterpret_cast<uint2*>(vout + i0) = pk.u;
            } else {
                *reinterpret_cast<float4*>(vout + i0) =
                    make_float4(to_acc(vs[0]), to_acc(vs[1]), to_acc(vs[2]), to_acc(vs[3]));
            }
        };
        if (!sk) {
            // no counters: four loads of w in flight per thread before the
            // stores (w is dead after this kernel: streamed past L2)
            constexpr unsigned U = 4;
            for (unsigned t0 = blockIdx.x * blockDim.x + threadIdx.x; t0 < n4; t0 += stride * U) {
                float4 w4[U];
#pragma unroll
                for (unsigned u = 0; u < U; ++u) {
                    const unsigned t = t0 + u * stride;
                    if (t < n4) w4[u] = __ldcs(reinterpret_cast<const float4*>(w) + t);
                }
#pragma unroll
                for (unsigned u = 0; u < U; ++u) {
                    const unsigned t = t0 + u * stride;
                    T vs[4];
                    if (t < n4) emit(t << 2, w4[u], vs);
                }
            }
        }
        for (unsigned t0 = blockIdx.x * blockDim.x; sk && t0 < n4; t0 += stride) {
            const unsigned t = t0 + threadIdx.x;
            if (t < n4) {
                const unsigned i0 = t << 2;
                const float4 w4 = *reinterpret_cast<const float4*>(w + i0);
                T vs[4];
                emit(i0, w4, vs);
                {
                    const uint4 ta = *reinterpret_cast<const uint4*>(tab + i0);
                    const uint4 tb = *reinterpret_cast<const uint4*>(tab + i0 + 2);
                    const uint2 ents[4] = {make_uint2(ta.x, ta.y), make_uint2(ta.z, ta.w), make_uint2(tb.x, tb.y),
                                           make_uint2(tb.z, tb.w)};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const long long qv = fixed_from(to_acc(vs[e]), S);
                        if (qv) scatter8(s_hi, s_lo, sp, qv, ents[e]);
                    }
                }
            }
            if (sk && ++round == fold_rounds) {
                __syncthreads();
                split_fold(s_hi, s_lo, s_wide, cnt);
                __syncthreads();
                round = 0;
            }
        }
        // the last n mod 4 elements
        if (blockIdx.x == 0 && threadIdx.x < (n & 3u)) {
            const unsigned i = (n4 << 2) + threadIdx.x;
            const Acc v = ((long long)i == prow) ? (Acc)1 : w[i] / hval;
            const T vsi = from_acc<T>(v);
            vout[i] = vsi;
            if (sk) {
                const long long qv = fixed_from(to_acc(vsi), S);
                if (qv) scatter8(s_hi, s_lo, sp, qv, tab[i]);
            }
        }
    } else if (any_ok) {
        T* vout = (T*)bf.V + (size_t)jn * g.ldv;
        const unsigned total = (unsigned)g.n << lbg;     // (i, rl) pairs this CTA's group covers
        const unsigned stride = gridDim.x * blockDim.x;
        const int fold_rounds = kFoldEvery / 256;
        int round = 0;
        for (unsigned t0 = blockIdx.x * blockDim.x; t0 < total; t0 += stride) {
            const unsigned t = t0 + threadIdx.x;
            const unsigned i = t >> lbg;
            const int rl = (int)(t & (unsigned)(Bg - 1));
            if (t < total && s_ok[rl]) {
                const unsigned e = (i << lb) + r0 + rl;
                const Acc v = ((long long)i == s_prow[rl]) ? (Acc)1 : w[e] / s_hval[rl];
                const T vs = from_acc<T>(v);
                vout[e] = vs;
                const long long fv = skip_sketch ? 0ll : fixed_from(to_acc(vs), F - s_e[rl]);
                const long long fw = (want_sw && !skip_sketch) ? fixed_from(v, F - s_e[rl]) : 0;
                if (fv || fw) {
                    int rows[16];
                    unsigned neg;
                    if (bf.sktab) {
                        const unsigned long long ent = bf.sktab[i];
                        neg = 0;
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const unsigned byte = (unsigned)(ent >> (8 * q)) & 0xFFu;
                            rows[q] = sp.lo[q] + (int)(byte & 0x7Fu);
                            neg |= (byte >> 7) << q;
                        }
                    } else if (sp.zeta == 8) {
                        sketch_column8(sp, i, rows, &neg);
                    } else {
                        sketch_column(sp, i, rows, &neg);
                    }
                    const int o1 = rl * sp.m_s, o2 = (Bg + rl) * sp.m_s;
                    if (sp.zeta == 8) {
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const bool ng = (neg >> q) & 1u;
                            if (f64) {
                                atomicAdd((unsigned long long*)&s_wide[o1 + rows[q]], (unsigned long long)(ng ? -fv : fv));
                                if (fw) atomicAdd((unsigned long long*)&s_wide[o2 + rows[q]], (unsigned long long)(ng ? -fw : fw));
                            } else {
                                split_add(s_hi, s_lo, o1 + rows[q], ng ? -fv : fv);
                                if (want_sw) split_add(s_hi, s_lo, o2 + rows[q], ng ? -fw : fw);
                            }
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < 16; ++q) {
                            if (q < sp.zeta) {
                                const bool ng = (neg >> q) & 1u;
                                if (f64) {
                                    atomicAdd((unsigned long long*)&s_wide[o1 + rows[q]], (unsigned long long)(ng ? -fv : fv));
                                    if (fw) atomicAdd((unsigned long long*)&s_wide[o2 + rows[q]], (unsigned long long)(ng ? -fw : fw));
                                } else {
                                    split_add(s_hi, s_lo, o1 + rows[q], ng ? -fv : fv);
                                    if (want_sw) split_add(s_hi, s_lo, o2 + rows[q], ng ? -fw : fw);
                                }
                            }
                        }
                    }
                }
            }
            if (!f64 && !skip_sketch && ++round == fold_rounds) {
                __syncthreads();
                split_fold(s_hi, s_lo, s_wide, cnt);
                __syncthreads();
                round = 0;
            }
        }
    }
    __syncthreads();
    if (!f64 && !skip_sketch) {
        split_fold(s_hi, s_lo, s_wide, cnt);
        __syncthreads();
    }
    const int K1 = g.k_max + 1;
    for (int t = threadIdx.x; t < (skip_sketch ? 0 : cnt); t += blockDim.x) {
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
            bf.colE[(size_t)r * K1 + jn] = s_e[rl];
            if (jn == 0) st->beta[r] = (double)s_hval[rl];
            else bf.H[(size_t)r * K1 * g.k_max + (size_t)K1 * j + jn] = (double)s_hval[rl];
            const long long e = row * B + r;
            atomicOr(&bf.ispiv[e >> 5], 1u << (unsigned)(e & 31));
            st->kdone[r] = jn;
        } else if (st->status[r] == IPF_OK) {
            st->status[r] = s_code[rl];
            // the generalized process stops as a whole; the other basis keeps
            // its completed columns
            if (bf.st_peer && bf.st_peer->status[r] == IPF_OK)
                bf.st_peer->status[r] = s_code[rl] == IPF_ERR_NONFINITE ? IPF_ERR_NONFINITE : IPF_BREAKDOWN;
            st->kdone[r] = (s_code[rl] == IPF_BREAKDOWN) ? jn : (jn > 0 ? jn - 1 : 0);
            if (jn == 0) st->beta[r] = 0.0;
        }
        st->key[kb ^ 1][r] = 0ull;
        if (f64 && rl == 0) { st->maxbits[kb ^ 1] = 0ull; st->minidx[kb ^ 1] = ~0ull; }
        if (g.sketch_defer && rl == 0) st->sk_pending = s_ok[0] ? jn : -1;   // one RHS
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
// deferred sketch: S v_c for the pending column c, the same exact integer
// sums as the normaliser's (so the result is bit-identical to sketching in
// the normaliser), read back from the stored column.  Every CTA reads the
// pending index first; the last CTA clears it, so a second launch before
// the next normalisation does nothing.
// ------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(256) k_sketch_col(Geom g, Bufs bf, SketchParams sp) {
    extern __shared__ unsigned char smem_raw[];
    const int cnt = sp.m_s;
    long long* s_wide = (long long*)smem_raw;
    int* s_hi = (int*)(s_wide + cnt);
    int* s_lo = s_hi + cnt;
    __shared__ bool s_last;
    DevState* st = bf.st;
    const int c = st->sk_pending;
    if (c >= 0 && c <= g.k_max) {
        for (int t = threadIdx.x; t < cnt; t += blockDim.x) { s_wide[t] = 0; s_hi[t] = 0; s_lo[t] = 0; }
        __syncthreads();
        const T* col = (const T*)bf.V + (size_t)c * g.ldv;
        const int S = kSplitS - bf.colE[c];
        const uint2* tab = (const uint2*)bf.sktab;
        const unsigned n = (unsigned)g.n, n4 = n >> 2;
        const unsigned stride = gridDim.x * blockDim.x;
        const int fold_rounds = kFoldEvery / (256 * 4);
        int round = 0;
        for (unsigned t0 = blockIdx.x * blockDim.x; t0 < n4; t0 += stride) {
            const unsigned t = t0 + threadIdx.x;
            if (t < n4) {
                const unsigned i0 = t << 2;
                T vs[4];
                if constexpr (sizeof(T) == 2) {
                    union { uint2 u; T t[4]; } pk;
                    pk.u = *reinterpret_cast<const uint2*>(col + i0);
#pragma unroll
                    for (int e = 0; e < 4; ++e) vs[e] = pk.t[e];
                } else {
                    const float4 f = *reinterpret_cast<const float4*>(col + i0);
                    vs[0] = f.x; vs[1] = f.y; vs[2] = f.z; vs[3] = f.w;
                }
                const uint4 ta = *reinterpret_cast<const uint4*>(tab + i0);
                const uint4 tb = *reinterpret_cast<const uint4*>(tab + i0 + 2);
                const uint2 ents[4] = {make_uint2(ta.x, ta.y), make_uint2(ta.z, ta.w), make_uint2(tb.x, tb.y),
                                       make_uint2(tb.z, tb.w)};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const long long qv = fixed_from(to_acc(vs[e]), S);
                    if (qv) scatter8(s_hi, s_lo, sp, qv, ents[e]);
                }
            }
            if (++round == fold_rounds) {
                __syncthreads();
                split_fold(s_hi, s_lo, s_wide, cnt);
                __syncthreads();
                round = 0;
            }
        }
        if (blockIdx.x == 0 && threadIdx.x < (n & 3u)) {
            const unsigned i = (n4 << 2) + threadIdx.x;
            const long long qv = fixed_from(to_acc(col[i]), S);
            if (qv) scatter8(s_hi, s_lo, sp, qv, tab[i]);
        }
        __syncthreads();
        split_fold(s_hi, s_lo, s_wide, cnt);
        __syncthreads();
        long long* dst = bf.accSV + (size_t)c * sp.m_s;            // one RHS: [k_max+1][m_s]
        for (int t = threadIdx.x; t < cnt; t += blockDim.x)
            if (s_wide[t]) atomicAdd((unsigned long long*)&dst[t], (unsigned long long)s_wide[t]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&st->sk_ctr, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        st->sk_pending = -1;
        st->sk_ctr = 0u;
        __threadfence();
    }
}

// ------------------------------------------------------------------------
// sampled pivoting (Sec. 3.2, Sec. 4): the pivot is the largest |w| over a
// random sample of `size` candidate rows.  Draw t of pivot choice c (c = j+1,
// 0 at the initialisation) is SplitMix64 output c*4096 + t of the generator
// started at `seed`, index floor(out * n / 2^64); draws that hit a pivot row
// or an already accepted row are discarded; at most 4096 draws.  If no more
// than `size` candidates remain, or every sampled |w| is zero, the full-max
// key left by the update stands.  One warp per right-hand side.
// ------------------------------------------------------------------------
template <class Acc>
__global__ void k_sample_pivot(Geom g, Bufs bf, unsigned long long seed, int size) {
    __shared__ long long s_draw[32];
    __shared__ int s_hit[32];
    __shared__ long long s_acc[64];
    __shared__ int s_cnt;
    const int r = blockIdx.x, lane = threadIdx.x;
    DevState* st = bf.st;
    if (st->status[r] != IPF_OK) return;
    const int jn = st->j + 1;
    if (jn > g.k_max) return;
    const long long n = g.n;
    const int B = g.B;
    // the full max |w| (left by the update) bounds |v_{j+1}| = |w| / |w(p)|
    if (lane == 0)
        st->wmax[r] = sizeof(Acc) == 4 ? (double)key_absval(st->key[jn & 1][r])
                                       : __longlong_as_double((long long)st->maxbits[jn & 1]);
    if (n - jn <= size) return;                       // every candidate: the full max stands
    if (lane == 0) s_cnt = 0;
    __syncwarp();
    for (int t0 = 0; t0 < 4096; t0 += 32) {
        const unsigned long long ctr = (unsigned long long)jn * 4096ull + (unsigned long long)(t0 + lane);
        const unsigned long long out = sm64_mix(seed + kGamma * (ctr + 1ull));
        const long long idx = (long long)__umul64hi(out, (unsigned long long)n);
        const long long e = idx * B + r;
        s_draw[lane] = idx;
        s_hit[lane] = (bf.ispiv[e >> 5] >> (unsigned)(e & 31)) & 1u;
        __syncwarp();
        if (lane == 0) {
            int cnt = s_cnt;
            for (int q = 0; q < 32 && cnt < size; ++q) {
                if (s_hit[q]) continue;
                bool dup = false;
                for (int a = 0; a < cnt; ++a) dup |= s_acc[a] == s_draw[q];
                if (!dup) s_acc[cnt++] = s_draw[q];
            }
            s_cnt = cnt;
        }
        __syncwarp();
        if (s_cnt >= size) break;
    }
    const int cnt = s_cnt;
    const Acc* w = (const Acc*)bf.w;
    if (sizeof(Acc) == 4) {
        unsigned long long best = 0ull;
        for (int a = lane; a < cnt; a += 32) {
            const long long idx = s_acc[a];
            const unsigned long long key = argmax_key((float)w[idx * B + r], (unsigned)idx);
            best = key > best ? key : best;
        }
        for (int off = 16; off > 0; off >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, best, off);
            best = o > best ? o : best;
        }
        if (lane == 0 && best != 0ull && key_absval(best) > 0.f) st->key[jn & 1][r] = best;
    } else {
        // F64 storage (one right-hand side): max |w| bits, then the lowest row
        unsigned long long bits = 0ull, row = ~0ull;
        for (int a = lane; a < cnt; a += 32) {
            const long long idx = s_acc[a];
            const unsigned long long bb = (unsigned long long)__double_as_longlong(fabs((double)w[idx]));
            if (bb > bits || (bb == bits && (unsigned long long)idx < row)) { bits = bb; row = (unsigned long long)idx; }
        }
        for (int off = 16; off > 0; off >>= 1) {
            const unsigned long long ob = __shfl_xor_sync(0xffffffffu, bits, off);
            const unsigned long long orow = __shfl_xor_sync(0xffffffffu, row, off);
            if (ob > bits || (ob == bits && orow < row)) { bits = ob; row = orow; }
        }
        if (lane == 0 && bits != 0ull) {
            st->maxbits[jn & 1] = bits;
            st->minidx[jn & 1] = row;
        }
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

// sketch table: the 8 rows and signs of column i, one byte per block
__global__ void k_sketch_table(SketchParams sp, long long n, unsigned long long* tab) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int rows[16];
        unsigned neg;
        sketch_column8(sp, i, rows, &neg);
        unsigned long long e = 0;
#pragma unroll
        for (int t = 0; t < 8; ++t)
            e |= (unsigned long long)((unsigned)(rows[t] - sp.lo[t]) | (((neg >> t) & 1u) << 7)) << (8 * t);
        tab[i] = e;
    }
}

// fresh DevState for a new solve (j = -1, all RHS OK, keys cleared)
__global__ void k_reset_state(DevState* st, int fwd) {
    const int t = threadIdx.x;
    if (t < kMaxRhs) {
        st->fwd[t] = fwd;
        st->status[t] = IPF_OK;
        st->kdone[t] = 0;
        st->beta[t] = 0.0;
        st->key[0][t] = 0ull;
        st->key[1][t] = 0ull;
    }
    if (t == 0) {
        st->j = -1;
        st->ctr = 0u;
        st->sk_pending = -1;
        st->sk_ctr = 0u;
        st->maxbits[0] = st->maxbits[1] = 0ull;
        st->minidx[0] = st->minidx[1] = ~0ull;
    }
}

}  // namespace

bool sketch_table_ok(const SketchParams& sp) {
    if (sp.zeta != 8) return false;
    for (int t = 0; t < 8; ++t)
        if (sp.lo[t + 1] - sp.lo[t] > 128) return false;
    return true;
}

cudaError_t launch_sketch_table(const SketchParams& sp, long long n, unsigned long long* tab, cudaStream_t s) {
    long long blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_sketch_table<<<(int)blocks, 256, 0, s>>>(sp, n, tab);
    return cudaGetLastError();
}

cudaError_t launch_reset_state(DevState* st, bool fwd, cudaStream_t s) {
    k_reset_state<<<1, 64, 0, s>>>(st, fwd ? 1 : 0);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------
// batched step: the update, normalisation and pivot-block solve of every
// active slot of the work list in one launch each (persistent CTAs over the
// (slot, tile) tables).  Per element the arithmetic is that of k_update_f,
// k_normalize, k_pivot_minv and k_pivot_apply for one right-hand side with
// float storage and the deferred sketch, so a solve gets the same bits
// whatever else is in the batch and however its elements are tiled.
// ------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(256, 4) kb_update(const SlotDesc* __restrict__ slots,
                                                    const TileRef* __restrict__ tiles, int ntiles) {
    constexpr int VEC = Vec16<T>::n;
    extern __shared__ unsigned char smem_raw[];
    float* s_coef = (float*)smem_raw;
    __shared__ unsigned long long s_key;
    __shared__ int s_j;
    for (int tt = blockIdx.x; tt < ntiles; tt += gridDim.x) {
        const TileRef tr = tiles[tt];
        const SlotDesc* sd = slots + tr.slot;
        const int j = slot_step(sd, &s_j);
        if (j < 0) continue;
        const Geom g = sd->g;
        const Bufs bf = sd->bf;
        const SketchParams sp = sd->sp;
        DevState* st = bf.st;
        const int nc = j + 1;
        const float* coef = (const float*)bf.coef;
        for (int t = threadIdx.x; t < nc; t += blockDim.x) s_coef[t] = coef[t];
        const int csk = (g.sketch_defer && st->sk_pending == j) ? j : -1;
        int* s_hi = (int*)(s_coef + ((nc + 3) & ~3));
        int* s_lo = s_hi + sp.m_s;
        if (csk >= 0)
            for (int t = threadIdx.x; t < 2 * sp.m_s; t += blockDim.x) s_hi[t] = 0;
        if (threadIdx.x == 0) s_key = 0ull;
        __syncthreads();
        const int Ssk = csk >= 0 ? kSplitS - bf.colE[csk] : 0;
        const uint2* tab = (const uint2*)bf.sktab;
        const T* V = (const T*)bf.V;
        float* w = (float*)bf.w;
        const unsigned N = (unsigned)g.N;
        const unsigned e0 = (unsigned)tr.tile * (unsigned)kBatchUpdTile;
        const unsigned e1 = min(N, e0 + (unsigned)kBatchUpdTile);
        const size_t ldv = (size_t)g.ldv;
        unsigned long long best = 0ull;
        for (unsigned base = e0 + threadIdx.x * VEC; base < e1; base += blockDim.x * VEC) {
            float acc[VEC];
            {
                const float4* wp = (const float4*)(w + base);
#pragma unroll
                for (int q = 0; q < VEC / 4; ++q) {
                    const float4 t4 = wp[q];
                    acc[4 * q] = t4.x; acc[4 * q + 1] = t4.y; acc[4 * q + 2] = t4.z; acc[4 * q + 3] = t4.w;
                }
            }
            const T* vb = V + base;
            if (csk >= 0) {
                const uint4 rv = *(const uint4*)(vb + (size_t)csk * ldv);
                const T* vv = (const T*)&rv;
#pragma unroll
                for (int q = 0; q < VEC; q += 2) {
                    const uint4 te = *(const uint4*)(tab + base + q);
                    if (base + q < N) {
                        const long long qv = fixed_from(to_acc(vv[q]), Ssk);
                        if (qv) scatter8(s_hi, s_lo, sp, qv, make_uint2(te.x, te.y));
                    }
                    if (base + q + 1 < N) {
                        const long long qv = fixed_from(to_acc(vv[q + 1]), Ssk);
                        if (qv) scatter8(s_hi, s_lo, sp, qv, make_uint2(te.z, te.w));
                    }
                }
            }
            int c = 0;
            for (; c + 8 <= nc; c += 8) {
                uint4 raw[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) raw[u] = __ldcs((const uint4*)(vb + (size_t)(c + u) * ldv));
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const T* vv = (const T*)&raw[u];
#pragma unroll
                    for (int q = 0; q < VEC; ++q) acc[q] = fmaf(-s_coef[c + u], to_acc(vv[q]), acc[q]);
                }
            }
            for (; c < nc; ++c) {
                const uint4 r1 = __ldcs((const uint4*)(vb + (size_t)c * ldv));
                const T* vv = (const T*)&r1;
#pragma unroll
                for (int q = 0; q < VEC; ++q) acc[q] = fmaf(-s_coef[c], to_acc(vv[q]), acc[q]);
            }
            const unsigned bits = bf.ispiv[base >> 5] >> (base & 31);
#pragma unroll
            for (int q = 0; q < VEC; ++q) {
                if ((bits >> q) & 1u) acc[q] = 0.f;
                const unsigned e = base + q;
                if (e < N) {
                    const unsigned long long k = argmax_key(acc[q], e);
                    best = k > best ? k : best;
                }
            }
            float4* wo = (float4*)(w + base);
#pragma unroll
            for (int q = 0; q < VEC / 4; ++q)
                wo[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, best, off);
            best = o > best ? o : best;
        }
        if ((threadIdx.x & 31) == 0 && best) atomicMax(&s_key, best);
        __syncthreads();
        if (threadIdx.x == 0 && s_key) atomicMax(&st->key[(j + 1) & 1][0], s_key);
        if (csk >= 0) {
            long long* dst = bf.accSV + (size_t)csk * sp.m_s;
            for (int t = threadIdx.x; t < sp.m_s; t += blockDim.x) {
                const long long v = ((long long)s_hi[t] << 17) + (long long)s_lo[t];
                if (v) atomicAdd((unsigned long long*)&dst[t], (unsigned long long)v);
            }
        }
    }
}

// the fast path of k_normalize (one RHS, float storage, the sketch deferred
// to the next update), over the tile's elements; tile 0 of a slot keeps its
// books and the slot's last tile advances its step counter
template <class T>
__global__ void __launch_bounds__(256) kb_normalize(const SlotDesc* __restrict__ slots,
                                                    const TileRef* __restrict__ tiles, int ntiles) {
    __shared__ long long s_prow;
    __shared__ float s_hval;
    __shared__ int s_ok, s_code, s_j;
    __shared__ bool s_last;
    for (int tt = blockIdx.x; tt < ntiles; tt += gridDim.x) {
        const TileRef tr = tiles[tt];
        const SlotDesc* sd = slots + tr.slot;
        const int j = slot_step(sd, &s_j);
        if (j < 0) continue;
        const Geom g = sd->g;
        const Bufs bf = sd->bf;
        DevState* st = bf.st;
        const int jn = j + 1;
        const int kb = jn & 1;
        const float* w = (const float*)bf.w;
        if (threadIdx.x == 0) {
            int ok = 1, code = IPF_OK;
            long long row = 0;
            float hv = 0.f;
            const unsigned long long key = st->key[kb][0];
            if (key == 0ull || key_absval(key) == 0.f) {
                ok = 0; code = IPF_BREAKDOWN;
            } else {
                row = (long long)key_row(key);
                hv = w[row];
                if (!isfinite(hv)) { ok = 0; code = IPF_ERR_NONFINITE; }
                else if (hv == 0.f) { ok = 0; code = IPF_BREAKDOWN; }
            }
            s_prow = row;
            s_hval = hv;
            s_ok = ok;
            s_code = code;
        }
        __syncthreads();
        const unsigned n = (unsigned)g.n;
        if (s_ok) {
            T* vout = (T*)bf.V + (size_t)jn * g.ldv;
            const unsigned n4 = n >> 2;
            const unsigned q0 = (unsigned)tr.tile * (kBatchNormTile / 4);
            const unsigned q1 = min(n4, q0 + kBatchNormTile / 4);
            const long long prow = s_prow;
            const float hval = s_hval;
            for (unsigned t = q0 + threadIdx.x; t < q1; t += blockDim.x) {
                const unsigned i0 = t << 2;
                const float4 w4 = *reinterpret_cast<const float4*>(w + i0);
                const float wv[4] = {w4.x, w4.y, w4.z, w4.w};
                T vs[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float v = ((long long)(i0 + e) == prow) ? 1.f : wv[e] / hval;
                    vs[e] = from_acc<T>(v);
                }
                if constexpr (sizeof(T) == 2) {
                    union { uint2 u; T t[4]; } pk;
#pragma unroll
                    for (int e = 0; e < 4; ++e) pk.t[e] = vs[e];
                    *reinterpret_cast<uint2*>(vout + i0) = pk.u;
                } else {
                    *reinterpret_cast<float4*>(vout + i0) =
                        make_float4(to_acc(vs[0]), to_acc(vs[1]), to_acc(vs[2]), to_acc(vs[3]));
                }
            }
            // the last n mod 4 elements belong to the tile holding element 4 n4
            if (4u * n4 >= (unsigned)tr.tile * kBatchNormTile && 4u * n4 < (unsigned)(tr.tile + 1) * kBatchNormTile &&
                threadIdx.x < (n & 3u)) {
                const unsigned i = (n4 << 2) + threadIdx.x;
                const float v = ((long long)i == prow) ? 1.f : w[i] / hval;
                vout[i] = from_acc<T>(v);
            }
        }
        if (tr.tile == 0 && threadIdx.x == 0) {
            const int K1 = g.k_max + 1;
            if (s_ok) {
                const long long row = s_prow;
                bf.piv[jn] = (int)row;
                bf.colE[jn] = 0;
                bf.H[(size_t)K1 * j + jn] = (double)s_hval;
                atomicOr(&bf.ispiv[row >> 5], 1u << (unsigned)(row & 31));
                st->kdone[0] = jn;
            } else if (st->status[0] == IPF_OK) {
                st->status[0] = s_code;
                st->kdone[0] = (s_code == IPF_BREAKDOWN) ? jn : (jn > 0 ? jn - 1 : 0);
            }
            st->key[kb ^ 1][0] = 0ull;
            if (g.sketch_defer) st->sk_pending = s_ok ? jn : -1;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            s_last = atomicAdd(&st->ctr, 1u) == (unsigned)sd->norm_tiles - 1u;
        }
        __syncthreads();
        if (s_last && threadIdx.x == 0) {
            st->j = jn;
            st->ctr = 0u;
            __threadfence();
        }
    }
}

// grid (column blocks, list entries)
template <class T>
__global__ void __launch_bounds__(256) kb_pivot_minv(const SlotDesc* __restrict__ slots,
                                                     const TileRef* __restrict__ list) {
    const SlotDesc* sd = slots + list[blockIdx.y].slot;
    if (sd->k_target <= 0) return;
    if (sd->bf.st->j >= sd->k_target) return;
    const Geom g = sd->g;
    const Bufs bf = sd->bf;
    pivot_minv_body<T>(g, bf, 0, blockIdx.x);
}

// grid (row blocks, list entries); dynamic shared memory pivot_apply_smem
template <class T>
__global__ void __launch_bounds__(256) kb_pivot_apply(const SlotDesc* __restrict__ slots,
                                                      const TileRef* __restrict__ list) {
    const SlotDesc* sd = slots + list[blockIdx.y].slot;
    if (sd->k_target <= 0) return;
    const DevState* st = sd->bf.st;
    if (st->j >= sd->k_target) return;
    const Geom g = sd->g;
    const Bufs bf = sd->bf;
    if (st->fwd[0]) {
        if (blockIdx.x == 0) pivot_fwd_body<T, float>(g, bf, 0);
        return;
    }
    pivot_apply_body<T, float>(g, bf, 0, blockIdx.x);
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

cudaError_t launch_pivot_minv(int storage, const Geom& g, const Bufs& bf, cudaStream_t s) {
    const dim3 grid((unsigned)((g.k_max + kMinvCols - 1) / kMinvCols), (unsigned)g.B);
    IPF_DISPATCH_STORAGE(storage, { k_pivot_minv<T><<<grid, 256, 0, s>>>(g, bf); });
    return cudaGetLastError();
}

cudaError_t launch_pivot_apply(int storage, const Geom& g, const Bufs& bf, cudaStream_t s) {
    const dim3 grid((unsigned)((g.k_max + kApplyRows - 1) / kApplyRows), (unsigned)g.B);   // rows 0 .. k_max - 1
    const size_t smem = pivot_apply_smem(g.k_max);
    IPF_DISPATCH_STORAGE(storage, {
        using Acc = typename AccOf<T>::type;
        k_pivot_apply<T, Acc><<<grid, 256, smem, s>>>(g, bf);
    });
    return cudaGetLastError();
}

cudaError_t launch_pivot_solve(int storage, const Geom& g, const Bufs& bf, cudaStream_t s) {
    cudaError_t e = launch_pivot_minv(storage, g, bf, s);
    if (e != cudaSuccess) return e;
    return launch_pivot_apply(storage, g, bf, s);
}

template <class T>
static cudaError_t update_B(const Geom& g, const Bufs& bf, const SketchParams& sp, int blocks, size_t smem,
                           cudaStream_t s) {
    auto go = [&](auto fn) -> cudaError_t {
        if (smem > 48 * 1024) {
            cudaError_t e = raise_smem(fn, (int)smem);
            if (e != cudaSuccess) return e;
        }
        fn<<<blocks, 256, smem, s>>>(g, bf, sp);
        return cudaGetLastError();
    };
    switch (g.B) {
        case 1: return go(k_update_f<T, 1>);
        case 2: return go(k_update_f<T, 2>);
        case 4: return go(k_update_f<T, 4>);
        case 8: return go(k_update_f<T, 8>);
        case 16: return go(k_update_f<T, 16>);
        case 32: return go(k_update_f<T, 32>);
        default: return cudaErrorInvalidValue;
    }
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
    size_t smem = (size_t)K1 * g.B * sizeof(float);
    if (g.sketch_defer) {
        // split counters after the coefficients; enough CTAs that none takes
        // more than kFoldEvery elements (one counter add per element)
        smem = (size_t)((K1 * g.B + 3) & ~3) * sizeof(float) + (size_t)2 * sp.m_s * sizeof(int);
        const long long need = (g.N + kFoldEvery - 1) / kFoldEvery;
        if (blocks < need) blocks = need;
    }
    switch (storage) {
        case IPF_STORE_F32: return update_B<float>(g, bf, sp, (int)blocks, smem, s);
        case IPF_STORE_BF16: return update_B<__nv_bfloat16>(g, bf, sp, (int)blocks, smem, s);
        case IPF_STORE_F16: return update_B<__half>(g, bf, sp, (int)blocks, smem, s);
        default: return cudaErrorInvalidValue;
    }
}

template <class T>
static cudaError_t gemv_B(const Geom& g, const Bufs& bf, int blocks, size_t smem, cudaStream_t s) {
    switch (g.B) {
        case 1: k_gemv<T, 1><<<blocks, 512, smem, s>>>(g, bf); break;
        case 2: k_gemv<T, 2><<<blocks, 512, smem, s>>>(g, bf); break;
        case 4: k_gemv<T, 4><<<blocks, 512, smem, s>>>(g, bf); break;
        case 8: k_gemv<T, 8><<<blocks, 512, smem, s>>>(g, bf); break;
        case 16: k_gemv<T, 16><<<blocks, 512, smem, s>>>(g, bf); break;
        case 32: k_gemv<T, 32><<<blocks, 512, smem, s>>>(g, bf); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_gemv(int storage, const Geom& g, const Bufs& bf, int num_sms, cudaStream_t s) {
    // one 512-thread CTA per SM: it co-resides with two operator CTAs, so the
    // HBM stream and the FP32 operator run on every SM at the same time
    int per_thread = 16 / (int)(storage == IPF_STORE_F32 ? 4 : 2);
    const long long chunks = (g.N + (long long)512 * per_thread - 1) / ((long long)512 * per_thread);
    long long blocks = (long long)num_sms;
    if (blocks > chunks) blocks = chunks < 1 ? 1 : chunks;
    const size_t smem = (size_t)(g.k_max + 1) * g.B * sizeof(float);
    switch (storage) {
        case IPF_STORE_F32: return gemv_B<float>(g, bf, (int)blocks, smem, s);
        case IPF_STORE_BF16: return gemv_B<__nv_bfloat16>(g, bf, (int)blocks, smem, s);
        case IPF_STORE_F16: return gemv_B<__half>(g, bf, (int)blocks, smem, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_combine(const Geom& g, const Bufs& bf, int num_sms, cudaStream_t s) {
    long long blocks = (g.N + 1023) / 1024;
    if (blocks > (long long)num_sms * 8) blocks = (long long)num_sms * 8;
    if (blocks < 1) blocks = 1;
    switch (g.B) {
        case 1: k_combine<1><<<(int)blocks, 256, 0, s>>>(g, bf); break;
        case 2: k_combine<2><<<(int)blocks, 256, 0, s>>>(g, bf); break;
        case 4: k_combine<4><<<(int)blocks, 256, 0, s>>>(g, bf); break;
        case 8: k_combine<8><<<(int)blocks, 256, 0, s>>>(g, bf); break;
        case 16: k_combine<16><<<(int)blocks, 256, 0, s>>>(g, bf); break;
        case 32: k_combine<32><<<(int)blocks, 256, 0, s>>>(g, bf); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
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
    int lbg = 0, lb = 0;
    while ((1 << lbg) < Bg) ++lbg;
    while ((1 << lb) < g.B) ++lb;
    long long bx = (work + 255) / 256;
    const int groups = g.B / Bg;
    long long cap = (long long)num_sms * 4 / groups;
    if (cap < 1) cap = 1;
    if (bx > cap) bx = cap;
    dim3 grid((unsigned)bx, (unsigned)groups);
    IPF_DISPATCH_STORAGE(storage, {
        using Acc = typename AccOf<T>::type;
        auto fn = k_normalize<T, Acc>;
        cudaError_t e = raise_smem(fn, (int)smem);
        if (e != cudaSuccess) return e;
        // programmatic dependent launch: overlaps this launch with the end of
        // the kernel before it in the stream (the kernel waits for it first)
        cudaLaunchConfig_t lc = {};
        lc.gridDim = grid;
        lc.blockDim = dim3(256);
        lc.dynamicSmemBytes = smem;
        lc.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        lc.attrs = at;
        lc.numAttrs = 1;
        e = cudaLaunchKernelEx(&lc, fn, g, bf, sp, want_sw ? 1 : 0, Bg, lbg, lb);
        if (e != cudaSuccess) return e;
    });
    return cudaGetLastError();
}

cudaError_t launch_sketch_col(int storage, const Geom& g, const Bufs& bf, const SketchParams& sp, int num_sms,
                              cudaStream_t s) {
    if (g.B != 1 || sp.zeta != 8 || !bf.sktab) return cudaErrorInvalidValue;
    const size_t smem = (size_t)sp.m_s * 16;
    long long blocks = (g.N / 4 + 255) / 256;
    if (blocks > (long long)num_sms * 4) blocks = (long long)num_sms * 4;
    if (blocks < 1) blocks = 1;
    switch (storage) {
        case IPF_STORE_F32: {
            cudaError_t e = raise_smem(k_sketch_col<float>, (int)smem);
            if (e != cudaSuccess) return e;
            k_sketch_col<float><<<(int)blocks, 256, smem, s>>>(g, bf, sp);
            break;
        }
        case IPF_STORE_BF16: {
            cudaError_t e = raise_smem(k_sketch_col<__nv_bfloat16>, (int)smem);
            if (e != cudaSuccess) return e;
            k_sketch_col<__nv_bfloat16><<<(int)blocks, 256, smem, s>>>(g, bf, sp);
            break;
        }
        case IPF_STORE_F16: {
            cudaError_t e = raise_smem(k_sketch_col<__half>, (int)smem);
            if (e != cudaSuccess) return e;
            k_sketch_col<__half><<<(int)blocks, 256, smem, s>>>(g, bf, sp);
            break;
        }
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_sample_pivot(int storage, const Geom& g, const Bufs& bf, unsigned long long seed, int size,
                                cudaStream_t s) {
    if (size < 1 || size > 64) return cudaErrorInvalidValue;
    if (storage == IPF_STORE_F64) k_sample_pivot<double><<<g.B, 32, 0, s>>>(g, bf, seed, size);
    else k_sample_pivot<float><<<g.B, 32, 0, s>>>(g, bf, seed, size);
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
    e = raise_smem(k_sketch_vec, (int)smem);
    if (e != cudaSuccess) return e;
    k_sketch_vec<<<(int)blocks, 256, smem, s>>>(x, n, sp, amax, acc);
    return cudaGetLastError();
}

cudaError_t launch_sketch_finish(const long long* acc, int m, long long n, int zeta, const unsigned* absmax,
                                 double* y, cudaStream_t s) {
    k_sketch_finish<<<(m + 255) / 256, 256, 0, s>>>(acc, m, n, zeta, absmax, y);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------
// batched step launchers
// ------------------------------------------------------------------------
cudaError_t launch_batch_pivot_solve(int storage, const SlotDesc* slots, const TileRef* list, int nslots, int k_max,
                                     cudaStream_t s) {
    if (nslots <= 0) return cudaSuccess;
    // k_max: the group's largest; blocks past a slot's own k_max return at once
    const dim3 gm((unsigned)((k_max + kMinvCols - 1) / kMinvCols), (unsigned)nslots);
    const dim3 ga((unsigned)((k_max + kApplyRows - 1) / kApplyRows), (unsigned)nslots);
    const size_t smem = pivot_apply_smem(k_max);
    auto go = [&](auto fm, auto fa) -> cudaError_t {
        fm<<<gm, 256, 0, s>>>(slots, list);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        fa<<<ga, 256, smem, s>>>(slots, list);
        return cudaGetLastError();
    };
    switch (storage) {
        case IPF_STORE_F32: return go(kb_pivot_minv<float>, kb_pivot_apply<float>);
        case IPF_STORE_BF16: return go(kb_pivot_minv<__nv_bfloat16>, kb_pivot_apply<__nv_bfloat16>);
        case IPF_STORE_F16: return go(kb_pivot_minv<__half>, kb_pivot_apply<__half>);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_batch_update(int storage, const SlotDesc* slots, const TileRef* tiles, int ntiles, int k_max,
                                int m_s_max, int num_sms, cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    const size_t smem = (size_t)((k_max + 1 + 3) & ~3) * sizeof(float) + (size_t)2 * m_s_max * sizeof(int);
    const int blocks = ntiles < num_sms * 4 ? ntiles : num_sms * 4;
    auto go = [&](auto fn) -> cudaError_t {
        if (smem > 48 * 1024) {
            cudaError_t e = raise_smem(fn, (int)smem);
            if (e != cudaSuccess) return e;
        }
        fn<<<blocks, 256, smem, s>>>(slots, tiles, ntiles);
        return cudaGetLastError();
    };
    switch (storage) {
        case IPF_STORE_F32: return go(kb_update<float>);
        case IPF_STORE_BF16: return go(kb_update<__nv_bfloat16>);
        case IPF_STORE_F16: return go(kb_update<__half>);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_batch_normalize(int storage, const SlotDesc* slots, const TileRef* tiles, int ntiles, int num_sms,
                                   cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    const int blocks = ntiles < num_sms * 8 ? ntiles : num_sms * 8;
    switch (storage) {
        case IPF_STORE_F32: kb_normalize<float><<<blocks, 256, 0, s>>>(slots, tiles, ntiles); break;
        case IPF_STORE_BF16: kb_normalize<__nv_bfloat16><<<blocks, 256, 0, s>>>(slots, tiles, ntiles); break;
        case IPF_STORE_F16: kb_normalize<__half><<<blocks, 256, 0, s>>>(slots, tiles, ntiles); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace ipf
