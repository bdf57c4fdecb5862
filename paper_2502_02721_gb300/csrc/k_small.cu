// The sketched projected problem (Sec. 3.2 Eq. sketched_LSLU, Sec. 3.3
// Eq. sketched_LSLU_hybrid, Algorithm 2's last two lines) in FP64, then
// x_k = V_k y:
//
//   k_form          M = [Z | c] with Z = S A V_k (m_s x k) and c = S b;
//                   T = S V_k when a sketched-x penalty is asked for
//   k_householder   Householder QR of every M (and T), R only; a
//                   cooperative launch, a group of CTAs per matrix, columns
//                   owned round-robin, reflectors passed on by column flags
//   k_small_solve   per (RHS, lambda): lambda = 0 back substitution on R_M;
//                   lambda > 0 QR of [R_M(:, 1:k); lambda R_T] (two stacked
//                   upper triangles, structure kept) then back substitution
//   k_reconstruct   x = V_k y for all lambdas in one pass over V_k
//
// ||c - Z y|| = ||R_M(:, k) - R_M(:, 1:k) y|| because M = Q R_M, and
// ||S V_k y|| = ||R_T y||, so only (k+1)- and k-sized triangles enter the
// per-lambda work.
#include "ipf_internal.cuh"

namespace ipf {

namespace {

struct SolveLayout {
    size_t bar_off, err_off, M_off, T_off, dM_off, dT_off, Y_off, S_off, W_off, total;
};

// workspace for k <= g.k_max and nl_max lambdas; the barrier counters and
// the error flag sit at fixed offsets at the start
SolveLayout layout_for(const Geom& g, int nl_max) {
    SolveLayout L;
    const size_t k = (size_t)g.k_max;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) & ~(size_t)255; return o; };
    L.bar_off = take(sizeof(unsigned) * (size_t)g.B * 2 * (g.k_max + 2));   // QR column flags per job
    L.err_off = take(sizeof(int) * 4);
    L.M_off = take(sizeof(double) * (size_t)g.B * g.m_s * (k + 1));
    L.T_off = take(sizeof(double) * (size_t)g.B * g.m_s * k);
    L.dM_off = take(sizeof(double) * (size_t)g.B * (k + 1));
    L.dT_off = take(sizeof(double) * (size_t)g.B * (k + 1));
    L.Y_off = take(sizeof(double) * (size_t)g.B * nl_max * (k + 1));
    L.S_off = take(sizeof(double) * (size_t)g.B * nl_max * (2 * k + 1) * (k + 1));
    L.W_off = take(sizeof(double) * (size_t)g.B * g.m_s * (k + 2));
    L.total = off;
    return L;
}

__device__ __forceinline__ int kuse_of(const DevState* st, int r, int k) {
    const int kd = st->kdone[r];
    return kd < k ? kd : k;
}

// the scale of a fixed-point sketch column with exponent e (see Bufs::colE)
__device__ __forceinline__ double col_scale(double scale, int e) { return e ? ldexp(scale, e) : scale; }

// M[r][col], T[r][col] (column-major, ld = m).  Column col < kb of M is
// z_col = S A v_col = (S V_{col+1}) h_col + H(col+1, col) (S w)_{col+1}, with
// (S w) the sketch of the unrounded normalised vector when the storage
// rounds it (use_sw, the DIRECT form) and S V otherwise (then the two forms
// coincide: S V_{kb+1} H); column kb is c = S b = beta * S (b / beta).
//
// qmr != 0 forms the quasi-minimal residual problem instead (Eq.
// Hessenber_LS): column col < kb is H(:, col) (rows 0..col+1, zero below)
// and column kb is beta e_1, so the same QR and per-lambda solves give
// y = argmin ||beta e_1 - H y||^2 + lambda^2 ||y||^2.
// W = S V_{kb+1} in FP64, column i scaled by its exponent: the factors of
// k_form's sums, formed once per entry instead of once per use
__global__ void k_scale_sv(Geom g, Bufs bf, int k, int zeta, double* Ww) {
    const int r = blockIdx.y;
    const int kb = kuse_of(bf.st, r, k);
    const int K1 = g.k_max + 1;
    const int m = g.m_s;
    const double scale = ldexp(1.0, -g.F) / sqrt((double)zeta);
    const long long* sv = bf.accSV + (size_t)r * K1 * m;
    const int* ce = bf.colE + (size_t)r * K1;
    double* W = Ww + (size_t)r * m * (k + 2);
    const long long total = (long long)m * (kb + 2 < K1 ? kb + 2 : K1);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t / m);
        W[t] = (double)sv[t] * col_scale(scale, ce[i]);
    }
}

__global__ void k_form(Geom g, Bufs bf, int k, int zeta, int use_sw, int need_T, double* Mw, double* Tw, int qmr,
                       const double* Ww) {
    const int r = blockIdx.y;
    const int kb = kuse_of(bf.st, r, k);
    const int K1 = g.k_max + 1;
    const int m = g.m_s;
    const double scale = ldexp(1.0, -g.F) / sqrt((double)zeta);
    const long long* sv = bf.accSV + (size_t)r * K1 * m;
    const long long* sw = bf.accSW + (size_t)r * K1 * m;
    // the penalty basis: S V itself, or S_1 L of the generalized process
    const long long* pv = bf.penSV ? bf.penSV + (size_t)r * K1 * m : sv;
    const double pscale = bf.penSV ? ldexp(1.0, -bf.penF) / sqrt((double)zeta) : scale;
    const int* ce = bf.colE + (size_t)r * K1;
    const int* pe = bf.penE ? bf.penE + (size_t)r * K1 : ce;
    const double* H = bf.H + (size_t)r * K1 * g.k_max;
    double* M = Mw + (size_t)r * m * (k + 1);
    double* T = Tw ? Tw + (size_t)r * m * k : nullptr;
    const double beta = bf.st->beta[r];
    const long long total = (long long)m * (kb + 1);
    // the work of column col grows with col (a sum over col + 2 terms):
    // the first blocks take the last columns, so the heaviest blocks start
    // first and the light ones fill the SMs behind them
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int cr = (int)(t / m), row = (int)(t - (long long)cr * m);
        const int col = kb - cr;
        double val;
        if (qmr) {
            if (col < kb) val = row <= col + 1 ? H[(size_t)K1 * col + row] : 0.0;
            else val = row == 0 ? beta : 0.0;
        } else if (bf.svd) {
            // Gaussian sketch: S V from the solve-time GEMM, c = S b
            auto svx = [&](int i) -> double {
                return bf.svd_f64 ? ((const double*)bf.svd)[(size_t)i * m + row]
                                  : (double)((const float*)bf.svd)[(size_t)i * m + row];
            };
            if (col < kb) {
                double s = 0.0;
                const double* Hc = H + (size_t)K1 * col;
                for (int i = 0; i <= col + 1; ++i) s = fma(svx(i), Hc[i], s);
                val = s;
                if (need_T) T[(size_t)col * m + row] = svx(col);
            } else {
                val = bf.cvec[row];
            }
        } else if (col < kb) {
            // Ww holds (double)sv * col_scale for every column: the same
            // factors, so the same bits as forming them here
            double s = 0.0;
            const double* Hc = H + (size_t)K1 * col;
            const double* W = Ww + (size_t)r * m * (k + 2) + row;
            for (int i = 0; i <= col; ++i) s = fma(W[(size_t)i * m], Hc[i], s);
            const long long* last = use_sw ? sw : sv;
            val = fma((double)last[(size_t)(col + 1) * m + row] * col_scale(scale, ce[col + 1]), Hc[col + 1], s);
            if (need_T) T[(size_t)col * m + row] = (double)pv[(size_t)col * m + row] * col_scale(pscale, pe[col]);
        } else {
            val = beta * (double)sw[row] * col_scale(scale, ce[0]);
        }
        M[(size_t)col * m + row] = val;
    }
}

// ------------------------------------------------------------------------
// cooperative Householder QR (R only).  job = 2*r + which (which 0: M with
// kb+1 columns, 1: T with kb columns).  cpj CTAs per job.
// ------------------------------------------------------------------------
// every thread gets the same sum: a shuffle tree per warp, then warp 0 adds
// the warps' sums by a second tree and shares the total (one warp doing
// those adds instead of every thread: FP64 issue is the scarce resource)
__device__ __forceinline__ double block_sum(double v, double* s_red) {
    __shared__ double s_total;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) s_red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        double t = lane < nw ? s_red[lane] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
            if (off < nw) t += __shfl_xor_sync(0xffffffffu, t, off);
        if (lane == 0) s_total = t;
    }
    __syncthreads();
    return s_total;
}

// bounded wait by thread 0 for a column flag set by another CTA of the job;
// every thread returns the same verdict (false: gave up or another CTA failed)
__device__ __forceinline__ bool wait_flag(const unsigned* flag, int* err) {
    __shared__ int s_fail;
    if (threadIdx.x == 0) {
        s_fail = 0;
        long long spins = 0;
        for (;;) {
            // acquire: the reflector written before the flag's release is
            // visible to this CTA once the barrier below has passed
            unsigned f;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(f) : "l"(flag) : "memory");
            if (f != 0u) break;
            if (*(volatile int*)err) { s_fail = 1; break; }
            if (++spins > (1ll << 22)) { atomicExch(err, 1); s_fail = 1; break; }
            __nanosleep(32);
        }
    }
    __syncthreads();
    return s_fail == 0;
}

// Reflector for column i (rows i..m-1 of col, every earlier reflector
// already applied): v = (col(i+1..) / (alpha - beta)) with v(i) = 1,
// tau = (beta - alpha) / beta, R(i,i) = beta.  v goes to buf (rows i..m-1)
// and back into the column below the diagonal, tau into the column's
// diagonal slot (R(i,i) lives in diag), then the column's flag is raised.
// col is the working copy (shared memory or the column itself); gcol, if
// not col, is the column in global memory, where v and tau are published.
__device__ __forceinline__ void make_reflector(double* col, double* gcol, int i, int m, double* buf, double* diag,
                                               unsigned* flag, double* s_red, double* s_tau) {
    __shared__ double s_inv;
    double part = 0.0;
    for (int row = i + threadIdx.x; row < m; row += blockDim.x) {
        const double x = col[row];
        buf[row] = x;
        if (row > i) part = fma(x, x, part);
    }
    const double sigma = block_sum(part, s_red);
    if (threadIdx.x == 0) {
        const double alpha = buf[i];
        double beta, tau, inv;
        if (sigma == 0.0) { beta = alpha; tau = 0.0; inv = 0.0; }
        else {
            const double nrm = sqrt(fma(alpha, alpha, sigma));
            beta = alpha <= 0.0 ? nrm : -nrm;
            tau = (beta - alpha) / beta;
            inv = 1.0 / (alpha - beta);
        }
        *diag = beta;
        *s_tau = tau;
        s_inv = inv;
        buf[i] = 1.0;
        col[i] = tau;
        if (gcol != col) gcol[i] = tau;
    }
    __syncthreads();
    const double inv = s_inv;
    for (int row = i + 1 + threadIdx.x; row < m; row += blockDim.x) {
        const double v = buf[row] * inv;
        buf[row] = v;
        col[row] = v;
        if (gcol != col) gcol[row] = v;
    }
    // the CTA's stores of v and tau, ordered before thread 0 by the barrier,
    // are published by the flag's release (cumulative at GPU scope)
    __syncthreads();
    if (threadIdx.x == 0) asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(flag), "r"(1u) : "memory");
}

// col -= tau v (v^T col) over rows i..m-1, the whole CTA (latency path)
__device__ __forceinline__ void apply_block(const double* v, double tau, double* col, int i, int m, double* s_red) {
    double d = 0.0;
    for (int row = i + threadIdx.x; row < m; row += blockDim.x) d = fma(v[row], col[row], d);
    const double f = tau * block_sum(d, s_red);
    for (int row = i + threadIdx.x; row < m; row += blockDim.x) col[row] = fma(-f, v[row], col[row]);
    __syncthreads();
}

// Householder QR (R only), pipelined by columns instead of a grid barrier
// per column.  Column j belongs to CTA j mod cpj of its job.  Reflector i is
// published by its owner (vector in the column below the diagonal, tau in
// the diagonal slot, then a flag); a CTA waits only for the flag of the
// reflector it applies next, and applies reflectors in order.  The owner of
// column i+1 applies reflector i to that column first and publishes
// reflector i+1 at once (lookahead), before its other columns; two shared
// buffers hold v_i and v_{i+1}.  csm: the CTA's own columns are worked on
// in shared memory (after the two buffers, m doubles each) and written back
// at the end, so the chain from one reflector to the next (apply it to the
// next column, form that column's reflector) reads and writes no global
// memory except the published reflector.  Cooperative launch: all CTAs
// co-resident.
__global__ void __launch_bounds__(256) k_householder(Geom g, const DevState* st, int k, int need_T, int cpj, int csm,
                                                      double* Mw, double* Tw, double* dM, double* dT,
                                                      unsigned* flags, int* err) {
    extern __shared__ unsigned char smem_raw[];
    const int m = g.m_s;
    double* s_buf = (double*)smem_raw;        // 2 x m doubles, then the own columns (csm)
    __shared__ double s_red[32];
    __shared__ double s_tau[2];
    const int jobs_per_rhs = need_T ? 2 : 1;
    const int job = blockIdx.x / cpj;
    const int q = blockIdx.x - job * cpj;
    const int njobs = g.B * jobs_per_rhs;
    if (job >= njobs) return;
    const int r = job / jobs_per_rhs, which = job - r * jobs_per_rhs;
    const int kb = kuse_of(st, r, k);
    double* A;
    double* diag;
    int ncols;
    if (which == 0) { A = Mw + (size_t)r * m * (k + 1); diag = dM + (size_t)r * (k + 1); ncols = kb + 1; }
    else { A = Tw + (size_t)r * m * k; diag = dT + (size_t)r * (k + 1); ncols = kb; }
    unsigned* flag = flags + (size_t)job * (g.k_max + 2);
    const int nsteps = ncols < m ? ncols : m;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    // own column jc (jc = q mod cpj): its working copy
    double* s_cols = s_buf + 2 * (size_t)m;
    auto colp = [&](int jc) -> double* { return csm ? s_cols + (size_t)((jc - q) / cpj) * m : A + (size_t)jc * m; };
    if (csm) {
        for (int jc = q; jc < ncols; jc += cpj) {
            double* d = colp(jc);
            const double* src = A + (size_t)jc * m;
            for (int row = threadIdx.x; row < m; row += blockDim.x) d[row] = src[row];
        }
        __syncthreads();
    }
    int have = -1;                            // reflector already made here by lookahead
    for (int i = 0; i < nsteps; ++i) {
        double* v = s_buf + (size_t)(i & 1) * m;
        double* ci = A + (size_t)i * m;
        double tau;
        if (i % cpj == q) {
            if (have != i) make_reflector(colp(i), ci, i, m, v, diag + i, flag + i, s_red, &s_tau[i & 1]);
            tau = s_tau[i & 1];
        } else {
            if (!wait_flag(flag + i, err)) return;
            // written by another CTA: read through L2
            for (int row = i + 1 + threadIdx.x; row < m; row += blockDim.x) v[row] = __ldcg(ci + row);
            if (threadIdx.x == 0) { v[i] = 1.0; s_tau[i & 1] = __ldcg(ci + i); }
            __syncthreads();
            tau = s_tau[i & 1];
        }
        // owned columns j > i: j = q, q + cpj, ...
        int j0 = q;
        if (j0 <= i) j0 += ((i - q) / cpj + 1) * cpj;
        if (j0 >= ncols) break;                // no column (and no reflector) left here
        int jrest = j0;
        if (j0 == i + 1) {
            // lookahead: the next reflector's column first, then that reflector
            if (tau != 0.0) apply_block(v, tau, colp(j0), i, m, s_red);
            if (i + 1 < nsteps) {
                double* vn = s_buf + (size_t)((i + 1) & 1) * m;
                make_reflector(colp(j0), A + (size_t)j0 * m, i + 1, m, vn, diag + i + 1, flag + i + 1, s_red,
                               &s_tau[(i + 1) & 1]);
                have = i + 1;
            }
            jrest = j0 + cpj;
        }
        if (tau != 0.0) {
            int idx = 0;
            for (int jc = jrest; jc < ncols; jc += cpj, ++idx) {
                if ((idx % nw) != warp) continue;
                double* cj = colp(jc);
                double d = 0.0;
                for (int row = i + lane; row < m; row += 32) d = fma(v[row], cj[row], d);
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) d += __shfl_xor_sync(0xffffffffu, d, off);
                const double f = tau * d;
                for (int row = i + lane; row < m; row += 32) cj[row] = fma(-f, v[row], cj[row]);
            }
        }
        __syncthreads();
    }
    // the own columns back to global memory: R above the diagonal (the
    // reflectors below it and tau were published already, the same values)
    if (csm) {
        __syncthreads();
        for (int jc = q; jc < ncols; jc += cpj) {
            const double* src = colp(jc);
            double* d = A + (size_t)jc * m;
            for (int row = threadIdx.x; row < m; row += blockDim.x) d[row] = src[row];
        }
    }
    // columns beyond m (never for m_s >= k+1) have no diagonal
}

// ------------------------------------------------------------------------
// per (RHS, lambda) small solve
// ------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_small_solve(Geom g, const DevState* st, int k, int nl, const double* lams,
                                                      int penalty, const double* Mw, const double* Tw,
                                                      const double* dM, const double* dT, double* Sw, double* Yw) {
    const int r = blockIdx.x / nl, l = blockIdx.x - (blockIdx.x / nl) * nl;
    const int kb = kuse_of(st, r, k);
    const int m = g.m_s;
    const double lam = lams[l];
    const double* M = Mw + (size_t)r * m * (k + 1);
    const double* dm = dM + (size_t)r * (k + 1);
    double* y = Yw + ((size_t)r * nl + l) * (k + 1);
    __shared__ double s_red[32];
    const int ld = 2 * kb + 1;
    double* S = Sw + ((size_t)r * nl + l) * (size_t)(2 * k + 1) * (k + 1);
    // top rows 0..kb: R_M restricted to columns 0..kb-1 plus rhs column kb
    // (lambda = 0: the back substitution reads R_M in place, only the rhs
    // column is copied)
    for (int t = lam == 0.0 ? kb * ld + threadIdx.x : threadIdx.x; t < (kb + 1) * ld; t += blockDim.x) {
        const int col = t / ld, row = t - col * ld;
        double v = 0.0;
        if (row <= kb) {
            if (row < col) v = M[(size_t)col * m + row];
            else if (row == col) v = dm[col];
        } else if (lam != 0.0 && col < kb) {
            const int br = row - kb - 1;          // bottom row index
            if (penalty == IPF_PEN_Y) v = (br == col) ? lam : 0.0;
            else {
                const double* T = Tw + (size_t)r * m * k;
                const double* dt = dT + (size_t)r * (k + 1);
                if (br < col) v = lam * T[(size_t)col * m + br];
                else if (br == col) v = lam * dt[col];
            }
        }
        S[(size_t)col * ld + row] = v;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (lam != 0.0) {
        for (int i = 0; i < kb; ++i) {
            // x = [top(i,i); bottom(0..i, i)]
            double* ci = S + (size_t)i * ld;
            double part = 0.0;
            for (int br = threadIdx.x; br <= i; br += blockDim.x) { const double x = ci[kb + 1 + br]; part = fma(x, x, part); }
            const double sigma = block_sum(part, s_red);
            const double alpha = ci[i];
            double beta, tau, inv;
            if (sigma == 0.0) { beta = alpha; tau = 0.0; inv = 0.0; }
            else {
                const double nrm = sqrt(fma(alpha, alpha, sigma));
                beta = alpha <= 0.0 ? nrm : -nrm;
                tau = (beta - alpha) / beta;
                inv = 1.0 / (alpha - beta);
            }
            __syncthreads();
            if (tau != 0.0) {
                for (int jc = i + 1 + warp; jc <= kb; jc += nw) {
                    double* cj = S + (size_t)jc * ld;
                    double d = (lane == 0) ? cj[i] : 0.0;
                    for (int br = lane; br <= i; br += 32) d = fma(ci[kb + 1 + br] * inv, cj[kb + 1 + br], d);
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) d += __shfl_xor_sync(0xffffffffu, d, off);
                    const double f = tau * d;
                    if (lane == 0) cj[i] -= f;
                    for (int br = lane; br <= i; br += 32) cj[kb + 1 + br] = fma(-f, ci[kb + 1 + br] * inv, cj[kb + 1 + br]);
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) ci[i] = beta;
            for (int br = threadIdx.x; br <= i; br += blockDim.x) ci[kb + 1 + br] = 0.0;
            __syncthreads();
        }
    }
    // back substitution top(0:kb, 0:kb) y = top(0:kb, kb) in blocks of 32
    // rows from the bottom: warp 0 solves a block's diagonal triangle alone
    // (y_i by a shuffle from the lane holding row i; the reciprocals of the
    // diagonal are formed in parallel first: FP64 division is scarce on
    // this GPU), one barrier publishes the block's y, and every thread
    // applies the block's columns to the rows above it.  Each row still
    // takes its updates in decreasing column order.
    __shared__ double s_inv[kSmallMaxK];
    double* rhs = S + (size_t)kb * ld;
    // R(row, i), row <= i: from R_M itself (lambda = 0) or the stacked QR
    auto Rv = [&](int row, int i) -> double {
        if (lam == 0.0) return row < i ? M[(size_t)i * m + row] : dm[i];
        return S[(size_t)i * ld + row];
    };
    for (int i = threadIdx.x; i < kb; i += blockDim.x) {
        const double d = Rv(i, i);
        s_inv[i] = d != 0.0 ? 1.0 / d : 0.0;
    }
    __syncthreads();
    // the diagonal block's triangle, staged by the whole CTA (coalesced along
    // columns) so that warp 0's chain of 32 dependent steps reads shared
    // memory instead of waiting on a global load per step
    __shared__ double s_blk[32][33];
    for (int hi = kb; hi > 0; hi -= 32) {
        const int lo = hi > 32 ? hi - 32 : 0;
        for (int t = threadIdx.x; t < 32 * 32; t += blockDim.x) {
            const int c = t >> 5, r = t & 31;                // column lo + c, row lo + r
            if (lo + c < hi && r < c) s_blk[r][c] = Rv(lo + r, lo + c);
        }
        __syncthreads();
        if (warp == 0) {
            const int row = lo + lane;                       // this lane's row of the block
            double b = row < hi ? rhs[row] : 0.0;
            for (int i = hi - 1; i >= lo; --i) {
                const double yi = __shfl_sync(0xffffffffu, b * s_inv[i < 0 ? 0 : i], i - lo);
                if (lane == 0) y[i] = yi;
                if (row < i) b = fma(-s_blk[lane][i - lo], yi, b);
                if (lane == i - lo) b = yi;                  // row i now holds y_i
            }
            if (row < hi) rhs[row] = b;                      // y of the block, for the rows above
        }
        __syncthreads();
        for (int row = threadIdx.x; row < lo; row += blockDim.x) {
            double b = rhs[row];
            for (int i = hi - 1; i >= lo; --i) b = fma(-Rv(row, i), rhs[i], b);
            rhs[row] = b;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------
// x = V_k y for up to NL lambdas in one pass over V_k; output [l][r][i].
// Each thread owns 16 bytes of every basis column per pass and keeps eight
// 128-bit column loads in flight.
// ------------------------------------------------------------------------
template <class T, int NL>
__global__ void __launch_bounds__(256) k_reconstruct(Geom g, Bufs bf, const DevState* st, int k, int nl,
                                                      const double* Yw, int l0, int nlc, float* x) {
    using Acc = typename AccOf<T>::type;
    constexpr int VEC = 16 / sizeof(T);
    extern __shared__ unsigned char smem_raw[];
    Acc* s_y = (Acc*)smem_raw;                 // [NL][B][k]
    __shared__ int s_kb[kMaxRhs];
    const int B = g.B;
    if (threadIdx.x < B) s_kb[threadIdx.x] = kuse_of(st, threadIdx.x, k);
    __syncthreads();
    for (int t = threadIdx.x; t < NL * B * k; t += blockDim.x) {
        const int l = t / (B * k), rem = t - l * B * k, r = rem / k, c = rem - r * k;
        s_y[t] = (l < nlc && c < s_kb[r]) ? (Acc)Yw[((size_t)r * nl + l0 + l) * (k + 1) + c] : (Acc)0;
    }
    int kmax = 0;
    for (int r = 0; r < B; ++r) kmax = s_kb[r] > kmax ? s_kb[r] : kmax;
    __syncthreads();
    const T* V = (const T*)bf.V;
    const size_t ldv = (size_t)g.ldv;
    const long long stride = (long long)gridDim.x * blockDim.x * VEC;
    for (long long base = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * VEC; base < g.N; base += stride) {
        Acc acc[NL][VEC];
#pragma unroll
        for (int l = 0; l < NL; ++l)
#pragma unroll
            for (int q = 0; q < VEC; ++q) acc[l][q] = 0;
        const T* vb = V + base;
        int c = 0;
        for (; c + 8 <= kmax; c += 8) {
            uint4 raw[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) raw[u] = __ldcs((const uint4*)(vb + (size_t)(c + u) * ldv));
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const T* vv = (const T*)&raw[u];
#pragma unroll
                for (int q = 0; q < VEC; ++q) {
                    const int rr = (int)((base + q) & (B - 1));
                    const Acc vq = to_acc(vv[q]);
#pragma unroll
                    for (int l = 0; l < NL; ++l) acc[l][q] = fma(s_y[((size_t)l * B + rr) * k + c + u], vq, acc[l][q]);
                }
            }
        }
        for (; c < kmax; ++c) {
            const uint4 r1 = __ldcs((const uint4*)(vb + (size_t)c * ldv));
            const T* vv = (const T*)&r1;
#pragma unroll
            for (int q = 0; q < VEC; ++q) {
                const int rr = (int)((base + q) & (B - 1));
                const Acc vq = to_acc(vv[q]);
#pragma unroll
                for (int l = 0; l < NL; ++l) acc[l][q] = fma(s_y[((size_t)l * B + rr) * k + c], vq, acc[l][q]);
            }
        }
#pragma unroll
        for (int q = 0; q < VEC; ++q) {
            const long long e = base + q;
            if (e >= g.N) break;
            const long long i = e / B;
            const int rr = (int)(e - i * B);
#pragma unroll
            for (int l = 0; l < NL; ++l)
                if (l < nlc) x[((size_t)(l0 + l) * B + rr) * g.n + i] = (float)acc[l][q];
        }
    }
}

}  // namespace

size_t solve_workspace_bytes(const Geom& g, int nl_max) { return layout_for(g, nl_max).total; }

cudaError_t solve_error_flag(const void* work, const Geom& g, int* flag) {
    const SolveLayout L = layout_for(g, 1);          // err_off does not depend on nl_max
    return cudaMemcpy(flag, (const char*)work + L.err_off, sizeof(int), cudaMemcpyDeviceToHost);
}

cudaError_t launch_solve_prepare(const Geom& g, const Bufs& bf, int zeta, int k, bool need_T, bool use_sw,
                                 void* work, int nl_max, int num_sms, cudaStream_t s, bool qmr) {
    SolveLayout L = layout_for(g, nl_max);
    char* base = (char*)work;
    double* Mw = (double*)(base + L.M_off);
    double* Tw = need_T ? (double*)(base + L.T_off) : nullptr;
    double* dM = (double*)(base + L.dM_off);
    double* dT = (double*)(base + L.dT_off);
    unsigned* bars = (unsigned*)(base + L.bar_off);
    int* err = (int*)(base + L.err_off);
    double* Ww = (double*)(base + L.W_off);
    cudaError_t e = cudaMemsetAsync(base, 0, L.M_off, s);
    if (e != cudaSuccess) return e;
    {
        dim3 grid((unsigned)((g.m_s * (k + 1) + 255) / 256), (unsigned)g.B);
        if (!qmr && !bf.svd) k_scale_sv<<<grid, 256, 0, s>>>(g, bf, k, zeta, Ww);
        k_form<<<grid, 256, 0, s>>>(g, bf, k, zeta, use_sw ? 1 : 0, need_T ? 1 : 0, Mw, Tw, qmr ? 1 : 0, Ww);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const int njobs = g.B * (need_T ? 2 : 1);
    // CTAs per job from the occupancy with the two reflector buffers, then
    // the own columns in shared memory too if all CTAs still co-reside
    size_t smem = 2 * sizeof(double) * (size_t)g.m_s;
    auto blocks_for = [&](size_t bytes, int* out) -> cudaError_t {
        cudaError_t ee = raise_smem(k_householder, (int)bytes);
        if (ee != cudaSuccess) return ee;
        int occ = 0;
        ee = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_householder, 256, bytes);
        *out = (occ < 1 ? 0 : occ) * num_sms;
        return ee;
    };
    int maxblocks = 0;
    if ((e = blocks_for(smem, &maxblocks)) != cudaSuccess) return e;
    if (maxblocks < 1) maxblocks = num_sms;
    int cpj = maxblocks / njobs;
    if (cpj > (k + 2) / 2) cpj = (k + 2) / 2;
    if (cpj < 1) cpj = 1;
    if (cpj * njobs > maxblocks) return cudaErrorInvalidConfiguration;   // cannot co-reside
    int csm = 0;
    const size_t own = (size_t)(k + 1 + cpj - 1) / cpj;                    // columns per CTA, at most
    const size_t smem_c = (2 + own) * sizeof(double) * (size_t)g.m_s;
    if (smem_c <= 200 * 1024) {
        int mb = 0;
        if (blocks_for(smem_c, &mb) == cudaSuccess && cpj * njobs <= mb) {
            csm = 1;
            smem = smem_c;
        }
    }
    const int nb = cpj * njobs;
    Geom gg = g;
    const DevState* stp = bf.st;
    int kk = k, nt = need_T ? 1 : 0, cp = cpj, cs = csm;
    void* args[] = {&gg, (void*)&stp, &kk, &nt, &cp, &cs, &Mw, &Tw, &dM, &dT, &bars, &err};
    return cudaLaunchCooperativeKernel((void*)k_householder, dim3(nb), dim3(256), args, smem, s);
}

cudaError_t launch_solve_lambdas(int storage, const Geom& g, const Bufs& bf, int k, bool need_T,
                                 const double* lambdas_dev, int nl, int penalty, void* work, int nl_max,
                                 float* x_dev, int num_sms, cudaStream_t s) {
    if (nl > nl_max) return cudaErrorInvalidValue;
    SolveLayout L = layout_for(g, nl_max);
    char* base = (char*)work;
    const double* Mw = (const double*)(base + L.M_off);
    const double* Tw = need_T ? (const double*)(base + L.T_off) : nullptr;
    const double* dM = (const double*)(base + L.dM_off);
    const double* dT = (const double*)(base + L.dT_off);
    double* Yw = (double*)(base + L.Y_off);
    double* Sw = (double*)(base + L.S_off);
    if (penalty == IPF_PEN_SKETCHED_X && !need_T) penalty = IPF_PEN_Y;   // no lambda > 0 in this call
    k_small_solve<<<g.B * nl, 256, 0, s>>>(g, bf.st, k, nl, lambdas_dev, penalty, Mw, Tw, dM, dT, Sw, Yw);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !x_dev) return e;
    // lambdas in chunks whose y fit in shared memory next to each other
    const size_t accsz = storage == IPF_STORE_F64 ? 8 : 4;
    int cap = 8;
    while (cap > 1 && accsz * cap * g.B * (k > 0 ? k : 1) > 96 * 1024) cap >>= 1;
    for (int l0 = 0; l0 < nl; l0 += cap) {
        const int nlc = nl - l0 < cap ? nl - l0 : cap;
        const int NLp = nlc <= 1 ? 1 : nlc <= 2 ? 2 : nlc <= 4 ? 4 : 8;
        auto launch = [&](auto kern, int vec) -> cudaError_t {
            const size_t smem = accsz * (size_t)NLp * g.B * (k > 0 ? k : 1);
            cudaError_t ee = raise_smem(kern, (int)smem);
            if (ee != cudaSuccess) return ee;
            long long chunks = (g.N + 256LL * vec - 1) / (256LL * vec);
            long long blocks = (long long)num_sms * 4;
            if (blocks > chunks) blocks = chunks < 1 ? 1 : chunks;
            kern<<<(int)blocks, 256, smem, s>>>(g, bf, bf.st, k, nl, Yw, l0, nlc, x_dev);
            return cudaGetLastError();
        };
        auto byNL = [&](auto tag, int vec) -> cudaError_t {
            using T = decltype(tag);
            switch (NLp) {
                case 1: return launch(k_reconstruct<T, 1>, vec);
                case 2: return launch(k_reconstruct<T, 2>, vec);
                case 4: return launch(k_reconstruct<T, 4>, vec);
                default: return launch(k_reconstruct<T, 8>, vec);
            }
        };
        switch (storage) {
            case IPF_STORE_F64: e = byNL(double(), 2); break;
            case IPF_STORE_F32: e = byNL(float(), 4); break;
            case IPF_STORE_BF16: e = byNL(__nv_bfloat16(), 8); break;
            case IPF_STORE_F16: e = byNL(__half(), 8); break;
            default: return cudaErrorInvalidValue;
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace ipf
