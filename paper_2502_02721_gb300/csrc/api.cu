// Host side of the C ABI declared in include/ipf.h: contexts, device memory,
// the per-step launch sequence (captured once in a CUDA graph and replayed),
// the projected solve, state export, and the standalone operator and sketch
// calls.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "ipf_internal.cuh"

using namespace ipf;

namespace {

constexpr int kLamChunk = 16;

size_t storage_bytes(int storage) {
    switch (storage) {
        case IPF_STORE_F64: return 8;
        case IPF_STORE_F32: return 4;
        default: return 2;
    }
}

int device_sms() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    return sms > 0 ? sms : 1;
}

bool pow2_le32(int b) { return b >= 1 && b <= 32 && (b & (b - 1)) == 0; }

long long op_n(const ipf_operator* op) {
    if (op->kind == IPF_OP_CSR) return op->cols;
    return (long long)op->rows * op->cols;
}

// length of A's output (the m-space of the generalized process)
long long op_m(const ipf_operator* op) {
    if (op->kind == IPF_OP_CSR) return op->rows;
    return (long long)op->rows * op->cols;
}

struct Alloc {
    ipf_alloc_fn fa = nullptr;
    ipf_free_fn ff = nullptr;
    void* user = nullptr;
    std::vector<void*> live;
    cudaError_t get(void** p, size_t bytes) {
        bytes = (bytes + 255) & ~(size_t)255;
        if (bytes == 0) bytes = 256;
        if (fa) {
            *p = fa(bytes, user);
            if (!*p) return cudaErrorMemoryAllocation;
        } else {
            cudaError_t e = cudaMalloc(p, bytes);
            if (e != cudaSuccess) return e;
        }
        live.push_back(*p);
        return cudaSuccess;
    }
    void release() {
        for (void* p : live) {
            if (ff) ff(p, user);
            else cudaFree(p);
        }
        live.clear();
    }
};

std::string fmt_cuda(const char* what, cudaError_t e) {
    return std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
}

// operator validation shared by ipf_create and ipf_op_create
ipf_status check_op(const ipf_operator* op, int nrhs, std::string* why) {
    if (!op) { *why = "operator is NULL"; return IPF_ERR_ARG; }
    if (op->rows <= 0 || op->cols <= 0) { *why = "operator rows/cols must be positive"; return IPF_ERR_ARG; }
    if (op->mem != IPF_MEM_HOST && op->mem != IPF_MEM_DEVICE) { *why = "operator mem flag"; return IPF_ERR_ARG; }
    switch (op->kind) {
        case IPF_OP_PSF2D:
            if (!op->psf || op->ph <= 0 || op->pw <= 0 || !(op->ph & 1) || !(op->pw & 1) || op->ph > 63 || op->pw > 63) {
                *why = "PSF2D needs an odd ph x pw PSF, sizes <= 63"; return IPF_ERR_ARG;
            }
            if (nrhs != 1) { *why = "PSF operators take one right-hand side per context"; return IPF_ERR_UNSUPPORTED; }
            return IPF_OK;
        case IPF_OP_PSF2D_SEP_MOTION:
            if (!op->sep_row || !op->sep_col || !op->motion || op->slen <= 0 || !(op->slen & 1) || op->slen > 63 ||
                op->mlen <= 0 || !(op->mlen & 1) || op->mlen > 15) {
                *why = "separable+motion needs odd slen <= 63 and odd mlen <= 15"; return IPF_ERR_ARG;
            }
            if (nrhs != 1) { *why = "PSF operators take one right-hand side per context"; return IPF_ERR_UNSUPPORTED; }
            return IPF_OK;
        case IPF_OP_CSR:
            if (!op->rowptr || (op->nnz > 0 && (!op->colind || !op->vals)) || op->nnz < 0) {
                *why = "CSR needs rowptr, colind, vals"; return IPF_ERR_ARG;
            }
            if (op->mem == IPF_MEM_HOST) {
                // host arrays are checked here so no kernel can index out of bounds;
                // device arrays are the caller's responsibility (documented in ipf.h)
                if (op->rowptr[0] != 0 || op->rowptr[op->rows] != op->nnz) {
                    *why = "CSR rowptr must start at 0 and end at nnz"; return IPF_ERR_ARG;
                }
                for (int r = 0; r < op->rows; ++r)
                    if (op->rowptr[r + 1] < op->rowptr[r]) { *why = "CSR rowptr must be non-decreasing"; return IPF_ERR_ARG; }
                for (long long t = 0; t < op->nnz; ++t)
                    if (op->colind[t] < 0 || op->colind[t] >= op->cols) { *why = "CSR column index out of range"; return IPF_ERR_ARG; }
            }
            return IPF_OK;
        default:
            *why = "unknown operator kind"; return IPF_ERR_ARG;
    }
}

// copy an operator to the device; CSR arrays already on the device are referenced
cudaError_t upload_op(const ipf_operator* op, Alloc& al, OpDev* d, cudaStream_t s) {
    memset(d, 0, sizeof(*d));
    d->kind = op->kind;
    d->rows = op->rows;
    d->cols = op->cols;
    const cudaMemcpyKind kind = op->mem == IPF_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    auto dup = [&](const void* src, size_t bytes, const void** dst) -> cudaError_t {
        void* p = nullptr;
        cudaError_t e = al.get(&p, bytes);
        if (e != cudaSuccess) return e;
        e = cudaMemcpyAsync(p, src, bytes, kind, s);
        *dst = p;
        return e;
    };
    cudaError_t e = cudaSuccess;
    if (op->kind == IPF_OP_PSF2D) {
        d->ph = op->ph; d->pw = op->pw;
        e = dup(op->psf, sizeof(float) * op->ph * op->pw, (const void**)&d->psf);
        if (e != cudaSuccess) return e;
        // packed pairs {F[ky][b], F[ky-1][b]} of the flipped PSF, zero-padded to a
        // square kw x kw, for the packed-FMA column convolution
        const int mk = op->ph > op->pw ? op->ph : op->pw;
        const int kw = mk <= 7 ? 7 : mk <= 15 ? 15 : mk <= 31 ? 31 : 0;
        if (kw) {
            std::vector<float> P((size_t)op->ph * op->pw);
            if (op->mem == IPF_MEM_HOST) memcpy(P.data(), op->psf, P.size() * sizeof(float));
            else if ((e = cudaMemcpy(P.data(), op->psf, P.size() * sizeof(float), cudaMemcpyDeviceToHost)) != cudaSuccess)
                return e;
            const int pady = (kw - op->ph) / 2, padx = (kw - op->pw) / 2;
            auto F = [&](int a, int bb) -> float {
                const int ka = a - pady, kb = bb - padx;
                if (a < 0 || a >= kw || ka < 0 || ka >= op->ph || kb < 0 || kb >= op->pw) return 0.f;
                return P[(size_t)(op->ph - 1 - ka) * op->pw + (op->pw - 1 - kb)];
            };
            std::vector<unsigned long long> pairs((size_t)kw * (kw + 1));
            for (int bb = 0; bb < kw; ++bb)
                for (int ky = 0; ky <= kw; ++ky) {
                    const float lo = F(ky, bb), hi = F(ky - 1, bb);
                    unsigned ulo, uhi;
                    memcpy(&ulo, &lo, 4);
                    memcpy(&uhi, &hi, 4);
                    pairs[(size_t)bb * (kw + 1) + ky] = (unsigned long long)ulo | ((unsigned long long)uhi << 32);
                }
            void* pp = nullptr;
            if ((e = al.get(&pp, pairs.size() * 8)) != cudaSuccess) return e;
            if ((e = cudaMemcpy(pp, pairs.data(), pairs.size() * 8, cudaMemcpyHostToDevice)) != cudaSuccess) return e;
            d->kw = kw;
            d->psf_pairs = (const unsigned long long*)pp;
            std::vector<unsigned short> img;
            const int KP = conv_tc_operand(kw, F, &img);
            if (KP) {
                void* pt = nullptr;
                if ((e = al.get(&pt, img.size() * 2)) != cudaSuccess) return e;
                if ((e = cudaMemcpy(pt, img.data(), img.size() * 2, cudaMemcpyHostToDevice)) != cudaSuccess) return e;
                d->tc_kp = KP;
                d->psf_tc = pt;
            }
        }
    } else if (op->kind == IPF_OP_PSF2D_SEP_MOTION) {
        d->slen = op->slen; d->mlen = op->mlen;
        if ((e = dup(op->sep_row, sizeof(float) * op->slen, (const void**)&d->sep_row)) != cudaSuccess) return e;
        if ((e = dup(op->sep_col, sizeof(float) * op->slen, (const void**)&d->sep_col)) != cudaSuccess) return e;
        e = dup(op->motion, sizeof(float) * op->mlen * op->mlen, (const void**)&d->motion);
    } else {
        d->nnz = op->nnz;
        if (op->mem == IPF_MEM_DEVICE) {
            d->rowptr = op->rowptr; d->colind = op->colind; d->vals = op->vals;
        } else {
            if ((e = dup(op->rowptr, sizeof(long long) * (op->rows + 1), (const void**)&d->rowptr)) != cudaSuccess) return e;
            if ((e = dup(op->colind, sizeof(int) * (op->nnz > 0 ? op->nnz : 1), (const void**)&d->colind)) != cudaSuccess) return e;
            e = dup(op->vals, sizeof(float) * (op->nnz > 0 ? op->nnz : 1), (const void**)&d->vals);
        }
    }
    return e;
}

// upload A^T: the convolution with the flipped PSF, or the CSR transpose
// (built on the host; device CSR arrays are read back once)
cudaError_t upload_transpose(const ipf_operator* op, Alloc& al, OpDev* d, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    ipf_operator t = *op;
    t.mem = IPF_MEM_HOST;
    if (op->kind == IPF_OP_PSF2D) {
        const size_t np = (size_t)op->ph * op->pw;
        std::vector<float> P(np), Pf(np);
        if (op->mem == IPF_MEM_HOST) memcpy(P.data(), op->psf, np * sizeof(float));
        else if ((e = cudaMemcpy(P.data(), op->psf, np * sizeof(float), cudaMemcpyDeviceToHost)) != cudaSuccess)
            return e;
        for (int a = 0; a < op->ph; ++a)
            for (int b = 0; b < op->pw; ++b)
                Pf[(size_t)a * op->pw + b] = P[(size_t)(op->ph - 1 - a) * op->pw + (op->pw - 1 - b)];
        t.psf = Pf.data();
        if ((e = upload_op(&t, al, d, s)) != cudaSuccess) return e;
        return cudaStreamSynchronize(s);
    }
    if (op->kind != IPF_OP_CSR) return cudaErrorInvalidValue;
    const int m = op->rows, n = op->cols;
    const long long nnz = op->nnz;
    std::vector<long long> rp(m + 1);
    std::vector<int> ci(nnz > 0 ? nnz : 1);
    std::vector<float> va(nnz > 0 ? nnz : 1);
    if (op->mem == IPF_MEM_HOST) {
        memcpy(rp.data(), op->rowptr, sizeof(long long) * (m + 1));
        if (nnz) memcpy(ci.data(), op->colind, sizeof(int) * nnz);
        if (nnz) memcpy(va.data(), op->vals, sizeof(float) * nnz);
    } else {
        if ((e = cudaMemcpy(rp.data(), op->rowptr, sizeof(long long) * (m + 1), cudaMemcpyDeviceToHost)) != cudaSuccess)
            return e;
        if (nnz && (e = cudaMemcpy(ci.data(), op->colind, sizeof(int) * nnz, cudaMemcpyDeviceToHost)) != cudaSuccess)
            return e;
        if (nnz && (e = cudaMemcpy(va.data(), op->vals, sizeof(float) * nnz, cudaMemcpyDeviceToHost)) != cudaSuccess)
            return e;
    }
    // counting sort by column; entries of a column keep their row order
    std::vector<long long> rpT(n + 1, 0);
    for (long long t2 = 0; t2 < nnz; ++t2) ++rpT[ci[t2] + 1];
    for (int c2 = 0; c2 < n; ++c2) rpT[c2 + 1] += rpT[c2];
    std::vector<long long> fill(rpT.begin(), rpT.end() - 1);
    std::vector<int> ciT(nnz > 0 ? nnz : 1);
    std::vector<float> vaT(nnz > 0 ? nnz : 1);
    for (int r = 0; r < m; ++r)
        for (long long t2 = rp[r]; t2 < rp[r + 1]; ++t2) {
            const long long dst = fill[ci[t2]]++;
            ciT[dst] = r;
            vaT[dst] = va[t2];
        }
    t.rows = n;
    t.cols = m;
    t.rowptr = rpT.data();
    t.colind = ciT.data();
    t.vals = vaT.data();
    if ((e = upload_op(&t, al, d, s)) != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

}  // namespace

struct ipf_ctx {
    ipf_config cfg;
    OpDev op;
    Alloc al;
    int storage = IPF_STORE_F32;
    int B = 1;
    Geom g;
    Bufs bf;
    SketchParams sp;
    int num_sms = 1;
    cudaStream_t s = nullptr;
    cudaStream_t s2 = nullptr;          // second stream of the split step (operator branch)
    cudaStream_t user = nullptr;
    cudaEvent_t ev = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool defer_sketch = false;          // S v_{j+1} taken by the next step's update (or before a solve)
    bool split = false;                 // operator overlapped with the V_j stream
    bool fork_piv = false;              // operator overlapped with the pivot-block solve
    // generalized process (SLSLU): g/bf/sp/op are the D side (m-space, A),
    // these the L side (n-space, A^T)
    bool gh = false;
    // Gaussian sketch: S (m_s x lds, storage type, row-major), S V_{k+1},
    // c = S b and the contraction's workspace (b rows, partial tiles)
    bool gauss = false;
    void* gS = nullptr;
    void* gSV = nullptr;
    double* gC = nullptr;
    void* gWs = nullptr;
    int gvariant = 0;                   // the contraction's pipeline (gauss_variant)
    OpDev opT;
    Geom g2;
    Bufs bf2;
    SketchParams sp2;
    int j_host = 0;                    // Hessenberg steps enqueued
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph_run = nullptr;    // kGraphSteps consecutive steps in one graph
    cudaGraphExec_t gexec_run = nullptr;
    ipf_status sticky = IPF_OK;
    std::string err;
    void* solve_ws = nullptr;
    size_t solve_ws_bytes = 0;
    double* lam_dev = nullptr;
    float* x_stage = nullptr;          // B*n floats (host output path)
    float* b_stage = nullptr;          // B*n floats (host b)
    // profile mode: event pairs recorded around each kernel
    struct Mark { int kind; double bytes; cudaEvent_t a, b; };
    std::vector<Mark> marks;
    std::vector<cudaEvent_t> spare;
    double prof_ms[kProfKinds] = {0};
    long long prof_n[kProfKinds] = {0};
    double prof_bytes[kProfKinds] = {0};
};

struct ipf_op {
    OpDev op;
    Alloc al;
};

namespace {

ipf_status fail(ipf_ctx* c, ipf_status st, const std::string& msg) {
    if (c) {
        if (c->sticky == IPF_OK) {
            c->sticky = st;
            c->err = msg;
        }
    }
    return st;
}

ipf_status cuda_fail(ipf_ctx* c, const char* what, cudaError_t e) {
    return fail(c, e == cudaErrorMemoryAllocation ? IPF_ERR_OOM : IPF_ERR_CUDA, fmt_cuda(what, e));
}

// user stream -> ctx stream ordering
cudaError_t enter(ipf_ctx* c) {
    cudaError_t e = cudaEventRecord(c->ev, c->user);
    if (e != cudaSuccess) return e;
    return cudaStreamWaitEvent(c->s, c->ev, 0);
}
cudaError_t leave(ipf_ctx* c) {
    cudaError_t e = cudaEventRecord(c->ev, c->s);
    if (e != cudaSuccess) return e;
    return cudaStreamWaitEvent(c->user, c->ev, 0);
}

}  // namespace

namespace {

cudaEvent_t take_event(ipf_ctx* c) {
    if (!c->spare.empty()) {
        cudaEvent_t e = c->spare.back();
        c->spare.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// run one launch, bracketed by events in profile mode
template <class F>
cudaError_t timed_on(ipf_ctx* c, cudaStream_t st, int kind, double bytes, F&& launch) {
    if (!c->cfg.profile) return launch();
    ipf_ctx::Mark m{kind, bytes, take_event(c), take_event(c)};
    cudaError_t e = cudaEventRecord(m.a, st);
    if (e != cudaSuccess) return e;
    e = launch();
    if (e != cudaSuccess) return e;
    e = cudaEventRecord(m.b, st);
    c->marks.push_back(m);
    return e;
}

template <class F>
cudaError_t timed(ipf_ctx* c, int kind, double bytes, F&& launch) {
    return timed_on(c, c->s, kind, bytes, launch);
}

size_t acc_bytes(const ipf_ctx* c) { return c->storage == IPF_STORE_F64 ? 8 : 4; }

double op_bytes(const ipf_ctx* c) {
    const double N = (double)c->g.N, sv = (double)storage_bytes(c->storage), ab = (double)acc_bytes(c);
    double b = N * sv + N * ab;
    if (c->op.kind == IPF_OP_CSR) b += (double)c->op.nnz * 8.0 + (double)(c->op.rows + 1) * 8.0;
    return b;
}

// the unrounded normalised vector differs from the stored one only for
// BF16/FP16 storage; its sketch then gives the DIRECT z_j by linearity
bool sw_on(const ipf_ctx* c) {
    return c->g.want_z && (c->storage == IPF_STORE_BF16 || c->storage == IPF_STORE_F16);
}

// sampled pivoting (config.pivot_sample > 0): after the update has left the
// full-max key, replace it by the largest |w| of the sample.  The second basis
// of the generalized process draws from its own seed.
cudaError_t sample_pivot(ipf_ctx* c, const Geom& g, const Bufs& bf) {
    if (c->cfg.pivot_sample <= 0) return cudaSuccess;
    const unsigned long long seed = c->cfg.seed ^ 0xA5A5A5A5A5A5A5A5ull ^
                                    (bf.st == c->bf.st ? 0ull : 0x5DEECE66DA3B1F27ull);
    return timed(c, 10, 0.0, [&] { return launch_sample_pivot(c->storage, g, bf, seed, c->cfg.pivot_sample, c->s); });
}

// the deferred sketch of the pending column on `st` (a no-op kernel when
// nothing is pending)
cudaError_t sketch_pending(ipf_ctx* c, cudaStream_t st) {
    if (!c->defer_sketch) return cudaSuccess;
    const double b = (double)c->g.N * storage_bytes(c->storage) + (double)c->g.n * 8.0;
    return timed_on(c, st, 11, b, [&] { return launch_sketch_col(c->storage, c->g, c->bf, c->sp, c->num_sms, st); });
}

// one Hessenberg step; every kernel takes j from device memory, so the same
// sequence serves every step and can be captured once.  `j` (host count) is
// only used to label profile bytes.
// half of a generalized step: the operator applied to the other basis's
// newest column, then this basis's elimination, update and normalisation
cudaError_t half_step(ipf_ctx* c, const OpDev& op, const Bufs& in, const Geom& gin, const Geom& g, const Bufs& bf,
                      const SketchParams& sp, int j) {
    cudaError_t e;
    const double N = (double)g.N, sv = (double)storage_bytes(c->storage), ab = (double)acc_bytes(c);
    const double ob = (double)gin.N * sv + N * ab +
                      (op.kind == IPF_OP_CSR ? (double)op.nnz * 8.0 + (double)(op.rows + 1) * 8.0 : 0.0);
    if ((e = timed(c, 0, ob, [&] {
             return launch_op_apply(op, c->storage, in.V, gin.ldv, gin.k_max + 1, &in.st->j, c->B, bf.w,
                                    bf.st->status, c->s);
         })) != cudaSuccess)
        return e;
    if ((e = timed(c, 1, 0.0, [&] { return launch_pivot_solve(c->storage, g, bf, c->s); })) != cudaSuccess) return e;
    if ((e = timed(c, 2, (double)(j + 1) * N * sv + 2.0 * N * ab + N / 8.0,
                   [&] { return launch_update(c->storage, g, bf, sp, c->num_sms, c->s); })) != cudaSuccess)
        return e;
    if ((e = sample_pivot(c, g, bf)) != cudaSuccess) return e;
    return timed(c, 3, N * ab + N * sv,
                 [&] { return launch_normalize(c->storage, g, bf, sp, false, c->num_sms, c->s); });
}

cudaError_t one_step(ipf_ctx* c, int j) {
    cudaError_t e;
    if (c->gh) {
        // u = A l_k eliminated against D (d_{k+1}), then q = A^T d_{k+1}
        // eliminated against L (l_{k+1})
        if ((e = half_step(c, c->op, c->bf2, c->g2, c->g, c->bf, c->sp, j)) != cudaSuccess) return e;
        return half_step(c, c->opT, c->bf, c->g, c->g2, c->bf2, c->sp2, j);
    }
    const double N = (double)c->g.N, sv = (double)storage_bytes(c->storage), ab = (double)acc_bytes(c);
    if (c->split) {
        // h first (products at the pivot rows + FP64 pivot-block solve, small),
        // then the operator on s2 overlapped with V_j h on s, joined before the
        // combine
        // the new rows of L_p and L_p^{-1} (pivots and basis only), the
        // products at the pivot rows, then h
        if ((e = timed(c, 1, 0.0, [&] { return launch_pivot_minv(c->storage, c->g, c->bf, c->s); })) != cudaSuccess)
            return e;
        if ((e = timed(c, 7, 0.0, [&] {
                 return launch_pivot_rows(c->op, c->storage, c->bf.V, c->g.ldv, c->bf.st, c->bf.piv, c->B, c->g.k_max,
                                          c->bf.gpiv, c->s);
             })) != cudaSuccess)
            return e;
        if ((e = timed(c, 1, 0.0, [&] { return launch_pivot_apply(c->storage, c->g, c->bf, c->s); })) != cudaSuccess)
            return e;
        if ((e = cudaEventRecord(c->ev_fork, c->s)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(c->s2, c->ev_fork, 0)) != cudaSuccess) return e;
        if ((e = timed_on(c, c->s2, 0, op_bytes(c), [&] {
                 return launch_op_apply(c->op, c->storage, c->bf.V, c->g.ldv, c->g.k_max + 1, &c->bf.st->j, c->B,
                                        c->bf.w, c->bf.st->status, c->s2);
             })) != cudaSuccess)
            return e;
        if ((e = cudaEventRecord(c->ev_join, c->s2)) != cudaSuccess) return e;
        if ((e = timed(c, 2, (double)(j + 1) * N * sv + 4.0 * N,
                       [&] { return launch_gemv(c->storage, c->g, c->bf, c->num_sms, c->s); })) != cudaSuccess)
            return e;
        if ((e = cudaStreamWaitEvent(c->s, c->ev_join, 0)) != cudaSuccess) return e;
        if ((e = timed(c, 8, 12.0 * N + N / 8.0, [&] { return launch_combine(c->g, c->bf, c->num_sms, c->s); })) !=
            cudaSuccess)
            return e;
        if ((e = sample_pivot(c, c->g, c->bf)) != cudaSuccess) return e;
        return timed(c, 3, N * ab + N * sv,
                     [&] { return launch_normalize(c->storage, c->g, c->bf, c->sp, sw_on(c), c->num_sms, c->s); });
    }
    if (c->fork_piv) {
        // the operator on s2 beside the pivot-row products and the FP64
        // pivot-block solve on s (which need only v_j and the pivots), joined
        // before the update that consumes both
        if ((e = cudaEventRecord(c->ev_fork, c->s)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(c->s2, c->ev_fork, 0)) != cudaSuccess) return e;
        if ((e = timed_on(c, c->s2, 0, op_bytes(c), [&] {
                 return launch_op_apply(c->op, c->storage, c->bf.V, c->g.ldv, c->g.k_max + 1, &c->bf.st->j, c->B,
                                        c->bf.w, c->bf.st->status, c->s2);
             })) != cudaSuccess)
            return e;
        if ((e = cudaEventRecord(c->ev_join, c->s2)) != cudaSuccess) return e;
        // the new rows of L_p and L_p^{-1} (pivots and basis only), the
        // products at the pivot rows, then h
        if ((e = timed(c, 1, 0.0, [&] { return launch_pivot_minv(c->storage, c->g, c->bf, c->s); })) != cudaSuccess)
            return e;
        if ((e = timed(c, 7, 0.0, [&] {
                 return launch_pivot_rows(c->op, c->storage, c->bf.V, c->g.ldv, c->bf.st, c->bf.piv, c->B, c->g.k_max,
                                          c->bf.gpiv, c->s);
             })) != cudaSuccess)
            return e;
        if ((e = timed(c, 1, 0.0, [&] { return launch_pivot_apply(c->storage, c->g, c->bf, c->s); })) != cudaSuccess)
            return e;
        if ((e = cudaStreamWaitEvent(c->s, c->ev_join, 0)) != cudaSuccess) return e;
        if ((e = timed(c, 2, (double)(j + 1) * N * sv + 2.0 * N * ab + N / 8.0 + (c->defer_sketch ? 8.0 * N : 0.0),
                       [&] { return launch_update(c->storage, c->g, c->bf, c->sp, c->num_sms, c->s); })) != cudaSuccess)
            return e;
        if ((e = sample_pivot(c, c->g, c->bf)) != cudaSuccess) return e;
        return timed(c, 3, N * ab + N * sv,
                     [&] { return launch_normalize(c->storage, c->g, c->bf, c->sp, sw_on(c), c->num_sms, c->s); });
    }
    if ((e = timed(c, 0, op_bytes(c), [&] {
             return launch_op_apply(c->op, c->storage, c->bf.V, c->g.ldv, c->g.k_max + 1, &c->bf.st->j, c->B, c->bf.w,
                                    c->bf.st->status, c->s);
         })) != cudaSuccess)
        return e;
    if ((e = timed(c, 1, 0.0, [&] { return launch_pivot_solve(c->storage, c->g, c->bf, c->s); })) != cudaSuccess)
        return e;
    if ((e = timed(c, 2, (double)(j + 1) * N * sv + 2.0 * N * ab + N / 8.0 + (c->defer_sketch ? 8.0 * N : 0.0),
                   [&] { return launch_update(c->storage, c->g, c->bf, c->sp, c->num_sms, c->s); })) != cudaSuccess)
        return e;
    if ((e = sample_pivot(c, c->g, c->bf)) != cudaSuccess) return e;
    return timed(c, 3, N * ab + N * sv,
                 [&] { return launch_normalize(c->storage, c->g, c->bf, c->sp, sw_on(c), c->num_sms, c->s); });
}

// clear the state and enqueue Algorithm 1's initialisation for b
cudaError_t init_solve(ipf_ctx* c, const float* bdev) {
    const Geom& g = c->g;
    const size_t K1 = (size_t)g.k_max + 1;
    const int B = c->B;
    cudaError_t e;
    if ((e = cudaMemsetAsync(c->bf.H, 0, B * K1 * g.k_max * sizeof(double), c->s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(c->bf.ispiv, 0, (g.ldv / 32 + 1) * sizeof(unsigned), c->s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(c->bf.accSV, 0, B * K1 * g.m_s * sizeof(long long), c->s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(c->bf.accSW, 0, B * K1 * g.m_s * sizeof(long long), c->s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(c->bf.colE, 0, B * K1 * sizeof(int), c->s)) != cudaSuccess) return e;
    if (c->gh) {
        const Geom& g2 = c->g2;
        if ((e = cudaMemsetAsync(c->bf2.H, 0, B * K1 * g2.k_max * sizeof(double), c->s)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(c->bf2.ispiv, 0, (g2.ldv / 32 + 1) * sizeof(unsigned), c->s)) != cudaSuccess)
            return e;
        if ((e = cudaMemsetAsync(c->bf2.accSV, 0, B * K1 * g2.m_s * sizeof(long long), c->s)) != cudaSuccess)
            return e;
        if ((e = cudaMemsetAsync(c->bf2.accSW, 0, B * K1 * g2.m_s * sizeof(long long), c->s)) != cudaSuccess)
            return e;
        if ((e = cudaMemsetAsync(c->bf2.colE, 0, B * K1 * sizeof(int), c->s)) != cudaSuccess) return e;
        if ((e = launch_reset_state(c->bf2.st, c->cfg.pivot_fwd != 0, c->s)) != cudaSuccess) return e;
    }
    e = timed(c, 4, 0.0, [&] {
        cudaError_t ee = launch_reset_state(c->bf.st, c->cfg.pivot_fwd != 0, c->s);
        if (ee != cudaSuccess) return ee;
        if ((ee = launch_load_rhs(c->storage, bdev, g, c->bf, c->s)) != cudaSuccess) return ee;
        if ((ee = launch_update(c->storage, g, c->bf, c->sp, c->num_sms, c->s)) != cudaSuccess) return ee;
        if ((ee = sample_pivot(c, g, c->bf)) != cudaSuccess) return ee;
        Geom gi = g;
        gi.sketch_defer = 0;                       // v_1 (and S b) sketched here
        return launch_normalize(c->storage, gi, c->bf, c->sp, true, c->num_sms, c->s);
    });
    if (e == cudaSuccess && c->gauss) e = launch_gauss_bparts(c->storage, bdev, g.n, c->gWs, c->s);
    if (e != cudaSuccess || !c->gh) return e;
    // l_1 = A^T d_1 / (A^T d_1)(g_1): the same vector as A^T r_0 / alpha, and
    // its pivot value is W(1,1)
    return timed(c, 4, 0.0, [&] {
        cudaError_t ee = launch_op_apply(c->opT, c->storage, c->bf.V, g.ldv, g.k_max + 1, &c->bf.st->j, B, c->bf2.w,
                                         c->bf2.st->status, c->s);
        if (ee != cudaSuccess) return ee;
        if ((ee = launch_update(c->storage, c->g2, c->bf2, c->sp2, c->num_sms, c->s)) != cudaSuccess) return ee;
        if ((ee = sample_pivot(c, c->g2, c->bf2)) != cudaSuccess) return ee;
        return launch_normalize(c->storage, c->g2, c->bf2, c->sp2, false, c->num_sms, c->s);
    });
}

}  // namespace

extern "C" {

void ipf_config_default(ipf_config* cfg) {
    if (!cfg) return;
    memset(cfg, 0, sizeof(*cfg));
    cfg->k_max = 50;
    cfg->m_s = 200;
    cfg->zeta = 8;
    cfg->seed = 1;
    cfg->storage = IPF_STORE_F32;
    cfg->penalty = IPF_PEN_SKETCHED_X;
    cfg->zform = IPF_Z_AUTO;
    cfg->overlap = 2;
    cfg->nrhs = 1;
    cfg->use_graphs = 1;
}

// stride between basis vectors: N rounded up to 64 elements (16-byte
// aligned columns for 128-bit loads and TMA)
static size_t ldv_for(long long N) { return (size_t)((N + 63) / 64 * 64); }

static int lam_chunk(int B) { return B >= kLamChunk ? 1 : kLamChunk / B; }
static size_t solve_ws_for(const Geom& g) { return solve_workspace_bytes(g, lam_chunk(g.B)); }

size_t ipf_footprint(const ipf_operator* op, const ipf_config* cfg) {
    if (!op || !cfg) return 0;
    const long long n = op_n(op);
    const int B = cfg->nrhs > 0 ? cfg->nrhs : 1;
    const size_t sb = storage_bytes(cfg->storage);
    const size_t acc = cfg->storage == IPF_STORE_F64 ? 8 : 4;
    const size_t K1 = (size_t)cfg->k_max + 1;
    // one basis of length np with its buffers
    auto basis = [&](long long np) -> size_t {
        const size_t l = ldv_for(np * B);
        size_t b = K1 * l * sb + l * acc + l / 8 + 4096;
        b += B * K1 * (2 * sizeof(int) + sizeof(double) * cfg->k_max + 2 * sizeof(double) * K1) + K1 * B * acc;
        return b + 2 * (size_t)B * K1 * cfg->m_s * 8 + l * 8;
    };
    const bool gh = cfg->method == IPF_METHOD_SLSLU;
    const size_t ldv = ldv_for(n * B);
    size_t bytes = basis(gh ? op_m(op) : n) + (gh ? basis(n) : 0);
    if (gh) bytes += 2 * (size_t)B * op_m(op) * 4;
    if (cfg->sketch == IPF_SKETCH_GAUSSIAN)
        bytes += gauss_s_bytes(cfg->storage, cfg->m_s, n) + (size_t)cfg->m_s * K1 * 8 + 8 * (size_t)cfg->m_s +
                 gauss_workspace_bytes(cfg->storage, cfg->m_s, n, cfg->k_max, device_sms()) + 3 * 256;
    Geom g; g.n = n; g.B = B; g.N = n * B; g.ldv = (long long)ldv; g.k_max = cfg->k_max; g.m_s = cfg->m_s; g.F = 0;
    bytes += solve_ws_for(g) + 2 * (size_t)B * n * 4 + 256 + ldv * 4 + B * K1 * 4;
    const size_t opb = op->kind == IPF_OP_CSR ? (size_t)(op->rows + 1) * 8 + (size_t)op->nnz * 8
                                              : (size_t)op->ph * op->pw * 4 + 32 * 33 * 8 + 40960;
    if (op->kind == IPF_OP_CSR && op->mem == IPF_MEM_HOST) bytes += opb;
    else if (op->kind == IPF_OP_PSF2D) bytes += opb;      // PSF, packed pairs, tensor-core operand
    if (gh) bytes += op->kind == IPF_OP_CSR ? (size_t)(op->cols + 1) * 8 + (size_t)op->nnz * 8 : opb;   // A^T
    return bytes;
}

ipf_status ipf_create(const ipf_operator* op, const float* b, int b_mem, const ipf_config* cfg_in, ipf_ctx** out) {
    if (!out) return IPF_ERR_ARG;
    *out = nullptr;
    if (!cfg_in || !b) return IPF_ERR_ARG;
    ipf_config cfg = *cfg_in;
    std::string why;
    const int B = cfg.nrhs;
    if (!pow2_le32(B)) return IPF_ERR_ARG;
    ipf_status st = check_op(op, B, &why);
    if (st != IPF_OK) return st;
    if (cfg.method != IPF_METHOD_SCMRH && cfg.method != IPF_METHOD_SLSLU) return IPF_ERR_ARG;
    if (cfg.pivot_sample < 0 || cfg.pivot_sample > 64) return IPF_ERR_ARG;
    if (cfg.sketch != IPF_SKETCH_SPARSE_SIGN && cfg.sketch != IPF_SKETCH_GAUSSIAN) return IPF_ERR_ARG;
    const bool gauss = cfg.sketch == IPF_SKETCH_GAUSSIAN;
    if (gauss && (B != 1 || cfg.method != IPF_METHOD_SCMRH)) return IPF_ERR_UNSUPPORTED;
    const bool gh = cfg.method == IPF_METHOD_SLSLU;
    if (!gh && op->kind == IPF_OP_CSR && op->rows != op->cols) return IPF_ERR_UNSUPPORTED;   // square A (sCMRH)
    if (gh && op->kind != IPF_OP_PSF2D && op->kind != IPF_OP_CSR) return IPF_ERR_UNSUPPORTED;
    if (cfg.k_max < 1 || cfg.zeta < 1 || cfg.zeta > 16 || cfg.m_s < cfg.zeta || cfg.m_s > 65536) return IPF_ERR_ARG;
    if (cfg.storage < IPF_STORE_F64 || cfg.storage > IPF_STORE_F16) return IPF_ERR_ARG;
    if (cfg.storage == IPF_STORE_F64 && B != 1) return IPF_ERR_UNSUPPORTED;
    if (cfg.penalty != IPF_PEN_SKETCHED_X && cfg.penalty != IPF_PEN_Y) return IPF_ERR_ARG;
    if (cfg.zform != IPF_Z_DIRECT && cfg.zform != IPF_Z_HESSENBERG && cfg.zform != IPF_Z_AUTO) return IPF_ERR_ARG;
    const bool z_ok = cfg.storage != IPF_STORE_F64;
    if (cfg.zform == IPF_Z_DIRECT && !z_ok) return IPF_ERR_UNSUPPORTED;
    if (cfg.k_max > kMaxK) return IPF_ERR_UNSUPPORTED;    // forward substitution's rows (512) in registers
    if (cfg.pivot_fwd != 0 && cfg.pivot_fwd != 1) return IPF_ERR_ARG;
    if (cfg.m_s > kMaxMs) return IPF_ERR_UNSUPPORTED;     // the normaliser's shared sketch counters
    // the Gaussian contraction's B tile: V_{k+1} rounded up, plus 8 rows of b, at most 256 rows
    if (gauss && (cfg.k_max + 1 + 8 + 15) / 16 * 16 > 256) return IPF_ERR_UNSUPPORTED;
    if (b_mem != IPF_MEM_HOST && b_mem != IPF_MEM_DEVICE) return IPF_ERR_ARG;
    const size_t accb = cfg.storage == IPF_STORE_F64 ? 8 : 4;

    const long long n = op_n(op);                 // length of x (the L space)
    const long long nD = gh ? op_m(op) : n;       // length of b (the D space)
    const long long nmax = n > nD ? n : nD;
    if (nmax * B >= (1ll << 31) || nmax >= (1ll << 29)) return IPF_ERR_UNSUPPORTED;
    if (gauss) {
        cfg.zform = IPF_Z_HESSENBERG;             // S A V_k = (S V_{k+1}) H from the solve-time GEMM
        if (cfg.overlap == 1) cfg.overlap = 0;
    }
    if (gh) {
        cfg.overlap = 0;                          // one stream per step
        cfg.zform = IPF_Z_HESSENBERG;
        cfg.penalty = IPF_PEN_SKETCHED_X;
    }

    ipf_ctx* c = new ipf_ctx();
    c->gh = gh;
    c->gauss = gauss;
    c->cfg = cfg;
    c->storage = cfg.storage;
    c->B = B;
    c->al.fa = cfg.alloc;
    c->al.ff = cfg.free;
    c->al.user = cfg.alloc_user;
    c->user = (cudaStream_t)cfg.stream;
    c->num_sms = device_sms();
    cudaError_t e;
#define CK(what, expr)                                              \
    do {                                                            \
        e = (expr);                                                 \
        if (e != cudaSuccess) {                                     \
            ipf_status code = cuda_fail(c, what, e);                \
            ipf_destroy(c);                                         \
            return code;                                            \
        }                                                           \
    } while (0)
    {
        // the elimination branch (V_j h) gets the higher priority so its CTAs are
        // placed first whenever the operator branch frees room
        int lo = 0, hi = 0;
        CK("priorities", cudaDeviceGetStreamPriorityRange(&lo, &hi));
        CK("stream", cudaStreamCreateWithPriority(&c->s, cudaStreamNonBlocking, hi));
        CK("stream", cudaStreamCreateWithPriority(&c->s2, cudaStreamNonBlocking, lo));
    }
    CK("event", cudaEventCreateWithFlags(&c->ev, cudaEventDisableTiming));
    CK("event", cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    CK("event", cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
    c->split = cfg.overlap == 1 && (op->kind == IPF_OP_PSF2D || op->kind == IPF_OP_CSR) && cfg.storage != IPF_STORE_F64;
    c->fork_piv = cfg.overlap == 2 && (op->kind == IPF_OP_PSF2D || op->kind == IPF_OP_CSR) && cfg.storage != IPF_STORE_F64;
    CK("order", enter(c));
    CK("operator upload", upload_op(op, c->al, &c->op, c->s));
    c->op.conv_fma = cfg.conv_fma ? 1 : 0;
    if (gh) {
        CK("transpose upload", upload_transpose(op, c->al, &c->opT, c->s));
        c->opT.conv_fma = c->op.conv_fma;
    }

    // one basis with its work vector, state, pivots, Hessenberg columns,
    // pivot block, sketches and sketch table
    auto alloc_proc = [&](Geom& g, Bufs& bf, SketchParams& sp, long long np, unsigned long long seed) -> cudaError_t {
        cudaError_t ee;
        g.n = np;
        g.B = B;
        g.N = np * B;
        g.ldv = (long long)ldv_for(g.N);
        g.k_max = cfg.k_max;
        g.m_s = cfg.m_s;
        g.F = cfg.storage == IPF_STORE_F64 ? fixed_exponent(np, 0) : kSplitS;
        g.want_z = cfg.zform == IPF_Z_DIRECT ? 1 : 0;
        g.sketch_off = gauss ? 1 : 0;
        sp = make_sketch_params(seed, cfg.m_s, cfg.zeta);
        const size_t K1 = (size_t)cfg.k_max + 1;
        const size_t sb = storage_bytes(cfg.storage);
#define AK(expr) do { if ((ee = (expr)) != cudaSuccess) return ee; } while (0)
        AK(c->al.get(&bf.V, K1 * g.ldv * sb));
        AK(c->al.get(&bf.w, g.ldv * accb));
        AK(c->al.get((void**)&bf.st, sizeof(DevState)));
        AK(c->al.get((void**)&bf.piv, B * K1 * sizeof(int)));
        AK(c->al.get((void**)&bf.H, B * K1 * cfg.k_max * sizeof(double)));
        AK(c->al.get(&bf.LpT, B * K1 * K1 * sizeof(double)));
        AK(c->al.get((void**)&bf.Minv, B * K1 * K1 * sizeof(double)));
        AK(c->al.get(&bf.coef, K1 * B * accb));
        AK(c->al.get((void**)&bf.ispiv, (g.ldv / 32 + 1) * sizeof(unsigned)));
        AK(c->al.get((void**)&bf.accSV, B * K1 * cfg.m_s * sizeof(long long)));
        AK(c->al.get((void**)&bf.accSW, B * K1 * cfg.m_s * sizeof(long long)));
        AK(c->al.get((void**)&bf.colE, B * K1 * sizeof(int)));
        bf.sampled = cfg.pivot_sample > 0 ? 1 : 0;
        bf.t = nullptr;
        bf.gpiv = nullptr;
        if (c->split) {
            AK(c->al.get((void**)&bf.t, g.ldv * sizeof(float)));
            AK(cudaMemsetAsync(bf.t, 0, g.ldv * sizeof(float), c->s));
        }
        if (c->split || c->fork_piv) AK(c->al.get((void**)&bf.gpiv, B * K1 * sizeof(float)));
        if (!gauss && sketch_table_ok(sp)) {
            unsigned long long* tab = nullptr;
            // ldv entries (the update reads the table 16 bytes at a time up to ldv)
            AK(c->al.get((void**)&tab, sizeof(unsigned long long) * (size_t)g.ldv));
            AK(cudaMemsetAsync(tab, 0, sizeof(unsigned long long) * (size_t)g.ldv, c->s));
            AK(launch_sketch_table(sp, np, tab, c->s));
            bf.sktab = tab;
        } else {
            bf.sktab = nullptr;
        }
        AK(cudaMemsetAsync(bf.V, 0, K1 * g.ldv * sb, c->s));
        AK(cudaMemsetAsync(bf.w, 0, g.ldv * accb, c->s));
        AK(cudaMemsetAsync(bf.LpT, 0, B * K1 * K1 * sizeof(double), c->s));
        AK(cudaMemsetAsync(bf.Minv, 0, B * K1 * K1 * sizeof(double), c->s));
        AK(cudaMemsetAsync(bf.piv, 0, B * K1 * sizeof(int), c->s));
        AK(cudaMemsetAsync(bf.coef, 0, K1 * B * accb, c->s));
#undef AK
        return cudaSuccess;
    };
    CK("alloc basis", alloc_proc(c->g, c->bf, c->sp, nD, cfg.seed));
    if (gh) {
        // S_1 gets its own counter-hash stream: the seed with fixed bits flipped
        CK("alloc second basis", alloc_proc(c->g2, c->bf2, c->sp2, n, cfg.seed ^ 0x5DEECE66DA3B1F27ull));
        c->bf.st_peer = c->bf2.st;
        c->bf2.st_peer = c->bf.st;
    }
    Geom& g = c->g;
    Bufs& bf = c->bf;
    // the sketch of each new column moves from the normaliser into the next
    // step's update, which streams that column anyway (one RHS, float
    // storage with the zeta = 8 table, no sketch of unrounded vectors)
    c->defer_sketch = B == 1 && !gh && !gauss && !c->split && c->storage != IPF_STORE_F64 && bf.sktab &&
                      cfg.zeta == 8 && !sw_on(c) &&
                      (((uintptr_t)bf.V | (uintptr_t)bf.sktab) & 15u) == 0 && (g.ldv & 7) == 0;
    g.sketch_defer = c->defer_sketch ? 1 : 0;
    if (gauss) {
        const size_t wsb = gauss_workspace_bytes(cfg.storage, cfg.m_s, n, cfg.k_max, c->num_sms);
        CK("alloc Gaussian S", c->al.get(&c->gS, gauss_s_bytes(cfg.storage, cfg.m_s, n)));
        CK("alloc S V", c->al.get(&c->gSV, (size_t)cfg.m_s * (cfg.k_max + 1) * (cfg.storage == IPF_STORE_F64 ? 8 : 4)));
        CK("alloc S b", c->al.get((void**)&c->gC, sizeof(double) * cfg.m_s));
        CK("alloc Gaussian workspace", c->al.get(&c->gWs, wsb));
        CK("memset Gaussian workspace", cudaMemsetAsync(c->gWs, 0, wsb, c->s));
        CK("Gaussian S", launch_gauss_fill_ctx(cfg.storage, c->gS, n, cfg.m_s, cfg.seed, c->num_sms, c->s));
        c->gvariant = gauss_variant(cfg.storage, c->gS, cfg.m_s, n, c->bf.V, c->g.ldv, cfg.k_max + 1, c->gWs, c->gSV,
                                    c->gC, &c->bf.st->status[0], c->num_sms, c->s);
    }
    c->solve_ws_bytes = solve_ws_for(g);
    CK("alloc solve", c->al.get(&c->solve_ws, c->solve_ws_bytes));
    CK("alloc lambdas", c->al.get((void**)&c->lam_dev, sizeof(double) * kLamChunk));
    CK("alloc x stage", c->al.get((void**)&c->x_stage, sizeof(float) * (size_t)n * B));
    CK("alloc b stage", c->al.get((void**)&c->b_stage, sizeof(float) * (size_t)nD * B));
    (void)bf;
    CK("memset solve", cudaMemsetAsync(c->solve_ws, 0, c->solve_ws_bytes, c->s));
    const float* bsrc = b;
    if (b_mem == IPF_MEM_HOST) {
        CK("b upload", cudaMemcpyAsync(c->b_stage, b, sizeof(float) * (size_t)nD * B, cudaMemcpyHostToDevice, c->s));
        bsrc = c->b_stage;
    }
    CK("init", init_solve(c, bsrc));
    CK("order", leave(c));
    if (b_mem == IPF_MEM_HOST) CK("sync", cudaStreamSynchronize(c->s));
#undef CK
    *out = c;
    return IPF_OK;
}

ipf_status ipf_reset(ipf_ctx* c, const float* b, int b_mem) {
    if (!c || !b) return IPF_ERR_ARG;
    if (b_mem != IPF_MEM_HOST && b_mem != IPF_MEM_DEVICE) return IPF_ERR_ARG;
    if (c->sticky == IPF_ERR_NONFINITE) { c->sticky = IPF_OK; c->err.clear(); }
    if (c->sticky != IPF_OK) return c->sticky;
    cudaError_t e = enter(c);
    if (e != cudaSuccess) return cuda_fail(c, "order", e);
    const float* bsrc = b;
    if (b_mem == IPF_MEM_HOST) {
        if ((e = cudaMemcpyAsync(c->b_stage, b, sizeof(float) * (size_t)c->g.n * c->B, cudaMemcpyHostToDevice,
                                 c->s)) != cudaSuccess)
            return cuda_fail(c, "b upload", e);
        bsrc = c->b_stage;
    }
    if ((e = init_solve(c, bsrc)) != cudaSuccess) return cuda_fail(c, "init", e);
    c->j_host = 0;
    if ((e = leave(c)) != cudaSuccess) return cuda_fail(c, "order", e);
    return IPF_OK;
}

ipf_status ipf_profile_read(ipf_ctx* c, double* ms, long long* launches, double* bytes) {
    if (!c) return IPF_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(c->s);
    if (e != cudaSuccess) return cuda_fail(c, "sync", e);
    for (auto& m : c->marks) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, m.a, m.b) == cudaSuccess) {
            c->prof_ms[m.kind] += t;
            c->prof_n[m.kind] += 1;
            c->prof_bytes[m.kind] += m.bytes;
        }
        c->spare.push_back(m.a);
        c->spare.push_back(m.b);
    }
    c->marks.clear();
    for (int k = 0; k < kProfKinds; ++k) {
        if (ms) ms[k] = c->prof_ms[k];
        if (launches) launches[k] = c->prof_n[k];
        if (bytes) bytes[k] = c->prof_bytes[k];
        c->prof_ms[k] = 0.0;
        c->prof_n[k] = 0;
        c->prof_bytes[k] = 0.0;
    }
    return IPF_OK;
}

// steps per graph launch once the one-step graph exists: one launch for
// kGraphSteps steps saves the gap between graph launches on the device
constexpr int kGraphSteps = 8;

ipf_status ipf_step(ipf_ctx* c, int nsteps, int* k_enqueued) {
    if (!c) return IPF_ERR_ARG;
    if (c->sticky != IPF_OK) return c->sticky;
    if (nsteps < 0) return IPF_ERR_ARG;
    int todo = nsteps;
    if (todo > c->g.k_max - c->j_host) todo = c->g.k_max - c->j_host;
    cudaError_t e = enter(c);
    if (e != cudaSuccess) return cuda_fail(c, "order", e);
    int t = 0;
    if (todo > 0 && c->cfg.use_graphs && !c->cfg.profile && !c->gexec) {
        // the first step runs eagerly (it sets the kernels' attributes), then
        // one step is captured and the rest replay the graph
        if ((e = one_step(c, c->j_host)) != cudaSuccess) return cuda_fail(c, "step", e);
        ++c->j_host;
        ++t;
        if (t < todo) {
            if ((e = cudaStreamBeginCapture(c->s, cudaStreamCaptureModeRelaxed)) != cudaSuccess)
                return cuda_fail(c, "capture", e);
            cudaError_t e1 = one_step(c, 0);
            cudaError_t e2 = cudaStreamEndCapture(c->s, &c->graph);
            if (e1 != cudaSuccess) return cuda_fail(c, "capture step", e1);
            if (e2 != cudaSuccess) return cuda_fail(c, "end capture", e2);
            if ((e = cudaGraphInstantiate(&c->gexec, c->graph, 0)) != cudaSuccess)
                return cuda_fail(c, "instantiate", e);
        }
    }
    if (c->gexec && !c->gexec_run && todo - t >= kGraphSteps) {
        // the same step kGraphSteps times in one capture (every kernel reads
        // j from device memory, so the steps differ only in their data)
        if ((e = cudaStreamBeginCapture(c->s, cudaStreamCaptureModeRelaxed)) != cudaSuccess)
            return cuda_fail(c, "capture", e);
        cudaError_t e1 = cudaSuccess;
        for (int q = 0; q < kGraphSteps && e1 == cudaSuccess; ++q) e1 = one_step(c, 0);
        cudaError_t e2 = cudaStreamEndCapture(c->s, &c->graph_run);
        if (e1 != cudaSuccess) return cuda_fail(c, "capture steps", e1);
        if (e2 != cudaSuccess) return cuda_fail(c, "end capture", e2);
        if ((e = cudaGraphInstantiate(&c->gexec_run, c->graph_run, 0)) != cudaSuccess)
            return cuda_fail(c, "instantiate", e);
    }
    while (t < todo) {
        if (c->gexec_run && todo - t >= kGraphSteps) {
            if ((e = cudaGraphLaunch(c->gexec_run, c->s)) != cudaSuccess) return cuda_fail(c, "graph launch", e);
            t += kGraphSteps;
            c->j_host += kGraphSteps;
            continue;
        }
        if (c->gexec && !c->cfg.profile) {
            if ((e = cudaGraphLaunch(c->gexec, c->s)) != cudaSuccess) return cuda_fail(c, "graph launch", e);
        } else {
            if ((e = one_step(c, c->j_host)) != cudaSuccess) return cuda_fail(c, "step", e);
        }
        ++t;
        ++c->j_host;
    }
    if ((e = leave(c)) != cudaSuccess) return cuda_fail(c, "order", e);
    if (k_enqueued) *k_enqueued = c->j_host;
    return IPF_OK;
}

static ipf_status read_state(ipf_ctx* c, DevState* h) {
    cudaError_t e = cudaStreamSynchronize(c->s);
    if (e != cudaSuccess) return cuda_fail(c, "sync", e);
    e = cudaMemcpy(h, c->bf.st, sizeof(DevState), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, "state readback", e);
    return IPF_OK;
}

static ipf_status worst(const DevState& h, int B) {
    ipf_status w = IPF_OK;
    for (int r = 0; r < B; ++r) {
        const int s = h.status[r];
        if (s < 0) return (ipf_status)s;
        if (s == IPF_BREAKDOWN) w = IPF_BREAKDOWN;
    }
    return w;
}

ipf_status ipf_sync(ipf_ctx* c, int* k_done) {
    if (!c) return IPF_ERR_ARG;
    if (c->sticky != IPF_OK) return c->sticky;
    DevState h;
    ipf_status st = read_state(c, &h);
    if (st != IPF_OK) return st;
    int errflag = 0;
    cudaError_t e = solve_error_flag(c->solve_ws, c->g, &errflag);
    if (e != cudaSuccess) return cuda_fail(c, "solve flag", e);
    if (errflag) return fail(c, IPF_ERR_TIMEOUT, "projected solve: a device-side barrier wait gave up");
    if (k_done)
        for (int r = 0; r < c->B; ++r) k_done[r] = h.kdone[r];
    return worst(h, c->B);
}

static ipf_status solve_impl(ipf_ctx* c, int k, const double* lambdas, int nl, float* x_out, int x_mem,
                             ipf_solve_info* info, bool qmr) {
    if (!c) return IPF_ERR_ARG;
    if (c->sticky != IPF_OK) return c->sticky;
    if (k < 0 || nl < 1 || !lambdas || !x_out) return IPF_ERR_ARG;
    if (x_mem != IPF_MEM_HOST && x_mem != IPF_MEM_DEVICE) return IPF_ERR_ARG;
    if (k > c->j_host) return IPF_ERR_STATE;
    for (int l = 0; l < nl; ++l)
        if (!(lambdas[l] >= 0.0) || !std::isfinite(lambdas[l])) return IPF_ERR_ARG;
    cudaError_t e = enter(c);
    if (e != cudaSuccess) return cuda_fail(c, "order", e);
    const Geom& g = c->g;
    const int nlm = lam_chunk(c->B);
    bool any_pos = false;
    for (int l = 0; l < nl; ++l) any_pos |= lambdas[l] > 0.0;
    if (qmr && k + 1 > g.m_s) return IPF_ERR_UNSUPPORTED;   // [H | beta e_1] fills the m_s-row workspace
    const bool need_T = !qmr && any_pos && c->cfg.penalty == IPF_PEN_SKETCHED_X;
    const int penalty = qmr ? IPF_PEN_Y : c->cfg.penalty;
    // generalized process: Z and c from the D side, the penalty S_1 L_k from
    // the L side, x = L_k y with the D side's completed-step count
    if ((e = sketch_pending(c, c->s)) != cudaSuccess) return cuda_fail(c, "sketch", e);
    Bufs bz = c->bf;
    Geom gx = g;
    Bufs bx = c->bf;
    if (c->gh) {
        bz.penSV = c->bf2.accSV;
        bz.penE = c->bf2.colE;
        bz.penF = c->g2.F;
        gx = c->g2;
        bx = c->bf2;
        bx.st = c->bf.st;
    }
    if (c->gauss && !qmr) {
        // [S V_{k+1} | S b] by one contraction with the stored Gaussian S
        const double sb = storage_bytes(c->storage);
        const double gb = (double)g.m_s * g.n * sb + (double)g.n * (k + 1) * sb;
        e = timed(c, 9, gb, [&] {
            return launch_gauss_sv(c->storage, c->gS, g.m_s, g.n, c->bf.V, g.ldv, g.k_max + 1, k + 1, c->gWs, c->gSV,
                                   c->gC, &c->bf.st->status[0], c->num_sms, c->gvariant, c->s);
        });
        if (e != cudaSuccess) return cuda_fail(c, "Gaussian sketch contraction", e);
        bz.svd = c->gSV;
        bz.svd_f64 = c->storage == IPF_STORE_F64 ? 1 : 0;
        bz.cvec = c->gC;
    }
    e = timed(c, 5, 0.0, [&] {
        return launch_solve_prepare(g, bz, c->cfg.zeta, k, need_T, sw_on(c), c->solve_ws, nlm, c->num_sms, c->s,
                                    qmr);
    });
    if (e != cudaSuccess) return cuda_fail(c, "solve prepare", e);
    const size_t slice = (size_t)gx.n * c->B;
    const int step = x_mem == IPF_MEM_DEVICE ? nlm : 1;
    for (int l0 = 0; l0 < nl; l0 += step) {
        const int nlc = nl - l0 < step ? nl - l0 : step;
        if ((e = cudaMemcpyAsync(c->lam_dev, lambdas + l0, sizeof(double) * nlc, cudaMemcpyHostToDevice, c->s)) != cudaSuccess)
            return cuda_fail(c, "lambda upload", e);
        float* dst = x_mem == IPF_MEM_DEVICE ? x_out + (size_t)l0 * slice : c->x_stage;
        const double xb = (double)k * gx.N * storage_bytes(c->storage) + (double)nlc * gx.N * 4.0;
        e = timed(c, 6, xb, [&] {
            return launch_solve_lambdas(c->storage, gx, bx, k, need_T, c->lam_dev, nlc, penalty, c->solve_ws, nlm,
                                        dst, c->num_sms, c->s);
        });
        if (e != cudaSuccess) return cuda_fail(c, "solve", e);
        if (x_mem == IPF_MEM_HOST) {
            if ((e = cudaMemcpyAsync(x_out + (size_t)l0 * slice, c->x_stage, sizeof(float) * slice,
                                     cudaMemcpyDeviceToHost, c->s)) != cudaSuccess)
                return cuda_fail(c, "x download", e);
        }
    }
    if ((e = leave(c)) != cudaSuccess) return cuda_fail(c, "order", e);
    if (x_mem == IPF_MEM_DEVICE && !info) return IPF_OK;      // asynchronous form
    DevState h;
    ipf_status st = read_state(c, &h);
    if (st != IPF_OK) return st;
    int errflag = 0;
    if ((e = solve_error_flag(c->solve_ws, g, &errflag)) != cudaSuccess) return cuda_fail(c, "solve flag", e);
    if (errflag) return fail(c, IPF_ERR_TIMEOUT, "projected solve: a device-side barrier wait gave up");
    if (info)
        for (int r = 0; r < c->B; ++r) {
            info[r].k_done = h.kdone[r];
            info[r].k_used = h.kdone[r] < k ? h.kdone[r] : k;
            info[r].status = h.status[r];
            info[r].pad = 0;
        }
    return worst(h, c->B);
}

ipf_status ipf_solve(ipf_ctx* c, int k, const double* lambdas, int nl, float* x_out, int x_mem, ipf_solve_info* info) {
    return solve_impl(c, k, lambdas, nl, x_out, x_mem, info, false);
}

ipf_status ipf_solve_qmr(ipf_ctx* c, int k, const double* lambdas, int nl, float* x_out, int x_mem,
                         ipf_solve_info* info) {
    return solve_impl(c, k, lambdas, nl, x_out, x_mem, info, true);
}

ipf_status ipf_export(ipf_ctx* c, int r, int* pivots, double* H, double* SV, double* SZ, double* cvec, double* beta) {
    if (!c) return IPF_ERR_ARG;
    if (c->sticky != IPF_OK) return c->sticky;
    if (r < 0 || r >= c->B) return IPF_ERR_ARG;
    cudaError_t e0 = sketch_pending(c, c->s);                 // the newest column's S v
    if (e0 != cudaSuccess) return cuda_fail(c, "sketch", e0);
    DevState h;
    ipf_status st = read_state(c, &h);
    if (st != IPF_OK) return st;
    const size_t K1 = (size_t)c->g.k_max + 1;
    const size_t km = (size_t)c->g.k_max;
    const int m = c->g.m_s;
    cudaError_t e = cudaSuccess;
    if (pivots) {
        std::vector<int> p(K1);
        e = cudaMemcpy(p.data(), c->bf.piv + r * K1, K1 * sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(c, "export piv", e);
        const int kd = h.kdone[r];
        const int np = (h.status[r] == IPF_BREAKDOWN) ? kd : kd + 1;
        for (int i = 0; i < (int)K1; ++i) pivots[i] = i < np ? p[i] : -1;
    }
    if (H) {
        e = cudaMemcpy(H, c->bf.H + r * K1 * km, K1 * km * sizeof(double), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(c, "export H", e);
    }
    const double sq = std::sqrt((double)c->cfg.zeta);
    std::vector<int> ce(K1);
    if ((e = cudaMemcpy(ce.data(), c->bf.colE + r * K1, K1 * sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(c, "export column exponents", e);
    // column t / m of a fixed-point sketch block carries the exponent ce[t / m]
    auto grab = [&](const long long* src, size_t count, double scale, double* dst) -> cudaError_t {
        std::vector<long long> a(count);
        cudaError_t ee = cudaMemcpy(a.data(), src, count * sizeof(long long), cudaMemcpyDeviceToHost);
        if (ee != cudaSuccess) return ee;
        for (size_t t = 0; t < count; ++t) dst[t] = (double)a[t] * std::ldexp(scale, ce[t / m]);
        return cudaSuccess;
    };
    if (SV && (e = grab(c->bf.accSV + r * K1 * m, K1 * m, std::ldexp(1.0, -c->g.F) / sq, SV)) != cudaSuccess)
        return cuda_fail(c, "export SV", e);
    if (SZ) {
        // z_j = S A v_j = S V_{j+1} h_j + H(j+1,j) (S w)_{j+1}, w the unrounded
        // normalised vector (the stored one unless the storage rounds)
        const double sc = std::ldexp(1.0, -c->g.F) / sq;
        std::vector<double> sv(K1 * m), sw(K1 * m), Hh(K1 * km);
        if ((e = grab(c->bf.accSV + r * K1 * m, K1 * m, sc, sv.data())) != cudaSuccess) return cuda_fail(c, "export SZ", e);
        if ((e = grab(c->bf.accSW + r * K1 * m, K1 * m, sc, sw.data())) != cudaSuccess) return cuda_fail(c, "export SZ", e);
        if ((e = cudaMemcpy(Hh.data(), c->bf.H + r * K1 * km, K1 * km * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(c, "export SZ", e);
        const bool use_sw = sw_on(c);
        for (size_t col = 0; col < km; ++col) {
            const double* hcol = Hh.data() + K1 * col;
            for (int row = 0; row < m; ++row) {
                double t = 0.0;
                for (size_t i = 0; i <= col; ++i) t += sv[i * m + row] * hcol[i];
                const std::vector<double>& last = use_sw ? sw : sv;
                t += last[(col + 1) * m + row] * hcol[col + 1];
                SZ[col * m + row] = t;
            }
        }
    }
    if (cvec) {
        if ((e = grab(c->bf.accSW + r * K1 * m, m, std::ldexp(1.0, -c->g.F) / sq, cvec)) != cudaSuccess)
            return cuda_fail(c, "export c", e);
        for (int t = 0; t < m; ++t) cvec[t] *= h.beta[r];
    }
    if (beta) *beta = h.beta[r];
    return IPF_OK;
}

static ipf_status export_column(ipf_ctx* c, const Geom& g, const Bufs& bf, int r, int j, float* v_out) {
    if (!c || !v_out) return IPF_ERR_ARG;
    if (c->sticky != IPF_OK) return c->sticky;
    if (r < 0 || r >= c->B || j < 0 || j > g.k_max) return IPF_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(c->s);
    if (e != cudaSuccess) return cuda_fail(c, "sync", e);
    const size_t sb = storage_bytes(c->storage);
    std::vector<unsigned char> raw((size_t)g.ldv * sb);
    e = cudaMemcpy(raw.data(), (const char*)bf.V + (size_t)j * g.ldv * sb, raw.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, "export basis", e);
    const long long n = g.n;
    const int B = c->B;
    for (long long i = 0; i < n; ++i) {
        const size_t el = (size_t)i * B + r;
        float v;
        switch (c->storage) {
            case IPF_STORE_F64: v = (float)((const double*)raw.data())[el]; break;
            case IPF_STORE_F32: v = ((const float*)raw.data())[el]; break;
            case IPF_STORE_BF16: {
                const unsigned short u = ((const unsigned short*)raw.data())[el];
                const unsigned w = (unsigned)u << 16;
                memcpy(&v, &w, 4);
                break;
            }
            default: {
                __half hv;
                memcpy(&hv, (const unsigned short*)raw.data() + el, 2);
                v = __half2float(hv);
            }
        }
        v_out[i] = v;
    }
    return IPF_OK;
}

ipf_status ipf_export_basis(ipf_ctx* c, int r, int j, float* v_out) {
    if (!c) return IPF_ERR_ARG;
    return export_column(c, c->g, c->bf, r, j, v_out);
}

ipf_status ipf_export_dual(ipf_ctx* c, int r, int* pivots_l, double* W, double* SL, double* w11) {
    if (!c) return IPF_ERR_ARG;
    if (c->sticky != IPF_OK) return c->sticky;
    if (!c->gh) return IPF_ERR_STATE;
    if (r < 0 || r >= c->B) return IPF_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(c->s);
    if (e != cudaSuccess) return cuda_fail(c, "sync", e);
    DevState h;
    if ((e = cudaMemcpy(&h, c->bf2.st, sizeof(DevState), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(c, "state readback", e);
    const size_t K1 = (size_t)c->g2.k_max + 1;
    const size_t km = (size_t)c->g2.k_max;
    const int m = c->g2.m_s;
    if (pivots_l) {
        std::vector<int> p(K1);
        if ((e = cudaMemcpy(p.data(), c->bf2.piv + r * K1, K1 * sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(c, "export piv", e);
        const int kd = h.kdone[r];
        const int np = (h.status[r] == IPF_BREAKDOWN) ? kd : kd + 1;
        for (int i = 0; i < (int)K1; ++i) pivots_l[i] = i < np ? p[i] : -1;
    }
    if (W && (e = cudaMemcpy(W, c->bf2.H + r * K1 * km, K1 * km * sizeof(double), cudaMemcpyDeviceToHost)) !=
                 cudaSuccess)
        return cuda_fail(c, "export W", e);
    if (SL) {
        std::vector<long long> a(K1 * m);
        if ((e = cudaMemcpy(a.data(), c->bf2.accSV + r * K1 * m, a.size() * sizeof(long long),
                            cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(c, "export SL", e);
        std::vector<int> ce(K1);
        if ((e = cudaMemcpy(ce.data(), c->bf2.colE + r * K1, K1 * sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(c, "export SL", e);
        const double sc = std::ldexp(1.0, -c->g2.F) / std::sqrt((double)c->cfg.zeta);
        for (size_t t = 0; t < a.size(); ++t) SL[t] = (double)a[t] * std::ldexp(sc, ce[t / m]);
    }
    if (w11) *w11 = h.beta[r];
    return IPF_OK;
}

ipf_status ipf_export_basis_l(ipf_ctx* c, int r, int j, float* l_out) {
    if (!c || !l_out) return IPF_ERR_ARG;
    if (!c->gh) return IPF_ERR_STATE;
    return export_column(c, c->g2, c->bf2, r, j, l_out);
}

void ipf_destroy(ipf_ctx* c) {
    if (!c) return;
    if (c->s) cudaStreamSynchronize(c->s);
    for (auto& m : c->marks) { cudaEventDestroy(m.a); cudaEventDestroy(m.b); }
    for (auto ev : c->spare) cudaEventDestroy(ev);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    if (c->gexec_run) cudaGraphExecDestroy(c->gexec_run);
    if (c->graph_run) cudaGraphDestroy(c->graph_run);
    c->al.release();
    if (c->ev) cudaEventDestroy(c->ev);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->s2) cudaStreamSynchronize(c->s2);
    if (c->s2) cudaStreamDestroy(c->s2);
    if (c->s) cudaStreamDestroy(c->s);
    delete c;
}

const char* ipf_status_str(ipf_status s) {
    switch (s) {
        case IPF_OK: return "IPF_OK";
        case IPF_BREAKDOWN: return "IPF_BREAKDOWN";
        case IPF_PENDING: return "IPF_PENDING";
        case IPF_ERR_ARG: return "IPF_ERR_ARG";
        case IPF_ERR_OOM: return "IPF_ERR_OOM";
        case IPF_ERR_CUDA: return "IPF_ERR_CUDA";
        case IPF_ERR_NONFINITE: return "IPF_ERR_NONFINITE";
        case IPF_ERR_TIMEOUT: return "IPF_ERR_TIMEOUT";
        case IPF_ERR_STATE: return "IPF_ERR_STATE";
        case IPF_ERR_UNSUPPORTED: return "IPF_ERR_UNSUPPORTED";
        case IPF_ERR_REJECTED: return "IPF_ERR_REJECTED";
        default: return "IPF_UNKNOWN";
    }
}

const char* ipf_last_error(const ipf_ctx* c) {
    if (!c) return "no context";
    return c->err.c_str();
}

ipf_status ipf_op_create(const ipf_operator* op, ipf_op** out) {
    if (!out) return IPF_ERR_ARG;
    *out = nullptr;
    std::string why;
    ipf_status st = check_op(op, 1, &why);
    if (st != IPF_OK) return st;
    ipf_op* h = new ipf_op();
    cudaError_t e = upload_op(op, h->al, &h->op, nullptr);
    if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
    if (e != cudaSuccess) {
        h->al.release();
        delete h;
        return e == cudaErrorMemoryAllocation ? IPF_ERR_OOM : IPF_ERR_CUDA;
    }
    *out = h;
    return IPF_OK;
}

ipf_status ipf_op_apply(ipf_op* h, const float* v_dev, float* w_dev, int nrhs, void* stream) {
    if (!h || !v_dev || !w_dev || nrhs < 1) return IPF_ERR_ARG;
    if (h->op.kind == IPF_OP_CSR && !pow2_le32(nrhs)) return IPF_ERR_ARG;
    cudaError_t e = launch_op_apply_f32_plain(h->op, v_dev, w_dev, nrhs, (cudaStream_t)stream);
    return e == cudaSuccess ? IPF_OK : IPF_ERR_CUDA;
}

ipf_status ipf_op_apply_bf16(ipf_op* h, const void* v_dev, float* w_dev, int use_fma, void* stream) {
    if (!h || !v_dev || !w_dev) return IPF_ERR_ARG;
    OpDev op = h->op;
    op.conv_fma = use_fma ? 1 : 0;
    cudaError_t e =
        launch_op_apply(op, IPF_STORE_BF16, v_dev, 0, 1, nullptr, 1, w_dev, nullptr, (cudaStream_t)stream);
    return e == cudaSuccess ? IPF_OK : IPF_ERR_CUDA;
}

void ipf_op_destroy(ipf_op* h) {
    if (!h) return;
    cudaDeviceSynchronize();
    h->al.release();
    delete h;
}

ipf_status ipf_sketch_apply(const float* x_dev, long long n, int m_s, int zeta, unsigned long long seed, double* y_dev,
                            void* stream) {
    if (!x_dev || !y_dev || n < 1 || zeta < 1 || zeta > 16 || m_s < zeta) return IPF_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int sms = device_sms();
    SketchParams sp = make_sketch_params(seed, m_s, zeta);
    void* scratch = nullptr;
    const size_t bytes = 256 + sizeof(long long) * (size_t)m_s;
    cudaError_t e = cudaMallocAsync(&scratch, bytes, s);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? IPF_ERR_OOM : IPF_ERR_CUDA;
    unsigned* amax = (unsigned*)scratch;
    long long* acc = (long long*)((char*)scratch + 256);
    e = cudaMemsetAsync(scratch, 0, bytes, s);
    if (e == cudaSuccess) e = launch_sketch_vector(x_dev, n, sp, 0, acc, (float*)amax, s, sms, true);
    if (e == cudaSuccess) e = launch_sketch_finish(acc, m_s, n, zeta, amax, y_dev, s);
    cudaError_t e2 = cudaFreeAsync(scratch, s);
    if (e != cudaSuccess || e2 != cudaSuccess) return IPF_ERR_CUDA;
    return IPF_OK;
}

ipf_status ipf_sketch_gaussian(int storage, unsigned long long seed, long long n, int m_s, void* S_dev, void* stream) {
    if (!S_dev || n < 1 || m_s < 1) return IPF_ERR_ARG;
    if (storage != IPF_STORE_F64 && storage != IPF_STORE_F32 && storage != IPF_STORE_BF16 && storage != IPF_STORE_F16)
        return IPF_ERR_ARG;
    const cudaError_t e = launch_gauss_fill(storage, S_dev, n, m_s, n, seed, device_sms(), (cudaStream_t)stream);
    return e == cudaSuccess ? IPF_OK : IPF_ERR_CUDA;
}

}  // extern "C"

namespace ipf {

cudaError_t raise_smem_ptr(const void* fn, size_t bytes) {
    static std::mutex mu;
    static std::vector<std::pair<const void*, size_t>> set;   // kernel, limit in force
    std::lock_guard<std::mutex> lk(mu);
    for (auto& e : set)
        if (e.first == fn) {
            if (e.second >= bytes) return cudaSuccess;
            const cudaError_t r = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
            if (r == cudaSuccess) e.second = bytes;
            return r;
        }
    const cudaError_t r = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (r == cudaSuccess) set.emplace_back(fn, bytes);
    return r;
}

// The batched step of the serving loop drives contexts whose every step is
// one of the batched kernels: one RHS, float storage, the sparse-sign sketch
// with its table and the deferred sketch, full pivoting, step mode 2 (the
// products at the pivot rows beside the operator), and a PSF on the FMA
// column path (kw 7, 15, 31; BF16 may use the tensor cores) or a CSR matrix.  Fills d (k_target and the tile counts are left
// to the caller) and returns true for such a context.
bool ctx_slot_desc(ipf_ctx* c, SlotDesc* d, int* storage) {
    if (!c || c->sticky != IPF_OK || c->gh || c->gauss || c->B != 1 || c->storage == IPF_STORE_F64) return false;
    // the batched step runs the pivot-row products beside the operator: the
    // context must have their buffer (step mode 2)
    if (!c->defer_sketch || c->split || !c->fork_piv || !c->bf.gpiv || c->cfg.pivot_sample != 0 || sw_on(c))
        return false;
    if (c->op.kind == IPF_OP_PSF2D) {
        if (!c->op.psf_pairs || (c->op.kw != 7 && c->op.kw != 15 && c->op.kw != 31)) return false;
    } else if (c->op.kind != IPF_OP_CSR) {
        return false;
    }
    memset(d, 0, sizeof(*d));
    d->g = c->g;
    d->bf = c->bf;
    d->sp = c->sp;
    d->op = c->op;
    *storage = c->storage;
    return true;
}

// the context's steps were taken by the batched step: k steps are enqueued
void ctx_steps_taken(ipf_ctx* c, int k) {
    if (c) c->j_host = k < c->g.k_max ? k : c->g.k_max;
}

}  // namespace ipf
