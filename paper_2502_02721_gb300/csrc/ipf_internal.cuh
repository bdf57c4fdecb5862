// Internal definitions shared by the libipf translation units: storage
// types, the sparse-sign counter hash, exact fixed-point sketch
// accumulation, argmax keys and the launcher prototypes.
#pragma once

#include <cuda_runtime.h>
#include <functional>
#include <vector>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "../../include/ipf.h"

namespace ipf {

// kernel kinds of the profile mode (ipf_profile_read)
constexpr int kProfKinds = 12;

// ---------------------------------------------------------------------------
// storage types: T is how basis vectors live in HBM, Acc the arithmetic type
// ---------------------------------------------------------------------------
template <class T> struct AccOf { using type = float; };
template <> struct AccOf<double> { using type = double; };

__device__ __forceinline__ float to_acc(float x) { return x; }
__device__ __forceinline__ double to_acc(double x) { return x; }
__device__ __forceinline__ float to_acc(__nv_bfloat16 x) { return __bfloat162float(x); }
__device__ __forceinline__ float to_acc(__half x) { return __half2float(x); }

template <class T> __device__ __forceinline__ T from_acc(float x);
template <> __device__ __forceinline__ float from_acc<float>(float x) { return x; }
template <> __device__ __forceinline__ __nv_bfloat16 from_acc<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <> __device__ __forceinline__ __half from_acc<__half>(float x) { return __float2half_rn(x); }
template <class T> __device__ __forceinline__ T from_acc(double x);
template <> __device__ __forceinline__ double from_acc<double>(double x) { return x; }

// ---------------------------------------------------------------------------
// sparse-sign sketch: column i has one +-1/sqrt(zeta) entry in each of zeta
// disjoint row blocks.  Row and sign come from SplitMix64 (Steele, Lea &
// Flood 2014): output number c of the generator started at `seed` is
// mix(seed + GAMMA*(c+1)); column i uses outputs W*i .. W*i+W-1,
// W = ceil(24*zeta/64), read as one little-endian bit string whose bits
// [24t, 24t+24) give block t: sign = bit 0 (1 = negative), r = the other
// 23 bits, row = lo_t + (r * size_t) >> 23 with lo_t = floor(t*m/zeta).
// ---------------------------------------------------------------------------
constexpr unsigned long long kGamma = 0x9E3779B97F4A7C15ull;

__host__ __device__ __forceinline__ unsigned long long sm64_mix(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

struct SketchParams {
    unsigned long long seed;
    int m_s;
    int zeta;
    int W;                   // 64-bit words per column
    int lo[17];              // block starts, lo[zeta] = m_s
};

inline SketchParams make_sketch_params(unsigned long long seed, int m_s, int zeta) {
    SketchParams p;
    p.seed = seed;
    p.m_s = m_s;
    p.zeta = zeta;
    p.W = (24 * zeta + 63) / 64;
    for (int t = 0; t <= zeta; ++t) p.lo[t] = (int)(((long long)t * m_s) / zeta);
    for (int t = zeta + 1; t <= 16; ++t) p.lo[t] = m_s;
    return p;
}

// rows[t], neg[t] for column i (t < zeta <= 16)
__device__ __forceinline__ void sketch_column(const SketchParams& sp, long long i, int* rows,
                                              unsigned* negmask) {
    unsigned long long w[6];
    const unsigned long long base = (unsigned long long)i * (unsigned long long)sp.W;
#pragma unroll
    for (int q = 0; q < 6; ++q)
        if (q < sp.W) w[q] = sm64_mix(sp.seed + kGamma * (base + q + 1));
    unsigned nm = 0;
#pragma unroll
    for (int t = 0; t < 16; ++t) {
        if (t < sp.zeta) {
            const int bit = 24 * t, q = bit >> 6, off = bit & 63;
            unsigned long long ch = w[q] >> off;
            if (off > 40) ch |= w[q + 1] << (64 - off);
            ch &= 0xFFFFFFull;
            nm |= (unsigned)(ch & 1ull) << t;
            const long long r = (long long)(ch >> 1);
            const int size = sp.lo[t + 1] - sp.lo[t];
            rows[t] = sp.lo[t] + (int)((r * size) >> 23);
        }
    }
    *negmask = nm;
}

// Specialisation for the common zeta = 8 (3 words, fixed chunk offsets).
__device__ __forceinline__ void sketch_column8(const SketchParams& sp, long long i, int* rows,
                                               unsigned* negmask) {
    const unsigned long long base = (unsigned long long)i * 3ull;
    const unsigned long long w0 = sm64_mix(sp.seed + kGamma * (base + 1));
    const unsigned long long w1 = sm64_mix(sp.seed + kGamma * (base + 2));
    const unsigned long long w2 = sm64_mix(sp.seed + kGamma * (base + 3));
    unsigned long long ch[8];
    ch[0] = w0;
    ch[1] = w0 >> 24;
    ch[2] = (w0 >> 48) | (w1 << 16);
    ch[3] = w1 >> 8;
    ch[4] = w1 >> 32;
    ch[5] = (w1 >> 56) | (w2 << 8);
    ch[6] = w2 >> 16;
    ch[7] = w2 >> 40;
    unsigned nm = 0;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const unsigned c = (unsigned)(ch[t] & 0xFFFFFFull);
        nm |= (c & 1u) << t;
        const int size = sp.lo[t + 1] - sp.lo[t];
        rows[t] = sp.lo[t] + (int)(((unsigned long long)(c >> 1) * (unsigned)size) >> 23);
    }
    *negmask = nm;
}

// ---------------------------------------------------------------------------
// exact sketch sums: each contribution is rounded once to a 64-bit fixed
// point value x * 2^F (F chosen per call so no sum can overflow), then all
// additions are integer and therefore independent of their order.
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long fixed_from(float v, int F) {
    const unsigned u = __float_as_uint(v);
    const int e = (int)((u >> 23) & 0xFFu);
    if (e == 0) return 0;
    const long long m = (long long)((u & 0x7FFFFFu) | 0x800000u);
    const int sh = e - 150 + F;
    long long q;
    if (sh >= 0) q = m << (sh > 38 ? 38 : sh);
    else if (sh > -26) q = (m + (1ll << (-sh - 1))) >> (-sh);
    else q = 0;
    return (u >> 31) ? -q : q;
}

__device__ __forceinline__ long long fixed_from(double v, int F) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    const int e = (int)((u >> 52) & 0x7FFull);
    if (e == 0) return 0;
    const long long m = (long long)((u & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);
    const int sh = e - 1075 + F;
    long long q;
    if (sh >= 0) q = m << (sh > 9 ? 9 : sh);
    else if (sh > -55) q = (m + (1ll << (-sh - 1))) >> (-sh);
    else q = 0;
    return (u >> 63) ? -q : q;
}

// Float modes: contributions |x| <= 2^e are rounded once to q = x * 2^S with
// S = kSplitS - e (|q| <= 2^34) and added into two int32 shared-memory
// counters, hi = q >> 17 and lo = q & (2^17 - 1); both stay exact for up to
// kFoldEvery contributions per counter, after which they are folded into an
// int64 (hi * 2^17 + lo) and cleared.  Integer sums make the result
// independent of thread order.
constexpr int kSplitS = 34;
constexpr int kFoldEvery = 8192;

__device__ __forceinline__ void split_add(int* hi, int* lo, int row, long long q) {
    atomicAdd(&hi[row], (int)(q >> 17));
    atomicAdd(&lo[row], (int)(q & 0x1FFFFll));
}

// fold hi/lo counters [0, cnt) into wide and clear them (whole CTA, between barriers)
__device__ __forceinline__ void split_fold(int* hi, int* lo, long long* wide, int cnt) {
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
        wide[t] += ((long long)hi[t] << 17) + (long long)lo[t];
        hi[t] = 0;
        lo[t] = 0;
    }
}

// fixed-point exponent for sums of at most `count` terms of magnitude <= 2^e_max
inline int fixed_exponent(long long count, int e_max) {
    int lg = 0;
    while ((1ll << lg) < count + 1) ++lg;
    return 61 - lg - e_max;
}

// ---------------------------------------------------------------------------
// argmax keys (float arithmetic): |w| bits in the high word, ~row in the low
// word, so the max key is the largest |w| with the lowest row on ties.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long argmax_key(float w, unsigned row) {
    return ((unsigned long long)__float_as_uint(fabsf(w)) << 32) | (unsigned long long)(0xFFFFFFFFu - row);
}
__device__ __forceinline__ unsigned key_row(unsigned long long k) { return 0xFFFFFFFFu - (unsigned)(k & 0xFFFFFFFFull); }
__device__ __forceinline__ float key_absval(unsigned long long k) { return __uint_as_float((unsigned)(k >> 32)); }

// ---------------------------------------------------------------------------
// device-side state of one context (one batch of nrhs right-hand sides)
// ---------------------------------------------------------------------------
constexpr int kMaxRhs = 32;

struct DevState {
    int j;                         // current step: basis v_0..v_{j} exists (j = -1 before init)
    unsigned ctr;                  // last-CTA ticket for the normalise kernel
    int status[kMaxRhs];           // per RHS: IPF_OK, IPF_BREAKDOWN, IPF_ERR_NONFINITE
    int kdone[kMaxRhs];            // completed Hessenberg steps per RHS
    double beta[kMaxRhs];          // b(p_1)
    unsigned long long key[2][kMaxRhs];      // argmax keys, double-buffered by step parity
    unsigned long long maxbits[2];           // F64 mode: max |w| bits (nrhs == 1)
    unsigned long long minidx[2];            // F64 mode: lowest row attaining it
    double wmax[kMaxRhs];          // sampled pivoting: max |w| over the candidates of this step
    int sk_pending;                // deferred sketch: column of V still to be sketched, or -1
    unsigned sk_ctr;               // last-CTA ticket for the deferred sketch kernel
    int fwd[kMaxRhs];              // per RHS: 1 = pivot block by forward substitution (chosen
                                   // at creation, or set when a row of L_p^{-1} grew past
                                   // kMinvGrowth), 0 = by the product with L_p^{-1}
};

// everything a kernel needs about the context, passed by value
struct Geom {
    long long n;        // unknowns per RHS
    int B;              // RHS count (interleaved, element e = i*B + r)
    long long N;        // n * B
    long long ldv;      // stride between basis vectors (elements), multiple of 64
    int k_max;
    int m_s;
    int F;              // fixed-point exponent of the sketch accumulators
    int want_z;         // DIRECT form: z_j = S A v_j (needs S of the unrounded vectors)
    int sketch_off = 0; // Gaussian sketch: no per-step sparse sketch (S V is formed at solve time)
    int sketch_defer = 0;  // the normaliser leaves S v_{j+1} to the next step's update (or to
                           // k_sketch_col before a solve) and marks the column pending
};

struct Bufs {
    void* V;                       // (k_max+1) x ldv storage-type basis
    void* w;                       // ldv Acc work vector (u in Algorithm 1)
    DevState* st;
    int* piv;                      // [B][k_max+1]
    double* H;                     // [B][(k_max+1)*k_max], column-major
    void* LpT;                     // [B][lp_stride] FP64, L_p packed by rows (strictly lower)
    double* Minv = nullptr;        // [B][lp_stride] FP64, L_p^{-1} packed the same way
    void* coef;                    // [(k_max+1)*B] Acc, h for the update
    unsigned* ispiv;               // bitmap over N elements
    long long* accSV;              // [B][k_max+1][m_s] fixed-point S V
    long long* accSW;              // [B][k_max+1][m_s] fixed-point S of the unrounded vectors
                                   // (column 0 = S (b / beta), others for BF16/FP16 storage)
    int* colE;                     // [B][k_max+1] column exponents: column j of accSV / accSW
                                   // holds S v_j * 2^(F - colE[j]), so |v_j| <= 2^colE[j] keeps
                                   // the fixed-point sums in range (0 unless pivots are sampled)
    int sampled;                   // pivots are sampled, so |v_j| may exceed 1
    const unsigned long long* sktab;  // n entries (zeta = 8, blocks <= 128 rows) or NULL:
                                      // byte t = row offset in block t | sign << 7
    float* t;                      // ldv FP32: V_j h (split step), else NULL
    float* gpiv;                   // [B][k_max+1] FP32: (A v_j)(p_i) (split step), else NULL
    // generalized process (two bases): the other basis's state, told when this
    // one stops, and for the projected solve the sketches of the penalty basis
    // (S_1 L) with their fixed-point exponent; NULL / 0 for one basis
    DevState* st_peer = nullptr;
    const long long* penSV = nullptr;
    const int* penE = nullptr;
    int penF = 0;
    // Gaussian sketch: S V_{k+1} (m_s x (k+1), column-major, FP64 if svd_f64
    // else FP32) and c = S b (m_s, FP64), formed at solve time; NULL otherwise
    const void* svd = nullptr;
    int svd_f64 = 0;
    const double* cvec = nullptr;
};

// operator on the device
struct OpDev {
    int kind;
    int rows, cols;
    int ph, pw;
    const float* psf;
    int slen;
    const float* sep_row;
    const float* sep_col;
    int mlen;
    const float* motion;
    const long long* rowptr;
    const int* colind;
    const float* vals;
    long long nnz;
    int kw;                        // PSF2D: padded square width (7, 15, 31) of psf_pairs, else 0
    const unsigned long long* psf_pairs;   // [kw][kw+1] packed {F[ky][b], F[ky-1][b]}, F flipped + padded
    int tc_kp;                     // PSF2D, kw 15 or 31: KP = kw + 1 of the tensor-core operand, else 0
    const void* psf_tc;            // [F_hi ; F_lo] BF16, 2KP x KP, K-major core-matrix layout
    int conv_fma;                  // 1: keep the FP32 FMA convolution for BF16 storage
};

// ---------------------------------------------------------------------------
// batched step: many one-RHS solves in flight advanced by one launch per
// phase.  The work list is a table of slots (each a context's geometry,
// buffers, sketch and operator, and the number of steps it takes) and, per
// phase, a flat table of (slot, tile) pairs; a CTA takes the table entries
// blockIdx.x, blockIdx.x + gridDim.x, ...  A slot is active in a step while
// its status is IPF_OK and its step counter is below k_target.
// ---------------------------------------------------------------------------
constexpr int kMaxSlots = 64;
constexpr int kMaxK = 480;                     // k_max (forward substitution's registers hold 512 rows)
// m_s of a context: the initial normalisation keeps two sets of exact sketch
// counters of one right-hand side (S v_1 and S b / beta; 8 + 4 + 4 bytes per
// row each) in dynamic shared memory, at most 227 KB per CTA less 1 KB for
// the kernel's static shared memory
constexpr int kMaxMs = (227 * 1024 - 1024) / 32;
constexpr int kSmallMaxK = 512;                // the projected solve's per-column shared arrays
static_assert(kMaxK <= kSmallMaxK, "projected solve arrays");
constexpr int kBatchUpdTile = kFoldEvery;      // update tile: the split counters' exact range
constexpr int kBatchNormTile = 4096;           // normalise tile (elements)
constexpr int kBatchCsrRows = 16;              // CSR rows per operator tile
constexpr int kCsrGroup = 16;                  // slots sharing one CSR matrix per pass over it
constexpr int kCsrGroupRec = kCsrGroup + 3;    // group record: count, slots, staging byte offset (2 words)

struct SlotDesc {
    Geom g;
    Bufs bf;
    SketchParams sp;
    OpDev op;
    int k_target;
    int norm_tiles;                // tiles of this slot in the normalise table (its last-tile ticket)
    int conv_cols;                 // operator tiles: PSF FMA path, tiles per image row of tiles; CSR 0
    int tc_kp;                     // tensor-core convolution: KP (16 or 32), 0 for the other operators
    int tc_ct, tc_rows;            // its column tiles and output rows per unit
};

struct TileRef {
    int slot;
    int tile;
};

// the slot's step index at the start of a phase (-1 if the slot takes no
// step now), read by thread 0 and shared with the CTA; also a barrier
// between the tiles a CTA takes
__device__ __forceinline__ int slot_step(const SlotDesc* sd, int* s_j) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int j = -1;
        if (sd->k_target > 0) {
            const DevState* st = sd->bf.st;
            j = st->j;
            if (st->status[0] != IPF_OK || j >= sd->k_target || j >= sd->g.k_max) j = -1;
        }
        *s_j = j;
    }
    __syncthreads();
    return *s_j;
}

// Raise a kernel's dynamic shared-memory limit to at least `bytes`, never
// lowering it: the limit is one process-wide attribute of the function, and
// a launch captured in a CUDA graph with a larger size (another context's or
// engine's k_max) must stay valid after a smaller launch elsewhere (api.cu;
// thread safe).
cudaError_t raise_smem_ptr(const void* fn, size_t bytes);
template <class F> inline cudaError_t raise_smem(F fn, size_t bytes) {
    return raise_smem_ptr(reinterpret_cast<const void*>(fn), bytes);
}

// ---------------------------------------------------------------------------
// launchers (defined in the .cu files)
// ---------------------------------------------------------------------------
// k_ops.cu
// vbase + (*jptr) * ldv is the input vector (jptr NULL: vbase itself)
// tensor-core convolution for BF16 storage (k_conv_tc.cu)
constexpr int kConvTcGroup = 8;    // image rows per MMA group
// BF16 bits of f rounded to nearest even (finite f), and back
unsigned short bf16_bits_rn(float f);
float bf16_bits_to_float(unsigned short h);
// the B operand of the tensor-core convolution for a kw x kw flipped PSF
// F(a, b) (kw 15 or 31); returns KP (16 or 32), or 0 if kw is not supported
int conv_tc_operand(int kw, const std::function<float(int, int)>& F, std::vector<unsigned short>* img);
bool conv_tc_eligible(const OpDev& op, const void* vbase, long long ldv);
cudaError_t launch_conv_tc(const OpDev& op, const void* vbase, long long ldv, long long vcols, const int* jptr,
                           float* w, int* err, cudaStream_t s);

// w = A v_j: vbase/ldv/vcols describe the basis (vcols columns), j read from
// jptr (column 0 when NULL); err receives IPF_ERR_TIMEOUT if a bounded wait
// inside the tensor-core convolution gives up (may be NULL)
cudaError_t launch_op_apply(const OpDev& op, int storage, const void* vbase, long long ldv, long long vcols,
                            const int* jptr, int B, void* w, int* err, cudaStream_t s);
// (A v_j)(p_i) for i <= j directly at the pivot rows (PSF2D and CSR); float accumulation
cudaError_t launch_pivot_rows(const OpDev& op, int storage, const void* vbase, long long ldv, const DevState* st,
                              const int* piv, int B, int k_max, float* gout, cudaStream_t s);
cudaError_t launch_op_apply_f32_plain(const OpDev& op, const float* v, float* w, int nrhs,
                                      cudaStream_t s);
// k_hess.cu
// fwd: the pivot block is solved by forward substitution from the first step
cudaError_t launch_reset_state(DevState* st, bool fwd, cudaStream_t s);
// Gaussian sketch (gauss.cu).  A context's S (launch_gauss_fill_ctx,
// gauss_s_bytes): for BF16 / FP16 storage tiled in units of 16 rows x 64
// elements (unit (r / 16, i / 64) at ((r / 16) ceil(n / 64) + i / 64) 1024
// elements, row-major inside, zero outside m x n), for FP32 / FP64 row-major
// with m rows of lds = gauss_lds(n) elements (entry (r, i) at r*lds + i);
// launch_gauss_fill writes the row-major form with any lds (the public
// ipf_sketch_gaussian).  The workspace holds the rows of b the contraction
// takes as extra B columns (zeroed at creation, written per right-hand side
// by launch_gauss_bparts) and the slices' partial tiles.
size_t gauss_s_bytes(int storage, int m, long long n);
cudaError_t launch_gauss_fill_ctx(int storage, void* S, long long n, int m, unsigned long long seed, int num_sms,
                                  cudaStream_t s);
long long gauss_lds(long long n);
size_t gauss_workspace_bytes(int storage, int m, long long n, int k_max, int num_sms);
cudaError_t launch_gauss_fill(int storage, void* S, long long n, int m, long long lds, unsigned long long seed,
                              int num_sms, cudaStream_t s);
cudaError_t launch_gauss_bparts(int storage, const float* b, long long n, void* ws, cudaStream_t s);
// [S V_{K1} | S b]: svd (column-major m x K1, FP64 for F64 storage, else
// FP32) and c = S b (FP64); err receives IPF_ERR_TIMEOUT if a bounded wait
// inside the tensor-core kernel gives up
// variant: the pipeline of the 16-bit tensor-core kernel (64 or 32 K elements
// per stage), from gauss_variant (timed once per shape by the autotuner)
cudaError_t launch_gauss_sv(int storage, const void* S, int m, long long n, const void* V, long long ldv, int kcols,
                            int K1, void* ws, void* svd, double* c, int* err, int num_sms, int variant,
                            cudaStream_t s);
int gauss_variant(int storage, const void* S, int m, long long n, const void* V, long long ldv, int kcols, void* ws,
                  void* svd, double* c, int* err, int num_sms, cudaStream_t s);
// sampled pivoting: overwrite the step's pivot choice (after the update)
cudaError_t launch_sample_pivot(int storage, const Geom& g, const Bufs& bf, unsigned long long seed, int size,
                                cudaStream_t s);
cudaError_t launch_load_rhs(int storage, const float* b, const Geom& g, const Bufs& bf, cudaStream_t s);
// the FP64 pivot-block solve h = L_p^{-1} u(p) in two launches: the new row
// of L_p and of L_p^{-1} (needs only the pivots and the basis), then the
// product with u(p) (or forward substitution where DevState::fwd is set);
// launch_pivot_solve issues both
cudaError_t launch_pivot_minv(int storage, const Geom& g, const Bufs& bf, cudaStream_t s);
cudaError_t launch_pivot_apply(int storage, const Geom& g, const Bufs& bf, cudaStream_t s);
cudaError_t launch_pivot_solve(int storage, const Geom& g, const Bufs& bf, cudaStream_t s);
cudaError_t launch_update(int storage, const Geom& g, const Bufs& bf, const SketchParams& sp, int num_sms,
                          cudaStream_t s);
// split step: t = V_j h, then u = w - t with pivots zeroed and argmax keys
cudaError_t launch_gemv(int storage, const Geom& g, const Bufs& bf, int num_sms, cudaStream_t s);
cudaError_t launch_combine(const Geom& g, const Bufs& bf, int num_sms, cudaStream_t s);
// S v_c for the pending column c (DevState::sk_pending) of a one-RHS float
// basis with the zeta = 8 sketch table; no-op when nothing is pending
cudaError_t launch_sketch_col(int storage, const Geom& g, const Bufs& bf, const SketchParams& sp, int num_sms,
                              cudaStream_t s);
cudaError_t launch_normalize(int storage, const Geom& g, const Bufs& bf, const SketchParams& sp,
                             bool want_sw, int num_sms, cudaStream_t s);
// precomputed sketch columns for zeta = 8 with every block <= 128 rows
bool sketch_table_ok(const SketchParams& sp);
cudaError_t launch_sketch_table(const SketchParams& sp, long long n, unsigned long long* tab, cudaStream_t s);
cudaError_t launch_sketch_vector(const float* x, long long n, const SketchParams& sp, int F,
                                 long long* acc, float* absmax_out, cudaStream_t s, int num_sms,
                                 bool find_max);
cudaError_t launch_fixed_to_double(const long long* acc, int m, double scale, double* y, cudaStream_t s);
cudaError_t launch_sketch_finish(const long long* acc, int m, long long n, int zeta, const unsigned* absmax,
                                 double* y, cudaStream_t s);
// batched step (k_hess.cu, k_ops.cu, k_conv_tc.cu): one launch per phase for
// the slots of one float storage type
// per entry of list (its slot field): the row of L_p^{-1}, then the product
cudaError_t launch_batch_pivot_solve(int storage, const SlotDesc* slots, const TileRef* list, int nslots, int k_max,
                                     cudaStream_t s);
cudaError_t launch_batch_update(int storage, const SlotDesc* slots, const TileRef* tiles, int ntiles, int k_max,
                                int m_s_max, int num_sms, cudaStream_t s);
cudaError_t launch_batch_normalize(int storage, const SlotDesc* slots, const TileRef* tiles, int ntiles, int num_sms,
                                   cudaStream_t s);
// (A v_j)(p_i) at the pivot rows into bf.gpiv: tile t of a slot = pivots 8t .. 8t+7
cudaError_t launch_batch_pivot_rows(int storage, const SlotDesc* slots, const TileRef* tiles, int ntiles, int num_sms,
                                    cudaStream_t s);
// CSR products of groups of slots sharing one matrix (groups: per group
// kCsrGroupRec ints, the count, the slots, the byte offset of its staging
// rows: cols x kCsrGroup values of the storage type; tile.slot = the group):
// the staging of each group's v_j (stage_tiles: 1024 columns each), then the
// products (tiles: kBatchCsrRows rows each)
cudaError_t launch_batch_csr_group(int storage, const SlotDesc* slots, const int* groups, unsigned char* stage,
                                   const TileRef* stage_tiles, int nstage, const TileRef* tiles, int ntiles,
                                   int num_sms, cudaStream_t s);
// PSF (FMA column convolution, kw 7 / 15 / 31) and CSR products
cudaError_t launch_batch_operator(int storage, const SlotDesc* slots, const TileRef* tiles, int ntiles, int num_sms,
                                  cudaStream_t s);
// tensor-core convolution (BF16) of the slots with tc_kp == kp; maps: the
// slots' tensor maps, kMaxSlots x conv_tc_map_bytes() bytes of host memory
// (entry s for slot s, built by conv_tc_map)
cudaError_t launch_batch_conv_tc(int kp, const void* maps, const SlotDesc* slots, const TileRef* units, int nunits,
                                 cudaStream_t s);
bool conv_tc_map(const OpDev& op, const void* vbase, long long ldv, long long vcols, void* map_out);
size_t conv_tc_map_bytes();

// api.cu: contexts the batched step can drive (see there)
bool ctx_slot_desc(ipf_ctx* c, SlotDesc* d, int* storage);
void ctx_steps_taken(ipf_ctx* c, int k);

// batch.cu: the project's autotuner cache (per process, and in the JSON file
// named by IPF_TUNE_CACHE): per key the chosen variant, its parameter and time
bool tune_lookup(const char* key, int* variant, int* param);
void tune_store(const char* key, int variant, int param, double us);

// batch.cu: the batched step of the serving loop (one engine per server,
// used from its scheduler thread only)
struct BatchEngine;
BatchEngine* batch_create();
void batch_destroy(BatchEngine* b);
// put a context in a free slot to take k steps (its initialisation enqueued
// before `ready`); returns the slot, or -1 if the context cannot be batched
// or no slot is free
int batch_add(BatchEngine* b, ipf_ctx* c, int k, cudaStream_t ready);
void batch_remove(BatchEngine* b, int slot);
int batch_steps(const BatchEngine* b, int slot);
int batch_used(const BatchEngine* b);
cudaError_t batch_run(BatchEngine* b, int steps, cudaEvent_t done);
void batch_counters(const BatchEngine* b, long long* graph_turns, long long* eager_turns, long long* captures);

// k_small.cu: workspace for k <= k_max and up to nl_max lambdas per chunk
size_t solve_workspace_bytes(const Geom& g, int nl_max);
// form M = [Z | c] (and T = S V_k) and their R factors
cudaError_t launch_solve_prepare(const Geom& g, const Bufs& bf, int zeta, int k, bool need_T, bool use_sw,
                                 void* work, int nl_max, int num_sms, cudaStream_t s, bool qmr = false);
// per lambda: y, then x = V_k y into x_dev ([l][r][n] float32)
cudaError_t launch_solve_lambdas(int storage, const Geom& g, const Bufs& bf, int k, bool need_T,
                                 const double* lambdas_dev, int nl, int penalty, void* work, int nl_max,
                                 float* x_dev, int num_sms, cudaStream_t s);
// device-side barrier timeout flag of the last prepare (host read, synchronous)
cudaError_t solve_error_flag(const void* work, const Geom& g, int* flag);

}  // namespace ipf
