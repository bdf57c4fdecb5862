/*
 * ipf.h -- C ABI of libipf, a GB300 (sm_103a) implementation of the sketched
 * inner-product-free Krylov method sCMRH of arXiv 2502.02721
 * ("Randomized and inner-product free Krylov methods for large-scale inverse
 * problems").
 *
 * Problem (Sec. 1, Eq. 1-3):  b = A x_true + e.  The library builds, with no
 * inner products, the pivoted Hessenberg basis V_{k+1} = L_{k+1} of
 * K_k(A, b) with A V_k = V_{k+1} H_{k+1,k} (Sec. 3.1, Eq. Hessenberg_s),
 * sketches it with a sparse-sign embedding S (Sec. 2), and solves the
 * sketched projected problem (Sec. 3.2 Eq. sketched_LSLU; Sec. 3.3
 * Eq. sketched_LSLU_hybrid)
 *      y = argmin || S (A V_k y - b) ||^2 + lambda^2 || S V_k y ||^2,
 *      x_k = V_k y                                      (x_0 = 0).
 * A is reached only through products A v (Sec. 1).
 *
 * Conventions for every entry point
 *  - Pointers are plain host or device addresses; which one is stated per
 *    argument (an *_mem flag selects where caller arrays live).
 *  - No exception crosses the ABI.  Every call returns an ipf_status.
 *  - Errors on a context are sticky: once a call fails with an IPF_ERR_*
 *    code, later calls on that context return the same code.
 *    ipf_last_error() gives a one-line message.
 *  - Work is enqueued on the context's own CUDA stream, ordered after all
 *    work already on the caller's stream (config.stream) at call time, and
 *    the caller's stream is made to wait for it before the call returns.
 *  - All device memory of a context is allocated at ipf_create (through the
 *    config's alloc/free callbacks when given, else cudaMalloc) and freed by
 *    ipf_destroy.
 */
#ifndef IPF_H
#define IPF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum ipf_status {
    IPF_OK = 0,
    IPF_BREAKDOWN = 1,        /* H(k+1,k) = 0 (Algorithm 1): not an error; the iterate at
                                 k_done is exact in K_{k_done}(A, b)                   */
    IPF_PENDING = 2,          /* serving: request not finished yet                    */
    IPF_ERR_ARG = -1,         /* invalid argument; nothing was enqueued               */
    IPF_ERR_OOM = -2,         /* device allocation failed                             */
    IPF_ERR_CUDA = -3,        /* a CUDA call failed (message in ipf_last_error)       */
    IPF_ERR_NONFINITE = -4,   /* a pivot value was NaN or Inf                         */
    IPF_ERR_TIMEOUT = -5,     /* a bounded device-side wait gave up                   */
    IPF_ERR_STATE = -6,       /* call not valid in the current state (e.g. k > steps) */
    IPF_ERR_UNSUPPORTED = -7, /* combination of options not implemented               */
    IPF_ERR_REJECTED = -8     /* serving: request can never fit the memory budget     */
} ipf_status;

enum ipf_op_kind {
    IPF_OP_PSF2D = 1,            /* w = P * v, odd ph x pw PSF, zero boundary          */
    IPF_OP_PSF2D_SEP_MOTION = 2, /* w = M * (g_col (x) g_row * v), both passes zero
                                    boundary, cropped to the image in between          */
    IPF_OP_CSR = 3               /* w = A v, CSR (int64 rowptr, int32 colind, f32 vals) */
};

enum ipf_mem { IPF_MEM_HOST = 0, IPF_MEM_DEVICE = 1 };

/* storage precision of the basis V; arithmetic is FP32-accumulate for
 * F32/BF16/F16 and FP64 for F64; the pivot-block solve and the projected
 * least-squares solve are FP64 in every mode.                              */
enum ipf_storage { IPF_STORE_F64 = 0, IPF_STORE_F32 = 1, IPF_STORE_BF16 = 2, IPF_STORE_F16 = 3 };

/* Tikhonov penalty: lambda^2 ||S V_k y||^2 (Eq. sketched_LSLU_hybrid with
 * S_1 = S) or lambda^2 ||y||^2 (the penalty of Eq. TSP).                   */
enum ipf_penalty { IPF_PEN_SKETCHED_X = 0, IPF_PEN_Y = 1 };

/* How S A V_k is assembled: DIRECT sketches each product u = A v_j before
 * the elimination (the sketched product of Algorithm 1, z_k = S u), HESSENBERG uses
 * S V_{k+1} H_k.  They agree in exact arithmetic; with BF16/FP16 storage
 * DIRECT is the sketched objective over the stored basis (the sketch of
 * each product is assembled by linearity from S of the stored basis and S
 * of the unrounded new vector, which costs a second sketch per step for
 * BF16/FP16).  DIRECT needs float storage.  AUTO uses HESSENBERG.          */
enum ipf_zform { IPF_Z_DIRECT = 0, IPF_Z_HESSENBERG = 1, IPF_Z_AUTO = 2 };

/* Which process builds the basis.
 * SCMRH  the pivoted Hessenberg process on a square A (Sec. 3.1 Eq.
 *        Hessenberg_s): x_k in K_k(A, b).
 * SLSLU  the generalized Hessenberg process (Sec. 3.1 Eq. Hessenberg_r;
 *        Algorithm 1, Algorithm 2) for any m x n PSF2D or CSR operator:
 *        A L_k = D_{k+1} H_{k+1,k} and A^T D_{k+1} = L_{k+1} W_{k+1} with two
 *        pivoted unit lower trapezoidal bases, D in R^m and L in R^n, and
 *        x_k = L_k y_k in K_k(A^T A, A^T b).  Each step applies A to l_k and
 *        A^T to d_{k+1}; S_2 (l x m, config.seed) sketches D, S_1 (l x n,
 *        seed config.seed XOR 0x5DEECE66DA3B1F27) sketches L; y minimises ||S_2 (A L_k y - b)||^2 +
 *        lambda^2 ||S_1 L_k y||^2.  b has m entries per RHS, x has n.  A^T is
 *        the convolution with the flipped PSF, or the CSR transpose (built on
 *        the host at create).  Steps run on one stream (config.overlap is
 *        ignored); the penalty is always the sketched-x form.               */
enum ipf_method { IPF_METHOD_SCMRH = 0, IPF_METHOD_SLSLU = 1 };

/* The sketching matrix S (m_s x n).
 * SPARSE_SIGN  the block sparse-sign embedding (see ipf_sketch_apply),
 *              applied to each basis vector as it is formed, exact sums.
 * GAUSSIAN     the Gaussian embedding of the paper's experiments (Sec. 2,
 *              Sec. 4): N(0, 1/m_s) entries from the SplitMix64 counter hash
 *              by Box-Muller (entry (r, i) from outputs 2c, 2c+1, c = r*n + i,
 *              of the generator started at config.seed; u = ((out >> 11) + 1)
 *              2^-53; z = sqrt(-2 ln u1) cos(2 pi u2); S = z / sqrt(m_s)),
 *              rounded to the storage type and kept in device memory
 *              (m_s x n elements; ipf_sketch_gaussian writes the same values
 *              row-major, the context keeps them in its own tiling).  No
 *              per-step sketch: at solve time one contraction forms
 *              [S V_{k+1} | S b] (the library's own kernels: tensor cores for
 *              BF16 / FP16 storage, with b entering as three exact parts of
 *              the storage type, and FP32 accumulation in slices of n added
 *              in FP64 in a fixed order; CUDA cores for FP32 / FP64
 *              storage).  SCMRH with nrhs == 1 only (else
 *              IPF_ERR_UNSUPPORTED); the Z form is HESSENBERG; ipf_export's
 *              SV, SZ and c are those of the sparse-sign path (zero here). */
enum ipf_sketch { IPF_SKETCH_SPARSE_SIGN = 0, IPF_SKETCH_GAUSSIAN = 1 };

/* Forward operator.  For PSF kinds n = rows*cols and images are row-major.
 * For CSR, rows x cols is m x n and the method needs m == n (square A).
 * mem says where psf/sep_row/sep_col/motion/rowptr/colind/vals live:
 *   IPF_MEM_HOST    the library copies them at ipf_create / ipf_op_create;
 *   IPF_MEM_DEVICE  PSF arrays are copied; CSR arrays are referenced, not
 *                   copied: the caller keeps them alive and unchanged for
 *                   the lifetime of every context or handle using them.
 * Host CSR arrays are validated (rowptr monotone from 0 to nnz, column
 * indices in [0, cols)); device CSR arrays must satisfy the same and are
 * not checked.                                                            */
typedef struct ipf_operator {
    int kind;
    int rows, cols;
    const float* psf;            int ph, pw;        /* IPF_OP_PSF2D, ph, pw odd <= 63   */
    const float* sep_row;        const float* sep_col; int slen;   /* odd <= 63        */
    const float* motion;         int mlen;          /* mlen x mlen, odd <= 15          */
    const long long* rowptr;     const int* colind; const float* vals; long long nnz;
    int mem;
} ipf_operator;

typedef void* (*ipf_alloc_fn)(size_t bytes, void* user);
typedef void (*ipf_free_fn)(void* ptr, void* user);

typedef struct ipf_config {
    int k_max;                   /* maximum Hessenberg steps, 1..480 (basis has k_max+1
                                    vectors); with the Gaussian sketch 1..247              */
    int m_s;                     /* sketch rows (l in Sec. 2); zeta <= m_s <= 7232 (the exact
                                    sketch counters of a right-hand side live in shared
                                    memory; larger: IPF_ERR_UNSUPPORTED)                    */
    int zeta;                    /* nonzeros per sketch column, 1..16                       */
    unsigned long long seed;     /* sketch seed (SplitMix64 state)                          */
    int storage;                 /* enum ipf_storage                                        */
    int penalty;                 /* enum ipf_penalty                                        */
    int zform;                   /* enum ipf_zform                                          */
    int nrhs;                    /* independent right-hand sides sharing A: 1, 2, 4 .. 32;
                                    PSF operators and F64 storage need nrhs == 1            */
    int use_graphs;              /* replay Hessenberg steps from CUDA graphs: one step and
                                    eight consecutive steps are captured once, and ipf_step
                                    launches the eight-step graph while 8 or more remain    */
    int profile;                 /* bracket every kernel with CUDA events on the context's
                                    stream (launches eagerly; read with ipf_profile_read)   */
    int overlap;                 /* PSF2D/CSR with float storage, second stream per step:
                                    0 one stream; 1 the operator beside V_j h; 2 (default)
                                    the operator beside the pivot-row products and the
                                    FP64 pivot-block solve.  In modes 0 and 2 with one
                                    RHS, float storage, zeta 8 and no DIRECT Z with
                                    BF16/FP16, the sketch S v_{j+1} of each new column is
                                    taken by the next step's update (which streams that
                                    column anyway) and the newest column's before a solve
                                    or export; the sums are the same exact integers      */
    int method;                  /* enum ipf_method (default IPF_METHOD_SCMRH)               */
    int sketch;                  /* enum ipf_sketch (default IPF_SKETCH_SPARSE_SIGN)        */
    int pivot_sample;            /* 0 (default): each pivot is the largest |.| over all
                                    candidate rows.  1..64: sampled pivoting (Sec. 3.2,
                                    Sec. 4): the largest |.| over that many candidate rows
                                    drawn for each pivot choice c (0 at the initialisation,
                                    j+1 at step j): draw t is SplitMix64 output c*4096 + t
                                    of the generator started at seed XOR 0xA5A5A5A5A5A5A5A5
                                    (SLSLU's L basis: also XOR 0x5DEECE66DA3B1F27), row
                                    floor(out * n / 2^64); draws hitting a pivot row or an
                                    accepted row are skipped, at most 4096 draws; if no more
                                    candidates remain than the sample size, or every sampled
                                    entry is zero, the full maximum is used                   */
    int conv_fma;                /* PSF2D with BF16 storage: 0 (default) runs the product on
                                    the tensor cores when the PSF pads to 15x15 or 31x31 and
                                    cols % 8 == 0; 1 keeps the FP32 FMA convolution         */
    int pivot_fwd;               /* the FP64 pivot-block solve h = L_p^{-1} u(p) of each step:
                                    0 (default) in inverse form: each step appends the row
                                    of L_p^{-1} that matches the new row of L_p and forms h
                                    as a product with independent rows, switching to forward
                                    substitution for the rest of the solve if a row of the
                                    inverse exceeds 2^20 in magnitude; 1 forward
                                    substitution throughout (one CTA)                     */
    void* stream;                /* cudaStream_t of the caller (NULL: legacy default)      */
    ipf_alloc_fn alloc;          /* optional device allocator (e.g. a framework's pool)    */
    ipf_free_fn free;
    void* alloc_user;
} ipf_config;

typedef struct ipf_solve_info {
    int k_used;                  /* iterations used for this right-hand side              */
    int k_done;                  /* completed Hessenberg steps                            */
    int status;                  /* IPF_OK, IPF_BREAKDOWN or an error                      */
    int pad;
} ipf_solve_info;

typedef struct ipf_ctx ipf_ctx;
typedef struct ipf_op ipf_op;

/* Fill *cfg with defaults: k_max 50, m_s 200, zeta 8, seed 1, F32 storage,
 * sketched-x penalty, AUTO Z, nrhs 1, graphs on, overlap 2, tensor-core
 * convolution where it applies, default stream, cudaMalloc.               */
void ipf_config_default(ipf_config* cfg);

/* Bytes of device memory ipf_create would allocate for this problem
 * (the serving loop admits requests by this number).                      */
size_t ipf_footprint(const ipf_operator* op, const ipf_config* cfg);

/* Create a solve context and enqueue the initialisation of Algorithm 1
 * (r_0 = b, pivot p_1 = argmax |b| with the lowest index on ties,
 * beta = b(p_1), v_1 = b / beta, c = S b).
 *   op    operator (see ipf_operator for ownership of its arrays)
 *   b     nrhs x n float32, right-hand side r stored at b + r*n; b_mem says
 *         whether it is host or device memory; copied, not retained.
 *   cfg   options; copied.
 *   out   receives the context (NULL on failure).
 * Errors: IPF_ERR_ARG (bad sizes or options), IPF_ERR_UNSUPPORTED,
 * IPF_ERR_OOM, IPF_ERR_CUDA.  A zero right-hand side is not an error: that
 * RHS reports IPF_BREAKDOWN with k_done 0 and solves to x = 0.             */
ipf_status ipf_create(const ipf_operator* op, const float* b, int b_mem,
                      const ipf_config* cfg, ipf_ctx** out);

/* Start a new solve on an existing context with a new right-hand side b
 * (same layout and ownership as in ipf_create), reusing all of its device
 * memory: clears the state and enqueues the initialisation.  Allocates
 * nothing.  Clears a sticky error only if it was IPF_ERR_NONFINITE.        */
ipf_status ipf_reset(ipf_ctx* ctx, const float* b, int b_mem);

/* Enqueue nsteps Hessenberg steps (the loop of Algorithm 1, square form):
 * u = A v_j; h = L_p^{-1} u(p) (the sequential elimination of Algorithm 1
 * as a unit-lower forward substitution on the pivot rows, FP64);
 * u -= V_j h with the pivot rows set to 0; p_{j+1} = argmax |u| over
 * non-pivot rows (lowest index on ties); H(j+1, j) = u(p_{j+1});
 * v_{j+1} = u / H(j+1, j) rounded to the storage type; S v_{j+1}.
 * Asynchronous.  A right-hand side that breaks down stops there; the
 * others continue.  nsteps is clipped to k_max minus the steps already
 * enqueued; *k_enqueued (may be NULL) receives the total enqueued.        */
ipf_status ipf_step(ipf_ctx* ctx, int nsteps, int* k_enqueued);

/* Wait for the context's work; k_done (nrhs entries, host, may be NULL)
 * receives the completed steps per RHS.  Returns the worst RHS status.    */
ipf_status ipf_sync(ipf_ctx* ctx, int* k_done);

/* Solve the sketched projected problem at k for each lambda and form
 * x = V_k y (Sec. 3.2, 3.3).  For RHS r, k_r = min(k, k_done_r).
 *   lambdas  nl >= 1 host doubles (0 gives the plain sketched LS problem)
 *   x_out    nl x nrhs x n float32, x for lambda l and RHS r at
 *            x_out + (l*nrhs + r)*n; host or device per x_mem.
 *   info     nrhs host entries, may be NULL.
 * Synchronises with the context's stream.  IPF_ERR_STATE if k exceeds the
 * steps enqueued.                                                          */
ipf_status ipf_solve(ipf_ctx* ctx, int k, const double* lambdas, int nl,
                     float* x_out, int x_mem, ipf_solve_info* info);
/* With x_mem == IPF_MEM_DEVICE and info == NULL, ipf_solve does not wait
 * for the GPU: it returns once the work is enqueued, and a device-side
 * failure of the solve is reported by the next ipf_sync.                  */

/* Kernel timings of a context created with config.profile = 1: for each
 * kind (0 operator, 1 pivot-block solve (two launches: the row of L_p^{-1},
 * then h), 2 update+argmax or V_j h,
 * 3 normalise (+ sketch unless deferred), 4 initialisation, 5 projected-solve
 * QR, 6 per-lambda solve + x = V_k y, 7 operator at the pivot rows,
 * 8 u = A v_j - V_j h with argmax, 9 the Gaussian sketch's [S V_{k+1} | S b],
 * 10 sampled pivot choice, 11 deferred sketch S v_j) the summed
 * milliseconds, launch counts and the summed algorithmic bytes of the
 * launches (0 where not defined), since the previous read.  With
 * config.overlap 1 a step runs the operator on a second stream beside V_j h,
 * so kinds 0 and 2 overlap in time; with overlap 2, kinds 0, 7, 1 and 11.
 * Arrays of 12 entries, host; synchronises.                               */
ipf_status ipf_profile_read(ipf_ctx* ctx, double* ms, long long* launches, double* bytes);

/* The quasi-minimal residual iterate of the same basis, without the sketch
 * (Eq. Hessenber_LS: CMRH for SCMRH contexts, LSLU for SLSLU contexts), with
 * the Tikhonov term of Eq. TSP for lambda > 0:
 *     y = argmin ||beta e_1 - H_{k+1,k} y||^2 + lambda^2 ||y||^2,
 * x = V_k y (L_k y for SLSLU).  The paper's non-sketched comparison method.
 * Arguments, layout and errors as ipf_solve; IPF_ERR_UNSUPPORTED if
 * k + 1 > m_s (the (k+1)-row problem is solved in the sketch's workspace). */
ipf_status ipf_solve_qmr(ipf_ctx* ctx, int k, const double* lambdas, int nl, float* x_out, int x_mem,
                         ipf_solve_info* info);

/* Copy the method's state for RHS r to host memory (any pointer may be
 * NULL): pivots (k_max+1 ints, 0-based rows, -1 past the last pivot),
 * H ((k_max+1) x k_max FP64, column-major, column j holds H(0..j+1, j)),
 * SV (m_s x (k_max+1) FP64, column-major: S v_j of the stored basis),
 * SZ (m_s x k_max FP64: z_j = S A v_j, zero unless the DIRECT form is in
 * use), c (m_s FP64: S b), beta (1 double).  Synchronises.                */
ipf_status ipf_export(ipf_ctx* ctx, int r, int* pivots, double* H, double* SV, double* SZ,
                      double* c, double* beta);

/* Copy basis vector j (0-based, j <= k_done) of RHS r as float32 (host). */
ipf_status ipf_export_basis(ipf_ctx* ctx, int r, int j, float* v_out);

/* SLSLU contexts: the second basis.  ipf_export and ipf_export_basis give
 * the D side (pivots t, H, S_2 D, c = S_2 b, beta); these give the L side:
 * pivots g (k_max + 1 entries, -1 past the last), a (k_max + 1) x k_max
 * column-major table of W (Eq. Hessenberg_r) whose column c (0-based) holds
 * W(1..c+1, c+2), the coefficients of q = A^T d_{c+2} on l_1..l_{c+1}, in
 * rows 0..c and the pivot W(c+2, c+2) in row c+1, S_1 L ((k_max + 1) x m_s),
 * and W(1, 1) = (A^T d_1)(g_1).  ipf_export_basis_l writes column j of L (n
 * floats).  IPF_ERR_STATE for SCMRH contexts.                             */
ipf_status ipf_export_dual(ipf_ctx* ctx, int r, int* pivots_l, double* W, double* SL, double* w11);
ipf_status ipf_export_basis_l(ipf_ctx* ctx, int r, int j, float* l_out);

void ipf_destroy(ipf_ctx* ctx);
const char* ipf_status_str(ipf_status s);
const char* ipf_last_error(const ipf_ctx* ctx);

/* ---- operator and sketch kernels as standalone calls (device pointers) ---- */

/* Upload an operator (see ipf_operator for ownership) and apply it:
 * w = A v for nrhs vectors (CSR: nrhs a power of two <= 32).  v is device
 * float32 nrhs x n (vector r at offset r*n), w device float32 nrhs x m
 * (m = rows for CSR, n otherwise); the caller guarantees those sizes.
 * Runs on `stream` (cudaStream_t, may be NULL).                           */
ipf_status ipf_op_create(const ipf_operator* op, ipf_op** out);
ipf_status ipf_op_apply(ipf_op* h, const float* v_dev, float* w_dev, int nrhs, void* stream);

/* w = A v for one vector stored in BF16 (v_dev: n BF16 values, device),
 * accumulated in FP32 (w_dev: m float32, device): the product a Hessenberg
 * step applies to a BF16 basis vector.  For PSF2D operators whose PSF pads
 * to 15x15 or 31x31 with cols % 8 == 0 it runs on the tensor cores, with
 * the PSF carried as the sum of two BF16 parts (about 2^-16 relative), unless
 * use_fma != 0, which selects the FP32 FMA convolution.  v_dev must be
 * 16-byte aligned for the tensor-core path.  Runs on `stream`; a stall of
 * seconds inside the tensor-core kernel (which then gives up) leaves w
 * unspecified and is not reported by this call.                           */
ipf_status ipf_op_apply_bf16(ipf_op* h, const void* v_dev, float* w_dev, int use_fma, void* stream);
void ipf_op_destroy(ipf_op* h);

/* y = S x for the block sparse-sign sketch S (m_s x n, zeta nonzeros
 * +-1/sqrt(zeta) per column, drawn from a SplitMix64 counter hash of seed;
 * Sec. 2 names sparse sign embeddings among the subspace embeddings).
 * x: device float32 (n); y: device float64 (m_s).  Sums are accumulated
 * exactly in 64-bit fixed point scaled to max|x|, so the result does not
 * depend on thread order.  Allocates its scratch with cudaMallocAsync on
 * `stream` and frees it before returning.                                  */
ipf_status ipf_sketch_apply(const float* x_dev, long long n, int m_s, int zeta,
                            unsigned long long seed, double* y_dev, void* stream);

/* Writes the Gaussian sketch S (m_s x n) of config.sketch = GAUSSIAN
 * (Sec. 2; Box-Muller on the SplitMix64 counter hash as described at
 * enum ipf_sketch) to S_dev, row-major (entry (r, i) at r*n + i, the entry's
 * counter), each entry the FP64 value z / sqrt(m_s) rounded to nearest-even
 * in `storage` (BF16 through FP32).  BF16 and F16 entries are evaluated in
 * FP32 with an error bound and recomputed in FP64 where the bound does not
 * fix the rounded value, so all storage types store the FP64 definition's
 * rounding.  S_dev: device, m_s * n elements of the storage type,
 * caller-owned.  Runs on `stream`, no allocation.  Errors: IPF_ERR_ARG (null
 * S_dev, n < 1, m_s < 1, unknown storage), IPF_ERR_CUDA (launch failure).  */
ipf_status ipf_sketch_gaussian(int storage, unsigned long long seed, long long n, int m_s, void* S_dev,
                               void* stream);

/* ---- serving: many solves in flight on one GPU ---- */

typedef struct ipf_server ipf_server;

typedef struct ipf_server_config {
    size_t hbm_budget_bytes;     /* device memory for in-flight requests, reserved at
                                    creation (0: 80% of the free memory)                  */
    size_t pinned_bytes;         /* pinned host staging for b and x (0: 1 GiB)             */
    int max_inflight;            /* requests on the GPU at once, 1..64                     */
    int steps_per_slice;         /* Hessenberg steps enqueued per request per turn (0: 8)  */
    int per_request;             /* 0 (default): requests the batched step can drive share
                                    it (see ipf_server_create); 1: every request steps on
                                    its own context and streams                           */
} ipf_server_config;

typedef struct ipf_request {
    ipf_operator op;             /* host arrays are copied at submit; device CSR arrays are
                                    referenced (kept alive by the caller until polled)    */
    const float* b;              /* host, nrhs x n, copied at submit                       */
    ipf_config cfg;              /* k_max, m_s, zeta, seed, storage, penalty, nrhs, ...;
                                    stream and allocator fields are ignored               */
    int k;                       /* Hessenberg steps, 1..cfg.k_max                         */
    double lambda;               /* Tikhonov parameter (0: plain sketched LS)              */
} ipf_request;

typedef struct ipf_result {
    int status;                  /* IPF_PENDING, IPF_OK, IPF_BREAKDOWN or an error         */
    int k_used;
    double t_submit, t_admit, t_done;   /* host steady-clock seconds                        */
} ipf_result;

/* Start a serving loop on the current device: a scheduler thread admits
 * requests when a slot is free and ipf_footprint(request) fits in what is
 * left of the budget (first come, first served), each into its own context
 * (its basis, pivots and sketches stay on the device until it retires).
 * Requests with one RHS, float storage, the sparse-sign sketch with zeta 8
 * and m_s <= 1024, full pivoting, no DIRECT Z form for BF16/FP16, and a PSF2D
 * operator whose PSF pads to 7x7, 15x15 or 31x31 or a CSR operator, share the
 * batched step: one turn advances every such in-flight request by
 * steps_per_slice Hessenberg steps with one launch per phase per step over
 * a device work list of all of them (requests of different n, k and step
 * counts in the same launches; a turn is replayed from a CUDA graph while
 * the set of requests stays the same).  For a BF16 PSF the product is the
 * FP32 FMA convolution or the tensor-core convolution with a band height
 * chosen by timing them on the request the first time its (PSF width, image
 * size) is seen, kept per process and, if the environment variable
 * IPF_TUNE_CACHE names a file, in that JSON file.  A request's result does not
 * depend on which other requests share its launches.  Other requests (and
 * all of them with per_request) step on their own streams.  After k steps
 * the request solves at k with lambda and copies x to the host.  All device
 * memory of requests comes from one arena reserved here, so admission and
 * retirement allocate nothing.  Errors: IPF_ERR_ARG, IPF_ERR_OOM (budget
 * cannot be reserved), IPF_ERR_CUDA.                                     */
ipf_status ipf_server_create(const ipf_server_config* cfg, ipf_server** out);

/* Queue a request; *ticket identifies it.  IPF_ERR_REJECTED if it can never
 * fit the budget; IPF_ERR_ARG for malformed requests.  Thread-safe.        */
ipf_status ipf_submit(ipf_server* s, const ipf_request* rq, unsigned long long* ticket);

/* IPF_PENDING until the request is done; then fills *res, copies x (nrhs x
 * n float32) to x_out if not NULL, forgets the ticket and returns the
 * request's status.  Thread-safe.                                         */
ipf_status ipf_poll(ipf_server* s, unsigned long long ticket, ipf_result* res, float* x_out);

/* Requests that took a slot of the batched step so far, and the engine's
 * turns launched from a CUDA graph, launched eagerly, and graph captures
 * (any pointer may be NULL).                                              */
ipf_status ipf_server_batch_stats(ipf_server* s, int* batched, long long* graph_turns, long long* eager_turns,
                                  long long* captures);

/* In-flight requests, queued requests and the budget they reserve.        */
ipf_status ipf_server_stats(ipf_server* s, int* inflight, int* queued, size_t* hbm_in_use);

/* Stop the scheduler, finish nothing further, release all memory.        */
void ipf_server_destroy(ipf_server* s);

/* ipf_sketch_apply without any device allocation.  The paper has no
 * counterpart: this is a service for callers that cannot allocate device
 * memory when they call, e.g. a runtime that owns and caps the GPU's memory
 * in pre-reserved pools, or a latency-critical path where an allocation's
 * cost or possible failure is not acceptable.  Same arguments, result and
 * kernels as ipf_sketch_apply; x and y are still the caller's.
 *  - Scratch is one fixed array of 33,024 bytes inside the library's device
 *    image (every GPU that loads libipf holds it until the process exits),
 *    so m_s must be <= 4096; larger m_s returns IPF_ERR_UNSUPPORTED.
 *  - The first call on a device looks up that array's device address with
 *    that device current; make that first call before any stream capture.
 *  - Every call shares the array and it keeps the last call's contents; each
 *    call clears the part it uses on `stream` first.  Calls whose work
 *    overlaps on the GPU (other streams, unordered host threads) race on it:
 *    order them on one stream or synchronise between them.
 * Errors: IPF_ERR_ARG as ipf_sketch_apply, IPF_ERR_UNSUPPORTED (m_s > 4096),
 * IPF_ERR_CUDA.                                                            */
ipf_status ipf_sketch_apply_noalloc(const float* x_dev, long long n, int m_s, int zeta,
                                    unsigned long long seed, double* y_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* IPF_H */
