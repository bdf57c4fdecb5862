// Zero-boundary 2-D convolution w = P * v on the 5th-generation tensor cores
// (tcgen05) for basis vectors stored in BF16, FP32 accumulation.
//
// With F the flipped PSF padded to KW x KW (KW = 15 or 31, c = KW/2),
//     w[y, x] = sum_{a,b} F[a][b] v[y - c + a, x - c + b],
// so image row iy reaches output row y through tap a = iy - y + c.  A CTA
// owns 128 output columns x0.. and a band of output rows, and takes the
// image rows in groups of G = 8 (iy0 .. iy0 + 7).  For one group
//     D[x, j] = sum_{r < G} sum_{b < KP} v[iy0 + r, x0 - c + x + b] B[j, (r, b)],
//     B[j, (r, b)] = F[r + j + 1 - G][b]   (zero outside 0..KW-1),
// is that group's whole contribution to output row y = iy0 + G - 1 + c - j,
// j = 0 .. KW + G - 2: a dense 128 x N x (G KP) contraction (KP = KW + 1),
// 2 G KP / 16 MMAs per group.  The CUDA cores only carry the KW - 1 output
// rows that straddle two groups (a shift register of partial sums).
//
// Operands, both K-major without swizzle in shared memory:
//   A  per image row, the Hankel matrix H[x, b] = v[iy, x0 - c + x + b].  A
//      K-major core matrix (8 rows x 8 elements) of it depends only on
//      (x/8 + b/8), so NQ = 16 + KP/8 - 1 blocks of 128 bytes hold it, block
//      q row s = v[iy, x0 - c + 8q + s .. +7]; the descriptor uses 128 bytes
//      for both the K and the M core-matrix strides.  Built from a staged row
//      segment by the builder warps.
//   B  [B_hi ; B_lo] (N = 2 NP rows, NP = KW + G - 1 rounded up to 8): B with
//      F rounded to BF16, and with the BF16 rounding of the remainder, so
//      hi + lo carries F to about 2^-16 relative; the halves land in separate
//      accumulator columns and are added in FP32.  Built once on the host
//      (conv_tc_operand) in this layout.
// Image rows arrive by TMA (3-D map over the basis: x, y, basis column j, j
// read from device memory), 8 rows of 160 elements per box starting at
// x0 - 16 (a multiple of 8 elements), zero-filled outside the image.
//
// One barrier wait, commit and arrive per group (each tcgen05 instruction
// and barrier test costs tens of cycles of issue latency in its thread).
// What bounds a group is shared-memory bandwidth: each MMA reads its A tile
// (4 KB) and B tile (N x 32 bytes) from shared memory, and the builders read
// the staged rows and store the Hankel blocks, about 1,000 128-byte
// wavefronts per group of 8 image rows; the B image therefore arrives by one
// bulk copy, and a builder lane writes two block rows from one set of loads.
// Warp roles (416 threads, one CTA per SM): warp 0 issues the TMA loads;
// warp 1 owns TMEM; one lane each of warps 1-3 and 12 issues the MMAs of
// every fourth group; warps 8-11 build A (every fourth group, two image rows
// at a time; the first group together); warps 4-7 read the accumulators (warp w reads TMEM lanes
// 32 (w % 4) ..) and finish the output rows.  Each ring slot is waited on by
// one role instance only (the slot counts are multiples of 4 and group g goes
// to instance g mod 4), so a parity wait can never match a phase two
// generations old.  Every wait is
// bounded in time; on a timeout the
// CTA stops issuing, drains its copies and MMAs, frees TMEM and reports
// IPF_ERR_TIMEOUT.
#include <cuda.h>

#include <cstring>
#include <functional>
#include <mutex>
#include <vector>

#include "ipf_internal.cuh"
#include "tc_common.cuh"

namespace ipf {

namespace {

constexpr int kThreads = 416;
constexpr int kBuilders = 4;         // builder warps: 8 .. 11
constexpr int kIssuers = 4;          // MMA-issuing warps: 1, 2, 3, 12
constexpr int kG = kConvTcGroup;     // image rows per MMA group
constexpr int kSegW = 160;           // elements per staged row segment
constexpr int kRB = 8;               // image rows per TMA box
constexpr int kNSeg = 4;             // boxes in flight
constexpr int kNHG = 8;              // A-operand groups in flight
constexpr int kNDG = 4;              // accumulator groups in flight
constexpr int kHankBytes = 2432;     // up to 19 blocks of 128 bytes
constexpr int kTmemCols = 512;
constexpr int kSegBytes = kRB * kSegW * 2;
constexpr int kBMax = 40960;         // B image bytes for KP = 32
constexpr int kOffB = 0;
constexpr int kOffSeg = kBMax;
constexpr int kOffHank = kOffSeg + kNSeg * kSegBytes;
constexpr int kOffBar = kOffHank + kNHG * kG * kHankBytes;
constexpr int kNBar = 2 * kNSeg + 2 * kNHG + 2 * kNDG + 1;
constexpr int kOffMisc = kOffBar + 8 * (kNBar + 1);       // + the B operand's barrier
constexpr int kSmemUsed = kOffMisc + 16;
constexpr int kSmemRequest = kSmemUsed + 1024;
static_assert(kRB == kG, "one staged box per group");
static_assert(kNHG % kIssuers == 0 && kNDG % kIssuers == 0 && kNHG % kBuilders == 0 && kNSeg % kBuilders == 0,
              "each ring slot belongs to one issuer and one builder");
static_assert(kSmemRequest > 116 * 1024 && kSmemRequest <= 227 * 1024, "one CTA per SM, within the SM");

// per KP: padded output rows per part, MMA N, K per group, B image bytes
template <int KP> struct TcShape {
    static constexpr int KW = KP - 1;
    static constexpr int NU = KW + kG - 1;              // output rows a group touches
    static constexpr int NP = (NU + 7) / 8 * 8;
    static constexpr int N = 2 * NP;                    // hi columns, then lo columns
    static constexpr int KG = kG * KP;
    static constexpr int BLBO = N * 16;                 // K-chunk stride of the B image
    static constexpr int BBYTES = KG * N * 2;
};
static_assert(TcShape<32>::BBYTES <= kBMax && TcShape<16>::BBYTES <= kBMax, "B image");

template <int NP>
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, uint32_t (&r)[NP]) {
    static_assert(NP == 40 || NP == 24, "column count");
    if constexpr (NP == 40) {
        tmem_ld32(taddr, r);
        tmem_ld8(taddr + 32, &r[32]);
    } else {
        tmem_ld16(taddr, r);
        tmem_ld8(taddr + 16, &r[16]);
    }
}

// one unit (128 output columns x R output rows: column tile unit % CT, row
// band unit / CT) of the convolution; vmap in parameter space
template <int KP>
__device__ __forceinline__ void conv_tc_body(const CUtensorMap* vmap, const int* __restrict__ jptr,
                                             float* __restrict__ w, int H, int W, int R, int CT,
                                             const uint4* __restrict__ bimg, int* __restrict__ err, int unit) {
    using S = TcShape<KP>;
    constexpr int KW = S::KW, NU = S::NU, NP = S::NP, N = S::N;
    constexpr int C = KW / 2;
    constexpr int NQ = 16 + KP / 8 - 1;        // A blocks per image row
    constexpr int OFF = 16 - C;                // segment index of v[iy, x0 - c]
    constexpr uint32_t IDESC = idesc_bf16(128, N);
    static_assert(KP == 16 || KP == 32, "KP");
    static_assert(OFF + 8 * (NQ - 1) + 7 + 7 < kSegW, "segment width");
    static_assert(NQ * 128 <= kHankBytes, "A operand size");
    static_assert(N % 16 == 0 && N <= 256 && kNDG * N <= kTmemCols, "MMA shape and TMEM columns");

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(sm);
    const uint32_t bar0 = sbase + kOffBar;
    auto seg_full = [&](int i) { return bar0 + 8u * i; };
    auto seg_empty = [&](int i) { return bar0 + 8u * (kNSeg + i); };
    auto h_full = [&](int i) { return bar0 + 8u * (2 * kNSeg + i); };
    auto h_empty = [&](int i) { return bar0 + 8u * (2 * kNSeg + kNHG + i); };
    auto d_full = [&](int i) { return bar0 + 8u * (2 * kNSeg + 2 * kNHG + i); };
    auto d_empty = [&](int i) { return bar0 + 8u * (2 * kNSeg + 2 * kNHG + kNDG + i); };
    const uint32_t done_bar = bar0 + 8u * (kNBar - 1);
    const uint32_t b_bar = bar0 + 8u * kNBar;               // the B operand has landed
    uint32_t* s_tmem = (uint32_t*)(sm + kOffMisc);
    volatile int* s_abort = (volatile int*)(sm + kOffMisc + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ct = unit % CT, sg = unit / CT;
    const int x0 = ct * 128, Y0 = sg * R;
    if (Y0 >= H) return;                                  // uniform for the CTA
    const int yEnd = min(Y0 + R, H);
    const int NR = (yEnd - Y0) + 2 * C;                   // image rows Y0 - c .. yEnd - 1 + c
    const int Ys = Y0 - C;
    const int NG = (NR + kG - 1) / kG;                    // row groups (one TMA box each)

    if (threadIdx.x == 0) {
        // seg_empty: one arrival per row of the box, once its builder warp has used it
        for (int i = 0; i < kNSeg; ++i) { mbar_init(seg_full(i), 1); mbar_init(seg_empty(i), kRB); }
        for (int i = 0; i < kNHG; ++i) { mbar_init(h_full(i), 32); mbar_init(h_empty(i), 1); }
        for (int i = 0; i < kNDG; ++i) { mbar_init(d_full(i), 1); mbar_init(d_empty(i), 128); }
        mbar_init(done_bar, kIssuers);
        mbar_init(b_bar, 1);
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        // the B operand by one bulk copy, landing while the first row boxes
        // are staged and built (the issuers wait for it before their first MMA)
        mbar_expect_tx(b_bar, (uint32_t)S::BBYTES);
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                sbase + (uint32_t)kOffB),
            "l"(bimg), "r"((uint32_t)S::BBYTES), "r"(b_bar)
            : "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(s_tmem)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;

    if (warp == 0) {
        // ---- TMA producer: one box of kRB = kG rows per group ----
        if (lane == 0) {
            const int z = jptr ? *jptr : 0;
            int issued = 0;
            for (int t = 0; t < NG; ++t) {
                const int sl = t % kNSeg;
                if (!mbar_wait(seg_empty(sl), ((t / kNSeg) & 1) ^ 1, s_abort, err)) break;
                mbar_expect_tx(seg_full(sl), kSegBytes);
                tma_load_3d(sbase + kOffSeg + sl * kSegBytes, vmap, x0 - 16, Ys + t * kRB, z, seg_full(sl));
                issued = t + 1;
            }
            // every issued copy lands before the CTA may exit
            for (int t = issued > kNSeg ? issued - kNSeg : 0; t < issued; ++t)
                mbar_wait(seg_full(t % kNSeg), (t / kNSeg) & 1, s_abort, err, false);
            mbar_wait(b_bar, 0, s_abort, err, false);
        }
    } else if (warp <= 3 || warp == 12) {
        // ---- MMA issuers: groups g = issuer (mod kIssuers) ----
        if (lane == 0) {
            const int issuer = warp == 12 ? 3 : warp - 1;
            const bool b_ok = mbar_wait(b_bar, 0, s_abort, err);
            for (int g = issuer; b_ok && g < NG; g += kIssuers) {
                const int hg = g % kNHG, dg = g % kNDG;
                if (!mbar_wait(h_full(hg), (g / kNHG) & 1, s_abort, err)) break;
                if (!mbar_wait(d_empty(dg), ((g / kNDG) & 1) ^ 1, s_abort, err)) break;
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(dg * N);
                const int rows = min(kG, NR - g * kG);
#pragma unroll
                for (int r = 0; r < kG; ++r) {
                    if (r < rows) {
                        const uint32_t a0 = sbase + kOffHank + (hg * kG + r) * kHankBytes;
#pragma unroll
                        for (int kk = 0; kk < KP / 16; ++kk) {
                            const int c16 = r * (KP / 16) + kk;           // 16-wide K slice of the group
                            mma_bf16(d, smem_desc(a0 + kk * 256, 128, 128),
                                     smem_desc(sbase + kOffB + c16 * 2 * S::BLBO, S::BLBO, 128), IDESC,
                                     c16 > 0 ? 1u : 0u);
                        }
                    }
                }
                mma_commit(d_full(dg));
                mma_commit(h_empty(hg));
            }
            // all MMAs issued by this thread complete before TMEM is freed
            mma_commit(done_bar);
            mbar_wait(done_bar, 0, s_abort, err, false);
        }
    } else if (warp >= 8 && warp < 12) {
        // ---- A builders: Hankel blocks from the staged box, one group per warp
        // (every fourth group), two image rows per pass; the first group is
        // built by all four warps, two rows each, so the first MMAs start
        // a quarter of a group's build time after the first box lands ----
        // two image rows r0, r0 + 1 of the box in slot sl into A slot hg; a
        // lane takes the core-matrix rows s = 2t and 2t + 1 of block q of one
        // of them: both 16-byte rows lie in the five source words from
        // (OFF + 8q + 2t) / 2 on, so the loads per stored byte are half those
        // of one row per lane (the staged segment's reads and the block
        // stores are the shared-memory traffic the convolution is bound by)
        auto build_pair = [&](int sl, int hg, int rows, int r0) {
            constexpr int JOBS = NQ * 4;                        // (q, t) per image row
            constexpr int NIT = (2 * JOBS + 31) / 32;
            uint32_t wv[NIT][5];
#pragma unroll
            for (int it = 0; it < NIT; ++it) {
                const int jb = it * 32 + lane;
                const int p = jb >= JOBS ? 1 : 0, rem = jb - p * JOBS;
                const int r = min(r0 + p, rows - 1);
                const uint32_t* src = (const uint32_t*)(sm + kOffSeg + sl * kSegBytes + r * kSegW * 2);
                const int e0 = OFF + 8 * (rem >> 2) + 2 * (rem & 3);
                const int wb = jb < 2 * JOBS ? (e0 >> 1) : 0;
#pragma unroll
                for (int k = 0; k < 5; ++k) wv[it][k] = src[wb + k];
            }
#pragma unroll
            for (int it = 0; it < NIT; ++it) {
                const int jb = it * 32 + lane;
                const int p = jb >= JOBS ? 1 : 0, rem = jb - p * JOBS;
                if (jb < 2 * JOBS && r0 + p < rows) {
                    unsigned char* dst = sm + kOffHank + (hg * kG + r0 + p) * kHankBytes;
                    const int q = rem >> 2, t = rem & 3;
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        // e = OFF + 8q + 2t + u has the parity of OFF + u: d
                        // words into wv, and a two-byte shift when e is odd
                        constexpr bool kOdd = (OFF & 1) != 0;
                        const int d = (kOdd && u == 1) ? 1 : 0;
                        const uint32_t sel = ((OFF + u) & 1) ? 0x5432u : 0x3210u;
                        const uint32_t w4 = d == 0 ? wv[it][4] : 0u;      // unused (aligned) when d = 1
                        uint4 o;
                        o.x = __byte_perm(wv[it][d], wv[it][d + 1], sel);
                        o.y = __byte_perm(wv[it][d + 1], wv[it][d + 2], sel);
                        o.z = __byte_perm(wv[it][d + 2], wv[it][d + 3], sel);
                        o.w = __byte_perm(wv[it][d + 3], w4, sel);
                        *(uint4*)(dst + q * 128 + (2 * t + u) * 16) = o;
                    }
                }
            }
            // every word read from the two staged rows has been consumed by a
            // store: they may be overwritten by the next box
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(seg_empty(sl));
                if (r0 + 1 < rows) mbar_arrive(seg_empty(sl));
            }
        };
        {
            // group 0 (box slot 0, A slot 0, both in their first phase)
            const int rows = min(kG, NR);
            const int r0 = 2 * (warp - 8);
            const bool ok = mbar_wait(seg_full(0), 0, s_abort, err) && mbar_wait(h_empty(0), 1, s_abort, err);
            if (ok && r0 < rows) build_pair(0, 0, rows, r0);
            fence_proxy_async_smem();
            asm volatile("bar.sync 1, 128;" ::: "memory");      // the four builder warps
            if (warp == 8 && !*s_abort) mbar_arrive(h_full(0));
        }
        for (int g = warp - 8 == 0 ? kBuilders : warp - 8; g < NG; g += kBuilders) {
            const int sl = g % kNSeg, hg = g % kNHG;
            if (!mbar_wait(seg_full(sl), (g / kNSeg) & 1, s_abort, err)) break;
            if (!mbar_wait(h_empty(hg), ((g / kNHG) & 1) ^ 1, s_abort, err)) break;
            const int rows = min(kG, NR - g * kG);
            for (int r0 = 0; r0 < rows; r0 += 2) build_pair(sl, hg, rows, r0);
            fence_proxy_async_smem();
            mbar_arrive(h_full(hg));
        }
    } else {
        // ---- epilogue ----
        // Before group g (image rows iy0 = Ys + g G ..), acc[t] holds output
        // row iy0 - c + t summed over the image rows above iy0 (t < KW - 1).
        // With the group's columns, total[t] = acc[t] + D[G + KW - 2 - t]
        // (hi + lo), t < NU; rows t < G are complete, the rest shift down by G.
        const int q = warp & 3;
        const int x = x0 + q * 32 + lane;
        const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16);
        float acc[KW - 1];
#pragma unroll
        for (int t = 0; t < KW - 1; ++t) acc[t] = 0.f;
        for (int g = 0; g < NG; ++g) {
            const int dg = g % kNDG;
            if (!__all_sync(0xffffffffu, mbar_wait(d_full(dg), (g / kNDG) & 1, s_abort, err))) break;
            tc_fence_after();
            uint32_t hi[NP], lo[NP];
            tmem_ld_cols<NP>(tl + (uint32_t)(dg * N), hi);
            tmem_ld_cols<NP>(tl + (uint32_t)(dg * N + NP), lo);
            tmem_wait_ld();
            tc_fence_before();
            mbar_arrive(d_empty(dg));
            float total[NU];
#pragma unroll
            for (int t = 0; t < NU; ++t) {
                const int j = kG + KW - 2 - t;
                const float d = __uint_as_float(hi[j]) + __uint_as_float(lo[j]);
                total[t] = t < KW - 1 ? acc[t] + d : d;
            }
#pragma unroll
            for (int t = 0; t < kG; ++t) {
                const int i = g * kG + t;                         // completing image row
                const int y = Y0 + i - 2 * C;
                if (i < NR && i >= 2 * C && y < yEnd && x < W) w[(size_t)y * W + x] = total[t];
            }
#pragma unroll
            for (int t = 0; t < KW - 1; ++t) acc[t] = total[t + kG];
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

template <int KP>
__global__ void __launch_bounds__(kThreads, 1)
    k_conv2d_tc(const __grid_constant__ CUtensorMap vmap, const int* __restrict__ jptr, float* __restrict__ w,
                int H, int W, int R, int CT, const uint4* __restrict__ bimg, int* __restrict__ err) {
    conv_tc_body<KP>(&vmap, jptr, w, H, W, R, CT, bimg, err, blockIdx.x);
}

// the batched step: one unit of one slot per CTA; every slot's tensor map
// travels in the parameter struct
struct TcMaps {
    CUtensorMap m[kMaxSlots];
};

template <int KP>
__global__ void __launch_bounds__(kThreads, 1)
    kb_conv_tc(const __grid_constant__ TcMaps maps, const SlotDesc* __restrict__ slots,
               const TileRef* __restrict__ units, int nunits) {
    __shared__ int s_j;
    if ((int)blockIdx.x >= nunits) return;
    const TileRef tr = units[blockIdx.x];
    const SlotDesc* sd = slots + tr.slot;
    if (slot_step(sd, &s_j) < 0) return;                 // uniform for the CTA
    DevState* st = sd->bf.st;
    conv_tc_body<KP>(&maps.m[tr.slot], &st->j, (float*)sd->bf.w, sd->op.rows, sd->op.cols, sd->tc_rows, sd->tc_ct,
                     (const uint4*)sd->op.psf_tc, &st->status[0], tr.tile);
}


template <int KP>
cudaError_t launch_kp(const CUtensorMap& map, const int* jptr, float* w, int H, int W, const void* bimg, int* err,
                      cudaStream_t s) {
    cudaError_t e = raise_smem(k_conv2d_tc<KP>, kSmemRequest);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 1;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int CT = (W + 127) / 128;
    int S = sms / CT;
    const int smax = (H + 31) / 32;                       // at least 32 output rows per CTA
    if (S > smax) S = smax;
    if (S < 1) S = 1;
    const int R = (H + S - 1) / S;
    const int units = CT * ((H + R - 1) / R);
    k_conv2d_tc<KP><<<units, kThreads, kSmemRequest, s>>>(map, jptr, w, H, W, R, CT, (const uint4*)bimg, err);
    return cudaGetLastError();
}

template <int KP>
void build_operand(const std::function<float(int, int)>& F, std::vector<unsigned short>* img) {
    using S = TcShape<KP>;
    img->assign(S::BBYTES / 2, 0);
    for (int n = 0; n < S::N; ++n) {
        const bool lo = n >= S::NP;
        const int j = lo ? n - S::NP : n;
        for (int k = 0; k < S::KG; ++k) {
            const int r = k / KP, b = k % KP;
            const int a = r + j + 1 - kG;
            float f = 0.f;
            if (j < S::NU && a >= 0 && a < S::KW && b < S::KW) f = F(a, b);
            const unsigned short h = bf16_bits_rn(f);
            const unsigned short v = lo ? bf16_bits_rn(f - bf16_bits_to_float(h)) : h;
            (*img)[(size_t)(k / 8) * S::N * 8 + (size_t)n * 8 + (k % 8)] = v;
        }
    }
}

}  // namespace

unsigned short bf16_bits_rn(float f) {
    unsigned u;
    memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (unsigned short)(u >> 16);
}

float bf16_bits_to_float(unsigned short h) {
    const unsigned u = (unsigned)h << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

int conv_tc_operand(int kw, const std::function<float(int, int)>& F, std::vector<unsigned short>* img) {
    if (kw == 31) { build_operand<32>(F, img); return 32; }
    if (kw == 15) { build_operand<16>(F, img); return 16; }
    return 0;
}

bool conv_tc_eligible(const OpDev& op, const void* vbase, long long ldv) {
    if (op.kind != IPF_OP_PSF2D || !op.psf_tc || op.conv_fma) return false;
    if (op.cols % 8 != 0 || ((uintptr_t)vbase & 15u) != 0 || (ldv * 2) % 16 != 0) return false;
    return encode_fn() != nullptr;
}

cudaError_t launch_conv_tc(const OpDev& op, const void* vbase, long long ldv, long long vcols, const int* jptr,
                           float* w, int* err, cudaStream_t s) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const int H = op.rows, W = op.cols;
    const long long colstride = ldv > 0 ? ldv : (long long)H * W;
    CUtensorMap map;
    const cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)(vcols > 0 ? vcols : 1)};
    const cuuint64_t strides[2] = {(cuuint64_t)W * 2, (cuuint64_t)colstride * 2};
    const cuuint32_t box[3] = {(cuuint32_t)kSegW, (cuuint32_t)kRB, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(vbase), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    if (op.tc_kp == 32) return launch_kp<32>(map, jptr, w, H, W, op.psf_tc, err, s);
    if (op.tc_kp == 16) return launch_kp<16>(map, jptr, w, H, W, op.psf_tc, err, s);
    return cudaErrorInvalidValue;
}

bool conv_tc_map(const OpDev& op, const void* vbase, long long ldv, long long vcols, void* map_out) {
    EncodeTiledFn enc = encode_fn();
    if (!enc || !conv_tc_eligible(op, vbase, ldv)) return false;
    const int H = op.rows, W = op.cols;
    const cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)(vcols > 0 ? vcols : 1)};
    const cuuint64_t strides[2] = {(cuuint64_t)W * 2, (cuuint64_t)ldv * 2};
    const cuuint32_t box[3] = {(cuuint32_t)kSegW, (cuuint32_t)kRB, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc((CUtensorMap*)map_out, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(vbase), dims, strides,
               box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t conv_tc_map_bytes() { return sizeof(CUtensorMap); }

cudaError_t launch_batch_conv_tc(int kp, const void* maps, const SlotDesc* slots, const TileRef* units, int nunits,
                                 cudaStream_t s) {
    if (nunits <= 0) return cudaSuccess;
    const TcMaps& m = *(const TcMaps*)maps;
    if (kp == 32) {
        cudaError_t e = raise_smem(kb_conv_tc<32>, kSmemRequest);
        if (e != cudaSuccess) return e;
        kb_conv_tc<32><<<nunits, kThreads, kSmemRequest, s>>>(m, slots, units, nunits);
    } else if (kp == 16) {
        cudaError_t e = raise_smem(kb_conv_tc<16>, kSmemRequest);
        if (e != cudaSuccess) return e;
        kb_conv_tc<16><<<nunits, kThreads, kSmemRequest, s>>>(m, slots, units, nunits);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace ipf
