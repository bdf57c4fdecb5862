// The Gaussian sketch (Sec. 2; the embedding of the paper's experiments):
// S (m_s x n) with N(0, 1/m_s) entries, drawn once per context from the
// SplitMix64 counter hash by the Box-Muller transform (Box & Muller 1958):
// entry (r, i) takes outputs 2c and 2c+1, c = r*n + i, of the generator
// started at the seed; u = ((out >> 11) + 1) * 2^-53 in (0, 1];
// z = sqrt(-2 ln u1) cos(2 pi u2); S[r, i] = z / sqrt(m_s), rounded to the
// storage type of the basis.  A context keeps S K-major (row-major for
// FP32 / FP64, entry (r, i) at r*lds + i; for BF16 / FP16 in units of 16
// rows x 64 elements, see k_gauss_fill_tiled), so S and the basis V (column
// j at j*ldv) are both K-major operands of the one contraction the method
// needs at solve time:
//
//     [S V_{k+1} | S b] = S [V_{k+1} | b]      (m_s x (k+2), K = n).
//
// For BF16 / FP16 storage it runs on the tensor cores (k_gauss_mma, tcgen05
// with TMEM accumulators, operands staged by TMA): b enters as three extra
// B rows b0 + b1 + b2 = b (each the storage-type rounding of what is left,
// so the split is exact for FP32 b), so c = S b costs no pass of its own.
// The n-long contraction is split into slices; each CTA sums one slice in
// FP32 in TMEM and writes its partial tile, and k_gauss_reduce adds the
// slices in FP64 in a fixed order (so the result does not depend on
// scheduling).  FP32 / FP64 storage use a CUDA-core kernel of the same
// structure (k_gauss_simt; FP32 / FP64 accumulation).
#include <atomic>
#include <cstdio>
#include <type_traits>

#include "tc_common.cuh"

namespace ipf {

namespace {

// One entry in FP64, the definition itself: v = z / sqrt(m).
__device__ __forceinline__ double gauss_f64(unsigned long long o1, unsigned long long o2, double sqrt_m) {
    const double u1 = ((double)(o1 >> 11) + 1.0) * 0x1.0p-53;
    const double u2 = ((double)(o2 >> 11) + 1.0) * 0x1.0p-53;
    const double z = sqrt(-2.0 * log(u1)) * cos(2.0 * 3.141592653589793 * u2);
    return z / sqrt_m;
}

// The same entry rounded to a 16-bit storage type, evaluated in FP32 with an
// error bound; when the bound's interval does not round to one value of the
// storage type the entry is recomputed in FP64, so the stored S equals the
// FP64 definition rounded to storage.
//  * ln u1: logf of u1 for u1 <= 1/2 (|ln u1| >= ln 2), else log1pf(-eps)
//    with eps = 1 - u1 formed exactly from the integer (2^53 - 1 - k1);
//    relative error <= 2.4e-7 (argument rounding 2^-24, 1 ulp of logf /
//    log1pf).
//  * cos(2 pi u2) = cos(pi t 2^-52), t = k2 + 1, reduced with integers:
//    cos(pi x) = -cos(pi (x - 1)), cos(pi y) = -cos(pi (1 - y)) for y > 1/2,
//    and cos(pi w) = sin(pi (1/2 - w)) for w > 1/4, so cospif or sinpif gets
//    an argument in [0, 1/4]; relative error <= 1.8e-7.
//  * R = sqrtf(-2 ln u1) (correctly rounded), v = R C / sqrt(m): relative
//    error <= 5.4e-7 in all; the interval used is twice that, plus an
//    absolute 2e-15 R / sqrt(m) for the FP64 definition's own rounding of
//    2 pi u2 (which matters only where C is near zero).
template <class T> __device__ __forceinline__ unsigned short store_bits(float v);
template <> __device__ __forceinline__ unsigned short store_bits<__nv_bfloat16>(float v) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}
template <> __device__ __forceinline__ unsigned short store_bits<__half>(float v) {
    return __half_as_ushort(__float2half_rn(v));
}

template <class T>
__device__ __forceinline__ bool gauss_fast(unsigned long long o1, unsigned long long o2, float inv_sqrt_m,
                                           unsigned short& bits) {
    const unsigned long long k1 = o1 >> 11, k2 = o2 >> 11;
    float L;
    if (k1 + 1ull <= (1ull << 52)) {
        L = logf(__ull2float_rn(k1 + 1ull) * 0x1.0p-53f);
    } else {
        const unsigned long long e = (1ull << 53) - 1ull - k1;
        if (e == 0ull) return false;                                 // u1 = 1
        L = log1pf(-(__ull2float_rn(e) * 0x1.0p-53f));
    }
    const float R = sqrtf(-2.f * L);
    const long long sft = (long long)(k2 + 1ull) - (1ll << 52);
    unsigned long long a = (unsigned long long)(sft < 0 ? -sft : sft);
    float sign = -1.f;
    if (a > (1ull << 51)) {
        a = (1ull << 52) - a;
        sign = -sign;
    }
    const float C = a <= (1ull << 50) ? cospif(__ull2float_rn(a) * 0x1.0p-52f)
                                      : sinpif(__ull2float_rn((1ull << 51) - a) * 0x1.0p-52f);
    const float v = __fmul_rn(__fmul_rn(R, sign * C), inv_sqrt_m);
    const float E = __fmaf_ru(1.2e-6f, fabsf(v), __fmul_ru(__fmul_ru(2e-15f, R), inv_sqrt_m));
    const unsigned short lo = store_bits<T>(__fsub_rd(v, E)), hi = store_bits<T>(__fadd_ru(v, E));
    if (lo != hi) return false;
    bits = lo;
    return true;
}

// entry with counter c = r*n + i in the storage type (16-bit types as bits)
template <class T>
__device__ __forceinline__ unsigned short gauss_bits16(unsigned long long c, unsigned long long seed, double sqrt_m,
                                                       float inv_sqrt_m) {
    const unsigned long long o1 = sm64_mix(seed + kGamma * (2ull * c + 1ull));
    const unsigned long long o2 = sm64_mix(seed + kGamma * (2ull * c + 2ull));
    unsigned short bits;
    if (!gauss_fast<T>(o1, o2, inv_sqrt_m, bits)) {
        const double v = gauss_f64(o1, o2, sqrt_m);
        if constexpr (std::is_same<T, __half>::value) bits = __half_as_ushort(__double2half(v));
        else bits = store_bits<T>((float)v);                 // FP64 -> FP32 -> BF16
    }
    return bits;
}

// The tiled layout of S for the tensor-core contraction (16-bit storage):
// units of 16 rows x 64 elements (2 KB, row-major inside), unit (rt, kb) =
// rows 16 rt .., elements 64 kb .. at offset (rt * nkb + kb) * 1024 elements,
// nkb = ceil(n / 64).  A stage of the contraction then reads whole 2 KB
// pieces of DRAM instead of 128 bytes of each of 128 rows 2n bytes apart.
// Entries outside m x n are zero (the basis is zero-filled there, and
// 0 x 0 must stay 0).
template <class T>
__global__ void __launch_bounds__(256) k_gauss_fill_tiled(T* __restrict__ S, long long n, int m, unsigned nkb,
                                                          unsigned long long total, unsigned long long seed,
                                                          double sqrt_m, float inv_sqrt_m) {
    unsigned short* S16 = reinterpret_cast<unsigned short*>(S);
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < total; t += stride) {
        const unsigned u = (unsigned)(t >> 10), w = (unsigned)(t & 1023u);
        const unsigned rt = u / nkb, kb = u - rt * nkb;
        const long long r = 16ll * rt + (w >> 6), i = 64ll * kb + (w & 63u);
        S16[t] = (r < m && i < n) ? gauss_bits16<T>((unsigned long long)(r * n + i), seed, sqrt_m, inv_sqrt_m)
                                  : (unsigned short)0;
    }
}

// entry c = r*n + i (the counter) goes to S[r*lds + i]; the walk carries
// (r, i) instead of a 64-bit division per entry
template <class T>
__global__ void __launch_bounds__(256) k_gauss_fill(T* __restrict__ S, long long n, int m, long long lds,
                                                    unsigned long long seed, double sqrt_m, float inv_sqrt_m) {
    const long long total = n * (long long)m;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long si = stride % n, sr = stride / n;
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long r = c / n, i = c - r * n;
    for (; c < total; c += stride) {
        const long long t = r * lds + i;
        if constexpr (sizeof(T) == 2) {
            reinterpret_cast<unsigned short*>(S)[t] = gauss_bits16<T>((unsigned long long)c, seed, sqrt_m, inv_sqrt_m);
        } else {
            const unsigned long long o1 = sm64_mix(seed + kGamma * (2ull * (unsigned long long)c + 1ull));
            const unsigned long long o2 = sm64_mix(seed + kGamma * (2ull * (unsigned long long)c + 2ull));
            S[t] = (T)gauss_f64(o1, o2, sqrt_m);
        }
        i += si;
        r += sr;
        if (i >= n) {
            i -= n;
            r += 1;
        }
    }
}

// b (FP32) as the extra B rows: for 16-bit storage three parts, part p the
// storage-type rounding of b - (parts before it), whose sum is b exactly for
// normal values (8 + 8 + 8 significant bits for BF16, 11 x 3 for FP16); for
// FP32 / FP64 storage b itself.  parts: [8][ldb], rows 3..7 stay zero.
template <class T>
__global__ void k_gauss_bparts(const float* __restrict__ b, long long n, long long ldb, T* __restrict__ parts) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float v = b[i];
        if constexpr (sizeof(T) == 2) {
            const T p0 = from_acc<T>(v);
            const float r1 = v - to_acc(p0);
            const T p1 = from_acc<T>(r1);
            const float r2 = r1 - to_acc(p1);
            parts[i] = p0;
            parts[ldb + i] = p1;
            parts[2 * ldb + i] = from_acc<T>(r2);
        } else {
            parts[i] = (T)v;
        }
    }
}

// ---------------------------------------------------------------------------
// tensor-core contraction.  CTA (slice s, row group q) sums K = i in
// [s*chunk, min(n, (s+1)*chunk)) for the rows rg q .. rg q + rg - 1 of S (rg
// = the rows per group, a multiple of 16 up to 256, the same for every
// group but the last, so that the CTAs carry equal shares of S: one or two
// M = 128 tiles, a tile of R < 128 rows loaded as boxes of 64, 32 and 16
// rows, its other TMEM lanes unused) against all N = Ntot rows of B = [V_0 .. V_{Nv-1};
// b0, b1, b2, 0 x 5] (Nv >= k + 1, Ntot = Nv + 8, a multiple of 16).  Per
// stage of 64 K elements (one 128-byte swizzle row): TMA brings the A tiles
// (128 rows x 128 bytes each) and B (Ntot rows) into shared memory with the
// 128-byte swizzle, zero-filled outside S, V and b; the MMA thread issues
// 4 x ntile tcgen05.mma (M 128, N Ntot, K 16) into TMEM (ntile x Ntot FP32
// columns) and commits to the stage's empty barrier.  Roles (192 threads,
// one CTA per SM): warp 0 TMA, warp 1 TMEM owner and MMA issuer, warps 2-5
// epilogue (warp w reads TMEM lanes 32 (w % 4) ..).  Every wait is bounded
// (2 s); on a timeout the CTA stops issuing, drains its copies and MMAs,
// frees TMEM, writes nothing and records IPF_ERR_TIMEOUT.
// ---------------------------------------------------------------------------
constexpr int kGmThreads = 192;
constexpr int kGmBRowsMax = 256;
constexpr int kGmBRows = 8;          // rows of the b block: 3 parts + 5 zero rows
constexpr int kGmChunkAlign = 64;    // slices start at multiples of 64 elements

// the two pipelines: BK K elements per stage (one swizzle row of 2 BK
// bytes), the stage slots fixed for the largest B
template <int BK> struct GmShape {
    static_assert(BK == 64 || BK == 32, "stage width");
    static constexpr int kRowBytes = 2 * BK;                    // 128 or 64: the swizzle span
    static constexpr int kStages = BK == 64 ? 3 : 7;
    static constexpr int kATile = 128 * kRowBytes;
    static constexpr int kStageBytes = 2 * kATile + kGmBRowsMax * kRowBytes;
    static constexpr int kOffBar = kStages * kStageBytes;
    static constexpr int kNBar = 2 * kStages + 1;
    static constexpr int kOffMisc = kOffBar + 8 * kNBar;
    static constexpr int kSmemRequest = kOffMisc + 16 + 1024;
    static_assert(kSmemRequest <= 227 * 1024, "shared memory per CTA");
    static_assert(kStageBytes % 1024 == 0 && kATile % 1024 == 0, "swizzle atoms stay aligned");
};

// shared-memory descriptor of a K-major tile in the stage's swizzle
template <int BK> __device__ __forceinline__ unsigned long long gm_desc(uint32_t addr);
template <> __device__ __forceinline__ unsigned long long gm_desc<64>(uint32_t addr) { return smem_desc_sw128(addr); }
template <> __device__ __forceinline__ unsigned long long gm_desc<32>(uint32_t addr) { return smem_desc_sw64(addr); }

// The tensor maps: S through four box heights (128, 64, 32, 16 rows); V
// through one box of all Nv rows (one CTA per row group), or, when the row
// groups of a slice form a cluster, five box heights (128 .. 8 rows) from
// which each CTA composes its share of V's rows, multicast to the cluster;
// b (8 rows)
struct GmMaps {
    CUtensorMap s[4];
    CUtensorMap v[5];
    CUtensorMap vall;
    CUtensorMap b;
};

template <bool BF16, int BK>
__global__ void __launch_bounds__(kGmThreads, 1)
    k_gauss_mma(const __grid_constant__ GmMaps maps, long long n, int m, long long chunk, int mg, int rg, int Nv,
                int Ntot, int clustered, float* __restrict__ part, int m_pad, int* __restrict__ err) {
    using G = GmShape<BK>;
    constexpr int kGmBK = BK;
    constexpr int kGmStages = G::kStages;
    constexpr int kGmATile = G::kATile;
    constexpr int kGmStageBytes = G::kStageBytes;
    constexpr int kGmOffBar = G::kOffBar;
    constexpr int kGmOffMisc = G::kOffMisc;
    constexpr int kRow = G::kRowBytes;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(sm);
    const uint32_t bar0 = sbase + kGmOffBar;
    auto full = [&](int i) { return bar0 + 8u * i; };
    auto empty = [&](int i) { return bar0 + 8u * (kGmStages + i); };
    const uint32_t done = bar0 + 8u * (2 * kGmStages);
    uint32_t* s_tmem = (uint32_t*)(sm + kGmOffMisc);
    volatile int* s_abort = (volatile int*)(sm + kGmOffMisc + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int slice = blockIdx.x / mg, q = blockIdx.x % mg;     // q = the cluster rank when clustered
    // clustered: this CTA loads V's 8-row units [u0, u1) for every CTA of the
    // cluster, and a stage slot is free again once all mg CTAs have consumed it
    const uint16_t cmask = (uint16_t)((1u << mg) - 1u);
    const int vu0 = q * (Nv / 8) / mg, vu1 = (q + 1) * (Nv / 8) / mg;
    const int row0 = q * rg;
    const int rows_q = min(rg, m - row0);                      // >= 1: q < mg, (mg - 1) rg < m
    const int ntile = (rows_q + 127) / 128;                    // 1 or 2
    // rows of each tile, rounded up to 16 (beyond m: TMA zero fill)
    const int R0 = min(128, (rows_q + 15) / 16 * 16);
    const int R1 = ntile > 1 ? (rows_q - 128 + 15) / 16 * 16 : 0;
    const long long i0 = (long long)slice * chunk;
    const long long i1 = min(n, i0 + chunk);
    const int nkb = (int)((i1 - i0 + kGmBK - 1) / kGmBK);      // >= 1: slices = ceil(n / chunk)

    if (threadIdx.x == 0) {
        for (int i = 0; i < kGmStages; ++i) { mbar_init(full(i), 1); mbar_init(empty(i), clustered ? mg : 1); }
        mbar_init(done, 1);
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(s_tmem)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncwarp();
    // clustered: every CTA's barriers exist before any copy or commit of
    // another CTA of the cluster can reach them
    if (clustered) cluster_sync();
    else __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;

    if (warp == 0) {
        if (lane == 0) {
            const uint32_t bytes = (uint32_t)((R0 + R1 + Ntot) * kRow);
            // S is read once: evict-first, so it does not push out the basis
            // tile the other row groups of the slice read from L2 after us
            const unsigned long long pol_s = l2_evict_first(), pol_v = l2_evict_last();
            int issued = 0;
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb % kGmStages;
                if (!mbar_wait(empty(s), ((kb / kGmStages) & 1) ^ 1, s_abort, err)) break;
                mbar_expect_tx(full(s), bytes);
                const int x = (int)(i0 + (long long)kb * kGmBK);
                const uint32_t st = sbase + (uint32_t)(s * kGmStageBytes);
                for (int t = 0; t < ntile; ++t) {
                    // Rt = 128, or the sum of the boxes 64, 32, 16 its bits select;
                    // each box lands at a multiple of 16 rows (1024-byte aligned)
                    // S is tiled (units of 16 rows x 64 elements): element x is
                    // (x mod 64) of unit column x / 64, row y of unit row y / 16
                    const int y0 = row0 + 128 * t;
                    const int Rt = t ? R1 : R0;
                    const int xu = x & 63, zu = x >> 6;
                    if (Rt == 128) {
                        tma_load_4d_hint(st + t * kGmATile, &maps.s[0], xu, 0, zu, y0 >> 4, full(s), pol_s);
                    } else {
                        int dn = 0;
#pragma unroll
                        for (int b = 1; b < 4; ++b) {
                            const int h = 128 >> b;
                            if (Rt & h) {
                                tma_load_4d_hint(st + t * kGmATile + dn * kRow, &maps.s[b], xu, 0, zu,
                                                 (y0 + dn) >> 4, full(s), pol_s);
                                dn += h;
                            }
                        }
                    }
                }
                const uint32_t vst = st + 2 * kGmATile;
                if (clustered) {
                    // this CTA's rows of V (a multiple of 8, as boxes of 128 .. 8
                    // rows at multiples of 8 rows: 1024-byte aligned), to every
                    // CTA of the cluster; the full barrier of each receives them
                    // (at most 128 rows: the launcher clusters only Nv <= 128 mg)
                    int r = 8 * vu0;
                    const int R = 8 * (vu1 - vu0);
                    if (R == 128) {
                        tma_load_2d_mc(vst + r * kRow, &maps.v[0], x, r, full(s), cmask, pol_v);
                    } else {
#pragma unroll
                        for (int b = 1; b < 5; ++b) {
                            const int h = 128 >> b;
                            if (R & h) {
                                tma_load_2d_mc(vst + r * kRow, &maps.v[b], x, r, full(s), cmask, pol_v);
                                r += h;
                            }
                        }
                    }
                } else {
                    tma_load_2d_hint(vst, &maps.vall, x, 0, full(s), pol_v);
                }
                tma_load_2d(vst + Nv * kRow, &maps.b, x, 0, full(s));
                issued = kb + 1;
            }
            // every issued copy lands before the CTA may exit
            for (int kb = issued > kGmStages ? issued - kGmStages : 0; kb < issued; ++kb)
                mbar_wait(full(kb % kGmStages), (kb / kGmStages) & 1, s_abort, err, false);
            // clustered: the other CTAs' last arrivals on this CTA's empty
            // barriers (their MMAs on the last stages) have come in
            if (clustered)
                for (int kb = nkb > kGmStages ? nkb - kGmStages : 0; kb < nkb; ++kb)
                    mbar_wait(empty(kb % kGmStages), (kb / kGmStages) & 1, s_abort, err, false);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_f16kind(128, Ntot, BF16);
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb % kGmStages;
                if (!mbar_wait(full(s), (kb / kGmStages) & 1, s_abort, err)) break;
                tc_fence_after();
                const uint32_t st = sbase + (uint32_t)(s * kGmStageBytes);
                for (int t = 0; t < ntile; ++t) {
#pragma unroll
                    for (int kk = 0; kk < kGmBK / 16; ++kk)
                        mma_bf16(tmem + (uint32_t)(t * Ntot), gm_desc<BK>(st + t * kGmATile + kk * 32),
                                 gm_desc<BK>(st + 2 * kGmATile + kk * 32), idesc, (kb > 0 || kk > 0) ? 1u : 0u);
                }
                if (clustered) mma_commit_mc(empty(s), cmask);
                else mma_commit(empty(s));
            }
            // arrives once every MMA issued above has completed
            mma_commit(done);
        }
    } else {
        // ---- epilogue: this slice's partial tile, FP32, to part[slice][row][col] ----
        const bool ok = mbar_wait(done, 0, s_abort, err, false);
        tc_fence_after();
        const int qw = warp & 3;
        const bool write = ok && !*s_abort;
        for (int t = 0; t < ntile; ++t) {
            const int rl = 32 * qw + lane;
            const int r = row0 + 128 * t + rl;
            float* dst = part + ((size_t)slice * m_pad + r) * Ntot;
            for (int c0 = 0; c0 < Ntot; c0 += 16) {
                uint32_t v[16];
                tmem_ld16(tmem + ((uint32_t)(32 * qw) << 16) + (uint32_t)(t * Ntot + c0), v);
                tmem_wait_ld();
                if (write && 128 * t + rl < rows_q) {          // this group's rows only (all < m)
#pragma unroll
                    for (int e = 0; e < 16; e += 4)
                        *reinterpret_cast<float4*>(dst + c0 + e) =
                            make_float4(__uint_as_float(v[e]), __uint_as_float(v[e + 1]), __uint_as_float(v[e + 2]),
                                        __uint_as_float(v[e + 3]));
                }
            }
        }
    }

    tc_fence_before();
    __syncwarp();
    // clustered: no CTA leaves while another may still write its shared
    // memory or signal its barriers
    if (clustered) cluster_sync();
    else __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    }
}

// CUDA-core contraction for FP32 / FP64 storage: CTA (slice, 16 rows, 16
// columns), the slice's K in chunks of 64 through shared memory; column
// Nv of B is b.  A = float for FP32 storage, double for FP64.
template <class T, class A>
__global__ void __launch_bounds__(256) k_gauss_simt(const T* __restrict__ S, long long lds, int m, long long n,
                                                    const T* __restrict__ V, long long ldv, int K1,
                                                    const T* __restrict__ bcol, long long chunk,
                                                    double* __restrict__ part, int m_pad, int Ntot) {
    __shared__ A sS[16][65];
    __shared__ A sV[16][65];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int slice = blockIdx.x;
    const int r0 = blockIdx.y * 16, c0 = blockIdx.z * 16;
    const long long i0 = (long long)slice * chunk, i1 = min(n, i0 + chunk);
    A acc = A(0);
    for (long long kb = i0; kb < i1; kb += 64) {
        for (int e = threadIdx.x; e < 16 * 64; e += 256) {
            const int rr = e >> 6, kk = e & 63;
            const long long i = kb + kk;
            const int r = r0 + rr, c = c0 + rr;
            sS[rr][kk] = (r < m && i < i1) ? (A)S[(size_t)r * lds + i] : A(0);
            const T* col = c < K1 ? V + (size_t)c * ldv : (c == K1 ? bcol : nullptr);
            sV[rr][kk] = (col && i < i1) ? (A)col[i] : A(0);
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < 64; ++kk) acc = fma(sS[ty][kk], sV[tx][kk], acc);
        __syncthreads();
    }
    const int r = r0 + ty, c = c0 + tx;
    if (r < m && c < Ntot) part[((size_t)slice * m_pad + r) * Ntot + c] = (double)acc;
}

// [S V | S b] = the sum of the slices' partial tiles, in FP64 and in slice
// order.  Thread (r, j): j < K1 gives (S V)(r, j) into svd (column-major
// m x K1, FP32 or FP64), j = K1 gives c(r) = sum over the nb b rows.
template <class P>
__global__ void k_gauss_reduce(const P* __restrict__ part, int nsplit, int m, int m_pad, int Ntot, int K1, int Nv,
                               int nb, float* __restrict__ svd32, double* __restrict__ svd64,
                               double* __restrict__ c) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int cols = K1 + 1;
    if (t >= (long long)m * cols) return;
    const int r = (int)(t / cols), j = (int)(t - (long long)r * cols);
    double sum = 0.0;
    if (j < K1) {
        for (int s = 0; s < nsplit; ++s) sum += (double)part[((size_t)s * m_pad + r) * Ntot + j];
        if (svd64) svd64[(size_t)j * m + r] = sum;
        else svd32[(size_t)j * m + r] = (float)sum;
    } else {
        for (int s = 0; s < nsplit; ++s)
            for (int p = 0; p < nb; ++p) sum += (double)part[((size_t)s * m_pad + r) * Ntot + Nv + p];
        c[r] = sum;
    }
}

// slices of the n-long contraction: `groups` CTAs per slice, at most one CTA
// per SM in all; chunk a multiple of 64 so slices never share a stage
void split_plan(long long n, int groups, int num_sms, long long* chunk, int* nsplit) {
    int target = num_sms / groups;
    if (target < 1) target = 1;
    long long ch = (n + target - 1) / target;
    ch = (ch + kGmChunkAlign - 1) / kGmChunkAlign * kGmChunkAlign;
    *chunk = ch;
    *nsplit = (int)((n + ch - 1) / ch);
}

// rows per row group: ceil(m / 256) groups of equal height, a multiple of 16
// (the smallest S box), the last group taking what is left
int gauss_group_rows(int m) {
    const int mg = (m + 255) / 256;
    const int rg = ((m + mg - 1) / mg + 15) / 16 * 16;
    return (mg - 1) * rg < m ? rg : 256;              // every group keeps at least one row
}

int v_rows(int K1) { return (K1 + kGmBRows + 15) / 16 * 16 - kGmBRows; }     // Nv: Nv + 8 a multiple of 16

bool is16(int storage) { return storage == IPF_STORE_BF16 || storage == IPF_STORE_F16; }

size_t part_bytes(int storage, int m, long long n, int K1max, int num_sms) {
    const int m_pad = (m + 255) / 256 * 256;
    long long chunk;
    int nsplit;
    if (is16(storage)) {
        split_plan(n, m_pad / 256, num_sms, &chunk, &nsplit);
        return (size_t)nsplit * m_pad * (v_rows(K1max) + kGmBRows) * sizeof(float);
    }
    split_plan(n, 1, num_sms, &chunk, &nsplit);
    return (size_t)nsplit * m_pad * (K1max + 1) * sizeof(double);
}

// clusters of mg CTAs of the contraction (either pipeline, whichever allows
// fewer) that fit on the GPU at once; 0 where the query fails.  Both
// pipelines use the same slicing, so their results stay bit-identical.
int gauss_max_clusters(bool bf16, int mg) {
    static std::atomic<int> cache[2][9];              // 0: not asked yet; else the answer + 1
    const int have = cache[bf16 ? 1 : 0][mg].load();
    if (have > 0) return have - 1;
    auto q = [&](auto kern, int smem) -> int {
        if (raise_smem(kern, smem) != cudaSuccess) return 0;
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3((unsigned)(mg * 64));
        lc.blockDim = dim3(kGmThreads);
        lc.dynamicSmemBytes = (size_t)smem;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)mg;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        lc.attrs = at;
        lc.numAttrs = 1;
        int c = 0;
        if (cudaOccupancyMaxActiveClusters(&c, kern, &lc) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return c;
    };
    const int a = bf16 ? q(k_gauss_mma<true, 64>, GmShape<64>::kSmemRequest)
                       : q(k_gauss_mma<false, 64>, GmShape<64>::kSmemRequest);
    const int b = bf16 ? q(k_gauss_mma<true, 32>, GmShape<32>::kSmemRequest)
                       : q(k_gauss_mma<false, 32>, GmShape<32>::kSmemRequest);
    const int r = a < b ? a : b;
    cache[bf16 ? 1 : 0][mg].store(r + 1);
    return r;
}

}  // namespace

// row stride of the row-major S (FP32 / FP64) and of the b rows: n rounded
// up to 64 elements
long long gauss_lds(long long n) { return (n + 63) / 64 * 64; }

size_t gauss_workspace_bytes(int storage, int m, long long n, int k_max, int num_sms) {
    const size_t sb = storage == IPF_STORE_F64 ? 8 : storage == IPF_STORE_F32 ? 4 : 2;
    return (size_t)kGmBRows * gauss_lds(n) * sb + 256 + part_bytes(storage, m, n, k_max + 1, num_sms);
}

cudaError_t launch_gauss_fill(int storage, void* S, long long n, int m, long long lds, unsigned long long seed,
                              int num_sms, cudaStream_t s) {
    if (n <= 0 || m <= 0) return cudaSuccess;
    const int blocks = num_sms * 8;
    const double sq = sqrt((double)m);
    const float inv = (float)(1.0 / sq);
    switch (storage) {
        case IPF_STORE_F64: k_gauss_fill<double><<<blocks, 256, 0, s>>>((double*)S, n, m, lds, seed, sq, inv); break;
        case IPF_STORE_F32: k_gauss_fill<float><<<blocks, 256, 0, s>>>((float*)S, n, m, lds, seed, sq, inv); break;
        case IPF_STORE_BF16:
            k_gauss_fill<__nv_bfloat16><<<blocks, 256, 0, s>>>((__nv_bfloat16*)S, n, m, lds, seed, sq, inv);
            break;
        case IPF_STORE_F16: k_gauss_fill<__half><<<blocks, 256, 0, s>>>((__half*)S, n, m, lds, seed, sq, inv); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

size_t gauss_s_bytes(int storage, int m, long long n) {
    if (is16(storage)) return (size_t)((m + 15) / 16) * (size_t)((n + 63) / 64) * 1024 * 2;
    const size_t sb = storage == IPF_STORE_F64 ? 8 : 4;
    return (size_t)m * gauss_lds(n) * sb;
}

cudaError_t launch_gauss_fill_ctx(int storage, void* S, long long n, int m, unsigned long long seed, int num_sms,
                                  cudaStream_t s) {
    if (n <= 0 || m <= 0) return cudaSuccess;
    if (!is16(storage)) return launch_gauss_fill(storage, S, n, m, gauss_lds(n), seed, num_sms, s);
    const unsigned nkb = (unsigned)((n + 63) / 64);
    const unsigned long long total = (unsigned long long)((m + 15) / 16) * nkb * 1024ull;
    if (total / 1024ull >= (1ull << 32)) return cudaErrorInvalidValue;
    const int blocks = num_sms * 8;
    const double sq = sqrt((double)m);
    const float inv = (float)(1.0 / sq);
    if (storage == IPF_STORE_BF16)
        k_gauss_fill_tiled<__nv_bfloat16><<<blocks, 256, 0, s>>>((__nv_bfloat16*)S, n, m, nkb, total, seed, sq, inv);
    else
        k_gauss_fill_tiled<__half><<<blocks, 256, 0, s>>>((__half*)S, n, m, nkb, total, seed, sq, inv);
    return cudaGetLastError();
}

cudaError_t launch_gauss_bparts(int storage, const float* b, long long n, void* ws, cudaStream_t s) {
    const long long ldb = gauss_lds(n);
    const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    switch (storage) {
        case IPF_STORE_F64: k_gauss_bparts<double><<<blocks, 256, 0, s>>>(b, n, ldb, (double*)ws); break;
        case IPF_STORE_F32: k_gauss_bparts<float><<<blocks, 256, 0, s>>>(b, n, ldb, (float*)ws); break;
        case IPF_STORE_BF16:
            k_gauss_bparts<__nv_bfloat16><<<blocks, 256, 0, s>>>(b, n, ldb, (__nv_bfloat16*)ws);
            break;
        case IPF_STORE_F16: k_gauss_bparts<__half><<<blocks, 256, 0, s>>>(b, n, ldb, (__half*)ws); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// [S V_{K1} | S b] for the basis columns 0 .. K1-1 (V: kcols columns of
// ldv elements) into svd (column-major m x K1, FP64 for F64 storage, else
// FP32) and c (m, FP64).  ws: the workspace of gauss_workspace_bytes (the b
// rows written by launch_gauss_bparts first, then the partial tiles).
cudaError_t launch_gauss_sv(int storage, const void* S, int m, long long n, const void* V, long long ldv, int kcols,
                            int K1, void* ws, void* svd, double* c, int* err, int num_sms, int variant,
                            cudaStream_t s) {
    if (K1 < 1 || K1 > kcols || m < 1 || n < 1) return cudaErrorInvalidValue;
    const long long lds = gauss_lds(n);
    const size_t sb = storage == IPF_STORE_F64 ? 8 : storage == IPF_STORE_F32 ? 4 : 2;
    const void* bpart = ws;
    void* part = (char*)ws + ((size_t)kGmBRows * lds * sb + 255) / 256 * 256;
    const int m_pad = (m + 255) / 256 * 256;
    const int rb = 256;
    if (is16(storage)) {
        EncodeTiledFn enc = encode_fn();
        if (!enc) return cudaErrorNotSupported;
        const int Nv = v_rows(K1), Ntot = Nv + kGmBRows;
        if (Ntot > kGmBRowsMax) return cudaErrorInvalidValue;
        const int BK = variant == 32 ? 32 : 64;
        const int mg = m_pad / 256;
        const int rg = gauss_group_rows(m);
        // the row groups of a slice as one cluster sharing V's tiles, when
        // they are 2..8 and each CTA's share of V is at most 128 rows; the
        // slices are then as many as clusters fit on the GPU at once
        const bool bf = storage == IPF_STORE_BF16;
        const int clusters = (mg >= 2 && mg <= 8 && Nv <= 128 * mg) ? gauss_max_clusters(bf, mg) : 0;
        const bool clustered = clusters > 0;
        long long chunk;
        int nsplit;
        split_plan(n, mg, clustered ? clusters * mg : num_sms, &chunk, &nsplit);
        const CUtensorMapDataType dt =
            storage == IPF_STORE_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
        const cuuint32_t estr[2] = {1, 1};
        GmMaps maps;
        auto make = [&](CUtensorMap* map, const void* base, cuuint64_t rows, cuuint64_t ld, cuuint32_t box_rows) {
            const cuuint64_t dims[2] = {(cuuint64_t)n, rows};
            const cuuint64_t strides[1] = {ld * 2};
            const cuuint32_t box[2] = {(cuuint32_t)BK, box_rows};
            return enc(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       BK == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        };
        // S tiled: dims (64 elements, 16 rows, nkb unit columns, nrt unit rows)
        const cuuint64_t nkb = (cuuint64_t)((n + 63) / 64), nrt = (cuuint64_t)((m + 15) / 16);
        for (int b = 0; b < 4; ++b) {
            const cuuint64_t dims[4] = {64, 16, nkb, nrt};
            const cuuint64_t strides[3] = {128, 2048, nkb * 2048};
            const cuuint32_t box[4] = {(cuuint32_t)BK, 16, 1, (cuuint32_t)(8 >> b)};
            const cuuint32_t e4[4] = {1, 1, 1, 1};
            if (enc(&maps.s[b], dt, 4, const_cast<void*>(S), dims, strides, box, e4, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    BK == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                return cudaErrorInvalidValue;
        }
        if (make(&maps.vall, V, (cuuint64_t)kcols, (cuuint64_t)ldv, (cuuint32_t)Nv) != CUDA_SUCCESS ||
            make(&maps.b, bpart, (cuuint64_t)kGmBRows, (cuuint64_t)lds, kGmBRows) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
        for (int b = 0; clustered && b < 5; ++b)
            if (make(&maps.v[b], V, (cuuint64_t)kcols, (cuuint64_t)ldv, (cuuint32_t)(128 >> b)) != CUDA_SUCCESS)
                return cudaErrorInvalidValue;
        auto go = [&](auto kern, int smem) -> cudaError_t {
            cudaError_t e = raise_smem(kern, smem);
            if (e != cudaSuccess) return e;
            cudaLaunchConfig_t lc = {};
            lc.gridDim = dim3((unsigned)(nsplit * mg));
            lc.blockDim = dim3(kGmThreads);
            lc.dynamicSmemBytes = (size_t)smem;
            lc.stream = s;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = clustered ? (unsigned)mg : 1u;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            lc.attrs = at;
            lc.numAttrs = clustered ? 1 : 0;
            return cudaLaunchKernelEx(&lc, kern, maps, n, m, chunk, mg, rg, Nv, Ntot, clustered ? 1 : 0,
                                      (float*)part, m_pad, err);
        };
        cudaError_t e;
        if (BK == 64) e = bf ? go(k_gauss_mma<true, 64>, GmShape<64>::kSmemRequest)
                             : go(k_gauss_mma<false, 64>, GmShape<64>::kSmemRequest);
        else e = bf ? go(k_gauss_mma<true, 32>, GmShape<32>::kSmemRequest)
                    : go(k_gauss_mma<false, 32>, GmShape<32>::kSmemRequest);
        if (e != cudaSuccess) return e;
        const long long th = (long long)m * (K1 + 1);
        k_gauss_reduce<float><<<(unsigned)((th + rb - 1) / rb), rb, 0, s>>>(
            (const float*)part, nsplit, m, m_pad, Ntot, K1, Nv, 3, (float*)svd, nullptr, c);
        return cudaGetLastError();
    }
    long long chunk;
    int nsplit;
    split_plan(n, 1, num_sms, &chunk, &nsplit);
    const int Ntot = K1 + 1;
    const dim3 grid(nsplit, (m + 15) / 16, (Ntot + 15) / 16);
    if (storage == IPF_STORE_F64)
        k_gauss_simt<double, double><<<grid, 256, 0, s>>>((const double*)S, lds, m, n, (const double*)V, ldv, K1,
                                                          (const double*)bpart, chunk, (double*)part, m_pad, Ntot);
    else
        k_gauss_simt<float, float><<<grid, 256, 0, s>>>((const float*)S, lds, m, n, (const float*)V, ldv, K1,
                                                        (const float*)bpart, chunk, (double*)part, m_pad, Ntot);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long th = (long long)m * (K1 + 1);
    k_gauss_reduce<double><<<(unsigned)((th + rb - 1) / rb), rb, 0, s>>>(
        (const double*)part, nsplit, m, m_pad, Ntot, K1, K1, 1,
        storage == IPF_STORE_F64 ? nullptr : (float*)svd, storage == IPF_STORE_F64 ? (double*)svd : nullptr, c);
    return cudaGetLastError();
}

// The contraction's pipeline for one shape: 64-element stages (3 in flight)
// or 32-element stages (7 in flight), whichever is faster on this GPU for
// (storage, m, n, kcols), timed once per shape (two launches each after a
// warm-up, on `s`, synchronising) and kept by the autotuner.  FP32 / FP64
// storage has one kernel (returns 0).
int gauss_variant(int storage, const void* S, int m, long long n, const void* V, long long ldv, int kcols, void* ws,
                  void* svd, double* c, int* err, int num_sms, cudaStream_t s) {
    if (!is16(storage)) return 0;
    char key[128];
    snprintf(key, sizeof key, "gauss/%s/m%d/n%lld/k%d", storage == IPF_STORE_BF16 ? "bf16" : "f16", m, n, kcols);
    int v = 0, p = 0;
    if (tune_lookup(key, &v, &p)) return v;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return 64;
    }
    int best = 64;
    float best_ms = 1e30f;
    for (int bk : {64, 32}) {
        bool ok = launch_gauss_sv(storage, S, m, n, V, ldv, kcols, kcols, ws, svd, c, err, num_sms, bk, s) ==
                  cudaSuccess;
        ok = ok && cudaEventRecord(e0, s) == cudaSuccess;
        for (int r = 0; r < 2 && ok; ++r)
            ok = launch_gauss_sv(storage, S, m, n, V, ldv, kcols, kcols, ws, svd, c, err, num_sms, bk, s) ==
                 cudaSuccess;
        ok = ok && cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
        float ms = 0.f;
        if (ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms / 2 < best_ms) {
            best_ms = ms / 2;
            best = bk;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    tune_store(key, best, 0, best_ms * 1e3);
    return best;
}

}  // namespace ipf
