// Forward operators w = A v (A is reached only through products, Sec. 1 of
// the paper), reading the basis vector in its storage type and accumulating
// in FP32 (FP64 for F64 storage).
//
//   k_conv2d      zero-boundary 2-D convolution with an odd PSF, output tile
//                 plus halo staged in shared memory, 4x8 outputs per thread
//                 with the PSF row and the input row segment in registers.
//   k_sep_motion  separable Gaussian (row pass, column pass), crop to the
//                 image, then the motion stencil, all in one tile.
//   k_csr         CSR product for B interleaved right-hand sides: one warp
//                 per row, lanes grouped by RHS so A is read once for all B.
#include <cstring>
#include <type_traits>

#include "ipf_internal.cuh"

namespace ipf {

namespace {

template <class T> __device__ __forceinline__ typename AccOf<T>::type ld_acc(const T* p) { return to_acc(*p); }

// ------------------------------------------------------------------------
// 2-D convolution.  KW = compile-time padded kernel width (odd), ph rows
// (runtime, odd).  Tile: TY x TX outputs, 256 threads as 16 x 16, each
// thread OY x OX = (TY/16) x (TX/16) outputs.
// ------------------------------------------------------------------------
template <class T, class Acc, int KW, int OY, int OX>
__global__ void __launch_bounds__(256, 3) k_conv2d(const T* __restrict__ vbase, long long ldv, const int* __restrict__ jptr,
                                                 Acc* __restrict__ w, int H, int W,
                                                 const float* __restrict__ psf, int ph, int pw) {
    const T* v = jptr ? vbase + (size_t)(*jptr) * ldv : vbase;
    constexpr int TY = 16 * OY, TX = 16 * OX;
    constexpr int IW = TX + KW - 1;                  // input tile width
    constexpr int IWP = (IW + 3) & ~3;
    extern __shared__ unsigned char smem_raw[];
    Acc* s_in = (Acc*)smem_raw;                      // (TY + ph - 1) x IWP
    Acc* s_k = s_in + (size_t)(TY + ph - 1) * IWP;   // ph x KW, flipped, width-padded
    const int cy = ph / 2, cx = KW / 2;
    const int y0 = blockIdx.y * TY, x0 = blockIdx.x * TX;
    const int IH = TY + ph - 1;
    // flipped, zero-padded kernel: s_k[a][b] multiplies v(y - cy + a, x - cx + b)
    const int padl = (KW - pw) / 2;
    for (int t = threadIdx.x; t < ph * KW; t += blockDim.x) {
        const int a = t / KW, bb = t - a * KW;
        const int kb = bb - padl;
        Acc val = 0;
        if (kb >= 0 && kb < pw) val = (Acc)psf[(ph - 1 - a) * pw + (pw - 1 - kb)];
        s_k[t] = val;
    }
    for (int t = threadIdx.x; t < IH * IWP; t += blockDim.x) {
        const int a = t / IWP, bb = t - a * IWP;
        const int yy = y0 - cy + a, xx = x0 - cx + bb;
        Acc val = 0;
        if (bb < IW && yy >= 0 && yy < H && xx >= 0 && xx < W) val = ld_acc(v + (size_t)yy * W + xx);
        s_in[t] = val;
    }
    __syncthreads();
    const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
    const int oy0 = ty * OY, ox0 = tx * OX;
    Acc acc[OY][OX];
#pragma unroll
    for (int a = 0; a < OY; ++a)
#pragma unroll
        for (int bb = 0; bb < OX; ++bb) acc[a][bb] = 0;
    for (int ky = 0; ky < ph; ++ky) {
        Acc kr[KW];
#pragma unroll
        for (int q = 0; q < KW; ++q) kr[q] = s_k[ky * KW + q];
#pragma unroll
        for (int a = 0; a < OY; ++a) {
            const Acc* row = s_in + (size_t)(oy0 + a + ky) * IWP + ox0;
            Acc in[OX + KW - 1];
#pragma unroll
            for (int q = 0; q < OX + KW - 1; ++q) in[q] = row[q];
#pragma unroll
            for (int q = 0; q < KW; ++q)
#pragma unroll
                for (int bb = 0; bb < OX; ++bb) acc[a][bb] = fma(kr[q], in[bb + q], acc[a][bb]);
        }
    }
#pragma unroll
    for (int a = 0; a < OY; ++a) {
        const int yy = y0 + oy0 + a;
        if (yy >= H) continue;
#pragma unroll
        for (int bb = 0; bb < OX; ++bb) {
            const int xx = x0 + ox0 + bb;
            if (xx < W) w[(size_t)yy * W + xx] = acc[a][bb];
        }
    }
}

// ------------------------------------------------------------------------
// 2-D convolution, FP32 accumulation, PSF width KW <= 31 (padded to KWP, a
// multiple of 4).  Same tile scheme as k_conv2d, but the flipped PSF row
// (KWP floats) and the thread's input row segment (NIN floats) are loaded
// as float4 into registers, so the inner loop is OX FMAs per kernel column
// with no shared-memory traffic.
// ------------------------------------------------------------------------
template <class T, int KW, int OY, int OX>
__global__ void __launch_bounds__(256, 2) k_conv2d_v(const T* __restrict__ vbase, long long ldv,
                                                    const int* __restrict__ jptr, float* __restrict__ w, int H,
                                                    int W, const float* __restrict__ psf, int ph, int pw) {
    const T* v = jptr ? vbase + (size_t)(*jptr) * ldv : vbase;
    constexpr int KWP = (KW + 3) & ~3;
    constexpr int TY = 16 * OY, TX = 16 * OX;
    constexpr int NIN = (OX + KW - 1 + 3) & ~3;       // input floats per output row segment
    constexpr int IWP = TX - OX + NIN;                // covers the last thread's segment
    static_assert(OX % 4 == 0, "OX must be a multiple of 4");
    extern __shared__ float4 smem_f4[];
    float* s_in = (float*)smem_f4;                    // (TY + ph - 1) x IWP
    float* s_k = s_in + (size_t)(TY + ph - 1) * IWP;  // ph x KWP
    const int cy = ph / 2, cx = KW / 2;
    const int y0 = blockIdx.y * TY, x0 = blockIdx.x * TX;
    const int IH = TY + ph - 1;
    const int padl = (KW - pw) / 2;
    for (int t = threadIdx.x; t < ph * KWP; t += blockDim.x) {
        const int a = t / KWP, bb = t - a * KWP;
        const int kb = bb - padl;
        float val = 0.f;
        if (bb < KW && kb >= 0 && kb < pw) val = psf[(ph - 1 - a) * pw + (pw - 1 - kb)];
        s_k[t] = val;
    }
    for (int t = threadIdx.x; t < IH * IWP; t += blockDim.x) {
        const int a = t / IWP, bb = t - a * IWP;
        const int yy = y0 - cy + a, xx = x0 - cx + bb;
        float val = 0.f;
        if (bb < TX + KW - 1 && yy >= 0 && yy < H && xx >= 0 && xx < W) val = to_acc(v[(size_t)yy * W + xx]);
        s_in[t] = val;
    }
    __syncthreads();
    const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
    const int oy0 = ty * OY, ox0 = tx * OX;
    float acc[OY][OX];
#pragma unroll
    for (int a = 0; a < OY; ++a)
#pragma unroll
        for (int bb = 0; bb < OX; ++bb) acc[a][bb] = 0.f;
    for (int ky = 0; ky < ph; ++ky) {
        float kr[KWP];
        const float4* kp = (const float4*)(s_k + ky * KWP);
#pragma unroll
        for (int q = 0; q < KWP / 4; ++q) {
            const float4 t4 = kp[q];
            kr[4 * q] = t4.x; kr[4 * q + 1] = t4.y; kr[4 * q + 2] = t4.z; kr[4 * q + 3] = t4.w;
        }
#pragma unroll
        for (int a = 0; a < OY; ++a) {
            const float4* rp = (const float4*)(s_in + (size_t)(oy0 + a + ky) * IWP + ox0);
            float in[NIN];
#pragma unroll
            for (int q = 0; q < NIN / 4; ++q) {
                const float4 t4 = rp[q];
                in[4 * q] = t4.x; in[4 * q + 1] = t4.y; in[4 * q + 2] = t4.z; in[4 * q + 3] = t4.w;
            }
#pragma unroll
            for (int q = 0; q < KW; ++q)
#pragma unroll
                for (int bb = 0; bb < OX; ++bb) acc[a][bb] = fmaf(kr[q], in[bb + q], acc[a][bb]);
        }
    }
#pragma unroll
    for (int a = 0; a < OY; ++a) {
        const int yy = y0 + oy0 + a;
        if (yy >= H) continue;
#pragma unroll
        for (int bb = 0; bb < OX; ++bb) {
            const int xx = x0 + ox0 + bb;
            if (xx < W) w[(size_t)yy * W + xx] = acc[a][bb];
        }
    }
}

// ------------------------------------------------------------------------
// 2-D convolution, FP32 accumulation, square-padded PSF KW x KW (KW <= 31),
// column formulation.  Thread t of a 256-thread block owns image column
// x0 + t of a 256-column tile and OY consecutive output rows.  For each kernel column b it loads the PSF column F[0..KW)[b] into
// registers, then walks the staged input column (OY + KW - 1 values, one
// conflict-free 4-byte shared load each: consecutive lanes read consecutive
// x) and adds F[r - a][b] * in[r] into the OY accumulators.
// ------------------------------------------------------------------------
template <class T, int KW, int OY>
__global__ void __launch_bounds__(256, 2) k_conv2d_c(const T* __restrict__ vbase, long long ldv,
                                                    const int* __restrict__ jptr, float* __restrict__ w, int H,
                                                    int W, const float* __restrict__ psf, int ph, int pw) {
    const T* v = jptr ? vbase + (size_t)(*jptr) * ldv : vbase;
    constexpr int TX = 256, TY = OY;
    constexpr int IH = TY + KW - 1, IW = TX + KW - 1;
    constexpr int IWP = IW + 1;                       // odd pitch keeps column walks conflict-free
    extern __shared__ float smem_c[];
    float* s_in = smem_c;                             // IH x IWP
    float* s_k = s_in + IH * IWP;                     // KW x KW flipped, zero-padded
    const int c = KW / 2;
    const int y0 = blockIdx.y * TY, x0 = blockIdx.x * TX;
    const int pady = (KW - ph) / 2, padx = (KW - pw) / 2;
    for (int t = threadIdx.x; t < KW * KW; t += blockDim.x) {
        const int a = t / KW, bb = t - a * KW;
        const int ka = a - pady, kb = bb - padx;
        float val = 0.f;
        if (ka >= 0 && ka < ph && kb >= 0 && kb < pw) val = psf[(ph - 1 - ka) * pw + (pw - 1 - kb)];
        s_k[t] = val;
    }
    for (int t = threadIdx.x; t < IH * IW; t += blockDim.x) {
        const int a = t / IW, bb = t - a * IW;
        const int yy = y0 - c + a, xx = x0 - c + bb;
        float val = 0.f;
        if (yy >= 0 && yy < H && xx >= 0 && xx < W) val = to_acc(v[(size_t)yy * W + xx]);
        s_in[a * IWP + bb] = val;
    }
    __syncthreads();
    const int ox = threadIdx.x;                        // 0..255
    float acc[OY];
#pragma unroll
    for (int a = 0; a < OY; ++a) acc[a] = 0.f;
    for (int b = 0; b < KW; ++b) {
        float f[KW];
#pragma unroll
        for (int a = 0; a < KW; ++a) f[a] = s_k[a * KW + b];
        const float* col = s_in + ox + b;
#pragma unroll
        for (int r = 0; r < IH; ++r) {
            const float x = col[r * IWP];
#pragma unroll
            for (int a = 0; a < OY; ++a) {
                const int ky = r - a;
                if (ky >= 0 && ky < KW) acc[a] = fmaf(f[ky], x, acc[a]);
            }
        }
    }
    const int xx = x0 + ox;
    if (xx < W) {
#pragma unroll
        for (int a = 0; a < OY; ++a) {
            const int yy = y0 + a;
            if (yy < H) w[(size_t)yy * W + xx] = acc[a];
        }
    }
}

// ------------------------------------------------------------------------
// Packed-FMA column convolution (Blackwell fma.rn.f32x2: two FP32 FMAs per
// instruction).  Like k_conv2d_c, but output rows are paired: for input row
// r and pair (2a, 2a+1), {acc[2a], acc[2a+1]} += {F[ky][b], F[ky-1][b]} * {x, x}
// with ky = r - 2a, so one loaded value feeds both rows and the PSF column
// lives in registers as KW+1 packed pairs (F[-1] = F[KW] = 0).
// ------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b,
                                                    unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
    return (unsigned long long)__float_as_uint(lo) | ((unsigned long long)__float_as_uint(hi) << 32);
}

// one 128 x OY output tile (tile column bx, tile row by), 128 threads
template <class T, int KW, int OY>
__device__ __forceinline__ void conv_c2_tile(const T* __restrict__ v, float* __restrict__ w, int H, int W,
                                             const unsigned long long* __restrict__ pairs, int bx, int by) {
    static_assert(OY % 2 == 0, "OY must be even");
    constexpr int TX = 128, TY = OY;
    constexpr int IH = TY + KW - 1, IW = TX + KW - 1;
    constexpr int IWP = IW + 1;
    constexpr int NP = KW + 1;                        // packed pairs per PSF column
    extern __shared__ float s_in[];                   // IH x IWP
    const int c = KW / 2;
    const int y0 = by * TY, x0 = bx * TX;
    for (int t = threadIdx.x; t < IH * IW; t += blockDim.x) {
        const int a = t / IW, bb = t - a * IW;
        const int yy = y0 - c + a, xx = x0 - c + bb;
        float val = 0.f;
        if (yy >= 0 && yy < H && xx >= 0 && xx < W) val = to_acc(v[(size_t)yy * W + xx]);
        s_in[a * IWP + bb] = val;
    }
    __syncthreads();
    const int ox = threadIdx.x;
    unsigned long long acc[OY / 2];
#pragma unroll
    for (int a = 0; a < OY / 2; ++a) acc[a] = 0ull;
    for (int b = 0; b < KW; ++b) {
        unsigned long long f2[NP];
#pragma unroll
        for (int q = 0; q < NP; ++q) f2[q] = __ldg(pairs + b * NP + q);   // same address for the whole CTA
        const float* col = s_in + ox + b;
#pragma unroll
        for (int r = 0; r < IH; ++r) {
            const float x = col[r * IWP];
            const unsigned long long xx = pack2(x, x);
#pragma unroll
            for (int a2 = 0; a2 < OY / 2; ++a2) {
                const int ky = r - 2 * a2;
                if (ky >= 0 && ky <= KW) acc[a2] = ffma2(f2[ky], xx, acc[a2]);
            }
        }
    }
    const int xo = x0 + ox;
    if (xo < W) {
#pragma unroll
        for (int a2 = 0; a2 < OY / 2; ++a2) {
            const int yy = y0 + 2 * a2;
            if (yy < H) w[(size_t)yy * W + xo] = __uint_as_float((unsigned)(acc[a2] & 0xFFFFFFFFull));
            if (yy + 1 < H) w[(size_t)(yy + 1) * W + xo] = __uint_as_float((unsigned)(acc[a2] >> 32));
        }
    }
}

template <class T, int KW, int OY>
__global__ void __launch_bounds__(128, 7) k_conv2d_c2(const T* __restrict__ vbase, long long ldv,
                                                     const int* __restrict__ jptr, float* __restrict__ w, int H,
                                                     int W, const unsigned long long* __restrict__ pairs) {
    const T* v = jptr ? vbase + (size_t)(*jptr) * ldv : vbase;
    conv_c2_tile<T, KW, OY>(v, w, H, W, pairs, blockIdx.x, blockIdx.y);
}

// ------------------------------------------------------------------------
// separable Gaussian then motion blur, each zero-boundary, fused per tile
// ------------------------------------------------------------------------
template <class T, class Acc, int TILE>
__global__ void __launch_bounds__(256) k_sep_motion(const T* __restrict__ vbase, long long ldv, const int* __restrict__ jptr,
                                                     Acc* __restrict__ w, int H, int W,
                                                     const float* __restrict__ grow, const float* __restrict__ gcol,
                                                     int slen, const float* __restrict__ mot, int mlen) {
    const T* v = jptr ? vbase + (size_t)(*jptr) * ldv : vbase;
    extern __shared__ unsigned char smem_raw[];
    const int hs = slen / 2, hm = mlen / 2;
    const int hal = hs + hm;
    const int A0 = TILE + 2 * hal;      // input tile side
    const int A1 = TILE + 2 * hm;       // after the separable pass
    Acc* s_in = (Acc*)smem_raw;                      // A0 x A0
    Acc* s_r = s_in + (size_t)A0 * A0;               // A0 rows x A1 cols (row pass)
    Acc* s_c = s_r + (size_t)A0 * A1;                // A1 x A1 (column pass, cropped)
    Acc* s_g = s_c + (size_t)A1 * A1;                // grow (slen), gcol (slen), motion (mlen^2)
    const int y0 = blockIdx.y * TILE, x0 = blockIdx.x * TILE;
    for (int t = threadIdx.x; t < slen; t += blockDim.x) {
        s_g[t] = (Acc)grow[t];
        s_g[slen + t] = (Acc)gcol[t];
    }
    for (int t = threadIdx.x; t < mlen * mlen; t += blockDim.x) s_g[2 * slen + t] = (Acc)mot[t];
    for (int t = threadIdx.x; t < A0 * A0; t += blockDim.x) {
        const int a = t / A0, bb = t - a * A0;
        const int yy = y0 - hal + a, xx = x0 - hal + bb;
        Acc val = 0;
        if (yy >= 0 && yy < H && xx >= 0 && xx < W) val = ld_acc(v + (size_t)yy * W + xx);
        s_in[t] = val;
    }
    __syncthreads();
    // row pass: s_r[a][c] = sum_q grow[q] * in[a][c + 2hs - q]   (c in 0..A1-1 -> x = x0-hm+c)
    for (int t = threadIdx.x; t < A0 * A1; t += blockDim.x) {
        const int a = t / A1, c = t - a * A1;
        const Acc* row = s_in + (size_t)a * A0 + c;
        Acc s = 0;
        for (int q = 0; q < slen; ++q) s = fma(s_g[q], row[2 * hs - q], s);
        s_r[t] = s;
    }
    __syncthreads();
    // column pass, then crop to the image: s_c[a][c] at (y0-hm+a, x0-hm+c)
    for (int t = threadIdx.x; t < A1 * A1; t += blockDim.x) {
        const int a = t / A1, c = t - a * A1;
        const int yy = y0 - hm + a, xx = x0 - hm + c;
        Acc s = 0;
        if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
            for (int q = 0; q < slen; ++q) s = fma(s_g[slen + q], s_r[(size_t)(a + 2 * hs - q) * A1 + c], s);
        }
        s_c[t] = s;
    }
    __syncthreads();
    const Acc* mk = s_g + 2 * slen;
    for (int t = threadIdx.x; t < TILE * TILE; t += blockDim.x) {
        const int a = t / TILE, c = t - a * TILE;
        const int yy = y0 + a, xx = x0 + c;
        if (yy >= H || xx >= W) continue;
        Acc s = 0;
        for (int p = 0; p < mlen; ++p)
            for (int q = 0; q < mlen; ++q)
                s = fma(mk[p * mlen + q], s_c[(size_t)(a + 2 * hm - p) * A1 + (c + 2 * hm - q)], s);
        w[(size_t)yy * W + xx] = s;
    }
}

// ------------------------------------------------------------------------
// CSR, B interleaved right-hand sides, one warp per row.  The summation
// order does not depend on B: the row's nonzeros are split into 32 classes
// by (p - rowstart) mod 32, each class is summed in order, and the classes
// are combined by the butterfly with offsets 16, 8, 4, 2, 1.  With G = 32/B
// lane groups, lane (g, r) owns classes g + G*u (u < B) of RHS r: offsets
// >= G pair classes inside a lane, smaller ones pair lanes g and g^o.  A
// right-hand side therefore gets the same bits alone or in any batch.
// ------------------------------------------------------------------------
// rows row0, row0 + step, ... below row1, one warp per row
template <class T, class Acc, int B>
__device__ __forceinline__ void csr_rows(const long long* __restrict__ rowptr, const int* __restrict__ colind,
                                         const float* __restrict__ vals, const T* __restrict__ v,
                                         Acc* __restrict__ w, long long row0, long long row1, long long step) {
    constexpr int G = 32 / B;
    const int lane = threadIdx.x & 31;
    const int g = lane / B, rr = lane - g * B;
    for (long long row = row0; row < row1; row += step) {
        const long long s = rowptr[row], e = rowptr[row + 1];
        Acc P[B];
#pragma unroll
        for (int u = 0; u < B; ++u) P[u] = 0;
        for (long long base = s; base < e; base += 32) {
#pragma unroll
            for (int u = 0; u < B; ++u) {
                const long long p = base + g + G * u;
                if (p < e) P[u] = fma((Acc)vals[p], to_acc(v[(size_t)colind[p] * B + rr]), P[u]);
            }
        }
        // in-lane levels: offsets o = 16 .. G pair classes c, c ^ o (u, u ^ o/G)
#pragma unroll
        for (int o = 16; o >= G && o >= 1; o >>= 1) {
            const int ou = o / G;
#pragma unroll
            for (int u = 0; u < B; ++u)
                if (!(u & ou)) P[u] = P[u] + P[u ^ ou];
        }
        Acc acc = P[0];
        // cross-lane levels: offsets o < G pair groups g, g ^ o
#pragma unroll
        for (int o = (G >= 2 ? G / 2 : 0); o >= 1; o >>= 1) acc = acc + __shfl_xor_sync(0xffffffffu, acc, o * B);
        if (g == 0) w[(size_t)row * B + rr] = acc;
    }
}

template <class T, class Acc, int B>
__global__ void __launch_bounds__(256) k_csr(const long long* __restrict__ rowptr, const int* __restrict__ colind,
                                              const float* __restrict__ vals, long long m,
                                              const T* __restrict__ vbase, long long ldv,
                                              const int* __restrict__ jptr, Acc* __restrict__ w) {
    const T* v = jptr ? vbase + (size_t)(*jptr) * ldv : vbase;
    const long long warps = (long long)gridDim.x * (blockDim.x / 32);
    csr_rows<T, Acc, B>(rowptr, colind, vals, v, w, (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, m,
                        warps);
}

template <class T, class Acc>
cudaError_t conv_dispatch(const OpDev& op, const T* v, long long ldv, const int* jp, Acc* w, cudaStream_t s) {
    const int H = op.rows, W = op.cols;
    auto go = [&](auto kern, int KW, int TY, int TX) -> cudaError_t {
        const int IWP = (TX + KW - 1 + 3) & ~3;
        const size_t smem = ((size_t)(TY + op.ph - 1) * IWP + (size_t)op.ph * KW) * sizeof(Acc);
        cudaError_t e = raise_smem(kern, (int)smem);
        if (e != cudaSuccess) return e;
        dim3 grid((W + TX - 1) / TX, (H + TY - 1) / TY);
        kern<<<grid, 256, smem, s>>>(v, ldv, jp, w, H, W, op.psf, op.ph, op.pw);
        return cudaGetLastError();
    };
    const int mx = op.pw;
    if constexpr (sizeof(Acc) == 4) {
        // register-blocked float path: 2 x 8 outputs per thread, 32 x 128 tiles
        auto gov = [&](auto kern, int KW) -> cudaError_t {
            constexpr int TY = 32, TX = 128, OX = 8;
            const int KWP = (KW + 3) & ~3;
            const int NIN = (OX + KW - 1 + 3) & ~3;
            const int IWP = TX - OX + NIN;
            const size_t smem = ((size_t)(TY + op.ph - 1) * IWP + (size_t)op.ph * KWP) * sizeof(float);
            cudaError_t e = raise_smem(kern, (int)smem);
            if (e != cudaSuccess) return e;
            dim3 grid((W + TX - 1) / TX, (H + TY - 1) / TY);
            kern<<<grid, 256, smem, s>>>(v, ldv, jp, (float*)w, H, W, op.psf, op.ph, op.pw);
            return cudaGetLastError();
        };
        // column formulation for square-paddable PSFs (ph <= KW, pw <= KW)
        auto goc = [&](auto kern, int KW, int OY) -> cudaError_t {
            const int IH = OY + KW - 1, IWP = 256 + KW;
            const size_t smem = ((size_t)IH * IWP + (size_t)KW * KW) * sizeof(float);
            cudaError_t e = raise_smem(kern, (int)smem);
            if (e != cudaSuccess) return e;
            dim3 grid((W + 255) / 256, (H + OY - 1) / OY);
            kern<<<grid, 256, smem, s>>>(v, ldv, jp, (float*)w, H, W, op.psf, op.ph, op.pw);
            return cudaGetLastError();
        };
        auto goc2 = [&](auto kern, int KW, int OY) -> cudaError_t {
            const int IH = OY + KW - 1, IWP = 128 + KW;
            const size_t smem = (size_t)IH * IWP * sizeof(float);
            cudaError_t e = raise_smem(kern, (int)smem);
            if (e != cudaSuccess) return e;
            dim3 grid((W + 127) / 128, (H + OY - 1) / OY);
            kern<<<grid, 128, smem, s>>>(v, ldv, jp, (float*)w, H, W, op.psf_pairs);
            return cudaGetLastError();
        };
        if (op.psf_pairs) {
            if (op.kw == 7) return goc2(k_conv2d_c2<T, 7, 16>, 7, 16);
            if (op.kw == 15) return goc2(k_conv2d_c2<T, 15, 16>, 15, 16);
            if (op.kw == 31) return goc2(k_conv2d_c2<T, 31, 16>, 31, 16);
        }
        const int mk = op.ph > op.pw ? op.ph : op.pw;
        if (mk <= 31) return goc(k_conv2d_c<T, 31, 16>, 31, 16);
        (void)gov;
        return go(k_conv2d<T, Acc, 63, 2, 4>, 63, 32, 64);
    } else {
        if (mx <= 7) return go(k_conv2d<T, Acc, 7, 2, 4>, 7, 32, 64);
        if (mx <= 15) return go(k_conv2d<T, Acc, 15, 2, 8>, 15, 32, 128);
        if (mx <= 31) return go(k_conv2d<T, Acc, 31, 2, 8>, 31, 32, 128);
        return go(k_conv2d<T, Acc, 63, 2, 4>, 63, 32, 64);
    }
}

template <class T, class Acc>
cudaError_t sep_dispatch(const OpDev& op, const T* v, long long ldv, const int* jp, Acc* w, cudaStream_t s) {
    constexpr int TILE = 32;
    const int hal = op.slen / 2 + op.mlen / 2;
    const int A0 = TILE + 2 * hal, A1 = TILE + 2 * (op.mlen / 2);
    const size_t smem = ((size_t)A0 * A0 + (size_t)A0 * A1 + (size_t)A1 * A1 + 2 * op.slen +
                         (size_t)op.mlen * op.mlen) * sizeof(Acc);
    auto kern = k_sep_motion<T, Acc, TILE>;
    cudaError_t e = raise_smem(kern, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((op.cols + TILE - 1) / TILE, (op.rows + TILE - 1) / TILE);
    kern<<<grid, 256, smem, s>>>(v, ldv, jp, w, op.rows, op.cols, op.sep_row, op.sep_col, op.slen, op.motion, op.mlen);
    return cudaGetLastError();
}

template <class T, class Acc>
cudaError_t csr_dispatch(const OpDev& op, const T* v, long long ldv, const int* jp, Acc* w, int B, cudaStream_t s) {
    const long long m = op.rows;
    long long blocks = (m + 7) / 8;
    if (blocks > 152 * 16) blocks = 152 * 16;
    const int nb = (int)blocks;
    switch (B) {
        case 1: k_csr<T, Acc, 1><<<nb, 256, 0, s>>>(op.rowptr, op.colind, op.vals, m, v, ldv, jp, w); break;
        case 2: k_csr<T, Acc, 2><<<nb, 256, 0, s>>>(op.rowptr, op.colind, op.vals, m, v, ldv, jp, w); break;
        case 4: k_csr<T, Acc, 4><<<nb, 256, 0, s>>>(op.rowptr, op.colind, op.vals, m, v, ldv, jp, w); break;
        case 8: k_csr<T, Acc, 8><<<nb, 256, 0, s>>>(op.rowptr, op.colind, op.vals, m, v, ldv, jp, w); break;
        case 16: k_csr<T, Acc, 16><<<nb, 256, 0, s>>>(op.rowptr, op.colind, op.vals, m, v, ldv, jp, w); break;
        case 32: k_csr<T, Acc, 32><<<nb, 256, 0, s>>>(op.rowptr, op.colind, op.vals, m, v, ldv, jp, w); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <class T>
cudaError_t apply_T(const OpDev& op, const void* v, long long ldv, long long vcols, const int* jp, void* w, int B,
                    int* err, cudaStream_t s) {
    using Acc = typename AccOf<T>::type;
    switch (op.kind) {
        case IPF_OP_PSF2D:
            if constexpr (std::is_same<T, __nv_bfloat16>::value) {
                if (conv_tc_eligible(op, v, ldv)) return launch_conv_tc(op, v, ldv, vcols, jp, (float*)w, err, s);
            }
            (void)vcols;
            (void)err;
            return conv_dispatch<T, Acc>(op, (const T*)v, ldv, jp, (Acc*)w, s);
        case IPF_OP_PSF2D_SEP_MOTION: return sep_dispatch<T, Acc>(op, (const T*)v, ldv, jp, (Acc*)w, s);
        case IPF_OP_CSR: return csr_dispatch<T, Acc>(op, (const T*)v, ldv, jp, (Acc*)w, B, s);
        default: return cudaErrorInvalidValue;
    }
}

// (A v_j)(p_i), i <= j, for the pivot-block solve.  PSF: four warps per
// pivot row, warp q taking the stencil rows q ceil(ph/4) .. (q+1) ceil(ph/4)
// - 1 with the lanes over the columns (every load of a warp issued before
// its FMAs: one round of loads for a 31 x 31 stencil), a fixed-order shuffle
// reduction in each warp and the four partial sums added in warp order.
// CSR: one warp per (pivot, RHS), lanes over the row's nonzeros, a
// fixed-order shuffle reduction.
constexpr int kPivParts = 4;                 // warps per PSF pivot row

template <class T>
__device__ __forceinline__ float pivot_row_psf_part(const T* __restrict__ v, int p, int H, int W,
                                                    const float* __restrict__ psf, int ph, int pw, int part) {
    const int lane = threadIdx.x & 31;
    const int py = p / W, px = p - py * W;
    const int cy = ph / 2, cx = pw / 2;
    const int per = (ph + kPivParts - 1) / kPivParts;
    const int ky0 = part * per, ky1 = min(ph, ky0 + per);
    float acc = 0.f;
    constexpr int U = 8;
    for (int kx = lane; kx < pw; kx += 32) {
        const int xx = px - kx + cx;
        const bool xin = xx >= 0 && xx < W;
        for (int ky = ky0; ky < ky1; ky += U) {
            float f[U], x[U];
            bool in[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int k = ky + u;
                const int yy = py - k + cy;
                in[u] = k < ky1 && xin && yy >= 0 && yy < H;
                f[u] = in[u] ? psf[k * pw + kx] : 0.f;
                x[u] = in[u] ? to_acc(v[(size_t)yy * W + xx]) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (in[u]) acc = fmaf(f[u], x[u], acc);
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    return acc;
}

// the four warps' partial sums of one pivot row, in warp order
__device__ __forceinline__ float pivot_parts_sum(const float* s) { return ((s[0] + s[1]) + s[2]) + s[3]; }

template <class T>
__device__ __forceinline__ float pivot_row_csr(const T* __restrict__ v, long long row, int B, int r,
                                               const long long* __restrict__ rowptr, const int* __restrict__ colind,
                                               const float* __restrict__ vals) {
    const int lane = threadIdx.x & 31;
    float acc = 0.f;
    for (long long q = rowptr[row] + lane; q < rowptr[row + 1]; q += 32)
        acc = fmaf(vals[q], to_acc(v[(size_t)colind[q] * B + r]), acc);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    return acc;
}

template <class T>
__global__ void __launch_bounds__(256) k_pivot_rows_psf(const T* __restrict__ vbase, long long ldv,
                                                         const DevState* __restrict__ st, const int* __restrict__ piv,
                                                         int H, int W, const float* __restrict__ psf, int ph, int pw,
                                                         float* __restrict__ gout) {
    // two pivot rows per CTA (8 warps, kPivParts per row)
    __shared__ float s_part[8];
    const int j = st->j;
    const int i0 = blockIdx.x * 2;
    if (j < 0 || i0 > j || st->status[0] != IPF_OK) return;          // uniform
    const int warp = threadIdx.x >> 5;
    const int i = i0 + warp / kPivParts;
    const T* v = vbase + (size_t)j * ldv;
    float acc = 0.f;
    if (i <= j) acc = pivot_row_psf_part<T>(v, piv[i], H, W, psf, ph, pw, warp % kPivParts);
    if ((threadIdx.x & 31) == 0) s_part[warp] = acc;
    __syncthreads();
    if (threadIdx.x < 2 && i0 + (int)threadIdx.x <= j) gout[i0 + threadIdx.x] = pivot_parts_sum(s_part + kPivParts * threadIdx.x);
}

template <class T>
__global__ void __launch_bounds__(256) k_pivot_rows_csr(const T* __restrict__ vbase, long long ldv,
                                                         const DevState* __restrict__ st, const int* __restrict__ piv,
                                                         int B, int K1, const long long* __restrict__ rowptr,
                                                         const int* __restrict__ colind, const float* __restrict__ vals,
                                                         float* __restrict__ gout) {
    const int j = st->j;
    const int wid = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int i = wid / B, r = wid - (wid / B) * B;
    if (j < 0 || i > j || r >= B || st->status[r] != IPF_OK) return;
    const T* v = vbase + (size_t)j * ldv;
    const float acc = pivot_row_csr<T>(v, piv[(size_t)r * K1 + i], B, r, rowptr, colind, vals);
    if ((threadIdx.x & 31) == 0) gout[(size_t)r * K1 + i] = acc;
}

__global__ void k_interleave(const float* __restrict__ src, float* __restrict__ dst, long long n, int B, int dir) {
    const long long N = n * B;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
        const long long i = e / B;
        const int r = (int)(e - i * B);
        if (dir == 0) dst[e] = src[(size_t)r * n + i];
        else dst[(size_t)r * n + i] = src[e];
    }
}

}  // namespace

cudaError_t launch_pivot_rows(const OpDev& op, int storage, const void* vbase, long long ldv, const DevState* st,
                              const int* piv, int B, int k_max, float* gout, cudaStream_t s) {
    const int K1 = k_max + 1;
    const int warps = K1 * (op.kind == IPF_OP_CSR ? B : 1);
    const int blocks = (warps + 7) / 8;
    auto go = [&](auto tag) -> cudaError_t {
        using T = decltype(tag);
        if (op.kind == IPF_OP_PSF2D)
            k_pivot_rows_psf<T><<<(K1 + 1) / 2, 256, 0, s>>>((const T*)vbase, ldv, st, piv, op.rows, op.cols, op.psf,
                                                             op.ph, op.pw, gout);
        else if (op.kind == IPF_OP_CSR)
            k_pivot_rows_csr<T><<<blocks, 256, 0, s>>>((const T*)vbase, ldv, st, piv, B, K1, op.rowptr, op.colind,
                                                       op.vals, gout);
        else
            return cudaErrorInvalidValue;
        return cudaGetLastError();
    };
    switch (storage) {
        case IPF_STORE_F32: return go(float());
        case IPF_STORE_BF16: return go(__nv_bfloat16());
        case IPF_STORE_F16: return go(__half());
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_op_apply(const OpDev& op, int storage, const void* vbase, long long ldv, long long vcols,
                            const int* jptr, int B, void* w, int* err, cudaStream_t s) {
    switch (storage) {
        case IPF_STORE_F64: return apply_T<double>(op, vbase, ldv, vcols, jptr, w, B, err, s);
        case IPF_STORE_F32: return apply_T<float>(op, vbase, ldv, vcols, jptr, w, B, err, s);
        case IPF_STORE_BF16: return apply_T<__nv_bfloat16>(op, vbase, ldv, vcols, jptr, w, B, err, s);
        case IPF_STORE_F16: return apply_T<__half>(op, vbase, ldv, vcols, jptr, w, B, err, s);
        default: return cudaErrorInvalidValue;
    }
}

// plain float32 vectors, RHS-major (input r*n + i, output r*m + i), for the
// standalone apply call
cudaError_t launch_op_apply_f32_plain(const OpDev& op, const float* v, float* w, int nrhs, cudaStream_t s) {
    const bool csr = op.kind == IPF_OP_CSR;
    const long long n = csr ? (long long)op.cols : (long long)op.rows * op.cols;
    const long long m = csr ? (long long)op.rows : n;
    if (nrhs == 1 || !csr) {
        for (int r = 0; r < nrhs; ++r) {
            cudaError_t e = apply_T<float>(op, v + (size_t)r * n, 0, 1, nullptr, w + (size_t)r * m, 1, nullptr, s);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    // CSR with several RHS: interleave into scratch, one product, de-interleave
    float* tmp = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&tmp, sizeof(float) * (size_t)(n + m) * nrhs, s);
    if (e != cudaSuccess) return e;
    float* vi = tmp;
    float* wi = tmp + (size_t)n * nrhs;
    const int blocks = 1024;
    k_interleave<<<blocks, 256, 0, s>>>(v, vi, n, nrhs, 0);
    e = apply_T<float>(op, vi, 0, 1, nullptr, wi, nrhs, nullptr, s);
    if (e == cudaSuccess) k_interleave<<<blocks, 256, 0, s>>>(wi, w, m, nrhs, 1);
    cudaError_t e2 = cudaFreeAsync(tmp, s);
    return e != cudaSuccess ? e : (e2 != cudaSuccess ? e2 : cudaGetLastError());
}

// ------------------------------------------------------------------------
// batched step: the products of every active slot of the work list whose
// operator is a PSF on the FMA column path (kw 7, 15, 31) or a CSR matrix,
// in one launch of 128-thread CTAs over the (slot, tile) table: a PSF tile
// is one 128 x 16 output tile of k_conv2d_c2, a CSR tile kBatchCsrRows rows
// of k_csr.  Same per-output arithmetic as those kernels.
// ------------------------------------------------------------------------
namespace {

template <class T>
__global__ void __launch_bounds__(128, 7) kb_operator(const SlotDesc* __restrict__ slots,
                                                      const TileRef* __restrict__ tiles, int ntiles) {
    __shared__ int s_j;
    for (int tt = blockIdx.x; tt < ntiles; tt += gridDim.x) {
        const TileRef tr = tiles[tt];
        const SlotDesc* sd = slots + tr.slot;
        const int j = slot_step(sd, &s_j);
        if (j < 0) continue;
        const T* v = (const T*)sd->bf.V + (size_t)j * sd->g.ldv;
        float* w = (float*)sd->bf.w;
        const OpDev& op = sd->op;
        if (op.kind == IPF_OP_CSR) {
            const long long r0 = (long long)tr.tile * kBatchCsrRows;
            const long long r1 = min((long long)op.rows, r0 + kBatchCsrRows);
            csr_rows<T, float, 1>(op.rowptr, op.colind, op.vals, v, w, r0 + threadIdx.x / 32, r1, blockDim.x / 32);
        } else {
            const int bx = tr.tile % sd->conv_cols, by = tr.tile / sd->conv_cols;
            switch (op.kw) {
                case 7: conv_c2_tile<T, 7, 16>(v, w, op.rows, op.cols, op.psf_pairs, bx, by); break;
                case 15: conv_c2_tile<T, 15, 16>(v, w, op.rows, op.cols, op.psf_pairs, bx, by); break;
                default: conv_c2_tile<T, 31, 16>(v, w, op.rows, op.cols, op.psf_pairs, bx, by); break;
            }
        }
    }
}

// (A v_j)(p_i), i <= j, of every active slot: tile t of a slot holds the
// the arithmetic of k_pivot_rows_*: tile t is CSR pivots 8t .. 8t + 7, a
// warp each, or PSF pivots 2t, 2t + 1, kPivParts warps each
template <class T>
__global__ void __launch_bounds__(256) kb_pivot_rows(const SlotDesc* __restrict__ slots,
                                                     const TileRef* __restrict__ tiles, int ntiles) {
    __shared__ int s_j;
    __shared__ float s_part[8];
    const int warp = threadIdx.x >> 5;
    for (int tt = blockIdx.x; tt < ntiles; tt += gridDim.x) {
        const TileRef tr = tiles[tt];
        const SlotDesc* sd = slots + tr.slot;
        const int j = slot_step(sd, &s_j);
        if (j < 0) continue;
        const T* v = (const T*)sd->bf.V + (size_t)j * sd->g.ldv;
        const OpDev& op = sd->op;
        if (op.kind == IPF_OP_CSR) {
            const int i = tr.tile * 8 + warp;
            if (i > j) continue;                           // uniform per warp
            const float acc = pivot_row_csr<T>(v, sd->bf.piv[i], 1, 0, op.rowptr, op.colind, op.vals);
            if ((threadIdx.x & 31) == 0) sd->bf.gpiv[i] = acc;
            continue;
        }
        const int i0 = tr.tile * 2;
        if (i0 > j) continue;                              // uniform
        const int i = i0 + warp / kPivParts;
        float acc = 0.f;
        if (i <= j) acc = pivot_row_psf_part<T>(v, sd->bf.piv[i], op.rows, op.cols, op.psf, op.ph, op.pw,
                                                warp % kPivParts);
        if ((threadIdx.x & 31) == 0) s_part[warp] = acc;
        __syncthreads();
        if (threadIdx.x < 2 && i0 + (int)threadIdx.x <= j)
            sd->bf.gpiv[i0 + threadIdx.x] = pivot_parts_sum(s_part + kPivParts * threadIdx.x);
        // (the next tile's slot_step starts with a barrier before s_part is reused)
    }
}

// CSR products of up to kCsrGroup slots that share one matrix.  A group's
// record (kCsrGroupRec ints): the count, the slots, and the byte offset of
// its staging rows in the engine's staging buffer (low, high word).  Step 1,
// kb_csr_stage: v_j of every slot of the group gathered into rows of
// kCsrGroup values, row c = (v_{q}(c), q < kCsrGroup) (zero where a slot is
// absent or idle), so that step 2 reads one row of 2 kCsrGroup bytes (4
// kCsrGroup for FP32) per nonzero for all slots instead of one scattered
// value per slot.
struct CsrGroupView {
    int count;
    const int* slot;
    size_t off;
};
__device__ __forceinline__ CsrGroupView csr_group(const int* groups, int g) {
    const int* rec = groups + (size_t)g * kCsrGroupRec;
    CsrGroupView v;
    v.count = rec[0];
    v.slot = rec + 1;
    v.off = (size_t)(unsigned)rec[kCsrGroup + 1] | ((size_t)(unsigned)rec[kCsrGroup + 2] << 32);
    return v;
}

// the step of each slot of a group, -1 where the slot does not step
__device__ __forceinline__ void csr_group_steps(const SlotDesc* slots, const CsrGroupView& gv, int* s_j) {
    if (threadIdx.x < kCsrGroup) {
        int j = -1;
        if ((int)threadIdx.x < gv.count) {
            const SlotDesc* sd = slots + gv.slot[threadIdx.x];
            if (sd->k_target > 0) {
                const DevState* st = sd->bf.st;
                j = st->j;
                if (st->status[0] != IPF_OK || j >= sd->k_target || j >= sd->g.k_max) j = -1;
            }
        }
        s_j[threadIdx.x] = j;
    }
}

// tile t of a group: staging rows 1024 t .. 1024 t + 1023
template <class T>
__global__ void __launch_bounds__(256) kb_csr_stage(const SlotDesc* __restrict__ slots, const int* __restrict__ groups,
                                                    unsigned char* __restrict__ stage,
                                                    const TileRef* __restrict__ tiles, int ntiles) {
    __shared__ int s_j[kCsrGroup];
    for (int tt = blockIdx.x; tt < ntiles; tt += gridDim.x) {
        const TileRef tr = tiles[tt];
        const CsrGroupView gv = csr_group(groups, tr.slot);
        __syncthreads();
        csr_group_steps(slots, gv, s_j);
        __syncthreads();
        const long long ncols = slots[gv.slot[0]].op.cols;
        T* rows = (T*)(stage + gv.off);
        const long long c0 = (long long)tr.tile * 1024;
        const long long c1 = min(ncols, c0 + 1024);
        for (long long c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
            T vals[kCsrGroup];
#pragma unroll
            for (int q = 0; q < kCsrGroup; ++q) {
                vals[q] = from_acc<T>(0.f);
                if (q < gv.count && s_j[q] >= 0) {
                    const SlotDesc* sd = slots + gv.slot[q];
                    vals[q] = ((const T*)sd->bf.V)[(size_t)s_j[q] * sd->g.ldv + c];
                }
            }
            // the row: kCsrGroup values, 16 bytes at a time
            constexpr int PER = 16 / sizeof(T);
            uint4* dst = reinterpret_cast<uint4*>(rows + (size_t)c * kCsrGroup);
#pragma unroll
            for (int h = 0; h < kCsrGroup / PER; ++h) {
                union { uint4 u; T t[PER]; } pk;
#pragma unroll
                for (int q = 0; q < PER; ++q) pk.t[q] = vals[h * PER + q];
                dst[h] = pk.u;
            }
        }
    }
}

// tile t of a group = its rows 16t .. 16t + 15, one warp per row; a row's
// nonzeros are loaded once for all slots of the group, each with one
// staging row, and each slot's sum runs over them in the order of csr_rows
// (lane-strided, then the same shuffle tree), so a slot gets the same bits
// as alone
template <class T>
__global__ void __launch_bounds__(128) kb_csr_group(const SlotDesc* __restrict__ slots,
                                                    const int* __restrict__ groups,
                                                    const unsigned char* __restrict__ stage,
                                                    const TileRef* __restrict__ tiles, int ntiles) {
    __shared__ int s_j[kCsrGroup];
    for (int tt = blockIdx.x; tt < ntiles; tt += gridDim.x) {
        const TileRef tr = tiles[tt];
        const CsrGroupView gv = csr_group(groups, tr.slot);
        __syncthreads();
        csr_group_steps(slots, gv, s_j);
        __syncthreads();
        const int ng = gv.count;
        const OpDev& op = slots[gv.slot[0]].op;
        const T* rows = (const T*)(stage + gv.off);
        const long long r0 = (long long)tr.tile * kBatchCsrRows;
        const long long r1 = min((long long)op.rows, r0 + kBatchCsrRows);
        const int lane = threadIdx.x & 31;
        for (long long row = r0 + threadIdx.x / 32; row < r1; row += blockDim.x / 32) {
            const long long b0 = op.rowptr[row], b1 = op.rowptr[row + 1];
            float P[kCsrGroup];
#pragma unroll
            for (int q = 0; q < kCsrGroup; ++q) P[q] = 0.f;
            // U chunks of 32 nonzeros per pass: every index, value and staged
            // row of the pass is requested before the first FMA (the loads of
            // a chunk depend on its column index), and each lane still adds
            // its nonzeros b0 + lane, b0 + lane + 32, ... in that order
            constexpr int PER = 16 / sizeof(T);
            constexpr int NH = kCsrGroup / PER;
            constexpr int U = 4;
            for (long long base = b0; base < b1; base += 32 * U) {
                float a[U];
                int c[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const long long pq = base + 32 * u + lane;
                    c[u] = pq < b1 ? op.colind[pq] : -1;
                    a[u] = pq < b1 ? op.vals[pq] : 0.f;
                }
                uint4 rv[U][NH];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const uint4* src = reinterpret_cast<const uint4*>(rows + (size_t)(c[u] < 0 ? 0 : c[u]) * kCsrGroup);
#pragma unroll
                    for (int h = 0; h < NH; ++h) rv[u][h] = c[u] >= 0 ? src[h] : make_uint4(0, 0, 0, 0);
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (c[u] < 0) continue;
#pragma unroll
                    for (int h = 0; h < NH; ++h) {
                        union { uint4 u4; T t[PER]; } pk;
                        pk.u4 = rv[u][h];
#pragma unroll
                        for (int q = 0; q < PER; ++q) P[h * PER + q] = fmaf(a[u], to_acc(pk.t[q]), P[h * PER + q]);
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < kCsrGroup; ++q) {
                if (q >= ng || s_j[q] < 0) continue;             // uniform for the warp
                float acc = P[q];
#pragma unroll
                for (int o = 16; o >= 1; o >>= 1) acc = acc + __shfl_xor_sync(0xffffffffu, acc, o);
                if (lane == 0) ((float*)slots[gv.slot[q]].bf.w)[row] = acc;
            }
        }
    }
}

}  // namespace

cudaError_t launch_batch_csr_group(int storage, const SlotDesc* slots, const int* groups, unsigned char* stage,
                                   const TileRef* stage_tiles, int nstage, const TileRef* tiles, int ntiles,
                                   int num_sms, cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    const int sb = nstage < num_sms * 8 ? nstage : num_sms * 8;
    const int blocks = ntiles < num_sms * 8 ? ntiles : num_sms * 8;
    switch (storage) {
        case IPF_STORE_F32:
            kb_csr_stage<float><<<sb, 256, 0, s>>>(slots, groups, stage, stage_tiles, nstage);
            kb_csr_group<float><<<blocks, 128, 0, s>>>(slots, groups, stage, tiles, ntiles);
            break;
        case IPF_STORE_BF16:
            kb_csr_stage<__nv_bfloat16><<<sb, 256, 0, s>>>(slots, groups, stage, stage_tiles, nstage);
            kb_csr_group<__nv_bfloat16><<<blocks, 128, 0, s>>>(slots, groups, stage, tiles, ntiles);
            break;
        case IPF_STORE_F16:
            kb_csr_stage<__half><<<sb, 256, 0, s>>>(slots, groups, stage, stage_tiles, nstage);
            kb_csr_group<__half><<<blocks, 128, 0, s>>>(slots, groups, stage, tiles, ntiles);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_batch_pivot_rows(int storage, const SlotDesc* slots, const TileRef* tiles, int ntiles, int num_sms,
                                    cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    const int blocks = ntiles < num_sms * 8 ? ntiles : num_sms * 8;
    switch (storage) {
        case IPF_STORE_F32: kb_pivot_rows<float><<<blocks, 256, 0, s>>>(slots, tiles, ntiles); break;
        case IPF_STORE_BF16: kb_pivot_rows<__nv_bfloat16><<<blocks, 256, 0, s>>>(slots, tiles, ntiles); break;
        case IPF_STORE_F16: kb_pivot_rows<__half><<<blocks, 256, 0, s>>>(slots, tiles, ntiles); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_batch_operator(int storage, const SlotDesc* slots, const TileRef* tiles, int ntiles, int num_sms,
                                  cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    // the largest tile of conv_c2_tile: (16 + 30) x (128 + 31) floats for kw 31
    const size_t smem = (size_t)(16 + 31 - 1) * (128 + 31) * sizeof(float);
    const int blocks = ntiles < num_sms * 7 ? ntiles : num_sms * 7;
    switch (storage) {
        case IPF_STORE_F32: kb_operator<float><<<blocks, 128, smem, s>>>(slots, tiles, ntiles); break;
        case IPF_STORE_BF16: kb_operator<__nv_bfloat16><<<blocks, 128, smem, s>>>(slots, tiles, ntiles); break;
        case IPF_STORE_F16: kb_operator<__half><<<blocks, 128, smem, s>>>(slots, tiles, ntiles); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace ipf
