// The Gaussian sketch (Sec. 2; the embedding of the paper's experiments):
// S (m_s x n) with N(0, 1/m_s) entries, drawn once per context from the
// SplitMix64 counter hash by the Box-Muller transform (Box & Muller 1958):
// entry (r, i) takes outputs 2c and 2c+1, c = r*n + i, of the generator
// started at the seed; u = ((out >> 11) + 1) * 2^-53 in (0, 1];
// z = sqrt(-2 ln u1) cos(2 pi u2); S[r, i] = z / sqrt(m_s), rounded to the
// storage type of the basis.  S is kept column-major (element (r, i) at
// r + i*m_s), so S V_{k+1} is one dense GEMM with the basis (leading
// dimension ldv), done at solve time by cuBLAS; c = S b is a reduction in
// a fixed order (FP32 runs of products added into FP64 sums).  cuBLAS is
// loaded on first use (dlopen), so the library does not depend on it unless
// the Gaussian sketch is asked for.
#include <cublas_v2.h>
#include <dlfcn.h>

#include <mutex>
#include <type_traits>

#include "ipf_internal.cuh"

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

// flat element t of S (column-major, t = r + i*m) walks with a carried
// (r, i) instead of a 64-bit division per element; the counter is c = r*n + i
template <class T>
__global__ void __launch_bounds__(256) k_gauss_fill(T* __restrict__ S, long long n, int m, unsigned long long seed,
                                                    double sqrt_m, float inv_sqrt_m) {
    const long long total = n * (long long)m;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long sr = stride % m, si = stride / m;
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long i = t / m, r = t - i * m;
    for (; t < total; t += stride) {
        const unsigned long long c = (unsigned long long)(r * n + i);
        const unsigned long long o1 = sm64_mix(seed + kGamma * (2ull * c + 1ull));
        const unsigned long long o2 = sm64_mix(seed + kGamma * (2ull * c + 2ull));
        if constexpr (sizeof(T) == 2) {
            unsigned short bits;
            if (!gauss_fast<T>(o1, o2, inv_sqrt_m, bits)) {
                const double v = gauss_f64(o1, o2, sqrt_m);
                if constexpr (std::is_same<T, __half>::value) bits = __half_as_ushort(__double2half(v));
                else bits = store_bits<T>((float)v);                 // FP64 -> FP32 -> BF16
            }
            reinterpret_cast<unsigned short*>(S)[t] = bits;
        } else {
            S[t] = (T)gauss_f64(o1, o2, sqrt_m);
        }
        r += sr;
        i += si;
        if (r >= m) {
            r -= m;
            i += 1;
        }
    }
}

// c = S b with a fixed summation order, in two passes.  Pass 1: CTA q takes
// the columns [q*n/Q, (q+1)*n/Q); a column of S is cut into vectors of V
// consecutive rows (16 bytes when the column is 16-byte aligned, else single
// rows), thread t owns vector t % mv of every column i = i0 + t / mv (mod
// cpi), so each load is one contiguous piece of a column.  Products are
// summed in FP32 over runs of kRun of the thread's columns (FP64 for F64
// storage: every product) and each run sum is added to an FP64 sum; the
// thread's sums go to part[(q * cpi + phase) * m + row].  Pass 2 adds the
// Q * cpi partial sums of each row in order.
constexpr int kRun = 32;

template <class T> struct RhsAcc { using type = float; };
template <> struct RhsAcc<double> { using type = double; };

template <class T, int V>
__global__ void __launch_bounds__(256) k_gauss_rhs_part(const T* __restrict__ S, const float* __restrict__ b,
                                                        long long n, int m, int mv, int cpi,
                                                        double* __restrict__ part) {
    using A = typename RhsAcc<T>::type;
    const int q = blockIdx.x;
    const long long i0 = n * q / kGaussRhsSlices, i1 = n * (q + 1) / kGaussRhsSlices;
    const int phase = mv <= (int)blockDim.x ? threadIdx.x / mv : 0;
    if (phase >= cpi) return;
    const int vr0 = mv <= (int)blockDim.x ? threadIdx.x % mv : threadIdx.x;
    const int vstep = mv <= (int)blockDim.x ? mv : blockDim.x;
    double* out = part + ((size_t)q * cpi + phase) * m;
    for (int vr = vr0; vr < mv; vr += vstep) {
        double tot[V];
#pragma unroll
        for (int e = 0; e < V; ++e) tot[e] = 0.0;
        long long i = i0 + phase;
        while (i < i1) {
            A run[V];
#pragma unroll
            for (int e = 0; e < V; ++e) run[e] = A(0);
#pragma unroll 4
            for (int c = 0; c < kRun; ++c) {
                if (i >= i1) break;
                const T* col = S + i * (long long)m + (long long)vr * V;
                const A bi = (A)__ldg(b + i);
                if constexpr (V > 1) {
                    union { uint4 u; T t[V]; } ld;
                    ld.u = __ldg(reinterpret_cast<const uint4*>(col));
#pragma unroll
                    for (int e = 0; e < V; ++e) run[e] = fma((A)to_acc(ld.t[e]), bi, run[e]);
                } else {
                    run[0] = fma((A)to_acc(col[0]), bi, run[0]);
                }
                i += cpi;
            }
#pragma unroll
            for (int e = 0; e < V; ++e) tot[e] += (double)run[e];
        }
#pragma unroll
        for (int e = 0; e < V; ++e) out[vr * V + e] = tot[e];
    }
}

__global__ void k_gauss_rhs_sum(const double* __restrict__ part, int nparts, int m, double* __restrict__ c) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= m) return;
    double t = 0.0;
    for (int q = 0; q < nparts; ++q) t += part[(size_t)q * m + r];
    c[r] = t;
}

template <class T>
cudaError_t rhs_typed(const T* S, const float* b, long long n, int m, double* c, double* part, cudaStream_t s) {
    constexpr int V = 16 / (int)sizeof(T);
    const bool vec = ((size_t)m * sizeof(T)) % 16 == 0 && ((uintptr_t)S & 15) == 0;
    const int mv = vec ? m / V : m;
    const int cpi = mv <= 256 ? 256 / mv : 1;
    if (vec) k_gauss_rhs_part<T, V><<<kGaussRhsSlices, 256, 0, s>>>(S, b, n, m, mv, cpi, part);
    else k_gauss_rhs_part<T, 1><<<kGaussRhsSlices, 256, 0, s>>>(S, b, n, m, mv, cpi, part);
    k_gauss_rhs_sum<<<(m + 255) / 256, 256, 0, s>>>(part, kGaussRhsSlices * cpi, m, c);
    return cudaGetLastError();
}

// cuBLAS entry points, resolved once
struct Blas {
    bool ok = false;
    cublasStatus_t (*create)(cublasHandle_t*) = nullptr;
    cublasStatus_t (*destroy)(cublasHandle_t) = nullptr;
    cublasStatus_t (*set_stream)(cublasHandle_t, cudaStream_t) = nullptr;
    cublasStatus_t (*gemm_ex)(cublasHandle_t, cublasOperation_t, cublasOperation_t, int, int, int, const void*,
                              const void*, cudaDataType, int, const void*, cudaDataType, int, const void*, void*,
                              cudaDataType, int, cublasComputeType_t, cublasGemmAlgo_t) = nullptr;
};

Blas& blas() {
    static Blas b;
    static std::once_flag once;
    std::call_once(once, [] {
        const char* names[] = {"libcublas.so.13", "/usr/local/cuda/lib64/libcublas.so.13", "libcublas.so"};
        void* h = nullptr;
        for (const char* nm : names)
            if ((h = dlopen(nm, RTLD_NOW | RTLD_LOCAL)) != nullptr) break;
        if (!h) return;
        b.create = (decltype(b.create))dlsym(h, "cublasCreate_v2");
        b.destroy = (decltype(b.destroy))dlsym(h, "cublasDestroy_v2");
        b.set_stream = (decltype(b.set_stream))dlsym(h, "cublasSetStream_v2");
        b.gemm_ex = (decltype(b.gemm_ex))dlsym(h, "cublasGemmEx");
        b.ok = b.create && b.destroy && b.set_stream && b.gemm_ex;
    });
    return b;
}

}  // namespace

cudaError_t launch_gauss_fill(int storage, void* S, long long n, int m, unsigned long long seed, int num_sms,
                              cudaStream_t s) {
    if (n <= 0 || m <= 0) return cudaSuccess;
    const int blocks = num_sms * 8;
    const double sm = sqrt((double)m);
    const float inv = (float)(1.0 / sm);
    switch (storage) {
        case IPF_STORE_F64: k_gauss_fill<double><<<blocks, 256, 0, s>>>((double*)S, n, m, seed, sm, inv); break;
        case IPF_STORE_F32: k_gauss_fill<float><<<blocks, 256, 0, s>>>((float*)S, n, m, seed, sm, inv); break;
        case IPF_STORE_BF16:
            k_gauss_fill<__nv_bfloat16><<<blocks, 256, 0, s>>>((__nv_bfloat16*)S, n, m, seed, sm, inv);
            break;
        case IPF_STORE_F16: k_gauss_fill<__half><<<blocks, 256, 0, s>>>((__half*)S, n, m, seed, sm, inv); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_gauss_rhs(int storage, const void* S, const float* b, long long n, int m, double* c,
                             double* part, cudaStream_t s) {
    switch (storage) {
        case IPF_STORE_F64: return rhs_typed((const double*)S, b, n, m, c, part, s);
        case IPF_STORE_F32: return rhs_typed((const float*)S, b, n, m, c, part, s);
        case IPF_STORE_BF16: return rhs_typed((const __nv_bfloat16*)S, b, n, m, c, part, s);
        case IPF_STORE_F16: return rhs_typed((const __half*)S, b, n, m, c, part, s);
        default: return cudaErrorInvalidValue;
    }
}

void* gauss_blas_create() {
    Blas& b = blas();
    if (!b.ok) return nullptr;
    cublasHandle_t h = nullptr;
    if (b.create(&h) != CUBLAS_STATUS_SUCCESS) return nullptr;
    return (void*)h;
}

void gauss_blas_destroy(void* h) {
    if (h && blas().ok) blas().destroy((cublasHandle_t)h);
}

// out (m x K, column-major; FP64 for F64 storage, else FP32) = S (m x n) V (n x K, leading dimension ldv)
cudaError_t launch_gauss_sv(void* handle, int storage, const void* S, int m, long long n, const void* V,
                            long long ldv, int K, void* out, cudaStream_t s) {
    Blas& b = blas();
    if (!b.ok || !handle) return cudaErrorNotSupported;
    cublasHandle_t h = (cublasHandle_t)handle;
    if (b.set_stream(h, s) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
    cudaDataType t;
    switch (storage) {
        case IPF_STORE_F64: t = CUDA_R_64F; break;
        case IPF_STORE_F32: t = CUDA_R_32F; break;
        case IPF_STORE_BF16: t = CUDA_R_16BF; break;
        case IPF_STORE_F16: t = CUDA_R_16F; break;
        default: return cudaErrorInvalidValue;
    }
    const bool f64 = storage == IPF_STORE_F64;
    const double a64 = 1.0, b64 = 0.0;
    const float a32 = 1.f, b32 = 0.f;
    const cublasStatus_t st = b.gemm_ex(h, CUBLAS_OP_N, CUBLAS_OP_N, m, K, (int)n, f64 ? (const void*)&a64 : &a32, S,
                                        t, m, V, t, (int)ldv, f64 ? (const void*)&b64 : &b32, out,
                                        f64 ? CUDA_R_64F : CUDA_R_32F, m,
                                        f64 ? CUBLAS_COMPUTE_64F : CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT);
    return st == CUBLAS_STATUS_SUCCESS ? cudaSuccess : cudaErrorUnknown;
}

}  // namespace ipf
