// The Gaussian sketch (Sec. 2; the embedding of the paper's experiments):
// S (m_s x n) with N(0, 1/m_s) entries, drawn once per context from the
// SplitMix64 counter hash by the Box-Muller transform (Box & Muller 1958):
// entry (r, i) takes outputs 2c and 2c+1, c = r*n + i, of the generator
// started at the seed; u = ((out >> 11) + 1) * 2^-53 in (0, 1];
// z = sqrt(-2 ln u1) cos(2 pi u2); S[r, i] = z / sqrt(m_s), rounded to the
// storage type of the basis.  S is kept column-major (element (r, i) at
// r + i*m_s), so S V_{k+1} is one dense GEMM with the basis (leading
// dimension ldv), done at solve time by cuBLAS; c = S b is a fixed-order
// FP64 reduction per row.  cuBLAS is loaded on first use (dlopen), so the
// library does not depend on it unless the Gaussian sketch is asked for.
#include <cublas_v2.h>
#include <dlfcn.h>

#include <mutex>

#include "ipf_internal.cuh"

namespace ipf {

namespace {

template <class T> __device__ __forceinline__ T from_double(double v);
template <> __device__ __forceinline__ double from_double<double>(double v) { return v; }
template <> __device__ __forceinline__ float from_double<float>(double v) { return (float)v; }
// through FP32, as the oracle rounds: FP64 -> FP32 -> BF16 (nearest even)
template <> __device__ __forceinline__ __nv_bfloat16 from_double<__nv_bfloat16>(double v) {
    return __float2bfloat16_rn((float)v);
}
template <> __device__ __forceinline__ __half from_double<__half>(double v) { return __double2half(v); }

template <class T>
__global__ void k_gauss_fill(T* __restrict__ S, long long n, int m, unsigned long long seed) {
    const long long total = n * (long long)m;
    const double scale = 1.0 / sqrt((double)m);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long i = t / m, r = t - i * m;                 // storage order: r + i*m
        const unsigned long long c = (unsigned long long)(r * n + i);
        const unsigned long long o1 = sm64_mix(seed + kGamma * (2ull * c + 1ull));
        const unsigned long long o2 = sm64_mix(seed + kGamma * (2ull * c + 2ull));
        const double u1 = ((double)(o1 >> 11) + 1.0) * 0x1.0p-53;
        const double u2 = ((double)(o2 >> 11) + 1.0) * 0x1.0p-53;
        const double z = sqrt(-2.0 * log(u1)) * cos(2.0 * 3.141592653589793 * u2);
        S[t] = from_double<T>(z * scale);
    }
}

// c[r] = sum_i S[r, i] b[i] in FP64, one CTA per row, fixed reduction order
template <class T>
__global__ void __launch_bounds__(256) k_gauss_rhs(const T* __restrict__ S, const float* __restrict__ b, long long n,
                                                   int m, double* __restrict__ c) {
    __shared__ double s_red[8];
    const int r = blockIdx.x;
    double acc = 0.0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x)
        acc = fma((double)to_acc(S[r + i * (long long)m]), (double)b[i], acc);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < 8; ++q) t += s_red[q];
        c[r] = t;
    }
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
    const int blocks = num_sms * 8;
    switch (storage) {
        case IPF_STORE_F64: k_gauss_fill<double><<<blocks, 256, 0, s>>>((double*)S, n, m, seed); break;
        case IPF_STORE_F32: k_gauss_fill<float><<<blocks, 256, 0, s>>>((float*)S, n, m, seed); break;
        case IPF_STORE_BF16: k_gauss_fill<__nv_bfloat16><<<blocks, 256, 0, s>>>((__nv_bfloat16*)S, n, m, seed); break;
        case IPF_STORE_F16: k_gauss_fill<__half><<<blocks, 256, 0, s>>>((__half*)S, n, m, seed); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_gauss_rhs(int storage, const void* S, const float* b, long long n, int m, double* c,
                             cudaStream_t s) {
    switch (storage) {
        case IPF_STORE_F64: k_gauss_rhs<double><<<m, 256, 0, s>>>((const double*)S, b, n, m, c); break;
        case IPF_STORE_F32: k_gauss_rhs<float><<<m, 256, 0, s>>>((const float*)S, b, n, m, c); break;
        case IPF_STORE_BF16: k_gauss_rhs<__nv_bfloat16><<<m, 256, 0, s>>>((const __nv_bfloat16*)S, b, n, m, c); break;
        case IPF_STORE_F16: k_gauss_rhs<__half><<<m, 256, 0, s>>>((const __half*)S, b, n, m, c); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
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
