// ipf_sketch_apply_noalloc: the standalone sparse-sign sketch y = S x with
// its scratch (the max-|x| word and the exact 64-bit row accumulators) in a
// fixed array of this library's device image instead of memory allocated
// per call.  It runs the same kernels as ipf_sketch_apply.
#include <mutex>

#include "ipf_internal.cuh"

namespace {

constexpr int kNoAllocMaxRows = 4096;                 // largest m_s accepted
constexpr size_t kNoAllocHeader = 256;                // max-|x| word, padded to 256 bytes
constexpr size_t kNoAllocBytes = kNoAllocHeader + sizeof(long long) * kNoAllocMaxRows;

// One copy per GPU that loads the library, kept until the process exits.
// In host code this name is a host-side stand-in, not a device address.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// device address of the scratch array on the current device, looked up once
// per device with that device current
cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        if (!p) return cudaErrorInvalidSymbol;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" ipf_status ipf_sketch_apply_noalloc(const float* x_dev, long long n, int m_s, int zeta,
                                               unsigned long long seed, double* y_dev, void* stream) {
    if (!x_dev || !y_dev || n < 1 || zeta < 1 || zeta > 16 || m_s < zeta) return IPF_ERR_ARG;
    if (m_s > kNoAllocMaxRows) return IPF_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    void* scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) return IPF_ERR_CUDA;
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) != cudaSuccess) return IPF_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return IPF_ERR_CUDA;
    unsigned* amax = (unsigned*)scratch;
    long long* acc = (long long*)((char*)scratch + kNoAllocHeader);
    // the array keeps the previous call's contents: clear the part used here
    if (cudaMemsetAsync(scratch, 0, kNoAllocHeader + sizeof(long long) * (size_t)m_s, s) != cudaSuccess)
        return IPF_ERR_CUDA;
    ipf::SketchParams sp = ipf::make_sketch_params(seed, m_s, zeta);
    cudaError_t e = ipf::launch_sketch_vector(x_dev, n, sp, 0, acc, (float*)amax, s, sms, true);
    if (e == cudaSuccess) e = ipf::launch_sketch_finish(acc, m_s, n, zeta, amax, y_dev, s);
    return e == cudaSuccess ? IPF_OK : IPF_ERR_CUDA;
}
