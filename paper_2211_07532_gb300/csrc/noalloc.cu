// aexp_wavelet_prox_static: the wavelet prox step with its scratch in a fixed device array
// owned by the library, for callers that cannot allocate device memory.
//
// The scratch (wavelet pyramid plus the intermediate approximation images) lives in
// g_prox_scratch below, a file-scope device array of kProxStaticBytes.  Every GPU that
// loads the library reserves it until the process exits.  Host code cannot use the
// array's name as a device address, so on the first call on each device (with that
// device current) its address is looked up with cudaGetSymbolAddress and cached.
#include <mutex>

#include "aexp_internal.cuh"

using namespace aexp;

namespace {

constexpr size_t kProxStaticBytes = size_t(4) << 20;  // 4 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_prox_scratch[kProxStaticBytes];

std::mutex g_static_mu;
void *g_static_ptr[kMaxDevices] = {};

// Device address of g_prox_scratch on the current device (looked up once per device).
cudaError_t static_scratch(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_prox_scratch);
        if (e != cudaSuccess) return e;
        g_static_ptr[dev] = p;
    }
    *out = g_static_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" AEXP_API int aexp_wavelet_prox_static(int nx, int ny, int wavelet, int levels, float tau, const void *in,
                                        void *out, void *stream) {
    if (nx < 1 || ny < 1 || levels < 1 || levels > 12) return AEXP_ERR_INVALID_ARG;
    if (wavelet != AEXP_WAVELET_HAAR && wavelet != AEXP_WAVELET_DB4) return AEXP_ERR_INVALID_ARG;
    if (!in || !out || !(tau >= 0.f)) return AEXP_ERR_INVALID_ARG;
    if (((uintptr_t)in % 8) || ((uintptr_t)out % 8)) return AEXP_ERR_MISALIGNED;
    WaveLayout W;
    wave_layout(nx, ny, wavelet, levels, &W);
    if (W.bytes > kProxStaticBytes) return AEXP_ERR_UNSUPPORTED;
    void *scratch = nullptr;
    cudaError_t e = static_scratch(&scratch);
    if (e != cudaSuccess) {
        aexp_set_last_cuda_error((int)e);
        return AEXP_ERR_CUDA;
    }
    // Every scratch byte read below is written earlier in the same call (the level-1 subbands and
    // approximation; the coarser levels live in the CTA's shared memory, or, for images too large
    // for that, in the array as well, each written before it is read), so nothing needs clearing.
    cudaStream_t st = (cudaStream_t)stream;
    e = wave_prox(W, (const float2 *)in, (char *)scratch, tau, nullptr, (float2 *)out, 0, 0.0, nullptr, nullptr, st);
    if (e != cudaSuccess) {
        aexp_set_last_cuda_error((int)e);
        return AEXP_ERR_CUDA;
    }
    return AEXP_OK;
}
