// noalloc.cu -- gint_vlocal_static: the FP64 H^V call without any device
// allocation.
//
// gint_vlocal takes the scratch of its orbital-value kernel from memory the
// handle allocated with cudaMalloc.  Some callers cannot let a library call
// cudaMalloc at compute time: cudaMalloc synchronises the device and can fail
// when a framework's caching allocator has already reserved the free memory,
// and some host code (schedulers with a fixed memory plan, allocator hooks)
// must not enter the CUDA allocator at all.  gint_vlocal_static runs the same
// FP64 kernel with its scratch in a fixed-size array that is part of the
// library image (kStaticScratchBytes per GPU, held from library load to
// process exit) and calls no allocating routine.
#include <mutex>

#include "gint_impl.cuh"

namespace gint {

gint_status simt_vlocal_on_scratch(gint_handle* h, const double* V, double* H, char* scratch, size_t cta_stride,
                                   int n_ctas, cudaStream_t st);
gint_status launch_mirror(gint_handle* h, double* H, cudaStream_t st);

constexpr size_t kStaticScratchBytes = size_t(64) << 20;  // 64 MiB on every GPU that loads the library
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

static std::mutex g_static_mu;
static void* g_static_addr[kMaxDevices];

// Device address of g_static_scratch on `dev` (which must be current), resolved
// once per device.  In host code the symbol is only a stand-in.
static gint_status static_scratch_address(int dev, void** out) {
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device ordinal %d out of range", dev);
        return GINT_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            set_error("cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
            return GINT_ERR_CUDA;
        }
        g_static_addr[dev] = p;
    }
    *out = g_static_addr[dev];
    return GINT_OK;
}

}  // namespace gint

using namespace gint;

extern "C" gint_status gint_vlocal_static(gint_handle* h, const double* V, double* H, gint_stream stream) {
    set_error("");
    if (!h || !V || !H) {
        set_error("gint_vlocal_static: NULL argument");
        return GINT_ERR_INVALID_ARG;
    }
    const size_t per_cta = (size_t)2 * (size_t)(h->max_brick_orb > 0 ? h->max_brick_orb : 1) * h->grid.bpad * sizeof(double);
    if (per_cta > kStaticScratchBytes) {
        set_error("gint_vlocal_static: a brick needs %zu bytes of scratch, more than the %zu-byte static array; "
                  "use smaller bricks", per_cta, kStaticScratchBytes);
        return GINT_ERR_UNSUPPORTED;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(h->device) != cudaSuccess) {
        set_error("cannot select device %d", h->device);
        return GINT_ERR_CUDA;
    }
    gint_status s = GINT_OK;
    void* scratch = nullptr;
    s = static_scratch_address(h->device, &scratch);
    if (s == GINT_OK) {
        cudaStream_t st = (cudaStream_t)stream;
        const int by_size = (int)(kStaticScratchBytes / per_cta);
        const int n_ctas = by_size < h->n_ctas ? by_size : h->n_ctas;
        cudaError_t e = cudaSuccess;
        if (h->n_values > 0) e = cudaMemsetAsync(H, 0, sizeof(double) * h->n_values, st);
        if (e != cudaSuccess) {
            set_error("cudaMemsetAsync: %s", cudaGetErrorString(e));
            s = GINT_ERR_CUDA;
        }
        if (s == GINT_OK) s = simt_vlocal_on_scratch(h, V, H, (char*)scratch, per_cta, n_ctas, st);
        if (s == GINT_OK) s = launch_mirror(h, H, st);
    }
    if (prev >= 0) cudaSetDevice(prev);
    return s;
}
