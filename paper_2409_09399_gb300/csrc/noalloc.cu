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
// library image (kStaticScratchBytes per GPU, reserved when gint_setup first
// runs on that GPU and held until the process exits) and calls no allocating
// routine.
#include "gint_impl.cuh"

namespace gint {

gint_status simt_vlocal_on_scratch(gint_handle* h, const double* V, double* H, char* scratch, size_t cta_stride,
                                   int n_ctas, cudaStream_t st);
gint_status launch_mirror(gint_handle* h, double* H, cudaStream_t st);

constexpr size_t kStaticScratchBytes = size_t(64) << 20;  // 64 MiB on every GPU that maps the array

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch on the current device.  Called by gint_setup, with the
// handle's device current, so that the module holding the array is loaded (and its 64 MiB
// reserved) at set-up, where allocating is allowed, rather than by the first
// gint_vlocal_static.  In host code the symbol itself is only a stand-in for that address.
gint_status static_scratch_resolve(void** out) {
    *out = nullptr;
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
        set_error("cudaGetSymbolAddress of the static scratch array failed: %s", cudaGetErrorString(e));
        return GINT_ERR_CUDA;
    }
    *out = p;
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
    void* scratch = h->d_static;  // resolved by gint_setup on this device
    if (!scratch) {
        set_error("gint_vlocal_static: the static scratch array was not mapped when the handle was set up");
        s = GINT_ERR_CUDA;
    }
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
