// api.cu -- C ABI compute entry points: gint_vlocal, gint_rho, gint_force_stress.
// Host-side validation, then enqueue on the caller's stream.
#include <algorithm>

#include "gint_impl.cuh"

namespace gint {
gint_status simt_run(gint_handle* h, int which, bool fp32, const double* V, const double* D, double* out,
                     double* acc, double* acc_e, cudaStream_t st);
gint_status launch_mirror(gint_handle* h, double* H, cudaStream_t st);
gint_status launch_rho_empty(gint_handle* h, double* rho, cudaStream_t st);
gint_status launch_force_finalize(gint_handle* h, double* F, double* sigma, double* virial, double* E,
                                  cudaStream_t st);
gint_status tc_vlocal(gint_handle* h, int form, const double* V, double* H, int accumulate, cudaStream_t st);
gint_status tc_vlocal_check(const gint_handle* h, int form);
gint_status tc_rhoforce_check(const gint_handle* h);
gint_status tc_rhoforce(gint_handle* h, int form, bool force, const double* V, const double* D, double* rho,
                        double* facc, double* acc_e, cudaStream_t st);

namespace {
// Selects the handle's device for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// FP64: SIMT FP64.  FP32: SIMT FP32.  BF16X3 / FP16X3: tensor cores (split
// 16-bit operands, three products, FP32 accumulation per brick).  FP16X4:
// tensor cores with an exactly accumulated 8-bit fixed-point leading product.
bool is_tc(const gint_handle* h) {
    return h->precision == GINT_BF16X3 || h->precision == GINT_FP16X3 || h->precision == GINT_FP16X4;
}
int tc_form(const gint_handle* h) { return h->precision == GINT_BF16X3 ? 1 : h->precision == GINT_FP16X4 ? 2 : 0; }
}  // namespace

// Tensor-core form of a handle's precision (0 fp16x3, 1 bf16x3, 2 fp16x4), -1 for the SIMT forms.
int tc_form_of(const gint_handle* h) { return is_tc(h) ? tc_form(h) : -1; }

namespace {

gint_status check_precision(const gint_handle* h, bool* fp32) {
    if (h->precision == GINT_FP64) { *fp32 = false; return GINT_OK; }
    if (h->precision == GINT_FP32 || h->precision == GINT_BF16X3 || h->precision == GINT_FP16X3 ||
        h->precision == GINT_FP16X4) {
        *fp32 = true;
        return GINT_OK;
    }
    set_error("precision %d is not implemented by this build", h->precision);
    return GINT_ERR_UNSUPPORTED;
}
}  // namespace
}  // namespace gint

using namespace gint;

extern "C" {

gint_status gint_vlocal(gint_handle* h, const double* V, double* H, int accumulate, gint_stream stream) {
    set_error("");
    if (!h || !V || !H) { set_error("gint_vlocal: NULL argument"); return GINT_ERR_INVALID_ARG; }
    if (accumulate != 0 && accumulate != 1) { set_error("gint_vlocal: accumulate must be 0 or 1"); return GINT_ERR_INVALID_ARG; }
    bool fp32 = false;
    gint_status s = check_precision(h, &fp32);
    if (s != GINT_OK) return s;
    DeviceGuard dg(h->device);
    if (!dg.ok) { set_error("cannot select device %d", h->device); return GINT_ERR_CUDA; }
    cudaStream_t st = (cudaStream_t)stream;
    if (!accumulate && h->n_values > 0) GINT_CUDA_TRY(cudaMemsetAsync(H, 0, sizeof(double) * h->n_values, st));
    if (is_tc(h))
        s = tc_vlocal(h, tc_form(h), V, H, accumulate, st);
    else
        s = simt_run(h, 0, fp32, V, nullptr, H, nullptr, nullptr, st);
    if (s != GINT_OK) return s;
    return launch_mirror(h, H, st);
}

gint_status gint_check(const gint_handle* h) {
    set_error("");
    if (!h) { set_error("gint_check: NULL handle"); return GINT_ERR_INVALID_ARG; }
    bool fp32 = false;
    gint_status s = check_precision(h, &fp32);
    if (s != GINT_OK || !is_tc(h)) return s;
    s = tc_vlocal_check(h, tc_form(h));
    if (s != GINT_OK) return s;
    return tc_rhoforce_check(h);
}

gint_status gint_rho(gint_handle* h, const double* D, double* rho, gint_stream stream) {
    set_error("");
    if (!h || !D || !rho) { set_error("gint_rho: NULL argument"); return GINT_ERR_INVALID_ARG; }
    bool fp32 = false;
    gint_status s = check_precision(h, &fp32);
    if (s != GINT_OK) return s;
    DeviceGuard dg(h->device);
    if (!dg.ok) { set_error("cannot select device %d", h->device); return GINT_ERR_CUDA; }
    cudaStream_t st = (cudaStream_t)stream;
    if (is_tc(h))
        s = tc_rhoforce(h, tc_form(h), false, nullptr, D, rho, nullptr, nullptr, st);
    else
        s = simt_run(h, 1, fp32, nullptr, D, rho, nullptr, nullptr, st);
    if (s != GINT_OK) return s;
    return launch_rho_empty(h, rho, st);
}

gint_status gint_force_stress(gint_handle* h, const double* V, const double* D, double* F, double* sigma,
                              double* virial_atom, double* E, gint_stream stream) {
    set_error("");
    if (!h || !V || !D) { set_error("gint_force_stress: NULL argument"); return GINT_ERR_INVALID_ARG; }
    if (!F && !sigma && !virial_atom && !E) { set_error("gint_force_stress: no output requested"); return GINT_ERR_INVALID_ARG; }
    bool fp32 = false;
    gint_status s = check_precision(h, &fp32);
    if (s != GINT_OK) return s;
    DeviceGuard dg(h->device);
    if (!dg.ok) { set_error("cannot select device %d", h->device); return GINT_ERR_CUDA; }
    cudaStream_t st = (cudaStream_t)stream;
    GINT_CUDA_TRY(cudaMemsetAsync(h->d_facc, 0, sizeof(double) * 12 * h->n_atoms, st));
    GINT_CUDA_TRY(cudaMemsetAsync(h->d_red, 0, sizeof(double), st));
    if (is_tc(h))
        s = tc_rhoforce(h, tc_form(h), true, V, D, nullptr, h->d_facc, h->d_red, st);
    else
        s = simt_run(h, 2, fp32, V, D, nullptr, h->d_facc, h->d_red, st);
    if (s != GINT_OK) return s;
    return launch_force_finalize(h, F, sigma, virial_atom, E, st);
}

}  // extern "C"
