// api.cu -- C ABI compute entry points: gint_vlocal, gint_rho, gint_force_stress.
// Host-side validation, then enqueue on the caller's stream.
#include <algorithm>

#include "gint_impl.cuh"
#include "nvtx.cuh"

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
// Accumulate the Pulay force, the per-atom virial and the energy (Eq. 4, 5) of the handle's
// precision into h->d_facc (12 per atom) and h->d_red[0].
gint_status force_accumulate(gint_handle* h, bool fp32, const double* V, const double* D, cudaStream_t st) {
    if (is_tc(h)) {  // limits first: a rejected call enqueues nothing
        gint_status c = tc_rhoforce_check(h);
        if (c != GINT_OK) return c;
    }
    GINT_CUDA_TRY(cudaMemsetAsync(h->d_facc, 0, sizeof(double) * 12 * h->n_atoms, st));
    GINT_CUDA_TRY(cudaMemsetAsync(h->d_red, 0, sizeof(double), st));
    if (is_tc(h)) return tc_rhoforce(h, tc_form(h), true, V, D, nullptr, h->d_facc, h->d_red, st);
    return simt_run(h, 2, fp32, V, D, nullptr, h->d_facc, h->d_red, st);
}

// x[i] *= c * (*g) (g NULL: 1), grid-stride.
__global__ void k_scale(double* x, int64_t n, double c, const double* g) {
    const double s = c * (g ? *g : 1.0);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] *= s;
}

// Energy gradients from the force accumulators: dE/dR_I = -F_I g, dE/d(eps) = sum_I Pi_I g
// (= -Omega sigma g), E = sum_g V rho dV.  One CTA; the virial sum runs over atoms in a fixed
// order per thread and a fixed tree, as in the force finalisation.
__global__ void k_energy_grad_finalize(int n_atoms, const double* acc, const double* acc_e, const double* g,
                                       double* dR, double* deps, double* E) {
    __shared__ double s[9][256];
    const double gs = g ? *g : 1.0;
    double v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = threadIdx.x; i < n_atoms; i += blockDim.x) {
        const double* a = acc + 12 * (size_t)i;
        if (dR) for (int c = 0; c < 3; ++c) dR[3 * (size_t)i + c] = -a[c] * gs;
        for (int c = 0; c < 9; ++c) v[c] += a[3 + c];
    }
    for (int c = 0; c < 9; ++c) s[c][threadIdx.x] = v[c];
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st)
            for (int c = 0; c < 9; ++c) s[c][threadIdx.x] += s[c][threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (deps) for (int c = 0; c < 9; ++c) deps[c] = s[c][0] * gs;
        if (E) *E = *acc_e;
    }
}

}  // namespace
}  // namespace gint

using namespace gint;

extern "C" {

gint_status gint_vlocal(gint_handle* h, const double* V, double* H, int accumulate, gint_stream stream) {
    gint::NvtxRange nvtx_range_("gint_vlocal");
    set_error("");
    if (!h || !V || !H) { set_error("gint_vlocal: NULL argument"); return GINT_ERR_INVALID_ARG; }
    if (accumulate != 0 && accumulate != 1) { set_error("gint_vlocal: accumulate must be 0 or 1"); return GINT_ERR_INVALID_ARG; }
    bool fp32 = false;
    gint_status s = check_precision(h, &fp32);
    if (s != GINT_OK) return s;
    DeviceGuard dg(h->device);
    if (!dg.ok) { set_error("cannot select device %d", h->device); return GINT_ERR_CUDA; }
    cudaStream_t st = (cudaStream_t)stream;
    if (is_tc(h)) {  // limits first: a rejected call enqueues nothing
        s = tc_vlocal_check(h, tc_form(h));
        if (s != GINT_OK) return s;
    }
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
    gint::NvtxRange nvtx_range_("gint_rho");
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
    gint::NvtxRange nvtx_range_("gint_force_stress");
    set_error("");
    if (!h || !V || !D) { set_error("gint_force_stress: NULL argument"); return GINT_ERR_INVALID_ARG; }
    if (!F && !sigma && !virial_atom && !E) { set_error("gint_force_stress: no output requested"); return GINT_ERR_INVALID_ARG; }
    bool fp32 = false;
    gint_status s = check_precision(h, &fp32);
    if (s != GINT_OK) return s;
    DeviceGuard dg(h->device);
    if (!dg.ok) { set_error("cannot select device %d", h->device); return GINT_ERR_CUDA; }
    cudaStream_t st = (cudaStream_t)stream;
    s = force_accumulate(h, fp32, V, D, st);
    if (s != GINT_OK) return s;
    return launch_force_finalize(h, F, sigma, virial_atom, E, st);
}

gint_status gint_energy_grads(gint_handle* h, const double* V, const double* D, const double* grad_E, double* dE_dR,
                              double* dE_deps, double* dE_dV, double* dE_dD, double* E, gint_stream stream) {
    gint::NvtxRange nvtx_range_("gint_energy_grads");
    set_error("");
    if (!h || !V || !D) { set_error("gint_energy_grads: NULL argument"); return GINT_ERR_INVALID_ARG; }
    if (!dE_dR && !dE_deps && !dE_dV && !dE_dD && !E) { set_error("gint_energy_grads: no output requested"); return GINT_ERR_INVALID_ARG; }
    bool fp32 = false;
    gint_status s = check_precision(h, &fp32);
    if (s != GINT_OK) return s;
    DeviceGuard dg(h->device);
    if (!dg.ok) { set_error("cannot select device %d", h->device); return GINT_ERR_CUDA; }
    cudaStream_t st = (cudaStream_t)stream;
    const int sms = std::max(1, h->sm_count);
    if (is_tc(h)) {  // limits of every kernel the call may run, before anything is enqueued
        if (dE_dD) s = tc_vlocal_check(h, tc_form(h));
        if (s == GINT_OK) s = tc_rhoforce_check(h);
        if (s != GINT_OK) return s;
    }
    if (dE_dR || dE_deps || E) {
        s = force_accumulate(h, fp32, V, D, st);
        if (s != GINT_OK) return s;
        k_energy_grad_finalize<<<1, 256, 0, st>>>(h->n_atoms, h->d_facc, h->d_red, grad_E, dE_dR, dE_deps, E);
        GINT_CUDA_TRY(cudaGetLastError());
    }
    if (dE_dV) {  // dE/dV_g = rho_g dV
        const int64_t ng0 = (int64_t)h->grid.n[0] * h->grid.n[1] * h->grid.n[2];
        // with a brick selection rho is written on the selected bricks only; E does not depend on V
        // elsewhere, so those elements of the gradient are zero
        if (h->selecting) GINT_CUDA_TRY(cudaMemsetAsync(dE_dV, 0, sizeof(double) * ng0, st));
        s = gint_rho(h, D, dE_dV, stream);
        if (s != GINT_OK) return s;
        const int64_t ng = (int64_t)h->grid.n[0] * h->grid.n[1] * h->grid.n[2];
        k_scale<<<4 * sms, 256, 0, st>>>(dE_dV, ng, h->grid.dV, grad_E);
        GINT_CUDA_TRY(cudaGetLastError());
    }
    if (dE_dD) {  // dE/dD = H^V (every block of the pattern)
        s = gint_vlocal(h, V, dE_dD, 0, stream);
        if (s != GINT_OK) return s;
        if (grad_E && h->n_values > 0) {
            k_scale<<<4 * sms, 256, 0, st>>>(dE_dD, h->n_values, 1.0, grad_E);
            GINT_CUDA_TRY(cudaGetLastError());
        }
    }
    return GINT_OK;
}

}  // extern "C"
