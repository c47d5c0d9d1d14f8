// hxc.cu -- the local potential from rho: Hartree and LDA exchange-correlation parts.
//
// V in Eq. 2 has three parts: the atoms' local pseudopotentials (an external input here,
// V_ext), the electrostatic (Hartree) potential of rho and the exchange-correlation
// potential (Section 2.2, the text after Eq. 2; Fig. 1 forms it from rho before the grid
// integrals).  Here:
//   V_H:  the periodic Poisson equation lap V_H = -4 pi (rho - mean rho), solved in
//         reciprocal space, V_H(G) = 4 pi rho(G) / |G|^2, V_H(G = 0) = 0;
//   v_xc: LDA, Slater exchange and the Perdew-Zunger (1981) fit of the Ceperley-Alder
//         correlation (spin unpolarised), zero where rho <= 0;
//   E_H = 1/2 sum_g rho_g V_H,g dV,  E_xc = sum_g rho_g eps_xc,g dV.
// The 3-D FFTs are a library step (cuFFT, loaded at run time, the way cuBLAS serves a
// plain GEMM); the G-space multiply and the fused pointwise pass with the FP64 energy
// reductions are the kernels below.  Both passes are bound by HBM bandwidth.
#include <cmath>
#include <dlfcn.h>
#include <mutex>

#include <cufft.h>

#include "gint_impl.cuh"
#include "nvtx.cuh"

namespace gint {

namespace {

// ------------------------------------------------------------ cuFFT, loaded at run time
struct CufftApi {
    cufftResult (*create)(cufftHandle*) = nullptr;
    cufftResult (*make3d)(cufftHandle, int, int, int, cufftType, size_t*) = nullptr;
    cufftResult (*exec_d2z)(cufftHandle, cufftDoubleReal*, cufftDoubleComplex*) = nullptr;
    cufftResult (*exec_z2d)(cufftHandle, cufftDoubleComplex*, cufftDoubleReal*) = nullptr;
    cufftResult (*set_stream)(cufftHandle, cudaStream_t) = nullptr;
    cufftResult (*destroy)(cufftHandle) = nullptr;
    bool ok = false;
};
CufftApi g_fft;
std::once_flag g_fft_once;

void load_cufft() {
    const char* names[] = {"libcufft.so.12", "libcufft.so.13", "libcufft.so.11", "libcufft.so"};
    void* lib = nullptr;
    for (const char* n : names)
        if ((lib = dlopen(n, RTLD_NOW | RTLD_LOCAL))) break;
    if (!lib) return;
    g_fft.create = (decltype(g_fft.create))dlsym(lib, "cufftCreate");
    g_fft.make3d = (decltype(g_fft.make3d))dlsym(lib, "cufftMakePlan3d");
    g_fft.exec_d2z = (decltype(g_fft.exec_d2z))dlsym(lib, "cufftExecD2Z");
    g_fft.exec_z2d = (decltype(g_fft.exec_z2d))dlsym(lib, "cufftExecZ2D");
    g_fft.set_stream = (decltype(g_fft.set_stream))dlsym(lib, "cufftSetStream");
    g_fft.destroy = (decltype(g_fft.destroy))dlsym(lib, "cufftDestroy");
    g_fft.ok = g_fft.create && g_fft.make3d && g_fft.exec_d2z && g_fft.exec_z2d && g_fft.set_stream && g_fft.destroy;
}

#define GINT_FFT_TRY(expr)                                                               \
    do {                                                                                 \
        cufftResult r_ = (expr);                                                         \
        if (r_ != CUFFT_SUCCESS) {                                                       \
            ::gint::set_error("%s failed: cuFFT status %d", #expr, (int)r_);             \
            return r_ == CUFFT_ALLOC_FAILED ? GINT_ERR_OOM : GINT_ERR_CUDA;              \
        }                                                                                \
    } while (0)

constexpr int kRedBlocks = 1024;  // blocks of the pointwise pass (fixed: fixed reduction order)
constexpr int kRedThreads = 256;

// Integer frequency of FFT index i on an axis of n points: 0..ceil(n/2)-1, then negative
// (the Nyquist index of an even axis is -n/2).
__device__ __forceinline__ int freq(int i, int n) { return i < (n + 1) / 2 ? i : i - n; }

// 1/x for x > 0 in FP64 from the FP32 reciprocal and one Newton-Raphson step
// y <- y (2 - x y), which squares the relative error (2^-23 -> below 2^-45).
__device__ __forceinline__ double recip(double x) {
    const double y = (double)__frcp_rn((float)x);
    return y * fma(-x, y, 2.0);
}

// 4 pi / |G|^2 for G = m0 b0 + m1 b1 + m2 b2 (b: reciprocal rows, b_i . a_j = 2 pi delta_ij).
__device__ __forceinline__ double coulomb(const double b[9], int m0, int m1, int m2) {
    const double gx = m0 * b[0] + m1 * b[3] + m2 * b[6];
    const double gy = m0 * b[1] + m1 * b[4] + m2 * b[7];
    const double gz = m0 * b[2] + m1 * b[5] + m2 * b[8];
    const double g2 = gx * gx + gy * gy + gz * gz;
    return g2 > 0.0 ? 4.0 * M_PI / g2 : 0.0;
}

struct Recip {
    double b[9];
};

// rho(G) -> V_H(G) / N in place on the half spectrum [n0][n1][n2/2 + 1].  A component on
// the Nyquist index of an even axis stands for both +n/2 and -n/2; the kernel there is the
// mean of the two assignments related by G -> -G, which keeps V_H(G) Hermitian (so the
// real inverse transform is exact) and equals the real part of the full complex transform
// with the -n/2 assignment.  One CTA per (i0, i1) row of the spectrum, threads along i2
// (contiguous), 32-bit index arithmetic; 1/|G|^2 from the FP32 reciprocal refined once in
// FP64 (two on the Nyquist planes).
__global__ void k_hartree_g(double2* spec, int n0, int n1, int n2, Recip R, double c4pi_n) {
    const int h2 = n2 / 2 + 1;
    for (int row = blockIdx.x; row < n0 * n1; row += gridDim.x) {
        const int i0 = row / n1, i1 = row - i0 * n1;
        const int m0 = freq(i0, n0), m1 = freq(i1, n1);
        const int q0 = (2 * i0 == n0) ? m0 : -m0;  // -G with each Nyquist component kept at -n/2
        const int q1 = (2 * i1 == n1) ? m1 : -m1;
        const bool nyq01 = (q0 == m0 && m0 != 0) || (q1 == m1 && m1 != 0);
        // in-plane part of G and of its partner
        const double gx = m0 * R.b[0] + m1 * R.b[3], gy = m0 * R.b[1] + m1 * R.b[4], gz = m0 * R.b[2] + m1 * R.b[5];
        const double qx = q0 * R.b[0] + q1 * R.b[3], qy = q0 * R.b[1] + q1 * R.b[4], qz = q0 * R.b[2] + q1 * R.b[5];
        double2* line = spec + (size_t)row * h2;
        for (int i2 = threadIdx.x; i2 < h2; i2 += blockDim.x) {
            const int m2 = freq(i2, n2);
            const double ax = fma((double)m2, R.b[6], gx), ay = fma((double)m2, R.b[7], gy);
            const double az = fma((double)m2, R.b[8], gz);
            const double g2 = fma(ax, ax, fma(ay, ay, az * az));
            double k = g2 > 0.0 ? c4pi_n * recip(g2) : 0.0;
            const bool nyq2 = 2 * i2 == n2;
            if (nyq01 || nyq2) {  // Nyquist planes: mean with the partner assignment
                const int q2 = nyq2 ? m2 : -m2;
                const double bx = fma((double)q2, R.b[6], qx), by = fma((double)q2, R.b[7], qy);
                const double bz = fma((double)q2, R.b[8], qz);
                const double p2 = fma(bx, bx, fma(by, by, bz * bz));
                k = 0.5 * (k + (p2 > 0.0 ? c4pi_n * recip(p2) : 0.0));
            }
            double2 v = line[i2];
            v.x *= k;
            v.y *= k;
            line[i2] = v;
        }
    }
}

// LDA exchange-correlation per electron and potential at density rho > 0 (hartree).
__device__ __forceinline__ void lda_xc(double rho, double& eps, double& v) {
    const double rs = cbrt(3.0 / (4.0 * M_PI * rho));
    constexpr double kSlater = -0.75 * 0.6108870577108572;  // -(3/4) (9 / (4 pi^2))^(1/3)
    const double ex = kSlater / rs;  // Slater exchange
    const double vx = (4.0 / 3.0) * ex;
    double ec, vc;
    if (rs >= 1.0) {  // Perdew-Zunger 1981, rs >= 1
        const double g = -0.1423, b1 = 1.0529, b2 = 0.3334;
        const double sq = sqrt(rs);
        const double den = 1.0 + b1 * sq + b2 * rs;
        ec = g / den;
        vc = ec * (1.0 + (7.0 / 6.0) * b1 * sq + (4.0 / 3.0) * b2 * rs) / den;
    } else {  // rs < 1
        const double A = 0.0311, B = -0.048, C = 0.0020, D = -0.0116;
        const double lr = log(rs);
        ec = A * lr + B + C * rs * lr + D * rs;
        vc = A * lr + (B - A / 3.0) + (2.0 / 3.0) * C * rs * lr + (2.0 * D - C) / 3.0 * rs;
    }
    eps = ex + ec;
    v = vx + vc;
}

// V_out = V_ext + V_H + v_xc(rho); per-block FP64 partial sums of rho V_H and rho eps_xc.
// V_H may alias V_out (each element is read before it is written by the same thread).
__global__ void __launch_bounds__(kRedThreads) k_local_potential(const double* __restrict__ rho, const double* V_ext,
                                                                 const double* V_H, double* V_out, int64_t n,
                                                                 double* part) {
    double eh = 0.0, ex = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double r = rho[i];
        const double vh = V_H[i];
        double eps = 0.0, vxc = 0.0;
        if (r > 0.0) lda_xc(r, eps, vxc);
        V_out[i] = (V_ext ? V_ext[i] : 0.0) + vh + vxc;
        eh += r * vh;
        ex += r * eps;
    }
    __shared__ double s[2][kRedThreads];
    s[0][threadIdx.x] = eh;
    s[1][threadIdx.x] = ex;
    __syncthreads();
    for (int st = kRedThreads / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) {
            s[0][threadIdx.x] += s[0][threadIdx.x + st];
            s[1][threadIdx.x] += s[1][threadIdx.x + st];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = s[0][0];
        part[2 * blockIdx.x + 1] = s[1][0];
    }
}

// energies[0] = 1/2 dV sum rho V_H, energies[1] = dV sum rho eps_xc (fixed order).
__global__ void k_local_energies(const double* part, int nb, double dV, double* energies) {
    __shared__ double s[2][kRedThreads];
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        a += part[2 * k];
        b += part[2 * k + 1];
    }
    s[0][threadIdx.x] = a;
    s[1][threadIdx.x] = b;
    __syncthreads();
    for (int st = kRedThreads / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) {
            s[0][threadIdx.x] += s[0][threadIdx.x + st];
            s[1][threadIdx.x] += s[1][threadIdx.x + st];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        energies[0] = 0.5 * s[0][0] * dV;
        energies[1] = s[1][0] * dV;
    }
}

// cuFFT plans and the half-spectrum buffer of the handle's grid, made on first use.
gint_status ensure_fft(gint_handle* h) {
    std::call_once(g_fft_once, load_cufft);
    if (!g_fft.ok) {
        set_error("the local potential needs cuFFT (libcufft), which could not be loaded");
        return GINT_ERR_UNSUPPORTED;
    }
    const int n0 = h->grid.n[0], n1 = h->grid.n[1], n2 = h->grid.n[2];
    if (!h->d_spec) {
        const size_t bytes = sizeof(double2) * (size_t)n0 * n1 * (n2 / 2 + 1);
        GINT_CUDA_TRY(dev_malloc(&h->d_spec, bytes));
    }
    if (!h->d_epart) GINT_CUDA_TRY(dev_malloc(&h->d_epart, sizeof(double) * 2 * kRedBlocks));
    if (h->fft_fwd < 0) {
        cufftHandle p;
        size_t ws = 0;
        GINT_FFT_TRY(g_fft.create(&p));
        const cufftResult r = g_fft.make3d(p, n0, n1, n2, CUFFT_D2Z, &ws);
        if (r != CUFFT_SUCCESS) {
            g_fft.destroy(p);
            set_error("cufftMakePlan3d (forward, %d x %d x %d) failed: cuFFT status %d", n0, n1, n2, (int)r);
            return r == CUFFT_ALLOC_FAILED ? GINT_ERR_OOM : GINT_ERR_CUDA;
        }
        h->fft_fwd = (int)p;
    }
    if (h->fft_inv < 0) {
        cufftHandle p;
        size_t ws = 0;
        GINT_FFT_TRY(g_fft.create(&p));
        const cufftResult r = g_fft.make3d(p, n0, n1, n2, CUFFT_Z2D, &ws);
        if (r != CUFFT_SUCCESS) {
            g_fft.destroy(p);
            set_error("cufftMakePlan3d (inverse, %d x %d x %d) failed: cuFFT status %d", n0, n1, n2, (int)r);
            return r == CUFFT_ALLOC_FAILED ? GINT_ERR_OOM : GINT_ERR_CUDA;
        }
        h->fft_inv = (int)p;
    }
    return GINT_OK;
}

}  // namespace

// Release the FFT plans of a handle (its buffers are freed with the rest).
void hxc_release(gint_handle* h) {
    if (g_fft.ok) {
        if (h->fft_fwd >= 0) g_fft.destroy((cufftHandle)h->fft_fwd);
        if (h->fft_inv >= 0) g_fft.destroy((cufftHandle)h->fft_inv);
    }
    h->fft_fwd = h->fft_inv = -1;
}

}  // namespace gint

using namespace gint;

extern "C" gint_status gint_local_potential(gint_handle* h, const double* rho, const double* V_ext, double* V_out,
                                            double* V_H, double* energies, gint_stream stream) {
    gint::NvtxRange nvtx_range_("gint_local_potential");
    set_error("");
    if (!h || !rho || !V_out) { set_error("gint_local_potential: NULL argument"); return GINT_ERR_INVALID_ARG; }
    const int64_t n0 = h->grid.n[0], n1 = h->grid.n[1], n2 = h->grid.n[2];
    if (n0 * n1 * n2 > INT32_MAX) {
        set_error("gint_local_potential: grids above 2^31 points are not supported");
        return GINT_ERR_UNSUPPORTED;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(h->device) != cudaSuccess) { set_error("cannot select device %d", h->device); return GINT_ERR_CUDA; }
    struct Restore {
        int d;
        ~Restore() { if (d >= 0) cudaSetDevice(d); }
    } restore{prev};
    gint_status s = ensure_fft(h);
    if (s != GINT_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    double2* spec = (double2*)h->d_spec;
    double* vh = V_H ? V_H : V_out;  // the inverse transform's output
    GINT_FFT_TRY(g_fft.set_stream((cufftHandle)h->fft_fwd, st));
    GINT_FFT_TRY(g_fft.set_stream((cufftHandle)h->fft_inv, st));
    GINT_FFT_TRY(g_fft.exec_d2z((cufftHandle)h->fft_fwd, const_cast<double*>(rho), (cufftDoubleComplex*)spec));
    Recip R;
    {
        // reciprocal rows b_j = 2 pi (A^-1)^T rows: b_j[c] = 2 pi Ainv[c][j]
        const double* a = h->cell;
        const double det = a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
                           a[2] * (a[3] * a[7] - a[4] * a[6]);
        const double inv[9] = {(a[4] * a[8] - a[5] * a[7]) / det, (a[2] * a[7] - a[1] * a[8]) / det,
                               (a[1] * a[5] - a[2] * a[4]) / det, (a[5] * a[6] - a[3] * a[8]) / det,
                               (a[0] * a[8] - a[2] * a[6]) / det, (a[2] * a[3] - a[0] * a[5]) / det,
                               (a[3] * a[7] - a[4] * a[6]) / det, (a[1] * a[6] - a[0] * a[7]) / det,
                               (a[0] * a[4] - a[1] * a[3]) / det};
        for (int j = 0; j < 3; ++j)
            for (int c = 0; c < 3; ++c) R.b[3 * j + c] = 2.0 * M_PI * inv[3 * c + j];
    }
    const int blocks = (int)std::min<int64_t>(n0 * n1, (int64_t)64 * std::max(1, h->sm_count));
    const int h2 = (int)(n2 / 2 + 1);
    const int threads = std::min(256, (h2 + 31) / 32 * 32);  // one pass over a spectrum row
    k_hartree_g<<<blocks, threads, 0, st>>>(spec, (int)n0, (int)n1, (int)n2, R, 4.0 * M_PI / (double)(n0 * n1 * n2));
    GINT_CUDA_TRY(cudaGetLastError());
    GINT_FFT_TRY(g_fft.exec_z2d((cufftHandle)h->fft_inv, (cufftDoubleComplex*)spec, vh));
    k_local_potential<<<kRedBlocks, kRedThreads, 0, st>>>(rho, V_ext, vh, V_out, n0 * n1 * n2, h->d_epart);
    GINT_CUDA_TRY(cudaGetLastError());
    if (energies) {
        k_local_energies<<<1, kRedThreads, 0, st>>>(h->d_epart, kRedBlocks, h->grid.dV, energies);
        GINT_CUDA_TRY(cudaGetLastError());
    }
    return GINT_OK;
}
