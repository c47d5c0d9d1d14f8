// fold.cu -- Bloch sum of the block-sparse H^V into a dense H(k):
//   H(k)_{I mu, J nu} = sum over the blocks (I, J, t) of exp(2 pi i kfrac . t) H_IJ(t)[mu, nu].
// The pattern is sorted by (I, J, t), so the blocks of one atom pair are
// contiguous: one warp per atom pair walks its blocks, sums the phased values in
// registers (FP64) and writes its nw_I x nw_J complex sub-matrix once (no atomics;
// the summation order is fixed).
#include <cmath>

#include "gint_impl.cuh"

namespace gint {

constexpr int kFoldMaxElems = 16 * 16;  // nw_I x nw_J <= 256 (kMaxNw is 32; checked on the host)
constexpr int kFoldPerLane = (kFoldMaxElems + 31) / 32;

__global__ void k_fold_k(Problem P, const int* nw_atom, const int64_t* orb_off, int64_t n_blocks, const double* H,
                         double k0, double k1, double k2, double2* Hk, int64_t ld) {
    const int64_t b0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (b0 >= n_blocks) return;
    const int32_t* key = P.blocks + 5 * b0;
    const int I = key[0], J = key[1];
    if (b0 > 0 && key[-5] == I && key[-4] == J) return;  // not the first block of its atom pair
    const int nI = nw_atom[I], nJ = nw_atom[J], ne = nI * nJ;
    double re[kFoldPerLane], im[kFoldPerLane];
#pragma unroll
    for (int q = 0; q < kFoldPerLane; ++q) re[q] = im[q] = 0.0;
    for (int64_t b = b0; b < n_blocks; ++b) {
        const int32_t* kb = P.blocks + 5 * b;
        if (kb[0] != I || kb[1] != J) break;
        // phase 2 pi (k . t), reduced to one turn before the sine and cosine
        double turns = k0 * kb[2] + k1 * kb[3] + k2 * kb[4];
        turns -= floor(turns);
        double s, c;
        sincospi(2.0 * turns, &s, &c);
        const double* Hb = H + P.offsets[b];
#pragma unroll
        for (int q = 0; q < kFoldPerLane; ++q) {
            const int e = lane + 32 * q;
            if (e < ne) {
                const double v = Hb[e];
                re[q] += c * v;
                im[q] += s * v;
            }
        }
    }
    const int64_t r0 = orb_off[I], c0 = orb_off[J];
#pragma unroll
    for (int q = 0; q < kFoldPerLane; ++q) {
        const int e = lane + 32 * q;
        if (e < ne) {
            const int mu = e / nJ, nu = e - mu * nJ;
            Hk[(r0 + mu) * ld + c0 + nu] = make_double2(re[q], im[q]);
        }
    }
}

}  // namespace gint

using namespace gint;

extern "C" gint_status gint_fold_k(const gint_handle* h, const double* H, const double kfrac[3], double* Hk, int64_t ld,
                                   gint_stream stream) {
    set_error("");
    if (!h || !H || !kfrac || !Hk) { set_error("gint_fold_k: NULL argument"); return GINT_ERR_INVALID_ARG; }
    if (ld < h->n_orbitals) { set_error("gint_fold_k: ld %lld < n_orbitals %lld", (long long)ld, (long long)h->n_orbitals); return GINT_ERR_INVALID_ARG; }
    for (int i = 0; i < 3; ++i)
        if (!std::isfinite(kfrac[i])) { set_error("gint_fold_k: k is not finite"); return GINT_ERR_INVALID_ARG; }
    if (h->max_nw > 16) { set_error("gint_fold_k: atoms with more than 16 orbitals are not supported"); return GINT_ERR_UNSUPPORTED; }
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    gint_status s = GINT_OK;
    cudaError_t e = cudaMemsetAsync(Hk, 0, sizeof(double) * 2 * (size_t)ld * (size_t)h->n_orbitals, st);
    if (e == cudaSuccess && h->n_blocks > 0) {
        const unsigned grid = (unsigned)((h->n_blocks * 32 + 255) / 256);
        k_fold_k<<<grid, 256, 0, st>>>(h->problem(), h->d_nw_atom, h->d_orb_off, h->n_blocks, H, kfrac[0], kfrac[1],
                                       kfrac[2], reinterpret_cast<double2*>(Hk), ld);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) { set_error("gint_fold_k: %s", cudaGetErrorString(e)); s = GINT_ERR_CUDA; }
    if (prev >= 0) cudaSetDevice(prev);
    return s;
}
