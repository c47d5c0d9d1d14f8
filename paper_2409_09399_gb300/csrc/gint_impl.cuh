// gint_impl.cuh -- internal structures and device helpers of libgint.
//
// Real-space grid integration of numerical-atomic-orbital DFT (paper
// Section 2.2): the grid is cut into bricks of grid points (the "batches" of
// Section 2.3.2); each brick carries the list of atom images whose cutoff
// sphere meets it (the "neighbouring atoms" of Section 2.3.2).  Kernels
// evaluate orbital values per brick and contract them (Section 2.3.3).
#pragma once

#include <cstdint>
#include <cstdio>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/gint.h"

namespace gint {

constexpr int kMaxRadial = 16;    // radial functions per species
constexpr int kMaxNw = 32;        // orbitals per atom
constexpr int kMaxL = 3;          // angular momentum
constexpr int kMaxBrickPts = 2048;  // points per brick (64 sub-tiles of 32)
constexpr int kMaxBrickAtoms = 160; // atom images per brick

// Per-species data on the device.  The radial table is stored per knot
// interval k as the cubic in t = r/dr - k, R = c0 + t (c1 + t (c2 + t c3)),
// for all radial functions of the species side by side:
// coef[tab_off + (k * n_radial + j) * 4 + c].
struct SpeciesDev {
    int n_radial;
    int n_orb;
    int lmax;
    int n_int;        // knot intervals
    double rc;
    double dr;
    double inv_dr;
    float rc_f;
    float inv_dr_f;
    int64_t tab_off;
    int64_t knot_off;  // offset of the species' FP32 knot table in float2 units
    int rad_l[kMaxRadial];
    signed char orb_rad[kMaxNw];  // radial function of each orbital
    signed char orb_l[kMaxNw];
    signed char orb_m[kMaxNw];    // m + l, 0..2l
    signed char orb_qe[kMaxNw];   // |phi_o(r)| <= 127 * 2^orb_qe for every r (fixed-point quantum)
    signed char orb_qeu[kMaxNw];  // the same for phi_o / ylm_norm(l, m) (unnormalised harmonic)
};

// Normalisation of the real solid harmonics in the orbital definition:
// phi_lm = R(r) / r^l * ylm_norm(l, m) * P_lm(x, y, z), with the polynomials
// P: l = 1: y, z, x; l = 2: xy, yz, 2z^2 - x^2 - y^2, xz, x^2 - y^2;
// l = 3: y(3x^2 - y^2), xyz, y(4z^2 - x^2 - y^2), z(2z^2 - 3x^2 - 3y^2),
// x(4z^2 - x^2 - y^2), z(x^2 - y^2), x(x^2 - 3y^2)  (m = -l..l).
__host__ __device__ inline double ylm_norm(int l, int mi) {  // mi = m + l
    switch (l) {
        case 0: return 0.28209479177387814;   // 1 / (2 sqrt(pi))
        case 1: return 0.48860251190291992;   // sqrt(3 / (4 pi))
        case 2: return (mi == 2) ? 0.31539156525252005 : (mi == 4) ? 0.54627421529603959 : 1.0925484305920792;
        default: {
            const double t[7] = {0.59004358992664352, 2.8906114426405538, 0.45704579946446572, 0.37317633259011540,
                                 0.45704579946446572, 1.4453057213202769, 0.59004358992664352};
            return t[mi];
        }
    }
}

// An atom image (I, T) whose cutoff sphere meets the grid.
struct ExtAtom {
    double p[3];  // R_I + T (bohr)
    int atom;     // I
    int species;
    int t[3];
    int pad;
};

// Grid and brick geometry.
struct GridDev {
    int n[3];        // grid points per axis
    int B[3];        // brick shape
    int nb[3];       // bricks per axis
    int bpts;        // B0*B1*B2
    int bpad;        // bpts rounded up to a multiple of 32
    int nsub;        // bpad / 32
    double step[3][3];  // step[i] = a_i / n_i
    float step_hi[3][3], step_lo[3][3];  // step = hi + lo, FP32 words (in-brick offsets without a scale bias)
    double dV;
};

// Everything a compute kernel needs (passed by value).
struct Problem {
    GridDev g;
    const SpeciesDev* sp;
    const double* coef64;
    const float* coef32;
    const float2* knot32;        // per knot and radial function (R(r_k), dr R'(r_k)) in FP32
    const ExtAtom* ext;
    const int64_t* brick_start;  // n_bricks + 1
    const int32_t* brick_atoms;  // ext indices, ascending per brick
    const int32_t* work;         // non-empty brick ids, natural order
    const int64_t* pair_start;   // n_bricks + 1: first entry of each brick's pair table
    const int32_t* pairs;        // per brick, na x na: block (I_a, I_b, t_b - t_a) of images a, b, -1 if none
    const unsigned long long* tile_mask;  // per work item and 128-point tile: images within rc of a tile point
    int n_work;
    const int32_t* blocks;       // n_blocks x 5
    const int64_t* offsets;      // n_blocks + 1
    const int64_t* row_start;    // n_atoms + 1
    int n_atoms;
    int n_species;
    int* err;                    // device error flags (bit set)
};

// One cell of a batched launch: its problem and its call's buffers, and the
// position of its bricks in the batch's work queue (items [item0, item0 + n_work)).
struct CellJob {
    Problem P;
    const double* V;
    double* H;
    const unsigned char* Dt;     // tensor-core copy of D
    const unsigned char* Dzero;  // a zero tile of it
    const int* dq;               // exact form: row maxima of D
    double* rho;
    double* facc;
    double* acc_e;
    int item0;
    int pad;
};

// The (cell, brick) queue of a batched launch: item w belongs to cell item_cell[w].
struct MultiArgs {
    const CellJob* jobs;
    const int* item_cell;
    int n_items;
};

// Device error bits.
enum : int {
    kErrPatternMissing = 1,
    kErrBrickTooLarge = 2,
    kErrTimeout = 4,  // a bounded wait on the tensor-core pipeline gave up
};

}  // namespace gint

// Host-side handle.
struct gint_handle {
    int device = 0;
    int n_atoms = 0;
    int n_species = 0;
    double cell[9] = {0};
    double omega = 0;
    int precision = GINT_FP64;
    gint::GridDev grid{};
    int max_nw = 0;
    int64_t n_bricks = 0;
    int64_t n_work = 0;
    int64_t n_empty = 0;
    int64_t n_ext = 0;
    int64_t n_blocks = 0;
    int64_t n_values = 0;
    int64_t n_orbitals = 0;           // sum of the atoms' orbitals (dimension of H(k))
    int64_t n_brick_atoms = 0;
    int64_t n_brick_pairs = 0;
    int max_brick_atoms = 0;
    int max_brick_orb = 0;
    // device memory owned by the handle
    gint::SpeciesDev* d_sp = nullptr;
    double* d_coef64 = nullptr;
    float* d_coef32 = nullptr;
    float2* d_knot32 = nullptr;
    gint::ExtAtom* d_ext = nullptr;
    int32_t* d_blocks = nullptr;
    int64_t* d_offsets = nullptr;
    int64_t* d_row_start = nullptr;
    int32_t* d_mirror = nullptr;      // for every block, the index of (J, I, -T)
    int64_t* d_brick_start = nullptr;
    int32_t* d_brick_atoms = nullptr;
    int32_t* d_work = nullptr;        // non-empty bricks
    int64_t* d_pair_start = nullptr;  // per-brick pair tables (see Problem::pairs)
    int32_t* d_pairs = nullptr;
    unsigned long long* d_tile_mask = nullptr;  // see Problem::tile_mask
    int32_t* d_empty = nullptr;       // empty bricks
    int* d_err = nullptr;             // [0] device check flags, [2] work counter
    int* d_nw_atom = nullptr;         // orbitals of every atom
    int* d_atom_sp = nullptr;         // species of every atom
    int64_t* d_orb_off = nullptr;     // first orbital (dense row) of every atom, n_atoms + 1
    double* d_facc = nullptr;         // per-atom force and virial accumulators, n_atoms x 12
    double* d_red = nullptr;          // small FP64 reduction buffer ([0] energy)
    void* d_dt = nullptr;             // per-call 16x16 tensor-core copy of D (1 KB per block)
    int* d_dq = nullptr;              // exact form: per (atom, orbital row) max |D| bits, n_atoms x 16
    void* d_zero = nullptr;           // one zero tile of the tensor-core copy of D
    void* d_scratch = nullptr;
    size_t scratch_bytes = 0;
    int n_ctas = 0;                   // persistent CTAs of the SIMT kernels
    int sm_count = 0;
    void* d_static = nullptr;         // device address of the library's static scratch array (not owned)
    void* d_spec = nullptr;           // local potential: half spectrum of the grid (complex128)
    double* d_epart = nullptr;        // local potential: per-block energy partial sums
    int fft_fwd = -1, fft_inv = -1;   // local potential: cuFFT plans (made on first use)
    long long wait_limit = 0;         // polls of a bounded tensor-core pipeline wait (0: the default)
    int generation = 0;               // bumped by gint_update_positions (batches built earlier are stale)
    int brick_opt[3] = {0, 0, 0};     // brick shape asked for at set-up (0: default)
    // host copy of the species tables and the atoms' species, for gint_update_positions
    std::vector<double> sp_rc;
    std::vector<int> sp_nrad, rad_l, rad_nk, atom_species;
    std::vector<double> rad_dr, rad_y, rad_dy;
    // bricks selected by gint_select_bricks (selecting == false: every brick)
    bool selecting = false;
    std::vector<int64_t> selection;

    gint::Problem problem() const {
        gint::Problem p;
        p.g = grid;
        p.sp = d_sp;
        p.coef64 = d_coef64;
        p.coef32 = d_coef32;
        p.knot32 = d_knot32;
        p.ext = d_ext;
        p.brick_start = d_brick_start;
        p.brick_atoms = d_brick_atoms;
        p.work = d_work;
        p.pair_start = d_pair_start;
        p.pairs = d_pairs;
        p.tile_mask = d_tile_mask;
        p.n_work = (int)n_work;
        p.blocks = d_blocks;
        p.offsets = d_offsets;
        p.row_start = d_row_start;
        p.n_atoms = n_atoms;
        p.n_species = n_species;
        p.err = d_err;
        return p;
    }
};

namespace gint {

// last-error message (thread local), set by the ABI layer
void set_error(const char* fmt, ...);

// Every device allocation of the library goes through dev_malloc, which a test hook
// (gint_debug_fail_alloc) can make fail as cudaMalloc does when the device is full.
cudaError_t dev_malloc_raw(void** p, size_t bytes);
template <typename T>
inline cudaError_t dev_malloc(T** p, size_t bytes) { return dev_malloc_raw(reinterpret_cast<void**>(p), bytes); }

// Polls of a bounded wait on the tensor-core pipelines (gint_set_wait_limit); the drains before
// tensor memory is released always use kDrainPolls.
constexpr long kDefaultWaitPolls = 1L << 26;
constexpr long kDrainPolls = 1L << 26;
inline long wait_polls(const gint_handle* h) { return h->wait_limit > 0 ? (long)h->wait_limit : kDefaultWaitPolls; }

#define GINT_CUDA_TRY(expr)                                                                     \
    do {                                                                                        \
        cudaError_t e_ = (expr);                                                                \
        if (e_ != cudaSuccess) {                                                                \
            ::gint::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, \
                              __LINE__);                                                        \
            return e_ == cudaErrorMemoryAllocation ? GINT_ERR_OOM : GINT_ERR_CUDA;               \
        }                                                                                       \
    } while (0)

// ------------------------------------------------------------------ device
// Binary search of block (I, J, t) in the sorted pattern row of atom I.
__device__ __forceinline__ int64_t find_block(const Problem& P, int I, int J, int t0, int t1, int t2) {
    int64_t lo = P.row_start[I], hi = P.row_start[I + 1] - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) >> 1;
        const int32_t* k = P.blocks + 5 * mid;
        int c = (k[1] != J) ? (k[1] < J ? -1 : 1)
              : (k[2] != t0) ? (k[2] < t0 ? -1 : 1)
              : (k[3] != t1) ? (k[3] < t1 ? -1 : 1)
              : (k[4] != t2) ? (k[4] < t2 ? -1 : 1) : 0;
        if (c == 0) return mid;
        if (c < 0) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

// Real solid harmonics S_lm = r^l Y_lm (normalised Y, no Condon-Shortley
// phase) for l = 0..lmax at (x, y, z), flattened as index l*l + (m + l).
// With grad != nullptr also dS/dx, dS/dy, dS/dz.
template <typename T>
__device__ __forceinline__ void solid_harm(int lmax, T x, T y, T z, T* S, T (*grad)[3]) {
    // normalisation constants sqrt((2l+1)/(4 pi) * ...), evaluated in double and rounded to T
    const T k00 = T(0.28209479177387814);   // 1/(2 sqrt(pi))
    const T k1 = T(0.48860251190291992);    // sqrt(3/(4 pi))
    const T k2a = T(1.0925484305920792);    // sqrt(15/(4 pi))
    const T k2b = T(0.31539156525252005);   // sqrt(5/(16 pi))
    const T k2c = T(0.54627421529603959);   // sqrt(15/(16 pi))
    const T k3a = T(0.59004358992664352);   // sqrt(35/(32 pi))
    const T k3b = T(2.8906114426405538);    // sqrt(105/(4 pi))
    const T k3c = T(0.45704579946446572);   // sqrt(21/(32 pi))
    const T k3d = T(0.37317633259011540);   // sqrt(7/(16 pi))
    const T k3e = T(1.4453057213202769);    // sqrt(105/(16 pi))
    S[0] = k00;
    if (grad) { grad[0][0] = T(0); grad[0][1] = T(0); grad[0][2] = T(0); }
    if (lmax < 1) return;
    S[1] = k1 * y; S[2] = k1 * z; S[3] = k1 * x;
    if (grad) {
        grad[1][0] = T(0); grad[1][1] = k1;   grad[1][2] = T(0);
        grad[2][0] = T(0); grad[2][1] = T(0); grad[2][2] = k1;
        grad[3][0] = k1;   grad[3][1] = T(0); grad[3][2] = T(0);
    }
    if (lmax < 2) return;
    const T xx = x * x, yy = y * y, zz = z * z;
    S[4] = k2a * (x * y);
    S[5] = k2a * (y * z);
    S[6] = k2b * (T(2) * zz - xx - yy);
    S[7] = k2a * (x * z);
    S[8] = k2c * (xx - yy);
    if (grad) {
        grad[4][0] = k2a * y; grad[4][1] = k2a * x; grad[4][2] = T(0);
        grad[5][0] = T(0); grad[5][1] = k2a * z; grad[5][2] = k2a * y;
        grad[6][0] = T(-2) * k2b * x; grad[6][1] = T(-2) * k2b * y; grad[6][2] = T(4) * k2b * z;
        grad[7][0] = k2a * z; grad[7][1] = T(0); grad[7][2] = k2a * x;
        grad[8][0] = T(2) * k2c * x; grad[8][1] = T(-2) * k2c * y; grad[8][2] = T(0);
    }
    if (lmax < 3) return;
    const T q = T(4) * zz - xx - yy;  // 5 z^2 - r^2
    S[9] = k3a * y * (T(3) * xx - yy);
    S[10] = k3b * x * y * z;
    S[11] = k3c * y * q;
    S[12] = k3d * z * (T(2) * zz - T(3) * xx - T(3) * yy);
    S[13] = k3c * x * q;
    S[14] = k3e * z * (xx - yy);
    S[15] = k3a * x * (xx - T(3) * yy);
    if (grad) {
        grad[9][0] = k3a * T(6) * x * y; grad[9][1] = k3a * T(3) * (xx - yy); grad[9][2] = T(0);
        grad[10][0] = k3b * y * z; grad[10][1] = k3b * x * z; grad[10][2] = k3b * x * y;
        grad[11][0] = k3c * T(-2) * x * y; grad[11][1] = k3c * (q - T(2) * yy); grad[11][2] = k3c * T(8) * y * z;
        grad[12][0] = k3d * T(-6) * x * z; grad[12][1] = k3d * T(-6) * y * z;
        grad[12][2] = k3d * (T(6) * zz - T(3) * xx - T(3) * yy);
        grad[13][0] = k3c * (q - T(2) * xx); grad[13][1] = k3c * T(-2) * x * y; grad[13][2] = k3c * T(8) * x * z;
        grad[14][0] = k3e * T(2) * x * z; grad[14][1] = k3e * T(-2) * y * z; grad[14][2] = k3e * (xx - yy);
        grad[15][0] = k3a * T(3) * (xx - yy); grad[15][1] = k3a * T(-6) * x * y; grad[15][2] = T(0);
    }
}

template <typename T> struct CoefPtr;
template <> struct CoefPtr<double> { static __device__ __forceinline__ const double* get(const Problem& P) { return P.coef64; } };
template <> struct CoefPtr<float> { static __device__ __forceinline__ const float* get(const Problem& P) { return P.coef32; } };

// Orbital values (and gradients when G != nullptr) of one atom of species
// `s` at displacement d = r - (R_I + T).  Returns false (nothing written)
// when |d| >= rc.  phi is written for o < n_orb.
//
// phi = u(r) S_lm(d) with u = R(r)/r^l; grad phi = u'(r) (d/r) S_lm + u grad S_lm,
// u' = R'/r^l - l R / r^(l+1).  At |d| < 1e-12 bohr the limits are used:
// phi = R(0) Y00 for l = 0 and 0 otherwise; grad phi = R'(0) grad S_1m for
// l = 1 and 0 otherwise.
template <typename T, bool kGrad>
__device__ __forceinline__ bool eval_atom(const Problem& P, const SpeciesDev& s, T dx, T dy, T dz,
                                          T* phi, T (*G)[3]) {
    const T r2 = dx * dx + dy * dy + dz * dz;
    const T rc = sizeof(T) == 8 ? T(s.rc) : T(s.rc_f);
    if (r2 >= rc * rc) return false;
    const T r = sqrt(r2);
    const bool tiny = r < T(1e-12);
    const T inv_dr = sizeof(T) == 8 ? T(s.inv_dr) : T(s.inv_dr_f);
    T x = r * inv_dr;
    int k = (int)x;
    if (k > s.n_int - 1) k = s.n_int - 1;
    const T t = x - T(k);
    const T* cf = CoefPtr<T>::get(P) + s.tab_off + (int64_t)k * s.n_radial * 4;
    T u[kMaxRadial], du[kMaxRadial];
    const T rinv = tiny ? T(0) : T(1) / r;
#pragma unroll 4
    for (int j = 0; j < s.n_radial; ++j) {
        const T c0 = cf[4 * j], c1 = cf[4 * j + 1], c2 = cf[4 * j + 2], c3 = cf[4 * j + 3];
        const int l = s.rad_l[j];
        if (tiny) {
            // c1 / dr = R'(0) on the first interval
            u[j] = (l == 0) ? c0 : (l == 1 ? c1 * inv_dr : T(0));
            du[j] = T(0);
            continue;
        }
        const T R = c0 + t * (c1 + t * (c2 + t * c3));
        T rl_inv = T(1);
        for (int q = 0; q < l; ++q) rl_inv *= rinv;
        u[j] = R * rl_inv;
        if (kGrad) {
            const T dR = (c1 + t * (T(2) * c2 + t * (T(3) * c3))) * inv_dr;
            du[j] = (dR - T(l) * R * rinv) * rl_inv;
        }
    }
    T S[16];
    T GS[16][3];
    solid_harm<T>(s.lmax, dx, dy, dz, S, kGrad ? GS : nullptr);
    for (int o = 0; o < s.n_orb; ++o) {
        const int j = s.orb_rad[o], l = s.orb_l[o];
        const int idx = l * l + s.orb_m[o];
        if (tiny) {
            phi[o] = (l == 0) ? u[j] * S[0] : T(0);
            if (kGrad) {
                const T gs = (l == 1) ? u[j] : T(0);
                G[o][0] = gs * GS[idx][0]; G[o][1] = gs * GS[idx][1]; G[o][2] = gs * GS[idx][2];
            }
            continue;
        }
        phi[o] = u[j] * S[idx];
        if (kGrad) {
            const T a = du[j] * rinv * S[idx];
            G[o][0] = a * dx + u[j] * GS[idx][0];
            G[o][1] = a * dy + u[j] * GS[idx][1];
            G[o][2] = a * dz + u[j] * GS[idx][2];
        }
    }
    return true;
}

// Grid point of local index p in brick (b0, b1, b2); false if p is padding or
// outside the grid.
__device__ __forceinline__ bool brick_point(const GridDev& g, int b0, int b1, int b2, int p, int& g0, int& g1, int& g2) {
    if (p >= g.bpts) return false;
    const int l2 = p % g.B[2];
    const int l1 = (p / g.B[2]) % g.B[1];
    const int l0 = p / (g.B[2] * g.B[1]);
    g0 = b0 * g.B[0] + l0;
    g1 = b1 * g.B[1] + l1;
    g2 = b2 * g.B[2] + l2;
    return g0 < g.n[0] && g1 < g.n[1] && g2 < g.n[2];
}

__device__ __forceinline__ void brick_coords(const GridDev& g, int b, int& b0, int& b1, int& b2) {
    b2 = b % g.nb[2];
    b1 = (b / g.nb[2]) % g.nb[1];
    b0 = b / (g.nb[2] * g.nb[1]);
}

// The three helpers below fix every rounding (no contraction left to the
// compiler), so that the set-up tile masks and the kernels that read them see
// the same offsets and the same in/out decisions.
//
// In-brick offset of local point p in FP32; the grid step is carried as two
// FP32 words (hi + lo), so the offset has rounding errors only.
__device__ __forceinline__ void point_offset(const GridDev& g, int p, float& fx, float& fy, float& fz) {
    const int l2 = p % g.B[2], l1 = (p / g.B[2]) % g.B[1], l0 = p / (g.B[2] * g.B[1]);
    const float f0 = (float)l0, f1 = (float)l1, f2 = (float)l2;
    float v[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float hi = __fmaf_rn(f2, g.step_hi[2][c], __fmaf_rn(f1, g.step_hi[1][c], __fmul_rn(f0, g.step_hi[0][c])));
        const float lo = __fmaf_rn(f2, g.step_lo[2][c], __fmaf_rn(f1, g.step_lo[1][c], __fmul_rn(f0, g.step_lo[0][c])));
        v[c] = __fadd_rn(hi, lo);
    }
    fx = v[0]; fy = v[1]; fz = v[2];
}

// (origin of brick (b0, b1, b2)) - (atom image position) in FP64, split into two FP32 words.
__device__ __forceinline__ void brick_atom_offset(const GridDev& g, int b0, int b1, int b2, const ExtAtom& X,
                                                  float c_hi[3], float c_lo[3]) {
    const double s0 = (double)(b0 * g.B[0]), s1 = (double)(b1 * g.B[1]), s2 = (double)(b2 * g.B[2]);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const double o = __dadd_rn(__dadd_rn(__dmul_rn(s0, g.step[0][q]), __dmul_rn(s1, g.step[1][q])), __dmul_rn(s2, g.step[2][q]));
        const double c = __dsub_rn(o, X.p[q]);
        c_hi[q] = __double2float_rn(c);
        c_lo[q] = __double2float_rn(__dsub_rn(c, (double)c_hi[q]));
    }
}

// |point - atom image| < rc for the point at in-brick offset f (FP32).
__device__ __forceinline__ bool point_within(const float c_hi[3], const float c_lo[3], float fx, float fy, float fz,
                                             float rc) {
    const float dx = __fadd_rn(__fadd_rn(c_hi[0], fx), c_lo[0]);
    const float dy = __fadd_rn(__fadd_rn(c_hi[1], fy), c_lo[1]);
    const float dz = __fadd_rn(__fadd_rn(c_hi[2], fz), c_lo[2]);
    return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx))) < __fmul_rn(rc, rc);
}

}  // namespace gint
