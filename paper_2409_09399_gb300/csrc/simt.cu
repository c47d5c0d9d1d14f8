// simt.cu -- SIMT (CUDA-core) kernels of the grid integrals, FP64 and FP32.
//
// One persistent CTA takes bricks from a work counter.  Per brick it
//   1. loads the brick's atom images and the weights W_p = V_p dV,
//   2. evaluates every orbital value of every atom image at every point of
//      the brick into its slice of device scratch, laid out [orbital][point]
//      (the paper's orbital-value kernel, Section 2.3.3), recording for each
//      atom image the 32-point sub-tiles where it is non-zero,
//   3. builds the brick's pair table: for atom images a1 <= a2 whose
//      sub-tile masks intersect, the offset of the canonical pattern block
//      (I1, I2, T2 - T1) (the brick's atoms are sorted by (I, t), so a1 < a2
//      always maps to a canonical block),
//   4. contracts: H blocks (Eq. 2), rho (Eq. 3) or force/virial (Eq. 4, 5).
// The FP64 form computes the displacement, orbital values and products in
// FP64.  The FP32 form takes the displacement in FP64, rounds it to FP32 and
// evaluates orbitals and per-brick products in FP32; accumulation into H,
// rho, F and the stress stays FP64.
#include <algorithm>
#include <cstring>

#include "gint_impl.cuh"

namespace gint {

struct AtomS {
    double p[3];
    int I;
    int sp;
    int nw;
    int off;  // first orbital of this atom image in the brick
    int t[3];
    int pad;
    unsigned long long mask;  // sub-tiles where the atom image is non-zero
};

struct SimtArgs {
    Problem P;
    int max_atoms;      // capacity of the smem atom / pair tables
    size_t cta_stride;  // scratch bytes per CTA
    char* scratch;      // n_ctas * cta_stride bytes
    int* counter;       // work counter (zero before launch)
};

size_t simt_smem_bytes(int max_atoms, int bpad) {
    return sizeof(AtomS) * max_atoms + sizeof(int64_t) * (size_t)max_atoms * max_atoms + sizeof(double) * bpad + 64;
}

struct SimtSmem {
    AtomS* at;
    int64_t* pairoff;
    double* W;
};

__device__ __forceinline__ SimtSmem simt_smem(unsigned char* smem, int max_atoms) {
    SimtSmem s;
    s.at = (AtomS*)smem;
    s.pairoff = (int64_t*)(s.at + max_atoms);
    s.W = (double*)(s.pairoff + (size_t)max_atoms * max_atoms);
    return s;
}

__device__ __forceinline__ int next_work(int* counter, int* s_slot) {
    if (threadIdx.x == 0) *s_slot = atomicAdd(counter, 1);
    __syncthreads();
    const int w = *s_slot;
    __syncthreads();
    return w;
}

// Shared prologue: load the brick, weights, orbital values, masks and pair table.
// kWeighted: also write W_p * phi into psiw.
template <typename T, bool kWeighted>
__device__ int brick_prologue(const Problem& P, int brick, const double* V, SimtSmem S, T* psi, T* psiw) {
    const GridDev& g = P.g;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int64_t s0 = P.brick_start[brick];
    const int na = (int)(P.brick_start[brick + 1] - s0);
    int b0, b1, b2;
    brick_coords(g, brick, b0, b1, b2);
    for (int i = tid; i < na; i += nth) {
        const ExtAtom X = P.ext[P.brick_atoms[s0 + i]];
        AtomS& a = S.at[i];
        a.p[0] = X.p[0]; a.p[1] = X.p[1]; a.p[2] = X.p[2];
        a.I = X.atom;
        a.sp = X.species;
        a.nw = P.sp[X.species].n_orb;
        a.t[0] = X.t[0]; a.t[1] = X.t[1]; a.t[2] = X.t[2];
        a.mask = 0ull;
    }
    for (int p = tid; p < g.bpad; p += nth) {
        int g0, g1, g2;
        double w = 0.0;
        if (V && brick_point(g, b0, b1, b2, p, g0, g1, g2))
            w = V[((int64_t)g0 * g.n[1] + g1) * g.n[2] + g2] * g.dV;
        S.W[p] = w;
    }
    __syncthreads();
    if (tid == 0) {
        int off = 0;
        for (int i = 0; i < na; ++i) { S.at[i].off = off; off += S.at[i].nw; }
    }
    __syncthreads();
    // orbital values: item = (atom image, point); a warp covers one sub-tile of one atom
    T phi[kMaxNw];
    const int nitems = na * g.bpad;
    for (int item0 = 0; item0 < nitems; item0 += nth) {
        const int item = item0 + tid;
        const bool live = item < nitems;
        const int a = live ? item / g.bpad : 0;
        const int p = live ? item - a * g.bpad : 0;
        bool inside = false;
        if (live) {
            const AtomS& X = S.at[a];
            int g0, g1, g2;
            if (brick_point(g, b0, b1, b2, p, g0, g1, g2)) {
                const double rx = g0 * g.step[0][0] + g1 * g.step[1][0] + g2 * g.step[2][0];
                const double ry = g0 * g.step[0][1] + g1 * g.step[1][1] + g2 * g.step[2][1];
                const double rz = g0 * g.step[0][2] + g1 * g.step[1][2] + g2 * g.step[2][2];
                const T dx = (T)(rx - X.p[0]), dy = (T)(ry - X.p[1]), dz = (T)(rz - X.p[2]);
                inside = eval_atom<T, false>(P, P.sp[X.sp], dx, dy, dz, phi, nullptr);
            }
            T* out = psi + (size_t)X.off * g.bpad + p;
            const T w = (T)S.W[p];
            for (int o = 0; o < X.nw; ++o) {
                const T v = inside ? phi[o] : T(0);
                out[(size_t)o * g.bpad] = v;
                if (kWeighted) psiw[(size_t)(X.off + o) * g.bpad + p] = v * w;
            }
        }
        // bpad is a multiple of 32 and nth a multiple of 32, so a warp's live
        // lanes share one atom image and one sub-tile
        const unsigned bal = __ballot_sync(0xffffffffu, inside);
        if ((threadIdx.x & 31) == 0 && bal) atomicOr(&S.at[a].mask, 1ull << (p >> 5));
    }
    __syncthreads();
    // pair table (dense na x na; both orientations hold the canonical block offset)
    for (int q = tid; q < na * na; q += nth) {
        const int a1 = q / na, a2 = q - a1 * na;
        if (a1 > a2) continue;
        int64_t off = -1;
        if (S.at[a1].mask & S.at[a2].mask) {
            // two images can reach one sub-tile without overlapping each other:
            // only pairs closer than rc1 + rc2 are in the pattern (and only those
            // have a non-zero product anywhere)
            const AtomS &X = S.at[a1], &Y = S.at[a2];
            const double dx = Y.p[0] - X.p[0], dy = Y.p[1] - X.p[1], dz = Y.p[2] - X.p[2];
            const double dist = sqrt(dx * dx + dy * dy + dz * dz);
            const double cut = P.sp[X.sp].rc + P.sp[Y.sp].rc;
            if (dist < cut + 1e-9) {
                const int64_t blk = find_block(P, X.I, Y.I, Y.t[0] - X.t[0], Y.t[1] - X.t[1], Y.t[2] - X.t[2]);
                if (blk >= 0) off = P.offsets[blk];
                else if (dist < cut - 1e-9) atomicOr(P.err, kErrPatternMissing);
            }
        }
        S.pairoff[a1 * na + a2] = off;
        S.pairoff[a2 * na + a1] = off;
    }
    __syncthreads();
    return na;
}

// ------------------------------------------------------------------- H^V
// Warps take atom-image pairs (a1 <= a2); a lane owns up to 8 elements of the
// nw1 x nw2 block per pass and sums psi[a1,mu](p) * W_p psi[a2,nu](p) over the
// points of the sub-tiles both atoms reach; the block is added to H with
// FP64 atomics (several bricks meet every block).
template <typename T>
__global__ void __launch_bounds__(256) k_vlocal_simt(SimtArgs A, const double* V, double* H) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_slot, s_next;
    const Problem& P = A.P;
    const GridDev& g = P.g;
    SimtSmem S = simt_smem(smem, A.max_atoms);
    T* psi = (T*)(A.scratch + (size_t)blockIdx.x * A.cta_stride);
    T* psiw = psi + (A.cta_stride / sizeof(T)) / 2;
    const int lane = threadIdx.x & 31;
    for (;;) {
        const int w = next_work(A.counter, &s_slot);
        if (w >= P.n_work) break;
        const int brick = P.work[w];
        if (threadIdx.x == 0) s_next = 0;
        const int na = brick_prologue<T, true>(P, brick, V, S, psi, psiw);
        for (;;) {
            int q = 0;
            if (lane == 0) q = atomicAdd(&s_next, 1);
            q = __shfl_sync(0xffffffffu, q, 0);
            if (q >= na * na) break;
            const int a1 = q / na, a2 = q - a1 * na;
            if (a1 > a2) continue;
            const int64_t off = S.pairoff[q];
            if (off < 0) continue;
            const AtomS &X = S.at[a1], &Y = S.at[a2];
            const unsigned long long m = X.mask & Y.mask;
            const int n1 = X.nw, n2 = Y.nw, ne = n1 * n2;
            for (int e0 = 0; e0 < ne; e0 += 256) {
                T acc[8];
                const T* ra[8];
                const T* rb[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    acc[k] = T(0);
                    int e = e0 + lane + 32 * k;
                    if (e >= ne) e = ne - 1;
                    const int mu = e / n2, nu = e - mu * n2;
                    ra[k] = psi + (size_t)(X.off + mu) * g.bpad;
                    rb[k] = psiw + (size_t)(Y.off + nu) * g.bpad;
                }
                unsigned long long mm = m;
                while (mm) {
                    const int s = __ffsll((long long)mm) - 1;
                    mm &= mm - 1;
                    for (int pp = 0; pp < 32; ++pp) {
                        const int p = 32 * s + pp;
#pragma unroll
                        for (int k = 0; k < 8; ++k) acc[k] += ra[k][p] * rb[k][p];
                    }
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int e = e0 + lane + 32 * k;
                    if (e < ne) atomicAdd(H + off + e, (double)acc[k]);
                }
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------- rho
// Warps take 32-point sub-tiles (lane = point).  For every pair a1 <= a2
// reaching the sub-tile, t = psi_a1(p)^T D_(a1,a2) psi_a2(p) with the
// canonical block; off-diagonal pairs count twice (D is symmetric).
template <typename T, int kNw>
__global__ void __launch_bounds__(256) k_rho_simt(SimtArgs A, const double* D, double* rho) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_slot, s_next;
    const Problem& P = A.P;
    const GridDev& g = P.g;
    SimtSmem S = simt_smem(smem, A.max_atoms);
    T* psi = (T*)(A.scratch + (size_t)blockIdx.x * A.cta_stride);
    const int lane = threadIdx.x & 31;
    for (;;) {
        const int w = next_work(A.counter, &s_slot);
        if (w >= P.n_work) break;
        const int brick = P.work[w];
        if (threadIdx.x == 0) s_next = 0;
        const int na = brick_prologue<T, false>(P, brick, nullptr, S, psi, nullptr);
        int b0, b1, b2;
        brick_coords(g, brick, b0, b1, b2);
        for (;;) {
            int s = 0;
            if (lane == 0) s = atomicAdd(&s_next, 1);
            s = __shfl_sync(0xffffffffu, s, 0);
            if (s >= g.nsub) break;
            const int p = 32 * s + lane;
            const unsigned long long bit = 1ull << s;
            double acc = 0.0;
            for (int a1 = 0; a1 < na; ++a1) {
                const AtomS& X = S.at[a1];
                if (!(X.mask & bit)) continue;
                T x1[kNw];
#pragma unroll
                for (int o = 0; o < kNw; ++o) x1[o] = o < X.nw ? psi[(size_t)(X.off + o) * g.bpad + p] : T(0);
                for (int a2 = a1; a2 < na; ++a2) {
                    const AtomS& Y = S.at[a2];
                    const int64_t off = S.pairoff[a1 * na + a2];
                    if (off < 0 || !(Y.mask & bit)) continue;
                    T x2[kNw];
#pragma unroll
                    for (int o = 0; o < kNw; ++o) x2[o] = o < Y.nw ? psi[(size_t)(Y.off + o) * g.bpad + p] : T(0);
                    const double* Db = D + off;
                    T t = T(0);
                    const int n2 = Y.nw;
#pragma unroll
                    for (int mu = 0; mu < kNw; ++mu) {
                        if (mu >= X.nw) break;
                        T r = T(0);
#pragma unroll
                        for (int nu = 0; nu < kNw; ++nu) {
                            if (nu >= n2) break;
                            r += (T)__ldg(Db + mu * n2 + nu) * x2[nu];
                        }
                        t += x1[mu] * r;
                    }
                    acc += (a1 == a2 ? 1.0 : 2.0) * (double)t;
                }
            }
            int g0, g1, g2;
            if (brick_point(g, b0, b1, b2, p, g0, g1, g2)) rho[((int64_t)g0 * g.n[1] + g1) * g.n[2] + g2] = acc;
        }
        __syncthreads();
    }
}

// Zero rho on bricks without atoms.
__global__ void k_rho_empty(GridDev g, const int32_t* empty, int64_t n_empty, double* rho) {
    for (int64_t w = blockIdx.x; w < n_empty; w += gridDim.x) {
        int b0, b1, b2;
        brick_coords(g, empty[w], b0, b1, b2);
        for (int p = threadIdx.x; p < g.bpts; p += blockDim.x) {
            int g0, g1, g2;
            if (brick_point(g, b0, b1, b2, p, g0, g1, g2)) rho[((int64_t)g0 * g.n[1] + g1) * g.n[2] + g2] = 0.0;
        }
    }
}

// ------------------------------------------------------- force and virial
// Warps take (sub-tile, atom image a1) items (lane = point):
//   G_mu = sum_{a2} sum_nu D_(a1,a2)[mu,nu] psi_a2,nu(p)   (both orientations)
//   f = 2 W_p sum_mu grad phi_a1,mu(p) G_mu ;  F_I1 += f ; Pi_I1 += f (x) d
//   E += W_p sum_mu phi_a1,mu(p) G_mu
// acc: per atom [F(3), Pi(9)] FP64, E at acc_e.
template <typename T, int kNw>
__global__ void __launch_bounds__(256) k_force_simt(SimtArgs A, const double* V, const double* D, double* acc,
                                                    double* acc_e) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_slot, s_next;
    __shared__ double s_e;
    const Problem& P = A.P;
    const GridDev& g = P.g;
    SimtSmem S = simt_smem(smem, A.max_atoms);
    T* psi = (T*)(A.scratch + (size_t)blockIdx.x * A.cta_stride);
    const int lane = threadIdx.x & 31;
    for (;;) {
        const int w = next_work(A.counter, &s_slot);
        if (w >= P.n_work) break;
        const int brick = P.work[w];
        if (threadIdx.x == 0) { s_next = 0; s_e = 0.0; }
        const int na = brick_prologue<T, false>(P, brick, V, S, psi, nullptr);
        int b0, b1, b2;
        brick_coords(g, brick, b0, b1, b2);
        double e_loc = 0.0;
        for (;;) {
            int q = 0;
            if (lane == 0) q = atomicAdd(&s_next, 1);
            q = __shfl_sync(0xffffffffu, q, 0);
            if (q >= g.nsub * na) break;
            const int s = q / na, a1 = q - s * na;
            const unsigned long long bit = 1ull << s;
            const AtomS& X = S.at[a1];
            if (!(X.mask & bit)) continue;
            const int p = 32 * s + lane;
            T G[kNw];
#pragma unroll
            for (int o = 0; o < kNw; ++o) G[o] = T(0);
            const int n1 = X.nw;
            for (int a2 = 0; a2 < na; ++a2) {
                const AtomS& Y = S.at[a2];
                const int64_t off = S.pairoff[a1 * na + a2];
                if (off < 0 || !(Y.mask & bit)) continue;
                T x2[kNw];
#pragma unroll
                for (int o = 0; o < kNw; ++o) x2[o] = o < Y.nw ? psi[(size_t)(Y.off + o) * g.bpad + p] : T(0);
                const double* Db = D + off;
                const int n2 = Y.nw;
                if (a1 <= a2) {
                    // canonical block (I1, I2) is n1 x n2
#pragma unroll
                    for (int mu = 0; mu < kNw; ++mu) {
                        if (mu >= n1) break;
                        T r = T(0);
#pragma unroll
                        for (int nu = 0; nu < kNw; ++nu) {
                            if (nu >= n2) break;
                            r += (T)__ldg(Db + mu * n2 + nu) * x2[nu];
                        }
                        G[mu] += r;
                    }
                } else {
                    // canonical block (I2, I1) is n2 x n1; use its transpose
#pragma unroll
                    for (int nu = 0; nu < kNw; ++nu) {
                        if (nu >= n2) break;
                        const T xv = x2[nu];
#pragma unroll
                        for (int mu = 0; mu < kNw; ++mu) {
                            if (mu >= n1) break;
                            G[mu] += (T)__ldg(Db + nu * n1 + mu) * xv;
                        }
                    }
                }
            }
            // gradient of a1's orbitals at p
            double f[3] = {0, 0, 0}, vir[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
            double e_pt = 0.0;
            int g0, g1, g2;
            if (brick_point(g, b0, b1, b2, p, g0, g1, g2)) {
                const double rx = g0 * g.step[0][0] + g1 * g.step[1][0] + g2 * g.step[2][0];
                const double ry = g0 * g.step[0][1] + g1 * g.step[1][1] + g2 * g.step[2][1];
                const double rz = g0 * g.step[0][2] + g1 * g.step[1][2] + g2 * g.step[2][2];
                const double ddx = rx - X.p[0], ddy = ry - X.p[1], ddz = rz - X.p[2];
                T phi[kMaxNw], gr[kMaxNw][3];
                if (eval_atom<T, true>(P, P.sp[X.sp], (T)ddx, (T)ddy, (T)ddz, phi, gr)) {
                    T fx = T(0), fy = T(0), fz = T(0), ee = T(0);
#pragma unroll
                    for (int mu = 0; mu < kNw; ++mu) {
                        if (mu >= n1) break;
                        fx += gr[mu][0] * G[mu];
                        fy += gr[mu][1] * G[mu];
                        fz += gr[mu][2] * G[mu];
                        ee += phi[mu] * G[mu];
                    }
                    const double wv = S.W[p];
                    f[0] = 2.0 * wv * (double)fx;
                    f[1] = 2.0 * wv * (double)fy;
                    f[2] = 2.0 * wv * (double)fz;
                    const double dd[3] = {ddx, ddy, ddz};
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b) vir[3 * a + b] = f[a] * dd[b];
                    e_pt = wv * (double)ee;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                for (int a = 0; a < 3; ++a) f[a] += __shfl_down_sync(0xffffffffu, f[a], o);
                for (int a = 0; a < 9; ++a) vir[a] += __shfl_down_sync(0xffffffffu, vir[a], o);
                e_pt += __shfl_down_sync(0xffffffffu, e_pt, o);
            }
            if (lane == 0) {
                double* out = acc + 12 * (size_t)X.I;
                for (int a = 0; a < 3; ++a) atomicAdd(out + a, f[a]);
                for (int a = 0; a < 9; ++a) atomicAdd(out + 3 + a, vir[a]);
                e_loc += e_pt;
            }
        }
        if (lane == 0 && e_loc != 0.0) atomicAdd(&s_e, e_loc);
        __syncthreads();
        if (threadIdx.x == 0 && s_e != 0.0) atomicAdd(acc_e, s_e);
        __syncthreads();
    }
}

// Rewrite every non-canonical block as the transpose of its mirror block.
__global__ void k_mirror_h(Problem P, const int32_t* mirror, const int* nw_atom, int64_t n_blocks, double* H) {
    const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (b >= n_blocks) return;
    const int32_t* k = P.blocks + 5 * b;
    const int I = k[0], J = k[1];
    const bool canon = (I < J) || (I == J && (k[2] > 0 || (k[2] == 0 && (k[3] > 0 || (k[3] == 0 && k[4] >= 0)))));
    if (canon) return;
    const int64_t m = mirror[b];
    if (m < 0) return;
    const int nI = nw_atom[I], nJ = nw_atom[J];
    const double* src = H + P.offsets[m];  // block (J, I, -T): nJ x nI
    double* dst = H + P.offsets[b];        // block (I, J, T):  nI x nJ
    for (int e = lane; e < nI * nJ; e += 32) {
        const int mu = e / nJ, nu = e - mu * nJ;
        dst[e] = src[nu * nI + mu];
    }
}

// F, per-atom virial, stress and energy from the accumulators.  One CTA;
// the stress sum runs over atoms in a fixed order per thread and a fixed tree.
__global__ void k_force_finalize(int n_atoms, double omega, const double* acc, const double* acc_e, double* F,
                                 double* sigma, double* virial, double* E) {
    __shared__ double s[9][256];
    double v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = threadIdx.x; i < n_atoms; i += blockDim.x) {
        const double* a = acc + 12 * (size_t)i;
        if (F) for (int c = 0; c < 3; ++c) F[3 * (size_t)i + c] = a[c];
        if (virial) for (int c = 0; c < 9; ++c) virial[9 * (size_t)i + c] = a[3 + c];
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
        if (sigma) for (int c = 0; c < 9; ++c) sigma[c] = -s[c][0] / omega;
        if (E) *E = *acc_e;
    }
}

// ----------------------------------------------------------------- host
static int simt_ctas_per_sm(size_t smem) {
    if (smem > 110 * 1024) return 1;
    return 2;
}

gint_status allocate_scratch(gint_handle* h) {
    const int bpad = h->grid.bpad;
    const size_t smem = simt_smem_bytes(std::max(1, h->max_brick_atoms), bpad);
    if (smem > 220 * 1024) {
        set_error("brick tables need %zu bytes of shared memory; use smaller bricks", smem);
        return GINT_ERR_UNSUPPORTED;
    }
    h->n_ctas = h->sm_count * simt_ctas_per_sm(smem);
    // psi and W*psi, FP64
    const size_t per_cta = (size_t)2 * std::max(1, h->max_brick_orb) * bpad * sizeof(double);
    h->scratch_bytes = per_cta * h->n_ctas + 256;
    GINT_CUDA_TRY(dev_malloc(&h->d_scratch, h->scratch_bytes));
    return GINT_OK;
}

template <typename T>
static gint_status launch_simt(gint_handle* h, int which, const double* V, const double* D, double* out0,
                               double* acc, double* acc_e, cudaStream_t st) {
    SimtArgs A;
    A.P = h->problem();
    A.max_atoms = std::max(1, h->max_brick_atoms);
    A.cta_stride = (size_t)2 * std::max(1, h->max_brick_orb) * h->grid.bpad * sizeof(double);
    A.scratch = (char*)h->d_scratch;
    A.counter = h->d_err + 2;
    GINT_CUDA_TRY(cudaMemsetAsync(A.counter, 0, sizeof(int), st));
    const size_t smem = simt_smem_bytes(A.max_atoms, h->grid.bpad);
    const int grid = h->n_ctas;
    if (which == 0) {
        GINT_CUDA_TRY(cudaFuncSetAttribute(k_vlocal_simt<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_vlocal_simt<T><<<grid, 256, smem, st>>>(A, V, out0);
    } else if (which == 1) {
        if (h->max_nw <= 16) {
            GINT_CUDA_TRY(cudaFuncSetAttribute(k_rho_simt<T, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_rho_simt<T, 16><<<grid, 256, smem, st>>>(A, D, out0);
        } else {
            GINT_CUDA_TRY(cudaFuncSetAttribute(k_rho_simt<T, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_rho_simt<T, 32><<<grid, 256, smem, st>>>(A, D, out0);
        }
    } else {
        if (h->max_nw <= 16) {
            GINT_CUDA_TRY(cudaFuncSetAttribute(k_force_simt<T, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_force_simt<T, 16><<<grid, 256, smem, st>>>(A, V, D, acc, acc_e);
        } else {
            GINT_CUDA_TRY(cudaFuncSetAttribute(k_force_simt<T, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_force_simt<T, 32><<<grid, 256, smem, st>>>(A, V, D, acc, acc_e);
        }
    }
    GINT_CUDA_TRY(cudaGetLastError());
    return GINT_OK;
}

gint_status simt_run(gint_handle* h, int which, bool fp32, const double* V, const double* D, double* out,
                     double* acc, double* acc_e, cudaStream_t st) {
    if (h->n_work == 0) return GINT_OK;
    return fp32 ? launch_simt<float>(h, which, V, D, out, acc, acc_e, st)
                : launch_simt<double>(h, which, V, D, out, acc, acc_e, st);
}

gint_status launch_mirror(gint_handle* h, double* H, cudaStream_t st) {
    if (h->n_blocks == 0) return GINT_OK;
    const int64_t threads = h->n_blocks * 32;
    k_mirror_h<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(h->problem(), h->d_mirror, h->d_nw_atom,
                                                                   h->n_blocks, H);
    GINT_CUDA_TRY(cudaGetLastError());
    return GINT_OK;
}

gint_status launch_rho_empty(gint_handle* h, double* rho, cudaStream_t st) {
    if (h->n_empty == 0) return GINT_OK;
    const int64_t nb = std::min<int64_t>(h->n_empty, (int64_t)h->sm_count * 16);
    k_rho_empty<<<(unsigned)nb, 256, 0, st>>>(h->grid, h->d_empty, h->n_empty, rho);
    GINT_CUDA_TRY(cudaGetLastError());
    return GINT_OK;
}

gint_status launch_force_finalize(gint_handle* h, double* F, double* sigma, double* virial, double* E,
                                  cudaStream_t st) {
    k_force_finalize<<<1, 256, 0, st>>>(h->n_atoms, h->omega, h->d_facc, h->d_red, F, sigma, virial, E);
    GINT_CUDA_TRY(cudaGetLastError());
    return GINT_OK;
}

}  // namespace gint

namespace gint {
// Launch the FP64 H^V SIMT kernel on caller-provided scratch (n_ctas slices of
// `cta_stride` bytes).  Used by the entry point that allocates nothing.
gint_status simt_vlocal_on_scratch(gint_handle* h, const double* V, double* H, char* scratch, size_t cta_stride,
                                   int n_ctas, cudaStream_t st) {
    if (h->n_work == 0) return GINT_OK;
    SimtArgs A;
    A.P = h->problem();
    A.max_atoms = std::max(1, h->max_brick_atoms);
    A.cta_stride = cta_stride;
    A.scratch = scratch;
    A.counter = h->d_err + 2;
    GINT_CUDA_TRY(cudaMemsetAsync(A.counter, 0, sizeof(int), st));
    const size_t smem = simt_smem_bytes(A.max_atoms, h->grid.bpad);
    GINT_CUDA_TRY(cudaFuncSetAttribute(k_vlocal_simt<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_vlocal_simt<double><<<n_ctas, 256, smem, st>>>(A, V, H);
    GINT_CUDA_TRY(cudaGetLastError());
    return GINT_OK;
}
}  // namespace gint
