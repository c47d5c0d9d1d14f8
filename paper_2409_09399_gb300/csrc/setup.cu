// setup.cu -- handle creation: tables, pair pattern, brick binner, ABI plumbing.
//
// The pair pattern is the overlapping-cutoff sparsity of Section 2.2 (blocks
// (I, J, T) with |R_J + T - R_I| < rc_I + rc_J).  The binner replaces the
// host-side sub-task generation of Section 2.3.2: for every brick of grid
// points it lists, on the device, the atom images whose cutoff sphere meets
// the brick (the "neighbouring atoms" of that batch).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <string>
#include <vector>

#include "gint_impl.cuh"
#include "nvtx.cuh"

namespace gint {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

// ------------------------------------------------------------ small scans
// Exclusive scan of n int64 values in place, out[n] = total.  Three kernels:
// per-tile sums, a serial scan of the tile sums, per-tile scans.
constexpr int kScanTile = 1024;

__global__ void k_scan_tile_sums(const int64_t* in, int64_t n, int64_t* sums) {
    __shared__ int64_t s[32];
    int64_t i = (int64_t)blockIdx.x * kScanTile + threadIdx.x;
    int64_t v = i < n ? in[i] : 0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = s[threadIdx.x];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) sums[blockIdx.x] = v;
    }
}

__global__ void k_scan_serial(int64_t* sums, int64_t m, int64_t* total) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int64_t acc = 0;
    for (int64_t i = 0; i < m; ++i) { int64_t v = sums[i]; sums[i] = acc; acc += v; }
    *total = acc;
}

__global__ void k_scan_apply(const int64_t* in, int64_t n, const int64_t* sums, int64_t* out) {
    __shared__ int64_t s[32];
    int64_t i = (int64_t)blockIdx.x * kScanTile + threadIdx.x;
    int64_t v = i < n ? in[i] : 0;
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s[w] = x;
    __syncthreads();
    if (w == 0) {
        int64_t t = s[lane];
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        s[lane] = t;
    }
    __syncthreads();
    int64_t excl = x - v + (w > 0 ? s[w - 1] : 0) + sums[blockIdx.x];
    if (i < n) out[i] = excl;
}

// in and out may alias; out must hold n + 1 values.
static gint_status scan_exclusive(const int64_t* in, int64_t n, int64_t* out, cudaStream_t st) {
    int64_t tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles == 0) {
        GINT_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(int64_t), st));
        return GINT_OK;
    }
    int64_t* sums = nullptr;
    GINT_CUDA_TRY(dev_malloc(&sums, sizeof(int64_t) * (tiles + 1)));
    k_scan_tile_sums<<<(unsigned)tiles, kScanTile, 0, st>>>(in, n, sums);
    k_scan_serial<<<1, 32, 0, st>>>(sums, tiles, sums + tiles);
    k_scan_apply<<<(unsigned)tiles, kScanTile, 0, st>>>(in, n, sums, out);
    cudaError_t e = cudaMemcpyAsync(out + n, sums + tiles, sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
    cudaError_t e2 = cudaStreamSynchronize(st);
    cudaFree(sums);
    GINT_CUDA_TRY(e);
    GINT_CUDA_TRY(e2);
    GINT_CUDA_TRY(cudaGetLastError());
    return GINT_OK;
}

// ------------------------------------------------------------- pattern
struct CellDev {
    double A[3][3];     // rows a_i
    double Ainv[3][3];  // fractional f = r Ainv
    double h[3];        // interplanar spacings
};

__device__ __forceinline__ void frac_of(const CellDev& c, const double r[3], double f[3]) {
    for (int i = 0; i < 3; ++i) f[i] = r[0] * c.Ainv[0][i] + r[1] * c.Ainv[1][i] + r[2] * c.Ainv[2][i];
}

// Visit the images t of J with |R_J + T - R_I| < rc_I + rc_J in lexicographic
// order; returns the count and (if out != null) writes (J, t0, t1, t2).
__device__ int pair_images(const CellDev& c, const double* pos, int I, int J, double cut, int32_t* out) {
    double d[3] = {pos[3 * J] - pos[3 * I], pos[3 * J + 1] - pos[3 * I + 1], pos[3 * J + 2] - pos[3 * I + 2]};
    double f[3];
    frac_of(c, d, f);
    int lo[3], hi[3];
    for (int i = 0; i < 3; ++i) {
        double w = cut / c.h[i];
        lo[i] = (int)ceil(-f[i] - w - 1e-9);
        hi[i] = (int)floor(-f[i] + w + 1e-9);
        if (lo[i] > hi[i]) return 0;
    }
    int n = 0;
    for (int t0 = lo[0]; t0 <= hi[0]; ++t0)
        for (int t1 = lo[1]; t1 <= hi[1]; ++t1)
            for (int t2 = lo[2]; t2 <= hi[2]; ++t2) {
                double v0 = d[0] + t0 * c.A[0][0] + t1 * c.A[1][0] + t2 * c.A[2][0];
                double v1 = d[1] + t0 * c.A[0][1] + t1 * c.A[1][1] + t2 * c.A[2][1];
                double v2 = d[2] + t0 * c.A[0][2] + t1 * c.A[1][2] + t2 * c.A[2][2];
                if (v0 * v0 + v1 * v1 + v2 * v2 < cut * cut) {
                    if (out) { out[4 * n] = J; out[4 * n + 1] = t0; out[4 * n + 2] = t1; out[4 * n + 3] = t2; }
                    ++n;
                }
            }
    return n;
}

// One CTA per atom I: count blocks and values of row I.
__global__ void k_pattern_count(CellDev c, int n_atoms, const double* pos, const int* spc, const double* rc_sp,
                                const int* nw_sp, int64_t* row_count, int64_t* row_vals) {
    int I = blockIdx.x;
    double rcI = rc_sp[spc[I]];
    int64_t cnt = 0, vals = 0;
    for (int J = threadIdx.x; J < n_atoms; J += blockDim.x) {
        int n = pair_images(c, pos, I, J, rcI + rc_sp[spc[J]], nullptr);
        cnt += n;
        vals += (int64_t)n * nw_sp[spc[I]] * nw_sp[spc[J]];
    }
    __shared__ int64_t sc[32], sv[32];
    for (int o = 16; o > 0; o >>= 1) {
        cnt += __shfl_down_sync(0xffffffffu, cnt, o);
        vals += __shfl_down_sync(0xffffffffu, vals, o);
    }
    if ((threadIdx.x & 31) == 0) { sc[threadIdx.x >> 5] = cnt; sv[threadIdx.x >> 5] = vals; }
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t a = 0, b = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += sc[w]; b += sv[w]; }
        row_count[I] = a;
        row_vals[I] = b;
    }
}

// One CTA (256 threads) per atom I: write the sorted blocks and offsets of row I.
// Candidates J are taken in chunks of 256; a block-wide exclusive scan of the
// per-J counts keeps the (J, t) order.
__global__ void k_pattern_fill(CellDev c, int n_atoms, const double* pos, const int* spc, const double* rc_sp,
                               const int* nw_sp, const int64_t* row_start, const int64_t* val_start,
                               int32_t* blocks, int64_t* offsets) {
    int I = blockIdx.x;
    double rcI = rc_sp[spc[I]];
    int nwI = nw_sp[spc[I]];
    __shared__ int64_t s_cnt[256], s_val[256];
    int64_t base_b = row_start[I], base_v = val_start[I];
    for (int J0 = 0; J0 < n_atoms; J0 += 256) {
        int J = J0 + threadIdx.x;
        int n = 0;
        if (J < n_atoms) n = pair_images(c, pos, I, J, rcI + rc_sp[spc[J]], nullptr);
        int64_t v = (J < n_atoms) ? (int64_t)n * nwI * nw_sp[spc[J]] : 0;
        s_cnt[threadIdx.x] = n;
        s_val[threadIdx.x] = v;
        __syncthreads();
        // serial scan of the 256 per-J counts by thread 0
        if (threadIdx.x == 0) {
            int64_t a = 0, b = 0;
            for (int k = 0; k < 256; ++k) {
                int64_t x = s_cnt[k], y = s_val[k];
                s_cnt[k] = a; s_val[k] = b;
                a += x; b += y;
            }
        }
        __syncthreads();
        if (J < n_atoms && n > 0) {
            int64_t bpos = base_b + s_cnt[threadIdx.x];
            int64_t vpos = base_v + s_val[threadIdx.x];
            int nwJ = nw_sp[spc[J]];
            // images are visited in lexicographic order; write in chunks of 64
            double d[3] = {pos[3 * J] - pos[3 * I], pos[3 * J + 1] - pos[3 * I + 1], pos[3 * J + 2] - pos[3 * I + 2]};
            double f[3];
            frac_of(c, d, f);
            double cut = rcI + rc_sp[spc[J]];
            int lo[3], hi[3];
            for (int i = 0; i < 3; ++i) {
                double w = cut / c.h[i];
                lo[i] = (int)ceil(-f[i] - w - 1e-9);
                hi[i] = (int)floor(-f[i] + w + 1e-9);
            }
            int q = 0;
            for (int t0 = lo[0]; t0 <= hi[0]; ++t0)
                for (int t1 = lo[1]; t1 <= hi[1]; ++t1)
                    for (int t2 = lo[2]; t2 <= hi[2]; ++t2) {
                        double v0 = d[0] + t0 * c.A[0][0] + t1 * c.A[1][0] + t2 * c.A[2][0];
                        double v1 = d[1] + t0 * c.A[0][1] + t1 * c.A[1][1] + t2 * c.A[2][1];
                        double v2 = d[2] + t0 * c.A[0][2] + t1 * c.A[1][2] + t2 * c.A[2][2];
                        if (v0 * v0 + v1 * v1 + v2 * v2 < cut * cut && q < n) {
                            int32_t* o = blocks + 5 * (bpos + q);
                            o[0] = I; o[1] = J; o[2] = t0; o[3] = t1; o[4] = t2;
                            offsets[bpos + q] = vpos + (int64_t)q * nwI * nwJ;
                            ++q;
                        }
                    }
        }
        __syncthreads();
        // advance the bases by this chunk's totals
        __shared__ int64_t tot_b, tot_v;
        if (threadIdx.x == 255) {
            tot_b = s_cnt[255] + n;
            tot_v = s_val[255] + v;
        }
        __syncthreads();
        base_b += tot_b;
        base_v += tot_v;
        __syncthreads();
    }
}

// Index of the mirror block (J, I, -T) of every block.
__global__ void k_mirror(Problem P, int64_t n_blocks, int32_t* mirror) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_blocks) return;
    const int32_t* k = P.blocks + 5 * b;
    int64_t m = find_block(P, k[1], k[0], -k[2], -k[3], -k[4]);
    mirror[b] = (int32_t)m;
    if (m < 0) atomicOr(P.err, kErrPatternMissing);
}

// ---------------------------------------------------------------- binner
// Squared distance from p to the parallelepiped {o + sum u_i e_i, u in [0,1]^3}.
// Exact: the minimiser lies in the relative interior of the whole box, of a
// face or of an edge (vertices are edge end points); each candidate is
// clamped into the box, so every candidate is feasible and the least one is
// the minimum.
__device__ double hull_dist2(const double p[3], const double o[3], const double e[3][3]) {
    double q[3] = {o[0] - p[0], o[1] - p[1], o[2] - p[2]};
    double G[3][3], b[3];
    for (int i = 0; i < 3; ++i) {
        b[i] = q[0] * e[i][0] + q[1] * e[i][1] + q[2] * e[i][2];
        for (int j = 0; j < 3; ++j) G[i][j] = e[i][0] * e[j][0] + e[i][1] * e[j][1] + e[i][2] * e[j][2];
    }
    auto dist2 = [&](const double u[3]) {
        double v0 = q[0] + u[0] * e[0][0] + u[1] * e[1][0] + u[2] * e[2][0];
        double v1 = q[1] + u[0] * e[0][1] + u[1] * e[1][1] + u[2] * e[2][1];
        double v2 = q[2] + u[0] * e[0][2] + u[1] * e[1][2] + u[2] * e[2][2];
        return v0 * v0 + v1 * v1 + v2 * v2;
    };
    auto clamp01 = [](double x) { return x < 0.0 ? 0.0 : (x > 1.0 ? 1.0 : x); };
    // interior: solve G u = -b
    double det = G[0][0] * (G[1][1] * G[2][2] - G[1][2] * G[2][1]) - G[0][1] * (G[1][0] * G[2][2] - G[1][2] * G[2][0]) +
                 G[0][2] * (G[1][0] * G[2][1] - G[1][1] * G[2][0]);
    double best = 1e300;
    if (fabs(det) > 1e-30) {
        double u[3];
        u[0] = (-b[0] * (G[1][1] * G[2][2] - G[1][2] * G[2][1]) + b[1] * (G[0][1] * G[2][2] - G[0][2] * G[2][1]) -
                b[2] * (G[0][1] * G[1][2] - G[0][2] * G[1][1])) / det;
        u[1] = (b[0] * (G[1][0] * G[2][2] - G[1][2] * G[2][0]) - b[1] * (G[0][0] * G[2][2] - G[0][2] * G[2][0]) +
                b[2] * (G[0][0] * G[1][2] - G[0][2] * G[1][0])) / det;
        u[2] = (-b[0] * (G[1][0] * G[2][1] - G[1][1] * G[2][0]) + b[1] * (G[0][0] * G[2][1] - G[0][1] * G[2][0]) -
                b[2] * (G[0][0] * G[1][1] - G[0][1] * G[1][0])) / det;
        if (u[0] >= 0 && u[0] <= 1 && u[1] >= 0 && u[1] <= 1 && u[2] >= 0 && u[2] <= 1) return 0.0;
        for (int i = 0; i < 3; ++i) u[i] = clamp01(u[i]);
        best = fmin(best, dist2(u));
    }
    // faces: coordinate k fixed at v, the other two free
    for (int k = 0; k < 3; ++k) {
        int i = (k + 1) % 3, j = (k + 2) % 3;
        for (int v = 0; v <= 1; ++v) {
            double bi = b[i] + v * G[k][i], bj = b[j] + v * G[k][j];
            double d2 = G[i][i] * G[j][j] - G[i][j] * G[i][j];
            double u[3];
            u[k] = v;
            if (fabs(d2) > 1e-30) {
                u[i] = clamp01((-bi * G[j][j] + bj * G[i][j]) / d2);
                u[j] = clamp01((-bj * G[i][i] + bi * G[i][j]) / d2);
            } else {
                u[i] = 0; u[j] = 0;
            }
            best = fmin(best, dist2(u));
            // edges of this face: coordinate j fixed at 0/1, i free (covers all 12 edges)
            for (int w = 0; w <= 1; ++w) {
                double u2[3];
                u2[k] = v; u2[j] = w;
                double bb = b[i] + v * G[k][i] + w * G[j][i];
                u2[i] = G[i][i] > 1e-30 ? clamp01(-bb / G[i][i]) : 0.0;
                best = fmin(best, dist2(u2));
            }
        }
    }
    return best;
}

struct BinArgs {
    CellDev c;
    GridDev g;
    const ExtAtom* ext;
    int64_t n_ext;
    const double* rc_sp;
};

// One warp per atom image: for every brick whose box of grid indices meets
// the image's cutoff sphere's fractional bounding box, test the exact
// brick-hull distance.  Pass 0 counts, pass 1 fills.
__global__ void k_bin(BinArgs a, int pass, int64_t* count, const int64_t* start, int64_t* fill, int32_t* atoms) {
    int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (e >= a.n_ext) return;
    const ExtAtom X = a.ext[e];
    double rc = a.rc_sp[X.species];
    double f[3];
    frac_of(a.c, X.p, f);
    int blo[3], bhi[3];
    for (int i = 0; i < 3; ++i) {
        double w = rc / a.c.h[i];
        long long glo = (long long)ceil((f[i] - w) * a.g.n[i] - 1e-9);
        long long ghi = (long long)floor((f[i] + w) * a.g.n[i] + 1e-9);
        if (glo < 0) glo = 0;
        if (ghi > a.g.n[i] - 1) ghi = a.g.n[i] - 1;
        if (glo > ghi) return;
        blo[i] = (int)(glo / a.g.B[i]);
        bhi[i] = (int)(ghi / a.g.B[i]);
    }
    int nb0 = bhi[0] - blo[0] + 1, nb1 = bhi[1] - blo[1] + 1, nb2 = bhi[2] - blo[2] + 1;
    int64_t total = (int64_t)nb0 * nb1 * nb2;
    const double rc2 = (rc + 1e-7) * (rc + 1e-7);
    for (int64_t q = lane; q < total; q += 32) {
        int c2 = (int)(q % nb2), c1 = (int)((q / nb2) % nb1), c0 = (int)(q / ((int64_t)nb2 * nb1));
        int b0 = blo[0] + c0, b1 = blo[1] + c1, b2 = blo[2] + c2;
        int lo[3] = {b0 * a.g.B[0], b1 * a.g.B[1], b2 * a.g.B[2]};
        int hi[3] = {min(lo[0] + a.g.B[0], a.g.n[0]) - 1, min(lo[1] + a.g.B[1], a.g.n[1]) - 1,
                     min(lo[2] + a.g.B[2], a.g.n[2]) - 1};
        double o[3], ed[3][3];
        for (int j = 0; j < 3; ++j) {
            o[j] = lo[0] * a.g.step[0][j] + lo[1] * a.g.step[1][j] + lo[2] * a.g.step[2][j];
            for (int i = 0; i < 3; ++i) ed[i][j] = (hi[i] - lo[i]) * a.g.step[i][j];
        }
        if (hull_dist2(X.p, o, ed) < rc2) {
            int64_t brick = ((int64_t)b0 * a.g.nb[1] + b1) * a.g.nb[2] + b2;
            if (pass == 0) {
                atomicAdd((unsigned long long*)&count[brick], 1ull);
            } else {
                unsigned long long slot = atomicAdd((unsigned long long*)&fill[brick], 1ull);
                if ((int64_t)slot < start[brick + 1] - start[brick]) atoms[start[brick] + (int64_t)slot] = (int32_t)e;
            }
        }
    }
}

// One warp per brick: sort its atom list ascending (rank sort, lists are short).
__global__ void k_sort_bricks(int64_t n_bricks, const int64_t* start, int32_t* atoms, int* err) {
    int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (b >= n_bricks) return;
    int64_t s = start[b];
    int n = (int)(start[b + 1] - s);
    if (n <= 1) return;
    if (n > kMaxBrickAtoms) {
        if (lane == 0) atomicOr(err, kErrBrickTooLarge);
        return;
    }
    int32_t vals[(kMaxBrickAtoms + 31) / 32];
    int ranks[(kMaxBrickAtoms + 31) / 32];
    int cnt = 0;
    for (int i = lane; i < n; i += 32, ++cnt) {
        int32_t v = atoms[s + i];
        int r = 0;
        for (int j = 0; j < n; ++j) {
            int32_t w = atoms[s + j];
            r += (w < v) || (w == v && j < i);
        }
        vals[cnt] = v;
        ranks[cnt] = r;
    }
    __syncwarp();
    for (int k = 0; k < cnt; ++k) atoms[s + ranks[k]] = vals[k];
}

// Per-brick statistics: orbital count, pattern pairs; work-list flags.
// Pair tables of the bricks (once per geometry): for images a, b of a brick
// (brick-local order), the block (I_a, I_b, t_b - t_a) when |R_b - R_a| <
// rc_a + rc_b (FP64, as the pattern), else -1.  One warp per brick.
__global__ void k_pair_count(int64_t n_bricks, const int64_t* brick_start, int64_t* cnt) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_bricks) return;
    const int64_t na = brick_start[b + 1] - brick_start[b];
    cnt[b] = na * na;
}

__global__ void k_brick_pairs(Problem P, int64_t n_bricks, const double* rc_sp, int32_t* pairs) {
    const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (b >= n_bricks) return;
    const int64_t s0 = P.brick_start[b];
    const int na = (int)(P.brick_start[b + 1] - s0);
    const int64_t ps = P.pair_start[b];
    for (int q = lane; q < na * na; q += 32) {
        const int a1 = q / na, a2 = q - a1 * na;
        const ExtAtom& X = P.ext[P.brick_atoms[s0 + a1]];
        const ExtAtom& Y = P.ext[P.brick_atoms[s0 + a2]];
        const double dx = Y.p[0] - X.p[0], dy = Y.p[1] - X.p[1], dz = Y.p[2] - X.p[2];
        const double cut = rc_sp[X.species] + rc_sp[Y.species];
        int64_t blk = -1;
        if (dx * dx + dy * dy + dz * dz < cut * cut) {
            blk = find_block(P, X.atom, Y.atom, Y.t[0] - X.t[0], Y.t[1] - X.t[1], Y.t[2] - X.t[2]);
            if (blk < 0) atomicOr(P.err, kErrPatternMissing);
        }
        pairs[ps + q] = (int32_t)blk;
    }
}

// Tile masks (once per geometry): for work item w and 128-point tile mt of its
// brick, bit a is set when brick image a lies within rc of a point of the tile
// (points p < bpts, the test the tensor-core rho and force kernels need; same
// helpers and roundings as those kernels).  One warp per (item, tile); a brick
// with more images than bits gets an empty mask (the tensor-core forms reject
// such handles).
__global__ void k_tile_mask(Problem P, int n_mt, unsigned long long* mask) {
    const int64_t id = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (id >= (int64_t)P.n_work * n_mt) return;
    const int w = (int)(id / n_mt), mt = (int)(id - (int64_t)w * n_mt);
    const GridDev& g = P.g;
    const int brick = P.work[w];
    int b0, b1, b2;
    brick_coords(g, brick, b0, b1, b2);
    const int64_t s0 = P.brick_start[brick];
    const int na = (int)(P.brick_start[brick + 1] - s0);
    unsigned long long m = 0ull;
    if (na <= 64) {
        float fx[4], fy[4], fz[4];
        bool pv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int p = mt * 128 + 32 * k + lane;
            pv[k] = p < g.bpts;
            fx[k] = fy[k] = fz[k] = 0.f;
            if (pv[k]) point_offset(g, p, fx[k], fy[k], fz[k]);
        }
        for (int a = 0; a < na; ++a) {
            const ExtAtom X = P.ext[P.brick_atoms[s0 + a]];
            float c_hi[3], c_lo[3];
            brick_atom_offset(g, b0, b1, b2, X, c_hi, c_lo);
            const float rc = P.sp[X.species].rc_f;
            bool in = false;
#pragma unroll
            for (int k = 0; k < 4; ++k) in = in || (pv[k] && point_within(c_hi, c_lo, fx[k], fy[k], fz[k], rc));
            if (__any_sync(0xffffffffu, in)) m |= 1ull << a;
        }
    }
    if (lane == 0) mask[id] = m;
}

__global__ void k_brick_stats(Problem P, int64_t n_bricks, const double* rc_sp, int64_t* nonempty_flag,
                              int64_t* pairs, int* max_atoms, int* max_orb) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_bricks) return;
    int64_t s = P.brick_start[b];
    int n = (int)(P.brick_start[b + 1] - s);
    nonempty_flag[b] = n > 0 ? 1 : 0;
    int norb = 0;
    int64_t np = 0;
    for (int i = 0; i < n; ++i) {
        const ExtAtom& A = P.ext[P.brick_atoms[s + i]];
        norb += P.sp[A.species].n_orb;
        for (int j = i; j < n; ++j) {
            const ExtAtom& B = P.ext[P.brick_atoms[s + j]];
            double d0 = B.p[0] - A.p[0], d1 = B.p[1] - A.p[1], d2 = B.p[2] - A.p[2];
            double cut = rc_sp[A.species] + rc_sp[B.species];
            np += (d0 * d0 + d1 * d1 + d2 * d2 < cut * cut);
        }
    }
    pairs[b] = np;
    atomicMax(max_atoms, n);
    atomicMax(max_orb, norb);
}

__global__ void k_compact(int64_t n, const int64_t* flag, const int64_t* pos, int32_t* out_set, int32_t* out_unset,
                          const int64_t* n_set) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (flag[i]) out_set[pos[i]] = (int32_t)i;
    else out_unset[i - pos[i]] = (int32_t)i;
}

__global__ void k_sum_i64(const int64_t* in, int64_t n, unsigned long long* out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t v = i < n ? in[i] : 0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(out, (unsigned long long)v);
}

// Exact per-point orbital counts: one warp per non-empty brick, lane = point.
__global__ void k_work_stats(Problem P, unsigned long long* out) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= P.n_work) return;
    const int brick = P.work[w];
    const GridDev& g = P.g;
    int b0, b1, b2;
    brick_coords(g, brick, b0, b1, b2);
    const int64_t s0 = P.brick_start[brick];
    const int na = (int)(P.brick_start[brick + 1] - s0);
    unsigned long long s1 = 0, s2 = 0;
    for (int p = lane; p < g.bpts; p += 32) {
        int g0, g1, g2;
        if (!brick_point(g, b0, b1, b2, p, g0, g1, g2)) continue;
        const double rx = g0 * g.step[0][0] + g1 * g.step[1][0] + g2 * g.step[2][0];
        const double ry = g0 * g.step[0][1] + g1 * g.step[1][1] + g2 * g.step[2][1];
        const double rz = g0 * g.step[0][2] + g1 * g.step[1][2] + g2 * g.step[2][2];
        unsigned long long no = 0;
        for (int i = 0; i < na; ++i) {
            const ExtAtom& X = P.ext[P.brick_atoms[s0 + i]];
            const double dx = rx - X.p[0], dy = ry - X.p[1], dz = rz - X.p[2];
            const double rc = P.sp[X.species].rc;
            if (dx * dx + dy * dy + dz * dz < rc * rc) no += P.sp[X.species].n_orb;
        }
        s1 += no;
        s2 += no * no;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
    }
    if (lane == 0) {
        atomicAdd(out, s1);
        atomicAdd(out + 1, s2);
    }
}

// ----------------------------------------------------- allocation hook
// gint_debug_fail_alloc(n): the n-th device allocation from then on fails the way cudaMalloc
// fails on a full device (cudaErrorMemoryAllocation), without touching the device.
static std::atomic<int> g_fail_alloc{0};

cudaError_t dev_malloc_raw(void** p, size_t bytes) {
    *p = nullptr;
    int n = g_fail_alloc.load();
    while (n > 0 && !g_fail_alloc.compare_exchange_weak(n, n - 1)) {
    }
    if (n == 1) return cudaErrorMemoryAllocation;
    return cudaMalloc(p, bytes);
}

// ----------------------------------------------------------- host helpers
static void inv3(const double a[9], double out[9]) {
    double d = a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) + a[2] * (a[3] * a[7] - a[4] * a[6]);
    out[0] = (a[4] * a[8] - a[5] * a[7]) / d;
    out[1] = (a[2] * a[7] - a[1] * a[8]) / d;
    out[2] = (a[1] * a[5] - a[2] * a[4]) / d;
    out[3] = (a[5] * a[6] - a[3] * a[8]) / d;
    out[4] = (a[0] * a[8] - a[2] * a[6]) / d;
    out[5] = (a[2] * a[3] - a[0] * a[5]) / d;
    out[6] = (a[3] * a[7] - a[4] * a[6]) / d;
    out[7] = (a[1] * a[6] - a[0] * a[7]) / d;
    out[8] = (a[0] * a[4] - a[1] * a[3]) / d;
}

template <typename T>
static gint_status dev_upload(T** dst, const T* src, size_t n) {
    *dst = nullptr;
    if (n == 0) n = 1;
    GINT_CUDA_TRY(dev_malloc((void**)dst, sizeof(T) * n));
    if (src) {
        const cudaError_t e = cudaMemcpy(*dst, src, sizeof(T) * n, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(*dst);
            *dst = nullptr;
            GINT_CUDA_TRY(e);
        }
    }
    return GINT_OK;
}

#define GINT_TRY(expr)                       \
    do {                                     \
        gint_status s_ = (expr);             \
        if (s_ != GINT_OK) return s_;        \
    } while (0)

gint_status allocate_scratch(gint_handle* h);  // simt.cu
gint_status static_scratch_resolve(void** out);  // noalloc.cu

static gint_status build_handle(gint_handle* h, int n_atoms, const double* pos, const int* species, const double* cell,
                                int n_species, const gint_species* sp, const int* grid, const gint_options* opt) {
    // ---- species tables
    std::vector<SpeciesDev> spd(n_species);
    std::vector<double> coef;
    std::vector<float2> knots;  // FP32 knot table: per species, per knot, per radial function
    std::vector<double> rc_sp(n_species);
    std::vector<int> nw_sp(n_species);
    int max_nw = 0;
    for (int s = 0; s < n_species; ++s) {
        const gint_species& S = sp[s];
        SpeciesDev& D = spd[s];
        memset(&D, 0, sizeof(D));
        D.n_radial = S.n_radial;
        D.rc = S.rc;
        D.rc_f = (float)S.rc;
        const gint_radial& r0 = S.radial[0];
        D.dr = r0.dr;
        D.inv_dr = 1.0 / r0.dr;
        D.inv_dr_f = (float)(1.0 / r0.dr);
        D.n_int = r0.n_knots - 1;
        D.tab_off = (int64_t)coef.size();
        D.knot_off = (int64_t)knots.size();
        for (int k = 0; k < r0.n_knots; ++k)
            for (int j = 0; j < S.n_radial; ++j) {
                const gint_radial& R = S.radial[j];
                knots.push_back(make_float2((float)R.y[k], (float)(R.dr * R.dy[k])));
            }
        int lmax = 0, norb = 0;
        for (int j = 0; j < S.n_radial; ++j) {
            D.rad_l[j] = S.radial[j].l;
            lmax = std::max(lmax, S.radial[j].l);
        }
        D.lmax = lmax;
        for (int l = 0; l <= kMaxL; ++l)
            for (int j = 0; j < S.n_radial; ++j)
                if (S.radial[j].l == l)
                    for (int m = 0; m <= 2 * l; ++m) {
                        D.orb_rad[norb] = (signed char)j;
                        D.orb_l[norb] = (signed char)l;
                        D.orb_m[norb] = (signed char)m;
                        ++norb;
                    }
        D.n_orb = norb;
        // fixed-point quantum of each orbital: |R| on a knot interval is at most
        // max |y| + (4/27) dr (|y'_k| + |y'_k+1|) (cubic Hermite basis bounds), and
        // |Y_lm| <= sqrt((2l + 1) / 4 pi) (addition theorem); 0.1 % margin for FP32
        for (int o = 0; o < norb; ++o) {
            const gint_radial& R = S.radial[D.orb_rad[o]];
            double bR = 0.0;
            for (int k = 0; k + 1 < R.n_knots; ++k) {
                const double dk = R.dy ? std::fabs(R.dy[k]) + std::fabs(R.dy[k + 1]) : 0.0;
                bR = std::max(bR, std::max(std::fabs(R.y[k]), std::fabs(R.y[k + 1])) + (4.0 / 27.0) * R.dr * dk);
            }
            const double bound = 1.001 * bR * std::sqrt((2.0 * D.orb_l[o] + 1.0) / (4.0 * M_PI));
            int e = 0;
            if (bound > 0.0) std::frexp(bound / 127.0, &e);  // bound / 127 < 2^e
            D.orb_qe[o] = (signed char)std::max(-100, std::min(100, e));
            e = 0;
            if (bound > 0.0) std::frexp(bound / ylm_norm(D.orb_l[o], D.orb_m[o]) / 127.0, &e);
            D.orb_qeu[o] = (signed char)std::max(-100, std::min(100, e));
        }
        nw_sp[s] = norb;
        rc_sp[s] = S.rc;
        max_nw = std::max(max_nw, norb);
        // interval cubics: c0 = y_k, c1 = dr y'_k, c2 = 3 (y_k+1 - y_k) - dr (2 y'_k + y'_k+1),
        // c3 = 2 (y_k - y_k+1) + dr (y'_k + y'_k+1)
        coef.resize(coef.size() + (size_t)D.n_int * S.n_radial * 4);
        double* c = coef.data() + D.tab_off;
        for (int k = 0; k < D.n_int; ++k)
            for (int j = 0; j < S.n_radial; ++j) {
                const gint_radial& R = S.radial[j];
                double y0 = R.y[k], y1 = R.y[k + 1], d0 = R.dr * R.dy[k], d1 = R.dr * R.dy[k + 1];
                double* o = c + ((size_t)k * S.n_radial + j) * 4;
                o[0] = y0;
                o[1] = d0;
                o[2] = 3.0 * (y1 - y0) - 2.0 * d0 - d1;
                o[3] = 2.0 * (y0 - y1) + d0 + d1;
            }
    }
    h->max_nw = max_nw;
    std::vector<float> coef32(coef.begin(), coef.end());
    GINT_TRY(dev_upload(&h->d_sp, spd.data(), spd.size()));
    GINT_TRY(dev_upload(&h->d_coef64, coef.data(), coef.size()));
    GINT_TRY(dev_upload(&h->d_coef32, coef32.data(), coef32.size()));
    GINT_TRY(dev_upload(&h->d_knot32, knots.data(), knots.size()));

    // ---- cell and grid
    CellDev c;
    double Ainv[9];
    inv3(cell, Ainv);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) { c.A[i][j] = cell[3 * i + j]; c.Ainv[i][j] = Ainv[3 * i + j]; }
    for (int i = 0; i < 3; ++i) {
        double b2 = Ainv[i] * Ainv[i] + Ainv[3 + i] * Ainv[3 + i] + Ainv[6 + i] * Ainv[6 + i];
        c.h[i] = 1.0 / sqrt(b2);
    }
    double det = cell[0] * (cell[4] * cell[8] - cell[5] * cell[7]) - cell[1] * (cell[3] * cell[8] - cell[5] * cell[6]) +
                 cell[2] * (cell[3] * cell[7] - cell[4] * cell[6]);
    h->omega = fabs(det);
    memcpy(h->cell, cell, sizeof(double) * 9);
    GridDev& g = h->grid;
    int Bdef[3] = {8, 8, 8};
    for (int i = 0; i < 3; ++i) {
        g.n[i] = grid[i];
        g.B[i] = (opt && opt->brick[i] > 0) ? opt->brick[i] : Bdef[i];
        if (g.B[i] > g.n[i]) g.B[i] = g.n[i];
        g.nb[i] = (g.n[i] + g.B[i] - 1) / g.B[i];
        for (int j = 0; j < 3; ++j) {
            g.step[i][j] = cell[3 * i + j] / grid[i];
            g.step_hi[i][j] = (float)g.step[i][j];
            g.step_lo[i][j] = (float)(g.step[i][j] - (double)g.step_hi[i][j]);
        }
    }
    g.bpts = g.B[0] * g.B[1] * g.B[2];
    if (g.bpts > kMaxBrickPts) {
        set_error("brick of %d points exceeds %d", g.bpts, kMaxBrickPts);
        return GINT_ERR_INVALID_ARG;
    }
    g.bpad = (g.bpts + 31) / 32 * 32;
    g.nsub = g.bpad / 32;
    g.dV = h->omega / ((double)grid[0] * grid[1] * grid[2]);
    h->n_bricks = (int64_t)g.nb[0] * g.nb[1] * g.nb[2];
    if (h->n_bricks > INT32_MAX) {
        set_error("too many bricks (%lld)", (long long)h->n_bricks);
        return GINT_ERR_UNSUPPORTED;
    }

    // ---- atoms
    std::vector<int> spc(species, species + n_atoms);
    double* d_pos = nullptr;
    int* d_spc = nullptr;
    double* d_rc = nullptr;
    int* d_nw = nullptr;
    // temporaries of the set-up, released on every return (each is listed as soon as it exists)
    struct Tmp {
        std::vector<void*> p;
        ~Tmp() { for (void* x : p) cudaFree(x); }
    } tmp;
    GINT_TRY(dev_upload(&d_pos, pos, (size_t)3 * n_atoms));
    tmp.p.push_back(d_pos);
    GINT_TRY(dev_upload(&d_spc, spc.data(), spc.size()));
    tmp.p.push_back(d_spc);
    GINT_TRY(dev_upload(&d_rc, rc_sp.data(), rc_sp.size()));
    tmp.p.push_back(d_rc);
    GINT_TRY(dev_upload(&d_nw, nw_sp.data(), nw_sp.size()));
    tmp.p.push_back(d_nw);
    cudaStream_t st = 0;

    // ---- pattern (Section 2.2 sparsity): rows I, sorted (J, t)
    int64_t *d_rc_cnt = nullptr, *d_rv = nullptr;
    GINT_CUDA_TRY(dev_malloc(&d_rc_cnt, sizeof(int64_t) * (n_atoms + 1)));
    tmp.p.push_back(d_rc_cnt);
    GINT_CUDA_TRY(dev_malloc(&d_rv, sizeof(int64_t) * (n_atoms + 1)));
    tmp.p.push_back(d_rv);
    k_pattern_count<<<n_atoms, 256, 0, st>>>(c, n_atoms, d_pos, d_spc, d_rc, d_nw, d_rc_cnt, d_rv);
    GINT_CUDA_TRY(cudaGetLastError());
    GINT_CUDA_TRY(dev_malloc(&h->d_row_start, sizeof(int64_t) * (n_atoms + 1)));
    GINT_TRY(scan_exclusive(d_rc_cnt, n_atoms, h->d_row_start, st));
    GINT_TRY(scan_exclusive(d_rv, n_atoms, d_rv, st));
    GINT_CUDA_TRY(cudaMemcpy(&h->n_blocks, h->d_row_start + n_atoms, sizeof(int64_t), cudaMemcpyDeviceToHost));
    GINT_CUDA_TRY(cudaMemcpy(&h->n_values, d_rv + n_atoms, sizeof(int64_t), cudaMemcpyDeviceToHost));
    if (h->n_blocks > INT32_MAX) {
        set_error("pattern has too many blocks (%lld)", (long long)h->n_blocks);
        return GINT_ERR_UNSUPPORTED;
    }
    GINT_CUDA_TRY(dev_malloc(&h->d_blocks, sizeof(int32_t) * 5 * std::max<int64_t>(1, h->n_blocks)));
    GINT_CUDA_TRY(dev_malloc(&h->d_offsets, sizeof(int64_t) * (h->n_blocks + 1)));
    k_pattern_fill<<<n_atoms, 256, 0, st>>>(c, n_atoms, d_pos, d_spc, d_rc, d_nw, h->d_row_start, d_rv, h->d_blocks,
                                            h->d_offsets);
    GINT_CUDA_TRY(cudaGetLastError());
    GINT_CUDA_TRY(cudaMemcpy(h->d_offsets + h->n_blocks, &h->n_values, sizeof(int64_t), cudaMemcpyHostToDevice));
    GINT_CUDA_TRY(dev_malloc(&h->d_err, sizeof(int) * 4));
    GINT_CUDA_TRY(cudaMemset(h->d_err, 0, sizeof(int) * 4));
    GINT_CUDA_TRY(dev_malloc(&h->d_red, sizeof(double) * 64));
    GINT_CUDA_TRY(dev_malloc(&h->d_facc, sizeof(double) * 12 * n_atoms));
    {
        std::vector<int> nwa(n_atoms);
        for (int i = 0; i < n_atoms; ++i) nwa[i] = nw_sp[spc[i]];
        GINT_TRY(dev_upload(&h->d_nw_atom, nwa.data(), nwa.size()));
        GINT_TRY(dev_upload(&h->d_atom_sp, spc.data(), spc.size()));
        std::vector<int64_t> oo(n_atoms + 1, 0);
        for (int i = 0; i < n_atoms; ++i) oo[i + 1] = oo[i] + nwa[i];
        h->n_orbitals = oo[n_atoms];
        GINT_TRY(dev_upload(&h->d_orb_off, oo.data(), oo.size()));
    }
    GINT_CUDA_TRY(dev_malloc(&h->d_mirror, sizeof(int32_t) * std::max<int64_t>(1, h->n_blocks)));
    {
        Problem P = h->problem();
        int64_t nb = h->n_blocks;
        if (nb > 0) k_mirror<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(P, nb, h->d_mirror);
        GINT_CUDA_TRY(cudaGetLastError());
    }

    // ---- atom images whose sphere meets the grid (host; sorted by (I, t))
    std::vector<ExtAtom> ext;
    for (int I = 0; I < n_atoms; ++I) {
        double rc = rc_sp[spc[I]];
        double f[3];
        for (int i = 0; i < 3; ++i)
            f[i] = pos[3 * I] * Ainv[i] + pos[3 * I + 1] * Ainv[3 + i] + pos[3 * I + 2] * Ainv[6 + i];
        int lo[3], hi[3];
        for (int i = 0; i < 3; ++i) {
            double w = rc / c.h[i];
            // the image's fractional coordinate f+t must lie in [-w, (n-1)/n + w]
            lo[i] = (int)ceil(-w - f[i] - 1e-9);
            hi[i] = (int)floor((double)(grid[i] - 1) / grid[i] + w - f[i] + 1e-9);
        }
        for (int t0 = lo[0]; t0 <= hi[0]; ++t0)
            for (int t1 = lo[1]; t1 <= hi[1]; ++t1)
                for (int t2 = lo[2]; t2 <= hi[2]; ++t2) {
                    ExtAtom X;
                    memset(&X, 0, sizeof(X));
                    for (int j = 0; j < 3; ++j) X.p[j] = pos[3 * I + j] + t0 * cell[j] + t1 * cell[3 + j] + t2 * cell[6 + j];
                    X.atom = I;
                    X.species = spc[I];
                    X.t[0] = t0; X.t[1] = t1; X.t[2] = t2;
                    ext.push_back(X);
                }
    }
    h->n_ext = (int64_t)ext.size();
    if (h->n_ext > INT32_MAX) {
        set_error("too many atom images");
        return GINT_ERR_UNSUPPORTED;
    }
    GINT_TRY(dev_upload(&h->d_ext, ext.data(), ext.size()));

    // ---- binner
    int64_t nbk = h->n_bricks;
    int64_t *d_count = nullptr, *d_fill = nullptr;
    GINT_CUDA_TRY(dev_malloc(&d_count, sizeof(int64_t) * (nbk + 1)));
    tmp.p.push_back(d_count);
    GINT_CUDA_TRY(dev_malloc(&d_fill, sizeof(int64_t) * (nbk + 1)));
    tmp.p.push_back(d_fill);
    GINT_CUDA_TRY(cudaMemset(d_count, 0, sizeof(int64_t) * (nbk + 1)));
    GINT_CUDA_TRY(cudaMemset(d_fill, 0, sizeof(int64_t) * (nbk + 1)));
    BinArgs ba;
    ba.c = c;
    ba.g = g;
    ba.ext = h->d_ext;
    ba.n_ext = h->n_ext;
    ba.rc_sp = d_rc;
    unsigned nblk = (unsigned)((h->n_ext * 32 + 255) / 256);
    if (h->n_ext > 0) k_bin<<<nblk, 256, 0, st>>>(ba, 0, d_count, nullptr, nullptr, nullptr);
    GINT_CUDA_TRY(cudaGetLastError());
    GINT_CUDA_TRY(dev_malloc(&h->d_brick_start, sizeof(int64_t) * (nbk + 1)));
    GINT_TRY(scan_exclusive(d_count, nbk, h->d_brick_start, st));
    GINT_CUDA_TRY(cudaMemcpy(&h->n_brick_atoms, h->d_brick_start + nbk, sizeof(int64_t), cudaMemcpyDeviceToHost));
    GINT_CUDA_TRY(dev_malloc(&h->d_brick_atoms, sizeof(int32_t) * std::max<int64_t>(1, h->n_brick_atoms)));
    if (h->n_ext > 0) k_bin<<<nblk, 256, 0, st>>>(ba, 1, nullptr, h->d_brick_start, d_fill, h->d_brick_atoms);
    GINT_CUDA_TRY(cudaGetLastError());
    k_sort_bricks<<<(unsigned)((nbk * 32 + 255) / 256), 256, 0, st>>>(nbk, h->d_brick_start, h->d_brick_atoms, h->d_err);
    GINT_CUDA_TRY(cudaGetLastError());

    // ---- statistics and work lists
    int64_t *d_flag = nullptr, *d_pairs = nullptr, *d_pos_ne = nullptr;
    int* d_max = nullptr;
    unsigned long long* d_sum = nullptr;
    GINT_CUDA_TRY(dev_malloc(&d_flag, sizeof(int64_t) * (nbk + 1)));
    tmp.p.push_back(d_flag);
    GINT_CUDA_TRY(dev_malloc(&d_pairs, sizeof(int64_t) * (nbk + 1)));
    tmp.p.push_back(d_pairs);
    GINT_CUDA_TRY(dev_malloc(&d_pos_ne, sizeof(int64_t) * (nbk + 1)));
    tmp.p.push_back(d_pos_ne);
    GINT_CUDA_TRY(dev_malloc(&d_max, sizeof(int) * 2));
    tmp.p.push_back(d_max);
    GINT_CUDA_TRY(dev_malloc(&d_sum, sizeof(unsigned long long)));
    tmp.p.push_back(d_sum);
    GINT_CUDA_TRY(cudaMemset(d_max, 0, sizeof(int) * 2));
    GINT_CUDA_TRY(cudaMemset(d_sum, 0, sizeof(unsigned long long)));
    {
        Problem P = h->problem();
        k_brick_stats<<<(unsigned)((nbk + 127) / 128), 128, 0, st>>>(P, nbk, d_rc, d_flag, d_pairs, d_max, d_max + 1);
        GINT_CUDA_TRY(cudaGetLastError());
        k_sum_i64<<<(unsigned)((nbk + 255) / 256), 256, 0, st>>>(d_pairs, nbk, d_sum);
        GINT_CUDA_TRY(cudaGetLastError());
    }
    // ---- per-brick pair tables
    {
        int64_t* d_pcnt = nullptr;
        GINT_CUDA_TRY(dev_malloc(&d_pcnt, sizeof(int64_t) * (nbk + 1)));
        tmp.p.push_back(d_pcnt);
        k_pair_count<<<(unsigned)((nbk + 255) / 256), 256, 0, st>>>(nbk, h->d_brick_start, d_pcnt);
        GINT_CUDA_TRY(cudaGetLastError());
        GINT_CUDA_TRY(dev_malloc(&h->d_pair_start, sizeof(int64_t) * (nbk + 1)));
        GINT_TRY(scan_exclusive(d_pcnt, nbk, h->d_pair_start, st));
        int64_t n_pair_entries = 0;
        GINT_CUDA_TRY(cudaMemcpy(&n_pair_entries, h->d_pair_start + nbk, sizeof(int64_t), cudaMemcpyDeviceToHost));
        GINT_CUDA_TRY(dev_malloc(&h->d_pairs, sizeof(int32_t) * std::max<int64_t>(1, n_pair_entries)));
        Problem P = h->problem();
        k_brick_pairs<<<(unsigned)((nbk * 32 + 255) / 256), 256, 0, st>>>(P, nbk, d_rc, h->d_pairs);
        GINT_CUDA_TRY(cudaGetLastError());
    }
    GINT_TRY(scan_exclusive(d_flag, nbk, d_pos_ne, st));
    GINT_CUDA_TRY(cudaMemcpy(&h->n_work, d_pos_ne + nbk, sizeof(int64_t), cudaMemcpyDeviceToHost));
    h->n_empty = nbk - h->n_work;
    GINT_CUDA_TRY(dev_malloc(&h->d_work, sizeof(int32_t) * std::max<int64_t>(1, h->n_work)));
    GINT_CUDA_TRY(dev_malloc(&h->d_empty, sizeof(int32_t) * std::max<int64_t>(1, h->n_empty)));
    k_compact<<<(unsigned)((nbk + 255) / 256), 256, 0, st>>>(nbk, d_flag, d_pos_ne, h->d_work, h->d_empty, nullptr);
    GINT_CUDA_TRY(cudaGetLastError());
    {
        const int n_mt = (h->grid.bpad + 127) / 128;
        const int64_t n_masks = h->n_work * n_mt;
        GINT_CUDA_TRY(dev_malloc(&h->d_tile_mask, sizeof(unsigned long long) * std::max<int64_t>(1, n_masks)));
        if (n_masks > 0) {
            Problem P = h->problem();
            k_tile_mask<<<(unsigned)((n_masks * 32 + 255) / 256), 256, 0, st>>>(P, n_mt, h->d_tile_mask);
            GINT_CUDA_TRY(cudaGetLastError());
        }
    }
    int mx[2];
    unsigned long long npairs = 0;
    GINT_CUDA_TRY(cudaMemcpy(mx, d_max, sizeof(int) * 2, cudaMemcpyDeviceToHost));
    GINT_CUDA_TRY(cudaMemcpy(&npairs, d_sum, sizeof(npairs), cudaMemcpyDeviceToHost));
    h->max_brick_atoms = mx[0];
    h->max_brick_orb = mx[1];
    h->n_brick_pairs = (int64_t)npairs;
    int herr = 0;
    GINT_CUDA_TRY(cudaDeviceSynchronize());
    GINT_CUDA_TRY(cudaMemcpy(&herr, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr & kErrPatternMissing) {
        set_error("pattern is not closed under (I, J, T) -> (J, I, -T)");
        return GINT_ERR_DEVICE;
    }
    if (h->max_brick_atoms > kMaxBrickAtoms || (herr & kErrBrickTooLarge)) {
        set_error("a brick meets %d atom images (limit %d); use smaller bricks", h->max_brick_atoms, kMaxBrickAtoms);
        return GINT_ERR_UNSUPPORTED;
    }
    GINT_TRY(allocate_scratch(h));
    // the static scratch of gint_vlocal_static: map it now, while allocating is allowed (a failure
    // here only disables that call, which then reports it)
    if (static_scratch_resolve(&h->d_static) != GINT_OK) {
        (void)cudaGetLastError();
        set_error("");
    }
    return GINT_OK;
}

void hxc_release(gint_handle* h);  // hxc.cu

static void free_handle(gint_handle* h) {
    if (!h) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(h->device);
    hxc_release(h);
    void* ptrs[] = {h->d_sp, h->d_coef64, h->d_coef32, h->d_knot32, h->d_ext, h->d_blocks, h->d_offsets, h->d_row_start,
                    h->d_mirror, h->d_brick_start, h->d_brick_atoms, h->d_work, h->d_pair_start, h->d_pairs, h->d_tile_mask, h->d_empty, h->d_err, h->d_red,
                    h->d_scratch, h->d_nw_atom, h->d_atom_sp, h->d_orb_off, h->d_facc, h->d_dt, h->d_dq, h->d_zero,
                    h->d_spec, h->d_epart};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (prev >= 0) cudaSetDevice(prev);
    delete h;
}

// Host copy of the species tables and the atoms' species (for gint_update_positions).
static void store_species(gint_handle* h, int n_atoms, const int* species, int n_species, const gint_species* sp,
                          const gint_options* opt) {
    h->atom_species.assign(species, species + n_atoms);
    h->sp_rc.clear(); h->sp_nrad.clear(); h->rad_l.clear(); h->rad_nk.clear();
    h->rad_dr.clear(); h->rad_y.clear(); h->rad_dy.clear();
    for (int s = 0; s < n_species; ++s) {
        h->sp_rc.push_back(sp[s].rc);
        h->sp_nrad.push_back(sp[s].n_radial);
        for (int j = 0; j < sp[s].n_radial; ++j) {
            const gint_radial& R = sp[s].radial[j];
            h->rad_l.push_back(R.l);
            h->rad_nk.push_back(R.n_knots);
            h->rad_dr.push_back(R.dr);
            h->rad_y.insert(h->rad_y.end(), R.y, R.y + R.n_knots);
            h->rad_dy.insert(h->rad_dy.end(), R.dy, R.dy + R.n_knots);
        }
    }
    for (int i = 0; i < 3; ++i) h->brick_opt[i] = opt ? opt->brick[i] : 0;
}

// gint_species views of the stored tables (pointers into h's vectors).
static void species_views(const gint_handle* h, std::vector<gint_species>& S, std::vector<gint_radial>& R) {
    R.resize(h->rad_l.size());
    S.resize(h->sp_rc.size());
    size_t j = 0, off = 0;
    for (size_t s = 0; s < S.size(); ++s) {
        S[s].rc = h->sp_rc[s];
        S[s].n_radial = h->sp_nrad[s];
        S[s].radial = R.data() + j;
        for (int k = 0; k < h->sp_nrad[s]; ++k, ++j) {
            R[j].l = h->rad_l[j];
            R[j].n_knots = h->rad_nk[j];
            R[j].dr = h->rad_dr[j];
            R[j].y = h->rad_y.data() + off;
            R[j].dy = h->rad_dy.data() + off;
            off += (size_t)h->rad_nk[j];
        }
    }
}

// Work lists (non-empty and empty bricks, natural order) of the selected bricks, and the
// tile masks of the new work list.  Synchronous.
static gint_status rebuild_work_lists(gint_handle* h) {
    const int64_t nbk = h->n_bricks;
    std::vector<int64_t> bs(nbk + 1);
    GINT_CUDA_TRY(cudaMemcpy(bs.data(), h->d_brick_start, sizeof(int64_t) * (nbk + 1), cudaMemcpyDeviceToHost));
    std::vector<char> sel(nbk, h->selecting ? 0 : 1);
    for (int64_t b : h->selection) sel[b] = 1;
    std::vector<int32_t> work, empty;
    for (int64_t b = 0; b < nbk; ++b)
        if (sel[b]) (bs[b + 1] > bs[b] ? work : empty).push_back((int32_t)b);
    int32_t *d_work = nullptr, *d_empty = nullptr;
    unsigned long long* d_mask = nullptr;
    const int n_mt = (h->grid.bpad + 127) / 128;
    const int64_t n_masks = (int64_t)work.size() * n_mt;
    cudaError_t e = dev_malloc(&d_work, sizeof(int32_t) * std::max<size_t>(1, work.size()));
    if (e == cudaSuccess) e = dev_malloc(&d_empty, sizeof(int32_t) * std::max<size_t>(1, empty.size()));
    if (e == cudaSuccess) e = dev_malloc(&d_mask, sizeof(unsigned long long) * std::max<int64_t>(1, n_masks));
    if (e == cudaSuccess && !work.empty())
        e = cudaMemcpy(d_work, work.data(), sizeof(int32_t) * work.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !empty.empty())
        e = cudaMemcpy(d_empty, empty.data(), sizeof(int32_t) * empty.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d_work); cudaFree(d_empty); cudaFree(d_mask);
        set_error("selecting bricks: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? GINT_ERR_OOM : GINT_ERR_CUDA;
    }
    cudaFree(h->d_work); cudaFree(h->d_empty); cudaFree(h->d_tile_mask);
    h->d_work = d_work;
    h->d_empty = d_empty;
    h->d_tile_mask = d_mask;
    h->n_work = (int64_t)work.size();
    h->n_empty = (int64_t)empty.size();
    if (n_masks > 0) {
        Problem P = h->problem();
        k_tile_mask<<<(unsigned)((n_masks * 32 + 255) / 256), 256>>>(P, n_mt, h->d_tile_mask);
        GINT_CUDA_TRY(cudaGetLastError());
    }
    GINT_CUDA_TRY(cudaDeviceSynchronize());
    return GINT_OK;
}

}  // namespace gint

using namespace gint;

extern "C" {

const char* gint_last_error(void) { return g_err; }

gint_status gint_setup(int n_atoms, const double* pos, const int* species, const double* cell, int n_species,
                       const gint_species* sp, const int* grid, const gint_options* opt, gint_handle** out) {
    gint::NvtxRange nvtx_range_("gint_setup");
    set_error("");
    if (!out) { set_error("out is NULL"); return GINT_ERR_INVALID_ARG; }
    *out = nullptr;
    if (n_atoms < 1 || !pos || !species || !cell || n_species < 1 || !sp || !grid) {
        set_error("invalid argument: need n_atoms >= 1, n_species >= 1 and non-NULL arrays");
        return GINT_ERR_INVALID_ARG;
    }
    for (int i = 0; i < 3; ++i)
        if (grid[i] < 1 || grid[i] > (1 << 24)) { set_error("grid[%d] = %d out of range", i, grid[i]); return GINT_ERR_INVALID_ARG; }
    if ((double)grid[0] * grid[1] * grid[2] > 4.0e12) { set_error("grid too large"); return GINT_ERR_INVALID_ARG; }
    double det = cell[0] * (cell[4] * cell[8] - cell[5] * cell[7]) - cell[1] * (cell[3] * cell[8] - cell[5] * cell[6]) +
                 cell[2] * (cell[3] * cell[7] - cell[4] * cell[6]);
    if (!(fabs(det) > 1e-12) || !std::isfinite(det)) { set_error("cell is singular"); return GINT_ERR_INVALID_ARG; }
    for (int i = 0; i < 3 * n_atoms; ++i)
        if (!std::isfinite(pos[i])) { set_error("pos[%d] is not finite", i); return GINT_ERR_INVALID_ARG; }
    for (int i = 0; i < n_atoms; ++i)
        if (species[i] < 0 || species[i] >= n_species) { set_error("species[%d] out of range", i); return GINT_ERR_INVALID_ARG; }
    for (int s = 0; s < n_species; ++s) {
        const gint_species& S = sp[s];
        if (!(S.rc > 0) || S.n_radial < 1 || S.n_radial > kMaxRadial || !S.radial) {
            set_error("species %d: need rc > 0 and 1..%d radial functions", s, kMaxRadial);
            return GINT_ERR_INVALID_ARG;
        }
        int norb = 0;
        for (int j = 0; j < S.n_radial; ++j) {
            const gint_radial& R = S.radial[j];
            if (R.l < 0 || R.l > kMaxL) { set_error("species %d radial %d: l = %d unsupported", s, j, R.l); return GINT_ERR_UNSUPPORTED; }
            if (R.n_knots < 2 || !(R.dr > 0) || !R.y) { set_error("species %d radial %d: bad table", s, j); return GINT_ERR_INVALID_ARG; }
            if (!R.dy) { set_error("species %d radial %d: derivative table required", s, j); return GINT_ERR_INVALID_ARG; }
            if (R.dr != S.radial[0].dr || R.n_knots != S.radial[0].n_knots) {
                set_error("species %d: all radial functions must share dr and n_knots", s);
                return GINT_ERR_UNSUPPORTED;
            }
            for (int k = 0; k < R.n_knots; ++k)
                if (!std::isfinite(R.y[k]) || !std::isfinite(R.dy[k])) {
                    set_error("species %d radial %d: non-finite table entry", s, j);
                    return GINT_ERR_INVALID_ARG;
                }
            norb += 2 * R.l + 1;
        }
        if (norb > kMaxNw) { set_error("species %d has %d orbitals (limit %d)", s, norb, kMaxNw); return GINT_ERR_UNSUPPORTED; }
        if ((S.radial[0].n_knots - 1) * S.radial[0].dr < S.rc * (1.0 - 1e-12)) {
            set_error("species %d: table ends before rc", s);
            return GINT_ERR_INVALID_ARG;
        }
    }
    if (opt) {
        for (int i = 0; i < 5; ++i)
            if (opt->reserved[i] != 0) { set_error("gint_options.reserved must be zero"); return GINT_ERR_INVALID_ARG; }
        for (int i = 0; i < 3; ++i)
            if (opt->brick[i] < 0 || opt->brick[i] > kMaxBrickPts) { set_error("brick[%d] out of range", i); return GINT_ERR_INVALID_ARG; }
        if (opt->precision < GINT_FP64 || opt->precision > GINT_FP16X4) { set_error("unknown precision"); return GINT_ERR_INVALID_ARG; }
    }
    int dev = (opt && opt->device >= 0) ? opt->device : -1;
    if (dev < 0) {
        if (cudaGetDevice(&dev) != cudaSuccess) { set_error("no CUDA device"); return GINT_ERR_CUDA; }
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(dev) != cudaSuccess) { set_error("cannot select device %d", dev); return GINT_ERR_CUDA; }
    gint_handle* h = new gint_handle();
    h->device = dev;
    h->n_atoms = n_atoms;
    h->n_species = n_species;
    h->precision = opt ? opt->precision : GINT_FP64;
    cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, dev);
    store_species(h, n_atoms, species, n_species, sp, opt);
    gint_status st = build_handle(h, n_atoms, pos, species, cell, n_species, sp, grid, opt);
    if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    if (st != GINT_OK) {
        free_handle(h);
        return st;
    }
    *out = h;
    return GINT_OK;
}

void gint_destroy(gint_handle* h) { free_handle(h); }

gint_status gint_pattern(const gint_handle* h, int64_t* n_blocks, int64_t* n_values, const int32_t** blocks,
                         const int64_t** offsets) {
    if (!h) { set_error("handle is NULL"); return GINT_ERR_INVALID_ARG; }
    if (n_blocks) *n_blocks = h->n_blocks;
    if (n_values) *n_values = h->n_values;
    if (blocks) *blocks = h->d_blocks;
    if (offsets) *offsets = h->d_offsets;
    return GINT_OK;
}

gint_status gint_set_precision(gint_handle* h, int precision) {
    if (!h) { set_error("handle is NULL"); return GINT_ERR_INVALID_ARG; }
    if (precision < GINT_FP64 || precision > GINT_FP16X4) { set_error("unknown precision %d", precision); return GINT_ERR_INVALID_ARG; }
    h->precision = precision;
    return GINT_OK;
}

gint_status gint_get_info(const gint_handle* h, gint_info* info) {
    if (!h || !info) { set_error("NULL argument"); return GINT_ERR_INVALID_ARG; }
    memset(info, 0, sizeof(*info));
    info->n_blocks = h->n_blocks;
    info->n_values = h->n_values;
    info->n_ext_atoms = h->n_ext;
    info->n_bricks = h->n_bricks;
    info->n_bricks_nonempty = h->n_work;
    info->n_brick_atoms = h->n_brick_atoms;
    info->n_brick_pairs = h->n_brick_pairs;
    info->max_brick_atoms = h->max_brick_atoms;
    info->max_brick_orbitals = h->max_brick_orb;
    for (int i = 0; i < 3; ++i) info->brick[i] = h->grid.B[i];
    info->precision = h->precision;
    info->scratch_bytes = (int64_t)h->scratch_bytes;
    info->n_orbitals = h->n_orbitals;
    return GINT_OK;
}

gint_status gint_work_stats(gint_handle* h, int64_t* sum_orbitals, int64_t* sum_orbitals_sq) {
    if (!h || !sum_orbitals || !sum_orbitals_sq) { set_error("NULL argument"); return GINT_ERR_INVALID_ARG; }
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(h->device) != cudaSuccess) { set_error("cannot select device %d", h->device); return GINT_ERR_CUDA; }
    unsigned long long* d = nullptr;
    unsigned long long hv[2] = {0, 0};
    cudaError_t e = dev_malloc(&d, sizeof(hv));
    if (e == cudaSuccess) e = cudaMemset(d, 0, sizeof(hv));
    if (e == cudaSuccess && h->n_work > 0) {
        const int64_t threads = h->n_work * 32;
        k_work_stats<<<(unsigned)((threads + 255) / 256), 256>>>(h->problem(), d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(hv, d, sizeof(hv), cudaMemcpyDeviceToHost);
    if (d) cudaFree(d);
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) { set_error("gint_work_stats: %s", cudaGetErrorString(e)); return GINT_ERR_CUDA; }
    *sum_orbitals = (int64_t)hv[0];
    *sum_orbitals_sq = (int64_t)hv[1];
    return GINT_OK;
}

gint_status gint_sync(gint_handle* h, gint_stream stream) {
    if (!h) { set_error("handle is NULL"); return GINT_ERR_INVALID_ARG; }
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(h->device);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    int flags = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&flags, h->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && flags) e = cudaMemset(h->d_err, 0, sizeof(int));
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) { set_error("gint_sync: %s", cudaGetErrorString(e)); return GINT_ERR_CUDA; }
    if (flags & kErrPatternMissing) { set_error("a pair of atoms met on the grid is missing from the pattern"); return GINT_ERR_PATTERN_MISMATCH; }
    if (flags & kErrTimeout) { set_error("a bounded wait on the tensor-core pipeline gave up"); return GINT_ERR_TIMEOUT; }
    if (flags) { set_error("device check failed (flags 0x%x)", flags); return GINT_ERR_DEVICE; }
    return GINT_OK;
}

gint_status gint_update_positions(gint_handle* h, const double* pos, const double* cell, int keep_pattern,
                                  int* pattern_changed) {
    gint::NvtxRange nvtx_range_("gint_update_positions");
    set_error("");
    if (!h || !pos) { set_error("gint_update_positions: NULL argument"); return GINT_ERR_INVALID_ARG; }
    if (keep_pattern != 0 && keep_pattern != 1) { set_error("keep_pattern must be 0 or 1"); return GINT_ERR_INVALID_ARG; }
    const double* cl = cell ? cell : h->cell;
    const double det = cl[0] * (cl[4] * cl[8] - cl[5] * cl[7]) - cl[1] * (cl[3] * cl[8] - cl[5] * cl[6]) +
                       cl[2] * (cl[3] * cl[7] - cl[4] * cl[6]);
    if (!(fabs(det) > 1e-12) || !std::isfinite(det)) { set_error("cell is singular"); return GINT_ERR_INVALID_ARG; }
    for (int i = 0; i < 3 * h->n_atoms; ++i)
        if (!std::isfinite(pos[i])) { set_error("pos[%d] is not finite", i); return GINT_ERR_INVALID_ARG; }
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(h->device) != cudaSuccess) { set_error("cannot select device %d", h->device); return GINT_ERR_CUDA; }
    // finish the work already queued on the handle's buffers before they are released
    if (cudaDeviceSynchronize() != cudaSuccess) {
        if (prev >= 0) cudaSetDevice(prev);
        set_error("gint_update_positions: device synchronisation failed");
        return GINT_ERR_CUDA;
    }
    gint_handle* hn = new gint_handle();
    hn->device = h->device;
    hn->n_atoms = h->n_atoms;
    hn->n_species = h->n_species;
    hn->precision = h->precision;
    hn->sm_count = h->sm_count;
    hn->sp_rc = h->sp_rc; hn->sp_nrad = h->sp_nrad; hn->rad_l = h->rad_l; hn->rad_nk = h->rad_nk;
    hn->rad_dr = h->rad_dr; hn->rad_y = h->rad_y; hn->rad_dy = h->rad_dy; hn->atom_species = h->atom_species;
    for (int i = 0; i < 3; ++i) hn->brick_opt[i] = h->brick_opt[i];
    std::vector<gint_species> S;
    std::vector<gint_radial> R;
    species_views(hn, S, R);
    gint_options opt;
    memset(&opt, 0, sizeof(opt));
    opt.precision = h->precision;
    opt.device = h->device;
    for (int i = 0; i < 3; ++i) opt.brick[i] = h->brick_opt[i];
    const int grid[3] = {h->grid.n[0], h->grid.n[1], h->grid.n[2]};
    gint_status st = build_handle(hn, h->n_atoms, pos, hn->atom_species.data(), cl, h->n_species, S.data(), grid, &opt);
    bool changed = false;
    if (st == GINT_OK) {
        changed = hn->n_blocks != h->n_blocks || hn->n_values != h->n_values;
        if (!changed && h->n_blocks > 0) {
            std::vector<int32_t> a((size_t)5 * h->n_blocks), b((size_t)5 * h->n_blocks);
            cudaError_t e = cudaMemcpy(a.data(), h->d_blocks, sizeof(int32_t) * a.size(), cudaMemcpyDeviceToHost);
            if (e == cudaSuccess) e = cudaMemcpy(b.data(), hn->d_blocks, sizeof(int32_t) * b.size(), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) { set_error("gint_update_positions: %s", cudaGetErrorString(e)); st = GINT_ERR_CUDA; }
            changed = a != b;
        }
    }
    if (st == GINT_OK && keep_pattern && changed) {
        set_error("the new positions need a different pair pattern (%lld blocks, was %lld); the handle is unchanged",
                  (long long)hn->n_blocks, (long long)h->n_blocks);
        st = GINT_ERR_PATTERN_MISMATCH;
    }
    if (st == GINT_OK) {
        hn->wait_limit = h->wait_limit;
        hn->generation = h->generation + 1;
        hn->selecting = h->selecting;
        hn->selection = h->selection;
        if (hn->selecting) st = rebuild_work_lists(hn);
    }
    if (st != GINT_OK) {
        free_handle(hn);
        if (prev >= 0) cudaSetDevice(prev);
        return st;
    }
    std::swap(*h, *hn);
    free_handle(hn);  // the old geometry's device memory
    if (prev >= 0) cudaSetDevice(prev);
    if (pattern_changed) *pattern_changed = changed ? 1 : 0;
    return GINT_OK;
}

gint_status gint_select_bricks(gint_handle* h, int64_t n, const int64_t* bricks) {
    set_error("");
    if (!h) { set_error("gint_select_bricks: NULL handle"); return GINT_ERR_INVALID_ARG; }
    if (bricks && n < 0) { set_error("gint_select_bricks: n < 0"); return GINT_ERR_INVALID_ARG; }
    if (bricks)
        for (int64_t i = 0; i < n; ++i)
            if (bricks[i] < 0 || bricks[i] >= h->n_bricks) {
                set_error("gint_select_bricks: brick %lld out of range [0, %lld)", (long long)bricks[i],
                          (long long)h->n_bricks);
                return GINT_ERR_INVALID_ARG;
            }
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(h->device) != cudaSuccess) { set_error("cannot select device %d", h->device); return GINT_ERR_CUDA; }
    gint_status st = GINT_OK;
    if (cudaDeviceSynchronize() != cudaSuccess) { set_error("gint_select_bricks: device synchronisation failed"); st = GINT_ERR_CUDA; }
    const bool was = h->selecting;
    std::vector<int64_t> old = h->selection;
    if (st == GINT_OK) {
        h->selecting = bricks != nullptr;
        if (bricks) h->selection.assign(bricks, bricks + n); else h->selection.clear();
        st = rebuild_work_lists(h);
        if (st != GINT_OK) { h->selecting = was; h->selection.swap(old); }
        else h->generation += 1;
    }
    if (prev >= 0) cudaSetDevice(prev);
    return st;
}

gint_status gint_brick_loads(const gint_handle* h, int64_t* n_images) {
    if (!h || !n_images) { set_error("gint_brick_loads: NULL argument"); return GINT_ERR_INVALID_ARG; }
    std::vector<int64_t> bs(h->n_bricks + 1);
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(h->device);
    cudaError_t e = cudaMemcpy(bs.data(), h->d_brick_start, sizeof(int64_t) * bs.size(), cudaMemcpyDeviceToHost);
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) { set_error("gint_brick_loads: %s", cudaGetErrorString(e)); return GINT_ERR_CUDA; }
    for (int64_t b = 0; b < h->n_bricks; ++b) n_images[b] = bs[b + 1] - bs[b];
    return GINT_OK;
}

gint_status gint_set_wait_limit(gint_handle* h, int64_t polls) {
    if (!h) { set_error("handle is NULL"); return GINT_ERR_INVALID_ARG; }
    if (polls < 0 || polls > ((int64_t)1 << 40)) { set_error("wait limit %lld out of range", (long long)polls); return GINT_ERR_INVALID_ARG; }
    h->wait_limit = polls;
    return GINT_OK;
}

gint_status gint_debug_fail_alloc(int n) {
    if (n < 0) { set_error("gint_debug_fail_alloc: n < 0"); return GINT_ERR_INVALID_ARG; }
    g_fail_alloc.store(n);
    return GINT_OK;
}

}  // extern "C"
