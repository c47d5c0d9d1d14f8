// tc_rho.cu -- tensor-core (tcgen05) form of rho (Eq. 3) and of the Pulay
// force and stress (Eq. 4, 5).
//
// Both need, at every point p of a brick, G_p = Psi_p D_b (Psi_p: orbital
// values at p over the brick's atom images, D_b the density-matrix blocks of
// those images).  Per 128-point M-tile of a brick:
//   * the tile's active atom images (within the cutoff of a point of the
//     tile; a bit mask per (brick, tile) made once per geometry at set-up)
//     give the N dimension: one 16-column slot per image (<= 512 TMEM
//     columns; 256 in the exact form, more images take further column
//     groups);
//   * the K dimension runs over active atom images, one MMA K-step (16) per
//     image (nw <= 16 orbitals, zero padded), two images per synchronisation:
//     A = Psi restricted to that image (128 points x 16, MN-major), B = the
//     image's D blocks against every image of the group, taken from a
//     per-call pre-formatted copy of D (every pattern block as a 16 x 16
//     tile of 16-bit pieces in K-major core-matrix order, the pieces
//     interleaved per 8-row group), so one slot of B is one bulk copy;
//   * three warp roles hand buffers over with mbarriers: eight warps
//     evaluate A, one warp issues the bulk copies of B, one thread issues
//     the MMAs (which never waits for earlier MMAs to complete);
//   * G accumulates in TMEM (lane = point), three products per step
//     (hi*hi + hi*lo + lo*hi);
//   * exact form (fp16x4): both operands in fixed point, x / q = n + l1 + l2
//     with n an integer of at most 8 bits and l1, l2 fp16 pieces of the
//     remainder; q is one power of two for all orbital values (the largest
//     per-orbital bound) and, for D, one per (atom, orbital row) taken from the
//     largest |D| of that row this call.  Products n*n accumulate exactly in
//     TMEM columns [0, 256) (K <= 1024, products below 2^14); the cross terms
//     n l1 + l1 n + l1 l1 + n l2 + l2 n go to columns [256, 512);
//   * the epilogue thread of point p reads G_p, re-evaluates the orbital
//     values (and gradients for the force) of every active image at p and
//     forms rho_p = sum phi G, or F_I += 2 W_p grad phi . G with the virial
//     and the energy, reduced per image in shared memory before FP64 atomics.
#include <algorithm>
#include <cstring>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fast_orb.cuh"
#include "gint_impl.cuh"
#include "tc_ptx.cuh"

namespace gint {

namespace {
// Warp roles: producer/epilogue warps in groups of 8 (a group fills every
// kGroups-th K step, 2 images x 128 points, one thread per (image, point)),
// then one warp for the bulk copies of B and one for the MMA issue.  rho in
// the exact form runs two groups (two steps produced at once); the force, whose
// epilogue needs 168 registers a thread, and the three-product form, whose
// B buffers leave no shared memory for the larger epilogue staging, one.
template <bool kForce, bool kExact> struct RfWarps {
    static constexpr int kProdWarps = (!kForce && kExact) ? 16 : 8;
    static constexpr int kGroups = kProdWarps / 8;
    static constexpr int kCopyWarp = kProdWarps;      // bulk copies of B
    static constexpr int kMmaWarp = kProdWarps + 1;   // MMA issue (one thread)
    static constexpr int kThreads = 32 * kProdWarps + 64;
};
constexpr int kMaxAtoms = 64;
constexpr int kMaxCols = 512;            // TMEM columns (packed orbitals of one M-tile)
// A pieces (128 points x 16 orbital slots) are MN-major: core matrix (point group
// pg = p / 8, orbital group og = o / 8) holds 8 orbital rows of 8 points (16 B);
// point groups are kASbo = 144 B apart (128 B + 16 B of padding, so that the 32
// points of a warp storing one orbital hit 16 different banks), orbital groups
// kALbo = 16 * 144 B apart.
constexpr int kASbo = 144;
constexpr int kALbo = 16 * kASbo;
constexpr int kAPiece = 2 * kALbo;
constexpr int kDtPiece = 512;            // one 16 x 16 piece of a pre-formatted D block
constexpr int kDtBytes = 3 * kDtPiece;   // per block: up to three pieces (exact form)

// Per form: pieces per operand and B rows (= output columns of a column group).
template <bool kExact> struct RfCfg {
    static constexpr int kPieces = kExact ? 3 : 2;
    static constexpr int kBRows = kExact ? 256 : 512;
    static constexpr int kBPiece = kBRows * 16 * 2;
};
constexpr int kMaxSpecies = 8;

struct Atom {
    float c_hi[3], c_lo[3];  // brick origin - image position (FP64 split into two FP32 words)
    int I, sp, nw;
    int t[3];
};

template <bool kExact, int kPW> struct Smem {
    using C = RfCfg<kExact>;
    unsigned char A[2][2][C::kPieces * kAPiece];   // [buffer][image of the step][pieces]
    unsigned char B[2][2][C::kPieces * C::kBPiece];
    Atom at[kMaxAtoms];
    int pairblk[kMaxAtoms * kMaxAtoms];  // block (I_a2, I_a1, T_a1 - T_a2) for K image a1, N image a2; -1 if none
    float W2[kMaxBrickPts];              // 2 V dV (force)
    double red[kMaxAtoms][13];           // per-image F(3), virial(9), energy
    float rho_part[128];                 // rho of the tile's points over earlier column groups
    float rho_q[kPW / 4 - 1][128];       // partial rho of warps 4 q .. 4 q + 3, q >= 1
    float qd[kMaxCols];                  // exact form: G scale 2^(qa + qD) of each output column of the group
    SpeciesFast spf[kMaxSpecies];
    unsigned char act[kMaxAtoms];
    unsigned char act_next[kMaxAtoms];  // copy warp: active images of the next M-tile
    uint64_t full[2];    // producers wrote A of buffer b (256 arrivals)
    uint64_t empty[2];   // MMAs reading buffer b completed (tcgen05.commit)
    uint64_t bfull[2];   // bulk copies of B into buffer b completed
    uint64_t done;       // all MMAs of a column group completed
    uint32_t tmem;
    int work, abort, nact, ncols;
};

static_assert(sizeof(Smem<false, 8>) + 1024 <= 232448, "shared memory of the rho/force kernel exceeds 227 KB");
static_assert(16 * 32 * 17 * sizeof(float) <= sizeof(Smem<true, 16>::A), "epilogue staging exceeds the A buffers");
static_assert(8 * 32 * 17 * sizeof(float) <= sizeof(Smem<false, 8>::A), "epilogue staging exceeds the A buffers");
static_assert(sizeof(Smem<true, 16>) + 1024 <= 232448, "shared memory of the exact rho/force kernel exceeds 227 KB");

// Exact form: s = n + l1 + l2 (n = rint(s), |s| <= 128; l1, l2 fp16 pieces of s - n).
__device__ __forceinline__ void fix_split3(float s, unsigned short& n16, unsigned short& l1, unsigned short& l2) {
    const float n = rintf(s);
    const float r = s - n;
    const __half h1 = __float2half_rn(r);
    n16 = __half_as_ushort(__float2half_rn(n));
    l1 = __half_as_ushort(h1);
    l2 = __half_as_ushort(__float2half_rn(r - __half2float(h1)));
}

template <typename H16> struct Split;
template <> struct Split<__half> {
    static __device__ __forceinline__ void run(float x, unsigned short& hi, unsigned short& lo) {
        __half h = __float2half_rn(x);
        hi = __half_as_ushort(h);
        lo = __half_as_ushort(__float2half_rn(x - __half2float(h)));
    }
    static constexpr int bf16 = 0;
};
template <> struct Split<__nv_bfloat16> {
    static __device__ __forceinline__ void run(float x, unsigned short& hi, unsigned short& lo) {
        __nv_bfloat16 h = __float2bfloat16_rn(x);
        hi = __bfloat16_as_ushort(h);
        lo = __bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(h)));
    }
    static constexpr int bf16 = 1;
};

// Pre-formatted D tile of one block (16 x 16, K-major core matrices): the pieces
// are interleaved per group of 8 rows, [rows 0-7: piece 0, 1(, 2)][rows 8-15: ...],
// 256 B per (row group, piece), so a tile is one contiguous copy into its image
// slot of B and each piece is a K-major operand with row-group stride kP * 256 B.
__device__ __forceinline__ int dt_off(int i, int j, int pc, int kP) {
    return ((((i >> 3) * kP + pc)) << 8) + ((j >> 3) << 7) + ((i & 7) << 4) + ((j & 7) << 1);
}

// byte offset of A element (point p, orbital slot o) in an MN-major A piece
__device__ __forceinline__ int amn(int p, int o) { return (o >> 3) * kALbo + (p >> 3) * kASbo + ((o & 7) << 4) + ((p & 7) << 1); }

// Sum 16 values over the 32 lanes of a warp with 16 shuffles (each step
// exchanges half of the remaining values with the partner lane).  Afterwards
// lanes L and L ^ 1 hold the total of value index
// 8 b4 + 4 b3 + 2 b2 + b1, b_k = bit k of L; the return value is that total.
__device__ __forceinline__ float warp_sum16(float (&v)[16], int lane) {
#pragma unroll
    for (int o = 16, c = 16; o >= 2; o >>= 1, c >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int k = 0; k < c / 2; ++k) {
            const float keep = up ? v[k + c / 2] : v[k];
            const float send = up ? v[k] : v[k + c / 2];
            v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}
__device__ __forceinline__ int warp_sum16_index(int lane) {
    return (((lane >> 4) & 1) << 3) | (((lane >> 3) & 1) << 2) | (((lane >> 2) & 1) << 1) | ((lane >> 1) & 1);
}

}  // namespace

// Pre-format D: every block b as a 16 x 16 tile (zero padded) of its 16-bit
// pieces (hi, lo; exact form n, l1, l2) in K-major core-matrix order (dt_off),
// values of block b taken from its canonical block (transposed when b is not
// canonical).  One warp per block.
// Largest |D| of every (atom I, orbital row i) over the blocks (I, J, T), as
// FP32 bits (non-negative floats order like their bit patterns).
__global__ void k_dmax(Problem P, const int32_t* mirror, const int* nw_atom, int64_t n_blocks, const double* D,
                       int* dq) {
    const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (b >= n_blocks) return;
    const int32_t* k = P.blocks + 5 * b;
    const int I = k[0], J = k[1];
    const bool canon = (I < J) || (I == J && (k[2] > 0 || (k[2] == 0 && (k[3] > 0 || (k[3] == 0 && k[4] >= 0)))));
    const int64_t src = canon ? b : (int64_t)mirror[b];
    if (src < 0) return;
    const int nI = nw_atom[I], nJ = nw_atom[J];
    const double* Ds = D + P.offsets[src];
    for (int e = lane; e < 256; e += 32) {
        const int i = e >> 4, j = e & 15;
        if (i < nI && j < nJ) {
            const float v = fabsf((float)(canon ? Ds[i * nJ + j] : Ds[j * nI + i]));
            if (v > 0.f) atomicMax(dq + 16 * I + i, __float_as_int(v));
        }
    }
}

// 2^e with |D row max| / 127 < 2^e (1 for an all-zero row)
__device__ __forceinline__ int dq_exp(int bits) {
    int e = 0;
    const float m = __int_as_float(bits);
    if (m > 0.f) frexpf(m * (1.f / 127.f), &e);
    return max(-100, min(100, e));
}
__device__ __forceinline__ float exp2f_i(int e) { return __int_as_float((127 + e) << 23); }  // |e| < 127

template <typename H16, bool kExact>
__global__ void k_format_d(Problem P, const int32_t* mirror, const int* nw_atom, int64_t n_blocks, const double* D,
                           const int* dq, unsigned char* Dt) {
    const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (b >= n_blocks) return;
    const int32_t* k = P.blocks + 5 * b;
    const int I = k[0], J = k[1];
    const bool canon = (I < J) || (I == J && (k[2] > 0 || (k[2] == 0 && (k[3] > 0 || (k[3] == 0 && k[4] >= 0)))));
    const int64_t src = canon ? b : (int64_t)mirror[b];
    const int nI = nw_atom[I], nJ = nw_atom[J];
    const double* Ds = D + P.offsets[src < 0 ? b : src];
    unsigned char* out = Dt + b * kDtBytes;
    for (int e = lane; e < 256; e += 32) {
        const int i = e >> 4, j = e & 15;
        float v = 0.f;
        if (i < nI && j < nJ && src >= 0) v = (float)(canon ? Ds[i * nJ + j] : Ds[j * nI + i]);
        unsigned short hi, lo, l2 = 0;
        if (kExact) fix_split3(v * exp2f_i(-dq_exp(dq[16 * I + i])), hi, lo, l2);
        else Split<H16>::run(v, hi, lo);
        constexpr int kP = kExact ? 3 : 2;
        *reinterpret_cast<unsigned short*>(out + dt_off(i, j, 0, kP)) = hi;
        *reinterpret_cast<unsigned short*>(out + dt_off(i, j, 1, kP)) = lo;
        if (kExact) *reinterpret_cast<unsigned short*>(out + dt_off(i, j, 2, kP)) = l2;
    }
}

// kMulti: the work queue spans the bricks of many cells (a batch, MultiArgs); the
// problem and the buffers of an item come from its cell's CellJob.
template <typename H16, bool kForce, bool kExact, bool kMulti>
__global__ void __launch_bounds__(RfWarps<kForce, kExact>::kThreads, 1) k_rhoforce_tc(const __grid_constant__ CellJob J_in, int* counter, const __grid_constant__ MultiArgs M,
                                                                 long wait_limit) {
    constexpr int kCols = kExact ? kMaxCols / 2 : kMaxCols;  // output columns of one column group
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    using Wr = RfWarps<kForce, kExact>;
    constexpr int kProdWarps = Wr::kProdWarps, kCopyWarp = Wr::kCopyWarp, kMmaWarp = Wr::kMmaWarp;
    constexpr int kThreads = Wr::kThreads;
    Smem<kExact, kProdWarps>& S = *reinterpret_cast<Smem<kExact, kProdWarps>*>(smem_raw);
    using C = RfCfg<kExact>;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const CellJob* Jc = &J_in;  // problem and buffers of the current item
    int cur_cell = -1;

    if (warp == 0) {
        tc::tmem_alloc(&S.tmem, kMaxCols);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&S.full[b], 256);  // one producer group
            tc::mbar_init(&S.empty[b], 1);
            tc::mbar_init(&S.bfull[b], 1);
        }
        tc::mbar_init(&S.done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        S.abort = 0;
    }
    if (!kMulti && tid < J_in.P.n_species) species_fast_from(J_in.P.sp[tid], S.spf[tid]);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = S.tmem;
    // exact form: one quantum 2^qa for every orbital value (the largest per-orbital quantum of the cell)
    float qa_inv = 1.f, qa_f = 1.f;
    auto set_qa = [&](const Problem& Q) {
        int qa = -126;
        for (int sp = 0; sp < Q.n_species; ++sp)
            for (int o = 0; o < S.spf[sp].nw; ++o) qa = max(qa, (int)S.spf[sp].qe[o]);
        qa_inv = exp2f_i(-qa);
        qa_f = exp2f_i(qa);
    };
    if (kExact && !kMulti) set_qa(J_in.P);
    uint32_t uses[2] = {0, 0};  // steps that used buffer b (every thread counts them)
    int a_rows0 = 16, a_rows1 = 16;  // producers: rows of their A column in buffer 0 / 1 that may be non-zero
    uint32_t dones = 0;         // completed phases of done
    uint32_t bissue[2] = {0, 0};  // copy warp: bulk-copy phases started per buffer
    int ahead = 0;                 // copy warp: steps of the coming column group already copied
    uint32_t chunk = 0;  // global chunk counter (buffer parity)

    for (;;) {
        if (tid == 0) S.work = atomicAdd(counter, 1);
        __syncthreads();
        const int w = S.work;
        if (w >= (kMulti ? M.n_items : J_in.P.n_work) || S.abort) break;
        int wl = w;
        if (kMulti) {
            const int c = M.item_cell[w];
            wl = w - M.jobs[c].item0;
            if (c != cur_cell) {  // uniform: every thread read the same item
                cur_cell = c;
                Jc = &M.jobs[c];
                if (tid < Jc->P.n_species) species_fast_from(Jc->P.sp[tid], S.spf[tid]);
                __syncthreads();
                if (kExact) set_qa(Jc->P);
            }
        }
        const Problem& P = Jc->P;
        const GridDev& g = P.g;
        const double* V = Jc->V;
        const unsigned char* Dt = Jc->Dt;
        const unsigned char* Dzero = Jc->Dzero;
        const int* dq = Jc->dq;
        double* rho = Jc->rho;
        double* facc = Jc->facc;
        double* acc_e = Jc->acc_e;
        const float2* knot2 = P.knot32;
        const int brick = P.work[wl];
        int b0, b1, b2;
        brick_coords(g, brick, b0, b1, b2);
        const int64_t s0 = P.brick_start[brick];
        const int na = (int)(P.brick_start[brick + 1] - s0);
        for (int i = tid; i < na; i += kThreads) {
            const ExtAtom X = P.ext[P.brick_atoms[s0 + i]];
            Atom& a = S.at[i];
            brick_atom_offset(g, b0, b1, b2, X, a.c_hi, a.c_lo);  // as in the set-up tile masks
            a.I = X.atom;
            a.sp = X.species;
            a.nw = P.sp[X.species].n_orb;
            a.t[0] = X.t[0]; a.t[1] = X.t[1]; a.t[2] = X.t[2];
        }
        if (kForce) {
            for (int p = tid; p < g.bpad; p += kThreads) {
                int g0, g1, g2;
                float wv = 0.f;
                if (brick_point(g, b0, b1, b2, p, g0, g1, g2))
                    wv = (float)(2.0 * ld_stream_f64(V + ((int64_t)g0 * g.n[1] + g1) * g.n[2] + g2) * g.dV);
                S.W2[p] = wv;
            }
        }
        __syncthreads();
        // ordered pair table: B rows of N image a2 for K image a1 come from block (I_a2, I_a1, T_a1 - T_a2),
        // entry (a2, a1) of the brick's pair table (built once per geometry)
        {
            const int32_t* pt = P.pairs + P.pair_start[brick];
            for (int q = tid; q < na * na; q += kThreads) {
                const int a1 = q / na, a2 = q - a1 * na;
                S.pairblk[q] = ld_stream_s32(pt + a2 * na + a1);
            }
        }
        __syncthreads();

        const int n_mtiles = (g.bpad + 127) / 128;
        // copy warp: the B copies of one step into buffer bb, K images actK[kk], actK[kk + 1] (nkk
        // of them) against the column images actN[n0 .. n0 + per_img); lane 0 waits until the
        // buffer's earlier MMAs and copies are done and opens the transaction phase
        auto copy_step = [&](int bb, const unsigned char* actK, int kk, int nkk, const unsigned char* actN, int n0,
                             int per_img) {
            int go = 0;
            if (lane == 0) {
                if (uses[bb] > 0 && !tc::mbar_wait(&S.empty[bb], (uses[bb] - 1) & 1, wait_limit)) atomicOr(&S.abort, 1);
                // at most one transaction phase of bfull[bb] is ever open: the copies issued
                // into this buffer before have landed (already true unless a wait gave up)
                if (bissue[bb] > 0 && !tc::mbar_wait(&S.bfull[bb], (bissue[bb] - 1) & 1, kDrainPolls))
                    atomicOr(&S.abort, 1);
                go = S.abort ? 0 : 1;  // after an abort no further copies are started
                if (go) {
                    tc::mbar_arrive_expect_tx(&S.bfull[bb], (uint32_t)(nkk * per_img * C::kPieces * kDtPiece));
                    bissue[bb] += 1;
                }
            }
            go = __shfl_sync(0xffffffffu, go, 0);
            for (int e = lane; go && e < nkk * per_img; e += 32) {
                const int jj = e / per_img, sl = e - jj * per_img;
                const int blk = S.pairblk[actK[kk + jj] * na + actN[n0 + sl]];
                const unsigned char* src = blk >= 0 ? Dt + (int64_t)blk * kDtBytes : Dzero;
                tc::bulk_copy_g2s(&S.B[bb][jj][sl * C::kPieces * kDtPiece], src, C::kPieces * kDtPiece, &S.bfull[bb]);
            }
            uses[bb] += 1;
        };
        for (int mt = 0; mt < n_mtiles && !S.abort; ++mt) {
            // ---- active atom images of this M-tile (images within rc of a point of the tile;
            //      tested once per geometry at set-up, k_tile_mask)
            if (warp == 0) {
                const unsigned long long m = __ldg(P.tile_mask + (int64_t)wl * n_mtiles + mt);  // bits < na only
                for (int h2 = 0; h2 < 2; ++h2) {
                    const int a = lane + 32 * h2;
                    if (m >> a & 1ull) S.act[__popcll(m & ((1ull << a) - 1ull))] = (unsigned char)a;
                }
                if (lane == 0) S.nact = __popcll(m);
            }
            __syncthreads();
            const int nact = S.nact;
            if (nact == 0) {
                if (!kForce && tid < 128) {
                    const int p = mt * 128 + tid;
                    int g0, g1, g2;
                    if (brick_point(g, b0, b1, b2, p, g0, g1, g2)) rho[((int64_t)g0 * g.n[1] + g1) * g.n[2] + g2] = 0.0;
                }
                continue;
            }
            if (S.abort) break;
            // column groups: consecutive active images, one 16-column slot each (a slot holds
            // an image's <= 16 orbitals, zero padded), at most kCols / 16 images per group
            for (int cg0 = 0; cg0 < nact && !S.abort;) {
            const int cg1 = min(nact, cg0 + kCols / 16);
            const int ncols = 16 * (cg1 - cg0);
            if (kExact)  // G scale of every output column: 2^qa x 2^qD(atom, orbital row); read after the K loop
                for (int e = tid; e < ncols; e += kThreads) {
                    const Atom& Y = S.at[S.act[cg0 + (e >> 4)]];
                    const int o = e & 15;
                    S.qd[e] = o < Y.nw ? qa_f * exp2f_i(dq_exp(__ldg(dq + 16 * Y.I + o))) : 0.f;
                }
            // ---- K loop over active images, two images (K = 32) per step.  Warps 0-7 produce
            // A (orbital values of the step's two K images at the tile's 128 points) into
            // buffer b = step & 1 and arrive on full[b]; warp 8 fetches B and lane 0 of it
            // issues the MMAs of a step once full[b] and bfull[b] complete, then commits
            // empty[b].  B (bulk asynchronous copies by warp 8): for K image a1 = act[k + j]
            // and the image a2 in slot s of the group, the pre-formatted tile of block
            // (I_a2, I_a1, T_a1 - T_a2) (a zero tile when the pair has no block), 512 B per
            // piece, is exactly the slot's 16-byte rows in the K-major B layout; the copies
            // of step s + 1 start as soon as the MMAs of step s - 1 complete.
            const int nsteps = (nact + 1) >> 1;
            // the previous group's epilogue staged its G values in the A buffers: no padding row
            // of A is known to be zero any more
            a_rows0 = a_rows1 = 16;
            if (warp < kProdWarps) {
                // group grp fills steps grp, grp + kGroups, ...; the previous use of a step's
                // buffer is then the group's own previous step (kGroups = 2) or the step before
                const int grp = warp >> 3, j = (tid >> 7) & 1, pl = tid & 127;
                for (int st = 0; st < nsteps; ++st) {
                    const int b = (chunk + st) & 1, k = 2 * st;
                    const int nk = min(2, nact - k);
                    if (Wr::kGroups > 1 && st % Wr::kGroups != grp) {
                        uses[b] += 1;
                        continue;
                    }
                    // buffer b is free once the MMAs of its previous step completed; a thread
                    // waits for that before its first store (with its knot loads in flight) or
                    // before it arrives
                    bool freed = uses[b] == 0;
                    auto ensure_free = [&]() {
                        if (freed) return;
                        if (!tc::mbar_wait(&S.empty[b], (uses[b] - 1) & 1, wait_limit)) atomicOr(&S.abort, 1);
                        freed = true;
                    };
                    if (j < nk && !S.abort) {
                        const Atom& X = S.at[S.act[k + j]];
                        const int p = mt * 128 + pl;
                        unsigned char* A0 = S.A[b][j];
                        bool inside = false;
                        if (p < g.bpts) {
                            float fx, fy, fz;
                            point_offset(g, p, fx, fy, fz);
                            const float dx = (X.c_hi[0] + fx) + X.c_lo[0];
                            const float dy = (X.c_hi[1] + fy) + X.c_lo[1];
                            const float dz = (X.c_hi[2] + fz) + X.c_lo[2];
                            auto put = [&](int o, float v, float, float, float) {
                                unsigned short hi, lo, l2 = 0;
                                if (kExact) fix_split3(v * qa_inv, hi, lo, l2);
                                else Split<H16>::run(v, hi, lo);
                                *reinterpret_cast<unsigned short*>(A0 + amn(pl, o)) = hi;
                                *reinterpret_cast<unsigned short*>(A0 + kAPiece + amn(pl, o)) = lo;
                                if (kExact) *reinterpret_cast<unsigned short*>(A0 + 2 * kAPiece + amn(pl, o)) = l2;
                            };
                            inside = orbitals_fast<false>(S.spf[X.sp], knot2, dx, dy, dz, put, ensure_free);
                        }
                        ensure_free();
                        // slot rows [nw, 16) must be zero; rows at or above the thread's last nw
                        // in this buffer already are (each thread owns one (slot, point) column)
                        const int dirty = b ? a_rows1 : a_rows0;
                        for (int o = X.nw; o < dirty; ++o)
                            for (int pc = 0; pc < C::kPieces; ++pc)
                                *reinterpret_cast<unsigned short*>(A0 + pc * kAPiece + amn(pl, o)) = 0;
                        if (b) a_rows1 = X.nw; else a_rows0 = X.nw;
                        if (!inside)
                            for (int o = 0; o < X.nw; ++o)
                                for (int pc = 0; pc < C::kPieces; ++pc)
                                    *reinterpret_cast<unsigned short*>(A0 + pc * kAPiece + amn(pl, o)) = 0;
                    }
                    ensure_free();
                    tc::fence_async_smem();
                    tc::mbar_arrive(&S.full[b]);
                    uses[b] += 1;
                }
            } else if (warp == kCopyWarp) {
                // B copies of every step; buffer b is refilled once the MMAs of the step
                // that last read it have completed (empty[b]).  The first `ahead` steps were
                // copied during the previous group's epilogue.
                for (int st = ahead; st < nsteps; ++st) {
                    const int kk = 2 * st;
                    copy_step((chunk + st) & 1, S.act, kk, min(2, nact - kk), S.act, cg0, cg1 - cg0);
                }
                ahead = 0;
            } else {
                // MMA issue: one thread waits for A (full) and B (bfull) of each step, issues
                // its MMAs and commits empty[b]; it never waits for earlier MMAs, so the
                // tensor pipe has the next step queued while the current one runs
                for (int st = 0; st < nsteps; ++st) {
                    const int b = (chunk + st) & 1, k = 2 * st;
                    const int nk = min(2, nact - k);
                    if (lane == 0) {
                        if (!S.abort && !tc::mbar_wait(&S.full[b], uses[b] & 1, wait_limit)) atomicOr(&S.abort, 1);
                        if (!S.abort && !tc::mbar_wait(&S.bfull[b], uses[b] & 1, wait_limit)) atomicOr(&S.abort, 1);
                        tc::fence_after_sync();
                        for (int jm = 0; jm < nk && !S.abort; ++jm) {
                            const uint32_t a_hi = tc::smem_u32(S.A[b][jm]), a_lo = a_hi + kAPiece, a_l2 = a_lo + kAPiece;
                            const uint32_t bb = tc::smem_u32(S.B[b][jm]);
                            for (int n0 = 0; n0 < ncols; n0 += 256) {
                                const int nn = min(256, ncols - n0);
                                const uint32_t idesc = tc::idesc_f16(128, nn, Split<H16>::bf16, 1, 0);  // A MN-major
                                // B pieces interleaved per row group: row-group stride kSboB, piece pc at + 256 pc
                                constexpr uint32_t kSboB = C::kPieces * 256;
                                const uint32_t b_hi = bb + (n0 >> 3) * kSboB, b_lo = b_hi + 256, b_l2 = b_hi + 512;
                                const uint32_t d = tmem + (uint32_t)n0;
                                // B K-major with 16 K-columns: LBO (K-adjacent cores) 128 B, SBO (row groups) kSboB;
                                // A MN-major: LBO (orbital groups) kALbo, SBO (point groups) kASbo
                                const uint32_t acc = (k + jm) > 0 ? 1u : 0u;
                                tc::mma_f16(d, tc::smem_desc(a_hi, kALbo, kASbo), tc::smem_desc(b_hi, 128, kSboB), idesc, acc);
                                if (kExact) {
                                    const uint32_t d1 = d + kCols;  // cross terms
                                    tc::mma_f16(d1, tc::smem_desc(a_hi, kALbo, kASbo), tc::smem_desc(b_lo, 128, kSboB), idesc, acc);
                                    tc::mma_f16(d1, tc::smem_desc(a_lo, kALbo, kASbo), tc::smem_desc(b_hi, 128, kSboB), idesc, 1u);
                                    tc::mma_f16(d1, tc::smem_desc(a_lo, kALbo, kASbo), tc::smem_desc(b_lo, 128, kSboB), idesc, 1u);
                                    tc::mma_f16(d1, tc::smem_desc(a_hi, kALbo, kASbo), tc::smem_desc(b_l2, 128, kSboB), idesc, 1u);
                                    tc::mma_f16(d1, tc::smem_desc(a_l2, kALbo, kASbo), tc::smem_desc(b_hi, 128, kSboB), idesc, 1u);
                                } else {
                                    tc::mma_f16(d, tc::smem_desc(a_hi, kALbo, kASbo), tc::smem_desc(b_lo, 128, kSboB), idesc, 1u);
                                    tc::mma_f16(d, tc::smem_desc(a_lo, kALbo, kASbo), tc::smem_desc(b_hi, 128, kSboB), idesc, 1u);
                                }
                            }
                        }
                        tc::mma_commit(&S.empty[b]);
                        if (st + 1 == nsteps) tc::mma_commit(&S.done);
                    }
                    __syncwarp();
                    uses[b] += 1;
                }
            }
            chunk += nsteps;
            // ---- all MMAs of this group complete (every thread waits on done)
            if (!tc::mbar_wait(&S.done, dones & 1, kDrainPolls)) atomicOr(&S.abort, 1);
            dones += 1;
            tc::fence_after_sync();
            if (kForce) {
                for (int e = tid; e < kMaxAtoms * 13; e += kThreads) (&S.red[0][0])[e] = 0.0;
            }
            __syncthreads();
            if (S.abort) break;
            // ---- epilogue: lane = point (TMEM lane 32 (warp & 3) + lane); warps w and w + 4
            //      take alternate atom images of the group
            {
                const int pl = (warp & 3) * 32 + lane;  // point within the tile
                const int p = mt * 128 + pl;
                int g0 = 0, g1 = 0, g2 = 0;
                const bool pv = brick_point(g, b0, b1, b2, p, g0, g1, g2);
                float fx = 0.f, fy = 0.f, fz = 0.f;
                if (p < g.bpts) point_offset(g, p, fx, fy, fz);
                float rho_p = (cg0 == 0 || warp >= 4) ? 0.f : S.rho_part[pl];
                for (int j = cg0 + (warp >> 2); warp < kProdWarps && j < cg1; j += kProdWarps / 4) {
                    const int a2 = S.act[j];
                    const Atom& Y = S.at[a2];
                    const int c0 = 16 * (j - cg0);  // the image's slot
                    constexpr int sh = 0;
                    float Gv[16];
                    const uint32_t ta = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)c0;
                    tc::tmem_ld16(ta, Gv);
                    // G values of the image for this lane (a padded row of 17), staged in the A
                    // buffers: every MMA of the group has completed, and the next group's
                    // producers write A only after the epilogue's closing barrier
                    float* gs = reinterpret_cast<float*>(&S.A[0][0][0]) + (warp * 32 + lane) * 17;
                    if (kExact) {
                        // G = (exact integer part + cross terms) x 2^qa x 2^qD(atom, row)
                        float G1[16];
                        tc::tmem_ld16(ta + kCols, G1);
                        const float* qc = S.qd + c0;
#pragma unroll
                        for (int o = 0; o < 16; ++o) gs[o] = (Gv[o] + G1[o]) * qc[o];
                    } else {
#pragma unroll
                        for (int o = 0; o < 16; ++o) gs[o] = Gv[o];
                    }
                    const float dx = (Y.c_hi[0] + fx) + Y.c_lo[0];
                    const float dy = (Y.c_hi[1] + fy) + Y.c_lo[1];
                    const float dz = (Y.c_hi[2] + fz) + Y.c_lo[2];
                    float e_j = 0.f, f0 = 0.f, f1 = 0.f, f2 = 0.f;
                    if (pv) {
                        auto put = [&](int o, float v, float gx, float gy, float gz) {
                            const float gv = gs[o + sh];
                            e_j += v * gv;
                            if (kForce) { f0 += gx * gv; f1 += gy * gv; f2 += gz * gv; }
                        };
                        (void)orbitals_fast<kForce>(S.spf[Y.sp], knot2, dx, dy, dz, put);
                    }
                    rho_p += e_j;
                    if (kForce) {
                        // per point in FP32, summed over the warp's 32 points in FP32,
                        // then accumulated per image in FP64
                        const float w2 = pv ? S.W2[p] : 0.f;
                        float v[16];
                        v[0] = w2 * f0; v[1] = w2 * f1; v[2] = w2 * f2;
                        const float d3[3] = {dx, dy, dz};
#pragma unroll
                        for (int a = 0; a < 3; ++a)
#pragma unroll
                            for (int c = 0; c < 3; ++c) v[3 + 3 * a + c] = v[a] * d3[c];
                        v[12] = 0.5f * w2 * e_j;
                        v[13] = v[14] = v[15] = 0.f;
                        const float tot = warp_sum16(v, lane);
                        const int q = warp_sum16_index(lane);
                        if (!(lane & 1) && q < 13) atomicAdd(&S.red[j][q], (double)tot);
                    }
                }
                if (warp >= 4 && warp < kProdWarps) S.rho_q[(warp >> 2) - 1][pl] = rho_p;
                // copy warp of the force kernel, while the others run the epilogue (the force's is
                // long enough to hide the copies; in rho it made the call slower): both B buffers are
                // free (every MMA of the group completed); copy the first two steps of the next
                // column group of the brick (the next group of this M-tile, else the first group of
                // the next M-tile)
                if (kForce && warp == kCopyWarp && !S.abort) {
                    const unsigned char* aK = S.act;
                    int nK = 0, n0 = 0;
                    if (cg1 < nact) {
                        nK = nact;
                        n0 = cg1;
                    } else if (mt + 1 < n_mtiles) {
                        const unsigned long long m = __ldg(P.tile_mask + (int64_t)wl * n_mtiles + mt + 1);
                        for (int h2 = 0; h2 < 2; ++h2) {
                            const int a = lane + 32 * h2;
                            if (m >> a & 1ull) S.act_next[__popcll(m & ((1ull << a) - 1ull))] = (unsigned char)a;
                        }
                        __syncwarp();
                        nK = __popcll(m);
                        aK = S.act_next;
                    }
                    if (nK > 0) {
                        const int nN = min(nK, n0 + kCols / 16) - n0;
                        ahead = min(2, (nK + 1) >> 1);
                        for (int st = 0; st < ahead; ++st)
                            copy_step((chunk + st) & 1, aK, 2 * st, min(2, nK - 2 * st), aK, n0, nN);
                    }
                }
                tc::fence_before_sync();
                __syncthreads();
                if (warp < 4) {
#pragma unroll
                    for (int q = 0; q < kProdWarps / 4 - 1; ++q) rho_p += S.rho_q[q][pl];
                    S.rho_part[pl] = rho_p;
                    if (!kForce && pv && cg1 == nact) rho[((int64_t)g0 * g.n[1] + g1) * g.n[2] + g2] = (double)rho_p;
                }
            }
            __syncthreads();
            if (kForce) {
                for (int e = tid; e < nact * 13; e += kThreads) {
                    const int j = e / 13, q = e - j * 13;
                    const double v = S.red[j][q];
                    if (v == 0.0) continue;
                    if (q < 12) atomicAdd(facc + 12 * (size_t)S.at[S.act[j]].I + q, v);
                    else atomicAdd(acc_e, v);
                }
                __syncthreads();
            }
            cg0 = cg1;
            }  // column groups
        }
        __syncthreads();
    }
    __syncthreads();
    // no MMA or bulk copy may be in flight when tensor memory and shared memory are released:
    // one more commit (completes after every earlier MMA) and the copies not yet waited for
    if (warp == kMmaWarp && lane == 0) {
        tc::mma_commit(&S.done);
        (void)tc::mbar_wait(&S.done, dones & 1, kDrainPolls);
    }
    if (warp == kCopyWarp && lane == 0)  // the last phase of each buffer covers every earlier copy
        for (int b = 0; b < 2; ++b)
            if (bissue[b] > 0) (void)tc::mbar_wait(&S.bfull[b], (bissue[b] - 1) & 1, kDrainPolls);
    if (S.abort && tid == 0) atomicOr(Jc->P.err, kErrTimeout);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kMaxCols);
}

// ------------------------------------------------------------------ host
static gint_status ensure_dt(gint_handle* h) {
    if (!h->d_dt) {
        const size_t bytes = (size_t)std::max<int64_t>(1, h->n_blocks) * kDtBytes;
        GINT_CUDA_TRY(dev_malloc(&h->d_dt, bytes));
    }
    if (!h->d_dq) GINT_CUDA_TRY(dev_malloc(&h->d_dq, sizeof(int) * 16 * (size_t)std::max(1, h->n_atoms)));
    if (!h->d_zero) {  // a zero D tile for atom-image pairs without a block
        GINT_CUDA_TRY(dev_malloc(&h->d_zero, kDtBytes));
        GINT_CUDA_TRY(cudaMemset(h->d_zero, 0, kDtBytes));
    }
    return GINT_OK;
}

// Allocations the tensor-core calls make on first use, done ahead of a graph capture.
gint_status tc_prepare(gint_handle* h) {
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(h->device);
    gint_status s = ensure_dt(h);
    if (prev >= 0) cudaSetDevice(prev);
    return s;
}

// form: 0 = fp16x3, 1 = bf16x3, 2 = fp16x4 (exact leading term)
gint_status tc_rhoforce_check(const gint_handle* h) {
    if (h->max_brick_atoms > kMaxAtoms || h->max_nw > 16 || h->n_species > kMaxSpecies) {
        set_error("tensor-core rho/force needs <= %d atom images per brick, <= 16 orbitals per atom and <= %d "
                  "species (have %d, %d, %d); use smaller bricks", kMaxAtoms, kMaxSpecies, h->max_brick_atoms,
                  h->max_nw, h->n_species);
        return GINT_ERR_UNSUPPORTED;
    }
    return GINT_OK;
}

// The per-call tensor-core copy of D (and, exact form, its row maxima).
gint_status tc_format_d(gint_handle* h, int form, const double* D, cudaStream_t st) {
    gint_status s = ensure_dt(h);
    if (s != GINT_OK) return s;
    if (h->n_blocks == 0) return GINT_OK;
    const Problem P = h->problem();
    const unsigned grid = (unsigned)((h->n_blocks * 32 + 255) / 256);
    unsigned char* dt = (unsigned char*)h->d_dt;
    if (form == 2) {
        GINT_CUDA_TRY(cudaMemsetAsync(h->d_dq, 0, sizeof(int) * 16 * (size_t)h->n_atoms, st));
        k_dmax<<<grid, 256, 0, st>>>(P, h->d_mirror, h->d_nw_atom, h->n_blocks, D, h->d_dq);
        k_format_d<__half, true><<<grid, 256, 0, st>>>(P, h->d_mirror, h->d_nw_atom, h->n_blocks, D, h->d_dq, dt);
    } else if (form == 1) {
        k_format_d<__nv_bfloat16, false><<<grid, 256, 0, st>>>(P, h->d_mirror, h->d_nw_atom, h->n_blocks, D, h->d_dq, dt);
    } else {
        k_format_d<__half, false><<<grid, 256, 0, st>>>(P, h->d_mirror, h->d_nw_atom, h->n_blocks, D, h->d_dq, dt);
    }
    GINT_CUDA_TRY(cudaGetLastError());
    return GINT_OK;
}

// A cell's job for the rho/force kernel (D already formatted by tc_format_d).
CellJob tc_cell_job(gint_handle* h, const double* V, double* H, double* rho, double* facc, double* acc_e) {
    CellJob J;
    memset(&J, 0, sizeof(J));
    J.P = h->problem();
    J.V = V;
    J.H = H;
    J.Dt = (const unsigned char*)h->d_dt;
    J.Dzero = (const unsigned char*)h->d_zero;
    J.dq = h->d_dq;
    J.rho = rho;
    J.facc = facc;
    J.acc_e = acc_e;
    return J;
}

// One launch of the rho or force kernel: one cell (M.n_items == 0: J) or a batch queue (M).
static gint_status launch_rf(int form, bool force, const CellJob& J, const MultiArgs& M, bool multi, int* counter,
                             int sm_count, long wait_limit, cudaStream_t st) {
    const bool exact = form == 2;
    GINT_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(int), st));
#define GINT_LAUNCH_RF(H16, F, X, MU)                                                                          \
    do {                                                                                                        \
        const size_t smem = sizeof(Smem<X, RfWarps<F, X>::kProdWarps>) + 1024;                                  \
        GINT_CUDA_TRY(cudaFuncSetAttribute(k_rhoforce_tc<H16, F, X, MU>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                           (int)smem));                                                         \
        k_rhoforce_tc<H16, F, X, MU><<<sm_count, RfWarps<F, X>::kThreads, smem, st>>>(J, counter, M, wait_limit);   \
    } while (0)
#define GINT_LAUNCH_RF2(H16, X, MU) \
    do { if (force) GINT_LAUNCH_RF(H16, true, X, MU); else GINT_LAUNCH_RF(H16, false, X, MU); } while (0)
    if (multi) {
        if (form == 1) GINT_LAUNCH_RF2(__nv_bfloat16, false, true);
        else if (exact) GINT_LAUNCH_RF2(__half, true, true);
        else GINT_LAUNCH_RF2(__half, false, true);
    } else {
        if (form == 1) GINT_LAUNCH_RF2(__nv_bfloat16, false, false);
        else if (exact) GINT_LAUNCH_RF2(__half, true, false);
        else GINT_LAUNCH_RF2(__half, false, false);
    }
#undef GINT_LAUNCH_RF2
#undef GINT_LAUNCH_RF
    GINT_CUDA_TRY(cudaGetLastError());
    return GINT_OK;
}

gint_status tc_rhoforce(gint_handle* h, int form, bool force, const double* V, const double* D, double* rho,
                        double* facc, double* acc_e, cudaStream_t st) {
    gint_status s = tc_rhoforce_check(h);
    if (s != GINT_OK) return s;
    s = tc_format_d(h, form, D, st);
    if (s != GINT_OK || h->n_work == 0) return s;
    return launch_rf(form, force, tc_cell_job(h, V, nullptr, rho, facc, acc_e), MultiArgs{}, false, h->d_err + 2,
                     h->sm_count, wait_polls(h), st);
}

// One launch over the (cell, brick) queue of a batch (every cell's D formatted, cells checked).
gint_status tc_rhoforce_multi(int form, bool force, const MultiArgs& M, int* counter, int sm_count, cudaStream_t st) {
    if (M.n_items == 0) return GINT_OK;
    CellJob none;
    memset(&none, 0, sizeof(none));
    return launch_rf(form, force, none, M, true, counter, sm_count, kDefaultWaitPolls, st);
}

}  // namespace gint
