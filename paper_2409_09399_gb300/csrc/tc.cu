// tc.cu -- tensor-core (tcgen05) form of the H^V grid integral (Eq. 2).
//
// Per brick of grid points the contraction H_b = Psi^T diag(W) Psi (Psi: brick
// points x brick orbitals, W_p = V_p dV) is a dense small GEMM (Section 2.2: taking
// the points in batches turns the per-point products into one matrix product).  Here it
// runs on the 5th-generation tensor cores:
//   * orbital rows of the brick are padded to tiles of 128; the upper-triangle
//     tile pairs (i <= j) accumulate in tensor memory (TMEM, 128 lanes x 512
//     FP32 columns: up to four 128 x 128 tiles per pass);
//   * the K dimension (points) is consumed in chunks of 16 points.  For each
//     chunk every thread of the CTA evaluates orbital values in FP32 and writes
//     them to shared memory as two 16-bit pieces, x = hi + lo, for both
//     operands A = 2^s W Psi and B = Psi, in the canonical no-swizzle layout
//     (8 x 8 core matrices of 128 bytes, K-major); one thread issues
//     A_hi B_hi + A_hi B_lo + A_lo B_hi as three tcgen05.mma per tile pair;
//     two chunk buffers alternate so orbital evaluation overlaps the MMAs;
//   * after the last chunk the accumulators are read back (tcgen05.ld), scaled
//     by 2^-s and added to the canonical H blocks with FP64 atomics.
// Measured errors of the three-product form grow with the number of MMA
// additions per element (96 per brick) the way a rounding biased towards zero
// in the FP32 accumulator predicts, and the bias does not average out over the
// bricks that add into one H element.  The exact form (fp16x4) avoids that
// bias for the leading term: the orbital values are taken without the
// harmonic normalisation (applied in FP64 in the epilogue, so that its FP32
// rounding does not scale whole rows of H), and every operand value x of row
// (orbital) o is written as x / q_o = n + l1 + l2 with q_o = 2^qe_o a
// per-orbital quantum (|x| <= 127 q_o at every point), n = rint(x / q_o) an
// integer of at most 8 bits and l1, l2 two fp16 pieces of the remainder.  Products n_a n_b are
// integers below 2^14, so their sums over <= 512 points stay below 2^23 and
// accumulate exactly in FP32; the cross terms n l1 + l1 n + l1 l1 + n l2 + l2 n
// (2^-7 of the leading term) go to a second accumulator.  Each output column
// then takes two TMEM columns, so a pass holds 256 output columns.
// The atom-to-brick displacement is taken in FP64 once per (brick, atom) and
// split into two FP32 words; in-brick offsets are FP32.
#include <algorithm>
#include <cstring>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fast_orb.cuh"
#include "gint_impl.cuh"
#include "tc_ptx.cuh"

namespace gint {

constexpr int kTcChunk = 16;        // points per K chunk (one MMA K step)
constexpr int kTcMaxAtoms = 64;     // atom images per brick
constexpr int kTcMaxSpecies = 8;
constexpr int kTcMaxSeg = 16;       // (row tile, column range) segments per brick

// Sizes of the two forms (up to 640 padded orbital rows, 5 tiles of 128, in both).
// Each form has one group of producer warps per operand buffer (a group fills
// every kGroups-th chunk), plus one MMA-issuing warp.
// Three-product form: pieces A_hi, A_lo, B_hi, B_lo over all rows; up to 1024
// points per brick; two operand buffers, two groups of 8 warps (17 warps).
// Exact form: pieces A_n, A_l1, A_l2 for the row tiles of the current pass only
// (a pass of <= 256 output columns spans at most three row tiles) and B_n, B_l1,
// B_l2 for the columns the pass's segments read only (at most 256 rows, packed
// in 16-row groups, plus one 16-row group that takes the stores of rows the pass
// does not read); up to 512 points per brick (the integer products of 512 points
// stay below 2^23); three operand buffers and three groups of 6 warps (19 warps
// with the issuer): three chunks are produced at once, a group waits for the
// MMAs of its own previous chunk only, and a pass of up to 24 atom images takes
// one item per thread.
template <bool kExact> struct TcCfg {
    static constexpr int kPieces = kExact ? 3 : 2;            // pieces per operand
    static constexpr int kRows = 640;
    static constexpr int kARows = kExact ? 384 : 640;         // rows held by an A piece
    static constexpr int kBRows = kExact ? 256 + 16 : 640;    // rows held by a B piece
    static constexpr int kBufs = kExact ? 3 : 2;              // operand buffers
    static constexpr int kPts = kExact ? 512 : 1024;
    static constexpr int kAPieceBytes = kARows * kTcChunk * 2;  // rows x 16 points x 2 B
    static constexpr int kBPieceBytes = kBRows * kTcChunk * 2;
    static constexpr int kBOff = kPieces * kAPieceBytes;        // first B piece in a buffer
    static constexpr int kBufBytes = kPieces * (kAPieceBytes + kBPieceBytes);
    static constexpr int kPassCols = kExact ? 256 : 512;      // output columns per pass
    static constexpr int kGroups = kBufs;                     // producer groups, one chunk in flight each
    static constexpr int kGroupWarps = kExact ? 6 : 8;
    static constexpr int kGroupThreads = 32 * kGroupWarps;
    static constexpr int kProdWarps = kGroups * kGroupWarps;
    static constexpr int kThreads = 32 * (kProdWarps + 1);    // + the MMA-issuing warp
    // A group's chunks use one buffer, so its previous chunk there (whose `empty` wait it
    // passed) orders the buffer's phases: a wait on the parity of phase u never runs while
    // the barrier is still in phase u - 2, which a parity wait cannot tell from phase u.
    static_assert(kGroups == kBufs, "one producer group per operand buffer");
};

struct TcAtom {
    float c_hi[3], c_lo[3];  // (brick origin - atom image position), FP64 split into two FP32 words
    int I;
    int sp;
    int nw;
    int off;
    int t[3];
};

struct TcArgs {
    Problem P;
    int* counter;
    long wait_limit;  // polls of a bounded hand-off wait (producers <-> MMA issue)
    int norm_after;  // exact form: leave the harmonic normalisation to k_norm_h (H not accumulated into)
};

template <bool kExact> struct TcSmem {
    using C = TcCfg<kExact>;
    unsigned char buf[C::kBufs][C::kBufBytes];
    TcAtom at[kTcMaxAtoms];
    int pairblk[kTcMaxAtoms * (kTcMaxAtoms + 1) / 2];  // block of image pair a1 <= a2 (index a2 (a2+1)/2 + a1), -1 if none
    float4 pt[C::kPts];             // in-brick offset of each point (x, y, z) and 2^s V dV
    SpeciesFast spf[kTcMaxSpecies];
    unsigned char row_atom[C::kRows];
    unsigned char row_mu[C::kRows];
    unsigned short rowtab[C::kRows];  // byte offset of row r's 16-byte segment in a piece
    unsigned short rowtabB[C::kRows]; // the same in a B piece (exact form: the pass's packed column rows)
    short grp_pos[C::kRows / 16];     // exact form: packed position of each 16-column group the pass reads, -1 if none
    double row_s[C::kRows];           // exact form: [ylm_norm x] 2^qeu of row r (FP64)
    float row_f[C::kRows];            // exact form: 2^qeu of row r
    unsigned char need_list[kTcMaxAtoms];  // atom images with rows the current pass reads
    int n_need;
    unsigned char seg_tile[kTcMaxSeg];  // segment: row tile, columns [c0, c1), TMEM column
    short seg_c0[kTcMaxSeg], seg_c1[kTcMaxSeg], seg_tcol[kTcMaxSeg];
    int pass_first[kTcMaxSeg + 1];      // first segment of each pass
    int npass, nrow, ncol;
    float wmax[C::kThreads / 32];  // per-warp maxima of |2^s V dV| (every warp of the form's CTA)
    uint64_t full[C::kBufs];   // producers of buffer b arrived (kGroupThreads arrivals)
    uint64_t empty[C::kBufs];  // MMAs reading buffer b completed (tcgen05.commit)
    uint64_t done;      // all MMAs of the pass completed
    uint32_t tmem;
    int work;
    int abort;
    float scale_inv;
};

static_assert(sizeof(TcSmem<false>) + 1024 <= 232448, "shared memory of the H^V kernel exceeds 227 KB");
static_assert(sizeof(TcSmem<true>) + 1024 <= 232448, "shared memory of the exact H^V kernel exceeds 227 KB");
__host__ __device__ constexpr int pair_index(int a1, int a2) { return a2 * (a2 + 1) / 2 + a1; }  // a1 <= a2

// Offset (bytes) of element (row r, point q) of one piece: core matrix
// (r / 8, q / 8) at ((r / 8) * 2 + q / 8) * 128, inside it row r % 8 of 16 bytes.
__device__ __forceinline__ int piece_off(int r, int q) {
    return (((r >> 3) * (kTcChunk / 8) + (q >> 3)) << 7) + ((r & 7) << 4) + ((q & 7) << 1);
}

template <typename H16> struct Conv;
template <> struct Conv<__half> {
    static __device__ __forceinline__ void split(float x, unsigned short& hi, unsigned short& lo) {
        __half h = __float2half_rn(x);
        __half l = __float2half_rn(x - __half2float(h));
        hi = __half_as_ushort(h);
        lo = __half_as_ushort(l);
    }
    static constexpr int bf16 = 0;
};
template <> struct Conv<__nv_bfloat16> {
    static __device__ __forceinline__ void split(float x, unsigned short& hi, unsigned short& lo) {
        __nv_bfloat16 h = __float2bfloat16_rn(x);
        __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
        hi = __bfloat16_as_ushort(h);
        lo = __bfloat16_as_ushort(l);
    }
    static constexpr int bf16 = 1;
};

// The same splits for two values at once (the two points of a producer item), packed
// as the 32-bit word stored for them: element of the first value in the low half.
__device__ __forceinline__ uint32_t h2_bits(__half2 h) { return *reinterpret_cast<uint32_t*>(&h); }
__device__ __forceinline__ uint32_t b2_bits(__nv_bfloat162 h) { return *reinterpret_cast<uint32_t*>(&h); }
template <typename H16> struct Conv2;
template <> struct Conv2<__half> {
    static __device__ __forceinline__ void split(float x0, float x1, uint32_t& hi, uint32_t& lo) {
        const __half2 h = __floats2half2_rn(x0, x1);
        const float2 f = __half22float2(h);
        hi = h2_bits(h);
        lo = h2_bits(__floats2half2_rn(x0 - f.x, x1 - f.y));
    }
};
template <> struct Conv2<__nv_bfloat16> {
    static __device__ __forceinline__ void split(float x0, float x1, uint32_t& hi, uint32_t& lo) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
        const float2 f = __bfloat1622float2(h);
        hi = b2_bits(h);
        lo = b2_bits(__floats2bfloat162_rn(x0 - f.x, x1 - f.y));
    }
};
// Exact form for two values: s = n + l1 + l2 (see fix_split3), packed pairs.
__device__ __forceinline__ void fix_split3_2(float s0, float s1, uint32_t& n, uint32_t& l1, uint32_t& l2) {
    const float n0 = rintf(s0), n1 = rintf(s1);
    const float r0 = s0 - n0, r1 = s1 - n1;
    const __half2 h = __floats2half2_rn(r0, r1);
    const float2 f = __half22float2(h);
    n = h2_bits(__floats2half2_rn(n0, n1));
    l1 = h2_bits(h);
    l2 = h2_bits(__floats2half2_rn(r0 - f.x, r1 - f.y));
}

// Exact form: s = n + l1 + l2 with n = rint(s) (|s| <= 128, so n is exact in
// fp16), l1 = fp16(s - n), l2 = fp16(s - n - l1) (both differences exact in FP32).
__device__ __forceinline__ void fix_split3(float s, unsigned short& n16, unsigned short& l1, unsigned short& l2) {
    const float n = rintf(s);
    const float r = s - n;
    const __half h1 = __float2half_rn(r);
    n16 = __half_as_ushort(__float2half_rn(n));
    l1 = __half_as_ushort(h1);
    l2 = __half_as_ushort(__float2half_rn(r - __half2float(h1)));
}
__device__ __forceinline__ float exp2i(int e) { return __int_as_float((127 + e) << 23); }  // 2^e, |e| < 127

// Exact FP32 -> FP64 widening with integer operations (sign, exponent rebias by
// 1023 - 127 = 896, mantissa shifted into place); zero and FP32 subnormals give 0.
__device__ __forceinline__ double f2d_exact(float x) {
    const uint32_t u = __float_as_uint(x);
    const uint32_t e = (u >> 23) & 0xffu;
    if (e == 0u) return 0.0;
    const uint32_t hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u >> 3) & 0xfffffu);
    return __hiloint2double((int)hi, (int)(u << 29));
}

// kMulti: the work queue spans the bricks of many cells (a batch, MultiArgs);
// the problem, V and H of an item come from its cell's CellJob.
template <typename H16, bool kExact, bool kMulti>
__global__ void __launch_bounds__(TcCfg<kExact>::kThreads, 1) k_vlocal_tc(const __grid_constant__ TcArgs A, const double* V_in, double* H_in,
                                                                const __grid_constant__ MultiArgs M) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TcSmem<kExact>& S = *reinterpret_cast<TcSmem<kExact>*>(smem_raw);
    using C = TcCfg<kExact>;
    constexpr int kPassCols = C::kPassCols;
    constexpr int kTcThreads = C::kThreads;
    constexpr int kAP = C::kAPieceBytes, kBP = C::kBPieceBytes, kBOff = C::kBOff;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const Problem* Pc = &A.P;  // problem, V and H of the current item
    const double* Vc = V_in;
    double* Hc = H_in;
    int cur_cell = -1;
    // per-cell tables: species (shared memory copy) and the in-brick point offsets (the same
    // for every brick of a cell): FP64, rounded once to FP32
    auto cell_setup = [&](const Problem& Q) {
        if (tid < Q.n_species) species_fast_from(Q.sp[tid], S.spf[tid]);
        const GridDev& gq = Q.g;
        for (int p = tid; p < gq.bpad && p < C::kPts; p += kTcThreads) {
            const int l2 = p % gq.B[2], l1 = (p / gq.B[2]) % gq.B[1], l0 = p / (gq.B[2] * gq.B[1]);
            float4 q4;
            q4.x = (float)(l0 * gq.step[0][0] + l1 * gq.step[1][0] + l2 * gq.step[2][0]);
            q4.y = (float)(l0 * gq.step[0][1] + l1 * gq.step[1][1] + l2 * gq.step[2][1]);
            q4.z = (float)(l0 * gq.step[0][2] + l1 * gq.step[1][2] + l2 * gq.step[2][2]);
            q4.w = 0.f;
            S.pt[p] = q4;
        }
    };

    if (warp == 0) {
        tc::tmem_alloc(&S.tmem, 512);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int b = 0; b < C::kBufs; ++b) {
            tc::mbar_init(&S.full[b], C::kGroupThreads);
            tc::mbar_init(&S.empty[b], 1);
        }
        tc::mbar_init(&S.done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        S.abort = 0;
    }
    if (!kMulti) cell_setup(A.P);
    for (int r = tid; r < C::kRows; r += kTcThreads) {
        S.rowtab[r] = (unsigned short)((((r >> 3) * (kTcChunk / 8)) << 7) + ((r & 7) << 4));
        if (!kExact) S.rowtabB[r] = S.rowtab[r];  // B holds every row
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = S.tmem;
    // completed phases of each barrier (every thread that waits on a barrier keeps its count)
    // chunks of every pass so far (every thread keeps the same count): the chunk with global index G
    // uses buffer G % kBufs, whose barriers' phase G / kBufs belongs to it
    uint32_t gchunk = 0;
    uint32_t dones = 0;
    const bool issuer_warp = warp == C::kProdWarps;
    const int grp = warp / C::kGroupWarps;  // producer group of warps 0 .. kProdWarps - 1
    const int lt = tid - grp * C::kGroupThreads;

    for (;;) {
        if (tid == 0) S.work = atomicAdd(A.counter, 1);
        __syncthreads();
        const int w = S.work;
        if (w >= (kMulti ? M.n_items : A.P.n_work) || S.abort) break;
        int wl = w;
        if (kMulti) {
            const int c = M.item_cell[w];
            const CellJob& J = M.jobs[c];
            wl = w - J.item0;
            if (c != cur_cell) {  // uniform: every thread read the same item
                cur_cell = c;
                Pc = &J.P;
                Vc = J.V;
                Hc = J.H;
                cell_setup(J.P);
                __syncthreads();
            }
        }
        const Problem& P = *Pc;
        const GridDev& g = P.g;
        const double* V = Vc;
        double* H = Hc;
        const float2* knot2 = P.knot32;
        const int brick = P.work[wl];
        int b0, b1, b2;
        brick_coords(g, brick, b0, b1, b2);
        const int64_t s0 = P.brick_start[brick];
        const int na = (int)(P.brick_start[brick + 1] - s0);
        // ---- brick tables
        const double ox = b0 * g.B[0] * g.step[0][0] + b1 * g.B[1] * g.step[1][0] + b2 * g.B[2] * g.step[2][0];
        const double oy = b0 * g.B[0] * g.step[0][1] + b1 * g.B[1] * g.step[1][1] + b2 * g.B[2] * g.step[2][1];
        const double oz = b0 * g.B[0] * g.step[0][2] + b1 * g.B[1] * g.step[1][2] + b2 * g.B[2] * g.step[2][2];
        for (int i = tid; i < na; i += kTcThreads) {
            const ExtAtom X = P.ext[P.brick_atoms[s0 + i]];
            TcAtom& a = S.at[i];
            const double c[3] = {ox - X.p[0], oy - X.p[1], oz - X.p[2]};
            for (int k = 0; k < 3; ++k) {
                a.c_hi[k] = (float)c[k];
                a.c_lo[k] = (float)(c[k] - (double)a.c_hi[k]);
            }
            a.I = X.atom;
            a.sp = X.species;
            a.nw = P.sp[X.species].n_orb;
            a.t[0] = X.t[0]; a.t[1] = X.t[1]; a.t[2] = X.t[2];
        }
        // in-brick point offsets, weights and their power-of-two scale (max |2^s W| in [0.5, 1))
        float wmax = 0.f;
        for (int p = tid; p < g.bpad; p += kTcThreads) {
            int g0, g1, g2;
            float wv = 0.f;
            if (brick_point(g, b0, b1, b2, p, g0, g1, g2))
                wv = (float)(ld_stream_f64(V + ((int64_t)g0 * g.n[1] + g1) * g.n[2] + g2) * g.dV);
            S.pt[p].w = p < g.bpts ? wv : 0.f;
            wmax = fmaxf(wmax, fabsf(wv));
        }
        for (int o = 16; o > 0; o >>= 1) wmax = fmaxf(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
        if (lane == 0) S.wmax[warp] = wmax;
        __syncthreads();
        if (tid == 0) {
            float m = 0.f;
            for (int k = 0; k < kTcThreads / 32; ++k) m = fmaxf(m, S.wmax[k]);
            int e = 0;
            if (m > 0.f) frexpf(m, &e);  // m = f 2^e, f in [0.5, 1)
            S.scale_inv = ldexpf(1.f, e);
            int off = 0;  // first row of each image (the row tables are filled by all threads below)
            for (int i = 0; i < na; ++i) {
                S.at[i].off = off;
                off += S.at[i].nw;
            }
            // row tiles of 128; tile i accumulates columns [128 i, ncol), cut into segments
            // so that each pass holds at most kPassCols output columns (512 TMEM columns)
            const int ncol = (off + 15) & ~15;
            const int nt = (off + 127) >> 7;
            int np = 0, used = 0, ns = 0;
            S.pass_first[0] = 0;
            for (int i = 0; i < nt; ++i) {
                int c = 128 * i;
                while (c < ncol) {
                    if (used == kPassCols) { S.pass_first[++np] = ns; used = 0; }
                    const int wdt = min(ncol - c, kPassCols - used);
                    S.seg_tile[ns] = (unsigned char)i;
                    S.seg_c0[ns] = (short)c;
                    S.seg_c1[ns] = (short)(c + wdt);
                    S.seg_tcol[ns] = (short)used;
                    ++ns;
                    used += wdt;
                    c += wdt;
                }
            }
            S.pass_first[++np] = ns;
            S.npass = np;
            S.nrow = off;
            S.ncol = ncol;
        }
        __syncthreads();
        const float wscale = 1.f / S.scale_inv;
        for (int p = tid; p < g.bpad; p += kTcThreads) S.pt[p].w *= wscale;
        const int nrow = S.nrow, npass = S.npass;
        // row tables: image and orbital of every row; exact form: the row's quantum 2^qeu (FP32)
        // and, in FP64, times the harmonic normalisation unless k_norm_h applies it afterwards
        for (int e = tid; e < na * kMaxNw; e += kTcThreads) {
            const int i = e / kMaxNw, o = e - i * kMaxNw;
            if (o >= S.at[i].nw) continue;
            const int r = S.at[i].off + o;
            S.row_atom[r] = (unsigned char)i;
            S.row_mu[r] = (unsigned char)o;
            if (kExact) {
                const SpeciesFast& sf = S.spf[S.at[i].sp];
                const SpeciesDev& sd = P.sp[S.at[i].sp];
                S.row_s[r] = (A.norm_after ? 1.0 : ylm_norm(sd.orb_l[o], sd.orb_m[o])) * (double)exp2i(sf.qeu[o]);
                S.row_f[r] = exp2i(sf.qeu[o]);
            }
        }
        // pair table of the brick (built once per geometry): block (I_a1, I_a2, t_a2 - t_a1), a1 <= a2
        {
            const int32_t* pt = P.pairs + P.pair_start[brick];
            for (int q = tid; q < na * na; q += kTcThreads) {
                const int a1 = q / na, a2 = q - a1 * na;
                if (a1 <= a2) S.pairblk[pair_index(a1, a2)] = ld_stream_s32(pt + q);
            }
        }
        // three-product form: zero the padding rows [nrow, round128(nrow)) of the chunk buffers
        // (A and B hold every row); the exact form zeroes its padding rows per pass
        const int nrow128 = (nrow + 127) & ~127;
        if (!kExact)
            for (int b = 0; b < C::kBufs; ++b)
                for (int e = tid; e < (nrow128 - nrow) * kTcChunk; e += kTcThreads) {
                    const int r = nrow + e / kTcChunk, q = e % kTcChunk;
                    const int o = piece_off(r, q);
                    for (int pc = 0; pc < C::kPieces; ++pc) {
                        *reinterpret_cast<unsigned short*>(&S.buf[b][kBOff + pc * kBP + o]) = 0;
                        *reinterpret_cast<unsigned short*>(&S.buf[b][pc * kAP + o]) = 0;
                    }
                }
        __syncthreads();

        const int nchunks = g.bpad / kTcChunk;
        for (int pass = 0; pass < npass && !S.abort; ++pass) {
            const int s0p = S.pass_first[pass], s1p = S.pass_first[pass + 1];
            const int t_lo = 128 * S.seg_tile[s0p], t_hi = 128 * (S.seg_tile[s1p - 1] + 1);
            // exact form: A pieces hold rows [a_lo, a_hi) of this pass's row tiles (<= 384 rows)
            const int a_lo = kExact ? t_lo : 0;
            const int a_hi = kExact ? t_hi : C::kRows;
            // the pass reads A rows of its row tiles [t_lo, t_hi) and B rows of its segments'
            // column ranges; only atom images with rows there are evaluated (listed by warp 0)
            if (warp == 0) {
                uint64_t m = 0;
                for (int h2 = 0; h2 < 2; ++h2) {
                    const int a = lane + 32 * h2;
                    bool nd = false;
                    if (a < na) {
                        const int r0 = S.at[a].off, r1 = r0 + S.at[a].nw;
                        nd = r0 < t_hi && r1 > t_lo;
                        for (int sg = s0p; sg < s1p; ++sg) nd = nd || (r0 < S.seg_c1[sg] && r1 > S.seg_c0[sg]);
                    }
                    m |= (uint64_t)__ballot_sync(0xffffffffu, nd) << (32 * h2);
                }
                for (int h2 = 0; h2 < 2; ++h2) {
                    const int a = lane + 32 * h2;
                    if (a < na && (m >> a & 1ull)) S.need_list[__popcll(m & ((1ull << a) - 1ull))] = (unsigned char)a;
                }
                if (lane == 0) S.n_need = __popcll(m);
            }
            if (kExact && tid == 32) {
                // packed B rows of this pass: the 16-column groups its segments read, in order
                const int ng = S.ncol >> 4;
                for (int gq = 0; gq < ng; ++gq) S.grp_pos[gq] = -1;
                for (int sg = s0p; sg < s1p; ++sg)
                    for (int gq = S.seg_c0[sg] >> 4; gq < (S.seg_c1[sg] >> 4); ++gq) S.grp_pos[gq] = 0;
                int pos = 0;
                for (int gq = 0; gq < ng; ++gq)
                    if (S.grp_pos[gq] >= 0) S.grp_pos[gq] = (short)(pos++);
            }
            if (kExact) {
                __syncthreads();
                // B row offsets of the pass (rows it does not read go to the spare group 256..271)
                for (int r = tid; r < S.ncol; r += kTcThreads) {
                    const int gp = S.grp_pos[r >> 4];
                    const int pr = gp >= 0 ? (gp << 4) + (r & 15) : 256 + (r & 15);
                    S.rowtabB[r] = (unsigned short)((((pr >> 3) * (kTcChunk / 8)) << 7) + ((pr & 7) << 4));
                }
                __syncthreads();
                // zero A rows [max(nrow, a_lo), a_hi) and the packed B rows of the padding rows
                // [nrow, ncol) in every buffer (they may hold rows of the previous pass; every MMA of
                // that pass has completed); no producer writes them in this pass
                const int z0 = max(nrow, a_lo);
                for (int b = 0; b < C::kBufs; ++b) {
                    for (int e = tid; e < (a_hi - z0) * kTcChunk; e += kTcThreads) {
                        const int r = z0 - a_lo + e / kTcChunk, q = e % kTcChunk;
                        const int o = piece_off(r, q);
                        for (int pc = 0; pc < C::kPieces; ++pc) *reinterpret_cast<unsigned short*>(&S.buf[b][pc * kAP + o]) = 0;
                    }
                    for (int e = tid; e < (S.ncol - nrow) * kTcChunk; e += kTcThreads) {
                        const int r = nrow + e / kTcChunk, q = e % kTcChunk;
                        if (S.grp_pos[r >> 4] < 0) continue;
                        const int o = S.rowtabB[r] + ((q >> 3) << 7) + ((q & 7) << 1);
                        for (int pc = 0; pc < C::kPieces; ++pc)
                            *reinterpret_cast<unsigned short*>(&S.buf[b][kBOff + pc * kBP + o]) = 0;
                    }
                }
            }
            __syncthreads();
            if (!issuer_warp) {
                // ---- producers: group g fills chunks c = g, g + kGroups, ... of the pass; chunk c
                //      (global index G) goes to buffer G % kBufs once the MMAs of chunk G - kBufs
                //      have read it
                for (int c = grp; c < nchunks; c += C::kGroups) {
                    const uint32_t G = gchunk + (uint32_t)c;
                    const int b = (int)(G % C::kBufs);
                    unsigned char* buf = S.buf[b];
                    // the buffer is free once the MMAs of chunk G - kBufs completed; a thread waits
                    // for that only before its first store (its first item's knot loads are then in
                    // flight) or before it arrives
                    bool freed = G < (uint32_t)C::kBufs;
                    auto ensure_free = [&]() {
                        if (freed) return;
                        if (!S.abort && !tc::mbar_wait(&S.empty[b], ((G / C::kBufs) - 1) & 1, A.wait_limit))
                            atomicOr(&S.abort, 1);
                        freed = true;
                    };
                    // orbital values at the chunk's points, two points per item, for the atom
                    // images of need_list: 8 items (point pairs) per image.  Items of the full
                    // blocks of 8 images: bits [1:0] point pair within a half chunk, [4:2] list
                    // entry within the block, [5] half chunk, [6..] block; so a warp stores 8
                    // atoms (distinct rows mod 8) x 4 point pairs of the same 16-byte row
                    // segment half: 32 different banks.  The r < 8 images of the last block take
                    // items j = qp r + (k mod 8) (at most two-way bank conflicts).
                    const int n_need = S.n_need;
                    const int n_full = (n_need >> 3) << 6;
                    const int r_last = n_need & 7;
                    const int n_items = 8 * n_need;
                    for (int item = lt; item < n_items; item += C::kGroupThreads) {
                        int k, qp;
                        if (item < n_full) {
                            k = ((item >> 6) << 3) | ((item >> 2) & 7);
                            qp = (((item >> 5) & 1) << 2) | (item & 3);
                        } else {
                            const int j = item - n_full;
                            qp = j / r_last;
                            k = (n_full >> 3) + (j - qp * r_last);
                        }
                        const TcAtom& X = S.at[S.need_list[k]];
                        const int q = 2 * qp;
                        const int p = c * kTcChunk + q;
                        const float4 u4 = S.pt[p], v4 = S.pt[p + 1];
                        const float ax = (X.c_hi[0] + u4.x) + X.c_lo[0];
                        const float ay = (X.c_hi[1] + u4.y) + X.c_lo[1];
                        const float az = (X.c_hi[2] + u4.z) + X.c_lo[2];
                        const float bx = (X.c_hi[0] + v4.x) + X.c_lo[0];
                        const float by = (X.c_hi[1] + v4.y) + X.c_lo[1];
                        const float bz = (X.c_hi[2] + v4.z) + X.c_lo[2];
                        const float wa = u4.w, wb = v4.w;  // zero at padding points
                        const int qoff = ((q >> 3) << 7) + ((q & 7) << 1);
                        const int rbase = X.off;
                        const SpeciesFast& sf = S.spf[X.sp];
                        auto put2 = [&](int o, float va, float vb) {
                            const int r = rbase + o;
                            const int offB = kBOff + S.rowtabB[r] + qoff;
                            auto st32 = [&](int off, uint32_t x) { *reinterpret_cast<uint32_t*>(&buf[off]) = x; };
                            if (kExact) {
                                const float qi = exp2i(-sf.qeu[o]);  // unnormalised orbital values
                                va *= qi;
                                vb *= qi;
                                uint32_t n, p, q;
                                if (r >= a_lo && r < a_hi) {
                                    const int offA = S.rowtab[r - a_lo] + qoff;
                                    fix_split3_2(va * wa, vb * wb, n, p, q);
                                    st32(offA, n); st32(offA + kAP, p); st32(offA + 2 * kAP, q);
                                }
                                fix_split3_2(va, vb, n, p, q);
                                st32(offB, n); st32(offB + kBP, p); st32(offB + 2 * kBP, q);
                            } else {
                                uint32_t ah, al, bh, bl;
                                Conv2<H16>::split(va * wa, vb * wb, ah, al);
                                Conv2<H16>::split(va, vb, bh, bl);
                                const int offA = S.rowtab[r] + qoff;
                                st32(offA, ah); st32(offA + kAP, al);
                                st32(offB, bh); st32(offB + kBP, bl);
                            }
                        };
                        if (!orbitals_fast2<!kExact>(sf, knot2, ax, ay, az, bx, by, bz, put2, ensure_free)) {
                            ensure_free();
                            for (int o = 0; o < X.nw; ++o) {
                                const int r = rbase + o;
                                const int offB = kBOff + S.rowtabB[r] + qoff;
                                const bool inA = r >= a_lo && r < a_hi;
                                const int offA = inA ? S.rowtab[r - a_lo] + qoff : 0;
                                for (int pc = 0; pc < C::kPieces; ++pc) {
                                    *reinterpret_cast<uint32_t*>(&buf[offB + pc * kBP]) = 0u;
                                    if (inA) *reinterpret_cast<uint32_t*>(&buf[offA + pc * kAP]) = 0u;
                                }
                            }
                        }
                    }
                    ensure_free();
                    tc::fence_async_smem();
                    tc::mbar_arrive(&S.full[b]);
                }
            } else if (lane == 0) {
                // ---- issuer: one thread waits for each chunk, issues its MMAs and commits
                const uint32_t lbo = 128, sbo = (kTcChunk / 8) * 128;
                for (int c = 0; c < nchunks; ++c) {
                    const uint32_t G = gchunk + (uint32_t)c;
                    const int b = (int)(G % C::kBufs);
                    if (!S.abort && !tc::mbar_wait(&S.full[b], (G / C::kBufs) & 1, A.wait_limit)) atomicOr(&S.abort, 1);
                    tc::fence_after_sync();
                    const uint32_t base = tc::smem_u32(S.buf[b]);
                    // K-major operands: LBO = distance of K-adjacent core matrices (128 B),
                    // SBO = distance of row-adjacent core matrices (2 * 128 B)
                    if (!S.abort) {
                        for (int sg = s0p; sg < s1p; ++sg) {
                            const int i = S.seg_tile[sg], c_end = S.seg_c1[sg];
                            const uint32_t arow = (uint32_t)((128 * i - a_lo) >> 3) * sbo;  // tile i in the A pieces
                            const uint32_t pa0 = base + arow;
                            const uint32_t pa1 = base + kAP + arow;
                            const uint32_t pa2 = base + 2 * kAP + arow;  // exact form
                            for (int c0 = S.seg_c0[sg]; c0 < c_end; c0 += 256) {
                                const int nn = min(256, c_end - c0);
                                const uint32_t idesc = tc::idesc_f16(128, nn, Conv<H16>::bf16, 0, 0);
                                // B rows of columns [c0, c0 + nn): packed position in the exact form
                                const int brow = kExact ? (S.grp_pos[c0 >> 4] << 4) : c0;
                                const uint32_t pb0 = base + kBOff + (uint32_t)(brow >> 3) * sbo;
                                const uint32_t pb1 = pb0 + kBP;
                                const uint32_t pb2 = pb0 + 2 * kBP;  // exact form
                                const uint32_t d = tmem + (uint32_t)(S.seg_tcol[sg] + c0 - S.seg_c0[sg]);
                                tc::mma_f16(d, tc::smem_desc(pa0, lbo, sbo), tc::smem_desc(pb0, lbo, sbo), idesc, c > 0 ? 1u : 0u);
                                if (kExact) {
                                    // integer products alone in d; the cross terms in d + 256
                                    const uint32_t d1 = d + 256;
                                    tc::mma_f16(d1, tc::smem_desc(pa0, lbo, sbo), tc::smem_desc(pb1, lbo, sbo), idesc, c > 0 ? 1u : 0u);
                                    tc::mma_f16(d1, tc::smem_desc(pa1, lbo, sbo), tc::smem_desc(pb0, lbo, sbo), idesc, 1u);
                                    tc::mma_f16(d1, tc::smem_desc(pa1, lbo, sbo), tc::smem_desc(pb1, lbo, sbo), idesc, 1u);
                                    tc::mma_f16(d1, tc::smem_desc(pa0, lbo, sbo), tc::smem_desc(pb2, lbo, sbo), idesc, 1u);
                                    tc::mma_f16(d1, tc::smem_desc(pa2, lbo, sbo), tc::smem_desc(pb0, lbo, sbo), idesc, 1u);
                                } else {
                                    tc::mma_f16(d, tc::smem_desc(pa0, lbo, sbo), tc::smem_desc(pb1, lbo, sbo), idesc, 1u);
                                    tc::mma_f16(d, tc::smem_desc(pa1, lbo, sbo), tc::smem_desc(pb0, lbo, sbo), idesc, 1u);
                                }
                            }
                        }
                    }
                    tc::mma_commit(&S.empty[b]);
                }
                tc::mma_commit(&S.done);
            }
            // ---- every thread: all MMAs of the pass complete.  Waited for even after an abort
            //      (the issuer commits `done` at the end of every pass), so that the phases of
            //      `done` stay in step and no MMA of the pass is in flight afterwards.
            __syncwarp();
            if (!tc::mbar_wait(&S.done, dones & 1, kDrainPolls)) atomicOr(&S.abort, 1);
            dones += 1;
            gchunk += (uint32_t)nchunks;
            tc::fence_after_sync();
            __syncthreads();
            if (S.abort) break;
            // ---- epilogue: warps 0-15; lanes = rows (lane group warp & 3), the four warps of a
            //      lane group take every fourth 16-column group
            if (warp < 16) {
                const int lane_base = (warp & 3) * 32;
                const float sinv = S.scale_inv;
                for (int sg = s0p; sg < s1p; ++sg) {
                    const int i = S.seg_tile[sg], cs0 = S.seg_c0[sg];
                    const int r = 128 * i + lane_base + lane;
                    const bool rvalid = r < nrow;
                    const int a1 = rvalid ? S.row_atom[r] : 0;
                    const int mu = rvalid ? S.row_mu[r] : 0;
                    const int ngrp = (S.seg_c1[sg] - cs0) >> 4;
                    const double qr = kExact && rvalid ? S.row_s[r] * (double)sinv : (double)sinv;
                    const float qrf = kExact && rvalid ? S.row_f[r] * sinv : sinv;  // powers of two
                    for (int gq = warp >> 2; gq < ngrp; gq += 4) {
                        float v[16], v1[16];
                        const uint32_t ta = tmem + ((uint32_t)lane_base << 16) + (uint32_t)(S.seg_tcol[sg] + 16 * gq);
                        tc::tmem_ld16(ta, v);
                        if (kExact) tc::tmem_ld16(ta + 256, v1);
                        if (!rvalid) continue;
                        // the block of (a1, a2) and its size change only where a2 does (about twice
                        // in 16 columns): looked up once per image
                        int a2c = -1, blk = -1, nw2 = 0;
                        int64_t off = 0;
#pragma unroll
                        for (int jj = 0; jj < 16; ++jj) {
                            const int col = cs0 + 16 * gq + jj;
                            if (col >= nrow) continue;
                            const int a2 = S.row_atom[col];
                            if (a2 != a2c) {
                                a2c = a2;
                                blk = a1 <= a2 ? S.pairblk[pair_index(a1, a2)] : -1;
                                off = blk >= 0 ? __ldg(P.offsets + blk) : 0;
                                nw2 = S.at[a2].nw;
                            }
                            if (blk < 0) continue;  // a1 > a2, or no block
                            const int nu = S.row_mu[col];
                            if (a1 == a2 && r > col) continue;  // same image: symmetric block, keep r <= col
                            auto emit = [&](double x) {
                                atomicAdd(H + off + mu * nw2 + nu, x);
                                if (a1 == a2 && mu != nu) atomicAdd(H + off + nu * nw2 + mu, x);
                            };
                            // Three-product form: power-of-two scale (exact), widened to FP64 by bit
                            // arithmetic (no FP64 pipe).  Exact form with norm_after: the factors are a
                            // power of two p2; both accumulators are scaled exactly, widened by bit
                            // arithmetic and added in FP64 (one DADD, one atomic; two FP32 values whose
                            // exponents differ by at most 28 add exactly in FP64, else the sum rounds at
                            // 2^-53 of the larger).  Exact form accumulating into H: FP64 row and column
                            // factors (normalisation x quantum).
                            if (!kExact) {
                                emit(f2d_exact(v[jj] * sinv));
                            } else if (A.norm_after) {
                                const float p2 = qrf * S.row_f[col];
                                emit(f2d_exact(v[jj] * p2) + f2d_exact(v1[jj] * p2));
                            } else {
                                emit(((double)v[jj] + (double)v1[jj]) * (qr * S.row_s[col]));
                            }
                        }
                    }
                }
            }
            tc::fence_before_sync();
            __syncthreads();
        }
        __syncthreads();
    }
    // ---- teardown: one more commit and a bounded wait, so that no MMA is in flight when
    //      tensor memory is released (every pass already waited on `done` unless it aborted)
    __syncthreads();
    if (issuer_warp && lane == 0) tc::mma_commit(&S.done);
    (void)tc::mbar_wait(&S.done, dones & 1, kDrainPolls);
    if (S.abort && tid == 0) atomicOr(Pc->err, kErrTimeout);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

template <bool kExact> size_t tc_smem_bytes() { return sizeof(TcSmem<kExact>) + 1024; }
template <bool kExact> constexpr int tc_threads() { return TcCfg<kExact>::kThreads; }

// Exact form: multiply every canonical H block by the harmonic normalisation of
// its row and column orbitals (FP64, once per element rather than once per brick).
__global__ void k_norm_h(Problem P, const int* atom_sp, int64_t n_blocks, double* H) {
    const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (b >= n_blocks) return;
    const int32_t* k = P.blocks + 5 * b;
    const int I = k[0], J = k[1];
    const bool canon = (I < J) || (I == J && (k[2] > 0 || (k[2] == 0 && (k[3] > 0 || (k[3] == 0 && k[4] >= 0)))));
    if (!canon) return;
    const SpeciesDev& si = P.sp[atom_sp[I]];
    const SpeciesDev& sj = P.sp[atom_sp[J]];
    const int nI = si.n_orb, nJ = sj.n_orb;
    double* Hb = H + P.offsets[b];
    for (int e = lane; e < nI * nJ; e += 32) {
        const int mu = e / nJ, nu = e - mu * nJ;
        Hb[e] *= ylm_norm(si.orb_l[mu], si.orb_m[mu]) * ylm_norm(sj.orb_l[nu], sj.orb_m[nu]);
    }
}

// form: 0 = fp16x3, 1 = bf16x3, 2 = fp16x4 (exact leading term)
gint_status tc_vlocal_check(const gint_handle* h, int form) {
    const bool exact = form == 2;
    const int max_rows = exact ? TcCfg<true>::kRows : TcCfg<false>::kRows;
    const int max_pts = exact ? TcCfg<true>::kPts : TcCfg<false>::kPts;
    if (h->max_brick_orb > max_rows || h->max_brick_atoms > kTcMaxAtoms || h->grid.bpad > max_pts ||
        h->grid.bpad % kTcChunk != 0 || h->n_species > kTcMaxSpecies) {
        set_error("tensor-core form needs <= %d orbitals, <= %d atom images and <= %d points per brick and "
                  "<= %d species (have %d, %d, %d, %d); use smaller bricks", max_rows, kTcMaxAtoms, max_pts,
                  kTcMaxSpecies, h->max_brick_orb, h->max_brick_atoms, h->grid.bpad, h->n_species);
        return GINT_ERR_UNSUPPORTED;
    }
    return GINT_OK;
}

gint_status tc_vlocal(gint_handle* h, int form, const double* V, double* H, int accumulate, cudaStream_t st) {
    gint_status s = tc_vlocal_check(h, form);
    if (s != GINT_OK || h->n_work == 0) return s;
    const bool exact = form == 2;
    TcArgs A;
    A.norm_after = exact && !accumulate ? 1 : 0;
    A.P = h->problem();
    A.counter = h->d_err + 2;
    A.wait_limit = wait_polls(h);
    GINT_CUDA_TRY(cudaMemsetAsync(A.counter, 0, sizeof(int), st));
    const size_t smem = exact ? tc_smem_bytes<true>() : tc_smem_bytes<false>();
#define GINT_LAUNCH_VL(H16, X)                                                                                 \
    do {                                                                                                       \
        GINT_CUDA_TRY(cudaFuncSetAttribute(k_vlocal_tc<H16, X, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                           (int)smem));                                                        \
        k_vlocal_tc<H16, X, false><<<h->sm_count, tc_threads<X>(), smem, st>>>(A, V, H, MultiArgs{});              \
    } while (0)
    if (form == 1) GINT_LAUNCH_VL(__nv_bfloat16, false);
    else if (form == 2) GINT_LAUNCH_VL(__half, true);
    else GINT_LAUNCH_VL(__half, false);
#undef GINT_LAUNCH_VL
    GINT_CUDA_TRY(cudaGetLastError());
    if (A.norm_after && h->n_blocks > 0) {
        k_norm_h<<<(unsigned)((h->n_blocks * 32 + 255) / 256), 256, 0, st>>>(A.P, h->d_atom_sp, h->n_blocks, H);
        GINT_CUDA_TRY(cudaGetLastError());
    }
    return GINT_OK;
}

// Exact form, H not accumulated into: the FP64 harmonic normalisation of a cell's H.
gint_status launch_norm_h(gint_handle* h, double* H, cudaStream_t st) {
    if (h->n_blocks == 0) return GINT_OK;
    k_norm_h<<<(unsigned)((h->n_blocks * 32 + 255) / 256), 256, 0, st>>>(h->problem(), h->d_atom_sp, h->n_blocks, H);
    GINT_CUDA_TRY(cudaGetLastError());
    return GINT_OK;
}

// One launch over the (cell, brick) queue of a batch: every cell's H (zeroed by the
// caller; the exact form leaves the normalisation to launch_norm_h).  The cells must
// pass tc_vlocal_check for `form`.
gint_status tc_vlocal_multi(int form, const MultiArgs& M, int* counter, int sm_count, cudaStream_t st) {
    if (M.n_items == 0) return GINT_OK;
    TcArgs A;
    memset(&A, 0, sizeof(A));
    A.counter = counter;
    A.wait_limit = kDefaultWaitPolls;
    A.norm_after = form == 2 ? 1 : 0;
    GINT_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(int), st));
    const size_t smem = form == 2 ? tc_smem_bytes<true>() : tc_smem_bytes<false>();
#define GINT_LAUNCH_VLM(H16, X)                                                                                \
    do {                                                                                                       \
        GINT_CUDA_TRY(cudaFuncSetAttribute(k_vlocal_tc<H16, X, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                           (int)smem));                                                        \
        k_vlocal_tc<H16, X, true><<<sm_count, tc_threads<X>(), smem, st>>>(A, nullptr, nullptr, M);                 \
    } while (0)
    if (form == 1) GINT_LAUNCH_VLM(__nv_bfloat16, false);
    else if (form == 2) GINT_LAUNCH_VLM(__half, true);
    else GINT_LAUNCH_VLM(__half, false);
#undef GINT_LAUNCH_VLM
    GINT_CUDA_TRY(cudaGetLastError());
    return GINT_OK;
}

}  // namespace gint
