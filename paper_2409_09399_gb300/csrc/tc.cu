// tc.cu -- tensor-core (tcgen05) form of the H^V grid integral (Eq. 2).
//
// Per brick of grid points the contraction H_b = Psi^T diag(W) Psi (Psi: brick
// points x brick orbitals, W_p = V_p dV) is a dense small GEMM (Section 2.2:
// "a batch of points turns vector products into a matrix product").  Here it
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
// The atom-to-brick displacement is taken in FP64 once per (brick, atom) and
// split into two FP32 words; in-brick offsets are FP32.
#include <algorithm>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fast_orb.cuh"
#include "gint_impl.cuh"
#include "tc_ptx.cuh"

namespace gint {

constexpr int kTcThreads = 256;
constexpr int kTcChunk = 16;        // points per K chunk (one MMA K step)
constexpr int kTcMaxRows = 640;     // padded brick orbitals (5 tiles of 128)
constexpr int kTcMaxAtoms = 64;     // atom images per brick
constexpr int kTcMaxPairsPerPass = 4;
constexpr int kTcMaxPts = 1024;     // points per brick on this path
constexpr int kTcMaxSpecies = 8;
constexpr long kWaitLimit = 1L << 26;  // bounded mbarrier polls

// bytes of one 16-bit operand piece for one chunk: rows x 16 points x 2 B
constexpr int kPieceBytes = kTcMaxRows * kTcChunk * 2;
constexpr int kBufBytes = 4 * kPieceBytes;  // A_hi, A_lo, B_hi, B_lo

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
};

struct TcSmem {
    unsigned char buf[2][kBufBytes];
    TcAtom at[kTcMaxAtoms];
    int64_t pairoff[kTcMaxAtoms * kTcMaxAtoms];
    float4 pt[kTcMaxPts];           // in-brick offset of each point (x, y, z) and 2^s V dV
    SpeciesFast spf[kTcMaxSpecies];
    unsigned char row_atom[kTcMaxRows];
    unsigned char row_mu[kTcMaxRows];
    uint64_t bar[2];
    uint32_t tmem;
    int work;
    int abort;
    float scale_inv;
};

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

template <typename H16>
__global__ void __launch_bounds__(kTcThreads, 1) k_vlocal_tc(TcArgs A, const double* V, double* H) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TcSmem& S = *reinterpret_cast<TcSmem*>(smem_raw);
    const Problem& P = A.P;
    const GridDev& g = P.g;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t idesc = tc::idesc_f16(128, 128, Conv<H16>::bf16, 0, 0);

    if (warp == 0) {
        tc::tmem_alloc(&S.tmem, 512);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(&S.bar[0], 1);
        tc::mbar_init(&S.bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        S.abort = 0;
    }
    if (tid < P.n_species) species_fast_from(P.sp[tid], S.spf[tid]);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = S.tmem;
    uint32_t commits[2] = {0, 0};  // completed-phase counters per buffer (same in every thread)
    const float4* coef4 = reinterpret_cast<const float4*>(P.coef32);

    for (;;) {
        if (tid == 0) S.work = atomicAdd(A.counter, 1);
        __syncthreads();
        const int w = S.work;
        if (w >= P.n_work || S.abort) break;
        const int brick = P.work[w];
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
                wv = (float)(V[((int64_t)g0 * g.n[1] + g1) * g.n[2] + g2] * g.dV);
            const int l2 = p % g.B[2], l1 = (p / g.B[2]) % g.B[1], l0 = p / (g.B[2] * g.B[1]);
            float4 q4;
            q4.x = (float)l0 * (float)g.step[0][0] + (float)l1 * (float)g.step[1][0] + (float)l2 * (float)g.step[2][0];
            q4.y = (float)l0 * (float)g.step[0][1] + (float)l1 * (float)g.step[1][1] + (float)l2 * (float)g.step[2][1];
            q4.z = (float)l0 * (float)g.step[0][2] + (float)l1 * (float)g.step[1][2] + (float)l2 * (float)g.step[2][2];
            q4.w = wv;
            S.pt[p] = q4;
            wmax = fmaxf(wmax, fabsf(wv));
        }
        for (int o = 16; o > 0; o >>= 1) wmax = fmaxf(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
        __shared__ float s_wmax[kTcThreads / 32];
        if (lane == 0) s_wmax[warp] = wmax;
        __syncthreads();
        if (tid == 0) {
            float m = 0.f;
            for (int k = 0; k < kTcThreads / 32; ++k) m = fmaxf(m, s_wmax[k]);
            int e = 0;
            if (m > 0.f) frexpf(m, &e);  // m = f 2^e, f in [0.5, 1)
            S.scale_inv = ldexpf(1.f, e);
            int off = 0;
            for (int i = 0; i < na; ++i) {
                S.at[i].off = off;
                for (int o = 0; o < S.at[i].nw; ++o) { S.row_atom[off + o] = (unsigned char)i; S.row_mu[off + o] = (unsigned char)o; }
                off += S.at[i].nw;
            }
        }
        __syncthreads();
        const float wscale = 1.f / S.scale_inv;
        for (int p = tid; p < g.bpad; p += kTcThreads) S.pt[p].w *= wscale;
        int nrow = 0;
        for (int i = 0; i < na; ++i) nrow += S.at[i].nw;
        const int nt = (nrow + 127) >> 7;
        // pair table: offsets of canonical blocks for pairs within cutoff
        for (int q = tid; q < na * na; q += kTcThreads) {
            const int a1 = q / na, a2 = q - a1 * na;
            if (a1 > a2) continue;
            int64_t off = -1;
            const TcAtom &X = S.at[a1], &Y = S.at[a2];
            // FP32 distance with a margin: only pairs within rc1 + rc2 are looked up
            const float dx = (Y.c_hi[0] - X.c_hi[0]) + (Y.c_lo[0] - X.c_lo[0]);
            const float dy = (Y.c_hi[1] - X.c_hi[1]) + (Y.c_lo[1] - X.c_lo[1]);
            const float dz = (Y.c_hi[2] - X.c_hi[2]) + (Y.c_lo[2] - X.c_lo[2]);
            const float dist = sqrtf(dx * dx + dy * dy + dz * dz);
            const float cut = P.sp[X.sp].rc_f + P.sp[Y.sp].rc_f;
            if (dist < cut + 1e-3f) {
                const int64_t blk = find_block(P, X.I, Y.I, Y.t[0] - X.t[0], Y.t[1] - X.t[1], Y.t[2] - X.t[2]);
                if (blk >= 0) off = P.offsets[blk];
                else if (dist < cut - 1e-3f) atomicOr(P.err, kErrPatternMissing);
            }
            S.pairoff[a1 * na + a2] = off;
        }
        // zero the padding rows [nrow, nt*128) of both chunk buffers
        for (int b = 0; b < 2; ++b)
            for (int e = tid; e < (nt * 128 - nrow) * kTcChunk; e += kTcThreads) {
                const int r = nrow + e / kTcChunk, q = e % kTcChunk;
                const int o = piece_off(r, q);
                for (int pc = 0; pc < 4; ++pc)
                    *reinterpret_cast<unsigned short*>(&S.buf[b][pc * kPieceBytes + o]) = 0;
            }
        __syncthreads();

        // ---- tile pairs (i <= j), processed in passes of up to four
        const int npairs = nt * (nt + 1) / 2;
        const int nchunks = g.bpad / kTcChunk;
        for (int pass0 = 0; pass0 < npairs && !S.abort; pass0 += kTcMaxPairsPerPass) {
            const int pass_n = min(kTcMaxPairsPerPass, npairs - pass0);
            // tiles whose rows this pass reads; only atom images with rows in them are produced
            unsigned need = 0;
            {
                int pi = 0, pj = 0;
                for (int t = 0; t < pass0 + pass_n; ++t) {
                    if (t >= pass0) need |= (1u << pi) | (1u << pj);
                    if (++pj >= nt) { ++pi; pj = pi; }
                }
            }
            for (int c = 0; c < nchunks; ++c) {
                const int b = c & 1;
                // the MMAs of the chunk that last used this buffer must be done
                if (commits[b] > 0) {
                    if (!tc::mbar_wait(&S.bar[b], (commits[b] - 1) & 1, kWaitLimit)) {
                        if (lane == 0) atomicOr(&S.abort, 1);
                    }
                }
                // orbital values of the needed atom images at the chunk's 16 points
                unsigned char* buf = S.buf[b];
                for (int item = tid; item < na * kTcChunk; item += kTcThreads) {
                    const int a = item / kTcChunk, q = item - a * kTcChunk;
                    const TcAtom& X = S.at[a];
                    const int t0 = X.off >> 7, t1 = (X.off + X.nw - 1) >> 7;
                    if (!((need >> t0) & 1u) && !((need >> t1) & 1u)) continue;
                    const int p = c * kTcChunk + q;
                    const float4 q4 = S.pt[p];
                    const float dx = (X.c_hi[0] + q4.x) + X.c_lo[0];
                    const float dy = (X.c_hi[1] + q4.y) + X.c_lo[1];
                    const float dz = (X.c_hi[2] + q4.z) + X.c_lo[2];
                    const float wv = q4.w;
                    const int rbase = X.off;
                    auto put = [&](int o, float v, float, float, float) {
                        unsigned short ah, al, bh, bl;
                        Conv<H16>::split(v * wv, ah, al);
                        Conv<H16>::split(v, bh, bl);
                        const int off = piece_off(rbase + o, q);
                        *reinterpret_cast<unsigned short*>(&buf[0 * kPieceBytes + off]) = ah;
                        *reinterpret_cast<unsigned short*>(&buf[1 * kPieceBytes + off]) = al;
                        *reinterpret_cast<unsigned short*>(&buf[2 * kPieceBytes + off]) = bh;
                        *reinterpret_cast<unsigned short*>(&buf[3 * kPieceBytes + off]) = bl;
                    };
                    const bool inside = p < g.bpts && orbitals_fast<false>(S.spf[X.sp], coef4, dx, dy, dz, put);
                    if (!inside)
                        for (int o = 0; o < X.nw; ++o) {
                            const int off = piece_off(rbase + o, q);
                            for (int pc = 0; pc < 4; ++pc) *reinterpret_cast<unsigned short*>(&buf[pc * kPieceBytes + off]) = 0;
                        }
                }
                tc::fence_async_smem();
                __syncthreads();
                if (S.abort) break;
                if (tid == 0) {
                    tc::fence_after_sync();
                    const uint32_t base = tc::smem_u32(buf);
                    // K-major operands: LBO = distance of K-adjacent core matrices (128 B),
                    // SBO = distance of row-adjacent core matrices (2 * 128 B)
                    const uint32_t lbo = 128, sbo = (kTcChunk / 8) * 128;
                    int pi = 0, pj = 0, k = 0;
                    for (int t = 0; t < pass0 + pass_n; ++t) {
                        if (t >= pass0) {
                            const uint32_t tile_bytes = 128 * kTcChunk * 2;  // 16 row groups
                            const uint32_t a_hi = base + 0 * kPieceBytes + pi * tile_bytes;
                            const uint32_t a_lo = base + 1 * kPieceBytes + pi * tile_bytes;
                            const uint32_t b_hi = base + 2 * kPieceBytes + pj * tile_bytes;
                            const uint32_t b_lo = base + 3 * kPieceBytes + pj * tile_bytes;
                            const uint32_t d = tmem + (uint32_t)((t - pass0) * 128);
                            tc::mma_f16(d, tc::smem_desc(a_hi, lbo, sbo), tc::smem_desc(b_hi, lbo, sbo), idesc, c > 0 ? 1u : 0u);
                            tc::mma_f16(d, tc::smem_desc(a_hi, lbo, sbo), tc::smem_desc(b_lo, lbo, sbo), idesc, 1u);
                            tc::mma_f16(d, tc::smem_desc(a_lo, lbo, sbo), tc::smem_desc(b_hi, lbo, sbo), idesc, 1u);
                        }
                        // next pair (i, j), i <= j, row-major over the upper triangle
                        ++k;
                        if (++pj >= nt) { ++pi; pj = pi; }
                    }
                    (void)k;
                    tc::mma_commit(&S.bar[b]);
                }
                commits[b] += 1;
            }
            // ---- wait for the last chunk's MMAs (the commit covers all earlier ones)
            {
                const int bl = (nchunks - 1) & 1;
                if (!tc::mbar_wait(&S.bar[bl], (commits[bl] - 1) & 1, kWaitLimit)) {
                    if (lane == 0) atomicOr(&S.abort, 1);
                }
                const int bo = bl ^ 1;
                if (commits[bo] > 0 && !tc::mbar_wait(&S.bar[bo], (commits[bo] - 1) & 1, kWaitLimit)) {
                    if (lane == 0) atomicOr(&S.abort, 1);
                }
            }
            tc::fence_after_sync();
            __syncthreads();
            if (S.abort) break;
            // ---- epilogue: warps 0-3 columns 0-63, warps 4-7 columns 64-127 of every tile of the pass
            {
                const int lane_base = (warp & 3) * 32;
                const int col0 = (warp >> 2) * 64;
                const float sinv = S.scale_inv;
                int pi = 0, pj = 0;
                for (int t = 0; t < pass0 + pass_n; ++t) {
                    if (t >= pass0) {
                        const int r = pi * 128 + lane_base + lane;
                        const bool rvalid = r < nrow;
                        const int a1 = rvalid ? S.row_atom[r] : 0;
                        const int mu = rvalid ? S.row_mu[r] : 0;
                        for (int cc = 0; cc < 64; cc += 16) {
                            float v[16];
                            tc::tmem_ld16(tmem + ((uint32_t)lane_base << 16) + (uint32_t)((t - pass0) * 128 + col0 + cc), v);
                            if (!rvalid) continue;
#pragma unroll
                            for (int jj = 0; jj < 16; ++jj) {
                                const int col = pj * 128 + col0 + cc + jj;
                                if (col >= nrow) continue;
                                const int a2 = S.row_atom[col];
                                if (a1 > a2) continue;
                                const int64_t off = S.pairoff[a1 * na + a2];
                                if (off < 0) continue;
                                const int nu = S.row_mu[col];
                                const double val = (double)(v[jj] * sinv);  // sinv is a power of two: exact
                                const int nw2 = S.at[a2].nw;
                                if (a1 == a2) {
                                    // same atom image: the block is symmetric; the tile grid only holds
                                    // r <= col for rows and columns in different tiles
                                    if (r > col) continue;
                                    atomicAdd(H + off + mu * nw2 + nu, val);
                                    if (mu != nu) atomicAdd(H + off + nu * nw2 + mu, val);
                                } else {
                                    atomicAdd(H + off + mu * nw2 + nu, val);
                                }
                            }
                        }
                    }
                    if (++pj >= nt) { ++pi; pj = pi; }
                }
            }
            tc::fence_before_sync();
            __syncthreads();
        }
        __syncthreads();
    }
    // ---- teardown: wait (bounded) for any MMA still in flight, then free TMEM
    __syncthreads();
    for (int b = 0; b < 2; ++b)
        if (commits[b] > 0) (void)tc::mbar_wait(&S.bar[b], (commits[b] - 1) & 1, kWaitLimit);
    if (S.abort && tid == 0) atomicOr(P.err, kErrTimeout);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

size_t tc_smem_bytes() { return sizeof(TcSmem) + 1024; }

gint_status tc_vlocal(gint_handle* h, int bf16, const double* V, double* H, cudaStream_t st) {
    if (h->n_work == 0) return GINT_OK;
    if (h->max_brick_orb > kTcMaxRows || h->max_brick_atoms > kTcMaxAtoms || h->grid.bpad > kTcMaxPts ||
        h->grid.bpad % kTcChunk != 0 || h->n_species > kTcMaxSpecies) {
        set_error("tensor-core form needs <= %d orbitals, <= %d atom images and <= %d points per brick and "
                  "<= %d species (have %d, %d, %d, %d); use smaller bricks", kTcMaxRows, kTcMaxAtoms, kTcMaxPts,
                  kTcMaxSpecies, h->max_brick_orb, h->max_brick_atoms, h->grid.bpad, h->n_species);
        return GINT_ERR_UNSUPPORTED;
    }
    TcArgs A;
    A.P = h->problem();
    A.counter = h->d_err + 2;
    GINT_CUDA_TRY(cudaMemsetAsync(A.counter, 0, sizeof(int), st));
    const size_t smem = tc_smem_bytes();
    if (bf16) {
        GINT_CUDA_TRY(cudaFuncSetAttribute(k_vlocal_tc<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_vlocal_tc<__nv_bfloat16><<<h->sm_count, kTcThreads, smem, st>>>(A, V, H);
    } else {
        GINT_CUDA_TRY(cudaFuncSetAttribute(k_vlocal_tc<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_vlocal_tc<__half><<<h->sm_count, kTcThreads, smem, st>>>(A, V, H);
    }
    GINT_CUDA_TRY(cudaGetLastError());
    return GINT_OK;
}

}  // namespace gint
