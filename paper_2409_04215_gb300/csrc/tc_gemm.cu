// One-body apply on the 5th-generation tensor cores: split-K multi-piece TF32 GEMM with tcgen05.
//
//   P[z][m][n] = sum_{k in chunk z} A[m][k] B[n][k]   (both operands K-major, FP32 pieces in memory)
//
// Every operand value x (an FP64 number) is stored as TF32 pieces, x ~ x0 + x1 (+ x2), each piece
// the round-to-nearest TF32 value of what the earlier pieces leave over.  Two pieces hold x to about
// 2^-22 and the product is formed from the three terms of order >= 2^-11 (3xTF32); three pieces hold
// it to about 2^-33 and the product keeps the six terms of order >= 2^-22 (6xTF32).  Each term is one
// tcgen05.mma.kind::tf32 per K step of 8, accumulated in FP32 in tensor memory (TMEM).  Plain FP32
// accumulation, not the product split, limits the accuracy, so the accumulations are kept short:
// the leading term x0*y0 goes to one of up to four "main" accumulators in turn (one per K stage), the
// correction terms (2^-11 smaller, so their rounding is negligible) to a separate one, the epilogue
// adds them with TwoSum into a (hi, lo) float pair, and K is split over CTAs (grid.z) in chunks of a
// few hundred whose pairs are summed in double-float arithmetic afterwards.  No FP64 arithmetic runs
// on the way (GB300's FP64 rate is a small fraction of its FP32 rate).
//
// The factor (B: U^T or W^T of the one-body SVD, Eq. pseudo) is the MMA's M side (128 rows per CTA),
// the gathered columns (A) its N side (<= 256), so a handful of bodies still fills the 128-row MMA.
// The factor is the bulk of the traffic, so it is stored as an FP32 pair (hi, lo) = (fl(x), fl(x - hi))
// (8 bytes per element, exact to about 2^-48) and cut into its TF32 pieces in shared memory after the
// TMA load; the columns arrive as pieces.
//
// Per CTA (192 threads): warp 0 lane 0 issues TMA loads (cp.async.bulk.tensor, 128-byte swizzle)
// into a two-stage ring, warps 2 to 5 cut each landed factor tile (hi, lo) into its TF32 pieces in
// place (the three tiles share one layout, so the cut is element-wise at equal offsets) and release it
// to warp 1 lane 0, which issues the MMAs and commits each stage back to the loader; warp 2 owns the
// TMEM allocation, and warps 0 to 3 read the accumulators with tcgen05.ld (warp w reads TMEM lanes
// 32w..32w+31) and write the (hi, lo) partials.  Every wait is bounded; on a timeout the CTA records an
// error flag, waits for the MMAs it issued, agrees (block vote), frees its TMEM and returns.
#include <cuda.h>

#include <cstring>

#include "common.cuh"
#include "kernels.h"

namespace mfs {

namespace tc {
constexpr int BM = 128;              // factor rows per CTA (MMA M)
constexpr int BK = 32;               // K elements per stage (128 bytes: one swizzle row)
constexpr int STAGES = 2;
constexpr int B_TILE = BM * BK * 4;  // bytes of one 128 x 32 FP32 factor tile (16 KB)
constexpr int THREADS = 192;         // warps 0-3: TMA, MMA, TMEM, epilogue; warps 2-5: cutting pieces
constexpr int CUTTERS = 128;         // threads of warps 2-5

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    // K-major operand, 128-byte swizzle: start address >> 4 (bits 0-13), leading byte offset unused
    // for this layout (encoded 1, bits 16-29), stride byte offset 1024 B between 8-row groups
    // (bits 32-45), descriptor version 1 (bits 46-47), swizzle mode 128B (value 2, bits 61-63).
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

__host__ __device__ constexpr uint32_t instr_desc_tf32(int M, int N) {
    // D = F32 (bits 4-5 = 1), A = B = TF32 (bits 7-9 = 2, bits 10-12 = 2), both K-major (bits 15, 16 = 0),
    // N >> 3 at bits 17-22, M >> 4 at bits 24-28.
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
        "[%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// The products kept: factor piece fa[t] times column piece fb[t], largest first.
template <int PIECES>
struct Terms;
template <>
struct Terms<2> {
    static constexpr int N = 3;
    __device__ static constexpr int fa(int t) { return t == 2 ? 1 : 0; }
    __device__ static constexpr int fb(int t) { return t == 1 ? 1 : 0; }
};
template <>
struct Terms<3> {
    static constexpr int N = 6;  // x0y0, x0y1, x1y0, x1y1, x0y2, x2y0
    __device__ static constexpr int fa(int t) { return t == 2 || t == 3 ? 1 : (t == 5 ? 2 : 0); }
    __device__ static constexpr int fb(int t) { return t == 1 || t == 3 ? 1 : (t == 4 ? 2 : 0); }
};

// (hi, lo) += v exactly up to the final rounding of lo (Knuth's TwoSum on the high part).
__device__ __forceinline__ void df_add(float &hi, float &lo, float v) {
    const float s = hi + v;
    const float bb = s - hi;
    lo += (hi - (s - bb)) + (v - bb);
    hi = s;
}

// (hi, lo) += (h, l), renormalised (double-float addition).
__device__ __forceinline__ void df_add2(float &hi, float &lo, float h, float l) {
    df_add(hi, lo, h);
    lo += l;
    const float s = hi + lo;
    lo = lo - (s - hi);
    hi = s;
}

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t t;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(x));
    return __uint_as_float(t);
}

// The nearest TF32 value (10 explicit mantissa bits), ties away from zero, by integer operations on the
// bits of a finite x: half a TF32 unit in the last place added to the magnitude, the 13 low bits cleared
// (a carry into the exponent is the rounding up into the next binade).
__device__ __forceinline__ float tf32_round_bits(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xffffe000u);
}

// The same split as split_pieces_df with the integer rounding (the cut inside the GEMM kernel).
__device__ __forceinline__ void split_pieces_bits(float hi, float lo, int pieces, float *p) {
    p[0] = tf32_round_bits(hi);
    const float rem = (hi - p[0]) + lo;
    p[1] = tf32_round_bits(rem);
    p[2] = pieces == 3 ? tf32_round_bits(rem - p[1]) : 0.f;
}

// (hi + lo) ~ p[0] + p[1] (+ p[2]) with FP32 arithmetic only: hi - tf32(hi) is exact.
__device__ __forceinline__ void split_pieces_df(float hi, float lo, int pieces, float *p) {
    p[0] = tf32_rna(hi);
    const float rem = (hi - p[0]) + lo;
    p[1] = tf32_rna(rem);
    p[2] = pieces == 3 ? tf32_rna(rem - p[1]) : 0.f;
}

// x ~ p[0] + p[1] (+ p[2]), each the nearest TF32 value of the remainder left by the earlier pieces.
__device__ __forceinline__ void split_pieces(double x, int pieces, float *p) {
    double rem = x;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        p[i] = i < pieces ? tf32_rna((float)rem) : 0.f;
        rem -= (double)p[i];
    }
}
}  // namespace tc

// grid: (ceil(n / 128), ceil(m / BN), chunks); block tc::THREADS; dynamic smem tc_gemm_smem(BN, PIECES)
template <int PIECES>
__global__ void __launch_bounds__(tc::THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ TcOperands ops, int m, int n, int k, int kchunk, int BN, int tmem_cols,
                   int nacc, float2 *P, int *err) {
    using namespace tc;
    using TT = Terms<PIECES>;
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[STAGES], cut_bar[STAGES], empty_bar[STAGES], done_bar;
    __shared__ uint32_t tmem_base_sh;
    // 1024-byte aligned tiles (128-byte swizzle atoms are 8 rows x 128 bytes)
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t a_tile = (uint32_t)BN * BK * 4;
    const uint32_t stage_bytes = PIECES * (B_TILE + a_tile);
    const uint32_t load_bytes = 2 * B_TILE + PIECES * a_tile;  // factor (hi, lo), column pieces
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n0 = blockIdx.x * BM, m0 = blockIdx.y * BN;
    const int kb0 = blockIdx.z * kchunk;
    const int kb1 = min(k, kb0 + kchunk);
    const int nk = (kb1 - kb0 + BK - 1) / BK;
    const long long limit = 1ll << 22;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&cut_bar[s], CUTTERS / 32);  // one arrival per cutting warp
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&done_bar, 1);
        fence_mbar_init();
    }
    if (warp == 2) {  // TMEM allocation (whole warp), address written to shared memory
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_sh;

    bool ok = true;
    if (warp == 0 && lane == 0) {  // TMA producer: factor pieces, then column pieces, per stage
        for (int i = 0; i < nk && ok; ++i) {
            const int s = i % STAGES;
            if (i >= STAGES) ok = mbar_wait_bounded(&empty_bar[s], (uint32_t)(((i / STAGES) - 1) & 1), err, limit);
            if (!ok) break;
            const uint32_t st = base + s * stage_bytes;
            const uint32_t fb = smem_u32(&full_bar[s]);
            mbar_arrive_expect_tx(&full_bar[s], load_bytes);
            const int kx = kb0 + i * BK;
#pragma unroll
            for (int p = 0; p < 2; ++p)  // factor hi and lo into piece slots 0 and 1
                tma_load_2d(st + p * B_TILE, reinterpret_cast<const CUtensorMap *>(&ops.b[p]), kx, n0, fb);
#pragma unroll
            for (int p = 0; p < PIECES; ++p)
                tma_load_2d(st + PIECES * B_TILE + p * a_tile, reinterpret_cast<const CUtensorMap *>(&ops.a[p]), kx,
                            m0, fb);
        }
    } else if (warp >= 2) {  // cut the landed factor tile (hi, lo) into TF32 pieces, in place
        const int ct = threadIdx.x - 64;  // 0 .. CUTTERS - 1
        for (int i = 0; i < nk && ok; ++i) {
            const int s = i % STAGES;
            ok = mbar_wait_bounded(&full_bar[s], (uint32_t)((i / STAGES) & 1), err, limit);
            if (!ok) break;
            float4 *t0 = reinterpret_cast<float4 *>(smem_raw + (base - raw) + s * stage_bytes);
            float4 *t1 = t0 + B_TILE / 16;
            float4 *t2 = t1 + B_TILE / 16;
            for (int v = ct; v < B_TILE / 16; v += CUTTERS) {
                const float4 h = t0[v], l = t1[v];
                float p0[4], p1[4], p2[4];
                const float hv[4] = {h.x, h.y, h.z, h.w}, lv[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    float q[3];
                    tc::split_pieces_bits(hv[e], lv[e], PIECES, q);
                    p0[e] = q[0];
                    p1[e] = q[1];
                    p2[e] = q[2];
                }
                t0[v] = make_float4(p0[0], p0[1], p0[2], p0[3]);
                t1[v] = make_float4(p1[0], p1[1], p1[2], p1[3]);
                if (PIECES == 3) t2[v] = make_float4(p2[0], p2[1], p2[2], p2[3]);
            }
            // the pieces are read by the tensor cores (async proxy) after this warp's release
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive_expect_tx(&cut_bar[s], 0);
        }
    } else if (warp == 1 && lane == 0) {  // MMA issuer
        const uint32_t idesc = instr_desc_tf32(BM, BN);
        const uint32_t dcorr = tmem + (uint32_t)(BN * nacc);  // correction terms, columns BN * nacc ...
        for (int i = 0; i < nk && ok; ++i) {
            const int s = i % STAGES;
            // the leading term of stage i goes to main accumulator i % nacc (TMEM columns BN * (i % nacc) ...)
            const uint32_t dmain = tmem + (uint32_t)(BN * (i % nacc));
            ok = mbar_wait_bounded(&cut_bar[s], (uint32_t)((i / STAGES) & 1), err, limit);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t st = base + s * stage_bytes;
#pragma unroll
            for (int kk = 0; kk < BK / 8; ++kk) {  // 8 TF32 = 32 bytes per MMA K step
                const uint32_t off = kk * 32;
#pragma unroll
                for (int t = 0; t < TT::N; ++t) {
                    const uint64_t fdesc = smem_desc(st + TT::fa(t) * B_TILE + off);
                    const uint64_t cdesc = smem_desc(st + PIECES * B_TILE + TT::fb(t) * a_tile + off);
                    if (t == 0)
                        mma_tf32(dmain, fdesc, cdesc, idesc, (i >= nacc || kk > 0) ? 1u : 0u);
                    else
                        mma_tf32(dcorr, fdesc, cdesc, idesc, (i > 0 || kk > 0 || t > 1) ? 1u : 0u);
                }
            }
            mma_commit(smem_u32(&empty_bar[s]));  // stage free once these MMAs have read it
        }
        // also after a timeout: the commit fires once every MMA issued so far has finished, so the TMEM
        // is never freed under a running MMA
        mma_commit(smem_u32(&done_bar));
    }
    __syncwarp();
    // everybody: wait for the accumulators (bounded), then agree on success
    bool good = mbar_wait_bounded(&done_bar, 0u, err, limit);
    good = __syncthreads_and(good && ok) != 0;
    if (good && warp < 4) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int row = n0 + 32 * warp + lane;  // TMEM lane = factor row
        const int used = min(nacc, nk);          // main accumulators written by at least one stage
        const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);
        float2 *Pz = P + (size_t)blockIdx.z * m * n;
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float hi[16], lo[16];
            tc::tmem_ld16(lane_base + (uint32_t)(BN * nacc + c0), hi);  // corrections first (smallest)
#pragma unroll
            for (int i = 0; i < 16; ++i) lo[i] = 0.f;
            for (int a = 0; a < used; ++a) {
                float v[16];
                tc::tmem_ld16(lane_base + (uint32_t)(BN * a + c0), v);
#pragma unroll
                for (int i = 0; i < 16; ++i) tc::df_add(hi[i], lo[i], v[i]);
            }
            if (row < n) {
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int col = m0 + c0 + i;
                    if (col < m) Pz[(size_t)col * n + row] = make_float2(hi[i], lo[i]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 2)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

// ---------------------------------------------------------------------------
// Operand pieces
// ---------------------------------------------------------------------------
// dst[0][c][r] = fl(src[r][c]), dst[1][c][r] = fl(src[r][c] - dst[0][c][r]): an FP64 factor stored
// [rows][cols] as K-major FP32 (hi, lo) planes [cols][ld_dst], columns rows..ld_dst zero.
__global__ void split_hilo_transpose_kernel(const double *src, int rows, int cols, float *dst, int ld_dst,
                                            size_t pstride) {
    const size_t total = (size_t)cols * ld_dst;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i / ld_dst), r = (int)(i % ld_dst);
        float hi = 0.f, lo = 0.f;
        if (r < rows) {
            const double x = src[(size_t)r * cols + c];
            hi = (float)x;
            lo = (float)(x - (double)hi);
        }
        dst[i] = hi;
        dst[pstride + i] = lo;
    }
}

// Double-float sum over the chunks of P[z] = (hi, lo) pairs, [rows][cols].
__device__ __forceinline__ void df_chunk_sum(int S, size_t mn, size_t i, const float2 *__restrict__ P, float &hi,
                                             float &lo) {
    hi = 0.f;
    lo = 0.f;
    for (int z = 0; z < S; ++z) {
        const float2 v = P[(size_t)z * mn + i];
        tc::df_add2(hi, lo, v.x, v.y);
    }
}

// C = sum_z P[z], written as pieces dst[p][row][col] (leading dimension ld_dst).
__global__ void reduce_pieces_kernel(int S, int rows, int cols, const float2 *__restrict__ P, float *dst, int ld_dst,
                                     size_t pstride, int pieces) {
    const size_t mn = (size_t)rows * cols;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < mn; i += (size_t)gridDim.x * blockDim.x) {
        float hi, lo, p[3];
        df_chunk_sum(S, mn, i, P, hi, lo);
        tc::split_pieces_df(hi, lo, pieces, p);
        const size_t o = (i / cols) * ld_dst + (i % cols);
#pragma unroll
        for (int q = 0; q < 3; ++q)
            if (q < pieces) dst[q * pstride + o] = p[q];
    }
}

// C = sum_z P[z] as FP64.
__global__ void reduce_f64_kernel(int S, size_t mn, const float2 *__restrict__ P, double *C) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < mn; i += (size_t)gridDim.x * blockDim.x) {
        float hi, lo;
        df_chunk_sum(S, mn, i, P, hi, lo);
        C[i] = (double)hi + (double)lo;
    }
}

// Gather and rotate into the body frame (as gather_rotate), written directly as pieces
// dst[p][col][ld_dst] of the FP64 values.
__global__ void gather_rotate_pieces_kernel(int D, const double *gamma, int sum_MD, const int *col_body,
                                            const int *col_rhs, const int *body_tgt_off, const double *rot, int ncols,
                                            int dM, float *dst, int ld_dst, size_t pstride, int pieces) {
    const int col = blockIdx.y;
    const int M = dM / D;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= M || col >= ncols) return;
    const int k = col_body[col], h = col_rhs[col];
    const double *gk = gamma + (size_t)h * sum_MD + (size_t)body_tgt_off[k] * D;
    float q[3];
    float *out = dst + (size_t)col * ld_dst;
    if (D == 1) {
        tc::split_pieces(gk[p], pieces, q);
#pragma unroll
        for (int j = 0; j < 3; ++j)
            if (j < pieces) out[j * pstride + p] = q[j];
    } else {
        const double *R = rot + 9 * k;  // row-major R; (R^T g)_a = sum_b R[b][a] g_b
        const double g0 = gk[3 * p], g1 = gk[3 * p + 1], g2 = gk[3 * p + 2];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            tc::split_pieces(R[a] * g0 + R[3 + a] * g1 + R[6 + a] * g2, pieces, q);
#pragma unroll
            for (int j = 0; j < 3; ++j)
                if (j < pieces) out[j * pstride + 3 * p + a] = q[j];
        }
    }
}

// dst[p][c][r] = src[p][r][c] for r < rows, c < cols, zero for r in [rows, ld_dst): the pieces of a
// factor laid out for the transposed product (a transposition of TF32 values, exact).  Tiles of
// 32 x 32 through shared memory (both sides coalesced).
__global__ void transpose_pieces_kernel(const float *src, int rows, int cols, int ld_src, size_t sstride, float *dst,
                                        int ld_dst, size_t dstride) {
    __shared__ float t[32][33];
    const int p = blockIdx.z;
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    const float *sp = src + p * sstride;
    float *dp = dst + p * dstride;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        t[i][threadIdx.x] = (r < rows && c < cols) ? sp[(size_t)r * ld_src + c] : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (c < cols && r < ld_dst) dp[(size_t)c * ld_dst + r] = t[threadIdx.x][i];
    }
}

cudaError_t transpose_pieces(const float *src, int rows, int cols, int ld_src, size_t sstride, float *dst, int ld_dst,
                             size_t dstride, int pieces, cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    if (pieces < 2 || pieces > 3 || ld_dst < rows || ld_src < cols) return cudaErrorInvalidValue;
    dim3 grid((cols + 31) / 32, (ld_dst + 31) / 32, pieces), block(32, 8);
    transpose_pieces_kernel<<<grid, block, 0, st>>>(src, rows, cols, ld_src, sstride, dst, ld_dst, dstride);
    return cudaGetLastError();
}

cudaError_t split_hilo_transpose(const double *src, int rows, int cols, float *dst, int ld_dst, size_t pstride,
                                 cudaStream_t st) {
    if (cols == 0) return cudaSuccess;
    split_hilo_transpose_kernel<<<1024, 256, 0, st>>>(src, rows, cols, dst, ld_dst, pstride);
    return cudaGetLastError();
}

cudaError_t reduce_pieces(int S, int rows, int cols, const float2 *P, float *dst, int ld_dst, size_t pstride,
                          int pieces, cudaStream_t st) {
    const size_t mn = (size_t)rows * cols;
    if (mn == 0) return cudaSuccess;
    if (pieces < 2 || pieces > 3) return cudaErrorInvalidValue;
    reduce_pieces_kernel<<<(unsigned)std::min<size_t>((mn + 255) / 256, 4096), 256, 0, st>>>(S, rows, cols, P, dst,
                                                                                               ld_dst, pstride, pieces);
    return cudaGetLastError();
}

cudaError_t reduce_f64(int S, size_t mn, const float2 *P, double *C, cudaStream_t st) {
    if (mn == 0) return cudaSuccess;
    reduce_f64_kernel<<<(unsigned)std::min<size_t>((mn + 255) / 256, 4096), 256, 0, st>>>(S, mn, P, C);
    return cudaGetLastError();
}

cudaError_t gather_rotate_pieces(int D, const double *gamma, int sum_MD, const int *col_body, const int *col_rhs,
                                 const int *body_tgt_off, const double *rot, int ncols, int dM, float *dst, int ld_dst,
                                 size_t pstride, int pieces, cudaStream_t st) {
    if (ncols == 0) return cudaSuccess;
    if (pieces < 2 || pieces > 3) return cudaErrorInvalidValue;
    const int M = dM / D;
    dim3 grid((M + 127) / 128, ncols);
    gather_rotate_pieces_kernel<<<grid, 128, 0, st>>>(D, gamma, sum_MD, col_body, col_rhs, body_tgt_off, rot, ncols,
                                                       dM, dst, ld_dst, pstride, pieces);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Host: tensor maps (driver entry point fetched through the runtime, no -lcuda)
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// 2-D FP32 tensor [rows][ld] (ld a multiple of 32), box 32 x box_rows, 128-byte swizzle, zero fill.
bool make_tc_map(TcMap &out, const float *ptr, int rows, int ld, int box_rows) {
    static_assert(sizeof(CUtensorMap) == sizeof(TcMap), "tensor map size");
    EncodeTiledFn fn = encode_fn();
    if (!fn || !ptr || rows < 1 || ld % 32 != 0 || box_rows < 8 || box_rows > 256 ||
        (reinterpret_cast<uintptr_t>(ptr) & 15))
        return false;
    CUtensorMap m;
    std::memset(&m, 0, sizeof(m));
    const cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
    const cuuint32_t box[2] = {32u, (cuuint32_t)box_rows};
    const cuuint32_t es[2] = {1u, 1u};
    if (fn(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(ptr), dims, strides, box, es,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    std::memcpy(&out, &m, sizeof(m));
    return true;
}

int tc_gemm_bn(int m, int pieces) {  // MMA N: columns per CTA, a multiple of 16; 128 at most for 3 pieces
    const int cap = pieces == 3 ? 128 : 256;
    const int b = ((m + 15) / 16) * 16;
    return b > cap ? cap : (b < 16 ? 16 : b);
}

size_t tc_gemm_smem(int BN, int pieces) {
    return (size_t)tc::STAGES * pieces * (tc::B_TILE + (size_t)BN * tc::BK * 4) + 1024;
}

int tc_gemm_chunks(int m, int n, int k, int sm_count, int pieces) {
    const int bn = tc_gemm_bn(m, pieces);
    const int tiles = ((n + tc::BM - 1) / tc::BM) * ((m + bn - 1) / bn);
    // whole waves: as many K chunks as fill the SMs once at the shared-memory occupancy (228 KB per
    // SM, 1 KB reserved per CTA), so no second, partly empty wave trails the first
    const size_t per_cta = tc_gemm_smem(bn, pieces) + 1024;
    int resident = (int)(233472 / per_cta);
    if (resident < 1) resident = 1;
    int s = (resident * sm_count) / tiles;
    const int smax = (k + 127) / 128;  // chunks of at least 128 K
    if (s > smax) s = smax;
    return s < 1 ? 1 : s;
}


int tc_gemm_sz(int k, int S) {
    const int kchunk = ((k + S - 1) / S + tc::BK - 1) / tc::BK * tc::BK;
    return (k + kchunk - 1) / kchunk;
}

// FP32 accumulators of BN columns (at most 4 main ones and the correction one) such that the CTAs
// resident on one SM together allocate
// no more than its 512 TMEM columns (an allocation beyond that would wait for a neighbour to finish).
template <int PIECES>
static cudaError_t tc_layout(int BN, int &nacc, int &cols) {
    static int cache[17] = {0};  // resident CTAs per SM, by BN / 16
    static bool attr = false;
    if (!attr) {  // the largest tile's shared memory, once: every BN then launches under it
        cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<PIECES>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)tc_gemm_smem(tc_gemm_bn(1 << 20, PIECES), PIECES));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const size_t smem = tc_gemm_smem(BN, PIECES);
    int &resident = cache[BN / 16];
    if (resident == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, tc_gemm_kernel<PIECES>, tc::THREADS,
                                                                      smem);
        if (e != cudaSuccess) return e;
        if (resident < 1) return cudaErrorInvalidConfiguration;
    }
    int cols_max = 512;
    while (cols_max * resident > 512) cols_max >>= 1;
    nacc = cols_max / BN - 1;  // main accumulators; one more holds the correction terms
    if (nacc > 4) nacc = 4;
    if (nacc < 1) return cudaErrorInvalidConfiguration;
    cols = 32;
    while (cols < (nacc + 1) * BN) cols <<= 1;
    return cudaSuccess;
}

template <int PIECES>
static cudaError_t tc_gemm_launch(const TcMap *b, const TcMap *a, int m, int n, int k, int S, float2 *P, int *err,
                                  cudaStream_t st) {
    const int BN = tc_gemm_bn(m, PIECES);
    int nacc = 1, cols = 32;
    cudaError_t e = tc_layout<PIECES>(BN, nacc, cols);
    if (e != cudaSuccess) return e;
    const int kchunk = ((k + S - 1) / S + tc::BK - 1) / tc::BK * tc::BK;
    const int Sz = (k + kchunk - 1) / kchunk;
    TcOperands ops;
    std::memset(&ops, 0, sizeof(ops));
    std::memcpy(ops.b, b, PIECES * sizeof(TcMap));
    std::memcpy(ops.a, a, PIECES * sizeof(TcMap));
    dim3 grid((n + tc::BM - 1) / tc::BM, (m + BN - 1) / BN, Sz);
    tc_gemm_kernel<PIECES><<<grid, tc::THREADS, tc_gemm_smem(BN, PIECES), st>>>(ops, m, n, k, kchunk, BN, cols, nacc, P,
                                                                            err);
    return cudaGetLastError();
}

cudaError_t tc_gemm(int pieces, const TcMap *b, const TcMap *a, int m, int n, int k, int S, float2 *P, int *err,
                    cudaStream_t st) {
    if (m == 0 || n == 0) return cudaSuccess;
    if (k <= 0 || S <= 0) return cudaErrorInvalidValue;
    if (pieces == 2) return tc_gemm_launch<2>(b, a, m, n, k, S, P, err, st);
    if (pieces == 3) return tc_gemm_launch<3>(b, a, m, n, k, S, P, err, st);
    return cudaErrorInvalidValue;
}

}  // namespace mfs
