// Pair-sum kernels: the all-pairs Laplace / Stokeslet evaluation from proxy
// sources to collocation targets (Algorithm 1 MATVEC step 2; Sec. 2.1 Eq. Skk,
// Sec. 2.2 Eq. stokeslet) with self pairs skipped (step 3 folded in) and the
// identity term of Eq. 2esysprec added in the epilogue.
//
// FP32 arithmetic:
//   r  = (c_target_body - c_source_body)  [FP64 difference, rounded once]
//        + x_local - y_local               [body-local rotated FP32 coordinates]
//   Laplace   u += alpha / r
//   Stokeslet u += (lambda + r (r . lambda) / r^2) / r
// 1/(4 pi) or 1/(8 pi mu) is applied once per target in the FP64 epilogue.
// Accumulation per target: a fresh FP32 partial per block of 32 sources, the
// block partials summed per source body, and each body sum added into an
// FP32 (hi, lo) pair by TwoSum; shares of different CTAs are added in FP64.
//
// Two compute policies share one persistent, stream-K staging loop:
//  * Scalar<D, NRHS, T>: T targets per thread, one FP32 instruction per target.
//  * PackedStokes<NRHS, TP>: 2*TP targets per thread held as TP f32x2 register
//    pairs; every Stokeslet operation is one packed f32x2 instruction for two
//    targets (sm_100+ add/mul/fma.rn.f32x2), halving the issue slots the FP32
//    pipe needs.  Source records then hold every value twice, so one 128-bit
//    shared-memory load yields two ready operand pairs.
#include <algorithm>
#include <atomic>
#include <mutex>

#include "../../include/mfs.h"
#include "common.cuh"
#include "kernels.h"

namespace mfs {

typedef unsigned long long u64;

// ---------------------------------------------------------------------------
// f32x2 helpers (inline PTX, sm_100+)
// ---------------------------------------------------------------------------
__device__ __forceinline__ u64 f2_add(u64 a, u64 b) {
    u64 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 f2_sub(u64 a, u64 b) {
    u64 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 f2_mul(u64 a, u64 b) {
    u64 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 f2_fma(u64 a, u64 b, u64 c) {
    u64 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ u64 f2_pack(float lo, float hi) {
    u64 d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
    return d;
}
__device__ __forceinline__ void f2_unpack(u64 v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
// 1/sqrt(x) by the hardware approximation with subnormals flushed: r^2 here is never subnormal
// (r >= Delta_sep or a padding distance), so the flush never triggers and the subnormal handling
// of the non-flushing form is pure overhead in the pair loop.
__device__ __forceinline__ float rsqrt_ftz(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ---------------------------------------------------------------------------
// Record layouts
// ---------------------------------------------------------------------------
// plain:  [x y z s_0 ... s_{C-1}] padded to a multiple of 4 floats
// packed: every value twice, [x x y y z z s_0 s_0 ...] padded to a multiple of 4 floats
__host__ __device__ constexpr int rec_floats(int D, int nrhs, bool packed) {
    return packed ? (2 * (3 + D * nrhs) + 3) / 4 * 4 : ((3 + D * nrhs) + 3) / 4 * 4;
}

struct Stage {
    int tile;      // -1: no stage
    int body;      // source body
    int rec0;      // first record (global)
    int nrec;      // records in this stage (multiple of 4)
    long long u;   // global unit index of the first block
    int nblk;      // blocks in this stage
};

// Last tile with u0 <= u (tiles are contiguous in unit space; empty tiles come before the tile they abut).
__device__ __forceinline__ int tile_of_unit(const PairTile *tiles, int ntiles, long long u) {
    int lo = 0, hi = ntiles - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (tiles[mid].u0 <= u) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// The stage that starts at global unit u (u < uend), at most max_blocks blocks long.
__device__ __forceinline__ Stage make_stage(const PairTile *tiles, int ntiles, const PairGeom &geo, long long u,
                                            long long uend, int max_blocks, int hint_tile) {
    Stage st;
    int t = hint_tile;
    if (t < 0 || !(tiles[t].u0 <= u && u < tiles[t].u1)) t = tile_of_unit(tiles, ntiles, u);
    const PairTile tl = tiles[t];
    const long long seg_end_u = tl.u1 < uend ? tl.u1 : uend;
    if (tl.L0 >= 0) {  // interaction list: the entry e with lst_cum[e] <= u < lst_cum[e + 1]
        int lo = tl.L0, hi = tl.L1 - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (geo.lst_cum[mid] <= u) lo = mid; else hi = mid - 1;
        }
        const int seg = geo.lst_seg[lo];
        const int blk = (int)(u - geo.lst_cum[lo]);
        const int seg_blocks = (int)(geo.lst_cum[lo + 1] - geo.lst_cum[lo]);
        int n = seg_blocks - blk;
        if (n > max_blocks) n = max_blocks;
        if (n > seg_end_u - u) n = (int)(seg_end_u - u);
        st.tile = t;
        st.body = seg;
        st.rec0 = geo.seg_rec0[seg] + blk * MFS_BS;
        int rec_end = geo.seg_rec0[seg] + (blk + n) * MFS_BS;
        if (rec_end > geo.seg_rec1[seg]) rec_end = geo.seg_rec1[seg];
        st.nrec = rec_end - st.rec0;
        st.u = u;
        st.nblk = n;
        return st;
    }
    const long long *blk_off = geo.blk_off;
    const int *src_off = geo.src_off;
    long long gbl = blk_off[tl.B0] + (u - tl.u0);
    if (tl.skip >= 0 && gbl >= blk_off[tl.skip]) gbl += blk_off[tl.skip + 1] - blk_off[tl.skip];
    int lo = tl.B0, hi = tl.B1 - 1;  // body with blk_off[b] <= gbl
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (blk_off[mid] <= gbl) lo = mid; else hi = mid - 1;
    }
    const int b = lo;
    const int blk = (int)(gbl - blk_off[b]);
    const int body_blocks = (int)(blk_off[b + 1] - blk_off[b]);
    const long long rem = seg_end_u - u;
    int n = body_blocks - blk;
    if (n > max_blocks) n = max_blocks;
    if (n > rem) n = (int)rem;
    st.tile = t;
    st.body = b;
    st.rec0 = src_off[b] + blk * MFS_BS;
    int rec_end = src_off[b] + (blk + n) * MFS_BS;
    if (rec_end > src_off[b + 1]) rec_end = src_off[b + 1];
    st.nrec = rec_end - st.rec0;
    st.u = u;
    st.nblk = n;
    return st;
}

// ---------------------------------------------------------------------------
// Compute policies
// ---------------------------------------------------------------------------
// Hooks every policy has; the gradient policy overrides them (target strengths, source-side sums).
struct PolicyBase {
    static constexpr int MINB = 1;  // minimum resident CTAs per SM requested from the compiler
    static constexpr bool GRID_DC = false;  // true: centre differences split into grid hi + lo (compensated)
    // idx: the target (a clamped duplicate when !valid: computed, never written)
    __device__ __forceinline__ void load_extra(int, int, bool, const PairGeom &) {}
    __device__ __forceinline__ void source_side(int, bool, double *) {}
};

template <int D, int NRHS, int T, int NT>
struct Scalar : PolicyBase {
    static constexpr int C = D * NRHS;
    static constexpr int REC = rec_floats(D, NRHS, false);
    static constexpr int TPT = T;  // targets per thread
    static constexpr int PSM = 0;  // all per-target state in registers
    float3 tp[T];
    int tb[T];
    float hi[T][C], lo[T][C], bsum[T][C];

    __device__ __forceinline__ void init(float *, int) {}
    __device__ __forceinline__ void set_target(int j, float4 p) {
        tp[j] = make_float3(p.x, p.y, p.z);
        tb[j] = __float_as_int(p.w);
    }
    __device__ __forceinline__ void reset() {
#pragma unroll
        for (int j = 0; j < T; ++j)
#pragma unroll
            for (int c = 0; c < C; ++c) hi[j][c] = lo[j][c] = bsum[j][c] = 0.f;
    }
    __device__ __forceinline__ void compute(const float *sb, int nrec, const float (*dc)[3], const float (*)[3],
                                            int kb0) {
        float3 xt[T];
#pragma unroll
        for (int j = 0; j < T; ++j) {
            const int r = tb[j] - kb0;
            xt[j] = make_float3(dc[r][0] + tp[j].x, dc[r][1] + tp[j].y, dc[r][2] + tp[j].z);
        }
        for (int s0 = 0; s0 < nrec; s0 += MFS_BS) {
            const int s1 = min(s0 + MFS_BS, nrec);
            float blk[T][C];
#pragma unroll
            for (int j = 0; j < T; ++j)
#pragma unroll
                for (int c = 0; c < C; ++c) blk[j][c] = 0.f;
            for (int s = s0; s < s1; s += 4) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float rec[REC];
#pragma unroll
                    for (int v = 0; v < REC / 4; ++v) {
                        const float4 f = reinterpret_cast<const float4 *>(sb + (s + q) * REC)[v];
                        rec[4 * v + 0] = f.x;
                        rec[4 * v + 1] = f.y;
                        rec[4 * v + 2] = f.z;
                        rec[4 * v + 3] = f.w;
                    }
#pragma unroll
                    for (int j = 0; j < T; ++j) {
                        const float dx = xt[j].x - rec[0];
                        const float dy = xt[j].y - rec[1];
                        const float dz = xt[j].z - rec[2];
                        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                        const float ri = rsqrt_ftz(r2);
                        if (D == 1) {
#pragma unroll
                            for (int h = 0; h < NRHS; ++h) blk[j][h] = fmaf(rec[3 + h], ri, blk[j][h]);
                        } else {
                            const float ri2 = ri * ri;
#pragma unroll
                            for (int h = 0; h < NRHS; ++h) {
                                const float lx = rec[3 + 3 * h], ly = rec[4 + 3 * h], lz = rec[5 + 3 * h];
                                const float dot = fmaf(dx, lx, fmaf(dy, ly, dz * lz));
                                const float sc = dot * ri2;
                                blk[j][3 * h + 0] = fmaf(fmaf(dx, sc, lx), ri, blk[j][3 * h + 0]);
                                blk[j][3 * h + 1] = fmaf(fmaf(dy, sc, ly), ri, blk[j][3 * h + 1]);
                                blk[j][3 * h + 2] = fmaf(fmaf(dz, sc, lz), ri, blk[j][3 * h + 2]);
                            }
                        }
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < T; ++j)
#pragma unroll
                for (int c = 0; c < C; ++c) bsum[j][c] += blk[j][c];
        }
    }
    __device__ __forceinline__ void end_body(int body, bool include_self) {
#pragma unroll
        for (int j = 0; j < T; ++j) {
            const bool keep = include_self || (tb[j] != body);
#pragma unroll
            for (int c = 0; c < C; ++c) {
                float s, e;
                two_sum(hi[j][c], keep ? bsum[j][c] : 0.f, s, e);
                hi[j][c] = s;
                lo[j][c] += e;
                bsum[j][c] = 0.f;
            }
        }
    }
    __device__ __forceinline__ float result(int j, int c, float &l) const {
        l = lo[j][c];
        return hi[j][c];
    }
};

template <int NRHS, int TP, int NT, bool OA = false>
struct PackedStokesT : PolicyBase {
    static constexpr int D = 3;
    static constexpr int C = 3 * NRHS;
    static constexpr int REC = rec_floats(3, NRHS, true);
    static constexpr int TPT = 2 * TP;  // targets per thread
    static constexpr int T = TPT;
    // Per-target state touched once per stage or per source body (position, body, hi, lo) lives in
    // shared memory, thread-contiguous ([field][target][thread]: conflict-free), which leaves the
    // registers to the packed inner loop.
    static constexpr int FIELDS = 4 + 2 * C;
    static constexpr int PSM = FIELDS * T;  // floats of shared memory per thread
    float *sm;
    int tid;
    u64 bsum[TP][C];

    __device__ __forceinline__ float &at(int f, int j) const { return sm[(f * T + j) * NT + tid]; }
    __device__ __forceinline__ void init(float *base, int t) {
        sm = base;
        tid = t;
    }
    __device__ __forceinline__ void set_target(int j, float4 p) {
        at(0, j) = p.x;
        at(1, j) = p.y;
        at(2, j) = p.z;
        at(3, j) = p.w;
    }
    __device__ __forceinline__ int body(int j) const { return __float_as_int(at(3, j)); }
    __device__ __forceinline__ void reset() {
#pragma unroll
        for (int j = 0; j < T; ++j)
#pragma unroll
            for (int c = 0; c < C; ++c) at(4 + c, j) = at(4 + C + c, j) = 0.f;
#pragma unroll
        for (int p = 0; p < TP; ++p)
#pragma unroll
            for (int c = 0; c < C; ++c) bsum[p][c] = 0ull;
    }
    __device__ __forceinline__ void compute(const float *sb, int nrec, const float (*dc)[3], const float (*)[3],
                                            int kb0) {
        u64 xt[TP][3];
#pragma unroll
        for (int p = 0; p < TP; ++p) {
            const int j0 = 2 * p, j1 = 2 * p + 1;
            const int r0 = body(j0) - kb0, r1 = body(j1) - kb0;
            xt[p][0] = f2_pack(dc[r0][0] + at(0, j0), dc[r1][0] + at(0, j1));
            xt[p][1] = f2_pack(dc[r0][1] + at(1, j0), dc[r1][1] + at(1, j1));
            xt[p][2] = f2_pack(dc[r0][2] + at(2, j0), dc[r1][2] + at(2, j1));
        }
        for (int s0 = 0; s0 < nrec; s0 += MFS_BS) {
            const int s1 = min(s0 + MFS_BS, nrec);
            u64 blk[TP][C];
#pragma unroll
            for (int p = 0; p < TP; ++p)
#pragma unroll
                for (int c = 0; c < C; ++c) blk[p][c] = 0ull;
            for (int s = s0; s < s1; s += 4) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    u64 rec[REC / 2];
#pragma unroll
                    for (int v = 0; v < REC / 4; ++v) {
                        const ulonglong2 f = reinterpret_cast<const ulonglong2 *>(sb + (s + q) * REC)[v];
                        rec[2 * v] = f.x;
                        rec[2 * v + 1] = f.y;
                    }
#pragma unroll
                    for (int p = 0; p < TP; ++p) {
                        const u64 dx = f2_sub(xt[p][0], rec[0]);
                        const u64 dy = f2_sub(xt[p][1], rec[1]);
                        const u64 dz = f2_sub(xt[p][2], rec[2]);
                        const u64 r2 = f2_fma(dx, dx, f2_fma(dy, dy, f2_mul(dz, dz)));
                        float a, b;
                        f2_unpack(r2, a, b);
                        const u64 ri = f2_pack(rsqrt_ftz(a), rsqrt_ftz(b));
                        const u64 ri2 = f2_mul(ri, ri);
#pragma unroll
                        for (int h = 0; h < NRHS; ++h) {
                            const u64 lx = rec[3 + 3 * h], ly = rec[4 + 3 * h], lz = rec[5 + 3 * h];
                            u64 dot, sc;
                            if constexpr (OA) {  // the operand shared by consecutive FMAs in slot A
                                dot = f2_fma(lx, dx, f2_fma(ly, dy, f2_mul(lz, dz)));
                                sc = f2_mul(ri2, dot);
                                blk[p][3 * h + 0] = f2_fma(ri, f2_fma(sc, dx, lx), blk[p][3 * h + 0]);
                                blk[p][3 * h + 1] = f2_fma(ri, f2_fma(sc, dy, ly), blk[p][3 * h + 1]);
                                blk[p][3 * h + 2] = f2_fma(ri, f2_fma(sc, dz, lz), blk[p][3 * h + 2]);
                            } else {
                                dot = f2_fma(dx, lx, f2_fma(dy, ly, f2_mul(dz, lz)));
                                sc = f2_mul(dot, ri2);
                                blk[p][3 * h + 0] = f2_fma(f2_fma(dx, sc, lx), ri, blk[p][3 * h + 0]);
                                blk[p][3 * h + 1] = f2_fma(f2_fma(dy, sc, ly), ri, blk[p][3 * h + 1]);
                                blk[p][3 * h + 2] = f2_fma(f2_fma(dz, sc, lz), ri, blk[p][3 * h + 2]);
                            }
                        }
                    }
                }
            }
#pragma unroll
            for (int p = 0; p < TP; ++p)
#pragma unroll
                for (int c = 0; c < C; ++c) bsum[p][c] = f2_add(bsum[p][c], blk[p][c]);
        }
    }
    __device__ __forceinline__ void end_body(int src_body, bool include_self) {
#pragma unroll
        for (int p = 0; p < TP; ++p) {
            const int j0 = 2 * p, j1 = 2 * p + 1;
            const bool k0 = include_self || (body(j0) != src_body);
            const bool k1 = include_self || (body(j1) != src_body);
#pragma unroll
            for (int c = 0; c < C; ++c) {
                float v0, v1, s, e;
                f2_unpack(bsum[p][c], v0, v1);
                two_sum(at(4 + c, j0), k0 ? v0 : 0.f, s, e);
                at(4 + c, j0) = s;
                at(4 + C + c, j0) += e;
                two_sum(at(4 + c, j1), k1 ? v1 : 0.f, s, e);
                at(4 + c, j1) = s;
                at(4 + C + c, j1) += e;
                bsum[p][c] = 0ull;
            }
        }
    }
    __device__ __forceinline__ float result(int j, int c, float &l) const {
        l = at(4 + C + c, j);
        return at(4 + c, j);
    }
};
template <int NRHS, int TP, int NT>
using PackedStokes = PackedStokesT<NRHS, TP, NT, false>;
template <int NRHS, int TP, int NT>
using PackedStokesOA = PackedStokesT<NRHS, TP, NT, true>;

// The same packed Stokeslet arithmetic with all per-target state in registers (more registers,
// more freedom for the compiler to interleave sources; the autotuner picks per geometry).
template <int NRHS, int TP, int NT>
struct PackedStokesReg : PolicyBase {
    static constexpr int D = 3;
    static constexpr int C = 3 * NRHS;
    static constexpr int REC = rec_floats(3, NRHS, true);
    static constexpr int TPT = 2 * TP;
    static constexpr int T = TPT;
    static constexpr int PSM = 0;
    float3 tp[T];
    int tb[T];
    float hi[T][C], lo[T][C];
    u64 bsum[TP][C];

    __device__ __forceinline__ void init(float *, int) {}
    __device__ __forceinline__ void set_target(int j, float4 p) {
        tp[j] = make_float3(p.x, p.y, p.z);
        tb[j] = __float_as_int(p.w);
    }
    __device__ __forceinline__ void reset() {
#pragma unroll
        for (int j = 0; j < T; ++j)
#pragma unroll
            for (int c = 0; c < C; ++c) hi[j][c] = lo[j][c] = 0.f;
#pragma unroll
        for (int p = 0; p < TP; ++p)
#pragma unroll
            for (int c = 0; c < C; ++c) bsum[p][c] = 0ull;
    }
    __device__ __forceinline__ void compute(const float *sb, int nrec, const float (*dc)[3], const float (*)[3],
                                            int kb0) {
        u64 xt[TP][3];
#pragma unroll
        for (int p = 0; p < TP; ++p) {
            const int r0 = tb[2 * p] - kb0, r1 = tb[2 * p + 1] - kb0;
            xt[p][0] = f2_pack(dc[r0][0] + tp[2 * p].x, dc[r1][0] + tp[2 * p + 1].x);
            xt[p][1] = f2_pack(dc[r0][1] + tp[2 * p].y, dc[r1][1] + tp[2 * p + 1].y);
            xt[p][2] = f2_pack(dc[r0][2] + tp[2 * p].z, dc[r1][2] + tp[2 * p + 1].z);
        }
        for (int s0 = 0; s0 < nrec; s0 += MFS_BS) {
            const int s1 = min(s0 + MFS_BS, nrec);
            u64 blk[TP][C];
#pragma unroll
            for (int p = 0; p < TP; ++p)
#pragma unroll
                for (int c = 0; c < C; ++c) blk[p][c] = 0ull;
            for (int s = s0; s < s1; s += 4) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    u64 rec[REC / 2];
#pragma unroll
                    for (int v = 0; v < REC / 4; ++v) {
                        const ulonglong2 f = reinterpret_cast<const ulonglong2 *>(sb + (s + q) * REC)[v];
                        rec[2 * v] = f.x;
                        rec[2 * v + 1] = f.y;
                    }
#pragma unroll
                    for (int p = 0; p < TP; ++p) {
                        const u64 dx = f2_sub(xt[p][0], rec[0]);
                        const u64 dy = f2_sub(xt[p][1], rec[1]);
                        const u64 dz = f2_sub(xt[p][2], rec[2]);
                        const u64 r2 = f2_fma(dx, dx, f2_fma(dy, dy, f2_mul(dz, dz)));
                        float a, b;
                        f2_unpack(r2, a, b);
                        const u64 ri = f2_pack(rsqrt_ftz(a), rsqrt_ftz(b));
                        const u64 ri2 = f2_mul(ri, ri);
#pragma unroll
                        for (int h = 0; h < NRHS; ++h) {
                            const u64 lx = rec[3 + 3 * h], ly = rec[4 + 3 * h], lz = rec[5 + 3 * h];
                            const u64 dot = f2_fma(dx, lx, f2_fma(dy, ly, f2_mul(dz, lz)));
                            const u64 sc = f2_mul(dot, ri2);
                            blk[p][3 * h + 0] = f2_fma(f2_fma(dx, sc, lx), ri, blk[p][3 * h + 0]);
                            blk[p][3 * h + 1] = f2_fma(f2_fma(dy, sc, ly), ri, blk[p][3 * h + 1]);
                            blk[p][3 * h + 2] = f2_fma(f2_fma(dz, sc, lz), ri, blk[p][3 * h + 2]);
                        }
                    }
                }
            }
#pragma unroll
            for (int p = 0; p < TP; ++p)
#pragma unroll
                for (int c = 0; c < C; ++c) bsum[p][c] = f2_add(bsum[p][c], blk[p][c]);
        }
    }
    __device__ __forceinline__ void end_body(int body, bool include_self) {
#pragma unroll
        for (int p = 0; p < TP; ++p) {
            const bool k0 = include_self || (tb[2 * p] != body);
            const bool k1 = include_self || (tb[2 * p + 1] != body);
#pragma unroll
            for (int c = 0; c < C; ++c) {
                float v0, v1, s, e;
                f2_unpack(bsum[p][c], v0, v1);
                two_sum(hi[2 * p][c], k0 ? v0 : 0.f, s, e);
                hi[2 * p][c] = s;
                lo[2 * p][c] += e;
                two_sum(hi[2 * p + 1][c], k1 ? v1 : 0.f, s, e);
                hi[2 * p + 1][c] = s;
                lo[2 * p + 1][c] += e;
                bsum[p][c] = 0ull;
            }
        }
    }
    __device__ __forceinline__ float result(int j, int c, float &l) const {
        l = lo[j][c];
        return hi[j][c];
    }
};

// Laplace pairs (K2) in packed f32x2 arithmetic: two targets per instruction, as the packed
// Stokeslet; per pair 3 subtractions, r^2, one MUFU rsqrt and one FMA per rhs.  The MUFU then bounds
// the kernel (16 rsqrt per clock per SM against 128 FP32 lanes).
template <int NRHS, int TP, int NT>
struct PackedLaplaceReg : PolicyBase {
    static constexpr int D = 1;
    static constexpr int C = NRHS;
    static constexpr int REC = rec_floats(1, NRHS, true);
    static constexpr int TPT = 2 * TP;
    static constexpr int T = TPT;
    static constexpr int PSM = 0;
    float3 tp[T];
    int tb[T];
    float hi[T][C], lo[T][C];
    u64 bsum[TP][C];

    __device__ __forceinline__ void init(float *, int) {}
    __device__ __forceinline__ void set_target(int j, float4 p) {
        tp[j] = make_float3(p.x, p.y, p.z);
        tb[j] = __float_as_int(p.w);
    }
    __device__ __forceinline__ void reset() {
#pragma unroll
        for (int j = 0; j < T; ++j)
#pragma unroll
            for (int c = 0; c < C; ++c) hi[j][c] = lo[j][c] = 0.f;
#pragma unroll
        for (int p = 0; p < TP; ++p)
#pragma unroll
            for (int c = 0; c < C; ++c) bsum[p][c] = 0ull;
    }
    __device__ __forceinline__ void compute(const float *sb, int nrec, const float (*dc)[3], const float (*)[3],
                                            int kb0) {
        u64 xt[TP][3];
#pragma unroll
        for (int p = 0; p < TP; ++p) {
            const int r0 = tb[2 * p] - kb0, r1 = tb[2 * p + 1] - kb0;
            xt[p][0] = f2_pack(dc[r0][0] + tp[2 * p].x, dc[r1][0] + tp[2 * p + 1].x);
            xt[p][1] = f2_pack(dc[r0][1] + tp[2 * p].y, dc[r1][1] + tp[2 * p + 1].y);
            xt[p][2] = f2_pack(dc[r0][2] + tp[2 * p].z, dc[r1][2] + tp[2 * p + 1].z);
        }
        for (int s0 = 0; s0 < nrec; s0 += MFS_BS) {
            const int s1 = min(s0 + MFS_BS, nrec);
            u64 blk[TP][C];
#pragma unroll
            for (int p = 0; p < TP; ++p)
#pragma unroll
                for (int c = 0; c < C; ++c) blk[p][c] = 0ull;
            for (int s = s0; s < s1; s += 4) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    u64 rec[REC / 2];
#pragma unroll
                    for (int v = 0; v < REC / 4; ++v) {
                        const ulonglong2 f = reinterpret_cast<const ulonglong2 *>(sb + (s + q) * REC)[v];
                        rec[2 * v] = f.x;
                        rec[2 * v + 1] = f.y;
                    }
#pragma unroll
                    for (int p = 0; p < TP; ++p) {
                        const u64 dx = f2_sub(xt[p][0], rec[0]);
                        const u64 dy = f2_sub(xt[p][1], rec[1]);
                        const u64 dz = f2_sub(xt[p][2], rec[2]);
                        const u64 r2 = f2_fma(dx, dx, f2_fma(dy, dy, f2_mul(dz, dz)));
                        float a, b;
                        f2_unpack(r2, a, b);
                        const u64 ri = f2_pack(rsqrt_ftz(a), rsqrt_ftz(b));
#pragma unroll
                        for (int h = 0; h < NRHS; ++h) blk[p][h] = f2_fma(rec[3 + h], ri, blk[p][h]);
                    }
                }
            }
#pragma unroll
            for (int p = 0; p < TP; ++p)
#pragma unroll
                for (int c = 0; c < C; ++c) bsum[p][c] = f2_add(bsum[p][c], blk[p][c]);
        }
    }
    __device__ __forceinline__ void end_body(int body, bool include_self) {
#pragma unroll
        for (int p = 0; p < TP; ++p) {
            const bool k0 = include_self || (tb[2 * p] != body);
            const bool k1 = include_self || (tb[2 * p + 1] != body);
#pragma unroll
            for (int c = 0; c < C; ++c) {
                float v0, v1, s, e;
                f2_unpack(bsum[p][c], v0, v1);
                two_sum(hi[2 * p][c], k0 ? v0 : 0.f, s, e);
                hi[2 * p][c] = s;
                lo[2 * p][c] += e;
                two_sum(hi[2 * p + 1][c], k1 ? v1 : 0.f, s, e);
                hi[2 * p + 1][c] = s;
                lo[2 * p + 1][c] += e;
                bsum[p][c] = 0ull;
            }
        }
    }
    __device__ __forceinline__ float result(int j, int c, float &l) const {
        l = lo[j][c];
        return hi[j][c];
    }
};

// Centre gradient for the adjoint: per pair, the gradient with respect to r = x_i - y_j of
// w_i^T G(r) mu_j summed over right-hand sides,
//   [ w_c (r.mu) + mu_c (w.r) - (w.mu) r_c - 3 (w.r)(r.mu) r_c / r^2 ] / r^3   (x 1/(8 pi mu) later),
// accumulated per target like the pair sums (self pairs left out) and, at every source-body
// boundary, reduced over the CTA's targets into src_grad[body] (one FP64 atomic per component).
template <int NRHS, int T, int NT>
struct GradStokes : PolicyBase {
    static constexpr int D = 3;
    static constexpr int C = 3;  // one gradient 3-vector per target
    static constexpr int REC = rec_floats(3, NRHS, false);
    static constexpr int TPT = T;
    static constexpr int PSM = 0;
    float3 tp[T];
    int tb[T];
    float w[T][3 * NRHS];
    float hi[T][3], lo[T][3], bsum[T][3];

    __device__ __forceinline__ void init(float *, int) {}
    __device__ __forceinline__ void set_target(int j, float4 p) {
        tp[j] = make_float3(p.x, p.y, p.z);
        tb[j] = __float_as_int(p.w);
    }
    __device__ __forceinline__ void load_extra(int j, int idx, bool valid, const PairGeom &geo) {
#pragma unroll
        for (int h = 0; h < NRHS; ++h)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                w[j][3 * h + c] = valid ? geo.tgt_w[((size_t)h * geo.ntargets + idx) * 3 + c] : 0.f;
    }
    __device__ __forceinline__ void reset() {
#pragma unroll
        for (int j = 0; j < T; ++j)
#pragma unroll
            for (int c = 0; c < 3; ++c) hi[j][c] = lo[j][c] = bsum[j][c] = 0.f;
    }
    __device__ __forceinline__ void compute(const float *sb, int nrec, const float (*dc)[3], const float (*)[3],
                                            int kb0) {
        float3 xt[T];
#pragma unroll
        for (int j = 0; j < T; ++j) {
            const int r = tb[j] - kb0;
            xt[j] = make_float3(dc[r][0] + tp[j].x, dc[r][1] + tp[j].y, dc[r][2] + tp[j].z);
        }
        for (int s0 = 0; s0 < nrec; s0 += MFS_BS) {
            const int s1 = min(s0 + MFS_BS, nrec);
            float blk[T][3];
#pragma unroll
            for (int j = 0; j < T; ++j)
#pragma unroll
                for (int c = 0; c < 3; ++c) blk[j][c] = 0.f;
            for (int s = s0; s < s1; ++s) {
                float rec[REC];
#pragma unroll
                for (int v = 0; v < REC / 4; ++v) {
                    const float4 f = reinterpret_cast<const float4 *>(sb + s * REC)[v];
                    rec[4 * v + 0] = f.x;
                    rec[4 * v + 1] = f.y;
                    rec[4 * v + 2] = f.z;
                    rec[4 * v + 3] = f.w;
                }
#pragma unroll
                for (int j = 0; j < T; ++j) {
                    const float dx = xt[j].x - rec[0], dy = xt[j].y - rec[1], dz = xt[j].z - rec[2];
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    const float ri = rsqrt_ftz(r2);
                    const float ri2 = ri * ri, ri3 = ri * ri2;
#pragma unroll
                    for (int h = 0; h < NRHS; ++h) {
                        const float mx = rec[3 + 3 * h], my = rec[4 + 3 * h], mz = rec[5 + 3 * h];
                        const float wx = w[j][3 * h], wy = w[j][3 * h + 1], wz = w[j][3 * h + 2];
                        const float wm = fmaf(wx, mx, fmaf(wy, my, wz * mz));
                        const float wr = fmaf(wx, dx, fmaf(wy, dy, wz * dz));
                        const float rm = fmaf(dx, mx, fmaf(dy, my, dz * mz));
                        const float q = -fmaf(3.f * wr * rm, ri2, wm);
                        blk[j][0] = fmaf(fmaf(dx, q, fmaf(wx, rm, mx * wr)), ri3, blk[j][0]);
                        blk[j][1] = fmaf(fmaf(dy, q, fmaf(wy, rm, my * wr)), ri3, blk[j][1]);
                        blk[j][2] = fmaf(fmaf(dz, q, fmaf(wz, rm, mz * wr)), ri3, blk[j][2]);
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < T; ++j)
#pragma unroll
                for (int c = 0; c < 3; ++c) bsum[j][c] += blk[j][c];
        }
    }
    // All threads of the CTA call this together (the source-body boundary is CTA-uniform).
    __device__ __forceinline__ void source_side(int body, bool include_self, double *src_grad) {
        if (!src_grad) return;  // no per-source-body reduction (a kernel argument: CTA-uniform)
        __shared__ float red[NT / 32][3];
        float s[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int j = 0; j < T; ++j)
            if (include_self || tb[j] != body)
#pragma unroll
                for (int c = 0; c < 3; ++c) s[c] += bsum[j][c];
#pragma unroll
        for (int c = 0; c < 3; ++c)
            for (int o = 16; o > 0; o >>= 1) s[c] += __shfl_xor_sync(0xffffffffu, s[c], o);
        if ((threadIdx.x & 31) == 0)
#pragma unroll
            for (int c = 0; c < 3; ++c) red[threadIdx.x >> 5][c] = s[c];
        __syncthreads();
        if (threadIdx.x < 3) {
            float v = 0.f;
            for (int q = 0; q < NT / 32; ++q) v += red[q][threadIdx.x];
            atomicAdd(&src_grad[3 * body + threadIdx.x], (double)v);
        }
        __syncthreads();
    }
    __device__ __forceinline__ void end_body(int body, bool include_self) {
#pragma unroll
        for (int j = 0; j < T; ++j) {
            const bool keep = include_self || (tb[j] != body);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float s, e;
                two_sum(hi[j][c], keep ? bsum[j][c] : 0.f, s, e);
                hi[j][c] = s;
                lo[j][c] += e;
                bsum[j][c] = 0.f;
            }
        }
    }
    __device__ __forceinline__ float result(int j, int c, float &l) const {
        l = lo[j][c];
        return hi[j][c];
    }
};

// Pressure and surface traction of the Stokeslet representation at evaluation points (Eq. traction),
// as a pair-kernel policy: for a target x with unit normal n (geo.tgt_w, FP32 [ntargets][3]; zero:
// pressure only) and a source y of strength lambda, r = x - y,
//   p   = (r . lambda) / r^3                  (x 1/(4 pi) in the epilogue)
//   T   = r (r . n)(r . lambda) / r^5         (x -3/(4 pi) afterwards),
// both independent of the viscosity; four outputs per right-hand side (p, T_x, T_y, T_z).  T targets
// per thread, sources as the pair sums' plain records; all pairs of the suspension (self included).
template <int NRHS, int T, int NT>
struct StressStokes : PolicyBase {
    static constexpr int D = 4;
    static constexpr int C = 4 * NRHS;
    static constexpr int REC = rec_floats(3, NRHS, false);
    static constexpr int TPT = T;
    static constexpr int PSM = 0;
    float3 tp[T];
    int tb[T];
    float nv[T][3];
    float hi[T][C], lo[T][C], bsum[T][C];

    __device__ __forceinline__ void init(float *, int) {}
    __device__ __forceinline__ void set_target(int j, float4 p) {
        tp[j] = make_float3(p.x, p.y, p.z);
        tb[j] = __float_as_int(p.w);
    }
    __device__ __forceinline__ void load_extra(int j, int idx, bool valid, const PairGeom &geo) {
#pragma unroll
        for (int c = 0; c < 3; ++c) nv[j][c] = (valid && geo.tgt_w) ? geo.tgt_w[(size_t)idx * 3 + c] : 0.f;
    }
    __device__ __forceinline__ void reset() {
#pragma unroll
        for (int j = 0; j < T; ++j)
#pragma unroll
            for (int c = 0; c < C; ++c) hi[j][c] = lo[j][c] = bsum[j][c] = 0.f;
    }
    __device__ __forceinline__ void compute(const float *sb, int nrec, const float (*dc)[3], const float (*)[3],
                                            int kb0) {
        float3 xt[T];
#pragma unroll
        for (int j = 0; j < T; ++j) {
            const int r = tb[j] - kb0;
            xt[j] = make_float3(dc[r][0] + tp[j].x, dc[r][1] + tp[j].y, dc[r][2] + tp[j].z);
        }
        for (int s0 = 0; s0 < nrec; s0 += MFS_BS) {
            const int s1 = min(s0 + MFS_BS, nrec);
            float blk[T][C];
#pragma unroll
            for (int j = 0; j < T; ++j)
#pragma unroll
                for (int c = 0; c < C; ++c) blk[j][c] = 0.f;
            for (int s = s0; s < s1; ++s) {
                float rec[REC];
#pragma unroll
                for (int v = 0; v < REC / 4; ++v) {
                    const float4 f = reinterpret_cast<const float4 *>(sb + s * REC)[v];
                    rec[4 * v + 0] = f.x;
                    rec[4 * v + 1] = f.y;
                    rec[4 * v + 2] = f.z;
                    rec[4 * v + 3] = f.w;
                }
#pragma unroll
                for (int j = 0; j < T; ++j) {
                    const float rx = xt[j].x - rec[0], ry = xt[j].y - rec[1], rz = xt[j].z - rec[2];
                    const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
                    const float ir = rsqrt_ftz(r2);
                    const float ir2 = ir * ir, ir3 = ir2 * ir;
                    const float rn = fmaf(rx, nv[j][0], fmaf(ry, nv[j][1], rz * nv[j][2]));
                    const float q5 = rn * ir3 * ir2;
#pragma unroll
                    for (int h = 0; h < NRHS; ++h) {
                        const float rl = fmaf(rx, rec[3 + 3 * h], fmaf(ry, rec[4 + 3 * h], rz * rec[5 + 3 * h]));
                        const float q = rl * q5;
                        blk[j][4 * h] = fmaf(rl, ir3, blk[j][4 * h]);
                        blk[j][4 * h + 1] = fmaf(rx, q, blk[j][4 * h + 1]);
                        blk[j][4 * h + 2] = fmaf(ry, q, blk[j][4 * h + 2]);
                        blk[j][4 * h + 3] = fmaf(rz, q, blk[j][4 * h + 3]);
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < T; ++j)
#pragma unroll
                for (int c = 0; c < C; ++c) bsum[j][c] += blk[j][c];
        }
    }
    __device__ __forceinline__ void end_body(int body, bool include_self) {
#pragma unroll
        for (int j = 0; j < T; ++j) {
            const bool keep = include_self || (tb[j] != body);
#pragma unroll
            for (int c = 0; c < C; ++c) {
                float s, e;
                two_sum(hi[j][c], keep ? bsum[j][c] : 0.f, s, e);
                hi[j][c] = s;
                lo[j][c] += e;
                bsum[j][c] = 0.f;
            }
        }
    }
    __device__ __forceinline__ float result(int j, int c, float &l) const {
        l = lo[j][c];
        return hi[j][c];
    }
};

// ---------------------------------------------------------------------------
// Compensated (double-FP32) pair sums: every pair term is carried as an unevaluated FP32 sum
// hi + lo, accurate to about 2^-28 of its size instead of FP32's 2^-24, and summed per target with
// TwoSum.  The FP32 policies above lose about eps_32 |G| |lambda| per pair; when the strengths are
// large and their fields cancel (the pseudo-inverse applied to a rough gamma, Eq. pseudo), that
// rounding noise is larger than 1e-6 of the result.  Exactness is arranged, not emulated:
//  * r = a + e: the body-local coordinates and the centre difference are split at multiples of
//    1/MFS_XGRID, so a = (dc_hi + x_hi) - y_hi is exact and |a|^2 is exact for |a| < 32;
//  * lambda = L + l with L an 11-bit block-floating value (one exponent per source), so a . L is
//    exact (three products of 11-bit integers on one scale) for |a| < 32;
//  * 1/r from the MUFU estimate y0 and the exactly computed residual h = 1 - r^2 y0^2 (one Newton
//    step carried in the low part);
//  * products and sums that feed the high part are split exactly (FMA product error, TwoSum).
// The intrinsics __fmul_rn / __fadd_rn keep the compiler from contracting the error-free
// transformations into FMAs.  Beyond |a| = 32 the squares and dot products round once (FP32
// accuracy for far pairs, whose terms are smaller by 1/r).
// Record: [y_hi(3) y_lo(3)] then per right-hand side Stokes [L(3) l(3) lambda_f32(3)], Laplace
// [lambda_hi lambda_lo].
// ---------------------------------------------------------------------------
__device__ __forceinline__ void df_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (hi, lo) += (th, tl)
__device__ __forceinline__ void df_acc(float &hi, float &lo, float th, float tl) {
    float s, e;
    df_two_sum(hi, th, s, e);
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(e, tl));
}

template <int D, int NRHS>
__host__ __device__ constexpr int comp_rec_floats() {
    return (6 + (D == 3 ? 9 : 2) * NRHS + 3) / 4 * 4;
}

template <int D, int NRHS, int T, int NT>
struct Comp : PolicyBase {
    static constexpr int DIM = D;
    static constexpr int C = D * NRHS;
    static constexpr int REC = comp_rec_floats<D, NRHS>();
    static constexpr int TPT = T;
    static constexpr int PSM = 0;
    static constexpr bool GRID_DC = true;
    float xh[T][3], xl[T][3];
    int tb[T];
    float Sh[T][C], Sl[T][C];  // finished source bodies (self left out)
    float Bh[T][C], Bl[T][C];  // the current source body

    __device__ __forceinline__ void init(float *, int) {}
    __device__ __forceinline__ void set_target(int j, float4 p) { tb[j] = __float_as_int(p.w); }
    __device__ __forceinline__ void load_extra(int j, int idx, bool, const PairGeom &geo) {
        const float4 h = geo.tgt_hi[idx], l = geo.tgt_lo[idx];
        xh[j][0] = h.x;
        xh[j][1] = h.y;
        xh[j][2] = h.z;
        xl[j][0] = l.x;
        xl[j][1] = l.y;
        xl[j][2] = l.z;
    }
    __device__ __forceinline__ void reset() {
#pragma unroll
        for (int j = 0; j < T; ++j)
#pragma unroll
            for (int c = 0; c < C; ++c) Sh[j][c] = Sl[j][c] = Bh[j][c] = Bl[j][c] = 0.f;
    }
    __device__ __forceinline__ void compute(const float *sb, int nrec, const float (*dch)[3], const float (*dcl)[3],
                                            int kb0) {
        float th_[T][3], tl_[T][3];  // target relative to the source body's centre, hi (exact) + lo
#pragma unroll
        for (int j = 0; j < T; ++j) {
            const int r = tb[j] - kb0;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                th_[j][c] = __fadd_rn(dch[r][c], xh[j][c]);
                tl_[j][c] = __fadd_rn(dcl[r][c], xl[j][c]);
            }
        }
#pragma unroll 1
        for (int s = 0; s < nrec; ++s) {
            float rec[REC];
#pragma unroll
            for (int v = 0; v < REC / 4; ++v) {
                const float4 f = reinterpret_cast<const float4 *>(sb + s * REC)[v];
                rec[4 * v + 0] = f.x;
                rec[4 * v + 1] = f.y;
                rec[4 * v + 2] = f.z;
                rec[4 * v + 3] = f.w;
            }
#pragma unroll
            for (int j = 0; j < T; ++j) {
                float a[3], e[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    a[c] = __fsub_rn(th_[j][c], rec[c]);      // exact (grid)
                    e[c] = __fsub_rn(tl_[j][c], rec[3 + c]);  // small
                }
                // r^2 = A + B: A = |a|^2 exact, B = e . (2a + e)
                const float A = __fmaf_rn(a[0], a[0], __fmaf_rn(a[1], a[1], __fmul_rn(a[2], a[2])));
                const float w0 = __fmaf_rn(2.f, a[0], e[0]), w1 = __fmaf_rn(2.f, a[1], e[1]),
                            w2 = __fmaf_rn(2.f, a[2], e[2]);
                const float B = __fmaf_rn(e[0], w0, __fmaf_rn(e[1], w1, __fmul_rn(e[2], w2)));
                const float r2h = __fadd_rn(A, B);
                const float r2l = __fadd_rn(__fsub_rn(A, r2h), B);
                // 1/r = y0 (1 + h/2), 1/r^2 = (q + qe)(1 + h), h = 1 - r^2 y0^2 computed exactly to first order
                const float y0 = rsqrt_ftz(r2h);
                const float q = __fmul_rn(y0, y0);
                const float qe = __fmaf_rn(y0, y0, -q);
                const float Pp = __fmul_rn(r2h, q);
                const float Pe = __fmaf_rn(r2h, q, -Pp);
                float h = __fsub_rn(__fsub_rn(1.f, Pp), Pe);
                h = __fmaf_rn(-r2h, qe, h);
                h = __fmaf_rn(-r2l, q, h);
                const float ril = __fmul_rn(__fmul_rn(0.5f, y0), h);
#pragma unroll
                for (int rh = 0; rh < NRHS; ++rh) {
                    if constexpr (D == 3) {
                        const float *L = rec + 6 + 9 * rh, *l = L + 3, *M = L + 6;
                        // r . lambda = (a . L) [exact] + (a . l + e . lambda)
                        const float doth = __fmaf_rn(a[0], L[0], __fmaf_rn(a[1], L[1], __fmul_rn(a[2], L[2])));
                        const float dotl = __fmaf_rn(
                            a[0], l[0],
                            __fmaf_rn(a[1], l[1],
                                      __fmaf_rn(a[2], l[2],
                                                __fmaf_rn(e[0], M[0], __fmaf_rn(e[1], M[1], __fmul_rn(e[2], M[2]))))));
                        // s = (r . lambda) / r^2 = sch + scl
                        const float sch = __fmul_rn(q, doth);
                        float scl = __fmaf_rn(q, doth, -sch);
                        scl = __fmaf_rn(q, __fmaf_rn(h, doth, dotl), scl);
                        scl = __fmaf_rn(qe, doth, scl);
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            // v = lambda + s r, then the term v / r
                            const float p = __fmul_rn(sch, a[c]);
                            const float pe = __fmaf_rn(sch, a[c], -p);
                            float vh, err;
                            df_two_sum(L[c], p, vh, err);
                            float vl = __fmaf_rn(sch, e[c], l[c]);
                            vl = __fmaf_rn(scl, a[c], vl);
                            vl = __fmaf_rn(scl, e[c], vl);
                            vl = __fadd_rn(__fadd_rn(vl, pe), err);
                            const float tH = __fmul_rn(y0, vh);
                            const float tE = __fmaf_rn(y0, vh, -tH);
                            const float tL = __fmaf_rn(y0, vl, __fmaf_rn(ril, vh, tE));
                            df_acc(Bh[j][3 * rh + c], Bl[j][3 * rh + c], tH, tL);
                        }
                    } else {
                        const float lh = rec[6 + 2 * rh], ll = rec[7 + 2 * rh];
                        const float tH = __fmul_rn(lh, y0);
                        const float tE = __fmaf_rn(lh, y0, -tH);
                        const float tL = __fmaf_rn(ll, y0, __fmaf_rn(lh, ril, tE));
                        df_acc(Bh[j][rh], Bl[j][rh], tH, tL);
                    }
                }
            }
        }
    }
    __device__ __forceinline__ void end_body(int body, bool include_self) {
#pragma unroll
        for (int j = 0; j < T; ++j) {
            const bool keep = include_self || (tb[j] != body);
#pragma unroll
            for (int c = 0; c < C; ++c) {
                if (keep) df_acc(Sh[j][c], Sl[j][c], Bh[j][c], Bl[j][c]);
                Bh[j][c] = Bl[j][c] = 0.f;
            }
        }
    }
    __device__ __forceinline__ float result(int j, int c, float &l) const {
        l = Sl[j][c];
        return Sh[j][c];
    }
};
template <int NRHS, int T, int NT>
using CompStokes = Comp<3, NRHS, T, NT>;
template <int NRHS, int T, int NT>
using CompLaplace = Comp<1, NRHS, T, NT>;

// ---------------------------------------------------------------------------
// The persistent stream-K kernel
// ---------------------------------------------------------------------------
template <class Pol, int NT>
struct StageCfg {
    static constexpr int REC = Pol::REC;
    // 16 KB stages; 12 KB when the policy keeps per-target state in shared memory (occupancy)
    static constexpr int STAGE_BYTES = Pol::PSM ? 12288 : 16384;
    static constexpr int STAGE_REC = (STAGE_BYTES / (REC * 4)) / MFS_BS * MFS_BS;
    static constexpr int STAGE_BLOCKS = STAGE_REC / MFS_BS;
    static constexpr int SMEM = 2 * STAGE_REC * REC * 4 + Pol::PSM * NT * 4;
};

// The same register-state policy compiled for more resident CTAs per SM: at most
// 65536 / (NT * MINB) registers per thread (more warps, possibly less interleaving); the autotuner
// decides per geometry.
template <int NRHS, int TP, int NT>
struct PackedStokesRegB4 : PackedStokesReg<NRHS, TP, NT> {
    static constexpr int MINB = 4;
};
template <int NRHS, int TP, int NT>
struct PackedStokesRegB5 : PackedStokesReg<NRHS, TP, NT> {
    static constexpr int MINB = 5;
};
template <int NRHS, int TP, int NT>
struct PackedStokesB4 : PackedStokes<NRHS, TP, NT> {
    static constexpr int MINB = 4;
};
template <int NRHS, int TP, int NT>
struct PackedStokesB5 : PackedStokes<NRHS, TP, NT> {
    static constexpr int MINB = 5;
};


template <class Pol, int NT, int MINB = Pol::MINB>
__global__ void __launch_bounds__(NT, MINB) pair_sum_kernel(PairGeom geo, PairWork work, int *err) {
    using Cfg = StageCfg<Pol, NT>;
    constexpr int REC = Cfg::REC, SREC = Cfg::STAGE_REC, C = Pol::C, TPT = Pol::TPT;
    extern __shared__ __align__(128) float smem[];
    __shared__ float dcs[2][MFS_MAX_TILE_BODIES][3];
    __shared__ float dcl[Pol::GRID_DC ? 2 : 1][Pol::GRID_DC ? MFS_MAX_TILE_BODIES : 1][3];
    __shared__ __align__(8) uint64_t bars[2];

    const int g = blockIdx.x;
    const long long W = work.total_units;
    const long long ubeg = (long long)g * W / work.G;
    const long long uend = (long long)(g + 1) * W / work.G;
    if (ubeg >= uend) return;
    const int tid = threadIdx.x;
    const long long wait_limit = 1ll << 22;

    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncthreads();

    const PairTile *tiles = work.tiles;
    Stage cur = make_stage(tiles, work.ntiles, geo, ubeg, uend, Cfg::STAGE_BLOCKS, -1);
    const int first_tile = cur.tile;
    if (tid == 0) {
        mbar_arrive_expect_tx(&bars[0], (uint32_t)(cur.nrec * REC * 4));
        bulk_g2s(smem, geo.src + (size_t)cur.rec0 * REC, (uint32_t)(cur.nrec * REC * 4), &bars[0]);
    }

    Pol pol;
    pol.init(smem + 2 * SREC * REC, tid);
    PairTile tl = tiles[cur.tile];
    long long seg_begin = ubeg;
    auto load_targets = [&](const PairTile &t_) {
#pragma unroll
        for (int j = 0; j < TPT; ++j) {
            int idx = t_.t0 + tid + j * NT;
            const bool in_tile = idx < t_.t1;
            if (!in_tile) idx = t_.t1 - 1;  // a clamped duplicate: computed, never written
            pol.set_target(j, geo.tgt[idx]);
            pol.load_extra(j, idx, in_tile, geo);
        }
        pol.reset();
    };
    load_targets(tl);

    int si = 0;
    while (true) {
        const int buf = si & 1;
        Stage nxt;
        nxt.tile = -1;
        const long long unext = cur.u + cur.nblk;
        if (unext < uend) {
            int hint = cur.tile;
            if (unext >= tiles[hint].u1) {  // next non-empty tile
                ++hint;
                while (hint < work.ntiles && tiles[hint].u1 <= unext) ++hint;
                if (hint >= work.ntiles) hint = -1;
            }
            nxt = make_stage(tiles, work.ntiles, geo, unext, uend, Cfg::STAGE_BLOCKS, hint);
            if (tid == 0) {
                mbar_arrive_expect_tx(&bars[buf ^ 1], (uint32_t)(nxt.nrec * REC * 4));
                bulk_g2s(smem + (buf ^ 1) * SREC * REC, geo.src + (size_t)nxt.rec0 * REC,
                         (uint32_t)(nxt.nrec * REC * 4), &bars[buf ^ 1]);
            }
        }
        // centre offsets of the tile's target bodies relative to this stage's source body
        for (int q = tid; q < tl.nb * 3; q += NT) {  // up to MFS_MAX_TILE_BODIES * 3 entries, NT may be fewer
            const int kb = tl.kb0 + q / 3, c = q % 3;
            const double d = geo.centres[kb * 3 + c] - geo.centres[cur.body * 3 + c];
            if constexpr (Pol::GRID_DC) {  // d = hi + lo with hi on the coordinate grid (exact in FP32)
                const double dh = rint(d * MFS_XGRID) / MFS_XGRID;
                dcs[buf][q / 3][c] = (float)dh;
                dcl[buf][q / 3][c] = (float)(d - dh);
            } else {
                dcs[buf][q / 3][c] = (float)d;
            }
        }
        const bool ok = mbar_wait_bounded(&bars[buf], (uint32_t)((si >> 1) & 1), err, wait_limit);
        if (__syncthreads_or(!ok)) {
            // give the other buffer's copy (if any) a bounded chance to land, then leave
            if (nxt.tile >= 0) mbar_wait_bounded(&bars[buf ^ 1], (uint32_t)(((si + 1) >> 1) & 1), nullptr, wait_limit);
            return;
        }

        pol.compute(smem + buf * SREC * REC, cur.nrec, dcs[buf], dcl[Pol::GRID_DC ? buf : 0], tl.kb0);

        // end of a source body (for this tile): fold into (hi, lo), leaving self pairs out
        if ((nxt.tile < 0) || nxt.tile != cur.tile || nxt.body != cur.body) {
            pol.source_side(cur.body, work.include_self, work.src_grad);  // CTA-uniform (may synchronise)
            pol.end_body(cur.body, work.include_self);
        }
        // end of this CTA's segment of the tile: write the tile's result
        if ((nxt.tile < 0) || nxt.tile != cur.tile) {
            const long long seg_end = cur.u + cur.nblk;
            const bool whole = (seg_begin == tl.u0) && (seg_end == tl.u1);
#pragma unroll
            for (int j = 0; j < TPT; ++j) {
                const int idx = tl.t0 + tid + j * NT;
                if (idx < tl.t1) {
                    double *dst;
                    if (whole) {
                        dst = work.direct + (size_t)idx * C;
                    } else {
                        const int slot = (cur.tile == first_tile) ? 0 : 1;
                        dst = work.partial + ((size_t)(g * 2 + slot) * work.tile_targets + (idx - tl.t0)) * C;
                    }
#pragma unroll
                    for (int c = 0; c < C; ++c) {
                        float l;
                        const float h = pol.result(j, c, l);
                        dst[c] = (double)h + (double)l;
                    }
                }
            }
            if (nxt.tile >= 0) {
                tl = tiles[nxt.tile];
                seg_begin = nxt.u;
                load_targets(tl);
            }
        }
        __syncthreads();  // all reads of `buf` and dcs[buf] done before they are refilled
        if (nxt.tile < 0) break;
        cur = nxt;
        ++si;
    }
}

// Epilogue: out[r][t][d] = beta * base[r][t][d] + scale * (sum of the CTA shares of target t).
// Blocks (tile, y): the CTAs that share the tile and the slot each wrote (0: the tile is where the
// CTA's range starts, 1: where it ends) are found once per block; the tile's (target, component)
// entries, contiguous in every array for one right-hand side, are spread over the gridDim.y blocks,
// and S consecutive lanes share an entry: lane k adds shares k, k + S, ... in that order (eight loads
// in flight), then the S partial sums meet in a fixed xor-shuffle tree.  The order is fixed, so the
// result is deterministic; with S = 1 it is the plain sum in CTA order.  Tiles shared by many CTAs
// (the far-field upward sums of the top nodes) are why S and the y blocks exist.
template <int D, int NRHS>
__global__ void __launch_bounds__(1024) pair_epilogue_kernel(PairWork work, const double *base, double beta, double scale, double *out,
                                     int ntargets, int S) {
    constexpr int C = D * NRHS;
    constexpr int MAXS = 256;
    __shared__ signed char slot_of[MAXS];  // per CTA gA + i: slot 0 / 1, -1 for an empty range
    const PairTile tl = work.tiles[blockIdx.x];
    const long long W = work.total_units;
    const int ns = (tl.gA >= 0 && tl.gA != tl.gB) ? tl.gB - tl.gA + 1 : 0;
    for (int i = threadIdx.x; i < ns && i < MAXS; i += blockDim.x) {
        const int gg = tl.gA + i;
        const long long b0 = (long long)gg * W / work.G, b1 = (long long)(gg + 1) * W / work.G;
        slot_of[i] = b0 >= b1 ? -1 : (b0 >= tl.u0 ? 0 : 1);
    }
    __syncthreads();
    const int E = (tl.t1 - tl.t0) * C;
    const int per_block = blockDim.x / S, sub = threadIdx.x % S;
    const size_t per_slot = (size_t)work.tile_targets * C;
    // the round count depends on the block only, so every lane of a warp reaches the shuffles
    for (int q0 = blockIdx.y * per_block; q0 < E; q0 += gridDim.y * per_block) {
        const int q = q0 + (int)threadIdx.x / S;
        double v = 0.0;
        if (q < E && tl.gA >= 0) {
            const int t = tl.t0 + q / C, c = q % C;
            if (tl.gA == tl.gB) {
                if (sub == 0) v = work.direct[(size_t)t * C + c];
            } else {
                const size_t within = (size_t)(t - tl.t0) * C + c;
                auto share = [&](int i) -> double {
                    int slot;
                    if (i < MAXS) {
                        slot = slot_of[i];
                    } else {
                        const int gg = tl.gA + i;
                        const long long b0 = (long long)gg * W / work.G, b1 = (long long)(gg + 1) * W / work.G;
                        slot = b0 >= b1 ? -1 : (b0 >= tl.u0 ? 0 : 1);
                    }
                    return slot < 0 ? 0.0 : work.partial[(size_t)((tl.gA + i) * 2 + slot) * per_slot + within];
                };
                int i = sub;
                for (; i + 7 * S < ns; i += 8 * S) {
                    double p[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) p[u] = share(i + u * S);
#pragma unroll
                    for (int u = 0; u < 8; ++u) v += p[u];
                }
                for (; i < ns; i += S) v += share(i);
            }
        }
        for (int o = S / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (q < E && sub == 0) {
            const int t = tl.t0 + q / C, c = q % C;
            const int h = c / D, d = c % D;
            const size_t o = ((size_t)h * ntargets + (work.tperm ? work.tperm[t] : t)) * D + d;
            const double b = base ? beta * base[o] : 0.0;
            out[o] = b + scale * v;
        }
    }
}

// Pack proxy strengths (FP64 [nrhs][sum_N][D], body-local rotated positions) into FP32 records.
// Padding records (beyond N_k in each body) sit at the body centre with zero strength, which
// contributes exactly zero to every target off that centre.
template <int D, int NRHS, bool PACKED>
__global__ void pack_sources_kernel(const float4 *src_pos, const int *src_pt_of_rec, const double *strength, int nsrc,
                                    int nrec, float *records) {
    constexpr int NV = 3 + D * NRHS, REC = rec_floats(D, NRHS, PACKED);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrec) return;
    float v[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) v[c] = 0.f;
    const int p = src_pt_of_rec[i];
    if (p >= 0) {
        const float4 y = src_pos[p];
        v[0] = y.x;
        v[1] = y.y;
        v[2] = y.z;
#pragma unroll
        for (int h = 0; h < NRHS; ++h)
#pragma unroll
            for (int d = 0; d < D; ++d) v[3 + h * D + d] = (float)strength[((size_t)h * nsrc + p) * D + d];
    }
    float r[REC];
#pragma unroll
    for (int c = 0; c < REC; ++c) r[c] = 0.f;
#pragma unroll
    for (int c = 0; c < NV; ++c) {
        if (PACKED) {
            r[2 * c] = v[c];
            r[2 * c + 1] = v[c];
        } else {
            r[c] = v[c];
        }
    }
    float4 *o = reinterpret_cast<float4 *>(records + (size_t)i * REC);
#pragma unroll
    for (int q = 0; q < REC / 4; ++q) o[q] = make_float4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
}

// Records of the compensated policies (layout above) from FP64 body-local positions and strengths.
// The block-floating part L of a Stokeslet strength keeps 11 significant bits on the scale of its
// largest component; l = lambda - L is rounded to FP32 (relative 2^-24 of a number below 2^-11 of
// lambda).  Padding records (rec_pt = -1) are all zero: the body centre with zero strength.
template <int D, int NRHS>
__global__ void pack_sources_comp_kernel(const double *src_local64, const int *src_pt_of_rec, const double *strength,
                                         int nsrc, int nrec, float *records) {
    constexpr int REC = comp_rec_floats<D, NRHS>();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrec) return;
    float r[REC];
#pragma unroll
    for (int c = 0; c < REC; ++c) r[c] = 0.f;
    const int p = src_pt_of_rec[i];
    if (p >= 0) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double y = src_local64[3 * (size_t)p + c];
            const double yh = rint(y * MFS_XGRID) / MFS_XGRID;
            r[c] = (float)yh;
            r[3 + c] = (float)(y - yh);
        }
#pragma unroll
        for (int h = 0; h < NRHS; ++h) {
            if (D == 3) {
                double lam[3], m = 0.0;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    lam[c] = strength[((size_t)h * nsrc + p) * 3 + c];
                    m = fmax(m, fabs(lam[c]));
                }
                double unit = 0.0;
                if (m > 0.0) {
                    int ex = 0;
                    frexp(m, &ex);  // m < 2^ex
                    unit = ldexp(1.0, ex - 11);
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const double L = unit > 0.0 ? rint(lam[c] / unit) * unit : 0.0;
                    r[6 + 9 * h + c] = (float)L;
                    r[9 + 9 * h + c] = (float)(lam[c] - L);
                    r[12 + 9 * h + c] = (float)lam[c];
                }
            } else {
                const double lam = strength[(size_t)h * nsrc + p];
                const float lh = (float)lam;
                r[6 + 2 * h] = lh;
                r[7 + 2 * h] = (float)(lam - (double)lh);
            }
        }
    }
    float4 *o = reinterpret_cast<float4 *>(records + (size_t)i * REC);
#pragma unroll
    for (int q = 0; q < REC / 4; ++q) o[q] = make_float4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
}

// ---------------------------------------------------------------------------
// Host side: variant table
// ---------------------------------------------------------------------------
template <class Pol, int NT, int MINB = Pol::MINB>
static cudaError_t launch_variant(const PairGeom &geo, const PairWork &work, int *err, cudaStream_t st) {
    using Cfg = StageCfg<Pol, NT>;
    auto kern = pair_sum_kernel<Pol, NT, MINB>;
    // the shared-memory limit is a per-device function attribute: set once on each device
    static std::atomic<unsigned long long> attr_devices{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0ull;
    if (!bit || !(attr_devices.load() & bit)) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
        if (e != cudaSuccess) return e;
        attr_devices.fetch_or(bit);
    }
    kern<<<work.G, NT, Cfg::SMEM, st>>>(geo, work, err);
    return cudaGetLastError();
}

template <class Pol, int NT, int MINB = Pol::MINB>
static int occupancy_variant() {
    using Cfg = StageCfg<Pol, NT>;
    auto kern = pair_sum_kernel<Pol, NT, MINB>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, NT, Cfg::SMEM) != cudaSuccess) return 0;
    return blocks;
}

// Scalar S(D, nrhs, targets per thread, threads); packed Stokes P(nrhs, target pairs per thread, threads)
// Scalar S(D, nrhs, T, NT); packed Stokes P(policy, nrhs, target pairs per thread, NT);
// centre-gradient G(nrhs, T, NT) for the adjoint; compensated X(policy, nrhs, T, NT) (precision = 3)
#define MFS_VARIANTS(S, P, G, X, Q)  \
    S(3, 1, 4, 128)         \
    S(3, 1, 2, 128)         \
    S(3, 1, 4, 256)         \
    S(3, 1, 2, 256)         \
    S(3, 2, 2, 128)         \
    S(3, 3, 2, 128)         \
    S(3, 4, 2, 128)         \
    S(3, 4, 1, 128)         \
    S(1, 1, 4, 128)         \
    S(1, 1, 8, 128)         \
    S(1, 1, 4, 256)         \
    S(1, 2, 4, 128)         \
    S(1, 3, 4, 128)         \
    S(1, 4, 4, 128)         \
    P(PackedStokesReg, 1, 1, 128) \
    P(PackedStokesReg, 1, 2, 128) \
    P(PackedStokesRegB4, 1, 2, 128) \
    P(PackedStokesRegB5, 1, 2, 128) \
    P(PackedStokesRegB4, 2, 1, 128) \
    P(PackedStokesRegB4, 4, 1, 128) \
    P(PackedStokesReg, 1, 1, 256) \
    P(PackedStokesReg, 2, 1, 128) \
    P(PackedStokesReg, 4, 1, 128) \
    P(PackedStokes, 1, 2, 128)    \
    P(PackedStokesB4, 1, 2, 128)  \
    P(PackedStokesB5, 1, 2, 128)  \
    P(PackedStokesB4, 1, 3, 128)  \
    P(PackedStokes, 1, 2, 256)    \
    P(PackedStokes, 1, 3, 128)    \
    P(PackedStokes, 1, 3, 64)     \
    P(PackedStokes, 1, 3, 256)    \
    P(PackedStokes, 1, 4, 128)    \
    P(PackedStokes, 1, 4, 64)     \
    P(PackedStokes, 2, 1, 128)    \
    P(PackedStokes, 4, 1, 128)    \
    P(PackedStokes, 4, 2, 64)     \
    P(PackedStokes, 4, 1, 64)     \
    P(PackedStokes, 2, 2, 64)     \
    P(PackedStokes, 1, 5, 64)     \
    P(PackedStokes, 1, 5, 128)    \
    P(PackedStokes, 1, 6, 64)     \
    P(PackedStokesOA, 1, 4, 64)   \
    P(PackedStokesOA, 1, 6, 64)   \
    P(PackedStokesOA, 1, 5, 64)   \
    P(PackedLaplaceReg, 1, 2, 128) \
    P(PackedLaplaceReg, 1, 4, 128) \
    P(PackedLaplaceReg, 1, 2, 256) \
    P(PackedLaplaceReg, 2, 2, 128) \
    P(PackedLaplaceReg, 4, 2, 128) \
    P(PackedLaplaceReg, 1, 8, 64)  \
    G(1, 4, 128)                  \
    G(2, 2, 128)                  \
    G(3, 2, 128)                  \
    G(4, 2, 128)                  \
    X(CompStokes, 1, 2, 128)      \
    X(CompStokes, 1, 4, 128)      \
    X(CompStokes, 1, 2, 256)      \
    X(CompStokes, 2, 2, 128)      \
    X(CompStokes, 3, 2, 128)      \
    X(CompStokes, 4, 1, 128)      \
    X(CompLaplace, 1, 4, 128)     \
    X(CompLaplace, 1, 2, 128)     \
    X(CompLaplace, 2, 2, 128)     \
    X(CompLaplace, 3, 2, 128)     \
    X(CompLaplace, 4, 2, 128)     \
    Q(1, 4, 128)                  \
    Q(2, 2, 128)                  \
    Q(3, 2, 128)                  \
    Q(4, 2, 128)

static const PairVariant kVariants[] = {
#define S(D_, R_, T_, N_) {D_, R_, T_, N_, N_ * T_, 0, 0, 0, "Scalar<" #D_ "," #R_ "," #T_ "," #N_ ">"},
#define P(POL_, R_, TP_, N_) \
    {POL_<R_, TP_, N_>::D, R_, 2 * TP_, N_, N_ * 2 * TP_, 1, 0, 0, #POL_ "<" #R_ "," #TP_ "," #N_ ">"},
#define G(R_, T_, N_) {3, R_, T_, N_, N_ * T_, 0, 1, 0, "GradStokes<" #R_ "," #T_ "," #N_ ">"},
#define X(POL_, R_, T_, N_) \
    {POL_<R_, T_, N_>::DIM, R_, T_, N_, N_ * T_, 0, 0, 1, #POL_ "<" #R_ "," #T_ "," #N_ ">"},
#define Q(R_, T_, N_) {4, R_, T_, N_, N_ * T_, 0, 2, 0, "StressStokes<" #R_ "," #T_ "," #N_ ">"},
    MFS_VARIANTS(S, P, G, X, Q)
#undef S
#undef P
#undef G
#undef X
#undef Q
};

const PairVariant *pair_variants(int *count) {
    *count = (int)(sizeof(kVariants) / sizeof(kVariants[0]));
    return kVariants;
}

int pair_record_floats(int D, int nrhs, int packed) {
    if (packed == 2) return D == 3 ? (6 + 9 * nrhs + 3) / 4 * 4 : (6 + 2 * nrhs + 3) / 4 * 4;  // compensated
    return rec_floats(D, nrhs, packed != 0);
}

int pair_occupancy(int vi) {
    int i = 0;
#define S(D_, R_, T_, N_) \
    if (vi == i++) return occupancy_variant<Scalar<D_, R_, T_, N_>, N_>();
#define P(POL_, R_, TP_, N_) \
    if (vi == i++) return occupancy_variant<POL_<R_, TP_, N_>, N_>();
#define G(R_, T_, N_) \
    if (vi == i++) return occupancy_variant<GradStokes<R_, T_, N_>, N_>();
#define X(POL_, R_, T_, N_) \
    if (vi == i++) return occupancy_variant<POL_<R_, T_, N_>, N_>();
#define Q(R_, T_, N_) \
    if (vi == i++) return occupancy_variant<StressStokes<R_, T_, N_>, N_>();
    MFS_VARIANTS(S, P, G, X, Q)
#undef S
#undef P
#undef G
#undef X
#undef Q
    return 0;
}

cudaError_t pair_launch(int vi, const PairGeom &geo, const PairWork &work, int *err, cudaStream_t st) {
    int i = 0;
#define S(D_, R_, T_, N_) \
    if (vi == i++) return launch_variant<Scalar<D_, R_, T_, N_>, N_>(geo, work, err, st);
#define P(POL_, R_, TP_, N_) \
    if (vi == i++) return launch_variant<POL_<R_, TP_, N_>, N_>(geo, work, err, st);
#define G(R_, T_, N_) \
    if (vi == i++) return launch_variant<GradStokes<R_, T_, N_>, N_>(geo, work, err, st);
#define X(POL_, R_, T_, N_) \
    if (vi == i++) return launch_variant<POL_<R_, T_, N_>, N_>(geo, work, err, st);
#define Q(R_, T_, N_) \
    if (vi == i++) return launch_variant<StressStokes<R_, T_, N_>, N_>(geo, work, err, st);
    MFS_VARIANTS(S, P, G, X, Q)
#undef S
#undef P
#undef G
#undef X
#undef Q
    return cudaErrorInvalidValue;
}

cudaError_t pair_epilogue(int D, int nrhs, const PairWork &work, const double *base, double beta, double scale,
                          double *out, int ntargets, cudaStream_t st) {
    const int threads = 1024;
    if (work.ntiles == 0) return cudaSuccess;
    // lanes per entry from the most CTAs on one tile; blocks per tile so that a tile's entries times
    // lanes fill about one 1024-thread block each (at most 16)
    const int S = work.max_share >= 64 ? 8 : (work.max_share >= 16 ? 4 : 1);
    const long long lanes = (long long)work.tile_targets * D * nrhs * S;
    const int Y = (int)std::min<long long>(16, std::max<long long>(1, (lanes + threads - 1) / threads));
    const dim3 grid((unsigned)work.ntiles, (unsigned)Y);
#define E(D_, R_)                                                                                      \
    if (D == D_ && nrhs == R_) {                                                                       \
        pair_epilogue_kernel<D_, R_><<<grid, threads, 0, st>>>(work, base, beta, scale, out, ntargets, S); \
        return cudaGetLastError();                                                                     \
    }
    E(3, 1) E(3, 2) E(3, 3) E(3, 4) E(1, 1) E(1, 2) E(1, 3) E(1, 4)
    E(4, 1) E(4, 2) E(4, 3) E(4, 4)  // pressure and traction
#undef E
    return cudaErrorInvalidValue;
}

cudaError_t pack_sources(int D, int nrhs, int packed, const float4 *src_pos, const int *src_pt_of_rec,
                         const double *strength, int nsrc, int nrec, float *records, cudaStream_t st) {
    const int threads = 256, blocks = (nrec + threads - 1) / threads;
    if (nrec == 0) return cudaSuccess;
#define PK(D_, R_, PA_)                                                                                 \
    if (D == D_ && nrhs == R_ && (packed != 0) == PA_) {                                                \
        pack_sources_kernel<D_, R_, PA_><<<blocks, threads, 0, st>>>(src_pos, src_pt_of_rec, strength, nsrc, nrec, \
                                                                     records);                         \
        return cudaGetLastError();                                                                      \
    }
    PK(3, 1, false) PK(3, 2, false) PK(3, 3, false) PK(3, 4, false)
    PK(1, 1, false) PK(1, 2, false) PK(1, 3, false) PK(1, 4, false)
    PK(3, 1, true) PK(3, 2, true) PK(3, 3, true) PK(3, 4, true)
    PK(1, 1, true) PK(1, 2, true) PK(1, 3, true) PK(1, 4, true)
#undef PK
    return cudaErrorInvalidValue;
}

cudaError_t pack_sources_comp(int D, int nrhs, const double *src_local64, const int *src_pt_of_rec,
                              const double *strength, int nsrc, int nrec, float *records, cudaStream_t st) {
    const int threads = 256, blocks = (nrec + threads - 1) / threads;
    if (nrec == 0) return cudaSuccess;
#define PK(D_, R_)                                                                                               \
    if (D == D_ && nrhs == R_) {                                                                                 \
        pack_sources_comp_kernel<D_, R_><<<blocks, threads, 0, st>>>(src_local64, src_pt_of_rec, strength, nsrc, \
                                                                     nrec, records);                             \
        return cudaGetLastError();                                                                               \
    }
    PK(3, 1) PK(3, 2) PK(3, 3) PK(3, 4) PK(1, 1) PK(1, 2) PK(1, 3) PK(1, 4)
#undef PK
    return cudaErrorInvalidValue;
}

}  // namespace mfs

// ===========================================================================
// Stokeslet sum without device allocation.
//
// For callers that cannot allocate device memory: code that runs where cudaMalloc is not
// allowed or not wanted (inside another library's memory pool, a plug-in host, or a
// pre-planned memory budget) still gets the packed FP32 pair kernel.  Every byte of
// scratch lives in one file-scope __device__ array of fixed size, reserved when the
// library is loaded.  The array is shared by all calls and keeps the last call's contents,
// so calls whose GPU work overlaps (different streams, or different host threads) race.
// A bounded device wait that gives up inside the pair kernel (the error path of every bulk copy)
// leaves the scratch partly written; the call then fills u with NaN instead of returning a sum
// built from stale scratch, and the caller sees the failure without a synchronising query.
// ===========================================================================
namespace mfs {
namespace noalloc {
using Pol = PackedStokesReg<1, 2, 128>;
constexpr int NT = 128;
constexpr int TT = NT * Pol::TPT;  // targets per tile
constexpr int REC = Pol::REC;
constexpr int kMaxTargets = MFS_NOALLOC_MAX_TARGETS;
constexpr int kMaxSources = MFS_NOALLOC_MAX_SOURCES;
constexpr int kMaxCTAs = 640;
constexpr int kMaxTiles = (kMaxTargets + TT - 1) / TT;
constexpr size_t al(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t oTgt = 0;
constexpr size_t oRec = oTgt + al(sizeof(float4) * kMaxTargets);
constexpr size_t oTiles = oRec + al(sizeof(float) * REC * (size_t)(kMaxSources + 4));
constexpr size_t oMeta = oTiles + al(sizeof(PairTile) * kMaxTiles);
constexpr size_t oPart = oMeta + 256;
constexpr size_t oDirect = oPart + al(sizeof(double) * 3 * (size_t)kMaxCTAs * 2 * TT);
constexpr size_t kBytes = oDirect + al(sizeof(double) * 3 * (size_t)kMaxTargets);
struct Meta {
    int src_off[2];
    int err;
    int pad;
    long long blk_off[2];
    double centre[3];
};
}  // namespace noalloc
}  // namespace mfs

static __device__ __align__(256) unsigned char g_noalloc_scratch[mfs::noalloc::kBytes];

namespace mfs {
namespace noalloc {

// Targets -> float4, sources -> duplicated FP32 records, the tile list of the stream-K split and
// the single-body offsets; every scratch word the pair kernel and the epilogue read is written here
// first.  Coordinates are taken relative to the first target in FP64 before the FP32 cast (the sum
// is translation invariant), so the FP32 separations keep their precision wherever the points sit.
__global__ void prep_kernel(const double *targets, int nt, const double *sources, const double *lam, int ns,
                            int nrec, int ntiles, long long nblk, int G, unsigned char *base) {
    float4 *tgt = reinterpret_cast<float4 *>(base + oTgt);
    float *rec = reinterpret_cast<float *>(base + oRec);
    PairTile *tiles = reinterpret_cast<PairTile *>(base + oTiles);
    Meta *meta = reinterpret_cast<Meta *>(base + oMeta);
    const long long W = (long long)ntiles * nblk;
    const int stride = gridDim.x * blockDim.x;
    const int i0 = blockIdx.x * blockDim.x + threadIdx.x;
    const double o0 = targets[0], o1 = targets[1], o2 = targets[2];  // nt >= 1
    for (int i = i0; i < nt; i += stride)
        tgt[i] = make_float4((float)(targets[3 * (size_t)i] - o0), (float)(targets[3 * (size_t)i + 1] - o1),
                             (float)(targets[3 * (size_t)i + 2] - o2), __int_as_float(0));
    for (int r = i0; r < nrec; r += stride) {
        float v[6];
        if (r < ns) {
            v[0] = (float)(sources[3 * (size_t)r] - o0);
            v[1] = (float)(sources[3 * (size_t)r + 1] - o1);
            v[2] = (float)(sources[3 * (size_t)r + 2] - o2);
            for (int c = 0; c < 3; ++c) v[3 + c] = (float)lam[3 * (size_t)r + c];
        } else {  // padding: far away, zero strength -> exactly zero contribution
            v[0] = v[1] = v[2] = 1e15f;
            v[3] = v[4] = v[5] = 0.f;
        }
        float *o = rec + (size_t)r * REC;
        for (int c = 0; c < 6; ++c) o[2 * c] = o[2 * c + 1] = v[c];
    }
    for (int t = i0; t < ntiles; t += stride) {
        PairTile tl;
        tl.t0 = t * TT;
        tl.t1 = min(nt, tl.t0 + TT);
        tl.kb0 = 0;
        tl.nb = 1;
        tl.skip = -1;
        tl.B0 = 0;
        tl.B1 = 1;
        tl.u0 = (long long)t * nblk;
        tl.u1 = tl.u0 + nblk;
        tl.gA = (int)(((tl.u0 + 1) * G - 1) / W);
        tl.gB = (int)((tl.u1 * G - 1) / W);
        tl.L0 = tl.L1 = -1;
        tiles[t] = tl;
    }
    if (i0 == 0) {
        meta->src_off[0] = 0;
        meta->src_off[1] = nrec;
        meta->err = 0;
        meta->blk_off[0] = 0;
        meta->blk_off[1] = nblk;
        meta->centre[0] = meta->centre[1] = meta->centre[2] = 0.0;
    }
}

// u = NaN everywhere when a bounded wait of the pair kernel gave up (err set): the scratch the
// epilogue read was then only partly written by this call.
__global__ void poison_on_timeout_kernel(const int *err, double *u, size_t n) {
    if (*err == 0) return;
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        u[i] = nan;
}

// Per device: the array's device address and the kernel's resident CTAs per SM, looked up on the
// first call on that device under a lock (several host threads may make their first calls at once).
struct DeviceScratch {
    std::mutex mu;
    void *ptr[64] = {};
    int occupancy[64] = {};
};
static DeviceScratch g_dev;

}  // namespace noalloc
}  // namespace mfs

extern "C" mfs_status mfs_stokeslet_sum_noalloc(const double *targets, int32_t num_targets, const double *sources,
                                                const double *strengths, int32_t num_sources, double mu, double *u,
                                                void *stream) {
    using namespace mfs;
    using namespace mfs::noalloc;
    if (!targets || !sources || !strengths || !u || num_targets < 0 || num_sources < 0 || !(mu > 0.0))
        return MFS_ERR_INVALID_ARG;
    if (num_targets > kMaxTargets || num_sources > kMaxSources) return MFS_ERR_INVALID_ARG;
    if (num_targets == 0) return MFS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return MFS_ERR_CUDA;
    unsigned char *base = nullptr;
    int occupancy = 0;
    {
        std::lock_guard<std::mutex> lock(g_dev.mu);
        if (!g_dev.ptr[dev]) {  // first call on this device: the array's device address
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return MFS_ERR_CUDA;
            g_dev.ptr[dev] = p;
        }
        if (g_dev.occupancy[dev] == 0) {
            int occ = 0;
            auto kern = pair_sum_kernel<Pol, NT>;
            if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, StageCfg<Pol, NT>::SMEM) !=
                    cudaSuccess ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, StageCfg<Pol, NT>::SMEM) !=
                    cudaSuccess ||
                occ <= 0)
                return MFS_ERR_CUDA;
            g_dev.occupancy[dev] = occ;
        }
        base = static_cast<unsigned char *>(g_dev.ptr[dev]);
        occupancy = g_dev.occupancy[dev];
    }
    if (num_sources == 0) return cudaMemsetAsync(u, 0, sizeof(double) * 3 * (size_t)num_targets, st) == cudaSuccess
                                     ? MFS_OK : MFS_ERR_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MFS_ERR_CUDA;
    const int nrec = (num_sources + 3) / 4 * 4;
    const long long nblk = (nrec + MFS_BS - 1) / MFS_BS;
    const int ntiles = (num_targets + TT - 1) / TT;
    const long long W = (long long)ntiles * nblk;
    long long G = std::min<long long>((long long)occupancy * sms, kMaxCTAs);
    if (G > W) G = W;
    prep_kernel<<<256, 256, 0, st>>>(targets, num_targets, sources, strengths, num_sources, nrec, ntiles, nblk,
                                     (int)G, base);
    if (cudaGetLastError() != cudaSuccess) return MFS_ERR_CUDA;
    Meta *meta = reinterpret_cast<Meta *>(base + oMeta);
    PairGeom geo;
    geo.tgt = reinterpret_cast<const float4 *>(base + oTgt);
    geo.src = reinterpret_cast<const float *>(base + oRec);
    geo.src_off = meta->src_off;
    geo.blk_off = meta->blk_off;
    geo.centres = meta->centre;
    geo.ntargets = num_targets;
    PairWork work;
    work.tiles = reinterpret_cast<const PairTile *>(base + oTiles);
    work.ntiles = ntiles;
    work.total_units = W;
    work.G = (int)G;
    work.partial = reinterpret_cast<double *>(base + oPart);
    work.direct = reinterpret_cast<double *>(base + oDirect);
    work.tile_targets = TT;
    work.include_self = 1;
    if (launch_variant<Pol, NT>(geo, work, &meta->err, st) != cudaSuccess) return MFS_ERR_CUDA;
    pair_epilogue_kernel<3, 1><<<ntiles, 1024, 0, st>>>(work, nullptr, 0.0, 1.0 / (8.0 * MFS_PI * mu), u,
                                                       num_targets, 1);
    poison_on_timeout_kernel<<<sms, 256, 0, st>>>(&meta->err, u, 3 * (size_t)num_targets);
    return cudaGetLastError() == cudaSuccess ? MFS_OK : MFS_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// FP32 FMA-rate probe: the throughput the pair kernel's roofline divides by
// ---------------------------------------------------------------------------
namespace mfs {
namespace fmaprobe {

constexpr int kChains = 8;     // independent dependency chains per thread
constexpr int kThreads = 256;  // threads per CTA
constexpr int kIters = 1 << 18;

// a <- a * b + c on kChains independent chains; b < 1 and c > 0 keep every value near c / (1 - b)
// (normal FP32 numbers), and the final test against a value the chains never reach keeps the
// compiler from removing them.
template <bool PACKED>
__global__ void __launch_bounds__(kThreads) fma_rate_kernel(float b, float c, int iters, float *sink) {
    const float seed = 0.5f + 1e-3f * (float)(threadIdx.x & 31);
    if (PACKED) {
        u64 a[kChains];
        const u64 bb = f2_pack(b, b), cc = f2_pack(c, c);
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = f2_pack(seed + (float)i, seed - (float)i);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int i = 0; i < kChains; ++i) a[i] = f2_fma(a[i], bb, cc);
        }
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < kChains; ++i) {
            float lo, hi;
            f2_unpack(a[i], lo, hi);
            s += lo + hi;
        }
        if (s == -1.0f) sink[blockIdx.x] = s;
    } else {
        float a[kChains];
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = seed + (float)i;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int i = 0; i < kChains; ++i) a[i] = fmaf(a[i], b, c);
        }
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < kChains; ++i) s += a[i];
        if (s == -1.0f) sink[blockIdx.x] = s;
    }
}

// f32x2 FMAs whose three operands are distinct registers, each rewritten every step (no operand
// is a loop constant, as in the pair kernel's inner loop, where dx, sc, lambda and the sums all
// change).  Half of the chains hold values near 1 (x), half values near t = 1e-15 (y):
// x' = x1 * y + x2 stays near x2 and y' = y1 * y2 + y3 near y3, so every value stays a normal
// FP32 number.  Two register banks alternate, so the kChains FMAs of a step are independent.
__global__ void __launch_bounds__(kThreads) fma_rate_distinct_kernel(float t, int iters, float *sink) {
    constexpr int H = kChains / 2;
    const float seed = 0.5f + 1e-3f * (float)(threadIdx.x & 31);
    u64 a[kChains], b[kChains];
#pragma unroll
    for (int i = 0; i < H; ++i) {
        a[i] = f2_pack(seed + (float)i, seed - 0.25f * (float)i);
        a[H + i] = f2_pack(t * (seed + (float)i), t * (seed + 0.5f * (float)i));
    }
    for (int it = 0; it < iters; it += 2) {
#pragma unroll
        for (int i = 0; i < H; ++i) {
            b[i] = f2_fma(a[(i + 1) % H], a[H + (i + 2) % H], a[(i + 3) % H]);
            b[H + i] = f2_fma(a[H + (i + 1) % H], a[H + (i + 2) % H], a[H + (i + 3) % H]);
        }
#pragma unroll
        for (int i = 0; i < H; ++i) {
            a[i] = f2_fma(b[(i + 1) % H], b[H + (i + 2) % H], b[(i + 3) % H]);
            a[H + i] = f2_fma(b[H + (i + 1) % H], b[H + (i + 2) % H], b[H + (i + 3) % H]);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
        float lo, hi;
        f2_unpack(a[i], lo, hi);
        s += lo + hi;
    }
    if (s == -1.0f) sink[blockIdx.x] = s;
}

}  // namespace fmaprobe
}  // namespace mfs

extern "C" mfs_status mfs_fp32_fma_rate(int32_t mode, double *tflops, void *stream) {
    using namespace mfs::fmaprobe;
    if (!tflops || mode < 0 || mode > 4) return MFS_ERR_INVALID_ARG;
    *tflops = 0.0;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        return MFS_ERR_CUDA;
    // modes 0-2: 4 CTAs of 8 warps per SM (32 warps); modes 3-4: one CTA (8 warps, 2 per scheduler)
    const int grid = sms * (mode >= 3 ? 1 : 4);
    const bool distinct = (mode == 2 || mode == 4);
    float *sink = nullptr;
    if (cudaMallocAsync(&sink, sizeof(float) * grid, st) != cudaSuccess) return MFS_ERR_OOM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    mfs_status rc = MFS_ERR_CUDA;
    if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
        auto launch = [&](int iters) {
            if (distinct)
                fma_rate_distinct_kernel<<<grid, kThreads, 0, st>>>(1e-15f, iters, sink);
            else if (mode != 0)
                fma_rate_kernel<true><<<grid, kThreads, 0, st>>>(0.9999999f, 1e-7f, iters, sink);
            else
                fma_rate_kernel<false><<<grid, kThreads, 0, st>>>(0.9999999f, 1e-7f, iters, sink);
        };
        launch(kIters / 16);  // warm-up (clocks up, code loaded)
        cudaEventRecord(e0, st);
        launch(kIters);
        cudaEventRecord(e1, st);
        float ms = 0.f;
        if (cudaGetLastError() == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
            cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.f) {
            const double fmas = (double)grid * kThreads * kChains * (mode != 0 ? 2.0 : 1.0) * kIters;
            *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
            rc = MFS_OK;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFreeAsync(sink, st);
    return rc;
}

// ---------------------------------------------------------------------------
// Self-test of the bounded device waits: a barrier phase that nothing completes
// ---------------------------------------------------------------------------
namespace mfs {
namespace selftest {

// One warp waits on phase 0 of a shared-memory mbarrier with the kernels' own bounded wait.  With
// `arrive`, thread 0 completes the phase first (an arrival with no expected bytes) and the wait
// succeeds; without, no thread ever arrives and every waiter gives up after `limit` polls and records
// the timeout flag, exactly as a lost bulk copy would make a pair or tensor-core kernel do.
__global__ void bounded_wait_kernel(int arrive, long long limit, int *err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (arrive && threadIdx.x == 0) mbar_arrive_expect_tx(&bar, 0);
    __syncthreads();
    mbar_wait_bounded(&bar, 0, err, limit);
}

}  // namespace selftest
}  // namespace mfs

extern "C" mfs_status mfs_selftest_bounded_wait(int32_t arrive, int64_t limit, void *stream) {
    if ((arrive != 0 && arrive != 1) || limit < 1 || limit > (1ll << 24)) return MFS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int *err = nullptr;
    if (cudaMallocAsync(&err, sizeof(int), st) != cudaSuccess) return MFS_ERR_OOM;
    mfs_status rc = MFS_ERR_CUDA;
    int h = -1;
    if (cudaMemsetAsync(err, 0, sizeof(int), st) == cudaSuccess) {
        mfs::selftest::bounded_wait_kernel<<<1, 32, 0, st>>>(arrive, (long long)limit, err);
        if (cudaGetLastError() == cudaSuccess &&
            cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
            cudaStreamSynchronize(st) == cudaSuccess)
            rc = (h & MFS_DEVERR_TIMEOUT) ? MFS_ERR_DEVICE_TIMEOUT : (h == 0 ? MFS_OK : MFS_ERR_CUDA);
    }
    cudaFreeAsync(err, st);
    cudaStreamSynchronize(st);
    return rc;
}
