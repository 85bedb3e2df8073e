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
#include "common.cuh"
#include "kernels.h"

namespace mfs {

template <int D, int NRHS>
struct Rec {
    static constexpr int C = D * NRHS;                 // strength components per source
    static constexpr int REC = ((3 + C) + 3) / 4 * 4;  // floats per packed source record
};

template <int D, int NRHS, int T, int NT>
struct PairCfg {
    static constexpr int C = Rec<D, NRHS>::C;
    static constexpr int REC = Rec<D, NRHS>::REC;
    static constexpr int STAGE_BYTES = 16384;
    static constexpr int STAGE_REC = (STAGE_BYTES / (REC * 4)) / MFS_BS * MFS_BS;
    static constexpr int STAGE_BLOCKS = STAGE_REC / MFS_BS;
    static constexpr int TT = NT * T;
    static constexpr int SMEM = 2 * STAGE_REC * REC * 4;
};

struct Stage {
    int tile;      // -1: no stage
    int body;      // source body
    int rec0;      // first record (global)
    int nrec;      // records in this stage (multiple of 4)
    long long u;   // global unit index of the first block
    int nblk;      // blocks in this stage
};

// First tile whose unit range contains u (tiles are contiguous in unit space; empty tiles skipped).
__device__ __forceinline__ int tile_of_unit(const PairTile *tiles, int ntiles, long long u) {
    int lo = 0, hi = ntiles - 1;
    while (lo < hi) {  // last tile with u0 <= u
        int mid = (lo + hi + 1) >> 1;
        if (tiles[mid].u0 <= u) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// The stage that starts at global unit u (u < uend), at most max_blocks blocks long.
__device__ __forceinline__ Stage make_stage(const PairTile *tiles, int ntiles, const long long *blk_off,
                                            const int *src_off, long long u, long long uend, int max_blocks,
                                            int hint_tile) {
    Stage st;
    int t = hint_tile;
    if (t < 0 || !(tiles[t].u0 <= u && u < tiles[t].u1)) t = tile_of_unit(tiles, ntiles, u);
    const PairTile tl = tiles[t];
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
    long long seg_end = tl.u1 < uend ? tl.u1 : uend;
    long long rem = seg_end - u;
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

template <int D, int NRHS, int T, int NT>
__global__ void __launch_bounds__(NT) pair_sum_kernel(PairGeom geo, PairWork work, int *err) {
    using Cfg = PairCfg<D, NRHS, T, NT>;
    constexpr int C = Cfg::C, REC = Cfg::REC, SREC = Cfg::STAGE_REC;
    extern __shared__ __align__(128) float smem[];
    __shared__ float dcs[2][MFS_MAX_TILE_BODIES][3];
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
    Stage cur = make_stage(tiles, work.ntiles, geo.blk_off, geo.src_off, ubeg, uend, Cfg::STAGE_BLOCKS, -1);
    const int first_tile = cur.tile;
    if (tid == 0) {
        mbar_arrive_expect_tx(&bars[0], (uint32_t)(cur.nrec * REC * 4));
        bulk_g2s(smem, geo.src + (size_t)cur.rec0 * REC, (uint32_t)(cur.nrec * REC * 4), &bars[0]);
    }

    // per-target state
    float3 tp[T];      // body-local target position
    int tb[T];         // target body
    float hi[T][C], lo[T][C], bsum[T][C];
    PairTile tl = tiles[cur.tile];
    long long seg_begin = ubeg;

    auto load_targets = [&](const PairTile &t_) {
#pragma unroll
        for (int j = 0; j < T; ++j) {
            int idx = t_.t0 + tid + j * NT;
            if (idx >= t_.t1) idx = t_.t1 - 1;
            float4 p = geo.tgt[idx];
            tp[j] = make_float3(p.x, p.y, p.z);
            tb[j] = __float_as_int(p.w);
#pragma unroll
            for (int c = 0; c < C; ++c) { hi[j][c] = 0.f; lo[j][c] = 0.f; bsum[j][c] = 0.f; }
        }
    };
    load_targets(tl);

    int si = 0;
    while (true) {
        const int buf = si & 1;
        // next stage (uniform across the CTA)
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
            nxt = make_stage(tiles, work.ntiles, geo.blk_off, geo.src_off, unext, uend, Cfg::STAGE_BLOCKS, hint);
            if (tid == 0) {
                mbar_arrive_expect_tx(&bars[buf ^ 1], (uint32_t)(nxt.nrec * REC * 4));
                bulk_g2s(smem + (buf ^ 1) * SREC * REC, geo.src + (size_t)nxt.rec0 * REC,
                         (uint32_t)(nxt.nrec * REC * 4), &bars[buf ^ 1]);
            }
        }
        // centre offsets of the tile's target bodies relative to this stage's source body
        if (tid < tl.nb * 3) {
            const int kb = tl.kb0 + tid / 3, c = tid % 3;
            dcs[buf][tid / 3][c] = (float)(geo.centres[kb * 3 + c] - geo.centres[cur.body * 3 + c]);
        }
        const bool ok = mbar_wait_bounded(&bars[buf], (uint32_t)((si >> 1) & 1), err, wait_limit);
        if (__syncthreads_or(!ok)) {
            // give the other buffer's copy (if any) a bounded chance to land, then leave
            if (nxt.tile >= 0) mbar_wait_bounded(&bars[buf ^ 1], (uint32_t)(((si + 1) >> 1) & 1), nullptr, wait_limit);
            return;
        }

        // ---- compute this stage ----
        const float *sb = smem + buf * SREC * REC;
        float3 xt[T];
#pragma unroll
        for (int j = 0; j < T; ++j) {
            const int r = tb[j] - tl.kb0;
            xt[j] = make_float3(dcs[buf][r][0] + tp[j].x, dcs[buf][r][1] + tp[j].y, dcs[buf][r][2] + tp[j].z);
        }
        for (int s0 = 0; s0 < cur.nrec; s0 += MFS_BS) {
            const int s1 = min(s0 + MFS_BS, cur.nrec);
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
                        const float ri = rsqrtf(r2);
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

        // ---- end of a source body (for this tile): fold into (hi, lo), leaving self pairs out ----
        const bool body_ends = (nxt.tile < 0) || nxt.tile != cur.tile || nxt.body != cur.body;
        if (body_ends) {
#pragma unroll
            for (int j = 0; j < T; ++j) {
                const bool keep = work.include_self || (tb[j] != cur.body);
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
        // ---- end of this CTA's segment of the tile: write the tile's result ----
        const bool tile_ends = (nxt.tile < 0) || nxt.tile != cur.tile;
        if (tile_ends) {
            const long long seg_end = cur.u + cur.nblk;
            const bool whole = (seg_begin == tl.u0) && (seg_end == tl.u1);
#pragma unroll
            for (int j = 0; j < T; ++j) {
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
                    for (int c = 0; c < C; ++c) dst[c] = (double)hi[j][c] + (double)lo[j][c];
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
template <int D, int NRHS>
__global__ void pair_epilogue_kernel(PairWork work, const double *base, double beta, double scale, double *out,
                                     int ntargets) {
    constexpr int C = D * NRHS;
    const PairTile tl = work.tiles[blockIdx.x];
    const long long W = work.total_units;
    for (int t = tl.t0 + threadIdx.x; t < tl.t1; t += blockDim.x) {
        double v[C];
#pragma unroll
        for (int c = 0; c < C; ++c) v[c] = 0.0;
        if (tl.gA >= 0) {
            if (tl.gA == tl.gB) {
#pragma unroll
                for (int c = 0; c < C; ++c) v[c] = work.direct[(size_t)t * C + c];
            } else {
                for (int gg = tl.gA; gg <= tl.gB; ++gg) {
                    const long long b0 = (long long)gg * W / work.G, b1 = (long long)(gg + 1) * W / work.G;
                    if (b0 >= b1) continue;
                    const int slot = (b0 >= tl.u0) ? 0 : 1;
                    const double *src = work.partial + ((size_t)(gg * 2 + slot) * work.tile_targets + (t - tl.t0)) * C;
#pragma unroll
                    for (int c = 0; c < C; ++c) v[c] += src[c];
                }
            }
        }
#pragma unroll
        for (int h = 0; h < NRHS; ++h)
#pragma unroll
            for (int d = 0; d < D; ++d) {
                const size_t o = ((size_t)h * ntargets + t) * D + d;
                const double b = base ? beta * base[o] : 0.0;
                out[o] = b + scale * v[h * D + d];
            }
    }
}

// Pack proxy strengths (FP64 [nrhs][sum_N][D], body-local rotated positions) into FP32 records.
// Padding records (beyond N_k in each body) sit at the body centre with zero strength, which
// contributes exactly zero to every target off that centre.
template <int D, int NRHS>
__global__ void pack_sources_kernel(const float4 *src_pos, const int *src_body_of_rec, const int *src_pt_of_rec,
                                    const double *strength, int nsrc, int nrec, float *records) {
    constexpr int C = D * NRHS, REC = Rec<D, NRHS>::REC;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrec) return;
    float r[REC];
#pragma unroll
    for (int c = 0; c < REC; ++c) r[c] = 0.f;
    const int p = src_pt_of_rec[i];
    if (p >= 0) {
        const float4 y = src_pos[p];
        r[0] = y.x;
        r[1] = y.y;
        r[2] = y.z;
#pragma unroll
        for (int h = 0; h < NRHS; ++h)
#pragma unroll
            for (int d = 0; d < D; ++d) r[3 + h * D + d] = (float)strength[((size_t)h * nsrc + p) * D + d];
    }
    float4 *o = reinterpret_cast<float4 *>(records + (size_t)i * REC);
#pragma unroll
    for (int v = 0; v < REC / 4; ++v) o[v] = make_float4(r[4 * v], r[4 * v + 1], r[4 * v + 2], r[4 * v + 3]);
    (void)src_body_of_rec;
    (void)C;
}

// ---------------------------------------------------------------------------
// Host side: variant table
// ---------------------------------------------------------------------------
template <int D, int NRHS, int T, int NT>
static cudaError_t launch_variant(const PairGeom &geo, const PairWork &work, int *err, cudaStream_t st) {
    using Cfg = PairCfg<D, NRHS, T, NT>;
    auto kern = pair_sum_kernel<D, NRHS, T, NT>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    kern<<<work.G, NT, Cfg::SMEM, st>>>(geo, work, err);
    return cudaGetLastError();
}

template <int D, int NRHS, int T, int NT>
static int occupancy_variant() {
    using Cfg = PairCfg<D, NRHS, T, NT>;
    auto kern = pair_sum_kernel<D, NRHS, T, NT>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, NT, Cfg::SMEM) != cudaSuccess) return 0;
    return blocks;
}

#define MFS_VARIANTS(X)      \
    X(3, 1, 4, 128)          \
    X(3, 1, 2, 128)          \
    X(3, 1, 4, 256)          \
    X(3, 1, 2, 256)          \
    X(3, 2, 2, 128)          \
    X(3, 3, 2, 128)          \
    X(3, 4, 2, 128)          \
    X(3, 4, 1, 128)          \
    X(1, 1, 4, 128)          \
    X(1, 1, 8, 128)          \
    X(1, 1, 4, 256)          \
    X(1, 2, 4, 128)          \
    X(1, 3, 4, 128)          \
    X(1, 4, 4, 128)

static const PairVariant kVariants[] = {
#define X(D_, R_, T_, N_) {D_, R_, T_, N_, N_ * T_},
    MFS_VARIANTS(X)
#undef X
};

const PairVariant *pair_variants(int *count) {
    *count = (int)(sizeof(kVariants) / sizeof(kVariants[0]));
    return kVariants;
}

int pair_record_floats(int D, int nrhs) { return ((3 + D * nrhs) + 3) / 4 * 4; }

int pair_occupancy(int vi) {
    int i = 0;
#define X(D_, R_, T_, N_) \
    if (vi == i++) return occupancy_variant<D_, R_, T_, N_>();
    MFS_VARIANTS(X)
#undef X
    return 0;
}

cudaError_t pair_launch(int vi, const PairGeom &geo, const PairWork &work, int *err, cudaStream_t st) {
    int i = 0;
#define X(D_, R_, T_, N_) \
    if (vi == i++) return launch_variant<D_, R_, T_, N_>(geo, work, err, st);
    MFS_VARIANTS(X)
#undef X
    return cudaErrorInvalidValue;
}

cudaError_t pair_epilogue(int D, int nrhs, const PairWork &work, const double *base, double beta, double scale,
                          double *out, int ntargets, cudaStream_t st) {
    const int threads = 256;
    if (work.ntiles == 0) return cudaSuccess;
#define E(D_, R_)                                                                                      \
    if (D == D_ && nrhs == R_) {                                                                       \
        pair_epilogue_kernel<D_, R_><<<work.ntiles, threads, 0, st>>>(work, base, beta, scale, out, ntargets); \
        return cudaGetLastError();                                                                     \
    }
    E(3, 1) E(3, 2) E(3, 3) E(3, 4) E(1, 1) E(1, 2) E(1, 3) E(1, 4)
#undef E
    return cudaErrorInvalidValue;
}

cudaError_t pack_sources(int D, int nrhs, const float4 *src_pos, const int *src_pt_of_rec, const double *strength,
                         int nsrc, int nrec, float *records, cudaStream_t st) {
    const int threads = 256, blocks = (nrec + threads - 1) / threads;
    if (nrec == 0) return cudaSuccess;
#define P(D_, R_)                                                                                        \
    if (D == D_ && nrhs == R_) {                                                                         \
        pack_sources_kernel<D_, R_><<<blocks, threads, 0, st>>>(src_pos, nullptr, src_pt_of_rec, strength, nsrc, \
                                                                 nrec, records);                         \
        return cudaGetLastError();                                                                       \
    }
    P(3, 1) P(3, 2) P(3, 3) P(3, 4) P(1, 1) P(1, 2) P(1, 3) P(1, 4)
#undef P
    return cudaErrorInvalidValue;
}

}  // namespace mfs
