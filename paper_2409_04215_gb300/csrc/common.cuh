// Shared definitions of libmfs (internal; not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#define MFS_PI 3.14159265358979323846

// Device error flags (bit mask written with atomicOr by kernels that give up).
#define MFS_DEVERR_TIMEOUT 1
#define MFS_DEVERR_BADARG 2

// ---------------------------------------------------------------------------
// Pair-sum work decomposition.
//
// Targets (collocation points) are numbered globally, bodies contiguous, the
// bodies of one suspension contiguous.  A tile is a range of at most
// `tile_targets` consecutive targets of one suspension spanning at most
// MFS_MAX_TILE_BODIES bodies.  Its work is the sequence of source "units"
// (blocks of MFS_BS consecutive source records of one body) of every body of
// its suspension, except the tile's own body when the tile lies inside one
// body and self pairs are excluded.  The units of all tiles are concatenated
// into one global sequence of `total_units`, cut into G equal shares, one per
// persistent CTA (a stream-K split), so that every CTA does the same work.
// ---------------------------------------------------------------------------
#define MFS_BS 32
#define MFS_MAX_TILE_BODIES 32

struct PairTile {
    int t0, t1;          // targets [t0, t1)
    int kb0, nb;         // target bodies kb0 .. kb0+nb-1
    int skip;            // source body left out entirely, or -1
    int B0, B1;          // source bodies of the suspension [B0, B1)
    long long u0, u1;    // global unit range of this tile
    int gA, gB;          // first and last CTA whose share meets this tile
    int L0, L1;          // L0 >= 0: the tile's sources are the segments of interaction-list entries
                         // [L0, L1) (PairGeom::lst_*) instead of the bodies [B0, B1)
};

// Compensated pair sums split body-local coordinates and centre differences at multiples of
// 1/MFS_XGRID: the "high" parts of a target and a source then differ by an exactly representable
// FP32 number, and its square is exact while it is shorter than 32 (11 significant bits).
#define MFS_XGRID 64.0

struct PairGeom {
    const float4 *tgt;         // [ntargets] body-local rotated target (x,y,z), w = body id (int bits)
    const float *src;          // [sum_Npad][REC] packed source records
    const int *src_off;        // [P+1] record offset of each body (padded to a multiple of 4)
    const long long *blk_off;  // [P+1] global block offset of each body (blocks of MFS_BS records)
    const double *centres;     // [P][3]
    int ntargets;
    const float *tgt_w = nullptr;  // gradient kernel only: target strengths w, FP32 [nrhs][ntargets][3]
    // compensated kernels only: body-local targets split as x = hi + lo, hi a multiple of 1/MFS_XGRID
    const float4 *tgt_hi = nullptr, *tgt_lo = nullptr;  // [ntargets] (x, y, z, unused)
    // interaction lists (tiles with L0 >= 0): entry e names source segment lst_seg[e], whose records
    // are [seg_rec0[s], seg_rec1[s]) (blocks of MFS_BS), and starts at global unit lst_cum[e]
    // (lst_cum has one entry more than lst_seg: the units of the last tile end at its last value)
    const int *lst_seg = nullptr;
    const long long *lst_cum = nullptr;
    const int *seg_rec0 = nullptr, *seg_rec1 = nullptr;
};

struct PairWork {
    const PairTile *tiles;
    int ntiles;
    long long total_units;
    int G;                     // persistent CTAs
    double *partial;           // [G][2][tile_targets][C]
    double *direct;            // [ntargets][C]
    int tile_targets;
    int include_self;          // 1: self pairs included (right-hand side u_0)
    double *src_grad = nullptr;  // gradient kernel only: per source body sums, FP64 [P][3] (atomic adds)
    const int *tperm = nullptr;  // epilogue: target t's value goes to (and its base is read at) tperm[t]
    int max_share = 1;           // epilogue: the most CTAs that share one tile
};

// ---------------------------------------------------------------------------
// Inline PTX: mbarrier + 1-D bulk copy (TMA engine), with bounded waits.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
        "r"(bytes)
        : "memory");
}

// Returns true when phase `parity` of the barrier has completed.
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after `limit` polls (each try_wait itself suspends for a
// hardware-defined interval), records MFS_DEVERR_TIMEOUT and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int *err, long long limit) {
    for (long long it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    if (err) atomicOr(err, MFS_DEVERR_TIMEOUT);
    return false;
}

// Bulk copy global -> shared, completion signalled on `bar` (bytes % 16 == 0, both addresses 16-B aligned).
__device__ __forceinline__ void bulk_g2s(void *dst_smem, const void *src_gmem, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Error-free transformation a + b = s + e (Knuth's TwoSum, 6 flops).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
