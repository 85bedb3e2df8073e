// One-body apply on the 5th-generation tensor cores: split-K 3xTF32 GEMM with tcgen05.
//
//   P[z][m][n] = sum_{k in chunk z} A[m][k] B[n][k]   (both operands K-major, FP32 in memory)
//
// Each operand x is held as hi = tf32(x) and lo = x - hi; the product is formed as
// hi*hi + hi*lo + lo*hi by three tcgen05.mma.kind::tf32 per K step, accumulated in FP32 in tensor
// memory (TMEM).  The factor (B: U^T or W^T of the one-body SVD, Eq. pseudo) is the MMA's M side
// (128 rows per CTA), the gathered columns (A) its N side (<= 256), so few columns still fill the
// 128-row MMA.  K is split over CTAs (grid.z) in chunks of a few hundred, and the FP32 chunk results
// are summed in FP64 afterwards (the same reduction as the CUDA-core split-K path), which keeps the
// FP32 accumulation short.
//
// Per CTA (128 threads): warp 0 lane 0 issues TMA loads (cp.async.bulk.tensor, 128-byte swizzle)
// into a two-stage ring, warp 1 lane 0 issues the MMAs and commits each stage back to the loader,
// warp 2 owns the TMEM allocation, and all four warps read the 128 x N accumulator with tcgen05.ld
// (warp w reads TMEM lanes 32w..32w+31) and write FP64 partials.  Every wait is bounded; on a
// timeout the CTA agrees (block vote), records an error flag, frees its TMEM and returns.
#include <cuda.h>

#include <cstring>

#include "common.cuh"
#include "kernels.h"

namespace mfs {

namespace tc {
constexpr int BM = 128;            // factor rows per CTA (MMA M)
constexpr int BK = 32;             // K elements per stage (128 bytes: one swizzle row)
constexpr int STAGES = 2;
constexpr int A_TILE = BM * BK * 4;  // bytes of one 128 x 32 FP32 tile (16 KB)

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
}  // namespace tc

// grid: (ceil(n / 128), ceil(m / BN), chunks); block 128; dynamic smem = STAGES * (2*A_TILE + 2*BN*128) + 1024
__global__ void __launch_bounds__(128, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap map_b_hi, const __grid_constant__ CUtensorMap map_b_lo,
                   const __grid_constant__ CUtensorMap map_a_hi, const __grid_constant__ CUtensorMap map_a_lo, int m,
                   int n, int k, int kchunk, int BN, int tmem_cols, double *P, int *err) {
    using namespace tc;
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], done_bar;
    __shared__ uint32_t tmem_base_sh;
    // 1024-byte aligned tiles (128-byte swizzle atoms are 8 rows x 128 bytes)
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t b_tile = A_TILE, a_tile = (uint32_t)BN * BK * 4;
    const uint32_t stage_bytes = 2 * b_tile + 2 * a_tile;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n0 = blockIdx.x * BM, m0 = blockIdx.y * BN;
    const int kb0 = blockIdx.z * kchunk;
    const int kb1 = min(k, kb0 + kchunk);
    const int nk = (kb1 - kb0 + BK - 1) / BK;
    const long long limit = 1ll << 22;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
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
    if (warp == 0 && lane == 0) {  // TMA producer
        for (int i = 0; i < nk && ok; ++i) {
            const int s = i % STAGES;
            if (i >= STAGES) ok = mbar_wait_bounded(&empty_bar[s], (uint32_t)(((i / STAGES) - 1) & 1), err, limit);
            if (!ok) break;
            const uint32_t st = base + s * stage_bytes;
            const uint32_t fb = smem_u32(&full_bar[s]);
            mbar_arrive_expect_tx(&full_bar[s], stage_bytes);
            const int kx = kb0 + i * BK;
            tma_load_2d(st, &map_b_hi, kx, n0, fb);
            tma_load_2d(st + b_tile, &map_b_lo, kx, n0, fb);
            tma_load_2d(st + 2 * b_tile, &map_a_hi, kx, m0, fb);
            tma_load_2d(st + 2 * b_tile + a_tile, &map_a_lo, kx, m0, fb);
        }
    } else if (warp == 1 && lane == 0) {  // MMA issuer
        const uint32_t idesc = instr_desc_tf32(BM, BN);
        for (int i = 0; i < nk && ok; ++i) {
            const int s = i % STAGES;
            ok = mbar_wait_bounded(&full_bar[s], (uint32_t)((i / STAGES) & 1), err, limit);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t st = base + s * stage_bytes;
#pragma unroll
            for (int kk = 0; kk < BK / 8; ++kk) {  // 8 TF32 = 32 bytes per MMA K step
                const uint32_t off = kk * 32;
                const uint64_t bh = smem_desc(st + off), bl = smem_desc(st + b_tile + off);
                const uint64_t ah = smem_desc(st + 2 * b_tile + off), al = smem_desc(st + 2 * b_tile + a_tile + off);
                mma_tf32(tmem, bh, ah, idesc, (i > 0 || kk > 0) ? 1u : 0u);
                mma_tf32(tmem, bh, al, idesc, 1u);
                mma_tf32(tmem, bl, ah, idesc, 1u);
            }
            mma_commit(smem_u32(&empty_bar[s]));  // stage free once these MMAs have read it
        }
        // also after a timeout: the commit fires once every MMA issued so far has finished, so the TMEM
        // is never freed under a running MMA
        mma_commit(smem_u32(&done_bar));
    }
    __syncwarp();
    // everybody: wait for the accumulator (bounded), then agree on success
    bool good = mbar_wait_bounded(&done_bar, 0u, err, limit);
    good = __syncthreads_and(good && ok) != 0;
    if (good) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int row = n0 + 32 * warp + lane;  // TMEM lane = factor row
        double *Pz = P + (size_t)blockIdx.z * m * n;
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
            if (row < n) {
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int col = m0 + c0 + i;
                    if (col < m) Pz[(size_t)col * n + row] = (double)v[i];
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 2)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t t;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(x));
    return __uint_as_float(t);
}

// hi = tf32(x), lo = tf32(x - hi) (round to nearest, ties away), rows x cols from a [rows][ld_src] array
// into [rows][ld_dst] arrays with zero padding columns cols..ld_dst.
__global__ void split_tf32_kernel(const float *src, int rows, int cols, int ld_src, float *hi, float *lo, int ld_dst) {
    const size_t total = (size_t)rows * ld_dst;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / ld_dst), c = (int)(i % ld_dst);
        float h = 0.f, l = 0.f;
        if (c < cols) {
            const float x = src[(size_t)r * ld_src + c];
            h = tf32_rna(x);
            l = tf32_rna(x - h);
        }
        hi[i] = h;
        lo[i] = l;
    }
}

// Transposed split: dst[c][r] from src[r][c] (a factor stored [k][n] becomes K-major [n][k]).
__global__ void split_tf32_transpose_kernel(const float *src, int rows, int cols, float *hi, float *lo, int ld_dst) {
    // src [rows][cols] -> dst [cols][ld_dst] with dst[c][r] = src[r][c]
    const size_t total = (size_t)cols * ld_dst;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i / ld_dst), r = (int)(i % ld_dst);
        float h = 0.f, l = 0.f;
        if (r < rows) {
            const float x = src[(size_t)r * cols + c];
            h = tf32_rna(x);
            l = tf32_rna(x - h);
        }
        hi[i] = h;
        lo[i] = l;
    }
}

cudaError_t split_tf32(const float *src, int rows, int cols, int ld_src, float *hi, float *lo, int ld_dst,
                       cudaStream_t st) {
    if (rows == 0) return cudaSuccess;
    split_tf32_kernel<<<1024, 256, 0, st>>>(src, rows, cols, ld_src, hi, lo, ld_dst);
    return cudaGetLastError();
}

cudaError_t split_tf32_transpose(const float *src, int rows, int cols, float *hi, float *lo, int ld_dst,
                                 cudaStream_t st) {
    if (cols == 0) return cudaSuccess;
    split_tf32_transpose_kernel<<<1024, 256, 0, st>>>(src, rows, cols, hi, lo, ld_dst);
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
    EncodeTiledFn fn = encode_fn();
    if (!fn || !ptr || ld % 32 != 0 || box_rows < 8 || box_rows > 256 || (reinterpret_cast<uintptr_t>(ptr) & 15))
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
    static_assert(sizeof(CUtensorMap) == sizeof(TcMap), "tensor map size");
    std::memcpy(&out, &m, sizeof(m));
    return true;
}

int tc_gemm_bn(int m) {  // MMA N: columns per CTA, a multiple of 16, at most 256
    const int b = ((m + 15) / 16) * 16;
    return b > 256 ? 256 : (b < 16 ? 16 : b);
}

int tc_gemm_chunks(int m, int n, int k, int sm_count) {
    const int tiles = ((n + tc::BM - 1) / tc::BM) * ((m + tc_gemm_bn(m) - 1) / tc_gemm_bn(m));
    int s = (2 * sm_count + tiles - 1) / tiles;  // about two CTAs per SM in total
    const int smax = (k + 255) / 256;            // chunks of at least 256 K
    if (s > smax) s = smax;
    return s < 1 ? 1 : s;
}

size_t tc_gemm_smem(int BN) { return (size_t)tc::STAGES * (2 * tc::A_TILE + 2 * (size_t)BN * tc::BK * 4) + 1024; }

// C partials P[z][m][n] = sum_{k in chunk z} A[m][k] B[n][k], A and B given as (hi, lo) tensor maps.
cudaError_t tc_gemm(const TcMap &b_hi, const TcMap &b_lo, const TcMap &a_hi, const TcMap &a_lo, int m, int n, int k,
                    int S, double *P, int *err, cudaStream_t st) {
    if (m == 0 || n == 0) return cudaSuccess;
    if (k <= 0 || S <= 0) return cudaErrorInvalidValue;
    const int BN = tc_gemm_bn(m);
    int cols = 32;
    while (cols < BN) cols <<= 1;
    const int kchunk = ((k + S - 1) / S + tc::BK - 1) / tc::BK * tc::BK;
    const int Sz = (k + kchunk - 1) / kchunk;
    const size_t smem = tc_gemm_smem(BN);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)tc_gemm_smem(256));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 grid((n + tc::BM - 1) / tc::BM, (m + BN - 1) / BN, Sz);
    CUtensorMap mb_hi, mb_lo, ma_hi, ma_lo;
    std::memcpy(&mb_hi, &b_hi, sizeof(mb_hi));
    std::memcpy(&mb_lo, &b_lo, sizeof(mb_lo));
    std::memcpy(&ma_hi, &a_hi, sizeof(ma_hi));
    std::memcpy(&ma_lo, &a_lo, sizeof(ma_lo));
    tc_gemm_kernel<<<grid, 128, smem, st>>>(mb_hi, mb_lo, ma_hi, ma_lo, m, n, k, kchunk, BN, cols, P, err);
    return cudaGetLastError();
}

int tc_gemm_sz(int k, int S) {
    const int kchunk = ((k + S - 1) / S + tc::BK - 1) / tc::BK * tc::BK;
    return (k + kchunk - 1) / kchunk;
}

}  // namespace mfs
