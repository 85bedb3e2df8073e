// Device-resident FP64 GMRES (Algorithm 1 SOLVE uses GMRES; zero initial guess, no restart
// within the basis capacity).  The vector of all lanes is one array; lane l (one right-hand
// side of one suspension) owns entries [seg_off[l], seg_off[l+1]) and has its own Arnoldi
// process, Hessenberg matrix and Givens rotations, so independent problems iterate together
// and stop separately (converged lanes are masked).  Orthogonalisation is classical
// Gram-Schmidt applied twice (CGS2); every reduction is deterministic (fixed block partials).
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace mfs {

#define GM_THREADS 256

__device__ __forceinline__ double block_sum(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    v = (threadIdx.x < blockDim.x / 32) ? sh[threadIdx.x] : 0.0;
    if (wid == 0)
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    return v;  // valid in thread 0
}

__device__ __forceinline__ void lane_chunk(const GmresDev &gd, int l, int b, long long &e0, long long &e1) {
    const long long s0 = gd.seg_off[l], s1 = gd.seg_off[l + 1], len = s1 - s0;
    e0 = s0 + len * b / gd.part_blocks;
    e1 = s0 + len * (b + 1) / gd.part_blocks;
}

// part[l][b][i] = sum over chunk b of lane l of V[i][e] * w[e], i = 0..j  (grid: PB x L).  Eight
// columns at a time: w[e] is read once per group, eight accumulators per thread, one grouped block
// reduction (warp shuffles, then the warps' sums added in a fixed order) per group.
__global__ void mdot_kernel(GmresDev gd, const double *w) {
    constexpr int G = 8;
    const int b = blockIdx.x, l = blockIdx.y;
    if (!gd.active[l]) return;
    const int j = *gd.jcur;
    __shared__ double sh[GM_THREADS / 32][G];
    long long e0, e1;
    lane_chunk(gd, l, b, e0, e1);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i0 = 0; i0 <= j; i0 += G) {
        const int ng = min(G, j + 1 - i0);
        double acc[G];
#pragma unroll
        for (int g = 0; g < G; ++g) acc[g] = 0.0;
        for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
            const double we = w[e];
#pragma unroll
            for (int g = 0; g < G; ++g)
                if (g < ng) acc[g] += gd.V[(size_t)(i0 + g) * gd.n + e] * we;
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
            double v = acc[g];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) sh[wid][g] = v;
        }
        __syncthreads();
        if (threadIdx.x < ng) {
            double s = 0.0;
            for (int q = 0; q < nw; ++q) s += sh[q][threadIdx.x];
            gd.part[((size_t)l * gd.part_blocks + b) * (gd.m + 1) + i0 + threadIdx.x] = s;
        }
        __syncthreads();
    }
}

// Sum over the block partials of lane l, entry i, by one warp (lanes stride over the blocks, then a
// fixed shuffle tree: the same order every call).
__device__ __forceinline__ double warp_part_sum(const GmresDev &gd, int l, int i) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int b = lane; b < gd.part_blocks; b += 32) s += gd.part[((size_t)l * gd.part_blocks + b) * (gd.m + 1) + i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// hbuf[l][i] (+)= sum_b part[l][b][i]   (grid: L, one warp per entry i <= j, warps striding)
__global__ void mdot_reduce_kernel(GmresDev gd, double *htmp, int accumulate) {
    const int l = blockIdx.x;
    if (!gd.active[l]) return;
    const int j = *gd.jcur;
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = warp; i <= j; i += nw) {
        const double s = warp_part_sum(gd, l, i);
        if ((threadIdx.x & 31) == 0) {
            htmp[(size_t)l * (gd.m + 1) + i] = s;
            if (accumulate) gd.hbuf[(size_t)l * (gd.m + 1) + i] += s;
            else gd.hbuf[(size_t)l * (gd.m + 1) + i] = s;
        }
    }
}

// w -= sum_{i<=j} htmp[l][i] V[i]   (grid: PB x L)
__global__ void update_kernel(GmresDev gd, double *w, const double *htmp) {
    const int b = blockIdx.x, l = blockIdx.y;
    if (!gd.active[l]) return;
    const int j = *gd.jcur;
    __shared__ double h[1024];
    for (int i = threadIdx.x; i <= j; i += blockDim.x) h[i] = htmp[(size_t)l * (gd.m + 1) + i];
    __syncthreads();
    long long e0, e1;
    lane_chunk(gd, l, b, e0, e1);
    for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        // four independent FP64 chains (GB300's FP64 latency would serialise a single one)
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int i = 0;
        for (; i + 3 <= j; i += 4) {
            s0 += h[i] * gd.V[(size_t)i * gd.n + e];
            s1 += h[i + 1] * gd.V[(size_t)(i + 1) * gd.n + e];
            s2 += h[i + 2] * gd.V[(size_t)(i + 2) * gd.n + e];
            s3 += h[i + 3] * gd.V[(size_t)(i + 3) * gd.n + e];
        }
        for (; i <= j; ++i) s0 += h[i] * gd.V[(size_t)i * gd.n + e];
        w[e] -= (s0 + s1) + (s2 + s3);
    }
}

// part[l][b][0] = sum over chunk of x*x  (norms)
__global__ void norm_part_kernel(GmresDev gd, const double *x, int all_lanes) {
    const int b = blockIdx.x, l = blockIdx.y;
    if (!all_lanes && !gd.active[l]) return;
    __shared__ double sh[32];
    long long e0, e1;
    lane_chunk(gd, l, b, e0, e1);
    double acc = 0.0;
    for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) acc += x[e] * x[e];
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) gd.part[((size_t)l * gd.part_blocks + b) * (gd.m + 1)] = acc;
}

// v_dst = x / ||x|| per lane, norm taken from the partials (grid: PB x L); vdst = V[j+1] when null
__global__ void normalise_kernel(GmresDev gd, const double *x, double *vdst, double *norm_out, int all_lanes) {
    const int b = blockIdx.x, l = blockIdx.y;
    if (!all_lanes && !gd.active[l]) return;
    if (!vdst) vdst = gd.V + (size_t)(*gd.jcur + 1) * gd.n;
    __shared__ double nrm_sh;
    if (threadIdx.x < 32) {  // the first warp sums the block partials of the squared norm
        const double s = warp_part_sum(gd, l, 0);
        if (threadIdx.x == 0) nrm_sh = sqrt(s);
    }
    __syncthreads();
    const double nrm = nrm_sh;
    if (b == 0 && threadIdx.x == 0 && norm_out) norm_out[l] = nrm;
    const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
    long long e0, e1;
    lane_chunk(gd, l, b, e0, e1);
    for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) vdst[e] = x[e] * inv;
}

__global__ void init_lanes_kernel(GmresDev gd) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= gd.L) return;
    const double b = gd.beta[l];
    gd.g[(size_t)l * (gd.m + 1)] = b;
    gd.active[l] = (b > 0.0 && isfinite(b)) ? 1 : 0;
    gd.iters[l] = 0;
    gd.resid[l] = (b > 0.0) ? 1.0 : 0.0;
    gd.status[l] = isfinite(b) ? 0 : 2;
}

// done = no lane active, j = 0 (one thread)
__global__ void init_done_kernel(GmresDev gd) {
    int any = 0;
    for (int l = 0; l < gd.L; ++l) any |= gd.active[l];
    *gd.done = any ? 0 : 1;
    *gd.jcur = 0;
}

__global__ void load_vj_kernel(GmresDev gd, double *vin) {
    const double *v = gd.V + (size_t)(*gd.jcur) * gd.n;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < gd.n; e += (long long)gridDim.x * blockDim.x)
        vin[e] = v[e];
}

// After column j: continue with j + 1 unless every lane stopped or the basis is full.
__global__ void advance_kernel(GmresDev gd, cudaGraphConditionalHandle cond, int cond_valid) {
    const int j = *gd.jcur;
    const int more = (*gd.done == 0) && (j + 1 < gd.m);
    if (more) *gd.jcur = j + 1;
    if (cond_valid) cudaGraphSetConditional(cond, more ? 1u : 0u);
}

// Givens update of column j for every active lane; sets done when no lane is active.
__global__ void givens_kernel(GmresDev gd, const double *hn) {
    const int l = threadIdx.x;
    const int j = *gd.jcur;
    __shared__ int any_active;
    if (l == 0) any_active = 0;
    __syncthreads();
    for (int ll = l; ll < gd.L; ll += blockDim.x) {
        if (!gd.active[ll]) continue;
        const int m = gd.m;
        double *H = gd.H + (size_t)ll * (m + 1) * m;  // H[i][jj] at i*m + jj
        double *cs = gd.cs + (size_t)ll * m, *sn = gd.sn + (size_t)ll * m, *g = gd.g + (size_t)ll * (m + 1);
        for (int i = 0; i <= j; ++i) H[i * m + j] = gd.hbuf[(size_t)ll * (m + 1) + i];
        const double h_next = hn[ll];
        H[(j + 1) * m + j] = h_next;
        for (int i = 0; i < j; ++i) {
            const double a = H[i * m + j], c = H[(i + 1) * m + j];
            H[i * m + j] = cs[i] * a + sn[i] * c;
            H[(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
        }
        const double a = H[j * m + j], c = H[(j + 1) * m + j];
        const double den = hypot(a, c);
        cs[j] = den > 0.0 ? a / den : 1.0;
        sn[j] = den > 0.0 ? c / den : 0.0;
        H[j * m + j] = den;
        H[(j + 1) * m + j] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        gd.iters[ll] = j + 1;
        const double res = fabs(g[j + 1]) / gd.beta[ll];
        gd.resid[ll] = res;
        int keep = 1;
        if (!isfinite(res) || !isfinite(den)) {
            gd.status[ll] = 2;  // breakdown
            keep = 0;
        } else if (res <= gd.tol || h_next == 0.0 || j + 1 >= m) {
            keep = 0;
        }
        gd.active[ll] = keep;
        if (keep) atomicOr(&any_active, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) *gd.done = any_active ? 0 : 1;
}

// y_l solves the k_l x k_l upper-triangular H_l y = g_l (one thread per lane)
__global__ void trisolve_kernel(GmresDev gd, double *y) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= gd.L) return;
    const int m = gd.m, k = gd.iters[l];
    const double *H = gd.H + (size_t)l * (m + 1) * m;
    const double *g = gd.g + (size_t)l * (m + 1);
    double *yl = y + (size_t)l * (m + 1);
    for (int i = k - 1; i >= 0; --i) {
        double s = g[i];
        for (int c = i + 1; c < k; ++c) s -= H[i * m + c] * yl[c];
        yl[i] = (H[i * m + i] != 0.0) ? s / H[i * m + i] : 0.0;
    }
}

// x = sum_{i<k_l} y_l[i] V[i]  (grid: PB x L)
__global__ void combine_kernel(GmresDev gd, const double *y, double *x) {
    const int b = blockIdx.x, l = blockIdx.y;
    const int k = gd.iters[l];
    long long e0, e1;
    lane_chunk(gd, l, b, e0, e1);
    const double *yl = y + (size_t)l * (gd.m + 1);
    for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < k; ++i) s += yl[i] * gd.V[(size_t)i * gd.n + e];
        x[e] = s;
    }
}

cudaError_t gmres_init(GmresDev &gd, const double *b, cudaStream_t st) {
    dim3 grid(gd.part_blocks, gd.L);
    norm_part_kernel<<<grid, GM_THREADS, 0, st>>>(gd, b, 1);
    normalise_kernel<<<grid, GM_THREADS, 0, st>>>(gd, b, gd.V, gd.beta, 1);
    cudaMemsetAsync(gd.H, 0, sizeof(double) * (size_t)gd.L * (gd.m + 1) * gd.m, st);
    cudaMemsetAsync(gd.g, 0, sizeof(double) * (size_t)gd.L * (gd.m + 1), st);
    init_lanes_kernel<<<(gd.L + 127) / 128, 128, 0, st>>>(gd);
    init_done_kernel<<<1, 1, 0, st>>>(gd);
    return cudaGetLastError();
}

cudaError_t gmres_arnoldi(GmresDev &gd, double *w, cudaStream_t st) {
    dim3 grid(gd.part_blocks, gd.L);
    for (int pass = 0; pass < 2; ++pass) {  // CGS2
        mdot_kernel<<<grid, GM_THREADS, 0, st>>>(gd, w);
        mdot_reduce_kernel<<<gd.L, 512, 0, st>>>(gd, gd.htmp, pass);  // 16 warps over the entries i <= j
        update_kernel<<<grid, GM_THREADS, 0, st>>>(gd, w, gd.htmp);
    }
    norm_part_kernel<<<grid, GM_THREADS, 0, st>>>(gd, w, 0);
    normalise_kernel<<<grid, GM_THREADS, 0, st>>>(gd, w, nullptr, gd.hn, 0);
    givens_kernel<<<1, 256, 0, st>>>(gd, gd.hn);
    return cudaGetLastError();
}

cudaError_t gmres_load_vj(GmresDev &gd, double *vin, cudaStream_t st) {
    load_vj_kernel<<<1024, 256, 0, st>>>(gd, vin);
    return cudaGetLastError();
}

cudaError_t gmres_advance(GmresDev &gd, cudaGraphConditionalHandle cond, int cond_valid, cudaStream_t st) {
    advance_kernel<<<1, 1, 0, st>>>(gd, cond, cond_valid);
    return cudaGetLastError();
}

cudaError_t gmres_solution(GmresDev &gd, double *x, double *y_small, cudaStream_t st) {
    trisolve_kernel<<<(gd.L + 127) / 128, 128, 0, st>>>(gd, y_small);
    dim3 grid(gd.part_blocks, gd.L);
    combine_kernel<<<grid, GM_THREADS, 0, st>>>(gd, y_small, x);
    return cudaGetLastError();
}

}  // namespace mfs
