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

#define MDOT_THREADS 512

// Columns i0 .. i0+G-1 of one block's chunk: part[l][b][i] = sum over the chunk of V[i][e] * w[e].
// The loop is bound by memory latency, not by the FP64 pipe: 16 warps per block, four elements per
// step (4 (G + 1) independent loads in flight per thread).  The block's G x MDOT_THREADS partials go
// to shared memory and warp g adds column g's values in a fixed order (16 per lane, then a shuffle
// tree): GB300 executes FP64 at about 2 DFMA per clock per SM, so the reduction costs 21 FP64
// instructions per column per block rather than a shuffle tree per thread and column.
template <int G>
__device__ __forceinline__ void mdot_group(const GmresDev &gd, const double *w, long long e0, long long e1, int i0,
                                           double *sh, double *dst) {
    double acc[G];
#pragma unroll
    for (int g = 0; g < G; ++g) acc[g] = 0.0;
    const double *V = gd.V + (size_t)i0 * gd.n;
    const long long step = blockDim.x;
    long long e = e0 + threadIdx.x;
    for (; e + 3 * step < e1; e += 4 * step) {
        double we[4], v[G][4];
#pragma unroll
        for (int u = 0; u < 4; ++u) we[u] = w[e + u * step];
#pragma unroll
        for (int g = 0; g < G; ++g)
#pragma unroll
            for (int u = 0; u < 4; ++u) v[g][u] = V[(size_t)g * gd.n + e + u * step];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int g = 0; g < G; ++g) acc[g] = fma(v[g][u], we[u], acc[g]);
    }
    for (; e < e1; e += step) {
        const double we = w[e];
#pragma unroll
        for (int g = 0; g < G; ++g) acc[g] = fma(V[(size_t)g * gd.n + e], we, acc[g]);
    }
#pragma unroll
    for (int g = 0; g < G; ++g) sh[g * MDOT_THREADS + threadIdx.x] = acc[g];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int g = warp; g < G; g += nw) {
        double r = 0.0;
        for (int k = lane; k < (int)blockDim.x; k += 32) r += sh[g * MDOT_THREADS + k];
        for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
        if (lane == 0) dst[i0 + g] = r;
    }
    __syncthreads();
}

// part[l][b][i] = sum over chunk b of lane l of V[i][e] * w[e], i = 0..j  (grid: PB x L, MDOT_THREADS
// threads): groups of 8 columns, then one group of 4, 2 and 1 for the rest (no predicated-off FP64
// work).
__global__ void __launch_bounds__(MDOT_THREADS) mdot_kernel(GmresDev gd, const double *w) {
    const int b = blockIdx.x, l = blockIdx.y;
    if (!gd.active[l]) return;
    const int j = *gd.jcur;
    __shared__ double sh[8 * MDOT_THREADS];
    long long e0, e1;
    lane_chunk(gd, l, b, e0, e1);
    double *dst = gd.part + ((size_t)l * gd.part_blocks + b) * (gd.m + 1);
    int i0 = 0;
    for (; i0 + 8 <= j + 1; i0 += 8) mdot_group<8>(gd, w, e0, e1, i0, sh, dst);
    if (j + 1 - i0 >= 4) { mdot_group<4>(gd, w, e0, e1, i0, sh, dst); i0 += 4; }
    if (j + 1 - i0 >= 2) { mdot_group<2>(gd, w, e0, e1, i0, sh, dst); i0 += 2; }
    if (j + 1 - i0 >= 1) mdot_group<1>(gd, w, e0, e1, i0, sh, dst);
}

// Sum over the block partials of lane l, entry i, by one warp: each lane adds its blocks (four
// independent loads per step), then a fixed shuffle tree -- the same order every call.
__device__ __forceinline__ double warp_part_sum(const GmresDev &gd, int l, int i) {
    const int lane = threadIdx.x & 31;
    const double *p = gd.part + (size_t)l * gd.part_blocks * (gd.m + 1) + i;
    const size_t stride = (size_t)(gd.m + 1);
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int b = lane;
    for (; b + 96 < gd.part_blocks; b += 128) {
        s0 += p[(size_t)b * stride];
        s1 += p[(size_t)(b + 32) * stride];
        s2 += p[(size_t)(b + 64) * stride];
        s3 += p[(size_t)(b + 96) * stride];
    }
    for (; b < gd.part_blocks; b += 32) s0 += p[(size_t)b * stride];
    double s = (s0 + s1) + (s2 + s3);
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

// w -= sum_{i<=j} htmp[l][i] V[i]   (grid: PB x L).  Four elements per step and eight columns per
// inner step, so that 32 independent loads are in flight per thread (the kernel is bound by memory
// latency); each element's sum runs over the columns in order (one FP64 chain per element).
__global__ void __launch_bounds__(2 * GM_THREADS) update_kernel(GmresDev gd, double *w, const double *htmp) {
    const int b = blockIdx.x, l = blockIdx.y;
    if (!gd.active[l]) return;
    const int j = *gd.jcur;
    __shared__ double h[1024];
    for (int i = threadIdx.x; i <= j; i += blockDim.x) h[i] = htmp[(size_t)l * (gd.m + 1) + i];
    __syncthreads();
    long long e0, e1;
    lane_chunk(gd, l, b, e0, e1);
    const long long step = blockDim.x;
    long long e = e0 + threadIdx.x;
    for (; e + 3 * step < e1; e += 4 * step) {
        double a[4] = {0.0, 0.0, 0.0, 0.0};
        int i = 0;
        for (; i + 8 <= j + 1; i += 8) {
            const double *V = gd.V + (size_t)i * gd.n + e;
            double v[8][4];
#pragma unroll
            for (int g = 0; g < 8; ++g)
#pragma unroll
                for (int u = 0; u < 4; ++u) v[g][u] = V[(size_t)g * gd.n + u * step];
#pragma unroll
            for (int g = 0; g < 8; ++g)
#pragma unroll
                for (int u = 0; u < 4; ++u) a[u] = fma(h[i + g], v[g][u], a[u]);
        }
        for (; i <= j; ++i) {
            const double *V = gd.V + (size_t)i * gd.n + e;
#pragma unroll
            for (int u = 0; u < 4; ++u) a[u] = fma(h[i], V[u * step], a[u]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) w[e + u * step] -= a[u];
    }
    for (; e < e1; e += step) {
        double a = 0.0;
        for (int i = 0; i <= j; ++i) a = fma(h[i], gd.V[(size_t)i * gd.n + e], a);
        w[e] -= a;
    }
}

// part[l][b][0] = sum over chunk of x*x  (norms)
__global__ void norm_part_kernel(GmresDev gd, const double *x, int all_lanes) {
    const int b = blockIdx.x, l = blockIdx.y;
    if (!all_lanes && !gd.active[l]) return;
    __shared__ double sh[32];
    long long e0, e1;
    lane_chunk(gd, l, b, e0, e1);
    // four elements per step: independent loads in flight (the loop is bound by memory latency)
    const long long step = blockDim.x;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    long long e = e0 + threadIdx.x;
    for (; e + 3 * step < e1; e += 4 * step) {
        const double x0 = x[e], x1 = x[e + step], x2 = x[e + 2 * step], x3 = x[e + 3 * step];
        a0 = fma(x0, x0, a0);
        a1 = fma(x1, x1, a1);
        a2 = fma(x2, x2, a2);
        a3 = fma(x3, x3, a3);
    }
    for (; e < e1; e += step) a0 = fma(x[e], x[e], a0);
    double acc = (a0 + a1) + (a2 + a3);
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
    const long long step = blockDim.x;
    long long e = e0 + threadIdx.x;
    for (; e + 3 * step < e1; e += 4 * step) {
        const double x0 = x[e], x1 = x[e + step], x2 = x[e + 2 * step], x3 = x[e + 3 * step];
        vdst[e] = x0 * inv;
        vdst[e + step] = x1 * inv;
        vdst[e + 2 * step] = x2 * inv;
        vdst[e + 3 * step] = x3 * inv;
    }
    for (; e < e1; e += step) vdst[e] = x[e] * inv;
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
        // column j from hbuf, rotated by the previous Givens rotations with one value carried in a
        // register (the loads of hbuf, cs and sn do not wait on the chain; H is written once)
        const double *hcol = gd.hbuf + (size_t)ll * (m + 1);
        const double h_next = hn[ll];
        double carry = hcol[0];
        for (int i = 0; i < j; ++i) {
            const double c = hcol[i + 1];
            H[i * m + j] = cs[i] * carry + sn[i] * c;
            carry = -sn[i] * carry + cs[i] * c;
        }
        const double a = carry, c = h_next;
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
        mdot_kernel<<<grid, MDOT_THREADS, 0, st>>>(gd, w);
        mdot_reduce_kernel<<<gd.L, 512, 0, st>>>(gd, gd.htmp, pass);  // 16 warps over the entries i <= j
        update_kernel<<<grid, 2 * GM_THREADS, 0, st>>>(gd, w, gd.htmp);  // latency-bound: more loads in flight
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
