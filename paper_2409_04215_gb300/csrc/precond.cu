// One-body preconditioner, setup and completion kernels.
//
//  * S_L = S^(00) (I - L) + L_r assembled in FP64 (Sec. 3.3; L, L_r of Sec. 3.1 and Eq. Lrsto),
//  * apply factors from its SVD S_L = U Sigma V^T (Eq. pseudo): U for the first step t = U^T g,
//    W = (I - L) V Sigma^+ for the second step of the projected apply used in the matvec
//    ((I - L^(k)) S_L^(k)+ of Eq. 2esysprec), and V Sigma^+ for the recovery lambda = S_L^+ gamma;
//    the product U^T-then-W is never formed (two-step apply, Eq. pseudo),
//  * rotation of congruent bodies: S_L^(k)+ = R_N V Sigma^+ U^T R_M^T (Remark congruent, Eq. Krot),
//  * completion strengths lambda_0 = K_N (K_N^T K_N)^{-1} [f; t] (Eq. lambda01, lambda02) and
//    alpha_0 = q/N 1 (Eq. al0); extraction U = -K_N^T lambda (Eq. getU), phi = -mean(alpha) (Eq. vkal).
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace mfs {

// (d)_x of Eq. Kdef: rows (0, d3, -d2), (-d3, 0, d1), (d2, -d1, 0); (d)_x w = w x d.
__device__ __forceinline__ double crossmat(const double *d, int row, int col) {
    const double m[3][3] = {{0.0, d[2], -d[1]}, {-d[2], 0.0, d[0]}, {d[1], -d[0], 0.0}};
    return m[row][col];
}

// Rigid-body matrix entry K[3q+b][m] for point p_q (Eq. Kdef).
__device__ __forceinline__ double kmat(const double *p, int b, int m) {
    return m < 3 ? (b == m ? 1.0 : 0.0) : crossmat(p, b, m - 3);
}

__device__ __forceinline__ double stokeslet(const double *x, const double *y, int a, int b, double mu) {
    const double r[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
    const double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    const double rn = sqrt(r2);
    return ((a == b ? 1.0 : 0.0) + r[a] * r[b] / r2) / (8.0 * MFS_PI * mu * rn);
}

__device__ __forceinline__ double laplace(const double *x, const double *y) {
    const double r[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
    return 1.0 / (4.0 * MFS_PI * sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]));
}

// P[row][m] = sum_j S0[row][j] K_N0[j][m] (Stokes, m < 6) or the row sum (Laplace, m = 0).
__global__ void build_P_kernel(int kind, int M, int N, const double *X0, const double *Y0, double mu, double *P) {
    const int row = blockIdx.x;
    const int D = kind == 1 ? 3 : 1;
    const int dN = D * N;
    const int i = row / D, a = row % D;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int col = threadIdx.x; col < dN; col += blockDim.x) {
        const int j = col / D, b = col % D;
        if (kind == 1) {
            const double s = stokeslet(X0 + 3 * i, Y0 + 3 * j, a, b, mu);
#pragma unroll
            for (int m = 0; m < 6; ++m) acc[m] += s * kmat(Y0 + 3 * j, b, m);
        } else {
            acc[0] += laplace(X0 + 3 * i, Y0 + 3 * j);
        }
    }
    __shared__ double red[6][256];
    for (int m = 0; m < 6; ++m) red[m][threadIdx.x] = acc[m];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int m = 0; m < 6; ++m) red[m][threadIdx.x] += red[m][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 6) P[(size_t)row * 6 + threadIdx.x] = red[threadIdx.x][0];
}

// SL (column-major dM x dN) = S0 - S0 L + L_r, or the bare self block S0 (Sec. 2.3) when bare.
__global__ void build_SL_kernel(int kind, int M, int N, const double *X0, const double *Y0, double mu,
                                const double *G0inv, const double *P, int bare, double *SL) {
    const int D = kind == 1 ? 3 : 1;
    const long long dM = (long long)D * M, dN = (long long)D * N;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= dM * dN) return;
    const int row = (int)(idx % dM), col = (int)(idx / dM);
    const int i = row / D, a = row % D, j = col / D, b = col % D;
    double v;
    if (bare) {
        v = kind == 1 ? stokeslet(X0 + 3 * i, Y0 + 3 * j, a, b, mu) : laplace(X0 + 3 * i, Y0 + 3 * j);
    } else if (kind == 1) {
        const double *y = Y0 + 3 * j, *x = X0 + 3 * i;
        double kn[6];
#pragma unroll
        for (int m = 0; m < 6; ++m) kn[m] = kmat(y, b, m);
        double sl = 0.0;  // (S0 K_N0) G0^{-1} K_N0^T
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            double q = 0.0;
#pragma unroll
            for (int n = 0; n < 6; ++n) q += G0inv[m * 6 + n] * kn[n];
            sl += P[(size_t)row * 6 + m] * q;
        }
        double lr = 0.0;  // K_M0 K_N0^T
#pragma unroll
        for (int m = 0; m < 6; ++m) lr += kmat(x, a, m) * kn[m];
        v = stokeslet(x, y, a, b, mu) - sl + lr;
    } else {
        v = laplace(X0 + 3 * i, Y0 + 3 * j) - P[(size_t)row * 6] / N + 1.0 / N;
    }
    SL[idx] = v;
}

cudaError_t build_SL(int kind, int M, int N, const double *X0, const double *Y0, double mu, const double *G0inv,
                     int bare, double *SL, cudaStream_t st) {
    const int D = kind == 1 ? 3 : 1;
    double *P = nullptr;
    cudaError_t e = cudaMallocAsync(&P, sizeof(double) * 6 * D * M, st);
    if (e != cudaSuccess) return e;
    if (!bare) build_P_kernel<<<D * M, 256, 0, st>>>(kind, M, N, X0, Y0, mu, P);
    const long long total = (long long)D * M * D * N;
    build_SL_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(kind, M, N, X0, Y0, mu, G0inv, P, bare, SL);
    e = cudaGetLastError();
    cudaFreeAsync(P, st);
    return e;
}

// B[j][m] = sum_q VT[j][q] K_N0[q][m] then times G0^{-1} (Stokes); row mean of VT (Laplace).
__global__ void vt_kn_kernel(int kind, int N, int r, const double *VTcm, const double *Y0, const double *G0inv,
                             double *Bp) {
    const int j = blockIdx.x;
    const int D = kind == 1 ? 3 : 1;
    const int dN = D * N;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int q = threadIdx.x; q < dN; q += blockDim.x) {
        const double v = VTcm[j + (size_t)q * r];
        if (kind == 1) {
            const int p = q / 3, b = q % 3;
#pragma unroll
            for (int m = 0; m < 6; ++m) acc[m] += v * kmat(Y0 + 3 * p, b, m);
        } else {
            acc[0] += v;
        }
    }
    __shared__ double red[6][256];
    for (int m = 0; m < 6; ++m) red[m][threadIdx.x] = acc[m];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int m = 0; m < 6; ++m) red[m][threadIdx.x] += red[m][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (kind == 1) {
            for (int m = 0; m < 6; ++m) {
                double s = 0.0;
                for (int n = 0; n < 6; ++n) s += red[n][0] * G0inv[n * 6 + m];  // (VT K_N0) G0^{-1}
                Bp[(size_t)j * 6 + m] = s;
            }
        } else {
            Bp[(size_t)j * 6] = red[0][0] / N;
        }
    }
}

__global__ void apply_factor_kernel(int kind, int N, int dM, int r, const double *Ucm, const double *sinv,
                                    const double *VTcm, const double *Y0, const double *Bp, int bare, float *U,
                                    float *Wp, float *Wr, double *U64, double *Wp64, double *Wr64) {
    const int D = kind == 1 ? 3 : 1;
    const int dN = D * N;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nU = (long long)dM * r, nW = (long long)r * dN;
    if (idx < nU) {  // U row-major [dM][r]
        const int i = (int)(idx / r), j = (int)(idx % r);
        const double u = Ucm[i + (size_t)j * dM];
        U[idx] = (float)u;
        if (U64) U64[idx] = u;
    }
    if (idx < nW) {  // W rows j, columns i (row-major [r][dN])
        const int j = (int)(idx / dN), i = (int)(idx % dN);
        const double vt = VTcm[j + (size_t)i * r];
        double proj;
        if (bare) {  // no projector: the Dirichlet apply V Sigma^+ U^T is used unprojected throughout
            proj = 0.0;
        } else if (kind == 1) {
            const int p = i / 3, b = i % 3;
            proj = 0.0;
#pragma unroll
            for (int m = 0; m < 6; ++m) proj += Bp[(size_t)j * 6 + m] * kmat(Y0 + 3 * p, b, m);
        } else {
            proj = Bp[(size_t)j * 6];
        }
        const double wr = sinv[j] * vt, wp = sinv[j] * (vt - proj);
        Wr[idx] = (float)wr;
        Wp[idx] = (float)wp;
        if (Wr64) {
            Wr64[idx] = wr;
            Wp64[idx] = wp;
        }
    }
}

cudaError_t build_apply_factors(int kind, int M, int N, const double *Ucm, const double *sigma, const double *VTcm,
                                const double *Y0, const double *G0inv, double eps_trunc, int bare, ShapeDev &sd,
                                cudaStream_t st) {
    const int D = kind == 1 ? 3 : 1;
    const int dM = D * M, dN = D * N, r = dN;
    // sigma is copied to the host by the caller; sinv computed here on the host copy
    double *hs = new double[r];
    cudaError_t e = cudaMemcpyAsync(hs, sigma, sizeof(double) * r, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        delete[] hs;
        return e;
    }
    double *hsinv = new double[r];
    sd.sigma1 = hs[0];
    sd.sigma_min = hs[0];
    for (int j = 0; j < r; ++j) {
        const bool keep = hs[j] > hs[0] * eps_trunc && hs[j] > 0.0;
        hsinv[j] = keep ? 1.0 / hs[j] : 0.0;
        if (keep) sd.sigma_min = hs[j];
    }
    double *sinv = nullptr, *Bp = nullptr;
    e = cudaMallocAsync(&sinv, sizeof(double) * r, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&Bp, sizeof(double) * 6 * r, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sinv, hsinv, sizeof(double) * r, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        if (!bare) vt_kn_kernel<<<r, 256, 0, st>>>(kind, N, r, VTcm, Y0, G0inv, Bp);
        const long long nmax = (long long)dM * r > (long long)r * dN ? (long long)dM * r : (long long)r * dN;
        apply_factor_kernel<<<(unsigned)((nmax + 255) / 256), 256, 0, st>>>(kind, N, dM, r, Ucm, sinv, VTcm, Y0, Bp,
                                                                             bare, sd.U, sd.Wp, sd.Wr, sd.U64,
                                                                             sd.Wp64, sd.Wr64);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFreeAsync(sinv, st);
    cudaFreeAsync(Bp, st);
    delete[] hs;
    delete[] hsinv;
    return e;
}

// ---------------------------------------------------------------------------
// Gather / scatter with per-body rotation
// ---------------------------------------------------------------------------
__global__ void gather_rotate_kernel(int D, const double *gamma, int sum_MD, const int *col_body, const int *col_rhs,
                                     const int *body_tgt_off, const double *rot, int ncols, int dM, float *A,
                                     double *A64) {
    const int col = blockIdx.y;
    const int M = dM / D;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= M || col >= ncols) return;
    const int k = col_body[col], h = col_rhs[col];
    const double *gk = gamma + (size_t)h * sum_MD + (size_t)body_tgt_off[k] * D;
    if (D == 1) {
        const double v = gk[p];
        A[(size_t)col * dM + p] = (float)v;
        if (A64) A64[(size_t)col * dM + p] = v;
    } else {
        const double *R = rot + 9 * k;  // row-major R (FP64); (R^T g)_a = sum_b R[b][a] g_b
        const double g0 = gk[3 * p], g1 = gk[3 * p + 1], g2 = gk[3 * p + 2];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double v = R[a] * g0 + R[3 + a] * g1 + R[6 + a] * g2;
            A[(size_t)col * dM + 3 * p + a] = (float)v;
            if (A64) A64[(size_t)col * dM + 3 * p + a] = v;
        }
    }
}

cudaError_t gather_rotate(int D, const double *gamma, int sum_MD, const int *col_body, const int *col_rhs,
                          const int *body_tgt_off, const double *rot, int ncols, int dM, float *A, double *A64,
                          cudaStream_t st) {
    if (ncols == 0) return cudaSuccess;
    const int M = dM / D;
    dim3 grid((M + 127) / 128, ncols);
    gather_rotate_kernel<<<grid, 128, 0, st>>>(D, gamma, sum_MD, col_body, col_rhs, body_tgt_off, rot, ncols, dM, A,
                                                A64);
    return cudaGetLastError();
}

__global__ void scatter_rotate_kernel(int D, const float *L, const double *L64, const int *col_body,
                                      const int *col_rhs, const int *body_src_off, const double *rot64, int ncols,
                                      int dN, int sum_N, double *lambda) {
    const int col = blockIdx.y;
    const int N = dN / D;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N || col >= ncols) return;
    const int k = col_body[col], h = col_rhs[col];
    double *out = lambda + ((size_t)h * sum_N + body_src_off[k]) * D;
    if (D == 1) {
        out[p] = L64 ? L64[(size_t)col * dN + p] : (double)L[(size_t)col * dN + p];
    } else {
        double v[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) v[a] = L64 ? L64[(size_t)col * dN + 3 * p + a] : (double)L[(size_t)col * dN + 3 * p + a];
        const double *R = rot64 + 9 * k;
#pragma unroll
        for (int a = 0; a < 3; ++a) out[3 * p + a] = R[3 * a] * v[0] + R[3 * a + 1] * v[1] + R[3 * a + 2] * v[2];
    }
}

cudaError_t scatter_rotate(int D, const float *L, const double *L64, const int *col_body, const int *col_rhs,
                           const int *body_src_off, const float *rot, const double *rot64, int ncols, int dN,
                           int sum_N, double *lambda, cudaStream_t st) {
    (void)rot;
    if (ncols == 0) return cudaSuccess;
    const int N = dN / D;
    dim3 grid((N + 127) / 128, ncols);
    scatter_rotate_kernel<<<grid, 128, 0, st>>>(D, L, L64, col_body, col_rhs, body_src_off, rot64, ncols, dN, sum_N,
                                                 lambda);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Row-major GEMM C[m][n] = A[m][k] B[k][n]: 64x64 output tile, 16-deep k slices in shared
// memory, 4x4 outputs per thread (256 threads).  FP32 (matvec) and FP64 (reference path, far-field
// fits).  With gridDim.z > 1, CTA z sums only k in [z kchunk, (z + 1) kchunk) and writes its partial
// product to C + z m n (a split over K, summed afterwards in a fixed order).
// ---------------------------------------------------------------------------
template <typename TT>
__global__ void __launch_bounds__(256) gemm_rm_kernel(int m, int n, int k, const TT *__restrict__ A,
                                                      const TT *__restrict__ B, TT *__restrict__ C, int kchunk) {
    constexpr int BM = 64, BN = 64, BK = 16;
    __shared__ TT As[BK][BM + 4];
    __shared__ TT Bs[BK][BN + 4];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int kbeg = blockIdx.z * kchunk, kend = min(k, kbeg + kchunk);
    C += (size_t)blockIdx.z * m * n;
    TT acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0;
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
        for (int e = threadIdx.x; e < BM * BK; e += 256) {  // A tile: rows m0.., cols k0..
            const int r = e / BK, c = e % BK;
            const int gm = m0 + r, gk = k0 + c;
            As[c][r] = (gm < m && gk < kend) ? A[(size_t)gm * k + gk] : TT(0);
        }
        for (int e = threadIdx.x; e < BK * BN; e += 256) {
            const int r = e / BN, c = e % BN;
            const int gk = k0 + r, gn = n0 + c;
            Bs[r][c] = (gk < kend && gn < n) ? B[(size_t)gk * n + gn] : TT(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            TT a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gm = m0 + ty * 4 + i, gn = n0 + tx * 4 + j;
            if (gm < m && gn < n) C[(size_t)gm * n + gn] = acc[i][j];
        }
}

// Split-K FP32 GEMM with compensated accumulation: CTA (x, y, z) computes the 64x64 tile (y, x)
// over the z-th chunk of k.  Each 16-deep k slice is summed in FP32 from zero and folded into a
// per-output (hi, lo) pair by TwoSum, so the rounding of a long sequential FP32 sum (which, over
// k = 3600, limits the solved velocities to ~2e-5) never builds up; the chunk results are
// written in FP64 and added in FP64 by splitk_reduce_kernel.
template <bool TRANS_B>  // TRANS_B: B is stored [n][k] (C = A B^T)
__global__ void __launch_bounds__(256) gemm_splitk_kernel(int m, int n, int k, int kchunk,
                                                          const float *__restrict__ A,
                                                          const float *__restrict__ B, double *__restrict__ P) {
    constexpr int BM = 64, BN = 64, BK = 16;
    __shared__ float As[BK][BM + 4];
    __shared__ float Bs[BK][BN + 4];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int kb = blockIdx.z * kchunk, ke = min(k, kb + kchunk);
    float hi[4][4], lo[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) hi[i][j] = lo[i][j] = 0.f;
    for (int k0 = kb; k0 < ke; k0 += BK) {
        for (int e = threadIdx.x; e < BM * BK; e += 256) {
            const int r = e / BK, c = e % BK;
            const int gm = m0 + r, gk = k0 + c;
            As[c][r] = (gm < m && gk < ke) ? A[(size_t)gm * k + gk] : 0.f;
        }
        for (int e = threadIdx.x; e < BK * BN; e += 256) {
            if (TRANS_B) {  // consecutive threads read consecutive k of one row of B[n][k]
                const int c = e / BK, r = e % BK;
                const int gk = k0 + r, gn = n0 + c;
                Bs[r][c] = (gk < ke && gn < n) ? B[(size_t)gn * k + gk] : 0.f;
            } else {
                const int r = e / BN, c = e % BN;
                const int gk = k0 + r, gn = n0 + c;
                Bs[r][c] = (gk < ke && gn < n) ? B[(size_t)gk * n + gn] : 0.f;
            }
        }
        __syncthreads();
        float s[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) s[i][j] = 0.f;
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) s[i][j] = fmaf(a[i], b[j], s[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float t, e;
                two_sum(hi[i][j], s[i][j], t, e);
                hi[i][j] = t;
                lo[i][j] += e;
            }
        __syncthreads();
    }
    double *Pz = P + (size_t)blockIdx.z * m * n;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gm = m0 + ty * 4 + i, gn = n0 + tx * 4 + j;
            if (gm < m && gn < n) Pz[(size_t)gm * n + gn] = (double)hi[i][j] + (double)lo[i][j];
        }
}

// C = sum_z P[z] in FP64, stored as FP32 (C32) or FP64 (C64).
__global__ void splitk_reduce_kernel(int S, size_t mn, const double *__restrict__ P, float *C32, double *C64) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < mn; i += (size_t)gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int z = 0; z < S; ++z) v += P[(size_t)z * mn + i];
        if (C64) C64[i] = v;
        else C32[i] = (float)v;
    }
}

cudaError_t splitk_reduce(int S, size_t mn, const double *P, float *C32, double *C64, cudaStream_t st) {
    if (mn == 0) return cudaSuccess;
    splitk_reduce_kernel<<<(unsigned)std::min<size_t>((mn + 255) / 256, 4096), 256, 0, st>>>(S, mn, P, C32, C64);
    return cudaGetLastError();
}

int gemm_splitk_chunks(int m, int n, int k, int sm_count) {
    const long long tiles = (long long)((n + 63) / 64) * ((m + 63) / 64);
    long long s = (4LL * sm_count + tiles - 1) / tiles;  // about four resident waves of CTAs
    const long long smax = (k + 63) / 64;                // at least 64 k per chunk
    if (s > smax) s = smax;
    if (s > 32) s = 32;
    return (int)(s < 1 ? 1 : s);
}

cudaError_t gemm_splitk(int m, int n, int k, int S, const float *A, const float *B, double *P, float *C32,
                        double *C64, cudaStream_t st, bool trans_b) {
    if (m == 0 || n == 0) return cudaSuccess;
    const int kchunk = ((k + S - 1) / S + 15) / 16 * 16;
    const int Sz = (k + kchunk - 1) / kchunk;
    dim3 grid((n + 63) / 64, (m + 63) / 64, Sz);
    if (trans_b)
        gemm_splitk_kernel<true><<<grid, 256, 0, st>>>(m, n, k, kchunk, A, B, P);
    else
        gemm_splitk_kernel<false><<<grid, 256, 0, st>>>(m, n, k, kchunk, A, B, P);
    const size_t mn = (size_t)m * n;
    splitk_reduce_kernel<<<(unsigned)std::min<size_t>((mn + 255) / 256, 4096), 256, 0, st>>>(Sz, mn, P, C32, C64);
    return cudaGetLastError();
}

cudaError_t gemm_rm(int m, int n, int k, const float *A, const float *B, float *C, cudaStream_t st) {
    if (m == 0 || n == 0) return cudaSuccess;
    dim3 grid((n + 63) / 64, (m + 63) / 64);
    gemm_rm_kernel<float><<<grid, 256, 0, st>>>(m, n, k, A, B, C, k);
    return cudaGetLastError();
}

cudaError_t gemm_rm64(int m, int n, int k, const double *A, const double *B, double *C, cudaStream_t st) {
    if (m == 0 || n == 0) return cudaSuccess;
    dim3 grid((n + 63) / 64, (m + 63) / 64);
    gemm_rm_kernel<double><<<grid, 256, 0, st>>>(m, n, k, A, B, C, k);
    return cudaGetLastError();
}

int gemm_rm64_chunks(int m, int n, int k, int sm_count) {
    const int tiles = ((n + 63) / 64) * ((m + 63) / 64);
    int s = (2 * sm_count) / std::max(tiles, 1);  // about two CTAs per SM
    s = std::min(s, (k + 127) / 128);               // chunks of at least 128 of K
    return std::max(s, 1);
}

__global__ void sum_chunks_kernel(int S, size_t mn, const double *__restrict__ P, double *__restrict__ C) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < mn; i += (size_t)gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int z = 0; z < S; ++z) v += P[(size_t)z * mn + i];
        C[i] = v;
    }
}

cudaError_t gemm_rm64_splitk(int m, int n, int k, int S, const double *A, const double *B, double *P, double *C,
                             cudaStream_t st) {
    if (m == 0 || n == 0) return cudaSuccess;
    if (S <= 1) return gemm_rm64(m, n, k, A, B, C, st);
    const int kchunk = ((k + S - 1) / S + 15) / 16 * 16;
    const int Sz = (k + kchunk - 1) / kchunk;
    dim3 grid((n + 63) / 64, (m + 63) / 64, Sz);
    gemm_rm_kernel<double><<<grid, 256, 0, st>>>(m, n, k, A, B, P, kchunk);
    const size_t mn = (size_t)m * n;
    sum_chunks_kernel<<<(unsigned)std::min<size_t>((mn + 255) / 256, 4096), 256, 0, st>>>(Sz, mn, P, C);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Completion and extraction (FP64)
// ---------------------------------------------------------------------------
__global__ void completion_stokes_kernel(const double *F, const double *T, int P, const double *rot64,
                                         const double *G0inv_shapes, const int *shape_id, const double *src_local64,
                                         const int *body_src_off, int sum_N, double *lam0) {
    const int k = blockIdx.x, h = blockIdx.y;
    __shared__ double nx[6];
    if (threadIdx.x == 0) {
        const double *R = rot64 + 9 * k;
        const double *f = F + ((size_t)h * P + k) * 3, *t = T + ((size_t)h * P + k) * 3;
        double ft0[6];
        for (int a = 0; a < 3; ++a) {  // body frame: R^T f, R^T t
            ft0[a] = R[a] * f[0] + R[3 + a] * f[1] + R[6 + a] * f[2];
            ft0[3 + a] = R[a] * t[0] + R[3 + a] * t[1] + R[6 + a] * t[2];
        }
        const double *Gi = G0inv_shapes + 36 * shape_id[k];
        double a6[6];
        for (int m = 0; m < 6; ++m) {
            double s = 0.0;
            for (int n = 0; n < 6; ++n) s += Gi[m * 6 + n] * ft0[n];
            a6[m] = s;
        }
        for (int a = 0; a < 3; ++a) {  // back to the global frame
            nx[a] = R[3 * a] * a6[0] + R[3 * a + 1] * a6[1] + R[3 * a + 2] * a6[2];
            nx[3 + a] = R[3 * a] * a6[3] + R[3 * a + 1] * a6[4] + R[3 * a + 2] * a6[5];
        }
    }
    __syncthreads();
    const int b0 = body_src_off[k], b1 = body_src_off[k + 1];
    for (int q = b0 + threadIdx.x; q < b1; q += blockDim.x) {
        const double *y = src_local64 + 3 * (size_t)q;  // rotated, relative to the centre
        double *o = lam0 + ((size_t)h * sum_N + q) * 3;
        // nu + xi x y
        o[0] = nx[0] + nx[4] * y[2] - nx[5] * y[1];
        o[1] = nx[1] + nx[5] * y[0] - nx[3] * y[2];
        o[2] = nx[2] + nx[3] * y[1] - nx[4] * y[0];
    }
}

cudaError_t completion_stokes(const double *F, const double *T, int nrhs, int P, const double *rot64,
                              const double *G0inv_shapes, const int *shape_id, const double *src_local64,
                              const int *body_src_off, int sum_N, double *lam0, cudaStream_t st) {
    dim3 grid(P, nrhs);
    completion_stokes_kernel<<<grid, 128, 0, st>>>(F, T, P, rot64, G0inv_shapes, shape_id, src_local64, body_src_off,
                                                    sum_N, lam0);
    return cudaGetLastError();
}

__global__ void completion_laplace_kernel(const double *Q, int P, const int *body_src_off, int sum_N, double *a0) {
    const int k = blockIdx.x, h = blockIdx.y;
    const int b0 = body_src_off[k], b1 = body_src_off[k + 1];
    const double v = Q[(size_t)h * P + k] / (double)(b1 - b0);
    for (int q = b0 + threadIdx.x; q < b1; q += blockDim.x) a0[(size_t)h * sum_N + q] = v;
}

cudaError_t completion_laplace(const double *Q, int nrhs, int P, const int *body_src_off, int sum_N, double *alpha0,
                               cudaStream_t st) {
    dim3 grid(P, nrhs);
    completion_laplace_kernel<<<grid, 128, 0, st>>>(Q, P, body_src_off, sum_N, alpha0);
    return cudaGetLastError();
}

// Dirichlet data of the resistance problem: b = K_M U, the rigid motion v + omega x (x - c) at every
// collocation point (Sec. 2.2, Eq. Kdef, Eq. Kbig); tgt_local64 holds x - c.
__global__ void dirichlet_rhs_stokes_kernel(const double *U, const double *Om, int P, const double *tgt_local64,
                                            const int *body_tgt_off, int sum_M, double *b) {
    const int k = blockIdx.x, h = blockIdx.y;
    const double *v = U + ((size_t)h * P + k) * 3, *w = Om + ((size_t)h * P + k) * 3;
    for (int i = body_tgt_off[k] + threadIdx.x; i < body_tgt_off[k + 1]; i += blockDim.x) {
        const double *x = tgt_local64 + 3 * (size_t)i;
        double *o = b + ((size_t)h * sum_M + i) * 3;
        o[0] = v[0] + w[1] * x[2] - w[2] * x[1];
        o[1] = v[1] + w[2] * x[0] - w[0] * x[2];
        o[2] = v[2] + w[0] * x[1] - w[1] * x[0];
    }
}

// Dirichlet data of the capacitance problem: eta^(k) = phi^(k) 1_M (Sec. 2.1).
__global__ void dirichlet_rhs_laplace_kernel(const double *phi, int P, const int *body_tgt_off, int sum_M,
                                             double *b) {
    const int k = blockIdx.x, h = blockIdx.y;
    const double v = phi[(size_t)h * P + k];
    for (int i = body_tgt_off[k] + threadIdx.x; i < body_tgt_off[k + 1]; i += blockDim.x) b[(size_t)h * sum_M + i] = v;
}

cudaError_t dirichlet_rhs_stokes(const double *U, const double *Om, int nrhs, int P, const double *tgt_local64,
                                 const int *body_tgt_off, int sum_M, double *b, cudaStream_t st) {
    dim3 grid(P, nrhs);
    dirichlet_rhs_stokes_kernel<<<grid, 128, 0, st>>>(U, Om, P, tgt_local64, body_tgt_off, sum_M, b);
    return cudaGetLastError();
}

cudaError_t dirichlet_rhs_laplace(const double *phi, int nrhs, int P, const int *body_tgt_off, int sum_M, double *b,
                                  cudaStream_t st) {
    dim3 grid(P, nrhs);
    dirichlet_rhs_laplace_kernel<<<grid, 128, 0, st>>>(phi, P, body_tgt_off, sum_M, b);
    return cudaGetLastError();
}

// [U; Omega] = sign * K_N^T lambda: sign -1 extracts velocities (Eq. getU), +1 forces and torques
// (Eq. force_def).
__global__ void extract_stokes_kernel(const double *lam, int P, const double *src_local64, const int *body_src_off,
                                      int sum_N, double sign, double *U, double *Om) {
    const int k = blockIdx.x, h = blockIdx.y;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int q = body_src_off[k] + threadIdx.x; q < body_src_off[k + 1]; q += blockDim.x) {
        const double *l = lam + ((size_t)h * sum_N + q) * 3;
        const double *y = src_local64 + 3 * (size_t)q;
        acc[0] += l[0];
        acc[1] += l[1];
        acc[2] += l[2];
        acc[3] += y[1] * l[2] - y[2] * l[1];  // (y - c) x lambda
        acc[4] += y[2] * l[0] - y[0] * l[2];
        acc[5] += y[0] * l[1] - y[1] * l[0];
    }
    __shared__ double red[6][128];
    for (int m = 0; m < 6; ++m) red[m][threadIdx.x] = acc[m];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int m = 0; m < 6; ++m) red[m][threadIdx.x] += red[m][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 3) {
        U[((size_t)h * P + k) * 3 + threadIdx.x] = sign * red[threadIdx.x][0];
        Om[((size_t)h * P + k) * 3 + threadIdx.x] = sign * red[3 + threadIdx.x][0];
    }
}

cudaError_t extract_stokes(const double *lam, int nrhs, int P, const double *src_local64, const int *body_src_off,
                           int sum_N, double *U, double *Om, cudaStream_t st, double sign) {
    dim3 grid(P, nrhs);
    extract_stokes_kernel<<<grid, 128, 0, st>>>(lam, P, src_local64, body_src_off, sum_N, sign, U, Om);
    return cudaGetLastError();
}

// V = -mean(alpha) per body (Eq. vkal), or the net charge sum(alpha) when sum (Eq. qkgauss).
__global__ void extract_laplace_kernel(const double *alpha, int P, const int *body_src_off, int sum_N, int sum,
                                       double *V) {
    const int k = blockIdx.x, h = blockIdx.y;
    double acc = 0.0;
    const int b0 = body_src_off[k], b1 = body_src_off[k + 1];
    for (int q = b0 + threadIdx.x; q < b1; q += blockDim.x) acc += alpha[(size_t)h * sum_N + q];
    __shared__ double red[128];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) V[(size_t)h * P + k] = sum ? red[0] : -red[0] / (double)(b1 - b0);
}

cudaError_t extract_laplace(const double *alpha, int nrhs, int P, const int *body_src_off, int sum_N, double *V,
                            cudaStream_t st, int sum) {
    dim3 grid(P, nrhs);
    extract_laplace_kernel<<<grid, 128, 0, st>>>(alpha, P, body_src_off, sum_N, sum, V);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64 reference pair sum (precision = 1): one thread per target, plain loops.
// out_raw holds the sum without the 1/(4 pi) or 1/(8 pi mu) factor, layout [nrhs][nt][D].
// ---------------------------------------------------------------------------
__global__ void pair_sum_fp64_kernel(int D, int nrhs, const double *tgt_local, const int *tgt_body, int nt,
                                     const double *src_local4, int nsrc, const int *susp_src_begin,
                                     const int *susp_src_end, const int *body_src_off, const double *centres,
                                     const double *strength, int include_self, double *out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const int kt = tgt_body[t];
    const double x[3] = {centres[3 * kt] + tgt_local[3 * t], centres[3 * kt + 1] + tgt_local[3 * t + 1],
                         centres[3 * kt + 2] + tgt_local[3 * t + 2]};
    double acc[12];
    for (int c = 0; c < 12; ++c) acc[c] = 0.0;
    const int self0 = body_src_off[kt], self1 = body_src_off[kt + 1];
    for (int s = susp_src_begin[kt]; s < susp_src_end[kt]; ++s) {
        if (!include_self && s >= self0 && s < self1) continue;
        const double *yl = src_local4 + 4 * (size_t)s;  // x, y, z (rotated, body-local), source body
        const int kb = (int)yl[3];
        const double r[3] = {x[0] - (centres[3 * kb] + yl[0]), x[1] - (centres[3 * kb + 1] + yl[1]),
                             x[2] - (centres[3 * kb + 2] + yl[2])};
        const double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        const double ri = 1.0 / sqrt(r2);
        for (int h = 0; h < nrhs; ++h) {
            if (D == 1) {
                acc[h] += strength[(size_t)h * nsrc + s] * ri;
            } else {
                const double *l = strength + ((size_t)h * nsrc + s) * 3;
                const double dot = r[0] * l[0] + r[1] * l[1] + r[2] * l[2];
                for (int a = 0; a < 3; ++a) acc[3 * h + a] += (l[a] + r[a] * dot / r2) * ri;
            }
        }
    }
    for (int h = 0; h < nrhs; ++h)
        for (int a = 0; a < D; ++a) out[((size_t)h * nt + t) * D + a] = acc[D * h + a];
}

// FP64 reference of the adjoint's pair gradient (precision = 1): one thread per target,
//   out_t = sum_h sum_{s in t's suspension, not on t's body} grad_r (tw_h(t)^T G(r) sigma_h(s)),  r = x_t - y_s,
// G = I / r + r r^T / r^3 (raw, without 1 / (8 pi mu)), so grad_r = [w (r.m) + m (w.r) - (w.m) r
// - 3 (w.r)(r.m) r / r^2] / r^3 with w = tw_h(t), m = sigma_h(s).  Layouts as pair_sum_fp64; tw is
// [nrhs][nt][3], out [nt][3].
__global__ void grad_pair_fp64_kernel(int nrhs, const double *tgt_local, const int *tgt_body, int nt, const double *tw,
                                      const double *src_local4, int nsrc, const int *susp_src_begin,
                                      const int *susp_src_end, const int *body_src_off, const double *centres,
                                      const double *strength, double *out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const int kt = tgt_body[t];
    const double x[3] = {centres[3 * kt] + tgt_local[3 * t], centres[3 * kt + 1] + tgt_local[3 * t + 1],
                         centres[3 * kt + 2] + tgt_local[3 * t + 2]};
    double acc[3] = {0.0, 0.0, 0.0};
    const int self0 = body_src_off[kt], self1 = body_src_off[kt + 1];
    for (int s = susp_src_begin[kt]; s < susp_src_end[kt]; ++s) {
        if (s >= self0 && s < self1) continue;
        const double *yl = src_local4 + 4 * (size_t)s;
        const int kb = (int)yl[3];
        const double r[3] = {x[0] - (centres[3 * kb] + yl[0]), x[1] - (centres[3 * kb + 1] + yl[1]),
                             x[2] - (centres[3 * kb + 2] + yl[2])};
        const double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        const double ri = 1.0 / sqrt(r2);
        const double ri3 = ri * ri * ri;
        for (int h = 0; h < nrhs; ++h) {
            const double *w = tw + ((size_t)h * nt + t) * 3;
            const double *m = strength + ((size_t)h * nsrc + s) * 3;
            const double wm = w[0] * m[0] + w[1] * m[1] + w[2] * m[2];
            const double wr = w[0] * r[0] + w[1] * r[1] + w[2] * r[2];
            const double rm = r[0] * m[0] + r[1] * m[1] + r[2] * m[2];
            const double q = -(wm + 3.0 * wr * rm / r2);
            for (int a = 0; a < 3; ++a) acc[a] += (r[a] * q + w[a] * rm + m[a] * wr) * ri3;
        }
    }
    for (int a = 0; a < 3; ++a) out[3 * (size_t)t + a] = acc[a];
}

cudaError_t grad_pair_fp64(int nrhs, const double *tgt_local, const int *tgt_body, int ntargets, const double *tw,
                           const double *src_local4, int nsrc, const int *susp_src_begin, const int *susp_src_end,
                           const int *body_src_off, const double *centres, const double *strength, double *out,
                           cudaStream_t st) {
    const int threads = 128;
    if (ntargets == 0) return cudaSuccess;
    grad_pair_fp64_kernel<<<(ntargets + threads - 1) / threads, threads, 0, st>>>(
        nrhs, tgt_local, tgt_body, ntargets, tw, src_local4, nsrc, susp_src_begin, susp_src_end, body_src_off, centres,
        strength, out);
    return cudaGetLastError();
}

cudaError_t pair_sum_fp64(int D, int nrhs, const double *tgt_local, const int *tgt_body, int ntargets,
                          const double *src_local4, int nsrc, const int *susp_src_begin, const int *susp_src_end,
                          const int *body_src_off, const double *centres, const double *strength, int include_self,
                          double *out_raw, cudaStream_t st) {
    const int threads = 128;
    if (ntargets == 0) return cudaSuccess;
    pair_sum_fp64_kernel<<<(ntargets + threads - 1) / threads, threads, 0, st>>>(
        D, nrhs, tgt_local, tgt_body, ntargets, src_local4, nsrc, susp_src_begin, susp_src_end, body_src_off, centres,
        strength, include_self, out_raw);
    return cudaGetLastError();
}

}  // namespace mfs
