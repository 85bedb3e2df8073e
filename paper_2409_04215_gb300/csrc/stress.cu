// Pressure and surface traction of the Stokeslet representation at evaluation points (Eq. traction):
// for a source of strength lambda at y and r = x - y,
//   p   = (r . lambda) / (4 pi r^3)                        (the pressure solution Pi = 2 r / r^3, x 1/(8 pi))
//   T_i = sigma_ik n_k = -3 r_i (r . n)(r . lambda) / (4 pi r^5),
// both independent of the viscosity.  One thread per evaluation point (points grouped by owner body),
// looping over every source of the owner's suspension (or, with the far-field treecode, over the
// owner's interaction list of bodies and tree nodes); sources are read as broadcasts (a warp's
// points mostly share a suspension).  FP32: body-relative coordinates r = (c_owner - c_src) + x_loc -
// y_loc and FP32 partials per source body added into (hi, lo) pairs by TwoSum, as in the pair kernel;
// FP64: plain double loops (the reference path).
#include "common.cuh"
#include "kernels.h"

namespace mfs {

namespace {
constexpr double kInv4Pi = 0.07957747154594767;  // 1 / (4 pi)

// One source segment (a body's proxy records, or a tree node's equivalent records) at the target
// xr (relative to the segment's centre), folded into the (hi, lo) sums by TwoSum.
template <int NRHS>
__device__ __forceinline__ void stress_segment(float xr, float yr, float zr, float n0, float n1, float n2,
                                               const float *__restrict__ rec, int rec_floats, int j0, int j1,
                                               float (&ph)[NRHS], float (&pl)[NRHS], float (&th)[NRHS][3],
                                               float (&tl)[NRHS][3]) {
    float bp[NRHS], bt[NRHS][3];
#pragma unroll
    for (int h = 0; h < NRHS; ++h) {
        bp[h] = 0.f;
        bt[h][0] = bt[h][1] = bt[h][2] = 0.f;
    }
    constexpr int RV = (3 + 3 * NRHS + 3) / 4;  // float4 loads per record (plain layout, padded to 4 floats)
    for (int j = j0; j < j1; ++j) {
        // the record in 16-byte loads: rec_floats is a multiple of 4 and the buffer 256-byte aligned
        const float4 *s4 = reinterpret_cast<const float4 *>(rec + (size_t)j * rec_floats);
        float s[4 * RV];
#pragma unroll
        for (int v = 0; v < RV; ++v) {
            const float4 f = __ldg(s4 + v);
            s[4 * v] = f.x;
            s[4 * v + 1] = f.y;
            s[4 * v + 2] = f.z;
            s[4 * v + 3] = f.w;
        }
        const float rx = xr - s[0], ry = yr - s[1], rz = zr - s[2];
        const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
        const float ir = rsqrtf(r2);
        const float ir3 = ir * ir * ir;
        const float rn = fmaf(rx, n0, fmaf(ry, n1, rz * n2));
        const float q5 = rn * ir3 * ir * ir;
#pragma unroll
        for (int h = 0; h < NRHS; ++h) {
            const float lx = s[3 + 3 * h], ly = s[4 + 3 * h], lz = s[5 + 3 * h];
            const float rl = fmaf(rx, lx, fmaf(ry, ly, rz * lz));
            bp[h] = fmaf(rl, ir3, bp[h]);
            const float q = rl * q5;
            bt[h][0] = fmaf(rx, q, bt[h][0]);
            bt[h][1] = fmaf(ry, q, bt[h][1]);
            bt[h][2] = fmaf(rz, q, bt[h][2]);
        }
    }
#pragma unroll
    for (int h = 0; h < NRHS; ++h) {
        float sum, err;
        two_sum(ph[h], bp[h], sum, err);
        ph[h] = sum;
        pl[h] += err;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            two_sum(th[h][c], bt[h][c], sum, err);
            th[h][c] = sum;
            tl[h][c] += err;
        }
    }
}

template <int NRHS>
__global__ void __launch_bounds__(128) stress_f32_kernel(const float4 *__restrict__ tgt, const float *__restrict__ nrm,
                                                         int np, const float *__restrict__ rec, int rec_floats,
                                                         const int *__restrict__ rec_off, const int *__restrict__ sb0,
                                                         const int *__restrict__ sb1, const double *__restrict__ centres,
                                                         double *p_out, double *t_out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= np) return;
    const float4 x4 = tgt[t];
    const int kt = __float_as_int(x4.w);
    const bool want_t = nrm != nullptr;
    float n0 = 0.f, n1 = 0.f, n2 = 0.f;
    if (want_t) {
        n0 = nrm[3 * (size_t)t];
        n1 = nrm[3 * (size_t)t + 1];
        n2 = nrm[3 * (size_t)t + 2];
    }
    float ph[NRHS], pl[NRHS], th[NRHS][3], tl[NRHS][3];
#pragma unroll
    for (int h = 0; h < NRHS; ++h) {
        ph[h] = pl[h] = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) th[h][c] = tl[h][c] = 0.f;
    }
    const double cx = centres[3 * kt], cy = centres[3 * kt + 1], cz = centres[3 * kt + 2];
    for (int kb = sb0[kt]; kb < sb1[kt]; ++kb) {
        const float xr = (float)(cx - centres[3 * kb]) + x4.x;
        const float yr = (float)(cy - centres[3 * kb + 1]) + x4.y;
        const float zr = (float)(cz - centres[3 * kb + 2]) + x4.z;
        stress_segment<NRHS>(xr, yr, zr, n0, n1, n2, rec, rec_floats, rec_off[kb], rec_off[kb + 1], ph, pl, th, tl);
    }
#pragma unroll
    for (int h = 0; h < NRHS; ++h) {
        if (p_out) p_out[(size_t)h * np + t] = kInv4Pi * ((double)ph[h] + (double)pl[h]);
        if (t_out && want_t)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                t_out[((size_t)h * np + t) * 3 + c] = -3.0 * kInv4Pi * ((double)th[h][c] + (double)tl[h][c]);
    }
}

// The same sums over an interaction list per owner (the far-field treecode): targets in the tree's
// order with the owner's tree position in w, segment seg = lst_seg[lst_off[q] ..] with its records
// [seg_rec0[seg], seg_rec1[seg]) and its centre at centres[seg]; results written to index perm[t].
template <int NRHS>
__global__ void __launch_bounds__(128) stress_list_f32_kernel(const float4 *__restrict__ tgt, const float *__restrict__ nrm,
                                                              int np, const float *__restrict__ rec, int rec_floats,
                                                              const int *__restrict__ lst_off,
                                                              const int *__restrict__ lst_seg,
                                                              const int *__restrict__ seg_rec0,
                                                              const int *__restrict__ seg_rec1,
                                                              const double *__restrict__ centres,
                                                              const int *__restrict__ perm, double *p_out,
                                                              double *t_out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= np) return;
    const float4 x4 = tgt[t];
    const int q = __float_as_int(x4.w);
    const bool want_t = nrm != nullptr;
    float n0 = 0.f, n1 = 0.f, n2 = 0.f;
    if (want_t) {
        n0 = nrm[3 * (size_t)t];
        n1 = nrm[3 * (size_t)t + 1];
        n2 = nrm[3 * (size_t)t + 2];
    }
    float ph[NRHS], pl[NRHS], th[NRHS][3], tl[NRHS][3];
#pragma unroll
    for (int h = 0; h < NRHS; ++h) {
        ph[h] = pl[h] = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) th[h][c] = tl[h][c] = 0.f;
    }
    const double cx = centres[3 * q], cy = centres[3 * q + 1], cz = centres[3 * q + 2];
    for (int i = lst_off[q]; i < lst_off[q + 1]; ++i) {
        const int sg = lst_seg[i];
        const float xr = (float)(cx - centres[3 * sg]) + x4.x;
        const float yr = (float)(cy - centres[3 * sg + 1]) + x4.y;
        const float zr = (float)(cz - centres[3 * sg + 2]) + x4.z;
        stress_segment<NRHS>(xr, yr, zr, n0, n1, n2, rec, rec_floats, seg_rec0[sg], seg_rec1[sg], ph, pl, th, tl);
    }
    const int o = perm[t];
#pragma unroll
    for (int h = 0; h < NRHS; ++h) {
        if (p_out) p_out[(size_t)h * np + o] = kInv4Pi * ((double)ph[h] + (double)pl[h]);
        if (t_out && want_t)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                t_out[((size_t)h * np + o) * 3 + c] = -3.0 * kInv4Pi * ((double)th[h][c] + (double)tl[h][c]);
    }
}

__global__ void __launch_bounds__(128) stress_f64_kernel(const double *__restrict__ tgt_local, const int *__restrict__ tbody,
                                                         const double *__restrict__ nrm, int np, int nrhs,
                                                         const double *__restrict__ src_local, const int *__restrict__ src_off,
                                                         int sum_N, const double *__restrict__ lam, const int *__restrict__ sb0,
                                                         const int *__restrict__ sb1, const double *__restrict__ centres,
                                                         double *p_out, double *t_out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= np) return;
    const int kt = tbody[t];
    for (int h = 0; h < nrhs; ++h) {
        double p = 0.0, T[3] = {0.0, 0.0, 0.0};
        for (int kb = sb0[kt]; kb < sb1[kt]; ++kb) {
            const double xr[3] = {centres[3 * kt] - centres[3 * kb] + tgt_local[3 * (size_t)t],
                                  centres[3 * kt + 1] - centres[3 * kb + 1] + tgt_local[3 * (size_t)t + 1],
                                  centres[3 * kt + 2] - centres[3 * kb + 2] + tgt_local[3 * (size_t)t + 2]};
            for (int j = src_off[kb]; j < src_off[kb + 1]; ++j) {
                const double r[3] = {xr[0] - src_local[3 * (size_t)j], xr[1] - src_local[3 * (size_t)j + 1],
                                     xr[2] - src_local[3 * (size_t)j + 2]};
                const double *l = lam + ((size_t)h * sum_N + j) * 3;
                const double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
                const double ir = 1.0 / sqrt(r2);
                const double ir3 = ir * ir * ir;
                const double rl = r[0] * l[0] + r[1] * l[1] + r[2] * l[2];
                p += rl * ir3;
                if (nrm) {
                    const double q = rl * (r[0] * nrm[3 * (size_t)t] + r[1] * nrm[3 * (size_t)t + 1] +
                                           r[2] * nrm[3 * (size_t)t + 2]) * ir3 * ir * ir;
                    for (int c = 0; c < 3; ++c) T[c] += r[c] * q;
                }
            }
        }
        if (p_out) p_out[(size_t)h * np + t] = kInv4Pi * p;
        if (t_out && nrm)
            for (int c = 0; c < 3; ++c) t_out[((size_t)h * np + t) * 3 + c] = -3.0 * kInv4Pi * T[c];
    }
}
}  // namespace

cudaError_t stress_f32(int nrhs, const float4 *tgt, const float *nrm, int np, const float *rec, int rec_floats,
                       const int *rec_off, const int *sb0, const int *sb1, const double *centres, double *p_out,
                       double *t_out, cudaStream_t st) {
    if (np == 0) return cudaSuccess;
    const unsigned grid = (unsigned)((np + 127) / 128);
    switch (nrhs) {
        case 1: stress_f32_kernel<1><<<grid, 128, 0, st>>>(tgt, nrm, np, rec, rec_floats, rec_off, sb0, sb1, centres, p_out, t_out); break;
        case 2: stress_f32_kernel<2><<<grid, 128, 0, st>>>(tgt, nrm, np, rec, rec_floats, rec_off, sb0, sb1, centres, p_out, t_out); break;
        case 3: stress_f32_kernel<3><<<grid, 128, 0, st>>>(tgt, nrm, np, rec, rec_floats, rec_off, sb0, sb1, centres, p_out, t_out); break;
        case 4: stress_f32_kernel<4><<<grid, 128, 0, st>>>(tgt, nrm, np, rec, rec_floats, rec_off, sb0, sb1, centres, p_out, t_out); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t stress_list_f32(int nrhs, const float4 *tgt, const float *nrm, int np, const float *rec, int rec_floats,
                            const int *lst_off, const int *lst_seg, const int *seg_rec0, const int *seg_rec1,
                            const double *centres, const int *perm, double *p_out, double *t_out, cudaStream_t st) {
    if (np == 0) return cudaSuccess;
    const unsigned grid = (unsigned)((np + 127) / 128);
#define SL(R_)                                                                                                 \
    stress_list_f32_kernel<R_><<<grid, 128, 0, st>>>(tgt, nrm, np, rec, rec_floats, lst_off, lst_seg, seg_rec0, \
                                                     seg_rec1, centres, perm, p_out, t_out)
    switch (nrhs) {
        case 1: SL(1); break;
        case 2: SL(2); break;
        case 3: SL(3); break;
        case 4: SL(4); break;
        default: return cudaErrorInvalidValue;
    }
#undef SL
    return cudaGetLastError();
}

cudaError_t stress_f64(int nrhs, const double *tgt_local, const int *tbody, const double *nrm, int np,
                       const double *src_local, const int *src_off, int sum_N, const double *lam, const int *sb0,
                       const int *sb1, const double *centres, double *p_out, double *t_out, cudaStream_t st) {
    if (np == 0) return cudaSuccess;
    stress_f64_kernel<<<(unsigned)((np + 127) / 128), 128, 0, st>>>(tgt_local, tbody, nrm, np, nrhs, src_local,
                                                                    src_off, sum_N, lam, sb0, sb1, centres, p_out,
                                                                    t_out);
    return cudaGetLastError();
}

}  // namespace mfs
