// FP64 reference (precision = 1) of the pressure and surface traction of the Stokeslet representation
// at evaluation points (Eq. traction): for a source of strength lambda at y and r = x - y,
//   p   = (r . lambda) / (4 pi r^3)                        (the pressure solution Pi = 2 r / r^3, x 1/(8 pi))
//   T_i = sigma_ik n_k = -3 r_i (r . n)(r . lambda) / (4 pi r^5),
// both independent of the viscosity.  One thread per evaluation point (points grouped by owner body),
// plain double loops over every source of the owner's suspension.  The FP32 path runs the same sums as
// the pair kernel's stress entry (StressStokes in pair_kernel.cu).
#include "common.cuh"
#include "kernels.h"

namespace mfs {

namespace {
constexpr double kInv4Pi = 0.07957747154594767;  // 1 / (4 pi)

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
