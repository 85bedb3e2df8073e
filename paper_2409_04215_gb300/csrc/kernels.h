// Internal host-side entry points of the libmfs kernels (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "common.cuh"

namespace mfs {

// ---- pair sums (pair_kernel.cu) ----
struct PairVariant {
    int D, nrhs, T, NT, tile_targets;
    int packed;  // 1: f32x2 Stokes policy with duplicated source records
    int grad;    // not a pair sum: 1 the adjoint's centre-gradient kernel, 2 pressure and traction (D = 4 outputs)
    int comp;    // 1: compensated double-FP32 arithmetic (precision = 3), records from pack_sources_comp
    const char *name;  // policy and template arguments, e.g. "PackedStokes<1,3,128>"
};
const PairVariant *pair_variants(int *count);
int pair_occupancy(int variant);  // resident CTAs per SM
int pair_record_floats(int D, int nrhs, int packed);
cudaError_t pair_launch(int variant, const PairGeom &geo, const PairWork &work, int *err, cudaStream_t st);
cudaError_t pair_epilogue(int D, int nrhs, const PairWork &work, const double *base, double beta, double scale,
                          double *out, int ntargets, cudaStream_t st);
cudaError_t pack_sources(int D, int nrhs, int packed, const float4 *src_pos, const int *src_pt_of_rec,
                         const double *strength, int nsrc, int nrec, float *records, cudaStream_t st);
// Records of the compensated kernels from FP64 body-local positions [nsrc][3] and strengths.
cudaError_t pack_sources_comp(int D, int nrhs, const double *src_local64, const int *src_pt_of_rec,
                              const double *strength, int nsrc, int nrec, float *records, cudaStream_t st);

// FP64 reference of the adjoint's pair gradient (precision = 1), per target: sum over the other
// bodies' sources of grad_r (tw^T G(r) strength), raw (no 1/(8 pi mu)); tw [nrhs][ntargets][3], out
// [ntargets][3]; the other arguments as pair_sum_fp64.
cudaError_t grad_pair_fp64(int nrhs, const double *tgt_local, const int *tgt_body, int ntargets, const double *tw,
                           const double *src_local4, int nsrc, const int *susp_src_begin, const int *susp_src_end,
                           const int *body_src_off, const double *centres, const double *strength, double *out,
                           cudaStream_t st);
// FP64 reference pair sum (precision = 1): one thread per target, direct loops; raw sums (no 1/(4pi) factor).
cudaError_t pair_sum_fp64(int D, int nrhs, const double *tgt_local, const int *tgt_body, int ntargets,
                          const double *src_local4, int nsrc, const int *susp_src_begin, const int *susp_src_end,
                          const int *body_src_off, const double *centres, const double *strength, int include_self,
                          double *out_raw, cudaStream_t st);

// ---- preconditioner and setup (precond.cu) ----
struct ShapeDev {
    int M, N, dM, dN, r;  // r = dN (rank kept; truncated sigmas give zero columns)
    float *U;             // [dM][r]  left singular vectors (GEMM 1: t = U^T g)
    float *Wp;            // [r][dN]  ((I - L0) V Sigma^+)^T (projected apply, matvec)
    float *Wr;            // [r][dN]  (V Sigma^+)^T (recovery apply)
    double *U64, *Wp64, *Wr64;  // FP64 copies (precision = 1)
    double *UT64 = nullptr, *WpT64 = nullptr, *WrT64 = nullptr;  // their transposes (the FP64 adjoint)
    double sigma1, sigma_min;   // largest / smallest kept singular value
};

// Build S_L = S0 (I - L) + L_r column-major (dM x dN) in FP64 on the device (Sec. 3.3); with bare,
// the self block S0 itself (the Dirichlet problems, Sec. 2.3).
cudaError_t build_SL(int kind, int M, int N, const double *X0, const double *Y0, double mu, const double *G0inv,
                     int bare, double *SL, cudaStream_t st);
// From the SVD (U col-major dM x r, sigma, VT col-major r x dN) write the FP32 / FP64 apply factors;
// with bare, Wp = Wr = (V Sigma^+)^T (no projector).
cudaError_t build_apply_factors(int kind, int M, int N, const double *Ucm, const double *sigma, const double *VTcm,
                                const double *Y0, const double *G0inv, double eps_trunc, int bare, ShapeDev &sd,
                                cudaStream_t st);

// Gather: A[col][i] = (R_k^T gamma_k)[i] as FP32 for the columns (body, rhs) of one shape.
cudaError_t gather_rotate(int D, const double *gamma, int sum_MD, const int *col_body, const int *col_rhs,
                          const int *body_tgt_off, const double *rot, int ncols, int dM, float *A, double *A64,
                          cudaStream_t st);
// C[m][n] = sum_k A[m][k] B[k][n]  (row-major; FP32 SIMT tiles, or FP64 when A64/B64 given).
cudaError_t gemm_rm(int m, int n, int k, const float *A, const float *B, float *C, cudaStream_t st);
// Split-K FP32 GEMM with TwoSum-compensated slices; chunk results (FP64, P [S][m][n]) summed in FP64
// into C32 (FP32) or C64 (FP64).  S from gemm_splitk_chunks; P must hold S*m*n doubles.
int gemm_splitk_chunks(int m, int n, int k, int sm_count);
cudaError_t splitk_reduce(int S, size_t mn, const double *P, float *C32, double *C64, cudaStream_t st);

// ---- tensor-core one-body apply (tc_gemm.cu): split-K multi-piece TF32 tcgen05 GEMM ----
struct alignas(64) TcMap {
    unsigned char bytes[128];  // an encoded CUtensorMap
};
struct TcOperands {  // kernel parameter: the factor as FP32 (hi, lo) planes (b[0], b[1]), the columns' TF32 pieces (a)
    TcMap b[3];
    TcMap a[3];
};
// 2-D FP32 tensor [rows][ld], ld % 32 == 0, box 32 x box_rows, 128-byte swizzle; false if not encodable.
bool make_tc_map(TcMap &out, const float *ptr, int rows, int ld, int box_rows);
int tc_gemm_bn(int m, int pieces);
int tc_gemm_chunks(int m, int n, int k, int sm_count, int pieces);
int tc_gemm_sz(int k, int S);
// P[z][m][n] = sum_{k in chunk z} A[m][k] B[n][k] as (hi, lo) float pairs, products of `pieces` (2 or 3)
// TF32 pieces per operand: the factor B given as FP32 (hi, lo) planes (maps b[0], b[1]; cut into pieces
// in shared memory), the columns A as pieces (maps a[0..pieces)); S from tc_gemm_chunks, P holds
// tc_gemm_sz(k, S) * m * n pairs.
cudaError_t tc_gemm(int pieces, const TcMap *b, const TcMap *a, int m, int n, int k, int S, float2 *P, int *err,
                    cudaStream_t st);
// FP64 [rows][cols] -> FP32 (hi, lo) planes dst[0 or 1][cols][ld_dst] (transposed, zero K padding).
cudaError_t split_hilo_transpose(const double *src, int rows, int cols, float *dst, int ld_dst, size_t pstride,
                                 cudaStream_t st);
// pieces src[p][rows][ld_src] (first cols valid) -> dst[p][cols][ld_dst] (transposed, zero padding to
// ld_dst >= rows), p at offsets p * sstride and p * dstride.
cudaError_t transpose_pieces(const float *src, int rows, int cols, int ld_src, size_t sstride, float *dst, int ld_dst,
                             size_t dstride, int pieces, cudaStream_t st);
// sum_z P[z] ([rows][cols], (hi, lo) pairs, double-float sums) -> pieces dst[p][rows][ld_dst].
cudaError_t reduce_pieces(int S, int rows, int cols, const float2 *P, float *dst, int ld_dst, size_t pstride,
                          int pieces, cudaStream_t st);
// sum_z P[z] ((hi, lo) pairs, double-float sums) -> C (FP64), mn entries.
cudaError_t reduce_f64(int S, size_t mn, const float2 *P, double *C, cudaStream_t st);
// gather_rotate with the FP64 values written as pieces dst[p][ncols][ld_dst].
cudaError_t gather_rotate_pieces(int D, const double *gamma, int sum_MD, const int *col_body, const int *col_rhs,
                                 const int *body_tgt_off, const double *rot, int ncols, int dM, float *dst, int ld_dst,
                                 size_t pstride, int pieces, cudaStream_t st);
cudaError_t gemm_splitk(int m, int n, int k, int S, const float *A, const float *B, double *P, float *C32,
                        double *C64, cudaStream_t st, bool trans_b = false);  // trans_b: B stored [n][k]
cudaError_t gemm_rm64(int m, int n, int k, const double *A, const double *B, double *C, cudaStream_t st);
// The same product split over K into S chunks (gemm_rm64_chunks), partials P [S][m][n] summed in chunk
// order into C (deterministic); S = 1 is gemm_rm64.
int gemm_rm64_chunks(int m, int n, int k, int sm_count);
cudaError_t gemm_rm64_splitk(int m, int n, int k, int S, const double *A, const double *B, double *P, double *C,
                             cudaStream_t st);
// Scatter: lambda (FP64 [nrhs][sum_N][D]) at the columns' bodies = R_k * Lcol (rotate back).
cudaError_t scatter_rotate(int D, const float *L, const double *L64, const int *col_body, const int *col_rhs,
                           const int *body_src_off, const float *rot, const double *rot64, int ncols, int dN,
                           int sum_N, double *lambda, cudaStream_t st);

// Completion strengths (Eq. lambda01-02 / Eq. al0) and extraction (Eq. getU / Eq. vkal).
cudaError_t completion_stokes(const double *F, const double *T, int nrhs, int P, const double *rot64,
                              const double *G0inv_shapes, const int *shape_id, const double *src_local64,
                              const int *body_src_off, int sum_N, double *lam0, cudaStream_t st);
cudaError_t completion_laplace(const double *Q, int nrhs, int P, const int *body_src_off, int sum_N, double *alpha0,
                               cudaStream_t st);
// sign -1: velocities (Eq. getU); +1: forces and torques (Eq. force_def).
cudaError_t extract_stokes(const double *lam, int nrhs, int P, const double *src_local64, const int *body_src_off,
                           int sum_N, double *U, double *Om, cudaStream_t st, double sign = -1.0);
// sum 0: potentials -mean(alpha) (Eq. vkal); 1: net charges sum(alpha) (Eq. qkgauss).
cudaError_t extract_laplace(const double *alpha, int nrhs, int P, const int *body_src_off, int sum_N, double *V,
                            cudaStream_t st, int sum = 0);
// Dirichlet data: rigid motion K_M U at the collocation points (Sec. 2.2) / phi 1_M (Sec. 2.1).
cudaError_t dirichlet_rhs_stokes(const double *U, const double *Om, int nrhs, int P, const double *tgt_local64,
                                 const int *body_tgt_off, int sum_M, double *b, cudaStream_t st);
cudaError_t dirichlet_rhs_laplace(const double *phi, int nrhs, int P, const int *body_tgt_off, int sum_M, double *b,
                                  cudaStream_t st);

// ---- pressure and traction at evaluation points (stress.cu, Eq. traction), FP64 reference ----
// Points tgt_local (owner-relative) with owners tbody, unit normals nrm [np][3] or null (no traction),
// FP64 body-local sources and strengths, per-body suspension body range [sb0, sb1); outputs p
// [nrhs][np], traction [nrhs][np][3] (either may be null).  The FP32 path is the pair kernel's stress
// entry (StressStokes).
cudaError_t stress_f64(int nrhs, const double *tgt_local, const int *tbody, const double *nrm, int np,
                       const double *src_local, const int *src_off, int sum_N, const double *lam, const int *sb0,
                       const int *sb1, const double *centres, double *p_out, double *t_out, cudaStream_t st);

// ---- far field of the pair sums: equivalent-source treecode (farfield.cu) ----
constexpr int FF_NE = 196;            // equivalent points per node (a Fibonacci sphere of radius r_e)
constexpr int FF_NC = 392;            // check points per node (radius FF_CHECK * r_e), least-squares fit
constexpr double FF_CHECK = 2.5;      // check radius / equivalent radius
constexpr double FF_SRC_RATIO = 0.83; // a node's source radius / its equivalent radius
// (a target at least mfs_options.farfield_separation equivalent radii from a node's centre sees the node
// through its equivalent points)
struct FFNode {
    double c[3] = {0, 0, 0};  // centre
    double rs = 0.0;          // radius of the node's proxy sources about c
    double re = 0.0;          // equivalent radius rs / FF_SRC_RATIO
    int body = -1;            // the body of a leaf, -1 for a group
    int first = 0, count = 0; // descendant bodies: order[first .. first + count)
    int nchild = 0;
    int child[8] = {0, 0, 0, 0, 0, 0, 0, 0};
};
struct FFTree {
    std::vector<FFNode> nodes;
    std::vector<int> order;  // bodies in tree (depth-first leaf) order
    std::vector<int> pos;    // pos[body] = its index in `order`
    std::vector<int> roots;  // one per suspension
};
// The 8-ary median-split tree of each suspension's bodies (centres [P][3], source radii rsrc [P]).
void ff_build_tree(int P, const double *centres, const double *rsrc, int S, const int *body_off, FFTree &t);
// Interaction list of the target bodies `tbodies` (original ids; target radii rtgt): segment ids, a
// body's proxy points as its tree position q < P, a node's equivalent points as P + node.  With
// self_skip, a single target body's own proxy points are left out.
void ff_interaction_list(const FFTree &t, int root, const std::vector<int> &tbodies, const double *centres,
                         const double *rtgt, double kappa, int self_skip, std::vector<int> &segs);
// mu[h][node][e][d] *= re[node] (the fit was made on the unit sphere; the kernels are homogeneous of
// degree -1).
cudaError_t ff_scale(double *mu, const double *re, int nodes, int per_node, int nrhs, cudaStream_t st);

// ---- GMRES (gmres.cu): L independent lanes, lane l owns vector entries [seg_off[l], seg_off[l+1]) ----
struct GmresDev {
    int L, m;                  // lanes, Krylov basis capacity (m <= 1023)
    long long n;               // vector length (all lanes)
    const long long *seg_off;  // [L+1] (device)
    double *V;                 // [(m+1)][n] basis
    double *H;                 // [L][m+1][m] Hessenberg, rotated to upper triangular
    double *cs, *sn, *g;       // [L][m], [L][m], [L][m+1]
    double *beta;              // [L] ||b||
    double *hbuf, *htmp;       // [L][m+1] current column, current CGS pass
    double *hn;                // [L] norm of the new Krylov vector
    double *part;              // [L][part_blocks][m+1] block partials
    int *active;               // [L] 1 while the lane iterates
    int *iters;                // [L] iterations done
    int *status;               // [L] 0 ok, 2 breakdown (non-finite)
    double *resid;             // [L] |g_k| / ||b||
    int *done;                 // [1] 1 when no lane is active
    int *jcur;                 // [1] the current Arnoldi column j (device-side, so a graph can loop)
    double tol;
    int part_blocks;           // blocks per lane in the reductions
};
// Start: v_0 = b / ||b|| per lane, lanes with b = 0 inactive, j = 0, done = (no lane active).
cudaError_t gmres_init(GmresDev &gd, const double *b, cudaStream_t st);
// Orthogonalise w = A v_j against v_0..v_j (CGS2), append v_{j+1}, Givens-update every active lane;
// j is read from gd.jcur.
cudaError_t gmres_arnoldi(GmresDev &gd, double *w, cudaStream_t st);
// vin = v_j (j from gd.jcur): the input of the next matvec at a fixed address.
cudaError_t gmres_load_vj(GmresDev &gd, double *vin, cudaStream_t st);
// j += 1 unless done or the basis is full; with a graph conditional handle (cond_valid), sets it to
// whether another iteration follows.
cudaError_t gmres_advance(GmresDev &gd, cudaGraphConditionalHandle cond, int cond_valid, cudaStream_t st);
// x = V y with H y = g per lane (y_small: [L][m+1] scratch).
cudaError_t gmres_solution(GmresDev &gd, double *x, double *y_small, cudaStream_t st);

}  // namespace mfs
