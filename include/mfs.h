/*
 * mfs.h -- C ABI of libmfs: the GMRES matvec hot path of the recompleted
 * method-of-fundamental-solutions (MFS) elastance and mobility solvers of
 * Broms, Barnett & Tornberg, "A Method of Fundamental Solutions for
 * Large-Scale 3D Elastance and Mobility Problems", on one GB300 (sm_103a).
 *
 * Conventions (all entry points)
 *  - Every user-facing number is FP64 and every index int32_t.  Arrays are
 *    row-major and contiguous.  "Host or device" pointers are accepted as either:
 *    the library asks the CUDA runtime what the pointer is, copies host data
 *    to the device itself and copies results back before returning.
 *  - Bodies are numbered 0..P-1; suspension s owns bodies
 *    [body_offsets[s], body_offsets[s+1]) and never interacts with another
 *    suspension.  Body k has M_k = colloc[shape_id[k]].n collocation points and
 *    N_k = proxy[shape_id[k]].n proxy points; sum_M = sum_k M_k, sum_N = sum_k N_k.
 *  - d = 1 (Laplace) or 3 (Stokes).  Surface vectors (gamma, y, u) are laid out
 *    [nrhs][sum_M][d]; proxy strength vectors (lambda, alpha) [nrhs][sum_N][d];
 *    forces, torques and velocities [nrhs][P][3]; charges and potentials [nrhs][P].
 *  - Kernels: Laplace G = 1/(4 pi r) (Sec. 2.1, Eq. Skk); Stokeslet
 *    (I + r r^T / r^2) / (8 pi mu r) (Sec. 2.2, Eq. stokeslet).  Torques are taken
 *    about the body centre.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Every launch
 *    goes on it; an entry point that returns results to host memory synchronises it.
 *  - No exception or longjmp crosses the ABI.  On error the status is returned
 *    and mfs_last_error() describes it; outputs are then unspecified, except for
 *    MFS_ERR_NOT_CONVERGED, where outputs hold the last iterate and `info` is filled.
 *  - A context is not thread safe: calls on one context must not overlap.
 */
#ifndef MFS_H_
#define MFS_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MFS_ABI_VERSION 4

typedef struct mfs_ctx mfs_ctx; /* opaque; owns all internal device memory */

typedef enum {
    MFS_OK = 0,
    MFS_ERR_INVALID_ARG = 1,     /* bad size, NULL pointer, non-finite input, wrong kind */
    MFS_ERR_CUDA = 2,            /* a CUDA runtime / library call failed */
    MFS_ERR_OOM = 3,             /* device allocation failed */
    MFS_ERR_NOT_CONVERGED = 4,   /* GMRES reached max_iter above the tolerance */
    MFS_ERR_BREAKDOWN = 5,       /* GMRES produced a non-finite residual */
    MFS_ERR_ILL_CONDITIONED = 6, /* a one-body SVD returned a non-finite or zero sigma_1 */
    MFS_ERR_DEVICE_TIMEOUT = 7   /* a device-side bounded wait gave up (kernel returned early) */
} mfs_status;

typedef enum { MFS_LAPLACE = 0, MFS_STOKES = 1 } mfs_kind;

/* A body-frame point set of one shape: n points, pts[n][3] (host memory), centred on the body centre. */
typedef struct {
    int32_t n;
    const double *pts;
} mfs_pointset;

/* The bodies (host memory).  quats [P][4] = (w, x, y, z) unit quaternions or NULL (identity);
 * shape_id [P] or NULL (all shape 0); body_offsets [S+1] or NULL (one suspension of P bodies). */
typedef struct {
    int32_t num_bodies;
    const double *centers; /* [P][3] */
    const double *quats;
    const int32_t *shape_id;
    int32_t num_suspensions;
    const int32_t *body_offsets;
} mfs_bodies;

typedef struct {
    double mu;         /* viscosity (Stokes); default 1 */
    double gmres_tol;  /* relative tolerance on the Arnoldi residual estimate; default 1e-7 */
    int32_t max_iter;  /* GMRES iteration cap per solve; default 200 */
    int32_t restart;   /* Krylov basis size before a restart; default 200 (no restart) */
    double eps_trunc;  /* singular values <= sigma_1 * eps_trunc are dropped (Eq. pseudo); default 0 */
    int32_t precision; /* 0: FP32 pair sums with compensated accumulation and FP32 one-body apply (default);
                          1: FP64 pair sums and FP64 one-body apply (reference GPU path), the adjoint
                             included (transposed sums, transposed apply and centre gradient in FP64);
                          2: FP32 pair sums, FP64 one-body apply;
                          3: compensated double-FP32 pair sums (every pair term carried as hi + lo
                             to about 2^-28 of its size, TwoSum accumulation) and FP64 one-body
                             apply: matvec and pair sums near FP64 accuracy on any input, including
                             rough gamma whose pseudo-inverse strengths are large and cancel, where
                             FP32 pair sums lose about eps_32 * |lambda| / |y|.  The transposed sums and
                             the evaluation at arbitrary points (mfs_evaluate*) stay FP32. */
    int32_t autotune;  /* 1: time pair-kernel variants on this geometry at setup (default 1) */
    int32_t max_rhs;   /* largest nrhs any later call will use (1..4); default 4 */
    int32_t profile;   /* 1: bracket every pair-kernel launch with CUDA events (no host sync) and report
                          their summed device time in mfs_solve_info.ms_pairs; default 0 */
    int32_t tensor_cores; /* precision-0 one-body apply (Eq. pseudo) on the tensor cores (tcgen05 TF32 MMAs,
                             FP32 accumulation over short K runs, double-float sums), operands cut from FP64
                             into TF32 pieces: 1 = three pieces, six products (FP32-level products);
                             2 = two pieces, three products (3xTF32, ~2^-21 products);
                             0 = CUDA-core split-K FP32 GEMM (TwoSum-compensated slices).  Default 1 */
    int32_t pair_variant; /* >= 0: use this entry of the pair-kernel table (mfs_pair_variant_info) for its
                             (d, nrhs) instead of the autotuner's pick; it must be a forward pair-sum
                             variant of the context's d, else mfs_setup fails with MFS_ERR_INVALID_ARG.
                             -1 (default): autotune or the built-in default. */
    int32_t graphs;       /* 1 (default): after the first GMRES iteration, the iteration loop runs as one CUDA
                             graph with a device-side while node (the matvec and Arnoldi kernels read the
                             iteration index from device memory; no host round trip per iteration).  Not
                             with profile = 1, whose per-launch events need the host loop.  0: host loop. */
    int32_t farfield;     /* 0 (default): every pair sum is a direct sum over all body pairs.  1: the forward
                             pair sums (matvec, right-hand side u_0) run as an equivalent-source treecode, the
                             GPU counterpart of the far-field acceleration the paper does with an FMM (Sec. 4):
                             an 8-ary tree of median splits over the body centres; every body and every node
                             gets 196 equivalent point sources on a sphere of radius r_e = (radius of its proxy
                             points) / 0.83, fitted in FP64 by least squares to its proxies' field at 392
                             check points at 2.5 r_e; targets at least 3 r_e from a node's centre see it
                             through those points, nearer ones its children, down to the proxy points of the
                             near bodies (direct, FP32 pair kernel).  Relative accuracy of the sums about
                             1e-7; the pair work drops from O(P^2) to about O(P log P).  Needs precision 0 or
                             2.  Every forward pair sum uses it (the solves, mfs_matvec, mfs_pair_sum); the
                             transposed sums of mfs_matvec_transposed and mfs_mobility_vjp use a second tree
                             with the roles swapped (collocation points as sources, proxy points as targets,
                             built on first use), and so does the VJP's centre gradient (its target side on
                             the first tree, its source side on the second); mfs_evaluate sums over the first
                             tree with interaction lists built for each call's points (each owner body's
                             radius that of its farthest point), and mfs_evaluate_stress likewise (the
                             pressure and traction of the equivalent Stokeslets in the far field; these are
                             derivatives of the field, matched to about 1e-5 relative at separation 3 where
                             velocities are matched to about 1e-7; a larger separation tightens both). */
    double farfield_separation; /* farfield = 1: a target uses a node's equivalent points when it is at least
                                   this many equivalent radii from the node's centre; default 3, allowed
                                   [2.5, 10] (2.5 = the check sphere; smaller is faster and less accurate). */
} mfs_options;

typedef struct {
    int32_t iters;        /* GMRES iterations (max over right-hand sides and suspensions) */
    int32_t converged;    /* 1 when every lane met gmres_tol */
    int32_t matvecs;      /* applications of the preconditioned operator */
    int32_t lanes;        /* independent Krylov solves = nrhs * num_suspensions */
    double rel_residual;  /* max over lanes of the final Arnoldi residual estimate / ||b|| */
    double ms_setup;      /* wall time of mfs_setup (ms) */
    double ms_solve;      /* device time of the solve (ms) */
    double ms_pairs;      /* device time spent in the pair-sum kernel (ms) */
    double pairs;         /* point pairs of the direct sums this solve represents (per right-hand side) */
    int32_t launches;     /* device kernels and memsets this call enqueued */
    int32_t pair_launches;/* pair-sum kernel launches of this call */
    double pairs_evaluated; /* target-source pairs the pair kernel evaluated (per right-hand side): `pairs`
                               for direct sums, fewer with farfield = 1 (near pairs, equivalent points) */
} mfs_solve_info;

/* Fill *opt with the defaults listed above. */
void mfs_default_options(mfs_options *opt);

/* Library ABI version (MFS_ABI_VERSION). */
int32_t mfs_abi_version(void);

/*
 * mfs_setup -- discretise the bodies and build every one-body factor (Sec. 2.3, Sec. 3.3).
 * Per shape, on the device in FP64: S^(00), K_N, K_M (Eq. Kdef), L and L_r (Sec. 3.1 / Eq. Lrsto),
 * S_L = S^(00)(I - L) + L_r and its thin SVD (Eq. pseudo); congruent rotated bodies share it
 * (Remark congruent, Eq. Krot).  Global points are c_k + R(q_k) X0.
 * proxy[s], colloc[s] (s < num_shapes) describe shape s; colloc[s].n must exceed proxy[s].n.
 * On success *out owns the new context (free with mfs_destroy).  All inputs are copied.
 */
mfs_status mfs_setup(mfs_ctx **out, mfs_kind kind, const mfs_bodies *bodies, int32_t num_shapes,
                     const mfs_pointset *proxy, const mfs_pointset *colloc, const mfs_options *opt,
                     void *stream);

/* Move the bodies: new centres [P][3] (host or device).  One-body factors are reused
 * (they depend on shape and orientation only, Remark congruent).  With farfield = 1 the treecode's
 * tree, node geometry and interaction lists are rebuilt for the new positions (host work and a few
 * uploads; captured graphs are dropped and recaptured on the next solve).  Synchronises the device. */
mfs_status mfs_update_centers(mfs_ctx *ctx, const double *centers, void *stream);

/*
 * mfs_matvec -- y = A gamma for the preconditioned square system Eq. 2esysprec:
 *   y^(k) = gamma^(k) + sum_{k' != k, same suspension} S^(kk') (I - L^(k')) S_L^(k')+ gamma^(k'),
 * with S_L^+ applied in two steps (Eq. pseudo) and self pairs never evaluated (Algorithm 1 MATVEC
 * steps 1-3 with step 3 folded into step 2).  gamma, y: [nrhs][sum_M][d], host or device; 1 <= nrhs <= max_rhs.
 */
mfs_status mfs_matvec(mfs_ctx *ctx, const double *gamma, double *y, int32_t nrhs, void *stream);

/*
 * mfs_matvec_transposed -- y = A^T w for the matrix A of Eq. 2esysprec (the operator the adjoint of
 * mfs_mobility_vjp solves with; the paper solves forward problems only):
 *   y^(k') = w^(k') + ((I - L^(k')) S_L^(k')+)^T sum_{k != k', same suspension} S^(kk')^T w^(k),
 * where S^(kk')^T is the Stokeslet pair sum with the collocation points of body k as sources and the
 * proxy points of body k' as targets (the Stokeslet is symmetric and even in r), and the transposed
 * one-body apply is R_M U W^T R_N^T (Eq. pseudo transposed).  Stokes contexts only (else
 * MFS_ERR_INVALID_ARG).  w, y: [nrhs][sum_M][3], host or device, 1 <= nrhs <= max_rhs.  FP32 pair
 * sums and an FP32-level one-body apply (on the tensor cores when tensor_cores != 0 and
 * precision = 0, else the CUDA-core split-K GEMM); with precision = 1 both in FP64.  The first call builds the
 * transposed-apply data (a one-off setup cost, synchronising).
 */
mfs_status mfs_matvec_transposed(mfs_ctx *ctx, const double *w, double *y, int32_t nrhs, void *stream);

/*
 * mfs_precond_apply -- lambda^(k) = S_L^(k)+ gamma^(k) (Eq. pseudo with Remark congruent), followed
 * by the projection (I - L^(k)) when project != 0 (Sec. 3.3, item 2).  gamma [nrhs][sum_M][d],
 * lambda [nrhs][sum_N][d], host or device.
 */
mfs_status mfs_precond_apply(mfs_ctx *ctx, const double *gamma, double *lambda, int32_t project, int32_t nrhs,
                             void *stream);

/*
 * mfs_pair_sum -- the bare MFS evaluation (Algorithm 1 MATVEC step 2):
 *   u^(k) = sum_{k' in the suspension of k, k' != k unless include_self} S^(kk') s^(k'),
 * strengths s [nrhs][sum_N][d] at the proxy points, u [nrhs][sum_M][d] at the collocation points,
 * host or device.  With include_self = 1 this is the right-hand side u_0 of Eq. erhsK / Eq. stou0.
 */
mfs_status mfs_pair_sum(mfs_ctx *ctx, const double *strengths, double *u, int32_t nrhs, int32_t include_self,
                        void *stream);

/*
 * mfs_solve_elastance -- potentials V [nrhs][P] of conductors with net charges Q [nrhs][P]
 * (Prop. 3.1): alpha_0 = q/N 1 (Eq. al0), u_0 by a pair sum over all pairs (Eq. erhsK), GMRES on
 * Eq. 2esysprec from a zero guess, alpha = S_L^+ gamma, V = -mean(alpha) (Eq. vkal).  Laplace only.
 * info may be NULL.
 */
mfs_status mfs_solve_elastance(mfs_ctx *ctx, const double *Q, double *V, int32_t nrhs, mfs_solve_info *info,
                               void *stream);

/*
 * mfs_solve_mobility -- velocities U and angular velocities Omega [nrhs][P][3] of rigid bodies
 * under forces F and torques T [nrhs][P][3] (Prop. 3.2): lambda_0 = K_N (K_N^T K_N)^-1 [f; t]
 * (Eq. lambda01, lambda02), u_0 over all pairs (Eq. stou0), GMRES on Eq. 2esysprec,
 * lambda = S_L^+ gamma, [U; Omega] = -K_N^T lambda (Eq. getU).  Stokes only.  info may be NULL.
 * The context keeps the solution for mfs_mobility_vjp.
 */
mfs_status mfs_solve_mobility(mfs_ctx *ctx, const double *F, const double *T, double *U, double *Omega,
                              int32_t nrhs, mfs_solve_info *info, void *stream);

/*
 * mfs_mobility_vjp -- reverse-mode derivative of the last mfs_solve_mobility (an adjoint the paper
 * does not give; derived from Eq. 2esysprec, Eq. stou0 and Eq. getU).  Given dL/dU and dL/dOmega
 * [nrhs][P][3], writes dL/dcenters [P][3] (summed over right-hand sides) and, when non-NULL,
 * dL/dF and dL/dT [nrhs][P][3].  Host or device pointers.
 */
mfs_status mfs_mobility_vjp(mfs_ctx *ctx, const double *dU, const double *dOmega, int32_t nrhs, double *dcenters,
                            double *dF, double *dT, void *stream);

/*
 * mfs_stokeslet_sum_noalloc -- the Stokeslet pair sum for callers that cannot allocate device
 * memory (code running inside another framework's memory pool, a plug-in host, or a fixed
 * memory budget, where a cudaMalloc is not allowed or not wanted).  The paper has no counterpart:
 * it is a packaging of the same FP32 pair kernel as mfs_pair_sum, without a context.
 *
 *   u_i = sum_j (I + r r^T / r^2) lambda_j / (8 pi mu r),  r = x_i - y_j,  over ALL pairs.
 *
 * targets [num_targets][3], sources [num_sources][3], strengths [num_sources][3] and the output
 * u [num_targets][3] are FP64 DEVICE pointers owned by the caller.  Coordinates are taken relative
 * to the first target in FP64 and then used as FP32 in the pair loop, so separations carry an
 * absolute rounding of about 6e-8 times the extent of the point set, wherever the set sits; a
 * target on top of a source gives a non-finite result.  If a bounded device wait inside the pair
 * kernel gives up (the kernels' timeout path, which a healthy GPU never takes), every entry of u is
 * set to NaN by the same call: the result is never assembled from another call's scratch.
 * Allocates nothing: its scratch (about 21 MB) is a fixed __device__ array inside libmfs that every
 * GPU which loads the library holds until the process exits.  Limits: num_targets and num_sources
 * at most MFS_NOALLOC_MAX_TARGETS / MFS_NOALLOC_MAX_SOURCES; larger sizes, NULL pointers or mu <= 0
 * return MFS_ERR_INVALID_ARG without launching anything.  All launches go on `stream`; the call
 * does not synchronise.  The first call on each device looks up the scratch array's device address
 * (cudaGetSymbolAddress) and the kernel's occupancy under a lock, so make that first call before any
 * stream capture; several devices in one process each get their own copy of the array.  Every call reuses
 * the same array, which keeps the previous call's contents: calls whose GPU work overlaps (other
 * streams or other host threads) race and must be serialised by the caller.
 */
#define MFS_NOALLOC_MAX_TARGETS 65536
#define MFS_NOALLOC_MAX_SOURCES 65536
mfs_status mfs_stokeslet_sum_noalloc(const double *targets, int32_t num_targets, const double *sources,
                                     const double *strengths, int32_t num_sources, double mu, double *u,
                                     void *stream);

/*
 * The Dirichlet problems (Sec. 2): capacitance (Sec. 2.1, Laplace) and resistance (Sec. 2.2, Stokes),
 * one-body preconditioned with the pseudo-inverse of the bare self block S^(kk) = R_M S^(00) R_N^T
 * (Sec. 2.3): GMRES on Eq. 2sysprec with the Dirichlet data as right-hand side (Algorithm 1).  The
 * first call of any of the four functions below computes the extra per-shape SVD of S^(00) (FP64,
 * on the device) and keeps its apply factors; the precision and tensor_cores options apply as for
 * the recompleted problems.  Layouts and pointer rules as everywhere in this header.
 *
 * mfs_dirichlet_apply -- alpha^(k) = S^(kk)+ gamma^(k) = R_N V Sigma^+ U^T R_M^T gamma^(k)
 *   (Eq. pseudo, two steps), gamma [nrhs][sum_M][d] -> alpha [nrhs][sum_N][d].
 * mfs_dirichlet_matvec -- y = gamma + sum_{k' != k} S^(kk') S^(k'k')+ gamma^(k') (Eq. 2sysprec;
 *   Algorithm 1 MATVEC, self pairs never added instead of subtracted).
 * mfs_solve_capacitance -- net charges q [nrhs][P] of conductors held at potentials phi [nrhs][P]:
 *   eta^(k) = phi^(k) 1_M, q^(k) = sum_j alpha_j^(k) (Eq. qkgauss).  Laplace contexts only.
 * mfs_solve_resistance -- forces F and torques T [nrhs][P][3] (about the body centres) on bodies
 *   moving rigidly with velocities U and angular velocities Omega [nrhs][P][3]: b = K_M [v; omega]
 *   (Eq. Kdef, Eq. Kbig), [f; t] = K_N^T lambda (Eq. force_def).  Stokes contexts only.
 * Errors as for the recompleted solves; info may be NULL.
 */
mfs_status mfs_dirichlet_apply(mfs_ctx *ctx, const double *gamma, double *alpha, int32_t nrhs, void *stream);
mfs_status mfs_dirichlet_matvec(mfs_ctx *ctx, const double *gamma, double *y, int32_t nrhs, void *stream);
mfs_status mfs_solve_capacitance(mfs_ctx *ctx, const double *phi, double *q, int32_t nrhs, mfs_solve_info *info,
                                 void *stream);
mfs_status mfs_solve_resistance(mfs_ctx *ctx, const double *U, const double *Omega, double *F, double *T,
                                int32_t nrhs, mfs_solve_info *info, void *stream);

/*
 * mfs_evaluate -- the solution field of the last solve on this context at arbitrary points: the
 * representation u(x) = sum_k sum_j G(x - y_j^(k)) beta_j^(k) (Eq. rep, Eq. repS) with the strengths
 * of that solve, beta = (I - L) S_L^+ gamma + lambda_0 after a mobility solve (Eq. multirep),
 * (I - L) S_L^+ gamma + alpha_0 after an elastance solve (Eq. erepK), S^+ gamma after a resistance
 * or capacitance solve (Eq. reconbal).  For the surface residual (Eq. residual) evaluate on a surface
 * point set finer than the collocation points.
 *   points [npoints][3] world coordinates, host or device; owner [npoints] (nullable; host or device):
 *   a body of the suspension the point belongs to -- only that suspension's sources contribute, and
 *   the point is expressed relative to that body's centre, so the nearest body is the most accurate
 *   choice.  NULL picks the nearest body (allowed with one suspension only).
 *   out [nrhs][npoints][d] (potential or velocity), host or device.  nrhs must equal the last solve's.
 * Points must lie outside the proxy surfaces (in the fluid or conductor exterior, or on the physical
 * surfaces); at a proxy point itself the kernel is singular and the value is not finite.
 * Errors: MFS_ERR_INVALID_ARG without a preceding solve, for a mismatched nrhs, an owner outside
 * [0, P), a non-finite point, or a NULL owner with several suspensions.
 */
mfs_status mfs_evaluate(mfs_ctx *ctx, const double *points, const int32_t *owner, int32_t npoints, double *out,
                        int32_t nrhs, void *stream);

/*
 * mfs_evaluate_stress -- pressure and surface traction of the last mobility or resistance solve at
 * arbitrary points (Stokes contexts): with the strengths beta of mfs_evaluate, the stress tensor
 * sigma = -p I + mu (grad u + grad u^T) of the representation (Eq. traction),
 *   p(x) = sum_j (r . beta_j) / (4 pi r^3),   T(x) = sigma n = -3 / (4 pi) sum_j r (r . n)(r . beta_j) / r^5,
 * r = x - y_j, over the sources of the point's suspension; both are independent of mu.  T is the force
 * per area the fluid exerts across a surface with unit normal n (pointing into the fluid): over a
 * body's surface it integrates to minus the force [f; t] = K_N^T lambda of a resistance solve
 * (Eq. forces).  The traction converges more slowly with N than the velocity (a derivative on the
 * surface, where the MFS error is largest).
 *   points [npoints][3], normals [npoints][3] unit (required when traction != NULL), owner as for
 *   mfs_evaluate; pressure [nrhs][npoints] and traction [nrhs][npoints][3] (either may be NULL, not
 *   both); all host or device.  Errors as for mfs_evaluate; MFS_ERR_INVALID_ARG for a Laplace context.
 */
mfs_status mfs_evaluate_stress(mfs_ctx *ctx, const double *points, const double *normals, const int32_t *owner,
                               int32_t npoints, double *pressure, double *traction, int32_t nrhs, void *stream);

/* The pair-kernel variant the forward pair sums of this context use for `nrhs` right-hand sides
 * (1..max_rhs): the autotuner's pick once a solve or matvec with that nrhs has run (autotune = 1),
 * else the built-in default.  A policy name with its template arguments, e.g.
 * "PackedStokes<1,3,128>" (rhs, target pairs per thread, threads per CTA).  Never NULL; "" for an
 * invalid ctx or nrhs.  Static storage.  Not in the paper: a profiling aid. */
const char *mfs_pair_variant(const mfs_ctx *ctx, int32_t nrhs);

/* Entry `index` of the pair-kernel table: its name (as mfs_pair_variant reports it), dimension d (1 or
 * 3; 4 for the stress entries), right-hand sides and whether it is a kernel other than a pair sum
 * (grad = 1: the adjoint's centre gradient; grad = 2: the pressure and traction of mfs_evaluate_stress,
 * four outputs per right-hand side).  NULL past the end of the table; the out-pointers may be NULL.
 * Static storage. */
const char *mfs_pair_variant_info(int32_t index, int32_t *d, int32_t *nrhs, int32_t *grad);

/*
 * mfs_fp32_fma_rate -- measured FP32 FMA throughput of the current device (TFLOP/s, an FMA counted as
 * two flops), the denominator check for the pair kernel's share of peak.  The paper has no
 * counterpart.  Each mode runs 8 dependency chains per thread of 256-thread CTAs, one launch of about
 * 10-20 ms after a short warm-up launch, timed with CUDA events on `stream` (the call synchronises
 * that stream):
 *   mode 0: scalar fma.rn.f32, a <- a b + c with loop-constant b and c, 32 resident warps per SM;
 *   mode 1: the f32x2 form the Stokeslet kernel issues, otherwise as mode 0;
 *   mode 2: f32x2 whose three operands are distinct registers rewritten every step (no operand is a
 *           loop constant, as in the pair kernel's inner loop), 32 warps per SM;
 *   mode 3: mode 1 at 8 resident warps per SM (two per scheduler, the Stokeslet kernel's occupancy);
 *   mode 4: mode 2 at 8 resident warps per SM.
 * Allocates and frees a few KB (stream-ordered).  *tflops is set to 0 on failure; a mode outside
 * 0..4 or a NULL tflops returns MFS_ERR_INVALID_ARG.
 */
mfs_status mfs_fp32_fma_rate(int32_t mode, double *tflops, void *stream);

/*
 * mfs_selftest_bounded_wait -- exercises the error path of the kernels' bounded device waits (the
 * paper has no counterpart).  A one-warp kernel waits on a shared-memory mbarrier phase with the same
 * bounded wait the pair and tensor-core kernels use; with arrive = 1 the phase is completed first and
 * the call returns MFS_OK, with arrive = 0 nothing completes it, the waiters give up after `limit`
 * polls (1 <= limit <= 2^24), set the device error flag and the call returns MFS_ERR_DEVICE_TIMEOUT
 * with the CUDA context intact.  Synchronises `stream`; allocates 4 bytes (stream-ordered).
 */
mfs_status mfs_selftest_bounded_wait(int32_t arrive, int64_t limit, void *stream);

/* Text of the last error on this context (never NULL; "" when none).  Valid until the next call. */
const char *mfs_last_error(const mfs_ctx *ctx);

/* Text of the last mfs_setup failure that could not return a context. */
const char *mfs_setup_error(void);

/* Release the context and all its device memory.  NULL is ignored. */
void mfs_destroy(mfs_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* MFS_H_ */
