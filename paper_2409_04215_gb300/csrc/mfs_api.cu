// libmfs host runtime and C ABI (see include/mfs.h).
#include <cusolverDn.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/mfs.h"
#include "common.cuh"
#include "kernels.h"

using namespace mfs;

namespace {

thread_local std::string g_setup_error;

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct PairPlan {
    int variant = -1;
    int include_self = 0;
    int tile_targets = 0;
    int G = 0;
    int ntiles = 0;
    long long total_units = 0;
    PairTile *tiles = nullptr;
    double *partial = nullptr;
    double *direct = nullptr;
    size_t partial_bytes = 0, direct_bytes = 0;
    int max_share = 1;  // the most CTAs that share one tile (sizes the epilogue)
};

// The one-body apply factors of one formulation for one shape, FP32 / FP64 and as tensor-core pieces.
struct FactorSet {
    bool built = false;
    ShapeDev dev{};
    bool tc_ready = false;
    float *Utp = nullptr, *Wptp = nullptr, *Wrtp = nullptr;  // FP32 (hi, lo) planes [2][r or dN][ld]
    size_t ut_stride = 0, wt_stride = 0;
    TcMap mU[3], mWp[3], mWr[3];
    // the transposed apply (adjoint), built on first use: (hi, lo) planes of U [dM][ld2] and of W^T [r][ld2]
    bool tcT_ready = false;
    float *Un = nullptr, *WpT = nullptr, *WrT = nullptr;
    size_t un_stride = 0;
    TcMap mUn[3], mWpT[3], mWrT[3];
};

struct ShapeHost {
    int M = 0, N = 0;
    std::vector<double> X0, Y0;  // body frame
    double G0inv[36];
    std::vector<int> bodies;     // bodies of this shape
    int *col_body = nullptr, *col_rhs = nullptr;  // device, [max_rhs * nbodies]
    float *A = nullptr, *Tm = nullptr, *Lm = nullptr;  // GEMM buffers
    double *Pk = nullptr;                              // split-K chunk results
    size_t Pk_count = 0;
    double *O64 = nullptr, *PkT = nullptr;             // adjoint: transposed-apply output and chunks
    float2 *PtcT = nullptr;                            // adjoint: tensor-core chunk results
    // tensor-core apply scratch: K-major TF32 pieces of the columns, chunk results
    int pieces = 0;        // TF32 pieces per operand (3: 6xTF32 products, 2: 3xTF32)
    int ld1 = 0, ld2 = 0;  // K extents padded to 32: roundup(dM, 32), roundup(r, 32)
    float *Ap = nullptr, *Tp = nullptr;  // [piece][columns][ld1 or ld2]
    size_t ap_stride = 0, tp_stride = 0;
    float2 *Ptc = nullptr;  // chunk results as (hi, lo) pairs
    std::map<int, std::array<TcMap, 6>> amaps;  // per column count: A pieces, T pieces
    double *A64 = nullptr, *T64 = nullptr, *L64 = nullptr;
    // one-body factors per formulation: [0] recompleted S_L (Sec. 3.3), [1] bare self block S^(00)
    // of the Dirichlet problems (Sec. 2.3), built on first use
    FactorSet fs[2];
};

}  // namespace

struct mfs_ctx {
    int kind = 0, D = 1;
    int fset = 0;  // factor set of the one-body apply: 0 recompleted (Sec. 3.3), 1 bare self block (Sec. 2.3)
    // GMRES iteration loops captured as CUDA graphs, by nrhs * 4 + fset * 2 + transposed
    struct SolveGraph {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        int launches = 0, pair_launches = 0;  // per iteration
    };
    std::map<int, SolveGraph> graphs;
    double *vin_d = nullptr;  // matvec input of a graph iteration (v_j copied to a fixed address)
    cudaStream_t cap_stream = nullptr;  // capture only (the legacy stream cannot capture); launches use the caller's
    void drop_graphs() {
        for (auto &kv : graphs) {
            if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
            if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
        }
        graphs.clear();
    }
    mfs_options opt{};
    int P = 0, S = 0, nshapes = 0;
    std::vector<double> centres, quats;
    std::vector<int> shape_id, body_off;
    std::vector<int> tgt_off, src_off, rec_off;  // [P+1] point / padded-record offsets
    std::vector<long long> blk_off;
    std::vector<int> tgt_body;                     // [sum_M]
    int sumM = 0, sumN = 0, nrec = 0;
    std::vector<double> rot;                       // [P][9]
    std::vector<ShapeHost> shapes;

    // device geometry
    double *centres_d = nullptr, *rot64_d = nullptr, *G0inv_d = nullptr;
    float *rot_d = nullptr;
    int *shape_id_d = nullptr;
    float4 *tgt_pos_d = nullptr, *src_pos_d = nullptr;
    float4 *tgt_hi_d = nullptr, *tgt_lo_d = nullptr;  // precision 3: grid-split body-local targets
    double *tgt_local64_d = nullptr, *src_local64_d = nullptr, *src_local4_d = nullptr;
    int *tgt_body_d = nullptr, *rec_pt_d = nullptr, *rec_off_d = nullptr, *tgt_off_d = nullptr,
        *src_off_d = nullptr, *susp_src_begin_d = nullptr, *susp_src_end_d = nullptr;
    long long *blk_off_d = nullptr;
    int *err_d = nullptr;

    // work buffers
    float *rec_d = nullptr;      // packed source records (max_rhs)
    int rec_floats = 0;          // floats per record allocated in rec_d (and recT_floats in recT_d)
    int recT_floats = 0;
    double *lam_d = nullptr;     // [max_rhs][sumN][D]
    double *raw_d = nullptr;     // FP64 reference pair sums [max_rhs][sumM][D]
    std::map<int, PairPlan> plans;  // key: variant * 4 + include_self * 2 + transposed
    int best_variant[2][5] = {{-1, -1, -1, -1, -1}, {-1, -1, -1, -1, -1}};  // [D==3][nrhs]

    // GMRES
    GmresDev gd{};
    size_t gd_n = 0;
    int gd_L = 0, gd_m = 0;
    long long *seg_off_d = nullptr;
    double *w_d = nullptr, *b_d = nullptr, *x_d = nullptr, *ysmall_d = nullptr;
    int *done_h = nullptr;

    // solution kept for the adjoint
    // the last solve, for mfs_mobility_vjp and mfs_evaluate: which problem, its GMRES solution gamma
    // [max_rhs][sum_M][D] and its inputs (F then T [nrhs][P][3], or Q [nrhs][P])
    int last_solve = 0;  // 0 none, 1 mobility, 2 elastance, 3 resistance, 4 capacitance
    double *keep_gamma = nullptr;
    double *keep_lam0 = nullptr;  // [max_rhs][P][6]
    int last_nrhs = 0;

    // adjoint: the transposed direction (proxy targets, collocation sources)
    bool trans_ready = false;
    std::vector<int> src_body, recT_off;
    std::vector<long long> blkT_off;
    int nrecT = 0;
    float4 *tgtT_pos_d = nullptr;
    // the FP64 transposed sums (precision = 1): proxy -> body, collocation points [sum_M][4] (body-local
    // x, y, z and the body id), each body's suspension as a collocation range
    int *src_body_d = nullptr, *colT_begin_d = nullptr, *colT_end_d = nullptr;
    double *colloc4_d = nullptr;
    float *recT_d = nullptr;
    int *recT_off_d = nullptr, *rec_ptT_d = nullptr;
    long long *blkT_off_d = nullptr;
    double *tmpM_d = nullptr;     // [max_rhs][sum_M][3]
    double *gradT_d = nullptr;    // [sum_M][3] per-target gradient sums
    double *src_grad_d = nullptr; // [P][3]
    double *six_d = nullptr;      // [max_rhs][P][6] scratch for -K_N^T z
    float *w32_d = nullptr;       // [max_rhs][sum_M][3] FP32 adjoint strengths
    double *eye6_d = nullptr;     // [nshapes][36] identity (K_N [u; w] expansion)

    // far field of the pair sums (opt.farfield = 1): equivalent-source treecode (farfield.cu)
    struct FarField {
        bool ready = false;
        // the roles of the point sets: forward sums (proxy sources, collocation targets) or the
        // adjoint's transposed sums (collocation sources, proxy targets)
        bool src_colloc = false;
        const float4 *src_pos = nullptr;             // [nsrc] body-local source positions
        const int *rec_pt = nullptr;                 // [nrec] source record -> point (-1: padding)
        const float4 *tgt_pos = nullptr;             // [ntgt] body-local target positions
        const std::vector<int> *rec_off = nullptr;   // [P + 1] padded record offsets of the sources
        const std::vector<int> *tgt_off = nullptr;   // [P + 1] target offsets
        int nsrc = 0, nrec = 0, ntgt = 0;
        FFTree tree;
        int nodes = 0;
        std::vector<double> rsrc, rtgt;              // per body: radius of its proxy / collocation points
        double *PinvT = nullptr;                     // [D FF_NC][D FF_NE]: transposed pseudo-inverse of the
                                                     // check <- equivalent map on the unit sphere (FP64)
        double *centres = nullptr;                   // [P + nodes][3]: bodies in tree order, then the nodes
        double *re = nullptr;                        // [nodes] equivalent radii
        float4 *eq_pos = nullptr;                    // [nodes FF_NE] equivalent points about their node's centre
        int *eq_pt = nullptr;                        // identity record -> point map (packing)
        float4 *chk_pos = nullptr;                   // [nodes FF_NC] check points, w = P + node
        float4 *tgt = nullptr;                       // [sum_M] targets in tree order, w = tree position
        int *tperm = nullptr;                        // [sum_M] tree-order target -> caller's target index
        int *seg_rec0 = nullptr, *seg_rec1 = nullptr;  // [P + nodes] record range of every segment
        std::vector<int> seg_rec0_h, seg_rec1_h;
        float *rec = nullptr;                        // proxy records, then equivalent records
        int rec_floats = 0;
        double *ucheck = nullptr;                    // [max_rhs][nodes FF_NC][D]
        double *mu = nullptr;                        // [max_rhs][nodes FF_NE][D]
        double *fit_chunks = nullptr;                // split-K partials of the fit product
        float *wt = nullptr;                         // [max_rhs][ntgt][3] target weights in tree order (gradient)
        struct Plan {
            PairPlan up, ev;
            int *lst_seg_up = nullptr, *lst_seg_ev = nullptr;
            long long *lst_cum_up = nullptr, *lst_cum_ev = nullptr;
            double pairs_up = 0.0, pairs_ev = 0.0;   // target-source pairs one application evaluates
        };
        std::map<int, Plan> plans;                   // key: variant * 2 + include_self
    } ff, ffT;                                       // forward sums; transposed sums (adjoint)

    int sm_count = 0;
    std::string last_error;
    std::vector<void *> allocs;
    double ms_setup = 0.0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, evp0 = nullptr, evp1 = nullptr;
    double pair_ms_acc = 0.0;
    int launches = 0;        // kernels + memsets enqueued by the current call
    int pair_launches = 0;   // pair-kernel launches of the current call
    std::vector<cudaEvent_t> pev;  // profile: event pairs around pair-kernel launches

    template <typename T>
    cudaError_t alloc(T **p, size_t count) {
        *p = nullptr;
        if (count == 0) count = 1;
        cudaError_t e = cudaMalloc((void **)p, sizeof(T) * count);
        if (e == cudaSuccess) allocs.push_back((void *)*p);
        return e;
    }
    void release(void *p) {
        if (!p) return;
        auto it = std::find(allocs.begin(), allocs.end(), p);
        if (it != allocs.end()) allocs.erase(it);
        cudaFree(p);
    }
    ~mfs_ctx() {
        drop_graphs();
        if (cap_stream) cudaStreamDestroy(cap_stream);
        for (void *p : allocs) cudaFree(p);
        if (done_h) cudaFreeHost(done_h);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        if (evp0) cudaEventDestroy(evp0);
        if (evp1) cudaEventDestroy(evp1);
        for (cudaEvent_t e : pev) cudaEventDestroy(e);
    }
};

static mfs_status ff_setup(mfs_ctx *ctx, mfs_ctx::FarField &F, cudaStream_t st);  // far-field structures

namespace {

#define CK(call)                                                                             \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            ctx->last_error = std::string(#call) + ": " + cudaGetErrorString(e_);            \
            return e_ == cudaErrorMemoryAllocation ? MFS_ERR_OOM : MFS_ERR_CUDA;              \
        }                                                                                    \
    } while (0)

#define CKS(call)                                  \
    do {                                           \
        mfs_status s_ = (call);                    \
        if (s_ != MFS_OK) return s_;               \
    } while (0)

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// A device view of a user pointer: either the pointer itself or a staged copy.
struct Staged {
    mfs_ctx *ctx = nullptr;
    double *d = nullptr;
    const void *user = nullptr;
    size_t count = 0;
    bool owned = false;
    ~Staged() {
        if (owned && d) cudaFree(d);
    }
};

mfs_status stage_in(mfs_ctx *ctx, Staged &s, const double *user, size_t count, cudaStream_t st) {
    s.ctx = ctx;
    s.user = user;
    s.count = count;
    if (is_device_ptr(user)) {
        s.d = const_cast<double *>(user);
        return MFS_OK;
    }
    CK(cudaMalloc(&s.d, sizeof(double) * std::max<size_t>(count, 1)));
    s.owned = true;
    CK(cudaMemcpyAsync(s.d, user, sizeof(double) * count, cudaMemcpyHostToDevice, st));
    return MFS_OK;
}

mfs_status stage_out_alloc(mfs_ctx *ctx, Staged &s, double *user, size_t count) {
    s.ctx = ctx;
    s.user = user;
    s.count = count;
    if (is_device_ptr(user)) {
        s.d = user;
        return MFS_OK;
    }
    CK(cudaMalloc(&s.d, sizeof(double) * std::max<size_t>(count, 1)));
    s.owned = true;
    return MFS_OK;
}

mfs_status stage_out_finish(mfs_ctx *ctx, Staged &s, cudaStream_t st) {
    if (s.owned) {
        CK(cudaMemcpyAsync(const_cast<void *>(s.user), s.d, sizeof(double) * s.count, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    return MFS_OK;
}

mfs_status check_device_error(mfs_ctx *ctx, cudaStream_t st) {
    int h = 0;
    CK(cudaMemcpyAsync(&h, ctx->err_d, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h) {
        ctx->last_error = (h & MFS_DEVERR_TIMEOUT) ? "a device-side bounded wait gave up" : "device argument error";
        cudaMemsetAsync(ctx->err_d, 0, sizeof(int), st);
        return MFS_ERR_DEVICE_TIMEOUT;
    }
    return MFS_OK;
}

void quat_to_rot(const double *q, double *R) {
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z); R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z); R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y); R[7] = 2 * (y * z + w * x); R[8] = 1 - 2 * (x * x + y * y);
}

// 6x6 inverse by Gauss-Jordan with partial pivoting; returns false when singular.
bool invert6(const double *A, double *Ainv) {
    double a[6][12];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 12; ++j) a[i][j] = j < 6 ? A[i * 6 + j] : (j - 6 == i ? 1.0 : 0.0);
    for (int c = 0; c < 6; ++c) {
        int p = c;
        for (int r = c + 1; r < 6; ++r)
            if (std::fabs(a[r][c]) > std::fabs(a[p][c])) p = r;
        if (a[p][c] == 0.0) return false;
        for (int j = 0; j < 12; ++j) std::swap(a[c][j], a[p][j]);
        const double inv = 1.0 / a[c][c];
        for (int j = 0; j < 12; ++j) a[c][j] *= inv;
        for (int r = 0; r < 6; ++r)
            if (r != c) {
                const double f = a[r][c];
                for (int j = 0; j < 12; ++j) a[r][j] -= f * a[c][j];
            }
    }
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) Ainv[i * 6 + j] = a[i][j + 6];
    return true;
}

// G0 = K_N0^T K_N0 for body-frame proxy points (Eq. lambda02 with Eq. Kdef).
void gram6(const std::vector<double> &Y0, double *G) {
    std::memset(G, 0, sizeof(double) * 36);
    const int n = (int)Y0.size() / 3;
    for (int q = 0; q < n; ++q) {
        const double *d = &Y0[3 * q];
        const double cm[3][3] = {{0.0, d[2], -d[1]}, {-d[2], 0.0, d[0]}, {d[1], -d[0], 0.0}};
        for (int b = 0; b < 3; ++b) {
            double row[6];
            for (int m = 0; m < 3; ++m) row[m] = (b == m) ? 1.0 : 0.0;
            for (int m = 0; m < 3; ++m) row[3 + m] = cm[b][m];
            for (int i = 0; i < 6; ++i)
                for (int j = 0; j < 6; ++j) G[i * 6 + j] += row[i] * row[j];
        }
    }
}

int default_variant(int D, int nrhs, int comp = 0) {
    int count = 0;
    const PairVariant *v = pair_variants(&count);
    // preferred variant per kind and nrhs when not autotuned: packed f32x2 for Stokes, scalar for Laplace
    const int wantT = (D == 3) ? (nrhs == 1 ? 4 : 2) : 4;
    const int wantNT = 128, wantPacked = (D == 3 && nrhs != 3) ? 1 : 0;
    if (!comp)
        for (int i = 0; i < count; ++i)
            if (!v[i].grad && !v[i].comp && v[i].D == D && v[i].nrhs == nrhs && v[i].T == wantT &&
                v[i].NT == wantNT && v[i].packed == wantPacked)
                return i;
    for (int i = 0; i < count; ++i)
        if (!v[i].grad && v[i].comp == comp && v[i].D == D && v[i].nrhs == nrhs) return i;
    return -1;
}

// The forward pair-sum variant of this context for nrhs: compensated kernels with precision = 3.
int forward_variant(const mfs_ctx *ctx, int nrhs) {
    const int tuned = ctx->best_variant[ctx->D == 3][nrhs];
    return tuned >= 0 ? tuned : default_variant(ctx->D, nrhs, ctx->opt.precision == 3);
}

// An FP32 (not compensated) variant for the sums that have no compensated form (transposed sums,
// evaluation at arbitrary points).
int fp32_variant(const mfs_ctx *ctx, int D, int nrhs) {
    if (ctx->opt.precision == 3) return default_variant(D, nrhs, 0);
    const int tuned = ctx->best_variant[D == 3][nrhs];
    return tuned >= 0 ? tuned : default_variant(D, nrhs, 0);
}

// Tiles and CTA shares for one pair-kernel variant.  transposed = 0: collocation targets, proxy
// sources (the matvec and u_0); transposed = 1: proxy targets, collocation sources (the adjoint's
// S^T sums).
// Work list of a pair sum over any target set grouped by body: targets of body k are
// [toff[k], toff[k+1]) and tbody[t] is the body of target t; source blocks per body from boff.
mfs_status build_plan_for(mfs_ctx *ctx, int variant, int include_self, const std::vector<int> &toff,
                          const std::vector<int> &tbody, const std::vector<long long> &boff, int ntargets,
                          PairPlan &plan) {
    int count = 0;
    const PairVariant *vv = pair_variants(&count);
    const PairVariant &v = vv[variant];
    const int TT = v.tile_targets;
    const int C = v.grad == 1 ? 3 : v.D * v.nrhs;  // the gradient kernel: one 3-vector per target
    std::vector<PairTile> tiles;
    long long units = 0;
    for (int s = 0; s < ctx->S; ++s) {
        const int B0 = ctx->body_off[s], B1 = ctx->body_off[s + 1];
        const int t_end = toff[B1];
        int t = toff[B0];
        while (t < t_end) {
            int t1 = std::min(t + TT, t_end);
            const int kb0 = tbody[t];
            int kb1 = tbody[t1 - 1];
            if (kb1 - kb0 + 1 > MFS_MAX_TILE_BODIES) {
                kb1 = kb0 + MFS_MAX_TILE_BODIES - 1;
                t1 = toff[kb1 + 1];
            }
            PairTile tl;
            tl.t0 = t;
            tl.t1 = t1;
            tl.kb0 = kb0;
            tl.nb = kb1 - kb0 + 1;
            tl.skip = (!include_self && tl.nb == 1) ? kb0 : -1;
            tl.B0 = B0;
            tl.B1 = B1;
            tl.L0 = tl.L1 = -1;
            long long u = 0;
            for (int b = B0; b < B1; ++b)
                if (b != tl.skip) u += boff[b + 1] - boff[b];
            tl.u0 = units;
            tl.u1 = units + u;
            units += u;
            tiles.push_back(tl);
            t = t1;
        }
    }
    const int occ = pair_occupancy(variant);
    if (occ <= 0) {
        ctx->last_error = "pair kernel variant cannot be resident on this GPU";
        return MFS_ERR_CUDA;
    }
    long long G = (long long)occ * ctx->sm_count;
    if (G > units) G = std::max<long long>(units, 1);
    const long long W = units;
    int max_share = 1;
    for (auto &tl : tiles) {
        if (tl.u1 == tl.u0) {
            tl.gA = tl.gB = -1;
            continue;
        }
        auto owner = [&](long long u) { return (int)(((u + 1) * G - 1) / W); };
        tl.gA = owner(tl.u0);
        tl.gB = owner(tl.u1 - 1);
        max_share = std::max(max_share, tl.gB - tl.gA + 1);
    }
    plan.variant = variant;
    plan.include_self = include_self;
    plan.tile_targets = TT;
    plan.G = (int)G;
    plan.ntiles = (int)tiles.size();
    plan.max_share = max_share;
    plan.total_units = units;
    CK(ctx->alloc(&plan.tiles, tiles.size()));
    CK(cudaMemcpy(plan.tiles, tiles.data(), sizeof(PairTile) * tiles.size(), cudaMemcpyHostToDevice));
    plan.partial_bytes = sizeof(double) * (size_t)G * 2 * TT * C;
    plan.direct_bytes = sizeof(double) * (size_t)ntargets * C;
    CK(ctx->alloc(&plan.partial, (size_t)G * 2 * TT * C));
    CK(ctx->alloc(&plan.direct, (size_t)std::max(ntargets, 1) * C));
    return MFS_OK;
}

mfs_status build_plan(mfs_ctx *ctx, int variant, int include_self, int transposed, PairPlan &plan) {
    return build_plan_for(ctx, variant, include_self, transposed ? ctx->src_off : ctx->tgt_off,
                          transposed ? ctx->src_body : ctx->tgt_body, transposed ? ctx->blkT_off : ctx->blk_off,
                          transposed ? ctx->sumN : ctx->sumM, plan);
}

void release_plan(mfs_ctx *ctx, PairPlan &plan) {
    ctx->release(plan.tiles);
    ctx->release(plan.partial);
    ctx->release(plan.direct);
    plan = PairPlan{};
}

mfs_status get_plan(mfs_ctx *ctx, int variant, int include_self, PairPlan **out, int transposed = 0) {
    const int key = variant * 4 + include_self * 2 + transposed;
    auto it = ctx->plans.find(key);
    if (it == ctx->plans.end()) {
        PairPlan p;
        CKS(build_plan(ctx, variant, include_self, transposed, p));
        it = ctx->plans.emplace(key, p).first;
    }
    *out = &it->second;
    return MFS_OK;
}

PairWork work_of(const PairPlan &p) {
    PairWork w;
    w.tiles = p.tiles;
    w.ntiles = p.ntiles;
    w.total_units = p.total_units;
    w.G = p.G;
    w.partial = p.partial;
    w.direct = p.direct;
    w.tile_targets = p.tile_targets;
    w.include_self = p.include_self;
    w.max_share = p.max_share;
    return w;
}

PairGeom geom_of(mfs_ctx *ctx) {
    PairGeom g;
    g.tgt = ctx->tgt_pos_d;
    g.src = ctx->rec_d;
    g.src_off = ctx->rec_off_d;
    g.blk_off = ctx->blk_off_d;
    g.centres = ctx->centres_d;
    g.ntargets = ctx->sumM;
    g.tgt_hi = ctx->tgt_hi_d;
    g.tgt_lo = ctx->tgt_lo_d;
    return g;
}

// Source records for `variant` from FP64 strengths [nrhs][sum_N][D].
cudaError_t pack_for(mfs_ctx *ctx, int variant, const double *strength, int nrhs, cudaStream_t st) {
    int vc = 0;
    const PairVariant *vv = pair_variants(&vc);
    // the record buffer holds every layout this context's entries use; anything else is refused
    if (pair_record_floats(ctx->D, nrhs, vv[variant].comp ? 2 : vv[variant].packed) > ctx->rec_floats)
        return cudaErrorInvalidValue;
    if (vv[variant].comp)
        return pack_sources_comp(ctx->D, nrhs, ctx->src_local64_d, ctx->rec_pt_d, strength, ctx->sumN, ctx->nrec,
                                 ctx->rec_d, st);
    return pack_sources(ctx->D, nrhs, vv[variant].packed, ctx->src_pos_d, ctx->rec_pt_d, strength, ctx->sumN,
                        ctx->nrec, ctx->rec_d, st);
}

double kernel_scale(mfs_ctx *ctx) {
    return ctx->kind == MFS_STOKES ? 1.0 / (8.0 * MFS_PI * ctx->opt.mu) : 1.0 / (4.0 * MFS_PI);
}

// out = beta * base + sign * (pair sum of strengths)  (strengths FP64 [nrhs][sumN][D] on device)
__global__ void combine_raw_kernel(const double *raw, const double *base, double beta, double scale, double *out,
                                   size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (base ? beta * base[i] : 0.0) + scale * raw[i];
}

mfs_status ff_pair_apply(mfs_ctx *ctx, mfs_ctx::FarField &F, int variant, const double *strength, double *out,
                         const double *base, double beta, double scale, int nrhs, int include_self, cudaStream_t st);

mfs_status pair_apply(mfs_ctx *ctx, const double *strength, double *out, const double *base, double beta,
                      double sign, int nrhs, int include_self, cudaStream_t st) {
    const double scale = sign * kernel_scale(ctx);
    if (ctx->opt.precision == 1) {
        CK(pair_sum_fp64(ctx->D, nrhs, ctx->tgt_local64_d, ctx->tgt_body_d, ctx->sumM, ctx->src_local4_d, ctx->sumN,
                         ctx->susp_src_begin_d, ctx->susp_src_end_d, ctx->src_off_d, ctx->centres_d, strength,
                         include_self, ctx->raw_d, st));
        const size_t n = (size_t)nrhs * ctx->sumM * ctx->D;
        combine_raw_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ctx->raw_d, base, beta, scale, out, n);
        CK(cudaGetLastError());
        ctx->launches += 2;
        ctx->pair_launches += 1;
        return MFS_OK;
    }
    const int variant = forward_variant(ctx, nrhs);
    if (variant < 0) {
        ctx->last_error = "no pair-kernel variant for this nrhs";
        return MFS_ERR_INVALID_ARG;
    }
    if (ctx->ff.ready)
        return ff_pair_apply(ctx, ctx->ff, variant, strength, out, base, beta, scale, nrhs, include_self, st);
    PairPlan *plan = nullptr;
    CKS(get_plan(ctx, variant, include_self, &plan));
    CK(pack_for(ctx, variant, strength, nrhs, st));
    const PairWork w = work_of(*plan);
    ctx->launches += 2;
    if (w.total_units > 0) {
        const size_t slot = 2 * (size_t)ctx->pair_launches;
        if (ctx->opt.profile) {
            while (ctx->pev.size() < slot + 2) {
                cudaEvent_t e;
                CK(cudaEventCreate(&e));
                ctx->pev.push_back(e);
            }
            CK(cudaEventRecord(ctx->pev[slot], st));
        }
        CK(pair_launch(variant, geom_of(ctx), w, ctx->err_d, st));
        if (ctx->opt.profile) CK(cudaEventRecord(ctx->pev[slot + 1], st));
        ctx->launches += 1;
        ctx->pair_launches += 1;
    }
    CK(pair_epilogue(ctx->D, nrhs, w, base, beta, scale, out, ctx->sumM, st));
    return MFS_OK;
}

// Tiles over targets grouped into consecutive groups (group g: targets [toff[g], toff[g+1]), its id in
// the geometry's centre table gid0 + g), never crossing a group boundary listed in `cuts`, each tile
// with the interaction list that list_of(g0, g1) gives for its groups g0..g1; seg_blocks[s] blocks of
// MFS_BS records per segment s.  Uploads the tiles and the lists (PairGeom::lst_seg, lst_cum).
template <class ListFn>
mfs_status build_plan_lists(mfs_ctx *ctx, int variant, int include_self, const std::vector<int> &toff, int gid0,
                            const std::vector<int> &cuts, const std::vector<long long> &seg_blocks,
                            const std::vector<int> &seg_recs, ListFn list_of, PairPlan &plan, int **lst_seg_d,
                            long long **lst_cum_d, double &pairs) {
    int count = 0;
    const PairVariant *vv = pair_variants(&count);
    const PairVariant &v = vv[variant];
    const int TT = v.tile_targets;
    const int C = v.grad == 1 ? 3 : v.D * v.nrhs;  // the gradient kernel: one 3-vector per target
    std::vector<PairTile> tiles;
    std::vector<int> lst;
    std::vector<long long> cum{0};
    std::vector<int> segs;
    long long units = 0;
    pairs = 0.0;
    const int ngroups = (int)toff.size() - 1;
    std::vector<int> tgroup(toff.back());
    for (int g = 0; g < ngroups; ++g)
        for (int t = toff[g]; t < toff[g + 1]; ++t) tgroup[t] = g;
    for (size_t ci = 0; ci + 1 < cuts.size(); ++ci) {
        const int t_end = toff[cuts[ci + 1]];
        int t = toff[cuts[ci]];
        while (t < t_end) {
            int t1 = std::min(t + TT, t_end);
            const int g0 = tgroup[t];
            int g1 = tgroup[t1 - 1];
            if (g1 - g0 + 1 > MFS_MAX_TILE_BODIES) {
                g1 = g0 + MFS_MAX_TILE_BODIES - 1;
                t1 = toff[g1 + 1];
            }
            PairTile tl;
            tl.t0 = t;
            tl.t1 = t1;
            tl.kb0 = gid0 + g0;
            tl.nb = g1 - g0 + 1;
            tl.skip = -1;
            tl.B0 = tl.B1 = 0;
            segs.clear();
            list_of(g0, g1, segs);
            tl.L0 = (int)lst.size();
            long long u = 0;
            for (int sgi : segs) {
                lst.push_back(sgi);
                u += seg_blocks[sgi];
                cum.push_back(units + u);
                pairs += (double)(t1 - t) * seg_recs[sgi];
            }
            tl.L1 = (int)lst.size();
            tl.u0 = units;
            tl.u1 = units + u;
            units += u;
            tiles.push_back(tl);
            t = t1;
        }
    }
    const int occ = pair_occupancy(variant);
    if (occ <= 0) {
        ctx->last_error = "pair kernel variant cannot be resident on this GPU";
        return MFS_ERR_CUDA;
    }
    long long G = (long long)occ * ctx->sm_count;
    if (G > units) G = std::max<long long>(units, 1);
    const long long W = std::max<long long>(units, 1);
    int max_share = 1;
    for (auto &tl : tiles) {
        if (tl.u1 == tl.u0) {
            tl.gA = tl.gB = -1;
            continue;
        }
        auto owner = [&](long long u) { return (int)(((u + 1) * G - 1) / W); };
        tl.gA = owner(tl.u0);
        tl.gB = owner(tl.u1 - 1);
        max_share = std::max(max_share, tl.gB - tl.gA + 1);
    }
    plan.variant = variant;
    plan.include_self = include_self;
    plan.tile_targets = TT;
    plan.G = (int)G;
    plan.ntiles = (int)tiles.size();
    plan.max_share = max_share;
    plan.total_units = units;
    CK(ctx->alloc(&plan.tiles, std::max<size_t>(tiles.size(), 1)));
    CK(cudaMemcpy(plan.tiles, tiles.data(), sizeof(PairTile) * tiles.size(), cudaMemcpyHostToDevice));
    CK(ctx->alloc(&plan.partial, (size_t)G * 2 * TT * C));
    CK(ctx->alloc(&plan.direct, (size_t)std::max(toff.back(), 1) * C));
    CK(ctx->alloc(lst_seg_d, std::max<size_t>(lst.size(), 1)));
    CK(ctx->alloc(lst_cum_d, cum.size()));
    if (!lst.empty()) CK(cudaMemcpy(*lst_seg_d, lst.data(), sizeof(int) * lst.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(*lst_cum_d, cum.data(), sizeof(long long) * cum.size(), cudaMemcpyHostToDevice));
    return MFS_OK;
}

// The far-field plans of one pair-kernel variant: the upward sums (each node's check points against
// its descendant bodies' proxy points) and the evaluation (targets in tree order against their
// interaction lists).
mfs_status ff_get_plan(mfs_ctx *ctx, mfs_ctx::FarField &F, int variant, int include_self,
                       mfs_ctx::FarField::Plan **out) {
    const int key = variant * 2 + include_self;
    auto it = F.plans.find(key);
    if (it != F.plans.end()) {
        *out = &it->second;
        return MFS_OK;
    }
    mfs_ctx::FarField::Plan pl;
    const int P = ctx->P, nodes = F.nodes;
    std::vector<long long> seg_blocks(P + nodes);
    std::vector<int> seg_recs(P + nodes);
    for (int sg = 0; sg < P + nodes; ++sg) {
        seg_recs[sg] = F.seg_rec1_h[sg] - F.seg_rec0_h[sg];
        seg_blocks[sg] = (seg_recs[sg] + MFS_BS - 1) / MFS_BS;
    }
    // upward: one group per node, tiles never span two nodes
    std::vector<int> toff_up(nodes + 1), cuts_up(nodes + 1);
    for (int n = 0; n <= nodes; ++n) {
        toff_up[n] = n * FF_NC;
        cuts_up[n] = n;
    }
    CKS(build_plan_lists(ctx, variant, 1, toff_up, P, cuts_up, seg_blocks, seg_recs,
                         [&](int g0, int g1, std::vector<int> &segs) {
                             for (int n = g0; n <= g1; ++n)
                                 for (int q = F.tree.nodes[n].first; q < F.tree.nodes[n].first + F.tree.nodes[n].count;
                                      ++q)
                                     segs.push_back(q);
                         },
                         pl.up, &pl.lst_seg_up, &pl.lst_cum_up, pl.pairs_up));
    // evaluation: groups are the bodies in tree order; tiles stay inside a suspension
    std::vector<int> toff_ev(P + 1, 0);
    for (int q = 0; q < P; ++q) {
        const int b = F.tree.order[q];
        toff_ev[q + 1] = toff_ev[q] + ((*F.tgt_off)[b + 1] - (*F.tgt_off)[b]);
    }
    std::vector<int> cuts_ev(ctx->S + 1);
    for (int sp = 0; sp <= ctx->S; ++sp) cuts_ev[sp] = ctx->body_off[sp];
    std::vector<int> suspension_of(P);
    for (int sp = 0; sp < ctx->S; ++sp)
        for (int b = ctx->body_off[sp]; b < ctx->body_off[sp + 1]; ++b) suspension_of[b] = sp;
    std::vector<int> tb;
    CKS(build_plan_lists(ctx, variant, include_self, toff_ev, 0, cuts_ev, seg_blocks, seg_recs,
                         [&](int g0, int g1, std::vector<int> &segs) {
                             tb.clear();
                             for (int q = g0; q <= g1; ++q) tb.push_back(F.tree.order[q]);
                             ff_interaction_list(F.tree, F.tree.roots[suspension_of[tb[0]]], tb, ctx->centres.data(),
                                                 F.rtgt.data(), ctx->opt.farfield_separation, !include_self, segs);
                         },
                         pl.ev, &pl.lst_seg_ev, &pl.lst_cum_ev, pl.pairs_ev));
    pl.ev.include_self = include_self;
    it = F.plans.emplace(key, pl).first;
    *out = &it->second;
    return MFS_OK;
}

// One pair-kernel launch on the far-field geometry, bracketed by profiling events like pair_apply's.
mfs_status ff_launch(mfs_ctx *ctx, int variant, const PairGeom &g, const PairWork &w, cudaStream_t st) {
    if (w.total_units == 0) return MFS_OK;
    const size_t slot = 2 * (size_t)ctx->pair_launches;
    if (ctx->opt.profile) {
        while (ctx->pev.size() < slot + 2) {
            cudaEvent_t e;
            CK(cudaEventCreate(&e));
            ctx->pev.push_back(e);
        }
        CK(cudaEventRecord(ctx->pev[slot], st));
    }
    CK(pair_launch(variant, g, w, ctx->err_d, st));
    if (ctx->opt.profile) CK(cudaEventRecord(ctx->pev[slot + 1], st));
    ctx->launches += 1;
    ctx->pair_launches += 1;
    return MFS_OK;
}

// The geometry of a far-field launch: the tree-ordered centres and the segments' record ranges.
static PairGeom ff_geom(const mfs_ctx::FarField &F) {
    PairGeom g;
    g.src = F.rec;
    g.src_off = nullptr;
    g.blk_off = nullptr;
    g.centres = F.centres;
    g.seg_rec0 = F.seg_rec0;
    g.seg_rec1 = F.seg_rec1;
    return g;
}

// The upward step of the treecode: the sources (records in the layout of `variant`, packed into
// F.rec) summed at every node's check points over the node's descendant bodies, then the node's
// equivalent strengths F.mu = (FP64 product with the pseudo-inverse) scaled by the radius.
static mfs_status ff_upward(mfs_ctx *ctx, mfs_ctx::FarField &F, int variant, const mfs_ctx::FarField::Plan *pl,
                            const double *strength, int nrhs, cudaStream_t st) {
    int vc = 0;
    const PairVariant *vv = pair_variants(&vc);
    const int D = ctx->D, nodes = F.nodes;
    if (pair_record_floats(D, nrhs, vv[variant].packed) > F.rec_floats) {
        ctx->last_error = "far field: record layout larger than its buffer";
        return MFS_ERR_INVALID_ARG;
    }
    CK(pack_sources(D, nrhs, vv[variant].packed, F.src_pos, F.rec_pt, strength, F.nsrc, F.nrec, F.rec, st));
    PairGeom g = ff_geom(F);
    g.lst_seg = pl->lst_seg_up;
    g.lst_cum = pl->lst_cum_up;
    g.tgt = F.chk_pos;
    g.ntargets = nodes * FF_NC;
    const PairWork wu = work_of(pl->up);
    CKS(ff_launch(ctx, variant, g, wu, st));
    CK(pair_epilogue(D, nrhs, wu, nullptr, 0.0, 1.0, F.ucheck, nodes * FF_NC, st));
    const int Sk = gemm_rm64_chunks(nrhs * nodes, D * FF_NE, D * FF_NC, ctx->sm_count);
    CK(gemm_rm64_splitk(nrhs * nodes, D * FF_NE, D * FF_NC, Sk, F.ucheck, F.PinvT, F.fit_chunks, F.mu, st));
    CK(ff_scale(F.mu, F.re, nodes, D * FF_NE, nrhs, st));
    ctx->launches += 4;
    return MFS_OK;
}

// out = beta * base + scale * (pair sum of strengths) through the treecode: the upward step, the
// equivalent strengths' records, then the evaluation over the interaction lists (results written
// back in the caller's target order).
mfs_status ff_pair_apply(mfs_ctx *ctx, mfs_ctx::FarField &F, int variant, const double *strength, double *out,
                         const double *base, double beta, double scale, int nrhs, int include_self, cudaStream_t st) {
    mfs_ctx::FarField::Plan *pl = nullptr;
    CKS(ff_get_plan(ctx, F, variant, include_self, &pl));
    int vc = 0;
    const PairVariant *vv = pair_variants(&vc);
    const int D = ctx->D, nodes = F.nodes;
    const int REC = pair_record_floats(D, nrhs, vv[variant].packed);
    CKS(ff_upward(ctx, F, variant, pl, strength, nrhs, st));
    CK(pack_sources(D, nrhs, vv[variant].packed, F.eq_pos, F.eq_pt, F.mu, nodes * FF_NE, nodes * FF_NE,
                    F.rec + (size_t)F.nrec * REC, st));
    PairGeom g = ff_geom(F);
    g.lst_seg = pl->lst_seg_ev;
    g.lst_cum = pl->lst_cum_ev;
    g.tgt = F.tgt;
    g.ntargets = F.ntgt;
    PairWork we = work_of(pl->ev);
    we.tperm = F.tperm;
    CKS(ff_launch(ctx, variant, g, we, st));
    CK(pair_epilogue(D, nrhs, we, base, beta, scale, out, F.ntgt, st));
    ctx->launches += 3;
    return MFS_OK;
}

// wt[h][t][c] = (float) v[h][perm[t]][c]: per-target weights in the tree's target order.
static __global__ void ff_gather_weights_kernel(const double *v, const int *perm, int n, int nrhs, float *wt) {
    const size_t total = (size_t)nrhs * n * 3;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const size_t h = e / ((size_t)n * 3), r = e % ((size_t)n * 3);
        const int t = (int)(r / 3), c = (int)(r % 3);
        wt[e] = (float)v[(h * n + perm[t]) * 3 + c];
    }
}

// The adjoint's pair gradient through the treecode, per target of F (scaled, FP64, caller's order):
//   out_t = scale * sum_h sum_{s not on t's body} grad_r (tw_h(t)^T G(r) sigma_h(s)),  r = x_t - y_s,
// with sigma the sources' strengths (near bodies directly, far nodes through the equivalent
// strengths fitted to sigma) and tw the targets' weights.  On the forward tree (targets the
// collocation points, tw = w, sigma = mu) it is the target side of the centre gradient; on the
// transposed tree (targets the proxy points, tw = mu, sigma = w) its source side with the sign
// reversed (G symmetric and even, so its gradient is odd).
mfs_status ff_grad_apply(mfs_ctx *ctx, mfs_ctx::FarField &F, int gv, const double *sigma, const double *tw, int nrhs,
                         double *out, cudaStream_t st) {
    const int fv = fp32_variant(ctx, 3, nrhs);  // the upward sums: the forward pair kernel
    mfs_ctx::FarField::Plan *pu = nullptr, *pg = nullptr;
    CKS(ff_get_plan(ctx, F, fv, 1, &pu));
    CKS(ff_get_plan(ctx, F, gv, 0, &pg));
    CKS(ff_upward(ctx, F, fv, pu, sigma, nrhs, st));
    // records of the gradient kernel (plain layout): the sources, then the equivalent points
    const int REC = pair_record_floats(3, nrhs, 0), nodes = F.nodes;
    CK(pack_sources(3, nrhs, 0, F.src_pos, F.rec_pt, sigma, F.nsrc, F.nrec, F.rec, st));
    CK(pack_sources(3, nrhs, 0, F.eq_pos, F.eq_pt, F.mu, nodes * FF_NE, nodes * FF_NE, F.rec + (size_t)F.nrec * REC,
                    st));
    if (!F.wt) CK(ctx->alloc(&F.wt, (size_t)ctx->opt.max_rhs * F.ntgt * 3));
    ff_gather_weights_kernel<<<1024, 256, 0, st>>>(tw, F.tperm, F.ntgt, nrhs, F.wt);
    CK(cudaGetLastError());
    PairGeom g = ff_geom(F);
    g.lst_seg = pg->lst_seg_ev;
    g.lst_cum = pg->lst_cum_ev;
    g.tgt = F.tgt;
    g.ntargets = F.ntgt;
    g.tgt_w = F.wt;
    PairWork we = work_of(pg->ev);
    we.tperm = F.tperm;
    we.src_grad = nullptr;  // segments are bodies and nodes here: no per-source-body reduction
    CKS(ff_launch(ctx, gv, g, we, st));
    CK(pair_epilogue(3, 1, we, nullptr, 0.0, kernel_scale(ctx), out, F.ntgt, st));
    ctx->launches += 5;
    return MFS_OK;
}

// pairs evaluated per right-hand side by one pair sum
double pair_count(mfs_ctx *ctx, int include_self) {
    double total = 0.0;
    for (int s = 0; s < ctx->S; ++s) {
        double sm = 0, sn = 0, self = 0;
        for (int k = ctx->body_off[s]; k < ctx->body_off[s + 1]; ++k) {
            const double m = ctx->tgt_off[k + 1] - ctx->tgt_off[k], n = ctx->src_off[k + 1] - ctx->src_off[k];
            sm += m;
            sn += n;
            self += m * n;
        }
        total += sm * sn - (include_self ? 0.0 : self);
    }
    return total;
}

// lambda = (I - L) S_L^+ gamma (project) or S_L^+ gamma  (Eq. pseudo, Remark congruent)
mfs_status precond_apply_dev(mfs_ctx *ctx, const double *gamma, double *lambda, int project, int nrhs,
                             cudaStream_t st) {
    const int D = ctx->D;
    for (auto &sh : ctx->shapes) {
        const int nb = (int)sh.bodies.size();
        if (nb == 0) continue;
        const int ncols = nb * nrhs;
        const FactorSet &fx = sh.fs[ctx->fset];
        const ShapeDev &sd = fx.dev;
        if (ctx->opt.precision >= 1) {  // FP64 one-body apply (reference and mixed modes)
            CK(gather_rotate(D, gamma, ctx->sumM * D, sh.col_body, sh.col_rhs, ctx->tgt_off_d, ctx->rot64_d, ncols,
                             sd.dM, sh.A, sh.A64, st));
            CK(gemm_rm64(ncols, sd.r, sd.dM, sh.A64, sd.U64, sh.T64, st));
            CK(gemm_rm64(ncols, sd.dN, sd.r, sh.T64, project ? sd.Wp64 : sd.Wr64, sh.L64, st));
            CK(scatter_rotate(D, nullptr, sh.L64, sh.col_body, sh.col_rhs, ctx->src_off_d, ctx->rot_d, ctx->rot64_d,
                              ncols, sd.dN, ctx->sumN, lambda, st));
        } else if (fx.tc_ready) {  // tensor cores: multi-piece TF32 tcgen05 GEMMs, double-float chunk sums
            const int np = sh.pieces;
            auto it = sh.amaps.find(ncols);
            if (it == sh.amaps.end()) {
                std::array<TcMap, 6> mp;
                const int bn = tc_gemm_bn(ncols, np);
                bool enc = true;
                for (int p = 0; p < np; ++p)
                    enc = enc && make_tc_map(mp[p], sh.Ap + p * sh.ap_stride, ncols, sh.ld1, bn) &&
                          make_tc_map(mp[3 + p], sh.Tp + p * sh.tp_stride, ncols, sh.ld2, bn);
                if (!enc) {
                    ctx->last_error = "tensor-map encoding for the tensor-core apply failed";
                    return MFS_ERR_CUDA;
                }
                it = sh.amaps.emplace(ncols, mp).first;
            }
            const std::array<TcMap, 6> &mp = it->second;
            // t = U^T g (Eq. pseudo): gathered columns as pieces, chunk sums re-cut into pieces of t
            CK(gather_rotate_pieces(D, gamma, ctx->sumM * D, sh.col_body, sh.col_rhs, ctx->tgt_off_d, ctx->rot64_d,
                                    ncols, sd.dM, sh.Ap, sh.ld1, sh.ap_stride, np, st));
            const int S1 = tc_gemm_chunks(ncols, sd.r, sd.dM, ctx->sm_count, np);
            CK(tc_gemm(np, fx.mU, mp.data(), ncols, sd.r, sd.dM, S1, sh.Ptc, ctx->err_d, st));
            CK(reduce_pieces(tc_gemm_sz(sd.dM, S1), ncols, sd.r, sh.Ptc, sh.Tp, sh.ld2, sh.tp_stride, np, st));
            // lambda = W t, kept in FP64
            const int S2 = tc_gemm_chunks(ncols, sd.dN, sd.r, ctx->sm_count, np);
            CK(tc_gemm(np, project ? fx.mWp : fx.mWr, mp.data() + 3, ncols, sd.dN, sd.r, S2, sh.Ptc, ctx->err_d, st));
            CK(reduce_f64(tc_gemm_sz(sd.r, S2), (size_t)ncols * sd.dN, sh.Ptc, sh.L64, st));
            CK(scatter_rotate(D, nullptr, sh.L64, sh.col_body, sh.col_rhs, ctx->src_off_d, ctx->rot_d, ctx->rot64_d,
                              ncols, sd.dN, ctx->sumN, lambda, st));
            ctx->launches += 2;
        } else {
            CK(gather_rotate(D, gamma, ctx->sumM * D, sh.col_body, sh.col_rhs, ctx->tgt_off_d, ctx->rot64_d, ncols,
                             sd.dM, sh.A, nullptr, st));
            // t = U^T g (FP32 result), then lambda = W t kept in FP64 (split-K, compensated; Eq. pseudo)
            const int S1 = gemm_splitk_chunks(ncols, sd.r, sd.dM, ctx->sm_count);
            const int S2 = gemm_splitk_chunks(ncols, sd.dN, sd.r, ctx->sm_count);
            CK(gemm_splitk(ncols, sd.r, sd.dM, S1, sh.A, sd.U, sh.Pk, sh.Tm, nullptr, st));
            CK(gemm_splitk(ncols, sd.dN, sd.r, S2, sh.Tm, project ? sd.Wp : sd.Wr, sh.Pk, nullptr, sh.L64, st));
            CK(scatter_rotate(D, nullptr, sh.L64, sh.col_body, sh.col_rhs, ctx->src_off_d, ctx->rot_d, ctx->rot64_d,
                              ncols, sd.dN, ctx->sumN, lambda, st));
            ctx->launches += 2;
        }
        ctx->launches += 4;
    }
    return MFS_OK;
}

// y = gamma + sum_{k' != k} S^(kk') (I - L^(k')) S_L^(k')+ gamma^(k')  (Eq. 2esysprec)
mfs_status matvec_dev(mfs_ctx *ctx, const double *gamma, double *y, int nrhs, cudaStream_t st) {
    CKS(precond_apply_dev(ctx, gamma, ctx->lam_d, 1, nrhs, st));
    CKS(pair_apply(ctx, ctx->lam_d, y, gamma, 1.0, 1.0, nrhs, 0, st));
    return MFS_OK;
}

mfs_status ensure_gmres(mfs_ctx *ctx, int nrhs) {
    const long long n = (long long)nrhs * ctx->sumM * ctx->D;
    const int L = nrhs * ctx->S;
    const int m = std::min(ctx->opt.restart, ctx->opt.max_iter);
    if (ctx->gd.V && ctx->gd_n == (size_t)n && ctx->gd_L == L && ctx->gd_m == m) return MFS_OK;
    // free old
    void *olds[] = {ctx->gd.V, ctx->gd.H, ctx->gd.cs, ctx->gd.sn, ctx->gd.g, ctx->gd.beta, ctx->gd.hbuf,
                    ctx->gd.htmp, ctx->gd.hn, ctx->gd.part, ctx->gd.active, ctx->gd.iters, ctx->gd.status,
                    ctx->gd.resid, ctx->gd.done, ctx->gd.jcur, ctx->seg_off_d, ctx->w_d, ctx->b_d, ctx->x_d,
                    ctx->ysmall_d, ctx->vin_d};
    ctx->drop_graphs();  // they hold the old buffers' addresses
    for (void *p : olds) ctx->release(p);
    ctx->vin_d = nullptr;
    GmresDev &gd = ctx->gd;
    gd = GmresDev{};
    gd.L = L;
    gd.m = m;
    gd.n = n;
    gd.tol = ctx->opt.gmres_tol;
    // blocks per lane: one wave over all lanes (SMs / L, so that no SM runs two blocks while others
    // run one), but at least ~2048 elements per block (8 per thread), so that the FP64 work of the dot
    // products outweighs their block reductions
    const long long per_lane = n / std::max(L, 1);
    gd.part_blocks = (int)std::max<long long>(1, std::min<long long>((long long)ctx->sm_count / std::max(L, 1),
                                                                     (per_lane + 2047) / 2048));
    gd.part_blocks = std::min(gd.part_blocks, 512);
    std::vector<long long> seg(L + 1);
    for (int h = 0; h < nrhs; ++h)
        for (int s = 0; s < ctx->S; ++s) {
            const int l = h * ctx->S + s;
            seg[l] = (long long)h * ctx->sumM * ctx->D + (long long)ctx->tgt_off[ctx->body_off[s]] * ctx->D;
        }
    seg[L] = n;
    CK(ctx->alloc(&ctx->seg_off_d, L + 1));
    CK(cudaMemcpy(ctx->seg_off_d, seg.data(), sizeof(long long) * (L + 1), cudaMemcpyHostToDevice));
    gd.seg_off = ctx->seg_off_d;
    CK(ctx->alloc(&gd.V, (size_t)(m + 1) * n));
    CK(cudaMemset(gd.V, 0, sizeof(double) * (size_t)(m + 1) * n));
    CK(ctx->alloc(&gd.H, (size_t)L * (m + 1) * m));
    CK(ctx->alloc(&gd.cs, (size_t)L * m));
    CK(ctx->alloc(&gd.sn, (size_t)L * m));
    CK(ctx->alloc(&gd.g, (size_t)L * (m + 1)));
    CK(ctx->alloc(&gd.beta, L));
    CK(ctx->alloc(&gd.hbuf, (size_t)L * (m + 1)));
    CK(ctx->alloc(&gd.htmp, (size_t)L * (m + 1)));
    CK(ctx->alloc(&gd.hn, L));
    CK(ctx->alloc(&gd.part, (size_t)L * gd.part_blocks * (m + 1)));
    CK(ctx->alloc(&gd.active, L));
    CK(ctx->alloc(&gd.iters, L));
    CK(ctx->alloc(&gd.status, L));
    CK(ctx->alloc(&gd.resid, L));
    CK(ctx->alloc(&gd.done, 1));
    CK(ctx->alloc(&gd.jcur, 1));
    CK(ctx->alloc(&ctx->vin_d, n));
    CK(ctx->alloc(&ctx->w_d, n));
    CK(ctx->alloc(&ctx->b_d, n));
    CK(ctx->alloc(&ctx->x_d, n));
    CK(ctx->alloc(&ctx->ysmall_d, (size_t)L * (m + 1)));
    ctx->gd_n = n;
    ctx->gd_L = L;
    ctx->gd_m = m;
    return MFS_OK;
}

// ---------------------------------------------------------------------------
// Adjoint (transposed) operators
// ---------------------------------------------------------------------------
// dst[c][r] = src[r][c], FP64 (setup of the FP64 adjoint's factor transposes).
static __global__ void transpose64_kernel(const double *src, int rows, int cols, double *dst) {
    const size_t n = (size_t)rows * cols;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[(i % cols) * rows + i / cols] = src[i];
}

// The transposed geometry: proxy points as targets (float4 with body bits), collocation points
// as sources packed into records with their own padded offsets; plus adjoint scratch; with
// farfield = 1 the treecode of the transposed sums (collocation sources, proxy targets).
mfs_status ensure_transposed(mfs_ctx *ctx) {
    if (ctx->trans_ready) return MFS_OK;
    const int P = ctx->P, R = ctx->opt.max_rhs;
    ctx->src_body.resize(ctx->sumN);
    for (int k = 0; k < P; ++k)
        for (int q = ctx->src_off[k]; q < ctx->src_off[k + 1]; ++q) ctx->src_body[q] = k;
    ctx->recT_off.assign(P + 1, 0);
    ctx->blkT_off.assign(P + 1, 0);
    for (int k = 0; k < P; ++k) {
        const int mpad = (ctx->tgt_off[k + 1] - ctx->tgt_off[k] + 3) / 4 * 4;
        ctx->recT_off[k + 1] = ctx->recT_off[k] + mpad;
        ctx->blkT_off[k + 1] = ctx->blkT_off[k] + (mpad + MFS_BS - 1) / MFS_BS;
    }
    ctx->nrecT = ctx->recT_off[P];
    std::vector<int> rec_pt(ctx->nrecT, -1);
    for (int k = 0; k < P; ++k)
        for (int i = 0; i < ctx->tgt_off[k + 1] - ctx->tgt_off[k]; ++i) rec_pt[ctx->recT_off[k] + i] = ctx->tgt_off[k] + i;
    // proxy targets: rotated local coordinates with the body id in w
    std::vector<float4> tp(ctx->sumN);
    std::vector<float> s4(4 * (size_t)ctx->sumN);
    CK(cudaMemcpy(tp.data(), ctx->src_pos_d, sizeof(float4) * ctx->sumN, cudaMemcpyDeviceToHost));
    for (int q = 0; q < ctx->sumN; ++q) {
        int k = ctx->src_body[q];
        float kb;
        std::memcpy(&kb, &k, sizeof(float));
        tp[q].w = kb;
    }
    const int recf = std::max(pair_record_floats(3, R, 0), pair_record_floats(3, R, 1));
    ctx->recT_floats = recf;
    CK(ctx->alloc(&ctx->tgtT_pos_d, ctx->sumN));
    CK(ctx->alloc(&ctx->recT_d, (size_t)ctx->nrecT * recf));
    CK(ctx->alloc(&ctx->recT_off_d, P + 1));
    CK(ctx->alloc(&ctx->rec_ptT_d, ctx->nrecT));
    CK(ctx->alloc(&ctx->blkT_off_d, P + 1));
    CK(ctx->alloc(&ctx->tmpM_d, (size_t)R * ctx->sumM * 3));
    CK(ctx->alloc(&ctx->gradT_d, (size_t)ctx->sumM * 3));
    CK(ctx->alloc(&ctx->src_grad_d, (size_t)P * 3));
    CK(ctx->alloc(&ctx->six_d, (size_t)R * P * 6));
    CK(ctx->alloc(&ctx->w32_d, (size_t)R * ctx->sumM * 3));
    CK(ctx->alloc(&ctx->eye6_d, (size_t)ctx->nshapes * 36));
    CK(cudaMemcpy(ctx->tgtT_pos_d, tp.data(), sizeof(float4) * ctx->sumN, cudaMemcpyHostToDevice));
    CK(cudaMemset(ctx->recT_d, 0, sizeof(float) * (size_t)ctx->nrecT * recf));
    CK(cudaMemcpy(ctx->recT_off_d, ctx->recT_off.data(), sizeof(int) * (P + 1), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->rec_ptT_d, rec_pt.data(), sizeof(int) * ctx->nrecT, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->blkT_off_d, ctx->blkT_off.data(), sizeof(long long) * (P + 1), cudaMemcpyHostToDevice));
    std::vector<double> eye(36 * (size_t)ctx->nshapes, 0.0);
    for (int s = 0; s < ctx->nshapes; ++s)
        for (int i = 0; i < 6; ++i) eye[36 * s + 7 * i] = 1.0;
    CK(cudaMemcpy(ctx->eye6_d, eye.data(), sizeof(double) * eye.size(), cudaMemcpyHostToDevice));
    for (auto &sh : ctx->shapes) {  // transposed-apply buffers
        const int nb = (int)sh.bodies.size();
        if (nb == 0) continue;
        const int m = sh.fs[0].dev.dM, n = sh.fs[0].dev.dN;
        size_t need = 0;
        for (int h = 1; h <= R; ++h) {
            const int rows = h * nb;
            need = std::max(need, (size_t)gemm_splitk_chunks(rows, n, n, ctx->sm_count) * rows * n);
            need = std::max(need, (size_t)gemm_splitk_chunks(rows, m, n, ctx->sm_count) * rows * m);
        }
        CK(ctx->alloc(&sh.PkT, need));
        CK(ctx->alloc(&sh.O64, (size_t)R * nb * m));
        FactorSet &fx = sh.fs[0];
        if (fx.tc_ready) {  // tensor cores: the factor planes transposed (exact), their maps, chunk results
            const int np = sh.pieces;
            fx.un_stride = (size_t)m * sh.ld2;
            CK(ctx->alloc(&fx.Un, 2 * fx.un_stride));
            CK(ctx->alloc(&fx.WpT, 2 * fx.wt_stride));
            CK(ctx->alloc(&fx.WrT, 2 * fx.wt_stride));
            // U^T planes [r][ld1] -> U planes [dM][ld2]; W planes [dN][ld2] -> W^T planes [r][ld2]
            CK(transpose_pieces(fx.Utp, n, m, sh.ld1, fx.ut_stride, fx.Un, sh.ld2, fx.un_stride, 2, 0));
            CK(transpose_pieces(fx.Wptp, n, n, sh.ld2, fx.wt_stride, fx.WpT, sh.ld2, fx.wt_stride, 2, 0));
            CK(transpose_pieces(fx.Wrtp, n, n, sh.ld2, fx.wt_stride, fx.WrT, sh.ld2, fx.wt_stride, 2, 0));
            CK(cudaDeviceSynchronize());
            bool enc = true;
            for (int p = 0; p < 2; ++p)
                enc = enc && make_tc_map(fx.mUn[p], fx.Un + p * fx.un_stride, m, sh.ld2, 128) &&
                      make_tc_map(fx.mWpT[p], fx.WpT + p * fx.wt_stride, n, sh.ld2, 128) &&
                      make_tc_map(fx.mWrT[p], fx.WrT + p * fx.wt_stride, n, sh.ld2, 128);
            if (!enc) {
                ctx->last_error = "tensor-map encoding for the transposed tensor-core apply failed";
                return MFS_ERR_CUDA;
            }
            size_t needT = 0;
            for (int h = 1; h <= R; ++h) {
                const int cols = h * nb;
                needT = std::max(needT, (size_t)tc_gemm_sz(n, tc_gemm_chunks(cols, n, n, ctx->sm_count, np)) * cols * n);
                needT = std::max(needT, (size_t)tc_gemm_sz(n, tc_gemm_chunks(cols, m, n, ctx->sm_count, np)) * cols * m);
            }
            CK(ctx->alloc(&sh.PtcT, needT));
            fx.tcT_ready = true;
        }
    }
    if (ctx->opt.precision == 1) {  // the FP64 transposed sums and one-body apply
        std::vector<double> tl(3 * (size_t)ctx->sumM), c4(4 * (size_t)ctx->sumM);
        CK(cudaMemcpy(tl.data(), ctx->tgt_local64_d, sizeof(double) * tl.size(), cudaMemcpyDeviceToHost));
        for (int i = 0; i < ctx->sumM; ++i) {
            for (int a = 0; a < 3; ++a) c4[4 * (size_t)i + a] = tl[3 * (size_t)i + a];
            c4[4 * (size_t)i + 3] = (double)ctx->tgt_body[i];
        }
        std::vector<int> cb(P), ce(P);
        for (int sp = 0; sp < ctx->S; ++sp)
            for (int k = ctx->body_off[sp]; k < ctx->body_off[sp + 1]; ++k) {
                cb[k] = ctx->tgt_off[ctx->body_off[sp]];
                ce[k] = ctx->tgt_off[ctx->body_off[sp + 1]];
            }
        CK(ctx->alloc(&ctx->src_body_d, ctx->sumN));
        CK(ctx->alloc(&ctx->colloc4_d, c4.size()));
        CK(ctx->alloc(&ctx->colT_begin_d, P));
        CK(ctx->alloc(&ctx->colT_end_d, P));
        CK(cudaMemcpy(ctx->src_body_d, ctx->src_body.data(), sizeof(int) * ctx->sumN, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(ctx->colloc4_d, c4.data(), sizeof(double) * c4.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(ctx->colT_begin_d, cb.data(), sizeof(int) * P, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(ctx->colT_end_d, ce.data(), sizeof(int) * P, cudaMemcpyHostToDevice));
        for (auto &sh : ctx->shapes) {
            if (sh.bodies.empty()) continue;
            ShapeDev &sd = sh.fs[0].dev;
            CK(ctx->alloc(&sd.UT64, (size_t)sd.dM * sd.r));
            CK(ctx->alloc(&sd.WpT64, (size_t)sd.r * sd.dN));
            CK(ctx->alloc(&sd.WrT64, (size_t)sd.r * sd.dN));
            transpose64_kernel<<<1024, 256>>>(sd.U64, sd.dM, sd.r, sd.UT64);
            transpose64_kernel<<<1024, 256>>>(sd.Wp64, sd.r, sd.dN, sd.WpT64);
            transpose64_kernel<<<1024, 256>>>(sd.Wr64, sd.r, sd.dN, sd.WrT64);
            CK(cudaGetLastError());
        }
        CK(cudaDeviceSynchronize());
    }
    if (ctx->opt.farfield) {
        auto &F = ctx->ffT;
        F.src_colloc = true;
        F.src_pos = ctx->tgt_pos_d;
        F.rec_pt = ctx->rec_ptT_d;
        F.nsrc = ctx->sumM;
        F.nrec = ctx->nrecT;
        F.rec_off = &ctx->recT_off;
        F.tgt_pos = ctx->tgtT_pos_d;
        F.tgt_off = &ctx->src_off;
        F.ntgt = ctx->sumN;
        CKS(ff_setup(ctx, F, 0));
    }
    ctx->trans_ready = true;
    return MFS_OK;
}

// z^(k') = sum_k S^(kk')^T w^(k) at the proxy points (the Stokeslet is symmetric and even in r),
// self pairs included or not.  w: [nrhs][sum_M][3], z: [nrhs][sum_N][3], both FP64 on the device.
mfs_status pair_apply_T(mfs_ctx *ctx, const double *w, double *z, int nrhs, int include_self, cudaStream_t st) {
    if (ctx->opt.precision == 1) {  // FP64 reference: the plain FP64 loops with the roles swapped
        CK(pair_sum_fp64(3, nrhs, ctx->src_local64_d, ctx->src_body_d, ctx->sumN, ctx->colloc4_d, ctx->sumM,
                         ctx->colT_begin_d, ctx->colT_end_d, ctx->tgt_off_d, ctx->centres_d, w, include_self,
                         ctx->raw_d, st));
        const size_t n = (size_t)nrhs * ctx->sumN * 3;
        combine_raw_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ctx->raw_d, nullptr, 0.0, kernel_scale(ctx), z,
                                                                        n);
        CK(cudaGetLastError());
        ctx->launches += 2;
        return MFS_OK;
    }
    const int variant = fp32_variant(ctx, 3, nrhs);
    if (ctx->ffT.ready)
        return ff_pair_apply(ctx, ctx->ffT, variant, w, z, nullptr, 0.0, kernel_scale(ctx), nrhs, include_self, st);
    int vc = 0;
    const PairVariant *vv = pair_variants(&vc);
    if (pair_record_floats(3, nrhs, vv[variant].packed) > ctx->recT_floats) {
        ctx->last_error = "transposed pair sum: record layout larger than its buffer";
        return MFS_ERR_INVALID_ARG;
    }
    PairPlan *plan = nullptr;
    CKS(get_plan(ctx, variant, include_self, &plan, 1));
    CK(pack_sources(3, nrhs, vv[variant].packed, ctx->tgt_pos_d, ctx->rec_ptT_d, w, ctx->sumM, ctx->nrecT,
                    ctx->recT_d, st));
    PairGeom g;
    g.tgt = ctx->tgtT_pos_d;
    g.src = ctx->recT_d;
    g.src_off = ctx->recT_off_d;
    g.blk_off = ctx->blkT_off_d;
    g.centres = ctx->centres_d;
    g.ntargets = ctx->sumN;
    const PairWork wk = work_of(*plan);
    if (wk.total_units > 0) {
        CK(pair_launch(variant, g, wk, ctx->err_d, st));
        ctx->launches += 1;
    }
    CK(pair_epilogue(3, nrhs, wk, nullptr, 0.0, kernel_scale(ctx), z, ctx->sumN, st));
    ctx->launches += 2;
    return MFS_OK;
}

// out^(k) = ((I - L^(k)) S_L^(k)+)^T z^(k) = R_M U W_p R_N^T z (project) or (S_L^(k)+)^T z = R_M U W_r R_N^T z,
// z [nrhs][sum_N][3] -> out [nrhs][sum_M][3] (transposes of the two-step apply, Eq. pseudo).
mfs_status precondT_dev(mfs_ctx *ctx, const double *z, double *out, int project, int nrhs, cudaStream_t st) {
    for (auto &sh : ctx->shapes) {
        const int nb = (int)sh.bodies.size();
        if (nb == 0) continue;
        const int ncols = nb * nrhs;
        const FactorSet &fx = sh.fs[0];
        const ShapeDev &sd = fx.dev;
        if (ctx->opt.precision == 1) {
            // FP64 reference: out = R_M U (W (R_N^T z)) with the transposed FP64 factors
            CK(gather_rotate(3, z, ctx->sumN * 3, sh.col_body, sh.col_rhs, ctx->src_off_d, ctx->rot64_d, ncols, sd.dN,
                             sh.A, sh.A64, st));
            CK(gemm_rm64(ncols, sd.r, sd.dN, sh.A64, project ? sd.WpT64 : sd.WrT64, sh.T64, st));
            CK(gemm_rm64(ncols, sd.dM, sd.r, sh.T64, sd.UT64, sh.O64, st));
            CK(scatter_rotate(3, nullptr, sh.O64, sh.col_body, sh.col_rhs, ctx->tgt_off_d, ctx->rot_d, ctx->rot64_d,
                              ncols, sd.dM, ctx->sumM, out, st));
            ctx->launches += 4;
            continue;
        }
        if (fx.tcT_ready && ctx->opt.precision == 0) {
            // tensor cores, as the forward apply: x = W^T (R_N^T z) with the K = dN column pieces in Tp,
            // x cut back into pieces (same layout, Tp reused), out = R_M U x kept in FP64
            const int np = sh.pieces;
            auto it = sh.amaps.find(ncols);
            if (it == sh.amaps.end()) {
                std::array<TcMap, 6> mp;
                const int bn = tc_gemm_bn(ncols, np);
                bool enc = true;
                for (int p = 0; p < np; ++p)
                    enc = enc && make_tc_map(mp[p], sh.Ap + p * sh.ap_stride, ncols, sh.ld1, bn) &&
                          make_tc_map(mp[3 + p], sh.Tp + p * sh.tp_stride, ncols, sh.ld2, bn);
                if (!enc) {
                    ctx->last_error = "tensor-map encoding for the tensor-core apply failed";
                    return MFS_ERR_CUDA;
                }
                it = sh.amaps.emplace(ncols, mp).first;
            }
            const TcMap *colmaps = it->second.data() + 3;
            CK(gather_rotate_pieces(3, z, ctx->sumN * 3, sh.col_body, sh.col_rhs, ctx->src_off_d, ctx->rot64_d, ncols,
                                    sd.dN, sh.Tp, sh.ld2, sh.tp_stride, np, st));
            const int S1 = tc_gemm_chunks(ncols, sd.r, sd.dN, ctx->sm_count, np);
            CK(tc_gemm(np, project ? fx.mWpT : fx.mWrT, colmaps, ncols, sd.r, sd.dN, S1, sh.PtcT, ctx->err_d, st));
            CK(reduce_pieces(tc_gemm_sz(sd.dN, S1), ncols, sd.r, sh.PtcT, sh.Tp, sh.ld2, sh.tp_stride, np, st));
            const int S2 = tc_gemm_chunks(ncols, sd.dM, sd.r, ctx->sm_count, np);
            CK(tc_gemm(np, fx.mUn, colmaps, ncols, sd.dM, sd.r, S2, sh.PtcT, ctx->err_d, st));
            CK(reduce_f64(tc_gemm_sz(sd.r, S2), (size_t)ncols * sd.dM, sh.PtcT, sh.O64, st));
            CK(scatter_rotate(3, nullptr, sh.O64, sh.col_body, sh.col_rhs, ctx->tgt_off_d, ctx->rot_d, ctx->rot64_d,
                              ncols, sd.dM, ctx->sumM, out, st));
            ctx->launches += 6;
            continue;
        }
        CK(gather_rotate(3, z, ctx->sumN * 3, sh.col_body, sh.col_rhs, ctx->src_off_d, ctx->rot64_d, ncols, sd.dN,
                         sh.A, nullptr, st));
        const int S1 = gemm_splitk_chunks(ncols, sd.r, sd.dN, ctx->sm_count);
        const int S2 = gemm_splitk_chunks(ncols, sd.dM, sd.r, ctx->sm_count);
        CK(gemm_splitk(ncols, sd.r, sd.dN, S1, sh.A, project ? sd.Wp : sd.Wr, sh.PkT, sh.Tm, nullptr, st, true));
        CK(gemm_splitk(ncols, sd.dM, sd.r, S2, sh.Tm, sd.U, sh.PkT, nullptr, sh.O64, st, true));
        CK(scatter_rotate(3, nullptr, sh.O64, sh.col_body, sh.col_rhs, ctx->tgt_off_d, ctx->rot_d, ctx->rot64_d,
                          ncols, sd.dM, ctx->sumM, out, st));
        ctx->launches += 6;
    }
    return MFS_OK;
}

// y = A^T w = w + [((I - L^(k')) S_L^(k')+)^T sum_{k != k'} S^(kk')^T w^(k)]_k'
mfs_status matvec_T_dev(mfs_ctx *ctx, const double *w, double *y, int nrhs, cudaStream_t st) {
    CKS(pair_apply_T(ctx, w, ctx->lam_d, nrhs, 0, st));
    CKS(precondT_dev(ctx, ctx->lam_d, ctx->tmpM_d, 1, nrhs, st));
    const size_t n = (size_t)nrhs * ctx->sumM * 3;
    combine_raw_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ctx->tmpM_d, w, 1.0, 1.0, y, n);
    CK(cudaGetLastError());
    ctx->launches += 1;
    return MFS_OK;
}

struct SolveStats {
    int iters = 0, converged = 1, matvecs = 0, breakdown = 0;
    double resid = 0.0;
};

// One GMRES iteration's matvec: w = A vin (or A^T vin).
mfs_status iteration_matvec(mfs_ctx *ctx, const double *vin, int nrhs, bool transposed, cudaStream_t st) {
    if (transposed) return matvec_T_dev(ctx, vin, ctx->w_d, nrhs, st);
    return matvec_dev(ctx, vin, ctx->w_d, nrhs, st);
}

// The loop of iterations j >= 1 as a CUDA graph: a while node whose body loads v_j, applies the
// matvec, orthogonalises (Arnoldi, Givens) and advances j, clearing the node's condition when every
// lane stopped or the basis is full (at most m - 1 passes).  Built on first use (the first iteration
// ran on the host loop, so every plan and tensor map the body needs exists) and kept per key.
mfs_status solve_graph(mfs_ctx *ctx, int nrhs, bool transposed, mfs_ctx::SolveGraph **out) {
    const int key = nrhs * 4 + ctx->fset * 2 + (transposed ? 1 : 0);
    auto it = ctx->graphs.find(key);
    if (it != ctx->graphs.end()) {
        *out = &it->second;
        return MFS_OK;
    }
    if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    cudaStream_t st = ctx->cap_stream;  // records the body; nothing executes on it
    mfs_ctx::SolveGraph g;
    GmresDev &gd = ctx->gd;
    CK(cudaGraphCreate(&g.graph, 0));
    auto fail = [&](cudaError_t e) {
        cudaGetLastError();
        if (g.graph) cudaGraphDestroy(g.graph);
        ctx->last_error = std::string("CUDA graph of the GMRES loop: ") + cudaGetErrorString(e);
        return MFS_ERR_CUDA;
    };
    cudaGraphConditionalHandle cond;
    cudaError_t e = cudaGraphConditionalHandleCreate(&cond, g.graph, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return fail(e);
    // the parameter union has no default constructor: zeroed storage, then the conditional member
    alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
    std::memset(cp_raw, 0, sizeof(cp_raw));
    cudaGraphNodeParams &cp = *reinterpret_cast<cudaGraphNodeParams *>(cp_raw);
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, g.graph, nullptr, nullptr, 0, &cp);
    if (e != cudaSuccess) return fail(e);
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    const int l0 = ctx->launches, p0 = ctx->pair_launches;
    e = cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return fail(e);
    mfs_status ms = MFS_OK;
    cudaError_t ce = gmres_load_vj(gd, ctx->vin_d, st);
    if (ce == cudaSuccess) ms = iteration_matvec(ctx, ctx->vin_d, nrhs, transposed, st);
    if (ce == cudaSuccess && ms == MFS_OK) ce = gmres_arnoldi(gd, ctx->w_d, st);
    if (ce == cudaSuccess && ms == MFS_OK) ce = gmres_advance(gd, cond, 1, st);
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(st, &captured);
    g.launches = ctx->launches - l0 + 11;
    g.pair_launches = ctx->pair_launches - p0;
    ctx->launches = l0;
    ctx->pair_launches = p0;
    if (ms != MFS_OK) {
        cudaGraphDestroy(g.graph);
        return ms;
    }
    if (ce != cudaSuccess) return fail(ce);
    if (e != cudaSuccess) return fail(e);
    e = cudaGraphInstantiate(&g.exec, g.graph, 0);
    if (e != cudaSuccess) return fail(e);
    it = ctx->graphs.emplace(key, g).first;
    *out = &it->second;
    return MFS_OK;
}

// Solve A x = b (or A^T x = b) with b = ctx->b_d for all lanes; x in ctx->x_d.
mfs_status gmres_solve(mfs_ctx *ctx, int nrhs, cudaStream_t st, SolveStats &stats, bool transposed = false) {
    GmresDev &gd = ctx->gd;
    CK(gmres_init(gd, ctx->b_d, st));
    ctx->launches += 6;
    const bool use_graph = ctx->opt.graphs && !ctx->opt.profile;
    for (int j = 0; j < gd.m; ++j) {
        CKS(iteration_matvec(ctx, gd.V + (size_t)j * gd.n, nrhs, transposed, st));
        CK(gmres_arnoldi(gd, ctx->w_d, st));
        CK(gmres_advance(gd, cudaGraphConditionalHandle(), 0, st));
        ctx->launches += 10;
        CK(cudaMemcpyAsync(ctx->done_h, gd.done, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        stats.matvecs = j + 1;
        if (*ctx->done_h || j + 1 >= gd.m) break;
        if (use_graph) {  // the remaining iterations as one graph launch
            mfs_ctx::SolveGraph *g = nullptr;
            CKS(solve_graph(ctx, nrhs, transposed, &g));
            CK(cudaGraphLaunch(g->exec, st));
            int jend = 0;
            CK(cudaMemcpyAsync(&jend, gd.jcur, sizeof(int), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            const int extra = jend - j;  // iterations the graph ran (j advanced from j + 1 to jend)
            ctx->launches += extra * g->launches;
            ctx->pair_launches += extra * g->pair_launches;
            stats.matvecs = jend + 1;
            break;
        }
    }
    CK(gmres_solution(gd, ctx->x_d, ctx->ysmall_d, st));
    ctx->launches += 2;
    std::vector<int> it(gd.L), status(gd.L), active(gd.L);
    std::vector<double> res(gd.L);
    CK(cudaMemcpyAsync(it.data(), gd.iters, sizeof(int) * gd.L, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(status.data(), gd.status, sizeof(int) * gd.L, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(res.data(), gd.resid, sizeof(double) * gd.L, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int l = 0; l < gd.L; ++l) {
        stats.iters = std::max(stats.iters, it[l]);
        stats.resid = std::max(stats.resid, res[l]);
        if (status[l] == 2) stats.breakdown = 1;
        if (!(res[l] <= gd.tol)) stats.converged = 0;
    }
    CKS(check_device_error(ctx, st));
    return MFS_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void mfs_default_options(mfs_options *opt) {
    if (!opt) return;
    opt->mu = 1.0;
    opt->gmres_tol = 1e-7;
    opt->max_iter = 200;
    opt->restart = 200;
    opt->eps_trunc = 0.0;
    opt->precision = 0;
    opt->autotune = 1;
    opt->max_rhs = 4;
    opt->profile = 0;
    opt->tensor_cores = 1;
    opt->pair_variant = -1;
    opt->graphs = 1;
    opt->farfield = 0;
    opt->farfield_separation = 3.0;
}

int32_t mfs_abi_version(void) { return MFS_ABI_VERSION; }

const char *mfs_pair_variant_info(int32_t index, int32_t *d, int32_t *nrhs, int32_t *grad) {
    int count = 0;
    const PairVariant *vv = pair_variants(&count);
    if (index < 0 || index >= count) return nullptr;
    if (d) *d = vv[index].D;
    if (nrhs) *nrhs = vv[index].nrhs;
    if (grad) *grad = vv[index].grad;
    return vv[index].name;
}

const char *mfs_pair_variant(const mfs_ctx *ctx, int32_t nrhs) {
    if (!ctx || nrhs < 1 || nrhs > 4 || nrhs > ctx->opt.max_rhs) return "";
    const int v = forward_variant(ctx, nrhs);
    int count = 0;
    const PairVariant *vv = pair_variants(&count);
    return (v >= 0 && v < count) ? vv[v].name : "";
}

const char *mfs_last_error(const mfs_ctx *ctx) { return ctx ? ctx->last_error.c_str() : ""; }

const char *mfs_setup_error(void) { return g_setup_error.c_str(); }

void mfs_destroy(mfs_ctx *ctx) { delete ctx; }

}  // extern "C"

// One formulation's one-body factors for shape s: the block (S_L, or the bare S^(00) when set = 1),
// its thin SVD in FP64 (cuSOLVER gesvd, Eq. pseudo), the FP32 / FP64 apply factors and, for the
// tensor cores, their TF32 pieces and tensor maps.
static mfs_status build_shape_factors(mfs_ctx *ctx, cusolverDnHandle_t solver, int s, int set, cudaStream_t st) {
    ShapeHost &sh = ctx->shapes[s];
    FactorSet &fx = sh.fs[set];
    ShapeDev &sd = fx.dev;
    const int D = ctx->D, kind = ctx->kind;
    sd.M = sh.M;
    sd.N = sh.N;
    sd.dM = D * sh.M;
    sd.dN = D * sh.N;
    sd.r = sd.dN;
    const int m = sd.dM, n = sd.dN;
    double *X0 = nullptr, *Y0 = nullptr, *G0i = nullptr, *SL = nullptr, *Ucm = nullptr, *sig = nullptr, *VT = nullptr,
           *work = nullptr;
    int *info_d = nullptr;
    auto cleanup = [&]() {
        cudaFree(X0); cudaFree(Y0); cudaFree(G0i); cudaFree(SL); cudaFree(Ucm); cudaFree(sig); cudaFree(VT);
        cudaFree(work); cudaFree(info_d);
    };
    auto fail = [&](const std::string &msg, mfs_status code) {
        cleanup();
        cudaGetLastError();
        ctx->last_error = msg;
        return code;
    };
    if (cudaMalloc(&X0, sizeof(double) * 3 * sh.M) != cudaSuccess ||
        cudaMalloc(&Y0, sizeof(double) * 3 * sh.N) != cudaSuccess ||
        cudaMalloc(&G0i, sizeof(double) * 36) != cudaSuccess ||
        cudaMalloc(&SL, sizeof(double) * (size_t)m * n) != cudaSuccess ||
        cudaMalloc(&Ucm, sizeof(double) * (size_t)m * n) != cudaSuccess ||
        cudaMalloc(&sig, sizeof(double) * n) != cudaSuccess ||
        cudaMalloc(&VT, sizeof(double) * (size_t)n * n) != cudaSuccess ||
        cudaMalloc(&info_d, sizeof(int)) != cudaSuccess)
        return fail("device allocation for the one-body SVD failed", MFS_ERR_OOM);
    cudaMemcpy(X0, sh.X0.data(), sizeof(double) * 3 * sh.M, cudaMemcpyHostToDevice);
    cudaMemcpy(Y0, sh.Y0.data(), sizeof(double) * 3 * sh.N, cudaMemcpyHostToDevice);
    cudaMemcpy(G0i, sh.G0inv, sizeof(double) * 36, cudaMemcpyHostToDevice);
    cudaError_t ce = build_SL(kind, sh.M, sh.N, X0, Y0, ctx->opt.mu, G0i, set, SL, st);
    int lwork = 0;
    if (ce == cudaSuccess && cusolverDnDgesvd_bufferSize(solver, m, n, &lwork) != CUSOLVER_STATUS_SUCCESS)
        ce = cudaErrorUnknown;
    if (ce == cudaSuccess) ce = cudaMalloc(&work, sizeof(double) * std::max(lwork, 1));
    if (ce == cudaSuccess) {
        signed char jobu = 'S', jobvt = 'S';
        cusolverStatus_t cs =
            cusolverDnDgesvd(solver, jobu, jobvt, m, n, SL, m, sig, Ucm, m, VT, n, work, lwork, nullptr, info_d);
        if (cs != CUSOLVER_STATUS_SUCCESS) ce = cudaErrorUnknown;
    }
    int info_h = 0;
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&info_h, info_d, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess || info_h != 0)
        return fail(std::string("one-body SVD failed: ") + (ce != cudaSuccess ? cudaGetErrorString(ce) : "gesvd info != 0"),
                    MFS_ERR_CUDA);
    // apply factors
    const bool want_tc = ctx->opt.tensor_cores != 0 && ctx->opt.precision == 0;
    bool ok = ctx->alloc(&sd.U, (size_t)m * n) == cudaSuccess && ctx->alloc(&sd.Wp, (size_t)n * n) == cudaSuccess &&
              ctx->alloc(&sd.Wr, (size_t)n * n) == cudaSuccess;
    if (ok && (ctx->opt.precision >= 1 || want_tc))  // the tensor-core pieces are cut from FP64 factors
        ok = ctx->alloc(&sd.U64, (size_t)m * n) == cudaSuccess && ctx->alloc(&sd.Wp64, (size_t)n * n) == cudaSuccess &&
             ctx->alloc(&sd.Wr64, (size_t)n * n) == cudaSuccess;
    if (!ok) return fail("device allocation for the apply factors failed", MFS_ERR_OOM);
    ce = build_apply_factors(kind, sh.M, sh.N, Ucm, sig, VT, Y0, G0i, ctx->opt.eps_trunc, set, sd, st);
    cleanup();
    if (ce != cudaSuccess) {
        ctx->last_error = std::string("apply factors: ") + cudaGetErrorString(ce);
        return MFS_ERR_CUDA;
    }
    if (!(sd.sigma1 > 0.0) || !std::isfinite(sd.sigma1)) {
        ctx->last_error = "one-body SVD returned a non-finite or zero largest singular value";
        return MFS_ERR_ILL_CONDITIONED;
    }
    if (want_tc) {
        // K-major FP32 (hi, lo) planes: U^T [r][ld1], Wp^T and Wr^T [dN][ld2], from the FP64 factors; zero
        // K padding.  The kernel cuts them into TF32 pieces in shared memory.
        sh.pieces = ctx->opt.tensor_cores == 2 ? 2 : 3;
        sh.ld1 = (m + 31) / 32 * 32;
        sh.ld2 = (n + 31) / 32 * 32;
        fx.ut_stride = (size_t)n * sh.ld1;
        fx.wt_stride = (size_t)n * sh.ld2;
        ok = ctx->alloc(&fx.Utp, 2 * fx.ut_stride) == cudaSuccess &&
             ctx->alloc(&fx.Wptp, 2 * fx.wt_stride) == cudaSuccess &&
             ctx->alloc(&fx.Wrtp, 2 * fx.wt_stride) == cudaSuccess;
        if (!ok) {
            ctx->last_error = "device allocation for the tensor-core factors failed";
            return MFS_ERR_OOM;
        }
        CK(split_hilo_transpose(sd.U64, m, n, fx.Utp, sh.ld1, fx.ut_stride, st));
        CK(split_hilo_transpose(sd.Wp64, n, n, fx.Wptp, sh.ld2, fx.wt_stride, st));
        CK(split_hilo_transpose(sd.Wr64, n, n, fx.Wrtp, sh.ld2, fx.wt_stride, st));
        CK(cudaStreamSynchronize(st));
        const int box = 128;  // factor rows per CTA (MMA M)
        bool enc = true;
        for (int p = 0; p < 2; ++p)
            enc = enc && make_tc_map(fx.mU[p], fx.Utp + p * fx.ut_stride, n, sh.ld1, box) &&
                  make_tc_map(fx.mWp[p], fx.Wptp + p * fx.wt_stride, n, sh.ld2, box) &&
                  make_tc_map(fx.mWr[p], fx.Wrtp + p * fx.wt_stride, n, sh.ld2, box);
        if (!enc) {
            ctx->last_error = "tensor-map encoding for the tensor-core apply failed";
            return MFS_ERR_CUDA;
        }
        fx.tc_ready = true;
        if (ctx->opt.precision == 0) {  // the FP64 factors were only the source of the pieces
            ctx->release(sd.U64);
            ctx->release(sd.Wp64);
            ctx->release(sd.Wr64);
            sd.U64 = sd.Wp64 = sd.Wr64 = nullptr;
        }
    }
    fx.built = true;
    return MFS_OK;
}

// Column lists and GEMM scratch of one shape's one-body apply (shared by the formulations).
static mfs_status alloc_apply_scratch(mfs_ctx *ctx, ShapeHost &sh, cudaStream_t st) {
    const int R = ctx->opt.max_rhs;
    const int m = sh.fs[0].dev.dM, n = sh.fs[0].dev.dN;
    const int nb = (int)sh.bodies.size();
    if (nb == 0) return MFS_OK;
    std::vector<int> cb(R * nb), cr(R * nb);
    for (int h = 0; h < R; ++h)
        for (int i = 0; i < nb; ++i) {
            cb[h * nb + i] = sh.bodies[i];
            cr[h * nb + i] = h;
        }
    bool ok = ctx->alloc(&sh.col_body, R * nb) == cudaSuccess && ctx->alloc(&sh.col_rhs, R * nb) == cudaSuccess &&
              ctx->alloc(&sh.A, (size_t)R * nb * m) == cudaSuccess &&
              ctx->alloc(&sh.Tm, (size_t)R * nb * n) == cudaSuccess &&
              ctx->alloc(&sh.Lm, (size_t)R * nb * n) == cudaSuccess;
    if (ok && ctx->opt.precision >= 1)
        ok = ctx->alloc(&sh.A64, (size_t)R * nb * m) == cudaSuccess &&
             ctx->alloc(&sh.T64, (size_t)R * nb * n) == cudaSuccess;
    if (ok) ok = ctx->alloc(&sh.L64, (size_t)R * nb * n) == cudaSuccess;
    if (ok) {  // split-K chunk results: the largest S * rows * cols over nrhs = 1..R and both GEMMs
        size_t need = 0;
        for (int h = 1; h <= R; ++h) {
            const int rows = h * nb;
            need = std::max(need, (size_t)gemm_splitk_chunks(rows, n, m, ctx->sm_count) * rows * n);
            need = std::max(need, (size_t)gemm_splitk_chunks(rows, n, n, ctx->sm_count) * rows * n);
        }
        sh.Pk_count = need;
        ok = ctx->alloc(&sh.Pk, need) == cudaSuccess;
    }
    if (ok && sh.pieces > 0) {  // tensor cores: column pieces and chunk results
        const int np = sh.pieces;
        const size_t cap = (size_t)R * nb;
        sh.ap_stride = cap * sh.ld1;
        sh.tp_stride = cap * sh.ld2;
        size_t need = 0;
        for (int h = 1; h <= R; ++h) {
            const int cols = h * nb;
            need = std::max(need, (size_t)tc_gemm_sz(m, tc_gemm_chunks(cols, n, m, ctx->sm_count, np)) * cols * n);
            need = std::max(need, (size_t)tc_gemm_sz(n, tc_gemm_chunks(cols, n, n, ctx->sm_count, np)) * cols * n);
        }
        ok = ctx->alloc(&sh.Ap, np * sh.ap_stride) == cudaSuccess &&
             ctx->alloc(&sh.Tp, np * sh.tp_stride) == cudaSuccess && ctx->alloc(&sh.Ptc, need) == cudaSuccess;
        // the padding columns of the column pieces stay zero: the kernels write only the first dM / r
        if (ok)
            ok = cudaMemsetAsync(sh.Ap, 0, sizeof(float) * np * sh.ap_stride, st) == cudaSuccess &&
                 cudaMemsetAsync(sh.Tp, 0, sizeof(float) * np * sh.tp_stride, st) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        ctx->last_error = "device allocation for the preconditioner buffers failed";
        return MFS_ERR_OOM;
    }
    CK(cudaMemcpy(sh.col_body, cb.data(), sizeof(int) * cb.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(sh.col_rhs, cr.data(), sizeof(int) * cr.size(), cudaMemcpyHostToDevice));
    return MFS_OK;
}

// The Dirichlet formulation's factors (bare self blocks), built on the first capacitance or
// resistance solve: one more SVD per shape.
static mfs_status ensure_dirichlet(mfs_ctx *ctx, cudaStream_t st) {
    bool all = true;
    for (auto &sh : ctx->shapes) all = all && sh.fs[1].built;
    if (all) return MFS_OK;
    cusolverDnHandle_t solver = nullptr;
    if (cusolverDnCreate(&solver) != CUSOLVER_STATUS_SUCCESS) {
        ctx->last_error = "cusolverDnCreate failed";
        return MFS_ERR_CUDA;
    }
    cusolverDnSetStream(solver, st);
    mfs_status status = MFS_OK;
    for (int s = 0; s < (int)ctx->shapes.size() && status == MFS_OK; ++s)
        if (!ctx->shapes[s].fs[1].built) status = build_shape_factors(ctx, solver, s, 1, st);
    cusolverDnDestroy(solver);
    return status;
}

// n points of the Fibonacci lattice on the unit sphere (z_i = 1 - (2i+1)/n, golden-angle longitudes).
static void unit_fibonacci(int n, std::vector<double> &p) {
    const double ga = 2.0 * MFS_PI / (((1.0 + std::sqrt(5.0)) / 2.0) * ((1.0 + std::sqrt(5.0)) / 2.0));
    p.resize(3 * (size_t)n);
    for (int i = 0; i < n; ++i) {
        const double z = 1.0 - (2.0 * i + 1.0) / n, rho = std::sqrt(std::max(0.0, 1.0 - z * z));
        p[3 * i] = rho * std::cos(ga * i);
        p[3 * i + 1] = rho * std::sin(ga * i);
        p[3 * i + 2] = z;
    }
}

// The transposed pseudo-inverse of the check <- equivalent map on the unit sphere (raw kernel: 1/r or
// (I + r r^T / r^2) / r), FP64, truncated at 1e-12 of the largest singular value; least squares
// (FF_NC > FF_NE).  It depends on the kernel only, so a context computes it once.
static mfs_status ff_unit_pinv(mfs_ctx *ctx, mfs_ctx::FarField &F, const std::vector<double> &ue,
                               const std::vector<double> &uc, cudaStream_t st) {
    const int D = ctx->D;
    const int m = D * FF_NC, n = D * FF_NE;
    std::vector<double> A((size_t)m * n);
    for (int i = 0; i < FF_NC; ++i)
        for (int j = 0; j < FF_NE; ++j) {
            double r[3], r2 = 0.0;
            for (int a = 0; a < 3; ++a) {
                r[a] = FF_CHECK * uc[3 * i + a] - ue[3 * j + a];
                r2 += r[a] * r[a];
            }
            const double ri = 1.0 / std::sqrt(r2);
            for (int a = 0; a < D; ++a)
                for (int b = 0; b < D; ++b) {
                    const double v = D == 1 ? ri : ((a == b ? ri : 0.0) + r[a] * r[b] * ri * ri * ri);
                    A[(size_t)(D * j + b) * m + (D * i + a)] = v;
                }
        }
    cusolverDnHandle_t solver = nullptr;
    if (cusolverDnCreate(&solver) != CUSOLVER_STATUS_SUCCESS) {
        ctx->last_error = "cusolverDnCreate failed";
        return MFS_ERR_CUDA;
    }
    cusolverDnSetStream(solver, st);
    double *A_d = nullptr, *U_d = nullptr, *S_d = nullptr, *VT_d = nullptr, *work = nullptr;
    int *info_d = nullptr, lwork = 0, info_h = 0;
    bool ok = cudaMalloc(&A_d, sizeof(double) * A.size()) == cudaSuccess &&
              cudaMalloc(&U_d, sizeof(double) * (size_t)m * n) == cudaSuccess &&
              cudaMalloc(&S_d, sizeof(double) * n) == cudaSuccess &&
              cudaMalloc(&VT_d, sizeof(double) * (size_t)n * n) == cudaSuccess &&
              cudaMalloc(&info_d, sizeof(int)) == cudaSuccess &&
              cudaMemcpy(A_d, A.data(), sizeof(double) * A.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
              cusolverDnDgesvd_bufferSize(solver, m, n, &lwork) == CUSOLVER_STATUS_SUCCESS &&
              cudaMalloc(&work, sizeof(double) * std::max(lwork, 1)) == cudaSuccess;
    signed char jobu = 'S', jobvt = 'S';
    ok = ok && cusolverDnDgesvd(solver, jobu, jobvt, m, n, A_d, m, S_d, U_d, m, VT_d, n, work, lwork, nullptr,
                                info_d) == CUSOLVER_STATUS_SUCCESS;
    std::vector<double> U((size_t)m * n), S(n), VT((size_t)n * n);
    ok = ok && cudaMemcpy(&info_h, info_d, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && info_h == 0 &&
         cudaMemcpy(U.data(), U_d, sizeof(double) * U.size(), cudaMemcpyDeviceToHost) == cudaSuccess &&
         cudaMemcpy(S.data(), S_d, sizeof(double) * n, cudaMemcpyDeviceToHost) == cudaSuccess &&
         cudaMemcpy(VT.data(), VT_d, sizeof(double) * VT.size(), cudaMemcpyDeviceToHost) == cudaSuccess;
    cudaFree(A_d); cudaFree(U_d); cudaFree(S_d); cudaFree(VT_d); cudaFree(work); cudaFree(info_d);
    cusolverDnDestroy(solver);
    if (!ok || !(S[0] > 0.0)) {
        cudaGetLastError();
        ctx->last_error = "far field: SVD of the check <- equivalent map failed";
        return MFS_ERR_CUDA;
    }
    // PinvT[i][j] = sum_k U[i][k] / s_k VT[k][j] (row-major m x n) over the kept singular values
    std::vector<double> PinvT((size_t)m * n, 0.0), row(n);
    for (int k = 0; k < n; ++k) {
        if (!(S[k] > 1e-12 * S[0])) continue;
        const double inv = 1.0 / S[k];
        for (int j = 0; j < n; ++j) row[j] = inv * VT[(size_t)j * n + k];
        for (int i = 0; i < m; ++i) {
            const double u = U[(size_t)k * m + i];
            double *o = &PinvT[(size_t)i * n];
            for (int j = 0; j < n; ++j) o[j] += u * row[j];
        }
    }
    CK(ctx->alloc(&F.PinvT, PinvT.size()));
    CK(cudaMemcpy(F.PinvT, PinvT.data(), sizeof(double) * PinvT.size(), cudaMemcpyHostToDevice));
    return MFS_OK;
}

// Frees the far-field structures that depend on the body centres (all but the pseudo-inverse) and
// drops the captured graphs that hold their addresses.
static void ff_release_geometry(mfs_ctx *ctx, mfs_ctx::FarField &F) {
    ctx->drop_graphs();
    for (auto &kv : F.plans) {
        auto &pl = kv.second;
        for (PairPlan *pp : {&pl.up, &pl.ev}) {
            ctx->release(pp->tiles);
            ctx->release(pp->partial);
            ctx->release(pp->direct);
        }
        ctx->release(pl.lst_seg_up);
        ctx->release(pl.lst_cum_up);
        ctx->release(pl.lst_seg_ev);
        ctx->release(pl.lst_cum_ev);
    }
    F.plans.clear();
    ctx->release(F.centres);
    ctx->release(F.re);
    ctx->release(F.eq_pos);
    ctx->release(F.eq_pt);
    ctx->release(F.chk_pos);
    ctx->release(F.tgt);
    ctx->release(F.tperm);
    ctx->release(F.seg_rec0);
    ctx->release(F.seg_rec1);
    ctx->release(F.rec);
    ctx->release(F.ucheck);
    ctx->release(F.mu);
    ctx->release(F.fit_chunks);
    F.centres = F.ucheck = F.mu = F.fit_chunks = F.re = nullptr;
    F.eq_pos = F.chk_pos = F.tgt = nullptr;
    F.eq_pt = F.tperm = F.seg_rec0 = F.seg_rec1 = nullptr;
    F.rec = nullptr;
    F.ready = false;
}

// The far-field structures (opt.farfield = 1): the tree, the FP64 pseudo-inverse of the map from
// equivalent strengths on the unit sphere to the field at the check points (ff_unit_pinv, once per
// context), and the tree-ordered geometry (again after every mfs_update_centers).
static mfs_status ff_setup(mfs_ctx *ctx, mfs_ctx::FarField &F, cudaStream_t st) {
    const int P = ctx->P, D = ctx->D;
    F.rsrc.assign(P, 0.0);
    F.rtgt.assign(P, 0.0);
    for (int k = 0; k < P; ++k) {
        const ShapeHost &sh = ctx->shapes[ctx->shape_id[k]];
        double rp = 0.0, rc = 0.0;  // radii of the proxy and collocation points about the centre
        for (int j = 0; j < sh.N; ++j)
            rp = std::max(rp, std::sqrt(sh.Y0[3 * j] * sh.Y0[3 * j] + sh.Y0[3 * j + 1] * sh.Y0[3 * j + 1] +
                                        sh.Y0[3 * j + 2] * sh.Y0[3 * j + 2]));
        for (int i = 0; i < sh.M; ++i)
            rc = std::max(rc, std::sqrt(sh.X0[3 * i] * sh.X0[3 * i] + sh.X0[3 * i + 1] * sh.X0[3 * i + 1] +
                                        sh.X0[3 * i + 2] * sh.X0[3 * i + 2]));
        F.rsrc[k] = F.src_colloc ? rc : rp;
        F.rtgt[k] = F.src_colloc ? rp : rc;
    }
    ff_build_tree(P, ctx->centres.data(), F.rsrc.data(), ctx->S, ctx->body_off.data(), F.tree);
    const int nodes = F.nodes = (int)F.tree.nodes.size();

    std::vector<double> ue, uc;
    unit_fibonacci(FF_NE, ue);
    unit_fibonacci(FF_NC, uc);
    if (!F.PinvT) {  // independent of the centres (kept across moves) and of the roles (shared)
        const auto &other = &F == &ctx->ff ? ctx->ffT : ctx->ff;
        if (other.PinvT) F.PinvT = other.PinvT;
        else CKS(ff_unit_pinv(ctx, F, ue, uc, st));
    }
    // tree-ordered geometry and segments: proxy segment q (tree position) = body order[q], node segment
    // P + node = its equivalent points
    std::vector<double> cen(3 * (size_t)(P + nodes)), re(nodes);
    for (int q = 0; q < P; ++q)
        for (int a = 0; a < 3; ++a) cen[3 * q + a] = ctx->centres[3 * F.tree.order[q] + a];
    for (int nd = 0; nd < nodes; ++nd) {
        for (int a = 0; a < 3; ++a) cen[3 * (P + nd) + a] = F.tree.nodes[nd].c[a];
        re[nd] = F.tree.nodes[nd].re;
    }
    std::vector<float4> eq((size_t)nodes * FF_NE), chk((size_t)nodes * FF_NC);
    std::vector<int> eq_pt((size_t)nodes * FF_NE);
    for (int nd = 0; nd < nodes; ++nd) {
        float w;
        const int id = P + nd;
        std::memcpy(&w, &id, sizeof(float));
        for (int e = 0; e < FF_NE; ++e) {
            eq[(size_t)nd * FF_NE + e] = make_float4((float)(re[nd] * ue[3 * e]), (float)(re[nd] * ue[3 * e + 1]),
                                                     (float)(re[nd] * ue[3 * e + 2]), 0.f);
            eq_pt[(size_t)nd * FF_NE + e] = nd * FF_NE + e;
        }
        for (int c = 0; c < FF_NC; ++c)
            chk[(size_t)nd * FF_NC + c] =
                make_float4((float)(FF_CHECK * re[nd] * uc[3 * c]), (float)(FF_CHECK * re[nd] * uc[3 * c + 1]),
                            (float)(FF_CHECK * re[nd] * uc[3 * c + 2]), w);
    }
    std::vector<float4> tpos(F.ntgt), tff(F.ntgt);
    CK(cudaMemcpy(tpos.data(), F.tgt_pos, sizeof(float4) * F.ntgt, cudaMemcpyDeviceToHost));
    std::vector<int> tperm(F.ntgt);
    int t = 0;
    for (int q = 0; q < P; ++q) {
        const int b = F.tree.order[q];
        float w;
        std::memcpy(&w, &q, sizeof(float));
        for (int i = (*F.tgt_off)[b]; i < (*F.tgt_off)[b + 1]; ++i, ++t) {
            tff[t] = make_float4(tpos[i].x, tpos[i].y, tpos[i].z, w);
            tperm[t] = i;
        }
    }
    F.seg_rec0_h.resize(P + nodes);
    F.seg_rec1_h.resize(P + nodes);
    for (int q = 0; q < P; ++q) {
        const int b = F.tree.order[q];
        F.seg_rec0_h[q] = (*F.rec_off)[b];
        F.seg_rec1_h[q] = (*F.rec_off)[b + 1];  // padded to a multiple of 4 (zero-strength padding records)
    }
    for (int nd = 0; nd < nodes; ++nd) {
        F.seg_rec0_h[P + nd] = F.nrec + nd * FF_NE;
        F.seg_rec1_h[P + nd] = F.nrec + (nd + 1) * FF_NE;
    }
    const int R = ctx->opt.max_rhs;
    F.rec_floats = std::max(pair_record_floats(D, R, 0), pair_record_floats(D, R, 1));  // plain or f32x2 policies
    CK(ctx->alloc(&F.centres, cen.size()));
    CK(ctx->alloc(&F.re, re.size()));
    CK(ctx->alloc(&F.eq_pos, eq.size()));
    CK(ctx->alloc(&F.eq_pt, eq_pt.size()));
    CK(ctx->alloc(&F.chk_pos, chk.size()));
    CK(ctx->alloc(&F.tgt, tff.size()));
    CK(ctx->alloc(&F.tperm, tperm.size()));
    CK(ctx->alloc(&F.seg_rec0, F.seg_rec0_h.size()));
    CK(ctx->alloc(&F.seg_rec1, F.seg_rec1_h.size()));
    CK(ctx->alloc(&F.rec, (size_t)(F.nrec + (size_t)nodes * FF_NE) * F.rec_floats));
    CK(ctx->alloc(&F.ucheck, (size_t)R * nodes * FF_NC * D));
    CK(ctx->alloc(&F.mu, (size_t)R * nodes * FF_NE * D));
    {
        size_t chunk_doubles = 1;
        for (int h = 1; h <= R; ++h) {
            const int S = gemm_rm64_chunks(h * nodes, D * FF_NE, D * FF_NC, ctx->sm_count);
            if (S > 1) chunk_doubles = std::max(chunk_doubles, (size_t)S * h * nodes * FF_NE * D);
        }
        CK(ctx->alloc(&F.fit_chunks, chunk_doubles));
    }
    CK(cudaMemcpy(F.centres, cen.data(), sizeof(double) * cen.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(F.re, re.data(), sizeof(double) * re.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(F.eq_pos, eq.data(), sizeof(float4) * eq.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(F.eq_pt, eq_pt.data(), sizeof(int) * eq_pt.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(F.chk_pos, chk.data(), sizeof(float4) * chk.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(F.tgt, tff.data(), sizeof(float4) * tff.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(F.tperm, tperm.data(), sizeof(int) * tperm.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(F.seg_rec0, F.seg_rec0_h.data(), sizeof(int) * F.seg_rec0_h.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(F.seg_rec1, F.seg_rec1_h.data(), sizeof(int) * F.seg_rec1_h.size(), cudaMemcpyHostToDevice));
    CK(cudaMemset(F.rec, 0, sizeof(float) * (size_t)(F.nrec + (size_t)nodes * FF_NE) * F.rec_floats));
    F.ready = true;
    return MFS_OK;
}

static mfs_status setup_impl(mfs_ctx *ctx, mfs_kind kind, const mfs_bodies *bodies, int32_t num_shapes,
                             const mfs_pointset *proxy, const mfs_pointset *colloc, cudaStream_t st) {
    auto t0 = std::chrono::steady_clock::now();
    ctx->kind = kind;
    ctx->D = kind == MFS_STOKES ? 3 : 1;
    const int P = bodies->num_bodies;
    ctx->P = P;
    ctx->nshapes = num_shapes;
    ctx->S = bodies->num_suspensions > 0 && bodies->body_offsets ? bodies->num_suspensions : 1;
    ctx->centres.assign(bodies->centers, bodies->centers + 3 * P);
    ctx->shape_id.resize(P);
    for (int k = 0; k < P; ++k) ctx->shape_id[k] = bodies->shape_id ? bodies->shape_id[k] : 0;
    if (bodies->body_offsets && bodies->num_suspensions > 0)
        ctx->body_off.assign(bodies->body_offsets, bodies->body_offsets + ctx->S + 1);
    else
        ctx->body_off = {0, P};
    // validation
    if (ctx->body_off.front() != 0 || ctx->body_off.back() != P) {
        ctx->last_error = "body_offsets must start at 0 and end at num_bodies";
        return MFS_ERR_INVALID_ARG;
    }
    for (int s = 0; s < ctx->S; ++s)
        if (ctx->body_off[s + 1] <= ctx->body_off[s]) {
            ctx->last_error = "every suspension needs at least one body";
            return MFS_ERR_INVALID_ARG;
        }
    for (int k = 0; k < P; ++k) {
        if (ctx->shape_id[k] < 0 || ctx->shape_id[k] >= num_shapes) {
            ctx->last_error = "shape_id out of range";
            return MFS_ERR_INVALID_ARG;
        }
        for (int c = 0; c < 3; ++c)
            if (!std::isfinite(ctx->centres[3 * k + c])) {
                ctx->last_error = "non-finite body centre";
                return MFS_ERR_INVALID_ARG;
            }
    }
    ctx->rot.resize(9 * P);
    for (int k = 0; k < P; ++k) {
        if (bodies->quats) {
            double q[4];
            double nq = 0.0;
            for (int c = 0; c < 4; ++c) {
                q[c] = bodies->quats[4 * k + c];
                nq += q[c] * q[c];
            }
            if (!(nq > 0.0) || !std::isfinite(nq)) {
                ctx->last_error = "quaternion must be non-zero and finite";
                return MFS_ERR_INVALID_ARG;
            }
            nq = std::sqrt(nq);
            for (int c = 0; c < 4; ++c) q[c] /= nq;
            quat_to_rot(q, &ctx->rot[9 * k]);
        } else {
            const double I[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
            std::memcpy(&ctx->rot[9 * k], I, sizeof(I));
        }
    }
    ctx->shapes.resize(num_shapes);
    for (int s = 0; s < num_shapes; ++s) {
        ShapeHost &sh = ctx->shapes[s];
        sh.M = colloc[s].n;
        sh.N = proxy[s].n;
        if (sh.N <= 0 || sh.M <= sh.N || !colloc[s].pts || !proxy[s].pts) {
            ctx->last_error = "each shape needs 0 < N < M points";
            return MFS_ERR_INVALID_ARG;
        }
        sh.X0.assign(colloc[s].pts, colloc[s].pts + 3 * sh.M);
        sh.Y0.assign(proxy[s].pts, proxy[s].pts + 3 * sh.N);
        for (double v : sh.X0)
            if (!std::isfinite(v)) { ctx->last_error = "non-finite collocation point"; return MFS_ERR_INVALID_ARG; }
        for (double v : sh.Y0)
            if (!std::isfinite(v)) { ctx->last_error = "non-finite proxy point"; return MFS_ERR_INVALID_ARG; }
        double G0[36];
        gram6(sh.Y0, G0);
        if (kind == MFS_STOKES) {
            if (!invert6(G0, sh.G0inv)) {
                ctx->last_error = "proxy points do not span rigid-body motions (singular K_N^T K_N)";
                return MFS_ERR_INVALID_ARG;
            }
        } else {
            std::memset(sh.G0inv, 0, sizeof(sh.G0inv));
        }
    }
    for (int k = 0; k < P; ++k) ctx->shapes[ctx->shape_id[k]].bodies.push_back(k);

    // offsets
    ctx->tgt_off.assign(P + 1, 0);
    ctx->src_off.assign(P + 1, 0);
    ctx->rec_off.assign(P + 1, 0);
    ctx->blk_off.assign(P + 1, 0);
    for (int k = 0; k < P; ++k) {
        const ShapeHost &sh = ctx->shapes[ctx->shape_id[k]];
        const int npad = (sh.N + 3) / 4 * 4;
        ctx->tgt_off[k + 1] = ctx->tgt_off[k] + sh.M;
        ctx->src_off[k + 1] = ctx->src_off[k] + sh.N;
        ctx->rec_off[k + 1] = ctx->rec_off[k] + npad;
        ctx->blk_off[k + 1] = ctx->blk_off[k] + (npad + MFS_BS - 1) / MFS_BS;
    }
    ctx->sumM = ctx->tgt_off[P];
    ctx->sumN = ctx->src_off[P];
    ctx->nrec = ctx->rec_off[P];
    ctx->tgt_body.resize(ctx->sumM);
    for (int k = 0; k < P; ++k)
        for (int i = ctx->tgt_off[k]; i < ctx->tgt_off[k + 1]; ++i) ctx->tgt_body[i] = k;

    // rotated body-local points
    std::vector<float4> tgt_pos(ctx->sumM), src_pos(ctx->sumN);
    std::vector<double> tgt64(3 * (size_t)ctx->sumM), src64(3 * (size_t)ctx->sumN), src4(4 * (size_t)ctx->sumN);
    std::vector<int> rec_pt(ctx->nrec, -1), susp_b(P), susp_e(P);
    for (int s = 0; s < ctx->S; ++s)
        for (int k = ctx->body_off[s]; k < ctx->body_off[s + 1]; ++k) {
            susp_b[k] = ctx->src_off[ctx->body_off[s]];
            susp_e[k] = ctx->src_off[ctx->body_off[s + 1]];
        }
    for (int k = 0; k < P; ++k) {
        const ShapeHost &sh = ctx->shapes[ctx->shape_id[k]];
        const double *R = &ctx->rot[9 * k];
        for (int i = 0; i < sh.M; ++i) {
            double x[3];
            for (int a = 0; a < 3; ++a)
                x[a] = R[3 * a] * sh.X0[3 * i] + R[3 * a + 1] * sh.X0[3 * i + 1] + R[3 * a + 2] * sh.X0[3 * i + 2];
            const int t = ctx->tgt_off[k] + i;
            float kb;
            std::memcpy(&kb, &k, sizeof(float));  // body id stored as int bits
            tgt_pos[t] = make_float4((float)x[0], (float)x[1], (float)x[2], kb);
            for (int a = 0; a < 3; ++a) tgt64[3 * (size_t)t + a] = x[a];
        }
        for (int j = 0; j < sh.N; ++j) {
            double y[3];
            for (int a = 0; a < 3; ++a)
                y[a] = R[3 * a] * sh.Y0[3 * j] + R[3 * a + 1] * sh.Y0[3 * j + 1] + R[3 * a + 2] * sh.Y0[3 * j + 2];
            const int q = ctx->src_off[k] + j;
            src_pos[q] = make_float4((float)y[0], (float)y[1], (float)y[2], 0.f);
            for (int a = 0; a < 3; ++a) {
                src64[3 * (size_t)q + a] = y[a];
                src4[4 * (size_t)q + a] = y[a];
            }
            src4[4 * (size_t)q + 3] = (double)k;
            rec_pt[ctx->rec_off[k] + j] = q;
        }
    }
    // padding records point at the body centre: rec_pt = -1 packs (0,0,0) with zero strength
    std::vector<float> rot32(9 * (size_t)P);
    for (size_t i = 0; i < rot32.size(); ++i) rot32[i] = (float)ctx->rot[i];

    CK(ctx->alloc(&ctx->centres_d, 3 * (size_t)P));
    CK(ctx->alloc(&ctx->rot64_d, 9 * (size_t)P));
    CK(ctx->alloc(&ctx->rot_d, 9 * (size_t)P));
    CK(ctx->alloc(&ctx->shape_id_d, P));
    CK(ctx->alloc(&ctx->tgt_pos_d, ctx->sumM));
    CK(ctx->alloc(&ctx->src_pos_d, ctx->sumN));
    CK(ctx->alloc(&ctx->tgt_local64_d, 3 * (size_t)ctx->sumM));
    CK(ctx->alloc(&ctx->src_local64_d, 3 * (size_t)ctx->sumN));
    CK(ctx->alloc(&ctx->src_local4_d, 4 * (size_t)ctx->sumN));
    CK(ctx->alloc(&ctx->tgt_body_d, ctx->sumM));
    CK(ctx->alloc(&ctx->rec_pt_d, ctx->nrec));
    CK(ctx->alloc(&ctx->rec_off_d, P + 1));
    CK(ctx->alloc(&ctx->blk_off_d, P + 1));
    CK(ctx->alloc(&ctx->tgt_off_d, P + 1));
    CK(ctx->alloc(&ctx->src_off_d, P + 1));
    CK(ctx->alloc(&ctx->susp_src_begin_d, P));
    CK(ctx->alloc(&ctx->susp_src_end_d, P));
    CK(ctx->alloc(&ctx->err_d, 1));
    CK(cudaMemset(ctx->err_d, 0, sizeof(int)));
    CK(cudaMemcpy(ctx->centres_d, ctx->centres.data(), sizeof(double) * 3 * P, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->rot64_d, ctx->rot.data(), sizeof(double) * 9 * P, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->rot_d, rot32.data(), sizeof(float) * 9 * P, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->shape_id_d, ctx->shape_id.data(), sizeof(int) * P, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->tgt_pos_d, tgt_pos.data(), sizeof(float4) * ctx->sumM, cudaMemcpyHostToDevice));
    if (ctx->opt.precision == 3) {  // compensated pair sums: x = hi + lo, hi on the 1/MFS_XGRID grid
        std::vector<float4> hi(ctx->sumM), lo(ctx->sumM);
        for (int t = 0; t < ctx->sumM; ++t) {
            float h[3], l[3];
            for (int a = 0; a < 3; ++a) {
                const double x = tgt64[3 * (size_t)t + a], xh = std::rint(x * MFS_XGRID) / MFS_XGRID;
                h[a] = (float)xh;
                l[a] = (float)(x - xh);
            }
            hi[t] = make_float4(h[0], h[1], h[2], 0.f);
            lo[t] = make_float4(l[0], l[1], l[2], 0.f);
        }
        CK(ctx->alloc(&ctx->tgt_hi_d, ctx->sumM));
        CK(ctx->alloc(&ctx->tgt_lo_d, ctx->sumM));
        CK(cudaMemcpy(ctx->tgt_hi_d, hi.data(), sizeof(float4) * ctx->sumM, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(ctx->tgt_lo_d, lo.data(), sizeof(float4) * ctx->sumM, cudaMemcpyHostToDevice));
    }
    CK(cudaMemcpy(ctx->src_pos_d, src_pos.data(), sizeof(float4) * ctx->sumN, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->tgt_local64_d, tgt64.data(), sizeof(double) * tgt64.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->src_local64_d, src64.data(), sizeof(double) * src64.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->src_local4_d, src4.data(), sizeof(double) * src4.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->tgt_body_d, ctx->tgt_body.data(), sizeof(int) * ctx->sumM, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->rec_pt_d, rec_pt.data(), sizeof(int) * ctx->nrec, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->rec_off_d, ctx->rec_off.data(), sizeof(int) * (P + 1), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->blk_off_d, ctx->blk_off.data(), sizeof(long long) * (P + 1), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->tgt_off_d, ctx->tgt_off.data(), sizeof(int) * (P + 1), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->src_off_d, ctx->src_off.data(), sizeof(int) * (P + 1), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->susp_src_begin_d, susp_b.data(), sizeof(int) * P, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->susp_src_end_d, susp_e.data(), sizeof(int) * P, cudaMemcpyHostToDevice));
    {
        std::vector<double> g0(36 * (size_t)num_shapes);
        for (int s = 0; s < num_shapes; ++s) std::memcpy(&g0[36 * s], ctx->shapes[s].G0inv, sizeof(double) * 36);
        CK(ctx->alloc(&ctx->G0inv_d, g0.size()));
        CK(cudaMemcpy(ctx->G0inv_d, g0.data(), sizeof(double) * g0.size(), cudaMemcpyHostToDevice));
    }

    // per-shape one-body factors: S_L and its SVD in FP64 (cuSOLVER), then the apply factors
    cusolverDnHandle_t solver = nullptr;
    if (cusolverDnCreate(&solver) != CUSOLVER_STATUS_SUCCESS) {
        ctx->last_error = "cusolverDnCreate failed";
        return MFS_ERR_CUDA;
    }
    cusolverDnSetStream(solver, st);
    const int D = ctx->D;
    const int R = ctx->opt.max_rhs;
    mfs_status status = MFS_OK;
    for (int s = 0; s < num_shapes && status == MFS_OK; ++s) status = build_shape_factors(ctx, solver, s, 0, st);
    for (int s = 0; s < num_shapes && status == MFS_OK; ++s) status = alloc_apply_scratch(ctx, ctx->shapes[s], st);
    cusolverDnDestroy(solver);
    if (status != MFS_OK) return status;

    // work buffers
    // every layout a forward pair-kernel entry of this kind may use: plain, f32x2 (Stokes and Laplace),
    // compensated
    const int recf = std::max({pair_record_floats(D, R, 0), pair_record_floats(D, R, 1),
                               ctx->opt.precision == 3 ? pair_record_floats(D, R, 2) : 0});
    ctx->rec_floats = recf;
    CK(ctx->alloc(&ctx->rec_d, (size_t)ctx->nrec * recf));
    CK(cudaMemset(ctx->rec_d, 0, sizeof(float) * (size_t)ctx->nrec * recf));
    CK(ctx->alloc(&ctx->lam_d, (size_t)R * ctx->sumN * D));
    if (ctx->opt.precision == 1) CK(ctx->alloc(&ctx->raw_d, (size_t)R * ctx->sumM * D));
    CK(cudaMallocHost(&ctx->done_h, sizeof(int)));
    CK(cudaEventCreate(&ctx->ev0));
    CK(cudaEventCreate(&ctx->ev1));
    CK(cudaEventCreate(&ctx->evp0));
    CK(cudaEventCreate(&ctx->evp1));
    if (ctx->opt.farfield) {  // forward sums: proxy sources, collocation targets
        auto &F = ctx->ff;
        F.src_colloc = false;
        F.src_pos = ctx->src_pos_d;
        F.rec_pt = ctx->rec_pt_d;
        F.nsrc = ctx->sumN;
        F.nrec = ctx->nrec;
        F.rec_off = &ctx->rec_off;
        F.tgt_pos = ctx->tgt_pos_d;
        F.tgt_off = &ctx->tgt_off;
        F.ntgt = ctx->sumM;
        CKS(ff_setup(ctx, F, st));
    }
    CK(cudaStreamSynchronize(st));
    ctx->ms_setup = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return MFS_OK;
}

// Time every pair-kernel variant for (D, nrhs) on the actual geometry and keep the fastest.
static mfs_status autotune(mfs_ctx *ctx, int nrhs, cudaStream_t st) {
    int count = 0;
    const PairVariant *v = pair_variants(&count);
    double best = 1e300;
    int best_i = -1;
    // zero strengths: the timing does not depend on the values
    CK(cudaMemsetAsync(ctx->lam_d, 0, sizeof(double) * (size_t)nrhs * ctx->sumN * ctx->D, st));
    // Large problems are timed on a sample: the targets of the first bodies of the first suspension
    // against all of its sources, about 4e10 pairs (tens of milliseconds, every SM busy), so that
    // trying every variant costs a fraction of one pair sum.
    const double sample_pairs = 4e10;
    bool sample = pair_count(ctx, 0) > 2.0 * sample_pairs;
    std::vector<int> toff_s;
    int nt_s = 0;
    if (sample) {
        const int B0 = ctx->body_off[0], B1 = ctx->body_off[1];
        const double ns = ctx->src_off[B1] - ctx->src_off[B0];
        int kb = B0;
        double acc = 0.0;
        while (kb < B1 && acc < sample_pairs) {
            acc += (double)(ctx->tgt_off[kb + 1] - ctx->tgt_off[kb]) * ns;
            ++kb;
        }
        toff_s.assign(ctx->tgt_off.begin(), ctx->tgt_off.end());
        for (int k = kb; k <= ctx->P; ++k) toff_s[k] = ctx->tgt_off[kb];
        nt_s = ctx->tgt_off[kb];
        sample = nt_s > 0;
    }
    for (int i = 0; i < count; ++i) {
        if (v[i].grad || v[i].D != ctx->D || v[i].nrhs != nrhs || v[i].comp != (ctx->opt.precision == 3)) continue;
        if (pair_occupancy(i) <= 0) continue;
        PairPlan local;
        PairPlan *plan = &local;
        if (sample)
            CKS(build_plan_for(ctx, i, 0, toff_s, ctx->tgt_body, ctx->blk_off, nt_s, local));
        else
            CKS(get_plan(ctx, i, 0, &plan));
        struct Release {
            mfs_ctx *c;
            PairPlan *p;
            ~Release() {
                if (p->tiles) release_plan(c, *p);
            }
        } release{ctx, &local};
        const PairWork w = work_of(*plan);
        if (w.total_units == 0) return MFS_OK;
        CK(pack_for(ctx, i, ctx->lam_d, nrhs, st));
        float ms_best = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            CK(cudaEventRecord(ctx->ev0, st));
            CK(pair_launch(i, geom_of(ctx), w, ctx->err_d, st));
            CK(cudaEventRecord(ctx->ev1, st));
            CK(cudaEventSynchronize(ctx->ev1));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
            if (rep > 0) ms_best = std::min(ms_best, ms);
        }
        if (ms_best < best) {
            best = ms_best;
            best_i = i;
        }
    }
    ctx->best_variant[ctx->D == 3][nrhs] = best_i;
    return check_device_error(ctx, st);
}

extern "C" {

mfs_status mfs_setup(mfs_ctx **out, mfs_kind kind, const mfs_bodies *bodies, int32_t num_shapes,
                     const mfs_pointset *proxy, const mfs_pointset *colloc, const mfs_options *opt, void *stream) {
    g_setup_error.clear();
    if (!out || !bodies || !proxy || !colloc || num_shapes <= 0 || bodies->num_bodies <= 0 || !bodies->centers ||
        (kind != MFS_LAPLACE && kind != MFS_STOKES)) {
        g_setup_error = "mfs_setup: invalid argument";
        return MFS_ERR_INVALID_ARG;
    }
    *out = nullptr;
    std::unique_ptr<mfs_ctx> ctx(new mfs_ctx());
    if (opt) ctx->opt = *opt; else mfs_default_options(&ctx->opt);
    if (ctx->opt.max_rhs < 1 || ctx->opt.max_rhs > 4 || ctx->opt.max_iter < 1 || ctx->opt.restart < 1 ||
        ctx->opt.restart > 1023 || !(ctx->opt.mu > 0.0) || !(ctx->opt.gmres_tol >= 0.0) ||
        ctx->opt.precision < 0 || ctx->opt.precision > 3 || !(ctx->opt.eps_trunc >= 0.0)) {
        g_setup_error = "mfs_setup: invalid options";
        return MFS_ERR_INVALID_ARG;
    }
    if (ctx->opt.farfield != 0 && (ctx->opt.farfield != 1 || (ctx->opt.precision != 0 && ctx->opt.precision != 2))) {
        g_setup_error = "mfs_setup: farfield must be 0 or 1, and 1 needs precision 0 or 2 (FP32 pair sums)";
        return MFS_ERR_INVALID_ARG;
    }
    if (ctx->opt.farfield == 1 && !(ctx->opt.farfield_separation >= FF_CHECK && ctx->opt.farfield_separation <= 10.0)) {
        g_setup_error = "mfs_setup: farfield_separation must lie in [2.5, 10]";
        return MFS_ERR_INVALID_ARG;
    }
    if (ctx->opt.max_iter > ctx->opt.restart) {
        g_setup_error = "mfs_setup: max_iter above restart is not supported (no restarted GMRES)";
        return MFS_ERR_INVALID_ARG;
    }
    if (ctx->opt.pair_variant >= 0) {  // a forced pair-kernel variant: a forward sum of this kind's d
        int count = 0;
        const PairVariant *vv = pair_variants(&count);
        const int pv = ctx->opt.pair_variant;
        if (pv >= count || vv[pv].grad || vv[pv].D != (kind == MFS_STOKES ? 3 : 1) ||
            vv[pv].nrhs > ctx->opt.max_rhs || vv[pv].comp != (ctx->opt.precision == 3)) {
            g_setup_error = "mfs_setup: pair_variant is not a forward pair-sum variant of this kind";
            return MFS_ERR_INVALID_ARG;
        }
        ctx->best_variant[kind == MFS_STOKES][vv[pv].nrhs] = pv;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        g_setup_error = "mfs_setup: no CUDA device";
        return MFS_ERR_CUDA;
    }
    cudaStream_t st = (cudaStream_t)stream;
    mfs_status s = setup_impl(ctx.get(), kind, bodies, num_shapes, proxy, colloc, st);
    if (s == MFS_OK && ctx->opt.autotune && ctx->opt.precision != 1 && ctx->best_variant[kind == MFS_STOKES][1] < 0) {
        // tune the single-rhs variant now; other nrhs on first use
        s = autotune(ctx.get(), 1, st);
    }
    if (s != MFS_OK) {
        g_setup_error = ctx->last_error;
        return s;
    }
    *out = ctx.release();
    return MFS_OK;
}

mfs_status mfs_update_centers(mfs_ctx *ctx, const double *centers, void *stream) {
    if (!ctx || !centers) return MFS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (is_device_ptr(centers)) {
        CK(cudaMemcpyAsync(ctx->centres.data(), centers, sizeof(double) * 3 * ctx->P, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    } else {
        std::memcpy(ctx->centres.data(), centers, sizeof(double) * 3 * ctx->P);
    }
    for (double v : ctx->centres)
        if (!std::isfinite(v)) {
            ctx->last_error = "non-finite body centre";
            return MFS_ERR_INVALID_ARG;
        }
    CK(cudaMemcpyAsync(ctx->centres_d, ctx->centres.data(), sizeof(double) * 3 * ctx->P, cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    for (auto *F : {&ctx->ff, &ctx->ffT}) {  // the treecodes' trees, node centres and lists follow the bodies
        if (!F->ready) continue;
        CK(cudaDeviceSynchronize());
        ff_release_geometry(ctx, *F);
        CKS(ff_setup(ctx, *F, st));
    }
    return MFS_OK;
}

mfs_status mfs_matvec(mfs_ctx *ctx, const double *gamma, double *y, int32_t nrhs, void *stream) {
    if (!ctx || !gamma || !y || nrhs < 1 || nrhs > ctx->opt.max_rhs) {
        if (ctx) ctx->last_error = "mfs_matvec: invalid argument";
        return MFS_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = (size_t)nrhs * ctx->sumM * ctx->D;
    Staged gi, yo;
    CKS(stage_in(ctx, gi, gamma, n, st));
    CKS(stage_out_alloc(ctx, yo, y, n));
    CKS(matvec_dev(ctx, gi.d, yo.d, nrhs, st));
    CKS(stage_out_finish(ctx, yo, st));
    return check_device_error(ctx, st);
}

mfs_status mfs_matvec_transposed(mfs_ctx *ctx, const double *w, double *y, int32_t nrhs, void *stream) {
    if (!ctx || !w || !y || nrhs < 1 || nrhs > ctx->opt.max_rhs) {
        if (ctx) ctx->last_error = "mfs_matvec_transposed: invalid argument";
        return MFS_ERR_INVALID_ARG;
    }
    if (ctx->kind != MFS_STOKES) {
        ctx->last_error = "mfs_matvec_transposed: Stokes contexts only";
        return MFS_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    CKS(ensure_transposed(ctx));
    const size_t n = (size_t)nrhs * ctx->sumM * 3;
    Staged wi, yo;
    CKS(stage_in(ctx, wi, w, n, st));
    CKS(stage_out_alloc(ctx, yo, y, n));
    CKS(matvec_T_dev(ctx, wi.d, yo.d, nrhs, st));
    CKS(stage_out_finish(ctx, yo, st));
    return check_device_error(ctx, st);
}

mfs_status mfs_precond_apply(mfs_ctx *ctx, const double *gamma, double *lambda, int32_t project, int32_t nrhs,
                             void *stream) {
    if (!ctx || !gamma || !lambda || nrhs < 1 || nrhs > ctx->opt.max_rhs) {
        if (ctx) ctx->last_error = "mfs_precond_apply: invalid argument";
        return MFS_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    Staged gi, lo;
    CKS(stage_in(ctx, gi, gamma, (size_t)nrhs * ctx->sumM * ctx->D, st));
    CKS(stage_out_alloc(ctx, lo, lambda, (size_t)nrhs * ctx->sumN * ctx->D));
    CKS(precond_apply_dev(ctx, gi.d, lo.d, project ? 1 : 0, nrhs, st));
    CKS(stage_out_finish(ctx, lo, st));
    return MFS_OK;
}

mfs_status mfs_pair_sum(mfs_ctx *ctx, const double *strengths, double *u, int32_t nrhs, int32_t include_self,
                        void *stream) {
    if (!ctx || !strengths || !u || nrhs < 1 || nrhs > ctx->opt.max_rhs) {
        if (ctx) ctx->last_error = "mfs_pair_sum: invalid argument";
        return MFS_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    Staged si, uo;
    CKS(stage_in(ctx, si, strengths, (size_t)nrhs * ctx->sumN * ctx->D, st));
    CKS(stage_out_alloc(ctx, uo, u, (size_t)nrhs * ctx->sumM * ctx->D));
    CKS(pair_apply(ctx, si.d, uo.d, nullptr, 0.0, 1.0, nrhs, include_self ? 1 : 0, st));
    CKS(stage_out_finish(ctx, uo, st));
    return check_device_error(ctx, st);
}

// Keep the GMRES solution gamma (ctx->x_d) and the inputs a (and b), n doubles each, of the solve
// just run (kind: 1 mobility, 2 elastance, 3 resistance, 4 capacitance).
static mfs_status keep_solution(mfs_ctx *ctx, int kind, int nrhs, const double *a, const double *b, size_t n,
                                cudaStream_t st) {
    if (!ctx->keep_gamma) {
        CK(ctx->alloc(&ctx->keep_gamma, (size_t)ctx->opt.max_rhs * ctx->sumM * ctx->D));
        CK(ctx->alloc(&ctx->keep_lam0, (size_t)ctx->opt.max_rhs * ctx->P * 6));
    }
    CK(cudaMemcpyAsync(ctx->keep_gamma, ctx->x_d, sizeof(double) * nrhs * ctx->sumM * ctx->D,
                       cudaMemcpyDeviceToDevice, st));
    if (a) CK(cudaMemcpyAsync(ctx->keep_lam0, a, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    if (b) CK(cudaMemcpyAsync(ctx->keep_lam0 + n, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    ctx->last_solve = kind;
    ctx->last_nrhs = nrhs;
    return MFS_OK;
}

static void begin_call(mfs_ctx *ctx) {
    ctx->launches = 0;
    ctx->pair_launches = 0;
    ctx->pair_ms_acc = 0.0;
}

static double pair_profile_ms(mfs_ctx *ctx) {
    if (!ctx->opt.profile) return 0.0;
    double total = 0.0;
    for (int i = 0; i < ctx->pair_launches && 2 * (size_t)i + 1 < ctx->pev.size(); ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ctx->pev[2 * i], ctx->pev[2 * i + 1]) == cudaSuccess) total += ms;
    }
    return total;
}

static mfs_status finish_info(mfs_ctx *ctx, mfs_solve_info *info, const SolveStats &ss, float ms, int nrhs,
                              bool rhs_pairs = true) {
    ctx->pair_ms_acc = pair_profile_ms(ctx);
    if (info) {
        info->launches = ctx->launches;
        info->pair_launches = ctx->pair_launches;
        info->iters = ss.iters;
        info->converged = ss.converged;
        info->matvecs = ss.matvecs;
        info->lanes = nrhs * ctx->S;
        info->rel_residual = ss.resid;
        info->ms_setup = ctx->ms_setup;
        info->ms_solve = ms;
        info->ms_pairs = ctx->pair_ms_acc;
        info->pairs = pair_count(ctx, 0) * ss.matvecs + (rhs_pairs ? pair_count(ctx, 1) : 0.0);
        info->pairs_evaluated = info->pairs;
        if (ctx->ff.ready) {  // what the treecode's launches evaluated for the same sums
            auto evaluated = [&](int include_self) {
                const auto it = ctx->ff.plans.find(forward_variant(ctx, nrhs) * 2 + include_self);
                return it == ctx->ff.plans.end() ? 0.0 : it->second.pairs_up + it->second.pairs_ev;
            };
            info->pairs_evaluated = evaluated(0) * ss.matvecs + (rhs_pairs ? evaluated(1) : 0.0);
        }
    }
    if (ss.breakdown) {
        ctx->last_error = "GMRES breakdown: non-finite residual";
        return MFS_ERR_BREAKDOWN;
    }
    if (!ss.converged) {
        ctx->last_error = "GMRES did not reach the tolerance within max_iter";
        return MFS_ERR_NOT_CONVERGED;
    }
    return MFS_OK;
}

mfs_status mfs_solve_mobility(mfs_ctx *ctx, const double *F, const double *T, double *U, double *Omega, int32_t nrhs,
                              mfs_solve_info *info, void *stream) {
    if (!ctx || !F || !T || !U || !Omega || nrhs < 1 || nrhs > ctx->opt.max_rhs) {
        if (ctx) ctx->last_error = "mfs_solve_mobility: invalid argument";
        return MFS_ERR_INVALID_ARG;
    }
    if (ctx->kind != MFS_STOKES) {
        ctx->last_error = "mfs_solve_mobility needs a Stokes context";
        return MFS_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nb = (size_t)nrhs * ctx->P * 3;
    Staged Fi, Ti, Uo, Oo;
    CKS(stage_in(ctx, Fi, F, nb, st));
    CKS(stage_in(ctx, Ti, T, nb, st));
    CKS(stage_out_alloc(ctx, Uo, U, nb));
    CKS(stage_out_alloc(ctx, Oo, Omega, nb));
    if (ctx->opt.autotune && ctx->opt.precision != 1 && ctx->best_variant[1][nrhs] < 0) CKS(autotune(ctx, nrhs, st));
    CKS(ensure_gmres(ctx, nrhs));
    begin_call(ctx);
    CK(cudaEventRecord(ctx->ev0, st));
    ctx->launches += 1;
    // lambda_0 and b = -u_0 (all pairs, Eq. stou0)
    CK(completion_stokes(Fi.d, Ti.d, nrhs, ctx->P, ctx->rot64_d, ctx->G0inv_d, ctx->shape_id_d, ctx->src_local64_d,
                         ctx->src_off_d, ctx->sumN, ctx->lam_d, st));
    CKS(pair_apply(ctx, ctx->lam_d, ctx->b_d, nullptr, 0.0, -1.0, nrhs, 1, st));
    SolveStats ss;
    CKS(gmres_solve(ctx, nrhs, st, ss));
    // lambda = S_L^+ gamma, [U; Omega] = -K_N^T lambda (Eq. getU)
    CKS(precond_apply_dev(ctx, ctx->x_d, ctx->lam_d, 0, nrhs, st));
    CK(extract_stokes(ctx->lam_d, nrhs, ctx->P, ctx->src_local64_d, ctx->src_off_d, ctx->sumN, Uo.d, Oo.d, st));
    ctx->launches += 1;
    CK(cudaEventRecord(ctx->ev1, st));
    // keep gamma, F and T for mfs_mobility_vjp and mfs_evaluate (outside the timed region)
    CKS(keep_solution(ctx, 1, nrhs, Fi.d, Ti.d, nb, st));
    CK(cudaEventSynchronize(ctx->ev1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    CKS(stage_out_finish(ctx, Uo, st));
    CKS(stage_out_finish(ctx, Oo, st));
    return finish_info(ctx, info, ss, ms, nrhs);
}

mfs_status mfs_solve_elastance(mfs_ctx *ctx, const double *Q, double *V, int32_t nrhs, mfs_solve_info *info,
                               void *stream) {
    if (!ctx || !Q || !V || nrhs < 1 || nrhs > ctx->opt.max_rhs) {
        if (ctx) ctx->last_error = "mfs_solve_elastance: invalid argument";
        return MFS_ERR_INVALID_ARG;
    }
    if (ctx->kind != MFS_LAPLACE) {
        ctx->last_error = "mfs_solve_elastance needs a Laplace context";
        return MFS_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nb = (size_t)nrhs * ctx->P;
    Staged Qi, Vo;
    CKS(stage_in(ctx, Qi, Q, nb, st));
    CKS(stage_out_alloc(ctx, Vo, V, nb));
    if (ctx->opt.autotune && ctx->opt.precision != 1 && ctx->best_variant[0][nrhs] < 0) CKS(autotune(ctx, nrhs, st));
    CKS(ensure_gmres(ctx, nrhs));
    begin_call(ctx);
    CK(cudaEventRecord(ctx->ev0, st));
    ctx->launches += 1;
    CK(completion_laplace(Qi.d, nrhs, ctx->P, ctx->src_off_d, ctx->sumN, ctx->lam_d, st));  // Eq. al0
    CKS(pair_apply(ctx, ctx->lam_d, ctx->b_d, nullptr, 0.0, -1.0, nrhs, 1, st));           // b = -u_0, Eq. erhsK
    SolveStats ss;
    CKS(gmres_solve(ctx, nrhs, st, ss));
    CKS(precond_apply_dev(ctx, ctx->x_d, ctx->lam_d, 0, nrhs, st));
    CK(extract_laplace(ctx->lam_d, nrhs, ctx->P, ctx->src_off_d, ctx->sumN, Vo.d, st));  // Eq. vkal
    ctx->launches += 1;
    CK(cudaEventRecord(ctx->ev1, st));
    CKS(keep_solution(ctx, 2, nrhs, Qi.d, nullptr, nb, st));
    CK(cudaEventSynchronize(ctx->ev1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    CKS(stage_out_finish(ctx, Vo, st));
    return finish_info(ctx, info, ss, ms, nrhs);
}

}  // extern "C"

namespace {
// Selects the Dirichlet factor set for the duration of one solve, on every return path.
struct DirichletScope {
    mfs_ctx *ctx;
    explicit DirichletScope(mfs_ctx *c) : ctx(c) { ctx->fset = 1; }
    ~DirichletScope() { ctx->fset = 0; }
};

// Algorithm 1 SOLVE with the Dirichlet data already in ctx->b_d: gamma by GMRES on Eq. 2sysprec, then
// the strengths alpha = S^+ gamma in ctx->lam_d.
mfs_status dirichlet_solve(mfs_ctx *ctx, int nrhs, cudaStream_t st, SolveStats &ss) {
    DirichletScope scope(ctx);
    CKS(gmres_solve(ctx, nrhs, st, ss));
    CKS(precond_apply_dev(ctx, ctx->x_d, ctx->lam_d, 0, nrhs, st));
    return MFS_OK;
}
}  // namespace

extern "C" {

mfs_status mfs_dirichlet_matvec(mfs_ctx *ctx, const double *gamma, double *y, int32_t nrhs, void *stream) {
    if (!ctx || !gamma || !y || nrhs < 1 || nrhs > ctx->opt.max_rhs) {
        if (ctx) ctx->last_error = "mfs_dirichlet_matvec: invalid argument";
        return MFS_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    CKS(ensure_dirichlet(ctx, st));
    Staged gi, yo;
    const size_t n = (size_t)nrhs * ctx->sumM * ctx->D;
    CKS(stage_in(ctx, gi, gamma, n, st));
    CKS(stage_out_alloc(ctx, yo, y, n));
    {
        DirichletScope scope(ctx);
        CKS(matvec_dev(ctx, gi.d, yo.d, nrhs, st));
    }
    CKS(stage_out_finish(ctx, yo, st));
    return check_device_error(ctx, st);
}

mfs_status mfs_dirichlet_apply(mfs_ctx *ctx, const double *gamma, double *alpha, int32_t nrhs, void *stream) {
    if (!ctx || !gamma || !alpha || nrhs < 1 || nrhs > ctx->opt.max_rhs) {
        if (ctx) ctx->last_error = "mfs_dirichlet_apply: invalid argument";
        return MFS_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    CKS(ensure_dirichlet(ctx, st));
    Staged gi, ao;
    CKS(stage_in(ctx, gi, gamma, (size_t)nrhs * ctx->sumM * ctx->D, st));
    CKS(stage_out_alloc(ctx, ao, alpha, (size_t)nrhs * ctx->sumN * ctx->D));
    {
        DirichletScope scope(ctx);
        CKS(precond_apply_dev(ctx, gi.d, ao.d, 0, nrhs, st));
    }
    CKS(stage_out_finish(ctx, ao, st));
    return check_device_error(ctx, st);
}

mfs_status mfs_solve_resistance(mfs_ctx *ctx, const double *U, const double *Omega, double *F, double *T,
                                int32_t nrhs, mfs_solve_info *info, void *stream) {
    if (!ctx || !U || !Omega || !F || !T || nrhs < 1 || nrhs > ctx->opt.max_rhs) {
        if (ctx) ctx->last_error = "mfs_solve_resistance: invalid argument";
        return MFS_ERR_INVALID_ARG;
    }
    if (ctx->kind != MFS_STOKES) {
        ctx->last_error = "mfs_solve_resistance needs a Stokes context";
        return MFS_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nb = (size_t)nrhs * ctx->P * 3;
    Staged Ui, Oi, Fo, To;
    CKS(stage_in(ctx, Ui, U, nb, st));
    CKS(stage_in(ctx, Oi, Omega, nb, st));
    CKS(stage_out_alloc(ctx, Fo, F, nb));
    CKS(stage_out_alloc(ctx, To, T, nb));
    CKS(ensure_dirichlet(ctx, st));
    if (ctx->opt.autotune && ctx->opt.precision != 1 && ctx->best_variant[1][nrhs] < 0) CKS(autotune(ctx, nrhs, st));
    CKS(ensure_gmres(ctx, nrhs));
    begin_call(ctx);
    CK(cudaEventRecord(ctx->ev0, st));
    // b = K_M U (Sec. 2.2), then Algorithm 1 and [f; t] = K_N^T lambda (Eq. force_def)
    CK(dirichlet_rhs_stokes(Ui.d, Oi.d, nrhs, ctx->P, ctx->tgt_local64_d, ctx->tgt_off_d, ctx->sumM, ctx->b_d, st));
    SolveStats ss;
    CKS(dirichlet_solve(ctx, nrhs, st, ss));
    CK(extract_stokes(ctx->lam_d, nrhs, ctx->P, ctx->src_local64_d, ctx->src_off_d, ctx->sumN, Fo.d, To.d, st, 1.0));
    ctx->launches += 2;
    CK(cudaEventRecord(ctx->ev1, st));
    CKS(keep_solution(ctx, 3, nrhs, nullptr, nullptr, 0, st));
    CK(cudaEventSynchronize(ctx->ev1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    CKS(stage_out_finish(ctx, Fo, st));
    CKS(stage_out_finish(ctx, To, st));
    return finish_info(ctx, info, ss, ms, nrhs, false);
}

mfs_status mfs_solve_capacitance(mfs_ctx *ctx, const double *phi, double *q, int32_t nrhs, mfs_solve_info *info,
                                 void *stream) {
    if (!ctx || !phi || !q || nrhs < 1 || nrhs > ctx->opt.max_rhs) {
        if (ctx) ctx->last_error = "mfs_solve_capacitance: invalid argument";
        return MFS_ERR_INVALID_ARG;
    }
    if (ctx->kind != MFS_LAPLACE) {
        ctx->last_error = "mfs_solve_capacitance needs a Laplace context";
        return MFS_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nb = (size_t)nrhs * ctx->P;
    Staged Pi, Qo;
    CKS(stage_in(ctx, Pi, phi, nb, st));
    CKS(stage_out_alloc(ctx, Qo, q, nb));
    CKS(ensure_dirichlet(ctx, st));
    if (ctx->opt.autotune && ctx->opt.precision != 1 && ctx->best_variant[0][nrhs] < 0) CKS(autotune(ctx, nrhs, st));
    CKS(ensure_gmres(ctx, nrhs));
    begin_call(ctx);
    CK(cudaEventRecord(ctx->ev0, st));
    // eta = phi 1_M (Sec. 2.1), then Algorithm 1 and q = sum alpha (Eq. qkgauss)
    CK(dirichlet_rhs_laplace(Pi.d, nrhs, ctx->P, ctx->tgt_off_d, ctx->sumM, ctx->b_d, st));
    SolveStats ss;
    CKS(dirichlet_solve(ctx, nrhs, st, ss));
    CK(extract_laplace(ctx->lam_d, nrhs, ctx->P, ctx->src_off_d, ctx->sumN, Qo.d, st, 1));
    ctx->launches += 2;
    CK(cudaEventRecord(ctx->ev1, st));
    CKS(keep_solution(ctx, 4, nrhs, nullptr, nullptr, 0, st));
    CK(cudaEventSynchronize(ctx->ev1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    CKS(stage_out_finish(ctx, Qo, st));
    return finish_info(ctx, info, ss, ms, nrhs, false);
}

}  // extern "C"

// FP64 -> FP32 (adjoint strengths for the gradient kernel)
static __global__ void to_f32_kernel(const double *x, float *y, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = (float)x[i];
}

// dL/dc_k = scale * (source-side sum of body k) - (sum over the targets of body k of their gradient sums)
static __global__ void centre_grad_kernel(const double *gradT, const int *tgt_off, const double *src_grad, double scale,
                                          double *dc) {
    const int k = blockIdx.x;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int i = tgt_off[k] + threadIdx.x; i < tgt_off[k + 1]; i += blockDim.x)
        for (int c = 0; c < 3; ++c) acc[c] += gradT[3 * (size_t)i + c];
    __shared__ double red[3][128];
    for (int c = 0; c < 3; ++c) red[c][threadIdx.x] = acc[c];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 3) dc[3 * k + threadIdx.x] = scale * src_grad[3 * k + threadIdx.x] - red[threadIdx.x][0];
}

// The centre gradient from the two treecode passes: dc_k = -(sum over body k's collocation points of gc)
// - (sum over its proxy points of gp), both already scaled.
static __global__ void centre_grad_ff_kernel(const double *gc, const int *tgt_off, const double *gp, const int *src_off,
                                             double *dc) {
    const int k = blockIdx.x;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int i = tgt_off[k] + threadIdx.x; i < tgt_off[k + 1]; i += blockDim.x)
        for (int c = 0; c < 3; ++c) acc[c] += gc[3 * (size_t)i + c];
    for (int j = src_off[k] + threadIdx.x; j < src_off[k + 1]; j += blockDim.x)
        for (int c = 0; c < 3; ++c) acc[c] += gp[3 * (size_t)j + c];
    __shared__ double red[3][128];
    for (int c = 0; c < 3; ++c) red[c][threadIdx.x] = acc[c];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 3) dc[3 * k + threadIdx.x] = -red[threadIdx.x][0];
}

// [dF; dT]_k = G_k^{-1} v_k with G_k = R_2 G_0 R_2^T (v = -K_N^T z, given as its force and torque parts)
static __global__ void gram_solve_kernel(const double *vf, const double *vt, int P, int nrhs, const double *rot64,
                                         const double *G0inv_shapes, const int *shape_id, double *dF, double *dT) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P * nrhs) return;
    const int k = i % P;
    const double *R = rot64 + 9 * k;
    const double *f = vf + 3 * (size_t)i, *t = vt + 3 * (size_t)i;
    double b[6], a[6];
    for (int c = 0; c < 3; ++c) {
        b[c] = R[c] * f[0] + R[3 + c] * f[1] + R[6 + c] * f[2];
        b[3 + c] = R[c] * t[0] + R[3 + c] * t[1] + R[6 + c] * t[2];
    }
    const double *Gi = G0inv_shapes + 36 * shape_id[k];
    for (int m = 0; m < 6; ++m) {
        double s = 0.0;
        for (int n = 0; n < 6; ++n) s += Gi[m * 6 + n] * b[n];
        a[m] = s;
    }
    for (int c = 0; c < 3; ++c) {
        dF[3 * (size_t)i + c] = R[3 * c] * a[0] + R[3 * c + 1] * a[1] + R[3 * c + 2] * a[2];
        dT[3 * (size_t)i + c] = R[3 * c] * a[3] + R[3 * c + 1] * a[4] + R[3 * c + 2] * a[5];
    }
}

extern "C" {

// Reverse mode of the last mfs_solve_mobility.  With U = E gamma, E = -K_N^T S_L^+ and A gamma = -u_0:
//   g = E^T dL/dU = -(S_L^+)^T K_N [dU; dOmega];  A^T w = g;  mu = lambda_0 + (I - L) S_L^+ gamma;
//   dL/dc_k = -sum_{i in k, j not in k} d/dr[w_i^T G mu_j] + sum_{j in k, i not in k} d/dr[w_i^T G mu_j];
//   dL/d[f; t]_k = -G_k^{-1} K_N^T (S^T w)_k over all pairs (Eq. stou0, Eq. lambda01-02).
mfs_status mfs_mobility_vjp(mfs_ctx *ctx, const double *dU, const double *dOmega, int32_t nrhs, double *dcenters,
                            double *dF, double *dT, void *stream) {
    if (!ctx || !dU || !dOmega || !dcenters || nrhs < 1 || nrhs > ctx->opt.max_rhs || (!dF) != (!dT)) {
        if (ctx) ctx->last_error = "mfs_mobility_vjp: invalid argument";
        return MFS_ERR_INVALID_ARG;
    }
    if (ctx->kind != MFS_STOKES || ctx->last_solve != 1 || ctx->last_nrhs != nrhs) {
        ctx->last_error = "mfs_mobility_vjp needs a preceding mfs_solve_mobility with the same nrhs";
        return MFS_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int P = ctx->P;
    const size_t nb = (size_t)nrhs * P * 3, nM = (size_t)nrhs * ctx->sumM * 3;
    Staged dUi, dWi, dco, dFo, dTo;
    CKS(stage_in(ctx, dUi, dU, nb, st));
    CKS(stage_in(ctx, dWi, dOmega, nb, st));
    CKS(stage_out_alloc(ctx, dco, dcenters, (size_t)P * 3));
    if (dF) {
        CKS(stage_out_alloc(ctx, dFo, dF, nb));
        CKS(stage_out_alloc(ctx, dTo, dT, nb));
    }
    CKS(ensure_transposed(ctx));
    CKS(ensure_gmres(ctx, nrhs));
    begin_call(ctx);
    // 1. seed g = -(S_L^+)^T K_N [dU; dOmega]
    CK(completion_stokes(dUi.d, dWi.d, nrhs, P, ctx->rot64_d, ctx->eye6_d, ctx->shape_id_d, ctx->src_local64_d,
                         ctx->src_off_d, ctx->sumN, ctx->lam_d, st));
    CKS(precondT_dev(ctx, ctx->lam_d, ctx->tmpM_d, 0, nrhs, st));
    combine_raw_kernel<<<(unsigned)((nM + 255) / 256), 256, 0, st>>>(ctx->tmpM_d, nullptr, 0.0, -1.0, ctx->b_d, nM);
    CK(cudaGetLastError());
    // 2. A^T w = g
    SolveStats ss;
    CKS(gmres_solve(ctx, nrhs, st, ss, true));
    if (ss.breakdown || !ss.converged) {
        ctx->last_error = "adjoint GMRES did not converge";
        return ss.breakdown ? MFS_ERR_BREAKDOWN : MFS_ERR_NOT_CONVERGED;
    }
    // 3. mu = lambda_0 + (I - L) S_L^+ gamma  (lambda_0 rebuilt from the kept F, T)
    double *lam0 = ctx->tmpM_d;  // [nrhs][sum_N][3] fits: sum_N < sum_M
    CK(completion_stokes(ctx->keep_lam0, ctx->keep_lam0 + nb, nrhs, P, ctx->rot64_d, ctx->G0inv_d, ctx->shape_id_d,
                         ctx->src_local64_d, ctx->src_off_d, ctx->sumN, lam0, st));
    CKS(precond_apply_dev(ctx, ctx->keep_gamma, ctx->lam_d, 1, nrhs, st));
    const size_t nN = (size_t)nrhs * ctx->sumN * 3;
    combine_raw_kernel<<<(unsigned)((nN + 255) / 256), 256, 0, st>>>(lam0, ctx->lam_d, 1.0, 1.0, ctx->lam_d, nN);
    CK(cudaGetLastError());
    // 4. centre gradient: pair kernel over off-diagonal pairs with target strengths w, source strengths mu
    int vc = 0, gv = -1;
    const PairVariant *vv = pair_variants(&vc);
    for (int i = 0; i < vc; ++i)
        if (vv[i].grad == 1 && vv[i].nrhs == nrhs) gv = i;  // the centre-gradient entry (not the stress one)
    if (gv < 0) {
        ctx->last_error = "no gradient kernel for this nrhs";
        return MFS_ERR_INVALID_ARG;
    }
    if (ctx->ff.ready && ctx->ffT.ready) {
        // through the treecodes: the target side on the forward tree (weights w at the collocation
        // points, sources mu), the source side on the transposed tree (weights mu at the proxy
        // points, sources w); tmpM_d (free again) takes the proxy-side gradient
        CKS(ff_grad_apply(ctx, ctx->ff, gv, ctx->lam_d, ctx->x_d, nrhs, ctx->gradT_d, st));
        CKS(ff_grad_apply(ctx, ctx->ffT, gv, ctx->x_d, ctx->lam_d, nrhs, ctx->tmpM_d, st));
        centre_grad_ff_kernel<<<P, 128, 0, st>>>(ctx->gradT_d, ctx->tgt_off_d, ctx->tmpM_d, ctx->src_off_d, dco.d);
        CK(cudaGetLastError());
        ctx->launches += 1;
    } else if (ctx->opt.precision == 1) {
        // FP64 reference, the same two sides as the treecode's: weights w at the collocation points
        // against mu, weights mu at the proxy points against w (roles swapped, sign folded into dc)
        CK(grad_pair_fp64(nrhs, ctx->tgt_local64_d, ctx->tgt_body_d, ctx->sumM, ctx->x_d, ctx->src_local4_d,
                          ctx->sumN, ctx->susp_src_begin_d, ctx->susp_src_end_d, ctx->src_off_d, ctx->centres_d,
                          ctx->lam_d, ctx->gradT_d, st));
        CK(grad_pair_fp64(nrhs, ctx->src_local64_d, ctx->src_body_d, ctx->sumN, ctx->lam_d, ctx->colloc4_d,
                          ctx->sumM, ctx->colT_begin_d, ctx->colT_end_d, ctx->tgt_off_d, ctx->centres_d, ctx->x_d,
                          ctx->tmpM_d, st));
        const double scale = kernel_scale(ctx);
        const size_t nc = (size_t)ctx->sumM * 3, np3 = (size_t)ctx->sumN * 3;
        combine_raw_kernel<<<(unsigned)((nc + 255) / 256), 256, 0, st>>>(ctx->gradT_d, nullptr, 0.0, scale,
                                                                         ctx->gradT_d, nc);
        combine_raw_kernel<<<(unsigned)((np3 + 255) / 256), 256, 0, st>>>(ctx->tmpM_d, nullptr, 0.0, scale,
                                                                          ctx->tmpM_d, np3);
        centre_grad_ff_kernel<<<P, 128, 0, st>>>(ctx->gradT_d, ctx->tgt_off_d, ctx->tmpM_d, ctx->src_off_d, dco.d);
        CK(cudaGetLastError());
        ctx->launches += 5;
    } else {
        to_f32_kernel<<<1024, 256, 0, st>>>(ctx->x_d, ctx->w32_d, nM);
        CK(pack_sources(3, nrhs, 0, ctx->src_pos_d, ctx->rec_pt_d, ctx->lam_d, ctx->sumN, ctx->nrec, ctx->rec_d, st));
        CK(cudaMemsetAsync(ctx->src_grad_d, 0, sizeof(double) * 3 * P, st));
        PairPlan *plan = nullptr;
        CKS(get_plan(ctx, gv, 0, &plan));
        PairGeom g = geom_of(ctx);
        g.tgt_w = ctx->w32_d;
        PairWork wk = work_of(*plan);
        wk.src_grad = ctx->src_grad_d;
        if (wk.total_units > 0) CK(pair_launch(gv, g, wk, ctx->err_d, st));
        CK(pair_epilogue(3, 1, wk, nullptr, 0.0, kernel_scale(ctx), ctx->gradT_d, ctx->sumM, st));
        centre_grad_kernel<<<P, 128, 0, st>>>(ctx->gradT_d, ctx->tgt_off_d, ctx->src_grad_d, kernel_scale(ctx), dco.d);
        CK(cudaGetLastError());
        ctx->launches += 6;
    }
    // 5. force and torque cotangents
    if (dF) {
        CKS(pair_apply_T(ctx, ctx->x_d, ctx->lam_d, nrhs, 1, st));
        CK(extract_stokes(ctx->lam_d, nrhs, P, ctx->src_local64_d, ctx->src_off_d, ctx->sumN, ctx->six_d,
                          ctx->six_d + nb, st));
        gram_solve_kernel<<<(unsigned)((P * nrhs + 127) / 128), 128, 0, st>>>(
            ctx->six_d, ctx->six_d + nb, P, nrhs, ctx->rot64_d, ctx->G0inv_d, ctx->shape_id_d, dFo.d, dTo.d);
        CK(cudaGetLastError());
        ctx->launches += 2;
        CKS(stage_out_finish(ctx, dFo, st));
        CKS(stage_out_finish(ctx, dTo, st));
    }
    CKS(stage_out_finish(ctx, dco, st));
    CK(cudaStreamSynchronize(st));
    return check_device_error(ctx, st);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Evaluation of the last solve's representation at arbitrary points
// ---------------------------------------------------------------------------
static __global__ void add_kernel(double *a, const double *b, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        a[i] += b[i];
}

// (p, T_x, T_y, T_z) per point and rhs -> pressure [n] and traction [n][3] (the -3 of Eq. traction).
static __global__ void split_stress_kernel(const double *o4, size_t n, double *p, double *t) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        if (p) p[e] = o4[4 * e];
        if (t)
            for (int c = 0; c < 3; ++c) t[3 * e + c] = -3.0 * o4[4 * e + 1 + c];
    }
}

// The stress entry of the pair-kernel table for nrhs (grad = 2), -1 if none.
static int stress_variant(int nrhs) {
    int count = 0;
    const PairVariant *vv = pair_variants(&count);
    for (int i = 0; i < count; ++i)
        if (vv[i].grad == 2 && vv[i].nrhs == nrhs) return i;
    return -1;
}

// out[h][order[i]][c] = in[h][i][c]: back from owner-sorted to the caller's point order.
static __global__ void unsort_kernel(const double *in, const int *order, int np, int D, int nrhs, double *out) {
    const size_t n = (size_t)nrhs * np * D;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const size_t h = e / ((size_t)np * D), r = e % ((size_t)np * D);
        const int i = (int)(r / D), c = (int)(r % D);
        out[(h * np + order[i]) * D + c] = in[e];
    }
}

// Evaluation points grouped by owner body (counting sort): order[j] is the caller's index of the j-th
// grouped point, toff[k] the first grouped point of body k; t4 / t64 the points relative to their
// owner's centre (FP32 with the owner id bits / FP64), nrm the grouped unit normals when given.
struct EvalTargets {
    std::vector<int> toff, order, tbody;
    std::vector<float4> t4;
    std::vector<double> t64;
    std::vector<float> nrm32;
    std::vector<double> nrm64;
};

static mfs_status group_targets(mfs_ctx *ctx, const double *points, const double *normals, const int32_t *owner,
                                int np, EvalTargets &e) {
    const int P = ctx->P;
    if (!owner && ctx->S > 1) {
        ctx->last_error = "evaluation: owner bodies are required with several suspensions";
        return MFS_ERR_INVALID_ARG;
    }
    std::vector<double> pts(3 * (size_t)np), nv;
    std::vector<int> own(np);
    CK(cudaMemcpy(pts.data(), points, sizeof(double) * pts.size(), cudaMemcpyDefault));
    if (normals) {
        nv.resize(3 * (size_t)np);
        CK(cudaMemcpy(nv.data(), normals, sizeof(double) * nv.size(), cudaMemcpyDefault));
    }
    if (owner) {
        CK(cudaMemcpy(own.data(), owner, sizeof(int) * np, cudaMemcpyDefault));
    } else {  // nearest body centre (single suspension)
        for (int i = 0; i < np; ++i) {
            double best = 1e300;
            int bk = 0;
            for (int k = 0; k < P; ++k) {
                double d2 = 0.0;
                for (int a = 0; a < 3; ++a) {
                    const double d = pts[3 * (size_t)i + a] - ctx->centres[3 * (size_t)k + a];
                    d2 += d * d;
                }
                if (d2 < best) {
                    best = d2;
                    bk = k;
                }
            }
            own[i] = bk;
        }
    }
    e.toff.assign(P + 1, 0);
    e.order.resize(np);
    e.tbody.resize(np);
    for (int i = 0; i < np; ++i) {
        bool finite = std::isfinite(pts[3 * (size_t)i]) && std::isfinite(pts[3 * (size_t)i + 1]) &&
                      std::isfinite(pts[3 * (size_t)i + 2]);
        if (normals)
            finite = finite && std::isfinite(nv[3 * (size_t)i]) && std::isfinite(nv[3 * (size_t)i + 1]) &&
                     std::isfinite(nv[3 * (size_t)i + 2]);
        if (own[i] < 0 || own[i] >= P || !finite) {
            ctx->last_error = "evaluation: owner out of range or non-finite point or normal";
            return MFS_ERR_INVALID_ARG;
        }
        e.toff[own[i] + 1]++;
    }
    for (int k = 0; k < P; ++k) e.toff[k + 1] += e.toff[k];
    e.t4.resize(np);
    e.t64.resize(3 * (size_t)np);
    if (normals) {
        e.nrm32.resize(3 * (size_t)np);
        e.nrm64.resize(3 * (size_t)np);
    }
    std::vector<int> fill(e.toff.begin(), e.toff.end() - 1);
    for (int i = 0; i < np; ++i) {
        const int k = own[i], j = fill[k]++;
        e.order[j] = i;
        e.tbody[j] = k;
        double x[3];
        for (int a = 0; a < 3; ++a) {
            x[a] = pts[3 * (size_t)i + a] - ctx->centres[3 * (size_t)k + a];
            e.t64[3 * (size_t)j + a] = x[a];
            if (normals) {
                e.nrm64[3 * (size_t)j + a] = nv[3 * (size_t)i + a];
                e.nrm32[3 * (size_t)j + a] = (float)nv[3 * (size_t)i + a];
            }
        }
        float kb;
        std::memcpy(&kb, &k, sizeof(float));  // body id stored as int bits
        e.t4[j] = make_float4((float)x[0], (float)x[1], (float)x[2], kb);
    }
    return MFS_OK;
}

namespace {
// The strengths of the representation of the last solve, [nrhs][sum_N][D] into ctx->lam_d:
// mobility (I - L) S_L^+ gamma + lambda_0 (Eq. multirep), elastance (I - L) S_L^+ gamma + alpha_0
// (Eq. erepK), resistance and capacitance S^+ gamma (Eq. reconbal).
mfs_status last_strengths(mfs_ctx *ctx, int nrhs, double *tmp, cudaStream_t st) {
    const int P = ctx->P;
    const size_t ns = (size_t)nrhs * ctx->sumN * ctx->D;
    if (ctx->last_solve >= 3) {
        DirichletScope scope(ctx);
        CKS(precond_apply_dev(ctx, ctx->keep_gamma, ctx->lam_d, 0, nrhs, st));
        return MFS_OK;
    }
    CKS(precond_apply_dev(ctx, ctx->keep_gamma, ctx->lam_d, 1, nrhs, st));
    if (ctx->last_solve == 1) {
        const size_t nb = (size_t)nrhs * P * 3;
        CK(completion_stokes(ctx->keep_lam0, ctx->keep_lam0 + nb, nrhs, P, ctx->rot64_d, ctx->G0inv_d,
                             ctx->shape_id_d, ctx->src_local64_d, ctx->src_off_d, ctx->sumN, tmp, st));
    } else {
        CK(completion_laplace(ctx->keep_lam0, nrhs, P, ctx->src_off_d, ctx->sumN, tmp, st));
    }
    add_kernel<<<(unsigned)std::min<size_t>((ns + 255) / 256, 4096), 256, 0, st>>>(ctx->lam_d, tmp, ns);
    CK(cudaGetLastError());
    return MFS_OK;
}
}  // namespace

// Sums at owner-grouped evaluation points through the treecode (farfield = 1): the upward step on the
// strengths in lam_d (a forward pair-sum entry), the proxy and equivalent records in the layout of
// `variant` (a pair sum for mfs_evaluate, the stress entry for mfs_evaluate_stress), the points
// reordered into the tree's body order, one-off interaction lists for them (each owner's radius that
// of its farthest point), and the launch of `variant` with per-point weights `tw_grouped` (the normals
// for the stress; may be null); results land in out_grouped [nrhs][np][dout] in the grouped order,
// scaled by `scale`.
static mfs_status ff_points(mfs_ctx *ctx, int variant, const EvalTargets &et, const float *tw_grouped, int nrhs,
                            int dout, double scale, double *out_grouped, cudaStream_t st) {
    auto &F = ctx->ff;
    const int P = ctx->P, D = ctx->D, np = (int)et.t4.size(), nodes = F.nodes;
    int vc = 0;
    const PairVariant *vv = pair_variants(&vc);
    const int fv = fp32_variant(ctx, D, nrhs);
    mfs_ctx::FarField::Plan *pu = nullptr;
    CKS(ff_get_plan(ctx, F, fv, 1, &pu));
    CKS(ff_upward(ctx, F, fv, pu, ctx->lam_d, nrhs, st));
    const int layout = vv[variant].packed, REC = pair_record_floats(D, nrhs, layout);
    if (REC > F.rec_floats) {
        ctx->last_error = "far field: record layout larger than its buffer";
        return MFS_ERR_INVALID_ARG;
    }
    CK(pack_sources(D, nrhs, layout, F.src_pos, F.rec_pt, ctx->lam_d, F.nsrc, F.nrec, F.rec, st));
    CK(pack_sources(D, nrhs, layout, F.eq_pos, F.eq_pt, F.mu, nodes * FF_NE, nodes * FF_NE,
                    F.rec + (size_t)F.nrec * REC, st));
    // tree order of the points; w = the owner's tree position; tperm: tree index -> grouped index
    std::vector<float4> tt(np);
    std::vector<float> tw(tw_grouped ? 3 * (size_t)np : 0);
    std::vector<int> tperm(np), toff(P + 1, 0);
    std::vector<double> rad(P, 0.0);
    int t = 0;
    for (int q = 0; q < P; ++q) {
        const int b = F.tree.order[q];
        float w;
        std::memcpy(&w, &q, sizeof(float));
        for (int j = et.toff[b]; j < et.toff[b + 1]; ++j, ++t) {
            tt[t] = make_float4(et.t4[j].x, et.t4[j].y, et.t4[j].z, w);
            if (tw_grouped)
                for (int a = 0; a < 3; ++a) tw[3 * (size_t)t + a] = tw_grouped[3 * (size_t)j + a];
            tperm[t] = j;
            const double *x = &et.t64[3 * (size_t)j];
            rad[b] = std::max(rad[b], std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]));
        }
        toff[q + 1] = t;
    }
    std::vector<long long> seg_blocks(P + nodes);
    std::vector<int> seg_recs(P + nodes);
    for (int sg = 0; sg < P + nodes; ++sg) {
        seg_recs[sg] = F.seg_rec1_h[sg] - F.seg_rec0_h[sg];
        seg_blocks[sg] = (seg_recs[sg] + MFS_BS - 1) / MFS_BS;
    }
    std::vector<int> cuts(ctx->S + 1), suspension_of(P), tb;
    for (int sp = 0; sp <= ctx->S; ++sp) cuts[sp] = ctx->body_off[sp];
    for (int sp = 0; sp < ctx->S; ++sp)
        for (int b = ctx->body_off[sp]; b < ctx->body_off[sp + 1]; ++b) suspension_of[b] = sp;
    PairPlan plan;
    int *lst_seg = nullptr, *perm_d = nullptr;
    long long *lst_cum = nullptr;
    float4 *tt_d = nullptr;
    float *tw_d = nullptr;
    double pairs = 0.0;
    mfs_status rc = build_plan_lists(
        ctx, variant, 1, toff, 0, cuts, seg_blocks, seg_recs,
        [&](int g0, int g1, std::vector<int> &segs) {
            tb.clear();
            for (int q = g0; q <= g1; ++q) tb.push_back(F.tree.order[q]);
            ff_interaction_list(F.tree, F.tree.roots[suspension_of[tb[0]]], tb, ctx->centres.data(), rad.data(),
                                ctx->opt.farfield_separation, 0, segs);
        },
        plan, &lst_seg, &lst_cum, pairs);
    if (rc == MFS_OK) {
        rc = [&]() -> mfs_status {
            CK(ctx->alloc(&tt_d, np));
            CK(ctx->alloc(&perm_d, np));
            CK(cudaMemcpyAsync(tt_d, tt.data(), sizeof(float4) * np, cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(perm_d, tperm.data(), sizeof(int) * np, cudaMemcpyHostToDevice, st));
            if (tw_grouped) {
                CK(ctx->alloc(&tw_d, tw.size()));
                CK(cudaMemcpyAsync(tw_d, tw.data(), sizeof(float) * tw.size(), cudaMemcpyHostToDevice, st));
            }
            PairGeom g = ff_geom(F);
            g.lst_seg = lst_seg;
            g.lst_cum = lst_cum;
            g.tgt = tt_d;
            g.ntargets = np;
            g.tgt_w = tw_d;
            PairWork we = work_of(plan);
            we.tperm = perm_d;
            CKS(ff_launch(ctx, variant, g, we, st));
            CK(pair_epilogue(dout, nrhs, we, nullptr, 0.0, scale, out_grouped, np, st));
            return MFS_OK;
        }();
    }
    cudaStreamSynchronize(st);  // the one-off lists and plan are freed below
    ctx->release(tt_d);
    ctx->release(tw_d);
    ctx->release(perm_d);
    ctx->release(lst_seg);
    ctx->release(lst_cum);
    if (plan.tiles) release_plan(ctx, plan);
    return rc;
}

extern "C" {

mfs_status mfs_evaluate(mfs_ctx *ctx, const double *points, const int32_t *owner, int32_t npoints, double *out,
                        int32_t nrhs, void *stream) {
    if (!ctx || (npoints > 0 && (!points || !out)) || npoints < 0 || nrhs < 1) {
        if (ctx) ctx->last_error = "mfs_evaluate: invalid argument";
        return MFS_ERR_INVALID_ARG;
    }
    if (ctx->last_solve == 0 || ctx->last_nrhs != nrhs) {
        ctx->last_error = "mfs_evaluate needs a preceding solve with the same nrhs";
        return MFS_ERR_INVALID_ARG;
    }
    if (npoints == 0) return MFS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int P = ctx->P, D = ctx->D, np = npoints;
    EvalTargets et;
    CKS(group_targets(ctx, points, nullptr, owner, np, et));
    std::vector<int> &toff = et.toff, &order = et.order, &tbody = et.tbody;
    std::vector<float4> &t4 = et.t4;
    std::vector<double> &t64 = et.t64;
    (void)P;
    Staged oo;
    CKS(stage_out_alloc(ctx, oo, out, (size_t)nrhs * np * D));
    float4 *t4_d = nullptr;
    int *order_d = nullptr, *tbody_d = nullptr;
    double *t64_d = nullptr, *sorted_d = nullptr, *tmp_d = nullptr, *raw_d = nullptr;
    PairPlan plan;
    auto cleanup = [&]() {
        cudaStreamSynchronize(st);
        void *ps[] = {t4_d, order_d, tbody_d, t64_d, sorted_d, tmp_d, raw_d};
        for (void *p : ps) ctx->release(p);
        if (plan.tiles) release_plan(ctx, plan);
    };
    mfs_status rc = [&]() -> mfs_status {
        CK(ctx->alloc(&t4_d, np));
        CK(ctx->alloc(&order_d, np));
        CK(ctx->alloc(&tbody_d, np));
        CK(ctx->alloc(&sorted_d, (size_t)nrhs * np * D));
        CK(ctx->alloc(&tmp_d, (size_t)nrhs * ctx->sumN * D));
        CK(cudaMemcpyAsync(t4_d, t4.data(), sizeof(float4) * np, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(order_d, order.data(), sizeof(int) * np, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(tbody_d, tbody.data(), sizeof(int) * np, cudaMemcpyHostToDevice, st));
        CKS(last_strengths(ctx, nrhs, tmp_d, st));
        const double scale = kernel_scale(ctx);
        if (ctx->opt.precision == 1) {  // FP64 direct sums
            CK(ctx->alloc(&t64_d, 3 * (size_t)np));
            CK(ctx->alloc(&raw_d, (size_t)nrhs * np * D));
            CK(cudaMemcpyAsync(t64_d, t64.data(), sizeof(double) * t64.size(), cudaMemcpyHostToDevice, st));
            CK(pair_sum_fp64(D, nrhs, t64_d, tbody_d, np, ctx->src_local4_d, ctx->sumN, ctx->susp_src_begin_d,
                             ctx->susp_src_end_d, ctx->src_off_d, ctx->centres_d, ctx->lam_d, 1, raw_d, st));
            const size_t n = (size_t)nrhs * np * D;
            combine_raw_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(raw_d, nullptr, 0.0, scale, sorted_d, n);
            CK(cudaGetLastError());
        } else {  // the FP32 pair kernel on the new targets, all pairs of the owner's suspension
            const int variant = fp32_variant(ctx, D, nrhs);
            if (variant < 0) {
                ctx->last_error = "no pair-kernel variant for this nrhs";
                return MFS_ERR_INVALID_ARG;
            }
            if (ctx->ff.ready) {  // through the treecode
                CKS(ff_points(ctx, variant, et, nullptr, nrhs, D, scale, sorted_d, st));
            } else {
                CKS(build_plan_for(ctx, variant, 1, toff, tbody, ctx->blk_off, np, plan));
                int vc = 0;
                const PairVariant *vv = pair_variants(&vc);
                CK(pack_sources(D, nrhs, vv[variant].packed, ctx->src_pos_d, ctx->rec_pt_d, ctx->lam_d, ctx->sumN,
                                ctx->nrec, ctx->rec_d, st));
                PairGeom g = geom_of(ctx);
                g.tgt = t4_d;
                g.ntargets = np;
                const PairWork w = work_of(plan);
                if (w.total_units > 0) CK(pair_launch(variant, g, w, ctx->err_d, st));
                CK(pair_epilogue(D, nrhs, w, nullptr, 0.0, scale, sorted_d, np, st));
            }
        }
        const size_t n = (size_t)nrhs * np * D;
        unsort_kernel<<<(unsigned)std::min<size_t>((n + 255) / 256, 4096), 256, 0, st>>>(sorted_d, order_d, np, D,
                                                                                          nrhs, oo.d);
        CK(cudaGetLastError());
        CKS(stage_out_finish(ctx, oo, st));
        return check_device_error(ctx, st);
    }();
    cleanup();
    return rc;
}

}  // extern "C"

extern "C" {

mfs_status mfs_evaluate_stress(mfs_ctx *ctx, const double *points, const double *normals, const int32_t *owner,
                               int32_t npoints, double *pressure, double *traction, int32_t nrhs, void *stream) {
    if (!ctx || npoints < 0 || nrhs < 1 || (npoints > 0 && (!points || (!pressure && !traction))) ||
        (traction && !normals)) {
        if (ctx) ctx->last_error = "mfs_evaluate_stress: invalid argument";
        return MFS_ERR_INVALID_ARG;
    }
    if (ctx->kind != MFS_STOKES) {
        ctx->last_error = "mfs_evaluate_stress needs a Stokes context";
        return MFS_ERR_INVALID_ARG;
    }
    if (ctx->last_solve == 0 || ctx->last_nrhs != nrhs) {
        ctx->last_error = "mfs_evaluate_stress needs a preceding solve with the same nrhs";
        return MFS_ERR_INVALID_ARG;
    }
    if (npoints == 0) return MFS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int P = ctx->P, np = npoints;
    EvalTargets et;
    CKS(group_targets(ctx, points, traction ? normals : nullptr, owner, np, et));
    // per body: the body range of its suspension
    std::vector<int> sb0(P), sb1(P);
    for (int s = 0; s < ctx->S; ++s)
        for (int k = ctx->body_off[s]; k < ctx->body_off[s + 1]; ++k) {
            sb0[k] = ctx->body_off[s];
            sb1[k] = ctx->body_off[s + 1];
        }
    Staged po, to;
    if (pressure) CKS(stage_out_alloc(ctx, po, pressure, (size_t)nrhs * np));
    if (traction) CKS(stage_out_alloc(ctx, to, traction, (size_t)nrhs * np * 3));
    float4 *t4_d = nullptr;
    float *n32_d = nullptr;
    int *order_d = nullptr, *tbody_d = nullptr, *sb0_d = nullptr, *sb1_d = nullptr;
    double *t64_d = nullptr, *n64_d = nullptr, *ps_d = nullptr, *ts_d = nullptr, *tmp_d = nullptr, *o4_d = nullptr;
    PairPlan splan;
    auto cleanup = [&]() {
        cudaStreamSynchronize(st);
        void *ps[] = {t4_d, n32_d, order_d, tbody_d, sb0_d, sb1_d, t64_d, n64_d, ps_d, ts_d, tmp_d, o4_d};
        for (void *p : ps) ctx->release(p);
        if (splan.tiles) release_plan(ctx, splan);
    };
    mfs_status rc = [&]() -> mfs_status {
        CK(ctx->alloc(&order_d, np));
        CK(ctx->alloc(&sb0_d, P));
        CK(ctx->alloc(&sb1_d, P));
        CK(ctx->alloc(&tmp_d, (size_t)nrhs * ctx->sumN * 3));
        if (pressure) CK(ctx->alloc(&ps_d, (size_t)nrhs * np));
        if (traction) CK(ctx->alloc(&ts_d, (size_t)nrhs * np * 3));
        CK(cudaMemcpyAsync(order_d, et.order.data(), sizeof(int) * np, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(sb0_d, sb0.data(), sizeof(int) * P, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(sb1_d, sb1.data(), sizeof(int) * P, cudaMemcpyHostToDevice, st));
        CKS(last_strengths(ctx, nrhs, tmp_d, st));
        if (ctx->opt.precision == 1) {
            CK(ctx->alloc(&t64_d, 3 * (size_t)np));
            CK(ctx->alloc(&tbody_d, np));
            CK(cudaMemcpyAsync(t64_d, et.t64.data(), sizeof(double) * et.t64.size(), cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(tbody_d, et.tbody.data(), sizeof(int) * np, cudaMemcpyHostToDevice, st));
            if (traction) {
                CK(ctx->alloc(&n64_d, 3 * (size_t)np));
                CK(cudaMemcpyAsync(n64_d, et.nrm64.data(), sizeof(double) * et.nrm64.size(), cudaMemcpyHostToDevice,
                                   st));
            }
            CK(stress_f64(nrhs, t64_d, tbody_d, n64_d, np, ctx->src_local64_d, ctx->src_off_d, ctx->sumN, ctx->lam_d,
                          sb0_d, sb1_d, ctx->centres_d, ps_d, ts_d, st));
        } else {  // the stress entry of the pair kernel (p, T per rhs), directly or through the treecode
            const int sv = stress_variant(nrhs);
            if (sv < 0) {
                ctx->last_error = "no stress kernel for this nrhs";
                return MFS_ERR_INVALID_ARG;
            }
            CK(ctx->alloc(&o4_d, (size_t)nrhs * np * 4));
            const double scale = 1.0 / (4.0 * MFS_PI);
            if (ctx->ff.ready) {
                CKS(ff_points(ctx, sv, et, traction ? et.nrm32.data() : nullptr, nrhs, 4, scale, o4_d, st));
            } else {
                CK(ctx->alloc(&t4_d, np));
                CK(cudaMemcpyAsync(t4_d, et.t4.data(), sizeof(float4) * np, cudaMemcpyHostToDevice, st));
                if (traction) {
                    CK(ctx->alloc(&n32_d, 3 * (size_t)np));
                    CK(cudaMemcpyAsync(n32_d, et.nrm32.data(), sizeof(float) * et.nrm32.size(),
                                       cudaMemcpyHostToDevice, st));
                }
                CKS(build_plan_for(ctx, sv, 1, et.toff, et.tbody, ctx->blk_off, np, splan));
                CK(pack_sources(3, nrhs, 0, ctx->src_pos_d, ctx->rec_pt_d, ctx->lam_d, ctx->sumN, ctx->nrec,
                                ctx->rec_d, st));
                PairGeom g = geom_of(ctx);
                g.tgt = t4_d;
                g.ntargets = np;
                g.tgt_w = n32_d;
                const PairWork w = work_of(splan);
                if (w.total_units > 0) CK(pair_launch(sv, g, w, ctx->err_d, st));
                CK(pair_epilogue(4, nrhs, w, nullptr, 0.0, scale, o4_d, np, st));
            }
            const size_t n = (size_t)nrhs * np;
            split_stress_kernel<<<(unsigned)std::min<size_t>((n + 255) / 256, 4096), 256, 0, st>>>(o4_d, n, ps_d,
                                                                                                  ts_d);
            CK(cudaGetLastError());
        }
        if (pressure) {
            const size_t n = (size_t)nrhs * np;
            unsort_kernel<<<(unsigned)std::min<size_t>((n + 255) / 256, 4096), 256, 0, st>>>(ps_d, order_d, np, 1,
                                                                                              nrhs, po.d);
            CK(cudaGetLastError());
            CKS(stage_out_finish(ctx, po, st));
        }
        if (traction) {
            const size_t n = (size_t)nrhs * np * 3;
            unsort_kernel<<<(unsigned)std::min<size_t>((n + 255) / 256, 4096), 256, 0, st>>>(ts_d, order_d, np, 3,
                                                                                              nrhs, to.d);
            CK(cudaGetLastError());
            CKS(stage_out_finish(ctx, to, st));
        }
        return check_device_error(ctx, st);
    }();
    cleanup();
    return rc;
}

}  // extern "C"
