// Far-field acceleration of the pair sums (host side): the tree over the bodies and the interaction
// lists of an equivalent-source treecode.
//
// The paper accelerates its pair sums with a fast multipole method on the CPU (Sec. 4: FMM3D, more
// than 90 % of its time).  Here the far field is represented the kernel-independent way, with the
// MFS's own device: every node of a tree over the bodies (each body, and each group of bodies) gets
// FF_NE equivalent point sources on a sphere of radius r_e around its centre whose field reproduces
// that of the node's proxy sources outside it.  The equivalent strengths are the least-squares fit
// of the sources' field on FF_NC check points at radius FF_CHECK * r_e (the "upward" step, run on the
// device), and a target at least kappa * r_e from a node's centre (kappa = farfield_separation, 3 by
// default) sees the node through them.
// Targets nearer than that see the node's children, down to the bodies' own proxy points.  Both the
// fit's right-hand side and the final sums are ordinary pair sums over interaction lists, so the
// device work is the pair kernel plus one FP64 matrix product per apply.
//
// This file builds, on the host: the tree (8-ary, by median splits of the body centres in x, then y,
// then z), the nodes' centres and radii, and the interaction list of a set of target bodies.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "kernels.h"

namespace mfs {

namespace {

struct Builder {
    const double *centres;
    const double *rsrc;
    std::vector<FFNode> &nodes;
    std::vector<int> &order;

    int leaf(int b) {
        FFNode n;
        for (int a = 0; a < 3; ++a) n.c[a] = centres[3 * b + a];
        n.rs = rsrc[b];
        n.body = b;
        n.first = (int)order.size();
        n.count = 1;
        order.push_back(b);
        nodes.push_back(n);
        return (int)nodes.size() - 1;
    }

    // Split ids into two halves (sizes differing by at most one) by the coordinate `axis`.
    static void halve(std::vector<int> &ids, int axis, const double *centres, std::vector<int> &lo,
                      std::vector<int> &hi) {
        std::sort(ids.begin(), ids.end(), [&](int a, int b) {
            const double xa = centres[3 * a + axis], xb = centres[3 * b + axis];
            return xa < xb || (xa == xb && a < b);
        });
        const size_t h = ids.size() / 2;
        lo.assign(ids.begin(), ids.begin() + h);
        hi.assign(ids.begin() + h, ids.end());
    }

    int build(std::vector<int> ids) {
        if (ids.size() == 1) return leaf(ids[0]);
        const int me = (int)nodes.size();
        nodes.push_back(FFNode());
        std::vector<std::vector<int>> groups;
        if (ids.size() <= 8) {
            for (int b : ids) groups.push_back({b});
        } else {
            std::vector<int> x0, x1;
            halve(ids, 0, centres, x0, x1);
            for (auto *gx : {&x0, &x1}) {
                std::vector<int> y0, y1;
                halve(*gx, 1, centres, y0, y1);
                for (auto *gy : {&y0, &y1}) {
                    std::vector<int> z0, z1;
                    halve(*gy, 2, centres, z0, z1);
                    if (!z0.empty()) groups.push_back(z0);
                    if (!z1.empty()) groups.push_back(z1);
                }
            }
        }
        const int first = (int)order.size();
        std::vector<int> kids;
        for (auto &g : groups) kids.push_back(build(g));
        FFNode n;
        n.body = -1;
        n.first = first;
        n.count = (int)order.size() - first;
        n.nchild = (int)kids.size();
        for (int i = 0; i < n.nchild; ++i) n.child[i] = kids[i];
        // centre: middle of the bounding box of the descendant bodies' centres; radius of its sources
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        for (int q = n.first; q < n.first + n.count; ++q)
            for (int a = 0; a < 3; ++a) {
                lo[a] = std::min(lo[a], centres[3 * order[q] + a]);
                hi[a] = std::max(hi[a], centres[3 * order[q] + a]);
            }
        for (int a = 0; a < 3; ++a) n.c[a] = 0.5 * (lo[a] + hi[a]);
        double rs = 0.0;
        for (int q = n.first; q < n.first + n.count; ++q) {
            const int b = order[q];
            double d2 = 0.0;
            for (int a = 0; a < 3; ++a) d2 += (centres[3 * b + a] - n.c[a]) * (centres[3 * b + a] - n.c[a]);
            rs = std::max(rs, std::sqrt(d2) + rsrc[b]);
        }
        n.rs = rs;
        nodes[me] = n;
        return me;
    }
};

}  // namespace

void ff_build_tree(int P, const double *centres, const double *rsrc, int S, const int *body_off, FFTree &t) {
    t.nodes.clear();
    t.order.clear();
    t.roots.clear();
    t.nodes.reserve(2 * (size_t)P);
    t.order.reserve(P);
    Builder bld{centres, rsrc, t.nodes, t.order};
    for (int s = 0; s < S; ++s) {
        std::vector<int> ids(body_off[s + 1] - body_off[s]);
        std::iota(ids.begin(), ids.end(), body_off[s]);
        t.roots.push_back(bld.build(ids));
    }
    t.pos.assign(P, 0);
    for (int q = 0; q < P; ++q) t.pos[t.order[q]] = q;
    for (auto &n : t.nodes) n.re = n.rs / FF_SRC_RATIO;
}

void ff_interaction_list(const FFTree &t, int root, const std::vector<int> &tbodies, const double *centres,
                         const double *rtgt, double kappa, int self_skip, std::vector<int> &segs) {
    const int P = (int)t.order.size();
    std::vector<int> stack{root};
    while (!stack.empty()) {
        const int ni = stack.back();
        stack.pop_back();
        const FFNode &n = t.nodes[ni];
        // far: every target point of the set is at least kappa r_e from the node's centre
        bool far = true;
        for (int b : tbodies) {
            double d2 = 0.0;
            for (int a = 0; a < 3; ++a) d2 += (centres[3 * b + a] - n.c[a]) * (centres[3 * b + a] - n.c[a]);
            if (std::sqrt(d2) - rtgt[b] < kappa * n.re) {
                far = false;
                break;
            }
        }
        if (far) {
            segs.push_back(P + ni);
        } else if (n.body >= 0) {
            if (!(self_skip && tbodies.size() == 1 && tbodies[0] == n.body)) segs.push_back(t.pos[n.body]);
        } else {
            for (int i = n.nchild - 1; i >= 0; --i) stack.push_back(n.child[i]);
        }
    }
}

__global__ void ff_scale_kernel(double *mu, const double *re, int nodes, int per_node, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        mu[i] *= re[(i / per_node) % nodes];
}

cudaError_t ff_scale(double *mu, const double *re, int nodes, int per_node, int nrhs, cudaStream_t st) {
    const size_t n = (size_t)nrhs * nodes * per_node;
    if (n == 0) return cudaSuccess;
    ff_scale_kernel<<<(unsigned)std::min<size_t>((n + 255) / 256, 4096), 256, 0, st>>>(mu, re, nodes, per_node, n);
    return cudaGetLastError();
}

}  // namespace mfs
