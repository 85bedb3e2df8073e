"""Host logic of the far-field treecode (farfield.cu), run on the CPU: a C++ driver compiled with the
library's own tree and interaction-list code (no device code is executed).

For seeded clusters (one suspension of grown ellipsoids, several suspensions of random spheres):
* the tree order is a permutation of each suspension's bodies, every node's descendant range
  agrees with its children, and every node's source radius encloses its bodies' proxy spheres;
* for every target body, the interaction list covers every other body of its suspension exactly
  once — directly as a proxy segment, or inside exactly one node seen through its equivalent
  points — and never a body of another suspension; its own body appears only when self pairs count;
* every node seen through its equivalent points is at least `separation` equivalent radii from every
  target point (the far criterion), and every body summed directly is not.
"""

import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2409_04215_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <vector>
#include "kernels.h"
using namespace mfs;
int main(int argc, char **argv) {
    FILE *f = std::fopen(argv[1], "r");
    int P, S; double kappa; int self_skip;
    if (std::fscanf(f, "%d %d %lf %d", &P, &S, &kappa, &self_skip) != 4) return 1;
    std::vector<int> off(S + 1);
    for (auto &o : off) if (std::fscanf(f, "%d", &o) != 1) return 1;
    std::vector<double> c(3 * P), rs(P), rt(P);
    for (int k = 0; k < P; ++k)
        if (std::fscanf(f, "%lf %lf %lf %lf %lf", &c[3 * k], &c[3 * k + 1], &c[3 * k + 2], &rs[k], &rt[k]) != 5)
            return 1;
    FFTree t;
    ff_build_tree(P, c.data(), rs.data(), S, off.data(), t);
    std::printf("order");
    for (int b : t.order) std::printf(" %d", b);
    std::printf("\nroots");
    for (int r : t.roots) std::printf(" %d", r);
    std::printf("\n");
    for (size_t i = 0; i < t.nodes.size(); ++i) {
        const FFNode &n = t.nodes[i];
        std::printf("node %zu %.17g %.17g %.17g %.17g %.17g %d %d %d %d", i, n.c[0], n.c[1], n.c[2], n.rs, n.re,
                    n.body, n.first, n.count, n.nchild);
        for (int j = 0; j < n.nchild; ++j) std::printf(" %d", n.child[j]);
        std::printf("\n");
    }
    for (int s = 0; s < S; ++s)
        for (int b = off[s]; b < off[s + 1]; ++b) {
            std::vector<int> segs;
            ff_interaction_list(t, t.roots[s], std::vector<int>{b}, c.data(), rt.data(), kappa, self_skip, segs);
            std::printf("list %d", b);
            for (int g : segs) std::printf(" %d", g);
            std::printf("\n");
        }
    return 0;
}
"""


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    d = tmp_path_factory.mktemp("ff")
    (d / "driver.cu").write_text(DRIVER)
    exe = d / "ff_probe"
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    subprocess.run([nvcc, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a", "-I", CSRC,
                    str(d / "driver.cu"), os.path.join(CSRC, "farfield.cu"), "-o", str(exe)], check=True)
    return exe, d


def _run(probe, centres, rsrc, rtgt, offsets, kappa, self_skip):
    exe, d = probe
    inp = d / "in.txt"
    with open(inp, "w") as f:
        f.write(f"{len(centres)} {len(offsets) - 1} {float(kappa)!r} {int(self_skip)}\n")
        f.write(" ".join(str(int(o)) for o in offsets) + "\n")
        for c, a, b in zip(centres, rsrc, rtgt):
            f.write(" ".join(repr(float(v)) for v in (c[0], c[1], c[2], a, b)) + "\n")
    out = subprocess.run([str(exe), str(inp)], capture_output=True, text=True, check=True).stdout.splitlines()
    order = [int(x) for x in out[0].split()[1:]]
    roots = [int(x) for x in out[1].split()[1:]]
    nodes, lists = [], {}
    for line in out[2:]:
        w = line.split()
        if w[0] == "node":
            nodes.append(dict(c=np.array([float(x) for x in w[2:5]]), rs=float(w[5]), re=float(w[6]), body=int(w[7]),
                              first=int(w[8]), count=int(w[9]), kids=[int(x) for x in w[11:11 + int(w[10])]]))
        else:
            lists[int(w[1])] = [int(x) for x in w[2:]]
    return order, roots, nodes, lists


def _check(probe, centres, rsrc, rtgt, offsets, kappa, self_skip):
    order, roots, nodes, lists = _run(probe, centres, rsrc, rtgt, offsets, kappa, self_skip)
    P = len(centres)
    assert sorted(order) == list(range(P))
    pos = {b: q for q, b in enumerate(order)}
    for s in range(len(offsets) - 1):  # each suspension's bodies occupy their own range of the tree order
        assert sorted(order[offsets[s]:offsets[s + 1]]) == list(range(offsets[s], offsets[s + 1]))
        assert nodes[roots[s]]["first"] == offsets[s] and nodes[roots[s]]["count"] == offsets[s + 1] - offsets[s]
    for n in nodes:
        desc = order[n["first"]:n["first"] + n["count"]]
        if n["body"] >= 0:
            assert desc == [n["body"]] and not n["kids"]
        else:
            kid_desc = [b for k in n["kids"] for b in order[nodes[k]["first"]:nodes[k]["first"] + nodes[k]["count"]]]
            assert kid_desc == desc and 1 < len(n["kids"]) <= 8
        for b in desc:  # the node's proxy sources lie inside its source radius
            assert np.linalg.norm(centres[b] - n["c"]) + rsrc[b] <= n["rs"] * (1 + 1e-12) + 1e-12
        assert abs(n["re"] - n["rs"] / 0.83) <= 1e-12 * n["re"]
    for s in range(len(offsets) - 1):
        for t in range(offsets[s], offsets[s + 1]):
            seen = []
            for g in lists[t]:
                if g < P:  # a body summed directly: not far from the target
                    b = order[g]
                    n = next(nd for nd in nodes if nd["body"] == b)
                    assert np.linalg.norm(centres[t] - n["c"]) - rtgt[t] < kappa * n["re"]
                    seen.append(b)
                else:  # a node seen through its equivalent points: far from every target point
                    n = nodes[g - P]
                    assert np.linalg.norm(centres[t] - n["c"]) - rtgt[t] >= kappa * n["re"]
                    seen += order[n["first"]:n["first"] + n["count"]]
            want = [b for b in range(offsets[s], offsets[s + 1]) if not (self_skip and b == t)]
            assert sorted(seen) == want, t
            assert pos[t] >= 0


def test_lists_grown_ellipsoid_cluster(probe):
    from mfs_inputs import make_workload

    wl = make_workload("ellipsoidT5000_mobility", count=300, n_v=12)
    sh = wl.shapes[0]
    rsrc = np.full(wl.num_bodies, np.linalg.norm(sh.proxy, axis=1).max())
    rtgt = np.full(wl.num_bodies, np.linalg.norm(sh.colloc, axis=1).max())
    for kappa in (3.0, 2.5):
        for self_skip in (True, False):
            _check(probe, wl.centres, rsrc, rtgt, wl.body_offsets, kappa, self_skip)


def test_lists_several_suspensions_mixed_radii(probe):
    from mfs_inputs import make_workload

    wl = make_workload("batched256_mobility", num_suspensions=7, p_lo=1, p_hi=70, m=60, n=30, seed=12)
    rsrc = np.array([np.linalg.norm(wl.shapes[i].proxy, axis=1).max() for i in wl.shape_id])
    rtgt = np.array([np.linalg.norm(wl.shapes[i].colloc, axis=1).max() for i in wl.shape_id])
    _check(probe, wl.centres, rsrc, rtgt, wl.body_offsets, 3.0, True)
