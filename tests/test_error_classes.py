"""The FP32-vs-FP64 error classification of the benchmark (bench.error_classes)
on hand-built states: node classes by distance to the faces, the face that
sets an edge node, and far-field face nodes whose Riemann branch differs."""
import numpy as np

import bench
from paper_2003_09926_gb300 import workloads as W

import states as ST


def test_classes_and_branch_flip(orc):
    gd = W.jet_grid(10, 8, 7)
    gd["stretch_c"] = 0.0
    o = orc.Oracle(gd, W.jet_flow())
    S = o.inner(o.S)
    nk, nj, ni = 7, 8, 10
    one = np.ones((nk, nj, ni))
    # subsonic everywhere, c = 1.01: the subsonic split u_n + 5 (c - 1) is
    # u_n + 0.05, at least 0.04 from zero on every far-field face
    c2 = 1.01 ** 2
    ref = ST.primitive_to_conserved(one, 0.5 * one, 0.01 * one, 0.0 * one, c2 * one / 1.4)
    got = ref.copy()
    # interior node (4, 1, 3) adjacent to the y- face node (4, 0, 3): v = 0.06
    # there makes the split -0.01, so that face node switches branch
    got[:, 3, 1, 4] = ST.primitive_to_conserved(1.0, 0.5, 0.06, 0.0, c2 / 1.4)
    got[1, 3, 0, 4] += 0.25           # the face node's own value differs
    got[0, 3, 3, 5] += 1e-6           # a node at distance 3 (i = 5, j = 3, k = 3)
    got[0, 0, 4, 0] += 1e-7           # an inflow-face node (x- wins its edge with z-)
    c = bench.error_classes(got, ref, S, gd["bc"])
    assert c["farfield_face_near_switch"]["nodes"] == 1
    assert c["farfield_face_near_switch"]["max_rel_per_variable"][1] == 0.25 / 0.5
    assert c["farfield_face_clear_of_switch"]["max_rel"] == 0.0
    assert abs(c["interior_d1"]["max_rel_per_variable"][2] - 0.05 / 0.01) < 1e-12
    assert abs(c["interior_d3plus"]["max_rel_per_variable"][0] - 1e-6) < 1e-15
    assert c["interior_d2"]["max_rel"] == 0.0
    assert abs(c["inflow_face"]["max_rel_per_variable"][0] - 1e-7) < 1e-15
    n_face = ni * nj * nk - (ni - 2) * (nj - 2) * (nk - 2)
    assert c["inflow_face"]["nodes"] == nj * nk
    assert c["farfield_face_clear_of_switch"]["nodes"] + 1 == n_face - nj * nk
    assert c["interior_d3plus"]["nodes"] == (ni - 6) * (nj - 6) * max(nk - 6, 0)
    assert c["all_nodes"]["nodes"] == ni * nj * nk


def test_riemann_branch_cases():
    n = np.array([[1.0], [0.0], [0.0]])
    q = lambda u, c: ST.primitive_to_conserved(np.array([1.0]), np.array([u]), np.array([0.0]), np.array([0.0]),  # noqa: E731
                                               np.array([c * c / 1.4]))
    assert bench.riemann_branch(q(1.2, 1.0), n)[0] == 3
    assert bench.riemann_branch(q(-1.2, 1.0), n)[0] == 0
    assert bench.riemann_branch(q(0.2, 1.0), n)[0] == 2
    assert bench.riemann_branch(q(-0.2, 1.0), n)[0] == 1
    # the subsonic split is the characteristic average: u_n + 5 (c - 1) > 0
    assert bench.riemann_branch(q(0.1, 0.97), n)[0] == 1
    assert bench.riemann_branch(q(-0.1, 1.03), n)[0] == 2
    br, m = bench.riemann_branch(q(-0.1, 1.0201), n, margin=True)
    assert br[0] == 2 and abs(m[0] - 0.0005) < 1e-12  # 5 (c - 1) - 0.1 = 0.0005
