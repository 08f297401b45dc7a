"""The multi-CTA build forms against the oracle on problems it finishes quickly.

The ID (Sec. 2.2) and the Gauss-Jordan steps of the block elimination (eq.
compressed-inverse) have several GPU forms: one CTA per box in shared memory,
a thread-block cluster per box, a cooperative launch with a grid barrier per
pivot step, and a launch per pivot step; the blocked Gauss-Jordan handles the
root.  The normal selection uses the last forms only for boxes too large for
the faster ones (the top levels of the 3D workloads), i.e. only at full size.
rs_set_path removes choices so that these forms run on small problems, and
rs_path_counts records which forms each build used.  Bars as in the other
parity tests: tree bit-exact, leaf ranks within +-2 of the oracle's,
solutions within 10 eps of the oracle's.
"""
import numpy as np
import pytest

import rs_inputs as ri
from oracle import rskel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = {
    "sphere": ("laplace3d", "sphere", 4096, 1e-6, 128, 216),
    "starfish": ("laplace2d", "starfish", 4096, 1e-10, 64, 64),
}
CASE_NAMES = list(CASES)

# spec -> (per case: forms of which at least one must have run; forms that
# must not have run).  A cooperative launch needs every CTA of the level
# resident at once: the 3D leaf boxes' column caches are too large for that,
# so there the selection falls through to the per-step launches.
FORCED = [
    ("id:coop", {"starfish": ["id_coop"], "sphere": ["id_coop", "id_step"]}, ["id_cta", "id_cluster"]),
    ("id:step", {"starfish": ["id_step"], "sphere": ["id_step"]}, ["id_cta", "id_cluster", "id_coop"]),
    ("id:big", {"starfish": ["id_cluster", "id_coop", "id_step"], "sphere": ["id_cluster", "id_coop", "id_step"]},
     ["id_cta"]),
    ("factor:big,gj:coop", {"starfish": ["gj_coop"], "sphere": ["gj_coop", "gj_step"]},
     ["factor_smem", "gj_cluster", "gj_blocked"]),
    ("factor:big,gj:step", {"starfish": ["gj_step"], "sphere": ["gj_step"]},
     ["factor_smem", "gj_cluster", "gj_blocked", "gj_coop"]),
    ("factor:big,gj:blocked", {"starfish": ["factor_big"], "sphere": ["factor_big"]}, ["factor_smem", "gj_cluster"]),
]


@pytest.fixture(scope="module", params=list(CASES), ids=str)
def case(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1110_3105_gb300 as rs
    kind, geom, n, eps, leaf, nproxy = CASES[request.param]
    pts, w = ri.geometry(geom, n)
    F = rskel.build(pts, rskel.Params(kind=kind, w=w, eps=eps, leaf=leaf, nproxy=nproxy))
    B = ri.rhs(n, 3, seed=61)
    return dict(name=request.param, rs=rs, kind=kind, n=n, eps=eps, leaf=leaf, nproxy=nproxy, pts=pts, w=w, F=F, B=B,
                Xo=F.solve(B))


@pytest.mark.parametrize("spec,must,mustnot", FORCED, ids=[f[0] for f in FORCED])
def test_forced_form_matches_oracle(case, spec, must, mustnot):
    rs = case["rs"]
    rs.rs_set_path(spec)
    rs.rs_path_counts(reset=True)
    try:
        H = rs.rs_build(case["pts"], case["kind"], case["w"], case["eps"], case["leaf"], case["nproxy"])
    finally:
        rs.rs_set_path(None)
    counts = rs.rs_path_counts(reset=True)
    try:
        F = case["F"]
        assert np.array_equal(rs.rs_tree_perm(H), F.tree.perm)
        L = F.tree.L
        _, k = rs.rs_box_ranks(H, L, F.tree.levels[L].nbox)
        assert np.max(np.abs(k - np.array([f.k for f in F.boxes[L]]))) <= 2
        X = np.zeros_like(case["B"])
        rs.rs_solve(H, case["B"], X)
        err = np.linalg.norm(X - case["Xo"], axis=0) / np.linalg.norm(case["Xo"], axis=0)
        assert np.all(err <= 10 * case["eps"]), (spec, counts, err)
    finally:
        H.free()
    assert any(counts[name] > 0 for name in must[case["name"]]), (spec, counts)
    for name in mustnot:
        assert counts[name] == 0, (spec, counts)


def test_normal_selection_recorded(case):
    """Without an override: the 2D boxes all fit one CTA or a cluster; the 3D
    sphere's top boxes (n ~ 500, m ~ 3000) fit neither, so its top ID level
    runs one launch per pivot step.  The counters say which forms ran."""
    rs = case["rs"]
    rs.rs_set_path(None)
    rs.rs_path_counts(reset=True)
    H = rs.rs_build(case["pts"], case["kind"], case["w"], case["eps"], case["leaf"], case["nproxy"])
    H.free()
    counts = rs.rs_path_counts(reset=True)
    assert counts["id_cta"] + counts["id_cluster"] + counts["id_coop"] + counts["id_step"] >= 1
    if case["name"] == "starfish":
        assert counts["id_coop"] == 0 and counts["id_step"] == 0, counts
    else:
        assert counts["id_step"] >= 1, counts
