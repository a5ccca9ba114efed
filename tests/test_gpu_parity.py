"""GPU path (C ABI) against the FP64 CPU oracle on the same seeded inputs.

Tolerances (relative L2 unless stated):
  direct FP64 matvec  1e-6   (differences: semi-analytical self integral with
                              N_k = 9 vs the exact one, ~1e-8, and summation order)
  direct FP32 matvec  1e-5
  treecode P = 6, theta = 0.5 (FP32 or FP64) 1e-4
  sigma_ext           1e-6 relative in direct FP64 mode, 1e-5 in refined direct FP32
                      mode (FP32 right-hand side); treecode P = 6, theta = 0.5: 3e-4
                      (the solve amplifies the ~1e-5 operator error near the
                      resonance); treecode P = 8: 1e-4
Near-singular classification is an integer decision: it must match exactly.
"""
import json
import os

import numpy as np
import pytest

from paper_1812_10722_gb300 import inputs as I

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def lspr():
    from paper_1812_10722_gb300 import build, lspr as L
    build.build()
    return L


def _ragged_mesh():
    # an open patch whose panel count is not a multiple of the 64-target block
    v, t = I.icosphere(3, 10.0)
    keep = np.ones(len(t), bool)
    keep[::29] = False
    return v, t[keep]


MESHES = {
    "sphere1280": lambda: I.icosphere(3, 10.0),
    "ragged1235": _ragged_mesh,
    "protein512": lambda: I.protein_like(3, seed=1812),
    "single": lambda: (np.array([[0, 0, 0], [1.0, 0, 0], [0, 1.0, 0]]), np.array([[0, 1, 2]], np.int32)),
}


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _rowmax(a, b):
    """Largest error of one element against the largest magnitude: max_i |a_i - b_i| / max_i |b_i|."""
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def _agree(a, b, tol, what="", tol_elem=None):
    """a matches b in the relative L2 norm (tol) and element by element (tol_elem, default tol): no
    single row may carry an error the norm would average away."""
    e2, ei = _rel(a, b), _rowmax(a, b)
    te = tol if tol_elem is None else tol_elem
    assert e2 < tol and ei < te, f"{what} relative L2 {e2:.3e}, largest element error {ei:.3e} (tol {tol:g}, {te:g})"


@pytest.mark.parametrize("name", list(MESHES))
def test_near_classification_exact(lspr, oracle, name):
    v, t = MESHES[name]()
    with lspr.Context(0) as ctx:
        ctx.mesh_upload(v, t)
        nnz = ctx.info()["n_near"]
    tot, cnt = oracle.near_pairs(v, t)
    assert nnz - len(t) == tot


# The semi-analytical self integral (N_k Gauss-Legendre nodes in the angle per
# edge) approaches the exact closed form of the oracle geometrically in N_k; on
# the irregular analyte-like mesh N_k = 9 leaves ~2e-6 and on the right triangle
# ~1e-3, so those run at N_k = 24 and 32.
NK = {"protein512": 24, "single": 32}


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("mode,tol", [("direct_fp64", 1e-6), ("direct_fp32", 1e-5)])
def test_matvec_direct(lspr, oracle, name, mode, tol):
    v, t = MESHES[name]()
    n = len(t)
    s = I.drude_eps(380.0) / I.EPS_WATER
    x = I.random_complex(2 * n, seed=11)
    yo = oracle.matvec(v, t, x, s)
    with lspr.Context(0) as ctx:
        ctx.mesh_upload(v, t, N_k=NK.get(name, 9))
        y = ctx.matvec(x, s, mode)
    _agree(y, yo, tol, name)


def test_self_integral_converges_in_Nk(lspr, oracle):
    # single-panel mesh: y_top = phi/2 - V_ii dphi isolates the semi-analytical V_ii
    rng = np.random.default_rng(3)
    for _ in range(5):
        v = rng.normal(size=(3, 3))
        t = np.array([[0, 1, 2]], np.int32)
        exact = oracle.self_V(v[0], v[1], v[2], v.mean(0))
        errs = []
        with lspr.Context(0) as ctx:
            for nk in (3, 6, 9, 16, 32):
                ctx.mesh_upload(v, t, N_k=nk)
                y = ctx.matvec(np.array([0.0, 1.0 + 0j]), 1.0, "direct_fp64")
                errs.append(abs(-y[0].real - exact) / exact)
        # geometric convergence: each step in N_k gains accuracy, 32 nodes reach <= 1e-6
        assert errs[-1] < 1e-6 and errs[-1] < 1e-4 * errs[0], errs
        assert all(errs[i + 1] <= errs[i] * 1.01 + 1e-15 for i in range(len(errs) - 1)), errs


@pytest.mark.parametrize("name", ["sphere1280", "ragged1235", "protein512"])
@pytest.mark.parametrize("mode", ["tree_fp32", "tree_fp64"])
@pytest.mark.parametrize("ncrit", [32, 300])
def test_matvec_tree(lspr, oracle, name, mode, ncrit):
    v, t = MESHES[name]()
    n = len(t)
    s = I.drude_eps(375.0) / I.EPS_WATER
    x = I.random_complex(2 * n, seed=5)
    yo = oracle.matvec(v, t, x, s)
    with lspr.Context(0) as ctx:
        ctx.mesh_upload(v, t)
        ctx.tree_build(0.5, 6, ncrit)
        info = ctx.info()
        y = ctx.matvec(x, s, mode)
    assert info["n_boxes"] >= 1
    _agree(y, yo, 1e-4, name)


def test_tree_error_falls_with_order(lspr, oracle):
    v, t = I.icosphere(3, 10.0)
    s = I.drude_eps(380.0) / I.EPS_WATER
    x = I.random_complex(2 * len(t), seed=2)
    yo = oracle.matvec(v, t, x, s)
    errs = []
    with lspr.Context(0) as ctx:
        ctx.mesh_upload(v, t)
        for P in (1, 2, 4, 6, 8):
            ctx.tree_build(0.5, P, 32)
            errs.append(_rel(ctx.matvec(x, s, "tree_fp64"), yo))
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1)), errs
    assert errs[-1] < 1e-6


def test_batched_matvec_and_device_pointers(lspr, oracle):
    torch = pytest.importorskip("torch")
    v, t = I.icosphere(3, 10.0)
    n = len(t)
    lam = I.wavelengths(350, 420, 3)
    s = I.drude_eps(lam) / I.EPS_WATER
    x = I.random_complex(2 * n, seed=9, batch=3)
    yo = oracle.matvec(v, t, x, s)
    with lspr.Context(0) as ctx:
        ctx.mesh_upload(torch.as_tensor(v, device="cuda"), torch.as_tensor(t, device="cuda"))
        ctx.tree_build(0.5, 6, 64)
        y_host = ctx.matvec(x, s, "tree_fp32")
        y_dev = ctx.matvec(torch.as_tensor(x, device="cuda"), s, "tree_fp32").cpu().numpy()
    for b in range(3):
        _agree(y_host[b], yo[b], 1e-4, b)
    # same product through device pointers; the FP32 far field accumulates with atomics
    # in a run-dependent order, so the two agree to FP32 rounding, not bit for bit
    assert _rel(y_dev, y_host) < 1e-6


def _golden(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


# FP32 operators leave a residual floor of a few 1e-6 near the resonance (rounding
# of the large, nearly cancelling layer potentials), so FP32 modes solve with FP64
# iterative refinement; the refined solution is that of the FP64 operator of the
# same kind (direct or treecode).
@pytest.mark.parametrize("mode,tol,gtol,refine", [("direct_fp64", 1e-6, 1e-8, False),
                                                  ("direct_fp32", 1e-5, 1e-8, True),
                                                  ("tree_fp64", 3e-4, 1e-8, False),
                                                  ("tree_fp32", 3e-4, 1e-8, True)])
def test_solve_sigma_sphere1280(lspr, mode, tol, gtol, refine):
    g = _golden("sphere1280_l380.json")
    v, t = I.icosphere(3, 10.0)
    ep = I.drude_eps(380.0)
    with lspr.Context(0) as ctx:
        ctx.mesh_upload(v, t)
        ctx.tree_build(0.5, 6, 300)
        r = ctx.solve(ep, I.EPS_WATER, 380.0, tol=gtol, mode=mode, restart=100, refine=refine)
    assert r.status[0] == 0
    assert abs(r.sigma_ext[0] - g["sigma_ext_nm2"]) / g["sigma_ext_nm2"] < tol
    p_ref = complex(*g["dipole"][2])
    assert abs(r.dipole[0, 2] - p_ref) / abs(p_ref) < tol


def test_fp32_refinement_matches_fp64_operator(lspr):
    # the refined FP32 solve reproduces the FP64 solve of the same operator, up to the
    # ~1e-7 FP32 error of its right-hand side amplified by the conditioning near resonance
    v, t = I.icosphere(3, 10.0)
    ep = I.drude_eps(375.0)
    with lspr.Context(0) as ctx:
        ctx.mesh_upload(v, t)
        ctx.tree_build(0.5, 6, 64)
        a = ctx.solve(ep, I.EPS_WATER, 375.0, tol=1e-9, mode="tree_fp64", restart=100)
        b = ctx.solve(ep, I.EPS_WATER, 375.0, tol=1e-9, mode="tree_fp32", refine=True, restart=100)
        c = ctx.solve(ep, I.EPS_WATER, 375.0, tol=3e-5, mode="tree_fp32", refine=False, restart=100)
    assert a.status[0] == 0 and b.status[0] == 0 and c.status[0] == 0
    assert abs(b.sigma_ext[0] - a.sigma_ext[0]) / a.sigma_ext[0] < 1e-5
    assert abs(c.sigma_ext[0] - a.sigma_ext[0]) / a.sigma_ext[0] < 2e-3


def test_treecode_order_8_meets_sigma_tolerance(lspr):
    g = _golden("sphere1280_l380.json")
    v, t = I.icosphere(3, 10.0)
    with lspr.Context(0) as ctx:
        ctx.mesh_upload(v, t)
        ctx.tree_build(0.5, 8, 64)
        r = ctx.solve(I.drude_eps(380.0), I.EPS_WATER, 380.0, tol=1e-8, mode="tree_fp32", refine=True)
    assert abs(r.sigma_ext[0] - g["sigma_ext_nm2"]) / g["sigma_ext_nm2"] < 1e-4


def test_solve_batched_wavelengths(lspr, oracle):
    v, t = I.icosphere(2, 10.0)
    lam = np.array([350.0, 370.0, 380.0, 420.0])
    ep = I.drude_eps(lam)
    dip, sig, its, bad = oracle.solve(v, t, ep, I.EPS_WATER, lam, tol=1e-9)
    with lspr.Context(0) as ctx:
        ctx.mesh_upload(v, t)
        ctx.tree_build(0.5, 6, 64)
        r = ctx.solve(ep, I.EPS_WATER, lam, tol=1e-9, mode="tree_fp32", refine=True, restart=60)
        r64 = ctx.solve(ep, I.EPS_WATER, lam, tol=1e-9, mode="direct_fp64", restart=60)
    assert np.all(r.status == 0) and np.all(r64.status == 0)
    assert np.max(np.abs(r.sigma_ext - sig) / sig) < 1e-4
    assert np.max(np.abs(r64.sigma_ext - sig) / sig) < 1e-6


def test_solve_polarisation_and_field_scaling(lspr):
    # sigma_ext does not depend on |E0|; for a sphere it does not depend on the direction either
    v, t = I.icosphere(3, 10.0)
    ep = I.drude_eps(390.0)
    with lspr.Context(0) as ctx:
        ctx.mesh_upload(v, t)
        a = ctx.solve(ep, I.EPS_WATER, 390.0, E0=(0, 0, 1), tol=1e-9, mode="direct_fp64").sigma_ext[0]
        b = ctx.solve(ep, I.EPS_WATER, 390.0, E0=(0, 0, -3.5), tol=1e-9, mode="direct_fp64").sigma_ext[0]
        c = ctx.solve(ep, I.EPS_WATER, 390.0, E0=(1, 1, 0), tol=1e-9, mode="direct_fp64").sigma_ext[0]
    assert abs(a - b) / a < 1e-7
    assert abs(a - c) / a < 2e-2    # icosphere is only approximately isotropic


def test_errors_are_status_codes(lspr):
    v, t = I.icosphere(1, 10.0)
    with lspr.Context(0) as ctx:
        with pytest.raises(lspr.LsprError) as e:
            ctx.tree_build(0.5, 6, 64)
        assert e.value.status == 2            # no mesh yet
        bad = t.copy()
        bad[0, 0] = len(v) + 5
        with pytest.raises(lspr.LsprError) as e:
            ctx.mesh_upload(v, bad)
        assert e.value.status == 1
        deg = t.copy()
        deg[0, 1] = deg[0, 0]
        with pytest.raises(lspr.LsprError) as e:
            ctx.mesh_upload(v, deg)
        assert e.value.status == 7
        with pytest.raises(lspr.LsprError) as e:
            ctx.mesh_upload(v, t, K=5)
        assert e.value.status == 1
        ctx.mesh_upload(v, t)
        with pytest.raises(lspr.LsprError) as e:
            ctx.matvec(np.zeros(2 * len(t), complex), 1.0, "tree_fp32")
        assert e.value.status == 2            # tree mode without a tree
        with pytest.raises(lspr.LsprError) as e:
            ctx.tree_build(0.5, 9, 64)
        assert e.value.status == 1
        r = ctx.solve(I.drude_eps(380.0), I.EPS_WATER, 380.0, tol=1e-12, maxiter=2, mode="direct_fp64",
                      check=False)
        assert r.status[0] == 5 and r.iterations[0] <= 2


@pytest.mark.slow
def _sampled_rows(oracle, v, t, x, s, blocks):
    """The oracle's product on blocks of 64 rows (top and bottom rows of those panels)."""
    n = len(t)
    idx, ref = [], []
    for i0 in blocks:
        yo = oracle.matvec_rows(v, t, x, s, (i0, i0 + 64))
        rows = np.r_[i0:i0 + 64, n + i0:n + i0 + 64]
        idx.append(rows)
        ref.append(yo[..., rows])
    return np.concatenate(idx), np.concatenate(ref, axis=-1)


@pytest.mark.slow
@pytest.mark.parametrize("tree", [(0.4, 5, 256), (0.5, 6, 300)])
def test_full_size_20480_rows_and_sigma(lspr, oracle, tree):
    # 20480-panel sphere at the tree the autotuner picks for the one-wavelength workload
    # (theta 0.4, P 5, Ncrit 256) and at the configuration's literal one: 256 rows (four blocks
    # of 64 across the Morton order) element by element against the oracle's rows; sigma_ext
    # of the refined FP32 solve against the oracle's stored solve
    v, t = I.icosphere(5, 10.0)
    n = len(t)
    s = I.drude_eps(380.0) / I.EPS_WATER
    x = I.random_complex(2 * n, seed=4)
    rows, yo = _sampled_rows(oracle, v, t, x, s, [0, n // 3, 2 * n // 3, n - 64])
    with lspr.Context(0) as ctx:
        ctx.mesh_upload(v, t)
        ctx.tree_build(*tree)
        y = ctx.matvec(x, s, "tree_fp32")
        r = ctx.solve(I.drude_eps(380.0), I.EPS_WATER, 380.0, tol=1e-6, mode="tree_fp32", refine=True, restart=50)
    _agree(y[rows], yo, 1e-4, tree)
    g = _golden("sphere20480_l380.json")
    err = abs(r.sigma_ext[0] - g["sigma_ext_nm2"]) / g["sigma_ext_nm2"]
    # the tuned tree meets the metric's 1e-4; the literal P = 6, theta = 0.5 tree truncates
    # at ~7e-4 (the reason the bench tunes it)
    assert err < (1e-4 if tree == (0.4, 5, 256) else 1e-3), err


@pytest.mark.slow
def test_full_size_81920_sweep(lspr, oracle):
    # the 64-wavelength sweep on the 81920-panel sphere at the tree the autotuner picks for it
    # (theta 0.4, P 7, Ncrit 512), tensor-core far field for 64 right-hand sides: 256 rows of
    # the 64-right-hand-side product element by element against the oracle's rows, then the
    # batched refined solve's sigma_ext against the oracle's stored solves at four wavelengths
    # (nearest the resonance, both ends, the middle)
    v, t = I.icosphere(6, 10.0)
    n = len(t)
    lam = I.wavelengths(350, 420, 64)
    ep = I.drude_eps(lam)
    s = ep / I.EPS_WATER
    x = I.random_complex(2 * n, seed=6, batch=64)
    rows, yo = _sampled_rows(oracle, v, t, x, s, [0, n // 3, 2 * n // 3, n - 64])
    with lspr.Context(0) as ctx:
        ctx.mesh_upload(v, t)
        ctx.tree_build(0.4, 7, 512)
        y = ctx.matvec(x, s, "tree_fp32")
        for b in range(64):
            _agree(y[b][rows], yo[b], 1e-4, b)
        r = ctx.solve(ep, I.EPS_WATER, lam, tol=1e-6, mode="tree_fp32", refine=True, restart=50, maxiter=2000)
        assert ctx.device_errors() == 0
    g = _golden("sphere81920_sweep64.json")
    for k, ref in zip(g["sweep_index"], g["sigma_ext_nm2"]):
        err = abs(r.sigma_ext[k] - ref) / ref
        assert err < 1e-4, (lam[k], err)


@pytest.mark.parametrize("mode,tol", [("direct_fp64", 1e-6), ("direct_fp32", 1e-5), ("tree_fp64", 1e-4),
                                      ("tree_fp32", 1e-4)])
def test_batched_matvec_ragged_chunks(lspr, oracle, mode, tol):
    # 11 right-hand sides: one full and one partial chunk of 8 (FP32) or 4 (FP64)
    v, t = _ragged_mesh()
    n = len(t)
    lam = I.wavelengths(350, 420, 11)
    s = I.drude_eps(lam) / I.EPS_WATER
    x = I.random_complex(2 * n, seed=17, batch=11)
    yo = oracle.matvec(v, t, x, s)
    with lspr.Context(0) as ctx:
        ctx.mesh_upload(v, t)
        ctx.tree_build(0.5, 6, 64)
        y = ctx.matvec(x, s, mode)
        y1 = ctx.matvec(x[5], s[5], mode)
    for b in range(11):
        _agree(y[b], yo[b], tol, b)
    # a batched column equals the single-RHS product (in FP32 modes up to FP32-level rounding:
    # several right-hand sides take the tensor-core M2P, one takes the FP32 pipe)
    assert _rel(y[5], y1) < (1e-6 if mode.endswith("fp64") else 1e-5)


def test_batched_solve_equals_single(lspr):
    v, t = I.icosphere(3, 10.0)
    lam = I.wavelengths(360, 400, 6)
    ep = I.drude_eps(lam)
    with lspr.Context(0) as ctx:
        ctx.mesh_upload(v, t)
        ctx.tree_build(0.5, 6, 64)
        rb = ctx.solve(ep, I.EPS_WATER, lam, tol=1e-9, mode="tree_fp32", refine=True, restart=60)
        singles = [ctx.solve(ep[b], I.EPS_WATER, lam[b], tol=1e-9, mode="tree_fp32", refine=True,
                             restart=60).sigma_ext[0] for b in range(len(lam))]
    assert np.all(rb.status == 0)
    assert np.max(np.abs(rb.sigma_ext - np.array(singles)) / np.array(singles)) < 1e-6


@pytest.mark.parametrize("name", ["sphere1280", "ragged1235"])
@pytest.mark.parametrize("kind,ncrit", [("direct", 300), ("tree", 32), ("tree", 300)])
def test_float_float_operator_matches_fp64(lspr, name, kind, ncrit):
    # float-float (hi + lo FP32 pairs) evaluation of the same operator: ~1e-13 per term
    v, t = MESHES[name]()
    n = len(t)
    lam = I.wavelengths(360, 400, 5)
    s = I.drude_eps(lam) / I.EPS_WATER
    x = I.random_complex(2 * n, seed=23, batch=5)
    with lspr.Context(0) as ctx:
        ctx.mesh_upload(v, t)
        ctx.tree_build(0.5, 6, ncrit)
        y64 = ctx.matvec(x, s, f"{kind}_fp64")
        yff = ctx.matvec(x, s, f"{kind}_ff")
        y1 = ctx.matvec(x[0], s[0], f"{kind}_ff")
    assert _rel(yff, y64) < 1e-11
    assert _rel(y1, y64[0]) < 1e-11


def test_refinement_residual_float_float_vs_fp64(lspr):
    v, t = I.icosphere(3, 10.0)
    ep = I.drude_eps(380.0)
    with lspr.Context(0) as ctx:
        ctx.mesh_upload(v, t)
        ctx.tree_build(0.5, 6, 64)
        a = ctx.solve(ep, I.EPS_WATER, 380.0, tol=1e-10, mode="tree_fp32", refine=1, restart=100)
        b = ctx.solve(ep, I.EPS_WATER, 380.0, tol=1e-10, mode="tree_fp32", refine=2, restart=100)
    assert a.status[0] == 0 and b.status[0] == 0 and a.residual[0] <= 1e-10
    assert abs(a.sigma_ext[0] - b.sigma_ext[0]) / b.sigma_ext[0] < 1e-8


@pytest.mark.parametrize("P", [1, 3, 8])
def test_float_float_operator_every_order(lspr, P):
    # the float-float M2P walks a term table for every order: ff = FP64 at P = 1, 3, 8
    v, t = MESHES["ragged1235"]()
    n = len(t)
    lam = I.wavelengths(360, 400, 5)
    s = I.drude_eps(lam) / I.EPS_WATER
    x = I.random_complex(2 * n, seed=29, batch=5)
    with lspr.Context(0) as ctx:
        ctx.mesh_upload(v, t)
        ctx.tree_build(0.5, P, 32)
        y64 = ctx.matvec(x, s, "tree_fp64")
        yff = ctx.matvec(x, s, "tree_ff")
        y1 = ctx.matvec(x[2], s[2], "tree_ff")
    assert _rel(yff, y64) < 1e-11
    assert _rel(y1, y64[2]) < 1e-11


@pytest.mark.parametrize("mode,refine,B,restart", [("direct_fp64", 0, 1, 50), ("direct_fp64", 0, 3, 12),
                                                   ("tree_fp32", 1, 1, 50), ("tree_fp32", 1, 4, 16),
                                                   ("tree_fp64", 0, 2, 10)])
def test_graph_cycles_match_host_cycles(lspr, mode, refine, B, restart):
    # Arnoldi cycles as device-driven graph loops give the host-driven cycles' result;
    # short restarts exercise several cycles, and the recorded graph is reused
    v, t = MESHES["sphere1280"]()
    lam = I.wavelengths(395, 420, B)
    ep = I.drude_eps(lam)
    kw = dict(tol=1e-9, mode=mode, refine=refine, restart=restart, maxiter=3000)
    with lspr.Context(0) as ctx:
        ctx.mesh_upload(v, t)
        ctx.tree_build(0.5, 6, 64)
        ctx.set_graphs(False)
        h = ctx.solve(ep, I.EPS_WATER, lam, **kw)
        assert ctx.graph_stats()["cycles"] == 0
        ctx.set_graphs(True)
        g = ctx.solve(ep, I.EPS_WATER, lam, **kw)
        ctx.mesh_upload(v, t)            # same sizes: the recorded graph stays valid
        ctx.tree_build(0.5, 6, 64)
        g2 = ctx.solve(ep, I.EPS_WATER, lam, **kw)
        st = ctx.graph_stats()
    assert np.all(h.status == 0) and np.all(g.status == 0) and np.all(g2.status == 0)
    assert st["cycles"] > 0 and st["recordings"] <= 2
    assert np.max(np.abs(g.sigma_ext - h.sigma_ext) / np.abs(h.sigma_ext)) < 1e-7
    # repeat: FP32 atomics make the far field's summation order vary from run to run
    assert np.max(np.abs(g2.sigma_ext - g.sigma_ext) / np.abs(g.sigma_ext)) < 1e-7
    if not refine:   # same kernels and stopping rule; the atomics' summation order varies from
        # run to run (host-driven runs alone differ), and where the explicit residual at a restart
        # lands within rounding of tol one run stops and the other takes part of another cycle
        assert np.all(np.abs(g.iterations - h.iterations) <= restart)


def test_graph_cycles_respect_iteration_limit(lspr):
    v, t = MESHES["protein512"]()
    ep = I.drude_eps(380.0)
    with lspr.Context(0) as ctx:
        ctx.mesh_upload(v, t)
        r = ctx.solve(ep, I.EPS_WATER, 380.0, tol=1e-14, mode="direct_fp64", restart=4, maxiter=10,
                      check=False)
        assert ctx.graph_stats()["cycles"] >= 3
    assert r.iterations[0] == 10 and r.status[0] != 0


def test_autotune_meets_sigma_bound(lspr):
    # the autotuner's choice, built in the context, reproduces the FP64 oracle's sigma_ext
    # within the requested bound
    v, t = I.icosphere(3, 10.0)
    g = _golden("sphere1280_l380.json")["sigma_ext_nm2"]
    ep = I.drude_eps(380.0)
    with lspr.Context(0) as ctx:
        ctx.mesh_upload(v, t)
        r = ctx.autotune(ep, I.EPS_WATER, 380.0, target_rel_err=1e-4, tol=1e-8)
        s = ctx.solve(ep, I.EPS_WATER, 380.0, tol=1e-8, mode="tree_fp32", refine=True)
    assert r["candidates"] == 60 and r["qualified"] >= 1 and r["rel_err"] <= 5e-5
    assert 4 <= r["P"] <= 8 and r["theta"] in (0.3, 0.4, 0.5, 0.6) and r["Ncrit"] in (128, 256, 512)
    assert r["ms"] <= r["ref_ms"]
    assert abs(s.sigma_ext[0] - g) / g < 1e-4


def test_autotune_batch_cost_and_solver(lspr):
    # batch tuning: candidates costed from product times at 24 right-hand sides (the faster P2P
    # path left set), then the restart and P2P path timed with full solves of the batch; the
    # chosen configuration solves the batch to the same sigma_ext as the FP64 treecode
    v, t = I.icosphere(3, 10.0)
    lam = I.wavelengths(355, 400, 24)
    ep = I.drude_eps(lam)
    lt = lam[[0, 10, 23]]
    with lspr.Context(0) as ctx:
        ctx.mesh_upload(v, t)
        r = ctx.autotune(I.drude_eps(lt), I.EPS_WATER, lt, target_rel_err=1e-4, tol=1e-8, coarse=True, time_rhs=24)
        assert r["candidates"] == 13 and r["qualified"] >= 1 and r["rel_err"] <= 5e-5   # 12 + the reference
        assert r["product_ms"] > 0 and r["residual_product_ms"] > 0 and r["iterations"] > 0
        assert r["tensor_cores"] in (1, 3)
        sv = ctx.tune_solver(ep, I.EPS_WATER, lam, restarts=(20, 40), tol=1e-8)
        assert sv["restart"] in (20, 40) and sv["tensor_cores"] in (1, 3) and sv["ms"] > 0
        a = ctx.solve(ep, I.EPS_WATER, lam, tol=1e-8, restart=sv["restart"], maxiter=3000, mode="tree_fp32",
                      refine=True)
        b = ctx.solve(ep, I.EPS_WATER, lam, tol=1e-8, restart=sv["restart"], maxiter=3000, mode="tree_fp64")
        with pytest.raises(lspr.LsprError):
            ctx.tune_solver(ep, I.EPS_WATER, lam, restarts=(0,))
        assert ctx.device_errors() == 0
    assert np.max(np.abs(a.sigma_ext - b.sigma_ext) / b.sigma_ext) < 1e-5


def _sensor_small():
    # sphere (surface 0) and two analytes at 0.5 and 1 nm: cross-surface near-singular pairs
    # (the analytes' skinny panels need N_k = 24 for the semi-analytical self integral to
    # match the exact one to ~1e-8)
    return I.sensor_geometry(2, 10.0, analytes=(("+z", 0.5), ("-x", 1.0)), analyte_sub=2)


@pytest.mark.parametrize("mode,tol", [("direct_fp64", 1e-6), ("direct_fp32", 1e-5), ("direct_ff", 1e-6),
                                      ("tree_fp64", 1e-4), ("tree_fp32", 1e-4)])
def test_multi_surface_matvec(lspr, oracle, mode, tol):
    # Eq. matrix_multi: self-surface interior rows, all-surface exterior rows with s_t weights
    v, t, surf = _sensor_small()
    n = len(t)
    lam = I.wavelengths(360, 400, 3)
    s = np.stack([I.drude_eps(lam) / I.EPS_WATER, np.full(3, 2.25 / I.EPS_WATER),
                  np.array([1.8, 2.0, 2.6]) / I.EPS_WATER + 0.01j], axis=1)
    x = I.random_complex(2 * n, seed=31, batch=3)
    yo = oracle.matvec_multi(v, t, surf, x, s)
    with lspr.Context(0) as ctx:
        ctx.mesh_upload(v, t, N_k=24, surf_id=surf)
        ctx.tree_build(0.5, 6, 32)
        y = ctx.matvec(x, s, mode)
        y1 = ctx.matvec(x[1], s[1], mode)
    for b in range(3):
        _agree(y[b], yo[b], tol, b)
    _agree(y1, yo[1], tol, "single")


@pytest.mark.parametrize("graphs", [True, False])
def test_multi_surface_solve(lspr, oracle, graphs):
    v, t, surf = _sensor_small()
    lam = np.array([370.0, 390.0])
    eps = np.stack([I.drude_eps(lam), np.full(2, 2.25), np.full(2, 2.0 + 0.05j)], axis=1)
    dref, sref, _, bad = oracle.solve_multi(v, t, surf, eps, I.EPS_WATER, lam, tol=1e-10)
    assert bad == 0
    with lspr.Context(0) as ctx:
        ctx.set_graphs(graphs)
        ctx.mesh_upload(v, t, N_k=24, surf_id=surf)
        r = ctx.solve(eps, I.EPS_WATER, lam, tol=1e-10, mode="direct_fp64", restart=100, maxiter=2000)
        ctx.tree_build(0.3, 8, 32)
        rt = ctx.solve(eps, I.EPS_WATER, lam, tol=1e-8, mode="tree_fp32", refine=True, restart=60, maxiter=2000)
        r1 = ctx.solve(eps[1], I.EPS_WATER, lam[1], tol=1e-8, mode="tree_fp32", refine=True, restart=60,
                       maxiter=2000)
    assert np.all(r.status == 0) and np.all(rt.status == 0)
    assert np.max(np.abs(r.sigma_ext - sref) / sref) < 1e-6
    assert np.max(np.abs(r.dipole - dref)) < 1e-6 * np.max(np.abs(dref))
    assert np.max(np.abs(rt.sigma_ext - sref) / sref) < 1e-4
    assert abs(r1.sigma_ext[0] - rt.sigma_ext[1]) / rt.sigma_ext[1] < 1e-6


def test_point_charges_solve(lspr, oracle):
    # charges inside the analytes add their Coulomb potential over 4 pi eps_t to the analytes'
    # interior rows (Eqs. integral_eq_lspr_system, matrix_multi); GPU against the oracle
    v, t, surf = _sensor_small()
    c = v[t].mean(axis=1)
    q1, q2 = c[surf == 1].mean(axis=0), c[surf == 2].mean(axis=0)
    charges = np.array([[*q1, 800.0], [*(q1 + [0.3, -0.2, 0.1]), -500.0], [*(q2 + [0.0, 0.2, 0.0]), 1200.0]])
    csurf = np.array([1, 1, 2], np.int32)
    lam = np.array([370.0, 390.0])
    eps = np.stack([I.drude_eps(lam), np.full(2, 2.25), np.full(2, 2.0 + 0.05j)], axis=1)
    dref, sref, _, bad = oracle.solve_multi(v, t, surf, eps, I.EPS_WATER, lam, tol=1e-10, charges=charges,
                                            charge_surf=csurf)
    d0, _, _, bad0 = oracle.solve_multi(v, t, surf, eps, I.EPS_WATER, lam, tol=1e-10)
    assert bad == 0 and bad0 == 0
    assert np.max(np.abs(dref - d0)) > 1e-3 * np.max(np.abs(d0))   # the charges matter
    with lspr.Context(0) as ctx:
        ctx.mesh_upload(v, t, N_k=24, surf_id=surf)
        ctx.set_charges(charges, csurf)
        r = ctx.solve(eps, I.EPS_WATER, lam, tol=1e-10, mode="direct_fp64", restart=100, maxiter=2000)
        ctx.tree_build(0.3, 8, 32)
        rt = ctx.solve(eps, I.EPS_WATER, lam, tol=1e-8, mode="tree_fp32", refine=True, restart=60, maxiter=2000)
        ctx.set_charges([[0.0, 0.0, 0.0, 1.0]], [3])   # no surface 3
        with pytest.raises(lspr.LsprError):
            ctx.solve(eps, I.EPS_WATER, lam, tol=1e-10, mode="direct_fp64", restart=100, maxiter=2000)
        ctx.set_charges(None)
        rn = ctx.solve(eps, I.EPS_WATER, lam, tol=1e-10, mode="direct_fp64", restart=100, maxiter=2000)
    assert np.all(r.status == 0) and np.all(rt.status == 0) and np.all(rn.status == 0)
    scale = np.max(np.abs(dref))
    assert np.max(np.abs(r.dipole - dref)) < 1e-6 * scale
    assert np.max(np.abs(r.sigma_ext - sref)) < 1e-6 * np.max(np.abs(sref))
    assert np.max(np.abs(rt.dipole - dref)) < 1e-4 * scale
    assert np.max(np.abs(rn.dipole - d0)) < 1e-6 * np.max(np.abs(d0))


def test_centred_charge_leaves_the_dipole(lspr):
    # a charge at the centre of a sphere adds a field of full symmetry: the dipole is unchanged
    v, t = I.icosphere(3, 10.0)
    lam = np.array([380.0])
    eps = I.drude_eps(lam)
    with lspr.Context(0) as ctx:
        ctx.mesh_upload(v, t)
        a = ctx.solve(eps, I.EPS_WATER, lam, tol=1e-10, mode="direct_fp64", restart=100, maxiter=2000)
        ctx.set_charges([[0.0, 0.0, 0.0, 5000.0]], [0])
        b = ctx.solve(eps, I.EPS_WATER, lam, tol=1e-10, mode="direct_fp64", restart=100, maxiter=2000)
    assert np.max(np.abs(b.dipole - a.dipole)) < 1e-8 * np.max(np.abs(a.dipole))


def test_off_centre_charge_in_the_particle(lspr, oracle):
    # a charge off the centre of the particle (surface 0) polarises it: dipole and sigma_ext of the
    # GPU solve against the oracle's (both take the dipole about the coordinate origin)
    v, t = I.icosphere(3, 10.0)
    surf = np.zeros(len(t), np.int32)
    lam = np.array([375.0, 395.0])
    eps = I.drude_eps(lam)
    charges = np.array([[2.0, -1.0, 3.5, 900.0]])
    dref, sref, _, bad = oracle.solve_multi(v, t, surf, eps.reshape(2, 1), I.EPS_WATER, lam, tol=1e-10,
                                            charges=charges, charge_surf=[0])
    d0, _, _, _ = oracle.solve_multi(v, t, surf, eps.reshape(2, 1), I.EPS_WATER, lam, tol=1e-10)
    assert bad == 0 and np.max(np.abs(dref - d0)) > 1e-3 * np.max(np.abs(d0))   # the charge matters
    with lspr.Context(0) as ctx:
        ctx.mesh_upload(v, t)
        ctx.set_charges(charges, [0])
        r = ctx.solve(eps, I.EPS_WATER, lam, tol=1e-10, mode="direct_fp64", restart=100, maxiter=2000)
    assert np.all(r.status == 0)
    assert np.max(np.abs(r.dipole - dref)) < 1e-6 * np.max(np.abs(dref))
    assert np.max(np.abs(r.sigma_ext - sref)) < 1e-6 * np.max(np.abs(sref))


def test_multi_surface_upload_errors(lspr):
    v, t, surf = _sensor_small()
    bad = surf.copy()
    bad[5] = 7
    with lspr.Context(0) as ctx:
        with pytest.raises(lspr.LsprError):
            ctx.mesh_upload(v, t, surf_id=bad, nsurf=3)
        ctx.mesh_upload(v, t, N_k=24, surf_id=surf)
        assert ctx.nsurf == 3


def test_grid_study_through_the_library(lspr, oracle):
    # the paper's Table 6 case (R = 8 nm, lossy water, K_fine = 37) on the GPU: errors
    # against Eq. an_sol at N = 512 and 2048 reproduce the printed 29.86 % and 7.33 %, the
    # observed order is ~1 and Richardson from 2048/8192 is much closer than 8192 alone
    from paper_1812_10722_gb300 import convergence as C
    em, ep, lam = 1.7972 + 8.5048e-9j, -3.3877 + 0.1922j, 380.0
    exact = oracle.sigma_closed_form(8.0, ep, em, lam)
    meshes = [I.octasphere(s, 8.0) for s in (3, 4, 5)]
    with lspr.Context(0) as ctx:
        out = C.grid_study([(v, t) for v, t in meshes], ep, em, lam, ctx=ctx, quad=dict(K_fine=37), tol=1e-10,
                           restart=100, maxiter=3000)
    err = [100 * (s - exact) / exact for s in out["sigma_ext"]]
    assert abs(err[0] - 29.86) <= 0.005 + 1e-9 and abs(err[1] - 7.33) <= 0.005 + 1e-9
    assert abs(err[2] - 1.9) <= 0.05
    assert 0.95 < out["order"] < 1.1
    assert abs(out["extrapolated"] - exact) < 0.1 * abs(out["sigma_ext"][2] - exact)


def test_lossy_host_matches_oracle(lspr, oracle):
    # complex host permittivity (k' = Re k in sigma_ext): GPU solve against the oracle's
    v, t = I.icosphere(3, 10.0)
    em = 1.7689 + 0.05j
    lam = np.array([370.0, 390.0])
    ep = I.drude_eps(lam)
    _, so, _, bad = oracle.solve(v, t, ep, em, lam, tol=1e-10)
    assert bad == 0
    with lspr.Context(0) as ctx:
        ctx.mesh_upload(v, t)
        r = ctx.solve(ep, em, lam, tol=1e-10, mode="direct_fp64", restart=100, maxiter=2000)
    assert np.max(np.abs(r.sigma_ext - so) / so) < 1e-6


@pytest.mark.parametrize("P,B", [(5, 5), (6, 16), (7, 40), (8, 20), (3, 2), (7, 64), (5, 70)])
def test_tensor_core_m2p_matches_fp32_pipe(lspr, oracle, P, B):
    # 3xTF32 products on the tensor cores give the FP32-pipe M2P's sums to FP32-level rounding
    # (the low parts are truncated to TF32: ~2^-21 per product, a few 1e-6 over the sum, inside
    # the FP32 product tolerance of 1e-5).  Units hold 16 right-hand sides up to B = 16, else
    # 32: B = 40 is one full and one partial unit of 32, B = 20 one partial unit of 32, B = 5
    # and B = 2 partial units of 16; P = 8 takes six stages of 32 terms per box, P = 3 one.
    v, t = I.icosphere(3, 10.0)
    n = len(t)
    lam = I.wavelengths(350, 420, B)
    s = I.drude_eps(lam) / I.EPS_WATER
    x = I.random_complex(2 * n, seed=37, batch=B)
    with lspr.Context(0) as ctx:
        ctx.mesh_upload(v, t)
        ctx.tree_build(0.5, P, 32)
        ytc = ctx.matvec(x, s, "tree_fp32")
        ytc2 = ctx.matvec(x, s, "tree_fp32")
        ctx.set_tensor_cores(3)   # the P2P on the tensor cores too
        ytp = ctx.matvec(x, s, "tree_fp32")
        assert ctx.device_errors() == 0
        ctx.set_tensor_cores(False)
        yfp = ctx.matvec(x, s, "tree_fp32")
        y64 = ctx.matvec(x, s, "tree_fp64")
    # every FP32-level variant (tensor-core M2P; tensor-core M2P and P2P; FP32 pipe) against the FP64
    # treecode of the same tree at the FP32 product tolerance.  The split operands hold 22
    # significant bits (two 11-bit TF32 parts, each rounded to nearest) against FP32's 24, so a
    # split product carries up to ~3 x 2^-22 relative error against ~2^-23 for an FP32 FMA: the
    # P2P, whose near pairs are the largest terms, may then show an element error a few times the
    # FP32 pipe's (measured 1.1e-5 against FP64 where the FP32 pipe stays below 1e-5), so the
    # variant with the tensor-core P2P is held to 3e-5 element by element (1e-5 in L2)
    for b in range(B):
        _agree(ytc2[b], ytc[b], 1e-6, b)
        _agree(ytc[b], y64[b], 1e-5, b)
        _agree(ytp[b], y64[b], 1e-5, b, tol_elem=3e-5)
        _agree(yfp[b], y64[b], 1e-5, b)
        _agree(ytp[b], yfp[b], 2e-5, b, tol_elem=4e-5)
        _agree(ytc[b], yfp[b], 2e-5, b)
    if P == 6:
        yo = oracle.matvec(v, t, x[:3], s[:3])
        for b in range(3):
            _agree(ytc[b], yo[b], 1e-4, b)


@pytest.mark.parametrize("B", [3, 24])
def test_tensor_core_m2p_partial_group(lspr, B):
    # 320 panels = five target blocks: the second group of four holds one block, and the
    # targets beyond the mesh get zero coefficients (M2P) and kernel values (P2P) and no
    # accumulation
    v, t = I.icosphere(2, 10.0)
    n = len(t)
    lam = I.wavelengths(350, 420, B)
    s = I.drude_eps(lam) / I.EPS_WATER
    x = I.random_complex(2 * n, seed=41, batch=B)
    with lspr.Context(0) as ctx:
        ctx.mesh_upload(v, t)
        ctx.tree_build(0.6, 4, 16)
        ytc = ctx.matvec(x, s, "tree_fp32")
        ctx.set_tensor_cores(3)
        ytp = ctx.matvec(x, s, "tree_fp32")
        assert ctx.device_errors() == 0
        ctx.set_tensor_cores(False)
        yfp = ctx.matvec(x, s, "tree_fp32")
        y64 = ctx.matvec(x, s, "tree_fp64")
    for b in range(B):
        _agree(ytc[b], y64[b], 1e-5, b)
        _agree(yfp[b], y64[b], 1e-5, b)
        _agree(ytp[b], y64[b], 1e-5, b, tol_elem=3e-5)   # split operands: 22 of FP32's 24 bits
        _agree(ytc[b], yfp[b], 2e-5, b)
        _agree(ytp[b], yfp[b], 2e-5, b, tol_elem=4e-5)


def test_bounded_wait_gives_up(lspr):
    # the pipeline waits of the tensor-core kernels end after about a second when nothing
    # arrives, raise the abort flag, and leave the context usable (a product still matches)
    v, t = I.icosphere(2, 10.0)
    n = len(t)
    s = I.drude_eps(np.array([370.0, 390.0])) / I.EPS_WATER
    x = I.random_complex(2 * n, seed=43, batch=2)
    with lspr.Context(0) as ctx:
        r = ctx.selftest_wait_timeout()
        assert r["succeeded"] == 0 and r["abort"] == 1
        assert 900 <= r["ms"] <= 5000
        ctx.mesh_upload(v, t)
        ctx.tree_build(0.6, 4, 16)
        ytc = ctx.matvec(x, s, "tree_fp32")
        assert ctx.device_errors() == 0
        ctx.set_tensor_cores(False)
        yfp = ctx.matvec(x, s, "tree_fp32")
    for b in range(2):
        assert _rel(ytc[b], yfp[b]) < 1e-5, b


def test_timed_out_wait_is_a_status(lspr):
    # the same bounded wait inside the real tensor-core M2P: with the check enabled it runs out
    # before any work is issued, and the product and the solve report LSPR_E_TIMEOUT (6); with
    # it disabled again, the same context gives the complete product
    v, t = I.icosphere(2, 10.0)
    n = len(t)
    lam = np.array([370.0, 390.0])
    s = I.drude_eps(lam) / I.EPS_WATER
    x = I.random_complex(2 * n, seed=44, batch=2)
    with lspr.Context(0) as ctx:
        ctx.mesh_upload(v, t)
        ctx.tree_build(0.6, 4, 16)
        y0 = ctx.matvec(x, s, "tree_fp32")
        assert ctx.device_errors() == 0
        ctx.selftest_gate_waits(True)
        with pytest.raises(lspr.LsprError) as e:
            ctx.matvec(x, s, "tree_fp32")
        assert e.value.status == 6
        assert ctx.device_errors() > 0
        with pytest.raises(lspr.LsprError) as e:
            ctx.solve(I.drude_eps(lam), I.EPS_WATER, lam, tol=1e-8, restart=2, maxiter=2, mode="tree_fp32")
        assert e.value.status == 6
        ctx.selftest_gate_waits(False)
        nerr = ctx.device_errors()
        y1 = ctx.matvec(x, s, "tree_fp32")
        assert ctx.device_errors() == nerr
    # the FP32 far field accumulates with atomics in a run-dependent order
    assert _rel(y0, y1) < 1e-6


def test_tensor_core_solve(lspr):
    v, t = I.icosphere(3, 10.0)
    lam = I.wavelengths(360, 400, 12)
    ep = I.drude_eps(lam)
    with lspr.Context(0) as ctx:
        ctx.mesh_upload(v, t)
        ctx.tree_build(0.4, 7, 64)
        a = ctx.solve(ep, I.EPS_WATER, lam, tol=1e-9, mode="tree_fp32", refine=True, restart=60, maxiter=3000)
        assert ctx.device_errors() == 0
        ctx.set_tensor_cores(False)
        b = ctx.solve(ep, I.EPS_WATER, lam, tol=1e-9, mode="tree_fp32", refine=True, restart=60, maxiter=3000)
    assert np.all(a.status == 0) and np.all(b.status == 0)
    assert np.max(np.abs(a.sigma_ext - b.sigma_ext) / b.sigma_ext) < 1e-7
