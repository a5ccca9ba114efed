"""The oracle's lockstep solve of several wavelengths (one shared operator application per
Arnoldi step) against the one-wavelength-at-a-time solve, which the other oracle pins tie to
the paper (Dense LU, Eq. an_sol, Table 6).  Each wavelength takes the same GMRES steps with
the same per-row accumulation order, so the results must agree bit for bit, also when the
wavelengths converge at different steps inside a restart cycle or hit the step limit."""
import numpy as np
import pytest

from paper_1812_10722_gb300 import inputs as I


@pytest.mark.parametrize("restart", [100, 7])
def test_batch_equals_one_at_a_time(oracle, restart):
    v, t = I.icosphere(2, 10.0)
    lam = np.array([350.0, 371.11, 385.0, 420.0])   # far from, at and past the dipole resonance
    ep = I.drude_eps(lam)
    d1, s1, i1, bad1 = oracle.solve(v, t, ep, I.EPS_WATER, lam, tol=1e-9, restart=restart)
    d2, s2, i2, rr, bad2 = oracle.solve_batch(v, t, ep, I.EPS_WATER, lam, tol=1e-9, restart=restart)
    assert bad1 == bad2 == 0
    assert np.array_equal(i1, i2)
    assert len(set(i1.tolist())) > 1            # the wavelengths stop at different steps
    assert np.array_equal(s1, s2) and np.array_equal(d1, d2)
    assert np.all(rr <= 1e-9)


def test_batch_step_limit(oracle):
    v, t = I.icosphere(2, 10.0)
    lam = np.array([360.0, 371.11])
    ep = I.drude_eps(lam)
    d1, s1, i1, bad1 = oracle.solve(v, t, ep, I.EPS_WATER, lam, tol=1e-14, restart=5, maxiter=12)
    d2, s2, i2, rr, bad2 = oracle.solve_batch(v, t, ep, I.EPS_WATER, lam, tol=1e-14, restart=5, maxiter=12)
    assert bad1 == bad2 == 2 and np.array_equal(i1, i2) and np.all(i2 == 12)
    assert np.array_equal(s1, s2) and np.array_equal(d1, d2)


def test_batch_several_surfaces(oracle):
    v, t, surf = I.sensor_geometry(2, 10.0, (("+z", 1.0),), 1)
    lam = np.array([365.0, 380.0, 400.0])
    e = np.full((3, 2), 2.25 + 0j)
    e[:, 0] = I.drude_eps(lam)
    d1, s1, i1, bad1 = oracle.solve_multi(v, t, surf, e, I.EPS_WATER, lam, tol=1e-9, restart=9)
    d2, s2, i2, rr, bad2 = oracle.solve_batch(v, t, e, I.EPS_WATER, lam, surf=surf, tol=1e-9, restart=9)
    assert bad1 == bad2 == 0 and np.array_equal(i1, i2)
    assert np.array_equal(s1, s2) and np.array_equal(d1, d2)


def test_row_block_of_the_product(oracle):
    # a block of rows of the product (used to time a bounded share of it) is those rows of the
    # whole product, bit for bit, for one and several right-hand sides
    v, t = I.icosphere(2, 10.0)
    n = len(t)
    lam = np.array([360.0, 380.0, 400.0])
    s = I.drude_eps(lam) / I.EPS_WATER
    x = I.random_complex(2 * n, seed=3, batch=3)
    y = oracle.matvec(v, t, x, s)
    yr = oracle.matvec_rows(v, t, x, s, (17, 101))
    rows = np.r_[17:101, n + 17:n + 101]
    assert np.array_equal(yr[:, rows], y[:, rows])
    assert not np.any(np.delete(yr, rows, axis=1))
    assert np.array_equal(oracle.matvec_rows(v, t, x[1], s[1], (0, n)), oracle.matvec(v, t, x[1], s[1]))
