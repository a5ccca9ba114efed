"""Oracle of several surfaces (Eqs. integral_eq_lspr_system and matrix_multi) against
what the physics fixes without it: one surface reduces to Eq. matrix_lspr exactly; two
distant spheres couple as point dipoles; an analyte of the host's own permittivity is not
there (its effect vanishes under mesh refinement); a distant analyte has no effect."""
import numpy as np
import pytest

from paper_1812_10722_gb300 import inputs as I


def test_one_surface_is_the_single_interface_operator(oracle):
    v, t = I.icosphere(2, 10.0)
    n = len(t)
    surf = np.zeros(n, np.int32)
    lam = np.array([380.0, 400.0])
    ep = I.drude_eps(lam)
    x = I.random_complex(2 * n, seed=5, batch=2)
    s = ep / I.EPS_WATER
    assert np.array_equal(oracle.matvec_multi(v, t, surf, x, s.reshape(2, 1)), oracle.matvec(v, t, x, s))
    assert np.array_equal(oracle.rhs_multi(v, t, surf, ep.reshape(2, 1), I.EPS_WATER),
                          oracle.rhs(v, t, ep, I.EPS_WATER))
    d1, s1, _, _ = oracle.solve_multi(v, t, surf, ep.reshape(2, 1), I.EPS_WATER, lam, tol=1e-10)
    d0, s0, _, _ = oracle.solve(v, t, ep, I.EPS_WATER, lam, tol=1e-10)
    assert np.array_equal(s1, s0) and np.array_equal(d1, d0)


@pytest.mark.parametrize("E0,sign", [((0.0, 0.0, 1.0), 2.0), ((1.0, 0.0, 0.0), -1.0)])
def test_two_spheres_couple_as_point_dipoles(oracle, E0, sign):
    # sphere 1 at distance d along z: its dipole field at sphere 0 is 2p/(4 pi eps_m d^3)
    # along the axis and -p/(4 pi eps_m d^3) across it, so p0 / p_single = 1 / (1 - c f (a/d)^3),
    # c = 2 or -1, f = (eps - eps_m)/(eps + 2 eps_m); higher multipoles add O((a/d)^2) of that
    a, d, ep, em = 10.0, 40.0, 2.25, 1.0
    vs, ts = I.icosphere(2, a)
    p1, _, _, _ = oracle.solve(vs, ts, ep, em, 500.0, E0=E0, tol=1e-11)
    v, t, surf = I.two_spheres(2, a, d)
    p2, _, _, _ = oracle.solve_multi(v, t, surf, [[ep, ep]], em, 500.0, E0=E0, tol=1e-11)
    k = int(np.argmax(np.abs(E0)))
    coupling = (p2[0][k] / p1[0][k]).real - 1.0
    f = (ep - em) / (ep + 2 * em)
    predicted = 1.0 / (1.0 - sign * f * (a / d) ** 3) - 1.0
    assert abs(coupling / predicted - 1.0) < 0.04
    assert np.max(np.abs(np.delete(p2[0], k))) < 1e-6 * abs(p2[0][k])


def test_transparent_analyte_vanishes_with_refinement(oracle):
    # eps_analyte = eps_host: no interface there; the discrete effect is a quadrature error
    # that falls with the analyte mesh (and stays far below a dielectric analyte's effect)
    lam, em = 380.0, I.EPS_WATER
    es = I.drude_eps(lam)
    vs, ts = I.icosphere(2, 10.0)
    _, s0, _, _ = oracle.solve(vs, ts, es, em, lam, tol=1e-10)
    effects = []
    for sub in (2, 3):
        v, t, surf = I.sensor_geometry(2, 10.0, analytes=(("+z", 3.0),), analyte_sub=sub)
        _, s1, _, _ = oracle.solve_multi(v, t, surf, [[es, em]], em, lam, tol=1e-10)
        _, s2, _, _ = oracle.solve_multi(v, t, surf, [[es, 2.25]], em, lam, tol=1e-10)
        effects.append((abs(s1[0] - s0[0]) / s0[0], abs(s2[0] - s0[0]) / s0[0]))
    assert effects[1][0] < effects[0][0] / 2.5          # ~O(h^2)
    assert effects[1][0] < 0.1 * effects[1][1]


def test_distant_analyte_has_no_effect(oracle):
    lam, em = 380.0, I.EPS_WATER
    es = I.drude_eps(lam)
    vs, ts = I.icosphere(2, 10.0)
    _, s0, _, _ = oracle.solve(vs, ts, es, em, lam, tol=1e-10)
    dev = []
    for gap in (1.0, 3.0, 10.0, 30.0):
        v, t, surf = I.sensor_geometry(2, 10.0, analytes=(("+z", gap),), analyte_sub=2)
        _, s, _, _ = oracle.solve_multi(v, t, surf, [[es, 2.25]], em, lam, tol=1e-10)
        dev.append(abs(s[0] - s0[0]) / s0[0])
    assert all(dev[k + 1] < dev[k] for k in range(3))
    assert dev[-1] < 0.02 * dev[0]


def test_placements_keep_the_gap():
    for axis in ("+z", "-z", "+x", "-x", "+y", "-y"):
        v, t, surf = I.sensor_geometry(1, 10.0, analytes=((axis, 2.0),), analyte_sub=1)
        va = v[np.unique(t[surf == 1])]
        assert abs(np.min(np.linalg.norm(va, axis=1)) - 12.0) < 1e-9
        c = va.mean(axis=0)
        assert np.argmax(np.abs(c)) == "xyz".index(axis[1]) and np.sign(c[np.argmax(np.abs(c))]) == (1 if axis[0] == "+" else -1)
