"""Point charges inside a surface (Eqs. integral_eq_lspr_system, matrix_multi: the Coulomb term
(1 / (4 pi eps_3)) sum_k q_k / |r - r_k| on the interior row of an analyte surface), pinned to
closed forms of a dielectric sphere (eps_in) in a host (eps_out) with no incident field:

- a centred charge (Born ion): the surface potential is q / (4 pi eps_out a) and the interior
  normal derivative -q / (4 pi eps_in a^2), uniform; the dipole vanishes by symmetry;
- an off-centre charge at distance d (Kirkwood): on the sphere the potential is
  sum_l (2l+1) q d^l / (4 pi (l eps_in + (l+1) eps_out) a^(l+1)) P_l(cos gamma).

Both follow from continuity of the potential and of eps dphi/dn across the surface; the
discrete solution converges to them as the panels shrink."""
import numpy as np
import pytest
from numpy.polynomial import legendre

import oracle
from paper_1812_10722_gb300 import inputs as I

EPS_IN, EPS_OUT = 2.25, 1.7689
A = 2.0


def _solve(sub, charges, surf_q):
    v, t = I.icosphere(sub, A)
    n = len(t)
    surf = np.zeros(n, np.int32)
    b = oracle.rhs_multi(v, t, surf, [EPS_IN], EPS_OUT, E0=(0.0, 0.0, 0.0))
    b = b + oracle.rhs_charges(v, t, surf, [EPS_IN], charges, surf_q)
    x, it, rr, ok = oracle.gmres_multi(v, t, surf, b[0], [EPS_IN / EPS_OUT], tol=1e-12, restart=200)
    assert ok
    return v, t, surf, x


def _centroids(v, t):
    return v[t].mean(axis=1)


@pytest.mark.parametrize("sub", [2, 3])
def test_born_ion(sub):
    q = 1.0
    v, t, surf, x = _solve(sub, [[0.0, 0.0, 0.0, q]], [0])
    n = len(t)
    phi, dphi = x[:n].real, x[n:].real
    phi0 = q / (4 * np.pi * EPS_OUT * A)
    dphi0 = -q / (4 * np.pi * EPS_IN * A * A)
    assert np.max(np.abs(x.imag)) < 1e-12
    # uniform over the panels of the symmetric mesh, and close to the closed form
    assert np.ptp(phi) < 0.02 * phi0 and np.ptp(dphi) < 0.05 * abs(dphi0)
    err = max(abs(phi.mean() / phi0 - 1), abs(dphi.mean() / dphi0 - 1))
    assert err < (0.025 if sub == 2 else 0.007), err   # second order: 1.5e-2, 3.8e-3 (phi)
    # the dipole of a centred charge vanishes by symmetry
    p = oracle.dipole_surface(v, t, surf, x, 0, EPS_IN, EPS_OUT, E0=(0.0, 0.0, 0.0))
    assert np.max(np.abs(p)) < 1e-10 * q * A


def _kirkwood(cosg, d, q=1.0, lmax=80):
    c = np.array([(2 * l + 1) * q * d ** l / (4 * np.pi * (l * EPS_IN + (l + 1) * EPS_OUT) * A ** (l + 1))
                  for l in range(lmax + 1)])
    return legendre.legval(cosg, c)


def test_kirkwood_offset_charge_converges():
    d = 0.5 * A
    errs = []
    for sub in (2, 3):
        v, t, surf, x = _solve(sub, [[0.0, 0.0, d, 1.0]], [0])
        n = len(t)
        c = _centroids(v, t)
        cosg = c[:, 2] / np.linalg.norm(c, axis=1)
        ref = _kirkwood(cosg, d)
        phi = x[:n].real
        errs.append(np.linalg.norm(phi - ref) / np.linalg.norm(ref))
    assert errs[1] < 0.007, errs          # 1.7e-2 at 320 panels, 4.3e-3 at 1280
    assert errs[1] < 0.35 * errs[0], errs  # second order


def test_charge_term_placement():
    # two spheres; a charge inside surface 1 touches only the interior rows of surface 1,
    # scaled by that surface's permittivity of each wavelength
    v, t, surf = I.two_spheres(2, 2.0, 6.0)
    n = len(t)
    eps = np.array([[-3.0 + 0.2j, 2.25], [-4.0 + 0.1j, 3.0 + 0.5j]])
    ch = [[0.0, 0.0, 6.5, 1.5]]
    b = oracle.rhs_charges(v, t, surf, eps, ch, [1])
    assert np.all(b[:, n:] == 0) and np.all(b[:, :n][:, surf == 0] == 0)
    c = _centroids(v, t)
    r = np.linalg.norm(c - np.array([0.0, 0.0, 6.5]), axis=1)
    for k in range(2):
        ref = 1.5 / (4 * np.pi * eps[k, 1] * r)
        got = b[k, :n]
        assert np.allclose(got[surf == 1], ref[surf == 1], rtol=1e-13, atol=0)
    with pytest.raises(RuntimeError):
        oracle.rhs_charges(v, t, surf, eps, ch, [2])


def test_charge_in_an_analyte_polarises_the_particle():
    # a centred charge q in an analyte sphere at distance D acts on the particle (radius R, eps_p)
    # through its exterior potential q / (4 pi eps_out r) (Born: independent of the analyte's
    # eps); the l = 1 part of that potential at the particle is the uniform field
    # -q / (4 pi eps_out D^2) z, so p = 4 pi eps_out R^3 f (-q / (4 pi eps_out D^2)) z with
    # f = (eps_p - eps_out) / (eps_p + 2 eps_out); mutual coupling enters at (R / D)^6 ~ 2e-5
    R, D, q = 2.0, 12.0, 50.0
    eps_p, eps_a = -8.0 + 0.3j, 2.25   # away from the resonance eps_p = -2 eps_out, which amplifies errors
    f = (eps_p - EPS_OUT) / (eps_p + 2 * EPS_OUT)
    p_ref = -R ** 3 * f * q / D ** 2
    errs = []
    for sub in (2, 3):
        v, t, surf = I.two_spheres(sub, R, D)
        n = len(t)
        eps = [eps_p, eps_a]
        b = oracle.rhs_charges(v, t, surf, eps, [[0.0, 0.0, D, q]], [1])
        x, it, rr, ok = oracle.gmres_multi(v, t, surf, b[0], [e / EPS_OUT for e in eps], tol=1e-12, restart=300)
        assert ok
        p = oracle.dipole_surface(v, t, surf, x, 0, eps_p, EPS_OUT, E0=(0.0, 0.0, 0.0))
        assert abs(p[0]) < 1e-9 * abs(p_ref) and abs(p[1]) < 1e-9 * abs(p_ref)   # axial symmetry
        errs.append(abs(p[2] - p_ref) / abs(p_ref))
    assert errs[1] < 0.02, errs            # 5.7e-2 at 2 x 320 panels, 1.5e-2 at 2 x 1280
    assert errs[1] < 0.35 * errs[0], errs  # second order
