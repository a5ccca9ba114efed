"""Pins of the oracle's discrete layer operators (Eq. layers_element, Eq. matrix_lspr).

Each check follows from the mathematics, not from the oracle's own formulas:

* Gauss identity: the double layer of a constant over any closed surface,
  evaluated on the surface, is -1/2 (outward normals).  Checked on a sphere and
  on a non-spherical perturbed ellipsoid (which also catches a transposed K).
* Sphere eigen-relations of the layer operators (interior harmonics r^l Y_l,
  exterior r^-(l+1) Y_l):  V Y_l = a/(2l+1) Y_l,  K Y_l = -Y_l/(2(2l+1)).
* Conductor pin for V: on an ellipsoid the equilibrium density
  sigma ~ 1/sqrt(x^2/a^4 + y^2/b^4 + z^2/c^4) gives a constant potential whose
  value is (Q/(8 pi)) int_0^inf ds / sqrt((a^2+s)(b^2+s)(c^2+s)).  Catches a
  transposed V (the panel areas sit on the wrong index) or a wrong 1/(4 pi).
* Brute force on a tiny mesh (20-panel icosahedron): every off-diagonal entry
  against an independent adaptive-subdivision integral, within the accuracy of
  the K / K_fine rules.
"""
import numpy as np
import pytest
from scipy.integrate import quad

from paper_1812_10722_gb300 import inputs as I


@pytest.fixture(scope="module")
def sphere(oracle):
    v, t = I.icosphere(3, 10.0)
    V, K = oracle.entries(v, t)
    c, n, a, L = oracle.panels(v, t)
    return dict(v=v, t=t, V=V, K=K, c=c, n=n, a=a)


def test_gauss_identity_sphere(sphere):
    rs = sphere["K"].sum(1)
    assert np.max(np.abs(rs + 0.5)) < 2e-4


def test_gauss_identity_nonspherical(oracle):
    v, t = I.protein_like(3, axes=(7.0, 4.0, 4.0), seed=5)
    _, K = oracle.entries(v, t)
    rs = K.sum(1)
    assert np.median(np.abs(rs + 0.5)) < 5e-3
    # a transposed operator would give column sums here instead
    c, n, a, L = oracle.panels(v, t)
    assert np.median(np.abs(K.T.sum(1) + 0.5)) > 5 * np.median(np.abs(rs + 0.5))


def test_sphere_eigen_relations(sphere):
    R = 10.0
    c, V, K = sphere["c"], sphere["V"], sphere["K"]
    r = np.linalg.norm(c, axis=1)
    one = np.ones(len(c))
    # l = 0: V 1 = a, K 1 = -1/2 (panel centroids lie slightly inside the sphere)
    assert np.allclose(V @ one, R, rtol=3e-3)
    # l = 1 harmonic z/r and l = 2 harmonic (3z^2 - r^2)/r^2 sampled at the centroids
    for l, f in [(1, c[:, 2] / r), (2, (3 * c[:, 2] ** 2 - r ** 2) / r ** 2)]:
        vl = V @ f
        kl = K @ f
        coef_v = (vl @ f) / (f @ f)
        coef_k = (kl @ f) / (f @ f)
        assert abs(coef_v - R / (2 * l + 1)) < 5e-3 * R / (2 * l + 1)
        assert abs(coef_k + 1.0 / (2 * (2 * l + 1))) < 4e-2 / (2 * (2 * l + 1))
        # eigenvector: residual small compared with the vector
        assert np.linalg.norm(vl - coef_v * f) < 2e-2 * np.linalg.norm(coef_v * f)


def test_conductor_ellipsoid_single_layer(oracle):
    a, b, cax = 3.0, 2.0, 1.5
    v, t = I.ellipsoid(4, (a, b, cax))
    V, _ = oracle.entries(v, t)
    c, n, area, L = oracle.panels(v, t)
    # project the centroids onto the ellipsoid to evaluate the density there
    s = np.sqrt((c[:, 0] / a) ** 2 + (c[:, 1] / b) ** 2 + (c[:, 2] / cax) ** 2)
    p = c / s[:, None]
    sigma = 1.0 / (4 * np.pi * a * b * cax * np.sqrt((p[:, 0] / a ** 2) ** 2 + (p[:, 1] / b ** 2) ** 2
                                                     + (p[:, 2] / cax ** 2) ** 2))
    Q = 1.0
    phi_exact = Q / (8 * np.pi) * quad(lambda u: 1 / np.sqrt((a * a + u) * (b * b + u) * (cax * cax + u)),
                                       0, np.inf, epsabs=1e-13)[0]
    phi = V @ sigma
    assert abs(np.median(phi) / phi_exact - 1) < 5e-3
    assert np.std(phi) / phi_exact < 1e-2
    # transposed V gives a clearly non-constant potential on this non-uniform mesh
    assert np.std(V.T @ sigma) > 3 * np.std(phi)


def _brute_entry(x, tri, nrm, depth=6):
    """int over the flat triangle of G and dG/dn_y at x by 4^depth sub-triangles x 3-point rule."""
    tris = tri[None, :, :]
    for _ in range(depth):
        a, b, c = tris[:, 0], tris[:, 1], tris[:, 2]
        ab, bc, ca = (a + b) / 2, (b + c) / 2, (c + a) / 2
        tris = np.concatenate([np.stack([a, ab, ca], 1), np.stack([ab, b, bc], 1),
                               np.stack([ca, bc, c], 1), np.stack([ab, bc, ca], 1)])
    area = 0.5 * np.linalg.norm(np.cross(tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0]), axis=1)
    V = 0.0; Kd = 0.0
    for lam in ([2 / 3, 1 / 6, 1 / 6], [1 / 6, 2 / 3, 1 / 6], [1 / 6, 1 / 6, 2 / 3]):
        y = lam[0] * tris[:, 0] + lam[1] * tris[:, 1] + lam[2] * tris[:, 2]
        d = x[None, :] - y
        r = np.linalg.norm(d, axis=1)
        V += np.sum(area / 3 / r)
        Kd += np.sum(area / 3 * (d @ nrm) / r ** 3)
    return V / (4 * np.pi), Kd / (4 * np.pi)


def test_entries_against_brute_force_icosahedron(oracle):
    v, t = I.icosphere(0, 1.0)
    V, K = oracle.entries(v, t, K=4, K_fine=37)
    c, n, a, L = oracle.panels(v, t)
    tot, cnt = oracle.near_pairs(v, t)
    assert tot > 0
    worst_v = worst_k = 0.0
    for i in range(len(t)):
        for j in range(len(t)):
            if i == j:
                continue
            bv, bk = _brute_entry(c[i], v[t[j]], n[j])
            worst_v = max(worst_v, abs(V[i, j] - bv) / abs(bv))
            worst_k = max(worst_k, abs(K[i, j] - bk) / (abs(bv) + abs(bk)))
    assert worst_v < 2e-3 and worst_k < 2e-3, (worst_v, worst_k)
    # self entries: exact, K_ii = 0
    for i in range(len(t)):
        assert K[i, i] == 0.0


def test_near_rule_beats_far_rule(oracle):
    # the K_fine rule must be closer to the exact integral than the K rule on near panels
    v, t = I.icosphere(1, 1.0)
    Vc, Kc = oracle.entries(v, t, K=4, K_fine=4)
    Vf, Kf = oracle.entries(v, t, K=4, K_fine=37)
    c, n, a, L = oracle.panels(v, t)
    i = 0
    near = np.where(np.abs(Vf[i] - Vc[i]) > 0)[0]
    assert len(near) > 3
    for j in near[:6]:
        if j == i:
            continue
        bv, bk = _brute_entry(c[i], v[t[j]], n[j])
        assert abs(Vf[i, j] - bv) < abs(Vc[i, j] - bv)
