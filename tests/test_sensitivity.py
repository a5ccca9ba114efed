"""Host logic of the resonance-shift studies (Sec. III.B "Resonance frequency shift" and
"Sensitivity calculations"): the peak locator against exact parabolas and the closed-form
sphere spectrum (Eq. an_sol), and the study geometries' placements and gaps."""
import numpy as np
import pytest

from paper_1812_10722_gb300 import inputs as I
from paper_1812_10722_gb300 import sensitivity as SN


def test_peak_of_a_parabola_and_of_a_lorentzian_is_exact():
    lam = np.linspace(370, 400, 32)
    for p in (371.3, 385.0, 398.9):
        sig = 5.0 - 0.7 * (lam - p) ** 2
        assert abs(SN.peak_wavelength(lam, sig, reciprocal=False) - p) < 1e-9
        lor = 1.0 / (0.3 + 2.0 * (lam - p) ** 2)
        assert abs(SN.peak_wavelength(lam, lor) - p) < 1e-9


def test_peak_and_shift_of_the_closed_form_sphere(oracle):
    # the quasistatic sphere's extinction peak (Eq. an_sol) for Drude silver in water sits near
    # 370.62 nm, where Re(eps) = -2 eps_m; on the 32-wavelength grid over 370-400 nm (0.97 nm
    # apart) the reciprocal-parabola vertex finds it, and the shift of a displaced spectrum,
    # within 0.005 nm; the plain parabola misses it by ~0.1 nm and a 0.4-nm shift by ~0.1 nm
    lam = I.wavelengths(370, 400, 32)
    f = lambda x, d=0.0: oracle.sigma_closed_form(10.0, I.drude_eps(x - d), I.EPS_WATER, x - d)  # noqa: E731
    fine = np.linspace(369.5, 372.0, 25001)
    exact = fine[np.argmax([f(x) for x in fine])]
    assert abs(exact - 370.62) < 0.01
    sig = np.array([f(x) for x in lam])
    p0 = SN.peak_wavelength(lam, sig)
    assert abs(p0 - exact) < 0.005
    for d in (0.25, 0.4, 0.75):
        p = SN.peak_wavelength(lam, np.array([f(x, d) for x in lam]))
        assert abs((p - p0) - d) < 0.005, d
    assert abs(SN.peak_wavelength(lam, sig, reciprocal=False) - exact) > 0.05


def test_peak_needs_an_interior_maximum():
    lam = np.linspace(370, 400, 8)
    with pytest.raises(ValueError):
        SN.peak_wavelength(lam, lam, reciprocal=False)   # monotone: the parabola opens upwards
    with pytest.raises(ValueError):
        SN.peak_wavelength(lam, lam)                      # the largest sample at the grid's end
    with pytest.raises(ValueError):
        SN.peak_wavelength(lam, 1.0 + (lam - 385.0) ** 2, reciprocal=False)   # a minimum, not a peak
    with pytest.raises(ValueError):
        SN.peak_wavelength(lam[:2], lam[:2])


def test_study_geometries():
    g = SN.axis_geometries(1.0, sphere_sub=2, analyte_sub=1)
    assert list(g) == ["z_1nm", "x_1nm", "y_1nm"]
    for name, (v, t, s) in g.items():
        ax = "xyz".index(name[0])
        for k in (1, 2):
            va = v[np.unique(t[s == k])]
            c = va.mean(0)
            # the analyte sits on its axis (both signs), 1 nm from the sphere
            assert abs(c[ax]) > 10.0 and np.all(np.abs(np.delete(c, ax)) < 2.0)
            assert abs(np.min(np.linalg.norm(va, axis=1)) - 11.0) < 1e-9
    gg = SN.gap_geometries([0.5, 4.0], sphere_sub=2, analyte_sub=1)
    for (name, (v, t, s)), gap in zip(gg.items(), (0.5, 4.0)):
        assert int(s.max()) == 6
        for k in range(1, 7):
            va = v[np.unique(t[s == k])]
            assert abs(np.min(np.linalg.norm(va, axis=1)) - (10.0 + gap)) < 1e-9
