"""Richardson arithmetic of the grid-convergence driver, checked on sequences with a known
limit and order, and on the oracle's own grid study of the paper's Table 6 case."""
import numpy as np
import pytest

from paper_1812_10722_gb300 import convergence as C
from paper_1812_10722_gb300 import inputs as I


@pytest.mark.parametrize("p", [1.0, 2.0, 0.5])
def test_exact_power_law(p):
    f = lambda n: 3.0 + 7.0 * n ** -p
    f1, f2, f3 = f(100.0), f(400.0), f(1600.0)
    assert abs(C.observed_order(f1, f2, f3, 4.0) - p) < 1e-9
    assert abs(C.richardson(f2, f3, 4.0, p) - 3.0) < 1e-9


def test_paper_table6_sequence():
    # the paper's printed errors (Table 6, sigma_ext of the isolated sphere at N = 512, 2048,
    # 8192) as values relative to Eq. an_sol: first order in 1/N, and the Richardson
    # estimate from the two finest meshes is ten times closer to the closed form
    g = _golden("paper_table6_errors.json")
    f = [1.0 + e / 100.0 for e in g["percent_error"][:3]]
    p = C.observed_order(*f, 4.0)
    x = C.richardson(f[1], f[2], 4.0, p)
    assert 0.95 < p < 1.1
    assert abs(x - 1.0) < 0.1 * abs(f[2] - 1.0)


def _golden(name):
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as fh:
        return json.load(fh)


def test_tabulated_permittivity_hook():
    # a table generated from the Drude model: exact at the nodes, converging between them
    lam_t = np.linspace(340.0, 440.0, 11)
    nk = np.sqrt(I.drude_eps(lam_t))
    assert np.allclose(I.tabulated_eps(lam_t, lam_t, nk.real, nk.imag), I.drude_eps(lam_t), rtol=1e-12)
    lam = np.array([355.0, 372.5, 418.0])
    errs = []
    for m in (11, 41, 161):
        lt = np.linspace(340.0, 440.0, m)
        nk = np.sqrt(I.drude_eps(lt))
        errs.append(np.max(np.abs(I.tabulated_eps(lam, lt, nk.real, nk.imag) - I.drude_eps(lam))))
    assert errs[1] < errs[0] / 10 and errs[2] < errs[1] / 10   # second order in the spacing
    with pytest.raises(ValueError):
        I.tabulated_eps(330.0, lt, nk.real, nk.imag)
