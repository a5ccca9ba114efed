"""Writes the stored expected values under tests/golden/ by calling only the oracle.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
from paper_1812_10722_gb300 import inputs as I  # noqa: E402


def write(name, obj):
    with open(os.path.join(HERE, name), "w") as f:
        json.dump(obj, f, indent=2)
        f.write("\n")


def sphere1280():
    v, t = I.icosphere(3, 10.0)
    ep = I.drude_eps(380.0)
    dip, sig, its, bad = O.solve(v, t, ep, I.EPS_WATER, 380.0, tol=1e-10)
    assert bad == 0
    write("sphere1280_l380.json", dict(
        workload="icosphere subdivision 3 (1280 triangles), R = 10 nm, Drude silver in water, lambda = 380 nm, "
                 "E0 = z, K = 4, K_fine = 19, threshold 0.5, GMRES tol 1e-10",
        writer="tests/golden/make_golden.py (oracle only)",
        sigma_ext_nm2=float(sig[0]),
        dipole=[[float(z.real), float(z.imag)] for z in dip[0]],
        closed_form_nm2=O.sigma_closed_form(10.0, ep, I.EPS_WATER, 380.0),
        gmres_iterations=int(its[0])))


def sphere20480():
    v, t = I.icosphere(5, 10.0)
    ep = I.drude_eps(380.0)
    dip, sig, its, bad = O.solve(v, t, ep, I.EPS_WATER, 380.0, tol=1e-8)
    assert bad == 0
    write("sphere20480_l380.json", dict(
        workload="icosphere subdivision 5 (20480 triangles), R = 10 nm, Drude silver in water, lambda = 380 nm, "
                 "E0 = z, K = 4, K_fine = 19, threshold 0.5, GMRES tol 1e-8",
        writer="tests/golden/make_golden.py (oracle only)",
        sigma_ext_nm2=float(sig[0]),
        dipole=[[float(z.real), float(z.imag)] for z in dip[0]],
        closed_form_nm2=O.sigma_closed_form(10.0, ep, I.EPS_WATER, 380.0),
        gmres_iterations=int(its[0])))


def sphere81920_sweep64():
    """sigma_ext at four wavelengths of the 64-wavelength sweep over 350-420 nm on the 81920-panel
    sphere: the one nearest the dipole resonance (smallest |eps + 2 eps_m|), both ends and the middle.
    The four are solved in lockstep (oracle.solve_batch: every matrix entry is evaluated once per
    product for all of them; each result equals the one-at-a-time solve bit for bit)."""
    v, t = I.icosphere(6, 10.0)
    lam_all = I.wavelengths(350.0, 420.0, 64)
    k = int(np.argmin(np.abs(I.drude_eps(lam_all) + 2 * I.EPS_WATER)))
    idx = sorted({k, 0, 32, 63})
    lam = lam_all[idx]
    ep = I.drude_eps(lam)
    dip, sig, its, rr, bad = O.solve_batch(v, t, ep, I.EPS_WATER, lam, tol=1e-8, restart=100)
    assert bad == 0
    write("sphere81920_sweep64.json", dict(
        workload="icosphere subdivision 6 (81920 triangles), R = 10 nm, Drude silver in water, 64 wavelengths "
                 "uniform over 350-420 nm (these are four of them), E0 = z, K = 4, K_fine = 19, threshold 0.5, "
                 "GMRES tol 1e-8, restart 100",
        writer="tests/golden/make_golden.py (oracle only)",
        sweep_index=[int(i) for i in idx],
        resonance_index=k,
        lambda_nm=[float(x) for x in lam],
        sigma_ext_nm2=[float(s) for s in sig],
        dipole=[[[float(z.real), float(z.imag)] for z in d] for d in dip],
        closed_form_nm2=[O.sigma_closed_form(10.0, e, I.EPS_WATER, L) for e, L in zip(ep, lam)],
        gmres_iterations=[int(i) for i in its],
        relative_residual=[float(r) for r in rr]))


if __name__ == "__main__":
    which = sys.argv[1:] or ["sphere1280"]
    for w in which:
        globals()[w]()
