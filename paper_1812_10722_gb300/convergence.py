"""Grid-convergence study and Richardson extrapolation (the verification method of
Sec. III.A, Table 6: sigma_ext on a sequence of meshes refined by a constant factor in
the panel count).

With a quantity f(N) = f* + c N^(-p) + ..., three meshes N, rN, r^2 N give the observed
order p = ln((f_1 - f_2) / (f_2 - f_3)) / ln r and the extrapolated value
f* ~ f_3 + (f_3 - f_2) / (r^p - 1), whose distance from f_3 estimates the discretisation
error of the finest mesh.  The solves run through the library (C ABI); this module only
drives them and does the arithmetic above.
"""
from __future__ import annotations

import math

import numpy as np


def observed_order(f1: float, f2: float, f3: float, ratio: float) -> float:
    """Order p of f(N) = f* + c N^-p from three values on meshes N, ratio N, ratio^2 N."""
    return math.log((f1 - f2) / (f2 - f3)) / math.log(ratio)


def richardson(f2: float, f3: float, ratio: float, order: float) -> float:
    """Extrapolated value from the two finest meshes (ratio between their panel counts)."""
    return f3 + (f3 - f2) / (ratio ** order - 1.0)


def grid_study(meshes, eps_in, eps_out, lambda_nm, E0=(0.0, 0.0, 1.0), ctx=None, tree=None, quad=None,
               **solve_kw):
    """sigma_ext on each mesh (verts, tris) of a sequence refined by a constant panel ratio,
    the observed order from the last three and the Richardson estimate.

    tree: None for the direct product, or (theta, P, Ncrit) for the treecode (then the
    solve's mode defaults to "tree_fp32" with refinement); quad: quadrature options of the
    mesh upload (K, K_fine, N_k, threshold)."""
    from . import lspr
    own = ctx is None
    ctx = ctx or lspr.Context(0)
    try:
        n, sig = [], []
        kw = dict(solve_kw)
        if tree is None:
            kw.setdefault("mode", "direct_fp64")
        else:
            kw.setdefault("mode", "tree_fp32")
            kw.setdefault("refine", True)
        for v, t in meshes:
            ctx.mesh_upload(v, t, **(quad or {}))
            if tree is not None:
                ctx.tree_build(*tree)
            r = ctx.solve(eps_in, eps_out, lambda_nm, E0=E0, **kw)
            n.append(len(t))
            sig.append(float(r.sigma_ext[0]))
    finally:
        if own:
            ctx.close()
    out = {"panels": n, "sigma_ext": sig}
    if len(sig) >= 3:
        ratio = n[-1] / n[-2]
        if not np.isclose(ratio, n[-2] / n[-3]):
            raise ValueError("the meshes must be refined by a constant panel ratio")
        p = observed_order(sig[-3], sig[-2], sig[-1], ratio)
        out.update(order=p, extrapolated=richardson(sig[-2], sig[-1], ratio, p), ratio=ratio)
        out["finest_error_estimate"] = abs(out["extrapolated"] - sig[-1]) / abs(out["extrapolated"])
    return out
