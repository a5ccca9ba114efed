"""Resonance-shift studies of the sensor-analyte system through the library.

The paper's sensing results (Sec. III.B, "Resonance frequency shift" and "Sensitivity
calculations") compare the extinction spectrum of the bare particle with the spectrum when
analytes sit near it: the plasmon peak moves to longer wavelengths by an amount that falls
with the particle-analyte distance and depends on where the analytes sit relative to the
incident polarisation (along the field, z, against across it, x and y).  This module drives
those studies: every geometry is solved for a whole wavelength sweep in one batched call
(Eq. matrix_multi, lspr_solve), and the peak is located from the three samples around the
largest cross-section (the vertex of the parabola through their reciprocals, exact for a Lorentzian peak; the plain
parabola's vertex is reported beside it).

Only the library's public binding is used; nothing here computes a layer potential.
"""
from __future__ import annotations

import time

import numpy as np

from . import inputs as I


def peak_wavelength(lam, sigma, reciprocal: bool = True) -> float:
    """Wavelength of the extinction peak from the three samples around the largest one (the end
    samples' neighbours when the largest sits at an end).

    reciprocal (default): vertex of the parabola through 1/sigma.  Near the resonance the
    particle's cross-section is a Lorentzian (Eq. an_sol: Im of a pole at eps = -2 eps_m, with
    eps nearly linear in the wavelength there), whose reciprocal is a parabola, so the vertex is
    exact for a pure Lorentzian; on the 0.97-nm grid of a 32-wavelength sweep over 370-400 nm it
    finds the closed-form sphere's peak to about 1e-3 nm.  reciprocal=False: vertex of the
    parabola through sigma itself, which on a peak as sharp as silver's in water is off by up to
    a tenth of the grid spacing and underestimates shifts (0.28 nm for a 0.4-nm shift)."""
    lam = np.asarray(lam, float)
    sigma = np.asarray(sigma, float)
    if len(lam) < 3:
        raise ValueError("a peak needs at least three wavelengths")
    k = int(np.clip(np.argmax(sigma), 1, len(sigma) - 2))
    x = lam[k - 1:k + 2] - lam[k]
    y = sigma[k - 1:k + 2]
    if reciprocal:
        if np.any(y <= 0):
            raise ValueError("the reciprocal fit needs positive cross-sections")
        a, b, _ = np.polyfit(x, 1.0 / y, 2)
        if not a > 0:
            raise ValueError("no interior maximum among the sampled wavelengths")
    else:
        a, b, _ = np.polyfit(x, y, 2)
        if not a < 0:
            raise ValueError("no interior maximum among the sampled wavelengths")
    peak = float(lam[k] - b / (2 * a))
    if not lam[k - 1] <= peak <= lam[k + 1]:
        raise ValueError("the maximum is not bracketed by the sampled wavelengths")
    return peak


def sweep(ctx, verts, tris, surf, lam, eps_analyte=2.25, eps_out=I.EPS_WATER, tree=(0.5, 7, 512), tol=1e-6,
          restart=50, refine=True, maxiter=4000, mesh_opts=None):
    """sigma_ext(lambda) of the particle (surface 0) for one geometry: Drude silver particle,
    analytes of permittivity eps_analyte, one batched solve of every wavelength.
    Returns (sigma [B], seconds, max Arnoldi steps)."""
    lam = np.asarray(lam, float)
    mo = mesh_opts or {}
    t0 = time.perf_counter()
    if surf is None:
        ctx.mesh_upload(verts, tris, **mo)
        eps = I.drude_eps(lam)
    else:
        ctx.mesh_upload(verts, tris, surf_id=surf, **mo)
        S = int(np.max(surf)) + 1
        eps = np.full((len(lam), S), complex(eps_analyte), np.complex128)
        eps[:, 0] = I.drude_eps(lam)
    ctx.tree_build(*tree)
    r = ctx.solve(eps, eps_out, lam, tol=tol, restart=restart, maxiter=maxiter, mode="tree_fp32", refine=refine)
    return np.asarray(r.sigma_ext), time.perf_counter() - t0, int(np.max(r.iterations))


def shift_study(ctx, geometries, lam, sphere_sub, R=10.0, **kw):
    """Peak shift of every geometry against the bare sphere of the same mesh.
    geometries: {name: (verts, tris, surf)}.  Returns {"bare": {...}, name: {...}} with each
    entry's peak wavelength, shift (nm), peak cross-section, solve seconds and Arnoldi steps."""
    vb, tb = I.icosphere(sphere_sub, R)
    sb, secs, its = sweep(ctx, vb, tb, None, lam, **kw)
    pb, pb2 = peak_wavelength(lam, sb), peak_wavelength(lam, sb, reciprocal=False)
    out = {"bare": {"peak_nm": pb, "peak_nm_parabola": pb2, "peak_sigma_nm2": float(np.max(sb)),
                    "seconds": round(secs, 2), "arnoldi_steps": its, "panels": len(tb)}}
    for name, (v, t, s) in geometries.items():
        sg, secs, its = sweep(ctx, v, t, s, lam, **kw)
        p, p2 = peak_wavelength(lam, sg), peak_wavelength(lam, sg, reciprocal=False)
        out[name] = {"peak_nm": p, "shift_nm": p - pb, "shift_nm_parabola": p2 - pb2,
                     "peak_sigma_nm2": float(np.max(sg)), "seconds": round(secs, 2), "arnoldi_steps": its,
                     "panels": len(t), "surfaces": int(np.max(s)) + 1}
    return out


def gap_geometries(gaps, placements=("+x", "-x", "+y", "-y", "+z", "-z"), sphere_sub=7, analyte_sub=6, R=10.0):
    """One geometry per gap: the sphere with an analyte at that gap on every placement axis."""
    return {f"gap_{g:g}nm": I.sensor_geometry(sphere_sub, R, tuple((a, g) for a in placements), analyte_sub)
            for g in gaps}


def axis_geometries(gap=1.0, sphere_sub=6, analyte_sub=6, R=10.0):
    """Two analytes at the same gap on +-z (along the incident field), on +-x and on +-y."""
    return {f"{ax}_{gap:g}nm": I.sensor_geometry(sphere_sub, R, ((f"+{ax}", gap), (f"-{ax}", gap)), analyte_sub)
            for ax in ("z", "x", "y")}
