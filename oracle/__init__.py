"""Plain FP64 CPU oracle of the quasistatic LSPR boundary-element method.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by ``bench.py``'s CPU-baseline / reference legs, never by the product
package.  The arithmetic lives in ``lspr_oracle.c`` (plain C, OpenMP over
rows); this module only compiles it with gcc and marshals numpy arrays.

Every function cites the passage of arXiv:1812.10722 it follows; the readings
of points the paper leaves open are listed at the top of ``lspr_oracle.c``.
Parity status: every function here is pinned by ``tests/test_oracle_*.py``
(closed forms, exactness, brute-force quadrature, invariants).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lspr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblspr_oracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_intp = ctypes.POINTER(ctypes.c_int)
_i64 = ctypes.c_int64
_d = ctypes.c_double
_i = ctypes.c_int


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            L.oracle_quad_rule.argtypes = [_i, _dp, _dp]
            L.oracle_quad_rule.restype = _i
            L.oracle_panels.argtypes = [_dp, _ip, _i64, _dp, _dp, _dp, _dp]
            L.oracle_self_V.argtypes = [_dp, _dp, _dp, _dp]
            L.oracle_self_V.restype = _d
            L.oracle_entries.argtypes = [_dp, _ip, _i64, _i, _i, _d, _i64, _i64, _dp, _dp]
            L.oracle_entries.restype = _i
            L.oracle_near_pairs.argtypes = [_dp, _ip, _i64, _d, _i64p]
            L.oracle_near_pairs.restype = _i64
            L.oracle_matvec.argtypes = [_dp, _ip, _i64, _i, _i, _d, _i, _dp, _dp, _dp, _i]
            L.oracle_matvec.restype = _i
            L.oracle_rhs.argtypes = [_dp, _ip, _i64, _i, _i, _d, _i, _dp, _d, _d, _dp, _dp, _i]
            L.oracle_rhs.restype = _i
            L.oracle_lu_solve.argtypes = [_i64, _dp, _dp]
            L.oracle_lu_solve.restype = _i
            L.oracle_gmres.argtypes = [_dp, _ip, _i64, _i, _i, _d, _d, _d, _dp, _dp, _d, _i, _i,
                                       _intp, _dp, _i]
            L.oracle_gmres.restype = _i
            L.oracle_dipole.argtypes = [_dp, _ip, _i64, _i64, _i64, _dp, _d, _d, _d, _d, _dp, _dp]
            L.oracle_sigma_ext.argtypes = [_dp, _d, _d, _dp, _d]
            L.oracle_sigma_ext.restype = _d
            L.oracle_sigma_closed_form.argtypes = [_d, _d, _d, _d, _d, _d]
            L.oracle_sigma_closed_form.restype = _d
            L.oracle_solve.argtypes = [_dp, _ip, _i64, _i, _i, _d, _i, _dp, _d, _d, _dp, _dp, _d, _i,
                                       _i, _dp, _dp, _intp, _i]
            L.oracle_solve.restype = _i
            L.oracle_matvec_multi.argtypes = [_dp, _ip, _ip, _i64, _i, _i, _i, _d, _i, _dp, _dp, _dp, _i]
            L.oracle_matvec_multi.restype = _i
            L.oracle_rhs_multi.argtypes = [_dp, _ip, _ip, _i64, _i, _i, _i, _d, _i, _dp, _d, _d, _dp, _dp, _i]
            L.oracle_rhs_multi.restype = _i
            L.oracle_gmres_multi.argtypes = [_dp, _ip, _ip, _i64, _i, _i, _i, _d, _dp, _dp, _dp, _d, _i, _i,
                                             _intp, _dp, _i]
            L.oracle_gmres_multi.restype = _i
            L.oracle_dipole_surface.argtypes = [_dp, _ip, _ip, _i64, _i, _dp, _d, _d, _d, _d, _dp, _dp]
            L.oracle_solve_multi.argtypes = [_dp, _ip, _ip, _i64, _i, _i, _i, _d, _i, _dp, _d, _d, _dp, _dp, _d,
                                             _i, _i, _dp, _dp, _intp, _i, _i64, _dp, _ip]
            L.oracle_solve_multi.restype = _i
            L.oracle_rhs_charges.argtypes = [_dp, _ip, _ip, _i64, _i, _i, _dp, _i64, _dp, _ip, _dp]
            L.oracle_rhs_charges.restype = _i
            L.oracle_matvec_rows.argtypes = [_dp, _ip, _i64, _i, _i, _d, _i, _dp, _dp, _dp, _i64, _i64, _i]
            L.oracle_matvec_rows.restype = _i
            L.oracle_solve_batch.argtypes = [_dp, _ip, _ip, _i64, _i, _i, _i, _d, _i, _dp, _d, _d, _dp, _dp, _d,
                                             _i, _i, _dp, _dp, _intp, _dp, _i]
            L.oracle_solve_batch.restype = _i
            _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _ptr(a, t=_dp):
    return a.ctypes.data_as(t)


def _mesh(verts, tris):
    v = _f64(verts)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    return v, t, len(t)


def quad_rule(K: int):
    """Dunavant rule with K points: (barycentric [K,3], weights [K] summing to 1).

    Sec. II.C "Integral evaluation": K in {1,3,4} far, K_fine in {19,25,37} near.
    """
    bary = np.zeros((37, 3))
    w = np.zeros(37)
    k = lib().oracle_quad_rule(K, _ptr(bary), _ptr(w))
    if k < 0:
        raise ValueError(f"no rule with {K} points")
    return bary[:k].copy(), w[:k].copy()


def panels(verts, tris):
    """Centroids, unit outward normals, areas, L = sqrt(2 A) (Sec. II.C)."""
    v, t, n = _mesh(verts, tris)
    c = np.zeros((n, 3)); nrm = np.zeros((n, 3)); a = np.zeros(n); L = np.zeros(n)
    lib().oracle_panels(_ptr(v), _ptr(t, _ip), n, _ptr(c), _ptr(nrm), _ptr(a), _ptr(L))
    return c, nrm, a, L


def self_V(v0, v1, v2, x):
    """(1/4pi) int_T 1/|x-y| dA, exact, x in the panel (singular integral, Sec. II.C)."""
    a = [_f64(q) for q in (v0, v1, v2, x)]
    return lib().oracle_self_V(*[_ptr(q) for q in a])


def entries(verts, tris, K=4, K_fine=19, threshold=0.5, rows=None):
    """Rows of V_ij and K_ij (Eq. layers_element) with the three-regime rule."""
    v, t, n = _mesh(verts, tris)
    i0, i1 = (0, n) if rows is None else rows
    V = np.zeros((i1 - i0, n)); Kd = np.zeros((i1 - i0, n))
    rc = lib().oracle_entries(_ptr(v), _ptr(t, _ip), n, K, K_fine, threshold, i0, i1, _ptr(V), _ptr(Kd))
    if rc:
        raise RuntimeError(f"oracle_entries failed ({rc})")
    return V, Kd


def near_pairs(verts, tris, threshold=0.5):
    """Per-row count of near-singular panels j != i (L_j/|c_i-c_j| >= threshold)."""
    v, t, n = _mesh(verts, tris)
    cnt = np.zeros(n, dtype=np.int64)
    tot = lib().oracle_near_pairs(_ptr(v), _ptr(t, _ip), n, threshold, _ptr(cnt, _i64p))
    return tot, cnt


def matvec(verts, tris, x, s, K=4, K_fine=19, threshold=0.5, nthreads=0):
    """y = A(s) x for Eq. matrix_lspr; x [2n] or [B,2n] complex, s scalar or [B]."""
    v, t, n = _mesh(verts, tris)
    x = _c128(x)
    squeeze = x.ndim == 1
    x2 = x.reshape(-1, 2 * n)
    B = x2.shape[0]
    s = _c128(np.broadcast_to(np.asarray(s, np.complex128), (B,)))
    y = np.zeros_like(x2)
    rc = lib().oracle_matvec(_ptr(v), _ptr(t, _ip), n, K, K_fine, threshold, B, _ptr(s.view(np.float64)),
                             _ptr(x2.view(np.float64)), _ptr(y.view(np.float64)), nthreads)
    if rc:
        raise RuntimeError(f"oracle_matvec failed ({rc})")
    return y[0] if squeeze else y


def rhs(verts, tris, eps_in, eps_out, E0=(0.0, 0.0, 1.0), K=4, K_fine=19, threshold=0.5, nthreads=0):
    """Right-hand side of Eq. matrix_lspr, [B,2n] for eps_in of shape [B]."""
    v, t, n = _mesh(verts, tris)
    e = _c128(np.atleast_1d(eps_in))
    B = len(e)
    b = np.zeros((B, 2 * n), np.complex128)
    E = _f64(E0)
    eo = complex(eps_out)
    rc = lib().oracle_rhs(_ptr(v), _ptr(t, _ip), n, K, K_fine, threshold, B, _ptr(e.view(np.float64)),
                          eo.real, eo.imag, _ptr(E), _ptr(b.view(np.float64)), nthreads)
    if rc:
        raise RuntimeError(f"oracle_rhs failed ({rc})")
    return b


def lu_solve(A, b):
    """Dense complex LU with partial pivoting (solves A x = b)."""
    A = _c128(A).copy()
    b = _c128(b).copy()
    rc = lib().oracle_lu_solve(len(b), _ptr(A.view(np.float64)), _ptr(b.view(np.float64)))
    if rc:
        raise RuntimeError("singular matrix")
    return b


def gmres(verts, tris, b, s, tol=1e-8, restart=100, maxiter=1000, K=4, K_fine=19, threshold=0.5,
          nthreads=0):
    """Complex GMRES(restart), right block-Jacobi preconditioner; returns (x, iters, relres, ok)."""
    v, t, n = _mesh(verts, tris)
    b = _c128(b)
    x = np.zeros(2 * n, np.complex128)
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0)
    s = complex(s)
    st = lib().oracle_gmres(_ptr(v), _ptr(t, _ip), n, K, K_fine, threshold, s.real, s.imag,
                            _ptr(b.view(np.float64)), _ptr(x.view(np.float64)), tol, restart, maxiter,
                            ctypes.byref(it), ctypes.byref(rr), nthreads)
    return x, it.value, rr.value, st == 0


def dipole(verts, tris, x, eps_in, eps_out, E0=(0.0, 0.0, 1.0), panels_range=None):
    """Dipole moment (Eq. dipole_def_gauss_i_final, outward-normal sign reading)."""
    v, t, n = _mesh(verts, tris)
    p0, p1 = (0, n) if panels_range is None else panels_range
    x = _c128(x)
    p = np.zeros(3, np.complex128)
    e1, e2 = complex(eps_in), complex(eps_out)
    E = _f64(E0)
    lib().oracle_dipole(_ptr(v), _ptr(t, _ip), n, p0, p1, _ptr(x.view(np.float64)), e1.real, e1.imag,
                        e2.real, e2.imag, _ptr(E), _ptr(p.view(np.float64)))
    return p


def sigma_ext(p, eps_out, lambda_nm, E0=(0.0, 0.0, 1.0)):
    """Extinction cross-section (nm^2) from the dipole (Eqs. scat_efield_long_range, cext_fwa)."""
    p = _c128(p)
    e2 = complex(eps_out)
    E = _f64(E0)
    return lib().oracle_sigma_ext(_ptr(p.view(np.float64)), e2.real, e2.imag, _ptr(E), float(lambda_nm))


def sigma_closed_form(R, eps_p, eps_m, lambda_nm):
    """Eq. an_sol: analytic extinction cross-section of a sphere of radius R (nm^2)."""
    ep, em = complex(eps_p), complex(eps_m)
    return lib().oracle_sigma_closed_form(float(R), ep.real, ep.imag, em.real, em.imag, float(lambda_nm))


def solve(verts, tris, eps_in, eps_out, lambda_nm, E0=(0.0, 0.0, 1.0), tol=1e-8, restart=100,
          maxiter=1000, K=4, K_fine=19, threshold=0.5, nthreads=0):
    """RHS + GMRES + dipole + sigma_ext for each wavelength; returns (dipoles [B,3], sigma [B], iters [B], n_bad)."""
    v, t, n = _mesh(verts, tris)
    e = _c128(np.atleast_1d(eps_in))
    lam = _f64(np.atleast_1d(lambda_nm))
    B = len(e)
    dip = np.zeros((B, 3), np.complex128)
    sig = np.zeros(B)
    its = np.zeros(B, dtype=np.int32)
    E = _f64(E0)
    e2 = complex(eps_out)
    bad = lib().oracle_solve(_ptr(v), _ptr(t, _ip), n, K, K_fine, threshold, B, _ptr(e.view(np.float64)),
                             e2.real, e2.imag, _ptr(E), _ptr(lam), tol, restart, maxiter,
                             _ptr(dip.view(np.float64)), _ptr(sig), its.ctypes.data_as(_intp), nthreads)
    return dip, sig, its, bad


# ------------------------------------------------------- several surfaces
# Eqs. integral_eq_lspr_system / matrix_multi: surfaces t = 0..S-1 (surf[i] = surface of
# panel i) with permittivities eps_t in one host eps_out; surface 0 is the particle whose
# sigma_ext is reported.


def _surf(surf, n):
    sf = np.ascontiguousarray(surf, dtype=np.int32)
    if sf.shape != (n,):
        raise ValueError("surf must hold one surface index per panel")
    return sf, int(sf.max()) + 1


def matvec_multi(verts, tris, surf, x, s, K=4, K_fine=19, threshold=0.5, nthreads=0):
    """y = A(s) x of several surfaces; x [2n] or [B,2n]; s [S] or [B,S] (eps_t/eps_out)."""
    v, t, n = _mesh(verts, tris)
    sf, S = _surf(surf, n)
    x = _c128(x)
    squeeze = x.ndim == 1
    x2 = x.reshape(-1, 2 * n)
    B = x2.shape[0]
    s = _c128(np.broadcast_to(np.asarray(s, np.complex128).reshape(-1, S), (B, S)))
    y = np.zeros_like(x2)
    rc = lib().oracle_matvec_multi(_ptr(v), _ptr(t, _ip), _ptr(sf, _ip), n, S, K, K_fine, threshold, B,
                                   _ptr(s.view(np.float64)), _ptr(x2.view(np.float64)), _ptr(y.view(np.float64)),
                                   nthreads)
    if rc:
        raise RuntimeError(f"oracle_matvec_multi failed ({rc})")
    return y[0] if squeeze else y


def rhs_multi(verts, tris, surf, eps_in, eps_out, E0=(0.0, 0.0, 1.0), K=4, K_fine=19, threshold=0.5,
              nthreads=0):
    """Right-hand side of several surfaces, [B,2n] for eps_in of shape [S] or [B,S]."""
    v, t, n = _mesh(verts, tris)
    sf, S = _surf(surf, n)
    e = _c128(np.asarray(eps_in, np.complex128).reshape(-1, S))
    B = e.shape[0]
    b = np.zeros((B, 2 * n), np.complex128)
    eo = complex(eps_out)
    rc = lib().oracle_rhs_multi(_ptr(v), _ptr(t, _ip), _ptr(sf, _ip), n, S, K, K_fine, threshold, B,
                                _ptr(e.view(np.float64)), eo.real, eo.imag, _ptr(_f64(E0)), _ptr(b.view(np.float64)),
                                nthreads)
    if rc:
        raise RuntimeError(f"oracle_rhs_multi failed ({rc})")
    return b


def gmres_multi(verts, tris, surf, b, s, tol=1e-8, restart=100, maxiter=1000, K=4, K_fine=19, threshold=0.5,
                nthreads=0):
    """GMRES of several surfaces for one wavelength, s [S]; returns (x, iters, relres, ok)."""
    v, t, n = _mesh(verts, tris)
    sf, S = _surf(surf, n)
    b = _c128(b)
    x = np.zeros(2 * n, np.complex128)
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0)
    s = _c128(np.asarray(s, np.complex128).reshape(S))
    st = lib().oracle_gmres_multi(_ptr(v), _ptr(t, _ip), _ptr(sf, _ip), n, S, K, K_fine, threshold,
                                  _ptr(s.view(np.float64)), _ptr(b.view(np.float64)), _ptr(x.view(np.float64)),
                                  tol, restart, maxiter, ctypes.byref(it), ctypes.byref(rr), nthreads)
    return x, it.value, rr.value, st == 0


def dipole_surface(verts, tris, surf, x, surface, eps_in, eps_out, E0=(0.0, 0.0, 1.0)):
    """Dipole moment of the panels of one surface (eps_in: that surface's permittivity)."""
    v, t, n = _mesh(verts, tris)
    sf, _ = _surf(surf, n)
    x = _c128(x)
    p = np.zeros(3, np.complex128)
    e1, e2 = complex(eps_in), complex(eps_out)
    lib().oracle_dipole_surface(_ptr(v), _ptr(t, _ip), _ptr(sf, _ip), n, int(surface), _ptr(x.view(np.float64)),
                                e1.real, e1.imag, e2.real, e2.imag, _ptr(_f64(E0)), _ptr(p.view(np.float64)))
    return p


def _charges(charges, charge_surf):
    if charges is None:
        return 0, None, None
    q = np.ascontiguousarray(np.asarray(charges, np.float64).reshape(-1, 4))
    qs = np.ascontiguousarray(np.asarray(charge_surf, np.int32).reshape(-1))
    if qs.shape[0] != q.shape[0]:
        raise ValueError("one surface index per charge")
    return q.shape[0], q, qs


def rhs_charges(verts, tris, surf, eps_in, charges, charge_surf):
    """Coulomb term of point charges inside surfaces on their interior rows, [B,2n]: charge
    (x, y, z, q) inside surface t adds q / (4 pi eps_t |c_i - r|) to row i of every panel of t
    (Eqs. integral_eq_lspr_system, matrix_multi).  eps_in [S] or [B,S]."""
    v, t, n = _mesh(verts, tris)
    sf, S = _surf(surf, n)
    e = _c128(np.asarray(eps_in, np.complex128).reshape(-1, S))
    B = e.shape[0]
    nq, q, qs = _charges(charges, charge_surf)
    b = np.zeros((B, 2 * n), np.complex128)
    if nq == 0:
        return b
    rc = lib().oracle_rhs_charges(_ptr(v), _ptr(t, _ip), _ptr(sf, _ip), n, S, B, _ptr(e.view(np.float64)), nq,
                                  _ptr(q), _ptr(qs, _ip), _ptr(b.view(np.float64)))
    if rc:
        raise RuntimeError(f"oracle_rhs_charges failed ({rc})")
    return b


def solve_multi(verts, tris, surf, eps_in, eps_out, lambda_nm, E0=(0.0, 0.0, 1.0), tol=1e-8, restart=100,
                maxiter=1000, K=4, K_fine=19, threshold=0.5, nthreads=0, charges=None, charge_surf=None):
    """Several surfaces: RHS (+ point charges, rhs_charges) + GMRES + dipole and sigma_ext of
    surface 0 per wavelength; eps_in [B,S]; returns (dipoles [B,3], sigma [B], iters [B], n_bad)."""
    v, t, n = _mesh(verts, tris)
    sf, S = _surf(surf, n)
    nq, q, qs = _charges(charges, charge_surf)
    e = _c128(np.asarray(eps_in, np.complex128).reshape(-1, S))
    lam = _f64(np.atleast_1d(lambda_nm))
    B = e.shape[0]
    dip = np.zeros((B, 3), np.complex128)
    sig = np.zeros(B)
    its = np.zeros(B, dtype=np.int32)
    e2 = complex(eps_out)
    bad = lib().oracle_solve_multi(_ptr(v), _ptr(t, _ip), _ptr(sf, _ip), n, S, K, K_fine, threshold, B,
                                   _ptr(e.view(np.float64)), e2.real, e2.imag, _ptr(_f64(E0)), _ptr(lam), tol,
                                   restart, maxiter, _ptr(dip.view(np.float64)), _ptr(sig), its.ctypes.data_as(_intp),
                                   nthreads, nq, _ptr(q) if nq else None, _ptr(qs, _ip) if nq else None)
    return dip, sig, its, bad


def solve_batch(verts, tris, eps_in, eps_out, lambda_nm, surf=None, E0=(0.0, 0.0, 1.0), tol=1e-8, restart=100,
                maxiter=1000, K=4, K_fine=19, threshold=0.5, nthreads=0):
    """The solve of ``solve`` (``surf`` None) or ``solve_multi`` for B wavelengths in lockstep, every
    operator application shared across the wavelengths still iterating (Sec. II.D GMRES; the matrix
    entries of Eq. layers_element are evaluated once per row for all of them).  Each wavelength's
    result is bit for bit the one-at-a-time result.  eps_in: [B] or [B, S] complex.
    Returns (dipoles [B,3], sigma [B], iters [B], relres [B], n_bad)."""
    v, t, n = _mesh(verts, tris)
    if surf is None:
        sf, S = None, 1
    else:
        sf, S = _surf(surf, n)
    lam = _f64(np.atleast_1d(lambda_nm))
    B = len(lam)
    e = _c128(np.asarray(eps_in, np.complex128).reshape(B, S))
    dip = np.zeros((B, 3), np.complex128)
    sig = np.zeros(B)
    its = np.zeros(B, dtype=np.int32)
    rr = np.zeros(B)
    E = _f64(E0)
    e2 = complex(eps_out)
    bad = lib().oracle_solve_batch(_ptr(v), _ptr(t, _ip), _ptr(sf, _ip) if sf is not None else None, n, S, K,
                                   K_fine, threshold, B, _ptr(e.view(np.float64)), e2.real, e2.imag, _ptr(E),
                                   _ptr(lam), tol, restart, maxiter, _ptr(dip.view(np.float64)), _ptr(sig),
                                   its.ctypes.data_as(_intp), _ptr(rr), nthreads)
    if bad < 0:
        raise RuntimeError("oracle_solve_batch: bad quadrature rule")
    return dip, sig, its, rr, bad


def matvec_rows(verts, tris, x, s, rows, K=4, K_fine=19, threshold=0.5, nthreads=0):
    """Rows [i0, i1) (panels) of y = A(s) x (Eq. matrix_lspr), top and bottom; x [2n] or [B, 2n].
    Returns y shaped like x with only those rows filled (the rest zero)."""
    v, t, n = _mesh(verts, tris)
    x = _c128(x)
    squeeze = x.ndim == 1
    x2 = x.reshape(-1, 2 * n)
    B = x2.shape[0]
    s = _c128(np.broadcast_to(np.atleast_1d(np.asarray(s, np.complex128)), (B,)))
    y = np.zeros_like(x2)
    i0, i1 = rows
    rc = lib().oracle_matvec_rows(_ptr(v), _ptr(t, _ip), n, K, K_fine, threshold, B, _ptr(s.view(np.float64)),
                                  _ptr(x2.view(np.float64)), _ptr(y.view(np.float64)), int(i0), int(i1), nthreads)
    if rc:
        raise RuntimeError(f"oracle_matvec_rows failed ({rc})")
    return y[0] if squeeze else y

