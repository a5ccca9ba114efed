"""Seeded synthetic inputs: triangle meshes, permittivities, wavelengths, vectors.

This module generates the workloads only.  It holds none of the boundary-element
arithmetic (no Green's function, quadrature, operator, solver or observable), so
both the CPU oracle and the CUDA path can consume the same inputs without
sharing any of the method.

Workloads (stand-ins for the paper's meshes and tabulated dielectric data,
which are not available):

* sphere: icosahedron subdivided ``s`` times (20*4**s flat triangles), every
  new vertex pushed onto the sphere of radius R after each subdivision, faces
  counter-clockwise seen from outside (outward normals).  The paper's own grid
  sequence 512/2048/8192/32768 (8*4**s) is reproduced with :func:`octasphere`.
* permittivity of silver: Drude model eps(w) = eps_inf - wp^2/(w^2 + i g w)
  with hbar*w[eV] = 1239.84198 / lambda[nm]; host water eps_m = 1.7689.
* protein-like analytes: a subdivided octahedron mapped onto an ellipsoid and
  perturbed radially by a seeded random real spherical-harmonic series.
"""
from __future__ import annotations

import numpy as np

HC_EV_NM = 1239.84198          # hbar*c in eV*nm: photon energy [eV] = HC_EV_NM / lambda [nm]
EPS_WATER = 1.7689             # host permittivity used by the sphere workloads
DRUDE_AG = dict(eps_inf=3.7, wp=9.0, gamma=0.018)   # eV


def _orient_outward(verts: np.ndarray, tris: np.ndarray) -> np.ndarray:
    """Flip faces whose normal points towards the origin (star-shaped closed surfaces)."""
    v0, v1, v2 = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    nrm = np.cross(v1 - v0, v2 - v0)
    c = (v0 + v1 + v2) / 3.0
    flip = np.einsum("ij,ij->i", nrm, c) < 0
    out = tris.copy()
    out[flip, 1], out[flip, 2] = tris[flip, 2], tris[flip, 1]
    return out


def _icosahedron():
    g = (1.0 + 5.0 ** 0.5) / 2.0
    v = []
    for a in (-1.0, 1.0):
        for b in (-g, g):
            v += [(0.0, a, b), (a, b, 0.0), (b, 0.0, a)]
    v = np.array(v)
    # faces = triples of mutually adjacent vertices (edge length 2)
    d = np.linalg.norm(v[:, None, :] - v[None, :, :], axis=2)
    adj = np.abs(d - 2.0) < 1e-9
    faces = []
    n = len(v)
    for i in range(n):
        for j in range(i + 1, n):
            if not adj[i, j]:
                continue
            for k in range(j + 1, n):
                if adj[i, k] and adj[j, k]:
                    faces.append((i, j, k))
    tris = np.array(faces, dtype=np.int64)
    assert tris.shape == (20, 3)
    return v, _orient_outward(v, tris)


def _octahedron():
    v = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float)
    faces = []
    for sx in (0, 1):
        for sy in (2, 3):
            for sz in (4, 5):
                faces.append((sx, sy, sz))
    return v, _orient_outward(v, np.array(faces, dtype=np.int64))


def _subdivide(verts: np.ndarray, tris: np.ndarray, radius: float | None):
    """Split every triangle into four at its edge midpoints (orientation kept)."""
    a, b, c = tris[:, 0], tris[:, 1], tris[:, 2]
    edges = np.concatenate([np.stack([a, b], 1), np.stack([b, c], 1), np.stack([c, a], 1)])
    key = np.sort(edges, axis=1)
    uniq, inv = np.unique(key, axis=0, return_inverse=True)
    inv = inv.reshape(-1)
    mid = 0.5 * (verts[uniq[:, 0]] + verts[uniq[:, 1]])
    if radius is not None:
        mid *= radius / np.linalg.norm(mid, axis=1, keepdims=True)
    base = len(verts)
    m = len(tris)
    ab, bc, ca = inv[:m] + base, inv[m:2 * m] + base, inv[2 * m:] + base
    new = np.concatenate([
        np.stack([a, ab, ca], 1), np.stack([b, bc, ab], 1),
        np.stack([c, ca, bc], 1), np.stack([ab, bc, ca], 1)])
    return np.concatenate([verts, mid]), new


def icosphere(subdivisions: int, radius: float = 10.0):
    """Sphere of 20*4**s flat triangles inscribed in radius ``radius`` (nm).

    Returns (verts float64 [nv,3], tris int32 [n,3]); faces are CCW seen from
    outside so (v1-v0)x(v2-v0) is the outward normal.
    """
    v, t = _icosahedron()
    v = v * (radius / np.linalg.norm(v, axis=1, keepdims=True))
    for _ in range(subdivisions):
        v, t = _subdivide(v, t, radius)
    return np.ascontiguousarray(v, dtype=np.float64), np.ascontiguousarray(t, dtype=np.int32)


def octasphere(subdivisions: int, radius: float = 8.0):
    """Sphere of 8*4**s triangles (512, 2048, 8192, 32768 for s = 3..6)."""
    v, t = _octahedron()
    v = v * radius
    for _ in range(subdivisions):
        v, t = _subdivide(v, t, radius)
    return np.ascontiguousarray(v, dtype=np.float64), np.ascontiguousarray(t, dtype=np.int32)


def ellipsoid(subdivisions: int, axes=(7.0, 4.0, 4.0)):
    """Octasphere mapped affinely onto an ellipsoid with the given semi-axes (nm)."""
    v, t = octasphere(subdivisions, 1.0)
    v = v * np.asarray(axes, float)[None, :]
    return np.ascontiguousarray(v), t


def _real_sph_harm(l: int, m: int, theta: np.ndarray, phi: np.ndarray) -> np.ndarray:
    from scipy.special import sph_harm_y
    y = sph_harm_y(l, abs(m), theta, phi)
    if m > 0:
        return np.sqrt(2.0) * (-1) ** m * y.real
    if m < 0:
        return np.sqrt(2.0) * (-1) ** m * y.imag
    return y.real


def protein_like(subdivisions: int = 6, axes=(7.0, 4.0, 4.0), lmax: int = 8,
                 amplitude: float = 0.10, seed: int = 1812):
    """Closed, star-shaped analyte surface: ellipsoid with a random SH bump field.

    r <- r * (1 + amplitude * g(theta, phi)), g = sum_{l=1..lmax} sum_m c_lm Y_lm
    with c_lm ~ N(0, 1/(2l+1)) drawn from numpy PCG64(seed), g scaled to max|g| = 1
    over the mesh vertices.  The long axis is x (the first semi-axis).
    """
    v, t = ellipsoid(subdivisions, axes)
    rng = np.random.Generator(np.random.PCG64(seed))
    r = np.linalg.norm(v, axis=1)
    theta = np.arccos(np.clip(v[:, 2] / r, -1.0, 1.0))
    phi = np.arctan2(v[:, 1], v[:, 0])
    g = np.zeros(len(v))
    for l in range(1, lmax + 1):
        for m in range(-l, l + 1):
            g += rng.normal(0.0, (1.0 / (2 * l + 1)) ** 0.5) * _real_sph_harm(l, m, theta, phi)
    g /= np.max(np.abs(g))
    v = v * (1.0 + amplitude * g)[:, None]
    return np.ascontiguousarray(v), _orient_outward(v, t.astype(np.int64)).astype(np.int32)


# Rotations that take a surface whose long axis is x to a placement axis: first x -> +z;
# the -z copy is the 180-degree rotation of the +z one about y, and +-x, +-y are 90-degree
# rotations of the +z placement (the sensor arrangements of Sec. III).
_TO_Z = np.array([[0.0, 0.0, -1.0], [0.0, 1.0, 0.0], [1.0, 0.0, 0.0]])
_FROM_Z = {
    "+z": np.eye(3),
    "-z": np.diag([-1.0, 1.0, -1.0]),
    "+x": np.array([[0.0, 0.0, 1.0], [0.0, 1.0, 0.0], [-1.0, 0.0, 0.0]]),
    "-x": np.array([[0.0, 0.0, -1.0], [0.0, 1.0, 0.0], [1.0, 0.0, 0.0]]),
    "+y": np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 1.0], [0.0, -1.0, 0.0]]),
    "-y": np.array([[1.0, 0.0, 0.0], [0.0, 0.0, -1.0], [0.0, 1.0, 0.0]]),
}
_AXIS = {"+z": (0, 0, 1), "-z": (0, 0, -1), "+x": (1, 0, 0), "-x": (-1, 0, 0), "+y": (0, 1, 0), "-y": (0, -1, 0)}


def place_analyte(verts: np.ndarray, axis: str, gap: float, R: float) -> np.ndarray:
    """Rotate a surface centred at the origin (long axis x) onto `axis` and move it along
    that axis until its closest vertex lies `gap` nm outside the sphere of radius R."""
    v = verts @ (_FROM_Z[axis] @ _TO_Z).T
    u = np.asarray(_AXIS[axis], float)

    def clearance(d):
        return np.min(np.linalg.norm(v + d * u, axis=1)) - R

    lo, hi = 0.0, R + gap + 2.0 * np.max(np.linalg.norm(v, axis=1))
    for _ in range(200):   # clearance grows with d once the surface is outside the sphere
        mid = 0.5 * (lo + hi)
        if clearance(mid) < gap:
            lo = mid
        else:
            hi = mid
    return np.ascontiguousarray(v + hi * u)


def sensor_geometry(sphere_sub: int = 6, R: float = 10.0, analytes=(("+z", 1.0), ("-z", 1.0)),
                    analyte_sub: int = 6, axes=(7.0, 4.0, 4.0), seed0: int = 1812):
    """Sphere (surface 0) plus protein-like analytes (surfaces 1, 2, ...) at the given
    (axis, gap) placements; analyte k is drawn with seed seed0 + k.  Returns (verts, tris, surf)."""
    vs, ts = icosphere(sphere_sub, R)
    parts_v, parts_t, surf = [vs], [ts], [np.zeros(len(ts), np.int32)]
    off = len(vs)
    for k, (axis, gap) in enumerate(analytes):
        va, ta = protein_like(analyte_sub, axes, seed=seed0 + k)
        va = place_analyte(va, axis, gap, R)
        parts_v.append(va)
        parts_t.append(ta + off)
        surf.append(np.full(len(ta), k + 1, np.int32))
        off += len(va)
    return (np.ascontiguousarray(np.concatenate(parts_v)), np.ascontiguousarray(np.concatenate(parts_t), np.int32),
            np.concatenate(surf))


def two_spheres(subdivisions: int, R: float, distance: float):
    """Two equal spheres, surface 0 at the origin and surface 1 centred at (0, 0, distance)."""
    v, t = icosphere(subdivisions, R)
    v1 = v + np.array([0.0, 0.0, distance])
    return (np.ascontiguousarray(np.concatenate([v, v1])),
            np.ascontiguousarray(np.concatenate([t, t + len(v)]), np.int32),
            np.concatenate([np.zeros(len(t), np.int32), np.ones(len(t), np.int32)]))


def drude_eps(lambda_nm, eps_inf=DRUDE_AG["eps_inf"], wp=DRUDE_AG["wp"], gamma=DRUDE_AG["gamma"]):
    """Drude permittivity eps_inf - wp^2/(w^2 + i*gamma*w), w = 1239.84198/lambda eV."""
    w = HC_EV_NM / np.asarray(lambda_nm, dtype=np.float64)
    return eps_inf - wp * wp / (w * w + 1j * gamma * w)


def tabulated_eps(lambda_nm, table_lambda_nm, table_n, table_k) -> np.ndarray:
    """Permittivity eps = (n + i k)^2 from a tabulated complex refractive index (e.g. the
    Johnson-Christy silver or Hale-Querry water tables the paper uses, Sec. III), with n and
    k interpolated linearly in the wavelength.  Wavelengths outside the table are refused."""
    lam = np.atleast_1d(np.asarray(lambda_nm, float))
    tl = np.asarray(table_lambda_nm, float)
    order = np.argsort(tl)
    tl = tl[order]
    if lam.min() < tl[0] or lam.max() > tl[-1]:
        raise ValueError("wavelength outside the tabulated range")
    n = np.interp(lam, tl, np.asarray(table_n, float)[order])
    k = np.interp(lam, tl, np.asarray(table_k, float)[order])
    return (n + 1j * k) ** 2


def wavelengths(lo: float, hi: float, count: int) -> np.ndarray:
    """``count`` wavelengths uniform over [lo, hi] nm, both ends included."""
    return np.linspace(lo, hi, count)


def random_complex(n: int, seed: int = 0, batch: int | None = None) -> np.ndarray:
    """Uniform [-1,1] + i[-1,1] complex128 vector(s) from numpy PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (n,) if batch is None else (batch, n)
    return rng.uniform(-1, 1, shape) + 1j * rng.uniform(-1, 1, shape)


# named workloads: sizes and parameters of the sphere benchmarks
SPHERE_WORKLOADS = {
    "sphere1280": dict(subdivisions=3, radius=10.0),
    "sphere5120": dict(subdivisions=4, radius=10.0),
    "sphere20480": dict(subdivisions=5, radius=10.0),
    "sphere81920": dict(subdivisions=6, radius=10.0),
    "sphere327680": dict(subdivisions=7, radius=10.0),
}
