"""Python binding of the C ABI in ``include/lspr.h`` (argument marshalling only).

Every numerical step runs in the sm_103a library ``_lib/liblspr_gb300.so``;
there is no CPU fallback: if the library is missing or no GPU is present the
calls raise.  Arrays may be numpy (host) or torch CUDA tensors (device; the
call then runs on torch's current stream of that device).
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

from . import build as _build

LIB_PATH = _build.LIB

DIRECT_FP64, DIRECT_FP32, TREE_FP64, TREE_FP32, DIRECT_FF, TREE_FF = 0, 1, 2, 3, 4, 5
MODES = {"direct_fp64": DIRECT_FP64, "direct_fp32": DIRECT_FP32, "tree_fp64": TREE_FP64, "tree_fp32": TREE_FP32,
         "direct_ff": DIRECT_FF, "tree_ff": TREE_FF}

STATUS = {0: "LSPR_OK", 1: "LSPR_E_ARG", 2: "LSPR_E_STATE", 3: "LSPR_E_CUDA", 4: "LSPR_E_OOM",
          5: "LSPR_E_NOT_CONVERGED", 6: "LSPR_E_TIMEOUT", 7: "LSPR_E_MESH"}

_lock = threading.Lock()
_lib = None


TIMER_NAMES = ["p2p", "m2p", "p2m", "near_assembly", "gmres", "tree", "mesh", "other", "p2p_fp64", "m2p_fp64",
               "p2m_fp64", "weights", "p2p_ff", "m2p_ff", "p2m_ff", "unused"]


class LsprError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        msg = f"{where}: {STATUS.get(status, status)} ({lib().lspr_status_string(status).decode()})"
        super().__init__(msg + (f": {detail}" if detail else ""))


class QuadOpts(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("K_fine", ctypes.c_int32), ("N_k", ctypes.c_int32),
                ("threshold", ctypes.c_double)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("restart", ctypes.c_int32), ("maxiter", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("refine", ctypes.c_int32)]


class SolveStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.POINTER(ctypes.c_int32)), ("residual", ctypes.POINTER(ctypes.c_double)),
                ("status", ctypes.POINTER(ctypes.c_int32)), ("seconds", ctypes.c_double),
                ("matvecs", ctypes.c_int64)]


_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_d = ctypes.c_double


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
            L = ctypes.CDLL(LIB_PATH)
            L.lspr_status_string.argtypes = [ctypes.c_int]
            L.lspr_status_string.restype = ctypes.c_char_p
            L.lspr_version.restype = ctypes.c_char_p
            L.lspr_last_error.argtypes = [_vp]
            L.lspr_last_error.restype = ctypes.c_char_p
            L.lspr_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, _vp]
            L.lspr_destroy.argtypes = [_vp]
            L.lspr_mesh_upload.argtypes = [_vp, _vp, _i64, _vp, _i64, _vp, _i32, ctypes.POINTER(QuadOpts), _i32]
            L.lspr_tree_build.argtypes = [_vp, _d, _i32, _i32]
            L.lspr_matvec.argtypes = [_vp, _vp, _vp, _i32, _vp, _i32, _i32]
            L.lspr_solve.argtypes = [_vp, _vp, _d, _d, _vp, _vp, _i32, ctypes.POINTER(SolveOpts), _vp, _vp,
                                     ctypes.POINTER(SolveStats)]
            L.lspr_get_info.argtypes = [_vp] + [ctypes.POINTER(_i64)] * 7
            L.lspr_get_timing_rhs.argtypes = [_vp, _vp]
            L.lspr_get_arnoldi_stats.argtypes = [_vp, _vp]
            L.lspr_tune_solver.argtypes = [_vp, _vp, _d, _d, _vp, _vp, _i32, ctypes.POINTER(SolveOpts), _vp, _i32,
                                           ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_d)]
            L.lspr_get_tc_info.argtypes = [_vp] + [ctypes.POINTER(_i64)] * 4
            L.lspr_set_timing.argtypes = [_vp, _i32]
            L.lspr_launch_count.argtypes = [_vp, ctypes.POINTER(_i64)]
            L.lspr_get_timing.argtypes = [_vp, _vp, _vp]
            L.lspr_set_graphs.argtypes = [_vp, _i32]
            L.lspr_set_tensor_cores.argtypes = [_vp, _i32]
            L.lspr_autotune.argtypes = [_vp, _vp, _d, _d, _vp, _vp, _i32, ctypes.POINTER(TuneOpts),
                                        ctypes.POINTER(TuneResult)]
            L.lspr_graph_stats.argtypes = [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]
            L.lspr_device_errors.argtypes = [_vp, ctypes.POINTER(_i32)]
            L.lspr_selftest_wait_timeout.argtypes = [_vp, ctypes.POINTER(_i32)]
            L.lspr_selftest_gate_waits.argtypes = [_vp, _i32]
            L.lspr_set_charges.argtypes = [_vp, _vp, _i64, _vp]
            for f in ("lspr_create", "lspr_destroy", "lspr_mesh_upload", "lspr_tree_build", "lspr_matvec",
                      "lspr_solve", "lspr_get_info", "lspr_set_timing", "lspr_get_timing", "lspr_launch_count",
                      "lspr_set_graphs", "lspr_graph_stats", "lspr_autotune", "lspr_set_tensor_cores",
                      "lspr_device_errors", "lspr_selftest_wait_timeout", "lspr_selftest_gate_waits",
                      "lspr_set_charges", "lspr_get_tc_info", "lspr_get_timing_rhs", "lspr_tune_solver",
                      "lspr_get_arnoldi_stats"):
                getattr(L, f).restype = ctypes.c_int
            _lib = L
    return _lib


def _check(rc: int, where: str, handle=None):
    if rc != 0:
        detail = lib().lspr_last_error(handle).decode() if handle else ""
        raise LsprError(rc, where, detail)


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _host_ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


class TuneOpts(ctypes.Structure):
    _fields_ = [("target_rel_err", ctypes.c_double), ("tol", ctypes.c_double), ("restart", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("refine", ctypes.c_int32), ("grid", ctypes.c_int32),
                ("time_rhs", ctypes.c_int32), ("pad_", ctypes.c_int32)]


class TuneResult(ctypes.Structure):
    _fields_ = [("theta", ctypes.c_double), ("P", ctypes.c_int32), ("Ncrit", ctypes.c_int32),
                ("rel_err", ctypes.c_double), ("ms", ctypes.c_double), ("ref_ms", ctypes.c_double),
                ("candidates", ctypes.c_int32), ("qualified", ctypes.c_int32), ("tensor_cores", ctypes.c_int32),
                ("iterations", ctypes.c_int32), ("product_ms", ctypes.c_double),
                ("residual_product_ms", ctypes.c_double)]


@dataclass
class SolveResult:
    dipole: np.ndarray        # [B, 3] complex
    sigma_ext: np.ndarray     # [B] nm^2
    iterations: np.ndarray    # [B]
    residual: np.ndarray      # [B]
    status: np.ndarray        # [B]
    seconds: float
    matvecs: int


class Context:
    """One GPU context: mesh, tree, operator and solver state (lspr_ctx)."""

    def __init__(self, device: int = 0, stream=None):
        self._h = ctypes.c_void_p()
        self.device = device
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream(device).cuda_stream
            except ImportError:
                stream = None
        _check(lib().lspr_create(ctypes.byref(self._h), device, ctypes.c_void_p(stream or 0)), "lspr_create")
        self.n = 0

    def close(self):
        if self._h:
            lib().lspr_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------------ mesh
    def mesh_upload(self, verts, tris, K=4, K_fine=19, N_k=9, threshold=0.5, surf_id=None, nsurf=None):
        """Panels and quadrature (host numpy or CUDA torch arrays).  surf_id: surface of
        each panel (surface 0 = the particle); nsurf defaults to max(surf_id) + 1."""
        q = QuadOpts(K, K_fine, N_k, threshold)
        if _is_torch(verts):
            assert verts.is_cuda and tris.is_cuda
            assert str(verts.dtype) == "torch.float64" and str(tris.dtype) == "torch.int32"
            verts, tris = verts.contiguous(), tris.contiguous()
            sid = None if surf_id is None else surf_id.contiguous()
            if sid is not None:
                assert sid.is_cuda and str(sid.dtype) == "torch.int32"
            ns = nsurf or (1 if sid is None else int(sid.max().item()) + 1)
            rc = lib().lspr_mesh_upload(self._h, ctypes.c_void_p(verts.data_ptr()), verts.shape[0],
                                        ctypes.c_void_p(tris.data_ptr()), tris.shape[0],
                                        None if sid is None else ctypes.c_void_p(sid.data_ptr()), ns,
                                        ctypes.byref(q), 1)
            n = tris.shape[0]
        else:
            v = np.ascontiguousarray(verts, dtype=np.float64)
            t = np.ascontiguousarray(tris, dtype=np.int32)
            sid = None if surf_id is None else np.ascontiguousarray(surf_id, dtype=np.int32)
            ns = nsurf or (1 if sid is None else int(sid.max()) + 1)
            rc = lib().lspr_mesh_upload(self._h, _host_ptr(v), len(v), _host_ptr(t), len(t),
                                        None if sid is None else _host_ptr(sid), ns, ctypes.byref(q), 0)
            n = len(t)
        _check(rc, "lspr_mesh_upload", self._h)
        self.n = int(n)
        self.nsurf = int(ns)

    def _per_surface(self, a, B):
        """[B, S] complex array from a scalar, [S], [B] (one surface) or [B, S] input."""
        a = np.asarray(a, np.complex128)
        S = getattr(self, "nsurf", 1)
        if S == 1:
            return np.ascontiguousarray(np.broadcast_to(a.reshape(-1), (B,)).reshape(B, 1))
        return np.ascontiguousarray(np.broadcast_to(a.reshape(-1, S), (B, S)))

    def tree_build(self, theta=0.5, P=6, Ncrit=300):
        _check(lib().lspr_tree_build(self._h, float(theta), int(P), int(Ncrit)), "lspr_tree_build", self._h)

    # ---------------------------------------------------------------- matvec
    def matvec(self, x, eps_ratio, mode="direct_fp64"):
        """y = A(s) x; x [2N] or [B, 2N] complex128 (numpy or torch CUDA)."""
        m = MODES[mode] if isinstance(mode, str) else int(mode)
        if _is_torch(x):
            import torch
            squeeze = x.dim() == 1
            xx = x.reshape(-1, 2 * self.n).contiguous()
            B = xx.shape[0]
            s = torch.as_tensor(self._per_surface(eps_ratio, B).copy(), device=x.device)
            y = torch.empty_like(xx)
            rc = lib().lspr_matvec(self._h, ctypes.c_void_p(xx.data_ptr()), ctypes.c_void_p(y.data_ptr()), B,
                                   ctypes.c_void_p(s.data_ptr()), m, 1)
            _check(rc, "lspr_matvec", self._h)
            return y[0] if squeeze else y
        x = np.ascontiguousarray(x, dtype=np.complex128)
        squeeze = x.ndim == 1
        xx = x.reshape(-1, 2 * self.n)
        B = xx.shape[0]
        s = self._per_surface(eps_ratio, B)
        y = np.zeros_like(xx)
        _check(lib().lspr_matvec(self._h, _host_ptr(xx), _host_ptr(y), B, _host_ptr(s), m, 0), "lspr_matvec", self._h)
        return y[0] if squeeze else y

    # ----------------------------------------------------------------- solve
    def solve(self, eps_in, eps_out, lambda_nm, E0=(0.0, 0.0, 1.0), tol=1e-6, restart=50, maxiter=500,
              mode="tree_fp32", refine=False, check=True) -> SolveResult:
        """eps_in: [B] (one surface) or [B, S] / [S] (several surfaces: permittivity of every
        surface per wavelength; sigma_ext and the dipole are surface 0's)."""
        m = MODES[mode] if isinstance(mode, str) else int(mode)
        S = getattr(self, "nsurf", 1)
        lam1 = np.atleast_1d(np.asarray(lambda_nm, np.float64))
        ea = np.asarray(eps_in, np.complex128)
        B = max(len(lam1), ea.size // S)
        e = self._per_surface(ea, B)
        lam = np.ascontiguousarray(np.broadcast_to(lam1, (B,)), dtype=np.float64)
        E = np.ascontiguousarray(E0, dtype=np.float64)
        dip = np.zeros((B, 3), np.complex128)
        sig = np.zeros(B)
        it = np.zeros(B, np.int32)
        rr = np.zeros(B)
        stt = np.zeros(B, np.int32)
        st = SolveStats(it.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                        rr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                        stt.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), 0.0, 0)
        # refine: False/0 plain, True/1 float-float residual, 2 native FP64 residual
        o = SolveOpts(float(tol), int(restart), int(maxiter), m, int(refine))
        eo = complex(eps_out)
        rc = lib().lspr_solve(self._h, _host_ptr(e), eo.real, eo.imag, _host_ptr(E), _host_ptr(lam), B,
                              ctypes.byref(o), _host_ptr(dip), _host_ptr(sig), ctypes.byref(st))
        if rc not in (0, 5) or (check and rc != 0):
            _check(rc, "lspr_solve", self._h)
        return SolveResult(dip, sig, it, rr, stt, st.seconds, st.matvecs)

    # ------------------------------------------------------------------ info
    def info(self) -> dict:
        vals = [ctypes.c_int64() for _ in range(7)]
        _check(lib().lspr_get_info(self._h, *[ctypes.byref(v) for v in vals]), "lspr_get_info", self._h)
        keys = ["n_panels", "n_sources", "n_near", "n_boxes", "n_p2p_items", "n_m2p_pairs", "n_p2p_pairs"]
        return {k: v.value for k, v in zip(keys, vals)}

    def tc_info(self) -> dict:
        """Sizes of the tensor-core work lists (0 until a product of several right-hand sides)."""
        vals = [ctypes.c_int64() for _ in range(4)]
        _check(lib().lspr_get_tc_info(self._h, *[ctypes.byref(v) for v in vals]), "lspr_get_tc_info", self._h)
        return dict(zip(["m2p_units", "m2p_group_boxes", "p2p_group_sources", "p2p_stages"], [v.value for v in vals]))

    def launch_count(self) -> int:
        n = ctypes.c_int64(0)
        _check(lib().lspr_launch_count(self._h, ctypes.byref(n)), "lspr_launch_count", self._h)
        return n.value

    def autotune(self, eps_in, eps_out, lambda_nm, E0=(0.0, 0.0, 1.0), target_rel_err=1e-4, tol=1e-6,
                 restart=50, mode="tree_fp32", refine=1, coarse=False, time_rhs=0) -> dict:
        """Cheapest (theta, P, Ncrit) whose sigma_ext stays within target_rel_err / 2 of the
        reference treecode solve; the chosen tree is left built.  time_rhs > 0: the cost is
        modelled from product times at that many right-hand sides (and the faster P2P path is
        left set), else it is the tuning solve's time."""
        eps = np.ascontiguousarray(np.atleast_1d(np.asarray(eps_in, np.complex128)))
        lam = np.ascontiguousarray(np.atleast_1d(np.asarray(lambda_nm, np.float64)))
        e0 = np.ascontiguousarray(np.asarray(E0, np.float64))
        eo = complex(eps_out)
        o = TuneOpts(float(target_rel_err), float(tol), int(restart), MODES[mode] if isinstance(mode, str) else int(mode),
                     int(refine), int(bool(coarse)), int(time_rhs), 0)
        r = TuneResult()
        _check(lib().lspr_autotune(self._h, _host_ptr(eps), eo.real, eo.imag, _host_ptr(e0), _host_ptr(lam),
                                   len(lam), ctypes.byref(o), ctypes.byref(r)), "lspr_autotune", self._h)
        return {k: getattr(r, k) for k, _ in TuneResult._fields_}

    def tune_solver(self, eps_in, eps_out, lambda_nm, restarts=(30, 50, 80), E0=(0.0, 0.0, 1.0), tol=1e-6,
                    maxiter=2000, mode="tree_fp32", refine=1) -> dict:
        """Fastest (GMRES restart, P2P path) for this batch, each timed with a full solve; the
        chosen tensor-core mask is left set.  Returns {"restart", "tensor_cores", "ms"}."""
        S = getattr(self, "nsurf", 1)
        lam1 = np.atleast_1d(np.asarray(lambda_nm, np.float64))
        ea = np.asarray(eps_in, np.complex128)
        B = max(len(lam1), ea.size // S)
        e = self._per_surface(ea, B)
        lam = np.ascontiguousarray(np.broadcast_to(lam1, (B,)), dtype=np.float64)
        E = np.ascontiguousarray(E0, dtype=np.float64)
        rs = np.ascontiguousarray(restarts, dtype=np.int32)
        o = SolveOpts(float(tol), 50, int(maxiter), MODES[mode] if isinstance(mode, str) else int(mode), int(refine))
        m, tc, ms = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_double(0.0)
        eo = complex(eps_out)
        _check(lib().lspr_tune_solver(self._h, _host_ptr(e), eo.real, eo.imag, _host_ptr(E), _host_ptr(lam), B,
                                      ctypes.byref(o), _host_ptr(rs), len(rs), ctypes.byref(m), ctypes.byref(tc),
                                      ctypes.byref(ms)), "lspr_tune_solver", self._h)
        return {"restart": m.value, "tensor_cores": tc.value, "ms": ms.value}

    def set_graphs(self, enable: bool):
        """Arnoldi cycles as CUDA graph launches (default) or host-driven."""
        _check(lib().lspr_set_graphs(self._h, int(bool(enable))), "lspr_set_graphs", self._h)

    def set_tensor_cores(self, enable):
        """Tensor cores for the FP32 far field of several right-hand sides: True / 1 = the M2P
        (default), 3 = M2P and P2P, False / 0 = the FP32-pipe kernels."""
        mask = int(enable) if not isinstance(enable, bool) else int(enable)
        _check(lib().lspr_set_tensor_cores(self._h, mask), "lspr_set_tensor_cores", self._h)

    def device_errors(self) -> int:
        """Bounded device waits that ran out since the context was created (0 when healthy)."""
        n = ctypes.c_int32(0)
        _check(lib().lspr_device_errors(self._h, ctypes.byref(n)), "lspr_device_errors", self._h)
        return n.value

    def set_charges(self, charges=None, surf=None):
        """Point charges (x, y, z, q) inside the given surfaces for later solves (None: remove)."""
        if charges is None:
            _check(lib().lspr_set_charges(self._h, None, 0, None), "lspr_set_charges", self._h)
            return
        q = np.ascontiguousarray(np.asarray(charges, np.float64).reshape(-1, 4))
        sq = np.ascontiguousarray(np.asarray(surf, np.int32).reshape(-1))
        if sq.shape[0] != q.shape[0]:
            raise ValueError("one surface index per charge")
        _check(lib().lspr_set_charges(self._h, q.ctypes.data, q.shape[0], sq.ctypes.data), "lspr_set_charges",
               self._h)

    def selftest_wait_timeout(self) -> dict:
        """Runs one bounded device wait that cannot complete: {"succeeded", "abort", "ms"}."""
        r = (ctypes.c_int32 * 3)()
        _check(lib().lspr_selftest_wait_timeout(self._h, r), "lspr_selftest_wait_timeout", self._h)
        return {"succeeded": r[0], "abort": r[1], "ms": r[2]}

    def selftest_gate_waits(self, enable: bool):
        """While enabled, every tensor-core far-field kernel gives up at once through its bounded
        wait (no work done, LSPR_E_TIMEOUT from the product or solve that launched it)."""
        _check(lib().lspr_selftest_gate_waits(self._h, int(bool(enable))), "lspr_selftest_gate_waits", self._h)

    def graph_stats(self) -> dict:
        c, r = ctypes.c_int64(0), ctypes.c_int64(0)
        _check(lib().lspr_graph_stats(self._h, ctypes.byref(c), ctypes.byref(r)), "lspr_graph_stats", self._h)
        return {"cycles": c.value, "recordings": r.value}

    def set_timing(self, enable: bool):
        _check(lib().lspr_set_timing(self._h, int(bool(enable))), "lspr_set_timing", self._h)

    def timing(self) -> dict:
        ms = np.zeros(16)
        n = np.zeros(16, np.int64)
        _check(lib().lspr_get_timing(self._h, _host_ptr(ms), _host_ptr(n)), "lspr_get_timing", self._h)
        return {k: (float(a), int(b)) for k, a, b in zip(TIMER_NAMES, ms, n)}

    def arnoldi_stats(self) -> dict:
        """Arnoldi work counters since the context was created (lspr_get_arnoldi_stats)."""
        r = np.zeros(4, np.int64)
        _check(lib().lspr_get_arnoldi_stats(self._h, _host_ptr(r)), "lspr_get_arnoldi_stats", self._h)
        return {"vectors": int(r[0]), "system_steps": int(r[1]), "vectors_second_pass": int(r[2]),
                "system_steps_second_pass": int(r[3])}

    def timing_rhs(self) -> dict:
        """Right-hand sides summed over the timed launches of each far-field slot."""
        r = np.zeros(16, np.int64)
        _check(lib().lspr_get_timing_rhs(self._h, _host_ptr(r)), "lspr_get_timing_rhs", self._h)
        return {k: int(v) for k, v in zip(TIMER_NAMES, r)}
