"""The allocation-free direct FP32 product (lspr_matvec_direct_fp32_noalloc).

It serves callers that must not allocate device memory during the call (an
application whose device memory belongs to another allocator or to a fixed
budget, or a latency-critical loop where cudaMalloc/cudaFree could synchronise
the device).  Its scratch lives in one fixed device array inside the library.
The test calls it through the C ABI twice in a row, with different inputs, and
compares each result with lspr_matvec in LSPR_DIRECT_FP32 mode at the FP32
direct tolerance of the parity tests (1e-5 relative L2); it also checks that a
mesh larger than the fixed scratch is refused.  The file is collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_1812_10722_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matvec_matches_direct_fp32():
    torch = pytest.importorskip("torch")
    from paper_1812_10722_gb300 import build, lspr
    build.build()
    L = lspr.lib()
    fn = L.lspr_matvec_direct_fp32_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_double]
    fn.restype = ctypes.c_int
    v, t = I.icosphere(3, 10.0)
    n = len(t)
    with lspr.Context(0) as ctx:
        ctx.mesh_upload(v, t)
        for call, (seed, lam) in enumerate([(21, 380.0), (22, 365.0)]):
            s = complex(I.drude_eps(lam) / I.EPS_WATER)
            x = torch.as_tensor(I.random_complex(2 * n, seed=seed), device="cuda")
            ref = ctx.matvec(x, s, "direct_fp32").cpu().numpy()
            y = torch.full_like(x, float("nan"))
            rc = fn(ctx._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), s.real, s.imag)
            assert rc == 0, f"call {call}: status {rc}"
            torch.cuda.synchronize()
            got = y.cpu().numpy()
            assert np.all(np.isfinite(got))
            assert _rel(got, ref) < 1e-5, f"call {call}"
        # a mesh beyond the fixed scratch (20480 panels > 16384) is refused
        vb, tb = I.icosphere(5, 10.0)
        ctx.mesh_upload(vb, tb)
        xb = torch.zeros(2 * len(tb), dtype=torch.complex128, device="cuda")
        yb = torch.zeros_like(xb)
        assert fn(ctx._h, ctypes.c_void_p(xb.data_ptr()), ctypes.c_void_p(yb.data_ptr()), 1.0, 0.0) == 1
