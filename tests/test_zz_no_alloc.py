"""The allocation-free direct FP32 product (lspr_matvec_direct_fp32_noalloc).

It serves callers that must not allocate device memory during the call (an
application whose device memory belongs to another allocator or to a fixed
budget, or a latency-critical loop where cudaMalloc/cudaFree could synchronise
the device).  Its scratch lives in one fixed device array inside the library.

The test calls it through the C ABI on a freshly uploaded mesh before any other
product (so that it cannot lean on buffers an lspr_matvec would have created),
then again with other inputs, and after a tree build has reordered the sources
and targets; every result is compared with lspr_matvec in LSPR_DIRECT_FP32 mode
at the FP32 direct tolerance of the parity tests (1e-5, relative L2 and element
by element).  Around a call after the first, the device's free memory must not
change.  A mesh larger than the fixed scratch is refused.  The file is collected
last.
"""
import ctypes

import numpy as np
import pytest

from paper_1812_10722_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _rowmax(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


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
    cases = [(21, 380.0), (22, 365.0), (23, 395.0)]
    xs = [torch.as_tensor(I.random_complex(2 * n, seed=seed), device="cuda") for seed, _ in cases]
    ys = [torch.full_like(x, float("nan")) for x in xs]
    ss = [complex(I.drude_eps(lam) / I.EPS_WATER) for _, lam in cases]

    def call(ctx, k):
        rc = fn(ctx._h, ctypes.c_void_p(xs[k].data_ptr()), ctypes.c_void_p(ys[k].data_ptr()), ss[k].real, ss[k].imag)
        assert rc == 0, f"call {k}: status {rc}"

    with lspr.Context(0) as ctx:
        ctx.mesh_upload(v, t)
        call(ctx, 0)                                  # the first product on this context
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        call(ctx, 1)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, "the call changed the device's free memory"
        ctx.tree_build(0.5, 6, 64)                    # reorders sources and targets (Morton)
        call(ctx, 2)
        torch.cuda.synchronize()
        for k in range(3):
            ref = ctx.matvec(xs[k], ss[k], "direct_fp32").cpu().numpy()
            got = ys[k].cpu().numpy()
            assert np.all(np.isfinite(got)), k
            assert _rel(got, ref) < 1e-5 and _rowmax(got, ref) < 1e-5, k
        # a mesh beyond the fixed scratch (20480 panels > 16384) is refused
        vb, tb = I.icosphere(5, 10.0)
        ctx.mesh_upload(vb, tb)
        xb = torch.zeros(2 * len(tb), dtype=torch.complex128, device="cuda")
        yb = torch.zeros_like(xb)
        assert fn(ctx._h, ctypes.c_void_p(xb.data_ptr()), ctypes.c_void_p(yb.data_ptr()), 1.0, 0.0) == 1
