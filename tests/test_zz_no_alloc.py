"""The allocation-free entry point kerr_trace_camera_static.

It serves callers that cannot allocate device memory (real-time hosts that
must not call cudaMalloc/cudaFree once running, hosts whose device memory is
budgeted by another framework's pool): all of its scratch lives in one fixed
device array inside the library.  Here it is called through the C ABI and its
outputs are compared with those of kerr_trace_camera, which allocates its
scratch in a context, on two calls in a row (the second call must start from
cleared counters, not from the first call's leftovers).

This file is named to be collected last, so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1706_07062_gb300 import kerr as K  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
GATE = 1e-5          # the FP32+Kahan parity tolerance used by the other tests


def _rel(a, b):
    a = a.detach().cpu().numpy()
    b = b.detach().cpu().numpy()
    den = np.maximum(np.linalg.norm(b, axis=0), 1e-300)
    return float((np.linalg.norm(a - b, axis=0) / den).max())


def _check_same(got, ref):
    assert torch.equal(got.status, ref.status)
    assert _rel(got.x[1:4], ref.x[1:4]) <= GATE
    assert _rel(got.k, ref.k) <= GATE
    assert torch.equal(got.steps, ref.steps)


@pytest.mark.parametrize("prec", [K.FP32_KAHAN, K.FP64])
def test_static_entry_point_matches_allocating_entry_point(prec):
    K.lib()
    cams = [K.camera(0.9, np.radians(60.0), 1000.0, 20.0, 160, 160),
            K.camera(0.5, np.radians(30.0), 1000.0, 12.0, 64, 32)]
    opts = K.default_opts(prec=prec, tol=1e-6)
    ctx = K.kerr_init(0.9)
    ref = K.kerr_trace_camera(ctx, cams, opts, device=DEV)
    torch.cuda.synchronize()
    ctx.close()
    # two calls in a row through the allocation-free entry point
    for _ in range(2):
        out = K.kerr_trace_camera_static(cams, opts, device=DEV)
        torch.cuda.synchronize()
        _check_same(out, ref)
    # a different, smaller call after them starts from cleared counters
    one = [cams[1]]
    ctx = K.kerr_init(0.5)
    ref1 = K.kerr_trace_camera(ctx, one, opts, device=DEV)
    torch.cuda.synchronize()
    ctx.close()
    out1 = K.kerr_trace_camera_static(one, opts, device=DEV)
    torch.cuda.synchronize()
    _check_same(out1, ref1)


def test_static_entry_point_limits():
    K.lib()
    too_big = K.camera(0.9, 1.0, 1000.0, 20.0, 512, 512)     # 262144 > 131072 rays
    with pytest.raises(K.KerrError, match="KERR_STATIC_MAX_GEODESICS"):
        K.kerr_trace_camera_static(too_big, device=DEV)
    small = K.camera(0.9, 1.0, 1000.0, 20.0, 8, 8)
    host = K.alloc_out(64)                                     # numpy (host) outputs
    with pytest.raises(K.KerrError, match="device memory"):
        K.kerr_trace_camera_static(small, out=host)
