"""The allocation-free entry point kerr_trace_camera_static.

It serves callers that cannot allocate device memory (real-time hosts that
must not call cudaMalloc/cudaFree once running, hosts whose device memory is
budgeted by another framework's pool): all of its scratch lives in one fixed
device array inside the library.  Here it is called through the C ABI and its
outputs are compared with those of kerr_trace_camera, which allocates its
scratch in a context, on two calls in a row (the second call must start from
cleared counters, not from the first call's leftovers).

Both entry points run the same kernels with the same launch configuration,
so their outputs agree bit for bit -- except when more geodesics enter the
FP64 zone than the array's zone buffer holds: those take their zone steps in
place (the same arithmetic in another launch), and the end points then agree
to rounding.

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


def _rel(a, b):
    a = a.detach().cpu().numpy()
    b = b.detach().cpu().numpy()
    den = np.maximum(np.linalg.norm(b, axis=0), 1e-300)
    return float((np.linalg.norm(a - b, axis=0) / den).max())


def _check_equal(got, ref):
    for f in ("x", "k", "status", "steps", "diag"):
        assert torch.equal(getattr(got, f), getattr(ref, f)), f


def _allocating(cams, opts):
    ctx = K.kerr_init(cams[0].a)
    ref = K.kerr_trace_camera(ctx, cams, opts, device=DEV)
    torch.cuda.synchronize()
    ctx.close()
    return ref


@pytest.mark.parametrize("prec", [K.FP32_KAHAN, K.FP64])
def test_static_entry_point_matches_allocating_entry_point(prec):
    K.lib()
    cams = [K.camera(0.9, np.radians(60.0), 1000.0, 20.0, 160, 160),
            K.camera(0.5, np.radians(30.0), 1000.0, 12.0, 64, 32)]
    opts = K.default_opts(prec=prec, tol=1e-6)
    ref = _allocating(cams, opts)
    # two calls in a row through the allocation-free entry point
    for _ in range(2):
        out = K.kerr_trace_camera_static(cams, opts, device=DEV)
        torch.cuda.synchronize()
        _check_equal(out, ref)
    # a different, smaller call after them starts from cleared counters
    one = [cams[1]]
    ref1 = _allocating(one, opts)
    out1 = K.kerr_trace_camera_static(one, opts, device=DEV)
    torch.cuda.synchronize()
    _check_equal(out1, ref1)


def test_static_entry_point_allocates_nothing_after_the_first_call():
    """After one call per precision (the set-up: the array's address and the
    kernels' lazy loading), further calls leave the device's free memory
    unchanged."""
    K.lib()
    cams = [K.camera(0.9, np.radians(60.0), 1000.0, 20.0, 96, 96)]
    outs = {}
    for prec in (K.FP32_KAHAN, K.FP64):
        outs[prec] = K.alloc_out(cams[0].nx * cams[0].ny, DEV)
        K.kerr_trace_camera_static(cams, K.default_opts(prec=prec), out=outs[prec])
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        for prec in (K.FP32_KAHAN, K.FP64):
            K.kerr_trace_camera_static(cams, K.default_opts(prec=prec), out=outs[prec])
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_zone_buffer_holds_every_deferred_geodesic():
    """A 256 x 256 image of the shadow itself: most of its 65536 rays enter the
    FP64 zone; the array's zone buffer holds one entry per geodesic, so all of
    them are deferred, as in the allocating entry point, and the two agree
    bit for bit."""
    K.lib()
    cams = [K.camera(0.9, 1.0, 1000.0, 3.0, 256, 256)]
    opts = K.default_opts(tol=1e-6)
    ctx = K.kerr_init(0.9)
    ref = K.kerr_trace_camera(ctx, cams, opts, device=DEV)
    torch.cuda.synchronize()
    s = K.kerr_get_stats(ctx)
    ctx.close()
    assert s.deferred > 65536 // 2 and s.queue_errors == 0   # most rays enter the zone
    for _ in range(2):
        out = K.kerr_trace_camera_static(cams, opts, device=DEV)
        torch.cuda.synchronize()
        _check_equal(out, ref)


@pytest.mark.parametrize("prec", [K.FP32_KAHAN, K.FP64])
def test_static_entry_point_at_its_ray_limit(prec):
    """Exactly KERR_STATIC_MAX_GEODESICS rays (512 x 256) are accepted and
    match the allocating entry point bit for bit."""
    K.lib()
    cams = [K.camera(0.9, np.radians(60.0), 1000.0, 20.0, 512, 256)]
    assert K.camera_rays(cams) == K.STATIC_MAX_GEODESICS
    opts = K.default_opts(prec=prec, tol=1e-6)
    ref = _allocating(cams, opts)
    out = K.kerr_trace_camera_static(cams, opts, device=DEV)
    torch.cuda.synchronize()
    _check_equal(out, ref)


def test_static_entry_point_limits():
    K.lib()
    too_big = K.camera(0.9, 1.0, 1000.0, 20.0, 512, 257)     # 131584 > 131072 rays
    with pytest.raises(K.KerrError, match="KERR_STATIC_MAX_GEODESICS"):
        K.kerr_trace_camera_static(too_big, device=DEV)
    small = K.camera(0.9, 1.0, 1000.0, 20.0, 8, 8)
    host = K.alloc_out(64)                                     # numpy (host) outputs
    with pytest.raises(K.KerrError, match="device memory"):
        K.kerr_trace_camera_static(small, out=host)
    # the same option and camera checks as kerr_trace_camera
    for bad in (dict(tol=float("inf")), dict(h0=float("inf")), dict(r_escape=float("nan"))):
        with pytest.raises(K.KerrError):
            K.kerr_trace_camera_static(small, K.default_opts(**bad), device=DEV)
    with pytest.raises(K.KerrError):
        K.kerr_trace_camera_static(K.camera(0.9, 1.0, 1000.0, float("inf"), 8, 8), device=DEV)
