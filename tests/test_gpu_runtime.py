"""Runtime services of the library on the GPU: deferred clipping, the abort
flag, resuming interrupted geodesics, allocation-failure injection, surrogate
parameter files, the autotuner with its cache, and the ALU-peak kernel.

Failures are made on the host (a flag the host sets, an allocation the
library is told to refuse, a step cap); nothing here faults or hangs the GPU.
"""
import threading
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import oracle as O  # noqa: E402
from paper_1706_07062_gb300 import kerr as K  # noqa: E402
from paper_1706_07062_gb300 import workloads as W  # noqa: E402
from parity import compare, rel_errors, to_np  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def cam(spec: W.CameraSpec) -> K.Camera:
    return K.camera(*spec.as_tuple())


# ---------------------------------------------------------------------------
# deferred clipping
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("zone_prec", [K.ZONE_FP64, K.ZONE_F32X2])
def test_deferred_clip_equals_in_place_clip(zone_prec):
    """Without crossing labels the FP32 path leaves the clipping of end points
    to the clip pass; with labels it clips inside the stepping loops.  Both
    run the same iteration from the same state, so end states, statuses and
    step counts are identical, and every end point but those of geodesics
    that start beyond the escape radius is clipped."""
    spec = W.CameraSpec(0.9, 1.0, 1000.0, 12.0, 96, 96)
    ctx = K.kerr_init(spec.a)
    opts = K.default_opts(zone_prec=zone_prec)
    deferred = K.alloc_out(spec.n, DEV)
    K.kerr_trace_camera(ctx, cam(spec), opts, out=deferred)
    s = K.kerr_get_stats(ctx)
    inplace = K.alloc_out(spec.n, DEV, cross=True)
    K.kerr_trace_camera(ctx, cam(spec), opts, out=inplace)
    s2 = K.kerr_get_stats(ctx)
    torch.cuda.synchronize()
    for f in ("x", "k", "status", "steps", "diag"):
        assert torch.equal(getattr(deferred, f), getattr(inplace, f)), f
    st = to_np(deferred.status)
    assert s.clips == int(np.isin(st, (K.ESCAPED, K.CAPTURED)).sum()) and s.clips > 0
    assert s.clip_rhs >= 8 * s.clips             # one right-hand side + >= 1 iteration
    assert s2.clips == 0                          # labels on: clipped in place
    ctx.close()


def test_deferred_clip_particles_end_on_their_end_time():
    ps = W.particles(n=3000, periods=2)
    ctx = K.kerr_init(ps.a)
    opts = K.default_opts(tol=1e-8, r_escape=-1.0, max_steps=10_000_000)
    out = K.kerr_trace_particles(ctx, torch.tensor(ps.x0, device=DEV),
                                 torch.tensor(ps.v0, device=DEV),
                                 torch.tensor(ps.t_end, device=DEV), opts)
    torch.cuda.synchronize()
    s = K.kerr_get_stats(ctx)
    st = to_np(out.status)
    ended = st == K.ENDTIME
    assert ended.sum() > 2000 and s.clips == int(np.isin(st, (K.ENDTIME, K.CAPTURED)).sum())
    t = to_np(out.x)[0]
    assert np.all(np.abs(t[ended] - ps.t_end[ended]) <= 3e-6 * np.abs(ps.t_end[ended]))
    ctx.close()


# ---------------------------------------------------------------------------
# abort flag and resume
# ---------------------------------------------------------------------------
def test_abort_flag_stops_a_running_launch():
    """The host sets the context's abort flag while a long FP64 launch runs:
    the launch returns early, unfinished geodesics end with KERR_TIMEOUT and
    their state; cleared, the flag lets the next call run to the end."""
    spec = W.CameraSpec(0.9, 1.0, 1000.0, 20.0, 384, 384)
    ctx = K.kerr_init(spec.a)
    flag = K.kerr_abort_flag(ctx)
    assert flag.value() == 0
    opts = K.default_opts(prec=K.FP64, tol=1e-13)
    out = K.alloc_out(spec.n, DEV, diag=False)
    K.kerr_trace_camera(ctx, cam(spec), opts, out=out)          # warm (graph, buffers)
    torch.cuda.synchronize()
    full_ms = K.kerr_get_stats(ctx).kernel_ms
    assert full_ms > 100.0, full_ms                              # long enough to interrupt
    assert (to_np(out.status) == K.TIMEOUT).sum() == 0
    t0 = time.perf_counter()
    K.kerr_trace_camera(ctx, cam(spec), opts, out=out)          # asynchronous
    threading.Timer(0.2 * full_ms * 1e-3, flag.set).start()
    torch.cuda.synchronize()
    wall_ms = (time.perf_counter() - t0) * 1e3
    s = K.kerr_get_stats(ctx)
    st = to_np(out.status)
    assert (st == K.TIMEOUT).sum() > 0
    assert set(np.unique(st)) <= {K.ESCAPED, K.CAPTURED, K.TIMEOUT}
    assert s.kernel_ms < 0.8 * full_ms and wall_ms < full_ms
    assert s.geodesics == spec.n and sum(s.status_count) == spec.n
    flag.clear()
    K.kerr_trace_camera(ctx, cam(spec), opts, out=out)
    torch.cuda.synchronize()
    assert (to_np(out.status) == K.TIMEOUT).sum() == 0
    ctx.close()


@pytest.mark.parametrize("prec", [K.FP64, K.FP32_KAHAN])
def test_resume_from_interrupted_states(prec):
    """Geodesics stopped after 30 attempts (KERR_MAXSTEPS) resume from their
    returned states through kerr_trace_rays.  FP64: the resumed end points
    equal the oracle's integration from the same returned states element by
    element (1e-9), and statuses match the uninterrupted oracle run.
    FP32+Kahan: the resumed end points meet the 1e-5 gate against the
    uninterrupted oracle.  The escape radius is fixed at 1000 M on both
    sides (a resumed geodesic's own start radius is where it stopped)."""
    spec = W.CAMERA_64
    fp32 = prec == K.FP32_KAHAN
    tol = 1e-6 if fp32 else W.TOL_64
    ctx = K.kerr_init(spec.a)
    idx = np.arange(spec.n)
    y0 = O.camera_ic(spec.a, spec.incl, spec.r_obs, spec.half_width, spec.nx, spec.ny, idx)
    first = K.kerr_trace_camera(ctx, cam(spec),
                                K.default_opts(prec=prec, tol=tol, max_steps=30, r_escape=1000.0),
                                device=DEV)
    torch.cuda.synchronize()
    st1 = to_np(first.status)
    stopped = st1 == K.MAXSTEPS
    assert stopped.mean() > 0.5
    resumed = K.kerr_trace_rays(ctx, first.x.contiguous(), first.k.contiguous(),
                                K.default_opts(prec=prec, tol=tol, r_escape=1000.0))
    torch.cuda.synchronize()
    oo = O.Opts(tol=tol, r_escape=1000.0)
    if fp32:
        s = compare("resume/fp32", spec.a, y0, oo, resumed, idx, 1e-5, fp32=True,
                    max_ill_frac=0.19)
        print(s)
    else:
        part = O.trace(spec.a, y0, O.Opts(tol=tol, r_escape=1000.0, max_steps=30))
        assert np.array_equal(part.status == O.MAXSTEPS, stopped)
        # the interrupted states lie on the same trajectories, but where along
        # them each stopped depends on the step lengths, whose last digits
        # follow the rounding of the error estimate far from the hole (where
        # it is tiny): they agree along the track to ~1e-5, not to the gate
        ex, ek, _ = rel_errors(to_np(first.x), to_np(first.k), part.y)
        assert max(ex.max(), ek.max()) < 1e-4
        # resuming is tracing from the returned states: against the oracle
        # from those very states, element by element
        y_stop = np.concatenate([to_np(first.x).T, to_np(first.k).T], axis=1)
        s = compare("resume/fp64", spec.a, y_stop, oo, resumed, idx, 1e-9, fp32=False,
                    max_ill_frac=0.01)
        print(s)
        full = O.trace(spec.a, y0, oo)
        same = to_np(resumed.status) == full.status
        assert same.mean() > 0.99
    ctx.close()


# ---------------------------------------------------------------------------
# allocation failure
# ---------------------------------------------------------------------------
def test_allocation_failure_returns_enomem_and_context_survives():
    spec = W.CameraSpec(0.9, 1.0, 1000.0, 12.0, 64, 48)
    ref_ctx = K.kerr_init(spec.a)
    ref = K.kerr_trace_camera(ref_ctx, cam(spec), K.default_opts(), device=DEV)
    torch.cuda.synchronize()
    ref_ctx.close()
    try:
        K.kerr_debug_fail_alloc(1)                 # kerr_init's scratch
        with pytest.raises(K.KerrError, match=r"\(-2\)"):
            K.kerr_init(spec.a)
        ctx = K.kerr_init(spec.a)
        for nth in (1, 2):                         # work buffer, then zone buffer
            K.kerr_debug_fail_alloc(nth)
            with pytest.raises(K.KerrError, match=r"\(-2\)"):
                K.kerr_trace_camera(ctx, cam(spec), K.default_opts(), device=DEV)
            K.kerr_debug_fail_alloc(0)
            out = K.kerr_trace_camera(ctx, cam(spec), K.default_opts(), device=DEV)
            torch.cuda.synchronize()
            for f in ("x", "k", "status", "steps"):
                assert torch.equal(getattr(out, f), getattr(ref, f)), (nth, f)
            ctx.close()
            ctx = K.kerr_init(spec.a)
        ctx.close()
    finally:
        K.kerr_debug_fail_alloc(0)


# ---------------------------------------------------------------------------
# surrogate parameter files
# ---------------------------------------------------------------------------
def test_surrogate_save_and_load(tmp_path):
    s = K.Surrogate(W.surrogate_init())
    rng = np.random.default_rng(11)
    x = torch.tensor(np.stack([rng.uniform(-1, 1, 4096), rng.uniform(-1, 1, 4096),
                               rng.uniform(0, 1, 4096), rng.uniform(0.1, 1, 4096)], 1),
                     dtype=torch.float32, device=DEV)
    y = torch.tensor(rng.normal(size=(4096, 8)), dtype=torch.float32, device=DEV)
    m = torch.ones((4096, 8), dtype=torch.float32, device=DEV)
    K.kerr_surrogate_train(s, x, y, m, epochs=2, batch=1024, lr=1e-3)   # non-trivial weights
    path = str(tmp_path / "surrogate.bin")
    K.kerr_surrogate_save(s, path)
    t = K.kerr_surrogate_load(path)
    assert np.array_equal(s.params(), t.params())
    assert np.array_equal(K.kerr_params_read(path), s.params())
    torch.cuda.synchronize()
    assert torch.equal(K.kerr_surrogate_forward(s, x), K.kerr_surrogate_forward(t, x))
    s.close()
    t.close()


# ---------------------------------------------------------------------------
# autotuner
# ---------------------------------------------------------------------------
def test_autotune_cameras_with_cache(tmp_path):
    cams = [K.camera(0.9, 1.0, 1000.0, 12.0, 64, 64), K.camera(0.5, 0.4, 1000.0, 20.0, 96, 48)]
    cache = str(tmp_path / "tune.txt")
    ctx = K.kerr_init(0.9)
    nvar, nz = K.kerr_num_variants(), K.kerr_num_zone_variants()
    t = K.kerr_autotune_cameras(ctx, cams, K.default_opts(), sample=4096, cache_path=cache)
    assert t.from_cache == 0 and t.timed == nvar + nz - 1
    assert 0 <= t.variant < nvar and 0 <= t.zone_variant < nz and t.ms > 0
    K.kerr_trace_camera(ctx, cams, K.default_opts(), device=DEV)
    torch.cuda.synchronize()
    assert K.kerr_get_stats(ctx).variant == t.variant      # applied to later calls
    # a new context reads the choice from the cache without timing
    ctx2 = K.kerr_init(0.9)
    t2 = K.kerr_autotune_cameras(ctx2, cams, K.default_opts(), sample=4096, cache_path=cache)
    assert t2.from_cache == 1 and t2.timed == 0
    assert (t2.variant, t2.zone_variant) == (t.variant, t.zone_variant)
    K.kerr_trace_camera(ctx2, cams, K.default_opts(), device=DEV)
    torch.cuda.synchronize()
    assert K.kerr_get_stats(ctx2).variant == t.variant
    # FP64: one-geodesic-per-thread variants only, no zone phase
    t64 = K.kerr_autotune_cameras(ctx2, cams, K.default_opts(prec=K.FP64), sample=2048)
    _, _, rays, _ = K.kerr_variant_shape(t64.variant)
    assert rays == 1 and t64.zone_variant == -1
    assert t64.timed == sum(K.kerr_variant_shape(v)[2] == 1 for v in range(nvar))
    gpu = f"{torch.cuda.get_device_name(0)} ({torch.cuda.get_device_properties(0).multi_processor_count} SMs)"
    key = K.kerr_tune_key_cameras(cams, K.default_opts())
    hit = K.kerr_tune_cache_lookup(cache, gpu, key)
    assert hit is not None and hit.variant == t.variant
    ctx.close()
    ctx2.close()


def test_autotune_particles():
    ps = W.particles(n=1 << 12, periods=1)
    ctx = K.kerr_init(ps.a)
    opts = K.default_opts(tol=1e-6, r_escape=-1.0, max_steps=10_000_000)
    x0 = torch.tensor(ps.x0, device=DEV)
    v0 = torch.tensor(ps.v0, device=DEV)
    te = torch.tensor(ps.t_end, device=DEV)
    t = K.kerr_autotune_particles(ctx, x0, v0, te, opts, sample=1024)
    assert t.from_cache == 0 and t.timed == K.kerr_num_variants() + K.kerr_num_zone_variants() - 1
    out = K.kerr_trace_particles(ctx, x0, v0, te, opts)
    torch.cuda.synchronize()
    assert K.kerr_get_stats(ctx).variant == t.variant
    assert set(np.unique(to_np(out.status))) <= {K.CAPTURED, K.ENDTIME, K.INVALID_IC}
    ctx.close()


# ---------------------------------------------------------------------------
# ALU peak kernel
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind", [K.PEAK_FP32, K.PEAK_FP32X2, K.PEAK_FP64])
def test_fma_chain_counts_its_flops(kind):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    sink = torch.zeros(sms * 4 * 256, dtype=torch.float32, device=DEV)
    rounds = 64
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    fl = K.kerr_fma_chain(kind, rounds, sink, 4)
    e1.record()
    torch.cuda.synchronize()
    per = 4 if kind == K.PEAK_FP32X2 else 2
    assert fl == per * sms * 4 * 256 * rounds * 16 * 8
    assert e0.elapsed_time(e1) > 0
    assert torch.count_nonzero(sink) == 0            # the chains never store
    with pytest.raises(K.KerrError):
        K.kerr_fma_chain(kind, 0, sink, 4)
