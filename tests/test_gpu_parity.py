"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Gates: 1e-9 relative end-point error for the FP64 path, 1e-5 for the FP32+Kahan
path, on every geodesic the oracle does not flag as ill-conditioned (rays
grazing the photon ring amplify any perturbation exponentially; see
parity.oracle_flags).  Status must agree on every well-conditioned geodesic.
"""
import math

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


@pytest.fixture(scope="module")
def ctx():
    K.lib()
    c = K.kerr_init(0.9)
    yield c
    c.close()


def cam(spec: W.CameraSpec) -> K.Camera:
    return K.camera(*spec.as_tuple())


def oracle_camera_ic(spec: W.CameraSpec, idx):
    return O.camera_ic(spec.a, spec.incl, spec.r_obs, spec.half_width, spec.nx, spec.ny, idx)


# ---------------------------------------------------------------------------
# 64 x 64 image, a = 0.9, i = 60 deg, tol 1e-10: every ray against the oracle
# ---------------------------------------------------------------------------
def test_camera64_fp64_every_ray(ctx):
    spec = W.CAMERA_64
    opts = K.default_opts(prec=K.FP64, tol=W.TOL_64)
    out = K.kerr_trace_camera(ctx, cam(spec), opts, device=DEV)
    torch.cuda.synchronize()
    idx = np.arange(spec.n)
    y0 = oracle_camera_ic(spec, idx)
    s = compare("camera64/fp64", spec.a, y0, O.Opts(tol=W.TOL_64), out, idx, 1e-9, fp32=False,
                max_ill_frac=0.01)
    print(s)


def test_camera64_fp32_every_ray(ctx):
    """The FP32 path at tol 1e-6 against the oracle at the same tolerance."""
    spec = W.CAMERA_64
    opts = K.default_opts(prec=K.FP32_KAHAN, tol=1e-6)
    out = K.kerr_trace_camera(ctx, cam(spec), opts, device=DEV)
    torch.cuda.synchronize()
    idx = np.arange(spec.n)
    y0 = oracle_camera_ic(spec, idx)
    s = compare("camera64/fp32", spec.a, y0, O.Opts(tol=1e-6), out, idx, 1e-5, fp32=True,
                max_ill_frac=0.19)
    print(s)


# ---------------------------------------------------------------------------
# 1024 x 1024 image, a = 0.99, i = 17 deg, tol 1e-6: full launch, seeded
# 4096-ray subset against the oracle (the benchmark's launch configuration)
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def c1024_oracle():
    spec = W.CAMERA_1024
    idx = W.camera_subset(spec)
    y0 = oracle_camera_ic(spec, idx)
    ref = O.trace(spec.a, y0, O.Opts(tol=W.TOL_1024))
    return idx, y0, ref


@pytest.mark.parametrize("prec,zone", [(K.FP32_KAHAN, K.ZONE_FP64), (K.FP32_KAHAN, K.ZONE_F32X2),
                                       (K.FP64, K.ZONE_FP64)])
def test_camera1024_full_launch_subset(ctx, c1024_oracle, prec, zone):
    spec = W.CAMERA_1024
    idx, y0, ref = c1024_oracle
    opts = K.default_opts(prec=prec, tol=W.TOL_1024, zone_prec=zone)
    out = K.kerr_trace_camera(ctx, cam(spec), opts, device=DEV)
    torch.cuda.synchronize()
    st = to_np(out.status)
    assert set(np.unique(st)) <= {K.ESCAPED, K.CAPTURED}
    gate = 1e-5 if prec == K.FP32_KAHAN else 1e-9
    s = compare(f"camera1024/{prec}/{zone}", spec.a, y0, O.Opts(tol=W.TOL_1024), out, idx, gate,
                fp32=(prec == K.FP32_KAHAN), ref=ref,
                max_ill_frac=0.11 if prec == K.FP32_KAHAN else 0.01)
    print(s)
    # null constraint reported per ray (FP64 diagnostics): |u^2| small
    u2 = to_np(out.diag)[3]
    kt = np.abs(to_np(out.k)[0])
    assert np.all(np.abs(u2) <= 1e-3 * np.maximum(1.0, kt) ** 2)


# ---------------------------------------------------------------------------
# entry points agree with each other
# ---------------------------------------------------------------------------
def test_trace_rays_matches_camera(ctx):
    spec = W.CameraSpec(0.9, 1.0, 1000.0, 12.0, 16, 16)
    opts = K.default_opts(prec=K.FP64, tol=1e-9)
    c2 = K.kerr_init(spec.a)
    cam_out = K.kerr_trace_camera(c2, cam(spec), opts, device=DEV)
    y0 = oracle_camera_ic(spec, np.arange(spec.n))
    x0 = torch.tensor(np.ascontiguousarray(y0[:, :4].T), device=DEV)
    k0 = torch.tensor(np.ascontiguousarray(y0[:, 4:].T), device=DEV)
    opts_r = K.default_opts(prec=K.FP64, tol=1e-9, r_escape=0.0)
    ray_out = K.kerr_trace_rays(c2, x0, k0, opts_r)
    torch.cuda.synchronize()
    ex, ek, _ = rel_errors(to_np(ray_out.x), to_np(ray_out.k),
                           np.concatenate([to_np(cam_out.x).T, to_np(cam_out.k).T], 1))
    assert np.array_equal(to_np(ray_out.status), to_np(cam_out.status))
    assert max(ex.max(), ek.max()) < 1e-9
    c2.close()


@pytest.mark.parametrize("prec", [K.FP32_KAHAN, K.FP64])
def test_host_and_device_buffers_agree(ctx, prec):
    """Pageable host outputs are staged through device memory; page-locked
    ones receive end points and diagnostics in place from the kernels (twice
    into the same buffers, so that the second call replays a cached graph)."""
    spec = W.CameraSpec(0.5, 0.7, 1000.0, 10.0, 33, 31)
    opts = K.default_opts(prec=prec, tol=1e-6)
    dev = K.kerr_trace_camera(ctx, cam(spec), opts, device=DEV)
    host = K.kerr_trace_camera(ctx, cam(spec), opts)               # numpy outputs
    pinned = K.alloc_out(spec.n, device="cpu", pinned=True)
    outs = [host]
    for _ in range(2):
        for t in (pinned.x, pinned.k, pinned.diag):
            t.fill_(np.nan)
        K.kerr_trace_camera(ctx, cam(spec), opts, out=pinned)
        outs.append(K.TraceOut(pinned.x.clone(), pinned.k.clone(), pinned.status.clone(),
                               pinned.steps.clone(), pinned.diag.clone()))
    torch.cuda.synchronize()
    for o in outs:
        assert np.array_equal(to_np(o.x), to_np(dev.x))
        assert np.array_equal(to_np(o.k), to_np(dev.k))
        assert np.array_equal(to_np(o.status), to_np(dev.status))
        assert np.array_equal(to_np(o.steps), to_np(dev.steps))
        assert np.array_equal(to_np(o.diag), to_np(dev.diag), equal_nan=True)


def test_batched_cameras_equal_single_cameras(ctx):
    specs = [W.CameraSpec(0.3, 0.4, 1000.0, 25.0, 17, 9), W.CameraSpec(0.95, 1.2, 800.0, 15.0, 32, 32),
             W.CameraSpec(0.0, 0.1, 1000.0, 8.0, 5, 7)]
    opts = K.default_opts(prec=K.FP32_KAHAN, tol=1e-6)
    batch = K.kerr_trace_camera(ctx, [cam(s) for s in specs], opts, device=DEV)
    off = 0
    for s in specs:
        one = K.kerr_trace_camera(ctx, cam(s), opts, device=DEV)
        torch.cuda.synchronize()
        sl = slice(off, off + s.n)
        assert torch.equal(batch.x[:, sl], one.x)
        assert torch.equal(batch.k[:, sl], one.k)
        assert torch.equal(batch.status[sl], one.status)
        off += s.n


# ---------------------------------------------------------------------------
# particles: time-like geodesics, per-particle end times
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [K.FP64, K.FP32_KAHAN])
def test_particles_subset(prec):
    """512 stratified particles of a 2^14 draw, one radial period each, at tol
    1e-8 in both precisions: element-wise end-point parity at 1e-9 (FP64) and
    1e-5 (FP32+Kahan).  Over more periods, or at tol 1e-6, particle end
    points at a fixed end time are not determined to 1e-5 by the method (the
    oracle's own tol/100, perturbation and FP32-rounding runs move them
    further: orbital phase error grows with every period), so longer runs are
    judged by their constants of motion (test_particles_full_size_sampled)."""
    ps = W.particles(n=1 << 14, periods=1)
    sub = W.particle_subset(ps, k=512)
    a = ps.a
    c = K.kerr_init(a)
    opts = K.default_opts(prec=prec, tol=1e-8, r_escape=-1.0, max_steps=10_000_000)
    x0 = torch.tensor(ps.x0, device=DEV)
    v0 = torch.tensor(ps.v0, device=DEV)
    te = torch.tensor(ps.t_end, device=DEV)
    out = K.kerr_trace_particles(c, x0, v0, te, opts)
    torch.cuda.synchronize()
    st = to_np(out.status)
    assert set(np.unique(st)) <= {K.CAPTURED, K.ENDTIME, K.INVALID_IC}
    y0, ok = O.particle_ic(a, ps.x0[:, sub].T, ps.v0[:, sub].T)
    assert np.array_equal(st[sub] == K.INVALID_IC, ~ok)
    keep = np.nonzero(ok)[0]
    oo = O.Opts(tol=opts.tol, r_escape=-1.0, max_steps=10_000_000)
    ref = O.trace(a, y0[keep], oo, t_end=ps.t_end[sub][keep])
    gate = 1e-9 if prec == K.FP64 else 1e-5
    s = compare(f"particles/{prec}", a, y0[keep], oo, out, sub[keep], gate,
                fp32=(prec == K.FP32_KAHAN), ref=ref, max_bad_frac=0.0,
                t_end=ps.t_end[sub][keep], max_ill_frac=0.01 if prec == K.FP64 else 0.10)
    print(s)
    c.close()


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------
def test_sizes_and_degenerate_states(ctx):
    a = 0.9
    rh = 1 + math.sqrt(1 - a * a)
    opts = K.default_opts(prec=K.FP64, tol=1e-8)
    for n in (1, 31, 32, 33, 1000):
        spec = W.CameraSpec(a, 0.5, 1000.0, 10.0, n, 1)
        out = K.kerr_trace_camera(ctx, cam(spec), opts, device=DEV)
        torch.cuda.synchronize()
        y0 = oracle_camera_ic(spec, np.arange(n))
        ref = O.trace(a, y0, O.Opts(tol=1e-8))
        assert np.array_equal(to_np(out.status), ref.status)
    # n = 0 is a no-op
    empty = K.alloc_out(0, DEV)
    K.kerr_trace_rays(ctx, torch.zeros((4, 0), dtype=torch.float64, device=DEV),
                      torch.zeros((4, 0), dtype=torch.float64, device=DEV), opts, out=empty)
    # NaN, inside the capture radius, max_steps
    y = np.array([[0, np.nan, 0, 0, -1, 0.1, 0, 0],
                  [0, 1.005 * rh, 0, 0, -1, 0.1, 0, 0],
                  oracle_camera_ic(W.CAMERA_64, [100])[0]])
    x0 = torch.tensor(np.ascontiguousarray(y[:, :4].T), device=DEV)
    k0 = torch.tensor(np.ascontiguousarray(y[:, 4:].T), device=DEV)
    for prec in (K.FP64, K.FP32_KAHAN):
        o = K.default_opts(prec=prec, tol=1e-8, max_steps=3)
        out = K.kerr_trace_rays(ctx, x0, k0, o)
        torch.cuda.synchronize()
        assert to_np(out.status).tolist() == [K.NONFINITE, K.CAPTURED, K.MAXSTEPS]
        assert to_np(out.steps).tolist() == [0, 0, 3]
        assert np.array_equal(to_np(out.x)[:, 1], y[1, :4])


def test_budget_gives_timeout_not_hang(ctx):
    spec = W.CameraSpec(0.9, 0.5, 1000.0, 20.0, 256, 256)
    opts = K.default_opts(prec=K.FP64, tol=1e-12, budget_ns=200_000)   # 0.2 ms
    out = K.kerr_trace_camera(ctx, cam(spec), opts, device=DEV)
    torch.cuda.synchronize()
    st = to_np(out.status)
    assert (st == K.TIMEOUT).sum() > 0
    assert set(np.unique(st)) <= {K.ESCAPED, K.CAPTURED, K.TIMEOUT}
    s = K.kerr_get_stats(ctx)
    assert s.geodesics == spec.n and sum(s.status_count) == spec.n


@pytest.mark.parametrize("every", [1, 8])
@pytest.mark.parametrize("prec", [K.FP64, K.FP32_KAHAN])
def test_renormalisation_matches_oracle(ctx, c1024_oracle, prec, every):
    """Null renormalisation (Sec. 2.2: k^t re-solved from the null condition,
    here every `every` accepted steps, on the root nearest the current k^t)
    against the oracle's renormalisation, element by element: every ray of
    the 64 x 64 image (FP64 at tol 1e-10, FP32+Kahan at tol 1e-6) and the
    1024 x 1024 image's seeded subset from a full launch (tol 1e-6), at the
    1e-9 (FP64) and 1e-5 (FP32) gates."""
    fp32 = prec == K.FP32_KAHAN
    gate = 1e-5 if fp32 else 1e-9
    spec = W.CAMERA_64
    tol = 1e-6 if fp32 else W.TOL_64
    out = K.kerr_trace_camera(ctx, cam(spec),
                              K.default_opts(prec=prec, tol=tol, renorm_every=every), device=DEV)
    torch.cuda.synchronize()
    idx = np.arange(spec.n)
    y0 = oracle_camera_ic(spec, idx)
    s = compare(f"renorm{every}/camera64/{prec}", spec.a, y0, O.Opts(tol=tol, renorm_every=every),
                out, idx, gate, fp32=fp32, max_ill_frac=0.19 if fp32 else 0.01)
    print(s)
    spec = W.CAMERA_1024
    idx, y0, _ = c1024_oracle
    oo = O.Opts(tol=W.TOL_1024, renorm_every=every)
    out = K.kerr_trace_camera(ctx, cam(spec),
                              K.default_opts(prec=prec, tol=W.TOL_1024, renorm_every=every),
                              device=DEV)
    torch.cuda.synchronize()
    s = compare(f"renorm{every}/camera1024/{prec}", spec.a, y0, oo, out, idx, gate, fp32=fp32,
                max_ill_frac=0.11 if fp32 else 0.01)
    print(s)


def test_renormalisation_keeps_null_constraint(ctx):
    """Renormalising after every accepted step keeps |g k k| of escaping rays
    no larger than without it."""
    spec = W.CameraSpec(0.99, 0.3, 1000.0, 6.0, 16, 16)
    for prec in (K.FP64, K.FP32_KAHAN):
        plain = K.kerr_trace_camera(ctx, cam(spec), K.default_opts(prec=prec), device=DEV)
        ren = K.kerr_trace_camera(ctx, cam(spec), K.default_opts(prec=prec, renorm_every=1),
                                  device=DEV)
        torch.cuda.synchronize()
        esc = to_np(ren.status) == K.ESCAPED
        assert np.abs(to_np(ren.diag)[3][esc]).max() <= np.abs(to_np(plain.diag)[3][esc]).max()


def test_invalid_arguments_are_rejected(ctx):
    with pytest.raises(K.KerrError):
        K.kerr_init(1.5)
    with pytest.raises(K.KerrError):
        K.kerr_trace_camera(ctx, K.camera(0.5, 0.3, 1000.0, 10.0, 0, 4), device=DEV)
    with pytest.raises(K.KerrError):
        K.kerr_trace_camera(ctx, K.camera(1.2, 0.3, 1000.0, 10.0, 4, 4), device=DEV)
    with pytest.raises(K.KerrError):
        K.kerr_trace_camera(ctx, K.camera(0.5, 0.3, 1000.0, 10.0, 4, 4),
                            K.default_opts(tol=-1.0), device=DEV)
    with pytest.raises(K.KerrError):
        K.kerr_trace_camera(ctx, K.camera(0.5, 0.3, 1000.0, 10.0, 4, 4),
                            K.default_opts(variant=99), device=DEV)


# FP32-phase right-hand-side mode of each stepping variant (0 inline, 1 call)
def variant_family(v):
    """(geodesics per thread, right-hand-side mode): variants of one family
    run the same arithmetic per geodesic."""
    _, _, rays, rhs_mode = K.kerr_variant_shape(v)
    return rays, rhs_mode


def test_every_variant_and_autotune(ctx):
    """Variants with the same right-hand-side code agree bit for bit (the
    launch shape only moves geodesics between lanes).  Inline and
    out-of-line FP32 right-hand sides may fuse multiply-adds differently, and
    so may the packed two-per-thread steps; FP32 rounding differences grow
    along a trajectory: each family is checked against the oracle at the FP32
    gate instead."""
    fams = {variant_family(v) for v in range(K.kerr_num_variants())}
    assert fams == {(1, 0), (1, 1), (2, 1)}
    spec = W.CameraSpec(0.9, 1.0, 1000.0, 20.0, 48, 48)
    outs = []
    for v in range(K.kerr_num_variants()):
        o = K.kerr_trace_camera(ctx, cam(spec), K.default_opts(variant=v), device=DEV)
        torch.cuda.synchronize()
        outs.append(o)
    first = {}
    for v, o in enumerate(outs):
        m = variant_family(v)
        if m not in first:
            first[m] = v
            continue
        b = outs[first[m]]
        assert torch.equal(o.x, b.x) and torch.equal(o.k, b.k) and torch.equal(o.status, b.status)
    idx = np.arange(spec.n)
    y0 = oracle_camera_ic(spec, idx)
    oo = O.Opts(tol=1e-6)
    ref = O.trace(spec.a, y0, oo)
    from parity import oracle_flags
    flags = oracle_flags(spec.a, y0, oo, ref, 1e-5, fp32=True)
    for m, v in first.items():
        s = compare(f"variant{v}/fp32", spec.a, y0, oo, outs[v], idx, 1e-5, fp32=True, ref=ref,
                    flags=flags, max_ill_frac=0.19)
        print(s)
    best = K.kerr_autotune(ctx, cam(spec), K.default_opts(), sample=2048)
    assert 0 <= best < K.kerr_num_variants()
    # two geodesics per thread is an FP32-only launch shape
    best64 = K.kerr_autotune(ctx, cam(spec), K.default_opts(prec=K.FP64), sample=1024)
    assert variant_family(best64)[0] == 1
    x2 = next(v for v in range(K.kerr_num_variants()) if variant_family(v)[0] == 2)
    with pytest.raises(K.KerrError):
        K.kerr_trace_camera(ctx, cam(spec), K.default_opts(prec=K.FP64, variant=x2), device=DEV)


def test_two_per_thread_edge_cases(ctx):
    """Two geodesics per thread with ragged counts (a last thread holding one
    geodesic, fewer geodesics than one warp's slots), particles with end
    times and crossing labels: the same end states, statuses, step counts
    and labels in every two-per-thread launch shape, and within the FP32 gate
    of the one-per-thread kernel with out-of-line right-hand sides."""
    x2 = [v for v in range(K.kerr_num_variants()) if variant_family(v)[0] == 2]
    ref_v = next(v for v in range(K.kerr_num_variants()) if variant_family(v) == (1, 1))
    for nx, ny in ((1, 1), (7, 5), (33, 31)):
        spec = W.CameraSpec(0.9, 1.0, 1000.0, 12.0, nx, ny)
        outs = []
        for v in x2 + [ref_v]:
            o = K.alloc_out(spec.n, DEV, cross=True)
            K.kerr_trace_camera(ctx, cam(spec), K.default_opts(variant=v), out=o)
            torch.cuda.synchronize()
            outs.append(o)
        for o in outs[1:-1]:
            for f in ("x", "k", "status", "steps"):
                assert torch.equal(getattr(o, f), getattr(outs[0], f)), (nx, ny, f)
            assert torch.equal(torch.nan_to_num(o.cross, 7.0), torch.nan_to_num(outs[0].cross, 7.0))
        r = outs[-1]
        assert torch.equal(r.status, outs[0].status)
        ex, ek, _ = rel_errors(to_np(outs[0].x), to_np(outs[0].k),
                               np.concatenate([to_np(r.x).T, to_np(r.k).T], 1))
        # two FP32 roundings of one method; end points on the capture sphere
        # amplify differences near the horizon
        assert np.median(np.maximum(ex, ek)) < 1e-4
    ps = W.particles(n=999, periods=3)
    c2 = K.kerr_init(ps.a)
    x0 = torch.tensor(ps.x0, device=DEV)
    v0 = torch.tensor(ps.v0, device=DEV)
    te = torch.tensor(ps.t_end, device=DEV)
    res = []
    for v in x2 + [ref_v]:
        o = K.default_opts(tol=1e-6, r_escape=-1.0, max_steps=10_000_000, variant=v)
        res.append(K.kerr_trace_particles(c2, x0, v0, te, o))
        torch.cuda.synchronize()
    for o in res[1:-1]:
        for f in ("x", "k", "status", "steps"):
            assert torch.equal(getattr(o, f), getattr(res[0], f)), f
    assert torch.equal(res[0].status, res[-1].status)
    ended = to_np(res[0].status) == K.ENDTIME
    # end-time clip tolerance of the FP32 steps: 2e-6 relative
    assert ended.any() and np.allclose(to_np(res[0].x)[0][ended], ps.t_end[ended], rtol=5e-6)
    c2.close()


# ---------------------------------------------------------------------------
# deferred FP64-zone phase
# ---------------------------------------------------------------------------
# zone variants: right-hand-side mode (0 inline, 1 one out-of-line copy, 2
# out-of-line pairs); variant 7 is variant 3 with two-lane attempts in the
# phase's tail, the same arithmetic
ZONE_RHS_MODE = [0, 0, 0, 1, 2, 2, 2, 1, 2]


def test_zone_launch_shapes_agree(ctx):
    """Zone-phase variants with the same right-hand-side code give identical
    end states (the launch shape only changes which lane runs a geodesic).
    Inline and out-of-line right-hand sides are the same source arithmetic,
    but the compiler may fuse a multiply-add differently across the call
    boundary: end states then agree to rounding, with the same statuses and
    step counts."""
    assert K.kerr_num_zone_variants() == len(ZONE_RHS_MODE)
    spec = W.CameraSpec(0.99, 0.3, 1000.0, 8.0, 96, 96)
    outs = [K.kerr_trace_camera(ctx, cam(spec), K.default_opts(zone_variant=v), device=DEV)
            for v in range(K.kerr_num_zone_variants())]
    torch.cuda.synchronize()
    first = {}
    for v, o in enumerate(outs):
        m = ZONE_RHS_MODE[v]
        if m in first:
            b = outs[first[m]]
            assert torch.equal(o.x, b.x) and torch.equal(o.k, b.k)
        else:
            first[m] = v
        b = outs[0]
        assert torch.equal(o.status, b.status) and torch.equal(o.steps, b.steps)
        ex, ek, _ = rel_errors(to_np(o.x), to_np(o.k),
                               np.concatenate([to_np(b.x).T, to_np(b.k).T], 1))
        assert max(ex.max(), ek.max()) < 1e-9


@pytest.mark.parametrize("one_lane,two_lane", [(3, 7), (4, 8)])
def test_two_lane_zone_attempts_are_exact(one_lane, two_lane):
    """Zone variants 7 and 8 take the zone phase's tail with two lanes per
    attempt (the full step on a helper lane, the half steps on the owner's)
    and re-pack the warps to at most 16 geodesics: the arithmetic is that of
    variants 3 and 4, so every output is bit-identical.  Nearly edge-on at
    a = 0.99 some geodesics orbit inside 1.5 r_h and come out again (FP32
    steps in the zone phase), so leaving the zone from a two-lane attempt is
    covered too."""
    spec = W.CameraSpec(0.99, np.radians(85.0), 1000.0, 8.0, 160, 160)
    c = K.kerr_init(spec.a)
    res = {}
    for zv in (one_lane, two_lane):
        o = K.alloc_out(spec.n, DEV, cross=True)
        K.kerr_trace_camera(c, cam(spec), K.default_opts(zone_variant=zv), out=o)
        torch.cuda.synchronize()
        res[zv] = (o, K.kerr_get_stats(c))
    c.close()
    (a, sa), (b, sb) = res[one_lane], res[two_lane]
    assert sa.attempts_fp32_zone_phase > 0 and sa.queue_errors == 0 and sb.queue_errors == 0
    assert sa.attempts_fp64 == sb.attempts_fp64
    for name in ("x", "k", "status", "steps"):
        assert torch.equal(getattr(a, name), getattr(b, name)), name
    assert torch.equal(torch.nan_to_num(a.cross, 7.0), torch.nan_to_num(b.cross, 7.0))


def test_zone_phase_counts(ctx):
    spec = W.CameraSpec(0.99, 0.3, 1000.0, 25.0, 128, 128)
    K.kerr_trace_camera(ctx, cam(spec), K.default_opts(), device=DEV)
    s = K.kerr_get_stats(ctx)
    assert s.geodesics == spec.n and sum(s.status_count) == spec.n
    assert s.deferred > 0 and s.attempts_fp64 > 0 and s.rhs_fp64 > 0
    assert all(t >= 0 for t in s.phase_ms) and s.phase_ms[1] > 0 and s.phase_ms[2] > 0
    assert abs(sum(s.phase_ms) - s.kernel_ms) < 0.05 * s.kernel_ms + 0.05
    assert s.queue_errors == 0
    K.kerr_trace_camera(ctx, cam(spec), K.default_opts(fp64_zone=0.0), device=DEV)
    s0 = K.kerr_get_stats(ctx)
    assert s0.deferred == 0 and s0.attempts_fp64 == 0 and s0.requeued == 0


@pytest.mark.parametrize("zone_prec", [K.ZONE_FP64, K.ZONE_F32X2])
def test_zone_requeue_is_exact(ctx, zone_prec):
    """Re-queueing zone geodesics (processor sharing) only moves a geodesic
    between lanes with its whole state, so every output is bit-identical for
    any quantum; a quantum of 1 hands geodesics over after every attempt.
    About half of the 320 x 320 rays enter the zone: more than the zone
    phase has lanes, so geodesics wait and get re-queued."""
    spec = W.CameraSpec(0.99, 0.3, 1000.0, 6.0, 320, 320)
    res = {}
    for q in (0, 1, 16):
        out = K.alloc_out(spec.n, DEV, cross=True)
        K.kerr_trace_camera(ctx, cam(spec), K.default_opts(zone_quantum=q, zone_prec=zone_prec),
                            out=out)
        torch.cuda.synchronize()
        res[q] = (out, K.kerr_get_stats(ctx))
    base, s0 = res[0]
    assert s0.requeued == 0 and s0.deferred > 0
    for q in (1, 16):
        out, s = res[q]
        assert s.queue_errors == 0
        assert s.requeued > 0
        assert s.geodesics == spec.n and sum(s.status_count[1:]) == spec.n
        for name in ("x", "k", "status", "steps", "diag", "cross"):
            a, b = getattr(out, name), getattr(base, name)
            if a.is_floating_point():
                assert torch.equal(a.isnan(), b.isnan()), name
                a, b = torch.nan_to_num(a), torch.nan_to_num(b)
            assert torch.equal(a, b), name
        assert s.attempts_fp64 == s0.attempts_fp64 and s.rhs_fp64 == s0.rhs_fp64


def test_zone_buffer_holds_every_deferred_geodesic(ctx):
    """A 512 x 512 image of the shadow itself: most rays enter the zone.  The
    zone buffer holds one entry per geodesic (each is deferred at most once),
    so every one of them is deferred, none is lost and re-queueing stays on;
    a fresh context and one whose buffers were grown by a larger image give
    the same result bit for bit."""
    spec = W.CameraSpec(0.9, 1.0, 1000.0, 3.0, 512, 512)
    opts = K.default_opts(tol=1e-6)
    fresh = K.kerr_init(spec.a)
    out1 = K.kerr_trace_camera(fresh, cam(spec), opts, device=DEV)
    torch.cuda.synchronize()
    s1 = K.kerr_get_stats(fresh)
    fresh.close()
    assert s1.deferred > spec.n // 2             # most rays enter the zone
    assert s1.queue_errors == 0 and s1.requeued > 0
    assert sum(s1.status_count[1:]) == spec.n
    big = K.kerr_init(spec.a)
    K.kerr_trace_camera(big, cam(W.CameraSpec(0.9, 1.0, 1000.0, 3.0, 1024, 1024)), opts,
                        device=DEV)                # grows the buffers to 2^20 geodesics
    out2 = K.kerr_trace_camera(big, cam(spec), opts, device=DEV)
    torch.cuda.synchronize()
    s2 = K.kerr_get_stats(big)
    big.close()
    assert s2.deferred == s1.deferred and s2.attempts_fp64 == s1.attempts_fp64
    for name in ("x", "k", "status", "steps"):
        assert torch.equal(getattr(out1, name), getattr(out2, name)), name


# ---------------------------------------------------------------------------
# equatorial-crossing labels
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec,tol,gate", [(K.FP64, 1e-10, 2e-7), (K.FP32_KAHAN, 1e-6, 5e-5)])
def test_crossing_labels_match_oracle(ctx, prec, tol, gate):
    """r1, phi1, r2, phi2, g1 against the oracle on every well-conditioned ray
    of a 48 x 48 image seen at 75 deg.  The labels are stored as floats, so
    the FP64 path's gate is set by float rounding (2e-7).  For the FP32 path
    the gate is 5e-5: first crossings at r ~ 2-5 M of rays near the shadow
    edge carry 1-3e-5 of FP32 error (their end points still meet 1e-5)."""
    spec = W.CameraSpec(0.9, np.radians(75.0), 1000.0, 15.0, 48, 48)
    out = K.alloc_out(spec.n, DEV, cross=True)
    K.kerr_trace_camera(ctx, cam(spec), K.default_opts(prec=prec, tol=tol), out=out)
    torch.cuda.synchronize()
    idx = np.arange(spec.n)
    y0 = oracle_camera_ic(spec, idx)
    oo = O.Opts(tol=tol)
    ref = O.trace(spec.a, y0, oo, crossings=True)
    from parity import label_flags, oracle_flags
    good = np.ones(spec.n, dtype=bool)
    # labels must be determined to half the gate by the oracle's own
    # perturbation runs (second crossings far out graze the plane and are
    # truncation-dominated)
    lgood = good[:, None] & ~label_flags(spec.a, y0, oo, ref, 0.5 * gate,
                                         fp32=(prec == K.FP32_KAHAN))
    good = good & ~oracle_flags(spec.a, y0, oo, ref, 1e-5 if prec == K.FP32_KAHAN else gate,
                                fp32=(prec == K.FP32_KAHAN))
    gc = to_np(out.cross).T.astype(np.float64)
    rc = ref.cross
    same_nan = np.isnan(gc) == np.isnan(rc)
    assert np.all(same_nan[lgood]), np.argwhere(~same_nan & lgood)[:5]
    both = lgood & ~np.isnan(gc) & ~np.isnan(rc)
    rel_r = np.abs(gc[:, [0, 2]] - rc[:, [0, 2]]) / rc[:, [0, 2]]
    dphi = np.abs((gc[:, [1, 3]] - rc[:, [1, 3]] + np.pi) % (2 * np.pi) - np.pi)
    rel_g = np.abs(gc[:, 4] - rc[:, 4]) / np.abs(rc[:, 4])
    assert np.all(rel_r[both[:, [0, 2]]] <= gate), np.sort(rel_r[both[:, [0, 2]]])[-5:]
    assert np.all(dphi[both[:, [1, 3]]] <= 2 * gate), np.sort(dphi[both[:, [1, 3]]])[-5:]
    assert np.all(rel_g[both[:, 4]] <= 2 * gate)
    assert both[:, 0].sum() > 1500 and both[:, 2].sum() > 20
    print(dict(labels=int((~np.isnan(rc)).sum()), ill_conditioned=int((~lgood & ~np.isnan(rc)).sum()),
               max_rel_r=float(rel_r[both[:, [0, 2]]].max()), max_dphi=float(dphi[both[:, [1, 3]]].max())))


# ---------------------------------------------------------------------------
# full-size configurations, sampled against the oracle
# ---------------------------------------------------------------------------
def batch64_sample(specs, per_image=16, seed=1708 + 1):
    """Seeded sample of `per_image` rays of every image of the batch: global
    ray indices, oracle start states and each ray's spin."""
    rng = np.random.default_rng(seed)
    off, rows, y0s, spins = 0, [], [], []
    for s in specs:
        loc = np.sort(rng.choice(s.n, size=per_image, replace=False))
        rows.append(off + loc)
        y0s.append(oracle_camera_ic(s, loc))
        spins.append(np.full(per_image, s.a))
        off += s.n
    return np.concatenate(rows), np.concatenate(y0s), np.concatenate(spins)


def test_batch64_full_size_sampled():
    """The 64-image batch (seed 1708, 34.9 M rays) in one launch, FP32+Kahan at
    tol 1e-6: 16 seeded rays per image against the oracle (each with its
    image's spin), the 1e-5 gate on every well-conditioned ray and status
    agreement on all of them."""
    specs = W.camera_batch()
    ctx = K.kerr_init(0.0)
    n = sum(s.n for s in specs)
    out = K.alloc_out(n, DEV, diag=False)
    K.kerr_trace_camera(ctx, [cam(s) for s in specs], K.default_opts(tol=1e-6), out=out)
    torch.cuda.synchronize()
    rows, y0, a = batch64_sample(specs)
    s = compare("batch64/fp32", a, y0, O.Opts(tol=1e-6), out, rows, 1e-5, fp32=True,
                max_ill_frac=0.14)
    print(s)
    ctx.close()


def test_particles_full_size_sampled():
    """2^20 particles for 100 radial periods (seed 1707), FP32+Kahan at tol 1e-6,
    the benchmark's launch: 96 stratified particles against the oracle.  After
    100 periods an end point at a fixed time is not determined to 1e-5 (the
    oracle's own 1e-7 perturbation run shifts the orbital phase by ~1e-4), so
    end points are compared only where the oracle finds them determined, and
    every particle that reaches its end time is judged by the drift of its
    constants of motion E, L_z and Carter's Q against the oracle's own drift
    at the same tolerance."""
    ps = W.particles()
    sub = W.particle_subset(ps, k=96)
    c = K.kerr_init(ps.a)
    opts = K.default_opts(tol=1e-6, r_escape=-1.0, max_steps=10_000_000)
    out = K.kerr_trace_particles(c, torch.tensor(ps.x0, device=DEV),
                                 torch.tensor(ps.v0, device=DEV),
                                 torch.tensor(ps.t_end, device=DEV), opts)
    torch.cuda.synchronize()
    y0, ok = O.particle_ic(ps.a, ps.x0[:, sub].T, ps.v0[:, sub].T)
    keep = np.nonzero(ok)[0]
    oo = O.Opts(tol=1e-6, r_escape=-1.0, max_steps=10_000_000)
    te = ps.t_end[sub][keep]
    ref = O.trace(ps.a, y0[keep], oo, t_end=te)
    s = compare("particles-full/fp32", ps.a, y0[keep], oo, out, sub[keep], 1e-5, fp32=True,
                ref=ref, t_end=te, max_ill_frac=1.0)
    s["determined_frac"] = 1.0 - s["ill_conditioned"] / s["n"]
    print(s)
    st = to_np(out.status)[sub][keep]
    fin = (st == K.ENDTIME) & (ref.status == K.ENDTIME)
    assert fin.sum() > 0.8 * len(keep)
    c0 = np.array([O.constants(ps.a, y) for y in y0[keep]])
    c_ref = np.array([O.constants(ps.a, y) for y in ref.y])
    c_gpu = to_np(out.diag)[:, sub][:, keep].T.astype(np.float64)
    E0, Lz0, Q0 = c0[fin, 0], c0[fin, 1], c0[fin, 2]
    # Carter's K = Q + (L_z - a E)^2 >= 0 scales Q (Q vanishes for equatorial orbits)
    K0 = Q0 + (Lz0 - ps.a * E0) ** 2
    scales = {0: np.abs(E0), 1: np.abs(Lz0) + 1e-3, 2: K0}
    for j, name in ((0, "E"), (1, "Lz"), (2, "Q")):
        d_gpu = np.abs(c_gpu[fin, j] - c0[fin, j]) / scales[j]
        d_ref = np.abs(c_ref[fin, j] - c0[fin, j]) / scales[j]
        print(name, "drift median/p90 gpu", np.median(d_gpu), np.percentile(d_gpu, 90),
              "oracle", np.median(d_ref), np.percentile(d_ref, 90))
        # diagnostics are stored as floats: 1e-7 of rounding on top of the drift
        assert np.median(d_gpu) <= 2 * np.median(d_ref) + 2e-7, name
        assert np.percentile(d_gpu, 90) <= 2 * np.percentile(d_ref, 90) + 2e-7, name
    c.close()
