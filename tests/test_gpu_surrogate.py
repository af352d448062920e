"""The learned surrogate (rows a11-a13): tensor-core forward and backward
against the FP64 reference network, training, target construction from the
integrator, the critical-curve gate and the integrator fallback."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import closed_forms as C  # noqa: E402
from oracle import mlp as M  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_1706_07062_gb300 import kerr as K  # noqa: E402
from parity import to_np  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def random_batch(n, seed):
    rng = np.random.default_rng(seed)
    x = np.stack([rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), rng.uniform(0, 1, n),
                  rng.uniform(0.1, 1, n)], 1)
    y = np.zeros((n, 8))
    y[:, 0] = rng.integers(0, 2, n)
    y[:, 1:] = rng.normal(size=(n, 7)) * 0.5
    m = (rng.uniform(size=(n, 8)) > 0.2).astype(np.float64)
    m[:, 0] = 1
    return x, y, m


def dev(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float32), device=DEV)


@pytest.mark.parametrize("impl", [K.SURR_FWD_TENSOR_CORE, K.SURR_FWD_GEMM])
@pytest.mark.parametrize("n", [1, 128, 129, 3000])
def test_forward_matches_reference_network(impl, n):
    """Both forward implementations (the fused tcgen05 kernel; the
    layer-by-layer tcgen05 GEMMs of the training path) against the FP64 reference
    network with the same bfloat16 rounding points, on ragged row counts."""
    p = M.init_params(11)
    p[M.B_OFF[1]:M.B_OFF[1] + 256] = np.random.default_rng(2).normal(size=256) * 0.2
    p[M.B_OFF[4]:M.B_OFF[4] + 8] = np.random.default_rng(4).normal(size=8) * 0.3
    s = K.Surrogate(p)
    x, _, _ = random_batch(n, 5)
    got = to_np(K.kerr_surrogate_forward(s, dev(x), impl=impl)).astype(np.float64)
    torch.cuda.synchronize()
    want_q = M.forward(p.astype(np.float64), x, quantize=True)
    want = M.forward(p.astype(np.float64), x, quantize=False)
    scale = 1.0 + np.abs(want_q)
    # same bfloat16 rounding points as the reference: only FP32 accumulation
    # order and rare flips of a bfloat16 rounding differ
    assert np.max(np.abs(got - want_q) / scale) < 2e-2
    assert np.median(np.abs(got - want_q) / scale) < 1e-3
    # against the unquantised FP64 network: the bfloat16 budget
    assert np.median(np.abs(got - want) / scale) < 2e-2
    s.close()


def test_fused_forward_many_tiles_per_cta():
    """300k rows: ~15 tiles per CTA of the persistent fused kernel (weights
    restaged per layer and tile, mbarrier phases over many tiles) agree with
    the GEMM path to accumulation order."""
    p = M.init_params(13)
    s = K.Surrogate(p)
    x, _, _ = random_batch(300_001, 9)
    xd = dev(x)
    a = K.kerr_surrogate_forward(s, xd, impl=K.SURR_FWD_TENSOR_CORE)
    b = K.kerr_surrogate_forward(s, xd, impl=K.SURR_FWD_GEMM)
    torch.cuda.synchronize()
    d = (a - b).abs() / (1 + b.abs())
    assert float(d.max()) < 2e-2 and float(d.median()) < 1e-3
    assert bool(torch.isfinite(a).all())
    s.close()


@pytest.mark.parametrize("impl", [K.SURR_TRAIN_FUSED, K.SURR_TRAIN_GEMM])
@pytest.mark.parametrize("n", [4096, 1000, 129, 37])
def test_gradient_matches_reference_network(impl, n):
    """Weight, bias and loss gradients of both training implementations (the
    fused chain / gradient kernels; the layer-by-layer GEMMs) against the FP64
    reference network, on batches that fill whole tiles and on ragged ones
    (partial row tiles, a partial last 64-row block of the batch-contracted
    weight gradients, split batches)."""
    p = M.init_params(12)
    s = K.Surrogate(p)
    x, y, m = random_batch(n, 6)
    loss = K.kerr_surrogate_grad(s, dev(x), dev(y), dev(m), impl=impl)
    g = s.grad().astype(np.float64)
    Lq, gq = M.grad(p.astype(np.float64), x, y, m, quantize=True)
    L, gref = M.grad(p.astype(np.float64), x, y, m, quantize=False)
    assert abs(loss - Lq) < 1e-3 * (1 + abs(Lq))
    Wg, bg = M.unpack(g)
    Wq, bq = M.unpack(gq)
    Wr, br = M.unpack(gref)
    for l in range(M.LAYERS):
        rel_q = np.linalg.norm(Wg[l] - Wq[l]) / np.linalg.norm(Wq[l])
        rel_r = np.linalg.norm(Wg[l] - Wr[l]) / np.linalg.norm(Wr[l])
        assert rel_q < 1e-2, (l, rel_q)
        assert rel_r < 5e-2, (l, rel_r)
        assert np.linalg.norm(bg[l] - bq[l]) <= 2e-2 * np.linalg.norm(bq[l]) + 1e-7
    # padding stays untouched
    assert np.all(Wg[0][:, 4:] == 0) and np.all(Wg[-1][8:] == 0)
    s.close()


@pytest.mark.parametrize("n", [20000, 8192 + 77])
def test_fused_and_gemm_gradients_agree(n):
    """The two training implementations on batches of more 128-row tiles than
    the GPU has SMs (several tiles per CTA of the chain kernel) and with a
    ragged tail: gradients equal to accumulation order (the GEMM path sums the
    bias gradient in fp32 before rounding, the fused path sums the bf16
    gradient as the reference network does)."""
    p = M.init_params(14)
    s = K.Surrogate(p)
    x, y, m = random_batch(n, 7)
    xd, yd, md = dev(x), dev(y), dev(m)
    lf = K.kerr_surrogate_grad(s, xd, yd, md, impl=K.SURR_TRAIN_FUSED)
    gf = s.grad().astype(np.float64)
    lg = K.kerr_surrogate_grad(s, xd, yd, md, impl=K.SURR_TRAIN_GEMM)
    gg = s.grad().astype(np.float64)
    assert abs(lf - lg) < 1e-5 * (1 + abs(lg))
    Wf, bf = M.unpack(gf)
    Wg, bg = M.unpack(gg)
    for l in range(M.LAYERS):
        assert np.linalg.norm(Wf[l] - Wg[l]) < 5e-3 * np.linalg.norm(Wg[l]), l
        assert np.linalg.norm(bf[l] - bg[l]) < 1e-2 * np.linalg.norm(bg[l]) + 1e-7, l
    s.close()


def test_training_implementations_share_the_weights():
    """After steps on the GEMM path the fused kernels see the updated weights
    (their packed copy is refreshed), and the reverse."""
    x, y, m = random_batch(4096, 8)
    xd, yd, md = dev(x), dev(y), dev(m)
    s = K.Surrogate(M.init_params(15))
    for first, second in ((K.SURR_TRAIN_GEMM, K.SURR_TRAIN_FUSED),
                          (K.SURR_TRAIN_FUSED, K.SURR_TRAIN_GEMM)):
        K.kerr_surrogate_train(s, xd, yd, md, epochs=1, batch=1024, lr=1e-3, impl=first)
        lf = K.kerr_surrogate_grad(s, xd, yd, md, impl=second)
        g2 = s.grad().astype(np.float64)
        lg = K.kerr_surrogate_grad(s, xd, yd, md, impl=first)
        g1 = s.grad().astype(np.float64)
        assert abs(lf - lg) < 1e-5 * (1 + abs(lg))
        assert np.linalg.norm(g2 - g1) < 1e-2 * np.linalg.norm(g1)
    s.close()


@pytest.mark.parametrize("impl", [K.SURR_TRAIN_FUSED, K.SURR_TRAIN_GEMM])
def test_training_fits_a_teacher_network(impl):
    """Adam on the tensor-core gradients fits targets made by another network."""
    teacher = M.init_params(21)
    rng = np.random.default_rng(4)
    n = 1 << 16
    x = np.stack([rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), rng.uniform(0, 1, n),
                  rng.uniform(0.1, 1, n)], 1)
    yt = M.forward(teacher.astype(np.float64), x)
    y = np.zeros((n, 8))
    y[:, 0] = (yt[:, 0] > 0).astype(float)
    y[:, 1:] = yt[:, 1:]
    m = np.ones((n, 8))
    s = K.Surrogate(M.init_params(22))
    losses = K.kerr_surrogate_train(s, dev(x), dev(y), dev(m), epochs=8, batch=4096, lr=2e-3,
                                    impl=impl)
    assert np.all(np.isfinite(losses))
    assert losses[-1] < 0.2 * losses[0], losses
    s.close()


def test_targets_follow_the_integrator():
    ctx = K.kerr_init(0.5)
    rng = np.random.default_rng(8)
    n = 1024
    pts = np.stack([rng.uniform(-25, 25, n), rng.uniform(-25, 25, n), rng.uniform(0, 0.998, n),
                    np.radians(rng.uniform(5, 85, n))], 1)
    inp, tgt, msk = K.kerr_surrogate_targets(ctx, torch.tensor(pts, device=DEV), 1000.0,
                                             K.default_opts(prec=K.FP64, tol=1e-9))
    inp, tgt, msk = to_np(inp), to_np(tgt), to_np(msk)
    np.testing.assert_allclose(inp[:, 0], pts[:, 0] / 25, rtol=1e-6)
    np.testing.assert_allclose(inp[:, 3], np.cos(pts[:, 3]), rtol=1e-6)
    y0 = np.concatenate([O.camera_ic(pts[i, 2], pts[i, 3], 1000.0, 1.0, 1, 1, [0]) for i in range(n)])
    for i in range(n):      # move the one-pixel camera's ray to the point
        si, ci = np.sin(pts[i, 3]), np.cos(pts[i, 3])
        y0[i, 1:4] = 1000.0 * np.array([si, 0, ci]) + pts[i, 0] * np.array([0, 1, 0]) \
            + pts[i, 1] * np.array([-ci, 0, si])
    fixed = []
    for i in range(n):
        g = O.metric(pts[i, 2], y0[i, :4])
        k = y0[i, 5:8]
        A, B, Cc = g[0, 0], 2 * g[0, 1:] @ k, k @ g[1:, 1:] @ k
        fixed.append(min(np.roots([A, B, Cc]).real))
    y0[:, 4] = fixed
    ref = O.trace(pts[:, 2], y0, O.Opts(tol=1e-9), crossings=True)
    assert np.array_equal(tgt[:, 0] == 1, ref.status == O.CAPTURED)
    has1 = ~np.isnan(ref.cross[:, 0])
    assert np.array_equal(msk[:, 1] == 1, has1)
    sel = has1
    np.testing.assert_allclose(tgt[sel, 1], 0.5 * (np.log(ref.cross[sel, 0]) - 2), atol=1e-4)
    np.testing.assert_allclose(tgt[sel, 2], np.cos(ref.cross[sel, 1]), atol=1e-4)
    ctx.close()


def test_render_fallback_everywhere_equals_integrator():
    cam = K.camera(0.9, np.radians(40), 1000.0, 12.0, 48, 40)
    ctx = K.kerr_init(0.9)
    s = K.Surrogate(M.init_params(31))
    opts = K.default_opts()
    out, fb, nfb = K.kerr_surrogate_render(ctx, s, cam, opts, p_lo=-1.0, p_hi=2.0, crit_dist=0.0)
    ref = K.kerr_trace_camera(ctx, cam, opts, out=K.alloc_out(cam.nx * cam.ny, DEV, cross=True))
    torch.cuda.synchronize()
    assert nfb == cam.nx * cam.ny and bool(fb.all())
    st = to_np(ref.status)
    assert np.array_equal(to_np(out[0]), (st == K.CAPTURED).astype(np.float32))
    np.testing.assert_array_equal(to_np(out[1:]), to_np(ref.cross))
    # no fallback at all: decoded network outputs
    out2, fb2, nfb2 = K.kerr_surrogate_render(ctx, s, cam, opts, p_lo=2.0, p_hi=-1.0,
                                              crit_dist=0.0)
    assert nfb2 == 0 and not bool(fb2.any())
    al = -12.0 + (np.arange(48) + 0.5) * 24.0 / 48
    be = -12.0 + (np.arange(40) + 0.5) * 24.0 / 40
    A, Bm = np.meshgrid(al, be)
    x = np.stack([A.ravel() / 25, Bm.ravel() / 25, np.full(A.size, 0.9),
                  np.full(A.size, np.cos(np.radians(40)))], 1)
    o = to_np(K.kerr_surrogate_forward(s, dev(x)))
    np.testing.assert_allclose(to_np(out2[0]), 1 / (1 + np.exp(-o[:, 0])), rtol=1e-5, atol=1e-6)
    ctx.close()
    s.close()


@pytest.mark.parametrize("a,incl", [(0.0, 60.0), (0.9, 60.0), (0.99, 17.0)])
def test_gate_finds_the_critical_curve(a, incl):
    """With the probability band empty, the fallback set is exactly the
    pixels within 0.5 M of Bardeen's critical curve (closed form)."""
    nx = 160
    cam = K.camera(a, np.radians(incl), 1000.0, 10.0, nx, nx)
    ctx = K.kerr_init(a)
    s = K.Surrogate(M.init_params(32))
    _, fb, nfb = K.kerr_surrogate_render(ctx, s, cam, K.default_opts(), p_lo=2.0, p_hi=-1.0,
                                         crit_dist=0.5)
    curve = C.bardeen_curve(a, np.radians(incl))
    al = -10.0 + (np.arange(nx) + 0.5) * 20.0 / nx
    A, B = np.meshgrid(al, al)
    P = np.stack([A.ravel(), B.ravel()], 1)
    d = np.min(np.linalg.norm(P[:, None, :] - curve[None, ::5, :], axis=2), axis=1)
    want = d < 0.5
    got = to_np(fb).astype(bool)
    unsure = np.abs(d - 0.5) < 0.02           # sampling of the curve on both sides
    assert np.array_equal(got[~unsure], want[~unsure])
    assert want.sum() > 500
    ctx.close()
    s.close()


def test_critical_curve_bounds_the_captured_region():
    """Integrator statuses along the alpha axis change within 0.05 M of the
    curve's crossings of beta = 0 (a = 0.9, i = 60 deg)."""
    a, incl = 0.9, np.radians(60.0)
    ctx = K.kerr_init(a)
    n = 1001
    cam = K.camera(a, incl, 1000.0, 8.0, n, 1)
    out = K.kerr_trace_camera(ctx, cam, K.default_opts(prec=K.FP64, tol=1e-10), device=DEV)
    torch.cuda.synchronize()
    st = to_np(out.status)
    al = -8.0 + (np.arange(n) + 0.5) * 16.0 / n
    cap = al[st == K.CAPTURED]
    curve = C.bardeen_curve(a, incl)
    lo, hi = curve[:, 0].min(), curve[:, 0].max()   # the extremes in alpha lie on beta = 0
    assert abs(cap.min() - lo) < 0.1 and abs(cap.max() - hi) < 0.1, (cap.min(), cap.max(), lo, hi)
    ctx.close()


def test_trained_surrogate_gains_over_the_integrator():
    """What the learned part buys: trained on 2M integrator rays (seeded as
    in the evaluation workload), the surrogate with fallback renders a
    2048 x 2048 image faster than the integrator alone, with no capture
    disagreement on the pixels it answers (checked against the FP64
    integrator and, on a sample, the FP64 oracle) and small label errors."""
    from paper_1706_07062_gb300 import workloads as W
    ctx = K.kerr_init(0.5)
    opts = K.default_opts()
    pts = torch.tensor(W.surrogate_points(2_000_000), device=DEV)
    inp, tgt, msk = K.kerr_surrogate_targets(ctx, pts, 1000.0, opts)
    s = K.Surrogate(W.surrogate_init())
    losses = K.kerr_surrogate_train(s, inp, tgt, msk, epochs=6, batch=8192, lr=2e-3)
    assert losses[-1] < 0.5 * losses[0]
    cs = W.CameraSpec(0.7, np.radians(50.0), 1000.0, 25.0, 2048, 2048)
    cam = K.camera(*cs.as_tuple())
    ref = K.alloc_out(cs.n, DEV, diag=False, cross=True)
    K.kerr_surrogate_render(ctx, s, cam, opts)                 # warm-up
    K.kerr_trace_camera(ctx, cam, opts, out=ref)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out, fb, nfb = K.kerr_surrogate_render(ctx, s, cam, opts)
    torch.cuda.synchronize()
    t_sur = time.perf_counter() - t0
    t0 = time.perf_counter()
    K.kerr_trace_camera(ctx, cam, opts, out=ref)
    torch.cuda.synchronize()
    t_int = time.perf_counter() - t0
    assert t_int / t_sur > 1.3, (t_int, t_sur)
    assert 0 < nfb < 0.1 * cs.n
    ref64 = K.alloc_out(cs.n, DEV, diag=False, cross=True)
    K.kerr_trace_camera(ctx, cam, K.default_opts(prec=K.FP64), out=ref64)
    o, f = to_np(out), to_np(fb).astype(bool)
    st = to_np(ref64.status)
    cr = to_np(ref64.cross)
    net = ~f
    assert np.mean((o[0][net] >= 0.5) != (st[net] == 2)) < 1e-4
    ok = net & ~np.isnan(o[1]) & ~np.isnan(cr[0])
    assert ok.sum() > 0.5 * cs.n
    r1 = np.abs(o[1][ok] - cr[0][ok]) / cr[0][ok]
    ph = np.abs(np.remainder(o[2][ok] - cr[1][ok] + np.pi, 2 * np.pi) - np.pi)
    assert np.median(r1) < 0.03 and np.percentile(r1, 99) < 0.2
    assert np.median(ph) < 0.03
    # fallback pixels carry the integrator's answer
    np.testing.assert_array_equal(o[0][f], (to_np(ref.status)[f] == 2).astype(np.float32))
    # a sample of network pixels against the FP64 oracle
    rng = np.random.default_rng(3)
    idx = np.sort(rng.choice(np.nonzero(net)[0], 256, replace=False))
    y0 = O.camera_ic(*cs.as_tuple(), idx)
    res = O.trace(cs.a, y0, O.Opts(tol=1e-8))
    assert np.mean((o[0][idx] >= 0.5) != (res.status == 2)) <= 1 / 256
    s.close()
    ctx.close()
