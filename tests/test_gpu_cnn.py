"""The learned denoiser's CUDA operations against the FP64 CNN oracle.

BF16 storage is reproduced on the oracle side (inputs, weights and hidden
activations rounded to bfloat16 as the kernels store them), so the
remaining differences are FP32 accumulation on the tensor cores and, where
a hidden activation sits next to a bfloat16 rounding boundary, one-ulp
flips (2^-8 relative) that propagate:
* one convolution, FP32 output: within 1e-5 of the largest magnitude;
  BF16 output: within 2^-8 relative per element (plus 1e-6 of the scale);
* the whole network n, its JVP and the gradients: within 2e-2 relative L2;
* weight gradient of one convolution (FP32 atomics): within 1e-5 relative;
* one Adam step (FP32 state, each step fed the kernel's own previous state):
  the moments within 1e-6 of the size of their terms, the parameter step
  within 1e-5 relative plus the FP32 rounding of the parameter.
Images of ragged sizes (partial 128-pixel tiles, borders) are included.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cnn_oracle as C
from paper_1911_01234_gb300 import binding as vb
from paper_1911_01234_gb300 import build, learned

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    vb.load()


# small and ragged images, and two large ones so that every CTA of a launch
# (at most 2 per SM) runs several tiles through the load pipeline
SIZES = [(13, 9), (16, 16), (5, 40), (1, 1), (32, 24), (3, 200), (40, 3), (256, 240),
         (200, 200)]


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _images(bands=2):
    ents = [(h, w, 0, w, i % bands, 0) for i, (h, w) in enumerate(SIZES)]
    return learned.Images(ents)


def _bf(x):
    return torch.from_numpy(np.ascontiguousarray(C.to_bf16(x).astype(np.float32))).cuda().to(
        torch.bfloat16)


def _split(im, arr):
    out, o = [], 0
    for (h, w) in SIZES:
        out.append(arr[o:o + h * w].reshape(h, w, -1))
        o += h * w
    return out


@pytest.mark.parametrize("cin,cout", [(16, 32), (32, 32), (32, 16), (16, 16)])
@pytest.mark.parametrize("mode", [0, 1, 2, 3])
@pytest.mark.parametrize("mirror", [0, 1])
def test_conv_matches_oracle(cin, cout, mode, mirror):
    rng = np.random.default_rng(cin * 100 + cout + 7 * mode + mirror)
    im = _images()
    P = im.pixels
    x = C.to_bf16(rng.standard_normal((P, cin)))
    w = rng.standard_normal((2, cout, 9, cin)).astype(np.float32) * 0.2
    bias = rng.standard_normal((2, cout)).astype(np.float32)
    mask = C.to_bf16(rng.standard_normal((P, cout)))
    wt = torch.from_numpy(w).cuda()
    img = torch.empty(2 * cout * 9 * cin, dtype=torch.bfloat16, device="cuda")
    L = learned.lib()
    vb.check(L.vdamp_cnn_pack_weights(wt.data_ptr(), 2, cin, cout, cin, cout, 0, img.data_ptr(),
                                      None), "pack")
    store = 3 if mode >= 2 else cout
    out = torch.zeros((P, store), dtype=torch.float32 if mode >= 2 else torch.bfloat16,
                      device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    bt = torch.from_numpy(bias).cuda()
    mt = _bf(mask)
    xt = _bf(x)   # kept alive until the kernel has run
    vb.check(L.vdamp_cnn_conv3x3(xt.data_ptr(), cin, img.data_ptr(), cout, bt.data_ptr(),
                                 mt.data_ptr(), out.data_ptr(), mode, mirror, store,
                                 im.dev.data_ptr(), im.n, im.ctiles, im.max_w, st.data_ptr(),
                                 None), "conv")
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    got = out.float().cpu().numpy()
    wr = C.to_bf16(w)
    for i, (xi, gi, mi) in enumerate(zip(_split(im, x), _split(im, got), _split(im, mask))):
        band = i % 2
        ref = C.conv3x3(xi, wr[band], None, mirror=bool(mirror))
        if mode in (0, 2):
            ref = ref + bias[band]
        if mode == 0:
            ref = np.maximum(ref, 0)
        if mode == 1:
            ref = np.where(mi > 0, ref, 0.0)
        ref = ref[..., :store]
        scale = max(np.abs(ref).max(), 1e-3)
        if mode >= 2:
            assert np.max(np.abs(gi - ref)) <= 1e-5 * scale, (i, np.max(np.abs(gi - ref)))
        else:
            assert np.all(np.abs(gi - ref) <= 2 ** -8 * np.abs(ref) + 1e-6 * scale), i


@pytest.mark.parametrize("cin,cout", [(16, 32), (32, 32), (32, 16)])
def test_weight_gradient_matches_oracle(cin, cout):
    rng = np.random.default_rng(cin + cout)
    im = _images()
    P = im.pixels
    x = C.to_bf16(rng.standard_normal((P, cin)))
    dy = C.to_bf16(rng.standard_normal((P, cout)))
    dw = torch.zeros((2, cout, 9, cin), dtype=torch.float32, device="cuda")
    db = torch.zeros((2, cout), dtype=torch.float32, device="cuda")
    xt, dyt = _bf(x), _bf(dy)   # kept alive until the kernel has run
    vb.check(learned.lib().vdamp_cnn_wgrad(xt.data_ptr(), cin, cin, dyt.data_ptr(), cout,
                                           cout, im.dev.data_ptr(), im.n, im.tiles,
                                           dw.data_ptr(), db.data_ptr(), None), "wgrad")
    torch.cuda.synchronize()
    ref_w = np.zeros((2, cout, 9, cin))
    ref_b = np.zeros((2, cout))
    for i, (xi, di) in enumerate(zip(_split(im, x), _split(im, dy))):
        w0 = np.zeros((cout, 9, cin))
        params = [(w0, np.zeros(cout))]
        g = C.backward(params, [xi, None], di)   # one layer: grads of sum(dy * conv(x))
        ref_w[i % 2] += g[0][0]
        ref_b[i % 2] += g[0][1]
    assert rel(dw.cpu().numpy(), ref_w) < 1e-5
    assert rel(db.cpu().numpy(), ref_b) < 1e-5


def _net_setup(seed=3):
    net = learned.SubbandCNN(bands=2, seed=seed)
    rng = np.random.default_rng(seed)
    for l in range(5):   # make every layer matter (the default last layer starts small)
        net.b[l].copy_(torch.from_numpy(
            (rng.standard_normal(net.b[l].shape) * 0.05).astype(np.float32)))
    with torch.no_grad():
        net.w[4].mul_(10.0)
        net.w[4][:, 2:] = 0
        net.b[4][:, 2:] = 0
        net.w[0][..., 3:] = 0
    net.pack()
    im = _images()
    N = im.pixels
    r = (rng.standard_normal(N) + 1j * rng.standard_normal(N)).astype(np.complex64)
    w0 = (r + 0.2 * (rng.standard_normal(N) + 1j * rng.standard_normal(N))).astype(np.complex64)
    # images read r at src_off = dense offset (pitch = width)
    ents = []
    o = 0
    for i, (h, w) in enumerate(SIZES):
        ents.append((h, w, o, w, i % 2, i % 2))
        o += h * w
    im = learned.Images(ents)
    tau = np.array([[0.3, 0.05], [0.3, 0.05]])
    return net, im, r, w0, tau


def test_network_forward_jvp_and_gradients_match_oracle():
    net, im, r, w0, tau = _net_setup()
    B = 2
    rd, w0d = torch.from_numpy(r).cuda(), torch.from_numpy(w0).cuda()
    td = torch.from_numpy(tau).cuda()
    x0 = net.input(im, rd, td, B)
    n, acts = net.forward(im, x0)
    seed = 11
    t0 = torch.empty((im.pixels, 16), dtype=torch.bfloat16, device="cuda")
    vb.check(learned.lib().vdamp_cnn_probe(seed, im.dev.data_ptr(), im.n, im.tiles,
                                           t0.data_ptr(), None), "probe")
    jn = net.jvp(im, acts, t0)
    f = torch.zeros_like(rd)
    sums = torch.zeros(2 * im.n, dtype=torch.float64, device="cuda")
    vb.check(learned.lib().vdamp_cnn_output(rd.data_ptr(), td.data_ptr(), B, im.dev.data_ptr(),
                                            im.n, im.tiles, n.data_ptr(), jn.data_ptr(), seed,
                                            f.data_ptr(), sums.data_ptr(), None), "output")
    grads = [torch.zeros_like(p) for p in net.params]
    dn = torch.empty((im.pixels, 16), dtype=torch.bfloat16, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    inv = 1.0 / im.pixels
    vb.check(learned.lib().vdamp_cnn_loss(rd.data_ptr(), w0d.data_ptr(), td.data_ptr(), B,
                                          im.dev.data_ptr(), im.n, im.tiles, n.data_ptr(), inv,
                                          dn.data_ptr(), loss.data_ptr(), None), "loss")
    net.backward(im, acts, dn, grads)
    torch.cuda.synchronize()
    assert int(net.status.item()) == 0
    n_g, jn_g, f_g, s_g = (n.cpu().numpy(), jn.cpu().numpy(), f.cpu().numpy(), sums.cpu().numpy())
    L_ref = 0.0
    gw = [np.zeros_like(g.cpu().numpy(), dtype=np.float64) for g in grads]
    o = 0
    for i, (h, w) in enumerate(SIZES):
        band = i % 2
        sl = slice(o, o + h * w)
        t = tau[band, band]
        params = net.oracle_params(band)
        ri = r[sl].astype(np.complex128).reshape(h, w)
        fi, ni, ai = C.denoise(params, ri, t, bf16=True)
        assert rel(n_g[sl].reshape(h, w, 2), ni) < 2e-2, i
        assert rel(f_g[sl].reshape(h, w), fi) < 2e-2, i
        keys = np.arange(o, o + h * w).reshape(h, w)
        eta = np.stack([C.rademacher(seed, keys, 0), C.rademacher(seed, keys, 1)], -1)
        t0o = np.concatenate([eta, np.zeros((h, w, 1))], -1)
        assert rel(jn_g[sl].reshape(h, w, 2), C.jvp(params, ai, t0o, bf16=True)) < 2e-2, i
        pr = float(np.sum(eta * C.jvp(params, ai, t0o, bf16=True)))
        assert abs(s_g[2 * i + 1] - pr) <= 2e-2 * max(np.sum(np.abs(eta)), 1.0), i
        assert abs(s_g[2 * i] - np.sum(np.abs(fi - ri) ** 2)) <= 2e-2 * np.sum(np.abs(fi - ri) ** 2) + 1e-9
        Li, dni, ai2 = C.loss(params, ri, w0[sl].astype(np.complex128).reshape(h, w), t, inv,
                              bf16=True)
        L_ref += Li
        g = C.backward(params, ai2, dni, bf16=True)
        for l, (rin, rout) in enumerate(learned.REAL):
            gw[l][band, :rout, :, :rin] += g[l][0]
            gw[5 + l][band, :rout] += g[l][1]
        o += h * w
    assert abs(float(loss.item()) - L_ref) < 2e-2 * L_ref
    for l in range(10):
        assert rel(grads[l].cpu().numpy(), gw[l]) < 3e-2, l


def test_training_reduces_the_loss():
    net, im, r, w0, tau = _net_setup(seed=5)
    B = 2
    rd, w0d = torch.from_numpy(r).cuda(), torch.from_numpy(w0).cuda()
    td = torch.from_numpy(tau).cuda()
    first = float(net.train_step(im, rd, w0d, td, B, 1e-3).item())
    for _ in range(60):
        last = net.train_step(im, rd, w0d, td, B, 1e-3)
    torch.cuda.synchronize()
    assert float(last.item()) < 0.8 * first
    assert int(net.status.item()) == 0
    # padded weights stay zero
    assert float(net.w[0][..., 3:].abs().max()) == 0.0
    assert float(net.w[4][:, 2:].abs().max()) == 0.0


def test_training_is_reproducible():
    """Two trainings from the same start on the same data give the same weights bit for bit:
    the weight gradients are reduced in a fixed order (per-CTA records added by band in
    record order), not by atomics whose order depends on scheduling."""
    states = []
    for _ in range(2):
        net, im, r, w0, tau = _net_setup(seed=5)
        B = 2
        rd, w0d = torch.from_numpy(r).cuda(), torch.from_numpy(w0).cuda()
        td = torch.from_numpy(tau).cuda()
        for _ in range(20):
            net.train_step(im, rd, w0d, td, B, 1e-3)
        torch.cuda.synchronize()
        states.append(net.state())
    for k in states[0]:
        assert np.array_equal(states[0][k], states[1][k]), k


def test_adam_matches_oracle():
    """vdamp_cnn_adam against the oracle's Adam step (Kingma and Ba, bias-corrected), six
    steps with fresh gradients; each step of the oracle starts from the kernel's FP32
    state, and the hyper-parameters are the FP32 values the kernel receives."""
    rng = np.random.default_rng(11)
    n = 10007
    f32 = lambda x: float(np.float32(x))
    lr, b1, b2, eps = f32(1e-3), f32(0.9), f32(0.999), f32(1e-8)
    p = torch.from_numpy(rng.standard_normal(n).astype(np.float32)).cuda()
    m = torch.zeros(n, dtype=torch.float32, device="cuda")
    v = torch.zeros_like(m)
    L = vb.load()
    for t in range(1, 7):
        g = torch.from_numpy((rng.standard_normal(n) * 10.0 ** rng.uniform(-3, 1, n))
                             .astype(np.float32)).cuda()
        p0, m0, v0 = (x.double().cpu().numpy() for x in (p, m, v))
        vb.check(L.vdamp_cnn_adam(p.data_ptr(), g.data_ptr(), m.data_ptr(), v.data_ptr(), n,
                                  lr, b1, b2, eps, t, None), "vdamp_cnn_adam")
        torch.cuda.synchronize()
        pw, mw, vw = C.adam_step(p0, g.double().cpu().numpy(), m0, v0, lr, b1, b2, eps, t)
        pg, mg, vg = (x.double().cpu().numpy() for x in (p, m, v))
        gd = g.double().cpu().numpy()
        # moments: within 1e-6 of the size of their two terms (m may cancel to ~0)
        m_scale = np.abs(b1 * m0) + np.abs((1 - b1) * gd)
        v_scale = np.abs(b2 * v0) + np.abs((1 - b2) * gd * gd)
        assert float(np.max(np.abs(mg - mw) / m_scale)) < 1e-6, t
        assert float(np.max(np.abs(vg - vw) / v_scale)) < 1e-6, t
        # parameters: the step within 1e-5 relative, plus the FP32 rounding of p itself
        bound = 1e-5 * np.abs(pw - p0) + 2.0 ** -24 * np.abs(pw)
        assert bool(np.all(np.abs(pg - pw) <= bound)), (t, float(np.max(np.abs(pg - pw) - bound)))


def test_conv_wait_that_runs_out_reports_a_timeout():
    """Failure detection of the bounded tensor-core waits, with no fault: with a first-wait
    limit of 0 polls every wait gives up at once, the kernel records the timeout, still waits
    (with the default limit) for the operations in flight, frees its tensor memory and
    returns; vdamp_cnn_status reports VDAMP_ETIMEOUT and the context stays usable: with the
    default limit back, the same convolution is complete and matches the oracle."""
    rng = np.random.default_rng(5)
    h, w = 24, 20
    x = C.to_bf16(rng.standard_normal((h * w, 32)))
    wt = (rng.standard_normal((1, 32, 9, 32)) * 0.2).astype(np.float32)
    bt = rng.standard_normal((1, 32)).astype(np.float32)
    im = learned.Images([(h, w, 0, w, 0, 0)])
    L = vb.load()
    wdev, bdev = torch.from_numpy(wt).cuda(), torch.from_numpy(bt).cuda()
    img = torch.empty(32 * 9 * 32, dtype=torch.bfloat16, device="cuda")
    xt = torch.from_numpy(x.astype(np.float32)).cuda().to(torch.bfloat16)
    out = torch.zeros((h * w, 32), dtype=torch.bfloat16, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    vb.check(L.vdamp_cnn_pack_weights(wdev.data_ptr(), 1, 32, 32, 32, 32, 0, img.data_ptr(),
                                      None), "vdamp_cnn_pack_weights")

    def conv():
        vb.check(L.vdamp_cnn_conv3x3(xt.data_ptr(), 32, img.data_ptr(), 32, bdev.data_ptr(),
                                     None, out.data_ptr(), 0, 0, 32, im.dev.data_ptr(), im.n,
                                     im.ctiles, im.max_w, status.data_ptr(), None),
                 "vdamp_cnn_conv3x3")

    default = vb.vdamp_cnn_default_wait_limit()
    assert default > 0
    prev = vb.vdamp_cnn_set_wait_limit(0)
    try:
        assert prev == default
        conv()
        assert vb.vdamp_cnn_status(status) == vb.VDAMP_ETIMEOUT
        assert "ran out" in vb.last_error()
        assert int(status.item()) == 0          # read and cleared
    finally:
        vb.vdamp_cnn_set_wait_limit(default)
    conv()
    assert vb.vdamp_cnn_status(status) == vb.VDAMP_OK
    ref = np.maximum(C.conv3x3(x.reshape(h, w, 32), C.to_bf16(wt[0]), bt[0]), 0).reshape(-1, 32)
    got = out.float().cpu().numpy()
    assert float(np.max(np.abs(got - ref) - 2 ** -8 * np.abs(ref))) <= 1e-5 * float(np.abs(ref).max())
