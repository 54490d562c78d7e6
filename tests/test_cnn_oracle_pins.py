"""Pins of the FP64 oracle of the learned denoiser (oracle/cnn_oracle.py).

Each pin ties the oracle to something other than itself: a library routine
(scipy's 2D correlation), an identity (adjointness of the transposed
convolution), central finite differences of the oracle's own forward pass
for its hand-written gradient and JVP, the exact Jacobian trace for the
Hutchinson estimate, Stein's identity checked by Monte Carlo for SURE, the
published first outputs of SplitMix64, and the bfloat16 rounding rule.
Adam's step is pinned by the closed forms that its bias correction makes
exact (the first step from zero moments and any constant gradient move each
parameter by lr g / (|g| + eps)), by where eps enters, by its invariance to
the scale of the gradients, and by its reduction to sign descent at
beta1 = beta2 = 0.
"""
import numpy as np
import pytest

from oracle import cnn_oracle as C


def test_splitmix64_published_outputs():
    # first outputs of SplitMix64 seeded with 0
    assert C.splitmix64(0, 1) == 0xE220A8397B1DCDAF
    assert C.splitmix64(0, 2) == 0x6E789E6AA1B965F4
    assert C.splitmix64(0, 3) == 0x06C45D188009454F


def test_rademacher_is_balanced_and_keyed():
    keys = np.arange(4000)
    a = C.rademacher(7, keys, 0)
    b = C.rademacher(7, keys, 1)
    assert set(np.unique(a)) == {-1.0, 1.0}
    assert abs(a.mean()) < 0.06 and abs(b.mean()) < 0.06
    assert abs(np.mean(a * b)) < 0.06           # re and im probes are independent
    assert not np.array_equal(a, C.rademacher(8, keys, 0))


def test_bf16_rounding():
    assert C.to_bf16(np.array([1.0]))[0] == 1.0
    assert C.to_bf16(np.array([1.0 + 2 ** -8]))[0] == 1.0                 # tie to even
    assert C.to_bf16(np.array([1.0 + 3 * 2 ** -8]))[0] == 1.0 + 2 ** -6   # tie to even
    assert C.to_bf16(np.array([1.0 + 2 ** -8 + 2 ** -12]))[0] == 1.0 + 2 ** -7
    x = np.random.default_rng(0).standard_normal(1000)
    r = C.to_bf16(x)
    assert np.all(np.abs(r - x) <= np.abs(x) * 2 ** -8 + 1e-300)
    assert np.array_equal(C.to_bf16(r), r)


def test_conv_matches_scipy_correlate():
    from scipy.signal import correlate2d
    rng = np.random.default_rng(1)
    x = rng.standard_normal((7, 5, 3))
    w = rng.standard_normal((4, 9, 3))
    b = rng.standard_normal(4)
    out = C.conv3x3(x, w, b)
    for co in range(4):
        ref = sum(correlate2d(x[:, :, ci], w[co, :, ci].reshape(3, 3), mode="same",
                              boundary="fill") for ci in range(3)) + b[co]
        assert np.allclose(out[:, :, co], ref, atol=1e-12)


def test_transposed_conv_is_the_adjoint():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((6, 8, 3))
    y = rng.standard_normal((6, 8, 5))
    w = rng.standard_normal((5, 9, 3))
    lhs = np.sum(C.conv3x3(x, w) * y)
    rhs = np.sum(x * C.conv3x3(y, C.transpose_weights(w), mirror=True))
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


def _tiny():
    rng = np.random.default_rng(3)
    params = C.init_params(rng, cin=3, hidden=4, cout=2)
    params = [(w, rng.standard_normal(b.shape) * 0.1) for w, b in params]
    r = (rng.standard_normal((6, 5)) + 1j * rng.standard_normal((6, 5))) * 0.3
    w0 = r + 0.1 * (rng.standard_normal((6, 5)) + 1j * rng.standard_normal((6, 5)))
    return params, r, w0, 0.04


def test_backward_matches_finite_differences():
    params, r, w0, tau = _tiny()
    L, dn, acts = C.loss(params, r, w0, tau, 1.0 / r.size)
    grads = C.backward(params, acts, dn)
    rng = np.random.default_rng(4)
    h = 1e-6
    for l in range(5):
        w, b = params[l]
        for _ in range(4):
            idx = tuple(rng.integers(0, s) for s in w.shape)
            wp, wm = w.copy(), w.copy()
            wp[idx] += h
            wm[idx] -= h
            pp = [(wp, b) if i == l else params[i] for i in range(5)]
            pm = [(wm, b) if i == l else params[i] for i in range(5)]
            fd = (C.loss(pp, r, w0, tau, 1.0 / r.size)[0] -
                  C.loss(pm, r, w0, tau, 1.0 / r.size)[0]) / (2 * h)
            assert abs(fd - grads[l][0][idx]) < 1e-6 + 1e-5 * abs(fd), (l, idx)
        j = rng.integers(0, b.shape[0])
        bp, bm = b.copy(), b.copy()
        bp[j] += h
        bm[j] -= h
        fd = (C.loss([(w, bp) if i == l else params[i] for i in range(5)], r, w0, tau,
                     1.0 / r.size)[0] -
              C.loss([(w, bm) if i == l else params[i] for i in range(5)], r, w0, tau,
                     1.0 / r.size)[0]) / (2 * h)
        assert abs(fd - grads[l][1][j]) < 1e-6 + 1e-5 * abs(fd), (l, j)


def test_jvp_matches_finite_differences():
    params, r, _, tau = _tiny()
    x0 = C.input_planes(r, tau)
    _, acts = C.forward(params, x0)
    rng = np.random.default_rng(5)
    t0 = np.zeros_like(x0)
    t0[..., :2] = rng.standard_normal(x0.shape[:2] + (2,))
    h = 1e-6
    fd = (C.forward(params, x0 + h * t0)[0] - C.forward(params, x0 - h * t0)[0]) / (2 * h)
    assert np.allclose(C.jvp(params, acts, t0), fd, atol=1e-7)


def test_hutchinson_estimates_the_jacobian_trace():
    params, r, _, tau = _tiny()
    x0 = C.input_planes(r, tau)
    _, acts = C.forward(params, x0)
    h, w = r.shape
    tr = 0.0   # exact trace of d n / d (first two planes), column by column
    for y in range(h):
        for x in range(w):
            for c in range(2):
                e = np.zeros_like(x0)
                e[y, x, c] = 1.0
                tr += C.jvp(params, acts, e)[y, x, c]
    keys = np.arange(h * w).reshape(h, w)
    est = [C.hutchinson_probe(params, acts, np.stack([C.rademacher(s, keys, 0),
                                                      C.rademacher(s, keys, 1)], -1))
           for s in range(400)]
    assert abs(np.mean(est) - tr) < 4 * np.std(est) / np.sqrt(len(est)) + 1e-9


def test_sure_of_a_linear_denoiser_is_unbiased():
    """f(r) = c r has div = 2 N c; E[SURE] = E |f - w|^2 (Stein) over Gaussian noise."""
    rng = np.random.default_rng(6)
    N, tau, c = 64, 0.3, 0.7
    w = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    s, m = [], []
    for _ in range(20000):
        r = w + np.sqrt(tau / 2) * (rng.standard_normal(N) + 1j * rng.standard_normal(N))
        f = c * r
        s.append(C.sure(f, r, tau, 2 * N * c))
        m.append(np.sum(np.abs(f - w) ** 2))
    d = np.array(s) - np.array(m)
    assert abs(d.mean()) < 4 * d.std() / np.sqrt(len(d))


def test_zero_output_layer_is_the_identity_denoiser():
    params, r, _, tau = _tiny()
    params[-1] = (np.zeros_like(params[-1][0]), np.zeros_like(params[-1][1]))
    f, _, acts = C.denoise(params, r, tau)
    assert np.array_equal(f, r)
    assert C.hutchinson_probe(params, acts, np.ones(r.shape + (2,))) == 0.0


def test_bf16_forward_stays_close_to_fp64():
    rng = np.random.default_rng(7)
    params = C.init_params(rng)
    r = rng.standard_normal((16, 16)) + 1j * rng.standard_normal((16, 16))
    n64, _ = C.forward(params, C.input_planes(r, 0.5))
    n16, _ = C.forward(params, C.input_planes(r, 0.5), bf16=True)
    assert np.linalg.norm(n16 - n64) / np.linalg.norm(n64) < 3e-2


# ---- Adam (Kingma and Ba 2015, Algorithm 1) ----------------------------------------

def test_adam_first_step_is_lr_times_normalised_gradient():
    rng = np.random.default_rng(3)
    p0, g = rng.standard_normal(50), rng.standard_normal(50)
    z = np.zeros(50)
    p1, m1, v1 = C.adam_step(p0, g, z, z, 1e-3, 0.9, 0.999, 1e-8, 1)
    # bias correction makes m_hat = g and v_hat = g^2 exactly at t = 1
    assert np.allclose(p1, p0 - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m1, 0.1 * g, rtol=1e-14) and np.allclose(v1, 0.001 * g * g, rtol=1e-12)


def test_adam_constant_gradient_moves_lr_per_step():
    # m_t = (1 - beta1^t) g and v_t = (1 - beta2^t) g^2: the corrected moments are g and g^2
    rng = np.random.default_rng(4)
    p, g = rng.standard_normal(20), rng.standard_normal(20)
    m = v = np.zeros(20)
    p0 = p.copy()
    for t in range(1, 61):
        p, m, v = C.adam_step(p, g, m, v, 1e-2, 0.9, 0.999, 0.0, t)
    assert np.allclose(p, p0 - 60 * 1e-2 * np.sign(g), rtol=0, atol=1e-12)


def test_adam_eps_is_added_after_the_square_root():
    g = np.array([1e-8, -1e-8])
    z = np.zeros(2)
    p1, _, _ = C.adam_step(np.zeros(2), g, z, z, 1.0, 0.9, 0.999, 1e-8, 1)
    assert np.allclose(p1, [-0.5, 0.5], rtol=1e-12)   # lr g / (|g| + eps) with |g| = eps


def test_adam_is_invariant_to_the_gradient_scale():
    rng = np.random.default_rng(5)
    gs = rng.standard_normal((8, 30))
    runs = []
    for c in (1.0, 1e3):
        p, m, v = np.ones(30), np.zeros(30), np.zeros(30)
        for t, g in enumerate(gs, start=1):
            p, m, v = C.adam_step(p, c * g, m, v, 1e-3, 0.9, 0.999, 0.0, t)
        runs.append(p)
    assert np.allclose(runs[0], runs[1], rtol=1e-13, atol=0)


def test_adam_without_momentum_is_sign_descent():
    rng = np.random.default_rng(6)
    p = rng.standard_normal(25)
    m = v = np.zeros(25)
    for t in range(1, 6):
        g = rng.standard_normal(25)
        q, m, v = C.adam_step(p, g, m, v, 0.1, 0.0, 0.0, 0.0, t)
        assert np.allclose(q, p - 0.1 * np.sign(g), rtol=0, atol=1e-15)
        p = q
