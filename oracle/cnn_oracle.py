"""FP64 oracle of the learned per-subband denoiser (test infrastructure only).

Only tests/, the smoke entry point and the benchmark's CPU baseline may import
this module; the library never does.  It shares no code with the CUDA path.

The paper only anticipates a learned denoiser in place of the soft threshold
(concluding section: VDAMP's state evolution lets any denoiser be tuned or
trained for the known colored noise); the network itself is this project's:
per subband index b, five 3x3 convolutions with 32 channels and ReLU,
  n_b(x): 3 -> 32 -> 32 -> 32 -> 32 -> 2 channels, zero padding,
applied to x = (Re r / sqrt(tau), Im r / sqrt(tau), 0.1 ln tau) and used in
residual form  f(r) = r - sqrt(tau) (n_0 + i n_1).  Tensors are [h][w][c];
weights [cout][9][cin] with tap t = 3 (dy + 1) + (dx + 1) reading the input
at (y + dy, x + dx) (zero outside the image).

The divergence that line 7 of Algorithm 1 needs (alpha = div f / (2 N_b),
the Wirtinger reading of the soft threshold's alpha) is estimated by
Hutchinson's method with Rademacher probes eta: E[eta . J eta] = tr J, with
J_f = I - J_n.  SURE of a denoiser (Stein, complex noise of variance tau,
tau/2 per real component):  sum |f - r|^2 - N tau + tau div_R f.
"""
from __future__ import annotations

import numpy as np

TAPS = [(dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15


def to_bf16(x: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def conv3x3(x: np.ndarray, w: np.ndarray, b=None, mirror: bool = False) -> np.ndarray:
    """out[y, x, co] = sum_t sum_ci in[y + dy_t, x + dx_t, ci] w[co, t, ci] (+ b[co]);
    mirror negates the offsets.  x [h][w][cin], w [cout][9][cin]."""
    h, wd, _ = x.shape
    xp = np.zeros((h + 2, wd + 2, x.shape[2]))
    xp[1:-1, 1:-1] = x
    out = np.zeros((h, wd, w.shape[0]))
    for t, (dy, dx) in enumerate(TAPS):
        if mirror:
            dy, dx = -dy, -dx
        out += xp[1 + dy:1 + dy + h, 1 + dx:1 + dx + wd] @ w[:, t, :].T
    if b is not None:
        out += b
    return out


def transpose_weights(w: np.ndarray) -> np.ndarray:
    """Weights of the adjoint convolution (used with mirror=True): [cin][9][cout]."""
    return np.transpose(w, (2, 1, 0)).copy()


def input_planes(r: np.ndarray, tau: float) -> np.ndarray:
    s = np.sqrt(tau)
    return np.stack([r.real / s, r.imag / s, np.full(r.shape, 0.1 * np.log(tau))], axis=-1)


def forward(params, x0: np.ndarray, bf16: bool = False):
    """n(x0) and the activations [x0, a1, ..., a5]; params = [(w, b)] * 5.  With bf16,
    inputs, weights and hidden activations are rounded to bfloat16 as stored."""
    rd = to_bf16 if bf16 else (lambda v: v)
    a = rd(x0)
    acts = [a]
    for l, (w, b) in enumerate(params):
        z = conv3x3(a, rd(w), b)
        a = rd(np.maximum(z, 0.0)) if l < len(params) - 1 else z
        acts.append(a)
    return a, acts


def denoise(params, r: np.ndarray, tau: float, bf16: bool = False):
    """f(r) = r - sqrt(tau) n(x) for one subband image r [h][w] (complex)."""
    n, acts = forward(params, input_planes(r, tau), bf16)
    return r - np.sqrt(tau) * (n[..., 0] + 1j * n[..., 1]), n, acts


def jvp(params, acts, t0: np.ndarray, bf16: bool = False) -> np.ndarray:
    """J_n t0: the tangent through the convolutions (no bias), gated by the primal ReLUs."""
    rd = to_bf16 if bf16 else (lambda v: v)
    t = rd(t0)
    for l, (w, _) in enumerate(params):
        t = conv3x3(t, rd(w))
        if l < len(params) - 1:
            t = rd(np.where(acts[l + 1] > 0, t, 0.0))
    return t


def backward(params, acts, dn: np.ndarray, bf16: bool = False):
    """Gradients [(dw, db)] of sum(dn * n) with respect to every layer."""
    rd = to_bf16 if bf16 else (lambda v: v)
    d = rd(dn)
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        w, _ = params[l]
        x = acts[l]
        h, wd, _ = x.shape
        xp = np.zeros((h + 2, wd + 2, x.shape[2]))
        xp[1:-1, 1:-1] = x
        dw = np.zeros_like(w)
        for t, (dy, dx) in enumerate(TAPS):
            sh = xp[1 + dy:1 + dy + h, 1 + dx:1 + dx + wd]
            dw[:, t, :] = np.einsum("yxo,yxi->oi", d, sh)
        grads[l] = (dw, d.sum(axis=(0, 1)))
        if l > 0:
            dx_ = conv3x3(d, transpose_weights(rd(w)), mirror=True)
            d = rd(np.where(acts[l] > 0, dx_, 0.0))
    return grads


def loss(params, r: np.ndarray, w0: np.ndarray, tau: float, inv_count: float, bf16=False):
    """inv_count * sum |f(r) - w0|^2 and dL/dn."""
    f, n, acts = denoise(params, r, tau, bf16)
    e = f - w0
    dn = np.stack([-2 * np.sqrt(tau) * e.real, -2 * np.sqrt(tau) * e.imag], -1) * inv_count
    return float(np.sum(np.abs(e) ** 2) * inv_count), dn, acts


def splitmix64(seed: int, n: int) -> int:
    """n-th output (n >= 1) of SplitMix64 seeded with `seed` (Steele, Lea, Flood 2014)."""
    z = (seed + GAMMA * n) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def rademacher(seed: int, keys: np.ndarray, c: int) -> np.ndarray:
    """+1 / -1 from bit 0 of output 2 key + c + 1 (c = 0 re, 1 im)."""
    return np.array([1.0 if splitmix64(seed, 2 * int(k) + c + 1) & 1 else -1.0
                     for k in np.ravel(keys)]).reshape(np.shape(keys))


def hutchinson_probe(params, acts, eta: np.ndarray, bf16: bool = False) -> float:
    """eta . J_n eta for a real probe eta [h][w][2]."""
    t0 = np.concatenate([eta, np.zeros(eta.shape[:2] + (acts[0].shape[2] - 2,))], -1)
    return float(np.sum(eta * jvp(params, acts, t0, bf16)))


def sure(f: np.ndarray, r: np.ndarray, tau: float, div: float) -> float:
    """Stein's unbiased risk estimate of a denoiser's complex output (div over R^2N)."""
    return float(np.sum(np.abs(f - r) ** 2) - r.size * tau + tau * div)


def adam_step(p: np.ndarray, g: np.ndarray, m: np.ndarray, v: np.ndarray, lr: float,
              beta1: float, beta2: float, eps: float, t: int):
    """One step of Adam (Kingma and Ba 2015, Algorithm 1) at step number t >= 1.

    Moment estimates m <- beta1 m + (1 - beta1) g and v <- beta2 v + (1 - beta2) g^2,
    their bias-corrected forms m_hat = m / (1 - beta1^t), v_hat = v / (1 - beta2^t),
    and the update p <- p - lr m_hat / (sqrt(v_hat) + eps) (eps added after the root).
    Returns the new (p, m, v); the inputs are not modified.
    """
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    return p - lr * m_hat / (np.sqrt(v_hat) + eps), m, v


def init_params(rng: np.random.Generator, cin=3, hidden=32, cout=2, layers=5):
    """He-normal weights, zero biases."""
    out = []
    dims = [cin] + [hidden] * (layers - 1) + [cout]
    for l in range(layers):
        fan = 9 * dims[l]
        out.append((rng.standard_normal((dims[l + 1], 9, dims[l])) * np.sqrt(2.0 / fan),
                    np.zeros(dims[l + 1])))
    return out
