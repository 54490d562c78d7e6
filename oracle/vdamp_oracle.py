"""FP64 CPU oracle for the VDAMP iteration (Algorithm 1) -- TEST INFRASTRUCTURE ONLY.

This module exists to check the CUDA path.  Only the test suite, the smoke
check and the benchmark's CPU-baseline leg may import it; the library never
does, and it imports nothing from the library (it shares no code, tables or
constants with the CUDA kernels).  It is deliberately plain and slow: every
step is a whole-array numpy pass in float64 / complex128, in the order of
Algorithm 1, with numpy's FFT and sort as the only library primitives.

Conventions fixed here (readings of passages the paper leaves open):

* F is the unitary 2D DFT on unshifted storage (DC at index 0); the SNR
  definition of Sec. 3 and S = |Phi Psi^H|^2 of Algorithm 1 (line 1) used as a
  variance map only agree with an orthonormal F and Psi.
* Psi is an orthonormal periodic 2D wavelet transform with s scales:
  a[n] = sum_k h[k] x[(2n+k) mod L], d[n] = sum_k g[k] x[(2n+k) mod L],
  g[k] = (-1)^k h[len-1-k]; rows (x) are filtered first, then columns (y).
* Coefficients are stored "packed": subbands in the order
  [A_s, H_s, V_s, D_s, H_{s-1}, V_{s-1}, D_{s-1}, ..., H_1, V_1, D_1] (coarse to
  fine), each row-major.  H is high-pass along x, V high-pass along y,
  D high-pass along both; the 1 + 3s subbands are the blocks of Eq. 6.
* The denoiser is complex soft thresholding with one threshold per subband
  (Eq. 7), chosen by the exact global minimiser of the complex colored SURE
  (Sec. 3, the unnumbered equation after Algorithm 1); alpha is the subband
  mean of the Wirtinger derivative, 1 - theta / (2|r|) above threshold.
* "w_k" in the return line of Algorithm 1 is the last denoiser output.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np

# ---------------------------------------------------------------------------
# Fourier operator (Sec. 1: Phi = M_Omega F)
# ---------------------------------------------------------------------------


def fft2u(x: np.ndarray) -> np.ndarray:
    """Unitary forward 2D DFT F (Sec. 1, Phi = M_Omega F)."""
    return np.fft.fft2(x, norm="ortho")


def ifft2u(k: np.ndarray) -> np.ndarray:
    """Unitary inverse 2D DFT F^H."""
    return np.fft.ifft2(k, norm="ortho")


# ---------------------------------------------------------------------------
# Orthogonal wavelet Psi (Sec. 1, Eq. 5-6; Sec. 3 uses Haar at s = 4)
# ---------------------------------------------------------------------------


def daubechies_lowpass(p: int) -> np.ndarray:
    """Orthonormal Daubechies low-pass filter with p vanishing moments (2p taps).

    Daubechies' spectral factorisation: |H(w)|^2 = 2 cos^{2p}(w/2) P(sin^2(w/2))
    with P(y) = sum_{k<p} C(p-1+k, k) y^k; each root y_r of P gives the pair
    z, 1/z of z^2 - (2 - 4 y_r) z + 1 and the factor with |z| < 1 is kept
    (minimum phase).  h[k] is the coefficient of z^{-k}; sum(h) = sqrt(2).
    p = 1 is Haar, p = 4 is the 8-tap "db4" filter.
    """
    coef = [math.comb(p - 1 + k, k) for k in range(p)]  # ascending powers of y
    poly = np.array([1.0 + 0.0j])
    for _ in range(p):
        poly = np.convolve(poly, [0.5, 0.5])
    if p > 1:
        for yr in np.roots(coef[::-1]):
            b = 2.0 - 4.0 * yr
            disc = np.sqrt(b * b - 4.0 + 0.0j)
            z1, z2 = (b + disc) / 2.0, (b - disc) / 2.0
            zr = z1 if abs(z1) < 1.0 else z2
            poly = np.convolve(poly, [1.0, -zr]) / (1.0 - zr)
    return math.sqrt(2.0) * poly.real


def wavelet_filters(name: str):
    """(h, g) for 'haar' or 'db4'; g[k] = (-1)^k h[len-1-k]."""
    p = {"haar": 1, "db4": 4}[name]
    h = daubechies_lowpass(p)
    n = len(h)
    g = np.array([(-1.0) ** k * h[n - 1 - k] for k in range(n)])
    return h, g


def _analysis_axis(x: np.ndarray, f: np.ndarray, axis: int) -> np.ndarray:
    """Periodic filter-and-decimate: out[n] = sum_k f[k] x[(2n+k) mod L] along axis."""
    n = x.shape[axis]
    out = 0.0
    for k, fk in enumerate(f):
        idx = (2 * np.arange(n // 2) + k) % n
        out = out + fk * np.take(x, idx, axis=axis)
    return out


def _synthesis_axis(c: np.ndarray, f: np.ndarray, axis: int) -> np.ndarray:
    """Adjoint of _analysis_axis: x[(2n+k) mod L] += f[k] c[n] along axis."""
    half = c.shape[axis]
    n = 2 * half
    cm = np.moveaxis(c, axis, 0)
    out = np.zeros((n,) + cm.shape[1:], dtype=np.result_type(c, np.float64))
    for k, fk in enumerate(f):
        idx = (2 * np.arange(half) + k) % n  # distinct for fixed k
        out[idx] += fk * cm
    return np.moveaxis(out, 0, axis)


@dataclass(frozen=True)
class Subband:
    index: int       # b in the packed order
    name: str        # "A4", "H2", ...
    level: int       # j (1 finest .. s coarsest)
    kind: str        # "A", "H", "V", "D"
    offset: int      # start in the packed vector
    shape: tuple     # (rows, cols)

    @property
    def size(self) -> int:
        return self.shape[0] * self.shape[1]


def subbands(ny: int, nx: int, s: int) -> List[Subband]:
    """The 1 + 3s subbands of Eq. 6 in packed order (coarse to fine)."""
    out = []
    hy, hx = ny >> s, nx >> s
    out.append(Subband(0, f"A{s}", s, "A", 0, (hy, hx)))
    off = hy * hx
    b = 1
    for j in range(s, 0, -1):
        hy, hx = ny >> j, nx >> j
        for kind in "HVD":
            out.append(Subband(b, f"{kind}{j}", j, kind, off, (hy, hx)))
            off += hy * hx
            b += 1
    assert off == ny * nx
    return out


def dwt2(x: np.ndarray, h: np.ndarray, g: np.ndarray, s: int) -> np.ndarray:
    """w = Psi x: s-scale periodic 2D analysis, returned packed (Eq. 5-6)."""
    ny, nx = x.shape
    details: Dict[int, tuple] = {}
    cur = x.astype(np.complex128)
    for j in range(1, s + 1):
        lx = _analysis_axis(cur, h, 1)
        hx = _analysis_axis(cur, g, 1)
        ll = _analysis_axis(lx, h, 0)
        v = _analysis_axis(lx, g, 0)
        hh = _analysis_axis(hx, h, 0)
        d = _analysis_axis(hx, g, 0)
        details[j] = (hh, v, d)
        cur = ll
    parts = [cur.ravel()]
    for j in range(s, 0, -1):
        parts.extend(p.ravel() for p in details[j])
    return np.concatenate(parts)


def idwt2(w: np.ndarray, h: np.ndarray, g: np.ndarray, s: int, ny: int, nx: int) -> np.ndarray:
    """x = Psi^H w: adjoint (= inverse) of dwt2 for packed coefficients."""
    bands = {sb.name: w[sb.offset:sb.offset + sb.size].reshape(sb.shape)
             for sb in subbands(ny, nx, s)}
    cur = bands[f"A{s}"].astype(np.complex128)
    for j in range(s, 0, -1):
        hh, v, d = bands[f"H{j}"], bands[f"V{j}"], bands[f"D{j}"]
        lx = _synthesis_axis(cur, h, 0) + _synthesis_axis(v, g, 0)
        hx = _synthesis_axis(hh, h, 0) + _synthesis_axis(d, g, 0)
        cur = _synthesis_axis(lx, h, 1) + _synthesis_axis(hx, g, 1)
    return cur


# ---------------------------------------------------------------------------
# S = |Phi Psi^H|^2 (Algorithm 1, line 1; 1 + 3s unique columns, Sec. 2)
# ---------------------------------------------------------------------------


def s_columns(ny: int, nx: int, h: np.ndarray, g: np.ndarray, s: int,
              position: Optional[List[int]] = None) -> np.ndarray:
    """One column of |F Psi^H|^2 per subband, by brute force: (1+3s, ny, nx).

    Column b is |F Psi^H e|^2 for a unit impulse e at coefficient `position[b]`
    of subband b (default: its first coefficient).  Rows of Phi are the rows of
    F on Omega, so S restricted to the sampled frequencies is S[:, mask].
    """
    out = []
    for sb in subbands(ny, nx, s):
        e = np.zeros(ny * nx, dtype=np.complex128)
        e[sb.offset + (0 if position is None else position[sb.index])] = 1.0
        out.append(np.abs(fft2u(idwt2(e, h, g, s, ny, nx))) ** 2)
    return np.stack(out)


# ---------------------------------------------------------------------------
# Denoiser: complex soft threshold tuned by colored SURE (Eq. 3, Eq. 7, Sec. 3)
# ---------------------------------------------------------------------------


def soft(r: np.ndarray, theta: float) -> np.ndarray:
    """Complex soft threshold: max(|r| - theta, 0) r / |r| (prox of theta |.|, Eq. 3)."""
    a = np.abs(r)
    scale = np.where(a > theta, 1.0 - theta / np.where(a > 0, a, 1.0), 0.0)
    return scale * r


def sure_value(a: np.ndarray, theta: float, tau: float) -> float:
    """Complex SURE of soft(., theta) for coefficients of magnitude a, variance tau.

    Per coefficient (Stein's lemma in R^2, each real part of variance tau/2):
    |r| <= theta: |r|^2 - tau;  |r| > theta: theta^2 + tau (1 - theta / |r|).
    """
    below = a <= theta
    above_val = theta * theta + tau * (1.0 - theta / np.where(below, 1.0, a))
    return float(np.sum(np.where(below, a * a - tau, above_val)))


def sure_threshold(a: np.ndarray, tau: float):
    """Exact global minimiser of SURE(theta) over theta in [0, max a].

    On [a_(m), a_(m+1)) SURE = C_m - m tau + K theta^2 + K tau - tau theta H_m with
    K = N - m, C_m the sum of the m smallest a^2 and H_m the sum of 1/a over the
    rest: a convex quadratic whose minimiser tau H_m / (2K) is clamped to the
    interval.  SURE drops by tau at each breakpoint, so a minimiser clamped to
    the right end is never the global one.  For theta >= max a SURE is constant
    and theta = max a is taken.  Ties within 1e-12 |SURE| go to the smallest theta.
    Returns (theta, sure_at_theta).
    """
    a = np.sort(np.asarray(a, dtype=np.float64))
    n = a.size
    c = np.concatenate([[0.0], np.cumsum(a * a)])                 # C_m, m = 0..n
    inv = np.where(a > 0, 1.0 / np.where(a > 0, a, 1.0), 0.0)
    hsum = np.concatenate([np.cumsum(inv[::-1])[::-1], [0.0]])    # H_m = sum_{i>=m} 1/a_(i)
    m = np.arange(n + 1)
    k = n - m
    lo = np.concatenate([[0.0], a])                               # a_(m), a_(0) = 0
    hi = np.concatenate([a, [np.inf]])                            # a_(m+1)
    kk = np.maximum(k, 1)
    th = np.maximum(tau * hsum / (2.0 * kk), lo)
    val = c - m * tau + k * th * th + k * tau - tau * th * hsum
    ok = th < hi
    ok[n] = True
    th[n] = a[-1]
    val[n] = c[n] - n * tau
    vals = np.where(ok, val, np.inf)
    vmin = vals.min()
    tol = 1e-12 * abs(vmin)
    cand = np.nonzero(vals <= vmin + tol)[0]
    best = cand[np.argmin(th[cand])]
    return float(th[best]), float(vals[best])


def sure_threshold_bruteforce(a: np.ndarray, tau: float, grid: int = 1_000_000):
    """Reference for tiny subbands: SURE on a dense theta grid plus all breakpoints."""
    a = np.asarray(a, dtype=np.float64)
    thetas = np.concatenate([np.linspace(0.0, a.max(), grid), a])
    a_safe = np.where(a > 0, a, 1.0)
    best_t, best_v = None, np.inf
    for chunk in np.array_split(thetas, max(1, thetas.size // 20000)):
        below = a[None, :] <= chunk[:, None]
        above_val = chunk[:, None] ** 2 + tau * (1.0 - chunk[:, None] / a_safe[None, :])
        v = np.where(below, a[None, :] ** 2 - tau, above_val).sum(axis=1)
        i = int(np.argmin(v))
        if v[i] < best_v:
            best_v, best_t = float(v[i]), float(chunk[i])
    return best_t, best_v


def soft_divergence_mean(a: np.ndarray, theta: float) -> float:
    """alpha = <g'(r)>: mean Wirtinger derivative of soft(., theta) (Algorithm 1, line 7).

    g' = 1 - theta / (2|r|) for |r| > theta and 0 otherwise (half the R^2 divergence).
    """
    above = a > theta
    return float(np.sum(np.where(above, 1.0 - theta / (2.0 * np.where(above, a, 1.0)), 0.0))
                 / a.size)


def denoise(r: np.ndarray, tau: np.ndarray, sbs: List[Subband]):
    """Algorithm 1, lines 6-7 with the SURE soft threshold: (w_hat, theta, alpha)."""
    w_hat = np.empty_like(r)
    theta = np.zeros(len(sbs))
    alpha = np.zeros(len(sbs))
    for sb in sbs:
        rb = r[sb.offset:sb.offset + sb.size]
        if tau[sb.index] <= 0.0:
            # No effective noise: keep r untouched and drop the Onsager term.
            w_hat[sb.offset:sb.offset + sb.size] = rb
            continue
        a = np.abs(rb)
        th, _ = sure_threshold(a, float(tau[sb.index]))
        theta[sb.index] = th
        alpha[sb.index] = soft_divergence_mean(a, th)
        w_hat[sb.offset:sb.offset + sb.size] = soft(rb, th)
    return w_hat, theta, alpha


def expand(per_band: np.ndarray, sbs: List[Subband]) -> np.ndarray:
    """Broadcast one value per subband to every coefficient (the form of Eq. 7)."""
    out = np.empty(sum(sb.size for sb in sbs), dtype=np.asarray(per_band).dtype)
    for sb in sbs:
        out[sb.offset:sb.offset + sb.size] = per_band[sb.index]
    return out


def onsager(w_hat: np.ndarray, r: np.ndarray, alpha: np.ndarray, sbs: List[Subband]):
    """Algorithm 1, line 8: r~ = (w_hat - alpha . r) / (1 - alpha), per subband."""
    al = expand(alpha, sbs)
    return (w_hat - al * r) / (1.0 - al)


# ---------------------------------------------------------------------------
# VDAMP (Algorithm 1)
# ---------------------------------------------------------------------------


@dataclass
class Operators:
    """Phi, Psi, P and S for one slice (Algorithm 1, Require line and line 1)."""
    ny: int
    nx: int
    levels: int
    h: np.ndarray
    g: np.ndarray
    mask: np.ndarray            # bool (ny, nx): Omega
    p: np.ndarray               # float64 (ny, nx): sampling probability
    sbs: List[Subband] = field(default_factory=list)
    S: Optional[np.ndarray] = None   # (1+3s, ny, nx) unique columns of |F Psi^H|^2

    def psi(self, x):
        return dwt2(x, self.h, self.g, self.levels)

    def psi_h(self, w):
        return idwt2(w, self.h, self.g, self.levels, self.ny, self.nx)

    def phi(self, x):
        """Phi x = M_Omega F x, returned as a full grid that is zero off Omega."""
        return np.where(self.mask, fft2u(x), 0.0)

    def phi_h(self, v):
        """Phi^H v = F^H M_Omega^T v."""
        return ifft2u(np.where(self.mask, v, 0.0))


def make_operators(mask: np.ndarray, p: np.ndarray, wavelet: str, levels: int) -> Operators:
    ny, nx = mask.shape
    h, g = wavelet_filters(wavelet)
    ops = Operators(ny, nx, levels, h, g, mask.astype(bool), p.astype(np.float64))
    ops.sbs = subbands(ny, nx, levels)
    ops.S = s_columns(ny, nx, h, g, levels)
    return ops


def tau_estimate(z: np.ndarray, ops: Operators, sigma2: float) -> np.ndarray:
    """Algorithm 1, line 5: tau = S^H P^{-1} [(P^{-1} - 1)|z|^2 + sigma^2 1_n].

    Only rows j in Omega take part (S = |Phi Psi^H|^2 has one row per sample).
    """
    om = ops.mask
    pinv = 1.0 / ops.p[om]
    v = pinv * ((pinv - 1.0) * np.abs(z[om]) ** 2 + sigma2)
    return ops.S[:, om] @ v


@dataclass
class Record:
    """What one iteration k produced (Algorithm 1, lines 3-8)."""
    r_tilde: np.ndarray     # r~_k (input of the iteration)
    z: np.ndarray           # z_k, zero off Omega
    r: np.ndarray           # r_k
    tau: np.ndarray         # tau_k, one per subband
    theta: np.ndarray       # absolute thresholds lambda_k tau_k
    alpha: np.ndarray       # alpha_k
    w_hat: np.ndarray       # w_hat_k
    x_hat: Optional[np.ndarray] = None   # return line applied to w_hat_k


def final_estimate(w: np.ndarray, y: np.ndarray, ops: Operators) -> np.ndarray:
    """Algorithm 1, return line: x = Psi^H w + Phi^H (y - Phi Psi^H w)."""
    u = ops.psi_h(w)
    return u + ops.phi_h(y - ops.phi(u))


def iterate(r_tilde: np.ndarray, y: np.ndarray, ops: Operators, sigma2: float,
            want_x: bool = False) -> Record:
    """One pass of Algorithm 1, lines 3-8, from a given r~_k."""
    z = np.where(ops.mask, y - ops.phi(ops.psi_h(r_tilde)), 0.0)          # line 3
    pz = np.where(ops.mask, z / np.where(ops.mask, ops.p, 1.0), 0.0)
    r = r_tilde + ops.psi(ops.phi_h(pz))                                 # line 4
    tau = tau_estimate(z, ops, sigma2)                                   # line 5
    w_hat, theta, alpha = denoise(r, tau, ops.sbs)                       # lines 6-7
    rec = Record(r_tilde=r_tilde, z=z, r=r, tau=tau, theta=theta, alpha=alpha, w_hat=w_hat)
    if want_x:
        rec.x_hat = final_estimate(w_hat, y, ops)
    return rec


def next_r_tilde(rec: Record, ops: Operators) -> np.ndarray:
    """Algorithm 1, line 8 applied to a record."""
    return onsager(rec.w_hat, rec.r, rec.alpha, ops.sbs)


@dataclass
class Result:
    x_hat: np.ndarray
    records: List[Record]
    r_tilde_next: np.ndarray

    @property
    def tau(self):
        return np.stack([r.tau for r in self.records])

    @property
    def theta(self):
        return np.stack([r.theta for r in self.records])

    @property
    def alpha(self):
        return np.stack([r.alpha for r in self.records])


def vdamp(y: np.ndarray, mask: np.ndarray, p: np.ndarray, sigma: float, wavelet: str,
          levels: int, iters: int, r_tilde0: Optional[np.ndarray] = None,
          want_x: bool = False, ops: Optional[Operators] = None) -> Result:
    """Algorithm 1 (VDAMP) with the SURE soft-threshold denoiser of Sec. 3.

    y, mask and p are (ny, nx) arrays on the unshifted grid (y is ignored off the
    mask); sigma is sigma_eps.  Returns x_hat and the per-iteration records.
    """
    if ops is None:
        ops = make_operators(mask, p, wavelet, levels)
    y = np.where(ops.mask, y.astype(np.complex128), 0.0)
    sigma2 = float(sigma) ** 2
    rt = np.zeros(ops.ny * ops.nx, dtype=np.complex128) if r_tilde0 is None \
        else r_tilde0.astype(np.complex128)                              # line 1
    records = []
    for _ in range(iters):                                               # line 2
        rec = iterate(rt, y, ops, sigma2, want_x)
        records.append(rec)
        rt = next_r_tilde(rec, ops)                                      # line 8
    x_hat = final_estimate(records[-1].w_hat, y, ops)                    # return line
    return Result(x_hat=x_hat, records=records, r_tilde_next=rt)


def nmse_db(x_hat: np.ndarray, x0: np.ndarray) -> float:
    """10 log10(||x_hat - x0||^2 / ||x0||^2) (Sec. 3)."""
    return 10.0 * math.log10(float(np.sum(np.abs(x_hat - x0) ** 2))
                             / float(np.sum(np.abs(x0) ** 2)))
