"""State-evolution diagnostics of a VDAMP run (Eq. 5; analogues of Fig. 3-5).

VDAMP's state evolution says that at every iteration k the effective
observation r_k equals the true wavelet coefficients w0 = Psi x0 plus
Gaussian noise whose variance in subband b is tau_b (white within a subband,
colored across subbands).  With a known ground truth (synthetic phantoms)
this module runs the iteration on the GPU through the C ABI (vdamp_iterate
for r_k and tau_k, vdamp_psi for w0, vdamp_solve for the per-iteration
estimates) and summarises, per iteration and subband:

  ratio     mean |r_k - w0|^2 / tau_b      (1 when tau predicts the error)
  skew_re, skew_im, kurt_re, kurt_im
            skewness and excess kurtosis of Re and Im of r_k - w0 (0 if Gaussian)
  ks        Kolmogorov-Smirnov distance between Re, Im of (r_k - w0)/sqrt(tau_b/2)
            and N(0, 1) (the largest gap of the QQ plot, in probability)
  lag1      correlation of horizontally adjacent errors inside the subband
            (0 for white noise)

and per iteration the NMSE of the return line applied to w_hat_k.  Only
these statistics are computed on the host, from the device results; every
step of the iteration runs in the library's kernels.
"""
from __future__ import annotations

import math
from typing import Dict, List

import numpy as np

from . import binding as vb


def _moments(v: np.ndarray):
    m = v.mean()
    d = v - m
    s2 = np.mean(d * d)
    if s2 <= 0:
        return 0.0, 0.0
    return float(np.mean(d ** 3) / s2 ** 1.5), float(np.mean(d ** 4) / s2 ** 2 - 3.0)


def _ks_normal(v: np.ndarray) -> float:
    x = np.sort(v)
    n = len(x)
    cdf = 0.5 * (1.0 + np.vectorize(math.erf)(x / math.sqrt(2.0)))
    hi = np.arange(1, n + 1) / n - cdf
    lo = cdf - np.arange(0, n) / n
    return float(max(hi.max(), lo.max()))


def subband_layout(ny: int, nx: int, levels: int) -> List[Dict]:
    """Packed subband order A_s, H_s, V_s, D_s, ..., H_1, V_1, D_1 with offsets and shapes."""
    out, off = [], 0
    h, w = ny >> levels, nx >> levels
    out.append({"name": f"A{levels}", "offset": off, "h": h, "w": w})
    off += h * w
    for j in range(levels, 0, -1):
        h, w = ny >> j, nx >> j
        for kind in "HVD":
            out.append({"name": f"{kind}{j}", "offset": off, "h": h, "w": w})
            off += h * w
    return out


def state_evolution(plan, y, mask, density, sigma: float, x0, iters: int) -> Dict:
    """Diagnostics of one slice.  y, mask, density: torch device tensors [1][ny][nx];
    x0: complex ground truth (numpy [ny][nx]).  Returns a dict of per-iteration lists."""
    import torch
    ny, nx, levels = plan.ny, plan.nx, plan.levels
    N, B = ny * nx, plan.B
    dev = y.device
    x0d = torch.from_numpy(np.ascontiguousarray(x0.astype(np.complex64)[None])).to(dev)
    w0d = torch.empty((1, N), dtype=torch.complex64, device=dev)
    vb.vdamp_psi(plan.handle, 1, x0d, w0d)
    rt = torch.zeros((1, N), dtype=torch.complex64, device=dev)
    r, rn = torch.empty_like(rt), torch.empty_like(rt)
    tau = torch.empty((1, B), dtype=torch.float64, device=dev)
    thr, alpha = torch.empty_like(tau), torch.empty_like(tau)
    sol = plan.solve(y, mask, density, [sigma], iters, want_iters=True)
    torch.cuda.synchronize()
    w0 = w0d.cpu().numpy()[0].astype(np.complex128)
    x0n = float(np.sum(np.abs(x0) ** 2))
    bands = subband_layout(ny, nx, levels)
    rows = []
    for k in range(iters):
        vb.vdamp_iterate(plan.handle, 1, rt, y, mask, density, [sigma], r, tau, thr, alpha, rn)
        torch.cuda.synchronize()
        e = r.cpu().numpy()[0].astype(np.complex128) - w0
        t = tau.cpu().numpy()[0]
        per = []
        for b, sb in enumerate(bands):
            n = sb["h"] * sb["w"]
            eb = e[sb["offset"]:sb["offset"] + n]
            sre, kre = _moments(eb.real)
            sim, kim = _moments(eb.imag)
            z = np.concatenate([eb.real, eb.imag]) / math.sqrt(max(t[b], 1e-300) / 2.0)
            g = eb.reshape(sb["h"], sb["w"])
            a, c = g[:, :-1].ravel(), g[:, 1:].ravel()
            den = math.sqrt(float(np.sum(np.abs(a) ** 2) * np.sum(np.abs(c) ** 2))) or 1.0
            per.append({"band": sb["name"], "size": n, "tau": float(t[b]),
                        "err": float(np.mean(np.abs(eb) ** 2)),
                        "ratio": float(np.mean(np.abs(eb) ** 2) / t[b]) if t[b] > 0 else float("nan"),
                        "skew_re": sre, "skew_im": sim, "kurt_re": kre, "kurt_im": kim,
                        "ks": _ks_normal(z) if n >= 64 else float("nan"),
                        "lag1": float(np.real(np.vdot(a, c)) / den) if a.size else float("nan"),
                        "theta": float(thr.cpu().numpy()[0][b]),
                        "alpha": float(alpha.cpu().numpy()[0][b])})
        xk = sol["x_hat_iters"][k, 0].cpu().numpy().astype(np.complex128)
        nm = 10.0 * math.log10(float(np.sum(np.abs(xk - x0) ** 2)) / x0n)
        rows.append({"k": k, "nmse_db": nm, "bands": per})
        rt, rn = rn, rt
    return {"ny": ny, "nx": nx, "levels": levels, "iters": iters, "rows": rows}


def to_markdown(d: Dict, min_size: int = 1024) -> str:
    """A compact table: per iteration, NMSE and the worst subband statistics over subbands
    of at least min_size coefficients."""
    out = ["| k | NMSE dB | ratio min | ratio max | max abs skew | max abs ex. kurtosis | "
           "max KS | lag-1 corr (mean) |", "|---|---|---|---|---|---|---|---|"]
    for row in d["rows"]:
        bs = [b for b in row["bands"] if b["size"] >= min_size]
        if not bs:
            continue
        out.append("| %d | %.2f | %.3f | %.3f | %.3f | %.3f | %.3f | %.3f |" % (
            row["k"], row["nmse_db"], min(b["ratio"] for b in bs), max(b["ratio"] for b in bs),
            max(max(abs(b["skew_re"]), abs(b["skew_im"])) for b in bs),
            max(max(abs(b["kurt_re"]), abs(b["kurt_im"])) for b in bs),
            max(b["ks"] for b in bs), float(np.mean([b["lag1"] for b in bs]))))
    return "\n".join(out)
