"""Seeded synthetic inputs for the VDAMP problem y = Phi x0 + eps (Eq. 1).

This module only *creates problems*: phantom images x0, variable-density
sampling probabilities p, Bernoulli masks Omega, the noise level and the
measurements y.  It holds none of the reconstruction arithmetic (no wavelet,
no threshold, no tau, no Onsager term), so the FP64 oracle and the CUDA path
can both consume its output without sharing any of the method's code.

Every value is a deterministic function of (workload id, slice index, stream
name) through numpy's SeedSequence, so a problem can be rebuilt anywhere.

Recipe (stands in for the 512x512 Shepp-Logan phantom of Sec. 3, whose table is
not available here, and for simulated brain slices):

* phantom: E random ellipses on [-1, 1]^2 painted in order (later ones
  overwrite), centre ~ U[-0.6, 0.6]^2, semi-axes ~ U[0.05, 0.45],
  angle ~ U[0, pi), intensity ~ U[0, 1]; optional texture multiplies the
  inside of each ellipse by 1 + 0.15 cos(2 pi (f1 x + f2 y) + psi),
  f ~ U[1, 4], psi ~ U[0, 2 pi); magnitude clipped to [0, 1]; smooth phase
  phi = (pi/2) (a1 x + a2 y + a3 x y + a4 x^2 + a5 y^2) / 2.5, a ~ U[-1, 1].
* density (Sec. 3 says only "polynomial variable density"): with signed
  frequencies kappa (unshifted storage, DC at index 0),
  rho = sqrt((ky/(ny/2))^2 + (kx/(nx/2))^2),
  p = min(1, c (1 - rho/sqrt(2))^4), a c x c centre forced to p = 1, and c
  found by 60 FP64 bisection steps so that sum(p) = N / R.
* mask: independent Bernoulli draws, Prob(j in Omega) = p_j (Sec. 1).
* noise: complex Gaussian with white phase on the sampled entries, variance
  sigma^2 chosen from the SNR definition ||F x0||^2 / (N sigma^2) of Sec. 3
  with a unitary F.
"""
from __future__ import annotations

import dataclasses
import functools
import math
from typing import List, Optional

import numpy as np

_ROOT_KEY = 0x1911

_STREAMS = {"phantom": 1, "mask": 2, "noise": 3, "snr": 4, "rate": 5}


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic workload: image size, wavelet, sampling and iterations."""
    name: str
    workload_id: int
    ny: int
    nx: int
    ellipses: int
    texture: bool
    wavelet: str          # "haar" or "db4"
    levels: int
    rate: float           # undersampling factor R (or lower end of a range)
    rate_hi: float        # upper end of the per-slice range (== rate if fixed)
    centre: int           # side of the fully sampled centre square
    snr_db: float
    snr_db_hi: float
    iters: int
    batch: int


# The workloads, by what they are.
PLAIN_64_HAAR3 = Workload("plain 64x64 Haar s=3 R=4 30dB K=20", 1, 64, 64, 8, False,
                          "haar", 3, 4.0, 4.0, 8, 30.0, 30.0, 20, 1)
PLAIN_256_DB4_4 = Workload("plain 256x256 db4 s=4 R=5 30dB K=30", 2, 256, 256, 20, True,
                           "db4", 4, 5.0, 5.0, 24, 30.0, 30.0, 30, 1)
BATCH_320_DB4_5 = Workload("batched 256 x 320x320 db4 s=5 R=6 30dB K=20", 5, 320, 320, 20,
                           True, "db4", 5, 6.0, 6.0, 24, 30.0, 30.0, 20, 256)


def mixed_batch_workloads() -> List[Workload]:
    """96 slices of mixed size: 32 each of 128^2, 256^2 and 384x320."""
    out = []
    for i, (ny, nx, c) in enumerate(((128, 128, 16), (256, 256, 24), (384, 320, 24))):
        out.append(Workload(f"batched 32 x {ny}x{nx} db4 s=4 R~U[3,8] SNR~U[25,40] K=30",
                            30 + i, ny, nx, 20, True, "db4", 4, 3.0, 8.0, c, 25.0, 40.0,
                            30, 32))
    return out


def _rng(workload_id: int, slice_idx: int, stream: str) -> np.random.Generator:
    ss = np.random.SeedSequence([_ROOT_KEY, workload_id, slice_idx, _STREAMS[stream]])
    return np.random.Generator(np.random.Philox(ss))


def signed_freq(n: int) -> np.ndarray:
    """Signed frequency of each unshifted DFT index: i for i < n/2, else i - n."""
    i = np.arange(n)
    return np.where(i < n // 2, i, i - n)


def phantom(ny: int, nx: int, ellipses: int, texture: bool, rng: np.random.Generator
            ) -> np.ndarray:
    """Random-ellipse phantom with smooth phase, complex128 (ny, nx)."""
    yy = (2.0 * (np.arange(ny) + 0.5) / ny - 1.0)[:, None] * np.ones((1, nx))
    xx = (2.0 * (np.arange(nx) + 0.5) / nx - 1.0)[None, :] * np.ones((ny, 1))
    mag = np.zeros((ny, nx))
    for _ in range(ellipses):
        cy, cx = rng.uniform(-0.6, 0.6, size=2)
        ay, ax = rng.uniform(0.05, 0.45, size=2)
        ang = rng.uniform(0.0, math.pi)
        val = rng.uniform(0.0, 1.0)
        ca, sa = math.cos(ang), math.sin(ang)
        dx, dy = xx - cx, yy - cy
        u = ca * dx + sa * dy
        v = -sa * dx + ca * dy
        inside = (u / ax) ** 2 + (v / ay) ** 2 <= 1.0
        if texture:
            f1, f2 = rng.uniform(1.0, 4.0, size=2)
            psi = rng.uniform(0.0, 2.0 * math.pi)
            tex = 1.0 + 0.15 * np.cos(2.0 * math.pi * (f1 * xx + f2 * yy) + psi)
            mag = np.where(inside, val * tex, mag)
        else:
            mag = np.where(inside, val, mag)
    mag = np.clip(mag, 0.0, 1.0)
    a = rng.uniform(-1.0, 1.0, size=5)
    phase = (math.pi / 2.0) * (a[0] * xx + a[1] * yy + a[2] * xx * yy + a[3] * xx ** 2
                               + a[4] * yy ** 2) / 2.5
    return mag * np.exp(1j * phase)


@functools.lru_cache(maxsize=64)
def poly_density(ny: int, nx: int, rate: float, centre: int) -> np.ndarray:
    """Polynomial variable density p (float64, unshifted, read-only), sum(p) = N / rate."""
    ky = signed_freq(ny)[:, None] / (ny / 2.0)
    kx = signed_freq(nx)[None, :] / (nx / 2.0)
    rho = np.sqrt(ky * ky + kx * kx)
    t = 1.0 - rho / math.sqrt(2.0)
    t2 = t * t
    base = t2 * t2
    cy = signed_freq(ny)[:, None]
    cx = signed_freq(nx)[None, :]
    h = centre // 2
    in_centre = (cy >= -h) & (cy <= centre - h - 1) & (cx >= -h) & (cx <= centre - h - 1)
    target = ny * nx / rate

    def total(c: float) -> float:
        return float(np.where(in_centre, 1.0, np.minimum(1.0, c * base)).sum())

    lo, hi = 0.0, 1.0
    while total(hi) < target and hi < 1e12:
        hi *= 2.0
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if total(mid) < target:
            lo = mid
        else:
            hi = mid
    c = 0.5 * (lo + hi)
    p = np.where(in_centre, 1.0, np.minimum(1.0, c * base))
    p.setflags(write=False)
    return p


@dataclasses.dataclass
class Problem:
    """One slice: ground truth, inputs of Algorithm 1 and the workload it came from.

    y, density and sigma are stored at the precision the GPU path consumes
    (complex64, float32, float32); the oracle upcasts these same values.
    """
    x0: np.ndarray          # complex128 (ny, nx) ground truth image
    y: np.ndarray           # complex64  (ny, nx) measurements, 0 off the mask
    mask: np.ndarray        # uint8      (ny, nx) 1 where sampled
    density: np.ndarray     # float32    (ny, nx) sampling probability p
    sigma: np.float32       # noise standard deviation sigma_eps
    wavelet: str
    levels: int
    iters: int
    rate: float
    snr_db: float


def make_problem(wl: Workload, slice_idx: int = 0, ny: Optional[int] = None,
                 nx: Optional[int] = None) -> Problem:
    """Build slice `slice_idx` of workload `wl` (sizes may be overridden)."""
    ny = wl.ny if ny is None else ny
    nx = wl.nx if nx is None else nx
    x0 = phantom(ny, nx, wl.ellipses, wl.texture, _rng(wl.workload_id, slice_idx, "phantom"))
    rate = wl.rate if wl.rate_hi == wl.rate else float(
        _rng(wl.workload_id, slice_idx, "rate").uniform(wl.rate, wl.rate_hi))
    snr = wl.snr_db if wl.snr_db_hi == wl.snr_db else float(
        _rng(wl.workload_id, slice_idx, "snr").uniform(wl.snr_db, wl.snr_db_hi))
    p64 = poly_density(ny, nx, rate, wl.centre)
    p32 = p64.astype(np.float32)
    u = _rng(wl.workload_id, slice_idx, "mask").random((ny, nx))
    mask = (u < p32.astype(np.float64)).astype(np.uint8)
    n_pix = ny * nx
    sigma2 = float(np.sum(np.abs(x0) ** 2)) / (n_pix * 10.0 ** (snr / 10.0))
    sigma32 = np.float32(math.sqrt(sigma2))
    s = float(sigma32)
    g = _rng(wl.workload_id, slice_idx, "noise")
    eps = (g.standard_normal((ny, nx)) + 1j * g.standard_normal((ny, nx))) * (s / math.sqrt(2.0))
    kspace = np.fft.fft2(x0, norm="ortho")  # acquisition model: unitary 2D DFT
    y = np.where(mask == 1, kspace + eps, 0.0).astype(np.complex64)
    return Problem(x0=x0, y=y, mask=mask, density=p32, sigma=sigma32, wavelet=wl.wavelet,
                   levels=wl.levels, iters=wl.iters, rate=rate, snr_db=snr)


def make_batch(wl: Workload, count: Optional[int] = None) -> List[Problem]:
    n = wl.batch if count is None else count
    return [make_problem(wl, i) for i in range(n)]
