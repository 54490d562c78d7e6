"""Learned VDAMP: a per-subband CNN denoiser in place of the soft threshold.

The paper anticipates denoisers beyond the soft threshold once the state
evolution makes the effective noise of every subband known (concluding
section).  Here, per subband index b, a network n_b of five 3x3
convolutions (3 -> 32 -> 32 -> 32 -> 32 -> 2 channels, ReLU, zero padding)
denoises in residual form

    f(r) = r - sqrt(tau_b) n_b(Re r / sqrt(tau_b), Im r / sqrt(tau_b), 0.1 ln tau_b),

its divergence for the Onsager term (Algorithm 1 line 7) comes from one
Hutchinson probe through the network's forward-mode derivative, and SURE
judges it per subband against the plain SURE soft threshold, which is kept
wherever the network's SURE is not lower (lines 6-8 in
vdamp_cnn_onsager).  Every convolution runs on the tcgen05 tensor cores
(BF16 operands, FP32 accumulation); the weight gradients, the loss, Adam
and all elementwise steps run in this library's kernels.  This module only
sequences the C-ABI calls and holds the buffers (torch device memory).

Training pairs (r_k, w0 = Psi x0) come from plain VDAMP itself, run on
seeded synthetic phantoms of the 256x256 db4 workload's kind (other slice
seeds than the ones evaluated).
"""
from __future__ import annotations

import math
from typing import Dict, List, Optional, Sequence

import numpy as np

from . import binding as vb
from . import diagnostics, synth

# (cin, cout) of the five layers as computed: the input has 16 channels (3
# used) and the output 16 (2 used); the padded weights start at zero and
# receive zero gradients, so they stay zero.
LAYERS = [(16, 32), (32, 32), (32, 32), (32, 32), (32, 16)]
REAL = [(3, 32), (32, 32), (32, 32), (32, 32), (32, 2)]

def lib():
    return vb.load()


def _p(t):
    return None if t is None else t.data_ptr()


def _st(stream):
    import torch
    return torch.cuda.current_stream().cuda_stream if stream is None else int(stream)


class Images:
    """Image list of one launch (see include/vdamp.h): entries
    (h, w, src_off, src_pitch, band, slice); dense pixels follow the list order;
    tiles / ctiles count the elementwise and the convolution tiles."""

    def __init__(self, entries: Sequence, device="cuda", dense_offsets=None):
        import torch
        rows, off, tile, ctile = [], 0, 0, 0
        for i, (h, w, src_off, pitch, band, slc) in enumerate(entries):
            o = off if dense_offsets is None else dense_offsets[i]
            rows.append([o, h, w, tile, src_off, pitch, band, slc, ctile])
            off += h * w
            tile += (h * w + 127) // 128
            wb = min(w, 30)   # convolution blocks: wb columns x floor(128 / (wb + 2)) rows
            ctile += ((w + wb - 1) // wb) * ((h + 128 // (wb + 2) - 1) // (128 // (wb + 2)))
        self.n = len(rows)
        self.tiles = tile
        self.ctiles = ctile
        self.max_w = max(e[1] for e in entries)
        self.pixels = off if dense_offsets is None else max(
            d + e[0] * e[1] for d, e in zip(dense_offsets, entries))
        self.rows = np.array(rows, dtype=np.int32)
        self.dev = torch.from_numpy(self.rows.reshape(-1).copy()).to(device)

    @staticmethod
    def subbands(ny: int, nx: int, levels: int, batch: int, device="cuda") -> "Images":
        """Every subband of every slice, dense layout = the packed layout."""
        N = ny * nx
        ents, offs = [], []
        for s in range(batch):
            for b, sb in enumerate(diagnostics.subband_layout(ny, nx, levels)):
                ents.append((sb["h"], sb["w"], s * N + sb["offset"], sb["w"], b, s))
                offs.append(s * N + sb["offset"])
        return Images(ents, device, dense_offsets=offs)


class SubbandCNN:
    """Weights (FP32 masters + BF16 operand images), Adam state and workspace."""

    def __init__(self, bands: int, seed: int = 0, device="cuda"):
        import torch
        self.bands = bands
        self.device = device
        rng = np.random.default_rng(seed)
        self.w, self.b = [], []
        for (cin, cout), (rin, rout) in zip(LAYERS, REAL):
            w = np.zeros((bands, cout, 9, cin), dtype=np.float32)
            w[:, :rout, :, :rin] = rng.standard_normal((bands, rout, 9, rin)) * math.sqrt(
                2.0 / (9 * rin))
            if rout == 2:   # start near the identity denoiser: a small last layer
                w *= 0.1
            self.w.append(torch.from_numpy(w).to(device))
            self.b.append(torch.zeros((bands, cout), dtype=torch.float32, device=device))
        self.params = self.w + self.b
        self.m = [torch.zeros_like(p) for p in self.params]
        self.v = [torch.zeros_like(p) for p in self.params]
        self.steps = 0
        self.wimg = [torch.empty(bands * cout * 9 * cin, dtype=torch.bfloat16, device=device)
                     for cin, cout in LAYERS]
        self.wimgT = [torch.empty(bands * cin * 9 * cout, dtype=torch.bfloat16, device=device)
                      for cin, cout in LAYERS]
        self.status = torch.zeros(1, dtype=torch.int32, device=device)
        self._ws: Dict[str, object] = {}
        self.pack()

    # ---------------------------------------------------------------- io ---
    def state(self) -> Dict[str, np.ndarray]:
        out = {}
        for l in range(5):
            out[f"w{l}"] = self.w[l].cpu().numpy()
            out[f"b{l}"] = self.b[l].cpu().numpy()
        return out

    def load_state(self, st: Dict[str, np.ndarray]):
        import torch
        for l in range(5):
            self.w[l].copy_(torch.from_numpy(st[f"w{l}"]))
            self.b[l].copy_(torch.from_numpy(st[f"b{l}"]))
        self.pack()

    def oracle_params(self, band: int):
        """This band's weights in the oracle's form (real channels only)."""
        out = []
        for l, ((rin, rout)) in enumerate(REAL):
            out.append((self.w[l][band, :rout, :, :rin].double().cpu().numpy(),
                        self.b[l][band, :rout].double().cpu().numpy()))
        return out

    def pack(self, stream=None):
        L, st = lib(), _st(stream)
        for l, (cin, cout) in enumerate(LAYERS):
            vb.check(L.vdamp_cnn_pack_weights(_p(self.w[l]), self.bands, cin, cout, cin, cout, 0,
                                              _p(self.wimg[l]), st), "vdamp_cnn_pack_weights")
            if l > 0:
                vb.check(L.vdamp_cnn_pack_weights(_p(self.w[l]), self.bands, cin, cout, cout,
                                                  cin, 1, _p(self.wimgT[l]), st),
                         "vdamp_cnn_pack_weights")

    # ---------------------------------------------------------- buffers ---
    def _buf(self, name, shape, dtype):
        import torch
        t = self._ws.get(name)
        n = int(np.prod(shape))
        if t is None or t.numel() < n or t.dtype != dtype:
            t = torch.empty(max(n, 1), dtype=dtype, device=self.device)
            self._ws[name] = t
        return t[:n].view(*shape)

    def conv(self, l, x, out, mode, im: Images, mask=None, transposed=False, cout_store=0,
             stream=None):
        cin, cout = LAYERS[l]
        if transposed:
            cin, cout = cout, cin
        img = self.wimgT[l] if transposed else self.wimg[l]
        vb.check(lib().vdamp_cnn_conv3x3(_p(x), cin, _p(img), cout, _p(self.b[l]), _p(mask),
                                         _p(out), mode, 1 if transposed else 0, cout_store,
                                         _p(im.dev), im.n, im.ctiles, im.max_w, _p(self.status),
                                         _st(stream)), "vdamp_cnn_conv3x3")

    # ---------------------------------------------------------- passes ---
    def forward(self, im: Images, x0, stream=None):
        """n (FP32 [pixels][2]) and the activations [x0, a1..a4]."""
        import torch
        acts = [x0]
        a = x0
        for l in range(4):
            o = self._buf(f"a{l + 1}", (im.pixels, LAYERS[l][1]), torch.bfloat16)
            self.conv(l, a, o, 0, im, stream=stream)
            acts.append(o)
            a = o
        n = self._buf("n", (im.pixels, 2), torch.float32)
        self.conv(4, a, n, 2, im, cout_store=2, stream=stream)
        return n, acts

    def jvp(self, im: Images, acts, t0, stream=None):
        import torch
        t = t0
        for l in range(4):
            o = self._buf(f"j{l % 2}", (im.pixels, LAYERS[l][1]), torch.bfloat16)
            self.conv(l, t, o, 1, im, mask=acts[l + 1], stream=stream)
            t = o
        jn = self._buf("jn", (im.pixels, 2), torch.float32)
        self.conv(4, t, jn, 3, im, cout_store=2, stream=stream)
        return jn

    def backward(self, im: Images, acts, dn, grads, stream=None):
        """Accumulate d(loss)/d(params) into grads (list like self.params) from dn."""
        import torch
        L, st = lib(), _st(stream)
        d = dn
        for l in range(4, -1, -1):
            cin, cout = LAYERS[l]
            vb.check(L.vdamp_cnn_wgrad(_p(acts[l]), cin, cin, _p(d), cout, cout, _p(im.dev),
                                       im.n, im.tiles, _p(grads[l]), _p(grads[5 + l]), st),
                     "vdamp_cnn_wgrad")
            if l > 0:
                o = self._buf(f"d{l % 2}", (im.pixels, cin), torch.bfloat16)
                self.conv(l, d, o, 1, im, mask=acts[l], transposed=True, stream=stream)
                d = o
        return grads

    def adam(self, grads, lr, stream=None, b1=0.9, b2=0.999, eps=1e-8):
        L, st = lib(), _st(stream)
        self.steps += 1
        for p, g, m, v in zip(self.params, grads, self.m, self.v):
            vb.check(L.vdamp_cnn_adam(_p(p), _p(g), _p(m), _p(v), p.numel(), lr, b1, b2, eps,
                                      self.steps, st), "vdamp_cnn_adam")
        self.pack(stream)

    def input(self, im: Images, r, tau, B, stream=None):
        import torch
        x0 = self._buf("x0", (im.pixels, 16), torch.bfloat16)
        vb.check(lib().vdamp_cnn_input(_p(r), _p(tau), B, _p(im.dev), im.n, im.tiles, _p(x0),
                                       _st(stream)), "vdamp_cnn_input")
        return x0

    def train_step(self, im: Images, r, w0, tau, B, lr, stream=None):
        """One Adam step on the images (patches of r with targets w0); returns the
        loss as a device scalar (mean |f - w0|^2 per coefficient)."""
        import torch
        L, st = lib(), _st(stream)
        x0 = self.input(im, r, tau, B, stream)
        n, acts = self.forward(im, x0, stream)
        dn = self._buf("dn", (im.pixels, 16), torch.bfloat16)
        loss = self._buf("loss", (1,), torch.float64)
        loss.zero_()
        vb.check(L.vdamp_cnn_loss(_p(r), _p(w0), _p(tau), B, _p(im.dev), im.n, im.tiles, _p(n),
                                  1.0 / im.pixels, _p(dn), _p(loss), st), "vdamp_cnn_loss")
        grads = [self._buf(f"g{i}", tuple(p.shape), torch.float32) for i, p in
                 enumerate(self.params)]
        for g in grads:
            g.zero_()
        self.backward(im, acts, dn, grads, stream)
        self.adam(grads, lr, stream)
        return loss

    def denoise(self, im: Images, r, tau, B, seed, f_out, sums, stream=None):
        """f = the network's output at every image, and per image (sum |f - r|^2,
        eta . J_n eta) for the probe `seed`."""
        import torch
        L, st = lib(), _st(stream)
        x0 = self.input(im, r, tau, B, stream)
        n, acts = self.forward(im, x0, stream)
        t0 = self._buf("t0", (im.pixels, 16), torch.bfloat16)
        vb.check(L.vdamp_cnn_probe(seed, _p(im.dev), im.n, im.tiles, _p(t0), st),
                 "vdamp_cnn_probe")
        jn = self.jvp(im, acts, t0, stream)
        sums.zero_()
        vb.check(L.vdamp_cnn_output(_p(r), _p(tau), B, _p(im.dev), im.n, im.tiles, _p(n),
                                    _p(jn), seed, _p(f_out), _p(sums), st), "vdamp_cnn_output")


# ------------------------------------------------------------ training ---

def make_pairs(ny, nx, wavelet, levels, slices, iters, workload_id=77, rate=5.0, stream=None):
    """Plain VDAMP (this library) on seeded phantoms of the given kind (20 textured
    ellipses, 24x24 centre, 30 dB, undersampling `rate`): returns (R [pairs][N]
    complex64, W0 [slices][N], TAU [pairs][B], slice of each pair)."""
    import torch
    wl = synth.Workload("training phantoms", workload_id, ny, nx, 20, True, wavelet, levels,
                        rate, rate, 24, 30.0, 30.0, iters, 1)
    plan = vb.Plan(ny, nx, wavelet, levels)
    N, B = ny * nx, plan.B
    R = torch.empty((slices * iters, N), dtype=torch.complex64, device="cuda")
    W0 = torch.empty((slices, N), dtype=torch.complex64, device="cuda")
    TAU = torch.empty((slices * iters, B), dtype=torch.float64, device="cuda")
    owner = np.repeat(np.arange(slices), iters)
    thr = torch.empty((1, B), dtype=torch.float64, device="cuda")
    alpha = torch.empty_like(thr)
    rt = torch.zeros((1, N), dtype=torch.complex64, device="cuda")
    rn = torch.empty_like(rt)
    for s in range(slices):
        pr = synth.make_problem(wl, s)
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a[None])).cuda()
        y, m, p = dev(pr.y), dev(pr.mask), dev(pr.density)
        vb.vdamp_psi(plan.handle, 1, dev(pr.x0.astype(np.complex64)), W0[s:s + 1])
        rt.zero_()
        for k in range(iters):
            i = s * iters + k
            vb.vdamp_iterate(plan.handle, 1, rt, y, m, p, [pr.sigma], R[i:i + 1], TAU[i:i + 1],
                             thr, alpha, rn)
            rt, rn = rn, rt
    torch.cuda.synchronize()
    plan.close()
    return R, W0, TAU, owner


def train(net: SubbandCNN, R, W0, TAU, owner, ny, nx, levels, steps=1500, patches=8,
          patch=32, lr=1e-3, seed=0, log_every=0):
    """Adam on random patches: each step takes `patches` patches of every subband
    (whole subbands when smaller than the patch) from random pairs."""
    import torch
    rng = np.random.default_rng(seed)
    layout = diagnostics.subband_layout(ny, nx, levels)
    N = ny * nx
    B = len(layout)
    pairs = R.shape[0]
    # targets: W0 per pair (index by slice) gathered once per step into a pair-major view
    hist = []
    for step in range(steps):
        ents = []
        for b, sb in enumerate(layout):
            ph, pw = min(patch, sb["h"]), min(patch, sb["w"])
            for _ in range(patches):
                i = int(rng.integers(pairs))
                y0 = int(rng.integers(sb["h"] - ph + 1))
                x0 = int(rng.integers(sb["w"] - pw + 1))
                ents.append((ph, pw, i * N + sb["offset"] + y0 * sb["w"] + x0, sb["w"], b, i))
        im = Images(ents)
        loss = net.train_step(im, R, _targets(W0, owner, R), TAU, B, lr)
        if log_every and step % log_every == 0:
            hist.append((step, float(loss.item())))
    return hist


_TGT = {}


def _targets(W0, owner, R):
    """W0 laid out pair by pair (the training kernels index targets like r)."""
    key = (W0.data_ptr(), R.shape[0])
    t = _TGT.get(key)
    if t is None:
        import torch
        t = W0[torch.from_numpy(owner).to(W0.device)]
        _TGT.clear()
        _TGT[key] = t
    return t


# ---------------------------------------------------------- learned solve ---

class LearnedSolver:
    """Algorithm 1 with the per-subband choice between the network and the SURE
    soft threshold at every iteration (net=None: the soft threshold everywhere,
    i.e. the plain method through the same steps).  Buffers are allocated once;
    capture() records a whole solve on the given inputs into a CUDA graph that
    replay() runs again (the inputs' memory and the sigma values are baked in)."""

    def __init__(self, plan, net: Optional[SubbandCNN], batch: int, iters: int, seed: int = 1,
                 want_iters: bool = False):
        import torch
        self.plan, self.net, self.batch, self.iters, self.seed = plan, net, batch, iters, seed
        ny, nx, B = plan.ny, plan.nx, plan.B
        N = ny * nx
        self.im = Images.subbands(ny, nx, plan.levels, batch)
        z = lambda: torch.zeros((batch, N), dtype=torch.complex64, device="cuda")
        self.rt, self.rt_soft, self.r, self.f, self.w_hat = z(), z(), z(), z(), z()
        d = lambda *s: torch.zeros(s, dtype=torch.float64, device="cuda")
        self.tau, self.thr, self.alpha, self.sure_soft = (d(batch, B) for _ in range(4))
        self.sums = d(2 * self.im.n)
        self.use = torch.zeros((iters, self.im.n), dtype=torch.int32, device="cuda")
        self.al = d(iters, self.im.n)
        self.taus, self.thrs = d(iters, batch, B), d(iters, batch, B)
        self.x_hat = torch.zeros((batch, ny, nx), dtype=torch.complex64, device="cuda")
        self.xs = torch.zeros((iters, batch, ny, nx), dtype=torch.complex64, device="cuda") \
            if want_iters else None
        self.graph = None

    def run(self, y, mask, density, sigma, stream=None, r_tilde0=None, k0=0):
        """Iterations k0 .. k0 + iters - 1 from r~ = r_tilde0 (None: 0, with k0 = 0); the
        probe of iteration k has seed + k, so a resumed run draws the probes the
        uninterrupted one would have."""
        L, st = lib(), _st(stream)
        plan, B = self.plan, self.plan.B
        if r_tilde0 is None:
            if k0 != 0:
                raise ValueError("k0 must be 0 for a cold start")
            self.rt.zero_()
        else:
            self.rt.copy_(r_tilde0)
        for k in range(self.iters):
            vb.vdamp_iterate(plan.handle, self.batch, self.rt, y, mask, density, sigma, self.r,
                             self.tau, self.thr, self.alpha, self.rt_soft, stream=st)
            vb.check(L.vdamp_last_sure(plan.handle, self.batch, _p(self.sure_soft), st),
                     "vdamp_last_sure")
            self.taus[k].copy_(self.tau)
            self.thrs[k].copy_(self.thr)
            if self.net is not None:
                self.net.denoise(self.im, self.r, self.tau, B, self.seed + k0 + k, self.f,
                                 self.sums, st)
            else:
                self.sums.zero_()
            vb.check(L.vdamp_cnn_onsager(_p(self.r), _p(self.f) if self.net is not None else None,
                                         _p(self.tau), _p(self.thr), _p(self.alpha),
                                         _p(self.sure_soft), B, _p(self.sums), _p(self.im.dev),
                                         self.im.n, self.im.tiles, _p(self.rt), _p(self.w_hat),
                                         _p(self.use[k]), _p(self.al[k]), st),
                     "vdamp_cnn_onsager")
            if self.xs is not None:
                vb.vdamp_final_estimate(plan.handle, self.batch, self.w_hat, y, mask, self.xs[k],
                                        stream=st)
        vb.vdamp_final_estimate(plan.handle, self.batch, self.w_hat, y, mask, self.x_hat,
                                stream=st)
        return self.outputs()

    def capture(self, y, mask, density, sigma):
        import torch
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.run(y, mask, density, sigma, stream=s.cuda_stream)   # warm-up (allocations)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=s):
            self.run(y, mask, density, sigma, stream=s.cuda_stream)
        torch.cuda.synchronize()
        return self

    def replay(self):
        self.graph.replay()
        return self.outputs()

    def check(self, stream=None):
        """Raise VdampError(VDAMP_ETIMEOUT) if a convolution's bounded wait for the tensor
        cores ran out since the last check (waits for `stream`; not inside a capture)."""
        if self.net is not None:
            vb.check(vb.vdamp_cnn_status(self.net.status, _st(stream)), "learned solve")

    def outputs(self):
        B = self.plan.B
        return {"x_hat": self.x_hat, "tau": self.taus, "thr": self.thrs, "r_tilde": self.rt,
                "use": self.use.view(self.iters, self.batch, B),
                "alpha": self.al.view(self.iters, self.batch, B), "x_hat_iters": self.xs}


def solve_learned(plan, net: Optional[SubbandCNN], y, mask, density, sigma, iters, seed=1,
                  want_iters=False, stream=None):
    """One learned solve (see LearnedSolver); returns x_hat, tau, thr (soft), the
    per-iteration network use [iters][batch][B], alpha [iters][batch][B] and, with
    want_iters, x_hat after every iteration [iters][batch][ny][nx]."""
    return LearnedSolver(plan, net, y.shape[0], iters, seed, want_iters).run(
        y, mask, density, sigma, stream)


def train_default(slices=52, iters=30, steps=1500, seed=0, log_every=100, timings=None):
    """The denoiser of the 256x256 db4 s=4 workload: about 20k subband pairs
    (52 phantoms x 30 iterations x 13 subbands) from plain VDAMP, then Adam on
    32x32 patches (8 per subband and step).  Returns the network and the
    loss history."""
    return train_for(256, 256, "db4", 4, 5.0, slices, iters, steps, 77, seed, log_every,
                     timings)


def train_for(ny, nx, wavelet, levels, rate, slices, iters, steps=1500, workload_id=77, seed=0,
              log_every=100, timings=None):
    """A denoiser for slices of one kind: slices x iters x (1 + 3 levels) subband
    pairs from plain VDAMP on seeded phantoms (seed `workload_id`), then Adam."""
    import time

    import torch
    t0 = time.perf_counter()
    R, W0, TAU, owner = make_pairs(ny, nx, wavelet, levels, slices, iters, workload_id, rate)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    net = SubbandCNN(bands=1 + 3 * levels, seed=seed)
    hist = train(net, R, W0, TAU, owner, ny, nx, levels, steps=steps, seed=seed,
                 log_every=log_every)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    if timings is not None:
        timings.update({"pairs_s": t1 - t0, "train_s": t2 - t1,
                        "pairs": int(R.shape[0]) * (1 + 3 * levels), "steps": steps})
    _TGT.clear()
    del R, W0, TAU
    return net, hist


def time_denoiser(batch: int = 64, reps: int = 10, seed: int = 0):
    """Times one denoiser application (input planes, the 5 convolutions, the
    probe, the 5 JVP convolutions, the output sums) on `batch` synthetic
    256x256 db4 s=4 slices; returns (ms, TFLOP/s of the convolutions)."""
    import torch
    net = SubbandCNN(13, seed=seed)
    im = Images.subbands(256, 256, 4, batch)
    g = torch.Generator(device="cuda").manual_seed(seed)
    r = torch.randn((batch, 65536), dtype=torch.complex64, device="cuda", generator=g)
    tau = torch.full((batch, 13), 0.5, dtype=torch.float64, device="cuda")
    f = torch.empty_like(r)
    sums = torch.zeros(2 * im.n, dtype=torch.float64, device="cuda")
    for _ in range(3):
        net.denoise(im, r, tau, 13, 7, f, sums)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        net.denoise(im, r, tau, 13, 7, f, sums)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    flop = batch * 65536 * 2 * sum(9 * ci * co for ci, co in LAYERS) * 2
    return ms, flop / ms / 1e9


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser(description="time the learned denoiser on synthetic slices")
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--reps", type=int, default=10)
    args = ap.parse_args()
    vb.load()
    ms, tf = time_denoiser(args.batch, args.reps)
    print(f"batch {args.batch}: denoise {ms:.3f} ms, {tf:.1f} TFLOP/s of convolution")
