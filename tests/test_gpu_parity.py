"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (FP32 kernels against FP64 arithmetic):
* transforms F, F^H, Psi, Psi^H: relative L2 error <= 2e-6 (a few FP32 ulps
  accumulated over log2(n) butterfly stages or s filter levels);
* the solve: x_hat and the tau vector within 1e-4 relative L2 at every
  iteration (each subband's tau within 1e-3 relative), thresholds within 1e-3
  relative, final NMSE within 0.01 dB;
* a threshold outside 1e-3 is accepted only as a SURE tie: the oracle's FP64
  SURE at both thresholds differs by at most 1e-6 of the scale of its terms
  (sum a^2 + N_b tau), the resolution of the kernel's FP32 curve.

On the 256x256 db4 workload the iteration itself amplifies perturbations by
about 1.5x per iteration (test_iteration_sensitivity_to_state_rounding in the
oracle pins): the FP64 oracle with its state merely rounded to complex64 drifts
to 1e-3 of itself by the end, and FP64 runs perturbed at 1e-7 end 0.017 dB
apart in NMSE.  An FP32 trajectory therefore follows the FP64 one to 1e-4 only
for its first iterations, and a SURE near-tie (two local minima whose order
flips under an FP32-level change of r_k) can send the two runs to different
thresholds.  The free-running test therefore holds the tolerances for k < 10
or until the runs first pick different thresholds (which must not happen
before k = 5); every iteration is held to them teacher-forced (each step
started from the oracle's own r~_k, where a threshold difference must be a
certified tie); and the final NMSE must fall within 4 standard deviations
(at least 0.02 dB) of the mean of FP64 oracle runs perturbed at the FP32 level
(state rounded to complex64, then multiplied by 1 + 1e-6 N(0, 1) before every
iteration).  24 such runs spread with a standard deviation of 0.014 dB over a
range of 0.054 dB; with 4e-6 the range widens to 0.077 dB.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import vdamp_oracle as O
from paper_1911_01234_gb300 import binding as vb
from paper_1911_01234_gb300 import build, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    vb.load()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def crand(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def tau_ok(t_gpu, t_orc):
    """tau vector within 1e-4 relative L2, every subband within 1e-3 relative."""
    return rel(t_gpu, t_orc) < 1e-4 and np.max(np.abs(t_gpu - t_orc) / t_orc) < 1e-3


def theta_ok(r, sbs, tau, th_gpu, th_orc):
    """Thresholds agree within 1e-3, or the oracle's SURE says they tie."""
    for sb in sbs:
        a, b = th_gpu[sb.index], th_orc[sb.index]
        if abs(a - b) <= 1e-3 * max(abs(b), 1e-30):
            continue
        mag = np.abs(r[sb.offset:sb.offset + sb.size])
        t = float(tau[sb.index])
        scale = float(np.sum(mag ** 2)) + sb.size * t
        if abs(O.sure_value(mag, a, t) - O.sure_value(mag, b, t)) > 1e-6 * scale:
            return False, sb.name
    return True, None


# ------------------------------------------------------------ transforms ---

@pytest.mark.parametrize("ny,nx", [(64, 64), (256, 256), (128, 128), (384, 320), (320, 320),
                                   (48, 80), (8, 8), (1024, 16), (24, 40)])
def test_fft2_matches_oracle(ny, nx):
    rng = np.random.default_rng(ny * 1000 + nx)
    plan = vb.Plan(ny, nx, "haar", 1, max_batch=2)
    x = crand(rng, (2, ny, nx)).astype(np.complex64)
    xd = dev(x)
    out = torch.empty_like(xd)
    back = torch.empty_like(xd)
    vb.vdamp_fft2(plan.handle, 2, xd, out, inverse=False)
    vb.vdamp_fft2(plan.handle, 2, out, back, inverse=True)
    torch.cuda.synchronize()
    x64 = x.astype(np.complex128)
    ref = np.stack([O.fft2u(xi) for xi in x64])
    assert rel(out.cpu().numpy(), ref) < 2e-6
    assert rel(back.cpu().numpy(), x64) < 2e-6
    plan.close()


@pytest.mark.parametrize("ny,nx", [(256, 256), (384, 320), (320, 384), (128, 128)])
@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("cb", [2, 8, 16])
def test_fft2_every_radix_plan_and_column_block(ny, nx, variant, cb):
    """The lengths with compiled radix plans (128, 256, 320, 384): each radix plan on both
    axes (compiled or run-time) and several column blocks, against the oracle's DFT."""
    rng = np.random.default_rng(ny + nx + 10 * variant + cb)
    plan = vb.Plan(ny, nx, "haar", 1, max_batch=2)
    t = plan.tuning()
    plan.set_tuning(dict(t, col_block=cb, radix_y=variant, radix_x=variant))
    x = crand(rng, (2, ny, nx)).astype(np.complex64)
    xd = dev(x)
    out = torch.empty_like(xd)
    back = torch.empty_like(xd)
    vb.vdamp_fft2(plan.handle, 2, xd, out, inverse=False)
    vb.vdamp_fft2(plan.handle, 2, out, back, inverse=True)
    torch.cuda.synchronize()
    x64 = x.astype(np.complex128)
    ref = np.stack([O.fft2u(xi) for xi in x64])
    assert rel(out.cpu().numpy(), ref) < 2e-6
    assert rel(back.cpu().numpy(), x64) < 2e-6
    plan.close()


@pytest.mark.parametrize("wav,ny,nx,s", [("haar", 64, 64, 3), ("db4", 256, 256, 4),
                                         ("db4", 48, 80, 2), ("db4", 384, 320, 4),
                                         ("db4", 320, 320, 5), ("haar", 16, 16, 4),
                                         ("db4", 32, 32, 3), ("db4", 24, 40, 3)])
def test_psi_and_adjoint_match_oracle(wav, ny, nx, s):
    rng = np.random.default_rng(ny + nx + s)
    plan = vb.Plan(ny, nx, wav, s, max_batch=2)
    h, g = O.wavelet_filters(wav)
    x = crand(rng, (2, ny, nx)).astype(np.complex64)
    w = torch.empty((2, ny * nx), dtype=torch.complex64, device="cuda")
    vb.vdamp_psi(plan.handle, 2, dev(x), w)
    c = crand(rng, (2, ny * nx)).astype(np.complex64)
    img = torch.empty((2, ny, nx), dtype=torch.complex64, device="cuda")
    vb.vdamp_psi_h(plan.handle, 2, dev(c), img)
    torch.cuda.synchronize()
    for i in range(2):
        assert rel(w.cpu().numpy()[i], O.dwt2(x[i].astype(np.complex128), h, g, s)) < 2e-6
        assert rel(img.cpu().numpy()[i],
                   O.idwt2(c[i].astype(np.complex128), h, g, s, ny, nx)) < 2e-6
    plan.close()


# ------------------------------------------------- one iteration, forced ---

def _problem_on_device(pr):
    return dev(pr.y[None]), dev(pr.mask[None]), dev(pr.density[None])


@pytest.mark.parametrize("wl,K,sure_parts", [(synth.PLAIN_64_HAAR3, 20, 0),
                                              (synth.PLAIN_64_HAAR3, 20, 1),
                                              (synth.PLAIN_256_DB4_4, 30, 0),
                                              (synth.PLAIN_256_DB4_4, 30, 1),
                                              (synth.PLAIN_256_DB4_4, 30, 8)])
def test_iteration_teacher_forced(wl, K, sure_parts):
    """Each iteration k from the oracle's own r~_k: lines 3-8 against the oracle, with each
    SURE search layout (0: automatic; 1: sort and search in one CTA per subband; 8: large
    subbands split into parts)."""
    pr = synth.make_problem(wl)
    ops = O.make_operators(pr.mask, pr.density, pr.wavelet, pr.levels)
    res = O.vdamp(pr.y, pr.mask, pr.density, pr.sigma, pr.wavelet, pr.levels, K, ops=ops)
    plan = vb.Plan(wl.ny, wl.nx, wl.wavelet, wl.levels)
    if sure_parts:
        plan.set_tuning(dict(plan.tuning(), sure_parts=sure_parts))
    y, m, p = _problem_on_device(pr)
    N, B = wl.ny * wl.nx, plan.B
    y64 = np.where(pr.mask == 1, pr.y.astype(np.complex128), 0.0)
    s2 = float(pr.sigma) ** 2
    r = torch.empty((1, N), dtype=torch.complex64, device="cuda")
    rn = torch.empty_like(r)
    tau = torch.empty((1, B), dtype=torch.float64, device="cuda")
    thr, alpha = torch.empty_like(tau), torch.empty_like(tau)
    for k in range(K):
        rt32 = res.records[k].r_tilde.astype(np.complex64)
        rec = O.iterate(rt32.astype(np.complex128), y64, ops, s2)
        vb.vdamp_iterate(plan.handle, 1, dev(rt32[None]), y, m, p, [pr.sigma], r, tau, thr, alpha,
                         rn)
        torch.cuda.synchronize()
        rg = r.cpu().numpy()[0]
        assert rel(rg, rec.r) < 1e-5, k
        tg = tau.cpu().numpy()[0]
        assert tau_ok(tg, rec.tau), (k, rel(tg, rec.tau))
        ok, band = theta_ok(rec.r, ops.sbs, rec.tau, thr.cpu().numpy()[0], rec.theta)
        assert ok, (k, band)
        if np.allclose(thr.cpu().numpy()[0], rec.theta, rtol=1e-3, atol=0):
            assert np.max(np.abs(alpha.cpu().numpy()[0] - rec.alpha)) < 1e-4, k
            assert rel(rn.cpu().numpy()[0], O.next_r_tilde(rec, ops)) < 1e-4, k
    assert vb.vdamp_device_status(plan.handle)[0] == vb.VDAMP_OK
    plan.close()


# ------------------------------------------------------ the whole solve ---

def _perturbed_oracle_nmse(wl, runs=8, eps=1e-6):
    """Final NMSE of FP64 oracle runs whose state is rounded to complex64 and perturbed by
    eps (relative) before every iteration: the spread the method itself gives an FP32 run."""
    out = []
    for seed in range(runs):
        pr = synth.make_problem(wl)
        ops = O.make_operators(pr.mask, pr.density, pr.wavelet, pr.levels)
        y = np.where(pr.mask == 1, pr.y.astype(np.complex128), 0.0)
        rt = np.zeros(wl.ny * wl.nx, dtype=np.complex128)
        rng = np.random.default_rng(1000 + seed)
        for _ in range(wl.iters):
            rt = rt.astype(np.complex64).astype(np.complex128)
            rt = rt * (1.0 + eps * rng.standard_normal(rt.shape))
            rec = O.iterate(rt, y, ops, float(pr.sigma) ** 2)
            rt = O.next_r_tilde(rec, ops)
        out.append(O.nmse_db(O.final_estimate(rec.w_hat, y, ops), pr.x0))
    return out


@pytest.mark.parametrize("wl,k_strict", [(synth.PLAIN_64_HAAR3, 20), (synth.PLAIN_256_DB4_4, 10)])
def test_solve_free_running(wl, k_strict):
    """Algorithm 1 end to end against the FP64 oracle (see the module docstring for k_strict)."""
    pr = synth.make_problem(wl)
    ops = O.make_operators(pr.mask, pr.density, pr.wavelet, pr.levels)
    res = O.vdamp(pr.y, pr.mask, pr.density, pr.sigma, pr.wavelet, pr.levels, wl.iters,
                  want_x=True, ops=ops)
    plan = vb.Plan(wl.ny, wl.nx, wl.wavelet, wl.levels)
    y, m, p = _problem_on_device(pr)
    out = plan.solve(y, m, p, [pr.sigma], wl.iters, want_iters=True)
    torch.cuda.synchronize()
    assert vb.vdamp_device_status(plan.handle)[0] == vb.VDAMP_OK
    xi = out["x_hat_iters"].cpu().numpy()[:, 0]
    tau = out["tau"].cpu().numpy()[0]
    thr = out["thr"].cpu().numpy()[0]
    parted = None
    for k, rec in enumerate(res.records[:k_strict]):
        assert tau_ok(tau[k], rec.tau), (k, rel(tau[k], rec.tau))   # tau_k precedes line 6
        if not np.allclose(thr[k], rec.theta, rtol=1e-3, atol=0):
            parted = k     # the two runs pick different SURE minima from r_k that differ
            break          # at the FP32 level: from here they follow different trajectories
        assert rel(xi[k], rec.x_hat) < 1e-4, k
    if parted is not None:
        assert wl.iters > k_strict, "the stable workload must not part"
        assert parted >= 5, parted
    xh = out["x_hat"].cpu().numpy()[0]
    assert np.array_equal(xh, xi[-1])
    nm_gpu = O.nmse_db(xh, pr.x0)
    if k_strict >= wl.iters:
        assert rel(xh, res.x_hat) < 1e-4
        assert abs(nm_gpu - O.nmse_db(res.x_hat, pr.x0)) < 0.01
    else:
        ens = np.array(_perturbed_oracle_nmse(wl) + [O.nmse_db(res.x_hat, pr.x0)])
        band = max(4.0 * ens.std(ddof=1), 0.02)
        assert abs(nm_gpu - ens.mean()) <= band, (nm_gpu, ens.mean(), band, ens)
    plan.close()


@pytest.mark.parametrize("ny,nx,wav,s,K", [(384, 320, "db4", 4, 3), (320, 320, "db4", 5, 3),
                                           (48, 80, "db4", 2, 6), (128, 128, "db4", 4, 4)])
def test_solve_other_sizes(ny, nx, wav, s, K):
    """Mixed radix (3, 5), non-square and deeper decompositions, ragged subbands."""
    wl = synth.Workload("t", 77, ny, nx, 12, True, wav, s, 5.0, 5.0, 16, 30.0, 30.0, K, 1)
    pr = synth.make_problem(wl)
    ops = O.make_operators(pr.mask, pr.density, wav, s)
    res = O.vdamp(pr.y, pr.mask, pr.density, pr.sigma, wav, s, K, want_x=True, ops=ops)
    plan = vb.Plan(ny, nx, wav, s)
    y, m, p = _problem_on_device(pr)
    out = plan.solve(y, m, p, [pr.sigma], K, want_iters=True)
    torch.cuda.synchronize()
    xi = out["x_hat_iters"].cpu().numpy()[:, 0]
    tau = out["tau"].cpu().numpy()[0]
    thr = out["thr"].cpu().numpy()[0]
    for k, rec in enumerate(res.records):
        assert rel(xi[k], rec.x_hat) < 1e-4, k
        assert tau_ok(tau[k], rec.tau), (k, rel(tau[k], rec.tau))
        assert theta_ok(rec.r, ops.sbs, rec.tau, thr[k], rec.theta)[0], k
    plan.close()


def test_return_line_consistency():
    """m F x_hat = y (Algorithm 1 return line, exact consistency, Sec. 2)."""
    wl = synth.PLAIN_64_HAAR3
    pr = synth.make_problem(wl)
    plan = vb.Plan(wl.ny, wl.nx, wl.wavelet, wl.levels)
    y, m, p = _problem_on_device(pr)
    out = plan.solve(y, m, p, [pr.sigma], 5)
    k = O.fft2u(out["x_hat"].cpu().numpy()[0].astype(np.complex128))
    sel = pr.mask == 1
    assert np.max(np.abs(k[sel] - pr.y[sel])) < 1e-5 * np.max(np.abs(pr.y))
    plan.close()


def test_resume_is_bit_identical():
    wl = synth.PLAIN_64_HAAR3
    pr = synth.make_problem(wl)
    plan = vb.Plan(wl.ny, wl.nx, wl.wavelet, wl.levels)
    y, m, p = _problem_on_device(pr)
    full = plan.solve(y, m, p, [pr.sigma], 12)
    a = plan.solve(y, m, p, [pr.sigma], 7, want_state=True)
    b = plan.solve(y, m, p, [pr.sigma], 5, r_tilde0=a["r_tilde"])
    torch.cuda.synchronize()
    assert torch.equal(full["tau"][:, 7:], b["tau"])
    assert torch.equal(full["thr"][:, 7:], b["thr"])
    assert torch.equal(full["x_hat"], b["x_hat"])
    plan.close()


def test_graph_and_direct_launches_agree():
    wl = synth.PLAIN_64_HAAR3
    pr = synth.make_problem(wl)
    plan = vb.Plan(wl.ny, wl.nx, wl.wavelet, wl.levels)
    y, m, p = _problem_on_device(pr)
    g = plan.solve(y, m, p, [pr.sigma], 6)
    vb.vdamp_plan_set_option(plan.handle, vb.VDAMP_OPT_GRAPH, 0)
    d = plan.solve(y, m, p, [pr.sigma], 6)
    torch.cuda.synchronize()
    assert torch.equal(g["x_hat"], d["x_hat"]) and torch.equal(g["tau"], d["tau"])
    plan.close()


@pytest.mark.parametrize("wl", [synth.PLAIN_64_HAAR3, synth.PLAIN_256_DB4_4], ids=lambda w: w.name[:16])
def test_overlapped_threshold_search_is_bit_identical(wl):
    """The finest subbands' threshold search on the plan's side stream (the split
    path of a lone slice) gives the same bits as the one-stream order, in a
    graph and in direct launches, with the per-iteration outputs too."""
    # (the pruned path of many slices: test_gpu_batched)
    pr = synth.make_problem(wl)
    plan = vb.Plan(wl.ny, wl.nx, wl.wavelet, wl.levels)
    y, m, p = _problem_on_device(pr)
    outs = []
    for overlap, graph in ((1, 1), (0, 1), (1, 0)):
        vb.vdamp_plan_set_option(plan.handle, vb.VDAMP_OPT_OVERLAP, overlap)
        vb.vdamp_plan_set_option(plan.handle, vb.VDAMP_OPT_GRAPH, graph)
        outs.append(plan.solve(y, m, p, [pr.sigma], 8, want_iters=True))
    torch.cuda.synchronize()
    st, _ = vb.vdamp_device_status(plan.handle)
    assert st == vb.VDAMP_OK
    for o in outs[1:]:
        for key in ("x_hat", "tau", "thr", "alpha", "x_hat_iters"):
            assert torch.equal(outs[0][key], o[key]), key
    plan.close()


def test_batch_matches_single_slices():
    wl = synth.PLAIN_64_HAAR3
    probs = [synth.make_problem(wl, i) for i in range(3)]
    plan = vb.Plan(wl.ny, wl.nx, wl.wavelet, wl.levels, max_batch=3)
    y = dev(np.stack([q.y for q in probs]))
    m = dev(np.stack([q.mask for q in probs]))
    p = dev(np.stack([q.density for q in probs]))
    sig = [q.sigma for q in probs]
    bat = plan.solve(y, m, p, sig, 8)
    for i in range(3):
        one = plan.solve(y[i:i + 1].contiguous(), m[i:i + 1].contiguous(),
                         p[i:i + 1].contiguous(), [sig[i]], 8)
        torch.cuda.synchronize()
        assert torch.equal(one["x_hat"][0], bat["x_hat"][i])
        assert torch.equal(one["tau"][0], bat["tau"][i])
    plan.close()


def test_host_buffer_entry_point_matches_device():
    wl = synth.PLAIN_64_HAAR3
    pr = synth.make_problem(wl)
    plan = vb.Plan(wl.ny, wl.nx, wl.wavelet, wl.levels)
    y, m, p = _problem_on_device(pr)
    K = 6
    d = plan.solve(y, m, p, [pr.sigma], K)
    torch.cuda.synchronize()
    x = np.zeros((1, wl.ny, wl.nx), np.complex64)
    tau = np.zeros((1, K, plan.B))
    thr, alpha = np.zeros_like(tau), np.zeros_like(tau)
    vb.vdamp_solve_host(plan.handle, 1, np.ascontiguousarray(pr.y[None]),
                        np.ascontiguousarray(pr.mask[None]), np.ascontiguousarray(pr.density[None]),
                        [pr.sigma], K, None, x, tau, thr, alpha, k0=0)
    assert np.array_equal(x, d["x_hat"].cpu().numpy())
    assert np.array_equal(tau, d["tau"].cpu().numpy())
    plan.close()


# ---------------------------------------------------------- edge cases ---

def test_full_sampling_noiseless_is_exact():
    """p = 1, sigma = 0: tau = 0, no thresholding, x_hat = x0 (degenerate case)."""
    wl = synth.PLAIN_64_HAAR3
    pr = synth.make_problem(wl)
    ones = np.ones_like(pr.mask)
    y = O.fft2u(pr.x0).astype(np.complex64)
    plan = vb.Plan(wl.ny, wl.nx, wl.wavelet, wl.levels)
    out = plan.solve(dev(y[None]), dev(ones[None]), dev(np.ones((1, 64, 64), np.float32)), [0.0], 3)
    torch.cuda.synchronize()
    assert torch.all(out["tau"] == 0) and torch.all(out["thr"] == 0)
    assert torch.all(out["alpha"] == 0)
    assert rel(out["x_hat"].cpu().numpy()[0], pr.x0) < 1e-6
    plan.close()


def test_empty_mask_gives_zero():
    wl = synth.PLAIN_64_HAAR3
    pr = synth.make_problem(wl)
    plan = vb.Plan(wl.ny, wl.nx, wl.wavelet, wl.levels)
    zero = np.zeros((1, 64, 64), np.uint8)
    out = plan.solve(dev(pr.y[None]), dev(zero), dev(pr.density[None]), [pr.sigma], 2)
    torch.cuda.synchronize()
    assert torch.all(out["x_hat"] == 0) and torch.all(out["tau"] == 0)
    plan.close()


def test_non_finite_input_is_reported():
    wl = synth.PLAIN_64_HAAR3
    pr = synth.make_problem(wl)
    y = pr.y.copy()
    idx = np.argwhere(pr.mask == 1)[5]
    y[tuple(idx)] = np.nan
    plan = vb.Plan(wl.ny, wl.nx, wl.wavelet, wl.levels)
    plan.solve(dev(y[None]), dev(pr.mask[None]), dev(pr.density[None]), [pr.sigma], 3)
    st, it = vb.vdamp_device_status(plan.handle)
    assert st == vb.VDAMP_ENUMERIC and it == 0
    plan.close()


def test_resume_reports_iterations_from_k0():
    """A resumed solve (r_tilde0 and k0 = 4) that meets a non-finite tau reports iteration
    k0 + k; a cold start with k0 != 0, or more iterations than the plan's max_iters, is
    refused before anything is launched."""
    wl = synth.PLAIN_64_HAAR3
    pr = synth.make_problem(wl)
    y = pr.y.copy()
    y[tuple(np.argwhere(pr.mask == 1)[5])] = np.nan
    plan = vb.Plan(wl.ny, wl.nx, wl.wavelet, wl.levels, max_iters=8)
    rt = torch.zeros((1, wl.ny * wl.nx), dtype=torch.complex64, device="cuda")
    plan.solve(dev(y[None]), dev(pr.mask[None]), dev(pr.density[None]), [pr.sigma], 3,
               r_tilde0=rt, k0=4)
    st, it = vb.vdamp_device_status(plan.handle)
    assert st == vb.VDAMP_ENUMERIC and it == 4
    yd, m, p = _problem_on_device(pr)
    with pytest.raises(vb.VdampError) as e:
        plan.solve(yd, m, p, [pr.sigma], 3, k0=2)
    assert e.value.status == vb.VDAMP_EINVAL
    with pytest.raises(vb.VdampError) as e:
        plan.solve(yd, m, p, [pr.sigma], 9)
    assert e.value.status == vb.VDAMP_EINVAL and "max_iters" in vb.last_error()
    plan.close()


@pytest.mark.parametrize("mag", [1.2, 0.0])
def test_one_cta_threshold_search_on_a_degenerate_subband(mag):
    """The one-CTA-per-subband threshold search (tuning entry 7 = 1) on a subband whose
    1024 magnitudes are all equal to mag sqrt(tau) (mag 1.2: one bucket far above the
    table's limit and holding the minimiser theta = max a, so the subband must take the
    full sort, and the running count shows it did), or zero (mag 0: magnitudes at the FP32
    rounding level, far below the noise: the flat top, pruned search); every other subband
    from the oracle's state.  r~ is chosen and y = m F Psi^H r~, so that z ~ 0 and r_k = r~
    up to FP32 rounding.  Teacher-forced against the oracle, on two calls in a row (the
    fallback list must empty itself)."""
    wl = synth.PLAIN_64_HAAR3
    pr = synth.make_problem(wl)
    ops = O.make_operators(pr.mask, pr.density, pr.wavelet, pr.levels)
    y0 = np.where(pr.mask == 1, pr.y.astype(np.complex128), 0.0)
    rec0 = O.iterate(np.zeros(wl.ny * wl.nx, np.complex128), y0, ops, float(pr.sigma) ** 2)
    rt = O.next_r_tilde(rec0, ops).astype(np.complex64)
    sb = ops.sbs[-1]   # D1, 32 x 32
    tau_d1 = float(O.tau_estimate(np.zeros((wl.ny, wl.nx)), ops, float(pr.sigma) ** 2)[sb.index])
    ph = np.exp(2j * np.pi * np.random.default_rng(3).random(sb.size))
    rt[sb.offset:sb.offset + sb.size] = (mag * math.sqrt(tau_d1) * ph).astype(np.complex64)
    y = np.where(pr.mask == 1, ops.phi(ops.psi_h(rt.astype(np.complex128))), 0.0)
    y32 = y.astype(np.complex64)
    rec = O.iterate(rt.astype(np.complex128), y32.astype(np.complex128), ops,
                    float(pr.sigma) ** 2)
    plan = vb.Plan(wl.ny, wl.nx, wl.wavelet, wl.levels)
    plan.set_tuning(vb.vdamp_plan_get_tuning(plan.handle)[:7] + [1])
    N, B = wl.ny * wl.nx, plan.B
    r = torch.empty((1, N), dtype=torch.complex64, device="cuda")
    rn = torch.empty_like(r)
    tau = torch.empty((1, B), dtype=torch.float64, device="cuda")
    thr, alpha = torch.empty_like(tau), torch.empty_like(tau)
    before = vb.vdamp_sure_fallback_count(plan.handle)
    for call in range(2):
        vb.vdamp_iterate(plan.handle, 1, dev(rt[None]), dev(y32[None]), dev(pr.mask[None]),
                         dev(pr.density[None]), [pr.sigma], r, tau, thr, alpha, rn)
        torch.cuda.synchronize()
        assert vb.vdamp_device_status(plan.handle)[0] == vb.VDAMP_OK
        assert rel(r.cpu().numpy()[0], rec.r) < 1e-5, call
        assert tau_ok(tau.cpu().numpy()[0], rec.tau), call
        ok, band = theta_ok(rec.r, ops.sbs, rec.tau, thr.cpu().numpy()[0], rec.theta)
        assert ok, (call, band)
    after = vb.vdamp_sure_fallback_count(plan.handle)
    assert after - before == (2 if mag > 0 else 0), (before, after)
    plan.close()


def test_invalid_solve_arguments_launch_nothing():
    wl = synth.PLAIN_64_HAAR3
    pr = synth.make_problem(wl)
    plan = vb.Plan(wl.ny, wl.nx, wl.wavelet, wl.levels)
    y, m, p = _problem_on_device(pr)
    with pytest.raises(vb.VdampError):
        plan.solve(y, m, p, [-1.0], 3)
    with pytest.raises(vb.VdampError):
        plan.solve(y, m, p, [float("nan")], 3)
    with pytest.raises(vb.VdampError):
        plan.solve(y, m, p, [pr.sigma], 0)
    plan.close()


def test_largest_supported_slice():
    """256 x 512: the largest finest subband (32768) the SURE kernel holds."""
    ny, nx, s, K = 256, 512, 4, 2
    wl = synth.Workload("big", 78, ny, nx, 20, True, "db4", s, 5.0, 5.0, 24, 30.0, 30.0, K, 1)
    pr = synth.make_problem(wl)
    ops = O.make_operators(pr.mask, pr.density, "db4", s)
    res = O.vdamp(pr.y, pr.mask, pr.density, pr.sigma, "db4", s, K, ops=ops)
    plan = vb.Plan(ny, nx, "db4", s)
    y, m, p = _problem_on_device(pr)
    out = plan.solve(y, m, p, [pr.sigma], K)
    torch.cuda.synchronize()
    assert rel(out["x_hat"].cpu().numpy()[0], res.x_hat) < 1e-4
    plan.close()


@pytest.mark.parametrize("wl", [synth.PLAIN_64_HAAR3, synth.PLAIN_256_DB4_4])
def test_persistent_cluster_solve_matches_oracle(wl):
    """The persistent cluster solve (VDAMP_OPT_FUSED = 1: the whole solve as one launch in
    which a thread-block cluster iterates the slice) against the FP64 oracle at every
    iteration (x_hat_k and tau_k to the solve tolerances, thresholds to 1e-3 or a certified
    tie), and against the one-kernel-per-step solve; the launch count shows which ran."""
    pr = synth.make_problem(wl)
    K = wl.iters if wl is synth.PLAIN_64_HAAR3 else 5
    ops = O.make_operators(pr.mask, pr.density, pr.wavelet, pr.levels)
    res = O.vdamp(pr.y, pr.mask, pr.density, pr.sigma, pr.wavelet, pr.levels, K, want_x=True,
                  ops=ops)
    plan = vb.Plan(wl.ny, wl.nx, wl.wavelet, wl.levels)
    y, m, p = _problem_on_device(pr)
    vb.vdamp_plan_set_option(plan.handle, vb.VDAMP_OPT_FUSED, 1)
    fused = plan.solve(y, m, p, [pr.sigma], K, want_iters=True)
    torch.cuda.synchronize()
    n_fused = vb.vdamp_last_launch_count(plan.handle)
    assert vb.vdamp_device_status(plan.handle)[0] == vb.VDAMP_OK
    vb.vdamp_plan_set_option(plan.handle, vb.VDAMP_OPT_FUSED, 0)
    step = plan.solve(y, m, p, [pr.sigma], K, want_iters=True)
    torch.cuda.synchronize()
    n_step = vb.vdamp_last_launch_count(plan.handle)
    assert n_fused == 2, n_fused            # the sigma upload and the one persistent launch
    assert n_step > 10 * K, n_step          # one kernel per step of every iteration
    xf = fused["x_hat_iters"].cpu().numpy()[:, 0]
    xs = step["x_hat_iters"].cpu().numpy()[:, 0]
    tf = fused["tau"].cpu().numpy()[0]
    thf = fused["thr"].cpu().numpy()[0]
    for k, rec in enumerate(res.records):
        assert rel(xf[k], rec.x_hat) < 1e-4, (k, rel(xf[k], rec.x_hat))
        assert tau_ok(tf[k], rec.tau), (k, rel(tf[k], rec.tau))
        assert theta_ok(rec.r, ops.sbs, rec.tau, thf[k], rec.theta)[0], k
        assert rel(xf[k], xs[k]) < 1e-5, k
        assert rel(tf[k], step["tau"].cpu().numpy()[0, k]) < 1e-5, k
    plan.close()


def test_paper_size_512_haar4():
    """The paper's image size and wavelet (512x512, Haar, 4 levels; Sec. 3): finest subbands
    of 65536 coefficients, more than one CTA holds, so their SURE search is split into parts
    whose magnitudes stream from global memory.  Teacher-forced steps against the oracle, a
    batch of three equal to single-slice solves bit for bit, and an empty mask (all-zero
    subbands: the exact zeros take no bucket) gives zero."""
    wl = synth.Workload("t", 78, 512, 512, 20, True, "haar", 4, 5.0, 5.0, 24, 30.0, 30.0, 3, 1)
    prs = [synth.make_problem(wl, i) for i in range(3)]
    pr = prs[0]
    ops = O.make_operators(pr.mask, pr.density, pr.wavelet, pr.levels)
    res = O.vdamp(pr.y, pr.mask, pr.density, pr.sigma, pr.wavelet, pr.levels, 3, ops=ops)
    plan = vb.Plan(512, 512, "haar", 4, max_batch=3)
    N, B = 512 * 512, plan.B
    y, m, p = _problem_on_device(pr)
    y64 = np.where(pr.mask == 1, pr.y.astype(np.complex128), 0.0)
    r = torch.empty((1, N), dtype=torch.complex64, device="cuda")
    rn = torch.empty_like(r)
    tau = torch.empty((1, B), dtype=torch.float64, device="cuda")
    thr, alpha = torch.empty_like(tau), torch.empty_like(tau)
    for k in (0, 2):
        rt32 = res.records[k].r_tilde.astype(np.complex64)
        rec = O.iterate(rt32.astype(np.complex128), y64, ops, float(pr.sigma) ** 2)
        vb.vdamp_iterate(plan.handle, 1, dev(rt32[None]), y, m, p, [pr.sigma], r, tau, thr, alpha,
                         rn)
        torch.cuda.synchronize()
        assert rel(r.cpu().numpy()[0], rec.r) < 1e-5, k
        tg = tau.cpu().numpy()[0]
        assert tau_ok(tg, rec.tau), (k, rel(tg, rec.tau))
        ok, band = theta_ok(rec.r, ops.sbs, rec.tau, thr.cpu().numpy()[0], rec.theta)
        assert ok, (k, band)
        if np.allclose(thr.cpu().numpy()[0], rec.theta, rtol=1e-3, atol=0):
            assert np.max(np.abs(alpha.cpu().numpy()[0] - rec.alpha)) < 1e-4, k
            assert rel(rn.cpu().numpy()[0], O.next_r_tilde(rec, ops)) < 1e-4, k
    assert vb.vdamp_device_status(plan.handle)[0] == vb.VDAMP_OK

    yb = dev(np.stack([q.y for q in prs]))
    mb = dev(np.stack([q.mask for q in prs]))
    pb = dev(np.stack([q.density for q in prs]))
    sig = [q.sigma for q in prs]
    bat = plan.solve(yb, mb, pb, sig, 3)
    for i in range(3):
        one = plan.solve(yb[i:i + 1].contiguous(), mb[i:i + 1].contiguous(),
                         pb[i:i + 1].contiguous(), [sig[i]], 3)
        torch.cuda.synchronize()
        assert torch.equal(one["x_hat"][0], bat["x_hat"][i]), i
        assert torch.equal(one["thr"][0], bat["thr"][i]), i
    assert vb.vdamp_device_status(plan.handle)[0] == vb.VDAMP_OK

    zero = torch.zeros((1, 512, 512), dtype=torch.uint8, device="cuda")
    out = plan.solve(y, zero, p, [pr.sigma], 2)
    torch.cuda.synchronize()
    assert torch.all(out["x_hat"] == 0) and torch.all(out["tau"] == 0)
    assert vb.vdamp_device_status(plan.handle)[0] == vb.VDAMP_OK
    plan.close()
