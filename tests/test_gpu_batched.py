"""Mixed-size batched solve, launch-shape tuning and the autotuner (CUDA path).

* vdamp_solve_groups runs several plans' solves as one graph launch; its
  results must equal the per-plan vdamp_solve results bit for bit (same
  kernels, same arguments, separate workspaces).
* Sampled slices of a mixed batch (sizes of the 96-slice mixed workload:
  128x128, 256x256, 384x320, db4 s=4, per-slice R and SNR) are checked against
  the FP64 oracle with the solve tolerances (x_hat and the tau vector within
  1e-4 relative L2, thresholds within 1e-3 or a certified SURE tie).
* Every tuning computes the same method: each launch shape is checked against
  the oracle, and unsupported shapes are refused.
* vdamp_solve_batched (slices in separate buffers, described one by one)
  groups slices of equal iteration count and start, and gives per slice the
  same results, bit for bit, as vdamp_solve on the same grouping.
"""
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


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _stack(prs, key):
    return torch.from_numpy(np.ascontiguousarray(np.stack([getattr(p, key) for p in prs]))).cuda()


def _groups(counts):
    out = []
    for wl, n in zip(synth.mixed_batch_workloads(), counts):
        prs = [synth.make_problem(wl, i) for i in range(n)]
        plan = vb.Plan(wl.ny, wl.nx, wl.wavelet, wl.levels, max_batch=n)
        out.append((wl, prs, plan))
    return out


def test_groups_equal_separate_solves():
    iters = 6
    groups = _groups((3, 2, 2))
    args = [(plan, _stack(prs, "y"), _stack(prs, "mask"), _stack(prs, "density"),
             [p.sigma for p in prs]) for _, prs, plan in groups]
    outs = vb.solve_groups(args, iters)
    again = vb.solve_groups(args, iters)   # replay of the cached graph
    torch.cuda.synchronize()
    for (wl, prs, plan), (_, y, m, d, sig), o, o2 in zip(groups, args, outs, again):
        ref = plan.solve(y, m, d, sig, iters)
        torch.cuda.synchronize()
        assert vb.vdamp_device_status(plan.handle)[0] == vb.VDAMP_OK
        for k in ("x_hat", "tau", "thr", "alpha"):
            assert torch.equal(o[k], ref[k]), (wl.name, k)
            assert torch.equal(o2[k], ref[k]), (wl.name, k)
        plan.close()


def _tie(r, sbs, tau, th_gpu, th_orc):
    """Thresholds agree within 1e-3, or the oracle's SURE at the two differs by at most
    1e-6 of the scale of its terms (a near-tie that FP32-level changes of r_k can flip)."""
    for sb in sbs:
        a, b = th_gpu[sb.index], th_orc[sb.index]
        if abs(a - b) <= 1e-3 * abs(b):
            continue
        mag = np.abs(r[sb.offset:sb.offset + sb.size])
        t = float(tau[sb.index])
        scale = float(np.sum(mag ** 2)) + sb.size * t
        if abs(O.sure_value(mag, a, t) - O.sure_value(mag, b, t)) > 1e-6 * scale:
            return False
    return True


def _forced_step_ok(plan, pr, ops, r_tilde, where):
    """One iteration (lines 3-8) of one slice started from the oracle's own r~_k: r, tau,
    the thresholds (or a certified tie) and, where the thresholds agree, alpha and r~_{k+1}
    against the oracle's step from the same r~_k."""
    N, B = pr.y.size, plan.B
    y64 = np.where(pr.mask == 1, pr.y.astype(np.complex128), 0.0)
    rt32 = r_tilde.astype(np.complex64)
    rec = O.iterate(rt32.astype(np.complex128), y64, ops, float(pr.sigma) ** 2)
    one = lambda a: torch.from_numpy(np.ascontiguousarray(a[None])).cuda()
    r = torch.empty((1, N), dtype=torch.complex64, device="cuda")
    rn = torch.empty_like(r)
    tau = torch.empty((1, B), dtype=torch.float64, device="cuda")
    thr, alpha = torch.empty_like(tau), torch.empty_like(tau)
    vb.vdamp_iterate(plan.handle, 1, one(rt32.reshape(-1)), one(pr.y), one(pr.mask),
                     one(pr.density), [pr.sigma], r, tau, thr, alpha, rn)
    torch.cuda.synchronize()
    assert rel(r.cpu().numpy()[0], rec.r) < 1e-5, where
    tg = tau.cpu().numpy()[0]
    assert rel(tg, rec.tau) < 1e-4 and np.max(np.abs(tg - rec.tau) / rec.tau) < 1e-3, where
    th = thr.cpu().numpy()[0]
    assert _tie(rec.r, ops.sbs, rec.tau, th, rec.theta), where
    if np.allclose(th, rec.theta, rtol=1e-3, atol=0):
        assert np.max(np.abs(alpha.cpu().numpy()[0] - rec.alpha)) < 1e-4, where
        assert rel(rn.cpu().numpy()[0], O.next_r_tilde(rec, ops)) < 1e-4, where
    return True


def test_groups_match_oracle_on_sampled_slices():
    iters = 5
    groups = _groups((2, 2, 2))
    args = [(plan, _stack(prs, "y"), _stack(prs, "mask"), _stack(prs, "density"),
             [p.sigma for p in prs]) for _, prs, plan in groups]
    outs = vb.solve_groups(args, iters)
    torch.cuda.synchronize()
    for (wl, prs, plan), o in zip(groups, outs):
        i = 1   # second slice of each group: its own R and SNR
        pr = prs[i]
        ops = O.make_operators(pr.mask, pr.density, pr.wavelet, pr.levels)
        res = O.vdamp(pr.y, pr.mask, pr.density, pr.sigma, pr.wavelet, pr.levels, iters, ops=ops)
        tau = o["tau"].cpu().numpy()[i]
        thr = o["thr"].cpu().numpy()[i]
        parted = None
        for k, rec in enumerate(res.records):
            assert rel(tau[k], rec.tau) < 1e-4, (wl.name, k)
            if not np.allclose(thr[k], rec.theta, rtol=1e-3, atol=0):
                # The free-running states have drifted apart at the FP32 level (the
                # iteration amplifies perturbations) and met a SURE near-tie, where a
                # relative change of 1e-6 in the magnitudes can flip the minimiser.  From
                # here the runs follow different, equally valid trajectories; the step
                # itself is held to the tolerances from the oracle's own r~_k.
                assert _forced_step_ok(plan, pr, ops, rec.r_tilde, (wl.name, k))
                parted = k
                break
        xg = o["x_hat"].cpu().numpy()[i]
        if parted is None:
            assert rel(xg, res.x_hat) < 1e-4, wl.name
        else:
            assert abs(O.nmse_db(xg, pr.x0) - O.nmse_db(res.x_hat, pr.x0)) < 0.1, wl.name
        plan.close()


def test_groups_reject_bad_arguments():
    (wl, prs, plan), = _groups((1,))
    y, m, d = _stack(prs, "y"), _stack(prs, "mask"), _stack(prs, "density")
    x = torch.empty((1, wl.ny, wl.nx), dtype=torch.complex64, device="cuda")
    t = torch.empty((1, 3, plan.B), dtype=torch.float64, device="cuda")
    g = {"plan": plan.handle, "batch": 1, "y": y, "mask": m, "density": d, "sigma": [prs[0].sigma],
         "iters": 3, "x_hat": x, "tau": t, "thr": t.clone(), "alpha": t.clone()}
    with pytest.raises(vb.VdampError) as e:
        vb.vdamp_solve_groups([g, dict(g)])   # the same plan twice would share a workspace
    assert e.value.status == vb.VDAMP_EINVAL
    with pytest.raises(vb.VdampError):
        vb.vdamp_solve_groups([dict(g, batch=2, sigma=[prs[0].sigma] * 2)])  # max_batch is 1
    with pytest.raises(vb.VdampError):
        vb.vdamp_solve_groups([dict(g, iters=0)])
    plan.close()


TUNINGS = [[2, 1, 16, 16, 0, 0, 1, 0], [4, 2, 32, 32, 1, 1, 0, 1], [8, 4, 64, 16, 2, 2, 1, 2],
           [16, 8, 32, 32, 0, 1, 0, 4], [2, 2, 64, 32, 1, 2, 1, 8], [4, 1, 16, 16, 0, 0, 2, 1],
           [8, 2, 32, 32, 2, 0, 2, 0]]


@pytest.mark.parametrize("ny,nx,wav,s", [(64, 64, "haar", 3), (48, 80, "db4", 2),
                                         (96, 160, "db4", 3)])
def test_every_tuning_matches_oracle(ny, nx, wav, s):
    wl = synth.Workload("t", 91, ny, nx, 10, True, wav, s, 4.0, 4.0, 8, 30.0, 30.0, 4, 1)
    pr = synth.make_problem(wl)
    res = O.vdamp(pr.y, pr.mask, pr.density, pr.sigma, wav, s, wl.iters)
    plan = vb.Plan(ny, nx, wav, s)
    y, m, d = (torch.from_numpy(np.ascontiguousarray(a[None])).cuda()
               for a in (pr.y, pr.mask, pr.density))
    tried = 0
    for t in TUNINGS:
        if nx % t[0]:
            with pytest.raises(vb.VdampError):
                vb.vdamp_plan_set_tuning(plan.handle, t)
            continue
        vb.vdamp_plan_set_tuning(plan.handle, t)
        assert vb.vdamp_plan_get_tuning(plan.handle) == t
        o = plan.solve(y, m, d, [pr.sigma], wl.iters)
        torch.cuda.synchronize()
        assert rel(o["x_hat"].cpu().numpy()[0], res.x_hat) < 1e-4, t
        for k, rec in enumerate(res.records):
            assert rel(o["tau"].cpu().numpy()[0, k], rec.tau) < 1e-4, (t, k)
        tried += 1
    assert tried >= 3
    for bad in ([3, 1, 16, 16, 0, 0, 0, 0], [8, 0, 16, 16, 0, 0, 0, 0], [8, 1, 24, 16, 0, 0, 0, 0],
                [8, 1, 16, 64, 0, 0, 0, 0], [8, 1, 16, 16, 3, 0, 0, 0], [8, 1, 16, 16, 0, 0, 3, 0],
                [8, 1, 16, 16, 0, 0, 0, 3], [8, 1, 16, 16, 0, 0, 0, 16]):
        with pytest.raises(vb.VdampError) as e:
            vb.vdamp_plan_set_tuning(plan.handle, bad)
        assert e.value.status == vb.VDAMP_EINVAL
    plan.close()


def test_autotune_picks_a_valid_tuning_that_still_matches():
    wl = synth.PLAIN_64_HAAR3
    pr = synth.make_problem(wl)
    plan = vb.Plan(wl.ny, wl.nx, wl.wavelet, wl.levels, max_batch=4)
    chosen = vb.vdamp_plan_autotune(plan.handle, 4, trials=2)
    torch.cuda.synchronize()
    assert chosen == vb.vdamp_plan_get_tuning(plan.handle)
    assert chosen[0] in (2, 4, 8, 16) and chosen[2] in (16, 32, 64) and chosen[3] in (16, 32)
    assert chosen[6] in (0, 1, 2) and chosen[7] in (0, 1, 2, 4)
    iters = 6
    res = O.vdamp(pr.y, pr.mask, pr.density, pr.sigma, pr.wavelet, pr.levels, iters)
    y, m, d = (torch.from_numpy(np.ascontiguousarray(a[None])).cuda()
               for a in (pr.y, pr.mask, pr.density))
    o = plan.solve(y, m, d, [pr.sigma], iters)
    torch.cuda.synchronize()
    assert rel(o["x_hat"].cpu().numpy()[0], res.x_hat) < 1e-4
    plan.close()


def test_full_size_batched_workload_on_sampled_slices():
    """256 slices of 320x320, db4 s=5, R=6 (the batched workload at full size) in the
    autotuned launch shape: with 16 subbands x 256 slices every subband's SURE runs as one
    CTA that sorts and searches (not the split parts of a few slices).  16 distinct problems
    are tiled over the batch: replicas must give bit-identical results (no cross-slice
    effects), and three of them are checked against the FP64 oracle, teacher-forced at
    iterations 0 and 4 (lines 3-8) and free-running for 3 iterations."""
    wl = synth.BATCH_320_DB4_5
    nb, distinct, K = 256, 16, 5
    prs = [synth.make_problem(wl, i) for i in range(distinct)]
    pick = [i % distinct for i in range(nb)]
    sampled = (0, 7, 13)
    plan = vb.Plan(wl.ny, wl.nx, wl.wavelet, wl.levels, max_batch=nb)
    assert plan.autotune(nb, trials=1)["sure_parts"] in (0, 1)   # one SURE CTA per subband
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(np.stack(a))).cuda()
    y = dev([prs[i].y for i in pick])
    m = dev([prs[i].mask for i in pick])
    d = dev([prs[i].density for i in pick])
    sig = [prs[i].sigma for i in pick]
    ora = {}
    for j in sampled:
        pr = prs[j]
        ops = O.make_operators(pr.mask, pr.density, pr.wavelet, pr.levels)
        ora[j] = (ops, O.vdamp(pr.y, pr.mask, pr.density, pr.sigma, pr.wavelet, pr.levels, K,
                               want_x=True, ops=ops))
    N, B = wl.ny * wl.nx, plan.B

    def same_as_first(t):
        t = t.reshape(nb, -1)
        return all(torch.equal(t[i], t[pick[i]]) for i in range(distinct, nb))

    # teacher-forced: the sampled slices start from the oracle's r~_k, the others from 0
    r = torch.empty((nb, N), dtype=torch.complex64, device="cuda")
    rn = torch.empty_like(r)
    tau = torch.empty((nb, B), dtype=torch.float64, device="cuda")
    thr, alpha = torch.empty_like(tau), torch.empty_like(tau)
    for k in (0, 4):
        rt = np.zeros((nb, N), dtype=np.complex64)
        for i in range(nb):
            if pick[i] in ora:
                rt[i] = ora[pick[i]][1].records[k].r_tilde.astype(np.complex64)
        vb.vdamp_iterate(plan.handle, nb, dev(list(rt)), y, m, d, sig, r, tau, thr, alpha, rn)
        torch.cuda.synchronize()
        for t in (r, tau, thr, alpha, rn):
            assert same_as_first(t), k
        for j in sampled:
            ops, res = ora[j]
            pr = prs[j]
            y64 = np.where(pr.mask == 1, pr.y.astype(np.complex128), 0.0)
            rt64 = res.records[k].r_tilde.astype(np.complex64).astype(np.complex128)
            rec = O.iterate(rt64, y64, ops, float(pr.sigma) ** 2)
            assert rel(r.cpu().numpy()[j], rec.r) < 1e-5, (j, k)
            tg = tau.cpu().numpy()[j]
            assert rel(tg, rec.tau) < 1e-4 and np.max(np.abs(tg - rec.tau) / rec.tau) < 1e-3
            th = thr.cpu().numpy()[j]
            assert _tie(rec.r, ops.sbs, rec.tau, th, rec.theta), (j, k)
            if np.allclose(th, rec.theta, rtol=1e-3, atol=0):
                assert np.max(np.abs(alpha.cpu().numpy()[j] - rec.alpha)) < 1e-4, (j, k)
                assert rel(rn.cpu().numpy()[j], O.next_r_tilde(rec, ops)) < 1e-4, (j, k)

    # free-running, 3 iterations
    o = plan.solve(y, m, d, sig, 3, want_iters=True)
    torch.cuda.synchronize()
    assert vb.vdamp_device_status(plan.handle)[0] == vb.VDAMP_OK
    for key in ("x_hat", "tau", "thr", "alpha"):
        assert same_as_first(o[key]), key
    xi = o["x_hat_iters"].cpu().numpy()
    for j in sampled:
        ops, res = ora[j]
        for k in range(3):
            rec = res.records[k]
            assert rel(o["tau"].cpu().numpy()[j, k], rec.tau) < 1e-4, (j, k)
            if not np.allclose(o["thr"].cpu().numpy()[j, k], rec.theta, rtol=1e-3, atol=0):
                # a SURE near-tie met by drifted states (see the sampled-slices test)
                assert _forced_step_ok(plan, prs[j], ops, rec.r_tilde, (j, k))
                break
            assert rel(xi[k, j], rec.x_hat) < 1e-4, (j, k)
    plan.close()


def test_solve_batched_descriptors_equal_solve():
    """Five slices in separate buffers: two groups of cold starts with different iteration
    counts (3 and 5 iterations) and one resumed slice (r_tilde0 after 3 iterations, k0 = 3);
    each result equals vdamp_solve on the same slices bit for bit, on two calls in a row."""
    wl = synth.PLAIN_64_HAAR3
    prs = [synth.make_problem(wl, i) for i in range(5)]
    plan = vb.Plan(wl.ny, wl.nx, wl.wavelet, wl.levels, max_batch=4)
    B, N = plan.B, wl.ny * wl.nx
    one = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ys = [one(q.y) for q in prs]
    ms = [one(q.mask) for q in prs]
    ps = [one(q.density) for q in prs]
    iters = [3, 5, 3, 2, 3]
    state = plan.solve(ys[3][None], ms[3][None], ps[3][None], [prs[3].sigma], 3,
                       want_state=True)["r_tilde"][0].clone()
    descs, outs = [], []
    for i, q in enumerate(prs):
        o = {"x_hat": torch.full((wl.ny, wl.nx), 7.0 + 0j, dtype=torch.complex64, device="cuda"),
             "tau": torch.full((iters[i], B), -1.0, dtype=torch.float64, device="cuda")}
        o["thr"], o["alpha"] = o["tau"].clone(), o["tau"].clone()
        outs.append(o)
        d = {"y": ys[i], "mask": ms[i], "density": ps[i], "sigma": q.sigma, "iters": iters[i], **o}
        if i == 3:
            d.update(r_tilde0=state, k0=3)
        descs.append(d)
    # references: the same groups through vdamp_solve
    stk = lambda xs, idx: torch.stack([xs[i] for i in idx]).contiguous()
    ref = {}
    for idx, K in (([0, 2, 4], 3), ([1], 5)):
        r = plan.solve(stk(ys, idx), stk(ms, idx), stk(ps, idx), [prs[i].sigma for i in idx], K)
        for j, i in enumerate(idx):
            ref[i] = {k: r[k][j] for k in ("x_hat", "tau", "thr", "alpha")}
    r = plan.solve(ys[3][None], ms[3][None], ps[3][None], [prs[3].sigma], 2,
                   r_tilde0=state[None].contiguous(), k0=3)
    ref[3] = {k: r[k][0] for k in ("x_hat", "tau", "thr", "alpha")}
    for call in range(2):
        vb.vdamp_solve_batched(plan.handle, descs)
        torch.cuda.synchronize()
        assert vb.vdamp_device_status(plan.handle)[0] == vb.VDAMP_OK
        for i in range(5):
            for k in ("x_hat", "tau", "thr", "alpha"):
                assert torch.equal(outs[i][k], ref[i][k]), (call, i, k)
    bad = dict(descs[0], iters=0)
    with pytest.raises(vb.VdampError):
        vb.vdamp_solve_batched(plan.handle, [descs[1], bad])
    plan.close()


def test_pruned_search_on_many_slices_equals_single_slices():
    """The batched threshold search (one CTA per large subband, two medium or
    four small ones per CTA, many waves of CTAs) must give each subband the
    result it gets when its slice is solved alone: per slice every output equals
    that of a one-slice solve, bit for bit, and no error is recorded."""
    wl = synth.BATCH_320_DB4_5
    n = 48   # 48 slices x 8 CTAs: several waves
    prs = [synth.make_problem(wl, i) for i in range(n)]
    plan = vb.Plan(wl.ny, wl.nx, wl.wavelet, wl.levels, max_batch=n)
    t = plan.tuning()
    t["sure_parts"] = 1
    plan.set_tuning(t)
    y, m, p = _stack(prs, "y"), _stack(prs, "mask"), _stack(prs, "density")
    sig = [q.sigma for q in prs]
    out = plan.solve(y, m, p, sig, 4)
    st, _ = vb.vdamp_device_status(plan.handle)
    assert st == vb.VDAMP_OK
    # the large subbands' search on the side stream or in line: the same bits
    vb.vdamp_plan_set_option(plan.handle, vb.VDAMP_OPT_OVERLAP, 0)
    inline = plan.solve(y, m, p, sig, 4)
    vb.vdamp_plan_set_option(plan.handle, vb.VDAMP_OPT_OVERLAP, 1)
    for key in ("x_hat", "tau", "thr", "alpha"):
        assert torch.equal(inline[key], out[key]), key
    for i in (0, 17, n - 1):
        one = plan.solve(y[i:i + 1], m[i:i + 1], p[i:i + 1], [sig[i]], 4)
        for key in ("x_hat", "tau", "thr", "alpha"):
            assert torch.equal(one[key][0], out[key][i]), (i, key)
    plan.close()
