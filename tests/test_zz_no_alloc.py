"""The no-allocation tau entry point agrees with the plan-based solver.

vdamp_tau_estimate_noalloc serves callers that cannot allocate device memory
(a fixed device memory pool or budget, hosts without an allocator, tools that
share a caching allocator).  It keeps its scratch in a fixed array inside the
library.  This test feeds it the residual z = m (y - F Psi^H r~) for an r~
reached by the solver, and compares its tau with the tau that vdamp_iterate
(the plan-based path) computes from the same r~, on two calls in a row, with
the tolerance the parity tests use: 1e-4 relative L2 on the tau vector and
1e-3 relative per subband.

A third test alternates two configurations (sizes, wavelets and levels) on one
stream with no synchronisation in between: each call fills the shared scratch
with its own tables on the device, so every result must still match.

This file is named to be collected last, so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1911_01234_gb300 import binding as vb
from paper_1911_01234_gb300 import build, synth

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("wl", [synth.PLAIN_256_DB4_4, synth.PLAIN_64_HAAR3])
def test_noalloc_tau_matches_plan_on_two_calls(wl):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    vb.load()
    pr = synth.make_problem(wl)
    ny, nx, N = wl.ny, wl.nx, wl.ny * wl.nx
    y = torch.from_numpy(pr.y[None].copy()).cuda()
    m = torch.from_numpy(pr.mask[None].copy()).cuda()
    p = torch.from_numpy(pr.density[None].copy()).cuda()
    plan = vb.Plan(ny, nx, wl.wavelet, wl.levels)
    B = plan.B
    img = torch.empty((1, ny, nx), dtype=torch.complex64, device="cuda")
    kspace = torch.empty_like(img)
    r = torch.empty((1, N), dtype=torch.complex64, device="cuda")
    rn = torch.empty_like(r)
    tau_ref = torch.empty((1, B), dtype=torch.float64, device="cuda")
    thr, alpha = torch.empty_like(tau_ref), torch.empty_like(tau_ref)
    tau_na = torch.empty(B, dtype=torch.float64, device="cuda")
    for call, iters in enumerate((2, 5)):
        r_tilde = plan.solve(y, m, p, [pr.sigma], iters, want_state=True)["r_tilde"]
        vb.vdamp_iterate(plan.handle, 1, r_tilde, y, m, p, [pr.sigma], r, tau_ref, thr, alpha, rn)
        vb.vdamp_psi_h(plan.handle, 1, r_tilde, img)
        vb.vdamp_fft2(plan.handle, 1, img, kspace)
        z = torch.where(m.bool(), y - kspace, torch.zeros_like(y)).contiguous()
        tau_na.fill_(-1.0)
        vb.vdamp_tau_estimate_noalloc(ny, nx, wl.wavelet, wl.levels, z[0], m[0], p[0],
                                      float(pr.sigma), tau_na)
        torch.cuda.synchronize()
        got = tau_na.cpu().numpy()
        want = tau_ref.cpu().numpy()[0]
        assert _rel(got, want) < 1e-4, (call, _rel(got, want))
        assert np.max(np.abs(got - want) / want) < 1e-3, call
    plan.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    vb.load()
    t = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(vb.VdampError) as e:
        vb.vdamp_tau_estimate_noalloc(2048, 64, "db4", 2, t, t, t, 0.1, t)
    assert e.value.status == vb.VDAMP_EINVAL
    assert "scratch limit" in vb.last_error()


def _reference_case(wl):
    """(device residual z, mask, density, sigma, tau from the plan path) for one workload."""
    pr = synth.make_problem(wl)
    ny, nx, N = wl.ny, wl.nx, wl.ny * wl.nx
    y = torch.from_numpy(pr.y[None].copy()).cuda()
    m = torch.from_numpy(pr.mask[None].copy()).cuda()
    p = torch.from_numpy(pr.density[None].copy()).cuda()
    plan = vb.Plan(ny, nx, wl.wavelet, wl.levels)
    img = torch.empty((1, ny, nx), dtype=torch.complex64, device="cuda")
    kspace = torch.empty_like(img)
    r = torch.empty((1, N), dtype=torch.complex64, device="cuda")
    rn = torch.empty_like(r)
    tau_ref = torch.empty((1, plan.B), dtype=torch.float64, device="cuda")
    thr, alpha = torch.empty_like(tau_ref), torch.empty_like(tau_ref)
    r_tilde = plan.solve(y, m, p, [pr.sigma], 3, want_state=True)["r_tilde"]
    vb.vdamp_iterate(plan.handle, 1, r_tilde, y, m, p, [pr.sigma], r, tau_ref, thr, alpha, rn)
    vb.vdamp_psi_h(plan.handle, 1, r_tilde, img)
    vb.vdamp_fft2(plan.handle, 1, img, kspace)
    z = torch.where(m.bool(), y - kspace, torch.zeros_like(y)).contiguous()
    torch.cuda.synchronize()
    want = tau_ref.cpu().numpy()[0]
    plan.close()
    return z[0], m[0].contiguous(), p[0].contiguous(), float(pr.sigma), want


def test_noalloc_alternating_configurations_on_one_stream():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    vb.load()
    cases = [(wl, _reference_case(wl)) for wl in (synth.PLAIN_256_DB4_4, synth.PLAIN_64_HAAR3)]
    outs = []
    for rep in range(2):   # A, B, A, B back to back, no host synchronisation between them
        for wl, (z, m, p, sigma, want) in cases:
            t = torch.full((len(want),), -1.0, dtype=torch.float64, device="cuda")
            vb.vdamp_tau_estimate_noalloc(wl.ny, wl.nx, wl.wavelet, wl.levels, z, m, p, sigma, t)
            outs.append((t, want, wl.name, rep))
    torch.cuda.synchronize()
    for t, want, name, rep in outs:
        got = t.cpu().numpy()
        assert _rel(got, want) < 1e-4, (name, rep, _rel(got, want))
        assert np.max(np.abs(got - want) / want) < 1e-3, (name, rep)
