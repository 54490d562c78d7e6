"""Host-side checks of the CUDA library that need no GPU.

The library loads and exports every function include/vdamp.h declares; its
host-side setup (wavelet filters from Daubechies' factorisation and the 1D
factors of S = |Phi Psi^H|^2, Algorithm 1 line 1) agrees with the oracle's
independent derivations; invalid plans are rejected before any CUDA call.
"""
import numpy as np
import pytest

from oracle import vdamp_oracle as O
from paper_1911_01234_gb300 import binding as vb
from paper_1911_01234_gb300 import build


@pytest.fixture(scope="module")
def lib():
    build.build()
    return vb.load()


def test_exports_every_header_symbol(lib):
    names = vb.header_functions()
    assert len(names) >= 16
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(vb._SIGS), "binding and header disagree"


@pytest.mark.parametrize("name", ["haar", "db4"])
def test_filters_match_oracle(lib, name):
    got = vb.vdamp_wavelet_filter(name)
    want, _ = O.wavelet_filters(name)
    assert got.shape == want.shape
    assert np.abs(got - want).max() < 1e-14


@pytest.mark.parametrize("name,ny,nx,s", [("haar", 32, 32, 3), ("db4", 32, 48, 3),
                                          ("db4", 64, 40, 2), ("db4", 16, 16, 4)])
def test_spectra_match_bruteforce_s(lib, name, ny, nx, s):
    h, g = O.wavelet_filters(name)
    S = O.s_columns(ny, nx, h, g, s)
    ey = vb.vdamp_subband_spectra(name, s, ny)
    ex = vb.vdamp_subband_spectra(name, s, nx)
    for sb in O.subbands(ny, nx, s):
        j = sb.level
        lo, hi = 2 * (j - 1), 2 * (j - 1) + 1
        ty, tx = {"A": (lo, lo), "H": (lo, hi), "V": (hi, lo), "D": (hi, hi)}[sb.kind]
        col = np.outer(ey[ty], ex[tx])
        assert np.abs(col - S[sb.index]).max() < 1e-13 * max(1.0, S[sb.index].max()), sb.name


@pytest.mark.parametrize("args", [
    (100, 64, "db4", 3),     # 100 is not divisible by 2^3
    (64, 64, "db4", 7),      # too many levels
    (64, 64, 3, 2),          # unknown wavelet
    (7 * 16, 64, "db4", 4),  # 7 is not an FFT radix
    (64, 4, "haar", 1),      # too small
    (2048, 64, "haar", 1),   # too large
    (64, 64, "db4", 3, 0),   # max_batch < 1
    (64, 64, "db4", 3, 1, 0),   # max_iters < 1
])
def test_plan_create_rejects_bad_arguments(lib, args):
    with pytest.raises(vb.VdampError) as e:
        vb.vdamp_plan_create(*args)
    assert e.value.status == vb.VDAMP_EINVAL
    assert "vdamp_plan_create" in vb.last_error()


def test_null_plan_calls_are_rejected(lib):
    assert lib.vdamp_plan_destroy(None) == vb.VDAMP_EINVAL
    assert lib.vdamp_num_subbands(None) == -1
    assert lib.vdamp_psi(None, 1, None, None, None) == vb.VDAMP_EINVAL
    assert lib.vdamp_solve(None, 1, *([None] * 4), 1, None, 0, *([None] * 7)) == vb.VDAMP_EINVAL
    assert lib.vdamp_solve_host(None, 1, *([None] * 4), 1, None, 0, *([None] * 5)) == \
        vb.VDAMP_EINVAL
    assert lib.vdamp_solve_batched(None, None, 1, None) == vb.VDAMP_EINVAL
    assert "vdamp_solve_batched" in vb.last_error()
