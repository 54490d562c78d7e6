"""Thin ctypes binding of libvdamp.so (include/vdamp.h), names as in the C ABI.

Only argument marshalling happens here: every step of the VDAMP iteration runs
in the library's CUDA kernels.  PyTorch supplies device memory and streams.
There is no fallback: if the library is missing or fails to load, every call
raises.
"""
from __future__ import annotations

import ctypes
import os
import re
from typing import Optional

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvdamp.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "vdamp.h")

VDAMP_OK, VDAMP_EINVAL, VDAMP_ENOMEM, VDAMP_ECUDA, VDAMP_ENUMERIC, VDAMP_ETIMEOUT = range(6)
STATUS_NAMES = {0: "VDAMP_OK", 1: "VDAMP_EINVAL", 2: "VDAMP_ENOMEM", 3: "VDAMP_ECUDA",
                4: "VDAMP_ENUMERIC", 5: "VDAMP_ETIMEOUT"}
VDAMP_HAAR, VDAMP_DB4 = 1, 4
WAVELETS = {"haar": VDAMP_HAAR, "db4": VDAMP_DB4}
VDAMP_OPT_GRAPH, VDAMP_OPT_KERNEL_TIMING, VDAMP_OPT_FUSED, VDAMP_OPT_OVERLAP = 1, 2, 3, 4
KERNEL_KINDS = ["idwt", "fft_rows", "col_pass", "dwt", "sure", "other", "fused"]


class VdampError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.POINTER(ctypes.c_double)
_SIGS = {
    "vdamp_last_error": (ctypes.c_char_p, []),
    "vdamp_plan_create": (_I, [ctypes.POINTER(_P), _I, _I, _I, _I, _I, _I]),
    "vdamp_plan_destroy": (_I, [_P]),
    "vdamp_num_subbands": (_I, [_P]),
    "vdamp_workspace_bytes": (ctypes.c_size_t, [_P]),
    "vdamp_plan_set_option": (_I, [_P, _I, _I]),
    "vdamp_last_launch_count": (_I, [_P]),
    "vdamp_solve": (_I, [_P, _I, _P, _P, _P, _P, _I, _P, _I, _P, _P, _P, _P, _P, _P, _P]),
    "vdamp_solve_host": (_I, [_P, _I, _P, _P, _P, _P, _I, _P, _I, _P, _P, _P, _P, _P]),
    "vdamp_solve_batched": (_I, [_P, _P, _I, _P]),
    "vdamp_iterate": (_I, [_P, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "vdamp_final_estimate": (_I, [_P, _I, _P, _P, _P, _P, _P]),
    "vdamp_psi": (_I, [_P, _I, _P, _P, _P]),
    "vdamp_psi_h": (_I, [_P, _I, _P, _P, _P]),
    "vdamp_fft2": (_I, [_P, _I, _P, _P, _I, _P]),
    "vdamp_device_status": (_I, [_P, ctypes.POINTER(_I), _P]),
    "vdamp_wavelet_filter": (_I, [_I, _D, ctypes.POINTER(_I)]),
    "vdamp_subband_spectra": (_I, [_I, _I, _I, _D]),
    "vdamp_kernel_times": (_I, [_P, _D, ctypes.POINTER(_I)]),
    "vdamp_tau_estimate_noalloc": (_I, [_I, _I, _I, _I, _P, _P, _P, ctypes.c_float, _P, _P]),
    "vdamp_plan_get_tuning": (_I, [_P, ctypes.POINTER(_I)]),
    "vdamp_plan_set_tuning": (_I, [_P, ctypes.POINTER(_I)]),
    "vdamp_plan_autotune": (_I, [_P, _I, _I, ctypes.POINTER(_I), _P]),
    "vdamp_solve_groups": (_I, [_P, _I, _P]),
    # learned per-subband denoiser
    "vdamp_cnn_conv3x3": (_I, [_P, _I, _P, _I, _P, _P, _P, _I, _I, _I, _P, _I, _I, _I, _P, _P]),
    "vdamp_cnn_pack_weights": (_I, [_P, _I, _I, _I, _I, _I, _I, _P, _P]),
    "vdamp_cnn_wgrad": (_I, [_P, _I, _I, _P, _I, _I, _P, _I, _I, _P, _P, _P]),
    "vdamp_cnn_input": (_I, [_P, _P, _I, _P, _I, _I, _P, _P]),
    "vdamp_cnn_probe": (_I, [ctypes.c_ulonglong, _P, _I, _I, _P, _P]),
    "vdamp_cnn_output": (_I, [_P, _P, _I, _P, _I, _I, _P, _P, ctypes.c_ulonglong, _P, _P, _P]),
    "vdamp_cnn_loss": (_I, [_P, _P, _P, _I, _P, _I, _I, _P, ctypes.c_float, _P, _P, _P]),
    "vdamp_cnn_adam": (_I, [_P, _P, _P, _P, ctypes.c_size_t, ctypes.c_float, ctypes.c_float,
                            ctypes.c_float, ctypes.c_float, _I, _P]),
    "vdamp_cnn_onsager": (_I, [_P] * 6 + [_I] + [_P] * 2 + [_I, _I] + [_P] * 5),
    "vdamp_last_sure": (_I, [_P, _I, _P, _P]),
    "vdamp_cnn_set_wait_limit": (_I, [ctypes.c_uint, ctypes.POINTER(ctypes.c_uint)]),
    "vdamp_cnn_default_wait_limit": (ctypes.c_uint, []),
    "vdamp_cnn_status": (_I, [_P, _P]),
    "vdamp_fma_peak": (_I, [_I, _I, _D, _D, _P]),
    "vdamp_sure_fallback_count": (_I, [_P, ctypes.POINTER(_I), _P]),
}

VDAMP_TUNING_LEN = 8
TUNING_FIELDS = ("col_block", "rows_per_cta", "idwt_tile", "dwt_tile", "radix_y", "radix_x",
                 "wavelet_cluster", "sure_parts")


class vdamp_group(ctypes.Structure):
    """struct vdamp_group of include/vdamp.h."""
    _fields_ = [("plan", _P), ("batch", _I), ("y", _P), ("mask", _P), ("density", _P),
                ("sigma", ctypes.POINTER(ctypes.c_float)), ("iters", _I), ("x_hat", _P),
                ("tau", _P), ("thr", _P), ("alpha", _P)]


class vdamp_slice_desc(ctypes.Structure):
    """struct vdamp_slice_desc of include/vdamp.h."""
    _fields_ = [("y", _P), ("mask", _P), ("density", _P), ("sigma", ctypes.c_float),
                ("iters", _I), ("r_tilde0", _P), ("k0", _I), ("x_hat", _P), ("tau", _P),
                ("thr", _P), ("alpha", _P)]


DEFAULT_MAX_ITERS = 64

_lib: Optional[ctypes.CDLL] = None


def load() -> ctypes.CDLL:
    """Load libvdamp.so (built by paper_1911_01234_gb300.build); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built: run paper_1911_01234_gb300.build.build()"
                               " (nvcc, sm_103a); there is no fallback path")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def header_functions():
    """Names of the functions include/vdamp.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vdamp_[a-z0-9_]+)\s*\(", text)))


def last_error() -> str:
    return load().vdamp_last_error().decode()


def check(status: int, where: str) -> None:
    if status != VDAMP_OK:
        raise VdampError(status, where, last_error())


def _ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(stream)


def _sigma_array(sigma, batch):
    arr = (ctypes.c_float * batch)()
    vals = [float(sigma)] * batch if not hasattr(sigma, "__len__") else [float(s) for s in sigma]
    if len(vals) != batch:
        raise ValueError("sigma needs one value per slice")
    for i, v in enumerate(vals):
        arr[i] = v
    return arr


# ------------------------------------------------------------ C-ABI calls ---

def vdamp_plan_create(ny: int, nx: int, wavelet, levels: int, max_batch: int = 1,
                      max_iters: int = DEFAULT_MAX_ITERS) -> int:
    w = WAVELETS.get(wavelet, wavelet) if isinstance(wavelet, str) else int(wavelet)
    h = _P()
    check(load().vdamp_plan_create(ctypes.byref(h), ny, nx, w, levels, max_iters, max_batch),
          "vdamp_plan_create")
    return h.value


def vdamp_plan_destroy(plan: int) -> None:
    check(load().vdamp_plan_destroy(plan), "vdamp_plan_destroy")


def vdamp_num_subbands(plan: int) -> int:
    return load().vdamp_num_subbands(plan)


def vdamp_workspace_bytes(plan: int) -> int:
    return load().vdamp_workspace_bytes(plan)


def vdamp_plan_set_option(plan: int, option: int, value: int) -> None:
    check(load().vdamp_plan_set_option(plan, option, value), "vdamp_plan_set_option")


def vdamp_last_launch_count(plan: int) -> int:
    return load().vdamp_last_launch_count(plan)


def vdamp_solve(plan, batch, y, mask, density, sigma, iters, r_tilde0, x_hat, tau, thr, alpha,
                r_tilde_out=None, x_hat_iters=None, stream=None, k0=0) -> None:
    """Device-buffer solve; tensors are CUDA torch tensors (complex64/uint8/float32/float64)."""
    sig = _sigma_array(sigma, batch)
    check(load().vdamp_solve(plan, batch, _ptr(y), _ptr(mask), _ptr(density), sig, iters,
                             _ptr(r_tilde0), int(k0), _ptr(x_hat), _ptr(tau), _ptr(thr),
                             _ptr(alpha),
                             _ptr(r_tilde_out), _ptr(x_hat_iters), _stream(stream)),
          "vdamp_solve")


def vdamp_solve_host(plan, batch, y, mask, density, sigma, iters, r_tilde0, x_hat, tau, thr,
                     alpha, stream=None, k0=0) -> None:
    """Host-buffer solve; arrays are C-contiguous numpy arrays of the header's types."""
    sig = _sigma_array(sigma, batch)

    def a(x):
        return None if x is None else x.ctypes.data
    check(load().vdamp_solve_host(plan, batch, a(y), a(mask), a(density), sig, iters,
                                  a(r_tilde0), int(k0), a(x_hat), a(tau), a(thr), a(alpha),
                                  _stream(stream)), "vdamp_solve_host")


def vdamp_solve_batched(plan, slices, stream=None) -> None:
    """slices: list of dicts with the vdamp_slice_desc fields (tensors for device arrays;
    r_tilde0 and k0 may be left out for a cold start)."""
    arr = (vdamp_slice_desc * len(slices))()
    for i, d in enumerate(slices):
        arr[i] = vdamp_slice_desc(_ptr(d["y"]), _ptr(d["mask"]), _ptr(d["density"]),
                                  float(d["sigma"]), int(d["iters"]), _ptr(d.get("r_tilde0")),
                                  int(d.get("k0", 0)), _ptr(d["x_hat"]), _ptr(d["tau"]),
                                  _ptr(d["thr"]), _ptr(d["alpha"]))
    check(load().vdamp_solve_batched(plan, ctypes.cast(arr, _P), len(slices), _stream(stream)),
          "vdamp_solve_batched")


def vdamp_iterate(plan, batch, r_tilde, y, mask, density, sigma, r, tau, thr, alpha,
                  r_tilde_next, stream=None) -> None:
    sig = _sigma_array(sigma, batch)
    check(load().vdamp_iterate(plan, batch, _ptr(r_tilde), _ptr(y), _ptr(mask), _ptr(density),
                               sig, _ptr(r), _ptr(tau), _ptr(thr), _ptr(alpha),
                               _ptr(r_tilde_next), _stream(stream)), "vdamp_iterate")


def vdamp_final_estimate(plan, batch, w, y, mask, x_hat, stream=None) -> None:
    check(load().vdamp_final_estimate(plan, batch, _ptr(w), _ptr(y), _ptr(mask), _ptr(x_hat),
                                      _stream(stream)), "vdamp_final_estimate")


def vdamp_psi(plan, batch, x, w, stream=None) -> None:
    check(load().vdamp_psi(plan, batch, _ptr(x), _ptr(w), _stream(stream)), "vdamp_psi")


def vdamp_psi_h(plan, batch, w, x, stream=None) -> None:
    check(load().vdamp_psi_h(plan, batch, _ptr(w), _ptr(x), _stream(stream)), "vdamp_psi_h")


def vdamp_fft2(plan, batch, x, out, inverse=False, stream=None) -> None:
    check(load().vdamp_fft2(plan, batch, _ptr(x), _ptr(out), 1 if inverse else 0,
                            _stream(stream)), "vdamp_fft2")


def vdamp_device_status(plan, stream=None):
    """(status, first_bad_iteration) after waiting for the plan's work on `stream`."""
    it = _I(-1)
    st = load().vdamp_device_status(plan, ctypes.byref(it), _stream(stream))
    return st, it.value


def vdamp_kernel_times(plan):
    """{kind: (total ms, launches)} of the timed launches since the last call."""
    n = len(KERNEL_KINDS)
    ms = (ctypes.c_double * n)()
    cnt = (_I * n)()
    check(load().vdamp_kernel_times(plan, ms, cnt), "vdamp_kernel_times")
    return {k: (ms[i], cnt[i]) for i, k in enumerate(KERNEL_KINDS)}


def vdamp_tau_estimate_noalloc(ny, nx, wavelet, levels, z, mask, density, sigma, tau,
                               stream=None) -> None:
    """The per-subband noise estimate tau from a residual z, with no device allocation and
    no plan (for callers that cannot allocate device memory; the paper has no counterpart)."""
    w = WAVELETS.get(wavelet, wavelet) if isinstance(wavelet, str) else int(wavelet)
    check(load().vdamp_tau_estimate_noalloc(ny, nx, w, levels, _ptr(z), _ptr(mask), _ptr(density),
                                            float(sigma), _ptr(tau), _stream(stream)),
          "vdamp_tau_estimate_noalloc")


def vdamp_fma_peak(precision, iters, stream=None):
    """(TFLOP/s, ms) of the FP32 (32) or FP64 (64) FMA-throughput kernel."""
    tf, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    check(load().vdamp_fma_peak(precision, iters, ctypes.byref(tf), ctypes.byref(ms),
                                _stream(stream)), "vdamp_fma_peak")
    return tf.value, ms.value


def vdamp_sure_fallback_count(plan, stream=None) -> int:
    """Subbands the pruned one-CTA threshold search left to the full sort (running total)."""
    n = _I(0)
    check(load().vdamp_sure_fallback_count(plan, ctypes.byref(n), _stream(stream)),
          "vdamp_sure_fallback_count")
    return n.value


def vdamp_cnn_set_wait_limit(polls):
    """Set the first-wait poll limit of later convolutions; returns the previous limit."""
    prev = ctypes.c_uint(0)
    check(load().vdamp_cnn_set_wait_limit(int(polls), ctypes.byref(prev)),
          "vdamp_cnn_set_wait_limit")
    return prev.value


def vdamp_cnn_default_wait_limit():
    return load().vdamp_cnn_default_wait_limit()


def vdamp_cnn_status(status, stream=None):
    """VDAMP_OK or VDAMP_ETIMEOUT from a convolution status word (read and cleared)."""
    return load().vdamp_cnn_status(_ptr(status), _stream(stream))


def vdamp_wavelet_filter(wavelet):
    import numpy as np
    w = WAVELETS.get(wavelet, wavelet) if isinstance(wavelet, str) else int(wavelet)
    h = (ctypes.c_double * 8)()
    n = _I(0)
    check(load().vdamp_wavelet_filter(w, h, ctypes.byref(n)), "vdamp_wavelet_filter")
    return np.array(h[:n.value])


def vdamp_subband_spectra(wavelet, levels, n):
    import numpy as np
    w = WAVELETS.get(wavelet, wavelet) if isinstance(wavelet, str) else int(wavelet)
    out = np.zeros(2 * levels * n)
    check(load().vdamp_subband_spectra(w, levels, n, out.ctypes.data_as(_D)),
          "vdamp_subband_spectra")
    return out.reshape(2 * levels, n)


def vdamp_plan_get_tuning(plan) -> list:
    t = (_I * VDAMP_TUNING_LEN)()
    check(load().vdamp_plan_get_tuning(plan, t), "vdamp_plan_get_tuning")
    return list(t)


def vdamp_plan_set_tuning(plan, tuning) -> None:
    t = (_I * VDAMP_TUNING_LEN)(*[int(v) for v in tuning])
    check(load().vdamp_plan_set_tuning(plan, t), "vdamp_plan_set_tuning")


def vdamp_plan_autotune(plan, batch, trials=5, stream=None) -> list:
    t = (_I * VDAMP_TUNING_LEN)()
    check(load().vdamp_plan_autotune(plan, batch, trials, t, _stream(stream)),
          "vdamp_plan_autotune")
    return list(t)


def vdamp_solve_groups(groups, stream=None) -> None:
    """groups: list of dicts with the vdamp_group fields (tensors for device arrays)."""
    arr = (vdamp_group * len(groups))()
    keep = []
    for i, g in enumerate(groups):
        sig = _sigma_array(g["sigma"], g["batch"])
        keep.append(sig)
        arr[i] = vdamp_group(g["plan"], g["batch"], _ptr(g["y"]), _ptr(g["mask"]),
                             _ptr(g["density"]), ctypes.cast(sig, ctypes.POINTER(ctypes.c_float)),
                             g["iters"], _ptr(g["x_hat"]), _ptr(g["tau"]), _ptr(g["thr"]),
                             _ptr(g["alpha"]))
    check(load().vdamp_solve_groups(ctypes.cast(arr, _P), len(groups), _stream(stream)),
          "vdamp_solve_groups")


# --------------------------------------------------------- convenience ---

class Plan:
    """Owns a vdamp_plan; solve() allocates outputs with torch on the plan's device."""

    def __init__(self, ny, nx, wavelet, levels, max_batch=1, max_iters=DEFAULT_MAX_ITERS):
        self.ny, self.nx, self.levels, self.max_batch = ny, nx, levels, max_batch
        self.wavelet, self.max_iters = wavelet, max_iters
        self.handle = vdamp_plan_create(ny, nx, wavelet, levels, max_batch, max_iters)
        self.B = vdamp_num_subbands(self.handle)

    def close(self):
        if self.handle:
            vdamp_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, y, mask, density, sigma, iters, r_tilde0=None, want_iters=False,
              want_state=False, stream=None, k0=0):
        import torch
        batch = y.shape[0] if y.dim() == 3 else 1
        dev = y.device
        x_hat = torch.empty((batch, self.ny, self.nx), dtype=torch.complex64, device=dev)
        tau = torch.empty((batch, iters, self.B), dtype=torch.float64, device=dev)
        thr = torch.empty_like(tau)
        alpha = torch.empty_like(tau)
        rt = torch.empty((batch, self.ny * self.nx), dtype=torch.complex64, device=dev) \
            if want_state else None
        xi = torch.empty((iters, batch, self.ny, self.nx), dtype=torch.complex64, device=dev) \
            if want_iters else None
        vdamp_solve(self.handle, batch, y, mask, density, sigma, iters, r_tilde0, x_hat, tau, thr,
                    alpha, rt, xi, stream, k0)
        return {"x_hat": x_hat, "tau": tau, "thr": thr, "alpha": alpha, "r_tilde": rt,
                "x_hat_iters": xi}

    def tuning(self):
        return dict(zip(TUNING_FIELDS, vdamp_plan_get_tuning(self.handle)))

    def set_tuning(self, tuning):
        vdamp_plan_set_tuning(self.handle, [tuning[k] for k in TUNING_FIELDS]
                              if isinstance(tuning, dict) else tuning)

    def autotune(self, batch=None, trials=5, stream=None):
        vdamp_plan_autotune(self.handle, batch or self.max_batch, trials, stream)
        return self.tuning()


def solve_groups(groups, iters, stream=None):
    """Mixed-size batched solve: groups = [(plan, y, mask, density, sigma), ...] with
    torch device tensors [batch][ny][nx]; returns one output dict per group."""
    import torch
    descs, outs = [], []
    for plan, y, mask, density, sigma in groups:
        batch = y.shape[0]
        dev = y.device
        o = {"x_hat": torch.empty((batch, plan.ny, plan.nx), dtype=torch.complex64, device=dev),
             "tau": torch.empty((batch, iters, plan.B), dtype=torch.float64, device=dev)}
        o["thr"] = torch.empty_like(o["tau"])
        o["alpha"] = torch.empty_like(o["tau"])
        outs.append(o)
        descs.append({"plan": plan.handle, "batch": batch, "y": y, "mask": mask,
                      "density": density, "sigma": sigma, "iters": iters, **o})
    vdamp_solve_groups(descs, stream)
    return outs
