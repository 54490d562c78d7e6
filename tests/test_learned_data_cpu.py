"""The learned denoiser is never evaluated on its training phantoms.

Training pairs come from plain VDAMP on phantoms of a workload seed of their
own (77 for the 256x256 network, 78 for the 320x320 one); the evaluated
slices come from the benchmark workloads' seeds.  The phantoms are checked
pairwise: no evaluated image equals, or nearly repeats (correlation of the
magnitudes above 0.99), a training image.
"""
import numpy as np

from paper_1911_01234_gb300 import synth


def _phantoms(wl, n):
    return [np.abs(synth.make_problem(wl, i).x0).ravel() for i in range(n)]


def _max_corr(a_list, b_list):
    A = np.stack([(a - a.mean()) / np.linalg.norm(a - a.mean()) for a in a_list])
    B = np.stack([(b - b.mean()) / np.linalg.norm(b - b.mean()) for b in b_list])
    return float(np.max(A @ B.T))


def test_training_and_evaluation_phantoms_are_disjoint():
    for train_id, ev, n_train, n_eval in ((77, synth.PLAIN_256_DB4_4, 52, 8),
                                          (78, synth.BATCH_320_DB4_5, 63, 16)):
        tr = synth.Workload("training phantoms", train_id, ev.ny, ev.nx, 20, True, ev.wavelet,
                            ev.levels, ev.rate, ev.rate_hi, 24, 30.0, 30.0, ev.iters, 1)
        assert tr.workload_id != ev.workload_id
        c = _max_corr(_phantoms(tr, n_train), _phantoms(ev, n_eval))
        assert c < 0.99, (train_id, c)
