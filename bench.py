"""Benchmark: plain VDAMP (Algorithm 1) on one 256x256 slice, db4 s=4, 30 iterations.

One step = one vdamp_solve of the whole hot path (30 iterations of lines 3-8
plus the return line) on one synthetic slice whose inputs are resident in
HBM.  Prints one JSON line.  `--impl reference` times the FP64 CPU oracle on
the host cores instead.  Under torchrun each rank solves its own 256x256 slice
for the headline (weak scaling), and the batched and mixed blocks partition
their slices over the ranks (balanced by pixels x iterations) and gather the
results on rank 0; no collective touches the data path.
"""
import os

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")   # the oracle baseline runs on one core

import argparse
import json
import math
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1911_01234_gb300 import synth  # noqa: E402

WL = synth.PLAIN_256_DB4_4
METRIC = "slice-iterations/s at 256x256 (plain VDAMP, db4 s=4, 30 iterations)"
UNIT = "slice-iterations/s"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def config_block(slices_per_gpu, world):
    return {"workload": WL.name, "ny": WL.ny, "nx": WL.nx, "wavelet": WL.wavelet,
            "levels": WL.levels, "iters": WL.iters, "rate": WL.rate, "snr_db": WL.snr_db,
            "slices_per_gpu": slices_per_gpu, "global_batch": slices_per_gpu * world,
            "parallelism": f"replicas x{world} (independent slices, no collective)",
            "l2": "flushed between steps (256 MiB write outside the step events)"}


# ------------------------------------------------------------ CPU oracle ---

class OracleRunner:
    """The FP64 oracle iterating the same workload; operators (S) built once."""

    def __init__(self, slice_idx=0):
        from oracle import vdamp_oracle as O
        self.O = O
        self.pr = synth.make_problem(WL, slice_idx)
        self.ops = O.make_operators(self.pr.mask, self.pr.density, self.pr.wavelet,
                                    self.pr.levels)
        self.y = np.where(self.pr.mask == 1, self.pr.y.astype(np.complex128), 0.0)
        self.s2 = float(self.pr.sigma) ** 2
        self.k = 0
        self.rt = np.zeros(WL.ny * WL.nx, dtype=np.complex128)

    def run(self, budget_s):
        """Iterate (lines 3-8; the return line after every 30th) for ~budget_s seconds."""
        O = self.O
        done = 0
        t0 = time.perf_counter()
        while True:
            rec = O.iterate(self.rt, self.y, self.ops, self.s2)
            self.rt = O.next_r_tilde(rec, self.ops)
            self.k += 1
            done += 1
            if self.k == WL.iters:
                O.final_estimate(rec.w_hat, self.y, self.ops)
                self.k = 0
                self.rt = np.zeros_like(self.rt)
            el = time.perf_counter() - t0
            if el >= budget_s:
                return done, el


_START = None


def _oracle_init(barrier):
    global _START
    _START = barrier


def _oracle_worker(job):
    """One host process: the oracle on its own slice, `warm` untimed seconds, then the
    timed budgets one after another (started together with the other workers)."""
    slice_idx, warm, budgets = job
    runner = OracleRunner(slice_idx)
    if warm > 0:
        runner.run(warm)
    if _START is not None:
        _START.wait(timeout=300)
    return [runner.run(b) for b in budgets]


def oracle_throughput(warm, budgets, workers):
    """FP64 oracle slice-iterations/s over all `workers` host processes (one slice each;
    spawned, so safe after CUDA is initialised).  Returns (per-budget list of
    (iterations summed over workers, slowest worker's seconds), workers used)."""
    if workers > 1:
        try:
            import multiprocessing as mp
            ctx = mp.get_context("spawn")
            barrier = ctx.Barrier(workers)
            with ctx.Pool(workers, initializer=_oracle_init, initargs=(barrier,)) as pool:
                job = pool.map_async(_oracle_worker, [(i, warm, budgets) for i in range(workers)])
                res = job.get(timeout=warm + sum(budgets) + 600)
            steps = [(sum(r[j][0] for r in res), max(r[j][1] for r in res))
                     for j in range(len(budgets))]
            return steps, workers
        except Exception:
            pass   # no process pool here: one process
    return _oracle_worker((0, warm, budgets)), 1


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    budget = max(0.2, min(args.ref_step_seconds, 150.0 / max(1, args.steps + args.warmup)))
    steps, cores = oracle_throughput(budget * args.warmup, [budget] * args.steps,
                                     args.ref_workers or os.cpu_count() or 1)
    total_it = sum(it for it, _ in steps)
    total_s = sum(el for _, el in steps)
    value = total_it / total_s
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_block(1, 1),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} steps of ~{budget:.2f} s of FP64 numpy "
                                       f"oracle iterations, one 256x256 slice per host "
                                       f"process ({cores} processes, {total_it} iterations)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ GPU arm ---

class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.marks = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.gpu)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return []
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        rows = []
        for ln in out.strip().splitlines():
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        return rows

    @staticmethod
    def summarize(rows):
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows)}


# Algorithmic bytes per launch of each kernel kind, per slice, for this
# workload (N = ny nx pixels, n = sampled frequencies).
def algorithmic_bytes(kind, N, n, levels):
    lv = [N / 4 ** (j - 1) for j in range(1, levels + 1)]   # pixels entering scale j
    if kind == "col_pass":     # k-space in + out, y and p on Omega, mask bits
        return 16 * N + 12 * n + N / 8
    if kind == "fft_rows":     # rows in + out
        return 16 * N
    if kind == "idwt":         # four bands in, one image out, mean over scales
        return statistics.mean(16 * v for v in lv)
    if kind == "dwt":          # image in, four bands out, r_{k-1} in for r~
        return statistics.mean(16 * v + 8 * v * (1.0 if j == levels else 0.75)
                               for j, v in enumerate(lv, start=1))
    if kind == "sure":         # r_k once
        return 8 * N
    return 0.0


# Measured with ncu (dram__bytes_read.sum + dram__bytes_write.sum per launch,
# mean over the launches of one iteration of the 256x256 db4 s=4 workload:
# 4 scales for idwt and dwt, the sort + search pairs for sure (the pairs of
# scales 1, 2, 3 and of the coarsest scale with the approximation band
# together: one iteration's threshold step, which the bench times as one
# event pair in its one-stream kernel-timing solve), the column pass) on the
# kernel build named by the hash of its sources; ignored (traffic null) once
# they changed.  ncu replays each launch with cold caches, and a launch's
# writes stay in L2.
MEASURED_TRAFFIC = {
    "idwt": {"bytes_per_launch": 241984, "source": "edb592202f1285cf"},
    "dwt": {"bytes_per_launch": 386368, "source": "edb592202f1285cf"},
    "sure": {"bytes_per_launch": 1626368, "source": "38dc34fea4bcea67"},
    "col_pass": {"bytes_per_launch": 863744, "source": "25a4268755cd2261"},
}


def taps(wavelet):
    return 2 if wavelet == "haar" else 8


def iteration_bytes(N, n):
    """Algorithmic bytes of one slice-iteration under the iteration's two global sync
    points: r_k in and r_{k+1} out (complex64), y and 1/p on Omega, the mask as bits."""
    return 16 * N + 12 * n + N / 8


def iteration_flops(ny, nx, levels, L):
    """Algorithmic FLOPs of one slice-iteration: the FFT pair (5 N log2 N each), the DWT
    pair (complex data, real L-tap filters, two 1D passes per scale: 8 L N_j per transform
    summed over the scales), and ~40 N elementwise (tau terms, line 8, threshold)."""
    N = ny * nx
    dwt = sum(8 * L * N / 4 ** j for j in range(levels))
    return 2 * 5 * N * math.log2(N) + 2 * dwt + 40 * N


def kernel_flops(kind, ny, nx, levels, L):
    """Algorithmic FLOPs per launch of one slice (the same kinds as algorithmic_bytes)."""
    N = ny * nx
    lv = [N / 4 ** (j - 1) for j in range(1, levels + 1)]
    if kind == "fft_rows":
        return 5 * N * math.log2(nx)
    if kind == "col_pass":
        return 2 * 5 * N * math.log2(ny) + 30 * N
    if kind in ("idwt", "dwt"):
        return statistics.mean(8 * L * v for v in lv)
    if kind == "sure":          # |r|, the prefix sums and one candidate quadratic per coefficient
        return 20 * N
    return 0.0


def bound_of(byts, flops, bw_gbs, p_tflops):
    """'hbm' or 'alu': the larger of the two lower bounds on the time."""
    if not p_tflops:
        return "hbm"
    return "alu" if flops / (p_tflops * 1e12) > byts / (bw_gbs * 1e9) else "hbm"


def iteration_roofline(s_per_slice_iter, ny, nx, n, levels, L, bw_gbs, p_fp32_tflops):
    """Whole-iteration roofline: T_roof = max(B_alg / BW, F_alg / P_fp32) against the
    measured time per slice-iteration, and the two partial fractions."""
    N = ny * nx
    b, f = iteration_bytes(N, n), iteration_flops(ny, nx, levels, L)
    t_hbm = b / (bw_gbs * 1e9)
    t_alu = f / (p_fp32_tflops * 1e12) if p_fp32_tflops else 0.0
    t_roof = max(t_hbm, t_alu)
    return {"bytes_per_slice_iter": b, "flops_per_slice_iter": f,
            "intensity_flop_per_byte": f / b, "us_per_slice_iter": s_per_slice_iter * 1e6,
            "t_roof_us": t_roof * 1e6, "frac": t_roof / s_per_slice_iter,
            "hbm_frac": t_hbm / s_per_slice_iter,
            "alu_frac": (t_alu / s_per_slice_iter) if p_fp32_tflops else None,
            "bound": "alu" if t_alu > t_hbm else "hbm",
            "peaks": {"hbm_gbs": bw_gbs, "fp32_tflops": p_fp32_tflops}}


def partition_slices(costs, world):
    """Slices to ranks, balanced by cost (pixels x iterations): longest first, each to the
    least-loaded rank (ties to the lower rank).  Returns one ascending index list per rank."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    out = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(i)
        load[r] += costs[i]
    return [sorted(x) for x in out]


def gather_by_slice(parts, world, rank, local, total):
    """Host gather of per-slice results to rank 0: `local` maps this rank's slice indices
    (parts[rank]) to result objects; rank 0 gets them back in slice order [0, total)."""
    if world <= 1:
        got = [local]
    else:
        import torch.distributed as dist
        got = [None] * world if rank == 0 else None
        dist.gather_object(local, got, dst=0)
    if rank != 0:
        return None
    out = [None] * total
    for r in range(world):
        for i, v in got[r].items():
            assert out[i] is None and i in parts[r], i
            out[i] = v
    assert all(v is not None for v in out)
    return out


def slowest_rank_ms(local_ms, world, device=None):
    """Max over ranks of the timed region (ms); the job's clock is its slowest rank."""
    if world <= 1:
        return float(local_ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, steps, iters_per_step, slices_per_rank, max_ms):
    """Whole-job slice-iterations/s: every rank's work over the slowest rank's time."""
    return world * slices_per_rank * steps * iters_per_step / (max_ms / 1e3)


# The sources each measured kernel is compiled from (its own code and the shared
# device helpers it inlines); its launch shape is fixed by the tuning named with
# the measurement.
KERNEL_SOURCES = {
    "idwt": ("dwt.cu", "dwt_dev.cuh", "vdamp_internal.cuh"),
    "dwt": ("dwt.cu", "dwt_dev.cuh", "vdamp_internal.cuh"),
    "sure": ("sure.cu", "sure_dev.cuh", "sure_prune_dev.cuh", "vdamp_internal.cuh"),
    "fft_rows": ("fft.cu", "fft_dev.cuh", "vdamp_internal.cuh"),
    "col_pass": ("fft_col.cu", "fft_dev.cuh", "vdamp_internal.cuh"),
}


def source_hash(kernel="idwt"):
    """Hash of the sources a kernel is built from: its measured traffic stays valid
    while they are unchanged."""
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1911_01234_gb300", "csrc")
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def timed_steps(torch, fn, steps, flush_buf, stream, world, warm=2):
    """Events around each of `steps` calls after `warm` untimed ones, L2 flushed before
    each (outside the events), barrier and synchronize on both sides; returns
    (this rank's total ms, the slowest rank's total ms)."""
    import torch.distributed as dist
    for i in range(warm):
        flush_buf.fill_(float(i))
        fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for i in range(steps):
        flush_buf.fill_(float(i))
        ev[i][0].record(stream)
        fn()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    return ms, slowest_rank_ms(ms, world, device="cuda")


def dominant_kernel(vb, plan, step, reps=1):
    """Per-kind event times of `reps` directly launched solves: (kind, {kind: (ms, n)})."""
    vb.vdamp_plan_set_option(plan.handle, vb.VDAMP_OPT_KERNEL_TIMING, 1)
    vb.vdamp_kernel_times(plan.handle)
    for _ in range(reps):
        step()
    kt = vb.vdamp_kernel_times(plan.handle)
    vb.vdamp_plan_set_option(plan.handle, vb.VDAMP_OPT_KERNEL_TIMING, 0)
    dom = max((k for k in kt if kt[k][1] > 0 and k != "other"), key=lambda k: kt[k][0])
    return dom, kt


def kernel_roofline(dom, kt, wl, slices, n_per_slice, peaks_, reps=1):
    """The dominant kernel's roofline: algorithmic bytes (and FLOPs) per launch over its
    mean event-timed launch, against the measured HBM peak (or FP32 peak if ALU-bound)."""
    hbm, src, p32 = peaks_["hbm_gbs"], peaks_["hbm_source"], peaks_.get("fp32_tflops")
    N = wl.ny * wl.nx
    L = taps(wl.wavelet)
    avg_s = kt[dom][0] / kt[dom][1] / 1e3
    if dom == "fused":
        byt = slices * wl.iters * iteration_bytes(N, n_per_slice)
        fl = slices * wl.iters * iteration_flops(wl.ny, wl.nx, wl.levels, L)
    else:
        byt = slices * algorithmic_bytes(dom, N, n_per_slice, wl.levels)
        fl = slices * kernel_flops(dom, wl.ny, wl.nx, wl.levels, L)
    bound = bound_of(byt, fl, hbm, p32)
    tot = sum(x[0] for x in kt.values())
    out = {"bound": bound, "kernel": dom, "avg_launch_us": avg_s * 1e6,
           "algorithmic_bytes_per_launch": byt, "algorithmic_flops_per_launch": fl,
           "time_share": {k: round(v[0] / tot, 4) for k, v in kt.items()},
           "launches_per_step": {k: v[1] // reps for k, v in kt.items()},
           "avg_us_by_kernel": {k: round(1e3 * v[0] / v[1], 2) for k, v in kt.items() if v[1]}}
    if bound == "hbm":
        out.update(achieved=byt / avg_s / 1e9, peak=hbm, peak_source=src, unit="GB/s",
                   frac=byt / avg_s / 1e9 / hbm)
    else:
        out.update(achieved=fl / avg_s / 1e12, peak=p32, peak_source="measured (vdamp_fma_peak)",
                   unit="TFLOP/s", frac=fl / avg_s / 1e12 / p32)
    out["hbm_frac"] = byt / avg_s / 1e9 / hbm
    out["alu_frac"] = (fl / avg_s / 1e12 / p32) if p32 else None
    return out


def run_batched(args, vb, torch, flush_buf, stream, rank, world, peaks_):
    """Batched workload: 256 slices of 320x320, db4 s=5, R=6, 30 dB, 20 iterations.  At
    N > 1 the slices are partitioned over the ranks (balanced by pixels x iterations),
    every rank solves its share, and x_hat, tau, theta, alpha are gathered on rank 0."""
    wl = synth.BATCH_320_DB4_5
    nb = args.batched_slices
    N = wl.ny * wl.nx
    parts = partition_slices([N * wl.iters] * nb, world)
    mine = parts[rank]
    probs = [synth.make_problem(wl, i) for i in mine]
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(np.stack(a))).cuda()
    y, m, p = dev([q.y for q in probs]), dev([q.mask for q in probs]), dev([q.density for q in probs])
    sig = [q.sigma for q in probs]
    n_samp = int(sum(int(q.mask.sum()) for q in probs))
    nm = len(mine)
    plan = vb.Plan(wl.ny, wl.nx, wl.wavelet, wl.levels, max_batch=nm)
    if args.path != "auto":
        vb.vdamp_plan_set_option(plan.handle, vb.VDAMP_OPT_FUSED, 1 if args.path == "fused" else 0)
    tuning = None if args.no_autotune else plan.autotune(nm, trials=3, stream=stream.cuda_stream)
    K = wl.iters
    x_hat = torch.empty((nm, wl.ny, wl.nx), dtype=torch.complex64, device="cuda")
    tau = torch.empty((nm, K, plan.B), dtype=torch.float64, device="cuda")
    thr, alpha = torch.empty_like(tau), torch.empty_like(tau)

    def step():
        vb.vdamp_solve(plan.handle, nm, y, m, p, sig, K, None, x_hat, tau, thr, alpha,
                       stream=stream.cuda_stream)
    steps = args.batched_steps
    _, max_ms = timed_steps(torch, step, steps, flush_buf, stream, world)
    if vb.vdamp_device_status(plan.handle)[0] != vb.VDAMP_OK:
        raise RuntimeError("batched solve reported a non-finite tau or alpha")
    # host gather of the results on rank 0 (outside the timed region)
    t0 = time.perf_counter()
    local = {i: (x_hat[j].cpu().numpy(), tau[j].cpu().numpy(), thr[j].cpu().numpy(),
                 alpha[j].cpu().numpy()) for j, i in enumerate(mine)}
    allres = gather_by_slice(parts, world, rank, local, nb)
    gather_s = time.perf_counter() - t0
    dom, kt = dominant_kernel(vb, plan, step)
    out = None
    if rank == 0:
        s_per = max_ms / 1e3 / (nb * K * steps)
        out = {"workload": wl.name, "slices": nb, "iters": K, "steps": steps,
               "value": nb * K * steps / (max_ms / 1e3), "unit": UNIT,
               "ms_per_step": max_ms / steps, "tuning": tuning,
               "partition": {"ranks": world, "slices_per_rank": [len(q) for q in parts],
                             "balance": "pixels x iterations, longest first",
                             "gathered_slices": sum(r is not None for r in allres),
                             "gather_s": round(gather_s, 3)},
               "roofline": kernel_roofline(dom, kt, wl, nm, n_samp / nm, peaks_),
               "iteration_roofline": iteration_roofline(
                   s_per, wl.ny, wl.nx, n_samp / nm, wl.levels, taps(wl.wavelet),
                   peaks_["hbm_gbs"], peaks_.get("fp32_tflops"))}
    plan.close()
    return out


def run_mixed(args, vb, torch, flush_buf, stream, rank, world):
    """Mixed-size batch: 32 slices each of 128x128, 256x256 and 384x320 (db4 s=4,
    per-slice R ~ U[3, 8] and SNR ~ U[25, 40] dB, 30 iterations) as one grouped
    graph launch, next to the same groups solved one after another.  At N > 1 the
    96 slices are partitioned over the ranks, balanced by pixels x iterations."""
    wls = synth.mixed_batch_workloads()
    K = wls[0].iters
    allsl = [(w, i) for w, wl in enumerate(wls) for i in range(wl.batch)]
    parts = partition_slices([wls[w].ny * wls[w].nx * K for w, _ in allsl], world)
    groups, plans, tunings = [], [], {}
    for w, wl in enumerate(wls):
        idx = [allsl[j][1] for j in parts[rank] if allsl[j][0] == w]
        if not idx:
            continue
        probs = [synth.make_problem(wl, i) for i in idx]
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(np.stack(a))).cuda()
        plan = vb.Plan(wl.ny, wl.nx, wl.wavelet, wl.levels, max_batch=len(idx))
        if not args.no_autotune:
            tunings[f"{wl.ny}x{wl.nx}"] = plan.autotune(len(idx), trials=3,
                                                         stream=stream.cuda_stream)
        plans.append(plan)
        groups.append((plan, dev([q.y for q in probs]), dev([q.mask for q in probs]),
                       dev([q.density for q in probs]), [q.sigma for q in probs]))
    slices = len(allsl)
    steps = args.batched_steps
    _, ms_grouped = timed_steps(torch, lambda: vb.solve_groups(groups, K,
                                                               stream=stream.cuda_stream),
                                steps, flush_buf, stream, world)
    _, ms_serial = timed_steps(torch, lambda: [g[0].solve(*g[1:], K, stream=stream.cuda_stream)
                                               for g in groups], steps, flush_buf, stream, world)
    for plan in plans:
        if vb.vdamp_device_status(plan.handle)[0] != vb.VDAMP_OK:
            raise RuntimeError("mixed solve reported a non-finite tau or alpha")
        plan.close()
    if rank != 0:
        return None
    return {"workload": "batched 96 mixed slices (32 x 128x128, 32 x 256x256, 32 x 384x320) "
                        "db4 s=4 R~U[3,8] SNR~U[25,40] K=30",
            "slices": slices, "iters": K, "steps": steps,
            "value": slices * K * steps / (ms_grouped / 1e3), "unit": UNIT,
            "ms_per_step": ms_grouped / steps,
            "one_group_after_another": {"value": slices * K * steps / (ms_serial / 1e3),
                                        "ms_per_step": ms_serial / steps},
            "partition": {"ranks": world, "slices_per_rank": [len(q) for q in parts]},
            "tuning": tunings or None}


def run_profile_case(args):
    """Untimed solves of one workload for a profiler (no JSON contract line)."""
    import torch
    from paper_1911_01234_gb300 import binding as vb
    from paper_1911_01234_gb300 import build
    build.build()
    vb.load()
    wl = WL if args.profile_case == "plain" else synth.BATCH_320_DB4_5
    nb = 1 if args.profile_case == "plain" else args.batched_slices
    probs = [synth.make_problem(wl, i) for i in range(nb)]
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(np.stack(a))).cuda()
    y, m, p = dev([q.y for q in probs]), dev([q.mask for q in probs]), dev([q.density for q in probs])
    plan = vb.Plan(wl.ny, wl.nx, wl.wavelet, wl.levels, max_batch=nb)
    if args.tuning:
        t = [int(v) for v in args.tuning.split(",")]
        plan.set_tuning(t + vb.vdamp_plan_get_tuning(plan.handle)[len(t):])   # rest: defaults
    for _ in range(args.warmup + args.steps):
        plan.solve(y, m, p, [q.sigma for q in probs], wl.iters)
    torch.cuda.synchronize()
    st = vb.vdamp_device_status(plan.handle)[0]
    plan.close()
    print(json.dumps({"profile_case": args.profile_case, "slices": nb, "solves":
                      args.warmup + args.steps, "tuning": args.tuning or "default",
                      "status": st}), flush=True)
    if st != vb.VDAMP_OK:
        raise SystemExit(1)


def run_fft_reference(vb, torch, stream):
    """The unitary 2D DFT of the library (row and column kernels, `vdamp_fft2`) timed beside
    cuFFT (torch.fft.fft2, norm="ortho") on the same data: a reference, not on the hot path
    (the iteration fuses the k-space step into the column transform instead)."""
    out = {}
    for ny, nx, batch, reps in ((256, 256, 1, 200), (320, 320, 256, 20)):
        plan = vb.Plan(ny, nx, "db4", 4, max_batch=batch)
        g = torch.Generator(device="cuda").manual_seed(7)
        x = torch.randn((batch, ny, nx), dtype=torch.complex64, device="cuda", generator=g)
        y_ours = torch.empty_like(x)

        def timed(fn):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            ts = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1) * 1e3)
            return statistics.median(ts)
        ours = timed(lambda: vb.vdamp_fft2(plan.handle, batch, x, y_ours,
                                           stream=stream.cuda_stream))
        cufft = timed(lambda: torch.fft.fft2(x, norm="ortho"))
        ref = torch.fft.fft2(x, norm="ortho")
        torch.cuda.synchronize()
        err = float((torch.linalg.vector_norm(y_ours - ref) / torch.linalg.vector_norm(ref)).item())
        out[f"{batch}x{ny}x{nx}"] = {"ours_us": round(ours, 2), "cufft_us": round(cufft, 2),
                                     "rel_l2_vs_cufft": err}
        plan.close()
    return out


def solve_closure(vb, torch, plan, y, m, p, sig, iters, stream):
    """A plain solve of `iters` iterations into preallocated outputs (so that every call
    replays the same cached graph)."""
    b = y.shape[0]
    x = torch.empty((b, plan.ny, plan.nx), dtype=torch.complex64, device="cuda")
    t = torch.empty((b, iters, plan.B), dtype=torch.float64, device="cuda")
    th, al = torch.empty_like(t), torch.empty_like(t)
    return lambda: vb.vdamp_solve(plan.handle, b, y, m, p, sig, iters, None, x, t, th, al,
                                  stream=stream.cuda_stream)


def first_reaching(curve, target):
    """1-based count of iterations after which `curve` (NMSE per iteration) is <= target."""
    return next((k + 1 for k, v in enumerate(curve) if v <= target), None)


def timed_mean_ms(torch, fn, flush_buf, stream, reps=5, warm=2):
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(reps)]
    for i in range(reps):
        flush_buf.fill_(float(i))
        ev[i][0].record(stream)
        fn()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev) / reps


def run_learned_batched(args, vb, torch, flush_buf, stream):
    """Learned VDAMP at scale: 256 slices of 320x320 db4 s=5 R=6 (a 16-subband network
    trained on pairs of that kind).  Both methods' mean-NMSE curves are measured per
    iteration; the target is the plain method's 30-iteration mean NMSE, and each method's
    time to it is the time of a solve of the iterations it needs to reach it."""
    from paper_1911_01234_gb300 import learned
    wl = synth.BATCH_320_DB4_5
    nb = args.batched_slices
    tim = {}
    net, _ = learned.train_for(wl.ny, wl.nx, wl.wavelet, wl.levels, wl.rate, 63, wl.iters,
                               steps=1500, workload_id=78, timings=tim)
    probs = [synth.make_problem(wl, i) for i in range(nb)]
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(np.stack(a))).cuda()
    y, m, p = dev([q.y for q in probs]), dev([q.mask for q in probs]), dev([q.density for q in probs])
    x0 = dev([q.x0.astype(np.complex64) for q in probs])
    x0n = (x0.abs().double() ** 2).sum(dim=(1, 2))
    sig = [q.sigma for q in probs]
    plan = vb.Plan(wl.ny, wl.nx, wl.wavelet, wl.levels, max_batch=nb)
    if not args.no_autotune:
        plan.autotune(nb, trials=3, stream=stream.cuda_stream)

    def slice_nmse(x):   # evaluation only: 10 log10 |x - x0|^2 / |x0|^2 per slice
        e = ((x - x0).abs().double() ** 2).sum(dim=(1, 2))
        return (10.0 * torch.log10(e / x0n)).cpu().numpy()

    def mean_nmse(x):
        return float(np.mean(slice_nmse(x)))

    plain = plan.solve(y, m, p, sig, 30, want_iters=True)
    torch.cuda.synchronize()
    plain_slices = np.stack([slice_nmse(plain["x_hat_iters"][k]) for k in range(30)])
    plain_curve = [float(v) for v in plain_slices.mean(1)]
    plain_median = [float(v) for v in np.median(plain_slices, 1)]
    # slices whose iteration diverges (final NMSE 3 dB above their best): an instability of
    # the method on some trajectories, which the FP64 oracle reproduces from the same state
    diverged = int(np.sum(plain_slices[-1] > plain_slices.min(0) + 3.0))
    del plain
    target = plain_curve[-1]
    need_plain = first_reaching(plain_curve, target)
    ms_plain = {k: timed_mean_ms(torch, solve_closure(vb, torch, plan, y, m, p, sig, k, stream),
                                 flush_buf, stream, reps=3)
                for k in sorted({1, need_plain, wl.iters, 30})}
    full = learned.LearnedSolver(plan, net, nb, wl.iters, want_iters=True)
    out = full.run(y, m, p, sig)
    torch.cuda.synchronize()
    full.check()
    learned_slices = np.stack([slice_nmse(out["x_hat_iters"][k]) for k in range(wl.iters)])
    curve = [float(v) for v in learned_slices.mean(1)]
    learned_median = [float(v) for v in np.median(learned_slices, 1)]
    use = out["use"].float().mean(dim=(0, 1)).cpu().numpy()
    del full, out
    need = first_reaching(curve, target)
    target_med = plain_median[-1]
    need_plain_med = first_reaching(plain_median, target_med)
    need_med = first_reaching(learned_median, target_med)
    ms_plain.update({k: timed_mean_ms(torch, solve_closure(vb, torch, plan, y, m, p, sig, k, stream),
                                      flush_buf, stream, reps=3)
                     for k in {need_plain_med} if k not in ms_plain})
    ms_learned = {}
    for k in sorted({1, wl.iters} | ({need} if need else set()) | ({need_med} if need_med else set())):
        solver = learned.LearnedSolver(plan, net, nb, k).capture(y, m, p, sig)
        ms_learned[k] = timed_mean_ms(torch, solver.replay, flush_buf, stream, reps=3)
        solver.check()
        del solver
    plan.close()
    per_it_plain = (ms_plain[30] - ms_plain[1]) / 29
    per_it_learned = (ms_learned[wl.iters] - ms_learned[1]) / max(1, wl.iters - 1)
    return {"workload": wl.name + ", learned per-subband CNN (16 networks) chosen by SURE",
            "metric": "time to reach the plain method's 30-iteration mean NMSE", "unit": "ms",
            "target_mean_nmse_db": target,
            "plain_mean_nmse_db_by_iter": [round(v, 4) for v in plain_curve],
            "learned_mean_nmse_db_by_iter": [round(v, 4) for v in curve],
            "plain_iters_to_target": need_plain, "ms_plain_to_target": ms_plain[need_plain],
            "learned_iters_to_target": need,
            "ms_learned_to_target": ms_learned.get(need) if need else None,
            "speedup_to_target": (ms_plain[need_plain] / ms_learned[need]) if need else None,
            "final_nmse_gain_db": plain_curve[wl.iters - 1] - curve[-1],
            "plain_slices_diverged": diverged,
            "median": {"target_nmse_db": target_med,
                       "plain_median_nmse_db_by_iter": [round(v, 4) for v in plain_median],
                       "learned_median_nmse_db_by_iter": [round(v, 4) for v in learned_median],
                       "plain_iters_to_target": need_plain_med,
                       "learned_iters_to_target": need_med,
                       "speedup_to_target": (ms_plain[need_plain_med] / ms_learned[need_med])
                       if need_med else None},
            "ms_plain_by_iters": ms_plain, "ms_learned_by_iters": ms_learned,
            "ms_per_iteration": {"plain": per_it_plain, "learned": per_it_learned,
                                 "learned_over_plain": per_it_learned / per_it_plain},
            "network_use_per_subband": [round(float(u), 2) for u in use],
            "training": tim}


def run_learned(args, vb, torch, flush_buf, stream, slices=4):
    """Learned VDAMP at 256x256 db4 s=4 (per-subband CNN chosen by SURE) on `slices`
    held-out slices: per slice, both NMSE curves, the first iteration at which each method
    reaches the plain method's own 30-iteration NMSE, and each method's time to get there
    (a solve of that many iterations); the medians over the slices are the headline."""
    from oracle import vdamp_oracle as O
    from paper_1911_01234_gb300 import learned
    tim = {}
    net, _ = learned.train_default(steps=1500, timings=tim)
    wl = WL
    plan = vb.Plan(wl.ny, wl.nx, wl.wavelet, wl.levels)
    if not args.no_autotune:
        plan.autotune(1, trials=3, stream=stream.cuda_stream)
    K = wl.iters
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a[None])).cuda()
    per_slice, uses = [], []
    for s_idx in range(slices):
        pr = synth.make_problem(wl, s_idx)
        y, m, p = d(pr.y), d(pr.mask), d(pr.density)
        plain = plan.solve(y, m, p, [pr.sigma], K, want_iters=True)
        torch.cuda.synchronize()
        nm_p = [O.nmse_db(plain["x_hat_iters"][k, 0].cpu().numpy(), pr.x0) for k in range(K)]
        solver = learned.LearnedSolver(plan, net, 1, K, want_iters=True)
        out = solver.run(y, m, p, [pr.sigma])
        torch.cuda.synchronize()
        solver.check()
        nm_l = [O.nmse_db(out["x_hat_iters"][k, 0].cpu().numpy(), pr.x0) for k in range(K)]
        uses.append(out["use"].cpu().numpy()[:, 0, :].mean(0))
        target = nm_p[-1]
        per_slice.append({"slice": s_idx, "plain_nmse_db_30": target,
                          "learned_nmse_db_30": nm_l[-1],
                          "plain_iters_to_target": first_reaching(nm_p, target),
                          "learned_iters_to_target": first_reaching(nm_l, target),
                          "plain_nmse_db_by_iter": [round(v, 4) for v in nm_p],
                          "learned_nmse_db_by_iter": [round(v, 4) for v in nm_l]})
    # solve times by iteration count (they do not depend on the slice's values)
    pr = synth.make_problem(wl, 0)
    y, m, p = d(pr.y), d(pr.mask), d(pr.density)
    ks_p = sorted({1, K} | {r["plain_iters_to_target"] for r in per_slice})
    ks_l = sorted({1, K} | {r["learned_iters_to_target"] for r in per_slice
                            if r["learned_iters_to_target"]})
    ms_p = {k: timed_mean_ms(torch, solve_closure(vb, torch, plan, y, m, p, [pr.sigma], k,
                                                  stream),
                             flush_buf, stream, reps=10, warm=3) for k in ks_p}
    ms_l = {}
    for k in ks_l:
        sv = learned.LearnedSolver(plan, net, 1, k).capture(y, m, p, [pr.sigma])
        ms_l[k] = timed_mean_ms(torch, sv.replay, flush_buf, stream, reps=10, warm=3)
        sv.check()
    plan.close()
    sp = []
    for r in per_slice:
        r["ms_plain_to_target"] = ms_p[r["plain_iters_to_target"]]
        kl = r["learned_iters_to_target"]
        r["ms_learned_to_target"] = ms_l[kl] if kl else None
        r["speedup_to_target"] = (r["ms_plain_to_target"] / ms_l[kl]) if kl else None
        if kl:
            sp.append(r["speedup_to_target"])
    per_it_p = (ms_p[K] - ms_p[1]) / (K - 1)
    per_it_l = (ms_l[K] - ms_l[1]) / (K - 1)
    return {"workload": "learned VDAMP, 256x256 db4 s=4 R=5 30 dB, per-subband 5-layer CNN "
                        "(32 ch, BF16 tcgen05) chosen by SURE, Hutchinson divergence",
            "metric": "time to reach the plain method's 30-iteration NMSE", "unit": "ms",
            "slices": slices,
            "median_speedup_to_target": statistics.median(sp) if sp else None,
            "median_final_nmse_gain_db": statistics.median(
                r["plain_nmse_db_30"] - r["learned_nmse_db_30"] for r in per_slice),
            "ms_plain_by_iters": ms_p, "ms_learned_by_iters": ms_l,
            "ms_per_iteration": {"plain": per_it_p, "learned": per_it_l,
                                 "learned_over_plain": per_it_l / per_it_p},
            "per_slice": per_slice,
            "network_use_per_subband": [round(float(u), 2) for u in np.mean(uses, axis=0)],
            "training": tim}


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_1911_01234_gb300 import binding as vb
    from paper_1911_01234_gb300 import build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    vb.load()

    pr = synth.make_problem(WL, slice_idx=rank)
    N = WL.ny * WL.nx
    n_samp = int(pr.mask.sum())
    y = torch.from_numpy(pr.y[None].copy()).cuda()
    m = torch.from_numpy(pr.mask[None].copy()).cuda()
    p = torch.from_numpy(pr.density[None].copy()).cuda()
    plan = vb.Plan(WL.ny, WL.nx, WL.wavelet, WL.levels)
    if args.path != "auto":
        vb.vdamp_plan_set_option(plan.handle, vb.VDAMP_OPT_FUSED, 1 if args.path == "fused" else 0)
    K = WL.iters
    x_hat = torch.empty((1, WL.ny, WL.nx), dtype=torch.complex64, device="cuda")
    tau = torch.empty((1, K, plan.B), dtype=torch.float64, device="cuda")
    thr, alpha = torch.empty_like(tau), torch.empty_like(tau)
    stream = torch.cuda.current_stream()
    if args.tuning:
        t = [int(v) for v in args.tuning.split(",")]
        plan.set_tuning(t + vb.vdamp_plan_get_tuning(plan.handle)[len(t):])   # rest: defaults
        tuning = plan.tuning()
    else:
        # 40 iterations per candidate: shapes differ by a few per cent at one slice
        tuning = None if args.no_autotune else plan.autotune(1, trials=40,
                                                             stream=stream.cuda_stream)
    flush_buf = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step():
        vb.vdamp_solve(plan.handle, 1, y, m, p, [pr.sigma], K, None, x_hat, tau, thr, alpha,
                       stream=stream.cuda_stream)

    for i in range(max(args.warmup, 3)):
        flush_buf.fill_(float(i))
        step()
    torch.cuda.synchronize()
    launches_per_step = vb.vdamp_last_launch_count(plan.handle)

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    for i in range(args.steps):
        flush_buf.fill_(float(i))
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    if world > 1:
        dist.barrier()
    rows = clocks.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    tot_ms = sum(step_ms)
    st, _ = vb.vdamp_device_status(plan.handle)
    if st != vb.VDAMP_OK:
        raise RuntimeError("solve reported a non-finite tau or alpha")
    max_ms = slowest_rank_ms(tot_ms, world, device="cuda")
    value = job_throughput(world, args.steps, K, 1, max_ms)

    # ---- peaks of this GPU: HBM from MEASURED_PEAKS.json, FP32 / FP64 FMA measured here
    hbm, src = peaks()
    p32, ms32 = vb.vdamp_fma_peak(32, 20000, stream=stream.cuda_stream)
    p64, ms64 = vb.vdamp_fma_peak(64, 400, stream=stream.cuda_stream)
    peaks_ = {"hbm_gbs": hbm, "hbm_source": src, "fp32_tflops": p32, "fp64_tflops": p64,
              "fma_kernel_ms": {"fp32": ms32, "fp64": ms64}}

    # ---- dominant kernel, timed live with CUDA events on the launching stream
    reps = 5

    def timed_reps():
        for i in range(reps):
            flush_buf.fill_(float(i))
            step()
    dom, kt = dominant_kernel(vb, plan, timed_reps, reps=1)
    roofline = kernel_roofline(dom, kt, WL, 1, n_samp, peaks_, reps=reps)
    meas = MEASURED_TRAFFIC.get(dom)
    roofline["traffic"] = meas["bytes_per_launch"] if meas and meas.get("source") == \
        source_hash(dom) else None
    roofline["iteration"] = iteration_roofline(max_ms / 1e3 / (args.steps * K), WL.ny, WL.nx,
                                               n_samp, WL.levels, taps(WL.wavelet), hbm, p32)

    # ---- end to end through the host-buffer entry point (pinned host memory); the L2
    # flush before each step is outside the wall-clock region
    hy = torch.from_numpy(pr.y[None].copy()).pin_memory()
    hm = torch.from_numpy(pr.mask[None].copy()).pin_memory()
    hp = torch.from_numpy(pr.density[None].copy()).pin_memory()
    hx = torch.empty((1, WL.ny, WL.nx), dtype=torch.complex64).pin_memory()
    ht = torch.empty((1, K, plan.B), dtype=torch.float64).pin_memory()
    hth, hal = torch.empty_like(ht).pin_memory(), torch.empty_like(ht).pin_memory()
    lib = vb.load()
    sig = vb._sigma_array([pr.sigma], 1)

    def e2e_step():
        vb.check(lib.vdamp_solve_host(plan.handle, 1, hy.data_ptr(), hm.data_ptr(),
                                      hp.data_ptr(), sig, K, None, 0, hx.data_ptr(), ht.data_ptr(),
                                      hth.data_ptr(), hal.data_ptr(), stream.cuda_stream),
                 "vdamp_solve_host")
    for i in range(3):
        e2e_step()
    e2e_steps = max(10, min(args.steps, 200))
    e2e_s = 0.0
    for i in range(e2e_steps):
        flush_buf.fill_(float(i))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_step()   # copies in, solve, copies out, and waits for them
        e2e_s += time.perf_counter() - t0
    e2e_val = world * e2e_steps * K / e2e_s
    h2d = 8 * N + N + 4 * N
    d2h = 8 * N + 3 * 8 * K * plan.B

    line = None
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": max_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic (seeded ellipse phantom, polynomial VD mask)",
                "config": dict(config_block(1, world), path=args.path, tuning=tuning),
                "clocks": ClockSampler.summarize(rows),
                "gpu_launches": launches_per_step * args.steps,
                "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "roofline": roofline, "peaks": peaks_,
                "wall_s_timed": wall}
    # the batched and mixed blocks run on every rank (slices partitioned over the ranks);
    # the learned blocks and the host baseline are single-GPU measurements
    if world > 1:
        args.no_learned = args.no_cpu_baseline = True
    if not args.no_batched:
        bat = run_batched(args, vb, torch, flush_buf, stream, rank, world, peaks_)
        mix = run_mixed(args, vb, torch, flush_buf, stream, rank, world)
        if rank == 0:
            line["batched"], line["mixed"] = bat, mix
            line["fft_reference"] = run_fft_reference(vb, torch, stream)
    if rank == 0:
        if not args.no_learned:
            line["learned"] = run_learned(args, vb, torch, flush_buf, stream)
            if not args.no_batched:
                line["learned_batched"] = run_learned_batched(args, vb, torch, flush_buf, stream)
        if not args.no_cpu_baseline:
            steps, cores = oracle_throughput(1.0, [args.cpu_seconds],
                                             args.ref_workers or os.cpu_count() or 1)
            it, el = steps[0]
            line["cpu_baseline"] = {"value": it / el, "unit": UNIT, "cores": cores,
                                    "kind": "oracle",
                                    "sample": f"{it} FP64 numpy oracle iterations in {el:.1f} s, "
                                              f"one 256x256 slice per host process "
                                              f"({cores} processes)"}
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-step-seconds", type=float, default=4.0)
    ap.add_argument("--ref-workers", type=int, default=0,
                    help="host processes of the oracle baseline (0: one per host core)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the 256 x 320x320 batched measurement")
    ap.add_argument("--batched-slices", type=int, default=256)
    ap.add_argument("--batched-steps", type=int, default=5)
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned-denoiser measurement (trains for a few seconds)")
    ap.add_argument("--tuning", default="",
                    help="explicit launch shapes for the 256x256 plan (comma-separated, "
                         "vdamp_plan_set_tuning order; entries left out keep the plan's "
                         "defaults) instead of autotuning it")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the plans' default launch shapes")
    ap.add_argument("--path", default="auto", choices=["auto", "fused", "steps"],
                    help="solve as one persistent cluster launch, or one kernel per step")
    ap.add_argument("--profile-case", default="", choices=["", "plain", "batched"],
                    help="only run solves of one workload, untimed (for ncu captures): "
                         "--warmup + --steps solves of the 256x256 slice or of "
                         "--batched-slices 320x320 slices, with --tuning if given")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.profile_case:
        run_profile_case(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
