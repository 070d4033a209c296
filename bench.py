"""Throughput of the SPOD hot path on the jet-shaped workload.

One step = fit (mean, blocks, window, FFT, weighted Gram, reduction, FP64
eigen-decomposition) + all modes, over X resident in HBM:
X = 512 x 256 grid x 3 variables, nt = 10 000 FP32 snapshots (15.7 GB),
nfft = 512, 50 % overlap (nb = 38), Hamming window, weights ~ r.
Metric: snapshot-GB/s = nt * M * sizeof(element) / (time per step).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16x3]
                    [--impl native|reference] [--no-compare] [--no-e2e] [--no-cpu]
    python bench.py --complex | --coeffs | --ooc | --backward | --batch     (separate measurements)

The default precision is bf16x3 (BF16 tensor-core Gram and modes with split
products); the same input is then also run through the plain FP32 GPU form
and reported under "vs_fp32".

N > 1 (torchrun): the paper's spatial decomposition (Sec. 3.1) -- every rank
owns one slab, a headline-sized grid of its own seed, of a domain N times the
headline grid (weak scaling); per step each rank fits its slab up to its part
of the Gram (spod_fit_partial), the parts are all-gathered in rank order (the
one exchange of the method), every rank sums them in that order and solves the
eigenproblems (spod_fit_from_grams), then computes the modes of its slab;
value = units of all ranks / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX, NR, NVARS, NT, NFFT = 512, 256, 3, 10000, 512
NOVERLAP = NFFT // 2
CPU_SAMPLE = 24576          # spatial columns of the oracle legs: ~10 s of oracle work per step on the host cores


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precision", default="bf16x3", choices=["fp32", "bf16x3", "bf16", "fp64"])
    ap.add_argument("--no-compare", action="store_true", help="skip the FP32 comparison run")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--small", action="store_true", help="a reduced grid for quick checks (not a bench value)")
    ap.add_argument("--grid", default=None, help="NXxNR grid for profiling runs (not a bench value)")
    ap.add_argument("--coeffs", action="store_true",
                    help="time the expansion coefficients + reconstruction (Eqs. coeffs, SPODrec) on a "
                         "256x128x2, nt=4096, nfft=256 grid; a separate measurement, not the headline line")
    ap.add_argument("--complex", action="store_true",
                    help="complex input of the same shape (the jet field + i x a second seed's field, "
                         "two-sided spectrum); a separate measurement, not the headline line")
    ap.add_argument("--backward", action="store_true",
                    help="time spod_backward (the adjoint of the eigenvalues) after a fit on the headline grid; "
                         "a separate measurement")
    ap.add_argument("--batch", action="store_true",
                    help="time spod_fit_batch on the six ERA5-shaped one-year datasets at full size (162 GB of "
                         "FP32 input resident in HBM), one graph launch per step, bf16x3 and FP32; a separate "
                         "measurement")
    ap.add_argument("--mean-pass", action="store_true",
                    help="take the time mean in a separate pass over X instead of inside the FFT pass "
                         "(spod_plan_desc.mean_in_fft = 0), for comparison")
    ap.add_argument("--bf16-input", action="store_true",
                    help="the headline grid stored as BF16 (the FP32 field rounded once to BF16); the plan reads "
                         "BF16 snapshots and computes at --precision; a separate measurement")
    ap.add_argument("--ooc", action="store_true",
                    help="time the out-of-core run (spod_run_host_ooc: X and Phi in pinned host memory, column "
                         "tiles over the host link) on the headline grid; a separate measurement")
    return ap.parse_args()


def workload_config(args, nb, nf, nmodes):
    cx = getattr(args, "complex", False)
    b16 = getattr(args, "bf16_input", False)
    esz = 8 if cx else (2 if b16 else 4)
    return {"workload": f"jet-shaped {NX}x{NR}x{NVARS}, nt={NT}, nfft={NFFT}, 50% overlap"
                        + (", complex (two-sided)" if cx else "") + (", stored as BF16" if b16 else ""),
            "npoints": NX * NR, "nvars": NVARS, "M": NX * NR * NVARS, "nt": NT, "nfft": NFFT,
            "noverlap": NOVERLAP, "nb": nb, "nf": nf, "nmodes": nmodes, "in_dtype": "c64" if cx else ("bf16" if b16 else "f32"),
            "precision": args.precision, "window": "hamming", "weights": "r-weighted",
            "l2": f"inputs larger than L2 ({NT * NX * NR * NVARS * esz / 1e9:.1f} GB per step)",
            "parallelism": "one GPU" if getattr(args, "gpus", 1) <= 1 else
                           f"{args.gpus} spatial slabs of one headline grid each, one all-gather of the slab Grams per step"}


# --------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        t_end = time.perf_counter() + 5.0           # let the sampler run before the timed region
        while not self.rows and time.perf_counter() < t_end and self.proc.poll() is None:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.perf_counter(), [x.strip() for x in line.split(",")]))

    def stop(self, t0=None, t1=None):
        """Median SM clock and active throttle reasons over the samples taken
        between host times t0 and t1 (the timed region), else over all."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        rows = [r for t, r in self.rows if t0 is None or t0 <= t <= t1]
        window = "timed region"
        if not rows:
            rows, window = [r for _, r in self.rows], "whole run (no sample fell inside the timed region)"
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            if len(r) >= 9:
                for i, n in enumerate(names):
                    if r[5 + i].lower().startswith("active"):
                        reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm), "window": window}


# --------------------------------------------------------------- oracle leg
def oracle_sample(wl_X_cpu_cols, W_cols, nmodes):
    """The FP64 oracle on a bounded spatial sample (all snapshots, P points)."""
    import oracle as O
    nt, P = wl_X_cpu_cols.shape
    d = O.Desc(nt=nt, M=P, nfft=NFFT, noverlap=NOVERLAP, window=O.WIN_HAMMING, weights=W_cols)
    t0 = time.perf_counter()
    fit = O.spod_fit(wl_X_cpu_cols, d, dft="fft")
    O.spod_modes(fit, d, nmodes)
    return time.perf_counter() - t0


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def sample_columns(X, P, seed=0):
    """P spatial columns spread over the grid (host FP64 copy of the stored values)."""
    import torch
    M = X.shape[1]
    idx = torch.linspace(0, M - 1, P).round().long().unique()
    cols = X[:, idx.to(X.device)].double().cpu().numpy()
    return cols, idx.numpy()


# --------------------------------------------------------------- main
def main():
    global MEAN_IN_FFT
    args = parse()
    MEAN_IN_FFT = not args.mean_pass
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if args.impl == "reference":
        return reference_leg(args, world, rank)
    if args.coeffs:
        return coeffs_leg(args, rank)
    if args.ooc:
        return ooc_leg(args, rank)
    if args.backward:
        return backward_leg(args, rank)
    if args.batch:
        return batch_leg(args, rank)

    import __graft_entry__ as g
    from paper_2309_11808_gb300 import _lib
    from workloads import jet_like

    g.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    nx, nr = (64, 64) if args.small else (NX, NR)
    if args.grid:
        nx, nr = (int(v) for v in args.grid.lower().split("x"))
    wl = jet_like(nx=nx, nr=nr, nvars=NVARS, nt=NT, nfft=NFFT, seed=rank, dtype=torch.float32, device=dev)
    if args.complex:
        im = jet_like(nx=nx, nr=nr, nvars=NVARS, nt=NT, nfft=NFFT, seed=rank + 1000, dtype=torch.float32,
                      device=dev).X
        wl.X = torch.complex(wl.X, im)
        del im
        torch.cuda.empty_cache()
        args.no_e2e = args.no_cpu = args.no_compare = True
    if args.bf16_input:
        wl.X = wl.X.to(torch.bfloat16)
        torch.cuda.empty_cache()
    X = wl.X
    M = X.shape[1]
    elem = X.element_size()
    bytes_step = NT * M * elem

    r = timed_run(args.precision, wl, args.steps, max(3, args.warmup), world, dev, clocks=True)
    sp, nb, nf, nmodes = r["sp"], r["nb"], r["nf"], r["nmodes"]
    ms_step, phase_ms, phase_launch, clk = r["ms_step"], r["phase_ms"], r["phase_launch"], r["clocks"]
    value = world * bytes_step / (ms_step * 1e-3) / 1e9

    # ---- roofline: every phase's kernel, the dominant one (largest time) on top
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except OSError:
        pass
    # one step launches each phase's kernels once (modes: the small coefficient
    # kernel + the mode GEMM), so the per-step phase time is the launch time
    per_phase = {k: kernel_roofline(k, phase_ms[k] / args.steps, M, nb, nf, nmodes, peaks, args.precision, elem,
                                    sp.mean_in_fft)
                 for k in phase_ms if phase_launch.get(k, 0) > 0}
    dom = max(per_phase, key=lambda k: phase_ms[k])
    roof = per_phase[dom]
    step_roof = step_roofline(ms_step, M, nb, nf, nmodes, peaks, args.precision)

    line = {"metric": "SPOD snapshot-GB/s (FFT+CSD+eig+modes)", "value": round(value, 3), "unit": "GB/s",
            "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup),
            "ms_per_step": round(ms_step, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE_NAME[args.precision],
            "data": "synthetic (seeded jet-shaped wave packets + AR(1) red noise)",
            "config": workload_config(args, nb, nf, nmodes), "roofline": roof,
            "step_roofline": step_roof,
            "phases_ms_per_step": {k: round(v / args.steps, 4) for k, v in phase_ms.items()},
            "phase_rooflines": per_phase,
            "gpu_launches": int(sum(phase_launch.values())), "clocks": clk,
            "snapshots_per_s": round(world * NT / (ms_step * 1e-3), 1),
            "mean_in_fft": bool(sp.mean_in_fft)}
    # fit alone (mean, FFT, Gram, reduction, eigen-solve: the phase events of
    # spod_fit, which runs its phases back to back on one stream)
    fit_ms = sum(phase_ms[k] for k in ("mean", "fft", "gram", "reduce", "eig")) / args.steps
    line["fit_only"] = {"ms_per_step": round(fit_ms, 4),
                        "value": round(world * bytes_step / (fit_ms * 1e-3) / 1e9, 3), "unit": "GB/s",
                        "snapshots_per_s": round(world * NT / (fit_ms * 1e-3), 1)}

    # ---- end to end through the C ABI with host buffers (right after the main
    # run: measured after the FP32 comparison run instead, the host-link copies
    # came out slower on this machine)
    if not args.no_e2e and rank == 0 and not args.small and not args.grid:
        if sp is None:
            sp = make_plan(args.precision, wl)
        line["e2e"] = e2e_leg(sp, X, nmodes, args, world)

    # ---- the plain FP32 GPU form on the same input (the comparison the metric names)
    if args.precision != "fp32" and not args.no_compare:
        sp.close()
        rf = timed_run("fp32", wl, max(2, args.steps // 2), 3, world, dev, clocks=False)
        rf["sp"].close()
        sp = None
        fv = world * bytes_step / (rf["ms_step"] * 1e-3) / 1e9
        line["vs_fp32"] = {"fp32_value": round(fv, 3), "fp32_ms_per_step": round(rf["ms_step"], 4),
                           "fp32_snapshots_per_s": round(world * NT / (rf["ms_step"] * 1e-3), 1),
                           "speedup": round(value / fv, 3), "fp32_steps": max(2, args.steps // 2),
                           "fp32_phases_ms_per_step": {k: round(v / max(2, args.steps // 2), 4)
                                                       for k, v in rf["phase_ms"].items()}}

    # ---- CPU oracle on a bounded sample
    if not args.no_cpu and rank == 0 and world == 1:
        cols, idx = sample_columns(X, min(CPU_SAMPLE, M))
        secs = oracle_sample(cols, wl.W.numpy()[idx], nmodes)
        line["cpu_baseline"] = {"value": round(NT * cols.shape[1] * elem / secs / 1e9, 5), "unit": "GB/s",
                                "cores": cpu_cores(), "kind": "oracle",
                                "sample": f"{cols.shape[1]} of {M} spatial columns, all {NT} snapshots, "
                                          f"fit + {nmodes} modes, numpy FFT step (oracle mode 'fft')",
                                "seconds": round(secs, 2)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if sp is not None:
        sp.close()
    if world > 1:
        dist.destroy_process_group()


DTYPE_NAME = {"fp32": "f32", "fp64": "f64", "bf16": "bf16", "bf16x3": "bf16x3"}
FP32_PEAK = 152 * 128 * 2 * 2.070e9 / 1e12      # TFLOP/s: SMs x FP32 lanes x FMA x max clock
FP64_PEAK = 1.25                                  # TFLOP/s: nominal GB300 FP64 rate


def max_over_ranks(x: float, dev) -> float:
    """The slowest rank's value (the job's time) when running under torch.distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_slab_grams(part, parts) -> None:
    """The one exchange of the spatial decomposition: every rank's slab Gram
    into parts[rank] on every rank (parts[r] holds rank r's part, so a sum in
    index order is the same sum on every rank).  A single process copies its
    own part."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_gather(list(parts.unbind(0)), part.contiguous())
    else:
        parts[0].copy_(part)


MEAN_IN_FFT = True      # --mean-pass clears it


def make_plan(precision, wl):
    from paper_2309_11808_gb300 import SPOD
    return SPOD(wl.npoints, NVARS, NT, NFFT, NOVERLAP, dtype=wl.X.dtype, precision=precision, weights=wl.W,
                mean_in_fft=MEAN_IN_FFT)


def timed_run(precision, wl, steps, warmup, world, dev, clocks):
    """W untimed steps, then K steps between CUDA events on the launching stream."""
    import torch
    import torch.distributed as dist
    from paper_2309_11808_gb300 import _lib
    X = wl.X
    sp = make_plan(precision, wl)
    nb, nf = sp.nb, sp.nf
    nmodes = nb
    cdt = torch.complex128 if precision == "fp64" else torch.complex64
    Phi = torch.empty((nf, nmodes, X.shape[1]), dtype=cdt, device=dev)
    stream = torch.cuda.current_stream(dev)

    if world > 1:
        # the slab Gram of this rank and the gathered parts of all ranks, in rank order
        part = torch.empty((nf, nb, nb, 2), dtype=torch.float64, device=dev)
        parts = torch.empty((world, nf, nb, nb, 2), dtype=torch.float64, device=dev)

        def step():
            _lib.spod_fit_partial(sp.handle, X, part, stream)
            gather_slab_grams(part, parts)
            _lib.spod_fit_from_grams(sp.handle, parts, world, stream)
            _lib.spod_modes(sp.handle, X, nmodes, Phi, stream)
    else:
        def step():
            _lib.spod_fit(sp.handle, X, stream)
            _lib.spod_modes(sp.handle, X, nmodes, Phi, stream)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    _lib.spod_profile_read(sp.handle)          # discard warm-up
    _lib.spod_profile_enable(sp.handle, True)
    sampler = ClockSampler(dev.index or 0) if clocks else None
    if sampler:
        sampler.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    h0 = time.perf_counter()
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    h1 = time.perf_counter()
    if world > 1:
        dist.barrier()
    clk = sampler.stop(h0, h1) if sampler else None
    ms_total = e0.elapsed_time(e1)
    phase_ms, phase_launch = _lib.spod_profile_read(sp.handle)
    _lib.spod_profile_enable(sp.handle, False)
    _lib.spod_sync(sp.handle, stream)
    ms_total = max_over_ranks(ms_total, dev)
    del Phi
    return {"sp": sp, "nb": nb, "nf": nf, "nmodes": nmodes, "ms_step": ms_total / steps, "phase_ms": phase_ms,
            "phase_launch": phase_launch, "clocks": clk}


# Kernel of each phase and precision (the phase timer brackets exactly these launches).
KERNELS = {
    "mean": "k_mean_partial + k_mean_finish",
    "fft": {"fp32": "k_fft_pipe", "fp64": "k_fft", "bf16": "k_fft_pipe", "bf16x3": "k_fft_pipe"},
    "gram": {"fp32": "k_gram_simt", "fp64": "k_gram_simt", "bf16": "k_gram_tc + k_gram_tc_collect",
             "bf16x3": "k_gram_tc + k_gram_tc_collect"},
    "reduce": {"fp32": "k_gram_reduce", "fp64": "k_gram_reduce", "bf16": "k_gram_tc_finish",
               "bf16x3": "k_gram_tc_finish"},
    "eig": "k_eig_tridiag",
    "modes": {"fp32": "k_mode_coeffs + k_modes_simt", "fp64": "k_mode_coeffs + k_modes_simt",
              "bf16": "k_mode_coeffs + k_mode_image + k_modes_tc",
              "bf16x3": "k_mode_coeffs + k_mode_image + k_modes_tc"},
}


def qhat_bytes_per_point(nb, nf, precision, folded=False):
    """Bytes of Qhat per spatial point: nf x 2 nb real entries (+ nf for the
    rho row when the time mean is taken inside the FFT pass)."""
    per = {"fp64": 8, "fp32": 4, "bf16": 2, "bf16x3": 4}[precision]
    return nf * (2 * nb + (1 if folded else 0)) * per


def kernel_roofline(phase, per_launch_ms, M, nb, nf, nmodes, peaks, precision, elem=4, folded=False):
    """Roofline of one launch of a phase's kernel on its ALGORITHMIC work.

    The method's compulsory traffic is X read once and the modes written
    (Phi, complex64 / complex128); everything else this pipeline moves -- the
    Qhat written by the FFT and read back by the Gram and the modes -- is
    implementation overhead, reported as ``overhead_bytes`` and counted
    against the kernel, not credited to it.  So: the mean and the FFT are
    credited with X read once, the modes with Phi written, the tensor-core
    Gram with its tensor FLOPs (8 nf nb^2 M per product, three products for
    bf16x3) against the sustained BF16 rate, the SIMT Gram / modes with their
    FP32 FLOPs, and the eigen-solver with its FP64 FLOPs against the nominal
    FP64 rate (it is bound by the latency of its dependent chains)."""
    hbm = peaks.get("hbm_gbs", 6800.0)
    src = "MEASURED_PEAKS.json hbm_gbs" if "hbm_gbs" in peaks else "fallback 6800 GB/s"
    t = per_launch_ms * 1e-3
    kern = KERNELS.get(phase, phase)
    if isinstance(kern, dict):
        kern = kern[precision]
    if phase == "fft" and elem == 8:
        kern = "k_fft_pipe (complex input)"
    q = qhat_bytes_per_point(nb, nf, precision, folded) * M
    phi = nf * nmodes * M * (16 if precision == "fp64" else 8)
    x = NT * M * (8 if precision == "fp64" and phase == "mean" else elem)
    traffic = TRAFFIC.get((phase, precision)) if elem == 4 else None

    def alu(flops, peak, peak_src, overhead=None):
        ach = flops / t / 1e12
        r = {"bound": "alu", "kernel": kern, "achieved": round(ach, 4), "peak": round(peak, 3), "unit": "TFLOP/s",
             "frac": round(ach / peak, 4), "traffic": traffic, "peak_source": peak_src, "flops_per_launch": flops,
             "ms": round(per_launch_ms, 4)}
        if overhead is not None:
            r["overhead_bytes"] = int(overhead)
        return r

    if phase == "gram" and precision in ("bf16", "bf16x3"):
        mult = 3 if precision == "bf16x3" else 1
        flops = mult * 8.0 * nf * nb * nb * M
        p_tc = peaks.get("bf16_tflops_sustained", 1700.0)
        ach = flops / t / 1e12
        return {"bound": "tensor", "kernel": kern, "achieved": round(ach, 2), "peak": p_tc, "unit": "TFLOP/s",
                "frac": round(ach / p_tc, 4), "traffic": traffic, "flops_per_launch": flops,
                "overhead_bytes": int(q),
                "peak_source": ("MEASURED_PEAKS.json bf16_tflops_sustained" if "bf16_tflops_sustained" in peaks
                                else "fallback 1700 TFLOP/s") + " (kernel timed inside a long step)",
                "note": "overhead_bytes = the Qhat read, not credited", "ms": round(per_launch_ms, 4)}
    if phase == "gram":
        return alu(4.0 * nf * nb * (nb + 1) * M, FP32_PEAK, "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz", q)
    if phase == "modes" and precision in ("fp32", "fp64"):
        return alu(8.0 * nf * nb * nmodes * M, FP32_PEAK, "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz", q)
    if phase == "eig":
        # Householder 16/3 n^3, Q formation 16/3 n^3, V = Q Z 4 n^3, Z rotations ~6 n^3 (real flops)
        flops = (16.0 / 3 + 16.0 / 3 + 4.0 + 6.0) * nb ** 3 * nf
        r = alu(flops, FP64_PEAK, "nominal GB300 FP64 rate (context only: the kernel is bound by the latency of "
                                  "its rotation chain; the non-FP64 plans run the reduction, the chain and the Z "
                                  "rotations in double-FP32 on the FP32 pipe)")
        r["traffic"] = None
        return r
    overhead = None
    if phase == "mean":
        byts = x
    elif phase == "fft":
        byts, overhead = x, q                      # Qhat written: overhead
    elif phase == "modes":
        byts, overhead = phi, q                    # Qhat read: overhead
    else:
        byts = nf * nb * nb * 16
    ach = byts / t / 1e9
    r = {"bound": "hbm", "kernel": kern, "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
         "frac": round(ach / hbm, 4), "traffic": traffic, "peak_source": src + " (burst)",
         "bytes_per_launch": int(byts), "ms": round(per_launch_ms, 4)}
    if overhead is not None:
        r["overhead_bytes"] = int(overhead)
        r["note"] = "bytes_per_launch = algorithmic bytes; overhead_bytes = Qhat traffic, not credited"
    return r


# DRAM bytes (read + write) per launch of a phase's main kernel from one ncu
# capture on the 64 x 64 x 3 grid (M = 12 288, same nt / nfft), scaled by the
# points processed (x 32) to the full grid; the summaries are in profiles/.
# Absent entries: no capture of the current kernel version.
TRAFFIC = {
    ("fft", "bf16x3"): int((497.484032 + 923.243520) * 1e6 * 32),    # k_fft_pipe<float, 1, 32, 512> (two-pass, mean inside)
    ("gram", "bf16x3"): int((979.395584 + 19.955456) * 1e6 * 32),    # k_gram_tc<1, 40> (packed Kahan drains, rho row)
    ("modes", "bf16x3"): int((996.140800 + 908.134400) * 1e6 * 32),  # k_modes_tc<1> (rho row, scales before the wait)
    ("gram", "fp32"): int((961.185 + 24.225792) * 1e6 * 32),         # k_gram_simt<float> (quad staging)
    ("modes", "fp32"): int((1017.999 + 917.710336) * 1e6 * 32),      # k_modes_simt<float, 13>
}


def step_roofline(ms_step, M, nb, nf, nmodes, peaks, precision):
    """Whole-step roofline of the method: t_roof = max(B / BW, F_gemm / P_tc, F_fft / P_fp32)
    with B = X read once + Phi written (no Qhat round trip), against the measured step."""
    hbm = peaks.get("hbm_gbs", 6800.0) * 1e9
    s = 8 if precision == "fp64" else 4
    B = NT * M * s + nf * nmodes * M * (16 if precision == "fp64" else 8)
    f_gram = 8.0 * nf * nb * nb * M
    f_modes = 8.0 * nf * nb * nmodes * M
    mult = {"bf16x3": 3, "bf16": 1}.get(precision)
    if mult:
        p_tc = peaks.get("bf16_tflops_sustained", 1700.0) * 1e12
        t_gemm = mult * (f_gram + f_modes) / p_tc
    else:
        t_gemm = (f_gram / 2 + f_modes) / (FP32_PEAK * 1e12)
    import math
    t_fft = 2.5 * NFFT * math.log2(NFFT) * nb * M / (FP32_PEAK * 1e12)
    t_hbm = B / hbm
    t_roof = max(t_hbm, t_gemm, t_fft)
    return {"t_roof_ms": round(t_roof * 1e3, 3), "frac": round(t_roof * 1e3 / ms_step, 4),
            "t_hbm_ms": round(t_hbm * 1e3, 3), "t_gemm_ms": round(t_gemm * 1e3, 3), "t_fft_ms": round(t_fft * 1e3, 3),
            "bytes": int(B), "note": "B = X read once + Phi written; a Qhat round trip counts against the step"}


def coeffs_leg(args, rank):
    """Expansion coefficients of the leading 2 modes at 16 bins (with their
    conjugates: K = 62 real basis vectors) and the reconstruction, timed with
    CUDA events after a fit + modes of the same grid."""
    import torch
    import __graft_entry__ as g
    from paper_2309_11808_gb300 import SPOD, _lib
    from workloads import jet_like
    g.build()
    dev = torch.device("cuda", 0)
    nx, nr, nv, nt, nfft = 256, 128, 2, 4096, 256
    wl = jet_like(nx=nx, nr=nr, nvars=nv, nt=nt, nfft=nfft, seed=rank, dtype=torch.float32, device=dev)
    sp = SPOD(wl.npoints, nv, nt, nfft, nfft // 2, dtype=torch.float32, precision=args.precision, weights=wl.W)
    X = wl.X
    M = X.shape[1]
    sp.fit(X)
    nmodes, nr_, fsel = 4, 2, list(range(0, 128, 8)) + [128]
    fsel = fsel[:16]
    Phi = sp.modes(X, nmodes)
    A = torch.empty((len(fsel), nr_, nt), dtype=torch.complex128, device=dev)
    Xr = torch.empty_like(X)
    st = torch.cuda.current_stream()

    def call():
        _lib.spod_coeffs(sp.handle, X, Phi, nmodes, nr_, fsel, A, st)
        _lib.spod_reconstruct(sp.handle, Phi, nmodes, nr_, fsel, A, Xr, st)
    for _ in range(max(3, args.warmup)):
        call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        call()
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    K = sum(nr_ * (1 if f in (0, nfft // 2) else 2) for f in fsel)
    flops = 2.0 * K * nt * M * 2 + 2.0 * K * K * M            # the two GEMMs and the basis Gram
    rel = float((Xr - X).float().pow(2).sum() / (X - X.mean(0)).float().pow(2).sum())
    line = {"metric": "SPOD expansion coefficients + reconstruction, ms per call", "value": round(ms, 3),
            "unit": "ms", "higher_is_better": False, "steps": args.steps, "warmup": max(3, args.warmup),
            "config": {"workload": f"jet-shaped {nx}x{nr}x{nv}, nt={nt}, nfft={nfft}", "M": M, "nt": nt,
                       "modes_per_bin": nr_, "bins": fsel, "real_basis_vectors": K, "fit_precision": args.precision,
                       "gemm": "library SIMT GEMM (k_gemm_simt), FP32; split over the points, parts summed in FP64"},
            "roofline": {"bound": "alu", "achieved": round(flops / (ms * 1e-3) / 1e12, 3), "peak": round(FP32_PEAK, 1),
                         "unit": "TFLOP/s", "frac": round(flops / (ms * 1e-3) / 1e12 / FP32_PEAK, 4),
                         "flops": flops},
            "relative_residual_energy": round(rel, 5)}
    print(json.dumps(line), flush=True)
    sp.close()


def backward_leg(args, rank):
    """spod_backward after one fit, timed with CUDA events on the launching
    stream, on two workloads: the headline jet grid with dL/dlambda = 1 for
    every eigenvalue (the loss sum_f tr M_f), and the differentiation workload
    (256 x 128 grid, 2 variables, nt = 4096, nfft = 256, cos-latitude weights)
    with the loss sum over bins 5..40 of lambda_1 + lambda_2.  The roofline is
    on the adjoint's algorithmic bytes, X read once and dL/dX written once."""
    import torch
    import __graft_entry__ as g
    from paper_2309_11808_gb300 import SPOD, _lib
    from workloads import diff_like, jet_like
    g.build()
    dev = torch.device("cuda", 0)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except OSError:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    runs = []
    for name in ("jet", "diff"):
        if name == "jet":
            wl = jet_like(nx=NX, nr=NR, nvars=NVARS, nt=NT, nfft=NFFT, seed=rank, dtype=torch.float32, device=dev)
            desc = f"jet-shaped {NX}x{NR}x{NVARS}, nt={NT}, nfft={NFFT}, 50% overlap"
        else:
            wl = diff_like(seed=rank, dtype=torch.float32, device=dev)
            desc = f"differentiation 256x128x2, nt={wl.nt}, nfft={wl.nfft}, 50% overlap, cos-latitude weights"
        X = wl.X
        M = X.shape[1]
        sp = SPOD(wl.npoints, wl.nvars, wl.nt, wl.nfft, wl.noverlap, dtype=torch.float32, precision=args.precision,
                  weights=wl.W)
        sp.fit(X)
        sp.eigs()                                   # the fit's status before timing
        nb, nf = sp.nb, sp.nf
        gl = torch.zeros((nf, nb), dtype=torch.float64, device=dev)
        if name == "jet":
            gl += 1.0
            loss = "sum of all eigenvalues (dL/dlambda = 1)"
        else:
            gl[5:41, :2] = 1.0
            loss = "sum over bins 5..40 of lambda_1 + lambda_2"
        dX = torch.empty(X.shape, dtype=torch.float64 if args.precision == "fp64" else torch.float32, device=dev)
        st = torch.cuda.current_stream()
        for _ in range(max(3, args.warmup)):
            _lib.spod_backward(sp.handle, gl, X, dX, st)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(args.steps):
            _lib.spod_backward(sp.handle, gl, X, dX, st)
        e1.record(st)
        torch.cuda.synchronize()
        _lib.spod_sync(sp.handle, st)
        ms = e0.elapsed_time(e1) / args.steps
        byts = wl.nt * M * X.element_size() + wl.nt * M * dX.element_size()
        ach = byts / (ms * 1e-3) / 1e9
        resident = sp.info.chunk_points >= M        # one spatial chunk: the fit's Qhat is reused
        runs.append({"workload": desc, "loss": loss, "nb": nb, "nf": nf, "ms_per_call": round(ms, 3),
                     "qhat": "resident from the fit" if resident else "recomputed per chunk",
                     "roofline": {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
                                  "frac": round(ach / hbm, 4), "bytes_per_call": int(byts),
                                  "note": "X read + dL/dX written (algorithmic); the Qhat and R traffic of "
                                          "this implementation is not credited"},
                     "finite": bool(torch.isfinite(dX).all())})
        sp.close()
        del wl, X, dX
        torch.cuda.empty_cache()
    line = {"metric": "SPOD adjoint (spod_backward) ms per call", "value": runs[0]["ms_per_call"], "unit": "ms",
            "higher_is_better": False, "steps": args.steps, "warmup": max(3, args.warmup),
            "config": {"workload": runs[0]["workload"], "precision": args.precision}, "runs": runs}
    print(json.dumps(line), flush=True)


def batch_leg(args, rank):
    """spod_fit_batch over the six ERA5-shaped one-year datasets (lat-lon grids
    181 x 360, 361 x 720 (x 2), 721 x 1440 (x 3), 2 variables, nt 2920 / 4380 /
    8760, nfft 256 / 384 / 512 / 720, cos-latitude weights): all inputs
    resident in HBM (162 GB FP32), one CUDA-graph launch fits all six (a
    branch per dataset); each plan's Qhat chunk is bounded so that the six
    workspaces fit beside the inputs.  Timed with CUDA events over graph
    launches after a capture and warm-up; the same datasets fitted one after
    another with spod_fit for comparison.  Metric: snapshot-GB/s over the six
    datasets (their FP32 bytes / time per launch)."""
    import torch
    import __graft_entry__ as g
    from paper_2309_11808_gb300 import SPOD, _lib
    from workloads import geo_datasets, geo_like
    g.build()
    dev = torch.device("cuda", 0)
    wls = []
    for i, ((nla, nlo), nt, nfft) in enumerate(geo_datasets()):
        wls.append(geo_like(nla, nlo, nt, nfft, seed=60 + i, dtype=torch.float32, device=dev))
    total = sum(w.X.numel() * 4 for w in wls)
    st = torch.cuda.current_stream()
    out = {}
    for prec in ("bf16x3", "fp32"):
        free = torch.cuda.mem_get_info()[0]
        budget = max(1 << 30, int(free * 0.8) // 6)          # Qhat bytes per plan
        sps = []
        for wl in wls:
            nb = (wl.nt - wl.noverlap) // (wl.nfft - wl.noverlap)
            per_pt = (wl.nfft // 2 + 1) * 2 * nb * 4
            chunk = max(64, min(wl.X.shape[1], budget // per_pt) // 64 * 64)
            sps.append(SPOD(wl.npoints, wl.nvars, wl.nt, wl.nfft, wl.noverlap, precision=prec, weights=wl.W,
                            chunk_points=chunk))
        handles = [sp.handle for sp in sps]
        Xs = [wl.X for wl in wls]
        for _ in range(max(3, args.warmup)):
            _lib.spod_fit_batch(handles, Xs, st)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(args.steps):
            _lib.spod_fit_batch(handles, Xs, st)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        for sp in sps:
            sp.eigs()                                          # status of every dataset
        # the same fits one after another
        e0.record(st)
        for sp, X in zip(sps, Xs):
            _lib.spod_fit(sp.handle, X, st)
        e1.record(st)
        torch.cuda.synchronize()
        ms_serial = e0.elapsed_time(e1)
        out[prec] = {"ms_per_launch": round(ms, 2), "value": round(total / (ms * 1e-3) / 1e9, 2),
                     "serial_ms": round(ms_serial, 2),
                     "chunks": [int(sp.info.chunk_points) for sp in sps],
                     "workspace_GB": round(sum(sp.info.workspace_bytes for sp in sps) / 1e9, 2)}
        for sp in sps:
            sp.close()
        torch.cuda.empty_cache()
    line = {"metric": "SPOD snapshot-GB/s over six ERA5-shaped datasets in one graph launch (fit)",
            "value": out["bf16x3"]["value"], "unit": "GB/s", "higher_is_better": True, "steps": args.steps,
            "warmup": max(3, args.warmup), "dtype": "bf16x3",
            "data": "synthetic (seeded AR(1) red noise + planted annual and diurnal-bin patterns)",
            "config": {"workload": "six one-year lat-lon records: " + ", ".join(
                f"{nla}x{nlo}x2 nt={nt} nfft={nfft}" for (nla, nlo), nt, nfft in geo_datasets()),
                "input_GB": round(total / 1e9, 1), "weights": "cos(latitude)"},
            "bf16x3": out["bf16x3"], "fp32": out["fp32"],
            "speedup_vs_fp32": round(out["fp32"]["ms_per_launch"] / out["bf16x3"]["ms_per_launch"], 3)}
    print(json.dumps(line), flush=True)


def ooc_leg(args, rank):
    """The out-of-core run on the headline grid: X (pinned host) is read in
    column tiles, the modes of every bin written back in tiles; the plan's Qhat
    chunk is one tile, so the device holds the plan's workspace and four tile
    buffers, not X, Qhat or Phi.  Wall-clock per call (the call synchronises)."""
    import torch
    import __graft_entry__ as g
    from paper_2309_11808_gb300 import SPOD, _lib
    from workloads import jet_like
    g.build()
    dev = torch.device("cuda", 0)
    wl = jet_like(nx=NX, nr=NR, nvars=NVARS, nt=NT, nfft=NFFT, seed=rank, dtype=torch.float32, device=dev)
    M = wl.X.shape[1]
    hX = torch.empty(wl.X.shape, dtype=torch.float32, pin_memory=True)
    hX.copy_(wl.X)
    W = wl.W.cpu()
    del wl
    torch.cuda.empty_cache()
    lines = []
    for ntile in (4, 8):
        tile = (M // ntile + 63) // 64 * 64
        sp = SPOD(NX * NR, NVARS, NT, NFFT, NOVERLAP, dtype=torch.float32, precision=args.precision, weights=W,
                  chunk_points=tile)
        nmodes = sp.nb
        cdt = torch.complex128 if args.precision == "fp64" else torch.complex64
        hPhi = torch.empty((sp.nf, nmodes, M), dtype=cdt, pin_memory=True)
        hlam = torch.empty((sp.nf, sp.nb), dtype=torch.float64, pin_memory=True)
        for _ in range(max(3, args.warmup)):
            _lib.spod_run_host_ooc(sp.handle, hX, nmodes, hPhi, hlam, tile)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            _lib.spod_run_host_ooc(sp.handle, hX, nmodes, hPhi, hlam, tile)
        dt = (time.perf_counter() - t0) / args.steps
        eb = hPhi.element_size()
        tiles_b = 2 * NT * tile * 4 + 2 * sp.nf * nmodes * tile * eb
        lines.append({"tile_points": tile, "tiles": (M + tile - 1) // tile, "ms_per_call": round(dt * 1e3, 2),
                      "GB_per_s": round(NT * M * 4 / dt / 1e9, 2),
                      "host_link_GB_per_s": round((2 * NT * M * 4 + hPhi.numel() * eb) / dt / 1e9, 1),
                      "device_bytes": int(sp.info.workspace_bytes + tiles_b),
                      "X_plus_Phi_bytes": int(NT * M * 4 + hPhi.numel() * eb)})
        sp.close()
        del hPhi
    line = {"metric": "SPOD out-of-core run (fit + all modes, host data), ms per call",
            "value": min(x["ms_per_call"] for x in lines), "unit": "ms", "higher_is_better": False,
            "steps": args.steps, "warmup": max(3, args.warmup),
            "config": {"workload": f"jet-shaped {NX}x{NR}x{NVARS}, nt={NT}, nfft={NFFT}, 50% overlap",
                       "precision": args.precision, "X": "pinned host memory", "Phi": "pinned host memory"},
            "runs": lines}
    print(json.dumps(line), flush=True)


def e2e_leg(sp, X, nmodes, args, world):
    import torch
    from paper_2309_11808_gb300 import _lib
    hX = torch.empty(X.shape, dtype=X.dtype, pin_memory=True)
    hX.copy_(X)
    cdt = np.complex128 if args.precision == "fp64" else np.complex64
    hPhi = torch.empty((sp.nf, nmodes, sp.M), dtype=torch.complex64 if cdt == np.complex64 else torch.complex128,
                       pin_memory=True)
    hlam = torch.empty((sp.nf, sp.nb), dtype=torch.float64, pin_memory=True)
    # the public host entry over the run's K timed steps (at least 2): each
    # step copies its X up and its modes and eigenvalues down (pinned host
    # buffers); step i + 1's upload overlaps step i's download
    # (spod_run_host_many)
    reps = max(2, args.steps)
    _lib.spod_run_host_many(sp.handle, [hX] * 2, nmodes, [hPhi] * 2, [hlam] * 2)   # warm-up (allocates staging)
    t0 = time.perf_counter()
    _lib.spod_run_host_many(sp.handle, [hX] * reps, nmodes, [hPhi] * reps, [hlam] * reps)
    dt = (time.perf_counter() - t0) / reps
    t1 = time.perf_counter()
    _lib.spod_run_host(sp.handle, hX, nmodes, hPhi, hlam)
    dt1 = time.perf_counter() - t1
    h2d = X.numel() * X.element_size()
    d2h = hPhi.numel() * hPhi.element_size() + hlam.numel() * hlam.element_size()
    return {"value": round(world * NT * sp.M * 4 / dt / 1e9, 3), "unit": "GB/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": round(dt * 1e3, 2), "steps_per_call": reps,
            "single_call_ms": round(dt1 * 1e3, 2)}


def reference_leg(args, world, rank):
    """The FP64 oracle, as it stands, timed on the host cores on the same
    bounded sample of the jet-shaped workload as the ``cpu_baseline`` leg:
    CPU_SAMPLE of the grid's spatial columns (spread evenly over it), all nt
    snapshots, fit + all modes per step.  The workload is generated with the
    same seeded generator as the native arm, on the GPU when there is one (on
    the host, 15.7 GB of it would take minutes), and only the sampled columns
    are copied to the host; the oracle itself runs on the host alone.  Under
    torchrun rank 0 alone runs and prints."""
    import torch
    from workloads import jet_like
    if rank != 0:
        return
    nx, nr = (64, 64) if args.small else (NX, NR)
    dev = "cuda:0" if torch.cuda.is_available() else "cpu"
    wl = jet_like(nx=nx, nr=nr, nvars=NVARS, nt=NT, nfft=NFFT, seed=0, dtype=torch.float32, device=dev)
    M = wl.X.shape[1]
    cols, idx = sample_columns(wl.X, min(CPU_SAMPLE, M))
    W = wl.W.numpy()[idx]
    del wl
    if dev != "cpu":
        torch.cuda.empty_cache()
    P = cols.shape[1]
    nb = (NT - NOVERLAP) // (NFFT - NOVERLAP)
    for _ in range(max(3, args.warmup)):
        oracle_sample(cols, W, nb)
    times = [oracle_sample(cols, W, nb) for _ in range(args.steps)]
    ms = 1e3 * sum(times) / len(times)
    val = NT * P * 4 / (ms * 1e-3) / 1e9
    sample = (f"{P} of {M} spatial columns (evenly spread) x all {NT} snapshots of the jet-shaped workload "
              f"per step, fit + {nb} modes, numpy FFT step (oracle mode 'fft'); the same sample as cpu_baseline")
    cfg = workload_config(args, nb, NFFT // 2 + 1, nb)
    cfg["sample"] = sample
    if args.small:
        cfg["workload"] += f" (reduced {nx}x{nr} grid)"
    line = {"impl": "reference", "metric": "SPOD snapshot-GB/s (FFT+CSD+eig+modes)", "value": round(val, 5),
            "unit": "GB/s", "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup),
            "ms_per_step": round(ms, 2), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic (seeded jet-shaped wave packets + AR(1) red noise)",
            "config": cfg,
            "cpu_baseline": {"kind": "oracle", "cores": cpu_cores(), "sample": sample, "value": round(val, 5)},
            "e2e": {"value": round(val, 5), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
