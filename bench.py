"""Throughput of the SPOD hot path on the jet-shaped workload.

One step = fit (mean, blocks, window, FFT, weighted Gram, reduction, FP64
eigen-decomposition) + all modes, over X resident in HBM:
X = 512 x 256 grid x 3 variables, nt = 10 000 FP32 snapshots (15.7 GB),
nfft = 512, 50 % overlap (nb = 38), Hamming window, weights ~ r.
Metric: snapshot-GB/s = nt * M * sizeof(element) / (time per step).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32]
                    [--impl native|reference]

N > 1 (torchrun): every rank runs its own full replica of the workload (no
collective on the data path); value = units of all ranks / max-over-ranks time.
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


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16x3", "bf16", "fp64"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--small", action="store_true", help="a reduced grid for quick checks (not a bench value)")
    return ap.parse_args()


def workload_config(args, nb, nf, nmodes):
    return {"workload": f"jet-shaped {NX}x{NR}x{NVARS}, nt={NT}, nfft={NFFT}, 50% overlap",
            "npoints": NX * NR, "nvars": NVARS, "M": NX * NR * NVARS, "nt": NT, "nfft": NFFT,
            "noverlap": NOVERLAP, "nb": nb, "nf": nf, "nmodes": nmodes, "in_dtype": "f32",
            "precision": args.precision, "window": "hamming", "weights": "r-weighted",
            "l2": "inputs larger than L2 (15.7 GB per step)"}


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
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) >= 9:
                for i, n in enumerate(names):
                    if r[5 + i].lower().startswith("active"):
                        reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


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
    args = parse()
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if args.impl == "reference":
        return reference_leg(args, world, rank)

    import __graft_entry__ as g
    from paper_2309_11808_gb300 import SPOD, _lib
    from workloads import jet_like

    g.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    nx, nr = (64, 64) if args.small else (NX, NR)
    wl = jet_like(nx=nx, nr=nr, nvars=NVARS, nt=NT, nfft=NFFT, seed=rank, dtype=torch.float32, device=dev)
    X = wl.X
    M = X.shape[1]
    sp = SPOD(wl.npoints, NVARS, NT, NFFT, NOVERLAP, dtype=torch.float32, precision=args.precision,
              weights=wl.W)
    nb, nf = sp.nb, sp.nf
    nmodes = nb
    cdt = torch.complex128 if args.precision == "fp64" else torch.complex64
    Phi = torch.empty((nf, nmodes, M), dtype=cdt, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        _lib.spod_fit(sp.handle, X, stream)
        _lib.spod_modes(sp.handle, X, nmodes, Phi, stream)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    _lib.spod_profile_read(sp.handle)          # discard warm-up
    _lib.spod_profile_enable(sp.handle, True)
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms_total = e0.elapsed_time(e1)
    phase_ms, phase_launch = _lib.spod_profile_read(sp.handle)
    _lib.spod_profile_enable(sp.handle, False)
    _lib.spod_sync(sp.handle, stream)
    if world > 1:
        t = torch.tensor([ms_total], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
    ms_step = ms_total / args.steps
    elem = 4
    bytes_step = NT * M * elem
    value = world * bytes_step / (ms_step * 1e-3) / 1e9

    # ---- roofline of the dominant kernel (phase with the largest time)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except OSError:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    fp32_peak = 152 * 128 * 2 * 2.070e9 / 1e12       # TFLOP/s: SMs x FP32 lanes x FMA x max clock
    dom = max(phase_ms, key=phase_ms.get)
    per_launch_ms = phase_ms[dom] / max(1, phase_launch[dom] if dom != "modes" else phase_launch[dom] // 2)
    roof = roofline(dom, per_launch_ms, M, nb, nf, nmodes, hbm_peak, fp32_peak, args.precision)

    line = {"metric": "SPOD snapshot-GB/s (FFT+CSD+eig+modes)", "value": round(value, 3), "unit": "GB/s",
            "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup),
            "ms_per_step": round(ms_step, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.precision != "fp64" else "f64",
            "data": "synthetic (seeded jet-shaped wave packets + AR(1) red noise)",
            "config": workload_config(args, nb, nf, nmodes), "roofline": roof,
            "phases_ms_per_step": {k: round(v / args.steps, 4) for k, v in phase_ms.items()},
            "gpu_launches": int(sum(phase_launch.values())), "clocks": clk,
            "snapshots_per_s": round(world * NT / (ms_step * 1e-3), 1)}

    # ---- end to end through the C ABI with host buffers
    if not args.no_e2e and rank == 0 and not args.small:
        line["e2e"] = e2e_leg(sp, X, nmodes, args, world)
    # ---- CPU oracle on a bounded sample
    if not args.no_cpu and rank == 0 and world == 1:
        P = 1024
        cols, idx = sample_columns(X, P)
        secs = oracle_sample(cols, wl.W.numpy()[idx], nmodes)
        line["cpu_baseline"] = {"value": round(NT * cols.shape[1] * elem / secs / 1e9, 5), "unit": "GB/s",
                                "cores": cpu_cores(), "kind": "oracle",
                                "sample": f"{cols.shape[1]} of {M} spatial columns, all {NT} snapshots, "
                                          f"fit + {nmodes} modes, numpy FFT step (oracle mode 'fft')",
                                "seconds": round(secs, 2)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    sp.close()
    if world > 1:
        dist.destroy_process_group()


def roofline(dom, per_launch_ms, M, nb, nf, nmodes, hbm_peak, fp32_peak, precision):
    """Algorithmic bytes / flops of one launch of the dominant phase's kernel."""
    R = 8 if precision == "fp64" else 4
    t = per_launch_ms * 1e-3
    if dom == "gram":
        flops = 4.0 * nf * nb * (nb + 1) * M            # Hermitian half of Q^H Q (complex MACs x 8 / 2)
        ach = flops / t / 1e12
        return {"bound": "alu", "kernel": "k_gram_simt", "achieved": round(ach, 3), "peak": round(fp32_peak, 1),
                "unit": "TFLOP/s", "frac": round(ach / fp32_peak, 4), "traffic": None,
                "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"}
    if dom == "modes":
        flops = 8.0 * nf * nb * nmodes * M
        ach = flops / t / 1e12
        return {"bound": "alu", "kernel": "k_modes_simt", "achieved": round(ach, 3), "peak": round(fp32_peak, 1),
                "unit": "TFLOP/s", "frac": round(ach / fp32_peak, 4), "traffic": None,
                "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"}
    if dom == "fft":
        byts = NT * M * 4 + nf * 2 * nb * M * R          # X read once + Qhat written
    elif dom == "mean":
        byts = NT * M * 4
    else:
        byts = nf * nb * nb * 16
    ach = byts / t / 1e9
    return {"bound": "hbm", "kernel": dom, "achieved": round(ach, 1), "peak": hbm_peak, "unit": "GB/s",
            "frac": round(ach / hbm_peak, 4), "traffic": None, "peak_source": "MEASURED_PEAKS.json hbm_gbs (burst)"}


def e2e_leg(sp, X, nmodes, args, world):
    import torch
    from paper_2309_11808_gb300 import _lib
    hX = torch.empty(X.shape, dtype=X.dtype, pin_memory=True)
    hX.copy_(X)
    cdt = np.complex128 if args.precision == "fp64" else np.complex64
    hPhi = torch.empty((sp.nf, nmodes, sp.M), dtype=torch.complex64 if cdt == np.complex64 else torch.complex128,
                       pin_memory=True)
    hlam = np.empty((sp.nf, sp.nb), dtype=np.float64)
    _lib.spod_run_host(sp.handle, hX, nmodes, hPhi, hlam)       # warm-up (allocates staging)
    reps = 2
    t0 = time.perf_counter()
    for _ in range(reps):
        _lib.spod_run_host(sp.handle, hX, nmodes, hPhi, hlam)
    dt = (time.perf_counter() - t0) / reps
    h2d = X.numel() * X.element_size()
    d2h = hPhi.numel() * hPhi.element_size() + hlam.nbytes
    return {"value": round(world * NT * sp.M * 4 / dt / 1e9, 3), "unit": "GB/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": round(dt * 1e3, 2)}


def reference_leg(args, world, rank):
    """The FP64 oracle timed on host cores on a bounded sample per step."""
    import torch
    from workloads import jet_like
    if rank != 0:
        return
    P = 512
    wl = jet_like(nx=32, nr=16, nvars=1, nt=NT, nfft=NFFT, seed=0, dtype=torch.float32)
    cols = wl.X[:, :P].double().numpy()
    W = wl.W.numpy()[:P]
    nb = (NT - NOVERLAP) // (NFFT - NOVERLAP)
    for _ in range(max(3, args.warmup)):
        oracle_sample(cols, W, nb)
    times = [oracle_sample(cols, W, nb) for _ in range(args.steps)]
    ms = 1e3 * sum(times) / len(times)
    val = NT * P * 4 / (ms * 1e-3) / 1e9
    sample = f"{P} spatial columns x {NT} snapshots of the jet-shaped workload per step, fit + {nb} modes"
    line = {"impl": "reference", "metric": "SPOD snapshot-GB/s (FFT+CSD+eig+modes)", "value": round(val, 5),
            "unit": "GB/s", "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup),
            "ms_per_step": round(ms, 2), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic (seeded jet-shaped)",
            "config": workload_config(args, nb, NFFT // 2 + 1, nb),
            "cpu_baseline": {"kind": "oracle", "cores": cpu_cores(), "sample": sample, "value": round(val, 5)},
            "e2e": {"value": round(val, 5), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
