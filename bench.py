#!/usr/bin/env python3
"""LSQML epoch throughput on GB300 (patterns/s), with roofline, CPU-oracle and
end-to-end figures, printed as one JSON line by rank 0.

A step is one LSQML epoch over the whole synthetic workload: for every
minibatch, the fused per-position pass (sub-pixel patch, probe modes, 2-D FFT,
intensity, data term, exit-wave change, inverse FFT, object/illumination
scatter), the probe reductions, the per-position FP64 step sizes and the
object/probe update. The default workload is the paper-shaped spiral case:
probe 128 x 128 with 5 Hermite-Gaussian modes, object 1024 x 1024, 4096
Fermat-spiral positions, minibatch 256, Poisson counts (1e6 per pattern).

--impl reference times the FP64 numpy oracle on host cores on a bounded
sample of the same workload (the reference arm; the paper's own code is not
available). With torchrun (N > 1) every rank runs an independent replica of
the workload (the path has no exchange step on one GPU): weak scaling.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "patterns/s per LSQML epoch (fwd+adjoint) vs plain FP32 at matched error"
UNIT = "patterns/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
FP32_LANES = 128   # FP32 lanes per SM; the ALU peak is SMs x lanes x 2 flop x the maximum SM clock


def alu_peak(dev):
    """Derived FP32 ALU peak (TFLOP/s) of `dev`: its SM count (queried) x 128
    lanes x 2 flop x its maximum SM clock (nvidia-smi's clocks.max.sm, else the
    measured maximum in MEASURED_PEAKS.json, else 2.07 GHz)."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    ghz, src = None, None
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(dev.index or 0), "--query-gpu=clocks.max.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=20)
        ghz, src = float(out.stdout.strip().splitlines()[0]) / 1e3, "nvidia-smi clocks.max.sm"
    except Exception:
        try:
            with open(PEAKS_FILE) as f:
                ghz, src = float(json.load(f)["sm_max_mhz"]) / 1e3, "MEASURED_PEAKS sm_max_mhz"
        except Exception:
            ghz, src = 2.07, "nominal"
    return sms * FP32_LANES * 2 * ghz * 1e-3, f"{sms} SM x {FP32_LANES} FP32 lanes x 2 flop x {ghz:.3f} GHz ({src}; derived)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["spiral128", "raster64", "uneven16", "uneven16opr", "spiral256", "multislice256",
                                           "multislice256-lsqml"], default="spiral128")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the FP32 vs split-BF16 comparison at matched reconstruction error")
    ap.add_argument("--precision", choices=["fp32", "bf16x3"], default="fp32",
                    help="far-field arithmetic of the timed epochs: FP32 FFTs or split-BF16 DFT-GEMMs")
    ap.add_argument("--ms-backward", choices=["recompute", "keep"], default="recompute",
                    help="multislice workloads: incident waves recomputed in the backward pass, or kept by the "
                         "forward pass (the other design is timed beside it unless --no-compare)")
    ap.add_argument("--variants", default="",
                    help="pin the kernel variants (pass1,pass2,probe_reduce, e.g. 0,0,1) instead of autotuning them: "
                         "profiling runs, where the autotuner's timings are distorted")
    ap.add_argument("--positions", type=int, default=0,
                    help="use only the first J positions of the workload (profiling runs)")
    return ap.parse_args()


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


FALLBACK_BF16_SUSTAINED = 1700.0


def bf16_peak():
    """Sustained dense BF16 tensor peak (TFLOP/s): the DFT-GEMM kernel runs inside a long step."""
    try:
        with open(PEAKS_FILE) as f:
            return float(json.load(f)["bf16_tflops_sustained"]), "measured (sustained bf16)"
    except Exception:
        return FALLBACK_BF16_SUSTAINED, "fallback (sustained bf16)"


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_pass1_traffic.txt")
PROFILE_EVERY = 5   # timed epochs between two whose dominant-kernel launches carry CUDA events
KERNEL_SOURCES = ["common.cuh", "fft.cuh", "kernels.cuh", "tc.cuh", "kernels_cluster.cuh", "pass_n128.cu", "api.cu"]


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in sorted(KERNEL_SOURCES):
        with open(os.path.join(ROOT, "paper_2510_20929_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel):
    """ncu DRAM bytes per launch recorded for `kernel`, or None if the kernel
    sources changed since the capture (or no capture is recorded)."""
    try:
        cur = kernel_source_hash()
        for line in open(TRAFFIC_FILE):
            f = line.split()
            if len(f) >= 6 and f[0] == "kernel" and f[1] == kernel and f[3] == cur:
                return float(f[5])
    except OSError:
        pass
    return None


def make_workload(name, positions=0):
    from paper_2510_20929_gb300 import synth
    w = synth.workload_spiral128() if name == "spiral128" else synth.workload_raster64()
    if positions and positions < w["J"]:
        w["pos"] = w["pos"][:positions]
        if w["counts_per"] == "all":
            w["total_counts"] *= positions / w["J"]
        w["J"] = positions
        w["name"] += f"-first{positions}"
    return w


def counts_total(w):
    return w["total_counts"] * (w["J"] if w["counts_per"] == "pattern" else 1)


# ----------------------------------------------------------------------------- algorithmic work
def pass1_work(N, M, B):
    """Per-launch algorithmic FLOPs and HBM bytes of the fused per-position pass.

    FLOPs: the forward and inverse 2-D FFT of every mode, 5 N^2 log2(N^2) each.
    Bytes: measured intensities read (4 N^2), the object tile read ((N+1)^2 x 8),
    the stored patch, g and h planes written ((2 + M) N^2 x 8) and the
    (dO, illum) accumulator read-modify-write ((N+1)^2 x 16 x 2).
    """
    flops = B * 2 * M * 5 * N * N * math.log2(N * N)
    nbytes = B * (4 * N * N + 8 * (N + 1) ** 2 + 8 * (2 + M) * N * N + 32 * (N + 1) ** 2)
    return flops, nbytes


def far_tc_work(N, M, B):
    """Per-launch tensor FLOPs of the split-BF16 DFT-GEMM far-field stage.

    Each 2-D transform is two passes of four real 128 x N x N GEMMs (the DFT
    operand has 128 rows, zero beyond N), each with three split terms; a
    position takes M forward and M inverse transforms.
    """
    per_transform = 2 * 4 * 3 * 2 * 128 * N * N
    return B * 2 * M * per_transform


# ----------------------------------------------------------------------------- clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        import tempfile
        try:
            fd, self.path = tempfile.mkstemp(prefix=f"ptycho_clocks_rank{self.index}_", suffix=".csv")
            self.f = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            lines = f.readlines()
        try:
            os.remove(self.path)
        except OSError:
            pass
        for line in lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- CPU oracle
# The amplitude data term's eps: one count. With a vanishing eps the modulus
# projection is ill-conditioned at dark predicted pixels that hold counts
# (from the flat start an FP32-sized perturbation of the probe moves the FP64
# oracle's spiral128 epoch by 1.7e-3); at one count it stays near 1e-7.
EPS = 1.0


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), or the machine type."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine()


def oracle_sample(w, nbatch, batch, seed=5):
    """Time the FP64 oracle on `nbatch` minibatches of the workload (its own
    intensities, Poisson-sampled from the oracle's forward model of the true
    object): returns (patterns/s, seconds of LSQML minibatch work)."""
    from oracle import ptycho_oracle as orc
    from paper_2510_20929_gb300 import synth
    order = synth.random_order(w["J"], seed)
    idx = order[: nbatch * batch]
    pos = w["pos"][idx]
    P = w["probe"]
    I = orc.forward(w["object"], P, pos)
    scale = counts_total(w) / (w["J"] * I.sum(axis=(1, 2)).mean())
    Im = synth.poisson_counts(I * scale, seed)
    P = P * math.sqrt(scale)
    O = __import__("numpy").ones_like(w["object"])
    opts = orc.LsqmlOptions(batch=batch, delta_o=0.1, delta_p=0.1, lam=1e-6, eps=EPS)
    t0 = time.perf_counter()
    for b0 in range(0, len(idx), batch):   # (a workload smaller than the sample has fewer minibatches)
        O, P, _, _ = orc.lsqml_batch(O, P, pos, Im, range(b0, min(b0 + batch, len(idx))), opts)
    dt = time.perf_counter() - t0
    return len(idx) / dt, dt


def _oracle_worker(name, positions, nbatch, batch, seed, barrier, queue):
    """One process of the all-cores leg: builds its sample, waits for the others, times it."""
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    w = make_workload(name, positions)
    barrier.wait()
    t0 = time.perf_counter()
    v, dt = oracle_sample(w, nbatch, batch, seed)
    queue.put((t0, t0 + dt, v * dt))


def oracle_all_cores(name, positions, nbatch, batch, procs):
    """The oracle on every host core: `procs` processes (spawned) each run
    `nbatch` minibatches of their own sample of the workload at the same time;
    throughput = all their positions over the span from the first start to the
    last finish. Minibatches of one epoch depend on each other, so this is an
    upper bound of what a split of each minibatch's positions over the cores
    (with a reduction of the accumulators) could reach."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    barrier, queue = ctx.Barrier(procs), ctx.Queue()
    ps = [ctx.Process(target=_oracle_worker, args=(name, positions, nbatch, batch, 100 + i, barrier, queue))
          for i in range(procs)]
    for p in ps:
        p.start()
    res = [queue.get(timeout=900) for _ in ps]
    for p in ps:
        p.join(timeout=60)
    span = max(r[1] for r in res) - min(r[0] for r in res)
    return sum(r[2] for r in res) / span, span


def cpu_baseline(name, positions, w, batch):
    """Single-thread and all-cores oracle legs, with the core count and the CPU model."""
    v1, dt1 = oracle_sample(w, 2, batch)
    ncores = os.cpu_count() or 1
    out = {"value": v1, "unit": UNIT, "cores": 1, "kind": "oracle", "cpu_model": cpu_model(), "nproc": ncores,
           "sample": f"2 LSQML minibatches of {batch} positions of {w['name']} (FP64 numpy oracle, one "
                     f"thread), {dt1:.1f} s"}
    try:
        vall, span = oracle_all_cores(name, positions, 1, batch, ncores)
        out["all_cores"] = {"value": vall, "unit": UNIT, "cores": ncores, "kind": "oracle",
                            "sample": f"{ncores} spawned processes, each one LSQML minibatch of {batch} positions "
                                      f"of its own sample of {w['name']} at the same time, {span:.1f} s span "
                                      "(an upper bound of a within-minibatch split over the cores)"}
    except Exception as e:   # the single-thread figure stands on its own
        out["all_cores"] = {"unavailable": f"{type(e).__name__}: {e}"}
    return out


def run_reference(args, rank):
    if rank != 0:
        return
    w = make_workload(args.workload, args.positions)
    batch = w["batch"]
    vals = []
    for s in range(args.warmup + args.steps):
        v, dt = oracle_sample(w, 1, batch, seed=5 + s)
        if s >= args.warmup:
            vals.append((v, dt))
    value = statistics.mean(v for v, _ in vals)
    ms = 1e3 * statistics.mean(dt for _, dt in vals)
    sample = (f"1 LSQML minibatch of {batch} positions of the {w['name']} workload per step "
              f"(object {w['H']}x{w['W']}, {w['M']} modes, {w['N']}^2), FP64 numpy oracle")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["name"], "J": w["J"], "N": w["N"], "M": w["M"], "H": w["H"], "W": w["W"],
                   "batch": batch, "eps": EPS},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                         "cpu_model": cpu_model(), "nproc": os.cpu_count()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ----------------------------------------------------------------------------- multi-rank
def max_over_ranks(x, world, device="cpu"):
    """Max of a per-rank float over all ranks (the slowest replica sets the time)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return t.item()


def job_throughput(units_per_rank, world, seconds):
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return world * units_per_rank / seconds


# ----------------------------------------------------------------------------- precision comparison
COMPARE_EPOCHS = 20


def object_error(O, O_true, pos, N):
    """Phase-aligned relative object error over the scanned region (the box of
    probe centres widened by N/4): min over a global phase of ||O e^{i phi} - O_true|| / ||O_true||."""
    import torch
    lo = (pos.min(dim=0).values - N / 4).floor().clamp(min=0).long().tolist()
    hi = (pos.max(dim=0).values + N / 4).ceil().long().tolist()
    a = O[lo[0]:hi[0], lo[1]:hi[1]].to(torch.complex128)
    b = O_true[lo[0]:hi[0], lo[1]:hi[1]].to(torch.complex128)
    c = (a.conj() * b).sum()
    ph = c / c.abs() if c.abs() > 0 else 1.0
    return ((a * ph - b).norm() / b.norm()).item()


def precision_comparison(api, O_true, P, pos, meas, order, B, steps, warmup, dev):
    """FP32 FFTs against split-BF16 DFT-GEMMs on the same seeded data: COMPARE_EPOCHS
    epochs from the same start (unit object, true probe) with each precision, the
    final loss and phase-aligned object error, and each precision's epoch time
    (CUDA events around `steps` epochs after `warmup`). Matched: object errors
    within 1 % of each other."""
    import torch
    res = {}
    H, W = O_true.shape
    stream = torch.cuda.current_stream()
    for prec in ("fp32", "bf16x3"):
        opts = api.make_opts(noise="gaussian", batch=B, delta_o=0.1, delta_p=0.1, lam=1e-6, eps=EPS,
                             precision=prec)
        O = torch.ones((H, W), dtype=torch.complex64, device=dev)
        Pe = P.clone()
        loss = None
        for _ in range(COMPARE_EPOCHS):
            loss, _ = api.lsqml_epoch(O, Pe, pos, meas, order, opts, check=False)
        api.workspace(api.dims_of(O, Pe, pos), B, dev, opts=opts).status()
        err = object_error(O, O_true, pos, P.shape[-1])
        for _ in range(warmup):
            api.lsqml_epoch(O, Pe, pos, meas, order, opts, check=False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            api.lsqml_epoch(O, Pe, pos, meas, order, opts, check=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        res[prec] = {"patterns_per_s": pos.shape[0] / (ms * 1e-3), "ms_per_epoch": ms,
                     "final_loss": loss.item(), "object_error": err}
    e32, e16 = res["fp32"]["object_error"], res["bf16x3"]["object_error"]
    res.update({"epochs": COMPARE_EPOCHS,
                "speedup_bf16x3_vs_fp32": res["bf16x3"]["patterns_per_s"] / res["fp32"]["patterns_per_s"],
                "object_error_rel_diff": abs(e16 - e32) / e32,
                "matched": abs(e16 - e32) <= 0.01 * e32,
                "start": "unit object, true probe; Gaussian data term, eps %g; same order and data" % EPS})
    return res


# ----------------------------------------------------------------------------- GPU
def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2510_20929_gb300 import api, synth

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    w = make_workload(args.workload, args.positions)
    H, W, N, M, J, B = w["H"], w["W"], w["N"], w["M"], w["J"], w["batch"]
    O_true = torch.tensor(w["object"], dtype=torch.complex64, device=dev)
    P = torch.tensor(w["probe"], dtype=torch.complex64, device=dev)
    pos = torch.tensor(w["pos"], dtype=torch.float32, device=dev)
    I0 = api.forward(O_true, P, pos)
    scale = counts_total(w) / (J * I0.sum(dim=(1, 2)).mean().item())
    P *= math.sqrt(scale)
    gen = torch.Generator(device=dev)
    gen.manual_seed(1234 + rank)
    meas = torch.poisson(I0 * scale, generator=gen).contiguous()
    del I0
    order = torch.tensor(synth.random_order(J, 5 + rank), dtype=torch.int32, device=dev)
    O = torch.ones((H, W), dtype=torch.complex64, device=dev)
    P_est = P.clone()
    opts = api.make_opts(noise="gaussian", batch=B, delta_o=0.1, delta_p=0.1, lam=1e-6, eps=EPS, autotune=True,
                         precision=args.precision)
    if args.variants:   # pinned entries are not retuned
        api.set_tuning(api.Dims(H, W, N, M, J), B, *[int(v) for v in args.variants.split(",")])
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        api.lsqml_epoch(O, P_est, pos, meas, order, opts, check=False)
    api.lsqml_epoch(O, P_est, pos, meas, order, opts, check=True)   # status check outside timing
    # per-kernel breakdown (every launch bracketed by events), before and
    # outside the timed region: names the dominant kernel and the shares
    api.profile_enable(True)
    api.profile_read()
    n_prof = min(max(args.steps, 1), 10)
    for _ in range(n_prof):
        api.lsqml_epoch(O, P_est, pos, meas, order, opts, check=False)
    prof = api.profile_read()
    api.profile_enable(False)
    dom_name = max(prof.items(), key=lambda kv: kv[1][1])[0]
    launches_per_epoch = sum(n for n, _ in prof.values()) / n_prof
    # timed region: the dominant kernel's launches carry an event pair in every
    # PROFILE_EVERY-th epoch (an event record between launches costs a few us
    # of launch overlap, so the other epochs run without)
    clocks = Clocks(local_rank)
    api.profile_enable(False, only=dom_name)
    api.profile_read()
    barrier()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    losses = []
    for i in range(args.steps):
        api.profile_enable(i % PROFILE_EVERY == 0, only=dom_name)
        loss, _ = api.lsqml_epoch(O, P_est, pos, meas, order, opts, check=False)
        losses.append(loss)
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    live = api.profile_read()
    api.profile_enable(False)
    ms = ev0.elapsed_time(ev1) / args.steps
    ms_max = max_over_ranks(ms, world, dev)
    value = job_throughput(J, world, ms_max * 1e-3)
    launches = int(round(launches_per_epoch * args.steps))

    # roofline of the dominant kernel (its launches timed live in the timed region)
    dom_n, dom_ms = live.get(dom_name, (0, 0.0))
    hbm, hbm_src = peaks()
    alu_tflops, alu_src = alu_peak(dev)
    if dom_name == "k_pass1":
        flops, nbytes = pass1_work(N, M, B)
        avg_s = dom_ms / dom_n * 1e-3
        # count the ragged last batch exactly: total work over total time
        nb_list = [min(B, J - b0) for b0 in range(0, J, B)]
        tot_flops = sum(pass1_work(N, M, nb)[0] for nb in nb_list) * (dom_n // len(nb_list))
        tot_bytes = sum(pass1_work(N, M, nb)[1] for nb in nb_list) * (dom_n // len(nb_list))
        t_s = dom_ms * 1e-3
        alu_ach = tot_flops / t_s * 1e-12
        hbm_ach = tot_bytes / t_s * 1e-9
        if alu_ach / alu_tflops >= hbm_ach / hbm:
            roof = {"bound": "alu", "achieved": alu_ach, "peak": alu_tflops, "unit": "TFLOP/s",
                    "frac": alu_ach / alu_tflops, "traffic": None,
                    "peak_source": alu_src}
        else:
            roof = {"bound": "hbm", "achieved": hbm_ach, "peak": hbm, "unit": "GB/s",
                    "frac": hbm_ach / hbm, "traffic": None, "peak_source": hbm_src}
        roof.update({"kernel": dom_name, "launch_ms": avg_s * 1e3,
                     "alu_frac": alu_ach / alu_tflops, "hbm_frac": hbm_ach / hbm,
                     "algorithmic_bytes_per_launch": nbytes, "algorithmic_flops_per_launch": flops})
        if N == 128 and M == 5 and B == 256:
            roof["traffic"] = recorded_traffic("k_pass1")
    elif dom_name == "k_far_tc":
        nb_list = [min(B, J - b0) for b0 in range(0, J, B)]
        tot_flops = sum(far_tc_work(N, M, nb) for nb in nb_list) * (dom_n // len(nb_list))
        t_s = dom_ms * 1e-3
        peak, src = bf16_peak()
        ach = tot_flops / t_s * 1e-12
        roof = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": None, "peak_source": src, "kernel": dom_name, "launch_ms": dom_ms / dom_n,
                "algorithmic_flops_per_launch": far_tc_work(N, M, B)}
    else:
        roof = {"bound": "hbm", "achieved": None, "peak": hbm, "unit": "GB/s", "frac": None,
                "traffic": None, "kernel": dom_name}

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "bf16x3 (f32 accumulate)",
        "data": "synthetic",
        "config": {"workload": w["name"], "J": J, "N": N, "M": M, "H": H, "W": W, "batch": B,
                   "noise": "gaussian", "eps": EPS, "precision": args.precision, "parallelism": f"replicas{world}" if world > 1 else "single",
                   "l2": "inputs larger than L2 (measured intensities %.0f MB read every epoch)"
                         % (J * N * N * 4 / 1e6),
                   "profiler": "CUDA event pair around every launch of the dominant kernel in every %d-th "
                               "timed epoch; the per-kernel breakdown from %d profiled epochs before the timed "
                               "region" % (PROFILE_EVERY, n_prof)},
        "roofline": roof,
        "gpu_launches": launches,
        "autotune": api.tuning(api.dims_of(O, P_est, pos), B),
        "kernels": {k: {"launches": n, "ms_per_launch": ms_ / max(n, 1), "share": ms_ / sum(
            v[1] for v in prof.values())} for k, (n, ms_) in prof.items()},
        "clocks": clk,
        "final_loss": losses[-1].item() if losses else None,
    }

    if not args.no_compare and N in (32, 64, 128):
        out["precision_comparison"] = precision_comparison(api, O_true, P, pos, meas, order, B,
                                                           min(args.steps, 20), args.warmup, dev)

    # end to end through the host-buffer entry point (pinned host memory)
    if not args.no_e2e:
        hO = torch.ones((H, W), dtype=torch.complex64).pin_memory()
        hP = P.cpu().pin_memory()
        hpos = pos.cpu().pin_memory()
        hmeas = meas.cpu().pin_memory()
        horder = order.cpu().pin_memory()
        del meas
        torch.cuda.empty_cache()
        for _ in range(max(1, args.warmup)):
            api.lsqml_epoch_host(hO, hP, hpos, hmeas, horder, opts, device=dev)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            api.lsqml_epoch_host(hO, hP, hpos, hmeas, horder, opts, device=dev)
        barrier()
        dt = max_over_ranks((time.perf_counter() - t0) / args.steps, world, dev)
        h2d = hO.numel() * 8 + hP.numel() * 8 + hpos.numel() * 4 + hmeas.numel() * 4 + horder.numel() * 4
        d2h = hO.numel() * 8 + hP.numel() * 8 + 8
        out["e2e"] = {"value": job_throughput(J, world, dt), "unit": UNIT, "h2d_bytes_per_step": h2d,
                      "d2h_bytes_per_step": d2h, "ms_per_step": dt * 1e3,
                      "entry": "ptycho_lsqml_epoch_host (pinned host buffers)"}

    if rank == 0 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(args.workload, args.positions, w, B)
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_uneven(args, rank, world, local_rank, opr_K=0):
    """Batched serving of 16 uneven reconstructions (windows 64/128/192/256, J ~ U[500, 20000]):
    one epoch of every reconstruction per step, batched (with and without graph
    replay) against the same reconstructions run one after the other. With
    opr_K > 0 every reconstruction relaxes its primary probe mode over opr_K
    eigenmodes (orthogonal probe relaxation, true weights N(1, 0.1), the
    reconstruction starting from unit weights) and the step also updates the
    eigenmodes and the weights."""
    import torch
    from paper_2510_20929_gb300 import api, synth
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    ws = synth.workload_uneven(16, seed=1005 + rank, opr_K=opr_K)
    recons, opts = [], []
    gen = torch.Generator(device=dev)
    gen.manual_seed(77 + rank)
    for w in ws:
        Ot = torch.tensor(w["object"], dtype=torch.complex64, device=dev)
        pos = torch.tensor(w["pos"], dtype=torch.float32, device=dev)
        order = torch.tensor(synth.random_order(w["J"], 3), dtype=torch.int32, device=dev)
        if opr_K:
            U = torch.tensor(w["opr_U"], dtype=torch.complex64, device=dev)
            wt = torch.tensor(w["opr_w"], dtype=torch.float32, device=dev)
            I0 = api.forward_opr(Ot, U, wt, None, pos)
            scale = w["total_counts"] / I0.sum().item()
            U *= math.sqrt(scale)
            meas = torch.poisson(I0 * scale, generator=gen)
            recons.append([torch.ones_like(Ot), U, torch.ones_like(wt), None, pos, meas, order])
        else:
            P = torch.tensor(w["probe"], dtype=torch.complex64, device=dev)
            I0 = api.forward(Ot, P, pos)
            scale = w["total_counts"] / I0.sum().item()
            P *= math.sqrt(scale)
            meas = torch.poisson(I0 * scale, generator=gen)
            recons.append([torch.ones_like(Ot), P, pos, meas, order])
        del Ot, I0
    total = sum(w["J"] for w in ws)

    def timed(fn, steps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    o_eager = [api.make_opts(batch=w["batch"]) for w in ws]
    o_graph = [api.make_opts(batch=w["batch"], graph=True) for w in ws]
    if opr_K:
        oprs = api.make_opr_opts(opr_K)

        def sequential():
            for r, o in zip(recons, o_eager):
                api.lsqml_epoch_opr(*r[:6], r[6], o, oprs, check=False)

        def batched(o):
            return api.lsqml_epoch_opr_batched(recons, o, oprs, check=False)

        def checked():
            return api.lsqml_epoch_opr_batched(recons, o_graph, oprs, check=True)
    else:
        def sequential():
            for (O, P, pos, meas, order), o in zip(recons, o_eager):
                api.lsqml_epoch(O, P, pos, meas, order, o, check=False)

        def batched(o):
            return api.lsqml_epoch_batched(recons, o, check=False)

        def checked():
            return api.lsqml_epoch_batched(recons, o_graph, check=True)

    ms_seq = timed(sequential, args.steps)
    ms_b = timed(lambda: batched(o_eager), args.steps)
    ms_g = timed(lambda: batched(o_graph), args.steps)
    checked()
    # each reconstruction's epoch alone: its minibatches form a dependency chain
    # (each reads the object and probe the previous one wrote), so the longest
    # of these bounds any schedule that runs the reconstructions together
    alone = []
    for i, o in enumerate(o_eager):
        if opr_K:
            r = recons[i]
            alone.append(timed(lambda: api.lsqml_epoch_opr(*r[:6], r[6], o, oprs, check=False), 1))
        else:
            O, P, pos, meas, order = recons[i]
            alone.append(timed(lambda: api.lsqml_epoch(O, P, pos, meas, order, o, check=False), 1))
    ms_max = max_over_ranks(ms_g, world, dev)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": job_throughput(total, world, ms_max * 1e-3), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "uneven16opr" if opr_K else "uneven16", "reconstructions": len(ws),
                       "positions": total, "windows": sorted({w["N"] for w in ws}), "J": [w["J"] for w in ws],
                       "opr_eigenmodes": opr_K},
            "batched_graph_ms": ms_g, "batched_eager_ms": ms_b, "sequential_ms": ms_seq,
            "speedup_vs_sequential": ms_seq / ms_g,
            "alone_ms": alone, "longest_chain_ms": max(alone),
            "batched_over_longest_chain": ms_g / max(alone),
            # the batched epoch against the reconstructions' epochs timed one by one,
            # and where those epochs spend their time, per window size
            "sum_alone_ms": sum(alone), "batched_over_sum_alone": ms_g / sum(alone),
            "alone_ms_per_window": {str(n): sum(a for a, w in zip(alone, ws) if w["N"] == n)
                                    for n in sorted({w["N"] for w in ws})},
        }), flush=True)


def run_ad256(args, rank, world, local_rank):
    """Differentiable case: probe 256^2 with 8 modes, object 2048^2, 10,000 spiral
    positions with N(0, 1.5 px) errors; a step is one Adam step on object, probe
    and positions (fused data term forward + adjoint over all positions)."""
    import torch
    from paper_2510_20929_gb300 import api, synth
    from paper_2510_20929_gb300.autograd import data_term
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    w = synth.workload_spiral256()
    if args.positions and args.positions < w["J"]:   # profiling runs: the first positions only
        w["pos"], w["pos_init"], w["J"] = w["pos"][:args.positions], w["pos_init"][:args.positions], args.positions
    O_true = torch.tensor(w["object"], dtype=torch.complex64, device=dev)
    P = torch.tensor(w["probe"], dtype=torch.complex64, device=dev)
    pos_true = torch.tensor(w["pos"], dtype=torch.float32, device=dev)
    I0 = api.forward(O_true, P, pos_true)
    scale = w["total_counts"] / I0.sum(dim=(1, 2)).mean().item()
    P *= math.sqrt(scale)
    gen = torch.Generator(device=dev)
    gen.manual_seed(99 + rank)
    meas = torch.poisson(I0 * scale, generator=gen)
    del I0
    O = O_true.clone().requires_grad_(True)
    Pe = P.clone().requires_grad_(True)
    pos = torch.tensor(w["pos_init"], dtype=torch.float32, device=dev).requires_grad_(True)
    opt = torch.optim.Adam([{"params": [O], "lr": 1e-3}, {"params": [Pe], "lr": 1e-3},
                            {"params": [pos], "lr": 0.05}])

    def step():
        opt.zero_grad(set_to_none=True)
        loss = data_term(O, Pe, pos, meas, "gaussian", 1e-9)
        loss.backward()
        opt.step()
        return loss

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    api.profile_enable(True)
    api.profile_read()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        loss = step()
    e1.record()
    torch.cuda.synchronize()
    prof = api.profile_read()
    api.profile_enable(False)
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": job_throughput(w["J"], world, ms * 1e-3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "spiral256-adam", "J": w["J"], "N": 256, "M": 8, "H": 2048, "W": 2048,
                       "step": "one Adam step on object, probe and positions (fused data term and adjoint)"},
            "kernels": {k: {"launches": n, "ms_per_launch": t / max(n, 1)} for k, (n, t) in prof.items()},
            "final_loss": loss.item(),
        }), flush=True)


def ms_designs(args):
    """Backward designs of a multislice run: the chosen one first, then the
    other one unless --no-compare."""
    other = "keep" if args.ms_backward == "recompute" else "recompute"
    return [args.ms_backward] if args.no_compare else [args.ms_backward, other]


def ms_design_report(api, w, mss, timed, opts):
    """Per backward design: time per step, throughput, workspace bytes and
    the per-position kernel's time per launch."""
    import ctypes
    d = api.Dims(w["slices"].shape[1], w["slices"].shape[2], 256, 4, w["J"])
    out = {}
    for name, (ms_step, prof, _) in timed.items():
        m = mss[name]
        if opts is None:
            ws = api.lib().ptycho_workspace_bytes_ms(ctypes.byref(d), ctypes.byref(m), w["batch"])
        else:
            ws = api.lib().ptycho_workspace_bytes_lsqml_ms(ctypes.byref(d), ctypes.byref(m), ctypes.byref(opts))
        p1 = prof.get("k_pass1_ms", (0, 0.0))
        out[name] = {"ms_per_step": ms_step, "value": w["J"] / (ms_step * 1e-3), "workspace_bytes": int(ws),
                     "k_pass1_ms_ms_per_launch": p1[1] / max(p1[0], 1)}
    return out


def run_ms256(args, rank, world, local_rank):
    """Multislice case: 4 slices of 2048^2, probe 256^2 with 4 modes, 8000
    positions; a step is one Adam step on the slices and the probe (fused
    multislice data term and adjoint over all positions, minibatches of 512
    inside the library call)."""
    import torch
    from paper_2510_20929_gb300 import api, synth
    from paper_2510_20929_gb300.autograd import data_term_ms
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    w = synth.workload_multislice256()
    if args.positions and args.positions < w["J"]:   # profiling runs: the first positions only
        w["pos"], w["J"] = w["pos"][:args.positions], args.positions
    designs = ms_designs(args)
    mss = {d: api.make_multislice(w["S"], w["dz"], w["wavelength"], w["pixel_size"], recompute=d == "recompute")
           for d in designs}
    ms = mss[designs[0]]
    Os_true = torch.tensor(w["slices"], dtype=torch.complex64, device=dev)
    P = torch.tensor(w["probe"], dtype=torch.complex64, device=dev)
    pos = torch.tensor(w["pos"], dtype=torch.float32, device=dev)
    I0 = api.forward_ms(Os_true, P, pos, ms, batch=w["batch"])
    scale = w["total_counts"] / I0.sum(dim=(1, 2)).mean().item()
    P *= math.sqrt(scale)
    gen = torch.Generator(device=dev)
    gen.manual_seed(101 + rank)
    meas = torch.poisson(I0 * scale, generator=gen)
    del I0
    Os = torch.ones_like(Os_true).requires_grad_(True)
    Pe = P.clone().requires_grad_(True)
    opt = torch.optim.Adam([{"params": [Os], "lr": 1e-2}, {"params": [Pe], "lr": 1e-3}])

    def step(m):
        opt.zero_grad(set_to_none=True)
        loss = data_term_ms(Os, Pe, pos, meas, m, "gaussian", 1e-9, w["batch"])
        loss.backward()
        opt.step()
        return loss

    timed = {}
    for d in designs:   # the headline design first, then the other one from where it left the parameters
        for _ in range(args.warmup):
            step(mss[d])
        torch.cuda.synchronize()
        api.profile_enable(True)
        api.profile_read()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            loss = step(mss[d])
        e1.record()
        torch.cuda.synchronize()
        prof_d = api.profile_read()
        api.profile_enable(False)
        timed[d] = (max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev), prof_d, loss)
    ms_step, prof, loss = timed[designs[0]]
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": job_throughput(w["J"], world, ms_step * 1e-3), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "multislice256-adam", "J": w["J"], "N": 256, "M": 4, "S": w["S"], "H": 2048,
                       "W": 2048, "dz_m": w["dz"], "wavelength_m": w["wavelength"], "pixel_m": w["pixel_size"],
                       "batch": w["batch"],
                       "backward": designs[0],
                       "step": "one Adam step on the object slices and the probe (fused multislice data term "
                               "and adjoint)"},
            "kernels": {k: {"launches": n, "ms_per_launch": t / max(n, 1)} for k, (n, t) in prof.items()},
            "backward_designs": ms_design_report(api, w, mss, timed, None),
            "final_loss": loss.item(),
        }), flush=True)


def run_ms256_lsqml(args, rank, world, local_rank):
    """Multislice LSQML: 4 slices of 2048^2, probe 256^2 with 4 modes, 8000
    positions, minibatches of 512; a step is one LSQML epoch over all positions
    (per-slice directions and step sizes), from flat slices and the true probe."""
    import torch
    from paper_2510_20929_gb300 import api, synth
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    w = synth.workload_multislice256()
    if args.positions and args.positions < w["J"]:   # profiling runs: the first positions only
        w["pos"], w["J"] = w["pos"][:args.positions], args.positions
    designs = ms_designs(args)
    mss = {d: api.make_multislice(w["S"], w["dz"], w["wavelength"], w["pixel_size"], recompute=d == "recompute")
           for d in designs}
    ms = mss[designs[0]]
    Os_true = torch.tensor(w["slices"], dtype=torch.complex64, device=dev)
    P = torch.tensor(w["probe"], dtype=torch.complex64, device=dev)
    pos = torch.tensor(w["pos"], dtype=torch.float32, device=dev)
    I0 = api.forward_ms(Os_true, P, pos, ms, batch=w["batch"])
    scale = w["total_counts"] / I0.sum(dim=(1, 2)).mean().item()
    P *= math.sqrt(scale)
    gen = torch.Generator(device=dev)
    gen.manual_seed(103 + rank)
    meas = torch.poisson(I0 * scale, generator=gen)
    del I0, Os_true
    order = torch.tensor(synth.random_order(w["J"], 9 + rank), dtype=torch.int32, device=dev)
    opts = api.make_opts(noise="gaussian", batch=w["batch"], delta_o=0.1, delta_p=0.1, lam=1e-6, eps=EPS)
    timed = {}
    for d in designs:   # each design from flat slices and the true probe
        Os = torch.ones((w["S"],) + tuple(w["slices"].shape[1:]), dtype=torch.complex64, device=dev)
        Pe = P.clone()
        for _ in range(args.warmup):
            api.lsqml_epoch_ms(Os, Pe, pos, meas, order, mss[d], opts, check=False)
        api.lsqml_epoch_ms(Os, Pe, pos, meas, order, mss[d], opts, check=True)
        torch.cuda.synchronize()
        api.profile_enable(True)
        api.profile_read()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        losses = []
        for _ in range(args.steps):
            loss, _ = api.lsqml_epoch_ms(Os, Pe, pos, meas, order, mss[d], opts, check=False)
            losses.append(loss)
        e1.record()
        torch.cuda.synchronize()
        prof_d = api.profile_read()
        api.profile_enable(False)
        timed[d] = (max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev), prof_d, losses)
        del Os, Pe
    ms_step, prof, losses = timed[designs[0]]
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": job_throughput(w["J"], world, ms_step * 1e-3), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "multislice256-lsqml", "J": w["J"], "N": 256, "M": 4, "S": w["S"], "H": 2048,
                       "W": 2048, "dz_m": w["dz"], "wavelength_m": w["wavelength"], "pixel_m": w["pixel_size"],
                       "batch": w["batch"], "eps": EPS, "backward": designs[0],
                       "step": "one LSQML epoch over all positions with per-slice directions and step sizes"},
            "kernels": {k: {"launches": n, "ms_per_launch": t / max(n, 1)} for k, (n, t) in prof.items()},
            "backward_designs": ms_design_report(api, w, mss, timed, opts),
            "losses": [l.item() for l in losses[:3]],
        }), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        if args.workload == "uneven16":
            run_uneven(args, rank, world, local_rank)
        elif args.workload == "uneven16opr":
            run_uneven(args, rank, world, local_rank, opr_K=8)
        elif args.workload == "spiral256":
            run_ad256(args, rank, world, local_rank)
        elif args.workload == "multislice256":
            run_ms256(args, rank, world, local_rank)
        elif args.workload == "multislice256-lsqml":
            run_ms256_lsqml(args, rank, world, local_rank)
        else:
            run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
