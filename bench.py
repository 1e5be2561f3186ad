"""Benchmark: CTF-MNMF-ISS iterations/s on one GB300 (and N independent replicas).

A step is one full solve of the plain single-mixture workload through the C ABI:
load the STFT, set the NMF init, run 100 iterations (ISS sweep + basis MU per bin,
activation MU + normalisation across bins). Workload: N=2 sources, M=3 microphones,
taps (2,1), F=513 bins, J=1000 frames, B=10 bases, seeded synthetic CTF mixture
(16 kHz speech-like shape, STFT 1024 / hop 256, -30 dB noise).

  value  : iterations/s of the whole job (all ranks), CUDA events on the solver's stream,
           inputs resident in HBM, L2 flushed (256 MiB write) between steps
  e2e    : the same through host buffers (pinned X, T0, V0 in; separated images out)
  roofline: the dominant kernel's algorithmic bytes per launch / its event-timed duration

--impl reference times the FP64 CPU oracle (one iteration of the same workload per step).
Under torchrun each rank solves its own mixture (seed = rank): weak scaling, no collective
on the data path; only the timing uses a barrier and a max-reduce.
"""
import os
import sys

if "--impl" in sys.argv and "reference" in sys.argv:
    for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(_v, "1")

import argparse
import json
import statistics
import subprocess
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CTF-MNMF-ISS iterations/s at 1 GB300 (plain vs batched vs fwd+bwd), % HBM roof"
UNIT = "iterations/s"
WORKLOAD = "C2"
FALLBACK_HBM_GBS = 6800.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=300)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--iters", type=int, default=None, help="iterations per step (default: workload's)")
    p.add_argument("--batched-steps", type=int, default=3,
                   help="timed steps of the 64-mixture batched workload (0 skips it)")
    p.add_argument("--batched-mixtures", type=int, default=64,
                   help="mixtures of the batched workload (seeds 0..n-1; fewer for small profiling captures)")
    p.add_argument("--fwdbwd-steps", type=int, default=3,
                   help="timed steps of the 16-mixture forward + backward workload (0 skips it)")
    p.add_argument("--fwdbwd-ckpt", type=int, default=0,
                   help="checkpoint segment length of the forward + backward workload (0: all iterations)")
    p.add_argument("--longj-steps", type=int, default=3,
                   help="timed steps of the long-J workload (F=513, J=16000; 0 skips it)")
    p.add_argument("--path", default="auto", choices=["auto", "persistent", "two_kernel"],
                   help="execution path of the plain workload (auto: the library times both)")
    p.add_argument("--bin-fpt", type=int, default=0,
                   help="frames per thread of the two-kernel bin phase (0: the library's choice)")
    p.add_argument("--ip-steps", type=int, default=3,
                   help="timed steps of the ISS-vs-IP comparison on the plain workload (0 skips it)")
    p.add_argument("--config-steps", type=int, default=3,
                   help="timed steps of each other single-mixture workload, C1 C3 P4 P6 P8 (0 skips them)")
    p.add_argument("--cpu-timings", type=int, default=1,
                   help="1: time the FP64 oracle on further workloads and thread counts (about a minute)")
    return p.parse_args()


def job_throughput(local_ms, world, iters, steps, dist=None, device="cpu"):
    """Whole-job rate: this rank's elapsed milliseconds maxed over the ranks (the job ends
    with its slowest rank), units = world * iters * steps. Returns (rate per second, max ms)."""
    import torch
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    return world * iters * steps / (ms / 1000.0), ms


def spec_for(rank):
    from paper_2510_02382_gb300 import synth
    return synth.scaled(synth.CONFIGS[WORKLOAD], seed=rank)


def workload_config(spec, l2_note):
    return {"workload": f"{WORKLOAD}: plain CTF-MNMF-ISS, N={spec.N} M={spec.M} taps={tuple(spec.taps())} "
                        f"F={spec.F} J={spec.J} B={spec.B}, {spec.iters} iterations per solve",
            "N": spec.N, "M": spec.M, "F": spec.F, "J": spec.J, "B": spec.B,
            "iterations_per_step": spec.iters, "l2": l2_note, "replicas": "one mixture per rank (seed = rank)"}


KERNEL_SOURCES = {   # the CUDA sources each profiled kernel is compiled from (besides the common headers)
    "persistent_kernel": lambda f: f == "persistent_kernel.cuh" or f.startswith("persistent"),
    "bin_phase_kernel": lambda f: f.startswith("bin_phase"),   # bin_phase.cu, bin_phase_kernels.cuh, bin_phase_m*.cu
    "frame_phase_kernel": lambda f: f == "kernels.cu",
}


def csrc_hash(kernel="persistent_kernel"):
    """Short hash of the sources a kernel is compiled from, matched against the one stored
    with a capture."""
    import hashlib
    d = os.path.join(ROOT, "paper_2510_02382_gb300", "csrc")
    pick = KERNEL_SOURCES[kernel]
    names = sorted(f for f in os.listdir(d) if f in ("internal.cuh", "phases.cuh") or pick(f))
    h = hashlib.sha256()
    for f in names:
        h.update(f.encode())
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def captured_traffic(kernel, launch_iters, want_iters):
    """DRAM bytes per launch from the committed ncu summary, if it matches these sources and
    the captured launch ran as many iterations as the timed one."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_C2.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    if d.get("csrc_sha256_16") != csrc_hash(kernel) or launch_iters != want_iters:
        return None
    return d["dram_bytes_per_launch"]


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        import tempfile
        try:
            fd, self.path = tempfile.mkstemp(prefix=f"ctfmnmf_clocks_{self.index}_", suffix=".csv")
            self.f = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as fh:
            lines = fh.readlines()
        os.unlink(self.path)
        for line in lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, r in rows for k in range(4) if r[k].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def cpu_baseline_sample(seconds=12.0):
    """The FP64 oracle, as it stands, on one host core: iterations of the full workload
    until `seconds` have passed (at least 2). Runs in a fresh interpreter."""
    code = f"""
import os, time, json, sys
sys.path.insert(0, {ROOT!r})
from paper_2510_02382_gb300 import synth
from oracle import ctfmnmf_oracle as O
spec = synth.CONFIGS[{WORKLOAD!r}]
mix = synth.make_mixture(spec)
x, W, b, v = O.init_state(mix.X, mix.T0, mix.V0)
n, t0 = 0, time.perf_counter()
while n < 2 or time.perf_counter() - t0 < {seconds}:
    W, b, v, y = O.iterate(x, W, b, v, mix.Ln)
    n += 1
dt = time.perf_counter() - t0
print(json.dumps({{"iters": n, "seconds": dt}}))
"""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
    if res.returncode != 0:
        return None
    d = json.loads(res.stdout.strip().splitlines()[-1])
    return {"value": d["iters"] / d["seconds"], "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{d['iters']} FP64 oracle iterations of the full {WORKLOAD} mixture in {d['seconds']:.1f} s "
                      f"(single thread)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import ctfmnmf_oracle as O
    from paper_2510_02382_gb300 import synth
    spec = spec_for(0)
    mix = synth.make_mixture(spec)
    x, W, b, v = O.init_state(mix.X, mix.T0, mix.V0)
    for _ in range(args.warmup):
        W, b, v, y = O.iterate(x, W, b, v, mix.Ln)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        W, b, v, y = O.iterate(x, W, b, v, mix.Ln)
    dt = time.perf_counter() - t0
    value = args.steps / dt
    sample = f"one FP64 oracle iteration of the full {WORKLOAD} mixture per step (single thread)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(spec, "host CPU run"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def batched_leg(args, peak):
    """The ragged batched workload: 64 mixtures (J ~ U[300, 3000], N in {2, 3}, M = N + 1,
    L in {2, 4, 8}, F = 513, B = 10, seeds 0..63), 50 iterations per step, one batch handle.
    Its working set (about 3 GB) is far larger than L2, so no flush is needed."""
    import torch
    from paper_2510_02382_gb300 import synth
    from paper_2510_02382_gb300.api import CTFMNMF, Batch
    specs = synth.batched_specs(count=args.batched_mixtures)
    solvers, bytes_it, binframes = [], 0, 0
    for sp in specs:
        mix = synth.make_mixture(sp)
        sv = CTFMNMF(sp.M, sp.N, sp.L, sp.B, sp.F, sp.J, Ln=mix.Ln, path="two_kernel")
        sv.load_stft(torch.from_numpy(mix.X).cuda())
        sv.set_init(torch.from_numpy(mix.T0).cuda(), torch.from_numpy(mix.V0).cuda())
        solvers.append(sv)
        bytes_it += 16 * sp.M * sp.F * sp.J + 8 * sp.N * sp.B * (sp.F + sp.J)
        binframes += sp.F * sp.J
    iters = specs[0].iters
    batch = Batch(solvers)
    batch.time(iters)
    ms = [batch.time(iters) for _ in range(args.batched_steps)]
    info = batch.info()
    batch.close()
    for sv in solvers:
        sv.close()
    t = statistics.median(ms) / 1000.0
    achieved = bytes_it * iters / t / 1e9
    return {"workload": f"{len(specs)} ragged mixtures: J ~ U[300, 3000], N in {{2,3}}, M = N+1, L in {{2,4,8}}, F=513, "
                        f"B=10, 50 iterations per step, seeds 0..{len(specs) - 1}",
            "batch_iterations_per_s": iters / t, "bin_frames_per_s": binframes * iters / t,
            "ms_per_step": 1000.0 * t, "steps": len(ms),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "algorithmic_bytes_per_iteration": bytes_it},
            "plan": info}


def fwd_bwd_leg(args, peak):
    """The differentiable workload: 16 mixtures (N=2, M=3, L=4, F=257, J=500, B=8, seeds
    0..15), 20 unrolled iterations (by default all of them on the forward pass's tape, one
    checkpoint segment; --fwdbwd-ckpt sets the segment length); a step = forward pass, MSE loss
    and its gradient, backward pass to X, T0, V0 (all in the library's kernels). Timed with
    CUDA events on the solver's stream; the forward pass alone (with the loss) is timed
    beside it for the fwd+bwd / fwd cost ratio."""
    import torch
    from paper_2510_02382_gb300 import synth
    from paper_2510_02382_gb300.api import Grad
    specs = synth.grad_specs()
    sp = specs[0]
    S, K = len(specs), sp.iters
    mixes = [synth.make_mixture(x) for x in specs]
    ckpt = args.fwdbwd_ckpt if args.fwdbwd_ckpt > 0 else K
    g = Grad(sp.M, sp.N, sp.L, sp.B, sp.F, sp.J, batch=S, n_iter=K, ckpt_every=ckpt, Ln=mixes[0].Ln)
    X = torch.from_numpy(np.stack([m.X for m in mixes])).cuda()
    T0 = torch.from_numpy(np.stack([m.T0 for m in mixes])).cuda()
    V0 = torch.from_numpy(np.stack([m.V0 for m in mixes])).cuda()
    Cref = torch.from_numpy(np.stack([m.images for m in mixes])).cuda()
    C = torch.empty(g.shapes()["C"], dtype=torch.complex64, device="cuda")
    gC = torch.empty_like(C)
    loss = torch.zeros((), dtype=torch.float64, device="cuda")
    st = g.stream

    def fwd():
        g.forward(X, T0, V0, out=C)
        g.mse(C, Cref, loss=loss)

    def fwd_bwd():
        fwd()
        g.mse(C, Cref, gC=gC)
        return g.backward(gC)

    def timed(fn, n):
        out = []
        for _ in range(n):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(st)
            fn()
            e1.record(st)
            torch.cuda.synchronize()
            out.append(e0.elapsed_time(e1))
        return statistics.median(out)

    fwd_bwd()                                   # first call builds the batch (autotuner)
    timed(fwd_bwd, 1)
    l0 = g.launch_count()
    ms = timed(fwd_bwd, args.fwdbwd_steps)
    launches = (g.launch_count() - l0) // args.fwdbwd_steps
    ms_fwd = timed(fwd, args.fwdbwd_steps)
    g.close()
    t = ms / 1000.0
    y_pass = 8 * sp.M * sp.F * sp.J * S         # one read or write of Y for the whole batch
    bytes_it = 6 * y_pass                       # fwd+bwd counted as 6 Y-passes per iteration
    achieved = bytes_it * K / t / 1e9
    return {"workload": f"16 mixtures N={sp.N} M={sp.M} L={sp.L} F={sp.F} J={sp.J} B={sp.B}, {K} unrolled "
                        f"iterations, checkpoint every {ckpt} (the last segment on the forward pass's tape), "
                        "loss = MSE of the separated images to the true "
                        "images, gradients to X, T0, V0; seeds 0..15",
            "iterations_per_s": K / t, "bin_frames_per_s": S * sp.F * sp.J * K / t,
            "ms_per_step": ms, "fwd_ms_per_step": ms_fwd, "fwd_bwd_over_fwd": ms / ms_fwd,
            "steps": args.fwdbwd_steps, "gpu_launches_per_step": launches,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "algorithmic_bytes_per_iteration": bytes_it}}


def ip_leg(args, spec, iters):
    """The paper's comparison on one GPU: the plain workload's iterations with the IP update
    (Eqs. 9-10) against the ISS update, both on the two-kernel path (the IP update runs
    there only), CUDA events around ctfmnmf_iterate on the solver's stream, median of the
    timed steps, L2 flushed between steps. The persistent ISS path is the headline value."""
    import torch
    from paper_2510_02382_gb300 import synth
    from paper_2510_02382_gb300.api import CTFMNMF
    mix = synth.make_mixture(spec)
    X = torch.from_numpy(mix.X).cuda()
    T0 = torch.from_numpy(mix.T0).cuda()
    V0 = torch.from_numpy(mix.V0).cuda()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    out = {}
    for upd in ("iss", "ip"):
        sv = CTFMNMF(spec.M, spec.N, spec.L, spec.B, spec.F, spec.J, Ln=mix.Ln, path="two_kernel", w_update=upd)
        st = sv.stream
        ms = []
        for k in range(args.ip_steps + 1):
            sv.load_stft(X)
            sv.set_init(T0, V0)
            flush.fill_(float(k))
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            sv.iterate(iters)
            e1.record(st)
            torch.cuda.synchronize()
            if k > 0:
                ms.append(e0.elapsed_time(e1))
        sv.close()
        out[upd] = iters / (statistics.median(ms) / 1000.0)
    return {"workload": "the plain workload, two-kernel path, ISS and IP updates", "steps": args.ip_steps,
            "iss_iterations_per_s": out["iss"], "ip_iterations_per_s": out["ip"],
            "iss_over_ip": out["iss"] / out["ip"]}


def longj_leg(args, peak):
    """Bins longer than one thread block: the long-J workload (N=2, M=3, L=4, F=513,
    J=16000, B=10; each bin over a cluster of 8 blocks), 10 iterations per step, CUDA events
    around ctfmnmf_iterate on the solver's stream, median of the timed steps. Its rows
    (197 MB) do not fit L2, so no flush is needed; the roofline is the cluster bin phase's
    own launch time from ctfmnmf_time_phases."""
    import torch
    from paper_2510_02382_gb300 import synth
    from paper_2510_02382_gb300.api import CTFMNMF
    sp = synth.CONFIGS["L1"]
    mix = synth.make_mixture(sp)
    sv = CTFMNMF(sp.M, sp.N, sp.L, sp.B, sp.F, sp.J, Ln=mix.Ln)
    X = torch.from_numpy(mix.X).cuda()
    T0 = torch.from_numpy(mix.T0).cuda()
    V0 = torch.from_numpy(mix.V0).cuda()
    st = sv.stream
    ms = []
    for k in range(args.longj_steps + 1):
        sv.load_stft(X)
        sv.set_init(T0, V0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        sv.iterate(sp.iters)
        e1.record(st)
        torch.cuda.synchronize()
        if k > 0:
            ms.append(e0.elapsed_time(e1))
    ms_bin, ms_frame = sv.time_phases(5)
    sv.close()
    t = statistics.median(ms) / 1000.0
    M, N, F, J, B = sp.M, sp.N, sp.F, sp.J, sp.B
    it_bytes = 16 * M * F * J + 8 * N * B * (F + J)
    bin_bytes = 16 * M * F * J + 8 * N * B * F + 4 * N * B * J
    return {"workload": f"long J: N={N} M={M} L={sp.L} F={F} J={J} B={B}, {sp.iters} iterations per step, "
                        "bins over clusters of 8 thread blocks", "steps": args.longj_steps,
            "iterations_per_s": sp.iters / t, "bin_frames_per_s": F * J * sp.iters / t,
            "ms_per_step": 1000.0 * t, "kernel_times": {"cluster_bin_phase_ms": ms_bin, "frame_phase_ms": ms_frame},
            "roofline": {"bound": "hbm", "kernel": "cluster_bin_kernel", "achieved": bin_bytes / (ms_bin * 1e-3) / 1e9,
                         "peak": peak, "unit": "GB/s", "frac": bin_bytes / (ms_bin * 1e-3) / 1e9 / peak,
                         "algorithmic_bytes_per_launch": bin_bytes},
            "iteration_roofline_frac": it_bytes * sp.iters / t / 1e9 / peak}


def plain_config_leg(name, args, peak):
    """One of the other single-mixture workloads (C1, C3 and the paper's Table I shapes
    P4/P6/P8) on the path AUTO picks: CUDA events around ctfmnmf_iterate(iters) on the solver's
    stream, median of the timed steps, L2 flushed between steps; the bin and frame phases timed
    alone (event pair around each launch) for the kernel roofline; the whole iteration's
    roofline from the graph-replayed rate."""
    import torch
    from paper_2510_02382_gb300 import synth
    from paper_2510_02382_gb300.api import CTFMNMF
    sp = synth.CONFIGS[name]
    mix = synth.make_mixture(sp)
    sv = CTFMNMF(sp.M, sp.N, sp.L, sp.B, sp.F, sp.J, Ln=mix.Ln)
    X = torch.from_numpy(mix.X).cuda()
    T0 = torch.from_numpy(mix.T0).cuda()
    V0 = torch.from_numpy(mix.V0).cuda()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    st = sv.stream
    ms = []
    for k in range(args.config_steps + 1):
        sv.load_stft(X)
        sv.set_init(T0, V0)
        flush.fill_(float(k))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        sv.iterate(sp.iters)
        e1.record(st)
        torch.cuda.synchronize()
        if k > 0:
            ms.append(e0.elapsed_time(e1))
    sv.load_stft(X)
    sv.set_init(T0, V0)
    sv.time_phases(3)
    ms_bin, ms_frame = sv.time_phases(20)
    path, shape = sv.path, sv.bin_shape()
    sv.close()
    t = statistics.median(ms) / 1000.0
    M, N, F, J, B = sp.M, sp.N, sp.F, sp.J, sp.B
    it_bytes = 16 * M * F * J + 8 * N * B * (F + J)
    bin_bytes = 16 * M * F * J + 8 * N * B * F + 4 * N * B * J
    bin_gbs = bin_bytes / (ms_bin * 1e-3) / 1e9
    return {"workload": f"{name}: N={N} M={M} taps={tuple(mix.Ln)} F={F} J={J} B={B}, {sp.iters} iterations per step",
            "steps": args.config_steps, "iterations_per_s": sp.iters / t, "bin_frames_per_s": F * J * sp.iters / t,
            "path": path, "bin_shape": {"frames_per_thread": shape[0], "threads": shape[1]},
            "kernel_times": {"bin_phase_ms": ms_bin, "frame_phase_ms": ms_frame},
            "roofline": {"bound": "hbm", "kernel": "bin_phase_kernel", "achieved": bin_gbs, "peak": peak, "unit": "GB/s",
                         "frac": bin_gbs / peak, "algorithmic_bytes_per_launch": bin_bytes},
            "iteration_roofline_frac": it_bytes * sp.iters / t / 1e9 / peak}


def cpu_oracle_timings(seconds=6.0):
    """The FP64 oracle, as it stands, on the host cores in the same run, beside the GPU numbers
    (a reported baseline, not the target): C2 with one thread and with every core, C3 with the
    ISS and with the IP update, and the batched workload as 4 of its mixtures x 5 iterations,
    extrapolated linearly in the sum of F*J*iterations over all 64 mixtures and 50 iterations.
    Each timing is a bounded sample of iterations (at least 2, until about `seconds`)."""
    code = f"""
import json, os, sys, time
sys.path.insert(0, {ROOT!r})
from paper_2510_02382_gb300 import synth
from oracle import ctfmnmf_oracle as O

def rate(spec, update, seconds):
    mix = synth.make_mixture(spec)
    x, W, b, v = O.init_state(mix.X, mix.T0, mix.V0)
    n, t0 = 0, time.perf_counter()
    while n < 2 or time.perf_counter() - t0 < seconds:
        W, b, v, y = O.iterate(x, W, b, v, mix.Ln, update=update)
        n += 1
    return n, time.perf_counter() - t0

out = {{}}
for name, upd in (("C2", "iss"), ("C3", "iss"), ("C3", "ip")):
    n, dt = rate(synth.CONFIGS[name], upd, {seconds})
    out[name + "_" + upd] = {{"iterations": n, "seconds": dt, "iterations_per_s": n / dt}}
specs = synth.batched_specs()
picks = [specs[k] for k in (0, 21, 42, 63)]
t = 0.0
for sp in picks:
    mix = synth.make_mixture(sp)
    x, W, b, v = O.init_state(mix.X, mix.T0, mix.V0)
    t0 = time.perf_counter()
    for _ in range(5):
        W, b, v, y = O.iterate(x, W, b, v, mix.Ln)
    t += time.perf_counter() - t0
work_sample = sum(sp.F * sp.J * 5 for sp in picks)
work_all = sum(sp.F * sp.J * sp.iters for sp in specs)
out["C4"] = {{"sample": "mixtures 0, 21, 42, 63 x 5 iterations", "seconds": t,
             "extrapolated_seconds_per_50_iterations": t * work_all / work_sample,
             "batch_iterations_per_s": specs[0].iters / (t * work_all / work_sample)}}
print(json.dumps(out))
"""
    ncores = os.cpu_count() or 1
    res = {"nproc": ncores}
    for label, threads in (("one_thread", 1), ("all_cores", ncores)):
        env = dict(os.environ, OMP_NUM_THREADS=str(threads), OPENBLAS_NUM_THREADS=str(threads),
                   MKL_NUM_THREADS=str(threads))
        if label == "all_cores":       # only C2 is rerun with every core
            c = code.replace('(("C2", "iss"), ("C3", "iss"), ("C3", "ip"))', '(("C2", "iss"),)')
            c = c[:c.index("specs = synth.batched_specs()")] + "print(json.dumps(out))\n"
        else:
            c = code
        r = subprocess.run([sys.executable, "-c", c], capture_output=True, text=True, env=env, timeout=900)
        if r.returncode != 0:
            res[label] = {"error": r.stderr.strip().splitlines()[-1] if r.stderr.strip() else "failed"}
            continue
        res[label] = json.loads(r.stdout.strip().splitlines()[-1])
        res[label]["threads"] = threads
    return res


def run_ours(args):
    import torch
    from paper_2510_02382_gb300 import synth
    from paper_2510_02382_gb300.api import CTFMNMF

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    spec = spec_for(rank)
    iters = args.iters or spec.iters
    mix = synth.make_mixture(spec)
    N, M, F, J, B = spec.N, spec.M, spec.F, spec.J, spec.B
    stream = torch.cuda.current_stream()
    solver = CTFMNMF(M, N, spec.L, B, F, J, Ln=mix.Ln, stream=stream, path=args.path, bin_fpt=args.bin_fpt)
    X_h = torch.from_numpy(mix.X).pin_memory()
    T0_h = torch.from_numpy(mix.T0).pin_memory()
    V0_h = torch.from_numpy(mix.V0).pin_memory()
    X_d, T0_d, V0_d = X_h.cuda(), T0_h.cuda(), V0_h.cuda()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MiB > L2

    def step():
        solver.load_stft(X_d)
        solver.set_init(T0_d, V0_d)
        solver.iterate(iters)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches0 = solver.launch_count()
    barrier()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    barrier()
    launches = solver.launch_count() - launches0
    total_ms = sum(a.elapsed_time(b) for a, b in ev)
    clocks = sampler.stop() if sampler else None
    value, total_ms = job_throughput(total_ms, world, iters, args.steps, dist, "cuda")

    # ---- end to end through host buffers
    out_h = torch.empty((N, M, F, J), dtype=torch.complex64).pin_memory()
    T0_e = torch.empty_like(T0_d)
    V0_e = torch.empty_like(V0_d)

    def step_e2e():
        solver.load_stft(X_h)
        T0_e.copy_(T0_h, non_blocking=True)
        V0_e.copy_(V0_h, non_blocking=True)
        solver.set_init(T0_e, V0_e)
        solver.iterate(iters)
        solver.get_separated(out_h)

    step_e2e()
    e2e_steps = max(1, min(args.steps, 50))
    ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(e2e_steps)]
    barrier()
    for k in range(e2e_steps):
        flush.zero_()
        ev2[k][0].record(stream)
        step_e2e()
        ev2[k][1].record(stream)
    barrier()
    e2e_ms = sum(a.elapsed_time(b) for a, b in ev2)
    e2e_value, _ = job_throughput(e2e_ms, world, iters, e2e_steps, dist, "cuda")
    h2d = X_h.numel() * 8 + T0_h.numel() * 4 + V0_h.numel() * 4
    d2h = out_h.numel() * 8

    # ---- per-kernel durations (event pairs around each launch, same stream) for the roofline
    solver.load_stft(X_d)
    solver.set_init(T0_d, V0_d)
    iter_bytes = 16 * M * F * J + 8 * N * B * (F + J)     # one HBM read + write of Y, T and V
    if solver.path == "persistent":
        solver.time_persistent(iters)
        runs = [solver.time_persistent(iters) for _ in range(5)]
        kms = statistics.median(r[0] for r in runs)
        kname, kbytes = "persistent_kernel", iters * iter_bytes
        phase = {"persistent_launch_ms": kms, "iterations_per_launch": iters,
                 "finalize_ms": statistics.median(r[1] for r in runs)}
    else:
        solver.time_phases(5)
        ms_bin, ms_frame = solver.time_phases(50)
        bytes_bin = 16 * M * F * J + 8 * N * B * F + 4 * N * B * J
        bytes_frame = 8 * N * F * J + 4 * N * F * B + 8 * N * B * J
        if ms_bin >= ms_frame:
            kname, kms, kbytes = "bin_phase_kernel", ms_bin, bytes_bin
        else:
            kname, kms, kbytes = "frame_phase_kernel", ms_frame, bytes_frame
        phase = {"bin_phase_ms": ms_bin, "frame_phase_ms": ms_frame}
    peak, peak_src = peaks()
    achieved = kbytes / (kms * 1e-3) / 1e9
    # the kernels inside the replayed graph: the timed step's time per iteration (a step also
    # loads the STFT and the init, about 1 % here), split between the phases in the ratio of
    # their isolated launch times (an estimate: events cannot sit inside a graph)
    it_us = 1000.0 * (total_ms / args.steps) / iters
    if solver.path == "persistent":
        in_graph = {"iteration_us": it_us}
    else:
        share = ms_bin / (ms_bin + ms_frame)
        in_graph = {"iteration_us": it_us, "bin_phase_us_est": share * it_us, "frame_phase_us_est": (1 - share) * it_us,
                    "bin_phase_frac_est": kbytes / (share * it_us * 1e-6) / 1e9 / peak if kname == "bin_phase_kernel" else None,
                    "method": "timed step per iteration, split by the ratio of the isolated launch times"}
    traffic = captured_traffic(kname, iters if kname == "persistent_kernel" else 1,
                               100 if kname == "persistent_kernel" else 1)
    # arithmetic view: about 23 M^2 (ISS) + 12 N B (NMF) flops per bin-frame and iteration
    flops = (23 * M * M + 12 * N * B) * F * J * (iters if kname == "persistent_kernel" else 1)
    fp32_peak = 152 * 128 * 2 * 2.07e9 / 1e12          # TFLOP/s: SMs x FP32 lanes x FMA x max clock
    solver_path = solver.path
    bin_fpt, bin_nt = solver.bin_shape()
    solver.close()
    batched = batched_leg(args, peak) if args.batched_steps > 0 else None
    fwdbwd = fwd_bwd_leg(args, peak) if args.fwdbwd_steps > 0 else None
    ipcmp = ip_leg(args, spec, iters) if args.ip_steps > 0 else None
    longj = longj_leg(args, peak) if args.longj_steps > 0 else None
    configs = ({name: plain_config_leg(name, args, peak) for name in ("C1", "C3", "P4", "P6", "P8")}
               if args.config_steps > 0 else None)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    cpu = cpu_baseline_sample() if world == 1 else None
    cpu_more = cpu_oracle_timings() if (world == 1 and args.cpu_timings) else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(spec, "flushed between steps (256 MiB write outside the timed events)"),
        "bin_frames_per_s": value * F * J,
        "roofline": {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak,
                     "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else "fallback",
                     "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "algorithmic_bytes_per_launch": kbytes, "avg_launch_ms": kms,
                     "alu": {"achieved_tflops": flops / (kms * 1e-3) / 1e12, "peak_tflops": fp32_peak,
                             "peak_source": "nominal, not measured: 152 SMs x 128 FP32 lanes x 2 (FMA) x 2.07 GHz",
                             "frac": flops / (kms * 1e-3) / 1e12 / fp32_peak},
                     "in_graph": in_graph},
        "path": solver_path,
        "bin_shape": {"frames_per_thread": bin_fpt, "threads": bin_nt},
        "kernel_times": phase,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": e2e_steps},
        "clocks": clocks,
        "gpu_launches": launches,
        "batched": batched,
        "fwd_bwd": fwdbwd,
        "iss_vs_ip": ipcmp,
        "long_j": longj,
        "plain_configs": configs,
        "cpu_oracle_timings": cpu_more,
    }
    if batched is not None:
        batched["vs_plain_bin_frames"] = batched["bin_frames_per_s"] / line["bin_frames_per_s"]
    if fwdbwd is not None:
        fwdbwd["vs_plain_bin_frames"] = fwdbwd["bin_frames_per_s"] / line["bin_frames_per_s"]
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
