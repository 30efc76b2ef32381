#!/usr/bin/env python
"""Benchmark of the fp64 spectral-element stiffness apply ("Ax", Listing 2)
on GB300, in the JSON-line format the round driver reads.

Workload (default): a box of 32^3 = 32768 perturbed trilinear hexahedra at
lx = 8 (N = 7), fp64 inputs resident in HBM (9 fields of 134 MB, together
far larger than the 129 MB L2, so no flush is needed between steps).  One
step = one fp64 ax_helm apply over all elements through the C ABI.

  value      GDOF/s = E * lx^3 local points per second, whole job (all ranks)
  roofline   achieved algorithmic HBM GB/s (72 * lx^3 bytes per element) of
             the apply kernel against the measured HBM copy bandwidth
  e2e        the same metric through the public API with pinned host inputs,
             host->device copies of every input and the device->host copy
             of w inside each timed step
  cpu_baseline  the CPU oracle (plain C loop nest, OpenMP) on a bounded
             sample of the same workload, on this host's cores
  extras     fp32/bf16 storage modes and the fp64-unit kernel, each timed
             the same way (GDOF/s and % of HBM)

``--impl reference`` times the CPU oracle instead (the reference arm).
Multi-GPU (torchrun): every rank applies the operator to its own copy of
the mesh (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Ax GDOF/s & % HBM roofline, FP64 vs mixed; CG time-to-1e-8 residual"
GKEYS = ("g11", "g22", "g33", "g12", "g13", "g23")
FALLBACK_HBM_GBS = 6800.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--n", type=int, default=32, help="elements per box edge")
    p.add_argument("--lx", type=int, default=8)
    p.add_argument("--no-extras", action="store_true")
    p.add_argument("--extras", default="modes,sweep,cg,cg_sweep,learned,batch,rates,tri_df",
                   help="comma list of extra sections to run")
    p.add_argument("--no-cpu-baseline", action="store_true")
    return p.parse_args()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append((time.time(), parts))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self, t0=None, t1=None):
        rows = [r for (t, r) in self.rows if (t0 is None or t >= t0) and (t1 is None or t <= t1)]
        window = "timed region"
        if not rows:  # a region shorter than the sampling period
            rows = [r for (_, r) in self.rows]
            window = "whole run (no sample fell inside the timed region)"
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max((float(r[2]) for r in rows if r[2].replace(".", "").isdigit()), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx,
                "reasons": reasons, "samples": len(rows), "window": window}


def source_hash(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


KERNEL_SOURCES = {
    "ax_eop_kernel": ["paper_2506_20994_gb300/csrc/ax_eo_persist.cuh",
                      "paper_2506_20994_gb300/csrc/df64.cuh",
                      "paper_2506_20994_gb300/csrc/guard.cuh",
                      "paper_2506_20994_gb300/csrc/common.cuh"],
    "ax_df64eo_kernel": ["paper_2506_20994_gb300/csrc/ax_df64_eo.cuh",
                         "paper_2506_20994_gb300/csrc/df64.cuh",
                         "paper_2506_20994_gb300/csrc/common.cuh"],
    "ax_df64_kernel": ["paper_2506_20994_gb300/csrc/ax_df64.cuh",
                       "paper_2506_20994_gb300/csrc/df64.cuh",
                       "paper_2506_20994_gb300/csrc/common.cuh"],
    "ax_kstep_kernel": ["paper_2506_20994_gb300/csrc/ax_kstep.cuh",
                        "paper_2506_20994_gb300/csrc/common.cuh"],
}


def ncu_traffic(kernel: str, lx: int, nel: int):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current source of the kernel (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    e = d.get(kernel)
    if not e or e.get("source_hash") != source_hash(KERNEL_SOURCES[kernel]):
        return None
    if e.get("lx") != lx:
        return None
    return float(e["dram_bytes_per_element"]) * nel


# ---------------------------------------------------------------------------
def setup_operator(n: int, lx: int, dev, seed: int = 0):
    import numpy as np
    import torch
    import paper_2506_20994_gb300 as ax
    from paper_2506_20994_gb300 import synth

    v = synth.box_vertices(n, seed=seed)
    g = ax.box_geometry(v, lx)
    shape = g["g11"].shape
    host = {"u": synth.uniform(shape, seed=seed + 1), "h1": np.ones(shape)}
    host["dx"], host["dxt"] = ax.dmat(lx)
    for k in GKEYS:
        host[k] = g[k]
    dev_t = {k: torch.as_tensor(a).to(dev) for k, a in host.items()}
    return host, dev_t, shape[0]


def time_region(fn, steps: int, warmup: int, stream, barrier=None):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    if barrier:
        barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    t_wall0 = time.time()
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    t_wall1 = time.time()
    if barrier:
        barrier()
    return e0.elapsed_time(e1), (t_wall0, t_wall1)


def cpu_baseline(lx: int, n: int, target_s: float = 10.0, single_s: float = 0.0):
    """The oracle on a bounded sample (2048 elements) of the workload, with
    all host threads; with single_s > 0 also one thread for about single_s
    seconds."""
    import numpy as np
    import oracle
    from paper_2506_20994_gb300 import synth

    nel = n ** 3
    m = min(nel, 2048)
    v = synth.box_vertices(n, seed=0)
    pick = np.arange(m)
    go = oracle.box_geometry(v, lx, elements=pick)
    u = synth.uniform((nel, lx, lx, lx), seed=1)[:m].copy()
    h1 = np.ones_like(u)
    dx, dxt = oracle.d_buffers(lx)
    G = [go[k] for k in GKEYS]
    def timed(seconds):
        oracle.ax_helm(u, dx, dxt, h1, *G, lx)  # warm
        reps, t0 = 0, time.perf_counter()
        while True:
            oracle.ax_helm(u, dx, dxt, h1, *G, lx)
            reps += 1
            el = time.perf_counter() - t0
            if el >= seconds or reps >= 10000:
                return reps, el

    threads = oracle.set_threads(0)
    reps, el = timed(target_s)
    out = {"value": reps * m * lx ** 3 / el / 1e9, "unit": "GDOF/s", "cores": threads,
           "kind": "oracle",
           "sample": f"{reps} applies of the oracle loop nest on {m} of the {nel} elements "
                     f"(lx={lx}), {el:.1f} s, {threads} OpenMP threads"}
    if single_s > 0:
        oracle.set_threads(1)
        try:
            r1, e1 = timed(single_s)
        finally:
            oracle.set_threads(threads)
        out["single_thread"] = {"value": r1 * m * lx ** 3 / e1 / 1e9, "unit": "GDOF/s",
                                "sample": f"{r1} applies, 1 thread, {e1:.1f} s"}
    return out


def errors_vs_oracle(ax, n: int, lx: int, u_host):
    """Relative L2 error of every operator mode against the fp64 oracle on a
    sample of the workload's elements (64 of the mesh, first and last
    included): the oracle computes their geometry itself, every mode is
    applied to exactly those inputs (h1 = 1), and the oracle applies
    Listing 2 to the same inputs in fp64."""
    import numpy as np
    import oracle
    from paper_2506_20994_gb300 import synth
    from bench_extras import mode_outputs, sample_elements
    nel = n ** 3
    pick = sample_elements(nel)
    v = synth.box_vertices(n, seed=0)
    go = oracle.box_geometry(v, lx, elements=pick)
    u = np.ascontiguousarray(u_host.reshape(nel, -1)[pick].reshape(-1, lx, lx, lx))
    h1 = np.ones_like(u)
    dx, dxt = oracle.d_buffers(lx)
    corners = oracle.element_corners(v)[pick]
    xi, wq = oracle.gll(lx)
    ref = oracle.ax_helm(u, dx, dxt, h1, *[go[k] for k in GKEYS], lx)
    got = mode_outputs(ax, lx, u, h1, dx, dxt, go, corners, xi, wq)
    out = {"elements": int(len(pick)), "of": nel,
           "method": "every mode on the same sampled elements and inputs as the oracle"}
    for name, w in got.items():
        out[name] = float(np.linalg.norm(w - ref) / np.linalg.norm(ref))
    return out


def run_reference(args, rank):
    if rank != 0:
        return
    base = cpu_baseline(args.lx, args.n, target_s=max(5.0, min(60.0, 0.01 * args.steps)))
    line = {
        "impl": "reference", "metric": METRIC, "value": base["value"], "unit": "GDOF/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "ms_per_step": None,
        "config": {"workload": f"fp64 ax_helm, box {args.n}^3 = {args.n ** 3} perturbed "
                               f"hexahedra, lx={args.lx}", "E": args.n ** 3, "lx": args.lx,
                   "points": args.n ** 3 * args.lx ** 3,
                   "entry": "oracle C loop nest (OpenMP over elements) on the host cores",
                   "parallelism": "rank 0 only"},
        "cpu_baseline": base,
        "e2e": {"value": base["value"], "unit": "GDOF/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import torch.distributed as dist
    import paper_2506_20994_gb300 as ax

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
        barrier = lambda: dist.barrier()
    else:
        barrier = None
    ax.lib()

    lx, n = args.lx, args.n
    host, d, nel = setup_operator(n, lx, dev)
    npts = nel * lx ** 3
    stream = torch.cuda.current_stream()
    w = torch.empty_like(d["u"])
    G = [d[k] for k in GKEYS]

    # the operator handle of one mesh: geometry prepared once (set-up, like
    # the geometric factors themselves), applied every step
    op = ax.Operator(lx, d["dx"], d["dxt"], d["h1"], *G)
    prepared = op.info()["prepared"]

    def step():
        op.apply(w, d["u"])

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ms, (tw0, tw1) = time_region(step, args.steps, max(3, args.warmup), stream, barrier)
    # A short timed region says little about sustained clocks: the same step
    # is timed again over about two seconds, with the clocks of that window.
    sustained = None
    if ms < 1000.0:
        n_s = int(min(200000, max(args.steps, 2000.0 / max(ms / args.steps, 1e-3))))
        ms_s, (ts0, ts1) = time_region(step, n_s, 3, stream, barrier)
        sustained = {"steps": n_s, "ms_per_step": round(ms_s / n_s, 5),
                     "value": round(world * npts * n_s / (ms_s * 1e-3) / 1e9, 3)}
    clocks.stop()
    if sustained is not None:
        sustained["clocks"] = clocks.summary(ts0, ts1)
    ms_t = torch.tensor([ms], device=dev, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(ms_t, op=dist.ReduceOp.MAX)
    ms_max = float(ms_t.item())
    value = world * npts * args.steps / (ms_max * 1e-3) / 1e9
    t_launch = ms / args.steps * 1e-3
    hbm_peak, peak_src = measured_peaks()
    bytes_alg = 72.0 * lx ** 3 * nel
    achieved = bytes_alg / t_launch / 1e9
    kname = ("ax_eop_kernel" if prepared else
             "ax_df64eo_kernel" if lx in (8, 10, 12) else
             "ax_df64_kernel" if lx <= 12 else "ax_kstep_kernel")
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak,
            "unit": "GB/s", "frac": round(achieved / hbm_peak, 4),
            "traffic": ncu_traffic(kname, lx, nel), "kernel": kname,
            "peak_source": f"{peak_src} HBM copy bandwidth (MEASURED_PEAKS.json)"}

    # end to end through the public C-ABI call on pinned host buffers
    # (ax_helm_host: every step moves all inputs in and the result out,
    # chunked so that the copies and the apply overlap)
    hp = {k: torch.as_tensor(host[k]).pin_memory() for k in host}
    w_host = torch.empty(w.shape, dtype=w.dtype).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in hp.values())
    d2h = w_host.numel() * w_host.element_size()

    def e2e_step():
        ax.ax_helm_host(w_host, hp["u"], hp["dx"], hp["dxt"], hp["h1"], *[hp[k] for k in GKEYS],
                        lx)

    e2e_steps = max(3, min(args.steps, 30))
    ms_e2e, _ = time_region(e2e_step, e2e_steps, 3, stream, barrier)
    if world > 1:  # the slowest rank, as for the main value
        t = torch.tensor([ms_e2e], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_e2e = float(t.item())
    e2e = {"value": world * npts * e2e_steps / (ms_e2e * 1e-3) / 1e9, "unit": "GDOF/s",
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "entry": "ax_helm_host (chunked copies in / apply / copies out overlapped)"}
    del hp

    extras = {}
    if not args.no_extras and rank == 0:
        from bench_extras import run_extras
        extras = run_extras(ax, host, d, lx, nel, stream, hbm_peak,
                            set(x for x in args.extras.split(",") if x))

    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "GDOF/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"fp64 ax_helm, box {n}^3 = {nel} perturbed hexahedra, lx={lx}",
                   "E": nel, "lx": lx, "points": npts,
                   "entry": "ax_op_apply (operator handle)",
                   "geometry": ("prepared once by ax_op_create into the persistent even-odd "
                                "kernel's double-float order (8 B per value, as fp64), staged "
                                "per element into shared memory by cp.async.bulk" if prepared
                                else "fp64 arrays"),
                   "e2e_entry": "ax_helm_host on pinned host fp64 arrays",
                   "gflop_per_step": round((12 * lx ** 4 + 18 * lx ** 3) * nel / 1e9, 4),
                   "l2": "inputs (9 x %.0f MB) larger than L2; no flush" % (npts * 8 / 1e6),
                   "parallelism": f"replicas x{world}"},
        "roofline": roof,
        "e2e": e2e,
        "gpu_launches": args.steps,
        "clocks": clocks.summary(tw0, tw1),
    }
    if sustained is not None:
        line["sustained"] = sustained
    line["gflops"] = round(line["config"]["gflop_per_step"] / (ms_max / args.steps * 1e-3), 1)
    if extras:
        line["extras"] = extras
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(lx, n, single_s=5.0)
        if not args.no_extras:  # outside the timed region: each mode against the oracle
            line.setdefault("extras", {})["errors_vs_oracle"] = errors_vs_oracle(
                ax, n, lx, host["u"])
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
