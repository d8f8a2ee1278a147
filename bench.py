"""Benchmark of the labeling hot path: edge x proposition labels per second.

One step = one planning query on one frame: resample the world proposition
planes at the agent pose (frame transform), label every roadmap edge (the
Boolean product of eq. 10) and, where the workload has one, run the safety
monitor fused into the labeling kernel.

  value  device-timed steps, inputs resident in HBM (CUDA events per step,
         L2 flushed before every step)
  e2e    the same steps through lbl_session_run with pinned host buffers:
         host->device copy of the planes and device->host copy of the labels
         (and monitor outputs) are inside the timed region

Multi-GPU (torchrun): every rank labels its own independent frames against
its own roadmap (weak scaling); ranks only meet at the barrier and the
max-over-ranks of the timings.

``--impl reference`` times the CPU oracle instead (rank 0 only), on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import json
import math
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "edge*prop labels/s"
UNIT = "labels/s"

WORKLOADS = {
    "large": "1,000,000 constant-curvature arcs swept on a 512x512 agent grid at 0.2 m (z-order), 64 propositions, "
             "world planes resampled at a random pose, 16-state safety monitor over 8 label bits fused",
    "driving": "100,000 arcs on a 256x256 agent grid at 0.25 m (z-order), 32 propositions, world planes resampled "
               "at a random pose",
    "plain": "2,000 arcs on a 64x64 grid at 0.5 m (z-order), 4 disc propositions",
    "paper": "1,097,702 short arcs on a 2048x1024 row-major grid at 0.1 m (2^21 cells), 2 propositions at ~1 % and "
             "~90 % fill",
    "serving": "request loop: Poisson arrivals at 2,000 req/s, each a random pose + 32 world planes (256x256 at "
               "0.25 m) against one of 8 resident roadmaps of 20k-1M edges; continuous batching over 2 lanes vs one "
               "request per launch; latency = scheduled arrival to labels in host memory",
    "paper3d": "1,097,702 arcs travelled at 8-15 m/s in a time-augmented (x, y, tau) workspace of 128x128x128 = 2^21 "
               "cells (0.4 m, 0.05 s; 3-D z-order), 2 propositions: moving vehicles (~1 %) and outside a lane loop "
               "(~90 %); 472 swept cells per edge",
    "batched": "64 frames/agents with roadmaps of log-uniform 10k-500k edges on 128^2-512^2 z-order grids at 0.25 m, "
               "8-64 propositions each, one CUDA-graph replay of the batched launch per step vs 64 frame-by-frame "
               "transform+label call pairs",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--workload", default="large", choices=sorted(WORKLOADS))
    ap.add_argument("--requests", type=int, default=20_000, help="serving: requests at the first rate")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--algo", default="quad", choices=["auto", "csr", "bittile", "sector", "quad", "mma"],
                    help="labeling form; auto = measure every form on the first frame and keep the fastest")
    ap.add_argument("--lanes", type=int, default=0)
    ap.add_argument("--early-exit", type=int, default=-1)
    ap.add_argument("--pipeline", type=int, default=0, help="1 registers, 2 bulk copies, 3 cp.async")
    ap.add_argument("--ctas", type=int, default=0)
    ap.add_argument("--depth", type=int, default=0)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--edges", type=int, default=None, help="shrink the workload (not for reported numbers)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-csr-form", action="store_true", help="skip timing the CSR form beside the quadtree form")
    ap.add_argument("--transform", default="auto", choices=["auto", "pyramid", "packed", "direct"],
                    help="frame transform: planes packed into words, then one gather per agent cell (pyramid: "
                         "the same kernel also builds the quadtree pyramid the labels gather from); or byte "
                         "gathers; auto packs as sessions do (planes of 8 MiB or more, world <= 4x agent cells) "
                         "and builds the pyramid in the transform for the quadtree form on z-order grids")
    ap.add_argument("--no-extras", action="store_true", help="skip the reduced batched and serving measurements "
                    "of the default line")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--clocks-csv", default=None, help="keep the raw clock samples in this file")
    ap.add_argument("--steps-csv", default=None, help="write every timed step's device times (ms) to this file")
    ap.add_argument("--rates", default="2000,5000,10000,15000", help="serving: request rates (req/s); the first is the "
                    "configured rate of the headline line, the others a saturation sweep")
    return ap.parse_args()


def rank_seed(seed: int, rank: int) -> int:
    """Every rank labels its own independent roadmap and frame."""
    return seed + 1000 * rank


def max_over_ranks(x: float, dist, device) -> float:
    """The job's time is the slowest rank's."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, edges: int, props: int, steps: int, total_ms: float) -> float:
    """Edge x proposition labels per second over all ranks (weak scaling:
    every rank labels edges x props per step)."""
    return world * edges * props * steps / (total_ms / 1e3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------- enqueue gate

class Gate:
    """Timed steps are enqueued in blocks, each behind a fixed-length spin
    kernel (torch.cuda._sleep) on the timing stream, with the device idle
    before it.  The host then queues the whole block while the device spins,
    so a host pause inside the block (pauses of 40-55 ms were seen on the GPU
    hosts, longer than the ~46 ms of work the driver queue holds) cannot
    leave the device idle between a step's events.  The spin and the idle
    time between blocks are outside every timed interval.  A block whose host
    enqueue took longer than the spin (a host pause longer than the spin) may
    hold device time spent waiting for the host: it is enqueued and timed
    again, up to `retries` times, its steps' events recorded anew.  `redone`
    counts those re-runs, `late` the blocks still late after them (0 = no
    timed step can have waited for the host)."""

    def __init__(self, torch, stream, block: int = 64, ms: float = 20.0, retries: int = 3):
        self.torch, self.stream, self.block, self.ms, self.retries = torch, stream, block, ms, retries
        self.host_ms = []
        self.redone = 0
        self.late = 0
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        cal = 2_000_000
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            a.record(stream)
            torch.cuda._sleep(cal)
            b.record(stream)
        torch.cuda.synchronize()
        self.cycles = int(cal * ms / max(a.elapsed_time(b), 1e-3))

    def blocks(self, n: int):
        for b0 in range(0, n, self.block):
            for attempt in range(1 + self.retries):
                self.torch.cuda.synchronize()
                with self.torch.cuda.stream(self.stream):
                    self.torch.cuda._sleep(self.cycles)
                t = time.perf_counter()
                yield range(b0, min(n, b0 + self.block))
                h = (time.perf_counter() - t) * 1e3
                self.host_ms.append(h)
                if h <= self.ms:
                    break
                if attempt == self.retries:
                    self.late += 1
                else:
                    self.redone += 1

    def summary(self) -> dict:
        return {"block_steps": self.block, "gate_ms": self.ms, "blocks": len(self.host_ms) - self.redone,
                "host_enqueue_ms_max": max(self.host_ms) if self.host_ms else 0.0,
                "redone": self.redone, "late": self.late}


# --------------------------------------------------------------------- clocks

CLOCK_FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    """nvidia-smi clock and throttle samples every 100 ms while the timed region
    runs, into `path` (a temporary file unless --clocks-csv names one)."""

    csv_path = None  # set from --clocks-csv

    def __init__(self, index: int, enabled: bool = True):
        self.proc = None
        self.path = None
        if not enabled:
            return
        try:
            if ClockSampler.csv_path:
                self.path = ClockSampler.csv_path
            else:
                fd, self.path = tempfile.mkstemp(prefix=f"lbl_clocks_gpu{index}_", suffix=".csv")
                os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={CLOCK_FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            # the sampler's start-up (its first query of the GPU) happens before
            # the timed region: wait, at most 1.5 s, for its first sample
            t_end = time.time() + 1.5
            while time.time() < t_end and self.proc.poll() is None and os.path.getsize(self.path) == 0:
                time.sleep(0.01)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self, t0: float, t1: float):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                ts = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                rows.append((ts, float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not ClockSampler.csv_path:
            try:
                os.remove(self.path)
            except OSError:
                pass
        inside = [r for r in rows if t0 - 1.0 <= r[0] <= t1 + 1.0] or rows
        if not inside:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in inside for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": float(np.median([r[1] for r in inside])), "sm_max_mhz": max(r[2] for r in inside),
                "reasons": reasons, "samples": len(inside)}


# ------------------------------------------------------------------- roofline

def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


def pyramid_words(cells: int, levels: int = 4) -> int:
    return sum(cells >> (2 * k) for k in range(levels + 1))


def pyramid_word_bytes(P: int) -> int:
    """Width of the per-frame pyramid words the library uses for P propositions."""
    return 1 if P <= 8 else 2 if P <= 16 else 4 if P <= 32 else 8


def label_bytes(wl, algo: str, n_bt: int | None, with_monitor: bool, n_sec: int | None = None,
                n_qd: int | None = None, from_pyramid: bool = False) -> int:
    """Algorithmic HBM bytes of one labeling call (each array read or written
    once; O, the bit planes and the pyramid counted once although they are
    re-read from L2).  from_pyramid: the quadtree call gathers from the
    pyramid the frame transform built (no O read, no pyramid written)."""
    E = wl.n_edges
    out = 8 * E + (10 * E if with_monitor else 0)
    if algo == "quad":  # pyramid: O read, pyramid written; stream: entries, rows, row order, pyramid once
        perm = 4 * E if 1 < E < 2**31 else 0  # the caller's edge of each row (rows are in locality order)
        pyr = pyramid_word_bytes(wl.P) * pyramid_words(wl.agent.cells)
        if from_pyramid:
            return 4 * n_qd + 8 * (E + 1) + perm + pyr + out
        return 4 * n_qd + 8 * (E + 1) + perm + 8 * wl.agent.cells + 2 * pyr + out
    if algo == "sector":
        return 4 * n_sec + 8 * (E + 1) + 8 * wl.agent.cells + out
    if algo == "mma":  # tile-block bits and ids, tile offsets, row order; per frame O read, B written and read
        n_mma, tiles = n_qd
        return (2048 + 4) * n_mma + 8 * (tiles + 1) + 4 * E + 8 * wl.agent.cells + 2 * mma_n(wl.P) * wl.agent.cells + out
    if algo == "bittile":
        blocks = (wl.agent.cells + 63) // 64
        return 12 * n_bt + 8 * (E + 1) + 8 * wl.agent.cells + 8 * wl.P * blocks + out
    return 4 * wl.nnz + 8 * (E + 1) + 8 * wl.agent.cells + out


def mma_n(P: int) -> int:
    """Columns of the tensor-core form's B operand for P propositions."""
    return 16 if P <= 16 else 32 if P <= 32 else 64


def committed_traffic(kernel_src: str, workload: str, algo: str):
    """Per-launch DRAM bytes from the committed ncu summary, if it was taken on
    the current kernel source (matching hash) and scaled to this workload."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    h = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()[:16]
    for line in open(path):
        t = line.split()
        if len(t) >= 4 and t[0] == workload and t[1] == algo and t[2] == h:
            return float(t[3])
    return None


def workload_config(args, wl, world: int) -> dict:
    """The `config` of both arms' JSON lines: the workload alone (which form
    and transform the GPU arm ran is reported beside it, under `path`)."""
    return {"workload": WORKLOADS[args.workload], "name": args.workload, "edges": int(wl.n_edges), "nnz": int(wl.nnz),
            "props": int(wl.P), "grid": "x".join(str(v) for v in (wl.agent.w, wl.agent.h, wl.agent.d) if v > 1),
            "monitor": wl.monitor is not None,
            "l2": f"flushed before every step (256 MiB write); CSR {(4 * wl.nnz) / 1e9:.3f} GB "
                  + ("> L2" if 4 * wl.nnz > (129 << 20) else "< L2 (each step starts with a flushed L2)"),
            "parallelism": f"replicas x{world}"}


def mma_roofline(wl, form, label_s: float, peaks, hbm_achieved: float, hbm_peak: float, lb: int) -> dict:
    """The tensor-core form against the fp8 tensor peak: 2 x 128 x N x 128
    flops per (tile, 128-cell block) pair.  The fp8 peak is the measured bf16
    burst peak times the nominal fp8/bf16 ratio of 2."""
    n_mma, tiles = form
    flops = 2.0 * 128 * mma_n(wl.P) * 128 * n_mma
    bf16 = (peaks or {}).get("bf16_tflops") or 1900.0
    peak = 2.0 * bf16
    achieved = flops / label_s / 1e12
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": None, "kernel": "label_mma", "flops_per_launch": flops, "tile_blocks": n_mma, "tiles": tiles,
            "peak_source": ("measured bf16 x 2 (fp8 nominal ratio)" if peaks else "fallback bf16 x 2"),
            "hbm": {"achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s", "frac": hbm_achieved / hbm_peak,
                    "algorithmic_bytes_per_launch": lb}}


def l1_roofline(kernel_src: str, workload: str, algo: str, E: int, label_s: float, clk, peaks):
    """The labeling call against its L1 ceiling: LSU data-pipe wavefronts per
    edge from the committed ncu capture (taken on a cut of the same workload,
    on the current kernel source: matching hash), scaled to E edges, per SM
    and clock, against the pipe's one wavefront per clock per SM."""
    path = os.path.join(ROOT, "profiles", "l1.txt")
    if not os.path.exists(path):
        return None
    h = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()[:16]
    for line in open(path):
        t = line.split()
        if len(t) >= 6 and t[0] == workload and t[1] == algo and t[2] == h:
            wpe, spe, sms = float(t[3]), float(t[4]), int(t[5])
            mhz = (clk or {}).get("sm_mhz") or (peaks or {}).get("sm_max_mhz") or 2070.0
            per_launch = wpe * E
            achieved = per_launch / label_s / (sms * mhz * 1e6)
            return {"unit": "LSU data-pipe wavefronts per SM-clock", "achieved": achieved, "peak": 1.0,
                    "frac": achieved, "wavefronts_per_launch": per_launch, "wavefronts_per_edge": wpe,
                    "l1_sectors_per_edge": spe, "sm_mhz": mhz, "sms": sms,
                    "source": "profiles/l1.txt (ncu, cut of the workload, scaled by edges)"}
    return None


# ------------------------------------------------------------------ reference

def cpu_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_step_times(wl, n_sample: int, threads: int):
    """Oracle times on a sample of one frame: (total, transform) seconds for the
    frame transform of the whole grid, labels of the first n_sample edges and
    the monitor on them."""
    import oracle
    rp = wl.rowptr[: n_sample + 1]
    ci = wl.colidx[: int(rp[-1])]
    t = time.perf_counter()
    if wl.agent.d > 1:
        O = oracle.frame_transform3(wl.world, wl.planes, wl.pose, wl.agent)
    else:
        O = oracle.frame_transform(wl.world, wl.planes, wl.pose, wl.agent)
    t_tr = time.perf_counter() - t
    Lw = oracle.label(rp, ci, O, wl.P, threads=threads)
    if wl.monitor is not None:
        m = wl.monitor
        oracle.monitor(m.n_states, m.m, m.relbits, m.delta, m.reject, Lw)
    return time.perf_counter() - t, t_tr


def oracle_step_rate(wl, n_sample: int, threads: int):
    return oracle_step_times(wl, n_sample, threads)[0]


def oracle_frame_seconds(wl, n_sample: int, t_total: float, t_transform: float) -> float:
    """A whole frame's oracle time from a sample: the transform once, the
    per-edge part scaled from n_sample edges to all of them."""
    return t_transform + (t_total - t_transform) * wl.n_edges / max(n_sample, 1)


def calibrate_sample(wl, seconds: float, threads: int) -> int:
    """Edges per oracle frame so that one frame takes about `seconds`: two
    probe sizes separate the fixed cost (whole-grid transform) from the
    per-edge cost."""
    n1 = min(wl.n_edges, 2000)
    n2 = min(wl.n_edges, 20000)
    t1 = oracle_step_rate(wl, n1, threads)
    if n2 == n1:
        return n1
    t2 = oracle_step_rate(wl, n2, threads)
    per_edge = max((t2 - t1) / (n2 - n1), 1e-9)
    fixed = max(t1 - per_edge * n1, 0.0)
    return int(min(wl.n_edges, max(1000, (seconds - fixed) / per_edge)))


def cpu_baseline(wl, seconds: float, with_monitor: bool) -> dict:
    """The oracle on the host: OpenMP over edges on every core this process may
    use (the baseline), and on one thread (a second, single-thread figure),
    each on a bounded sample of one frame."""
    E, P = wl.n_edges, wl.P
    threads = cpu_cores()
    n = calibrate_sample(wl, seconds, threads)
    dt, dtr = oracle_step_times(wl, n, threads)
    n1 = calibrate_sample(wl, seconds / 3.0, 1)
    dt1, dtr1 = oracle_step_times(wl, n1, 1)
    what = " + monitor" if with_monitor else ""
    return {"value": E * P / oracle_frame_seconds(wl, n, dt, dtr), "unit": UNIT, "cores": threads,
            "cores_total": os.cpu_count(), "kind": "oracle",
            "sample": f"one frame: whole-grid frame transform + labels of the first {n} of {E} edges{what} "
                      f"({dt:.1f} s on {threads} threads); a whole frame's time = transform + label time x {E}/{n}",
            "single_thread": {"value": E * P / oracle_frame_seconds(wl, n1, dt1, dtr1), "unit": UNIT, "cores": 1,
                              "sample": f"the same on one thread, first {n1} edges ({dt1:.1f} s)"}}


def run_reference(args, rank, world):
    if rank != 0:
        return
    if args.workload == "paper3d":
        wl = synth.make_paper3d(seed=args.seed, threads=cpu_cores(), **({"edges": args.edges} if args.edges else {}))
    else:
        wl = synth.make(args.workload, seed=args.seed, edges=args.edges, threads=cpu_cores())
    threads = cpu_cores()
    # about two minutes for the whole run: each step a sample of ~120 s / steps
    # (at least 1,000 edges, at most the whole frame)
    per_step = min(6.0, 120.0 / max(args.steps + args.warmup, 1))
    n = calibrate_sample(wl, per_step, threads)
    for _ in range(args.warmup):
        oracle_step_rate(wl, n, threads)
    samples = [oracle_step_times(wl, n, threads) for _ in range(args.steps)]
    tot = sum(oracle_frame_seconds(wl, n, a, b) for a, b in samples)
    value = wl.n_edges * wl.P * args.steps / tot
    sample = (f"per step: whole-grid frame transform + labels (and monitor) of the first {n} of {wl.n_edges} "
              f"edges; a whole frame's time = transform + label time x {wl.n_edges}/{n}; {args.steps} steps, "
              f"{sum(a for a, b in samples):.1f} s of oracle work")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": workload_config(args, wl, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "cores_total": os.cpu_count(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------ ours

def main():
    args = parse()
    ClockSampler.csv_path = args.clocks_csv
    rank, world, local = dist_env()
    if args.impl == "reference":
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("gloo")
        run_reference(args, rank, world)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import paper_1810_02612_gb300 as L
    from paper_1810_02612_gb300.lbl import lbl_config

    if args.workload == "serving":
        run_serving(args, rank, world, local, dist, torch, L)
        if dist:
            dist.destroy_process_group()
        return
    if args.workload == "batched":
        run_batched(args, rank, world, local, dist, torch, L)
        if dist:
            dist.destroy_process_group()
        return

    # ---- inputs: every rank its own independent roadmap and frame
    t_gen = time.perf_counter()
    if args.workload == "paper3d":
        wl = synth.make_paper3d(seed=rank_seed(args.seed, rank), threads=cpu_cores(),
                                **({"edges": args.edges} if args.edges else {}))
    else:
        wl = synth.make(args.workload, seed=rank_seed(args.seed, rank), edges=args.edges, threads=cpu_cores())
    t_gen = time.perf_counter() - t_gen
    algo = {"auto": L.LBL_ALGO_AUTO, "csr": L.LBL_ALGO_CSR, "bittile": L.LBL_ALGO_BITTILE,
            "sector": L.LBL_ALGO_SECTOR, "quad": L.LBL_ALGO_QUAD, "mma": L.LBL_ALGO_MMA}[args.algo]
    flags = ((L.LBL_UPLOAD_BITTILE if args.algo in ("auto", "bittile") else 0)
             | (L.LBL_UPLOAD_SECTOR if args.algo in ("auto", "sector") else 0)
             | (L.LBL_UPLOAD_QUAD if args.algo in ("auto", "quad") else 0)
             | (L.LBL_UPLOAD_MMA if args.algo == "mma" else 0))
    stream = torch.cuda.Stream()
    t_up = time.perf_counter()
    rm = L.lbl_roadmap_upload(wl.agent, wl.rowptr, wl.colidx, flags=flags, stream=stream)
    t_up = time.perf_counter() - t_up
    mon = None
    if wl.monitor is not None:
        m = wl.monitor
        mon = L.lbl_monitor_create(m.n_states, m.m, m.relbits, m.delta, m.reject)
    E, P = wl.n_edges, wl.P
    cfg = lbl_config(algo, args.lanes, args.early_exit, args.ctas, args.pipeline, args.depth)
    with torch.cuda.stream(stream):
        d_planes = torch.from_numpy(wl.planes).to("cuda", non_blocking=False)
        d_O = torch.empty(wl.agent.cells, dtype=torch.uint64, device="cuda")
        d_L = torch.empty(E, dtype=torch.uint64, device="cuda")
        d_next = torch.empty(E, dtype=torch.uint64, device="cuda") if mon else None
        d_viol = torch.empty(E, dtype=torch.uint16, device="cuda") if mon else None
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        d_words = torch.empty(wl.world.cells, dtype=getattr(torch, L.packed_word_dtype(P)), device="cuda")
    torch.cuda.synchronize()
    auto_transform = args.transform == "auto"
    if auto_transform:
        args.transform = ("packed" if P * wl.world.cells >= (8 << 20) and wl.world.cells <= 4 * wl.agent.cells
                          else "direct")

    def transform():
        if args.transform in ("packed", "pyramid"):
            L.lbl_pack_planes(wl.world, d_planes, P, d_words, stream=stream)
        if args.transform == "pyramid":
            L.lbl_frame_transform_pyramid(rm, wl.world, d_words, P, wl.pose, d_O, stream=stream)
        elif args.transform == "packed":
            L.lbl_frame_transform_words(wl.world, d_words, P, wl.pose, wl.agent, d_O, stream=stream)
        else:
            L.lbl_frame_transform(wl.world, d_planes, P, wl.pose, wl.agent, d_O, stream=stream)

    def label():
        if args.transform == "pyramid":
            L.lbl_label_pyramid(rm, P, d_L, mon, d_next, d_viol, cfg, stream=stream)
        else:
            L.lbl_label(rm, d_O, P, d_L, mon, d_next, d_viol, cfg, stream=stream)

    def step():
        transform()
        label()

    # AUTO: measure every labeling variant on this frame once (untimed) and
    # let the roadmap keep the fastest
    tuned = None
    if args.algo == "auto":
        transform()
        tuned = L.lbl_roadmap_autotune(rm, d_O, P, d_L, mon, d_next, d_viol, reps=5, stream=stream)
        used = {L.LBL_ALGO_BITTILE: "bittile", L.LBL_ALGO_SECTOR: "sector",
                L.LBL_ALGO_QUAD: "quad", L.LBL_ALGO_MMA: "mma"}.get(tuned["algo"], "csr")
    else:
        used = args.algo
    # the transform builds the pyramid in one launch on z-order grids and on 2-D
    # row-major grids of whole 16 x 16 tiles (the quadtree form's tiled order)
    one_launch = (wl.agent.order == synth.MORTON
                  or (wl.agent.d <= 1 and wl.agent.w % 16 == 0 and wl.agent.h % 16 == 0))
    if auto_transform and used == "quad" and one_launch and P > 0:
        args.transform = "pyramid"  # measured at least as fast as either transform + pyramid launch
    if args.transform == "pyramid" and (used != "quad" or not one_launch):
        raise SystemExit("--transform pyramid needs the quadtree form on a z-order or tiled row-major agent grid")
    launches_per_step = (2 + (1 if used in ("bittile", "quad", "mma") and args.transform != "pyramid" else 0)
                         + (1 if args.transform in ("packed", "pyramid") else 0))  # + planes / pyramid / B, packing

    # ---- warm-up (the flush fills too: a kernel's first launch in the process
    # loads its module and can wait for the device)
    for w in range(args.warmup):
        with torch.cuda.stream(stream):
            flush.fill_(w & 255)
        step()
    torch.cuda.synchronize()

    # ---- device-timed steps (L2 flushed before each)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local, enabled=not args.no_clocks and rank == 0)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    gate = Gate(torch, stream)
    gc.disable()  # no collector pause while the host enqueues the timed steps
    t0 = time.time()
    for blk in gate.blocks(args.steps):
        for i in blk:
            with torch.cuda.stream(stream):
                flush.fill_(i & 255)
            ev[i][0].record(stream)
            transform()
            ev[i][1].record(stream)
            label()
            ev[i][2].record(stream)
    torch.cuda.synchronize()
    t1 = time.time()
    gc.enable()
    gates = {"steps": gate.summary()}
    if dist:
        dist.barrier()
    step_ms = np.array([a.elapsed_time(c) for a, b, c in ev])
    frame_ms = np.array([a.elapsed_time(b) for a, b, c in ev])
    label_ms = np.array([b.elapsed_time(c) for a, b, c in ev])
    clk = clocks.stop(t0, t1)
    if args.steps_csv and rank == 0:
        np.savetxt(args.steps_csv, np.stack([step_ms, frame_ms, label_ms], 1), fmt="%.5f",
                   header="step_ms,transform_ms,label_ms", delimiter=",")
    total_ms = max_over_ranks(float(step_ms.sum()), dist, "cuda")
    value = job_throughput(world, E, P, args.steps, total_ms)

    # ---- the CSR form on the same frame and roadmap, for its roofline (the
    # quadtree form moves five times fewer bytes, so its fraction is lower)
    csr_line = None
    if used == "quad" and not args.no_csr_form:
        csr_cfg = lbl_config(L.LBL_ALGO_CSR, 0, 0, args.ctas, 0, 0)
        n_csr = max(10, min(args.steps, 200))
        cev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_csr)]
        for _ in range(3):
            L.lbl_label(rm, d_O, P, d_L, mon, d_next, d_viol, csr_cfg, stream=stream)
        cgate = Gate(torch, stream)
        for blk in cgate.blocks(n_csr):
            for i in blk:
                with torch.cuda.stream(stream):
                    flush.fill_(i & 255)
                cev[i][0].record(stream)
                L.lbl_label(rm, d_O, P, d_L, mon, d_next, d_viol, csr_cfg, stream=stream)
                cev[i][1].record(stream)
        torch.cuda.synchronize()
        gates["csr_form"] = cgate.summary()
        csr_s = float(np.mean([a.elapsed_time(b) for a, b in cev])) / 1e3
        csr_b = label_bytes(wl, "csr", None, mon is not None)
        peaks0 = measured_peaks()
        pk = peaks0["hbm_gbs"] if peaks0 else 6800.0
        csr_line = {"bound": "hbm", "achieved": csr_b / csr_s / 1e9, "peak": pk, "unit": "GB/s",
                    "frac": csr_b / csr_s / 1e9 / pk, "label_ms": csr_s * 1e3, "launches": n_csr,
                    "traffic": committed_traffic(os.path.join(ROOT, "paper_1810_02612_gb300", "csrc", "k_label.cu"),
                                                 args.workload, "csr") if args.edges is None else None,
                    "kernel": "label_csr", "algorithmic_bytes_per_launch": csr_b,
                    "peak_source": "measured" if peaks0 else "fallback"}

    # ---- end to end through the session API with pinned host buffers
    ss = L.lbl_session_create(rm, wl.world, P, mon, cfg)
    h_planes = torch.from_numpy(wl.planes).pin_memory()
    h_L = torch.empty(E, dtype=torch.uint64).pin_memory()
    h_next = torch.empty(E, dtype=torch.uint64).pin_memory() if mon else None
    h_viol = torch.empty(E, dtype=torch.uint16).pin_memory() if mon else None
    for _ in range(args.warmup):
        L.lbl_session_run(ss, h_planes, wl.pose, h_L, h_next, h_viol, stream=stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    # (1) frame latency: each frame alone, L2 flushed and the device idle
    # before it (so its host-to-device copy starts inside the timed region)
    n_lat = min(args.steps, 400)
    e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_lat)]
    for i in range(n_lat):
        with torch.cuda.stream(stream):
            flush.fill_(i & 255)
        torch.cuda.synchronize()
        e_ev[i][0].record(stream)
        L.lbl_session_run(ss, h_planes, wl.pose, h_L, h_next, h_viol, stream=stream)
        e_ev[i][1].record(stream)
    torch.cuda.synchronize()
    e2e_ms_steps = np.array([a.elapsed_time(b) for a, b in e_ev])
    # (2) throughput: frames back to back, every frame's H2D and D2H inside
    # the timed region (the roadmap rows exceed L2, so no flush is needed)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    # (not gated: the session's own streams do not wait for the caller's stream,
    # so a spin there would overlap the frames instead of preceding them)
    t_a, t_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    gc.disable()
    t_a.record(stream)
    for i in range(args.steps):
        L.lbl_session_run(ss, h_planes, wl.pose, h_L, h_next, h_viol, stream=stream)
    t_b.record(stream)
    torch.cuda.synchronize()
    gc.enable()
    e2e_ms = max_over_ranks(float(t_a.elapsed_time(t_b)), dist, "cuda")
    e2e_value = job_throughput(world, E, P, args.steps, e2e_ms)
    h2d = int(wl.planes.nbytes)
    d2h = 8 * E + ((8 + 2) * E if mon else 0)
    L.lbl_session_free(ss)

    # ---- roofline of the dominant kernel (labeling)
    info = L.lbl_roadmap_info(rm)
    qd_or_mma = L.lbl_roadmap_form_info(rm, L.LBL_ALGO_MMA) if used == "mma" else info[4]
    lb = label_bytes(wl, used, info[2], mon is not None, info[3], qd_or_mma, from_pyramid=args.transform == "pyramid")
    label_avg_s = float(label_ms.mean()) / 1e3
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    achieved = lb / label_avg_s / 1e9
    kernel_src = os.path.join(ROOT, "paper_1810_02612_gb300", "csrc", "k_label.cu")
    full_size = args.edges is None
    # the committed captures are of the default call; for the quadtree form that
    # is the front alone, gathering from the pyramid the transform built
    pin = used if used != "quad" or args.transform == "pyramid" else "quad_with_pyramid_kernel"
    traffic = committed_traffic(kernel_src, args.workload, pin) if full_size else None
    l1 = l1_roofline(kernel_src, args.workload, pin, E, label_avg_s, clk, peaks)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl, args.cpu_seconds, mon is not None)

    more = {}
    if world == 1 and args.workload == "large" and not args.no_extras:
        more = extras(args, rank, torch, L)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": workload_config(args, wl, world),
            "path": {"algo": used, "tuned": tuned, "transform": args.transform,
                     "cfg": {"lanes_per_edge": args.lanes, "early_exit": args.early_exit, "ctas_per_sm": args.ctas,
                             "pipeline": args.pipeline, "depth": args.depth}},
            "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                           "frame_transform_avg": float(frame_ms.mean()), "label_avg": float(label_ms.mean()),
                           "e2e_p50": float(np.percentile(e2e_ms_steps, 50)),
                           "e2e_p99": float(np.percentile(e2e_ms_steps, 99))},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": e2e_ms / args.steps,
                    "mode": "lbl_session_run frames back to back from pinned host memory; each frame's "
                            "H2D planes and D2H labels/monitor outputs inside the timed region"},
            "gpu_launches": launches_per_step * args.steps,
            "mma_probe": mma_probe(L) if used == "mma" else None,
            "roofline": mma_roofline(wl, qd_or_mma, label_avg_s, peaks, achieved, peak, lb) if used == "mma" else
                        {"bound": "l1" if l1 and l1["frac"] >= achieved / peak else "hbm",  # the fuller one
                         "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": f"label_{used}", "algorithmic_bytes_per_launch": lb,
                         "csr_equivalent_gbs": label_bytes(wl, "csr", None, mon is not None) / label_avg_s / 1e9,
                         "peak_source": "measured" if peaks else "fallback", "l1": l1},
            "roofline_csr_form": csr_line,
            "cpu_baseline": cpu,
            "clocks": clk,
            "enqueue_gates": gates,
            "setup_s": {"generate": t_gen, "upload": t_up},
        }
        line.update(more)
        print(json.dumps(line), flush=True)

    if mon:
        L.lbl_monitor_free(mon)
    L.lbl_roadmap_free(rm)
    if dist:
        dist.destroy_process_group()


def measure_batched(torch, L, frames, steps: int, warmup: int, algo: str, dist=None, clocks=None, tune=True):
    """Batched frames: one graph replay of the batched launches per step against
    the same frames labeled by frame-by-frame transform + label call pairs (same
    buffers, L2 flushed before every step), checked bit for bit.  With `tune`
    the batch's label plan is chosen by lbl_batch_autotune before the graph is
    captured (and checked bit for bit again)."""
    stream = torch.cuda.Stream()
    rms, fr = [], []
    quad = algo in ("quad", "auto")
    for f in frames:
        rms.append(L.lbl_roadmap_upload(f.agent, f.rowptr, f.colidx, flags=L.LBL_UPLOAD_QUAD if quad else 0,
                                        stream=stream))
    for f in frames:
        d_pl = torch.from_numpy(np.ascontiguousarray(f.planes)).cuda()
        fr.append(dict(world=f.world, d_planes=d_pl, pose=f.pose,
                       d_O=torch.empty(f.agent.cells, dtype=torch.uint64, device="cuda"),
                       d_L=torch.empty(f.n_edges, dtype=torch.uint64, device="cuda")))

    def frame_transform(f, d):
        L.lbl_frame_transform(f.world, d["d_planes"], f.P, f.pose, f.agent, d["d_O"], stream=stream)
    torch.cuda.synchronize()  # frame buffers were filled on the default stream; the launches use `stream`
    b = L.lbl_batch_create(rms, [f.P for f in frames])
    L.lbl_batch_set_frames(b, fr)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def plain_step():
        for f, r, d in zip(frames, rms, fr):
            frame_transform(f, d)
            L.lbl_label(r, d["d_O"], f.P, d["d_L"], stream=stream)

    # correctness: batched == frame by frame, bit for bit
    plain_step()
    torch.cuda.synchronize()
    ref = [d["d_L"].clone() for d in fr]
    for d in fr:
        d["d_L"].zero_()
    L.lbl_batch_launch(b, stream=stream)
    torch.cuda.synchronize()
    match = all(torch.equal(a.view(torch.int64), d["d_L"].view(torch.int64)) for a, d in zip(ref, fr))
    tuning = None
    if tune:
        tuning = [t for t in L.lbl_batch_autotune(b, reps=5, stream=stream) if t["items"] > 0]
        for d in fr:
            d["d_L"].zero_()
        torch.cuda.synchronize()
        L.lbl_batch_launch(b, stream=stream)
        torch.cuda.synchronize()
        match = match and all(torch.equal(a.view(torch.int64), d["d_L"].view(torch.int64)) for a, d in zip(ref, fr))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        L.lbl_batch_launch(b, stream=torch.cuda.current_stream())

    gates = {}

    def timed(fn, n, name="", cmds=4, ms=20.0):
        # cmds: commands one step queues; a gated block holds at most ~800
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        gate = Gate(torch, stream, block=max(1, min(64, 800 // cmds)), ms=ms)
        for blk in gate.blocks(n):
            for i in blk:
                with torch.cuda.stream(stream):
                    flush.fill_(i & 255)
                ev[i][0].record(stream)
                fn()
                ev[i][1].record(stream)
        torch.cuda.synchronize()
        if name:
            gates[name] = gate.summary()
        return np.array([a.elapsed_time(c) for a, c in ev])

    for w in range(warmup):
        with torch.cuda.stream(stream):
            flush.fill_(w & 255)
        plain_step()
        g.replay()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.time()
    with torch.cuda.stream(stream):
        batched_ms = timed(lambda: g.replay(), steps, "batched")
    t1 = time.time()
    clk = clocks.stop(t0, t1) if clocks else None
    nf = len(frames)
    plain_ms = timed(plain_step, steps, "plain", cmds=3 + 4 * nf, ms=50.0)
    # where the time goes: each stage alone, batched and frame by frame
    n_br = max(5, steps // 5)
    with torch.cuda.stream(stream):
        b_tr = timed(lambda: L.lbl_batch_launch(b, L.LBL_STAGE_TRANSFORM, stream=stream), n_br, cmds=6)
        b_lb = timed(lambda: L.lbl_batch_launch(b, L.LBL_STAGE_LABEL, stream=stream), n_br, cmds=8)
    p_tr = timed(lambda: [frame_transform(f, d) for f, d in zip(frames, fr)], n_br, cmds=3 + nf, ms=50.0)
    p_lb = timed(lambda: [L.lbl_label(r, d["d_O"], f.P, d["d_L"], stream=stream)
                          for f, r, d in zip(frames, rms, fr)], n_br, cmds=3 + 3 * nf, ms=50.0)
    entries = [L.lbl_roadmap_info(r)[4] if quad else f.nnz for f, r in zip(frames, rms)]
    L.lbl_batch_free(b)
    for r in rms:
        L.lbl_roadmap_free(r)
    packs = any(f.P > 0 and f.world.cells <= 4 * f.agent.cells for f in frames)  # frames the batch packs
    label_classes = len({pyramid_word_bytes(f.P) if quad else 8 for f in frames})  # one label launch per word width
    bytes_step = sum(4 * n + 16 * f.n_edges + 8 * f.agent.cells + f.P * f.world.cells
                     + (2 * pyramid_word_bytes(f.P) * pyramid_words(f.agent.cells) if quad else 0)
                     for f, n in zip(frames, entries))
    return {"batched_ms": batched_ms, "plain_ms": plain_ms, "match": bool(match), "clk": clk, "tuning": tuning,
            "gates": gates,
            "units": sum(f.n_edges * f.P for f in frames), "entries": int(sum(entries)), "bytes_step": bytes_step,
            "launches": 1 + int(packs) + int(quad) + label_classes,  # (pack,) transform, (pyramid,) labels
            "plain_launches": len(frames) * (3 if quad else 2),  # transform, (pyramid,) label per frame
            "stage_ms": {"batched_transform": float(np.median(b_tr)), "batched_label": float(np.median(b_lb)),
                         "plain_transform": float(np.median(p_tr)), "plain_label": float(np.median(p_lb))}}


def batched_summary(m: dict, frames, steps: int) -> dict:
    """The batched-vs-plain comparison as one JSON object."""
    units = m["units"]
    tb, tp = float(m["batched_ms"].sum()), float(m["plain_ms"].sum())
    return {"frames": len(frames), "edges": int(sum(f.n_edges for f in frames)), "steps": steps,
            "value": units * steps / (tb / 1e3), "plain_value": units * steps / (tp / 1e3), "unit": UNIT,
            "batched_ms_per_step": tb / steps, "plain_ms_per_step": tp / steps, "speedup": tp / tb,
            "bit_exact_match": m["match"],
            "batched_p50_ms": float(np.percentile(m["batched_ms"], 50)),
            "batched_p99_ms": float(np.percentile(m["batched_ms"], 99)),
            "plain_p50_ms": float(np.percentile(m["plain_ms"], 50)),
            "plain_p99_ms": float(np.percentile(m["plain_ms"], 99)),
            "batched_launches_per_step": m["launches"], "plain_launches_per_step": m["plain_launches"],
            "stage_ms": m["stage_ms"], "tuning": m["tuning"], "enqueue_gates": m["gates"]}


def run_batched(args, rank, world, local, dist, torch, L):
    """64 frames of uneven roadmaps: one graph replay of the batched launch per
    step against 64 frame-by-frame call pairs, same frames and buffers."""
    t_gen = time.perf_counter()
    frames = synth.make_batch(seed=rank_seed(args.seed, rank), threads=cpu_cores())
    t_gen = time.perf_counter() - t_gen
    clocks = ClockSampler(local, enabled=not args.no_clocks and rank == 0)
    m = measure_batched(torch, L, frames, args.steps, args.warmup, args.algo, dist, clocks)
    quad = args.algo in ("quad", "auto")
    total_b = max_over_ranks(float(m["batched_ms"].sum()), dist, "cuda")
    total_p = max_over_ranks(float(m["plain_ms"].sum()), dist, "cuda")
    value = job_throughput(world, m["units"], 1, args.steps, total_b)
    plain_value = job_throughput(world, m["units"], 1, args.steps, total_p)
    nnz = sum(f.nnz for f in frames)
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    achieved = m["bytes_step"] / (total_b / args.steps / 1e3) / 1e9
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_b / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOADS["batched"], "name": "batched", "frames": len(frames),
                       "edges": sum(f.n_edges for f in frames), "nnz": nnz,
                       "l2": "flushed before every step (256 MiB write)", "parallelism": f"replicas x{world}"},
            "path": {"algo": "quad" if quad else "csr", "streamed_entries": m["entries"]},
            "batched_vs_plain": {"plain_value": plain_value, "plain_ms_per_step": total_p / args.steps,
                                 "speedup": total_p / total_b, "bit_exact_match": m["match"],
                                 "plain_launches_per_step": m["plain_launches"],
                                 "batched_launches_per_step": m["launches"], "stage_ms": m["stage_ms"],
                                 "tuning": m["tuning"]},
            "latency_ms": {"batched_p50": float(np.percentile(m["batched_ms"], 50)),
                           "batched_p99": float(np.percentile(m["batched_ms"], 99)),
                           "plain_p50": float(np.percentile(m["plain_ms"], 50)),
                           "plain_p99": float(np.percentile(m["plain_ms"], 99))},
            "gpu_launches": m["launches"] * args.steps,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "kernel": "batched step (frame transforms + labels)",
                         "algorithmic_bytes_per_launch": m["bytes_step"],
                         "peak_source": "measured" if peaks else "fallback"},
            "clocks": m["clk"], "setup_s": {"generate": t_gen},
        }
        print(json.dumps(line), flush=True)


SERVING_SIZES = [20_000, 35_000, 61_000, 107_000, 187_000, 327_000, 572_000, 1_000_000]


def serving_setup(torch, L, seed: int, n_max: int, algo: str, sizes=SERVING_SIZES):
    """Resident roadmaps (prefixes of one pool of arcs on a 256x256 grid), eight
    32-proposition world plane sets in pinned memory, and the seeded request
    stream (unit gaps, roadmap and plane-set choice, pose per request)."""
    rng = np.random.default_rng(seed)
    agent = synth.agent_grid(256, 0.25, synth.MORTON)
    wgrid = synth.world_grid(256, 256, 0.25)
    arcs = synth.sample_arcs(rng, sizes[-1], agent, (-0.3, 0.3), (5.0, 40.0))
    rowptr, colidx = synth.sweep_csr(arcs, 1.2, agent, cpu_cores())
    P = 32
    plane_sets = [torch.from_numpy(synth.planes_mixed(rng, P, wgrid)).pin_memory() for _ in range(8)]
    quad = algo in ("quad", "auto")
    rms = [L.lbl_roadmap_upload(agent, rowptr[: n + 1], colidx[: int(rowptr[n])],
                                flags=L.LBL_UPLOAD_QUAD if quad else 0) for n in sizes]
    req = {"unit_gaps": rng.exponential(1.0, size=n_max), "which": rng.integers(0, len(sizes), size=n_max),
           "sets": rng.integers(0, len(plane_sets), size=n_max),
           "poses": [synth.random_pose(rng, wgrid) for _ in range(n_max)]}
    return {"sizes": sizes, "P": P, "wgrid": wgrid, "plane_sets": plane_sets, "rms": rms, "req": req, "quad": quad,
            "nnz_largest": int(rowptr[-1]),
            "outs": [torch.empty(sizes[-1], dtype=torch.uint64).pin_memory() for _ in range(256)]}


def serve(L, st: dict, max_batch: int, rate: float, n_req: int, warm: int) -> dict:
    """Replay the first n_req requests of the stream at `rate` from a host
    thread; latency = scheduled arrival -> labels in host memory."""
    import threading
    sizes, P, req, outs = st["sizes"], st["P"], st["req"], st["outs"]
    ring = len(outs)
    gaps = req["unit_gaps"][:n_req] / rate
    srv = L.lbl_server_create(st["rms"], [P] * len(sizes), None, lanes=2, mem_budget=4 << 30, max_batch=max_batch)
    tickets = [None] * n_req
    lat = np.zeros(n_req)
    done_t = np.zeros(n_req)
    submitted = threading.Semaphore(0)

    def waiter():
        for i in range(n_req):
            submitted.acquire()
            lat[i] = L.lbl_server_wait(srv, tickets[i], 60000) / 1e6
            done_t[i] = time.monotonic_ns()

    th = threading.Thread(target=waiter)
    th.start()
    t0 = time.monotonic_ns() + 20_000_000
    arrival = t0 + np.cumsum(gaps * 1e9).astype(np.int64)
    for i in range(n_req):
        while time.monotonic_ns() < arrival[i]:
            pass
        if i >= ring:  # the output buffer of request i - ring is free again
            while done_t[i - ring] == 0:
                time.sleep(0)
        k = int(req["which"][i])
        tickets[i] = L.lbl_server_submit(srv, k, st["wgrid"], st["plane_sets"][int(req["sets"][i])],
                                         req["poses"][i], outs[i % ring][: sizes[k]], arrival_ns=int(arrival[i]))
        submitted.release()
    th.join()
    stats = L.lbl_server_stats(srv)
    L.lbl_server_free(srv)
    sel = slice(warm, n_req)
    span_s = (done_t[n_req - 1] - arrival[warm]) / 1e9
    labels = float(sum(sizes[int(k)] for k in req["which"][warm:n_req])) * P
    return {"rate_req_s": rate, "requests": n_req, "warmup": warm,
            "labels_per_s": labels / span_s, "p50_ms": float(np.percentile(lat[sel], 50)),
            "p99_ms": float(np.percentile(lat[sel], 99)), "p999_ms": float(np.percentile(lat[sel], 99.9)),
            "mean_ms": float(lat[sel].mean()), "achieved_req_per_s": (n_req - warm) / span_s,
            "batches": stats["batches"], "mean_batch": n_req / max(stats["batches"], 1),
            "max_batch": stats["max_batch"]}


def run_serving(args, rank, world, local, dist, torch, L):
    """Poisson request stream against 8 resident roadmaps; the same stream is
    served with continuous batching and with one request per launch."""
    rates = [float(x) for x in args.rates.split(",")]
    rate = rates[0]
    n_max = args.requests
    t_gen = time.perf_counter()
    st = serving_setup(torch, L, rank_seed(args.seed, rank), n_max, args.algo)
    t_gen = time.perf_counter() - t_gen
    warm = min(args.warmup * 100, n_max // 10)
    clocks = ClockSampler(local, enabled=not args.no_clocks and rank == 0)
    t0 = time.time()
    cont = serve(L, st, 128, rate, n_max, warm)
    t1 = time.time()
    clk = clocks.stop(t0, t1)
    plain = serve(L, st, 1, rate, n_max, warm)
    sweep = []
    for r in rates[1:]:
        n = min(n_max, 10_000)
        c, p = serve(L, st, 128, r, n, min(warm, n // 10)), serve(L, st, 1, r, n, min(warm, n // 10))
        sweep.append({"rate_req_s": r, "continuous_batching": c, "one_request_per_launch": p,
                      "throughput_gain": c["labels_per_s"] / p["labels_per_s"], "p99_gain": p["p99_ms"] / c["p99_ms"]})
    value = cont["labels_per_s"]
    sizes, P, wgrid, which = st["sizes"], st["P"], st["wgrid"], st["req"]["which"]
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": n_max, "warmup": cont["warmup"],
            "ms_per_step": cont["mean_ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOADS["serving"], "name": "serving", "requests": n_max, "rate_req_s": rate,
                       "roadmap_edges": sizes, "nnz_largest": st["nnz_largest"], "props": P,
                       "parallelism": f"replicas x{world}"},
            "path": {"algo": "quad" if st["quad"] else "csr"},
            "gpu_launches": int(cont["batches"]) * (3 if st["quad"] else 2),
            "serving": {"continuous_batching": cont, "one_request_per_launch": plain,
                        "p99_gain": plain["p99_ms"] / cont["p99_ms"], "saturation_sweep": sweep},
            "latency_ms": {"p50": cont["p50_ms"], "p99": cont["p99_ms"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": P * wgrid.cells,
                    "d2h_bytes_per_step": int(8 * np.mean([sizes[int(k)] for k in which[:n_max]]))},
            "clocks": clk, "setup_s": {"generate": t_gen},
        }
        print(json.dumps(line), flush=True)
    for r in st["rms"]:
        L.lbl_roadmap_free(r)


def extras(args, rank, torch, L) -> dict:
    """Reduced batched and serving measurements for the default line: 16 frames
    of 10k-200k edges (one graph replay vs 16 call pairs, 200 steps), and 2 s of
    Poisson arrivals at 2,000 req/s against the 8 resident roadmaps, then the
    same requests at 10,000 req/s (continuous batching vs one request per
    launch, each)."""
    out = {}
    t = time.perf_counter()
    frames = synth.make_batch(seed=rank_seed(args.seed, rank) + 17, frames=16, edges=(10_000, 200_000),
                              threads=cpu_cores())
    m = measure_batched(torch, L, frames, 200, 5, "quad")
    out["batched"] = batched_summary(m, frames, 200)
    out["batched"]["workload"] = ("16 frames/agents, roadmaps of log-uniform 10k-200k edges on 128^2-512^2 z-order "
                                  "grids at 0.25 m, 8-64 propositions; one CUDA-graph replay of the batched launches "
                                  "vs 16 frame-by-frame transform+label call pairs; L2 flushed before every step")
    n_req, rate, rate_hi = 4000, 2000.0, 10000.0
    st = serving_setup(torch, L, rank_seed(args.seed, rank) + 29, n_req, "quad")
    cont = serve(L, st, 128, rate, n_req, 400)
    plain = serve(L, st, 1, rate, n_req, 400)
    cont_hi = serve(L, st, 128, rate_hi, n_req, 400)
    plain_hi = serve(L, st, 1, rate_hi, n_req, 400)
    for r in st["rms"]:
        L.lbl_roadmap_free(r)
    out["serving"] = {"workload": f"{n_req} requests (2 s) of Poisson arrivals at {rate:.0f} req/s, each a random "
                                  "pose + 32 world planes (256x256 at 0.25 m) against one of 8 resident roadmaps of "
                                  "20k-1M edges; 2 lanes; latency = scheduled arrival to labels in host memory",
                      "continuous_batching": cont, "one_request_per_launch": plain,
                      "p99_gain": plain["p99_ms"] / cont["p99_ms"],
                      "throughput_gain": cont["labels_per_s"] / plain["labels_per_s"],
                      "loaded": {"workload": f"the same {n_req} requests arriving at {rate_hi:.0f} req/s",
                                 "continuous_batching": cont_hi, "one_request_per_launch": plain_hi,
                                 "p99_gain": plain_hi["p99_ms"] / cont_hi["p99_ms"],
                                 "throughput_gain": cont_hi["labels_per_s"] / plain_hi["labels_per_s"]}}
    out["mma_probe"] = mma_probe(L)
    out["extras_s"] = time.perf_counter() - t
    return out


def mma_probe(L) -> dict:
    """Measured tcgen05 rates behind the tensor-core form (lbl_mma_probe): e4m3
    (the form's kind::f8f6f4) at the form's widths and bf16 for comparison; the
    int8 kind does not exist on sm_103a."""
    res = {}
    for kind, n, name in ((0, 64, "e4m3_n64"), (0, 128, "e4m3_n128"), (0, 16, "e4m3_n16"), (1, 64, "bf16_n64")):
        r = L.lbl_mma_probe(kind, n, reps=4000, ctas_per_sm=4)
        res[name] = {"tflops": r["tflops"], "exact": r["exact"]}
    res["int8"] = "tcgen05.mma kind::i8 is rejected by ptxas for sm_103a; the form multiplies 0/1 in e4m3 instead"
    return res


if __name__ == "__main__":
    main()
