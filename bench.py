"""Benchmark of the single-GPU short-range MD hot path.

Headline workload: LJ fluid, N = 16,777,216, density 0.8442, T = 1.2,
r_cut = 2.5, r_skin = 0.4, dt = 0.005, mixed precision (FP32 forces with
compensated accumulation, FP64 positions and integration).  A step is one full
velocity-Verlet step of the hot path: integrate + half-skin rebuild check,
conditional cell binning / space-filling-curve sort / neighbour-list build,
pair forces, second half-kick, thermo every 100 steps; 100-step CUDA graphs.

Metric: particle-timesteps/s (N * steps / wall), higher is better; TPS is
reported beside it.  Also reported: the plain FP64 path on the same state and
the batched 256-replica ensemble, the pair kernel's HBM roofline fraction, the
CPU oracle on a bounded sample, and an end-to-end figure with host buffers.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

For N > 1 (torchrun) each rank runs an independent replica of the workload
(replicas only: the path does not shard), value = all ranks' particle-steps /
the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1412_3387_gb300 import inputs  # noqa: E402

METRIC = "particle-timesteps/s"
UNIT = "particle-steps/s"
HEADLINE = dict(workload="lj-16.7M", n=16_777_216, rho=0.8442, T=1.2, r_cut=2.5, r_skin=0.4,
                dt=0.005)
CPU_SAMPLE_N = 65_536  # the 64k sub-run of the same fluid


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=HEADLINE["n"], help="particles (headline 16,777,216)")
    ap.add_argument("--equil", type=int, default=1000, help="equilibration steps before timing")
    ap.add_argument("--forms", default="all", choices=["all", "mixed"])
    ap.add_argument("--fp64-steps", type=int, default=100)
    ap.add_argument("--batched-steps", type=int, default=200)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tuning", default="", help="fixed launch config, e.g. nlist:640:1,pair:128:1")
    ap.add_argument("--profile-pass", action="store_true",
                    help="after timing, one forced list build + one pair launch inside the "
                         "NVTX range 'md_profile' (for ncu --nvtx-include md_profile/)")
    return ap.parse_args()


def workload_config(args):
    return {"workload": HEADLINE["workload"] if args.n == HEADLINE["n"] else f"lj-{args.n}",
            "n_particles": args.n, "density": HEADLINE["rho"], "T": HEADLINE["T"],
            "r_cut": HEADLINE["r_cut"], "r_skin": HEADLINE["r_skin"], "dt": HEADLINE["dt"],
            "precision": "mixed (FP32 forces, Kahan; FP64 positions)",
            "graph_steps": 100, "thermo_period": 100, "sort_period": 1,
            "l2": "inputs larger than L2 (about 40 B/particle resident state x 16.7M)"}


# --------------------------------------------------------------------------
# clocks

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.proc = None
        # raw samples in a temporary file; the summary goes into the JSON line
        self.path = os.path.join(tempfile.gettempdir(), f"md_bench_clocks_{os.getpid()}.csv")
        self.idx = device_index

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "200"]
            if self.idx is not None:
                cmd += ["-i", str(self.idx)]
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------------------------
# CPU oracle baseline (bounded sample of the same fluid)

def cpu_oracle_rate(seconds: float):
    """Times the oracle's O(N) MD loop (as it stands) on CPU_SAMPLE_N particles
    of the headline fluid, on all host cores; returns (rate, cores, sample)."""
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    st = inputs.lj_fluid(CPU_SAMPLE_N, HEADLINE["rho"], HEADLINE["T"], seed=12345, jitter=0.05)
    kw = dict(r_cut=HEADLINE["r_cut"], r_skin=HEADLINE["r_skin"], dt=HEADLINE["dt"], max_nb=192)
    t0 = time.perf_counter()
    oracle.run(st.pos, st.vel, st.image, st.box[0], 2, **kw)
    probe = max(time.perf_counter() - t0, 1e-3) / 3.0  # forces at start + 2 steps
    steps = int(max(3, min(2000, seconds / probe)))
    t0 = time.perf_counter()
    oracle.run(st.pos, st.vel, st.image, st.box[0], steps, **kw)
    dt = time.perf_counter() - t0
    rate = CPU_SAMPLE_N * steps / dt
    return rate, cores, f"LJ N={CPU_SAMPLE_N} (same density, T, r_cut, skin), {steps} steps, " \
                        f"{dt:.1f} s, {cores} threads"


# --------------------------------------------------------------------------

def dist_setup(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch
        import torch.distributed as dist
        if args.impl == "gb300":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl")
        else:
            dist.init_process_group("gloo")
        pg = dist
    return rank, world, local, pg


def slowest_rank_time(elapsed, dist, device):
    """Length of the timed region: the slowest rank's (max over ranks; every
    rank gets it)."""
    if not dist:
        return elapsed
    import torch
    t = torch.tensor([elapsed], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(n_per_rank, steps, world, t_max):
    """Particle-steps per second of the whole job: every rank advanced its own
    n_per_rank particles by `steps` steps within t_max."""
    return n_per_rank * steps * world / t_max


def run_reference(args, rank, world):
    """Reference arm: the CPU FP64 oracle, as it stands, on the host cores."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    n = CPU_SAMPLE_N
    st = inputs.lj_fluid(n, HEADLINE["rho"], HEADLINE["T"], seed=12345, jitter=0.05)
    kw = dict(r_cut=HEADLINE["r_cut"], r_skin=HEADLINE["r_skin"], dt=HEADLINE["dt"], max_nb=192)
    state = (st.pos, st.vel, st.image)
    # each step of this arm = one oracle MD step of the 65,536-particle sample
    if args.warmup:
        out = oracle.run(*state, st.box[0], args.warmup, **kw)
        state = (out["pos"], out["vel"], out["image"])
    t0 = time.perf_counter()
    oracle.run(*state, st.box[0], args.steps, **kw)
    dt = time.perf_counter() - t0
    value = n * args.steps / dt
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference", "config": workload_config(args),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"LJ N={n} sample of the headline fluid, one oracle MD "
                                   f"step per bench step, {cores} threads"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


PAIR_SOURCES = ("pair_impl.cuh", "brick.cuh", "md_internal.cuh")


def pair_source_hash():
    h = hashlib.sha256()
    for name in PAIR_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_1412_3387_gb300", "csrc", name), "rb").read())
    return h.hexdigest()[:16]


def pair_traffic_record():
    """DRAM bytes per pair-kernel launch (scaled to this workload) from the
    committed ncu summary, if it was taken on the current kernel sources;
    else None."""
    path = os.path.join(ROOT, "profiles", "pair_lj_mixed_traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path))
    if rec.get("pair_sources_sha256_16") != pair_source_hash():
        return None
    return rec


def time_steps(sysm, steps, stream, torch):
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    sysm.run(steps, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def main():
    args = parse()
    rank, world, local, dist = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    from paper_1412_3387_gb300 import md

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    H = HEADLINE
    st = inputs.lj_fluid(args.n, H["rho"], H["T"], seed=12345 + rank)
    # sort_period=1: particles are re-sorted along the space-filling curve at
    # every list rebuild, which keeps the cell members contiguous in memory
    common = dict(r_cut=H["r_cut"], r_skin=H["r_skin"], dt=H["dt"], thermo_period=100,
                  graph_steps=100, sort_period=1, device=dev)
    with torch.cuda.stream(stream):
        sysm = md.MDSystem(st, precision="mixed", stream=stream, **common)
        sysm.prepare(stream)
        if args.tuning:
            for item in args.tuning.split(","):
                name, b, w = item.split(":")
                sysm.set_tuning(md.KERNEL_NLIST if name == "nlist" else md.KERNEL_PAIR,
                                int(b), int(w))
            sysm.prepare(stream)
        sysm.run(args.equil, stream=stream)  # melt the lattice start; sorts along the way
        if not args.tuning and not args.no_autotune:
            sysm.autotune(n_samples=5, block_stride=2, stream=stream)
        sysm.run(args.warmup, stream=stream)
        torch.cuda.synchronize()
        builds0 = sysm.info()["n_builds"]
        # ---- timed region ---------------------------------------------------
        dev_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local] \
            if "CUDA_VISIBLE_DEVICES" in os.environ else local
        with Clocks(dev_index) as clk:
            if dist:
                dist.barrier()
            elapsed = time_steps(sysm, args.steps, stream, torch)
            if dist:
                dist.barrier()
        sysm.check_error()
        builds = sysm.info()["n_builds"] - builds0
        t_max = slowest_rank_time(elapsed, dist, dev)
        value = whole_job_rate(args.n, args.steps, world, t_max)
        ms_per_step = 1e3 * t_max / args.steps

        if args.profile_pass:
            torch.cuda.nvtx.range_push("md_profile")
            sysm.build_nlist(True, stream)
            sysm.compute_pair(False, stream)
            sysm.integrate(1, stream)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()

        # ---- pair-kernel roofline (CUDA events on the launching stream) ----
        counts, _ = sysm.nlist(stream)
        nbar = float(counts.double().mean().item())
        del _
        n_launch = 30
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        sysm.compute_pair(False, stream)
        torch.cuda.synchronize()
        e0.record(stream)
        for _k in range(n_launch):
            sysm.compute_pair(False, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        pair_ms = e0.elapsed_time(e1) / n_launch
        bytes_per_particle = 4.0 * nbar + 4 + 16 + 16 + 16
        achieved = args.n * bytes_per_particle / (pair_ms * 1e-3) / 1e9
        peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
        if os.path.exists(peaks_path):
            peak, peak_src = float(json.load(open(peaks_path))["hbm_gbs"]), "measured"
        else:
            peak, peak_src = 6800.0, "fallback"
        rec = pair_traffic_record()
        traffic = None
        if rec:  # scaled by the particles of one launch
            traffic = rec["dram_bytes_per_particle"] * args.n
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "traffic": traffic,
                    "kernel": "k_pair<LJ, mixed>", "peak_source": peak_src,
                    "ms_per_launch": pair_ms, "algorithmic_bytes_per_particle": bytes_per_particle,
                    "mean_neighbours": nbar}

        # ---- end to end through the public API with host buffers ----------
        host = {k: getattr(sysm, k).cpu().pin_memory() for k in ("pos", "vel", "image", "tag", "type")}
        back = {k: torch.empty_like(host[k]).pin_memory() for k in ("pos", "vel")}
        torch.cuda.synchronize()
        e0.record(stream)
        for k, v in host.items():
            getattr(sysm, k).copy_(v, non_blocking=True)
        sysm.run(args.steps, stream=stream)
        for k in back:
            back[k].copy_(getattr(sysm, k), non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_s = e0.elapsed_time(e1) / 1e3
        h2d = sum(v.numel() * v.element_size() for v in host.values())
        d2h = sum(v.numel() * v.element_size() for v in back.values())
        e2e = {"value": args.n * args.steps * world / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps}
        sysm.check_error()
        tune_used = sysm.tuning()
        max_nb = sysm.max_nb
        eq_state = sysm.state_numpy()
        sysm.close()
        del sysm
        torch.cuda.empty_cache()

        # launches in the timed region: per step integrate(1) (with the
        # previous step's second half-kick folded in) + 8 binning (7 cell-list
        # kernels + brick descriptors) + 2 sort + nlist + pair; per 100-step
        # graph the closing half-kick integrate(2) and 2 thermo kernels.  The
        # binning, sort and list kernels return at once on steps without a
        # rebuild.
        launches = args.steps * (1 + 8 + 2 + 1 + 1) + 3 * (args.steps // 100)

        forms = {"mixed": {"value": value, "ms_per_step": ms_per_step, "steps": args.steps}}
        if args.forms == "all":
            # plain FP64 path on the equilibrated state
            st64 = st.copy()
            for k in ("pos", "vel", "image", "tag", "type"):
                setattr(st64, k, eq_state[k])
            s64 = md.MDSystem(st64, precision="fp64", stream=stream, max_nb=max_nb, **common)
            for kern, name in ((md.KERNEL_PAIR, "pair"), (md.KERNEL_NLIST, "nlist")):
                try:
                    s64.set_tuning(kern, *tune_used[name])
                except md.MDError:
                    pass  # the FP64 kernel may not fit the mixed kernel's block size
            s64.run(3, stream=stream)
            t64 = time_steps(s64, args.fp64_steps, stream, torch)
            s64.check_error()
            forms["fp64"] = {"value": args.n * args.fp64_steps / t64,
                             "ms_per_step": 1e3 * t64 / args.fp64_steps, "steps": args.fp64_steps}
            s64.close()
            del s64
            torch.cuda.empty_cache()
            # batched ensemble: 256 LJ replicas, N log-uniform in [2000, 64000]
            ens = inputs.replica_ensemble(256, seed=777 + rank)
            sb = md.MDSystem(ens, r_cut=2.5, r_skin=0.3, dt=0.005, precision="mixed",
                             thermo_period=100, graph_steps=100, sort_period=1, device=dev,
                             stream=stream)
            sb.prepare(stream)
            sb.run(300, stream=stream)
            if not args.no_autotune:
                sb.autotune(n_samples=3, block_stride=4, stream=stream)
            sb.run(20, stream=stream)
            tb = time_steps(sb, args.batched_steps, stream, torch)
            sb.check_error()
            forms["batched"] = {"value": ens.n * args.batched_steps / tb,
                                "ms_per_step": 1e3 * tb / args.batched_steps,
                                "steps": args.batched_steps, "replicas": 256,
                                "n_particles": ens.n}
            sb.close()

    if rank != 0:
        return
    cpu_rate, cores, sample = cpu_oracle_rate(args.cpu_seconds)
    cfg = workload_config(args)
    cfg["tuning"] = tune_used
    cfg["builds_in_timed_region"] = builds
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "tps": 1e3 / ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic (seeded fcc start, melted over the equilibration steps)",
        "config": cfg, "roofline": roofline, "clocks": clk.summary(),
        "cpu_baseline": {"value": cpu_rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": e2e, "gpu_launches": launches, "forms": forms,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
