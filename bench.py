"""Benchmark of the single-GPU short-range MD hot path.

Headline workload: LJ fluid, N = 16,777,216, density 0.8442, T = 1.2,
r_cut = 2.5, r_skin = 0.4, dt = 0.005, mixed precision (FP32 forces with
compensated accumulation, FP64 positions and integration).  A step is one full
velocity-Verlet step of the hot path: integrate + half-skin rebuild check,
conditional cell binning / space-filling-curve sort / neighbour-list build,
pair forces, second half-kick (folded into the next step's first inside a
graph), thermo once per graph.  The timed steps always replay CUDA graphs: the
graph length is the largest divisor of --steps up to 100, and the graph is
captured and instantiated before the timed region starts.

Metric: particle-timesteps/s (N * steps / wall), higher is better; TPS is
reported beside it.  Also reported ("forms"): the plain FP64 path on the same
state; the 256-replica ensemble (mixed) and the same replicas as 256
sequential FP64 runs; the 4,000-particle FP64 fluid; the 8,000,000-particle
DPD fluid; the 4,194,304-bead diblock melt (mixed and FP64); the Gaussian,
Morse and Yukawa pairs on the 2,097,152-particle fluid (mixed); each form's force
error against the CPU oracle; the pair kernels' rooflines; the CPU oracle on
bounded samples (all host threads and one thread); an end-to-end figure with
host buffers.

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
MAX_GRAPH = 100


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=HEADLINE["n"], help="particles (headline 16,777,216)")
    ap.add_argument("--equil", type=int, default=1000, help="equilibration steps before timing")
    ap.add_argument("--forms", default="all", help="all, mixed, or a comma list of forms")
    ap.add_argument("--fp64-steps", type=int, default=100)
    ap.add_argument("--batched-steps", type=int, default=200)
    ap.add_argument("--dpd-steps", type=int, default=200)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tuning", default="", help="fixed launch config, e.g. nlist:640:1,pair:128:1")
    ap.add_argument("--profile-pass", action="store_true",
                    help="after timing, one forced list build + one pair launch inside the "
                         "NVTX range 'md_profile' (for ncu --nvtx-include md_profile/)")
    ap.add_argument("--oracle-rate", type=float, default=0.0, help=argparse.SUPPRESS)
    return ap.parse_args(argv)


HEADLINE_SORT_PERIOD = 100


def graph_len(steps: int, cap: int = MAX_GRAPH) -> int:
    """Steps per CUDA graph for a timed region of `steps` steps: the largest
    divisor of steps not above cap, so the region is whole graph replays."""
    if steps <= 0:
        return 1
    for g in range(min(cap, steps), 0, -1):
        if steps % g == 0:
            return g
    return 1


def align_steps(step: int, g: int) -> int:
    """Untimed steps that bring the step counter to a multiple of g (graph
    replays start on thermo boundaries)."""
    return (-step) % g


def workload_config(args, g=None):
    g = g or graph_len(args.steps)
    return {"workload": HEADLINE["workload"] if args.n == HEADLINE["n"] else f"lj-{args.n}",
            "n_particles": args.n, "density": HEADLINE["rho"], "T": HEADLINE["T"],
            "r_cut": HEADLINE["r_cut"], "r_skin": HEADLINE["r_skin"], "dt": HEADLINE["dt"],
            "precision": "mixed (FP32 forces, Kahan; FP64 positions)",
            "timed_path": "cuda-graph replays", "graph_steps_used": g, "thermo_period": g,
            "sort_period": HEADLINE_SORT_PERIOD,
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

def _oracle_sample_rate(seconds: float):
    import oracle
    oracle.build()
    st = inputs.lj_fluid(CPU_SAMPLE_N, HEADLINE["rho"], HEADLINE["T"], seed=12345, jitter=0.05)
    kw = dict(r_cut=HEADLINE["r_cut"], r_skin=HEADLINE["r_skin"], dt=HEADLINE["dt"], max_nb=192)
    t0 = time.perf_counter()
    oracle.run(st.pos, st.vel, st.image, st.box[0], 2, **kw)
    probe = max(time.perf_counter() - t0, 1e-3) / 3.0  # forces at start + 2 steps
    steps = int(max(3, min(2000, seconds / probe)))
    t0 = time.perf_counter()
    oracle.run(st.pos, st.vel, st.image, st.box[0], steps, **kw)
    dt = time.perf_counter() - t0
    return CPU_SAMPLE_N * steps / dt, steps, dt


def cpu_oracle_rate(seconds: float, threads: int | None = None):
    """Times the oracle's O(N) MD loop (as it stands) on CPU_SAMPLE_N particles
    of the headline fluid; threads=None uses all host cores in this process,
    threads=k runs a child process with OMP_NUM_THREADS=k.  Returns
    (rate, cores, sample)."""
    cores = os.cpu_count() or 1
    if threads is None:
        rate, steps, dt = _oracle_sample_rate(seconds)
        used = cores
    else:
        env = dict(os.environ, OMP_NUM_THREADS=str(threads))
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-rate",
                            str(seconds)], env=env, capture_output=True, text=True, timeout=600)
        rec = json.loads(r.stdout.strip().splitlines()[-1])
        rate, steps, dt, used = rec["rate"], rec["steps"], rec["seconds"], threads
    return rate, used, (f"LJ N={CPU_SAMPLE_N} (same density, T, r_cut, skin), {steps} steps, "
                        f"{dt:.1f} s, {used} threads")


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


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return float(json.load(open(path))["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def time_run(sysm, steps, stream, torch):
    """CUDA-event time of sysm.run(steps) on `stream` (synchronised on both
    sides)."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    sysm.run(steps, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def ready_for_graphs(sysm, g, stream, torch):
    """Untimed: capture the g-step graph (one replay) and align the step
    counter to a multiple of g, so that a timed run of k g steps is k graph
    replays and nothing else."""
    sysm.run(g + align_steps(sysm.get_step() + g, g), stream=stream)
    torch.cuda.synchronize()
    assert sysm.get_step() % g == 0


def pair_launch_ms(sysm, stream, torch, n_launch=30):
    """Mean CUDA-event duration of back-to-back pair-kernel launches on the
    launching stream, on the system's current list."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    sysm.compute_pair(False, stream)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(n_launch):
        sysm.compute_pair(False, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / n_launch


def nlist_build_ms(sysm, stream, torch, n_launch=5):
    """Mean CUDA-event duration of back-to-back forced list builds on the
    launching stream (the first, untimed call rebins the particles, so the
    timed launches are the list kernel alone)."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    sysm.build_nlist(True, stream)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(n_launch):
        sysm.build_nlist(True, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / n_launch


def mean_neighbours(sysm, stream):
    counts, rows = sysm.nlist(stream)
    del rows
    return float(counts.double().mean().item())


def force_error(f, ref, absf):
    """RMS and max relative force error over particles with |F| >= 1e-2 S
    (S = sum_j |f_ij|, the oracle's), as in the parity tests."""
    d = np.linalg.norm(f[:, :3] - ref[:, :3], axis=1)
    F = np.linalg.norm(ref[:, :3], axis=1)
    big = (F >= 1e-2 * absf) & (absf > 0)
    rel = d[big] / F[big]
    return {"rms_rel": float(np.sqrt(np.mean(rel ** 2))), "max_rel": float(rel.max()),
            "particles": int(big.sum())}


# --------------------------------------------------------------------------
# the forms beside the headline

def fp64_peak(stream, torch):
    """Measured FP64 rate (DFMA chains filling every SM; best of 5 launches,
    CUDA events on the launching stream), TFLOP/s."""
    import ctypes as C
    from paper_1412_3387_gb300 import build as _b
    lib = C.CDLL(_b.RATE_LIB)
    lib.mdrate_dfma.restype = C.c_double
    lib.mdrate_dfma.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p]
    nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    blocks = nsm * 8
    out = torch.empty(blocks * 256, dtype=torch.float64, device="cuda")
    best = 0.0
    for _ in range(6):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        flops = lib.mdrate_dfma(C.c_void_p(out.data_ptr()), blocks, 200, C.c_void_p(stream.cuda_stream))
        e1.record(stream)
        torch.cuda.synchronize()
        if flops < 0:
            return None
        best = max(best, flops / (e0.elapsed_time(e1) * 1e-3) / 1e12)
    return best


def lj_error_subrun(md, dev, stream):
    """Mixed and FP64 force errors against the oracle on the 65,536-particle
    sub-run of the headline fluid: a jittered fcc start advanced 200 steps by
    the oracle, then forces from both GPU forms and the oracle."""
    import oracle
    H = HEADLINE
    st = inputs.lj_fluid(CPU_SAMPLE_N, H["rho"], H["T"], seed=12345, jitter=0.1)
    L = st.box[0]
    out = oracle.run(st.pos, st.vel, st.image, L, 200, r_cut=H["r_cut"], r_skin=H["r_skin"],
                     dt=H["dt"], max_nb=192)
    snap = st.copy()
    snap.pos, snap.vel, snap.image = out["pos"], out["vel"], out["image"]
    nl = oracle.neighbors(snap.pos, L, H["r_cut"] + H["r_skin"], max_nb=192, method="cells")
    ref, vref, absf = oracle.lj_forces(snap.pos, L, H["r_cut"], nlist=nl)
    th_ref = oracle.thermo(snap.vel, ref, vref, L)
    res = {"sample": f"LJ N={CPU_SAMPLE_N}, oracle-advanced 200 steps from a jittered fcc start"}
    for prec in ("mixed", "fp64"):
        s = md.MDSystem(snap, r_cut=H["r_cut"], r_skin=H["r_skin"], dt=H["dt"], precision=prec,
                        device=dev, stream=stream)
        s.prepare(stream)
        s.compute_pair(True, stream)
        f = s.forces(stream=stream).cpu().numpy()
        th = s.thermo(stream).cpu().numpy()[0]
        s.check_error()
        e = force_error(f, ref, absf)
        e["pe_rel"] = abs(th[1] - th_ref["pe"]) / abs(th_ref["pe"])
        e["virial_rel"] = abs(th[2] - th_ref["virial"]) / abs(th_ref["virial"])
        res[prec] = e
        s.close()
    return res


def batched_forms(md, dev, stream, torch, args, rank):
    """The 256-replica ensemble in one launch per kernel (mixed), its force
    error against the oracle on sampled replicas, and the same replicas as
    256 sequential FP64 runs of 100 steps."""
    import oracle
    ens = inputs.replica_ensemble(256, seed=777 + rank)
    kw = dict(r_cut=2.5, r_skin=0.3, dt=0.005, device=dev, stream=stream)
    out = {}
    g = graph_len(args.batched_steps)
    sb = md.MDSystem(ens, precision="mixed", thermo_period=g, graph_steps=g, sort_period=1, **kw)
    sb.prepare(stream)
    sb.run(300, stream=stream)
    if not args.no_autotune:
        sb.autotune(n_samples=3, block_stride=4, stream=stream)
    ready_for_graphs(sb, g, stream, torch)
    tb = time_run(sb, args.batched_steps, stream, torch)
    sb.check_error()
    out["batched"] = {"value": ens.n * args.batched_steps / tb,
                      "ms_per_step": 1e3 * tb / args.batched_steps, "steps": args.batched_steps,
                      "graph_steps_used": g, "replicas": 256, "n_particles": ens.n,
                      "tuning": sb.tuning()}
    # force error on sampled replicas of the equilibrated ensemble
    sb.compute_pair(False, stream)
    fb = sb.forces(stream=stream).cpu().numpy()
    eq = sb.state_numpy()
    sb.close()
    sizes = np.diff(ens.offsets)
    pick = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), 17, 101, 211})
    rms, mx, nparts = [], [], 0
    for r in pick:
        o0, o1 = int(ens.offsets[r]), int(ens.offsets[r + 1])
        L = ens.box[r]
        nl = oracle.neighbors(eq["pos"][o0:o1], L, 2.8, max_nb=256, method="cells")
        ref, _, absf = oracle.lj_forces(eq["pos"][o0:o1], L, 2.5, nlist=nl)
        e = force_error(fb[o0:o1], ref, absf)
        rms.append(e["rms_rel"])
        mx.append(e["max_rel"])
        nparts += o1 - o0
    out["batched"]["error_vs_oracle"] = {
        "rms_rel_max_over_replicas": max(rms), "max_rel": max(mx), "replicas": pick,
        "particles": nparts, "state": "after 300 + tuning + timed steps of the batched run"}
    # 256 sequential plain FP64 runs of the same replicas (100 steps each)
    t_seq, ps = 0.0, 0
    for r in range(256):
        sub = inputs.select_replica(ens, r)
        a = md.MDSystem(sub, precision="fp64", thermo_period=100, graph_steps=100, sort_period=1,
                        **kw)
        a.prepare(stream)
        a.run(100, stream=stream)  # captures the graph
        t_seq += time_run(a, 100, stream, torch)
        a.check_error()
        ps += sub.n * 100
        a.close()
    out["sequential_fp64"] = {"value": ps / t_seq, "ms_total": 1e3 * t_seq, "runs": 256,
                              "steps_per_run": 100, "graph_steps_used": 100,
                              "n_particles": ens.n}
    return out


def small_fp64_form(md, dev, stream, torch):
    """The 4,000-particle LJ fluid, FP64 throughout, 100 steps (one graph)."""
    st = inputs.lj_fluid(4000, 0.8442, 1.44, seed=12345)
    s = md.MDSystem(st, r_cut=2.5, r_skin=0.3, dt=0.005, precision="fp64", thermo_period=100,
                    graph_steps=100, sort_period=1, device=dev, stream=stream)
    s.prepare(stream)
    s.run(200, stream=stream)  # melt and capture
    t = time_run(s, 100, stream, torch)
    s.check_error()
    s.close()
    return {"value": 4000 * 100 / t, "tps": 100 / t, "ms_per_step": 1e3 * t / 100,
            "steps": 100, "graph_steps_used": 100, "n_particles": 4000}


# Gaussian, Morse and Yukawa pairs (Sec. 3's list): the paper's 2,097,152-
# particle benchmark fluid (rho 0.8442, T 1.2) with each potential in the
# mixed form, 100 untimed steps from the lattice, then timed graph replays
POTENTIALS = (("gauss", [[1.0, 1.0]]), ("morse", [[1.0, 6.0, 1.12]]), ("yukawa", [[1.0, 1.0]]))


def potential_forms(md, dev, stream, torch, tune_used, n=2_097_152, steps=200):
    out = {}
    for name, coeff in POTENTIALS:
        st = inputs.lj_fluid(n, 0.8442, 1.2, seed=2727)
        g = graph_len(steps)
        s = md.MDSystem(st, r_cut=2.5, r_skin=0.4, dt=0.005, pair=name, coeff=coeff,
                        precision="mixed", sort_period=1, thermo_period=g, graph_steps=g,
                        max_nb=192, stream=stream)
        try:
            for kern, k in ((md.KERNEL_PAIR, "pair"), (md.KERNEL_NLIST, "nlist")):
                s.set_tuning(kern, *tune_used[k])
            s.run(100, stream=stream)
            ready_for_graphs(s, g, stream, torch)
            t = time_run(s, steps, stream, torch)
            s.check_error()
            out[name] = {"value": n * steps / t, "ms_per_step": 1e3 * t / steps, "steps": steps,
                         "graph_steps_used": g, "n_particles": n, "coeff": coeff,
                         "pair_ms_per_launch": pair_launch_ms(s, stream, torch, 10)}
        except md.MDError as e:  # a side leg never hides the headline
            out[name] = {"error": str(e), "coeff": coeff}
        s.close()
        del s
        torch.cuda.empty_cache()
    return {"potentials_2M_mixed": out}


def dpd_forms(md, dev, stream, torch, args):
    """DPD fluid (8,000,000, rho 3, A 25, gamma 4.5, kT 1, dt 0.02, mixed) and
    the diblock melt (131,072 chains x 32 beads, A_AB 40, K 4), each with its
    pair-kernel roofline and the force error against the oracle on a
    65,536-particle sample of the same composition."""
    import oracle
    out = {}
    g = graph_len(args.dpd_steps)
    peak, peak_src = hbm_peak()
    coeff_f = [[25.0, 4.5]]
    coeff_d = np.array([[[25.0, 4.5], [40.0, 4.5]], [[40.0, 4.5], [25.0, 4.5]]])
    # the diblock melt starts as overlapping random-walk chains: its first
    # lists hold rows of up to ~130 neighbours (~45 once the melt has relaxed)
    cases = [
        ("dpd", "dpd-8M", lambda n: inputs.dpd_fluid(n, 3.0, 1.0, seed=4242), 8_000_000,
         coeff_f, ("mixed",), 96),
        ("diblock", "diblock-4.2M",
         lambda n: inputs.diblock_melt(n // 32, 32, 3.0, 1.0, seed=4343), 4_194_304, coeff_d,
         ("mixed", "fp64"), 192),
    ]
    for key, name, make, n, coeff, precs, max_nb in cases:
        st = make(n)
        rec = {"workload": name, "n_particles": st.n}
        for prec in precs:
            steps = args.dpd_steps if prec == "mixed" else max(g, args.dpd_steps // 4)
            gp = graph_len(steps)
            s = md.MDSystem(st, r_cut=1.0, r_skin=0.3, dt=0.02, pair="dpd", coeff=coeff, kT=1.0,
                            seed=99, precision=prec, thermo_period=gp, graph_steps=gp,
                            sort_period=1, bond_K=4.0, bond_r0=0.0, max_nb=max_nb, device=dev,
                            stream=stream)
            s.prepare(stream)
            s.run(100, stream=stream)
            if prec == "mixed" and not args.no_autotune:
                s.autotune(n_samples=3, block_stride=4, stream=stream)
            ready_for_graphs(s, gp, stream, torch)
            t = time_run(s, steps, stream, torch)
            s.check_error()
            r = {"value": st.n * steps / t, "ms_per_step": 1e3 * t / steps, "steps": steps,
                 "graph_steps_used": gp, "tuning": s.tuning()}
            if prec == "mixed":
                nbar = mean_neighbours(s, stream)
                ms = pair_launch_ms(s, stream, torch)
                bpp = 4.0 * nbar + 4 + 2 * (16 + 16) + 16
                ach = st.n * bpp / (ms * 1e-3) / 1e9
                r["pair_roofline"] = {"kernel": "k_pair<DPD, mixed>", "bound": "hbm",
                                      "achieved": ach, "peak": peak, "unit": "GB/s",
                                      "frac": ach / peak, "peak_source": peak_src,
                                      "ms_per_launch": ms, "mean_neighbours": nbar,
                                      "algorithmic_bytes_per_particle": bpp}
            rec[prec] = r
            s.close()
            torch.cuda.empty_cache()
        # force error on a 65,536-particle sample of the same composition
        smp = make(65_536)
        L = smp.box[0]
        step, seed = 7, 99
        nl = oracle.neighbors(smp.pos, L, 1.3, max_nb=max_nb, method="cells")
        ref, _, absf = oracle.dpd_forces(smp.pos, smp.vel, L, 1.0, coeff, 1.0, 0.02, step, seed,
                                         type=smp.type, tag=smp.tag, nlist=nl)
        if len(smp.bonds):
            ref, _, absf = oracle.bond_forces(smp.bonds, smp.pos, L, 4.0, 0.0, ref, None, absf)
        errs = {}
        for prec in precs:
            s = md.MDSystem(smp, r_cut=1.0, r_skin=0.3, dt=0.02, pair="dpd", coeff=coeff, kT=1.0,
                            seed=seed, precision=prec, bond_K=4.0, bond_r0=0.0, max_nb=max_nb,
                            device=dev, stream=stream)
            s.set_step(step, stream)
            s.prepare(stream)
            errs[prec] = force_error(s.forces(stream=stream).cpu().numpy(), ref, absf)
            s.close()
        rec["error_vs_oracle"] = dict(errs, sample="65,536 particles of the same composition, "
                                                   "seeded start, step 7")
        out[key] = rec
    return out


def main():
    args = parse()
    if args.oracle_rate:
        rate, steps, dt = _oracle_sample_rate(args.oracle_rate)
        print(json.dumps({"rate": rate, "steps": steps, "seconds": dt}))
        return
    rank, world, local, dist = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    from paper_1412_3387_gb300 import md

    forms_wanted = set(args.forms.split(","))
    want = lambda name: "all" in forms_wanted or name in forms_wanted
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    H = HEADLINE
    g = graph_len(args.steps)
    st = inputs.lj_fluid(args.n, H["rho"], H["T"], seed=12345 + rank)
    # the particles are re-sorted along the space-filling curve at the first
    # rebuild 100 or more steps after the last sort (a sort at every rebuild
    # keeps the cell members exactly contiguous but costs more than it saves)
    common = dict(r_cut=H["r_cut"], r_skin=H["r_skin"], dt=H["dt"], thermo_period=g,
                  graph_steps=g, sort_period=HEADLINE_SORT_PERIOD, device=dev)
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
        ready_for_graphs(sysm, g, stream, torch)
        builds0 = sysm.info()["n_builds"]
        # ---- timed region: args.steps / g replays of the g-step graph -------
        dev_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local] \
            if "CUDA_VISIBLE_DEVICES" in os.environ else local
        with Clocks(dev_index) as clk:
            if dist:
                dist.barrier()
            elapsed = time_run(sysm, args.steps, stream, torch)
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
        nbar = mean_neighbours(sysm, stream)
        pair_ms = pair_launch_ms(sysm, stream, torch)
        nlist_ms = nlist_build_ms(sysm, stream, torch)
        bytes_per_particle = 4.0 * nbar + 4 + 16 + 16 + 16
        achieved = args.n * bytes_per_particle / (pair_ms * 1e-3) / 1e9
        peak, peak_src = hbm_peak()
        rec = pair_traffic_record()
        traffic = rec["dram_bytes_per_particle"] * args.n if rec else None
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "traffic": traffic,
                    "kernel": "k_pair<LJ, mixed>", "peak_source": peak_src,
                    "ms_per_launch": pair_ms, "algorithmic_bytes_per_particle": bytes_per_particle,
                    "mean_neighbours": nbar}

        # ---- end to end through the public API with host buffers ----------
        ready_for_graphs(sysm, g, stream, torch)
        host = {k: getattr(sysm, k).cpu().pin_memory() for k in ("pos", "vel", "image", "tag", "type")}
        back = {k: torch.empty_like(host[k]).pin_memory() for k in ("pos", "vel")}
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
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
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "copies": "whole particle state in before the steps, pos and vel out after"}
        sysm.check_error()
        tune_used = sysm.tuning()
        max_nb = sysm.max_nb
        eq_state = sysm.state_numpy()
        sysm.close()
        del sysm
        torch.cuda.empty_cache()

        # launches in the timed region: per step integrate(1) (with the
        # previous step's second half-kick folded in) + 8 binning (7 cell-list
        # kernels + brick descriptors) + 2 sort + nlist + pair; per g-step
        # graph the closing half-kick integrate(2) and 2 thermo kernels.  The
        # binning, sort and list kernels return at once on steps without a
        # rebuild.
        launches = args.steps * (1 + 8 + 2 + 1 + 1) + 3 * (args.steps // g)

        forms = {"mixed": {"value": value, "ms_per_step": ms_per_step, "steps": args.steps,
                           "graph_steps_used": g, "nlist_ms_per_build": nlist_ms,
                           "builds": builds}}
        if want("fp64"):
            # plain FP64 path on the equilibrated state
            st64 = st.copy()
            for k in ("pos", "vel", "image", "tag", "type"):
                setattr(st64, k, eq_state[k])
            g64 = graph_len(args.fp64_steps)
            # the FP64 pair kernel reads each in-range neighbour's FP64 position
            # from global memory: sorted at every rebuild, those reads stay local
            c64 = dict(common, thermo_period=g64, graph_steps=g64, sort_period=1)
            s64 = md.MDSystem(st64, precision="fp64", stream=stream, max_nb=max_nb, **c64)
            for kern, name in ((md.KERNEL_PAIR, "pair"), (md.KERNEL_NLIST, "nlist")):
                try:
                    s64.set_tuning(kern, *tune_used[name])
                except md.MDError:
                    pass  # the FP64 kernel may not fit the mixed kernel's block size
            ready_for_graphs(s64, g64, stream, torch)
            t64 = time_run(s64, args.fp64_steps, stream, torch)
            s64.check_error()
            ms64 = pair_launch_ms(s64, stream, torch, 5)
            peak64 = fp64_peak(stream, torch)
            # FP64 pair kernel: bound by the FP64 pipe.  Per pair inside r_cut
            # it issues about 40 FP64 instructions (the exact minimum-image
            # distance: 3 sub, 3 mul, 3 round, 3 mul, 3 sub, 3 mul, 2 add; the
            # LJ force: the reciprocal ~ 8, 2 mul for r^-6, 4 for the magnitude,
            # 3 mul and 3 add for the components); each occupies the pipe like
            # one DFMA, counted as 2 FLOPs against the DFMA peak.  55.3 pairs
            # per particle inside r_cut at this density.
            fl = 2.0 * 40.0 * 55.3 * args.n / (ms64 * 1e-3) / 1e12
            forms["fp64"] = {"value": args.n * args.fp64_steps / t64,
                             "ms_per_step": 1e3 * t64 / args.fp64_steps, "steps": args.fp64_steps,
                             "graph_steps_used": g64, "pair_ms_per_launch": ms64,
                             "pair_roofline": {"kernel": "k_pair<LJ, FP64>", "bound": "fp64",
                                               "achieved": fl, "peak": peak64, "unit": "TFLOP/s",
                                               "frac": fl / peak64 if peak64 else None,
                                               "peak_source": "measured (DFMA chains, this run)",
                                               "fp64_instructions_per_pair": 40.0,
                                               "pairs_per_particle": 55.3}}
            # the same FP64 run with the half list (Newton's third law): each
            # pair's FP64 arithmetic once, the partner's share by atomic adds
            s64.set_newton(True)
            ready_for_graphs(s64, g64, stream, torch)
            tn64 = time_run(s64, args.fp64_steps, stream, torch)
            s64.check_error()
            forms["fp64_newton"] = {"value": args.n * args.fp64_steps / tn64,
                                    "ms_per_step": 1e3 * tn64 / args.fp64_steps,
                                    "steps": args.fp64_steps, "graph_steps_used": g64,
                                    "pair_ms_per_launch": pair_launch_ms(s64, stream, torch, 5)}
            s64.close()
            del s64
            torch.cuda.empty_cache()
        if want("nvt"):
            # the same fluid under a Nose-Hoover thermostat (the ensemble of the
            # paper's weak-scaling benchmark: one kinetic-energy sum per step)
            stn = st.copy()
            for k in ("pos", "vel", "image", "tag", "type"):
                setattr(stn, k, eq_state[k])
            gn = graph_len(args.fp64_steps)
            sn = md.MDSystem(stn, precision="mixed", stream=stream, max_nb=max_nb,
                             **dict(common, thermo_period=gn, graph_steps=gn))
            for kern, name in ((md.KERNEL_PAIR, "pair"), (md.KERNEL_NLIST, "nlist")):
                sn.set_tuning(kern, *tune_used[name])
            sn.set_integrator("nose-hoover", kT=H["T"], param=0.5)
            ready_for_graphs(sn, gn, stream, torch)
            tn = time_run(sn, args.fp64_steps, stream, torch)
            sn.check_error()
            forms["nvt_nose_hoover"] = {"value": args.n * args.fp64_steps / tn,
                                        "ms_per_step": 1e3 * tn / args.fp64_steps,
                                        "steps": args.fp64_steps, "graph_steps_used": gn,
                                        "kT": H["T"], "tau": 0.5}
            sn.close()
            del sn
            torch.cuda.empty_cache()
        if want("errors"):
            forms["error_vs_oracle_64k"] = lj_error_subrun(md, dev, stream)
        if want("batched"):
            forms.update(batched_forms(md, dev, stream, torch, args, rank))
        if want("lj4000"):
            forms["lj4000_fp64"] = small_fp64_form(md, dev, stream, torch)
        if want("dpd"):
            forms.update(dpd_forms(md, dev, stream, torch, args))
        if want("potentials"):
            forms.update(potential_forms(md, dev, stream, torch, tune_used))

    if rank != 0:
        return
    cpu_rate, cores, sample = cpu_oracle_rate(args.cpu_seconds)
    cpu1 = None
    if want("cpu1"):
        r1, c1, s1 = cpu_oracle_rate(min(args.cpu_seconds, 8.0), threads=1)
        cpu1 = {"value": r1, "unit": UNIT, "cores": c1, "kind": "oracle", "sample": s1}
    cfg = workload_config(args, g)
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
        "cpu_baseline_1core": cpu1,
        "e2e": e2e, "gpu_launches": launches, "forms": forms,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
