#!/usr/bin/env python
"""Benchmark of the APR SPH hot path on one GB300 (replicas on N GPUs).

Headline workload: the flyby disc (8,000,000 particles: a locally isothermal
disc on R in [1, 10] around a unit star, a unit perturber on a parabolic orbit
with periastron 20 started at true anomaly -120 degrees, and a two-level
refinement sphere R = (7.5, 5.0) that follows the perturber).  A step is one
whole pass of the hot path through the C ABI: kick, drift, accretion, zones
moved onto their sinks, split/merge, neighbour index, density solve, forces
with point-mass gravity, kick, conservation sums.  Metric: particle-steps per
second, counting the particles the density and force passes ran on; the
FP32-mixed path is the value, the FP64 path is timed beside it.

The zone starts at r = 80 and at periastron reaches in to R = 12.5, outside
the disc's edge at R = 10, so no gas enters it: on this workload the split and
merge passes find nothing to do.  The disc with a planet (1.13 M particles,
particles entering and leaving the planet's zone every step) is measured as a
second full line in the same JSON object.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
(whole steps of the same workload recipe at a bounded particle count) instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "APR particle-steps/s (density+force), FP32-mixed vs FP64 GPU, at stated error"
UNIT = "particle-steps/s"

# workload name -> (generator, default particle count, capacity factor, neighbour list length)
# the discs' Gaussian vertical tails put up to ~1240 particles inside 2.25 h of a
# tail particle (measured on the oracle's converged state): lists of 2048
WORKLOADS = {
    "flyby": ("flyby", 8_000_000, 1.2, 2048),
    "disc_planet": ("disc_planet", 1_000_000, 1.6, 2048),
    "sod": ("c2_sod", 123_480, 3.0, 0),
}

# Algorithmic FP32 (or FP64) work per pair, counted once from the kernel source
# (FMA = 2): density, per pair inside 2h per Newton-Raphson iteration: relative
# coords 3, r^2 5, sqrt 1, q 1, M4 f and f' 8, two compensated sums 11, f'' and the
# third compensated sum (mu q^2 f'', for the step acceptance) 10  -> 39;
# force, per pair inside max(2h_a, 2h_b): coords/r^2/rsqrt/r/q 12, two M4
# derivatives 8, F_a F_b 5, v.r 9, viscosity on approaching pairs 6, pressure term 5,
# three compensated components 15, energy 7, conductivity 13, signal speed 3 -> 83.
FLOPS_PER_PAIR = {"density": 39.0, "force": 83.0}
# Algorithmic bytes of the neighbour-list build: per particle its lattice
# coordinates and level (16 B), squared threshold (8 B) and per-axis bound (4 B)
# read, its entry count written (4 B); per list entry 4 B written.
LIST_BYTES_PER_PARTICLE = 32.0
LIST_BYTES_PER_ENTRY = 4.0
GROUPS = ("sort", "tree", "lists", "density", "force", "refine", "other")
# relative tolerances of the sampled parity (the same as the GPU tests)
PARITY_TOL = {"fp32": {"rho": 1e-5, "h": 1e-5, "omega": 1e-4, "a": 1e-4},
              "fp64": {"rho": 1e-12, "h": 1e-12, "omega": 1e-10, "a": 1e-9}}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="flyby", choices=sorted(WORKLOADS))
    ap.add_argument("--n", type=int, default=0, help="particle count (0: the workload's own)")
    ap.add_argument("--fp64-steps", type=int, default=5)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--parity-sample", type=int, default=1000)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle leg (cpu_baseline, parity)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-second", action="store_true", help="skip the disc-with-planet line")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the side measurements (tube, bins, sound wave, split adjoint)")
    ap.add_argument("--extra-steps", type=int, default=10)
    ap.add_argument("--ncu-range", action="store_true",
                    help="bracket the timed steps with cudaProfilerStart/Stop (for ncu "
                         "--profile-from-start off)")
    ap.add_argument("--table", action="store_true",
                    help="the per-configuration table (C1-C5): GPU FP32-mixed and FP64 rates, "
                         "the oracle's rate on the host cores, sampled errors against the "
                         "oracle, the dominant kernel's roofline fraction; one JSON line")
    ap.add_argument("--profile-workload", choices=["disc_planet", "disc_planet_bins"], default=None,
                    help="profiling only: initialise this workload, take --warmup steps, "
                         "then --steps steps inside cudaProfilerStart/Stop (the _bins form: "
                         "steps of 32 times the smallest limit in time-step bins 0..5)")
    return ap.parse_args()


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def make_workload(name, n=0):
    import apr_synth
    gen, n0, capf, mn = WORKLOADS[name]
    f = getattr(apr_synth, gen)
    w = f() if name == "sod" or not n else f(n)
    return w, capf, mn


def workload_label(name, w):
    n = len(w["p"]["x"])
    return {"flyby": f"flyby_disc_{n}p_periastron20_2level_sphere",
            "disc_planet": f"disc_planet_{n}p_3level_sphere",
            "sod": f"sod_shock_tube_3d_{n}p_2level_slab"}[name]


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """SM clock and clock-event reasons sampled while the timed region runs.

    Reads NVML (libnvidia-ml, read-only queries) from a thread every 2 ms; falls
    back to ``nvidia-smi -lms 200`` if NVML cannot be loaded.  Nothing is set."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    # NVML clock-event reason bits
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, uuid=None):
        self.sm, self.mx, self.bits = [], [], 0
        self.source = None
        self._stop = False
        try:
            self._nvml_start(uuid)
            self.source = "nvml"
        except Exception:
            self._smi_start()
            self.source = "nvidia-smi"

    def _nvml_start(self, uuid):
        import ctypes
        import threading
        L = ctypes.CDLL("libnvidia-ml.so.1")
        if L.nvmlInit_v2() != 0:
            raise OSError("nvmlInit")
        h = ctypes.c_void_p()
        if uuid:
            rc = L.nvmlDeviceGetHandleByUUID(str(uuid).encode(), ctypes.byref(h))
        else:
            cnt = ctypes.c_uint(0)
            L.nvmlDeviceGetCount_v2(ctypes.byref(cnt))
            if cnt.value != 1:
                raise OSError("several GPUs and no UUID")
            rc = L.nvmlDeviceGetHandleByIndex_v2(0, ctypes.byref(h))
        if rc != 0:
            raise OSError("nvml handle")
        reasons = getattr(L, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            L.nvmlDeviceGetCurrentClocksThrottleReasons
        mx = ctypes.c_uint(0)
        L.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx))
        self.mx.append(float(mx.value))

        def run():
            clk, bits = ctypes.c_uint(0), ctypes.c_ulonglong(0)
            while not self._stop:
                if L.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk)) == 0:
                    self.sm.append(float(clk.value))
                if reasons(h, ctypes.byref(bits)) == 0:
                    self.bits |= bits.value
                time.sleep(0.002)

        self.thread = threading.Thread(target=run, daemon=True)
        self.thread.start()
        time.sleep(0.01)  # first samples before the timed region starts

    def _smi_start(self):
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "200"]
        try:
            self.proc = subprocess.Popen(cmd, stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.source == "nvml":
            self._stop = True
            self.thread.join(timeout=2)
            reasons = sorted(v for b, v in self.REASONS.items() if self.bits & b)
            return {"sm_mhz": statistics.median(self.sm) if self.sm else None,
                    "sm_max_mhz": max(self.mx) if self.mx else None, "reasons": reasons,
                    "samples": len(self.sm), "source": "nvml, every 2 ms"}
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [l.strip().split(", ") for l in self.file.read().splitlines() if l.strip()]
        os.unlink(self.file.name)
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[k] for r in rows if len(r) >= 9 for k in range(4)
                          if r[5 + k].strip().lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(sm), "source": "nvidia-smi -lms 200"}


# ----------------------------------------------------------- our arm

# The bound arrays go into Morton order (apr_reorder) after the initial refinement
# and again every REORDER_EVERY steps; a reorder that falls on a timed step is
# timed with it.
REORDER_EVERY = 16


def advance(sim, dt=0.0):
    """One step through apr_step, then the periodic reorder."""
    out = sim.step(dt)
    sim.steps_taken = getattr(sim, "steps_taken", 0) + 1
    if REORDER_EVERY and sim.steps_taken % REORDER_EVERY == 0:
        sim.reorder()
    return out


def timed_steps(sim, torch, k, flush):
    """Device time of k steps (CUDA events on the library's stream), L2 flushed
    (256 MB written) before each step, outside the events."""
    st = sim.stream
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(k)]
    psteps = 0
    for i in range(k):
        with torch.cuda.stream(st):
            flush.zero_()
        ev[i][0].record(st)
        advance(sim)
        ev[i][1].record(st)
        psteps += sim.n
    st.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    return ms, psteps


SAMPLE_FIELDS = ("rho", "h", "omega", "ax", "ay", "az", "dudt", "pres")


def sample_fields(sim, ids):
    """The fields the parity block compares, at the particles with these ids."""
    import numpy as np
    gid = sim.get("id")
    order = np.argsort(gid)
    pos = order[np.searchsorted(gid[order], ids)]
    assert np.array_equal(gid[pos], ids)
    return {f: sim.get(f)[pos] for f in SAMPLE_FIELDS}


def traffic_record(kernel, workload):
    """DRAM bytes per launch from a committed ncu summary
    (profiles/<kernel>_traffic_<workload>.md, lines "key: value"), if it was taken on
    the current source of the kernel's file (else None)."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_traffic_{workload}.md")
    if not os.path.exists(path):
        return None
    rec = {}
    with open(path) as f:
        for line in f:
            k, sep, v = line.partition(":")
            if sep and k.strip() in ("dram_bytes_per_launch", "n", "source_sha256_16", "source"):
                rec[k.strip()] = v.strip()
    src = os.path.join(ROOT, "paper_2409_11470_gb300", "csrc", rec.get("source", "apr_sph.cu"))
    if not os.path.exists(src):
        return None
    with open(src, "rb") as f:
        digest = hashlib.sha256(f.read()).hexdigest()[:16]
    if rec.get("source_sha256_16") != digest or "dram_bytes_per_launch" not in rec or "n" not in rec:
        return None
    return {"dram_bytes_per_launch": float(rec["dram_bytes_per_launch"]), "n": float(rec["n"])}


def replica_totals(torch, ms, psteps, world, device):
    """Whole-job totals of independent replicas: the slowest rank's time and the
    particle-steps of all ranks (the only collective of a multi-GPU run)."""
    ms_t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    ps_t = torch.tensor([float(psteps)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(ms_t, op=dist.ReduceOp.MAX)
        dist.all_reduce(ps_t, op=dist.ReduceOp.SUM)
    return float(ms_t.item()), float(ps_t.item())


def measure_peaks(torch, uuid=None):
    """Measured FMA-pipe peaks of this GPU (apr_probe_fma_peak), with the SM clock
    sampled while each probe runs."""
    from paper_2409_11470_gb300.binding import probe_fma_peak
    out = {}
    for prec, iters in (("fp32", 40000), ("fp64", 1000)):
        probe_fma_peak(prec, max(1, iters // 10))  # warm-up of the clocks
        cs = ClockSampler(uuid)
        best = 0.0
        for _ in range(3):
            tf, ms = probe_fma_peak(prec, iters)
            best = max(best, tf)
        clk = cs.stop()
        out[prec] = {"tflops": best, "ms_per_launch": ms, "sm_mhz": clk["sm_mhz"],
                     "reasons": clk["reasons"]}
    return out


def rooflines(prof, steps, ms_total, n_mean, peaks, precision):
    """One roofline entry per kernel group that takes at least 10% of the timed
    steps: density and force against the measured FMA peak of their precision
    (algorithmic FLOPs per launch over the launch's average CUDA-event time), the
    neighbour lists against the measured copy bandwidth (algorithmic bytes)."""
    hbm = measured_hbm()
    rows = []
    for g in GROUPS:
        ms = prof[g]["ms"]
        calls = max(prof[g]["calls"], 1)
        share = ms / ms_total if ms_total > 0 else 0.0
        if share < 0.10:
            continue
        ms_launch = ms / calls
        row = {"group": g, "share": share, "ms_per_launch": ms_launch, "launches": calls}
        if g in FLOPS_PER_PAIR:
            pk = peaks[precision]["tflops"]
            work = prof[g]["pairs"] * FLOPS_PER_PAIR[g] / calls
            ach = work / (ms_launch / 1e3) / 1e12
            ker = f"k_{g}<{'float' if precision == 'fp32' else 'double'}>"
            row.update({"kernel": ker, "bound": "alu", "achieved": ach, "peak": pk,
                        "unit": "TFLOP/s", "frac": ach / pk,
                        "peak_source": f"measured FMA-chain probe ({precision}), of measured",
                        "pairs_per_launch": prof[g]["pairs"] / calls,
                        "flops_per_pair": FLOPS_PER_PAIR[g]})
        elif g == "lists":
            entries = prof[g]["pairs"] / calls
            byts = n_mean * LIST_BYTES_PER_PARTICLE + entries * LIST_BYTES_PER_ENTRY
            ach = byts / (ms_launch / 1e3) / 1e9
            row.update({"kernel": "k_candidates + k_thresholds + k_lists", "bound": "hbm",
                        "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                        "peak_source": "MEASURED_PEAKS.json hbm_gbs, of measured",
                        "list_entries_per_launch": entries,
                        "algorithmic_bytes_per_launch": byts})
        else:
            row.update({"bound": "hbm", "note": "several kernels; no single algorithmic figure"})
        rows.append(row)
    return rows


def measured_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0  # the recipe's fallback


def measure(w, precision, steps, warmup, torch, flush, cap_factor, max_neigh, sample_ids=None,
            uuid=None, world=1, ncu_range=False, keep=False):
    """Initialise a workload, keep the sampled fields of the initialised state,
    take warm-up steps, then time `steps` steps with the profiler on."""
    from paper_2409_11470_gb300.binding import Simulation
    n0 = len(w["p"]["x"])
    sim = Simulation(w, capacity=int(cap_factor * n0) + 1024, precision=precision,
                     max_neigh=max_neigh)
    t0 = time.perf_counter()
    sim.init()
    sim.stream.synchronize()
    init_s = time.perf_counter() - t0
    sim.reorder()
    n_init = sim.n
    sample = sample_fields(sim, sample_ids) if sample_ids is not None else None
    m_sinks0 = [k["m"] for k in sim.sinks()]
    for _ in range(warmup):
        advance(sim)
    sim.profile_enable(True)  # clears the counters
    launches0 = sim.profile()["launches"]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(uuid)
    if ncu_range:
        torch.cuda.cudart().cudaProfilerStart()
    t_wall = time.perf_counter()
    ms, psteps = timed_steps(sim, torch, steps, flush)
    torch.cuda.synchronize()
    if ncu_range:
        torch.cuda.cudart().cudaProfilerStop()
    t_wall = time.perf_counter() - t_wall
    clocks = sampler.stop()
    prof = sim.profile()
    sim.profile_enable(False)
    res = {"ms": ms, "psteps": psteps, "prof": prof, "launches": prof["launches"] - launches0,
           "clocks": clocks, "sample": sample, "n_initial": n0, "n_after_init": n_init,
           "n_last": sim.n, "init_s": init_s, "wall_s_timed": t_wall,
           "sink_mass_gain": [k["m"] - m for k, m in zip(sim.sinks(), m_sinks0)]}
    if keep:
        res["sim"] = sim
    else:
        sim.close()
    return res


DF_GROUPS = ("sort", "tree", "lists", "density", "force")


def summary(r, steps, peaks, precision):
    """value, per-step breakdown and rooflines of one measured run."""
    prof = r["prof"]
    n_mean = r["psteps"] / steps
    rows = rooflines(prof, steps, r["ms"], n_mean, peaks, precision)
    # the index, density and force alone (quantise and sort, radix tree, cells and
    # lists, density solve, forces): the groups' device time per step
    df_ms = sum(prof[g]["ms"] for g in DF_GROUPS)
    return {"value": r["psteps"] / (r["ms"] / 1e3), "unit": UNIT, "ms_per_step": r["ms"] / steps,
            "density_force_only": {"value": r["psteps"] / (df_ms / 1e3) if df_ms > 0 else None,
                                   "unit": UNIT, "ms_per_step": df_ms / steps,
                                   "groups": list(DF_GROUPS)},
            "steps": steps, "n_initial": r["n_initial"], "n_after_init": r["n_after_init"],
            "n_last": r["n_last"],
            "breakdown_ms_per_step": {g: round(prof[g]["ms"] / steps, 4) for g in GROUPS},
            "density_attempts_per_step": prof["density_attempts"] / steps,
            "retried_particles_per_step": prof["uncovered"] / steps,
            "sink_mass_gain": r["sink_mass_gain"], "rooflines": rows}


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    w, capf, mn = make_workload(args.workload, args.n)
    label = workload_label(args.workload, w)
    n0 = len(w["p"]["x"])
    props = torch.cuda.get_device_properties(local)
    uuid = getattr(props, "uuid", None)
    uuid = f"GPU-{uuid}" if uuid is not None and not str(uuid).startswith("GPU-") else uuid
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    peaks = measure_peaks(torch, uuid)
    rng = np.random.default_rng(12345)
    sample_ids = np.sort(rng.choice(np.asarray(w["p"]["id"]), min(args.parity_sample, n0),
                                    replace=False)).astype(np.uint64)

    r32 = measure(w, "fp32", args.steps, args.warmup, torch, flush, capf, mn, sample_ids, uuid,
                  world, args.ncu_range, keep=not args.no_e2e)
    ms_max, ps_all = replica_totals(torch, r32["ms"], r32["psteps"], world, "cuda")
    value = ps_all / (ms_max / 1e3)
    s32 = summary(r32, args.steps, peaks, "fp32")
    dom = max(s32["rooflines"], key=lambda x: x["share"]) if s32["rooflines"] else None
    roofline = None
    if dom is not None and "frac" in dom:
        tr = None
        if dom["group"] in FLOPS_PER_PAIR:
            tr = traffic_record(f"k_{dom['group']}_f32", args.workload)
        elif dom["group"] == "lists":
            tr = traffic_record("lists", args.workload)
        roofline = {"bound": dom["bound"], "achieved": dom["achieved"], "peak": dom["peak"],
                    "unit": dom["unit"], "frac": dom["frac"],
                    "traffic": tr["dram_bytes_per_launch"] * (r32["n_after_init"] / tr["n"])
                    if tr else None,
                    "kernel": dom["kernel"], "group": dom["group"], "share": dom["share"],
                    "peak_source": dom["peak_source"], "ms_per_launch": dom["ms_per_launch"]}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": label, "n_initial": n0, "n_after_init": r32["n_after_init"],
                      "n_last": r32["n_last"],
                      "precision": "fp32-mixed (pair sums f32 compensated on relative lattice "
                                   "coordinates; state, integration, reductions f64)",
                      "l2": "flushed by a 256 MB write before every timed step (the state is "
                            "also far larger than L2)",
                      "parallelism": "replicas" if world > 1 else "single GPU",
                      "zone": "follows the perturber (r = 80 at the start, 20 at periastron); "
                              "its outer radius 7.5 never reaches the disc (R <= 10), so no gas "
                              "is split or merged in these steps" if args.workload == "flyby"
                              else None,
                      "layout": f"particle arrays put in Morton order (apr_reorder) after "
                                f"init and every {REORDER_EVERY} steps, inside the timed steps",
                      "wall_s_timed": r32["wall_s_timed"]},
           "roofline": roofline, "rooflines": s32["rooflines"],
           "breakdown_ms_per_step": s32["breakdown_ms_per_step"],
           "density_force_only": s32["density_force_only"],
           "gpu_launches": r32["launches"], "clocks": r32["clocks"], "peaks": peaks}

    r64 = None
    if rank == 0 and not args.no_fp64:
        r64 = measure(w, "fp64", args.fp64_steps, max(1, args.warmup // 2), torch, flush, capf, mn,
                      sample_ids, uuid)
        s64 = summary(r64, args.fp64_steps, peaks, "fp64")
        out["fp64"] = {k: s64[k] for k in ("value", "ms_per_step", "steps", "breakdown_ms_per_step",
                                            "density_force_only", "rooflines")}
        out["fp32_over_fp64"] = value / s64["value"]

    if rank == 0 and not args.no_e2e:
        out["e2e"] = e2e_rate(r32["sim"], torch, args.steps, flush)
    if "sim" in r32:
        r32["sim"].close()

    if rank == 0 and world == 1 and not args.no_cpu:
        leg = oracle_leg(w, args.workload, sample_ids, r32["sample"],
                         r64["sample"] if r64 else None, args.cpu_seconds)
        out["cpu_baseline"] = leg["cpu_baseline"]
        out["parity"] = leg["parity"]

    if rank == 0 and not args.no_second and args.workload == "flyby":
        out["disc_planet_line"] = second_line(torch, flush, peaks, args)

    if rank == 0 and not args.no_extra:
        out["other_workloads"] = side_measurements(args, torch, flush)

    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def e2e_rate(sim, torch, steps, flush):
    """The same steps through the C ABI with host buffers: every step uploads the
    pinned host state (apr_upload), steps, and downloads it (apr_download); the
    step length is the cached limit, read before the upload drops it."""
    from paper_2409_11470_gb300.binding import F64_FIELDS
    fields = list(F64_FIELDS) + ["level", "flags", "id"]
    host = {f: b for f, b in sim.host_buffers().items() if f in fields}
    sim.download(host)
    st = sim.stream
    evs = []
    bi = bo = 0
    ps_e = 0
    for _ in range(steps):
        n = sim.n
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(st):
            flush.zero_()
        dt = sim.timestep()
        e0.record(st)
        sim.upload(host, n)
        advance(sim, dt)
        n2 = sim.download(host)
        e1.record(st)
        st.synchronize()
        evs.append(e0.elapsed_time(e1))
        bi += sum(n * host[f].element_size() for f in fields)
        bo += sum(n2 * host[f].element_size() for f in fields)
        ps_e += n2
    return {"value": ps_e / (sum(evs) / 1e3), "unit": UNIT, "h2d_bytes_per_step": bi // steps,
            "d2h_bytes_per_step": bo // steps}


def second_line(torch, flush, peaks, args):
    """The disc with a planet (zone busy every step) as a second full line:
    FP32-mixed and FP64 particle-steps/s, breakdown and rooflines."""
    try:
        w, capf, mn = make_workload("disc_planet", 0)
        k = max(1, args.extra_steps)
        r32 = measure(w, "fp32", k, 2, torch, flush, capf, mn)
        s32 = summary(r32, k, peaks, "fp32")
        line = {"workload": workload_label("disc_planet", w), "fp32": s32,
                "gpu_launches": r32["launches"], "clocks": r32["clocks"]}
        if not args.no_fp64:
            k64 = max(2, k // 3)
            r64 = measure(w, "fp64", k64, 1, torch, flush, capf, mn)
            s64 = summary(r64, k64, peaks, "fp64")
            line["fp64"] = {x: s64[x] for x in ("value", "ms_per_step", "steps",
                                                 "breakdown_ms_per_step", "density_force_only",
                                                 "rooflines")}
            line["fp32_over_fp64"] = s32["value"] / s64["value"]
        return line
    except Exception as e:  # a second line never takes the headline down
        return {"error": f"{type(e).__name__}: {e}"}


# ------------------------------------------------------- side measurements

def side_measurements(args, torch, flush):
    """The shock tube (FP32-mixed and FP64 whole steps), time-step bins, the
    sound-wave box and the split adjoint, each on its own."""
    import apr_synth
    out = {}
    k = max(1, args.extra_steps)
    try:
        w, capf, mn = make_workload("sod", 0)
        r = {"workload": workload_label("sod", w)}
        r32 = measure(w, "fp32", k, 3, torch, flush, capf, mn)
        r["fp32"] = {"value": r32["psteps"] / (r32["ms"] / 1e3), "ms_per_step": r32["ms"] / k,
                     "breakdown_ms_per_step": {g: round(r32["prof"][g]["ms"] / k, 4) for g in GROUPS}}
        r64 = measure(w, "fp64", max(2, k // 3), 1, torch, flush, capf, mn)
        r["fp64"] = {"value": r64["psteps"] / (r64["ms"] / 1e3),
                     "ms_per_step": r64["ms"] / max(2, k // 3)}
        r["fp32_over_fp64"] = r["fp32"]["value"] / r["fp64"]["value"]
        out["sod_shock_tube"] = r
    except Exception as e:
        out["sod_shock_tube"] = {"error": f"{type(e).__name__}: {e}"}
    for name, make, Bs, big, capf, mn in (
            ("sod_time_step_bins", apr_synth.c2_sod, (3,), 4, 3.0, 0),
            ("disc_planet_1e6_time_step_bins", apr_synth.disc_planet, (3, 5), 2, 1.6, 2048)):
        try:
            out[name] = bins_measurement(torch, make(), Bs, big, capf, mn)
        except Exception as e:
            out[name] = {"error": f"{type(e).__name__}: {e}"}
    try:
        out["sound_wave_box_56832p_cylinder_zone"] = sound_wave_measurement(torch)
    except Exception as e:
        out["sound_wave_box_56832p_cylinder_zone"] = {"error": f"{type(e).__name__}: {e}"}
    try:
        out["split_adjoint_c5_2000376p"] = adjoint_rate(torch, k)
    except Exception as e:
        out["split_adjoint_c5_2000376p"] = {"error": f"{type(e).__name__}: {e}"}
    return out


def bins_measurement(torch, w, Bs, big_steps, cap_factor=3.0, max_neigh=0):
    """A workload advanced with one global step (B = 0, the smallest limit taken
    afresh every step) and with individual time steps in bins (Sec. 2.5; dt_max =
    2^B times the smallest limit, taken afresh every step of dt_max), all runs
    over the same simulated time: device time per unit of simulated time, force
    updates per particle and unit time, and the device time by group."""
    from paper_2409_11470_gb300.binding import Simulation
    n0 = len(w["p"]["x"])
    res = {"n_initial": n0}
    t_end = None
    for B in (0,) + tuple(b for b in Bs if b > 0):
        g = Simulation(w, capacity=int(cap_factor * n0) + 1024, precision="fp32",
                       max_neigh=max_neigh)
        g.init()
        if t_end is None:
            t_end = big_steps * g.timestep() * (1 << max(Bs))
        g.profile(reset=True)
        g.profile_enable(True)
        st = g.stream
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        t, upd, sat, steps, first, acc = 0.0, 0, 0, 0, True, 0
        while t < t_end:
            dt_max = g.timestep() * (1 << B)
            c, u, sa, _ = g.step_bins(dt_max, B, init_bins=first)
            first = False
            t += dt_max
            upd += u
            sat += sa
            acc += c.n_accreted
            steps += 1
        e1.record(st)
        st.synchronize()
        ms = e0.elapsed_time(e1)
        prof = g.profile()
        g.profile_enable(False)
        res[f"B{B}"] = {"steps_of_dt_max": steps, "t_sim": t, "ms_per_unit_time": ms / t,
                        "updates_per_particle_per_unit_time": upd / g.n / t,
                        "saturated_updates": sat, "accreted": acc, "n_last": g.n,
                        "breakdown_ms_per_unit_time": {
                            k: round(prof[k]["ms"] / t, 2) for k in
                            ("sort", "tree", "lists", "density", "force", "refine", "other")}}
        g.close()
    b0 = res["B0"]["ms_per_unit_time"]
    for B in Bs:
        if B > 0:
            res[f"B{B}"]["speedup_vs_global_step"] = b0 / res[f"B{B}"]["ms_per_unit_time"]
    return res


def sound_wave_measurement(torch, t_end=2.0):
    """The appendix sound-wave box (56,832 particles, circular zone switched on at
    t = 0.5) run to t = 2 with and without the zone: whole-step particle-steps/s of
    the zoned run, the density blip at the boundary (largest difference of the
    binned cross-section densities, in units of the initial mean density) and how
    far the mixed-level transition reaches past the boundary (in level-0 h)."""
    import numpy as np

    import apr_synth
    from paper_2409_11470_gb300.binding import Simulation
    w = apr_synth.sound_wave_box()
    n0 = len(w["p"]["x"])
    t_on, regs = w["regions_at"]

    def run(zone, relax=False):
        g = Simulation(w, capacity=3 * n0, precision="fp32")
        g.init()
        rho0 = float(np.mean(g.get("rho")))
        st = g.stream
        t, on, steps, psteps, ms = 0.0, False, 0, 0, 0.0
        while t < t_end - 1e-12:
            if zone and not on and t >= t_on - 1e-12:
                g.set_regions(regs)
                on = True
                if relax:  # split now, then relax the children (Sec. 2.4, the paper's 0.5% / 50)
                    ref = g.snapshot()
                    g.split_merge()
                    g.relax(ref, 50, 0.005)
            dt = min(g.timestep(), t_end - t, (t_on - t) if (zone and not on) else 1e9)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            g.step(dt)
            e1.record(st)
            st.synchronize()
            ms += e0.elapsed_time(e1)
            steps += 1
            psteps += g.n
            t += dt
        return g, rho0, ms, steps, psteps

    ref, rho_ic, _, _, _ = run(False)
    apr, _, ms, steps, psteps = run(True)
    rel_run = run(True, relax=True)[0]
    _, pr = apr_synth.wave_profile(ref.get("x"), ref.get("y"), ref.get("rho"), w["Ly"])

    def blip_fuzz(g):
        _, pa = apr_synth.wave_profile(g.get("x"), g.get("y"), g.get("rho"), w["Ly"])
        return (float(np.max(np.abs(pa - pr)) / rho_ic),
                apr_synth.zone_fuzz(g.get("x"), g.get("y"), g.get("level"), g.get("h")))

    blip, fuzz = blip_fuzz(apr)
    blip_r, fuzz_r = blip_fuzz(rel_run)
    res = {"value": psteps / (ms / 1e3), "unit": UNIT, "steps": steps, "ms_per_step": ms / steps,
           "n_initial": n0, "n_last": apr.n, "t_end": t_end, "blip_over_rho0": blip,
           "transition_over_h": fuzz, "relaxed_at_split": {"blip_over_rho0": blip_r,
                                                          "transition_over_h": fuzz_r},
           "paper": "blip below 5% of the initial density; transition about 10% of h"}
    for g in (ref, apr, rel_run):
        g.close()
    return res


def adjoint_rate(torch, k):
    """apr_density_loss_grad on the 126^3 jittered lattice, first split pass of the
    R = 0.35 zone: evaluations (J and the full gradient) per second."""
    import apr_synth
    from paper_2409_11470_gb300.binding import Simulation
    w = apr_synth.c5_adjoint_lattice()
    prob = apr_synth.adjoint_problem(w)
    n, npar = len(w["p"]["x"]), len(prob["parent"])
    sim = Simulation(w, capacity=n + 2 * npar, precision="fp32")
    dev = sim.device
    par = torch.as_tensor(prob["parent"], device=dev)
    d = torch.as_tensor(prob["d"], device=dev)
    hc = torch.as_tensor(prob["hc"], device=dev)
    for _ in range(2):
        J0 = sim.density_loss_grad(par, d, hc)[0]
    st = sim.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(k):
        sim.density_loss_grad(par, d, hc)
    e1.record(st)
    st.synchronize()
    ms = e0.elapsed_time(e1) / k
    sim.close()
    return {"evals_per_s": 1e3 / ms, "ms_per_eval": ms, "particles": n, "splits": npar,
            "children": 2 * npar, "children_per_s": 2 * npar * 1e3 / ms, "J": J0,
            "precision": "fp32 pair sums, fp64 reduction",
            "note": "one evaluation = children placed, index over the combined set, forward "
                    "and reverse sweeps, chain rule to the offsets, J read back"}


# ------------------------------------------------------------ the oracle

# bounded particle counts of the oracle's whole steps (the same recipe, seeded
# alike): about a second per step on 16 host cores
ORACLE_STEP_N = {"flyby": 250_000, "disc_planet": 250_000, "sod": 0}


def _oracle_sample_errors(g, o, idx, adiabatic):
    import numpy as np
    rho, h, om, P = o["rho"][idx], o["h"][idx], o["omega"][idx], o["pres"][idx]
    a_o = np.stack([o["ax"][idx], o["ay"][idx], o["az"][idx]], 1)
    a_g = np.stack([g["ax"], g["ay"], g["az"]], 1)
    scale = np.linalg.norm(a_o, axis=1) + P / (rho * h)
    e = {"rho": float(np.max(np.abs(g["rho"] - rho) / rho)),
         "h": float(np.max(np.abs(g["h"] - h) / h)),
         "omega": float(np.max(np.abs(g["omega"] - om))),
         "a": float(np.max(np.abs(a_g - a_o) / scale[:, None]))}
    if adiabatic:
        cs = o["cs"][idx]
        sd = np.abs(o["dudt"][idx]) + P / rho * cs / h
        e["dudt"] = float(np.max(np.abs(g["dudt"] - o["dudt"][idx]) / sd))
    return e


def oracle_leg(w, workload, sample_ids, s32, s64, seconds):
    """The CPU-baseline leg: the FP64 oracle as it stands, on the host cores.

    parity: from the same seeded input, the oracle solves the initialised
    state's density (every particle, exact roots) and the forces of the sampled
    particles; the GPU's initialised values at those particles (FP32-mixed and
    FP64) are compared with it, per quantity: rho and h relative, Omega
    absolute, a (and du/dt) relative to |a| + P/(rho h).
    cpu_baseline: whole oracle steps of the same workload recipe at a bounded
    particle count, particle-steps/s."""
    import numpy as np

    import oracle
    _, _, capf, _ = WORKLOADS[workload]
    n = len(w["p"]["x"])
    o = oracle.Oracle(w, capacity=int(capf * n) + 16)
    t0 = time.perf_counter()
    o.track_regions()
    bad = o.density()
    cnt = o.split_merge(0)
    changed = sum(cnt.n_split) + sum(cnt.n_merge)
    if changed:  # the zones split or merge at the start: the full initial refinement
        o = oracle.Oracle(w, capacity=int(capf * n) + 16)
        o.init()
        bad = 0
    t_dens = time.perf_counter() - t0
    oid = o["id"]
    order = np.argsort(oid)
    idx = order[np.searchsorted(oid[order], sample_ids)]
    assert np.array_equal(oid[idx], sample_ids)
    t0 = time.perf_counter()
    if not changed:
        o.force(idx)
        if o.nsink:
            o.sink_gravity()
    t_force = time.perf_counter() - t0
    adiabatic = int(w["cfg"]["eos"]) == 0
    parity = {"sample": int(len(idx)), "kind": "sampled particles of the initialised state "
              "against the oracle's solve of the same seeded input",
              "oracle_s": {"density_all": t_dens, "force_sample": t_force},
              "oracle_unconverged": int(bad), "tolerance": PARITY_TOL}
    for name, s in (("fp32", s32), ("fp64", s64)):
        if s is None:
            continue
        e = _oracle_sample_errors(s, o, idx, adiabatic)
        tol = PARITY_TOL[name]
        parity[name] = {"max_err": e, "within_tolerance": all(e[k] <= tol[k if k != "dudt" else "a"]
                                                              for k in e)}
    del o
    base = oracle_step_rate(workload, seconds)
    return {"parity": parity, "cpu_baseline": base}


def oracle_step_rate(workload, seconds, steps=0, warmup=0):
    """Whole FP64 oracle steps (kick, drift, accretion, zones, split/merge, density,
    forces, point masses, kick) of the workload recipe at a bounded particle count:
    particle-steps/s, the threads used and what was run."""
    import oracle
    nb = ORACLE_STEP_N[workload]
    w, capf, _ = make_workload(workload, nb)
    o = oracle.Oracle(w, capacity=int(capf * len(w["p"]["x"])) + 16)
    o.init()
    for _ in range(warmup):
        o.step(o.timestep())
    total, done, k = 0.0, 0, 0
    while (steps and k < steps) or (not steps and (total < seconds or k < 2)):
        dt = o.timestep()
        t0 = time.perf_counter()
        o.step(dt)
        total += time.perf_counter() - t0
        done += o.n
        k += 1
    return {"value": done / total, "unit": UNIT, "cores": o.threads(), "kind": "oracle",
            "sample": f"{k} whole FP64 oracle steps (k-d tree enumeration, OpenMP) of the "
                      f"{workload_label(workload, w)} recipe ({len(w['p']['x'])} particles at the "
                      f"start, {o.n} after), {total:.1f} s",
            "steps": k, "seconds": total}


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return
    w, _, _ = make_workload(args.workload, args.n)
    base = oracle_step_rate(args.workload, 0.0, steps=args.steps, warmup=args.warmup)
    value = base["value"]
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * base["seconds"] / max(base["steps"], 1), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": workload_label(args.workload, w), "n_initial": len(w["p"]["x"])},
           "cpu_baseline": {k: base[k] for k in ("value", "unit", "cores", "kind", "sample")},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_profile_workload(args):
    """A side workload's steps bracketed for ``ncu --profile-from-start off``."""
    import torch

    import apr_synth
    from paper_2409_11470_gb300.binding import Simulation
    w = apr_synth.disc_planet()
    n0 = len(w["p"]["x"])
    sim = Simulation(w, capacity=int(1.6 * n0) + 1024, precision="fp32", max_neigh=2048)
    sim.init()
    sim.reorder()
    bins = args.profile_workload.endswith("_bins")

    def one(first):
        if bins:
            sim.step_bins(32 * sim.timestep(), 5, init_bins=first)
        else:
            advance(sim)

    for k in range(args.warmup):
        one(k == 0)
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStart()
    for k in range(args.steps):
        one(args.warmup == 0 and k == 0)
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStop()
    print(json.dumps({"profile_workload": w["name"], "steps": args.steps, "n": sim.n}), flush=True)
    sim.close()


# --------------------------------------------------------- the C1-C5 table

def _gpu_init_sample(w, precision, capf, mn, ids):
    """GPU init of a workload and its sampled fields (the state the oracle rows
    are compared on)."""
    from paper_2409_11470_gb300.binding import Simulation
    n0 = len(w["p"]["x"])
    sim = Simulation(w, capacity=int(capf * n0) + 1024, precision=precision, max_neigh=mn)
    sim.init()
    out = sample_fields(sim, ids)
    sim.close()
    return out


def oracle_table_leg(rows, torch):
    """The oracle's side of the table (part of the CPU-baseline leg): per
    configuration, its rate on the host cores and the GPU's sampled errors
    against it (rows carry the GPU's sampled fields)."""
    import numpy as np

    import apr_synth
    import oracle
    from paper_2409_11470_gb300.binding import Simulation
    out = {}
    # C1: one split pass, then density and force of all 4376 particles (brute force and tree)
    w = apr_synth.c1_lattice()
    res = {}
    for mode, enum in (("brute_force", 0), ("k_d_tree", 1)):
        o = oracle.Oracle(w, capacity=3 * 4096, enumerate=enum)
        o.split_merge(0)
        t0 = time.perf_counter()
        o.density()
        o.force()
        res[mode] = o.n / (time.perf_counter() - t0)
    g = rows["C1"]["sample"]
    errs = {p: _oracle_sample_errors(g[p], o, np.arange(o.n), False) for p in g}
    out["C1"] = {"oracle_particle_steps_per_s": res, "cores": o.threads(),
                 "oracle_kind": "split pass, then density + force of every particle", "errors": errs}
    # C2, C3, C4: the oracle's whole steps; errors on the GPU's sampled initial state
    for cname, wl in (("C2", "sod"), ("C3", "disc_planet"), ("C4", "flyby")):
        wfull, capf, _ = make_workload(wl, 0)
        ids = rows[cname]["ids"]
        n = len(wfull["p"]["x"])
        o = oracle.Oracle(wfull, capacity=int(capf * n) + 16)
        t0 = time.perf_counter()
        if cname == "C4":  # no particle is in the zone: density of all, forces of the sample
            o.track_regions()
            o.density()
            o.split_merge(0)
            oid = o["id"]
            order = np.argsort(oid)
            idx = order[np.searchsorted(oid[order], ids)]
            o.force(idx)
            o.sink_gravity()
        else:
            o.init()
            oid = o["id"]
            order = np.argsort(oid)
            idx = order[np.searchsorted(oid[order], ids)]
        t_init = time.perf_counter() - t0
        errs = {p: _oracle_sample_errors(rows[cname]["sample"][p], o, idx,
                                         int(wfull["cfg"]["eos"]) == 0)
                for p in rows[cname]["sample"]}
        if cname == "C4":
            del o
            rate = oracle_step_rate("flyby", 20.0)
            rate["note"] = "the same recipe at 250,000 particles (scaled; the oracle's cost per particle-step is set by the neighbour count, the same at either size)"
        else:
            rate = {"value": 0.0}
            dt = o.timestep()
            t0 = time.perf_counter()
            k = 0
            while k < 2 or time.perf_counter() - t0 < 10.0:
                o.step(dt)
                k += 1
            rate = {"value": k * o.n / (time.perf_counter() - t0), "steps": k, "cores": o.threads()}
        out[cname] = {"oracle_step": rate, "oracle_init_s": t_init, "errors": errs}
    # C5: the oracle's gradient on the 2048 splits nearest the centre
    w = apr_synth.c5_adjoint_lattice()
    prob = apr_synth.adjoint_problem(w)
    t0 = time.perf_counter()
    Jo, gdo, gho = oracle.Oracle(w).split_loss_grad(prob["parent"], prob["d"], prob["hc"],
                                                    prob["want"])
    t_o = time.perf_counter() - t0
    want = prob["want"]
    e = {}
    for p, (J, gd, gh) in rows["C5"]["grad"].items():
        e[p] = {"J": abs(J - Jo) / Jo,
                "grad_d_rel_l2": float(np.linalg.norm(gd[want] - gdo[want]) / np.linalg.norm(gdo[want])),
                "grad_h_rel_l2": float(np.linalg.norm(gh[np.repeat(want, 2)] - gho[np.repeat(want, 2)])
                                       / np.linalg.norm(gho[np.repeat(want, 2)]))}
    out["C5"] = {"oracle_s": t_o, "oracle_kind": "J and the gradient on the 2048-split subset "
                 "(every child's density error enters J)", "errors": e}
    return out


def run_table(args):
    """The C1-C5 table: one JSON line."""
    import numpy as np
    import torch

    import apr_synth
    from paper_2409_11470_gb300.binding import Simulation
    torch.cuda.set_device(0)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    peaks = measure_peaks(torch)
    rows = {}
    # C1: density + force after the split pass, repeated
    w = apr_synth.c1_lattice()
    c1 = {"config": "C1 lattice 16^3 + one split pass (4096 -> 4376)", "sample": {}}
    for prec in ("fp32", "fp64"):
        sim = Simulation(w, capacity=3 * 4096, precision=prec)
        sim.split_merge()
        sim.density()
        sim.force()
        st = sim.stream
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 50
        e0.record(st)
        for _ in range(reps):
            sim.density()
            sim.force()
        e1.record(st)
        st.synchronize()
        ms = e0.elapsed_time(e1) / reps
        c1[prec] = {"value": sim.n / (ms / 1e3), "ms_per_eval": ms}
        c1["sample"][prec] = {f: sim.get(f) for f in SAMPLE_FIELDS}
        c1["n"] = sim.n
        sim.close()
    rows["C1"] = c1
    rng = np.random.default_rng(4321)
    for cname, wl, k in (("C2", "sod", 20), ("C3", "disc_planet", 10), ("C4", "flyby", 10)):
        wfull, capf, mn = make_workload(wl, 0)
        n0 = len(wfull["p"]["x"])
        row = {"config": workload_label(wl, wfull), "sample": {}}
        if cname == "C4":
            ids = np.sort(rng.choice(n0, 1000, replace=False)).astype(np.uint64)
        else:  # ids after the initial refinement: children get new ids, so sample the GPU's
            sim = Simulation(wfull, capacity=int(capf * n0) + 1024, precision="fp64", max_neigh=mn)
            sim.init()
            ids = np.sort(rng.choice(sim.get("id"), 1000, replace=False))
            sim.close()
        row["ids"] = ids
        for prec, steps in (("fp32", k), ("fp64", max(2, k // 4))):
            r = measure(wfull, prec, steps, 2, torch, flush, capf, mn, ids)
            sm = summary(r, steps, peaks, prec)
            dom = max(sm["rooflines"], key=lambda x: x["share"]) if sm["rooflines"] else {}
            row[prec] = {"value": sm["value"], "ms_per_step": sm["ms_per_step"],
                         "n_after_init": sm["n_after_init"],
                         "dominant": {x: dom.get(x) for x in ("group", "kernel", "share", "bound",
                                                               "frac")}}
            row["sample"][prec] = r["sample"]
        row["fp32_over_fp64"] = row["fp32"]["value"] / row["fp64"]["value"]
        rows[cname] = row
    # C5: loss + gradient evaluations
    w = apr_synth.c5_adjoint_lattice()
    prob = apr_synth.adjoint_problem(w)
    n, npar = len(w["p"]["x"]), len(prob["parent"])
    c5 = {"config": "C5 126^3 lattice, split adjoint (2,000,376 particles)", "grad": {}}
    for prec in ("fp32", "fp64"):
        sim = Simulation(w, capacity=n + 2 * npar, precision=prec)
        dev = sim.device
        par = torch.as_tensor(prob["parent"], device=dev)
        d = torch.as_tensor(prob["d"], device=dev)
        hc = torch.as_tensor(prob["hc"], device=dev)
        J, gd, gh = sim.density_loss_grad(par, d, hc)
        st = sim.stream
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5 if prec == "fp32" else 2
        e0.record(st)
        for _ in range(reps):
            sim.density_loss_grad(par, d, hc)
        e1.record(st)
        st.synchronize()
        ms = e0.elapsed_time(e1) / reps
        c5[prec] = {"evals_per_s": 1e3 / ms, "ms_per_eval": ms}
        c5["grad"][prec] = (J, gd.cpu().numpy(), gh.cpu().numpy())
        sim.close()
    c5["fp32_over_fp64"] = c5["fp32"]["evals_per_s"] / c5["fp64"]["evals_per_s"]
    rows["C5"] = c5
    orc = oracle_table_leg(rows, torch)
    table = {}
    for cname, row in rows.items():
        t = {k: v for k, v in row.items() if k not in ("sample", "ids", "grad")}
        t["oracle"] = orc[cname]
        table[cname] = t
    print(json.dumps({"table": table, "peaks": peaks, "unit": UNIT}), flush=True)


def main():
    args = parse()
    if args.table:
        run_table(args)
        return
    if args.profile_workload:
        run_profile_workload(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
