#!/usr/bin/env python
"""Benchmark of the APR SPH hot path on one GB300 (replicas on N GPUs).

Workload: the full three-dimensional Sod shock tube (140x28x28 + 70x14x14 =
123,480 equal-mass particles, ~210k after the initial two-level refinement of
the slab |x| < 0.15 / 0.10).  A step is one whole pass of the hot path
(kick, drift, accretion, zones, split/merge, neighbour index, density solve,
forces, kick) through the C ABI.  Metric: particle-steps per second, counting
the particles the density and force passes ran on.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
(density + force on a bounded sample of the same state) instead.
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
WORKLOAD = "sod_shock_tube_3d_123480p_2level_slab"

# Algorithmic FP32 work per pair, counted once from the kernel source (FMA = 2):
# density, per pair inside 2h per Newton-Raphson iteration: relative coords 3,
# r^2 5, sqrt 1, q 1, M4 f and f' 8, two compensated sums 11, f'' and the third
# compensated sum (mu q^2 f'', for the step acceptance of the FP32 kernel) 10  -> 39;
# force, per pair inside max(2h_a, 2h_b): coords/r^2/rsqrt/r/q 12, two M4
# derivatives 8, F_a F_b 5, v.r 9, viscosity on approaching pairs (half) 6,
# pressure term 5, three compensated components 15, energy 7, conductivity 13,
# signal speed 3  -> 83.
FLOPS_PER_PAIR = {"density": 39.0, "force": 83.0}
FP32_LANES_PER_SM = 128
NUM_SMS = 152


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=5)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the side measurements (disc, flyby, split adjoint)")
    ap.add_argument("--extra-steps", type=int, default=10)
    ap.add_argument("--nL", type=int, default=28, help="shock-tube resolution (28 = full size)")
    ap.add_argument("--ncu-range", action="store_true",
                    help="bracket the timed steps with cudaProfilerStart/Stop (for ncu "
                         "--profile-from-start off)")
    ap.add_argument("--profile-workload", choices=["disc_planet", "disc_planet_bins"], default=None,
                    help="profiling only: initialise this workload, take --warmup steps, "
                         "then --steps steps inside cudaProfilerStart/Stop (the _bins form: "
                         "steps of 32 times the smallest limit in time-step bins 0..5)")
    return ap.parse_args()


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def workload(nL):
    import apr_synth
    return apr_synth.c2_sod() if nL == 28 else apr_synth.sod(nL)


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
        sim.step(0.0)
        ev[i][1].record(st)
        psteps += sim.n
    st.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    return ms, psteps


def traffic_record(kernel):
    """DRAM bytes per launch from a committed ncu summary (profiles/<kernel>_traffic_*.md,
    lines "key: value"), if it was taken on the current kernel source (else None)."""
    import glob
    paths = sorted(glob.glob(os.path.join(ROOT, "profiles", f"{kernel}_traffic_*.md")))
    if not paths:
        return None
    rec = {}
    with open(paths[0]) as f:
        for line in f:
            k, sep, v = line.partition(":")
            if sep and k.strip() in ("dram_bytes_per_launch", "n", "source_sha256_16"):
                rec[k.strip()] = v.strip()
    src = os.path.join(ROOT, "paper_2409_11470_gb300", "csrc", "apr_sph.cu")
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


def run_ours(args):
    import numpy as np
    import torch

    import apr_synth  # noqa: F401
    from paper_2409_11470_gb300.binding import F64_FIELDS, Simulation

    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    w = workload(args.nL)
    n0 = len(w["p"]["x"])
    cap = 3 * n0
    sim = Simulation(w, capacity=cap, precision="fp32")
    sim.init()
    n_init = sim.n
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        sim.step(0.0)
    props = torch.cuda.get_device_properties(local)
    uuid = getattr(props, "uuid", None)
    uuid = f"GPU-{uuid}" if uuid is not None and not str(uuid).startswith("GPU-") else uuid
    sim.profile_enable(True)
    launches0 = sim.profile()["launches"]  # kernels launched before the timed region
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(uuid)
    if args.ncu_range:
        torch.cuda.cudart().cudaProfilerStart()
    t_wall = time.perf_counter()
    ms, psteps = timed_steps(sim, torch, args.steps, flush)
    torch.cuda.synchronize()
    if args.ncu_range:
        torch.cuda.cudart().cudaProfilerStop()
    t_wall = time.perf_counter() - t_wall
    clocks = sampler.stop()
    prof = sim.profile()
    sim.profile_enable(False)
    launches = prof["launches"] - launches0
    ms_max, ps_all = replica_totals(torch, ms, psteps, world, "cuda")
    value = ps_all / (ms_max / 1e3)

    # roofline of the dominant kernel (live events on the library's stream)
    groups = {g: prof[g] for g in ("sort", "tree", "lists", "density", "force", "refine", "other")}
    dom = max(("density", "force"), key=lambda g: groups[g]["ms"])
    gd = groups[dom]
    sm_max = clocks["sm_max_mhz"] or 2070.0
    peak = NUM_SMS * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    flops_launch = gd["pairs"] * FLOPS_PER_PAIR[dom] / max(gd["calls"], 1)
    ms_launch = gd["ms"] / max(gd["calls"], 1)
    achieved = flops_launch / (ms_launch / 1e3) / 1e12
    tr = traffic_record(f"k_{dom}_f32")
    roofline = {"bound": "alu", "kernel": f"k_{dom}<float>", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": tr["dram_bytes_per_launch"] * (n_init / tr["n"]) if tr else None,
                "peak_note": f"FP32 FMA pipes: {NUM_SMS} SMs x {FP32_LANES_PER_SM} lanes x 2 x "
                             f"{sm_max:.0f} MHz (derived, no measured FP32 peak)",
                "pairs_per_launch": gd["pairs"] / max(gd["calls"], 1),
                "flops_per_pair": FLOPS_PER_PAIR[dom], "ms_per_launch": ms_launch}
    breakdown = {g: round(v["ms"] / args.steps, 4) for g, v in groups.items()}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": WORKLOAD if args.nL == 28 else f"sod_nL{args.nL}",
                      "n_initial": n0, "n_after_init": n_init, "n_last": sim.n,
                      "precision": "fp32-mixed (pair sums f32 compensated; state, integration, "
                                   "reductions f64)",
                      "l2": "flushed by a 256 MB write before every timed step",
                      "parallelism": "replicas" if world > 1 else "single GPU",
                      "wall_s_timed": t_wall, "launches_before_timed": launches0},
           "roofline": roofline, "breakdown_ms_per_step": breakdown,
           "gpu_launches": launches, "clocks": clocks}

    if rank == 0 and not args.no_fp64:
        s64 = Simulation(w, capacity=cap, precision="fp64")
        s64.init()
        for _ in range(max(1, args.warmup // 2)):
            s64.step(0.0)
        ms64, ps64 = timed_steps(s64, torch, args.fp64_steps, flush)
        v64 = ps64 / (ms64 / 1e3)
        out["fp64"] = {"value": v64, "ms_per_step": ms64 / args.fp64_steps,
                       "steps": args.fp64_steps}
        out["fp32_over_fp64"] = value / v64
        s64.close()

    if rank == 0 and not args.no_e2e:
        # the same steps through the C ABI with host buffers: every step uploads the
        # pinned host state (apr_upload), steps, and downloads it (apr_download); the
        # step length is the cached limit, read before the upload drops it
        fields = list(F64_FIELDS) + ["level", "flags", "id"]
        host = {f: b for f, b in sim.host_buffers().items() if f in fields}
        sim.download(host)
        st = sim.stream
        evs = []
        bi = bo = 0
        ps_e = 0
        for _ in range(args.steps):
            n = sim.n
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(st):
                flush.zero_()
            dt = sim.timestep()
            e0.record(st)
            sim.upload(host, n)
            sim.step(dt)
            n2 = sim.download(host)
            e1.record(st)
            st.synchronize()
            evs.append(e0.elapsed_time(e1))
            bi += sum(n * host[f].element_size() for f in fields)
            bo += sum(n2 * host[f].element_size() for f in fields)
            ps_e += n2
        out["e2e"] = {"value": ps_e / (sum(evs) / 1e3), "unit": UNIT,
                      "h2d_bytes_per_step": bi // args.steps, "d2h_bytes_per_step": bo // args.steps}

    if rank == 0 and world == 1 and not args.no_cpu:
        out["cpu_baseline"] = oracle_baseline(w, cap, args.cpu_seconds)

    if rank == 0 and not args.no_extra:
        sim.close()
        out["other_workloads"] = side_measurements(args, torch, flush)

    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    sim.close()  # idempotent
    if rank == 0:
        print(json.dumps(out), flush=True)


# ------------------------------------------------------- side measurements

def _workload_rate(w, precision, steps, warmup, torch, flush, cap_factor, max_neigh=0):
    from paper_2409_11470_gb300.binding import Simulation
    n0 = len(w["p"]["x"])
    sim = Simulation(w, capacity=int(cap_factor * n0) + 1024, precision=precision,
                     max_neigh=max_neigh)
    sim.init()
    n_init = sim.n
    m_sinks0 = sum(k["m"] for k in sim.sinks())
    for _ in range(warmup):
        sim.step(0.0)
    sim.profile(reset=True)
    sim.profile_enable(True)
    ms, psteps = timed_steps(sim, torch, steps, flush)
    prof = sim.profile()
    sim.profile_enable(False)
    res = {"value": psteps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps, "steps": steps,
           "n_after_init": n_init, "n_last": sim.n,
           "sink_mass_gain": sum(k["m"] for k in sim.sinks()) - m_sinks0,
           "breakdown_ms_per_step": {g: round(prof[g]["ms"] / steps, 3) for g in
                                     ("sort", "tree", "lists", "density", "force", "refine",
                                      "other")},
           "density_attempts_per_step": prof["density_attempts"] / steps,
           "retried_particles_per_step": prof["uncovered"] / steps,
           "shrunk_particles_per_step": prof["shrunk"] / steps}
    sim.close()
    return res


def side_measurements(args, torch, flush):
    """The disc workloads and the split adjoint, each on its own: particle-steps/s
    of whole steps (FP32-mixed and FP64) and loss+gradient evaluations/s."""
    import apr_synth
    out = {}
    k = max(1, args.extra_steps)
    # the discs' Gaussian vertical tails put up to ~1240 particles inside 2.25 h of a
    # tail particle (measured on the oracle's converged state): lists of 2048
    for name, make, cap_factor, fp64 in (
            ("disc_planet_1e6_3level_sphere", apr_synth.disc_planet, 1.6, True),
            ("flyby_disc_8e6_2level_sphere", apr_synth.flyby, 1.2, True)):
        try:
            w = make()
            r = {"n_initial": len(w["p"]["x"]), "max_neigh": 2048,
                 "fp32": _workload_rate(w, "fp32", k, 2, torch, flush, cap_factor, 2048)}
            if fp64:
                r["fp64"] = _workload_rate(w, "fp64", max(2, k // 3), 1, torch, flush, cap_factor,
                                           2048)
                r["fp32_over_fp64"] = r["fp32"]["value"] / r["fp64"]["value"]
            out[name] = r
        except Exception as e:  # a side measurement never takes the headline down
            out[name] = {"error": f"{type(e).__name__}: {e}"}
    for name, make, Bs, big, capf, mn in (
            ("sod_time_step_bins", apr_synth.c2_sod, (2, 3), 4, 3.0, 0),
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

def oracle_baseline(w, cap, seconds):
    """Density + force of the FP64 oracle (as it stands) on a bounded sample of the
    initialised state; returns particle-steps/s and how it was measured."""
    import numpy as np

    import oracle
    o = oracle.Oracle(w, capacity=cap)
    o.init()
    rng = np.random.default_rng(0)
    m = 256
    t = 0.0
    while True:
        sample = rng.choice(o.n, m, replace=False)
        t0 = time.perf_counter()
        o.density(sample)
        o.force(sample)
        t = time.perf_counter() - t0
        if t * 4 > seconds or m >= o.n:
            break
        m = min(o.n, int(m * max(2.0, 0.5 * seconds / max(t, 1e-3))))
    total = 0.0
    done = 0
    steps = max(1, int(round(seconds / max(t, 1e-3))))
    for _ in range(steps):
        sample = rng.choice(o.n, m, replace=False)
        t0 = time.perf_counter()
        o.density(sample)
        o.force(sample)
        total += time.perf_counter() - t0
        done += m
    return {"value": done / total, "unit": UNIT, "cores": o.threads(), "kind": "oracle",
            "sample": f"density+force of {m} random particles of the initialised "
                      f"{o.n}-particle shock tube, cell-list enumeration, "
                      f"{steps} sample(s), {total:.1f} s"}


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return
    w = workload(args.nL)
    n0 = len(w["p"]["x"])
    import numpy as np

    import oracle
    o = oracle.Oracle(w, capacity=3 * n0)
    o.init()
    rng = np.random.default_rng(0)
    per_step = max(1.0, 60.0 / max(args.steps + args.warmup, 1))  # whole run within minutes
    m = 256
    while True:
        sample = rng.choice(o.n, m, replace=False)
        t0 = time.perf_counter()
        o.density(sample)
        o.force(sample)
        t = time.perf_counter() - t0
        if t * 2 > per_step or m >= o.n:
            break
        m = min(o.n, int(m * max(2.0, 0.8 * per_step / max(t, 1e-3))))
    for _ in range(args.warmup):
        s = rng.choice(o.n, m, replace=False)
        o.density(s)
        o.force(s)
    total = 0.0
    for _ in range(args.steps):
        s = rng.choice(o.n, m, replace=False)
        t0 = time.perf_counter()
        o.density(s)
        o.force(s)
        total += time.perf_counter() - t0
    value = args.steps * m / total
    sample = (f"each step: density+force of {m} random particles of the initialised "
              f"{o.n}-particle shock tube (FP64 oracle, cell-list enumeration)")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD if args.nL == 28 else f"sod_nL{args.nL}",
                      "n_initial": n0, "n_after_init": o.n},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": o.threads(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
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
    bins = args.profile_workload.endswith("_bins")

    def one(first):
        if bins:
            sim.step_bins(32 * sim.timestep(), 5, init_bins=first)
        else:
            sim.step(0.0)

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


def main():
    args = parse()
    if args.profile_workload:
        run_profile_workload(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
