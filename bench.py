#!/usr/bin/env python
"""Benchmark of the direct-summation Hermite hot path on GB300.

Default workload: a Plummer sphere of N = 65536 equal masses, eps = 1e-3,
block time steps (Aarseth eta = 0.01, dt_max = 1/16), FP32 pair math with
double-single relative coordinates and accumulation (NB_F32DS), FP64 state.
One bench step advances the system by 1/16 N-body time unit through nb_step:
every block step inside runs the scheduler (K5), the j-predictor (K1), the
pair-force kernel (K2) with its partial-sum reduction (K3) and the Hermite
corrector (K4). The metric is pair interactions (N_active * N summed over the
block steps) per second, in G/s, and its fraction of FP32 peak at 60 flops per
acc+jerk interaction.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload block65536|h6block65536|full2p20|batch4096|serve|ext65536|bridge32768|small1024]

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (rank 0 only under torchrun). Multi-GPU runs are
independent replicas (the workload does not shard; weak scaling).
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "G pair-interactions/s (acc+jerk)"
UNIT = "G interactions/s"
FLOPS_PER_INTERACTION = 60
# the 6th-order pair adds the snap: a_ij (3), |v|^2 + r.a (6), beta (3), the three
# scale factors (3) and S = m a r^-3 - 6 alpha J - 3 beta A with its sum (3 x 6 + 3)
FLOPS_PER_INTERACTION6 = 97
FP64_NOMINAL_TFLOPS = 1.25
# algorithmic bytes per particle of the per-particle stages (FP64 SoA state):
# predictor: t, dt, m, x, v, a, j read (120 B) + x_p, v_p and the 48-B j-record written (96 B)
# corrector: index, t, dt, x_p, v_p, a, j, new a, j read (164 B) + x, v, a, j, t, dt written (112 B)
# DRAM bytes per launch of the dominant kernel (dram__bytes_read.sum + dram__bytes_write.sum,
# one-pass ncu capture of the same launch): full N = 2^20 F32-DS evaluation with the
# built-in plan (2048 i-blocks x 4 j-splits of k_force_tile32, 256-record j-tiles)
MEASURED_TRAFFIC = {("full2p20", "f32ds", 1 << 20): 348.6e6}
PREDICT_BYTES = 216
CORRECT_BYTES = 276
L2_FLUSH_BYTES = 256 << 20

WORKLOADS = {
    "block65536": dict(n=65536, eps=1e-3, eta=0.01, dt_max=1.0 / 16, shared_dt=0.0,
                       variant="f32ds", masses="equal", step_t=1.0 / 16, kind="evolve",
                       desc="Plummer N=65536 equal masses, eps=1e-3, block steps "
                            "(Aarseth eta=0.01, dt_max=1/16); one bench step = 1/16 time unit"),
    "full2p20": dict(n=2 ** 20, eps=1e-4, variant="f32ds", masses="lognormal", kind="force",
                     desc="Plummer N=2^20 log-normal masses (sigma 0.5), eps=1e-4; one bench "
                          "step = one full N^2 acc/jerk/pot evaluation (predict + force)"),
    "batch4096": dict(n=4096, n_lo=16, n_hi=4096, dt=1.0 / 512, variant="f32ds", kind="batch",
                      step_t=1.0 / 16, eps=None, masses="equal",
                      desc="4096 independent Plummer clusters, N log-uniform in [16, 4096], "
                           "eps = 1/(4 N^(1/3)), shared dt = 1/512, F32-DS; one bench step = "
                           "1/16 time unit = 32 graph-replayed steps of all clusters"),
    "serve": dict(n=64, n_lo=2 ** 8, n_hi=2 ** 18, t_span=0.125, eta=0.01, dt_max=1.0 / 16,
                  variant="f32ds", kind="serve", eps=None, masses="galaxy",
                  rates=(1e6,), sweep_fracs=(0.1, 0.5, 1.0, 2.0),
                  desc="Poisson stream of 64 requests on subsystems of 11 Plummer galaxies "
                       "with a 1% central point mass, N log-uniform in [2^8, 2^18], half one "
                       "force evaluation, half 1/8 time unit of block steps (eta=0.01, "
                       "dt_max=1/16), eps = 1/(4 N^(1/3)); one bench step = the whole stream at "
                       "the saturating rate (all requests at once); then the arrival rate is "
                       "swept at 0.1x-2x the measured saturation rate"),
    "ext65536": dict(n=65536, n_ext=65536, eps=1e-3, variant="f32ds", masses="equal", kind="ext",
                     desc="field-particle service (nb_force_ext): the force of a Plummer j-set of "
                          "N=65536 (eps=1e-3) on 65536 external particles of a second Plummer "
                          "sphere offset by (0.5, 0, 0); one bench step = one call with host "
                          "arrays in and out"),
    "bridge32768": dict(n=32768, eps=1e-3, eta=0.01, dt_max=1.0 / 16, variant="f32ds",
                        masses="equal", kind="bridge", step_t=1.0 / 16,
                        desc="bridge (Sect. V): two Plummer clusters of N=32768 (half mass, "
                             "radius x0.25) 2 length units apart, each advanced with its own "
                             "block-step Hermite (eta=0.01, dt_max=1/16), kicked by the other "
                             "every 1/16 time unit; one bench step = one nb_bridge_step"),
    "h6block65536": dict(n=65536, eps=1e-3, eta=0.02, eta_s=0.01, dt_max=1.0 / 16, shared_dt=0.0,
                         variant="f32ds", masses="equal", step_t=1.0 / 16, kind="evolve",
                         order=6,
                         desc="Plummer N=65536 equal masses, eps=1e-3, block steps of the "
                              "6th-order Hermite scheme (acc, jerk, snap per pair; Aarseth "
                              "criterion on a, jerk, snap, crackle with eta=0.02, eta_s=0.01, "
                              "dt_max=1/16); one bench step = 1/16 time unit"),
    "small1024": dict(n=1024, eps=1.0 / 64, eta=0.01, dt_max=1.0 / 16, shared_dt=1.0 / 256,
                      variant="f64", masses="equal", step_t=1.0 / 16, kind="evolve",
                      desc="Plummer N=1024, eps=1/64, shared dt=1/256, FP64 pairs; one bench "
                           "step = 16 shared steps"),
}


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="block65536")
    ap.add_argument("--variant", choices=["f32", "f32ds", "f64"], default=None)
    ap.add_argument("--n", type=int, default=None,
                    help="override the workload's particle count (profiling of smaller cases)")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="skip the library's autotuner (nb_autotune / nb_batch_autotune), which "
                         "otherwise runs in the untimed set-up; plans are then the built-in "
                         "heuristic")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fused-max-na", type=int, default=0,
                    help="largest due set the fused block-step kernel takes (0: library default)")
    ap.add_argument("--n-corr", type=int, default=0,
                    help="force evaluations + corrections per block step (P(EC)^n; 0/1: PEC)")
    ap.add_argument("--requests", type=int, default=None,
                    help="serve: requests in the stream (default 64)")
    ap.add_argument("--n-hi", type=int, default=None, help="serve: largest request N")
    ap.add_argument("--n-i", type=int, default=None,
                    help="full2p20: evaluate the force on a seeded i-subset of this size only "
                         "(profiling of the mid-size due sets of block steps)")
    ap.add_argument("--no-extras", action="store_true",
                    help="block65536: skip the full2p20 and serve measurements that the default "
                         "line carries as extra keys")
    return ap.parse_args(argv)


def workload(args):
    wl = dict(WORKLOADS[args.workload])
    if wl["kind"] == "serve":
        if args.requests:
            wl["n"] = args.requests
        if args.n_hi:
            wl["n_hi"] = args.n_hi
            wl["desc"] += " [N range overridden to [%d, %d]]" % (wl["n_lo"], args.n_hi)
        return wl
    if args.n:
        wl["n"] = args.n
        wl["desc"] = wl["desc"] + " [N overridden to %d]" % args.n
    return wl


# ---------------------------------------------------------------------------
# distributed plumbing (replicas: a barrier and a max over ranks, no data path)
# ---------------------------------------------------------------------------

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def aggregate(per_rank):
    """Whole-job numbers from per-rank (units, seconds) pairs: units summed over the
    replicas, time the slowest rank's."""
    units = sum(u for u, _ in per_rank)
    secs = max(s for _, s in per_rank)
    return units, secs


def emit(args, line):
    """Print the JSON line, or hand it to the caller that measures a sub-workload."""
    cap = getattr(args, "capture", None)
    if cap is not None:
        cap.append(line)
    else:
        print(json.dumps(line), flush=True)


class Dist:
    def __init__(self, world, backend):
        self.world = world
        self.pg = None
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend=backend)
            self.dist = dist

    def barrier(self):
        if self.world > 1:
            self.dist.barrier()

    def gather_pairs(self, units, secs, device=None):
        if self.world == 1:
            return [(units, secs)]
        import torch
        t = torch.tensor([units, secs], dtype=torch.float64, device=device)
        out = [torch.zeros_like(t) for _ in range(self.world)]
        self.dist.all_gather(out, t)
        return [(float(o[0]), float(o[1])) for o in out]

    def close(self):
        if self.world > 1:
            self.dist.destroy_process_group()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        reasons = sorted({self.NAMES[k] for _, _, fl in rows for k, v in enumerate(fl)
                          if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------
# peaks
# ---------------------------------------------------------------------------

def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            return json.load(open(path))
        except ValueError:
            return {}
    return {}


def fp32_peak_tflops(sm_count, sm_mhz):
    """FP32 peak: SMs x 128 FP32 lanes x 2 flops (FMA) x SM clock."""
    return sm_count * 128 * 2 * sm_mhz * 1e6 / 1e12


def stage_bandwidth(wl, n, fused_steps, fused_stage_ms, other_ms, planned_inter, peaks):
    """HBM-side rates of the O(N) stages: the fused kernel's predict stage (all N
    particles per fused step) and the planned-path corrector (the due particles of the
    planned steps), in GB/s of algorithmic bytes against the measured copy bandwidth."""
    if wl["kind"] != "evolve":
        return None
    hbm = float(peaks.get("hbm_gbs") or 0.0) or None
    out = {"hbm_peak_gbs": hbm, "predict_bytes_per_particle": PREDICT_BYTES,
           "correct_bytes_per_particle": CORRECT_BYTES}
    if fused_steps and fused_stage_ms[0] > 0:
        g = PREDICT_BYTES * n * fused_steps / (fused_stage_ms[0] / 1e3) / 1e9
        out["fused_predict_stage_gbs"] = g
        out["fused_predict_stage_us_per_step"] = 1e3 * fused_stage_ms[0] / fused_steps
    if fused_steps and fused_stage_ms[1] > 0:
        # the j-records every fused step's force stage reads (48 B per particle, from L2)
        out["fused_force_stage_record_gbs"] = 48.0 * n * fused_steps / (fused_stage_ms[1] / 1e3) / 1e9
        out["fused_force_stage_us_per_step"] = 1e3 * fused_stage_ms[1] / fused_steps
    if other_ms.get("correct_ms"):
        g = CORRECT_BYTES * (planned_inter / n) / (other_ms["correct_ms"] / 1e3) / 1e9
        out["planned_correct_gbs"] = g
    if hbm:
        for k in ("fused_predict_stage_gbs", "planned_correct_gbs"):
            if k in out:
                out[k.replace("_gbs", "_frac")] = out[k] / hbm
    return out


# ---------------------------------------------------------------------------
# the CPU oracle sample (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------

ORACLE_BLOCK_STEPS = 64


def oracle_sample(wl, particles, keep=None):
    """One bounded oracle sample of the workload; returns (interactions, seconds, desc).
    keep (a dict), for a full evaluation: receives the sample's indices and the oracle's
    acc, jerk, pot on them."""
    import oracle
    if wl["kind"] == "batch":
        # 32 seeded clusters spanning the size range, 64 shared steps each
        from paper_1409_5474_gb300 import ic
        sizes = np.rint(np.exp(np.linspace(np.log(wl["n_lo"]), np.log(wl["n_hi"]), 32)))
        inter = 0.0
        t0 = time.perf_counter()
        for c, n in enumerate(sizes.astype(int)):
            p = ic.plummer(int(n), int(ic.key(ic.MASTER_SEED, 8, c)))
            st = oracle.State(p.m, p.pos, p.vel)
            _, it = oracle.hermite_run(st, math.inf, float(ic.cluster_eps(n)) ** 2,
                                       dt_shared=wl["dt"], max_steps=64)
            inter += it
        dt = time.perf_counter() - t0
        return inter, dt, ("oracle shared-step Hermite on 32 clusters with N log-spaced in "
                           "[%d, %d]: initial evaluation + 64 steps each" % (wl["n_lo"], wl["n_hi"]))
    if wl["kind"] == "serve":
        # the force requests of the stream, smallest first, for about 10 s
        from paper_1409_5474_gb300 import ic
        reqs = ic.request_stream(wl["n"], 1.0, n_lo=wl["n_lo"], n_hi=wl["n_hi"],
                                 t_span=wl["t_span"])
        inter, used = 0.0, 0
        t0 = time.perf_counter()
        for r in sorted(reqs, key=lambda q: q.n):
            if r.kind != "force":
                continue
            q = ic.request_particles(r)
            e = float(ic.cluster_eps(r.n))
            oracle.force(q.m, q.pos, q.vel, e * e)
            inter += float(r.n) * r.n
            used += 1
            if time.perf_counter() - t0 > 10.0:
                break
        return inter, time.perf_counter() - t0, (
            "oracle force on the %d smallest force requests of the stream" % used)
    eps2 = wl["eps"] ** 2
    if wl["kind"] == "ext":
        from paper_1409_5474_gb300 import ic
        q = ic.plummer(wl["n_ext"], ic.MASTER_SEED + 7)
        ni = 2048
        t0 = time.perf_counter()
        oracle.force_ext(particles.m, particles.pos, particles.vel, eps2,
                         q.pos[:ni] + np.array([0.5, 0.0, 0.0]), q.vel[:ni])
        dt = time.perf_counter() - t0
        return float(ni) * particles.n, dt, (
            "oracle force_ext of the j-set on the first %d external particles" % ni)
    if wl["kind"] == "force":
        rng = np.random.default_rng(2014)
        ni = 4096
        idx = rng.choice(particles.n, size=ni, replace=False).astype(np.int32)
        t0 = time.perf_counter()
        ra, rj, rp = oracle.force(particles.m, particles.pos, particles.vel, eps2, idx=idx)
        dt = time.perf_counter() - t0
        if keep is not None:
            keep.update(idx=idx, acc=ra, jerk=rj, pot=rp)
        return float(ni) * particles.n, dt, (
            f"oracle force on a seeded {ni}-particle i-subset against all {particles.n} j")
    if wl.get("order", 4) == 6:
        st = oracle.State6(particles.m, particles.pos, particles.vel)
        t0 = time.perf_counter()
        steps, inter = oracle.hermite6_run(st, math.inf, eps2, eta=wl["eta"], eta_s=wl["eta_s"],
                                           dt_max=wl["dt_max"], max_steps=ORACLE_BLOCK_STEPS)
        return inter, time.perf_counter() - t0, (
            f"oracle 6th-order block-step Hermite of the same system from t=0: two-pass "
            f"start-up + first {ORACLE_BLOCK_STEPS} block steps")
    st = oracle.State(particles.m, particles.pos, particles.vel)
    t0 = time.perf_counter()
    if wl.get("shared_dt", 0.0) > 0:
        steps, inter = oracle.hermite_run(st, math.inf, eps2, dt_shared=wl["shared_dt"],
                                          max_steps=16)
        desc = "oracle shared-step Hermite: initial evaluation + 16 steps from t=0"
    else:
        steps, inter = oracle.hermite_run(st, math.inf, eps2, eta=wl["eta"],
                                          dt_max=wl["dt_max"], max_steps=ORACLE_BLOCK_STEPS)
        desc = (f"oracle block-step Hermite of the same system from t=0: initial full "
                f"evaluation + first {ORACLE_BLOCK_STEPS} block steps")
    dt = time.perf_counter() - t0
    return inter, dt, desc


def make_particles(wl):
    from paper_1409_5474_gb300 import ic
    return ic.plummer(wl["n"], ic.MASTER_SEED + (3 if wl["masses"] == "lognormal" else 0),
                      masses=wl["masses"])


# ---------------------------------------------------------------------------
# arms
# ---------------------------------------------------------------------------

def config_of(wl, name, variant):
    c = {"workload": name, "n": wl["n"], "eps": wl["eps"], "variant": variant,
         "desc": wl["desc"], "inputs": "seeded synthetic Plummer sphere",
         "l2": "flushed between timed steps (256 MB write)"}
    if wl["kind"] == "evolve":
        c.update({"eta": wl["eta"], "dt_max": wl["dt_max"], "shared_dt": wl["shared_dt"],
                  "step_time_units": wl["step_t"], "order": wl.get("order", 4)})
        if wl.get("order", 4) == 6:
            c["eta_s"] = wl["eta_s"]
    if wl["kind"] == "batch":
        c.update({"n_clusters": wl["n"], "n_range": [wl["n_lo"], wl["n_hi"]], "shared_dt": wl["dt"],
                  "eps": "1/(4 N^(1/3)) per cluster", "step_time_units": wl["step_t"],
                  "l2": "working set (~1 GB) larger than L2"})
    return c


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    wl = workload(args)
    variant = args.variant or wl["variant"]
    p = make_particles(wl) if wl["kind"] not in ("batch", "serve") else None
    inter_t = secs_t = 0.0
    desc = ""
    for k in range(args.warmup + args.steps):
        inter, secs, desc = oracle_sample(wl, p)
        if k >= args.warmup:
            inter_t += inter
            secs_t += secs
    value = inter_t / secs_t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs_t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(wl, args.workload, variant),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle", "build": oracle.CFLAGS,
                             "sample": desc + " (per step)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (there is no CPU path)")
    torch.cuda.set_device(local)
    dist = Dist(world, "nccl")
    from paper_1409_5474_gb300 import nbody

    nbody.load()
    wl = workload(args)
    variant = args.variant or wl["variant"]
    if wl["kind"] == "batch":
        return run_batch(args, wl, variant, dist, rank, world, local)
    if wl["kind"] == "serve":
        return run_serve(args, wl, variant, dist, rank, world, local)
    if wl["kind"] == "ext":
        return run_ext(args, wl, variant, dist, rank, world, local)
    if wl["kind"] == "bridge":
        return run_bridge(args, wl, variant, dist, rank, world, local)
    p = make_particles(wl)
    stream = torch.cuda.Stream()          # the stream every kernel of the step runs on
    torch.cuda.set_stream(stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    cfg = dict(variant=variant, eps=wl["eps"], device=local, flags=nbody.NB_FLAG_TIMING,
               fused_max_na=args.fused_max_na, n_corr=args.n_corr)
    order = wl.get("order", 4)
    fpi = FLOPS_PER_INTERACTION6 if order == 6 else FLOPS_PER_INTERACTION
    if wl["kind"] == "evolve":
        cfg.update(eta=wl["eta"], dt_max=wl["dt_max"], shared_dt=wl["shared_dt"])
    if order == 6:
        cfg.update(order=6, eta_s=wl["eta_s"])
    sysm = nbody.System(p.m, p.pos, p.vel, **cfg)
    h = sysm.h
    nbody.nb_set_stream(h, stream.cuda_stream)
    n = p.n
    t_tune = time.perf_counter()
    # block steps use every N_active bucket: tune them all; a full evaluation uses one
    # plan, which the built-in heuristic already takes from a sweep
    # (a force on an i-subset, --n-i, is tuned too: profiling of the block steps' plans)
    plan_table = (nbody.nb_autotune(h, 3)
                  if args.autotune and (wl["kind"] == "evolve" or args.n_i)
                  else None)
    t_tune = time.perf_counter() - t_tune

    def one_step(k, host_state):
        """One bench step; returns (interactions, device_ms, wall_s, launches, stats, state)."""
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        if wl["kind"] == "evolve":
            w0 = time.perf_counter()
            if host_state is not None:
                nbody.nb_set_state(h, host_state)          # H2D of the whole state
                if order == 6:
                    nbody.nb_set_snap(h, host_state["snap"], host_state["crackle"])
            e0.record(stream)
            st = nbody.nb_step(h, (k + 1) * wl["step_t"])
            e1.record(stream)
            out = nbody.nb_get_state(h)                    # D2H of the whole state
            if order == 6:
                out["snap"], out["crackle"] = nbody.nb_get_snap(h)
            w1 = time.perf_counter()
            stream.synchronize()
            return st["interactions"], e0.elapsed_time(e1), w1 - w0, st["kernel_launches"], st, out
        # full evaluation: predict to t0 and one N^2 force (or the force on an i-subset)
        before = nbody.nb_get_stats(h)
        w0 = time.perf_counter()
        if host_state is not None:
            nbody.nb_set_particles(h, p.m, p.pos.T, p.vel.T, 0.0)
        e0.record(stream)
        nbody.nb_predict(h, 0.0)
        nbody.nb_force_dev(h, d_idx.data_ptr() if d_idx is not None else 0, n_i,
                           bufs[0:3].data_ptr(), bufs[3:6].data_ptr(), bufs[6].data_ptr())
        e1.record(stream)
        host = bufs.cpu()                                  # D2H of acc, jerk, pot
        w1 = time.perf_counter()
        stream.synchronize()
        after = nbody.nb_get_stats(h)
        d = {k_: after[k_] - before[k_] for k_ in ("interactions", "force_ms", "reduce_ms",
                                                    "predict_ms", "kernel_launches",
                                                    "force_launches")}
        return d["interactions"], e0.elapsed_time(e1), w1 - w0, d["kernel_launches"], d, host

    n_i = min(args.n_i, n) if (args.n_i and wl["kind"] == "force") else n
    d_idx = None
    if n_i < n:
        sub_idx = np.sort(np.random.default_rng(1500).choice(n, size=n_i, replace=False))
        d_idx = torch.from_numpy(sub_idx.astype(np.int32)).cuda()
    bufs = torch.empty((7, n_i), dtype=torch.float64, device="cuda") if wl["kind"] == "force" else None
    host_state = None
    for k in range(args.warmup):
        one_step(k, None)
    energy0 = None
    if wl["kind"] == "evolve":
        host_state = nbody.nb_get_state(h)
        if order == 6:
            host_state["snap"], host_state["crackle"] = nbody.nb_get_snap(h)
        energy0 = sum(nbody.nb_energy(h))          # untimed: softened E at a synchronised time
    else:
        host_state = True
    nbody.nb_reset_stats(h)
    torch.cuda.synchronize()
    dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    tot_inter = tot_ms = tot_wall = 0.0
    launches = 0
    force_ms = reduce_ms = 0.0
    force_launches = 0
    other_ms = {"sched_ms": 0.0, "predict_ms": 0.0, "correct_ms": 0.0, "fused_ms": 0.0}
    fused_steps = 0
    block_steps = 0
    hist = {"active_hist": [0] * 32, "force_ms_hist": [0.0] * 32, "inter_hist": [0.0] * 32,
            "fused_step_ms_hist": [0.0] * 32}
    fused_stage_ms = [0.0] * 4
    torch.cuda.nvtx.range_push("timed")  # profilers can select the timed steps by this range
    for k in range(args.warmup, args.warmup + args.steps):
        flush.fill_(float(k))                              # L2 flush between timed steps
        inter, ms, wall, nl, st, host_state = one_step(k, host_state)
        tot_inter += inter
        tot_ms += ms
        tot_wall += wall
        launches += nl
        force_ms += st["force_ms"]
        reduce_ms += st["reduce_ms"]
        force_launches += st["force_launches"]
        for key in other_ms:
            other_ms[key] += st.get(key, 0.0)
        block_steps += st.get("block_steps", 0)
        fused_steps += st.get("fused_steps", 0)
        for q, x in enumerate(st.get("fused_stage_ms", [0.0] * 4)):
            fused_stage_ms[q] += x
        for key in hist:
            for b, x in enumerate(st.get(key, [0] * 32)):
                hist[key][b] += x
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    clocks = sampler.stop()
    energy1 = sum(nbody.nb_energy(h)) if energy0 is not None else None  # untimed
    dist.barrier()
    pairs = dist.gather_pairs(tot_inter, tot_ms / 1e3, device="cuda")
    units, secs = aggregate(pairs)
    wall_pairs = dist.gather_pairs(tot_inter, tot_wall, device="cuda")
    e2e_units, e2e_secs = aggregate(wall_pairs)
    if rank != 0:
        sysm.close()
        dist.close()
        return 0
    props = torch.cuda.get_device_properties(local)
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz") or (clocks or {}).get("sm_max_mhz") or 2070.0)
    peak = fp32_peak_tflops(props.multi_processor_count, sm_max)
    peak_source = ("SMs x 128 x 2 x max SM clock %.0f MHz (derived; FP32 is not in "
                   "MEASURED_PEAKS.json)" % sm_max)
    if variant == "f64":
        # the FP64 pair path is bound by GB300's FP64 rate
        peak = FP64_NOMINAL_TFLOPS
        peak_source = "GB300 nominal dense FP64 rate (not measured)"
    value = units / secs / 1e9
    # the planned force launches' own interactions (the fused kernel's steps are
    # timed as a whole and reported apart)
    planned_inter = float(sum(hist["inter_hist"])) if wl["kind"] == "evolve" else tot_inter
    achieved = fpi * planned_inter / (force_ms / 1e3) / 1e12 if force_ms else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if variant == "f64" else "f32",
        "data": "synthetic (seeded Plummer sphere, N-body units)",
        "config": dict(config_of(wl, args.workload, variant),
                       parallelism=("replicas%d" % world) if world > 1 else "single GPU",
                       corrector=("P(EC)^%d" % args.n_corr) if args.n_corr > 1 else "PEC",
                       integrator="Hermite order %d" % order),
        "fp32_peak_frac": fpi * value * 1e9 / (peak * 1e12),
        "roofline": {"bound": "alu",
                     "kernel": ("k_force6_tile32 / k_force6_tile64 (6th-order pair force)"
                                if order == 6 else
                                "k_force_tile64/k_force_jmode64 (planned FP64 pair force)"
                                if variant == "f64" else
                                "k_force_tile32/k_force_wgrp32/k_force_tiny32 (planned pair force)"),
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": (achieved / peak) if achieved else None,
                     "traffic": (MEASURED_TRAFFIC.get((args.workload, variant, n))
                                 if not args.autotune or wl["kind"] != "evolve" else None),
                     "peak_source": peak_source,
                     "flops_per_interaction": fpi,
                     "force_ms": force_ms, "reduce_ms": reduce_ms,
                     "force_launches": force_launches, "interactions": planned_inter},
        "kernel_ms": dict(other_ms, force_ms=force_ms, reduce_ms=reduce_ms),
        "block_steps": block_steps,
        "fused_steps": fused_steps,
        "stage_bandwidth": (stage_bandwidth(wl, n, fused_steps, fused_stage_ms, other_ms,
                                            float(sum(hist["inter_hist"])), peaks)
                            if order == 4 else None),
        "energy": ({"E0": energy0, "E1": energy1,
                    "rel_drift": abs(energy1 - energy0) / abs(energy0),
                    "over_time_units": args.steps * wl["step_t"]}
                   if energy0 is not None else None),
        "fused_stage_ms": {"predict": fused_stage_ms[0], "force": fused_stage_ms[1],
                           "reduce_correct": fused_stage_ms[2], "step_barrier": fused_stage_ms[3]},
        "by_log2_active": {k: [round(x, 3) if isinstance(x, float) else x for x in v]
                           for k, v in hist.items()},
        "e2e": {"value": e2e_units / e2e_secs / 1e9, "unit": UNIT,
                "h2d_bytes_per_step": (n * (15 if order == 4 else 21) * 8)
                if wl["kind"] == "evolve" else n * 7 * 8,
                "d2h_bytes_per_step": (n * (15 if order == 4 else 21) * 8)
                if wl["kind"] == "evolve" else n_i * 7 * 8},
        "gpu_launches": launches,
        "plans": ("autotuned (nb_autotune, %.1f s untimed set-up)" % t_tune) if plan_table
                 else "built-in heuristic",
        "plan_table": ([list(e) for e in plan_table[:nbody_bucket(n) + 1]] if plan_table else None),
        "interactions": tot_inter,
        "clocks": clocks,
    }
    if n_i < n:
        line["config"]["n_i"] = n_i
        line["config"]["desc"] += " [force on a seeded %d-particle i-subset]" % n_i
    if world == 1 and not args.no_cpu_baseline:
        import oracle
        keep = {}
        inter, secs_c, desc = oracle_sample(wl, p, keep)
        line["cpu_baseline"] = {"value": inter / secs_c / 1e9, "unit": UNIT,
                                "cores": oracle.num_threads(), "kind": "oracle", "build": oracle.CFLAGS, "sample": desc,
                                "seconds": secs_c}
        if wl["kind"] == "force" and n_i == n and "idx" in keep:
            # the GPU's last evaluation against the oracle's values on the timed sample
            g = np.asarray(host_state)[:, keep["idx"]]
            line["cpu_baseline"]["gpu_error"] = force_errors(
                g[0:3].T, g[3:6].T, g[6], keep["acc"], keep["jerk"], keep["pot"])
    sysm.close()
    if (args.workload == "block65536" and world == 1 and not args.no_extras
            and getattr(args, "capture", None) is None):
        line.update(extras(args))
    emit(args, line)
    dist.close()
    return 0


def nbody_bucket(n):
    """Plan-table bucket of an i-set of n: ceil(log2 n)."""
    return max(0, int(math.ceil(math.log2(max(1, n)))))


def force_errors(acc, jerk, pot, ra, rj, rp):
    """Error of GPU forces against the oracle's on the same particles: relative RMS over
    the set and the per-particle max and median of |d_i| / |ref_i|, per quantity."""
    out = {}
    for name, got, ref in (("acc", acc, ra), ("jerk", jerk, rj), ("pot", pot, rp)):
        got = np.asarray(got, dtype=np.float64)
        ref = np.asarray(ref, dtype=np.float64)
        d = got - ref
        if ref.ndim == 1:
            per = np.abs(d) / np.abs(ref)
        else:
            per = np.linalg.norm(d, axis=1) / np.linalg.norm(ref, axis=1)
        out[name] = {"rel_rms": float(np.sqrt((d ** 2).sum() / (ref ** 2).sum())),
                     "max": float(per.max()), "median": float(np.median(per))}
    out["particles"] = int(np.asarray(rp).shape[0])
    return out


def extras(args):
    """The two targets that the default line carries beside block65536: one full N = 2^20
    evaluation (three timed repeats, its roofline and its error against the oracle on the
    cpu_baseline sample) and the request loop on the config-5 stream at the saturating
    rate (p50 / p99 latency and G/s against one request per launch; no rate sweep)."""
    out = {}
    sub = argparse.Namespace(**vars(args))
    sub.workload, sub.steps, sub.warmup, sub.n, sub.n_i = "full2p20", 3, 1, None, None
    sub.variant, sub.capture, sub.no_extras = None, [], True
    run_ours(sub)
    f = sub.capture[0]
    out["full2p20"] = {k: f.get(k) for k in ("value", "unit", "steps", "warmup", "ms_per_step",
                                             "fp32_peak_frac", "roofline", "e2e", "clocks",
                                             "gpu_launches", "cpu_baseline", "config")}
    sub = argparse.Namespace(**vars(args))
    sub.workload, sub.steps, sub.warmup, sub.variant = "serve", 1, 1, None
    sub.requests, sub.n_hi, sub.capture, sub.no_extras = None, None, [], True
    sub.no_cpu_baseline, sub.serve_sweep = True, False
    run_serve(sub, workload(sub), "f32ds", Dist(1, None), 0, 1,
              int(os.environ.get("LOCAL_RANK", "0")))
    v = sub.capture[0]
    one = v["one_request_per_launch"]
    out["serve"] = {"value": v["value"], "unit": v["unit"], "latency": v["latency"],
                    "makespan_s": v["sweep"][-1]["server"]["makespan_s"],
                    "one_request_per_launch": {"value": one["throughput"], "unit": UNIT,
                                               "latency": one["latency"],
                                               "makespan_s": one["makespan_s"]},
                    "fp32_peak_frac": v["fp32_peak_frac"], "clocks": v["clocks"],
                    "gpu_launches": v["gpu_launches"], "server_stats": v["server_stats"],
                    "config": v["config"]}
    return out


def run_batch(args, wl, variant, dist, rank, world, local):
    """Config 4: many clusters, one graph-replayed shared step of all of them at a time."""
    import torch
    from paper_1409_5474_gb300 import ic, nbody

    systems = ic.cluster_batch(wl["n"], wl["n_lo"], wl["n_hi"])
    sizes = np.array([len(p.m) for p in systems])
    eps = ic.cluster_eps(sizes)
    bt = nbody.Batch(systems, eps, wl["dt"], variant=variant, device=local,
                     flags=nbody.NB_FLAG_TIMING)
    threads = bt.autotune() if args.autotune else None
    steps_per = int(round(wl["step_t"] / wl["dt"]))
    m = np.concatenate([p.m for p in systems])
    for _ in range(args.warmup):
        bt.step(steps_per)
    pos, vel, _ = bt.get()
    torch.cuda.synchronize()
    dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    tot_inter = tot_dev = tot_wall = force_ms = 0.0
    launches = 0
    for k in range(args.steps):
        w0 = time.perf_counter()
        nbody.nb_batch_set(bt.b, m, pos, vel, (args.warmup + k) * wl["step_t"])  # H2D
        e0 = time.perf_counter()
        st = bt.step(steps_per)
        e1 = time.perf_counter()
        pos, vel, _ = bt.get()                                                    # D2H
        w1 = time.perf_counter()
        inter = st["interactions"] - float((sizes.astype(np.float64) ** 2).sum())  # minus init
        tot_inter += inter
        tot_dev += e1 - e0
        tot_wall += w1 - w0
        force_ms += st["force_ms"]
        launches += st["kernel_launches"]
    clocks = sampler.stop()
    dist.barrier()
    units, secs = aggregate(dist.gather_pairs(tot_inter, tot_dev, device="cuda"))
    e2e_units, e2e_secs = aggregate(dist.gather_pairs(tot_inter, tot_wall, device="cuda"))
    if rank != 0:
        bt.close()
        dist.close()
        return 0
    props = torch.cuda.get_device_properties(local)
    sm_max = float(measured_peaks().get("sm_max_mhz") or 2070.0)
    peak = fp32_peak_tflops(props.multi_processor_count, sm_max)
    value = units / secs / 1e9
    achieved = FLOPS_PER_INTERACTION * tot_inter / (force_ms / 1e3) / 1e12 if force_ms else None
    ntot = int(sizes.sum())
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded Plummer clusters, N-body units)",
        "config": dict(config_of(wl, args.workload, variant),
                       parallelism=("replicas%d" % world) if world > 1 else "single GPU",
                       cta_threads=threads or "default 128", particles=ntot),
        "fp32_peak_frac": FLOPS_PER_INTERACTION * value * 1e9 / (peak * 1e12),
        "roofline": {"bound": "alu", "kernel": "k_force_items32 (batched pair force)",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": None,
                     "peak_source": "SMs x 128 x 2 x max SM clock %.0f MHz (derived)" % sm_max,
                     "force_ms": force_ms},
        "e2e": {"value": e2e_units / e2e_secs / 1e9, "unit": UNIT,
                "h2d_bytes_per_step": ntot * 7 * 8, "d2h_bytes_per_step": ntot * 6 * 8,
                "note": "host set includes a fresh initial evaluation, not counted as work"},
        "gpu_launches": launches,
        "interactions": tot_inter,
        "clocks": clocks,
        "timing": "host wall clock around nb_batch_step (synchronous) for value",
    }
    if world == 1 and not args.no_cpu_baseline:
        import oracle
        inter, secs_c, desc = oracle_sample(wl, None)
        line["cpu_baseline"] = {"value": inter / secs_c / 1e9, "unit": UNIT,
                                "cores": oracle.num_threads(), "kind": "oracle", "build": oracle.CFLAGS, "sample": desc,
                                "seconds": secs_c}
    emit(args, line)
    bt.close()
    dist.close()
    return 0

# ---------------------------------------------------------------------------
# the field-particle service (nb_force_ext): an i-set disjoint from the j-set
# ---------------------------------------------------------------------------

def run_ext(args, wl, variant, dist, rank, world, local):
    """The force of the predicted j-set on an external i-set, as a hybrid code would call
    it every bridge kick (host arrays in and out: the call is end to end by design)."""
    import torch
    from paper_1409_5474_gb300 import ic, nbody

    p = make_particles(wl)
    q = ic.plummer(wl["n_ext"], ic.MASTER_SEED + 7)
    ipos = (q.pos + np.array([0.5, 0.0, 0.0])).T.copy()
    ivel = q.vel.T.copy()
    sysm = nbody.System(p.m, p.pos, p.vel, variant=variant, eps=wl["eps"], device=local,
                        flags=nbody.NB_FLAG_TIMING)
    h = sysm.h
    nbody.nb_predict(h, 0.0)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        nbody.nb_force_ext(h, ipos, ivel)
    nbody.nb_reset_stats(h)
    torch.cuda.synchronize()
    dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    wall = 0.0
    for k in range(args.steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nbody.nb_force_ext(h, ipos, ivel)
        wall += time.perf_counter() - t0
    clocks = sampler.stop()
    st = nbody.nb_get_stats(h)
    inter = float(wl["n_ext"]) * p.n * args.steps
    units, secs = aggregate(dist.gather_pairs(inter, wall, device="cuda"))
    if rank != 0:
        sysm.close()
        dist.close()
        return 0
    props = torch.cuda.get_device_properties(local)
    sm_max = float(measured_peaks().get("sm_max_mhz") or 2070.0)
    peak = fp32_peak_tflops(props.multi_processor_count, sm_max)
    value = units / secs / 1e9
    force_ms = st["force_ms"]
    achieved = FLOPS_PER_INTERACTION * inter / (force_ms / 1e3) / 1e12 if force_ms else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded Plummer spheres, N-body units)",
        "config": dict(config_of(wl, args.workload, variant), n_ext=wl["n_ext"],
                       parallelism="single GPU", timing="host wall clock around the call"),
        "fp32_peak_frac": FLOPS_PER_INTERACTION * value * 1e9 / (peak * 1e12),
        "roofline": {"bound": "alu", "kernel": "k_force_tile32 (planned pair force, external i)",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak if achieved else None, "traffic": None,
                     "force_ms": force_ms,
                     "peak_source": "SMs x 128 x 2 x max SM clock %.0f MHz (derived)" % sm_max},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 48 * wl["n_ext"],
                "d2h_bytes_per_step": 56 * wl["n_ext"],
                "note": "the call takes and returns host arrays: value is end to end"},
        "gpu_launches": int(st["kernel_launches"]),
        "clocks": clocks,
    }
    if world == 1 and not args.no_cpu_baseline:
        import oracle
        ni = 2048
        t0 = time.perf_counter()
        oracle.force_ext(p.m, p.pos, p.vel, wl["eps"] ** 2, ipos[:, :ni].T, ivel[:, :ni].T)
        secs_c = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": ni * p.n / secs_c / 1e9, "unit": UNIT,
                                "cores": oracle.num_threads(), "kind": "oracle", "build": oracle.CFLAGS,
                                "sample": "oracle force_ext of the j-set on the first %d "
                                          "external particles" % ni, "seconds": secs_c}
    emit(args, line)
    sysm.close()
    dist.close()
    return 0


def run_bridge(args, wl, variant, dist, rank, world, local):
    """Two systems coupled by the bridge; interactions = both systems' own block-step
    evaluations plus the four cross evaluations (kicks) per step."""
    import torch
    from paper_1409_5474_gb300 import ic, nbody

    n = wl["n"]
    a = ic.plummer(n, ic.MASTER_SEED + 11)
    b = ic.plummer(n, ic.MASTER_SEED + 12)
    off = np.array([1.0, 0.0, 0.0])
    vorb = np.array([0.0, 0.5 * math.sqrt(1.0 / 2.0), 0.0])   # mutual orbit of two halves
    kw = dict(variant=variant, eps=wl["eps"], eta=wl["eta"], dt_max=wl["dt_max"], device=local,
              flags=nbody.NB_FLAG_TIMING)
    A = nbody.System(a.m * 0.5, a.pos * 0.25 - off, a.vel * math.sqrt(2.0) - vorb, **kw)
    B = nbody.System(b.m * 0.5, b.pos * 0.25 + off, b.vel * math.sqrt(2.0) + vorb, **kw)
    for _ in range(args.warmup):
        nbody.nb_bridge_step(A.h, B.h, wl["step_t"])
    nbody.nb_reset_stats(A.h)
    nbody.nb_reset_stats(B.h)
    torch.cuda.synchronize()
    dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        nbody.nb_bridge_step(A.h, B.h, wl["step_t"])
    wall = time.perf_counter() - t0
    clocks = sampler.stop()
    sa, sb = nbody.nb_get_stats(A.h), nbody.nb_get_stats(B.h)
    inter = sa["interactions"] + sb["interactions"]
    units, secs = aggregate(dist.gather_pairs(inter, wall, device="cuda"))
    if rank != 0:
        A.close()
        B.close()
        dist.close()
        return 0
    props = torch.cuda.get_device_properties(local)
    sm_max = float(measured_peaks().get("sm_max_mhz") or 2070.0)
    peak = fp32_peak_tflops(props.multi_processor_count, sm_max)
    value = units / secs / 1e9
    force_ms = sa["force_ms"] + sb["force_ms"]
    planned = float(sum(sa["inter_hist"]) + sum(sb["inter_hist"]))
    achieved = FLOPS_PER_INTERACTION * planned / (force_ms / 1e3) / 1e12 if force_ms else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded Plummer spheres, N-body units)",
        "config": dict(config_of(wl, args.workload, variant), systems=2,
                       parallelism="single GPU", timing="host wall clock around the call"),
        "fp32_peak_frac": FLOPS_PER_INTERACTION * value * 1e9 / (peak * 1e12),
        "roofline": {"bound": "alu", "kernel": "planned pair force kernels (both systems)",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak if achieved else None, "traffic": None,
                     "force_ms": force_ms,
                     "peak_source": "SMs x 128 x 2 x max SM clock %.0f MHz (derived)" % sm_max},
        "block_steps": sa["block_steps"] + sb["block_steps"],
        "fused_steps": sa["fused_steps"] + sb["fused_steps"],
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0,
                "note": "the state stays on the device; value is the call's wall clock"},
        "gpu_launches": int(sa["kernel_launches"] + sb["kernel_launches"]),
        "clocks": clocks,
    }
    emit(args, line)
    A.close()
    B.close()
    dist.close()
    return 0


# ---------------------------------------------------------------------------
# config 5: the request loop
# ---------------------------------------------------------------------------

def _pct(xs, q):
    return float(np.percentile(np.asarray(xs, dtype=np.float64), q)) if len(xs) else None


def _lat(xs):
    return {"p50_s": _pct(xs, 50), "p99_s": _pct(xs, 99), "mean_s": float(np.mean(xs)),
            "max_s": float(np.max(xs))}


def run_serve(args, wl, variant, dist, rank, world, local):
    """Config 5: a Poisson stream of force / evolve requests through the request loop
    (nb_submit / nb_wait: continuous batching, one batched force launch per tick), and the
    same requests served one at a time through the plain engine calls (nb_set_particles +
    nb_predict + nb_force, or nb_step), in arrival order."""
    import threading
    import torch
    from paper_1409_5474_gb300 import ic, nbody

    base = ic.request_stream(wl["n"], 1.0, n_lo=wl["n_lo"], n_hi=wl["n_hi"], t_span=wl["t_span"])
    parts = [ic.request_particles(r) for r in base]
    eps = [float(ic.cluster_eps(r.n)) for r in base]
    var = nbody.VARIANTS[variant]
    srv = nbody.Server(variant=var, device=local, budget_bytes=64 << 30, max_inflight=64,
                       max_queue=4096, eta=wl["eta"], dt_max=wl["dt_max"])

    def submit(r, i, force_only=False):
        p = parts[i]
        if force_only or r.kind == "force":
            return srv.force(p.m, p.pos.T, p.vel.T, eps[i])
        return srv.evolve(p.m, p.pos.T, p.vel.T, eps[i], r.t_span)

    def run_stream(rate, force_only=False):
        """Replay the stream at `rate` (a submitter thread sleeps until each arrival);
        returns the results (server clock) in request order."""
        reqs = ic.request_stream(wl["n"], rate, n_lo=wl["n_lo"], n_hi=wl["n_hi"],
                                 t_span=wl["t_span"])
        tickets = [None] * len(reqs)
        ready = [threading.Event() for _ in reqs]
        t0 = time.perf_counter()

        def submitter():
            for i, r in enumerate(reqs):
                d = t0 + r.arrival - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                tickets[i] = submit(r, i, force_only)
                ready[i].set()

        th = threading.Thread(target=submitter)
        th.start()
        res = []
        for i in range(len(reqs)):
            ready[i].wait()
            res.append(srv.wait(tickets[i], timeout_s=7200))
        th.join()
        bad = [r for r in res if r["status"] != nbody.NB_STATUS_DONE]
        if bad:
            raise RuntimeError("request failed: %s" % bad[0])
        return reqs, res

    def summarise(reqs, res):
        lat = [r["t_done"] - r["t_submit"] for r in res]
        span = max(r["t_done"] for r in res) - min(r["t_submit"] for r in res)
        inter = sum(r["interactions"] for r in res)
        out = {"throughput": inter / span / 1e9, "makespan_s": span, "interactions": inter,
               "latency": _lat(lat)}
        for kind in ("force", "evolve"):
            xs = [x for x, q in zip(lat, reqs) if q.kind == kind]
            if xs:
                out["latency_" + kind] = _lat(xs)
        return out

    # warm-up: the stream as force requests only (fills the handle pool, loads the kernels)
    for _ in range(args.warmup):
        run_stream(wl["rates"][-1], force_only=True)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    st0 = srv.stats()
    timed = []
    for _ in range(args.steps):
        timed.append(summarise(*run_stream(wl["rates"][-1])))
    st1 = srv.stats()
    clocks = sampler.stop()
    # arrival rates relative to saturation: the requests per second the server sustains
    # when all arrive at once (count / makespan of the timed streams)
    r_sat = len(base) / (sum(t["makespan_s"] for t in timed) / len(timed))
    sweep = []
    for frac in (wl["sweep_fracs"] if getattr(args, "serve_sweep", True) else ()):
        rate = frac * r_sat
        reqs, res = run_stream(rate)
        sweep.append({"rate_hz": rate, "frac_of_saturation": frac,
                      "server": summarise(reqs, res)})

    # one request per launch: pre-created engine handles, requests served in arrival order
    systems = [nbody.System(p.m, p.pos, p.vel, variant=variant, eps=e, eta=wl["eta"],
                            dt_max=wl["dt_max"], device=local) for p, e in zip(parts, eps)]
    service, b_inter = [], []
    for r, p, sy in zip(base, parts, systems):
        t0 = time.perf_counter()
        nbody.nb_set_particles(sy.h, p.m, p.pos.T, p.vel.T, 0.0)
        if r.kind == "force":
            nbody.nb_predict(sy.h, 0.0)
            nbody.nb_force(sy.h)
            it = float(r.n) * r.n
        else:
            it = nbody.nb_step(sy.h, r.t_span)["interactions"]
            nbody.nb_get_particles(sy.h)
        service.append(time.perf_counter() - t0)
        b_inter.append(it)
    for sy in systems:
        sy.close()

    def fifo(rate):
        reqs = ic.request_stream(wl["n"], rate, n_lo=wl["n_lo"], n_hi=wl["n_hi"],
                                 t_span=wl["t_span"])
        fin, lat = 0.0, []
        for q, sv in zip(reqs, service):
            fin = max(q.arrival, fin) + sv
            lat.append(fin - q.arrival)
        out = {"throughput": sum(b_inter) / (fin - reqs[0].arrival) / 1e9,
               "makespan_s": fin - reqs[0].arrival, "latency": _lat(lat)}
        for kind in ("force", "evolve"):
            xs = [x for x, q in zip(lat, reqs) if q.kind == kind]
            if xs:
                out["latency_" + kind] = _lat(xs)
        return out

    for row in sweep:
        row["one_request_per_launch"] = fifo(row["rate_hz"])
    sat = {"rate_hz": wl["rates"][-1], "frac_of_saturation": None, "server": timed[-1],
           "one_request_per_launch": fifo(wl["rates"][-1]), "saturation_rate_hz": r_sat}
    sweep.append(sat)
    srv_stats = {k: st1[k] - st0[k] for k in ("ticks", "force_launches", "interactions",
                                               "busy_s", "completed", "kernel_launches")}
    props = torch.cuda.get_device_properties(local)
    sm_max = float(measured_peaks().get("sm_max_mhz") or 2070.0)
    peak = fp32_peak_tflops(props.multi_processor_count, sm_max)
    inter = sum(t["interactions"] for t in timed)
    secs = sum(t["makespan_s"] for t in timed)
    value = inter / secs / 1e9
    h2d = sum(8 * 7 * r.n for r in base)
    d2h = sum(8 * (7 if r.kind == "force" else 6) * r.n for r in base)
    line = {
        "metric": METRIC + "; p50/p99 request latency", "value": value, "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded galaxies with a central point mass, N-body units)",
        "config": {"workload": args.workload, "requests": wl["n"], "n_range": [wl["n_lo"], wl["n_hi"]],
                   "t_span": wl["t_span"], "eta": wl["eta"], "dt_max": wl["dt_max"],
                   "variant": variant, "eps": "1/(4 N^(1/3)) per request", "desc": wl["desc"],
                   "max_inflight": 64, "budget_bytes": 64 << 30,
                   "l2": "working set of the stream (GBs) larger than L2",
                   "parallelism": "single GPU"},
        "latency": timed[-1]["latency"],
        "fp32_peak_frac": FLOPS_PER_INTERACTION * value * 1e9 / (peak * 1e12),
        "roofline": {"bound": "alu", "kernel": "k_force_items32 (batched pair force)",
                     "achieved": FLOPS_PER_INTERACTION * value * 1e9 / 1e12, "peak": peak,
                     "unit": "TFLOP/s", "frac": FLOPS_PER_INTERACTION * value * 1e9 / (peak * 1e12),
                     "traffic": None,
                     "note": "whole-loop throughput (makespan incl. host ticks), not the kernel alone",
                     "peak_source": "SMs x 128 x 2 x max SM clock %.0f MHz (derived)" % sm_max},
        "one_request_per_launch": sat["one_request_per_launch"],
        "sweep": sweep,
        "server_stats": srv_stats,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "note": "requests carry host arrays in and out: the request loop is end to end"},
        "gpu_launches": None,
        "clocks": clocks,
    }
    line["gpu_launches"] = int(srv_stats["kernel_launches"])
    if world == 1 and not args.no_cpu_baseline:
        import oracle
        t0 = time.perf_counter()
        inter_c, used = 0.0, 0
        for r, p, e in sorted(zip(base, parts, eps), key=lambda x: x[0].n):
            if r.kind != "force":
                continue
            oracle.force(p.m, p.pos, p.vel, e * e)
            inter_c += float(r.n) * r.n
            used += 1
            if time.perf_counter() - t0 > 10.0:
                break
        secs_c = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": inter_c / secs_c / 1e9, "unit": UNIT,
                                "cores": oracle.num_threads(), "kind": "oracle", "build": oracle.CFLAGS,
                                "sample": "oracle force on the %d smallest force requests" % used,
                                "seconds": secs_c}
    if rank == 0:
        emit(args, line)
    srv.close()
    dist.close()
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
