#!/usr/bin/env python
"""MD atom-steps/s of the Allegro energy+force path on GB300.

One step = neighbour-list rebuild (no skin) + energy + forces (forward pair
passes, FP64 energy reduction, hand-written adjoint) + FP64 velocity-Verlet
update + per-step >5 sigma outlier count, replayed as a captured CUDA graph.
Workloads (synthetic liquid ammonia at 0.68 g/cm^3, seeded Gaussian weights):
  fp32_6912   6,912 atoms (1,728 NH3), 2 layers, l_max 2, 16 channels,
              latent [128, 128], energy [32], r_cut 5 A, dt 0.25 fs, FP32 path.
Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
the host cores on a bounded sample of the same workload.
Multi-GPU: independent replicas, one per rank (no data-path collective).
"""
import argparse
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
sys.path.insert(0, ROOT)

KB_T200 = 8.617333e-5 * 200.0
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x FMA x max clock

# Algorithmic multiply-adds per pair of each pass for the 2-layer l_max 2
# model (D 128, C 16, E 32; 11 coupling paths, 83 CG terms per channel).  Each
# model operation is counted once forward and once in its adjoint (input
# gradients only); the forward recomputed inside the adjoint passes is not.
ALG_MAC_PER_PAIR = {
    "pass_a": 1536 + 16384 + 2048 + 144,                        # two-body, env1, scatter
    "pass_b": 6144 + 1328 + 8960 + 22528 + 16384 + 2048 + 144,  # embed, TP, mix, latent, env2
    "pass_c": (144 + 22528 + 16384 + 4096 + 32) * 2,            # layer 2 + energy, fwd + adjoint
    "pass_b_adjoint": 288 + 2048 + 16384 + 22528 + 8960 + 2656 + 6144 + 288,
    "pass_a_adjoint": 288 + 2048 + 16384 + 1536,
}

WORKLOADS = {
    "fp32_6912": dict(n_mol=1728, precision=0, dt=0.25, model="main", dtype="f32"),
    "bf16_110592": dict(n_mol=27648, precision=1, dt=0.25, model="main", dtype="bf16"),
    "bf16_6912": dict(n_mol=1728, precision=1, dt=0.25, model="main", dtype="bf16"),
}


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _energy_scale(name):
    with open(os.path.join(ROOT, "tests", "golden", "energy_scale.json")) as f:
        return json.load(f)[name]["sigma"]


def _workload(name):
    import synth
    w = WORKLOADS[name]
    cfg = synth.MAIN if w["model"] == "main" else synth.TINY
    blob = synth.make_blob(cfg, 42, sigma=_energy_scale(w["model"]))
    pos, sp, cell = synth.make_ammonia(w["n_mol"], 0)
    vel = synth.make_velocities(sp, 200.0, 1)
    return w, cfg, blob, pos, sp, cell, vel


def cpu_baseline(name, max_seconds=30.0):
    """FP64 oracle on the host cores: velocity-Verlet steps of the full
    workload until max_seconds of CPU work (at least one step)."""
    import torch
    from oracle.md import velocity_verlet
    from oracle.model import OracleModel
    torch.set_num_threads(os.cpu_count() or 1)
    w, cfg, blob, pos, sp, cell, vel = _workload(name)
    orc = OracleModel(blob)
    L = np.diag(cell)
    import synth
    f = lambda p: orc.energy_forces(p, sp, L)[:2]      # noqa: E731
    t0 = time.perf_counter()
    f(pos)                                               # initial forces (not counted)
    t1 = time.perf_counter()
    steps = max(1, int(max_seconds // max(t1 - t0, 1e-3)) - 1)
    steps = min(steps, 3)
    t2 = time.perf_counter()
    velocity_verlet(f, pos, vel, synth.MASS_AMU[sp], L, w["dt"], steps)
    t3 = time.perf_counter()
    # velocity_verlet evaluates forces once up front and once per step
    per_step = (t3 - t2) / (steps + 1)
    return {"value": len(sp) / per_step, "unit": "atom-steps/s", "cores": torch.get_num_threads(),
            "kind": "oracle",
            "sample": f"{steps} FP64 velocity-Verlet step(s) of the full {len(sp)}-atom workload "
                      f"(torch-CPU float64 + autograd forces), {per_step:.2f} s/step"}


def run_reference(args):
    """The FP64 oracle as the reference arm, on the host cores."""
    rank = _env_int("RANK", 0)
    if rank != 0:
        return 0
    import torch
    from oracle.md import velocity_verlet
    from oracle.model import OracleModel
    import synth
    torch.set_num_threads(os.cpu_count() or 1)
    w, cfg, blob, _, _, _, _ = _workload(args.config)
    # bounded sample: 432 atoms (108 NH3) of the same generator and density
    pos, sp, cell = synth.make_ammonia(108, 0)
    vel = synth.make_velocities(sp, 200.0, 1)
    L = np.diag(cell)
    orc = OracleModel(blob)
    f = lambda p: orc.energy_forces(p, sp, L)[:2]      # noqa: E731
    state = velocity_verlet(f, pos, vel, synth.MASS_AMU[sp], L, w["dt"], max(args.warmup, 1))
    t0 = time.perf_counter()
    velocity_verlet(f, state["pos"], state["vel"], synth.MASS_AMU[sp], L, w["dt"], 1)
    est = time.perf_counter() - t0
    steps = int(min(args.steps, max(3, 150.0 // max(est, 1e-3))))
    t0 = time.perf_counter()
    velocity_verlet(f, state["pos"], state["vel"], synth.MASS_AMU[sp], L, w["dt"], steps)
    el = time.perf_counter() - t0
    value = len(sp) * steps / el
    line = {
        "impl": "reference", "metric": "MD atom-steps/s on 1 GB300 (E+F)", "value": value,
        "unit": "atom-steps/s", "n_gpus": 0, "steps": steps, "steps_requested": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * el / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.config, "sample_atoms": len(sp)},
        "cpu_baseline": {"value": value, "unit": "atom-steps/s", "cores": torch.get_num_threads(),
                         "kind": "oracle",
                         "sample": f"{steps} FP64 velocity-Verlet steps of a {len(sp)}-atom sample "
                                   f"(same generator, density and model)"},
        "e2e": {"value": value, "unit": "atom-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    import paper_2303_08169_gb300 as al

    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local = _env_int("LOCAL_RANK", 0)
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w, cfg, blob, pos, sp, cell, vel = _workload(args.config)
    N = len(sp)
    ctx = al.allegro_create(blob, np.array([14.007, 1.008]), cfg.r_cut, cfg.l_max, cfg.n_layers)
    stream = torch.cuda.Stream(device=dev)
    al.allegro_set_stream(ctx, stream)
    al.allegro_set_md_precision(ctx, w["precision"])
    pos_d = torch.tensor(pos, device=dev)
    vel_d = torch.tensor(vel, device=dev)
    sp_d = torch.tensor(sp, device=dev, dtype=torch.int32)
    al.allegro_md_init(ctx, pos_d, vel_d, sp_d, cell)
    K, W = args.steps, args.warmup
    outl = torch.zeros(K, dtype=torch.int64, device=dev)
    ener = torch.zeros((K, 3), dtype=torch.float64, device=dev)
    al.allegro_md_step_nve(ctx, w["dt"], W)                 # graph capture + warm-up
    n_pairs = al.allegro_query(ctx, al.ALLEGRO_Q_N_PAIRS)
    step_kernels = al.allegro_query(ctx, al.ALLEGRO_Q_STEP_KERNELS)
    clocks = ClockSampler(local)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    al.allegro_md_step_nve(ctx, w["dt"], K, outl, ener)
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    if dist:
        t = torch.tensor([ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    en = ener.cpu().numpy()
    drift = float(np.abs(en[:, 2] - en[0, 2]).max() / (N * KB_T200))
    outliers = outl.cpu().numpy()

    # per-kernel device times (CUDA events on the library stream) at the final state
    phases = al.allegro_phase_times(ctx, 20)
    dom = max(ALG_MAC_PER_PAIR, key=lambda k: phases[k])
    achieved = 2.0 * ALG_MAC_PER_PAIR[dom] * n_pairs / (phases[dom] * 1e-3) / 1e12

    # end to end: energy+forces through the C ABI from pinned host positions to
    # pinned host forces (H2D + rebuild + passes + D2H inside the timed region)
    pos_h = torch.tensor(pos, dtype=torch.float64).pin_memory()
    F_h = torch.empty((N, 3), dtype=torch.float32).pin_memory()
    for _ in range(3):
        al.allegro_energy_forces(ctx, pos_h, sp_d, cell, F_h, None, w["precision"])
    n_e2e = max(10, min(K, 200))
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(n_e2e):
        al.allegro_energy_forces(ctx, pos_h, sp_d, cell, F_h, None, w["precision"])
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / n_e2e

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.config)
    al.allegro_destroy(ctx)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    line = {
        "metric": "MD atom-steps/s on 1 GB300 (E+F), BF16 vs FP32 path at stated force error",
        "value": world * N * K / (ms * 1e-3),
        "unit": "atom-steps/s",
        "n_gpus": world,
        "steps": K,
        "warmup": W,
        "ms_per_step": ms / K,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": w["dtype"],
        "data": "synthetic",
        "config": {"workload": args.config, "atoms": N, "pairs": n_pairs, "dt_fs": w["dt"],
                   "l2": "working set above L2 (per-pair state ~1 GB per step)",
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": N / (e2e_ms * 1e-3), "unit": "atom-steps/s",
                "h2d_bytes_per_step": 24 * N, "d2h_bytes_per_step": 12 * N + 8,
                "note": "allegro_energy_forces with pinned host positions in and host forces out"},
        "gpu_launches": int(step_kernels * K),
        "roofline": {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": FP32_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS, "traffic": None,
                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"},
        "phases_ms": phases,
        "physics": {"energy_drift_over_NkT": drift, "outliers_last": int(outliers[-1]),
                    "outliers_max": int(outliers.max())},
        "clocks": clk,
    }
    if cpu:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="fp32_6912", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
