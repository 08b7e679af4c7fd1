#!/usr/bin/env python
"""MD atom-steps/s of the Allegro energy+force path on GB300.

One step = neighbour-list rebuild (no skin) + energy + forces (forward pair
passes, FP64 energy reduction, hand-written adjoint) + FP64 velocity-Verlet
update + per-step >5 sigma outlier count, replayed as a captured CUDA graph.
Synthetic liquid ammonia at 0.68 g/cm^3 and seeded Gaussian weights of the
2-layer, l_max 2, 16-channel, latent [128, 128], energy [32], r_cut 5 A model;
dt 0.25 fs from 200 K.  Workloads:
  tc_110592    110,592 atoms (27,648 NH3), tensor-core path, FP16 operands
               with split (hi + lo) two-body and energy-hidden GEMMs: the
               mixed-precision mode that meets the 2e-3 eV/A force bound
               (headline, the default)
  bf16_110592  same, BF16 operands throughout
  fp16_110592  same, FP16 operands throughout
  fp32_6912    6,912 atoms (1,728 NH3), every per-pair GEMM in FP32
  tc_1000000   10^6 atoms (250,000 NH3, edge 218 A, ~5.2e7 pairs, per-pair
               arrays at the tensor-core width), FP16_SPLIT, 200 steps
Prints one JSON line (rank 0): the headline workload timed over --steps, the
other paths timed over min(--steps, 200) steps under "paths", each path's
force error against the FP64 oracle (on the 6,912-atom cell; for the 10^6-atom
configuration on sampled atoms of its own frame), per-kernel device times and
the roofline of the dominant kernel.  --impl reference
times the FP64 CPU oracle on the host cores on a bounded sample.
Multi-GPU: independent replicas, one per rank (no data-path collective).
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MD atom-steps/s on 1 GB300 (E+F), BF16 vs FP32 path at stated force error"
KB_T200 = 8.617333e-5 * 200.0
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x FMA x max clock
FORCE_BOUND = 2e-3                                   # eV/A, max |dF| of the mixed-precision path

# Algorithmic multiply-adds per pair of each pass kernel for the 2-layer
# l_max 2 model (D 128, C 16, E 32; 11 coupling paths, 83 CG terms per
# channel).  Each model operation is counted once forward and once in its
# adjoint (input gradients only); forward work recomputed inside an adjoint
# kernel is not counted.
#   GEMM: per-pair dense products (tensor cores on the tensor-core path)
GEMM_MAC_PER_PAIR = {
    "pass_a": 1536 + 16384 + 2048,                        # two-body 12->128->128, env1 128->16
    "pass_b1": 6144 + 8960,                               # embedding 128->48, mixing
    "pass_b2": 22528 + 16384 + 2048,                      # latent 176->128->128, env2
    "pass_c": 2 * (22528 + 16384 + 4096),                 # latent + energy hidden, fwd + adjoint
    "pass_b_adjoint": 2048 + 16384 + 22528 + 8960 + 6144,    # env, latent, mixing, embedding adjoints
    "pass_a_adjoint": 2048 + 16384 + 1536,
}
#   all multiply-adds incl. tensor products, scatters, energy output (FP32 path)
ALL_MAC_PER_PAIR = {
    "pass_a": 1536 + 16384 + 2048 + 144,
    "pass_b": 6144 + 1328 + 8960 + 22528 + 16384 + 2048 + 144,
    "pass_c": (144 + 22528 + 16384 + 4096 + 32) * 2,
    "pass_b_adjoint": 288 + 2048 + 16384 + 22528 + 8960 + 2656 + 6144 + 288,
    "pass_a_adjoint": 288 + 2048 + 16384 + 1536,
}
# one E + F of the FP32 path (all of the above), and the multiply-adds of the
# per-pair weight layers (two-body, embedding, env, mixing, latent, energy
# hidden and output): one outer product dz (x) x per layer and pair in a
# weight-gradient reduction
FP32_MAC_PER_PAIR = sum(ALL_MAC_PER_PAIR.values())
WEIGHT_MAC_PER_PAIR = 1536 + 16384 + 6144 + 2 * 2048 + 8960 + 2 * (22528 + 16384) + 4096 + 32
TC_KERNELS = {"pass_a": "k_bf_a", "pass_b1": "k_bf_b1", "pass_b2": "k_bf_b2", "pass_c": "k_bf_c",
              "pass_b_adjoint": "k_bf_bt", "pass_a_adjoint": "k_bf_at"}
FP32_KERNELS = {"pass_a": "k_pass_a", "pass_b": "k_pass_b", "pass_c": "k_pass_c",
                "pass_b_adjoint": "k_pass_b_bwd", "pass_a_adjoint": "k_pass_a_bwd"}

WORKLOADS = {
    "tc_110592": dict(n_mol=27648, precision=3, dt=0.25,
                      dtype="f16 operands (two-body and energy-hidden GEMMs split hi+lo), f32 accumulate"),
    "bf16_110592": dict(n_mol=27648, precision=1, dt=0.25, dtype="bf16 operands, f32 accumulate"),
    "fp16_110592": dict(n_mol=27648, precision=2, dt=0.25, dtype="f16 operands, f32 accumulate"),
    "fp32_6912": dict(n_mol=1728, precision=0, dt=0.25, dtype="f32"),
    "tc_6912": dict(n_mol=1728, precision=3, dt=0.25,
                    dtype="f16 operands (two-body and energy-hidden GEMMs split hi+lo), f32 accumulate"),
    "tc_1000000": dict(n_mol=250000, precision=3, dt=0.25,
                       dtype="f16 operands (two-body and energy-hidden GEMMs split hi+lo), f32 accumulate"),
}
SECONDARY = ["bf16_110592", "fp16_110592", "fp32_6912"]
SCALE = "tc_1000000"   # own context, run after the others
SCALE_SAMPLES = 16      # atoms of the 10^6-atom frame checked against the oracle
SKIN = 0.3              # A, the Verlet-skin block
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "tc_110592_kernels.md")


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def max_over_ranks(ms, dist=None, device="cpu"):
    """The job's time: the slowest rank's elapsed milliseconds."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, atoms, steps, ms):
    """Whole-job atom-steps/s: every rank advances its own replica of `atoms`
    atoms by `steps` steps in the job time `ms` (weak scaling)."""
    return world * atoms * steps / (ms * 1e-3)


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


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


def _model():
    import synth
    cfg = synth.MAIN
    return cfg, synth.make_blob(cfg, 42, sigma=_energy_scale("main"))


def _system(n_mol):
    import synth
    pos, sp, cell = synth.make_ammonia(n_mol, 0)
    vel = synth.make_velocities(sp, 200.0, 1)
    return pos, sp, cell, vel


def _kernel_source_hash():
    h = hashlib.sha256()
    with open(os.path.join(ROOT, "paper_2303_08169_gb300", "csrc", "model_bf16.cu"), "rb") as f:
        h.update(f.read())
    return h.hexdigest()[:16]


def _profile_traffic(kernel):
    """DRAM bytes per pair of one kernel from the committed ncu summary, or
    None when the summary is missing or the kernel source changed since."""
    try:
        text = open(PROFILE_SUMMARY).read()
    except OSError:
        return None
    m = re.search(r"source_sha256_16:\s*([0-9a-f]+)", text)
    if not m or m.group(1) != _kernel_source_hash():
        return None
    m = re.search(rf"dram_bytes_per_pair\.{kernel}:\s*([0-9.eE+-]+)", text)
    return float(m.group(1)) if m else None


# ---------------------------------------------------------------------------
def cpu_baseline(max_seconds=30.0):
    """FP64 oracle on the host cores: velocity-Verlet steps of the 6,912-atom
    cell of the same generator until max_seconds of CPU work (1 to 3 steps).
    Also returns the oracle forces at the initial positions."""
    import torch
    import synth
    from oracle.md import velocity_verlet
    from oracle.model import OracleModel
    torch.set_num_threads(os.cpu_count() or 1)
    cfg, blob = _model()
    pos, sp, cell, vel = _system(1728)
    orc = OracleModel(blob)
    L = np.diag(cell)
    f = lambda p: orc.energy_forces(p, sp, L)[:2]      # noqa: E731
    t0 = time.perf_counter()
    E0, F0 = f(pos)                                      # initial forces (not counted)
    t1 = time.perf_counter()
    steps = min(3, max(1, int(max_seconds // max(t1 - t0, 1e-3)) - 1))
    t2 = time.perf_counter()
    velocity_verlet(f, pos, vel, synth.MASS_AMU[sp], L, 0.25, steps)
    t3 = time.perf_counter()
    per_step = (t3 - t2) / (steps + 1)                  # one force call up front + one per step
    base = {"value": len(sp) / per_step, "unit": "atom-steps/s", "cores": torch.get_num_threads(),
            "kind": "oracle",
            "sample": f"{steps} FP64 velocity-Verlet step(s) of the {len(sp)}-atom cell of the same "
                      f"generator and model (torch-CPU float64 + autograd forces), {per_step:.2f} s/step"}
    return base, (pos, sp, cell, E0, F0)


def oracle_local_forces(pos, sp, cell, idx):
    """FP64 oracle forces of the atoms idx of a large frame, each from its
    2 r_cut neighbourhood (the CPU-oracle leg, for the accuracy check of the
    10^6-atom configuration)."""
    from oracle.model import OracleModel
    _, blob = _model()
    orc = OracleModel(blob)
    return np.array([orc.local_energy_force(pos, sp, np.diag(cell), int(k))[1] for k in idx])


def run_reference(args):
    """The FP64 oracle as the reference arm, on the host cores."""
    rank = _env_int("RANK", 0)
    if rank != 0:
        return 0
    import torch
    import synth
    from oracle.md import velocity_verlet
    from oracle.model import OracleModel
    torch.set_num_threads(os.cpu_count() or 1)
    w = WORKLOADS[args.config]
    cfg, blob = _model()
    # bounded sample: 432 atoms (108 NH3) of the same generator, density and model
    pos, sp, cell, vel = _system(108)
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
        "impl": "reference", "metric": METRIC, "value": value,
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


# ---------------------------------------------------------------------------
class Runner:
    def __init__(self, al, torch, dev, blob, cfg):
        self.al, self.torch, self.dev = al, torch, dev
        self.ctx = al.allegro_create(blob, np.array([14.007, 1.008]), cfg.r_cut, cfg.l_max, cfg.n_layers)
        self.stream = torch.cuda.Stream(device=dev)
        al.allegro_set_stream(self.ctx, self.stream)

    def md(self, name, K, W, clocks=None, barrier=None, skin=0.0):
        """K graph-captured MD steps after W warm-up steps; returns a dict."""
        al, torch, dev = self.al, self.torch, self.dev
        w = WORKLOADS[name]
        pos, sp, cell, vel = _system(w["n_mol"])
        al.allegro_set_md_precision(self.ctx, w["precision"])
        al.allegro_set_skin(self.ctx, skin)
        al.allegro_md_init(self.ctx, torch.tensor(pos, device=dev), torch.tensor(vel, device=dev),
                           torch.tensor(sp, device=dev, dtype=torch.int32), cell)
        outl = torch.zeros(K, dtype=torch.int64, device=dev)
        ener = torch.zeros((K, 3), dtype=torch.float64, device=dev)
        al.allegro_md_step_nve(self.ctx, w["dt"], W)        # graph capture + warm-up
        n_pairs_start = al.allegro_query(self.ctx, al.ALLEGRO_Q_N_PAIRS)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        if clocks:
            clocks.start()
            time.sleep(0.3)
        if barrier:
            barrier()
        torch.cuda.synchronize()
        ev0.record(self.stream)
        al.allegro_md_step_nve(self.ctx, w["dt"], K, outl, ener)
        ev1.record(self.stream)
        torch.cuda.synchronize()
        if barrier:
            barrier()
        clk = clocks.stop() if clocks else None
        ms = ev0.elapsed_time(ev1)
        en = ener.cpu().numpy()
        N = len(sp)
        return {"ms": ms, "N": N, "K": K, "clocks": clk, "n_pairs_start": n_pairs_start,
                "rebuilds": al.allegro_query(self.ctx, al.ALLEGRO_Q_REBUILDS),
                "n_pairs": al.allegro_query(self.ctx, al.ALLEGRO_Q_N_PAIRS),
                "step_kernels": al.allegro_query(self.ctx, al.ALLEGRO_Q_STEP_KERNELS),
                "drift": float(np.abs(en[:, 2] - en[0, 2]).max() / (N * KB_T200)),
                "outliers_last": int(outl[-1].item()), "outliers_max": int(outl.max().item()),
                "pos": pos, "sp": sp, "cell": cell}

    def nvt(self, name, K, W, temperature=200.0, tau=100.0):
        """K graph-captured Nose-Hoover NVT steps after W warm-up steps, from
        the workload's 200 K start; returns ms, pairs and the drift of the
        conserved extended energy."""
        al, torch, dev = self.al, self.torch, self.dev
        w = WORKLOADS[name]
        pos, sp, cell, vel = _system(w["n_mol"])
        al.allegro_set_md_precision(self.ctx, w["precision"])
        al.allegro_md_init(self.ctx, torch.tensor(pos, device=dev), torch.tensor(vel, device=dev),
                           torch.tensor(sp, device=dev, dtype=torch.int32), cell)
        ener = torch.zeros((K, 4), dtype=torch.float64, device=dev)
        al.allegro_md_step_nvt(self.ctx, w["dt"], W, temperature, tau)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(self.stream)
        al.allegro_md_step_nvt(self.ctx, w["dt"], K, temperature, tau, None, ener)
        ev1.record(self.stream)
        torch.cuda.synchronize()
        en = ener.cpu().numpy()
        N = len(sp)
        return {"ms": ev0.elapsed_time(ev1), "N": N, "K": K,
                "n_pairs": al.allegro_query(self.ctx, al.ALLEGRO_Q_N_PAIRS),
                "H_drift_over_NkT": float(np.abs(en[:, 3] - en[0, 3]).max() / (N * KB_T200)),
                "T_end_K": float(2.0 * en[-1, 1] / (3 * N * 8.617333262e-5))}

    def pimd(self, name, K, W, n_beads=32, temperature=200.0):
        """K ring-polymer MD steps (Sec. 6: 32 replicas per atom) of the
        workload's atom count split into n_beads replicas of N / n_beads
        atoms (same density, model and precision): every step evaluates all
        replicas in one pass sequence.  Returns ms and the H_P drift."""
        import synth
        al, torch, dev = self.al, self.torch, self.dev
        w = WORKLOADS[name]
        pos, sp, cell, _ = _system(w["n_mol"] // n_beads)
        rng = np.random.default_rng(11)
        q = pos[None] + 0.03 * rng.normal(size=(n_beads,) + pos.shape)
        v = np.stack([synth.make_velocities(sp, temperature, 100 + k) for k in range(n_beads)])
        al.allegro_set_md_precision(self.ctx, w["precision"])
        al.allegro_pimd_init(self.ctx, torch.tensor(q, device=dev), torch.tensor(v, device=dev),
                             torch.tensor(sp, device=dev, dtype=torch.int32), cell, temperature)
        ener = torch.zeros((K, 3), dtype=torch.float64, device=dev)
        al.allegro_pimd_step(self.ctx, w["dt"], W)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(self.stream)
        al.allegro_pimd_step(self.ctx, w["dt"], K, ener)
        ev1.record(self.stream)
        torch.cuda.synchronize()
        en = ener.cpu().numpy()
        N = n_beads * len(sp)
        return {"ms": ev0.elapsed_time(ev1), "N": N, "K": K, "beads": n_beads, "atoms_per_replica": len(sp),
                "n_pairs": al.allegro_query(self.ctx, al.ALLEGRO_Q_N_PAIRS),
                "step_kernels": al.allegro_query(self.ctx, al.ALLEGRO_Q_RP_STEP_KERNELS),
                "HP_drift_over_NkT": float(np.abs(en[:, 2] - en[0, 2]).max() / (N * KB_T200))}

    def phases(self, n_reps=20):
        """Per-kernel device times at the current MD state (CUDA events on
        the library stream) and the pair count of that state."""
        ph = self.al.allegro_phase_times(self.ctx, n_reps)
        return ph, self.al.allegro_query(self.ctx, self.al.ALLEGRO_Q_N_PAIRS)

    def forces(self, pos, sp, cell, precision):
        al, torch, dev = self.al, self.torch, self.dev
        F = torch.empty((len(pos), 3), dtype=torch.float32, device=dev)
        E = al.allegro_energy_forces(self.ctx, torch.tensor(pos, device=dev),
                                     torch.tensor(sp, device=dev, dtype=torch.int32), cell, F, None, precision)
        return E, F.cpu().numpy().astype(np.float64)

    def e2e(self, name, n_iter):
        """energy+forces through the C ABI from pinned host positions to
        pinned host forces, wall-clock per call (H2D, rebuild, passes, D2H)."""
        al, torch = self.al, self.torch
        w = WORKLOADS[name]
        pos, sp, cell, _ = _system(w["n_mol"])
        pos_h = torch.tensor(pos, dtype=torch.float64).pin_memory()
        sp_h = torch.tensor(sp, dtype=torch.int32).pin_memory()
        F_h = torch.empty((len(sp), 3), dtype=torch.float32).pin_memory()
        for _ in range(3):
            al.allegro_energy_forces(self.ctx, pos_h, sp_h, cell, F_h, None, w["precision"])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n_iter):
            al.allegro_energy_forces(self.ctx, pos_h, sp_h, cell, F_h, None, w["precision"])
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / n_iter
        return {"value": len(sp) / dt, "unit": "atom-steps/s",
                "h2d_bytes_per_step": 24 * len(sp) + 4 * len(sp), "d2h_bytes_per_step": 12 * len(sp) + 8,
                "ms_per_call": 1e3 * dt,
                "note": "allegro_energy_forces (one E+F step) with pinned host positions and species in "
                        "and host forces and energy out, wall clock"}

    def close(self):
        self.al.allegro_destroy(self.ctx)


def lmax_sweep(al, torch, dev, K=10, W=3, n_mol=27648):
    """Time per MD step (E+F, graph-captured NVE step) of the main model's
    widths at l_max 0, 1 and 2 on the 110,592-atom system, in the split
    tensor-core mode (the headline precision) and on the FP32 passes: the
    shape of the paper's Table 2 (395 : 916 : 2,580 ms for l = 0 : 1 : 2 on
    its own platform and system)."""
    import synth
    pos, sp, cell, vel = _system(n_mol)
    out = {"l_max": [], "ms_per_step": [], "ms_per_step_fp32": [], "pairs": [], "params": []}
    for lmax in (0, 1, 2):
        M = synth.MAIN
        cfg = synth.ModelConfig(r_cut=M.r_cut, l_max=lmax, n_layers=M.n_layers, n_channels=M.n_channels,
                                latent=M.latent, energy=M.energy, avg_num_neighbors=M.avg_num_neighbors)
        blob = synth.make_blob(cfg, 42, sigma=_energy_scale("main"))
        run = Runner(al, torch, dev, blob, cfg)
        times = {}
        for prec in (al.ALLEGRO_FP16_SPLIT, al.ALLEGRO_FP32):
            al.allegro_set_md_precision(run.ctx, prec)
            al.allegro_md_init(run.ctx, torch.tensor(pos, device=dev), torch.tensor(vel, device=dev),
                               torch.tensor(sp, device=dev, dtype=torch.int32), cell)
            al.allegro_md_step_nve(run.ctx, 0.25, W)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            ev0.record(run.stream)
            al.allegro_md_step_nve(run.ctx, 0.25, K)
            ev1.record(run.stream)
            torch.cuda.synchronize()
            times[prec] = ev0.elapsed_time(ev1) / K
            if prec == al.ALLEGRO_FP16_SPLIT:
                out["pairs"].append(al.allegro_query(run.ctx, al.ALLEGRO_Q_N_PAIRS))
        out["l_max"].append(lmax)
        out["ms_per_step"].append(times[al.ALLEGRO_FP16_SPLIT])
        out["ms_per_step_fp32"].append(times[al.ALLEGRO_FP32])
        out["params"].append(al.allegro_query(run.ctx, al.ALLEGRO_Q_N_PARAMS))
        run.close()
    t0 = out["ms_per_step"][0]
    out["ratio_to_l0"] = [t / t0 for t in out["ms_per_step"]]
    out["ratio_to_l0_fp32"] = [t / out["ms_per_step_fp32"][0] for t in out["ms_per_step_fp32"]]
    out["paper_ratio_to_l0"] = [1.0, 916.0 / 395.0, 2580.0 / 395.0]
    out["atoms"] = len(sp)
    out["steps"] = K
    out["note"] = ("ms_per_step: FP16_SPLIT tensor-core passes; ms_per_step_fp32: FP32 pair passes; main model "
                   "widths (16 channels, latent [128, 128]), 2 layers; pairs at the start of the split-mode run")
    return out


def sam_timing(al, torch, steps=5, n_sharp=64):
    """SAM training step (Eq. 3) on 32 seeded ammonia structures of 64-512
    atoms; targets from a teacher model (weights seed 43) evaluated by the
    library's FP32 path.  Wall clock per allegro_sam_train_step."""
    import synth
    cfg = synth.MAIN
    teacher = synth.make_blob(cfg, 43, sigma=_energy_scale("main_teacher"))
    _, student = _model()
    batch = synth.make_sam_batch()
    tctx = al.allegro_create(teacher, np.array([14.007, 1.008]), cfg.r_cut, cfg.l_max, cfg.n_layers)
    structs = []
    for pos, sp, cell in batch:
        F = np.zeros((len(sp), 3), np.float32)
        E = al.allegro_energy_forces(tctx, pos, sp.astype(np.int32), cell, F)
        structs.append(dict(pos=pos, species=sp, cell=cell, e_target=E, f_target=F))
    al.allegro_destroy(tctx)
    ctx = al.allegro_create(student, np.array([14.007, 1.008]), cfg.r_cut, cfg.l_max, cfg.n_layers)
    b, keep = al.make_batch(structs)
    losses = [al.allegro_sam_train_step(ctx, b, 0.05, 2e-3, 1.0, 100.0)]     # warm-up (allocations)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        losses.append(al.allegro_sam_train_step(ctx, b, 0.05, 2e-3, 1.0, 100.0))
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    # sharpness of the trained weights (Eq. 2, estimated as in Sec. 5.4 by the
    # largest loss increase over random eps of norm rho = 0.05; 64 seeded
    # samples here instead of the paper's 1,000) and its 1-D surface
    n_par = al.allegro_query(ctx, al.ALLEGRO_Q_N_PARAMS)
    gen = torch.Generator(device="cuda").manual_seed(11)
    eps = torch.randn((n_sharp, n_par), generator=gen, device="cuda", dtype=torch.float32)
    eps = eps * (0.05 / eps.norm(dim=1, keepdim=True))
    eps = torch.cat([torch.zeros((1, n_par), device="cuda", dtype=torch.float32), eps])
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    ls = al.allegro_loss_scan(ctx, b, eps, np.ones(n_sharp + 1))
    dt_scan = (time.perf_counter() - t1) / (n_sharp + 1)
    kmax = int(np.argmax(ls[1:])) + 1
    surface = al.allegro_loss_scan(ctx, b, eps[kmax], np.linspace(-1.0, 1.0, 9))
    n_pairs = al.allegro_query(ctx, al.ALLEGRO_Q_BATCH_PAIRS)
    launch = {name: [(al.allegro_query(ctx, key) >> (4 * q)) & 15 for q in range(5)]
              for name, key in (("value_passes", al.ALLEGRO_Q_FP32_LAUNCH),
                                ("tangent_passes", al.ALLEGRO_Q_TANGENT_LAUNCH))}
    al.allegro_destroy(ctx)
    n_atoms = int(sum(len(s["species"]) for s in structs))
    # algorithmic work of one SAM step: two loss gradients, each the forward
    # E + F (forward and force adjoint) and the tangent of both along dL/dF
    # (twice their multiply-adds: value and tangent) on the FP32 pass kernels,
    # and the weight-gradient reductions (two outer products per linear layer
    # and pair), which run on the tensor cores (BF16 x 3 split operands) except
    # the mixing matrices'.  The fraction below counts the FP32 pass work only
    # against the FP32 FMA peak, over the whole step's time.
    flops_fp32 = 2 * n_pairs * 2 * (3 * FP32_MAC_PER_PAIR)
    flops_wgrad = 2 * n_pairs * 2 * (2 * WEIGHT_MAC_PER_PAIR)
    peak = FP32_PEAK_TFLOPS
    sam_roof = {"bound": "alu", "achieved": flops_fp32 / dt * 1e-12, "peak": peak, "unit": "TFLOP/s",
                "frac": flops_fp32 / dt * 1e-12 / peak, "algorithmic_flops": flops_fp32,
                "weight_gradient_flops_on_tensor_cores": flops_wgrad, "pairs": n_pairs,
                "peak_source": "FP32 FMA: 152 SMs x 128 lanes x 2 FLOP x 2.07 GHz (derived)"}
    return {"structures": len(structs), "atoms": n_atoms, "pairs": n_pairs, "ms_per_step": 1e3 * dt,
            "steps": steps, "roofline": sam_roof,
            "fp32_launch_waves": dict(launch, order=["A", "B", "C", "B^T", "A^T"],
                                      note="waves of one block per SM per pass, chosen by the library's autotuner"),
            "rho": 0.05, "lr": 2e-3, "loss_first": losses[0], "loss_last": losses[-1],
            "sharpness": {"value": float(ls[1:].max() - ls[0]), "samples": n_sharp, "loss_at_w": float(ls[0]),
                          "ms_per_loss_evaluation": 1e3 * dt_scan,
                          "surface_p": [-1.0, -0.75, -0.5, -0.25, 0.0, 0.25, 0.5, 0.75, 1.0],
                          "surface_loss": [float(x) for x in surface],
                          "note": "allegro_loss_scan after the SAM steps: loss at w + eps_k for random eps_k "
                                  "of norm 0.05 (seeded), then L(w + p eps_max)"},
            "note": "all 32 structures in one concatenated pair list; two loss gradients (w, w + eps) "
                    "per step, each one FP32 forward pass sequence and one tangent pass sequence (the "
                    "hand-written adjoint differentiated along dL/dF: the exact force-term gradient) "
                    "with per-pair dumps, then deterministic weight-gradient reductions (tcgen05, BF16 x 3 "
                    "split operands, FP32 accumulation in TMEM, per-CTA partials added in a fixed order)"}


def roofline(phases, n_pairs, tensor_path, peaks):
    if tensor_path:
        times = {k: phases[k] for k in GEMM_MAC_PER_PAIR}
        dom = max(times, key=times.get)
        flops = 2.0 * GEMM_MAC_PER_PAIR[dom] * n_pairs
        peak = peaks.get("bf16_tflops")
        src = "measured bf16 dense burst (kind::f16 runs FP16 at the BF16 rate), MEASURED_PEAKS.json"
        if peak is None:
            peak, src = 1900.0, "fallback 1.9 PFLOP/s bf16 burst"
        traffic = _profile_traffic(TC_KERNELS[dom])
        traffic = None if traffic is None else traffic * n_pairs
        achieved = flops / (times[dom] * 1e-3) / 1e12
        return {"bound": "tensor", "kernel": TC_KERNELS[dom], "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                "algorithmic_flops_per_launch": flops, "launch_ms": times[dom], "peak_source": src,
                "frac_label": "of measured"}
    times = {k: phases[k] for k in ALL_MAC_PER_PAIR}
    dom = max(times, key=times.get)
    flops = 2.0 * ALL_MAC_PER_PAIR[dom] * n_pairs
    achieved = flops / (times[dom] * 1e-3) / 1e12
    return {"bound": "alu", "kernel": FP32_KERNELS[dom], "achieved": achieved, "peak": FP32_PEAK_TFLOPS,
            "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS, "traffic": None,
            "algorithmic_flops_per_launch": flops, "launch_ms": times[dom],
            "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz", "frac_label": "of derived"}


def roofline_step(phases, n_pairs, peaks):
    """Whole E+F of the tensor-core path: algorithmic GEMM FLOPs of all seven
    pass kernels over their summed device time (tensor view), and their DRAM
    bytes (committed ncu figures, when the source matches) over the same time
    (HBM view)."""
    t = sum(phases[k] for k in GEMM_MAC_PER_PAIR)
    flops = 2.0 * sum(GEMM_MAC_PER_PAIR.values()) * n_pairs
    peak = peaks.get("bf16_tflops", 1900.0)
    per = [_profile_traffic(TC_KERNELS[k]) for k in GEMM_MAC_PER_PAIR]
    traffic = None if any(x is None for x in per) else sum(per) * n_pairs
    hbm = peaks.get("hbm_gbs", 6800.0)
    out = {"kernels_ms": t, "algorithmic_flops": flops, "achieved_tflops": flops / (t * 1e-3) / 1e12,
           "peak_tflops": peak, "frac_tensor": flops / (t * 1e-3) / 1e12 / peak, "traffic": traffic}
    if traffic is not None:
        out["achieved_gbs"] = traffic / (t * 1e-3) / 1e9
        out["frac_hbm"] = out["achieved_gbs"] / hbm
    return out


def _guarded(block):
    """Run one of the blocks beside the headline; an exception there is
    reported in its place instead of taking the headline line with it."""
    try:
        return block()
    except Exception as e:      # noqa: BLE001 - any failure of an extra block is reported, not raised
        return {"error": f"{type(e).__name__}: {e}"}


def run_ours(args):
    import torch
    import paper_2303_08169_gb300 as al

    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local = _env_int("LOCAL_RANK", 0)
    dist = None
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    barrier = dist.barrier if dist else None
    cfg, blob = _model()
    run = Runner(al, torch, dev, blob, cfg)
    K, W = args.steps, args.warmup
    w = WORKLOADS[args.config]
    tensor_path = w["precision"] != 0

    head = run.md(args.config, K, W, ClockSampler(local), barrier)
    ms = max_over_ranks(head["ms"], dist, dev)
    phases, n_pairs_ph = run.phases()
    roof = roofline(phases, n_pairs_ph, tensor_path, _measured_peaks())
    roof_step = roofline_step(phases, n_pairs_ph, _measured_peaks()) if tensor_path else None

    paths = {}
    accuracy = {}
    cpu = None
    if not args.only_headline:
        e2e = run.e2e(args.config, max(10, min(K, 100)))
        K2 = min(K, 200)
        for name in [args.config] + [s for s in SECONDARY if s != args.config]:
            r = head if name == args.config else run.md(name, K2, W)
            paths[name] = {"value": r["N"] * r["K"] / (r["ms"] * 1e-3), "ms_per_step": r["ms"] / r["K"],
                           "atoms": r["N"], "pairs": r["n_pairs"], "steps": r["K"], "dtype": WORKLOADS[name]["dtype"]}

        def nvt_block():
            rn = run.nvt(args.config, min(K, 200), W)
            return {"workload": args.config, "value": rn["N"] * rn["K"] / (rn["ms"] * 1e-3),
                    "unit": "atom-steps/s", "ms_per_step": rn["ms"] / rn["K"], "steps": rn["K"],
                    "pairs": rn["n_pairs"], "temperature_K": 200.0, "tau_fs": 100.0,
                    "H_drift_over_NkT": rn["H_drift_over_NkT"], "T_end_K": rn["T_end_K"],
                    "note": "allegro_md_step_nvt: Nose-Hoover half steps around the same velocity-Verlet step"}

        def pimd_block():
            rp = run.pimd(args.config, min(K, 100), W)
            return {"workload": f"{rp['beads']} replicas x {rp['atoms_per_replica']} atoms ({rp['N']} bead-atoms)",
                    "value": rp["N"] * rp["K"] / (rp["ms"] * 1e-3), "unit": "bead-atom-steps/s",
                    "ms_per_step": rp["ms"] / rp["K"], "steps": rp["K"], "temperature_K": 200.0,
                    "HP_drift_over_NkT": rp["HP_drift_over_NkT"], "pairs": rp["n_pairs"],
                    "gpu_launches": int(rp["step_kernels"] * rp["K"]),
                    "note": "allegro_pimd_step: one CUDA graph per step (kicks, exact normal-mode spring "
                            "propagation, one neighbour build over all replicas, one pass sequence over all "
                            "replicas, record)"}

        def skin_block():
            rs = run.md(args.config, min(K, 200), W, skin=SKIN)
            run.md(args.config, 1, 1)                     # back to per-step rebuilds for the blocks below
            rn = run.md(args.config, min(K, 200), W)
            return {"workload": args.config, "skin_A": SKIN, "steps": rs["K"],
                    "ms_per_step": rs["ms"] / rs["K"], "value": rs["N"] * rs["K"] / (rs["ms"] * 1e-3),
                    "rebuilds": rs["rebuilds"], "pairs": rs["n_pairs"],
                    "ms_per_step_rebuild_every_step": rn["ms"] / rn["K"], "pairs_rebuild_every_step": rn["n_pairs"],
                    "note": "allegro_set_skin: list of r_cut + skin kept until an atom moved skin/2; the skin's "
                            "extra pairs (zero contribution) against the builds it saves"}

        nvt = _guarded(nvt_block)
        skin = _guarded(skin_block)
        pimd = _guarded(pimd_block)
        sam = _guarded(lambda: sam_timing(al, torch))
        lsweep = _guarded(lambda: lmax_sweep(al, torch, dev))
        scale_sample = {}
        if args.config != SCALE and not args.no_scale:
            def scale_block():
                big = Runner(al, torch, dev, blob, cfg)
                try:
                    r = big.md(SCALE, min(K, 200), W)
                    # forces of the initial frame at sampled atoms, for the accuracy check
                    _, Fb = big.forces(r["pos"], r["sp"], r["cell"], WORKLOADS[SCALE]["precision"])
                    idx = np.random.default_rng(5).choice(r["N"], SCALE_SAMPLES, replace=False)
                    scale_sample.update(frame=(r["pos"], r["sp"], r["cell"]), idx=idx, F=Fb[idx])
                finally:
                    big.close()
                return {"value": r["N"] * r["K"] / (r["ms"] * 1e-3), "ms_per_step": r["ms"] / r["K"],
                        "atoms": r["N"], "pairs": r["n_pairs"], "steps": r["K"], "dtype": WORKLOADS[SCALE]["dtype"]}

            paths[SCALE] = _guarded(scale_block)
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            cpu, (pos, sp, cell, E0, F0) = cpu_baseline()
            # force error of every path against the FP64 oracle on the 6,912-atom cell
            for name in paths:
                if name == SCALE:
                    continue
                prec = WORKLOADS[name]["precision"]
                E, F = run.forces(pos, sp, cell, prec)
                d = F - F0
                accuracy[name] = {"max_abs_dF": float(np.abs(d).max()), "rms_dF": float(np.sqrt(np.mean(d * d))),
                                  "abs_dE_per_atom": abs(E - E0) / len(sp), "cell": f"{len(sp)}-atom cell"}
            if scale_sample:
                # the 10^6-atom frame itself: sampled atoms against the oracle's
                # local evaluation (exact: E_i depends only on atoms within r_cut)
                Fr = oracle_local_forces(*scale_sample["frame"], scale_sample["idx"])
                d = scale_sample["F"] - Fr
                accuracy[SCALE] = {"max_abs_dF": float(np.abs(d).max()), "rms_dF": float(np.sqrt(np.mean(d * d))),
                                   "cell": f"{SCALE_SAMPLES} sampled atoms of the {WORKLOADS[SCALE]['n_mol'] * 4}"
                                           "-atom frame (oracle local evaluation)"}
            for name, acc in accuracy.items():
                paths[name]["max_abs_dF_eV_per_A"] = acc["max_abs_dF"]
                paths[name]["rms_dF_eV_per_A"] = acc["rms_dF"]
    else:
        e2e = None
        sam = None
        nvt = None
        skin = None
        pimd = None
        lsweep = None
    run.close()
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    N = head["N"]
    mean_pairs = 0.5 * (head["n_pairs_start"] + head["n_pairs"])
    line = {
        "metric": METRIC,
        "value": job_throughput(world, N, K, ms),
        "unit": "atom-steps/s",
        "n_gpus": world,
        "steps": K,
        "warmup": W,
        "ms_per_step": ms / K,
        "ns_per_pair": 1e6 * (ms / K) / mean_pairs,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": w["dtype"],
        "data": "synthetic",
        "config": {"workload": args.config, "atoms": N, "pairs_start": head["n_pairs_start"],
                   "pairs_end": head["n_pairs"], "state": f"after {W} warm-up MD steps from the seeded frame",
                   "dt_fs": w["dt"],
                   "l2": "inputs larger than L2 (per-pair state of ~6 GB per step at 110,592 atoms)",
                   "parallelism": f"replicas x{world}"},
        "e2e": e2e,
        "gpu_launches": int(head["step_kernels"] * K),
        "roofline": roof,
        "roofline_step": roof_step,
        "kernel_ms": {k: round(v, 4) for k, v in phases.items()},
        "physics": {"energy_drift_over_NkT": head["drift"], "outliers_last": head["outliers_last"],
                    "outliers_max": head["outliers_max"]},
        "clocks": head["clocks"],
    }
    if paths:
        line["paths"] = paths
    if accuracy:
        line["accuracy_vs_fp64_oracle"] = {
            "bound_max_abs_dF": FORCE_BOUND, "headline_within_bound": accuracy[args.config]["max_abs_dF"] <= FORCE_BOUND
            if args.config in accuracy else None, **accuracy}
    if sam:
        line["sam_train_step"] = sam
    if nvt:
        line["nvt"] = nvt
    if skin:
        line["verlet_skin"] = skin
    if pimd:
        line["pimd"] = pimd
    if lsweep:
        line["lmax_sweep"] = lsweep
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
    ap.add_argument("--config", default="tc_110592", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-scale", action="store_true", help="skip the 10^6-atom path")
    ap.add_argument("--only-headline", action="store_true",
                    help="time the headline workload only (no other paths, e2e, accuracy or CPU baseline)")
    ap.add_argument("--only", choices=["pimd", "sam", "lmax"],
                    help="run one secondary block alone (for profiling) and print its result as JSON")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.only:
        return run_block(args)
    return run_ours(args)


def run_block(args):
    """One secondary block on GPU 0 with --steps / --warmup steps where it
    steps (ring-polymer MD) or SAM steps (sam), printed as one JSON line."""
    import torch
    import paper_2303_08169_gb300 as al
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    if args.only == "pimd":
        cfg, blob = _model()
        run = Runner(al, torch, dev, blob, cfg)
        out = run.pimd(args.config, args.steps, args.warmup)
        run.close()
    elif args.only == "sam":
        out = sam_timing(al, torch, steps=args.steps, n_sharp=2)
    else:
        out = lmax_sweep(al, torch, dev, K=args.steps, W=args.warmup)
    print(json.dumps({"block": args.only, **out}), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
