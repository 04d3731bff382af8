"""Benchmark of the explicit OTM material-point update on GB300.

Workload (default): the scaled-up Johnson-Cook Taylor rod with adiabatic heating, R 3.2 mm,
L 25.4 mm, h 0.12 mm: 501,189 nodes, 2,854,368 material points (synthetic, seeded). A step is one
pass of Algorithm 1 over all points (node update, kinematics, return map, linked-cell search,
LME shape functions, node-major lists). Metric: material-point-steps/s = n_mps * steps / time.

The configured run is 1000 steps. The cost of a step grows while the elastic wave from the
impact sweeps the rod (the LME solve needs Newton iterations wherever the material deforms), so
the timed window sits mid-run: --start-step untimed steps (default 500), then W warm-up and K
timed steps.

value       : FP64 path (--precision mixed: the mixed path alone), inputs resident in HBM, CUDA
              events on the library's stream.
whole_run   : the same metric over all 1000 configured steps of the run (the spin-up, the window
              and the rest, each timed with CUDA events).
mixed       : the mixed path (FP32 force scatter, node update and kinematics gather; double-float
              Newton Hessian sums; FP64 weights, residual, F and return map), from the FP64 path's
              state at the same step.
adjoint     : adjoint/forward time ratio of the hand-written GPU adjoint on the 202,752-MP rod.
e2e         : the same metric through the C ABI from page-locked host memory: the state at the
              window's start loaded from a host snapshot (H2D of every node, MP and support array),
              then every step followed by a D2H of the node positions (after one untimed load).
roofline    : the dominant kernel of the step (largest phase time) against the FP64 peak, with
              the method's algorithmic flops (frac) and the kernel's executed flops (frac_executed).
cpu_baseline: the serial FP64 oracle on a bounded sample of the same workload (a contiguous
              block of material points in the middle of the rod, with the full node set), started
              from the GPU's state at the window's start; cpu_baseline_all_cores: the oracle's
              OpenMP build (the same arithmetic) on every host core, same sample and state.
chip        : the orthogonal-cutting block (4 x 1 x 0.4 mm, 2,996,352 MPs, mixed precision, erosion
              and compaction in every step): a window from the start (tool one spacing away) and a
              window with the tool embedded 1.5 spacings (contact, plastic flow).

--gpus N under torchrun: N independent replicas (one rod per GPU, no collective in the data
path; "scaling": "weak"); the timing is bracketed by barriers and the max over ranks is taken.
--impl reference: times the oracle (the CPU reference) on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import scenarios  # noqa: E402

METRIC = "material-point-steps/s on 1 GB300 (FP64 vs mixed); adjoint/forward time ratio"
UNIT = "MP-steps/s"
MIXED_DTYPE = ("f32 scatter/node update/kinematics gather/row N d, double-float LME Hessian sums, "
               "f64 exponent, N, Z, residual, F and return map")

# Arithmetic per pair of the LME kernel (FP64; an FMA counts 2 flops), Newton evaluations per
# solve = 1 + k (k the mean Newton iterations, measured):
#  algorithmic, the method's own work (the exp not counted as flops): per evaluation 25 (exponent
#  lambda . d + prior: 6; Z, r, J = sum w d d^T: 1 + 6 + 12), once 15 (d_a and the prior term,
#  N, grad N) and 17 (mass and force contributions): (1 + k) 25 + 32.
#  executed in FP64 by this kernel: setup 10 (d, prior exponent), per evaluation 29 (exponent 6,
#  the table exp's two FMAs 4 (its range reduction in integer operations, its polynomial in
#  double-float on the FP32 pipe), w d 3, Z 1, r 3, J 12), final 20 (N 1, e = N d 3, mass 1,
#  force Q e 15): 30 + 29 (1 + k).
LME_ALG_PER_EVAL, LME_ALG_ONCE = 25, 32
LME_EXEC_PER_EVAL, LME_EXEC_ONCE = 29, 30
#  k_search (FP32): 8 flops per candidate (3 sub, 1 mul, 2 fma); candidates ~ 3.73 x support.
#  k_kinematics (FP64): 24 flops per pair (x_p: 3 fma, G = sum du (x) e: 9 fma).
SEARCH_PER_CAND, CAND_PER_PAIR = 8, 3.73
KIN_PER_PAIR = 24
# DRAM bytes per pair of one k_lme launch, from the ncu capture of the h 0.29 mm rod at step 302
# (dram__bytes_read.sum + dram__bytes_write.sum = 3.959 GB over 54.11 M pairs); the traffic of
# a launch scales with its pairs (shape and contribution writes, ID and rank reads)
LME_DRAM_BYTES_PER_PAIR = (0.395994e9 + 3.563405e9) / (202752 * 266.871)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12   # 2 FP64 FMA lanes / SM / clock at 2070 MHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


def aggregate(ms_local: float, n_mps: int, steps: int, world: int, dist, device="cpu"):
    """Replicas: every rank runs its own rod; the job time is the slowest rank's (max over ranks)
    and the value counts the material-point steps of all ranks."""
    import torch
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    return ms, world * n_mps * steps / (ms / 1e3)


def workload(name: str, seed: int = 0):
    if name == "taylor_jc_h0.12":
        return scenarios.config_taylor_jc(h=0.12e-3, seed=seed)
    if name == "taylor_jc_h0.103":
        return scenarios.config_taylor_jc(h=0.103e-3, seed=seed)
    if name == "taylor_jc_h0.29":
        return scenarios.taylor_rod(h=0.29e-3, material=scenarios.copper_jc(), seed=seed,
                                    name="taylor_jc_h0.29")
    if name == "taylor_j2_h0.8":
        return scenarios.config_taylor_j2(seed=seed)
    raise ValueError(name)


def cpu_sample(prob, layers: int = 4):
    """A bounded sample of the workload for the oracle: the material points of `layers` cell
    layers in the middle of the rod (complete supports), with the full node set. Returns the
    sample problem and the sampled MP indices."""
    per_layer = prob.n_mps // int(round(prob.meta["L"] / prob.h))
    k0 = int(round(prob.meta["L"] / prob.h)) // 2
    sl = np.arange(k0 * per_layer, (k0 + layers) * per_layer)
    import copy
    s = copy.copy(prob)
    s.mp_x = prob.mp_x[sl].copy()
    s.mp_vol = prob.mp_vol[sl].copy()
    s.mp_mass = prob.mp_mass[sl].copy()
    s.mp_material = prob.mp_material[sl].copy()
    return s, sl


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ---------------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (SM clock, throttle reasons) taken during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm_, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm_)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------------- GPU arm
STATE_FIELDS = ["node_x", "node_du", "mp_x", "F", "be", "sigma", "vol", "ebar", "T", "lam"]


def timed_steps(sim, n, torch):
    """n steps enqueued back to back, timed with CUDA events on the library's stream (ms)."""
    if n <= 0:
        return 0.0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(sim.stream)
    st = sim.step(n, sync=False)
    e1.record(sim.stream)
    torch.cuda.synchronize()
    code, fid = sim.error()
    if st != 0 or code != 0:
        raise RuntimeError(f"steps failed: {st} {code} {fid}")
    return e0.elapsed_time(e1)


def time_gpu(prob, precision, steps, warmup, torch, dist, start: int = 0, snap=None, save_snaps: bool = False,
             profile_window: bool = False, save_state: bool = False):
    """K timed steps after W warm-up steps, from the state after `start` spin-up steps (timed as
    well, for the whole-run figure) or from the snapshot `snap`. With save_snaps the state there
    is also returned as a device and a page-locked host snapshot, with save_state as host arrays."""
    from paper_2206_08772_gb300.otm import OTM
    sim = OTM(prob, precision=precision)
    stream = sim.stream
    spin_ms = 0.0
    if snap is not None:
        sim.restore(snap)
    elif start > 0:
        spin_ms = timed_steps(sim, start, torch)
    snaps = (sim.snapshot(), sim.snapshot(host=True)) if save_snaps else None
    state = {f: sim.get(f) for f in STATE_FIELDS} if save_state else None
    warm_ms = timed_steps(sim, warmup, torch)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = sim.launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if profile_window:   # marks the timed steps for a profiler started with --profile-from-start off
        import torch.cuda.profiler
        torch.cuda.profiler.start()
    e0.record(stream)
    st = sim.step(steps, sync=False)
    e1.record(stream)
    torch.cuda.synchronize()
    if profile_window:
        torch.cuda.profiler.stop()
    if dist is not None:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    code, fid = sim.error()
    if st != 0 or code != 0:
        raise RuntimeError(f"timed steps failed: {st} {code} {fid}")
    launches = sim.launches() - l0
    cnt = sim.get("support_count").astype(np.float64)
    it = sim.get("newton_it").astype(np.float64)
    info = dict(ms=ms, spin_ms=spin_ms, warm_ms=warm_ms, launches=launches, mean_support=float(cnt.mean()),
                mean_newton_it=float(it.mean()), snaps=snaps, state=state)
    return sim, info


def phase_profile(sim, steps: int = 3):
    """Per-phase average milliseconds (CUDA events around each phase on the library stream) and
    the total of the profiled steps."""
    sim.phase_times()
    sim.phase_timing(True)
    t0 = time.perf_counter()
    st = sim.step(steps)
    wall = time.perf_counter() - t0
    pt = sim.phase_times()
    sim.phase_timing(False)
    if st != 0:
        raise RuntimeError(f"profiled steps failed: {st}")
    return {k: (ms / n if n else 0.0) for k, (ms, n) in pt.items()}, 1e3 * wall


def time_e2e(sim, prob, steps, torch, host_snap):
    """Through the C ABI from page-locked host memory, on an existing handle of the problem: the
    state at the start of the timed window is loaded from a host snapshot (H2D of every node, MP
    and support array, then the shape functions regenerated), then per step otm_step + a D2H
    read of the node positions."""

    def pinned(a):
        t = torch.empty(a.shape, dtype=getattr(torch, str(a.dtype)), pin_memory=True)
        t.numpy()[...] = a
        return t.numpy()

    out = pinned(np.zeros((prob.n_nodes, 3)))
    h2d = host_snap[0].numel()
    # one untimed load first: the GPU's first pass over a freshly written page-locked buffer pays
    # for setting up its address translation (about 8 GB/s instead of 28+)
    sim.restore(host_snap)
    sim.get("node_x", out=out)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim.restore(host_snap)
    t_restore = time.perf_counter() - t0
    for _ in range(steps):
        st = sim.step(1, sync=False)
        if st != 0:
            raise RuntimeError(f"e2e step failed {st}")
        sim.get("node_x", out=out)
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    return dict(value=prob.n_mps * steps / t, unit=UNIT, h2d_bytes_per_step=int(h2d // max(steps, 1)),
                d2h_bytes_per_step=int(out.nbytes), seconds=t, restore_seconds=t_restore)


def time_adjoint(steps: int, torch):
    """Adjoint/forward time ratio on the 202,752-MP Johnson-Cook rod (h 0.29 mm): forward of
    `steps` steps from the impact with ceil(sqrt(steps)) checkpoints, then the backward pass
    (segment recompute + backward steps) for one objective."""
    import math

    from paper_2206_08772_gb300.adjoint import backward_pass, objectives_and_seeds
    from paper_2206_08772_gb300.otm import OTM
    prob = workload("taylor_jc_h0.29")
    every = int(math.ceil(math.sqrt(steps)))
    sim = OTM(prob, precision="fp64")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    checkpoints = {0: sim.snapshot()}
    for k in range(steps):
        if sim.step(1) != 0:
            raise RuntimeError("adjoint forward failed")
        if (k + 1) % every == 0 and k + 1 < steps:
            checkpoints[k + 1] = sim.snapshot()
    final = sim.snapshot()
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    vals, seeds, _ = objectives_and_seeds(sim.get("node_x"), sim.get("node_mass"), prob.h)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    grad = backward_pass(sim, prob, steps, every, checkpoints, final, seeds[0])
    torch.cuda.synchronize()
    t_bwd = time.perf_counter() - t0
    sim.close()
    return {"workload": "taylor_jc_h0.29 (38,181 nodes, 202,752 MPs), JC copper", "steps": steps,
            "checkpoint_every": every, "forward_s": t_fwd, "backward_s": t_bwd, "ratio": t_bwd / t_fwd,
            "objective": "final length", "dL_dtheta": dict(zip(("A", "B", "n", "C", "m", "v0"), grad.tolist()))}


def timed_oracle_steps(sim, n_mps, steps, min_seconds, max_steps):
    """`steps` oracle steps, or (steps None) as many as fill min_seconds (at most max_steps)."""
    t0 = time.perf_counter()
    if steps is not None:
        st = sim.step(steps)
    else:
        steps, st = 0, 0
        while st == 0 and steps < max_steps and (steps == 0 or time.perf_counter() - t0 < min_seconds):
            st = sim.step(1)
            steps += 1
    t = time.perf_counter() - t0
    if st != 0:
        raise RuntimeError(f"oracle step failed {st}")
    return n_mps * steps / t, steps, t


def time_oracle_midrun(prob, state, step, omp: bool, min_seconds: float = 10.0, max_steps: int = 60):
    """The oracle on the bounded sample, started from the GPU's state at `step` (the start of the
    benchmark window): the sample's MP fields and every node's position and increment are set,
    the supports and shape functions rebuilt (untimed), then the timed steps."""
    import oracle
    samp, sel = cpu_sample(prob)
    sim = oracle.Sim(samp, omp=omp)
    sim.set("node_x", state["node_x"])
    sim.set("node_du", state["node_du"])
    for f in STATE_FIELDS[2:]:
        sim.set(f, state[f][sel])
    st = sim.refresh()
    if st != 0:
        raise RuntimeError(f"oracle refresh failed {st}")
    value, steps, t = timed_oracle_steps(sim, samp.n_mps, None, min_seconds, max_steps)
    cores = host_cores() if omp else 1
    return dict(value=value, unit=UNIT, cores=cores, kind="oracle",
                sample=(f"{samp.n_mps} MPs (4 cell layers at mid-length) of the {prob.n_mps}-MP rod with all "
                        f"{prob.n_nodes} nodes, started from the GPU state at step {step} (the benchmark "
                        f"window's start), {steps} oracle steps in {t:.1f} s; "
                        + (f"OpenMP build on {cores} threads" if omp else "serial C, 1 thread")),
                seconds=t)


def time_oracle(prob, steps: int | None, warmup: int = 0, omp: bool = True, min_seconds: float = 10.0,
                max_steps: int = 60):
    """The oracle on the bounded sample from the impact (the reference arm: no GPU state)."""
    import oracle
    samp, _ = cpu_sample(prob)
    t0 = time.perf_counter()
    sim = oracle.Sim(samp, omp=omp)
    t_init = time.perf_counter() - t0
    for _ in range(warmup):
        sim.step(1)
    value, steps, t = timed_oracle_steps(sim, samp.n_mps, steps, min_seconds, max_steps)
    cores = host_cores() if omp else 1
    return dict(value=value, unit=UNIT, cores=cores, kind="oracle",
                sample=(f"{samp.n_mps} MPs (4 cell layers at mid-length) of the {prob.n_mps}-MP rod with all "
                        f"{prob.n_nodes} nodes, {steps} oracle steps ({t:.1f} s) after init ({t_init:.1f} s) "
                        f"and {warmup} warm-up steps, counted from the impact; "
                        + (f"OpenMP build on {cores} threads" if omp else "serial C, 1 thread")),
                seconds=t)


def run_chip(torch, steps: int, warmup: int):
    """Config 3's block at full size in the mixed path with erosion on (compaction runs every
    step): a window from the start of the run (the tool one spacing from the block, as
    configured) and one with the tool embedded 1.5 spacings (contact, plastic flow)."""
    from paper_2206_08772_gb300.otm import OTM
    out = {}
    for name, embed in (("start", 0.0), ("tool_embedded_1.5h", 1.5)):
        h = 1.0e-3 / 68
        prob = scenarios.config_chip(h=h, embed=embed * h)
        sim = OTM(prob, precision="mixed", max_support=384)
        warm_ms = timed_steps(sim, warmup, torch)
        l0 = sim.launches()
        ms = timed_steps(sim, steps, torch)
        c = sim.counts()
        out[name] = {"value": c["n_mps"] * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps,
                     "steps": steps, "warmup": warmup, "n_mps": prob.n_mps, "n_mps_after": c["n_mps"],
                     "n_nodes_after": c["n_nodes"], "gpu_launches": sim.launches() - l0,
                     "mean_newton_iterations": float(sim.get("newton_it").mean()),
                     "plastic_mps": int((sim.get("ebar") > 0).sum()), "warmup_ms": warm_ms}
        sim.close()
        del sim
        torch.cuda.empty_cache()
    return {"workload": "chip 4 x 1 x 0.4 mm, h 1/68 mm: 527,436 nodes, 2,996,352 MPs, Ti-6Al-4V-like JC with "
                        "fracture, tool rake 0, clearance 7 deg, depth 0.2 mm, 5 m/s, mixed precision",
            **out}


def sweep_run(prob, precision, steps, torch):
    """One rod of the sweep: up to `steps` steps, one call per step, timed with CUDA events on
    the library's stream. Returns (sim, ms, steps done, error or None); with an error the state is
    that of the failing step."""
    from paper_2206_08772_gb300.otm import OTM
    sim = OTM(prob, precision=precision)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(sim.stream)
    done, err = 0, None
    for _ in range(steps):
        st = sim.step(1)
        if st != 0:
            err = {"code": st, "mp_or_node_id": sim.error()[1], "at_step": done + 1}
            break
        done += 1
    e1.record(sim.stream)
    torch.cuda.synchronize()
    return sim, e0.elapsed_time(e1), done, err


def run_sweep(args, torch):
    """The mixed-precision sweep: 16 Johnson-Cook rods (R 3.2, L 25.4 mm) with h log-spaced from
    0.5 to 0.12 mm, v0 ~ U(150, 300) m/s, A and B scaled by U(0.9, 1.1) (seeded); each run up to
    `sweep_steps` steps in FP64 and in the mixed path, with node insertion on. The step is
    proportional to h, so 1000 steps of a coarse rod span up to 4x the physical time of the
    finest; where a run meets a failure of the discretization first (an inverted neighbourhood
    at the flattened impact face, or a point that leaves its support's hull beyond what inserted
    nodes repair), both paths are timed and compared over the steps before it and the row
    says so. Reported per rod: the time per step of each path (CUDA events) and the
    final-geometry difference of the mixed path from the FP64 path (which matches the oracle to
    1e-10): final length and footprint radius."""
    from paper_2206_08772_gb300.adjoint import objectives_and_seeds
    rng = np.random.default_rng(2024)
    rows = []
    for i, h in enumerate(np.geomspace(0.5e-3, 0.12e-3, 16)):
        v0 = float(rng.uniform(150.0, 300.0))
        A, B = 90e6 * float(rng.uniform(0.9, 1.1)), 292e6 * float(rng.uniform(0.9, 1.1))
        prob = scenarios.taylor_rod(h=float(h), material=scenarios.copper_jc(A=A, B=B), v0=v0, seed=i,
                                    name=f"sweep_{i}")
        prob.max_insert = max(1000, prob.n_nodes // 20)
        steps = args.sweep_steps
        stop = None
        res = {}
        for attempt in range(3):
            res = {}
            for prec in ("fp64", "mixed"):
                sim, ms, done, err = sweep_run(prob, prec, steps, torch)
                if err is not None:
                    res = None
                    stop = dict(err, precision=prec)
                    steps = done          # the steps before the failure, for both paths
                    sim.close()
                    torch.cuda.empty_cache()
                    break
                L_, R_ = objectives_and_seeds(sim.get("node_x"), sim.get("node_mass"), prob.h)[0]
                res[prec] = (ms, L_, R_, sim.counts()["n_nodes"] - prob.n_nodes)
                sim.close()
                del sim
                torch.cuda.empty_cache()
            if res is not None:
                break
        if not res or steps == 0:
            rows.append({"h_mm": float(h) * 1e3, "n_mps": prob.n_mps, "v0": v0, "failed": stop})
            continue
        (t64, L64, R64, ins64), (t32, L32, R32, ins32) = res["fp64"], res["mixed"]
        rows.append({"h_mm": float(h) * 1e3, "n_mps": prob.n_mps, "v0": v0, "A": A, "B": B, "steps": steps,
                     "stopped_by": stop, "fp64_ms_per_step": t64 / steps, "mixed_ms_per_step": t32 / steps,
                     "speedup": t64 / t32, "rel_err_length": abs(L32 - L64) / L64,
                     "rel_err_radius": abs(R32 - R64) / R64, "inserted_nodes_fp64": ins64,
                     "inserted_nodes_mixed": ins32})
        print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    ok = [r for r in rows if "speedup" in r]
    print(json.dumps({"sweep": "mixed vs fp64, 16 JC rods", "max_steps": args.sweep_steps, "rods": rows,
                      "speedup_median": float(np.median([r["speedup"] for r in ok])),
                      "speedup_weighted": float(sum(r["n_mps"] * r["steps"] * r["fp64_ms_per_step"] for r in ok)
                                                / sum(r["n_mps"] * r["steps"] * r["mixed_ms_per_step"] for r in ok)),
                      "max_rel_err_length": max(r["rel_err_length"] for r in ok),
                      "max_rel_err_radius": max(r["rel_err_radius"] for r in ok)}))


def run_eps_sweep(torch):
    """The stabilised OTM (Eq. 7-8) over a range of penalties eps = c E h^2 (the paper gives no
    value): (a) the plain J2 Taylor rod (R 3.2, L 25.4 mm, h 0.8 mm, 100 steps): final length and
    footprint radius against eps = 0, and the time per step; (b) an elastic rod (no yield, no wall,
    axial velocity gradient 4e3 1/s, L 6.4 mm, 60 steps): drift of the total energy (kinetic from
    the central velocity and the lumped mass, Hencky strain energy of F) against eps = 0."""
    from paper_2206_08772_gb300.adjoint import objectives_and_seeds
    from paper_2206_08772_gb300.otm import OTM

    def strain_energy(sim, p):
        F = sim.get("F").reshape(-1, 3, 3)
        w = np.linalg.eigvalsh(F @ np.transpose(F, (0, 2, 1)))
        e = 0.5 * np.log(w)
        tr = e.sum(1)
        dev = e - tr[:, None] / 3
        mat = p.materials[0]
        return (p.mp_vol * (0.5 * mat.K * tr ** 2 + mat.mu * (dev * dev).sum(1))).sum()

    def energy(sim, p):   # at time n; advances one step
        du_n = sim.get("node_du").copy()
        se = strain_energy(sim, p)
        assert sim.step(1) == 0
        v = (du_n + sim.get("node_du")) / (2 * p.dt)
        return se + 0.5 * (sim.get("node_mass") * (v * v).sum(1)).sum()

    rows = []
    base = None
    for c in (0.0, 1e-4, 1e-3, 1e-2, 1e-1):
        p = scenarios.config_taylor_j2()
        mat = p.materials[0]
        p.eps_stab = c * mat.E * p.h ** 2
        sim = OTM(p)
        ms = timed_steps(sim, 100, torch)
        (L, R), _, _ = objectives_and_seeds(sim.get("node_x"), sim.get("node_mass"), p.h)
        sim.close()
        q = scenarios.taylor_rod(h=0.8e-3, R=3.2e-3, L=6.4e-3, wall=False,
                                 material=scenarios.copper_j2(), name="elastic_rod")
        q.materials[0].sigma_y0 = 1e30
        zc = q.node_x[:, 2].mean()
        q.node_du0 = np.zeros_like(q.node_x)
        q.node_du0[:, 2] = 4e3 * (q.node_x[:, 2] - zc) * q.dt
        q.eps_stab = c * q.materials[0].E * q.h ** 2
        se = OTM(q)
        e0 = energy(se, q)
        assert se.step(58) == 0
        e1 = energy(se, q)
        se.close()
        row = {"c": c, "eps_N": p.eps_stab, "ms_per_step": ms / 100, "final_length_mm": L * 1e3,
               "footprint_radius_mm": R * 1e3, "elastic_energy_drift": abs(e1 - e0) / e0}
        if base is None:
            base = row
        row["length_change_vs_eps0"] = (L * 1e3 - base["final_length_mm"]) / base["final_length_mm"]
        row["radius_change_vs_eps0"] = (R * 1e3 - base["footprint_radius_mm"]) / base["footprint_radius_mm"]
        rows.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
    print(json.dumps({"eps_sweep": "stabilised OTM, eps = c E h^2", "rows": rows}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="taylor_jc_h0.12")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                    help="path of the main timed run (mixed: the mixed path alone, no second leg)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-whole-run", action="store_true")
    ap.add_argument("--no-chip", action="store_true")
    ap.add_argument("--adjoint-steps", type=int, default=500)
    ap.add_argument("--run-steps", type=int, default=1000, help="configured length of the run (whole-run figure)")
    ap.add_argument("--start-step", type=int, default=500,
                    help="untimed steps before the warm-up (the timed window sits mid-run)")
    ap.add_argument("--sweep", action="store_true", help="run the 16-rod mixed-precision sweep instead")
    ap.add_argument("--profile-window", action="store_true",
                    help="cudaProfilerStart/Stop around the timed FP64 steps (for ncu --profile-from-start off)")
    ap.add_argument("--sweep-steps", type=int, default=1000)
    ap.add_argument("--eps-sweep", action="store_true", help="run the stabilisation penalty sweep instead")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    prob = workload(args.workload)
    config = {"workload": f"{prob.name}: Taylor rod R 3.2 mm, L 25.4 mm, Johnson-Cook copper + adiabatic heating",
              "n_nodes": prob.n_nodes, "n_mps": prob.n_mps, "h_mm": prob.h * 1e3, "gamma": prob.gamma,
              "support_tol": prob.support_tol, "dt_s": prob.dt, "max_support": 384,
              "l2": "inputs larger than L2 (pair arrays of tens of GB)", "parallelism": f"replicas x{args.gpus}",
              "run_steps": args.run_steps, "start_step": args.start_step,
              "timed_window": f"steps {args.start_step + args.warmup + 1}-{args.start_step + args.warmup + args.steps}"}

    if args.impl == "reference":
        if rank != 0:
            return
        o = time_oracle(prob, args.steps, args.warmup, omp=True)
        line = {"impl": "reference", "metric": METRIC, "value": o["value"], "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * o["seconds"] / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": config,
                "cpu_baseline": {"value": o["value"], "unit": UNIT, "cores": o["cores"], "kind": "oracle",
                                 "sample": o["sample"]},
                "e2e": {"value": o["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist_
        torch.cuda.set_device(local)
        dist_.init_process_group("nccl")
        dist = dist_
    else:
        torch.cuda.set_device(0)

    if args.eps_sweep:
        if rank == 0:
            run_eps_sweep(torch)
        if dist is not None:
            dist.destroy_process_group()
        return
    if args.sweep:
        if rank == 0:
            run_sweep(args, torch)
        if dist is not None:
            dist.destroy_process_group()
        return

    with ClockSampler(local) as clk:
        sim, info = time_gpu(prob, args.precision, args.steps, args.warmup, torch, dist, start=args.start_step,
                             save_snaps=True, profile_window=args.profile_window,
                             save_state=not args.no_cpu_baseline and rank == 0)
    snap_dev, snap_host = info.pop("snaps")
    state = info.pop("state")
    phases, prof_ms = phase_profile(sim)
    ms, value = aggregate(info["ms"], prob.n_mps, args.steps, world, dist, device="cuda")

    whole = None
    if not args.no_whole_run:
        done = args.start_step + args.warmup + args.steps + 3
        rest_ms = timed_steps(sim, args.run_steps - done, torch)
        total_ms = info["spin_ms"] + info["warm_ms"] + info["ms"] + prof_ms + rest_ms
        whole = {"value": prob.n_mps * args.run_steps / (total_ms / 1e3), "unit": UNIT, "steps": args.run_steps,
                 "seconds": total_ms / 1e3,
                 "note": "steps 1-%d: spin-up, warm-up, window and the rest timed with CUDA events; the 3 "
                         "phase-profiled steps by wall clock" % args.run_steps}

    mixed = None
    if not args.no_mixed and args.precision == "fp64":
        simm, infom = time_gpu(prob, "mixed", args.steps, args.warmup, torch, dist, snap=snap_dev)
        phases_m, _ = phase_profile(simm)
        simm.close()
        del simm
        torch.cuda.empty_cache()
        mv = world * prob.n_mps * args.steps / (infom["ms"] / 1e3)
        mixed = {"value": mv, "unit": UNIT, "ms_per_step": infom["ms"] / args.steps,
                 "speedup_vs_fp64": mv / value,
                 "dtype": MIXED_DTYPE,
                 "phases_ms": phases_m}
    adjoint = None
    if not args.no_adjoint and rank == 0:
        adjoint = time_adjoint(args.adjoint_steps, torch)
        torch.cuda.empty_cache()
    e2e = None
    if not args.no_e2e:
        e2e = time_e2e(sim, prob, args.steps, torch, snap_host)
        e2e["value"] *= world
    sim.close()
    del sim, snap_dev, snap_host
    torch.cuda.empty_cache()
    chip = None
    if not args.no_chip and rank == 0:
        chip = run_chip(torch, args.steps, args.warmup)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    n_bar, k_bar = info["mean_support"], info["mean_newton_it"]
    pairs = n_bar * prob.n_mps
    lme_alg = pairs * (LME_ALG_PER_EVAL * (1 + k_bar) + LME_ALG_ONCE) / 1e12
    lme_exec = pairs * (LME_EXEC_PER_EVAL * (1 + k_bar) + LME_EXEC_ONCE) / 1e12
    work = {"lme": (lme_alg, FP64_PEAK_TFLOPS, "fp64")}   # kernel -> (algorithmic TFLOP per launch, peak, kind)
    if phases.get("kinematics", 0.0) > 0.0:     # separate kernels
        work["search"] = (pairs * CAND_PER_PAIR * SEARCH_PER_CAND / 1e12, FP32_PEAK_TFLOPS, "fp32")
        work["kinematics"] = (pairs * KIN_PER_PAIR / 1e12, FP64_PEAK_TFLOPS, "fp64")
    else:                                        # fused kinematics + search: its FP64 part
        work["search"] = (pairs * KIN_PER_PAIR / 1e12, FP64_PEAK_TFLOPS, "fp64")
    kernels = {}
    for k, (tf, peak, kind) in work.items():
        ms_k = phases[k]
        kernels[k] = {"ms": ms_k, "achieved_tflops": tf / (ms_k / 1e3), "peak": peak, "kind": kind,
                      "frac": tf / (ms_k / 1e3) / peak}
    dom = max(kernels, key=lambda k: kernels[k]["ms"])
    kd = kernels[dom]
    roofline = {"kernel": f"k_{dom}", "bound": "alu", "achieved": kd["achieved_tflops"], "peak": kd["peak"],
                "unit": "TFLOP/s", "frac": kd["frac"],
                # the executed-flop count and the captured DRAM bytes are those of the FP64 path's kernel
                "frac_executed": ((lme_exec / (kd["ms"] / 1e3) / kd["peak"])
                                  if dom == "lme" and args.precision == "fp64" else None),
                "flops_per_pair": {"algorithmic": LME_ALG_PER_EVAL * (1 + k_bar) + LME_ALG_ONCE,
                                   "executed": (LME_EXEC_PER_EVAL * (1 + k_bar) + LME_EXEC_ONCE
                                                if args.precision == "fp64" else None)},
                "traffic": LME_DRAM_BYTES_PER_PAIR * pairs if dom == "lme" and args.precision == "fp64" else None,
                "traffic_note": ("bytes per launch: DRAM bytes per pair of the ncu capture on the 202,752-MP rod "
                                 "(profiles/) x this launch's pairs"),
                "peak_source": ("derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2070 MHz (no FP64 entry in the "
                                "measured peaks)" if kd["kind"] == "fp64"
                                else "derived: 152 SMs x 128 FP32 FMA/clk x 2 x 2070 MHz"),
                "kernel_ms": kd["ms"], "share_of_step": kd["ms"] / (ms / args.steps), "kernels": kernels}
    cpu = cpu_all = None
    if not args.no_cpu_baseline:
        o = time_oracle_midrun(prob, state, args.start_step, omp=False)
        cpu = {k: o[k] for k in ("value", "unit", "cores", "kind", "sample")}
        o = time_oracle_midrun(prob, state, args.start_step, omp=True)
        cpu_all = {k: o[k] for k in ("value", "unit", "cores", "kind", "sample")}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else MIXED_DTYPE, "data": "synthetic",
            "config": config,
            "gpu_launches": info["launches"], "whole_run": whole, "mixed": mixed, "e2e": e2e,
            "roofline": roofline, "adjoint": adjoint, "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_all,
            "chip": chip, "clocks": clk.summary(),
            "stats": {"mean_support": n_bar, "mean_newton_iterations": k_bar},
            "phases_ms": phases}
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
