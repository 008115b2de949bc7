#!/usr/bin/env python
"""Benchmark of the MoP effective-potential path (V_eff of Eq. 3 and its gradient) on B300.

One step = one full evaluation of V_eff and dV_eff/dR of a Q = 150,000-atom, N = 64-bead path
(synthetic chains + water system) through the C ABI: mop_set_path (device copy of the step's
coordinates) + mop_veff_and_grad.  value = N * Q * evaluations / s (bead-atoms/s), summed over
ranks.  Inputs are larger than L2 (coordinates 115 MB per step, fields > 1 GB).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "path-gradient evals/s (bead·atoms/s) at Q=150k, N=64; adjoint vs FD-HVP at tol"
UNIT = "bead*atoms/s"
# Canonical flop counts per unique in-cutoff pair of the hot-path scope: about 30 FP32 flops for
# the force and 40 for the adjoint HVP.  The itemised counts of the written formulas (FADD/FMUL =
# 1, FFMA = 2, rsqrt not counted) are 36 and 59; both fractions are reported.
FLOPS_FORCE = 30
FLOPS_HVP = 40
FLOPS_FORCE_ITEMISED = 36
FLOPS_HVP_ITEMISED = 59
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2032.0
FD_SWEEP = (1e-5, 3e-5, 1e-4, 3e-4, 1e-3)
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the pair kernels on
# this workload, from the --set full capture in profiles/k_pairb_cfg5_Q150k_N64.md.  Valid only
# for the kernel sources they were measured on: any change to them makes `traffic` null.
PAIR_TRAFFIC = {"sources_sha256_16": "f0310ddf08aabd60", "k_pairb<0,RF,full>": 516.9e6,
                "k_pairb<1,RF,half>": 1253.5e6}
PAIR_SOURCES = ("mop_pairb.cu", "mop_pairmath.cuh", "mop_prep.cu", "mop_internal.cuh")
# arithmetic of the mixed-precision path, quantity by quantity
PRECISION = {"pair_arithmetic": "f32 (two beads per f32x2 instruction)",
             "forces_F": "double-float (f32 hi + lo): f32 pair sums folded by TwoSum (full list, no j-side "
                         "sums); bonded f32 added exactly",
             "eta": "double-float from the exact R^{n+1} - R^n and the double-float c F; f32 copy for the HVP",
             "H_eta": "f32 pair terms; i-side sums folded into double-floats, the j-atoms' shares of the "
                      "owner-entry pass as 64-bit fixed point (integer atomics: exact, order-independent, scaled "
                      "per bead by a power of two); stored as f32, bonded f32 added",
             "gradient_G": "double-float K (eta^{n-1} - eta^n) + H eta / 2 (- F^1), written as f64",
             "energies": "double-float per warp, f64 per block and across blocks",
             "ewald_j_side_and_grids": "int64 fixed point (2^-23 forces, 2^-40 SPME charge grids)"}


def pair_sources_sha() -> str:
    import hashlib
    csrc = ROOT / "paper_2501_11962_b300" / "csrc"
    return hashlib.sha256(b"".join((csrc / f).read_bytes() for f in PAIR_SOURCES)).hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--config", type=int, default=5)
    ap.add_argument("--beads", type=int, default=None)
    ap.add_argument("--no-fd", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="keep the default neighbour-search geometry")
    ap.add_argument("--no-metad", action="store_true", help="skip the metadynamics production-loop timing")
    ap.add_argument("--no-batch", action="store_true", help="skip the multi-path batching timing")
    ap.add_argument("--no-pme", action="store_true", help="skip the Ewald / SPME electrostatics timing")
    ap.add_argument("--no-skin", action="store_true", help="skip the Verlet-skin (kept pair list) timing")
    return ap.parse_args()


def workload_name(cfg, N, Q, relaxed=False):
    names = {5: "chains+water membrane-sized synthetic system", 4: "water+ion", 3: "water", 2: "water", 1: "LJ fcc"}
    return f"cfg{cfg} {names.get(cfg, '')}{' (relaxed)' if relaxed else ''}: Q={Q}, N={N}"


# Relaxed base structures (200 steps of capped steepest descent on the oracle's forces, written by
# tests/golden/relax_inputs.py); the beads are drawn around them
RELAXED = ROOT / "tests" / "golden" / "relaxed"


def workload(cfg, n_beads=None):
    """The benchmark workload: the relaxed structure when it is stored, else the generated one."""
    from paper_2501_11962_b300 import synth
    f = RELAXED / f"cfg{cfg}.npy"
    base = np.load(f) if f.exists() else None
    return synth.config(cfg, n_beads=n_beads, base=base), base is not None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50",
                 "-i", str(self.dev)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int, device) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------------------------------
# CPU oracle (baseline arm and the cpu_baseline leg)


def oracle_sample_time(w, n_beads_sample: int):
    """Time one oracle V_eff + gradient (analytic HVP, OpenMP over beads) of a sub-path."""
    import oracle
    o = oracle.Oracle(w.system)
    X = np.ascontiguousarray(w.paths[0][:n_beads_sample].astype(np.float64))
    t0 = time.perf_counter()
    o.veff(X)
    dt = time.perf_counter() - t0
    return dt, oracle.num_threads()


def cpu_sample_beads(w):
    import oracle
    return int(min(w.paths[0].shape[0], oracle.num_threads() + 1))


def run_reference(args, world, rank):
    from paper_2501_11962_b300 import synth
    if rank != 0:
        return
    w, relaxed = workload(args.config, args.beads)
    N, Q = w.paths[0].shape[:2]
    ns = cpu_sample_beads(w)
    times = []
    for k in range(args.warmup + args.steps):
        dt, cores = oracle_sample_time(w, ns)
        if k >= args.warmup:
            times.append(dt)
    t = float(np.mean(times))
    value = ns * Q / t
    sample = (f"oracle V_eff+gradient (analytic HVP) of a {ns}-bead sub-path of the workload, "
              f"OpenMP over beads; value = {ns}*Q/time")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args.config, N, Q, relaxed), "Q": Q, "N": N, "paths": 1},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ------------------------------------------------------------------------------------------
# CUDA path


def run_ours(args, world, rank, local):
    import ctypes as C
    import torch
    from paper_2501_11962_b300 import mop, synth

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    w, relaxed = workload(args.config, args.beads)
    X = w.paths[0]
    N, Q = X.shape[:2]
    prec = mop.MOP_PREC_FP64 if w.precision == "fp64" else mop.MOP_PREC_MIXED
    eng = mop.Engine(w.system, precision=prec, device=local)
    Xd = torch.tensor(X, device=dev)
    eng.set_path(0, Xd)
    tuned = eng.tuning()
    if not args.no_tune:
        tuned, _ = eng.autotune(0)              # neighbour-search geometry (not timed)
    eng.set_profiling(True)
    veff = torch.empty(1, dtype=torch.float64, device=dev)
    grad = torch.empty((N, Q, 3), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        eng.set_path(0, Xd, stream=stream.cuda_stream)
        eng.veff_and_grad_device(veff, grad, 0, stream=stream.cuda_stream)

    passes = []
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    # mop_set_path copies device input with cudaMemcpyAsync (no kernel of the library)
    launches_per_step = eng.last_launch_count()
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        e0.record(stream)
        for _ in range(args.steps):
            step()
            passes.append(eng.pass_ms())
        e1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(ms, world, dev)
    value = world * N * Q / (ms * 1e-3)
    mean_pass = {k: float(np.mean([p[k] for p in passes])) for k in passes[0]}

    # roofline of the dominant pair kernel (FP32 ALU bound).  The pass times come from the
    # library's CUDA events on the launching stream; the pair passes are one pair-kernel launch
    # each, plus the small bead-1 energy kernel in the force pass.
    unique, listed = eng.count_pairs(0)
    flops = {"pair_force": unique * FLOPS_FORCE, "pair_hvp": unique * FLOPS_HVP}
    flops_it = {"pair_force": unique * FLOPS_FORCE_ITEMISED, "pair_hvp": unique * FLOPS_HVP_ITEMISED}
    dom = max(("pair_force", "pair_hvp"), key=lambda k: mean_pass[k])
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sms * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    achieved = flops[dom] / (mean_pass[dom] * 1e-3) / 1e12
    achieved_it = flops_it[dom] / (mean_pass[dom] * 1e-3) / 1e12
    fma_peak = mop.measure_fp32_peak(local)      # dependent-FMA microkernel on this GPU, now
    ach_force = flops["pair_force"] / (mean_pass["pair_force"] * 1e-3) / 1e12
    pk = os.environ.get("MOP_PAIR_KERNELS", "")
    half = pk == "half" or prec == mop.MOP_PREC_FP64
    mode = "0" if dom == "pair_force" else "1"
    kname = (f"k_pair<float,{mode}>" if prec != mop.MOP_PREC_FP64 else f"k_pair<double,{mode}>") if half \
        else f"k_pairb<{mode},RF,{'half' if pk == 'blhalf' or (mode == '1' and pk != 'blfull') else 'full'}>"
    traffic = PAIR_TRAFFIC.get(kname) if (args.config == 5 and N == 64 and not half and
                                          pair_sources_sha() == PAIR_TRAFFIC["sources_sha256_16"]) else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "traffic_unit": "bytes per launch", "kernel": kname,
                "unique_pairs_per_launch": unique, "evaluated_pairs_per_launch": listed,
                "flops_per_unique_pair": FLOPS_FORCE if dom == "pair_force" else FLOPS_HVP,
                "peak_note": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flops x {SM_MAX_MHZ:.0f} MHz",
                "peak_measured_fma": fma_peak, "frac_of_measured_fma": achieved / fma_peak,
                "itemised": {"flops_per_unique_pair": FLOPS_FORCE_ITEMISED if dom == "pair_force" else FLOPS_HVP_ITEMISED,
                             "achieved": achieved_it, "frac": achieved_it / peak},
                "pair_force": {"achieved": ach_force, "frac": ach_force / peak,
                               "frac_of_measured_fma": ach_force / fma_peak,
                               "itemised_frac": flops_it["pair_force"] / (mean_pass["pair_force"] * 1e-3) / 1e12 / peak}}

    # end to end through the C ABI with page-locked host buffers, copies inside the timed region.
    # Two ways: one synchronous call pair per step, and the pipelined form (MOP_ASYNC) in which
    # a step's upload and download overlap the next step's evaluation (two buffer sets, taking
    # turns; each step still copies its coordinates in and its V_eff and gradient out).
    xh = [torch.tensor(X).pin_memory() for _ in range(2)]
    gh = [torch.empty((N, Q, 3), dtype=torch.float64).pin_memory() for _ in range(2)]
    vh = [torch.zeros(1, dtype=torch.float64).pin_memory() for _ in range(2)]
    L = eng.L

    def e2e_sync(k):
        st = L.mop_set_path(eng.h, 0, N, C.c_void_p(xh[0].data_ptr()), 0, C.c_void_p(stream.cuda_stream))
        eng._check(st, "mop_set_path")
        st = L.mop_veff_and_grad(eng.h, 0, C.c_void_p(vh[0].data_ptr()), C.c_void_p(gh[0].data_ptr()), 0,
                                 C.c_void_p(stream.cuda_stream))
        eng._check(st, "mop_veff_and_grad")

    def e2e_async(k):
        eng.set_path_async(0, xh[k % 2], stream=stream.cuda_stream)
        eng.veff_and_grad_async(vh[k % 2], gh[k % 2], 0, stream=stream.cuda_stream)

    def time_e2e(step, finish):
        for k in range(2):
            step(k)
        finish()
        barrier(world)
        t0 = time.perf_counter()
        for k in range(args.steps):
            step(k)
        finish()
        return max_over_ranks((time.perf_counter() - t0) / args.steps, world, dev)

    sync_s = time_e2e(e2e_sync, torch.cuda.synchronize)
    e2e_s = time_e2e(e2e_async, lambda: (eng.wait(), torch.cuda.synchronize()))
    assert np.isfinite(vh[(args.steps - 1) % 2].item())
    e2e = {"value": world * N * Q / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(N * Q * 3 * 4),
           "d2h_bytes_per_step": int(N * Q * 3 * 8 + 8), "ms_per_step": e2e_s * 1e3,
           "form": "pipelined (MOP_ASYNC): a step's copies overlap the next step's evaluation",
           "synchronous": {"value": world * N * Q / sync_s, "ms_per_step": sync_s * 1e3}}

    # FD-HVP comparison path (paper Eq. 5) at the same workload
    fd = None
    if not args.no_fd and rank == 0:
        ref_H = eng.get_field(0, mop.MOP_FIELD_HETA)[:N - 1]
        errs, vals = {}, {}
        for h in FD_SWEEP:
            ef = mop.Engine(w.system, precision=prec, hvp_mode=mop.MOP_HVP_FD, fd_h=h, device=local)
            ef.set_path(0, Xd, stream=stream.cuda_stream)
            ef.veff_and_grad_device(veff, grad, 0, stream=stream.cuda_stream)
            torch.cuda.synchronize()
            H = ef.get_field(0, mop.MOP_FIELD_HETA)[:N - 1]
            errs[h] = float(np.linalg.norm(H - ref_H) / np.linalg.norm(ref_H))
            if h == FD_SWEEP[0] or errs[h] <= min(errs.values()):
                k = max(3, args.steps // 2)
                ef.set_path(0, Xd, stream=stream.cuda_stream)
                ef.veff_and_grad_device(veff, grad, 0, stream=stream.cuda_stream)
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                for _ in range(k):
                    ef.set_path(0, Xd, stream=stream.cuda_stream)
                    ef.veff_and_grad_device(veff, grad, 0, stream=stream.cuda_stream)
                b.record(stream)
                torch.cuda.synchronize()
                vals[h] = N * Q / (a.elapsed_time(b) / k * 1e-3)
            ef.close()
        best = min(errs, key=errs.get)
        fd = {"value": vals.get(best), "unit": UNIT, "best_h_nm": best, "hvp_rel_err_best": errs[best],
              "hvp_rel_err_by_h": {f"{h:g}": e for h, e in errs.items()},
              "reaches_1e-4": bool(errs[best] <= 1e-4),
              "adjoint_over_fd_speed": value / world / vals[best] if vals.get(best) else None}

    # The metadynamics production loop (mop_metadynamics, graph mode): BAOAB MD of all beads with
    # one Gaussian deposited per round on a centre-of-mass end-to-end CV.  The time step is the
    # stable one of this action: its c F term gives the path Hessian eigenvalues
    # dt_path omega^4 / (2 nu) for a physical vibration omega, about (5,100 ps^-1)^2 for the
    # flexible O-H bond at dt_path = 2 fs and nu = 5 ps^-1, so velocity Verlet needs dt < 0.39 fs;
    # 0.2 fs is used.  The path starts stationary (every bead at the relaxed base structure) and
    # the thermostat spreads it; the beads of the evaluation workload, independent displacements
    # of 0.01 nm, are far from a solution of Eq. 1 and heat up violently under these dynamics.
    # It runs on the relaxed water box (config 3, Q = 24,000) and on this workload.  Every captured step
    # rebuilds the pair lists; a list that outgrows the capacity the graph was sized for makes
    # mop_step restore its state and repeat the batch with a larger capacity.
    def metad_run(wm, Nm, label):
        Qm = wm.system.n_atoms
        Xm = np.repeat(np.asarray(wm.system.extra["base"], np.float32)[None], Nm, axis=0)
        em = mop.Engine(wm.system, precision=prec, device=local)
        em.set_path(0, Xm)
        em.veff_and_grad(0, want_grad=False)
        _, pairs0 = em.count_pairs(0)
        pos = Xm[-1].astype(np.float64)
        ga = synth.nearest_group(pos, np.asarray(wm.system.box), pos[0], 8)
        gb = synth.nearest_group(pos, np.asarray(wm.system.box), pos[Qm // 2], 8)
        em.add_bias(0, 0.0, 0.0, 0.1, groups=(ga, gb), e2e=True, com=True)
        em.set_graph_mode(True)
        rounds, stride, dt_md = 4, 25, 2e-4
        b0, _ = em.list_stats(0)
        failed = None
        try:
            em.metadynamics(1, 2, dt_md, 5.0, 3, 1.0, 0.1)         # capture and warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            em.metadynamics(rounds, stride, dt_md, 5.0, 3, 1.0, 0.1)
            torch.cuda.synchronize()
            t = time.perf_counter() - t0
            failed = False
        except mop.MopError as e:
            if e.status not in (mop.MOP_ERR_STATE, mop.MOP_ERR_OOM, mop.MOP_ERR_NONFINITE):
                raise
            failed, t = e.status, float("nan")
        b1, _ = em.list_stats(0)
        pairs1 = None
        if not failed:
            em.veff_and_grad(0, want_grad=False)
            _, pairs1 = em.count_pairs(0)
        out = {"workload": label, "start": "stationary path (all beads at the relaxed base structure)",
               "evaluated_pairs_per_launch_at_start": pairs0, "evaluated_pairs_per_launch_at_end": pairs1,
               "md_steps_per_s": rounds * stride / t,
               "ms_per_md_step": t / (rounds * stride) * 1e3, "bead_atom_steps_per_s": Nm * Qm * rounds * stride / t,
               "rounds": rounds, "stride": stride, "dt_ps": dt_md, "gamma_per_ps": 5.0, "graph_mode": True,
               "failed_with_status": failed, "step_batches_rerun_after_list_overflow": em.list_overflows(0),
               "synchronous_list_builds": b1 - b0,
               "note": "host wall clock over the rounds, including one synchronous re-evaluation per deposit"}
        em.close()
        return out

    metad = None
    if not args.no_metad and rank == 0:
        w3, rel3 = workload(3, n_beads=N)
        metad = {"water": metad_run(w3, N, workload_name(3, N, w3.system.n_atoms, rel3)),
                 "this_workload": metad_run(w, N, workload_name(args.config, N, Q, relaxed))}

    # batching: the 8 paths of uneven length of the water + ion workload (config 4, 968 beads)
    # in one call, every pass one launch over all paths, against the same paths one call each
    batch = None
    if not args.no_batch and rank == 0:
        w4 = synth.config(4)
        eb = mop.Engine(w4.system, precision=mop.MOP_PREC_MIXED, device=local)
        nbeads = 0
        for pid, Xp in enumerate(w4.paths):
            eb.set_path(pid, Xp)
            nbeads += Xp.shape[0]
        Q4 = w4.system.n_atoms

        def timed(fn, reps=5):
            fn()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                fn()
            torch.cuda.synchronize()
            return (time.perf_counter() - t0) / reps

        t_all = timed(lambda: eb.veff_and_grad(-1, want_grad=False))
        t_one = timed(lambda: [eb.veff_and_grad(pid, want_grad=False) for pid in range(len(w4.paths))])
        batch = {"workload": f"config 4: {len(w4.paths)} paths, N = {[p.shape[0] for p in w4.paths]}, Q = {Q4}",
                 "value": nbeads * Q4 / t_all, "unit": UNIT, "ms_per_call": t_all * 1e3,
                 "one_call_per_path_ms": t_one * 1e3, "speedup_over_one_call_per_path": t_one / t_all,
                 "note": "host wall clock of the synchronous C-ABI call (V_eff only read back)"}
        eb.close()

    # Ewald electrostatics on the same path: real-space erfc with exclusion corrections alone, then
    # with the SPME reciprocal part (order-4 B-splines, grid spacing <= 0.12 nm, erfc(beta rc) =
    # 1e-5); the difference is the cost of the reciprocal part (spread, FFTs, gather, both passes)
    pme = None
    if not args.no_pme and rank == 0 and prec == mop.MOP_PREC_MIXED:
        import dataclasses
        sys_pme = synth.with_pme(w.system)
        pme = {"grid": list(sys_pme.pme_grid), "order": sys_pme.pme_order, "ew_beta_per_nm": sys_pme.ew_beta}
        for label, sysx in (("real_space_only", dataclasses.replace(sys_pme, pme_grid=(0, 0, 0))),
                            ("spme", sys_pme)):
            ep = mop.Engine(sysx, precision=prec, device=local)
            ep.set_tuning(tuned["col_factor"], tuned["bin_factor"])
            ep.set_profiling(True)

            def pstep():
                ep.set_path(0, Xd, stream=stream.cuda_stream)
                ep.veff_and_grad_device(veff, grad, 0, stream=stream.cuda_stream)

            for _ in range(3):
                pstep()
            torch.cuda.synchronize()
            k = max(3, args.steps // 2)
            pp = []
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(k):
                pstep()
                pp.append(ep.pass_ms())
            b.record(stream)
            torch.cuda.synchronize()
            t = a.elapsed_time(b) / k
            pme[label] = {"ms_per_step": t, "value": N * Q / (t * 1e-3), "unit": UNIT,
                          "pass_ms": {kk: float(np.mean([q[kk] for q in pp])) for kk in pp[0]}}
            ep.close()
        pme["reciprocal_ms_per_step"] = pme["spme"]["ms_per_step"] - pme["real_space_only"]["ms_per_step"]
        pme["reaction_field_ms_per_step"] = ms

    # Verlet skin: evaluations of the same path that keep the list built for rc + skin (the sort
    # and the list build are skipped; the pair kernels walk the longer list)
    skin = None
    if not args.no_skin and rank == 0 and prec == mop.MOP_PREC_MIXED:
        skin = {"rebuilt_every_evaluation_ms": ms}
        for sk in (0.02, 0.05):
            es = mop.Engine(w.system, precision=prec, device=local)
            es.set_tuning(tuned["col_factor"], tuned["bin_factor"])
            es.set_list_skin(sk)
            es.set_profiling(True)
            es.set_path(0, Xd, stream=stream.cuda_stream)
            es.veff_and_grad_device(veff, grad, 0, stream=stream.cuda_stream)   # builds the list
            torch.cuda.synchronize()
            for _ in range(2):
                es.veff_and_grad_device(veff, grad, 0, stream=stream.cuda_stream)
            torch.cuda.synchronize()
            k = max(3, args.steps // 2)
            pp = []
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(k):
                es.veff_and_grad_device(veff, grad, 0, stream=stream.cuda_stream)
                pp.append(es.pass_ms())
            b.record(stream)
            torch.cuda.synchronize()
            _, listed_sk = es.count_pairs(0)
            builds, reuses = es.list_stats(0)
            skin[f"{sk:g}_nm"] = {"kept_list_ms": a.elapsed_time(b) / k, "listed_pairs_per_launch": listed_sk,
                                  "builds": builds, "reuses": reuses,
                                  "pass_ms": {kk: float(np.mean([q[kk] for q in pp])) for kk in pp[0]}}
            es.close()
        skin["listed_pairs_per_launch_without_skin"] = listed

    cpu = None
    if not args.no_cpu and rank == 0 and world == 1:
        ns = cpu_sample_beads(w)
        dt, cores = oracle_sample_time(w, ns)
        cpu = {"value": ns * Q / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"one oracle V_eff+gradient (analytic HVP) of a {ns}-bead sub-path of the workload "
                         f"({dt:.1f} s, OpenMP over beads); value = {ns}*Q/time"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec == 0 else "f64",
            "precision": PRECISION if prec == 0 else "f64 everywhere",
            "data": "synthetic",
            "config": {"workload": workload_name(args.config, N, Q, relaxed), "Q": Q, "N": N, "paths": 1,
                       "hvp": "adjoint", "l2": "inputs larger than L2 (115 MB coordinates per step, >1 GB fields)",
                       "parallelism": f"{world} independent replica(s), one per GPU"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "fd_hvp": fd, "metad": metad, "batch": batch,
            "pme": pme, "skin": skin,
            "pass_ms": mean_pass, "tuning": tuned, "gpu_launches": launches_per_step * args.steps,
            "clocks": clocks.summary(),
        }
        print(json.dumps(line))


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
