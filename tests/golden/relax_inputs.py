"""Writes the relaxed base structures of workloads 2-5 to tests/golden/relaxed/cfg<k>.npy.

The synthetic-input recipe relaxes each generated structure by 200 steps of capped steepest
descent before the beads are drawn around it: every step moves atom i by alpha F_i, shortened to
at most `cap` nm, with F the FP64 forces of the oracle (nonbonded reaction field and bonded
terms).  alpha = 2e-6 nm^2 mol/kJ keeps the stiffest term stable (alpha k < 1 for the
345,000 kJ/mol/nm^2 bonds).  Only the seeded generator and oracle/ run here; the files are
stored as float32 and read by the tests and the benchmark through synth.config(base=...).

  python tests/golden/relax_inputs.py [k ...]
"""
from __future__ import annotations

import sys
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

import oracle  # noqa: E402
from paper_2501_11962_b300 import synth  # noqa: E402

OUT = Path(__file__).resolve().parent / "relaxed"
STEPS, ALPHA, CAP = 200, 2e-6, 0.01


def relax(k: int) -> np.ndarray:
    w = synth.config(k, n_beads=1)
    x = np.array(w.system.extra["base"], np.float64)
    o = oracle.Oracle(w.system)
    t0 = time.time()
    for step in range(STEPS):
        F, U = o.forces(x)
        if step % 50 == 0:
            print(f"cfg{k} step {step}: U = {U:.6e} kJ/mol, max |F| = {np.abs(F).max():.3e} "
                  f"({time.time() - t0:.0f} s)", flush=True)
        fn = np.linalg.norm(F, axis=1, keepdims=True)
        d = ALPHA * F * np.minimum(1.0, CAP / np.maximum(ALPHA * fn, 1e-300))
        x = x + d
    F, U = o.forces(x)
    print(f"cfg{k} relaxed: U = {U:.6e} kJ/mol, max |F| = {np.abs(F).max():.3e}", flush=True)
    return x.astype(np.float32)


def path(k: int) -> Path:
    return OUT / f"cfg{k}.npy"


def load(k: int):
    """The stored relaxed base structure of workload k (None if it was not written)."""
    p = path(k)
    return np.load(p) if p.exists() else None


if __name__ == "__main__":
    OUT.mkdir(exist_ok=True)
    for k in [int(a) for a in sys.argv[1:]] or [2, 3, 4, 5]:
        np.save(path(k), relax(k))
