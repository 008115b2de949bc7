"""The rational erfcx table of the Ewald pair kernels (csrc/mop_pairmath.cuh) against math.erfc: the
coefficients as compiled (FP32) reproduce erfc(x) exp(x^2) to 3e-7 in FP64 arithmetic and to 6e-7
in an FP32 Horner evaluation with fused multiply-adds, over the range of beta r the kernels use."""
import math
import re
from pathlib import Path

import numpy as np

SRC = Path(__file__).resolve().parents[1] / "paper_2501_11962_b300" / "csrc" / "mop_pairmath.cuh"


def table(name):
    m = re.search(name + r"\[\d+\] = \{([^}]*)\}", SRC.read_text())
    return np.array([np.float32(float(v.strip().rstrip("f"))) for v in m.group(1).split(",")])


def erfc_ref(x):
    return np.array([math.erfc(v) for v in x])


def test_erfcx_table_matches_erfc():
    P, Q = table("kErfcxP"), table("kErfcxQ")
    assert len(P) == 4 and len(Q) == 5 and (P > 0).all() and (Q > 0).all()
    x = np.linspace(0.0, 6.0, 60001)
    ref = erfc_ref(x)
    p64 = np.polyval(P[::-1].astype(np.float64), x)
    q64 = np.polyval(Q[::-1].astype(np.float64), x)
    rel64 = np.abs(np.exp(-x * x) * p64 / q64 - ref) / ref
    assert rel64.max() < 3e-7, rel64.max()
    # FP32 with fused multiply-adds: products of two floats are exact in FP64, one rounding per step
    x32 = x.astype(np.float32)

    def horner(C):
        a = np.float32(C[-1])
        for c in C[-2::-1]:
            a = (np.float64(a) * np.float64(x32) + np.float64(c)).astype(np.float32)
        return a

    r32 = (np.float64(horner(P)) * np.float64(np.float32(1.0) / horner(Q))).astype(np.float32)
    rel32 = np.abs(np.exp(-np.float64(x32) ** 2) * np.float64(r32) - erfc_ref(np.float64(x32))) / erfc_ref(np.float64(x32))
    assert rel32.max() < 6e-7, rel32.max()
    # special values: erfc(0) = 1; erfc(x) ~ exp(-x^2) / (x sqrt(pi)) far out
    assert abs(P[0] / Q[0] - 1.0) < 1e-7
    assert abs(p64[-1] / q64[-1] * 6.0 * math.sqrt(math.pi) - 1.0) < 0.02
