"""Generates the rational approximation of the scaled complementary error function used by the
Ewald real-space pair kernels: erfcx(x) = exp(x^2) erfc(x) ~ P(x) / Q(x) on [0, XMAX], P of degree
3 and Q of degree 4 (Q(0) = 1), all coefficients positive, so that an FP32 Horner evaluation has no
cancellation.  The kernels then form erfc(beta r) = exp(-beta^2 r^2) P/Q and reuse the Gaussian for
the force term 2 beta / sqrt(pi) exp(-beta^2 r^2).

The fit is linearised least squares on the relative error (Sanathanan-Koerner iteration: each
step solves min sum w (P - y Q)^2 / (Q_prev y)^2), with weights raised where the error peaks, at
Chebyshev nodes of [0, XMAX].  Run it to print the C table that csrc/mop_pairmath.cuh holds.
"""
from __future__ import annotations

import numpy as np

XMAX = 6.0          # beta rc up to 6: erfc(6) = 2e-17, beyond any useful real-space tolerance
DEG_P, DEG_Q = 3, 4


def fit(xmax: float = XMAX, m: int = DEG_P, n: int = DEG_Q, nodes: int = 6000, iters: int = 40):
    from scipy.special import erfcx
    k = np.arange(nodes)
    x = 0.5 * xmax * (1.0 - np.cos(np.pi * (k + 0.5) / nodes))
    y = erfcx(x)
    q = np.ones(nodes)
    w = np.ones(nodes)
    for _ in range(iters):
        A = np.hstack([np.vander(x, m + 1, increasing=True),
                       -(y[:, None] * np.vander(x, n + 1, increasing=True)[:, 1:])])
        s = w / (q * y)
        sol, *_ = np.linalg.lstsq(A * s[:, None], y * s, rcond=None)
        P, Q = sol[:m + 1], np.concatenate([[1.0], sol[m + 1:]])
        q = np.polyval(Q[::-1], x)
        r = (np.polyval(P[::-1], x) / q - y) / y
        w = w * (1.0 + 30.0 * np.abs(r) / np.abs(r).max())
    return P, Q


def c_table(P, Q) -> str:
    fmt = lambda v: ", ".join(f"{c:.9e}f" for c in v)   # noqa: E731
    return (f"constexpr float kErfcxP[{len(P)}] = {{{fmt(P)}}};\n"
            f"constexpr float kErfcxQ[{len(Q)}] = {{{fmt(Q)}}};")


if __name__ == "__main__":
    P, Q = fit()
    assert (P > 0).all() and (Q > 0).all()
    print(c_table(P, Q))
