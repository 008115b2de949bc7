"""Reciprocal-space Ewald electrostatics for the FP64 oracle (test infrastructure only).

Smooth particle-mesh Ewald (Essmann et al., J. Chem. Phys. 103, 8577 (1995)): charges spread with
cardinal B-splines of order p onto a K1 x K2 x K3 grid of the orthorhombic box, convolved with the
Ewald reciprocal kernel through FFTs (numpy.fft), forces by differentiating the splines.  The
Hessian-vector product is the forward derivative of every step (the derivative of the charge grid
takes its own FFT).  `ewald_recip` is the direct reciprocal-space Ewald sum the pins compare
against.

Conventions: energies kJ/mol, lengths nm, charges e, f = 138.935458 kJ mol^-1 nm e^-2.
"""
from __future__ import annotations

import numpy as np

F_COULOMB = 138.935458


def _spline_values(w, p):
    """M_p(w + t) for t = 0..p-1 (w in [0, 1), any dtype): the p nonzero B-spline weights of a
    point, by the recursion M_n(x) = (x M_{n-1}(x) + (n - x) M_{n-1}(x - 1)) / (n - 1)."""
    A = [w, 1.0 - w]                        # M_2(w), M_2(w + 1)
    for n in range(2, p):
        B = []
        for t in range(n + 1):
            x = w + t
            a = A[t] if t < n else 0.0
            b = A[t - 1] if t >= 1 else 0.0
            B.append((x * a + (n + 1 - x) * b) / n)
        A = B
    return A


def _spline_weights(u, p):
    """Grid offsets and weights of fractional grid coordinates u (shape (Q,)): for t = 0..p-1 the
    point floor(u) - t carries M_p(w + t), with w = u - floor(u), and its first and second
    derivatives, M_p' = M_{p-1}(x) - M_{p-1}(x - 1) and M_p'' = M_{p-2}(x) - 2 M_{p-2}(x - 1) +
    M_{p-2}(x - 2)."""
    base = np.floor(u).astype(np.int64)
    w = u - base

    def shifted(vals, t, k):   # M_n(w + t - k) from the list of M_n(w + s), s = 0..n-1
        s_ = t - k
        return vals[s_] if 0 <= s_ < len(vals) else 0.0

    Mp = _spline_values(w, p)
    Mq = _spline_values(w, p - 1)
    Mr = _spline_values(w, p - 2)
    dM = [shifted(Mq, t, 0) - shifted(Mq, t, 1) for t in range(p)]
    d2M = [shifted(Mr, t, 0) - 2.0 * shifted(Mr, t, 1) + shifted(Mr, t, 2) for t in range(p)]
    return base, np.stack(Mp, 1), np.stack([np.broadcast_to(a, w.shape) for a in dM], 1), \
        np.stack([np.broadcast_to(a, w.shape) for a in d2M], 1)


def _bspline_moduli(K, p):
    """|b(m)|^2 of the Euler exponential splines for m = 0..K-1."""
    m = np.arange(K)
    Mp = _spline_values(np.float64(0.0), p)          # M_p(t) for t = 0..p-1 (M_p(0) = 0)
    den = np.zeros(K, complex)
    for k in range(p - 1):
        den += Mp[k + 1] * np.exp(2j * np.pi * m * k / K)
    return 1.0 / np.abs(den) ** 2


def _kernel(box, K, p, beta, f):
    """theta(m) = f exp(-pi^2 |m~|^2 / beta^2) / (pi V |m~|^2) B(m), m~ the reciprocal vector."""
    box = np.asarray(box, float)
    V = float(np.prod(box))
    mm = [np.fft.fftfreq(K[d], 1.0 / K[d]) / box[d] for d in range(3)]    # m_d / L_d
    m2 = mm[0][:, None, None] ** 2 + mm[1][None, :, None] ** 2 + mm[2][None, None, :] ** 2
    with np.errstate(divide="ignore"):
        th = f * np.exp(-np.pi ** 2 * m2 / beta ** 2) / (np.pi * V * m2)
    th[0, 0, 0] = 0.0
    B = (_bspline_moduli(K[0], p)[:, None, None] * _bspline_moduli(K[1], p)[None, :, None] *
         _bspline_moduli(K[2], p)[None, None, :])
    return th * B


def spme(x, q, box, K, p, beta, f=F_COULOMB, v=None):
    """Reciprocal-space energy and forces (E, F[Q][3]) of charges q at positions x (Q x 3).  With
    a direction v (Q x 3) also the Hessian-vector product H v = -dF(x + e v)/de at e = 0, by
    forward differentiation of every step (the grid's derivative takes its own FFT)."""
    x = np.asarray(x, float)
    box = np.asarray(box, float)
    K = tuple(int(k) for k in K)
    Qn = x.shape[0]
    u = [K[d] * x[:, d] / box[d] for d in range(3)]
    sw = [_spline_weights(u[d], p) for d in range(3)]
    t = np.arange(p)
    idx = [np.mod(sw[d][0][:, None] - t[None, :], K[d]) for d in range(3)]   # (Q, p) grid indices
    M = [sw[d][1] for d in range(3)]
    dM = [sw[d][2] * (K[d] / box[d]) for d in range(3)]                      # d/dx of M
    d2M = [sw[d][3] * (K[d] / box[d]) ** 2 for d in range(3)]

    def outer(a, b, c):
        return a[:, :, None, None] * b[:, None, :, None] * c[:, None, None, :]

    shape = (Qn, p, p, p)
    I0 = np.broadcast_to(idx[0][:, :, None, None], shape).ravel()
    I1 = np.broadcast_to(idx[1][:, None, :, None], shape).ravel()
    I2 = np.broadcast_to(idx[2][:, None, None, :], shape).ravel()

    def spread(W):
        grid = np.zeros(K)
        np.add.at(grid, (I0, I1, I2), W.ravel())
        return grid

    theta = _kernel(box, K, p, beta, f)

    def conv(grid):   # the Ewald kernel applied to a charge grid (real, symmetric)
        return (np.fft.ifftn(np.fft.fftn(grid) * theta) * (K[0] * K[1] * K[2])).real

    W = q[:, None, None, None] * outer(M[0], M[1], M[2])
    grid = spread(W)
    phi = conv(grid)
    E = 0.5 * float(np.sum(grid * phi))
    ph = phi[I0, I1, I2].reshape(shape)
    F = np.zeros((Qn, 3))
    for d in range(3):
        parts = [M[0], M[1], M[2]]
        parts[d] = dM[d]
        F[:, d] = -q * np.sum(outer(*parts) * ph, axis=(1, 2, 3))
    if v is None:
        return E, F
    v = np.asarray(v, float)
    # derivatives along v: M' = dM v_d, dM' = d2M v_d
    Mv = [dM[d] * v[:, d, None] for d in range(3)]
    dMv = [d2M[d] * v[:, d, None] for d in range(3)]
    Wv = q[:, None, None, None] * (outer(Mv[0], M[1], M[2]) + outer(M[0], Mv[1], M[2]) + outer(M[0], M[1], Mv[2]))
    phv = conv(spread(Wv))[I0, I1, I2].reshape(shape)
    H = np.zeros((Qn, 3))
    for d in range(3):
        parts = [M[0], M[1], M[2]]
        parts[d] = dM[d]
        dparts = [Mv[0], Mv[1], Mv[2]]
        dparts[d] = dMv[d]
        Gv = sum(outer(*[dparts[e] if e == k else parts[e] for e in range(3)]) for k in range(3))
        H[:, d] = q * np.sum(Gv * ph + outer(*parts) * phv, axis=(1, 2, 3))
    return E, F, H


def spme_hvp(x, q, box, K, p, beta, v, f=F_COULOMB):
    """H v of the reciprocal-space energy (see spme)."""
    return spme(x, q, box, K, p, beta, f, v=v)[2]


def ewald_recip(x, q, box, beta, mmax, f=F_COULOMB):
    """Direct reciprocal-space Ewald sum over |m_d| <= mmax[d]: energy and forces."""
    x = np.asarray(x, float)
    box = np.asarray(box, float)
    V = float(np.prod(box))
    g = [np.arange(-mmax[d], mmax[d] + 1) / box[d] for d in range(3)]
    m = np.stack(np.meshgrid(*g, indexing="ij"), -1).reshape(-1, 3)
    m = m[np.any(m != 0, axis=1)]
    m2 = np.sum(m * m, 1)
    a = f * np.exp(-np.pi ** 2 * m2 / beta ** 2) / (2.0 * np.pi * V * m2)
    ph = 2.0 * np.pi * x @ m.T                                            # (Q, M)
    S = q @ np.exp(1j * ph)                                               # structure factors
    E = float(np.sum(a * np.abs(S) ** 2))
    # F_i = -dE/dx_i = 4 pi sum_m a m q_i Im(exp(i 2 pi m.x_i) conj(S))
    t = q[:, None] * np.imag(np.exp(1j * ph) * np.conj(S)[None, :]) * a[None, :]
    F = 4.0 * np.pi * t @ m
    return E, F
