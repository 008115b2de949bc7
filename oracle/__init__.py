"""ctypes front end of the FP64 CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package.  The product path (the CUDA library and its Python binding) never does.
"""
from __future__ import annotations

import ctypes as C
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "oracle.cpp"
_LIB = _HERE / "liboracle.so"

HVP_ANALYTIC = 0
HVP_COMPLEX = 1
HVP_FD_EQ5 = 2


def build(force: bool = False) -> Path:
    """Compile oracle.cpp into liboracle.so (g++ -O2, OpenMP)."""
    if force or not _LIB.exists() or _LIB.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _LIB.with_suffix(".so.tmp")
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-o", str(tmp), str(_SRC)]
        subprocess.run(cmd, check=True)
        tmp.replace(_LIB)
    return _LIB


class OrcSystem(C.Structure):
    _fields_ = [
        ("Q", C.c_int32), ("n_types", C.c_int32), ("box", C.c_double * 3),
        ("type", C.c_void_p), ("sigma", C.c_void_p), ("eps", C.c_void_p),
        ("charge", C.c_void_p), ("mass", C.c_void_p),
        ("mol_id", C.c_void_p), ("mol_local", C.c_void_p),
        ("n_bonds", C.c_int32), ("bond_ij", C.c_void_p), ("bond_r0", C.c_void_p), ("bond_k", C.c_void_p),
        ("n_angles", C.c_int32), ("angle_ijk", C.c_void_p), ("angle_th0", C.c_void_p), ("angle_k", C.c_void_p),
        ("rc", C.c_double), ("eps_rf", C.c_double), ("cutoff_mode", C.c_int32),
        ("dt_path", C.c_double), ("nu_path", C.c_double),
        ("elec", C.c_int32), ("ew_beta", C.c_double),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(str(build()))
        d, i, p = C.c_double, C.c_int, C.c_void_p
        _lib.orc_forces.argtypes = [p, p, p, p, i]
        _lib.orc_forces_complex.argtypes = [p, p, p, d, p, p, p]
        _lib.orc_hvp.argtypes = [p, p, p, p, i, d]
        _lib.orc_hessian_dense.argtypes = [p, p, p]
        _lib.orc_veff.argtypes = [p, i, p, i, d, p, p, p, p, p, p]
        _lib.orc_veff_complex_dir.argtypes = [p, i, p, p, d, p]
        _lib.orc_philox4x32_10.argtypes = [p, p, p]
        _lib.orc_gauss3.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32, p]
        _lib.orc_cv_distance.argtypes = [p, p, p, i, p, i, p, d]
        _lib.orc_cv_distance.restype = d
        _lib.orc_bias.argtypes = [p, i, p, p, i, p, i, i, i, p, p, p, p, p]
        _lib.orc_bias.restype = d
        _lib.orc_step.argtypes = [p, i, p, p, p, d, d, d, C.c_uint64, C.c_uint64, i]
        _lib.orc_step.restype = d
        _lib.orc_cv_com.argtypes = [p, p, p, i, p, i, i, p, d]
        _lib.orc_cv_com.restype = d
        _lib.orc_bias_com.argtypes = [p, i, p, p, i, p, i, i, i, i, p, p, p, p, p]
        _lib.orc_bias_com.restype = d
        _lib.orc_metad.argtypes = [p, i, p, p, d, d, d, C.c_uint64, C.c_uint64, i, i, p, i, p, i, i, i, d, d, i,
                                   p, p, p, i]
        _lib.orc_metad.restype = d
        _lib.orc_bias_multi.argtypes = [p, i, p, i, p, p, p, p, p, p, i, p, p, p, p, p]
        _lib.orc_bias_multi.restype = d
        _lib.orc_metad_multi.argtypes = [p, i, p, p, d, d, d, C.c_uint64, C.c_uint64, i, i, i, p, p, p, p, p, p,
                                         d, p, i, p, p, p, i]
        _lib.orc_metad_multi.restype = d
        _lib.orc_num_threads.restype = i
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class Oracle:
    """Holds the contiguous parameter arrays of one system and calls the C++ oracle."""

    def __init__(self, system):
        s = system
        self.system = s
        self.Q = s.n_atoms
        keep = dict(
            type=np.ascontiguousarray(s.type, np.int32),
            sigma=np.ascontiguousarray(s.lj_sigma, np.float64),
            eps=np.ascontiguousarray(s.lj_eps, np.float64),
            charge=np.ascontiguousarray(s.charge, np.float64),
            mass=np.ascontiguousarray(s.mass, np.float64),
            mol_id=np.ascontiguousarray(s.mol_id, np.int32),
            mol_local=np.ascontiguousarray(s.mol_local, np.int32),
            bond_ij=np.ascontiguousarray(s.bond_ij, np.int32).reshape(-1),
            bond_r0=np.ascontiguousarray(s.bond_r0, np.float64),
            bond_k=np.ascontiguousarray(s.bond_k, np.float64),
            angle_ijk=np.ascontiguousarray(s.angle_ijk, np.int32).reshape(-1),
            angle_th0=np.ascontiguousarray(s.angle_th0, np.float64),
            angle_k=np.ascontiguousarray(s.angle_k, np.float64),
        )
        self._keep = keep
        st = OrcSystem()
        st.Q = self.Q
        st.n_types = s.n_types
        for k in range(3):
            st.box[k] = float(s.box[k])
        for name in ("type", "sigma", "eps", "charge", "mass", "mol_id", "mol_local",
                     "bond_ij", "bond_r0", "bond_k", "angle_ijk", "angle_th0", "angle_k"):
            setattr(st, name, keep[name].ctypes.data)
        st.n_bonds = int(s.bond_ij.shape[0])
        st.n_angles = int(s.angle_ijk.shape[0])
        st.rc = float(s.rc)
        st.eps_rf = float(s.eps_rf)
        st.cutoff_mode = int(s.cutoff_mode)
        st.dt_path = float(s.dt_path)
        st.nu_path = float(s.nu_path)
        st.elec = int(getattr(s, "elec", 0))
        st.ew_beta = float(getattr(s, "ew_beta", 0.0))
        self._st = st
        self._sp = C.cast(C.pointer(st), C.c_void_p)
        self.L = lib()

    # --- single configuration -----------------------------------------------------------
    def forces(self, x, method: int = 0):
        x = np.ascontiguousarray(x, np.float64).reshape(self.Q, 3)
        F = np.zeros((self.Q, 3))
        U = np.zeros(1)
        self.L.orc_forces(self._sp, _ptr(x), _ptr(F), _ptr(U), method)
        return F, float(U[0])

    def forces_complex(self, x, v, h):
        x = np.ascontiguousarray(x, np.float64).reshape(self.Q, 3)
        v = np.ascontiguousarray(v, np.float64).reshape(self.Q, 3)
        Fr, Fi, Uc = np.zeros((self.Q, 3)), np.zeros((self.Q, 3)), np.zeros(2)
        self.L.orc_forces_complex(self._sp, _ptr(x), _ptr(v), float(h), _ptr(Fr), _ptr(Fi), _ptr(Uc))
        return Fr, Fi, Uc

    def hvp(self, x, v, mode: int = HVP_ANALYTIC, h: float = 0.0):
        x = np.ascontiguousarray(x, np.float64).reshape(self.Q, 3)
        v = np.ascontiguousarray(v, np.float64).reshape(self.Q, 3)
        out = np.zeros((self.Q, 3))
        self.L.orc_hvp(self._sp, _ptr(x), _ptr(v), _ptr(out), mode, float(h))
        return out

    def hessian(self, x):
        x = np.ascontiguousarray(x, np.float64).reshape(self.Q, 3)
        H = np.zeros((3 * self.Q, 3 * self.Q))
        self.L.orc_hessian_dense(self._sp, _ptr(x), _ptr(H))
        return H

    # --- paths --------------------------------------------------------------------------
    def veff(self, X, hvp_mode: int = HVP_ANALYTIC, fd_h: float = 0.0, want=("G",)):
        X = np.ascontiguousarray(X, np.float64)
        N = X.shape[0]
        shp = (N, self.Q, 3)
        out = {k: (np.zeros(shp) if k in want else None) for k in ("G", "F", "eta", "Heta")}
        v = np.zeros(1)
        parts = np.zeros(2)
        self.L.orc_veff(self._sp, N, _ptr(X), hvp_mode, float(fd_h), _ptr(v), _ptr(out["G"]), _ptr(out["F"]),
                        _ptr(out["eta"]), _ptr(out["Heta"]), _ptr(parts))
        res = {k: a for k, a in out.items() if a is not None}
        res.update(veff=float(v[0]), U1=float(parts[0]), Espring=float(parts[1]))
        return res

    # --- Ewald electrostatics (ELEC_PME): real space, exclusions and self term in the C++ code,
    # reciprocal space by SPME in numpy (oracle/pme.py)
    def recip(self, x, v=None):
        """Reciprocal-space energy and forces (and H v with a direction v) of one configuration."""
        from . import pme
        s = self.system
        return pme.spme(np.asarray(x, np.float64), np.asarray(s.charge, np.float64), s.box, s.pme_grid,
                        s.pme_order, s.ew_beta, v=v)

    def veff_pme(self, X):
        """V_eff (Eq. 3) and its exact gradient (Eqs. 5-7, FD term replaced by -H eta / 2) with
        Ewald electrostatics: per bead F = F_real+bonded + F_recip, H eta likewise."""
        s = self.system
        X = np.ascontiguousarray(X, np.float64)
        N = X.shape[0]
        m = np.asarray(s.mass, np.float64)[:, None]
        K = m * s.nu_path / (2.0 * s.dt_path)
        c = s.dt_path / (m * s.nu_path)
        n_force = 1 if N == 1 else N - 1
        F = np.zeros_like(X)
        U1 = 0.0
        for n in range(n_force):
            Fr, Ur = self.forces(X[n])
            Er, Fk = self.recip(X[n])
            F[n] = Fr + Fk
            if n == 0:
                U1 = Ur + Er
        eta = np.zeros_like(X)
        Heta = np.zeros_like(X)
        for n in range(N - 1):
            eta[n] = X[n + 1] - X[n] - c * F[n]
            Heta[n] = self.hvp(X[n], eta[n]) + self.recip(X[n], v=eta[n])[2]
        Es = float(np.sum(0.5 * K * eta[:N - 1] ** 2))
        G = np.zeros_like(X)
        if N == 1:
            G[0] = -F[0]
        else:
            G[0] = -F[0] - K * eta[0] + 0.5 * Heta[0]
            for n in range(1, N - 1):
                G[n] = K * eta[n - 1] - K * eta[n] + 0.5 * Heta[n]
            G[N - 1] = K * eta[N - 2]
        return dict(veff=U1 + Es, U1=U1, Espring=Es, G=G, F=F, eta=eta, Heta=Heta)

    def veff_complex_dir(self, X, D, h: float = 1e-20) -> float:
        X = np.ascontiguousarray(X, np.float64)
        D = np.ascontiguousarray(D, np.float64)
        out = np.zeros(1)
        self.L.orc_veff_complex_dir(self._sp, X.shape[0], _ptr(X), _ptr(D), float(h), _ptr(out))
        return float(out[0])

    def cv_distance(self, x, ga, gb):
        x = np.ascontiguousarray(x, np.float64)
        ga = np.ascontiguousarray(ga, np.int32)
        gb = np.ascontiguousarray(gb, np.int32)
        ds = np.zeros((self.Q, 3))
        s = self.L.orc_cv_distance(self._sp, _ptr(x), _ptr(ga), len(ga), _ptr(gb), len(gb), _ptr(ds), 1.0)
        return s, ds

    def bias(self, X, ga, gb, centers, heights, widths, e2e: bool = False):
        X = np.ascontiguousarray(X, np.float64)
        ga = np.ascontiguousarray(ga, np.int32)
        gb = np.ascontiguousarray(gb, np.int32)
        c = np.ascontiguousarray(centers, np.float64)
        h = np.ascontiguousarray(heights, np.float64)
        w = np.ascontiguousarray(widths, np.float64)
        G = np.zeros(X.shape)
        cv = np.zeros(1)
        V = self.L.orc_bias(self._sp, X.shape[0], _ptr(X), _ptr(ga), len(ga), _ptr(gb), len(gb), int(e2e),
                            len(c), _ptr(c), _ptr(h), _ptr(w), _ptr(G), _ptr(cv))
        return V, G, float(cv[0])

    def cv_com(self, x, ga, gb, com: bool):
        """CV with optional mass weighting (orc_cv_com): s and ds/dx [Q][3]."""
        x = np.ascontiguousarray(x, np.float64)
        ga = np.ascontiguousarray(ga, np.int32)
        gb = np.ascontiguousarray(gb, np.int32)
        ds = np.zeros((self.Q, 3))
        s = self.L.orc_cv_com(self._sp, _ptr(x), _ptr(ga), len(ga), _ptr(gb), len(gb), int(com), _ptr(ds), 1.0)
        return s, ds

    def bias_com(self, X, ga, gb, centers, heights, widths, e2e: bool = False, com: bool = False):
        X = np.ascontiguousarray(X, np.float64)
        ga = np.ascontiguousarray(ga, np.int32)
        gb = np.ascontiguousarray(gb, np.int32)
        c = np.ascontiguousarray(centers, np.float64)
        h = np.ascontiguousarray(heights, np.float64)
        w = np.ascontiguousarray(widths, np.float64)
        G = np.zeros(X.shape)
        cv = np.zeros(1)
        V = self.L.orc_bias_com(self._sp, X.shape[0], _ptr(X), _ptr(ga), len(ga), _ptr(gb), len(gb), int(e2e),
                                int(com), len(c), _ptr(c), _ptr(h), _ptr(w), _ptr(G), _ptr(cv))
        return V, G, float(cv[0])

    def metad(self, X, Vel, dt, gamma, temperature, seed, step0, n_deposits, stride, ga, gb, height, width,
              e2e=False, com=False, gaussians=None, round_f32=True):
        """Metadynamics of paths (orc_metad), X and Vel updated in place.  Returns V_eff + V_bias
        at the final positions and the Gaussians (centers, heights, widths) after the run."""
        ga = np.ascontiguousarray(ga, np.int32)
        gb = np.ascontiguousarray(gb, np.int32)
        g0 = [] if gaussians is None else list(zip(*gaussians))
        n0 = len(g0)
        c = np.zeros(n0 + n_deposits)
        h = np.zeros(n0 + n_deposits)
        w = np.zeros(n0 + n_deposits)
        for k, (ck, hk, wk) in enumerate(g0):
            c[k], h[k], w[k] = ck, hk, wk
        V = self.L.orc_metad(self._sp, X.shape[0], _ptr(X), _ptr(Vel), float(dt), float(gamma), float(temperature),
                             int(seed), int(step0), int(n_deposits), int(stride), _ptr(ga), len(ga), _ptr(gb),
                             len(gb), int(e2e), int(com), float(height), float(width), n0, _ptr(c), _ptr(h),
                             _ptr(w), int(round_f32))
        return V, (c, h, w)

    @staticmethod
    def _cv_arrays(cvs):
        """cvs: [(group A, group B, e2e, com), ...] -> concatenated groups, offsets and flags."""
        ga = np.concatenate([np.asarray(c[0], np.int32) for c in cvs]).astype(np.int32)
        gb = np.concatenate([np.asarray(c[1], np.int32) for c in cvs]).astype(np.int32)
        ga_off = np.concatenate([[0], np.cumsum([len(c[0]) for c in cvs])]).astype(np.int32)
        gb_off = np.concatenate([[0], np.cumsum([len(c[1]) for c in cvs])]).astype(np.int32)
        e2e = np.asarray([int(bool(c[2])) for c in cvs], np.int32)
        com = np.asarray([int(bool(c[3])) for c in cvs], np.int32)
        return ga, ga_off, gb, gb_off, e2e, com

    def bias_multi(self, X, cvs, centers, widths, heights):
        """Multi-CV bias (orc_bias_multi): returns V_b, dV_b/dX and the CV values."""
        X = np.ascontiguousarray(X, np.float64)
        arrs = self._cv_arrays(cvs)
        n = len(cvs)
        c = np.ascontiguousarray(np.reshape(centers, (-1, n)), np.float64)
        w = np.ascontiguousarray(np.reshape(widths, (-1, n)), np.float64)
        h = np.ascontiguousarray(heights, np.float64)
        G = np.zeros(X.shape)
        cv = np.zeros(n)
        V = self.L.orc_bias_multi(self._sp, X.shape[0], _ptr(X), n, *[_ptr(a) for a in arrs], len(h), _ptr(c),
                                  _ptr(w), _ptr(h), _ptr(G), _ptr(cv))
        return V, G, cv

    def metad_multi(self, X, Vel, dt, gamma, temperature, seed, step0, n_deposits, stride, cvs, height, dep_widths,
                    gaussians=None, round_f32=True):
        """Multi-CV metadynamics (orc_metad_multi), X and Vel in place.  gaussians = (centers [k][n],
        widths [k][n], heights [k]) already present.  Returns V and the Gaussians after the run."""
        arrs = self._cv_arrays(cvs)
        n = len(cvs)
        k0 = 0 if gaussians is None else len(gaussians[2])
        c = np.zeros((k0 + n_deposits, n))
        w = np.zeros((k0 + n_deposits, n))
        h = np.zeros(k0 + n_deposits)
        if k0:
            c[:k0], w[:k0], h[:k0] = np.reshape(gaussians[0], (k0, n)), np.reshape(gaussians[1], (k0, n)), gaussians[2]
        dw = np.ascontiguousarray(dep_widths, np.float64)
        V = self.L.orc_metad_multi(self._sp, X.shape[0], _ptr(X), _ptr(Vel), float(dt), float(gamma),
                                   float(temperature), int(seed), int(step0), int(n_deposits), int(stride), n,
                                   *[_ptr(a) for a in arrs], float(height), _ptr(dw), k0, _ptr(c), _ptr(w), _ptr(h),
                                   int(round_f32))
        return V, (c, w, h)

    def step(self, X, V, G, dt, gamma, temperature, seed, step, round_f32=True):
        """One BAOAB / velocity-Verlet step in place; returns V_eff at the new positions."""
        return self.L.orc_step(self._sp, X.shape[0], _ptr(X), _ptr(V), _ptr(G), float(dt), float(gamma),
                               float(temperature), int(seed), int(step), int(round_f32))


def philox4x32_10(counter, key):
    c = np.ascontiguousarray(counter, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def gauss3(seed, step, bead, atom):
    out = np.zeros(3)
    lib().orc_gauss3(int(seed), int(step), int(bead), int(atom), _ptr(out))
    return out


def num_threads() -> int:
    return int(lib().orc_num_threads())
