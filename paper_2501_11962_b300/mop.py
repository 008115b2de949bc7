"""Thin ctypes binding of libmop.so (include/mop.h) and a torch.autograd.Function.

Argument marshalling only: every step of the evaluation runs in the CUDA library.  When the
library cannot be loaded, every call raises; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

import numpy as np

from . import build as _build

MOP_OK, MOP_ERR_ARG, MOP_ERR_CUDA, MOP_ERR_OOM, MOP_ERR_NONFINITE, MOP_ERR_BOX, MOP_ERR_STATE, MOP_ERR_TIMEOUT = range(8)
STATUS_NAMES = ["MOP_OK", "MOP_ERR_ARG", "MOP_ERR_CUDA", "MOP_ERR_OOM", "MOP_ERR_NONFINITE", "MOP_ERR_BOX",
                "MOP_ERR_STATE", "MOP_ERR_TIMEOUT"]
MOP_SHIFTED_FORCE, MOP_POT_SHIFT = 0, 1
MOP_HVP_ADJOINT, MOP_HVP_FD = 0, 1
MOP_PREC_MIXED, MOP_PREC_FP64 = 0, 1
MOP_DEVPTR, MOP_INPUT_F64, MOP_E2E, MOP_COM, MOP_ASYNC = 1, 2, 4, 8, 16
MOP_ELEC_RF, MOP_ELEC_PME = 0, 1
MOP_FIELD_FORCE, MOP_FIELD_ETA, MOP_FIELD_HETA = 0, 1, 2

EXPORTS = ("mop_create", "mop_destroy", "mop_set_path", "mop_get_path", "mop_veff_and_grad", "mop_get_field",
           "mop_get_energies", "mop_add_bias", "mop_step", "mop_kinetic_energy", "mop_last_launch_count",
           "mop_set_profiling", "mop_last_pass_ms", "mop_count_pairs", "mop_spring_energy_noalloc",
           "mop_set_graph_mode", "mop_set_tuning", "mop_get_tuning", "mop_autotune", "mop_measure_fp32_peak",
           "mop_metadynamics", "mop_get_gaussians", "mop_add_cv", "mop_add_gaussian",
           "mop_set_list_skin", "mop_get_list_stats", "mop_get_list_overflows", "mop_wait", "mop_last_error")


class MopError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {msg}")


class mop_tuning(C.Structure):
    _fields_ = [("col_factor", C.c_double), ("bin_factor", C.c_double)]


class mop_system_desc(C.Structure):
    _fields_ = [
        ("n_atoms", C.c_int32), ("box", C.c_double * 3),
        ("type", C.c_void_p), ("n_types", C.c_int32), ("lj_sigma", C.c_void_p), ("lj_eps", C.c_void_p),
        ("charge", C.c_void_p), ("mass", C.c_void_p), ("mol_id", C.c_void_p), ("mol_local", C.c_void_p),
        ("n_bonds", C.c_int32), ("bond_ij", C.c_void_p), ("bond_r0", C.c_void_p), ("bond_k", C.c_void_p),
        ("n_angles", C.c_int32), ("angle_ijk", C.c_void_p), ("angle_th0", C.c_void_p), ("angle_k", C.c_void_p),
        ("rc", C.c_double), ("eps_rf", C.c_double), ("cutoff_mode", C.c_int32),
        ("dt_path", C.c_double), ("nu_path", C.c_double), ("temperature", C.c_double),
        ("hvp_mode", C.c_int32), ("fd_h", C.c_double), ("precision", C.c_int32),
        ("elec", C.c_int32), ("ew_beta", C.c_double), ("pme_grid", C.c_int32 * 3), ("pme_order", C.c_int32),
    ]


_lib = None


def lib_path() -> Path:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load libmop.so (compiling it first when stale and nvcc is available)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_needed:
        try:
            _build.build()
        except (FileNotFoundError, OSError):
            if not _build.LIB.exists():
                raise
    L = C.CDLL(str(_build.LIB))
    p, i32, d = C.c_void_p, C.c_int32, C.c_double
    L.mop_create.argtypes = [p, C.c_int, C.POINTER(p)]
    L.mop_destroy.argtypes = [p]
    L.mop_set_path.argtypes = [p, i32, i32, p, i32, p]
    L.mop_get_path.argtypes = [p, i32, p, i32, p]
    L.mop_veff_and_grad.argtypes = [p, i32, p, p, i32, p]
    L.mop_get_field.argtypes = [p, i32, i32, p, i32, p]
    L.mop_get_energies.argtypes = [p, i32, p]
    L.mop_add_bias.argtypes = [p, p, i32, p, i32, d, d, d, i32, i32]
    L.mop_step.argtypes = [p, i32, d, d, C.c_uint64, p]
    L.mop_metadynamics.argtypes = [p, i32, i32, d, d, C.c_uint64, d, d, p]
    L.mop_get_gaussians.argtypes = [p, i32, p, p, p, i32, p, p]
    L.mop_add_cv.argtypes = [p, i32, p, i32, p, i32, i32, d, p]
    L.mop_add_gaussian.argtypes = [p, i32, d, p, p]
    L.mop_kinetic_energy.argtypes = [p, i32, p]
    L.mop_last_launch_count.argtypes = [p]
    L.mop_last_launch_count.restype = i32
    L.mop_set_profiling.argtypes = [p, i32]
    L.mop_last_pass_ms.argtypes = [p, p, i32]
    L.mop_count_pairs.argtypes = [p, i32, p, p]
    L.mop_spring_energy_noalloc.argtypes = [p, p, i32, i32, d, d, p, p]
    L.mop_set_graph_mode.argtypes = [p, i32]
    L.mop_set_tuning.argtypes = [p, p]
    L.mop_get_tuning.argtypes = [p, p]
    L.mop_autotune.argtypes = [p, i32, p, p]
    L.mop_set_list_skin.argtypes = [p, d]
    L.mop_get_list_stats.argtypes = [p, i32, p, p]
    L.mop_get_list_overflows.argtypes = [p, i32, p]
    L.mop_last_error.argtypes = [p]
    L.mop_last_error.restype = C.c_char_p
    for name in EXPORTS:
        if name not in ("mop_last_launch_count", "mop_last_error"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _np_ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def _stream_ptr(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(int(stream))


class Engine:
    """One mop_handle: a system on one GPU plus up to 64 paths."""

    def __init__(self, system, hvp_mode: int = MOP_HVP_ADJOINT, precision: int = MOP_PREC_MIXED,
                 fd_h: float = 1e-5, device: int = 0):
        self.L = load()
        s = system
        self.system = s
        self.Q = s.n_atoms
        self.precision = precision
        keep = dict(
            type=np.ascontiguousarray(s.type, np.int32), sigma=np.ascontiguousarray(s.lj_sigma, np.float64),
            eps=np.ascontiguousarray(s.lj_eps, np.float64), charge=np.ascontiguousarray(s.charge, np.float64),
            mass=np.ascontiguousarray(s.mass, np.float64), mol=np.ascontiguousarray(s.mol_id, np.int32),
            loc=np.ascontiguousarray(s.mol_local, np.int32),
            bij=np.ascontiguousarray(s.bond_ij, np.int32).reshape(-1), br0=np.ascontiguousarray(s.bond_r0, np.float64),
            bk=np.ascontiguousarray(s.bond_k, np.float64),
            aijk=np.ascontiguousarray(s.angle_ijk, np.int32).reshape(-1),
            ath=np.ascontiguousarray(s.angle_th0, np.float64), ak=np.ascontiguousarray(s.angle_k, np.float64))
        d = mop_system_desc()
        d.n_atoms = self.Q
        for k in range(3):
            d.box[k] = float(s.box[k])
        d.type, d.n_types = keep["type"].ctypes.data, s.n_types
        d.lj_sigma, d.lj_eps = keep["sigma"].ctypes.data, keep["eps"].ctypes.data
        d.charge, d.mass = keep["charge"].ctypes.data, keep["mass"].ctypes.data
        d.mol_id, d.mol_local = keep["mol"].ctypes.data, keep["loc"].ctypes.data
        d.n_bonds = int(s.bond_ij.shape[0])
        d.bond_ij, d.bond_r0, d.bond_k = keep["bij"].ctypes.data, keep["br0"].ctypes.data, keep["bk"].ctypes.data
        d.n_angles = int(s.angle_ijk.shape[0])
        d.angle_ijk, d.angle_th0, d.angle_k = keep["aijk"].ctypes.data, keep["ath"].ctypes.data, keep["ak"].ctypes.data
        d.rc, d.eps_rf, d.cutoff_mode = float(s.rc), float(s.eps_rf), int(s.cutoff_mode)
        d.dt_path, d.nu_path, d.temperature = float(s.dt_path), float(s.nu_path), float(s.temperature)
        d.hvp_mode, d.fd_h, d.precision = int(hvp_mode), float(fd_h), int(precision)
        d.elec, d.ew_beta = int(getattr(s, "elec", MOP_ELEC_RF)), float(getattr(s, "ew_beta", 0.0))
        for k, g in enumerate(getattr(s, "pme_grid", (0, 0, 0))):
            d.pme_grid[k] = int(g)
        d.pme_order = int(getattr(s, "pme_order", 4))
        h = C.c_void_p()
        st = self.L.mop_create(C.byref(d), device, C.byref(h))
        if st != MOP_OK:
            raise MopError(st, "mop_create rejected the system description")
        self.h = h
        self.n_beads = {}

    def close(self):
        if getattr(self, "h", None):
            self.L.mop_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int, what: str):
        if st != MOP_OK:
            msg = self.L.mop_last_error(self.h)
            raise MopError(st, f"{what}: {msg.decode() if msg else ''}")

    # ---- paths --------------------------------------------------------------------------
    def set_path(self, path_id: int, xyz, stream=None):
        """xyz: [N, Q, 3] float32/float64 numpy array (host) or CUDA tensor (device)."""
        if isinstance(xyz, np.ndarray):
            a = np.ascontiguousarray(xyz)
            flags = MOP_INPUT_F64 if a.dtype == np.float64 else 0
            if a.dtype not in (np.float32, np.float64):
                a = a.astype(np.float32)
            st = self.L.mop_set_path(self.h, path_id, a.shape[0], _np_ptr(a), flags, None)
        else:
            t = xyz.contiguous()
            flags = MOP_DEVPTR | (MOP_INPUT_F64 if str(t.dtype) == "torch.float64" else 0)
            st = self.L.mop_set_path(self.h, path_id, t.shape[0], C.c_void_p(t.data_ptr()), flags,
                                     _stream_ptr(stream))
            self._keep_alive = t
        self._check(st, "mop_set_path")
        self.n_beads[path_id] = int(xyz.shape[0])

    def get_path(self, path_id: int) -> np.ndarray:
        out = np.empty((self.n_beads[path_id], self.Q, 3), np.float32)
        self._check(self.L.mop_get_path(self.h, path_id, _np_ptr(out), 0, None), "mop_get_path")
        return out

    def veff_and_grad(self, path_id: int = -1, want_grad: bool = True):
        """Host call: returns (veff array [P], grad array [sum N, Q, 3] or None)."""
        ids = [path_id] if path_id >= 0 else sorted(self.n_beads)
        nb = sum(self.n_beads.get(i, 0) for i in ids)
        v = np.empty(len(ids))
        g = np.empty((nb, self.Q, 3)) if want_grad else None
        st = self.L.mop_veff_and_grad(self.h, path_id, _np_ptr(v), _np_ptr(g) if (want_grad and nb) else None, 0,
                                      None)
        self._check(st, "mop_veff_and_grad")
        return v, g

    def veff_and_grad_device(self, veff, grad, path_id: int = -1, stream=None):
        """Device call: veff, grad are CUDA float64 tensors; asynchronous on `stream`."""
        st = self.L.mop_veff_and_grad(self.h, path_id, C.c_void_p(veff.data_ptr()),
                                      C.c_void_p(grad.data_ptr()) if grad is not None else None, MOP_DEVPTR,
                                      _stream_ptr(stream))
        self._check(st, "mop_veff_and_grad")

    def set_path_async(self, path_id: int, xyz, stream=None):
        """Enqueue coordinates from a page-locked float32 host tensor [N, Q, 3] (MOP_ASYNC); the
        tensor must stay untouched until wait()."""
        N = int(xyz.shape[0])
        self._check(self.L.mop_set_path(self.h, path_id, N, C.c_void_p(xyz.data_ptr()), MOP_ASYNC,
                                        _stream_ptr(stream)), "mop_set_path")
        self.n_beads[path_id] = N

    def veff_and_grad_async(self, veff, grad, path_id: int = -1, stream=None):
        """Enqueue an evaluation whose V_eff and gradient land in page-locked float64 host tensors
        (MOP_ASYNC); they are filled when wait() returns."""
        st = self.L.mop_veff_and_grad(self.h, path_id, C.c_void_p(veff.data_ptr()),
                                      C.c_void_p(grad.data_ptr()) if grad is not None else None, MOP_ASYNC,
                                      _stream_ptr(stream))
        self._check(st, "mop_veff_and_grad")

    def wait(self):
        self._check(self.L.mop_wait(self.h), "mop_wait")

    def get_field(self, path_id: int, field: int) -> np.ndarray:
        out = np.empty((self.n_beads[path_id], self.Q, 3))
        self._check(self.L.mop_get_field(self.h, path_id, field, _np_ptr(out), 0, None), "mop_get_field")
        return out

    def energies(self, path_id: int) -> dict:
        out = np.zeros(4)
        self._check(self.L.mop_get_energies(self.h, path_id, _np_ptr(out)), "mop_get_energies")
        return dict(U1=out[0], Espring=out[1], Ebias=out[2], cv=out[3])

    def add_bias(self, path_id: int, s_center: float, height: float, width: float, groups=None, e2e=False,
                 com=False):
        if groups is not None:
            ga = np.ascontiguousarray(groups[0], np.int32)
            gb = np.ascontiguousarray(groups[1], np.int32)
            flags = (MOP_E2E if e2e else 0) | (MOP_COM if com else 0)
            st = self.L.mop_add_bias(self.h, _np_ptr(ga), len(ga), _np_ptr(gb), len(gb), s_center, height, width,
                                     path_id, flags)
        else:
            st = self.L.mop_add_bias(self.h, None, 0, None, 0, s_center, height, width, path_id, 0)
        self._check(st, "mop_add_bias")

    def tuning(self) -> dict:
        t = mop_tuning()
        self._check(self.L.mop_get_tuning(self.h, C.byref(t)), "mop_get_tuning")
        return dict(col_factor=t.col_factor, bin_factor=t.bin_factor)

    def set_tuning(self, col_factor: float, bin_factor: float):
        t = mop_tuning(col_factor, bin_factor)
        self._check(self.L.mop_set_tuning(self.h, C.byref(t)), "mop_set_tuning")

    def autotune(self, path_id: int = 0):
        """Runs mop_autotune; returns (tuning dict, ms per evaluation)."""
        t, ms = mop_tuning(), C.c_double()
        self._check(self.L.mop_autotune(self.h, path_id, C.byref(t), C.byref(ms)), "mop_autotune")
        return dict(col_factor=t.col_factor, bin_factor=t.bin_factor), ms.value

    def set_list_skin(self, skin_nm: float):
        """Verlet skin of the pair lists (0: rebuild at every evaluation)."""
        self._check(self.L.mop_set_list_skin(self.h, float(skin_nm)), "mop_set_list_skin")

    def list_stats(self, path_id: int) -> tuple:
        """(lists built, lists reused) by the evaluations of path_id."""
        b, r = C.c_int64(), C.c_int64()
        self._check(self.L.mop_get_list_stats(self.h, path_id, C.byref(b), C.byref(r)), "mop_get_list_stats")
        return b.value, r.value

    def list_overflows(self, path_id: int) -> int:
        """Graph-mode step batches of path_id run again after a pair list outgrew its capacity."""
        n = C.c_int64()
        self._check(self.L.mop_get_list_overflows(self.h, path_id, C.byref(n)), "mop_get_list_overflows")
        return n.value

    def set_graph_mode(self, on: bool = True):
        self._check(self.L.mop_set_graph_mode(self.h, int(on)), "mop_set_graph_mode")

    def step(self, n_steps: int, dt: float, gamma: float = 0.0, seed: int = 1):
        self._check(self.L.mop_step(self.h, n_steps, dt, gamma, seed, None), "mop_step")

    def gaussians(self, path_id: int):
        """(centers [k][n_cv], heights [k], widths [k][n_cv]) of a path's Gaussians, in the order
        they were added."""
        n, ncv = np.zeros(1, np.int32), np.zeros(1, np.int32)
        self._check(self.L.mop_get_gaussians(self.h, path_id, None, None, None, 0, _np_ptr(n), _np_ptr(ncv)),
                    "mop_get_gaussians")
        k, q = int(n[0]), int(ncv[0])
        c, hh, w = np.zeros((k, q)), np.zeros(k), np.zeros((k, q))
        self._check(self.L.mop_get_gaussians(self.h, path_id, _np_ptr(c), _np_ptr(hh), _np_ptr(w), k, _np_ptr(n),
                                             None), "mop_get_gaussians")
        return c, hh, w

    def add_cv(self, path_id: int, groups, e2e=False, com=False, deposit_width: float = 0.0) -> int:
        """Adds a CV (mop_add_cv); returns its index."""
        ga = np.ascontiguousarray(groups[0], np.int32)
        gb = np.ascontiguousarray(groups[1], np.int32)
        idx = np.zeros(1, np.int32)
        flags = (MOP_E2E if e2e else 0) | (MOP_COM if com else 0)
        self._check(self.L.mop_add_cv(self.h, path_id, _np_ptr(ga), len(ga), _np_ptr(gb), len(gb), flags,
                                      float(deposit_width), _np_ptr(idx)), "mop_add_cv")
        return int(idx[0])

    def add_gaussian(self, path_id: int, height: float, centers, widths):
        """Appends one Gaussian on all CVs of the path (mop_add_gaussian)."""
        c = np.ascontiguousarray(centers, np.float64)
        w = np.ascontiguousarray(widths, np.float64)
        self._check(self.L.mop_add_gaussian(self.h, path_id, float(height), _np_ptr(c), _np_ptr(w)),
                    "mop_add_gaussian")

    def metadynamics(self, n_deposits: int, stride: int, dt: float, gamma: float, seed: int, height: float,
                     width: float):
        """n_deposits rounds of `stride` MD steps, each followed by one Gaussian at the current CV
        of every path with CV groups (mop_metadynamics)."""
        self._check(self.L.mop_metadynamics(self.h, n_deposits, stride, dt, gamma, seed, height, width, None),
                    "mop_metadynamics")

    def kinetic_energy(self, path_id: int) -> float:
        out = np.zeros(1)
        self._check(self.L.mop_kinetic_energy(self.h, path_id, _np_ptr(out)), "mop_kinetic_energy")
        return float(out[0])

    def last_launch_count(self) -> int:
        return int(self.L.mop_last_launch_count(self.h))

    PASSES = ("prep", "pair_force", "bonded_eta", "pair_hvp", "bonded_hvp_grad", "bias_reduce")

    def set_profiling(self, on: bool = True):
        self._check(self.L.mop_set_profiling(self.h, int(on)), "mop_set_profiling")

    def pass_ms(self) -> dict:
        out = np.zeros(6, np.float32)
        self._check(self.L.mop_last_pass_ms(self.h, _np_ptr(out), 6), "mop_last_pass_ms")
        return dict(zip(self.PASSES, out.astype(float).tolist()))

    def count_pairs(self, path_id: int):
        u, l = np.zeros(1, np.int64), np.zeros(1, np.int64)
        self._check(self.L.mop_count_pairs(self.h, path_id, _np_ptr(u), _np_ptr(l)), "mop_count_pairs")
        return int(u[0]), int(l[0])


def measure_fp32_peak(device: int = 0) -> float:
    """Measured FP32 FMA throughput of `device` in TFLOP/s (mop_measure_fp32_peak)."""
    L = load()
    t = np.zeros(1, np.float64)
    st = L.mop_measure_fp32_peak(int(device), _np_ptr(t))
    if st != 0:
        raise MopError(st, "mop_measure_fp32_peak")
    return float(t[0])


def _autograd_function():
    import torch

    class VeffFunction(torch.autograd.Function):
        """V_eff(R) of one path (Eq. 3) with its exact gradient (Eqs. 5-7 with the adjoint HVP).

        forward(coords [N, Q, 3] CUDA float32/float64, engine, path_id) -> 0-dim float64 tensor;
        backward returns grad_out * dV_eff/dR in the dtype of coords.
        """

        @staticmethod
        def forward(ctx, coords, engine, path_id):
            engine.set_path(path_id, coords.detach())
            veff = torch.empty(1, dtype=torch.float64, device=coords.device)
            grad = torch.empty(coords.shape, dtype=torch.float64, device=coords.device)
            engine.veff_and_grad_device(veff, grad, path_id)
            ctx.save_for_backward(grad)
            ctx.in_dtype = coords.dtype
            return veff[0]

        @staticmethod
        def backward(ctx, grad_out):
            (grad,) = ctx.saved_tensors
            return (grad_out * grad).to(ctx.in_dtype), None, None

    return VeffFunction


_VEFF = None


def veff(coords, engine: Engine, path_id: int = 0):
    """Differentiable V_eff of `coords` ([N, Q, 3] CUDA tensor) through `engine`."""
    global _VEFF
    if _VEFF is None:
        _VEFF = _autograd_function()
    return _VEFF.apply(coords, engine, path_id)
