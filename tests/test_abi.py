"""The C-ABI library builds, loads and exports every symbol include/mop.h declares; host-side
validation of mop_create runs without a GPU."""
import ctypes as C
import re
from pathlib import Path

import numpy as np
import pytest

from paper_2501_11962_b300 import mop, synth

HEADER = Path(__file__).resolve().parents[1] / "include" / "mop.h"


def declared_functions():
    text = HEADER.read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mop_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_function():
    lib = mop.load()
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(mop.EXPORTS) == names


def _desc(system, **over):
    eng_keep = {}
    s = system
    arrs = dict(
        type=np.ascontiguousarray(s.type, np.int32), sigma=np.ascontiguousarray(s.lj_sigma),
        eps=np.ascontiguousarray(s.lj_eps), charge=np.ascontiguousarray(s.charge),
        mass=np.ascontiguousarray(s.mass), mol=np.ascontiguousarray(s.mol_id, np.int32),
        loc=np.ascontiguousarray(s.mol_local, np.int32))
    arrs.update({k: v for k, v in over.items() if isinstance(v, np.ndarray)})
    d = mop.mop_system_desc()
    d.n_atoms = s.n_atoms
    for k in range(3):
        d.box[k] = float(over.get("box", s.box)[k])
    d.type, d.n_types = arrs["type"].ctypes.data, over.get("n_types", s.n_types)
    d.lj_sigma, d.lj_eps = arrs["sigma"].ctypes.data, arrs["eps"].ctypes.data
    d.charge, d.mass = arrs["charge"].ctypes.data, arrs["mass"].ctypes.data
    d.mol_id, d.mol_local = arrs["mol"].ctypes.data, arrs["loc"].ctypes.data
    d.rc, d.eps_rf, d.cutoff_mode = over.get("rc", s.rc), over.get("eps_rf", 78.0), 0
    d.dt_path, d.nu_path, d.temperature = 0.002, 5.0, 300.0
    d.hvp_mode, d.fd_h, d.precision = over.get("hvp_mode", 0), 1e-5, 0
    eng_keep["arrs"] = arrs
    return d, eng_keep


def _create(d):
    h = C.c_void_p()
    st = mop.load().mop_create(C.byref(d), 0, C.byref(h))
    if st == mop.MOP_OK:
        mop.load().mop_destroy(h)
    return st


@pytest.fixture(scope="module")
def fcc():
    return synth.lj_fcc()[0]


def test_create_rejects_cutoff_beyond_half_box(fcc):
    d, keep = _desc(fcc, rc=1.2)   # box 2.33 nm
    assert _create(d) == mop.MOP_ERR_BOX


def test_create_rejects_nonfinite_parameters(fcc):
    m = np.ascontiguousarray(fcc.mass.copy())
    m[3] = np.nan
    d, keep = _desc(fcc, mass=m)
    assert _create(d) == mop.MOP_ERR_NONFINITE


def test_create_rejects_bad_type_and_mass(fcc):
    t = np.ascontiguousarray(fcc.type.copy())
    t[0] = 5
    d, keep = _desc(fcc, type=t)
    assert _create(d) == mop.MOP_ERR_ARG
    m = np.ascontiguousarray(fcc.mass.copy())
    m[0] = -1.0
    d, keep = _desc(fcc, mass=m)
    assert _create(d) == mop.MOP_ERR_ARG
    d, keep = _desc(fcc, hvp_mode=7)
    assert _create(d) == mop.MOP_ERR_ARG


def test_null_handle_calls_fail_cleanly():
    lib = mop.load()
    assert lib.mop_destroy(None) == mop.MOP_OK
    assert lib.mop_veff_and_grad(None, 0, None, None, 0, None) == mop.MOP_ERR_ARG
    assert lib.mop_last_launch_count(None) == 0
    assert lib.mop_last_error(None) == b"null handle"
    assert lib.mop_count_pairs(None, 0, None, None) == mop.MOP_ERR_ARG
    assert lib.mop_set_profiling(None, 1) == mop.MOP_ERR_ARG


def _pme(d, grid=(24, 24, 24), order=4, beta=3.0, hvp=0):
    d.elec, d.ew_beta, d.pme_order, d.hvp_mode = mop.MOP_ELEC_PME, beta, order, hvp
    for k in range(3):
        d.pme_grid[k] = grid[k]
    return d


def test_create_validates_the_ewald_parameters(fcc):
    d, keep = _desc(fcc, rc=1.0)
    # the finite-difference HVP has no reciprocal-space counterpart; a grid-free Ewald is fine to check
    assert _create(_pme(d, hvp=1)) == mop.MOP_ERR_ARG
    # odd B-spline orders need odd grids (the moduli vanish at an even grid's Nyquist frequency)
    assert _create(_pme(d, order=5)) == mop.MOP_ERR_ARG
    assert _create(_pme(d, order=3)) == mop.MOP_ERR_ARG
    assert _create(_pme(d, order=9, grid=(25, 25, 25))) == mop.MOP_ERR_ARG
    assert _create(_pme(d, grid=(24, 3, 24))) == mop.MOP_ERR_ARG
    assert _create(_pme(d, beta=-1.0)) == mop.MOP_ERR_ARG
    assert _create(_pme(d, beta=float("nan"))) == mop.MOP_ERR_ARG
    # Ewald runs in mixed precision only
    d.precision = mop.MOP_PREC_FP64
    assert _create(_pme(d)) == mop.MOP_ERR_ARG


def test_create_rejects_an_empty_system(fcc):
    d, keep = _desc(fcc)
    d.n_atoms = 0
    assert _create(d) == mop.MOP_ERR_ARG
