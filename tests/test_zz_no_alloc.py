"""mop_spring_energy_noalloc: the spring energy for callers that cannot allocate device memory
(for example code replayed inside another framework's CUDA graph, or a plug-in whose host owns
all allocations).  It must agree with the spring energy mop_veff_and_grad reports, call after
call, while using only its fixed static scratch array.  This file is collected last."""
import ctypes as C

import numpy as np
import pytest

from paper_2501_11962_b300 import mop
from tests.conftest import workload

TOL_V = 1e-6   # the V_eff / energy tolerance of the parity tests

pytestmark = pytest.mark.gpu


def test_spring_energy_noalloc_matches_engine_twice():
    import torch
    w = workload(2, n_beads=16)
    X = w.paths[0]
    N = X.shape[0]
    eng = mop.Engine(w.system)
    eng.set_path(0, X)
    eng.veff_and_grad(0)
    ref = eng.energies(0)["Espring"]
    eta = torch.tensor(eng.get_field(0, mop.MOP_FIELD_ETA)[:N - 1], device="cuda", dtype=torch.float64)
    mass = torch.tensor(w.system.mass, device="cuda", dtype=torch.float64)
    out = torch.empty(1, device="cuda", dtype=torch.float64)
    lib = mop.load()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        out.fill_(float("nan"))   # the entry point must overwrite whatever the output held
        st = lib.mop_spring_energy_noalloc(C.c_void_p(eta.data_ptr()), C.c_void_p(mass.data_ptr()), N - 1,
                                           w.system.n_atoms, w.system.dt_path, w.system.nu_path,
                                           C.c_void_p(out.data_ptr()), stream)
        assert st == mop.MOP_OK
        torch.cuda.synchronize()
        got = out.item()
        assert abs(got - ref) / abs(ref) < TOL_V, (got, ref)


def test_spring_energy_noalloc_rejects_oversized_input():
    import torch
    lib = mop.load()
    t = torch.zeros(3, device="cuda", dtype=torch.float64)
    p = C.c_void_p(t.data_ptr())
    # 65,537 tiles of 256 atoms exceed the 65,536 partial sums of the static array
    st = lib.mop_spring_energy_noalloc(p, p, 1, 65537 * 256, 0.002, 5.0, p, None)
    assert st == mop.MOP_ERR_ARG


def test_spring_energy_noalloc_at_the_spring_limit():
    """65,536 springs of 256 atoms: exactly the 65,536 block sums the static array holds, with
    more springs than one grid dimension of 65,535 could carry."""
    import torch
    lib = mop.load()
    S, Q = 65536, 256
    g = torch.Generator(device="cpu").manual_seed(1234)
    eta_h = torch.randn(S, Q, 3, generator=g, dtype=torch.float64) * 0.01
    mass_h = torch.rand(Q, generator=g, dtype=torch.float64) * 30.0 + 1.0
    dt, nu = 0.002, 5.0
    K = mass_h.numpy() * nu / (2.0 * dt)
    ref = float(np.sum(0.5 * K[None, :] * np.sum(eta_h.numpy() ** 2, axis=2)))
    eta, mass = eta_h.cuda(), mass_h.cuda()
    out = torch.empty(1, device="cuda", dtype=torch.float64)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        out.fill_(float("nan"))
        st = lib.mop_spring_energy_noalloc(C.c_void_p(eta.data_ptr()), C.c_void_p(mass.data_ptr()), S, Q, dt, nu,
                                           C.c_void_p(out.data_ptr()), stream)
        assert st == mop.MOP_OK
        torch.cuda.synchronize()
        assert abs(out.item() - ref) / abs(ref) < 1e-12, (out.item(), ref)
    # one spring more does not fit
    st = lib.mop_spring_energy_noalloc(C.c_void_p(eta.data_ptr()), C.c_void_p(mass.data_ptr()), S + 1, Q, dt, nu,
                                       C.c_void_p(out.data_ptr()), stream)
    assert st == mop.MOP_ERR_ARG


def test_spring_energy_noalloc_rejects_the_largest_atom_count():
    """n_atoms = 2^31 - 1 must be rejected by the size check (no 32-bit overflow of the tile
    count), before any memory is touched."""
    import torch
    lib = mop.load()
    t = torch.zeros(3, device="cuda", dtype=torch.float64)
    p = C.c_void_p(t.data_ptr())
    st = lib.mop_spring_energy_noalloc(p, p, 1, 2**31 - 1, 0.002, 5.0, p, None)
    assert st == mop.MOP_ERR_ARG
