"""mop_veff_and_grad into pinned host memory.  With the earlier half-list kernels
(MOP_PAIR_KERNELS=half) the HVP pass runs in bead chunks and each chunk's gradient rows are
copied while later chunks compute (the rows the bias touches after the last chunk); the bead-lane
kernels copy after the kernels.  The result must equal, bit for bit, the device-pointer call and
the pageable-host call."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2501_11962_b300 import mop
from tests.conftest import workload

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kernels", ["default", "half"])
@pytest.mark.parametrize("bias", [None, "end", "e2e"])
def test_pinned_host_gradient_equals_device_result(monkeypatch, bias, kernels):
    if kernels == "half":
        monkeypatch.setenv("MOP_PAIR_KERNELS", "half")
    else:
        monkeypatch.delenv("MOP_PAIR_KERNELS", raising=False)
    w = workload(4, n_beads=24)
    X = w.paths[0]
    N, Q = X.shape[:2]
    eng = mop.Engine(w.system)
    eng.set_path(0, X)
    if bias is not None:
        ga, gb = w.cv_groups
        eng.add_bias(0, 1.0, 2.0, 0.1, groups=(ga, gb), e2e=bias == "e2e")
    # device pointers
    vd = torch.empty(1, dtype=torch.float64, device="cuda")
    gd = torch.empty((N, Q, 3), dtype=torch.float64, device="cuda")
    eng.veff_and_grad_device(vd, gd, 0)
    torch.cuda.synchronize()
    # pinned host buffers (chunked copies) and pageable host buffers (one copy at the end)
    gp = torch.empty((N, Q, 3), dtype=torch.float64).pin_memory()
    vp = np.zeros(1)
    st = eng.L.mop_veff_and_grad(eng.h, 0, vp.ctypes.data_as(C.c_void_p), C.c_void_p(gp.data_ptr()), 0, None)
    eng._check(st, "mop_veff_and_grad")
    v_page, g_page = eng.veff_and_grad(0)
    assert vp[0] == vd.item() == v_page[0]
    assert np.array_equal(gp.numpy(), gd.cpu().numpy())
    assert np.array_equal(g_page, gd.cpu().numpy())


def test_async_pipeline_equals_synchronous_calls():
    """MOP_ASYNC: three evaluations enqueued back to back from page-locked buffers (uploads and
    downloads on the handle's streams, overlapping the next evaluation) give, after mop_wait, the
    bits of the synchronous calls on the same coordinates; a mop_step after them waits for the
    downloads and continues from the last path."""
    w = workload(4, n_beads=24)
    X = w.paths[0]
    N, Q = X.shape[:2]
    rng = np.random.default_rng(3)
    xs = [(X + rng.normal(0.0, 0.002, X.shape)).astype(np.float32) for _ in range(3)]
    ref = []
    eng = mop.Engine(w.system)
    for x in xs:
        eng.set_path(0, x)
        ref.append(eng.veff_and_grad(0))
    xh = [torch.tensor(x).pin_memory() for x in xs]
    vh = [torch.zeros(1, dtype=torch.float64).pin_memory() for _ in xs]
    gh = [torch.empty((N, Q, 3), dtype=torch.float64).pin_memory() for _ in xs]
    for k in range(3):
        eng.set_path_async(0, xh[k])
        eng.veff_and_grad_async(vh[k], gh[k], 0)
    eng.wait()
    for k in range(3):
        assert vh[k].item() == ref[k][0][0]
        assert np.array_equal(gh[k].numpy(), ref[k][1])
    # a step right after asynchronous calls (no wait in between) starts from the last path
    eng.set_path_async(0, xh[0])
    eng.veff_and_grad_async(vh[0], gh[0], 0)
    eng.step(1, 1e-5, 0.0, seed=1)
    eng.wait()
    assert np.array_equal(gh[0].numpy(), ref[0][1])
    assert np.isfinite(eng.get_path(0)).all()


def test_async_all_paths_equals_synchronous_call():
    """MOP_ASYNC with path_id = -1: the V_eff of every set path and the concatenated gradient land
    in the page-locked buffers as the synchronous call returns them; mop_wait on a handle with
    nothing pending returns at once."""
    w = workload(4)
    eng = mop.Engine(w.system)
    eng.wait()
    for p in (0, 1, 2):
        eng.set_path(p, w.paths[p])
    v_ref, g_ref = eng.veff_and_grad(-1)
    vh = torch.zeros(3, dtype=torch.float64).pin_memory()
    gh = torch.empty(g_ref.shape, dtype=torch.float64).pin_memory()
    eng.veff_and_grad_async(vh, gh, -1)
    eng.wait()
    assert np.array_equal(vh.numpy(), v_ref)
    assert np.array_equal(gh.numpy(), g_ref)
