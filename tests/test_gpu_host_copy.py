"""mop_veff_and_grad into pinned host memory: the HVP pass runs in bead chunks and each chunk's
gradient rows are copied while later chunks compute (the rows the bias touches after the last
chunk).  The result must equal, bit for bit, the device-pointer call and the pageable-host call."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2501_11962_b300 import mop
from tests.conftest import workload

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("bias", [None, "end", "e2e"])
def test_pinned_host_gradient_equals_device_result(bias):
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
