"""The scale of the j-side shares of the H eta pass rests on a bound (8 max|eta| (16 gmax + 1e3),
with gmax the largest |g| of the force pass) that is argued, not proved.  The check library
(libmop_jcheck.so: the same kernels with MOP_BL_JCHECK=1) writes NaN into the rows of any bead
whose shares left the promised range (2^24 after scaling; 2^30 for the unscaled force shares of
the half list).  Every workload, around the strained and the relaxed structures, with adjoint and
FD H eta, on the default lists and on the half list, must evaluate to a finite gradient that
equals the product library's bit for bit; a path with two oxygens 0.08 nm apart must trip the
check.  Each library runs in a process of its own."""
import json
import os
import subprocess
import sys
from pathlib import Path

import pytest

pytestmark = pytest.mark.gpu

ROOT = Path(__file__).resolve().parents[1]

SCRIPT = r"""
import json, os, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2501_11962_b300 import build as B
if sys.argv[2] == "check":
    B.LIB = B.CHECK_LIB
from paper_2501_11962_b300 import mop, synth
mop.load(build_if_needed=False)
from tests.conftest import workload
out = []
for k, relaxed, kernels, fd, pme, overlap in json.loads(sys.argv[3]):
    if kernels:
        os.environ["MOP_PAIR_KERNELS"] = kernels
    else:
        os.environ.pop("MOP_PAIR_KERNELS", None)
    w = workload(k, relaxed=relaxed)
    system = synth.with_pme(w.system) if pme else w.system
    kw = dict(hvp_mode=mop.MOP_HVP_FD, fd_h=1e-3) if fd else {}
    eng = mop.Engine(system, **kw)
    for p, X in enumerate(w.paths):
        if overlap:
            # the oxygen of molecule 1 0.08 nm from that of molecule 0 in every bead: an LJ force
            # of ~6e9 kJ/mol/nm, beyond the range the unscaled force shares are promised
            X = X.copy()
            X[:, 3] = X[:, 0] + np.float32([0.08, 0.0, 0.0])
        eng.set_path(p, X)
    try:
        v, G = eng.veff_and_grad(-1)
        res = dict(finite=bool(np.isfinite(G).all() and np.isfinite(v).all()),
                   sig=[float(np.sum(G)), float(np.sum(np.abs(G))), [float(x) for x in v]])
    except mop.MopError as e:
        res = dict(finite=False, error=str(e))
    eng.close()
    out.append(res)
print(json.dumps(out))
"""

CASES = [
    (2, False, "", False, False, False), (2, True, "", False, False, False), (2, False, "", True, False, False),
    (2, True, "", True, False, False), (2, False, "blhalf", False, False, False),
    (2, False, "blhalf", True, False, False), (2, False, "", False, True, False), (3, True, "", False, False, False),
    (4, False, "", False, False, False), (4, True, "", False, False, False), (4, False, "blhalf", False, False, False),
    (5, False, "", False, False, False), (5, True, "", False, False, False),
]
# the positive control: a share the check must catch
CONTROL = [(2, False, "blhalf", False, False, True)]


def run(lib, cases):
    env = dict(os.environ)
    env.pop("MOP_PAIR_KERNELS", None)
    r = subprocess.run([sys.executable, "-c", SCRIPT, str(ROOT), lib, json.dumps(cases)], capture_output=True,
                       text=True, env=env, cwd=str(ROOT), timeout=1800)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_j_side_shares_stay_in_range_on_every_workload():
    from paper_2501_11962_b300 import build as B
    assert B.CHECK_LIB.exists(), "libmop_jcheck.so is built by build_check()"
    checked = run("check", CASES + CONTROL)
    product = run("product", CASES)
    for case, c, p in zip(CASES, checked, product):
        assert c["finite"], (case, c)
        assert c["sig"] == p["sig"], (case, c, p)
    assert not checked[-1]["finite"], checked[-1]   # the check is live
