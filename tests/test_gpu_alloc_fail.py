"""Allocation failure is reported, not fatal.  MOP_FAIL_ALLOC makes chosen device allocations fail
on the host side (no device fault): the entry point must return MOP_ERR_OOM and leave the
handle usable, so that the next call succeeds and gives the same result as a handle that never
failed.  Runs in a child process, because the variable is read once per process."""
import os
import subprocess
import sys
from pathlib import Path

import pytest

pytestmark = pytest.mark.gpu

ROOT = Path(__file__).resolve().parents[1]

CHILD = r"""
import numpy as np
from paper_2501_11962_b300 import mop, synth

w = synth.config(2, n_beads=4)
X = w.paths[0]

def expect(status, fn):
    try:
        fn()
    except mop.MopError as e:
        assert e.status == status, (e.status, str(e))
        return
    raise AssertionError("no error, expected %d" % status)

# reference from a handle that never failed (its allocations come after every planned failure)
expect(mop.MOP_ERR_OOM, lambda: mop.Engine(w.system))          # the 3rd allocation of mop_create
eng = mop.Engine(w.system)                                        # that failure is spent: works
expect(mop.MOP_ERR_OOM, lambda: eng.set_path(0, X))            # the 2nd allocation of mop_set_path
expect(mop.MOP_ERR_STATE, lambda: eng.veff_and_grad(0))        # the path was left unset
eng.set_path(0, X)
expect(mop.MOP_ERR_OOM, lambda: eng.veff_and_grad(0))          # the 5th allocation of an evaluation
v1, G1 = eng.veff_and_grad(0)
ref = mop.Engine(w.system)
ref.set_path(0, X)
v0, G0 = ref.veff_and_grad(0)
assert np.array_equal(v1, v0) and np.array_equal(G1, G0)
print("OK")
"""


def test_allocation_failure_returns_oom_and_leaves_the_handle_usable():
    env = dict(os.environ, MOP_FAIL_ALLOC="mop_create:3,mop_set_path:2,mop_veff_and_grad:5")
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    print(r.stdout, r.stderr[-2000:])
    assert r.returncode == 0 and "OK" in r.stdout
