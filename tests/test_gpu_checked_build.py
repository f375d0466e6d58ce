"""The checked build (libgradsim_check.so: step kernels compiled with
-DGS_CHECK, every mesh-table index range-checked on the device before use)
on the small parity cases: the status word stays clear (gs_mesh_check is
GS_OK, never GS_EINDEX) and the results still match the FP64 oracle.  Runs
in a child process, which loads the checked library instead of the regular
one (GRADSIM_CHECKED=1)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import os, sys
import numpy as np
ROOT = sys.argv[1]
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))
import torch
from paper_2104_02646_gb300 import gradsim as gs
from paper_2104_02646_gb300 import inputs as I
from gpu_util import (CLOTH_KEYS, POS_CONTACT, TET_KEYS, check_grads, check_state, make_target, run_gpu,
                      run_oracle)

L = gs.load()
assert L.gs_build_flags() & gs.GS_BUILD_CHECKED, "not the checked build"
assert os.path.basename(gs.library_path()) == "libgradsim_check.so"
ctx = gs.Context(0)


def case(p, S, keys, **kw):
    tgt = make_target(p, S)
    ref = run_oracle(p, S, tgt)
    out = run_gpu(gs, ctx, p, S, tgt, **kw)
    st = out["mesh"].check_finite()
    assert st == gs.GS_OK, (p.name, st, L.gs_last_error())
    check_state(out["x"], out["v"], ref["x"], ref["v"], p.x0, POS_CONTACT, vel_entry=False)
    check_grads(out, ref, keys)
    out["mesh"].close()


case(I.bar("b", steps=1000), 1000, TET_KEYS)
case(I.block(n=8, steps=60, seed=3), 60, TET_KEYS, patch_elems=300)
case(I.block(n=6, steps=57, seed=5), 57, TET_KEYS, K=8, patch_elems=200)
case(I.cloth("3s", n=24, steps=120, grid_scaled=True, height=0.29), 120, CLOTH_KEYS, patch_elems=128)
thrown = I.cloth_throw(n=12, steps=80)
case(thrown, 80, CLOTH_KEYS, patch_elems=128)

# a batch of three meshes in one launch per step
probs = [I.batch_member(i, steps=50, lo=500, hi=3000) for i in range(3)]
rng = np.random.default_rng(1)
for p in probs:
    p.v0 = rng.normal(0.0, 0.1, p.X.shape)
meshes = [gs.Mesh(ctx, p, patch_elems=128) for p in probs]
batch = gs.Batch(ctx, meshes)
tg = [torch.tensor(make_target(p, 50), dtype=torch.float32, device="cuda") for p in probs]
loss = torch.zeros(3, dtype=torch.float64, device="cuda")
batch.rollout([p.dt for p in probs], 50, 1, tg, loss)
grads = [{k: torch.zeros(p.n_elems, dtype=torch.float64, device="cuda") for k in ("d_mu", "d_lambda")}
         for p in probs]
batch.adjoint(grads)
torch.cuda.synchronize()
for m in meshes:
    assert m.check_finite() == gs.GS_OK, L.gs_last_error()
print("CHECKED BUILD OK")
"""


def test_checked_build_status_clear_and_parity():
    from paper_2104_02646_gb300 import _build
    _build.build()
    assert os.path.exists(_build.LIB_CHECKED)
    env = dict(os.environ, GRADSIM_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "CHECKED BUILD OK" in r.stdout
