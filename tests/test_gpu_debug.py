"""The bounds-checked debug build (GS_DEBUG=1, libgaloissat_debug.so).

In the debug build every row index a kernel gathers is compared with the problem's variable
count; an index out of range sets a sticky status bit that gs_sync_status reports, and the load is
skipped (no trap). On valid inputs the checks never fire and the arithmetic is the release
build's code, so the two builds must agree bitwise. Both builds run in child processes (the
library is chosen when the binding first loads it) on the same seeded inputs: forward, backward,
fused steps in the shared-variable and owned-variable forms, the exact check and a
straight-through step.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import os, sys
sys.path.insert(0, sys.argv[1])
import numpy as np, torch
from paper_2603_28796_b300 import _abi, build, synth
from paper_2603_28796_b300.engine import Engine, STEngine
out = {"lib": np.array([os.path.basename(build.LIB_DEBUG if os.environ.get("GS_DEBUG") == "1" else build.LIB)])}
cases = {
    "sat3": (synth.planted_ksat(3000, 12780, 3, seed=31), 200, "f32", 0),
    "mixed": (synth.mixed_powerlaw(4000, 14000, seed=32), 96, "bf16", 0),
    "comm": (synth.community(16 * 300, 4 * 16 * 300, 16, seed=33), 32, "bf16", 2),
}
for name, (cnf, B, dt, split) in cases.items():
    prob = _abi.gs_load_cnf(cnf.n_vars, cnf.clause_ptr, cnf.lits)
    if split:
        _abi.gs_set_tuning(prob, var_split=split, loss_mode=1)
    eng = Engine(prob, B, dt, seed=34)
    out[name + "_fwd"] = _abi.gs_forward(prob, eng.x_cur).cpu().numpy()
    out[name + "_bwd"] = _abi.gs_backward(prob, eng.x_cur).float().cpu().numpy()
    for _ in range(3):
        eng.step()
    torch.cuda.synchronize()
    for key in ("delta", "m", "v", "loss", "unsat", "best", "bits"):
        out[name + "_" + key] = getattr(eng, key).float().cpu().numpy() if key in ("delta", "m", "v") else \
            getattr(eng, key).cpu().numpy()
    _abi.gs_sync_status(prob)
    del eng
    prob.close()
cnf = cases["sat3"][0]
prob = _abi.gs_load_cnf(cnf.n_vars, cnf.clause_ptr, cnf.lits)
st = STEngine(prob, 128, seed=35, noise_seed=36)
for _ in range(3):
    st.step()
torch.cuda.synchronize()
out["st_delta"] = st.delta.cpu().numpy()
out["st_bits"] = st.bits_cur.cpu().numpy()
out["st_unsat"] = st.unsat.cpu().numpy()
_abi.gs_sync_status(prob)
np.savez(sys.argv[2], **out)
print("ok")
"""


def _run(tmp_path, debug):
    path = str(tmp_path / ("dbg.npz" if debug else "rel.npz"))
    env = dict(os.environ, GS_DEBUG="1" if debug else "0")
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT, path], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return dict(np.load(path))


def test_debug_build_raises_no_flag_and_matches_release(tmp_path):
    rel = _run(tmp_path, False)
    dbg = _run(tmp_path, True)
    assert rel.pop("lib")[0] == "libgaloissat.so"
    assert dbg.pop("lib")[0] == "libgaloissat_debug.so"
    assert set(rel) == set(dbg)
    for key in rel:
        assert np.array_equal(rel[key], dbg[key]), key
