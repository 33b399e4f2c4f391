"""The allocation-free forward entry point against the regular one and the FP64 oracle.

gs_forward_noalloc exists for host programs that may not allocate device memory while they
run (their memory is pre-reserved by another allocator, or an allocation's implicit
synchronisation is not acceptable). It keeps its scratch in a fixed array inside the library,
so these checks call it twice in a row on different inputs — the second call must not see the
first call's leftovers — and compare each result with gs_forward on the same input (the same
kernels, chunking and reduction order: bitwise equal) and with the FP64 oracle (the 1e-5
relative loss bar of the other parity tests). The lane caps of the forward pass are varied
(gs_set_tuning), since a tuned cap changes the chunking both entry points must follow. This file
is collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2603_28796_b300 import _abi, synth  # noqa: E402
from tests import _gpu_helpers as H  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,fwd_lanes", [("f32", 0), ("bf16", 0), ("f32", 4), ("bf16", 8), ("f32", 16)])
def test_noalloc_forward_matches_forward_and_oracle_on_two_calls(dtype, fwd_lanes):
    cnf = synth.planted_ksat(3000, 12780, 3, seed=91)
    prob = H.load(cnf)
    if fwd_lanes:
        _abi.gs_set_tuning(prob, fwd_lanes=fwd_lanes)
    B = 300
    for call, seed in enumerate((92, 93)):
        xh = synth.uniform_values(cnf.n_vars, B, seed=seed)
        x = H.device_cands(xh, B, dtype)
        ref = _abi.gs_forward(prob, x)
        out = torch.full((1, B), -1.0, dtype=torch.float64, device="cuda")
        _abi.gs_forward_noalloc(prob, x, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()[0]
        assert np.array_equal(got, ref.cpu().numpy()[0]), "no-alloc call %d differs from gs_forward" % (call + 1)
        l_ref, _ = oracle.forward(cnf.n_vars, cnf.clause_ptr, cnf.lits, H.host64(x))
        H.assert_loss(got, l_ref, "no-alloc call %d vs oracle" % (call + 1))
    _abi.gs_sync_status(prob)


def test_noalloc_forward_rejects_sizes_beyond_its_scratch():
    cnf = synth.planted_ksat(2000, 60000, 3, seed=94)
    prob = H.load(cnf)
    tiles = prob.info()["n_fwd_tiles"]
    B = 128 * (-(-(16 << 20) // (tiles * 4 * 128)) + 1)       # tiles * B * 4 > 16 MiB
    assert tiles * B * 4 > (16 << 20)
    x = H.device_cands(np.zeros((cnf.n_vars, B), np.float32), B)
    out = torch.zeros((1, B), dtype=torch.float64, device="cuda")
    with pytest.raises(_abi.GSError) as ei:
        _abi.gs_forward_noalloc(prob, x, out)
    assert ei.value.status == 5 and "16 MiB" in str(ei.value)
