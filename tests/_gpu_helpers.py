"""Shared helpers of the GPU parity tests: device placement, dtype rounding of inputs, and the
tolerances derived from the float32 arithmetic of the kernels."""
from __future__ import annotations

import numpy as np
import torch

from paper_2603_28796_b300 import _abi, synth

TORCH_DT = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}
U32 = 2.0 ** -24          # unit roundoff of float32
GRAD_RTOL = 1e-5          # the gradient / loss bar: 1e-5 relative


def device_cands(a: np.ndarray, B: int, dtype="f32") -> torch.Tensor:
    """float host [n, >=B] -> device [n, B] view of a padded [n, ldB] buffer in dtype
    (16-bit dtypes round to nearest even: the rounding belongs to input generation)."""
    dt = TORCH_DT[dtype]
    n = a.shape[0]
    ld = synth.padded_ld(B, torch.empty(0, dtype=dt).element_size())
    buf = torch.zeros((n, ld), dtype=dt, device="cuda")
    buf[:, :B] = torch.from_numpy(np.ascontiguousarray(a[:, :B], dtype=np.float32)).to("cuda").to(dt)
    return buf[:, :B]


def host64(t: torch.Tensor) -> np.ndarray:
    """Exact float64 image of a device tensor (float32/bfloat16/float16 -> float64 is exact)."""
    return t.detach().to(torch.float64).cpu().numpy()


def load(cnf) -> _abi.Problem:
    return _abi.gs_load_cnf(cnf.n_vars, cnf.clause_ptr, cnf.lits)


def assert_loss(l_gpu, l_ref, what="loss"):
    err = np.abs(l_gpu - l_ref)
    tol = GRAD_RTOL * np.abs(l_ref) + 1e-30
    bad = err > tol
    assert not bad.any(), "%s: %d of %d beyond 1e-5 relative; worst %.3e at %s" % (
        what, bad.sum(), bad.size, (err / np.maximum(np.abs(l_ref), 1e-300)).max(), np.argwhere(bad)[:3].tolist())


def assert_grad(g_gpu, g_ref, scale, what="grad"):
    """|g - g_ref| <= 1e-5 * max(|g_ref|, A), A = sum |leave-one-out| (cancellation scale)."""
    err = np.abs(g_gpu - g_ref)
    tol = GRAD_RTOL * np.maximum(np.abs(g_ref), scale) + 1e-30
    bad = err > tol
    assert not bad.any(), "%s: %d of %d beyond tolerance; worst ratio %.3f at %s" % (
        what, bad.sum(), bad.size, (err / tol).max(), np.argwhere(bad)[:3].tolist())


def adam_tolerances(d0, m0, v0, g_ref, scale, t, lr=1.0, b1=0.9, b2=0.999, eps=1e-8, tau=1.0, g_rel=None, z=None,
                    z_err=None):
    """Element-wise bounds on |out_gpu - out_oracle| for delta', m', v' after one Adam step,
    propagated from (i) the gradient error bound (1e-5 * max(|g|, A), or g_rel * |g| when the
    gradient is an exact input) and (ii) a few float32 roundings in each operation. The chain
    factor is taken at z = delta / tau, or at the given z (the straight-through form passes
    (delta + noise) / tau, whose float32 rounding z_err moves the chain factor y (1 - y) by
    z_err |1 - 2y| relative)."""
    d0, m0, v0, g = (np.asarray(a, dtype=np.float64) for a in (d0, m0, v0, g_ref))
    z = d0 / tau if z is None else np.asarray(z, dtype=np.float64) / tau
    sp, sn = 1.0 / (1.0 + np.exp(-z)), 1.0 / (1.0 + np.exp(z))
    chain = sp * sn / tau
    if g_rel is None:
        eg = GRAD_RTOL * np.maximum(np.abs(g), scale)            # absolute error of dL/dx
    else:
        eg = g_rel * np.abs(g)
    gd = g * chain
    egd = eg * chain + 8 * U32 * np.abs(gd)                     # chain factor: expf, divide, products
    if z_err is not None:
        egd = egd + np.abs(gd) * np.asarray(z_err, dtype=np.float64) * np.abs(1.0 - 2.0 * sp)
    m1 = b1 * m0 + (1 - b1) * gd
    v1 = b2 * v0 + (1 - b2) * gd * gd
    em = (1 - b1) * egd + 4 * U32 * (np.abs(m1) + b1 * np.abs(m0))
    ev = (1 - b2) * (2 * np.abs(gd) * egd + egd * egd) + 4 * U32 * (np.abs(v1) + b2 * np.abs(v0))
    bc1, bc2 = 1 - b1 ** t, 1 - b2 ** t
    sv = np.sqrt(v1 / bc2)
    den = sv + eps
    u = lr * (m1 / bc1) / den
    with np.errstate(divide="ignore", invalid="ignore"):
        dv = np.where(v1 > 0, 0.5 / np.sqrt(np.maximum(v1, 1e-300) * bc2), 0.0)
    eu = lr / bc1 * (em / den + np.abs(m1) * ev * dv / (den * den)) + 8 * U32 * np.abs(u)
    eu = np.minimum(eu, 2 * lr / bc1 * np.abs(m1) / np.maximum(den, 1e-300) + 2 * lr * em / bc1 / eps)
    ed = eu + 2 * U32 * (np.abs(d0) + np.abs(u))
    return dict(delta=ed, m=em, v=ev, u=u)


def check_adam(out_gpu, ref, tol, what=""):
    for key in ("delta", "m", "v"):
        err = np.abs(out_gpu[key] - ref[key])
        bad = err > tol[key] + 1e-38
        assert not bad.any(), "%s %s: %d of %d beyond the derived bound; worst ratio %.3f at %s" % (
            what, key, bad.sum(), bad.size, (err / (tol[key] + 1e-38)).max(), np.argwhere(bad)[:3].tolist())


def unpack_bits(bits: torch.Tensor, n: int, B: int) -> np.ndarray:
    w = bits.cpu().numpy().view(np.uint64)[:n]
    out = np.zeros((n, B), dtype=np.uint8)
    for b in range(B):
        out[:, b] = ((w[:, b // 64] >> np.uint64(b % 64)) & np.uint64(1)).astype(np.uint8)
    return out


def padding_bits_zero(bits: torch.Tensor, n: int, B: int) -> bool:
    w = bits.cpu().numpy().view(np.uint64)[:n]
    nwd = (B + 63) // 64
    if B % 64 == 0:
        return True
    mask = np.uint64((1 << (B % 64)) - 1)
    return bool(np.all((w[:, nwd - 1] & ~mask) == 0))
