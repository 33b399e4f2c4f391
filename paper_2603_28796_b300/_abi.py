"""ctypes binding of the C ABI declared in ``include/gs.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls. Candidate arrays are torch
tensors of shape ``[n, B]`` on the problem's device, var-major, unit column stride; their row
stride is passed as ``ldB`` (so a ``[n, B]`` view of a ``[n, ldB]`` buffer is accepted). All
compute runs in the library's kernels on the given (default: current) CUDA stream; nothing
here computes on the host, and there is no fallback: if ``libgaloissat.so`` is missing or
fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import build as _build

GS_OK = 0
GS_F32, GS_BF16, GS_F16 = 0, 1, 2
STATUS_NAMES = {
    0: "GS_OK", 1: "GS_ERR_INVALID_ARG", 2: "GS_ERR_PARSE", 3: "GS_ERR_OOM", 4: "GS_ERR_CUDA",
    5: "GS_ERR_UNSUPPORTED", 6: "GS_ERR_TIMEOUT", 7: "GS_ERR_STATE",
}

# Every symbol include/gs.h declares.
EXPORTED = (
    "gs_adam_default", "gs_load_cnf", "gs_load_batch", "gs_load_batch_opts", "gs_load_dimacs", "gs_inspect_cnf", "gs_info_get",
    "gs_set_tuning", "gs_get_tuning", "gs_autotune", "gs_reserve", "gs_relax", "gs_forward", "gs_forward_noalloc", "gs_backward", "gs_step", "gs_round_check", "gs_check_bits",
    "gs_st_noise", "gs_st_sample", "gs_st_step", "gs_tseitin3", "gs_pool_sample", "gs_branch_vars",
    "gs_gather_probe", "gs_wait_selftest", "gs_sync_status", "gs_free", "gs_status_str", "gs_last_error",
)


class GSError(RuntimeError):
    """A C-ABI call returned a status other than GS_OK."""

    def __init__(self, status: int, call: str, detail: str):
        self.status = status
        super().__init__("%s failed: %s (%s)" % (call, STATUS_NAMES.get(status, status), detail))


class GsInfo(ctypes.Structure):
    _fields_ = [
        ("n_vars", ctypes.c_int64), ("n_clauses", ctypes.c_int64), ("nnz", ctypes.c_int64),
        ("n_inst", ctypes.c_int32), ("max_k", ctypes.c_int32), ("n_empty", ctypes.c_int64),
        ("n_unit", ctypes.c_int64), ("n_taut", ctypes.c_int64), ("n_dup", ctypes.c_int64),
        ("n_occ_codes", ctypes.c_int64), ("n_fwd_tiles", ctypes.c_int64), ("n_var_tiles", ctypes.c_int64),
        ("n_split", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
        ("fwd_tile_codes", ctypes.c_int32), ("var_tile_codes", ctypes.c_int32), ("own_item_codes", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]

    def as_dict(self) -> dict:
        return {name: int(getattr(self, name)) for name, _ in self._fields_}


class GsPlanOpts(ctypes.Structure):
    _fields_ = [("fwd_tile_codes", ctypes.c_int32), ("var_tile_codes", ctypes.c_int32),
                ("own_item_codes", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class GsTuning(ctypes.Structure):
    _fields_ = [("var_lanes", ctypes.c_int32), ("fwd_lanes", ctypes.c_int32), ("var_gather", ctypes.c_int32),
                ("loss_mode", ctypes.c_int32), ("var_split", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {"var_lanes": int(self.var_lanes), "fwd_lanes": int(self.fwd_lanes),
                "var_gather": int(self.var_gather), "loss_mode": int(self.loss_mode),
                "var_split": int(self.var_split)}


class GsAdam(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("eps", ctypes.c_double), ("tau", ctypes.c_double)]


_lib = None


def library_path() -> str:
    return _build.LIB


def lib():
    """The loaded ``libgaloissat.so`` (raises if it has not been built); with the environment
    variable ``GS_DEBUG=1`` the bounds-checked ``libgaloissat_debug.so`` instead."""
    global _lib
    if _lib is None:
        path = _build.LIB_DEBUG if os.environ.get("GS_DEBUG", "") not in ("", "0") else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError("%s is not built (run __graft_entry__.build() or "
                               "python -m paper_2603_28796_b300.build); there is no CPU fallback"
                               % os.path.basename(path))
        L = ctypes.CDLL(path)
        i32, i64, vp, cp = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_char_p
        pp = ctypes.POINTER(ctypes.c_void_p)
        sig = {
            "gs_adam_default": (None, [ctypes.POINTER(GsAdam)]),
            "gs_load_cnf": (ctypes.c_int, [i64, i64, vp, vp, vp, pp]),
            "gs_load_batch": (ctypes.c_int, [i32, vp, vp, vp, vp, vp, pp]),
            "gs_load_batch_opts": (ctypes.c_int, [i32, vp, vp, vp, vp, ctypes.POINTER(GsPlanOpts), vp, pp]),
            "gs_load_dimacs": (ctypes.c_int, [cp, vp, pp]),
            "gs_inspect_cnf": (ctypes.c_int, [i64, i64, vp, vp, ctypes.POINTER(GsInfo)]),
            "gs_info_get": (ctypes.c_int, [vp, ctypes.POINTER(GsInfo)]),
            "gs_set_tuning": (ctypes.c_int, [vp, ctypes.POINTER(GsTuning)]),
            "gs_get_tuning": (ctypes.c_int, [vp, ctypes.POINTER(GsTuning)]),
            "gs_autotune": (ctypes.c_int, [vp, i32, ctypes.c_int, vp, ctypes.POINTER(GsTuning)]),
            "gs_reserve": (ctypes.c_int, [vp, i32, ctypes.c_int]),
            "gs_relax": (ctypes.c_int, [vp, vp, vp, ctypes.c_int, i32, i64, ctypes.c_float, vp]),
            "gs_forward": (ctypes.c_int, [vp, vp, ctypes.c_int, i32, i64, vp, vp]),
            "gs_forward_noalloc": (ctypes.c_int, [vp, vp, ctypes.c_int, i32, i64, vp, vp]),
            "gs_backward": (ctypes.c_int, [vp, vp, ctypes.c_int, i32, i64, vp, vp, vp]),
            "gs_step": (ctypes.c_int, [vp, vp, vp, vp, vp, vp, vp, ctypes.c_int, i32, i64, i64,
                                       ctypes.POINTER(GsAdam), vp, vp, vp]),
            "gs_round_check": (ctypes.c_int, [vp, vp, i32, i64, vp, vp, vp, vp]),
            "gs_check_bits": (ctypes.c_int, [vp, vp, i32, vp, vp, vp]),
            "gs_tseitin3": (ctypes.c_int, [i64, i64, vp, vp, vp, vp, vp, vp, vp]),
            "gs_pool_sample": (ctypes.c_int, [vp, vp, i64, i32, vp, i64, ctypes.c_uint64, i32, i32, vp, vp, vp]),
            "gs_branch_vars": (ctypes.c_int, [vp, vp, i64, i32, i32, vp, vp]),
            "gs_st_noise": (ctypes.c_int, [vp, ctypes.c_uint64, i64, vp, i32, i64, vp]),
            "gs_st_sample": (ctypes.c_int, [vp, vp, vp, ctypes.c_uint64, i64, i32, i64, vp, vp]),
            "gs_st_step": (ctypes.c_int, [vp, vp, vp, vp, vp, vp, vp, vp, vp, ctypes.c_uint64, i64, i32, i64,
                                          ctypes.POINTER(GsAdam), vp]),
            "gs_gather_probe": (ctypes.c_int, [vp, i64, i64, i32, vp, i64, vp, vp]),
            "gs_wait_selftest": (ctypes.c_int, [vp, ctypes.c_uint32, vp]),
            "gs_sync_status": (ctypes.c_int, [vp]),
            "gs_free": (None, [vp]),
            "gs_status_str": (ctypes.c_char_p, [ctypes.c_int]),
            "gs_last_error": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status: int, call: str) -> None:
    if status != GS_OK:
        detail = lib().gs_last_error().decode(errors="replace")
        raise GSError(status, call, detail)


# ------------------------------------------------------------------------------------------
# torch marshalling helpers (imported lazily so that host-only users need no torch import)
def _torch():
    import torch
    return torch


def _dtype_code(t) -> int:
    torch = _torch()
    if t.dtype == torch.float32:
        return GS_F32
    if t.dtype == torch.bfloat16:
        return GS_BF16
    if t.dtype == torch.float16:
        return GS_F16
    raise TypeError("relaxed values must be float32, bfloat16 or float16, got %s" % t.dtype)


def _stream(stream) -> Optional[int]:
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else stream


def _cand(t, name: str, n: Optional[int] = None):
    """(B, ldB) of a var-major candidate tensor [n, B] with unit column stride."""
    if t.dim() != 2:
        raise ValueError("%s must be 2-D [n, B]" % name)
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if n is not None and t.shape[0] != n:
        raise ValueError("%s has %d rows, the problem has %d variables" % (name, t.shape[0], n))
    if t.shape[1] > 1 and t.stride(1) != 1:
        raise ValueError("%s must have unit column stride" % name)
    ldB = t.stride(0) if t.shape[0] > 0 else t.shape[1]
    return int(t.shape[1]), int(ldB)


def _ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


def _np_ptr(a) -> Optional[int]:
    return None if a is None else a.ctypes.data


# ------------------------------------------------------------------------------------------
class Problem:
    """Owning handle of a ``gs_problem*`` (freed by ``gs_free`` on close / garbage collection)."""

    def __init__(self, handle: int):
        self._h = ctypes.c_void_p(handle)
        self._info = None

    @property
    def handle(self) -> ctypes.c_void_p:
        if not self._h:
            raise RuntimeError("problem already freed")
        return self._h

    def info(self) -> dict:
        if self._info is None:
            gi = GsInfo()
            _check(lib().gs_info_get(self.handle, ctypes.byref(gi)), "gs_info_get")
            self._info = gi.as_dict()
        return self._info

    @property
    def n_vars(self) -> int:
        return self.info()["n_vars"]

    @property
    def n_inst(self) -> int:
        return self.info()["n_inst"]

    def close(self) -> None:
        if self._h:
            lib().gs_free(self._h)
            self._h = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _csr(clause_ptr, lits):
    cp = np.ascontiguousarray(clause_ptr, dtype=np.int64)
    lt = np.ascontiguousarray(lits, dtype=np.int32)
    return cp, lt


def gs_adam_default() -> GsAdam:
    a = GsAdam()
    lib().gs_adam_default(ctypes.byref(a))
    return a


def gs_load_cnf(n_vars: int, clause_ptr, lits, stream=None) -> Problem:
    cp, lt = _csr(clause_ptr, lits)
    out = ctypes.c_void_p()
    _check(lib().gs_load_cnf(int(n_vars), cp.size - 1, _np_ptr(cp), _np_ptr(lt) if lt.size else None,
                             _stream(stream), ctypes.byref(out)), "gs_load_cnf")
    return Problem(out.value)


def gs_load_batch(n_vars, n_clauses, clause_ptr, lits, stream=None) -> Problem:
    nv = np.ascontiguousarray(n_vars, dtype=np.int64)
    nc = np.ascontiguousarray(n_clauses, dtype=np.int64)
    cp, lt = _csr(clause_ptr, lits)
    out = ctypes.c_void_p()
    _check(lib().gs_load_batch(nv.size, _np_ptr(nv), _np_ptr(nc), _np_ptr(cp), _np_ptr(lt) if lt.size else None,
                               _stream(stream), ctypes.byref(out)), "gs_load_batch")
    return Problem(out.value)


def gs_load_batch_opts(n_vars, n_clauses, clause_ptr, lits, fwd_tile_codes: int = 0, var_tile_codes: int = 0,
                       own_item_codes: int = 0, stream=None) -> Problem:
    """gs_load_batch with explicit tile sizes (0 = default); a single formula is a batch of one."""
    nv = np.atleast_1d(np.ascontiguousarray(n_vars, dtype=np.int64))
    nc = np.atleast_1d(np.ascontiguousarray(n_clauses, dtype=np.int64))
    cp, lt = _csr(clause_ptr, lits)
    opts = GsPlanOpts(int(fwd_tile_codes), int(var_tile_codes), int(own_item_codes), 0)
    out = ctypes.c_void_p()
    _check(lib().gs_load_batch_opts(nv.size, _np_ptr(nv), _np_ptr(nc), _np_ptr(cp), _np_ptr(lt) if lt.size else None,
                                    ctypes.byref(opts), _stream(stream), ctypes.byref(out)), "gs_load_batch_opts")
    return Problem(out.value)


def gs_load_dimacs(path: str, stream=None) -> Problem:
    out = ctypes.c_void_p()
    _check(lib().gs_load_dimacs(os.fsencode(path), _stream(stream), ctypes.byref(out)), "gs_load_dimacs")
    return Problem(out.value)


def gs_inspect_cnf(n_vars: int, clause_ptr, lits) -> dict:
    """Validation + statistics on the host only (needs no GPU)."""
    cp, lt = _csr(clause_ptr, lits)
    gi = GsInfo()
    _check(lib().gs_inspect_cnf(int(n_vars), cp.size - 1, _np_ptr(cp), _np_ptr(lt) if lt.size else None,
                                ctypes.byref(gi)), "gs_inspect_cnf")
    return gi.as_dict()


def gs_tseitin3(n_vars: int, clause_ptr, lits):
    """Width-3 chain normalisation (Eq. 6-8) on the host: returns (n', clause_ptr', lits'); the
    first n_vars variables are the input's, the rest are the chains' fresh variables."""
    cp, lt = _csr(clause_ptr, lits)
    n2, m2, z2 = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    args = (int(n_vars), cp.size - 1, _np_ptr(cp), _np_ptr(lt) if lt.size else None)
    _check(lib().gs_tseitin3(*args, ctypes.byref(n2), ctypes.byref(m2), ctypes.byref(z2), None, None), "gs_tseitin3")
    cp2 = np.zeros(m2.value + 1, dtype=np.int64)
    lt2 = np.zeros(max(z2.value, 1), dtype=np.int32)
    _check(lib().gs_tseitin3(*args, ctypes.byref(n2), ctypes.byref(m2), ctypes.byref(z2), _np_ptr(cp2), _np_ptr(lt2)),
           "gs_tseitin3")
    return int(n2.value), cp2, lt2[: z2.value]


def gs_info_get(prob: Problem) -> dict:
    return prob.info()


def gs_set_tuning(prob: Problem, var_lanes: int = 0, fwd_lanes: int = 0, var_gather: int = 0,
                  loss_mode: int = 0, var_split: int = 0) -> None:
    t = GsTuning(int(var_lanes), int(fwd_lanes), int(var_gather), int(loss_mode), int(var_split))
    _check(lib().gs_set_tuning(prob.handle, ctypes.byref(t)), "gs_set_tuning")


def gs_get_tuning(prob: Problem) -> dict:
    t = GsTuning()
    _check(lib().gs_get_tuning(prob.handle, ctypes.byref(t)), "gs_get_tuning")
    return t.as_dict()


def _dtype_arg(dtype) -> int:
    """A gs_dtype code from an int code, a name ("f32", "bf16", "f16") or a torch dtype."""
    if isinstance(dtype, int):
        return dtype
    code = {"f32": GS_F32, "bf16": GS_BF16, "f16": GS_F16}.get(dtype) if isinstance(dtype, str) else None
    return code if code is not None else _dtype_code(_torch().empty(0, dtype=dtype))


def gs_autotune(prob: Problem, B: int, dtype, stream=None) -> dict:
    code = _dtype_arg(dtype)
    t = GsTuning()
    _check(lib().gs_autotune(prob.handle, int(B), code, _stream(stream), ctypes.byref(t)), "gs_autotune")
    return t.as_dict()


def gs_reserve(prob: Problem, B: int, dtype) -> None:
    code = _dtype_arg(dtype)
    _check(lib().gs_reserve(prob.handle, int(B), code), "gs_reserve")


def gs_relax(prob: Problem, delta, x, tau: float = 1.0, stream=None):
    B, ldB = _cand(delta, "delta", prob.n_vars)
    Bx, ldx = _cand(x, "x", prob.n_vars)
    if (B, ldB) != (Bx, ldx):
        raise ValueError("delta and x must share B and ldB")
    _check(lib().gs_relax(prob.handle, _ptr(delta), _ptr(x), _dtype_code(x), B, ldB, float(tau), _stream(stream)),
           "gs_relax")
    return x


def gs_forward(prob: Problem, x, loss=None, stream=None):
    torch = _torch()
    B, ldB = _cand(x, "x", prob.n_vars)
    if loss is None:
        loss = torch.empty((prob.n_inst, B), dtype=torch.float64, device=x.device)
    _check(lib().gs_forward(prob.handle, _ptr(x), _dtype_code(x), B, ldB, _ptr(loss), _stream(stream)), "gs_forward")
    return loss


def gs_forward_noalloc(prob: Problem, x, loss, stream=None):
    """gs_forward for callers that must not allocate: ``loss`` (float64 [n_inst, B]) is required,
    and the library's fixed scratch replaces the workspace (see include/gs.h)."""
    B, ldB = _cand(x, "x", prob.n_vars)
    _check(lib().gs_forward_noalloc(prob.handle, _ptr(x), _dtype_code(x), B, ldB, _ptr(loss), _stream(stream)),
           "gs_forward_noalloc")
    return loss


def gs_backward(prob: Problem, x, dloss=None, grad=None, stream=None):
    torch = _torch()
    B, ldB = _cand(x, "x", prob.n_vars)
    if grad is None:
        grad = torch.empty((prob.n_vars, ldB), dtype=torch.float32, device=x.device)[:, :B]
    Bg, ldg = _cand(grad, "grad", prob.n_vars)
    if (Bg, ldg) != (B, ldB):
        raise ValueError("grad must have the same B and ldB as x")
    if dloss is not None:
        dloss = dloss.contiguous()
        if dloss.dtype != torch.float64 or dloss.numel() != prob.n_inst * B:
            raise ValueError("dloss must be float64 [n_inst, B]")
    _check(lib().gs_backward(prob.handle, _ptr(x), _dtype_code(x), B, ldB, _ptr(dloss), _ptr(grad), _stream(stream)),
           "gs_backward")
    return grad


def _adam(adam) -> Optional[GsAdam]:
    if adam is None:
        return None
    if isinstance(adam, GsAdam):
        return adam
    a = gs_adam_default()
    for k, v in dict(adam).items():
        setattr(a, k, float(v))
    return a


def gs_step(prob: Problem, delta, m, v, step: int, grad=None, x_in=None, x_out=None, adam=None, loss=None,
            bits=None, stream=None) -> None:
    B, ldB = _cand(delta, "delta", prob.n_vars)
    for t, name in ((m, "m"), (v, "v"), (grad, "grad")):
        if t is not None and _cand(t, name, prob.n_vars) != (B, ldB):
            raise ValueError("%s must have the same B and ldB as delta" % name)
    xref = x_out if x_out is not None else x_in
    dtype = _dtype_code(xref) if xref is not None else GS_F32
    for t, name in ((x_in, "x_in"), (x_out, "x_out")):
        if t is not None and _cand(t, name, prob.n_vars) != (B, ldB):
            raise ValueError("%s must have the same B and ldB as delta" % name)
    a = _adam(adam)
    _check(lib().gs_step(prob.handle, _ptr(delta), _ptr(m), _ptr(v), _ptr(grad), _ptr(x_in), _ptr(x_out), dtype, B,
                         ldB, int(step), ctypes.byref(a) if a is not None else None, _ptr(loss), _ptr(bits),
                         _stream(stream)), "gs_step")


def gs_round_check(prob: Problem, delta, bits=None, unsat=None, best=None, stream=None):
    torch = _torch()
    B, ldB = _cand(delta, "delta", prob.n_vars)
    if unsat is None:
        unsat = torch.empty((prob.n_inst, B), dtype=torch.int32, device=delta.device)
    if best is None:
        best = torch.empty(prob.n_inst, dtype=torch.int32, device=delta.device)
    _check(lib().gs_round_check(prob.handle, _ptr(delta), B, ldB, _ptr(bits), _ptr(unsat), _ptr(best),
                                _stream(stream)), "gs_round_check")
    return unsat, best


def gs_check_bits(prob: Problem, bits, B: int, unsat=None, best=None, stream=None):
    torch = _torch()
    if unsat is None:
        unsat = torch.empty((prob.n_inst, B), dtype=torch.int32, device=bits.device)
    if best is None:
        best = torch.empty(prob.n_inst, dtype=torch.int32, device=bits.device)
    _check(lib().gs_check_bits(prob.handle, _ptr(bits), int(B), _ptr(unsat), _ptr(best), _stream(stream)),
           "gs_check_bits")
    return unsat, best


# ------------------------------------------------------------------------------------------
# Straight-through Gumbel training (Eq. 3 with noise, Eq. 4 in the forward pass).
def _seed(seed) -> int:
    return int(seed) & (2 ** 64 - 1)


def gs_st_noise(prob: Problem, seed: int, step: int, noise, stream=None) -> None:
    """Logistic noise l of one step into a float32 [n, B] candidate tensor."""
    B, ldB = _cand(noise, "noise", prob.n_vars)
    _check(lib().gs_st_noise(prob.handle, _seed(seed), int(step), _ptr(noise), B, ldB, _stream(stream)),
           "gs_st_noise")


def gs_st_sample(prob: Problem, delta, bits, seed: int = 0, step: int = 1, noise=None, stream=None) -> None:
    """bits = [delta + l > 0] (l from ``noise`` or generated from (seed, step))."""
    B, ldB = _cand(delta, "delta", prob.n_vars)
    if noise is not None and _cand(noise, "noise", prob.n_vars) != (B, ldB):
        raise ValueError("noise must have the same B and ldB as delta")
    _check(lib().gs_st_sample(prob.handle, _ptr(delta), _ptr(noise), _seed(seed), int(step), B, ldB, _ptr(bits),
                              _stream(stream)), "gs_st_sample")


def gs_st_step(prob: Problem, delta, m, v, bits_in, bits_out, step: int, seed: int = 0, noise=None, noise_next=None,
               noise_next_out=None, adam=None, stream=None) -> None:
    """One straight-through Gumbel step t: gradient at the hard point bits_in, soft chain, Adam,
    bits_out = [delta' + l_{t+1} > 0]. noise / noise_next: float32 [n, B] tensors or None
    (generated); noise_next_out receives the generated l_{t+1}."""
    B, ldB = _cand(delta, "delta", prob.n_vars)
    for t, name in ((m, "m"), (v, "v"), (noise, "noise"), (noise_next, "noise_next"), (noise_next_out, "noise_next_out")):
        if t is not None and _cand(t, name, prob.n_vars) != (B, ldB):
            raise ValueError("%s must have the same B and ldB as delta" % name)
    a = _adam(adam)
    _check(lib().gs_st_step(prob.handle, _ptr(delta), _ptr(m), _ptr(v), _ptr(bits_in), _ptr(bits_out), _ptr(noise),
                            _ptr(noise_next), _ptr(noise_next_out), _seed(seed), int(step), B, ldB,
                            ctypes.byref(a) if a is not None else None, _stream(stream)), "gs_st_step")


# ------------------------------------------------------------------------------------------
# Candidate pool and branching variables.
def _column(delta, b: int):
    """(device pointer, stride) of candidate column b of a var-major float32 [n, B] tensor."""
    if delta.dtype != _torch().float32:
        raise ValueError("delta must be float32")
    if not (0 <= b < delta.shape[1]):
        raise ValueError("candidate index out of range")
    return delta.data_ptr() + 4 * int(b) * delta.stride(1), delta.stride(0)


def gs_pool_sample(prob: Problem, delta, b: int, N: int, S: int, seed: int = 0, n_rows=None, noise=None,
                   bits=None, stream=None):
    """N noisy samples around candidate b of delta and each sample's S most confident rows.
    Returns (bits [n_rows, ceil(N/64)] int64, sel [N, S] int32) on the device."""
    torch = _torch()
    ptr, stride = _column(delta, b)
    nr = prob.n_vars if n_rows is None else int(n_rows)
    if bits is None:
        bits = torch.zeros((max(nr, 1), (int(N) + 63) // 64), dtype=torch.int64, device=delta.device)
    sel = torch.empty((int(N), int(S)), dtype=torch.int32, device=delta.device)
    ldN = 0
    if noise is not None:
        if noise.dtype != torch.float32 or noise.stride(1) != 1 or noise.shape[1] < N:
            raise ValueError("noise must be float32 [n_rows, >= N] with unit column stride")
        ldN = noise.stride(0)
    _check(lib().gs_pool_sample(prob.handle, ptr, stride, nr, _ptr(noise), ldN, _seed(seed), int(N), int(S),
                                _ptr(bits), _ptr(sel), _stream(stream)), "gs_pool_sample")
    return bits, sel


def gs_branch_vars(prob: Problem, delta, b: int, d: int, n_rows=None, stream=None):
    """The d rows of candidate b with the smallest |delta| (least confident), ascending."""
    ptr, stride = _column(delta, b)
    nr = prob.n_vars if n_rows is None else int(n_rows)
    out = _torch().empty(int(d), dtype=_torch().int32, device=delta.device)
    _check(lib().gs_branch_vars(prob.handle, ptr, stride, nr, int(d), _ptr(out), _stream(stream)), "gs_branch_vars")
    return out


def gs_gather_probe(src, row_bytes: int, idx, sink=None, stream=None):
    """Random row gathers (measurement kernel): ``src`` is a 2-D device tensor whose rows are read
    ``row_bytes`` bytes at a time from column 0 (row stride = its row stride in bytes), ``idx``
    a device int32/uint32 tensor of row indices; returns the uint32 sink tensor."""
    torch = _torch()
    if src.dim() != 2 or src.stride(1) != 1:
        raise ValueError("src must be a 2-D tensor with unit column stride")
    if idx.dtype not in (torch.int32,) or not idx.is_contiguous():
        raise ValueError("idx must be a contiguous int32 tensor")
    if sink is None:
        sink = torch.zeros(1, dtype=torch.int32, device=src.device)
    stride = src.stride(0) * src.element_size()
    _check(lib().gs_gather_probe(_ptr(src), int(src.shape[0]), int(stride), int(row_bytes), _ptr(idx),
                                 int(idx.numel()), _ptr(sink), _stream(stream)), "gs_gather_probe")
    return sink


def gs_wait_selftest(prob: Problem, limit_us: int = 1000, stream=None) -> None:
    _check(lib().gs_wait_selftest(prob.handle, int(limit_us), _stream(stream)), "gs_wait_selftest")


def gs_sync_status(prob: Problem) -> None:
    _check(lib().gs_sync_status(prob.handle), "gs_sync_status")


def gs_free(prob: Problem) -> None:
    prob.close()


def gs_status_str(status: int) -> str:
    return lib().gs_status_str(int(status)).decode()


def gs_last_error() -> str:
    return lib().gs_last_error().decode(errors="replace")
