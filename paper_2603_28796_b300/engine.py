"""Training engine of the differentiable solving stage on the C-ABI library.

``GSLoss`` is a ``torch.autograd.Function`` over ``gs_forward`` / ``gs_backward``: its forward
keeps only the relaxed values x (nothing per literal) and its backward recomputes the clause
products (Sec. "Differentiable SAT Formulation": forward of Eq. 2 + Eq. 5, back-propagation
through them).

``STEngine`` runs the paper's own training forward instead: straight-through Gumbel-softmax
(Eq. 3 with noise, Eq. 4 in the forward pass), whose forward is the bit-packed hard assignment.

``Engine`` owns one batch of B candidates of a problem: the float32 logit differences delta,
the Adam moments, two ping-pong buffers of relaxed values x = sigma(delta / tau) in the storage
dtype, the bit-packed rounded assignments and the per-candidate results. One ``step()`` is the
whole hot path: fused gradient + Adam + relaxed values + rounding + forward loss
(``gs_step`` with ``grad=None``), then the exact check (``gs_check_bits``). ``run(steps)``
captures the steps into one CUDA graph and replays it.
"""
from __future__ import annotations

from typing import Optional

import numpy as np
import torch

from . import _abi, synth

_DTYPES = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16,
           torch.float32: torch.float32, torch.bfloat16: torch.bfloat16, torch.float16: torch.float16}
_CODES = {torch.float32: _abi.GS_F32, torch.bfloat16: _abi.GS_BF16, torch.float16: _abi.GS_F16}


def candidates(n: int, B: int, dtype=torch.float32, device="cuda", fill: float = 0.0) -> torch.Tensor:
    """A var-major [n, B] view of a [n, ldB] buffer whose rows start on 16-byte boundaries."""
    dtype = _DTYPES[dtype]
    ld = synth.padded_ld(B, torch.empty(0, dtype=dtype).element_size())
    return torch.full((max(n, 0), ld), fill, dtype=dtype, device=device)[:, :B]


class GSLoss(torch.autograd.Function):
    """loss[i, b] = sum over clauses t of instance i of prod_{literals of t} f  (Eq. 2 + Eq. 5,
    kept non-negative: equals m_i + L_paper). Gradient with respect to x through gs_backward."""

    @staticmethod
    def forward(ctx, x: torch.Tensor, prob: _abi.Problem) -> torch.Tensor:
        loss = _abi.gs_forward(prob, x)
        ctx.save_for_backward(x)
        ctx.prob = prob
        return loss

    @staticmethod
    def backward(ctx, dloss: torch.Tensor):
        (x,) = ctx.saved_tensors
        grad = _abi.gs_backward(ctx.prob, x, dloss=dloss.to(torch.float64).contiguous())
        if x.dtype != torch.float32:
            grad = grad.to(x.dtype)
        return grad, None


def gs_loss(prob: _abi.Problem, x: torch.Tensor) -> torch.Tensor:
    return GSLoss.apply(x, prob)


class Engine:
    def __init__(self, prob: _abi.Problem, B: int, dtype="f32", adam: Optional[dict] = None, seed: int = 0,
                 delta0: Optional[np.ndarray] = None, device="cuda", autotune: bool = False):
        self.prob = prob
        self.B = int(B)
        self.dtype = _DTYPES[dtype]
        self.device = torch.device(device)
        self.adam = _abi._adam(adam) if adam is not None else None
        n = prob.n_vars
        self.n = n
        self.delta = candidates(n, B, torch.float32, device)
        self.m = candidates(n, B, torch.float32, device)
        self.v = candidates(n, B, torch.float32, device)
        self.x = [candidates(n, B, self.dtype, device), candidates(n, B, self.dtype, device)]
        self.nwd = (self.B + 63) // 64
        self.bits = torch.zeros((max(n, 1), self.nwd), dtype=torch.int64, device=device)
        self.loss = torch.zeros((prob.n_inst, B), dtype=torch.float64, device=device)
        self.unsat = torch.zeros((prob.n_inst, B), dtype=torch.int32, device=device)
        self.best = torch.zeros(prob.n_inst, dtype=torch.int32, device=device)
        self.cur = 0
        self.t = 0
        if autotune:
            self.tuning = _abi.gs_autotune(prob, B, _CODES[self.dtype])
        _abi.gs_reserve(prob, B, _CODES[self.dtype])
        self.reset(seed, delta0)

    def reset(self, seed: int = 0, delta0: Optional[np.ndarray] = None) -> None:
        """delta from delta0 (float32 [n, >=B]) or the seeded uniform-probability initialisation;
        Adam state zeroed; x = sigma(delta / tau)."""
        if delta0 is None:
            delta0 = synth.init_delta(self.n, self.B, seed)
        d = torch.from_numpy(np.ascontiguousarray(delta0[:, :self.B], dtype=np.float32))
        self.delta.copy_(d.to(self.device))
        self.m.zero_()
        self.v.zero_()
        self.t = 0
        self.cur = 0
        tau = self.adam.tau if self.adam is not None else 1.0
        _abi.gs_relax(self.prob, self.delta, self.x[0], tau=tau)

    @property
    def x_cur(self) -> torch.Tensor:
        return self.x[self.cur]

    def step(self, loss: bool = True, check: bool = True) -> None:
        """One pass of the hot path over the batch (asynchronous on the current stream)."""
        self.t += 1
        _abi.gs_step(self.prob, self.delta, self.m, self.v, self.t, grad=None, x_in=self.x[self.cur],
                     x_out=self.x[self.cur ^ 1], adam=self.adam, loss=self.loss if loss else None,
                     bits=self.bits if check else None)
        self.cur ^= 1
        if check:
            _abi.gs_check_bits(self.prob, self.bits, self.B, self.unsat, self.best)

    def capture(self, steps: int, loss: bool = True, check: bool = True) -> torch.cuda.CUDAGraph:
        """Records the next ``steps`` steps (t advancing) into a CUDA graph. The engine's state
        (t, ping-pong index) is advanced as if they had run; replay the graph exactly once."""
        if steps % 2:
            raise ValueError("capture an even number of steps so the ping-pong buffers line up")
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                for _ in range(steps):
                    self.step(loss=loss, check=check)
        torch.cuda.current_stream().wait_stream(s)
        return g

    def run(self, steps: int, graph: bool = True, loss: bool = True, check: bool = True) -> None:
        if graph and steps >= 2:
            even = steps - (steps % 2)
            g = self.capture(even, loss, check)
            g.replay()
            for _ in range(steps - even):
                self.step(loss, check)
        else:
            for _ in range(steps):
                self.step(loss, check)

    def state_dict(self) -> dict:
        """Everything the next step reads: logits, Adam moments, the current relaxed values, the
        step counter and the ping-pong index (host copies; torch.save-able)."""
        return {"kind": "relaxed", "n": self.n, "B": self.B, "dtype": str(self.dtype), "t": self.t,
                "delta": self.delta.detach().cpu().clone(), "m": self.m.detach().cpu().clone(),
                "v": self.v.detach().cpu().clone(), "x": self.x[self.cur].detach().cpu().clone()}

    def load_state_dict(self, st: dict) -> None:
        """Resume from state_dict(): the following steps are bitwise those of the saved run."""
        if st.get("kind") != "relaxed" or st["n"] != self.n or st["B"] != self.B or st["dtype"] != str(self.dtype):
            raise ValueError("state does not match this engine (kind, n, B, dtype)")
        self.delta.copy_(st["delta"].to(self.device))
        self.m.copy_(st["m"].to(self.device))
        self.v.copy_(st["v"].to(self.device))
        self.cur = 0
        self.x[0].copy_(st["x"].to(self.device))
        self.t = int(st["t"])

    def round_check(self):
        """Fresh rounding + check of the current delta: (unsat [n_inst, B], best [n_inst])."""
        return _abi.gs_round_check(self.prob, self.delta, bits=self.bits, unsat=self.unsat, best=self.best)

    def assignment(self, b: int) -> np.ndarray:
        """Rounded assignment of candidate b as 0/1 bytes (host)."""
        words = self.bits[:, b // 64].cpu().numpy().view(np.uint64)
        return ((words >> np.uint64(b % 64)) & np.uint64(1)).astype(np.uint8)[: self.n]


class STEngine:
    """Straight-through Gumbel training of one batch of B candidates (Eq. 3 with noise, Eq. 4 in
    the forward pass): step t evaluates the loss at the hard assignment x_hat_t = [delta + l_t > 0]
    (exact unsatisfied-clause counts), takes the integer gradient there through the soft chain
    y (1 - y) / tau, applies Adam and draws x_hat_{t+1}. The noise l is generated inside the
    kernels from (noise_seed, step). With ``noise_ring`` (default) each step also stores the next
    step's noise, which the next step reads instead of drawing it again (two [n, B] float32
    buffers); without it nothing per candidate is stored besides two bit-packed assignments."""

    def __init__(self, prob: _abi.Problem, B: int, adam: Optional[dict] = None, seed: int = 0, noise_seed: int = 1,
                 delta0: Optional[np.ndarray] = None, device="cuda", noise_ring: bool = True):
        self.prob = prob
        self.B = int(B)
        self.device = torch.device(device)
        self.adam = _abi._adam(adam) if adam is not None else None
        self.noise_seed = int(noise_seed)
        n = prob.n_vars
        self.n = n
        self.delta = candidates(n, B, torch.float32, device)
        self.m = candidates(n, B, torch.float32, device)
        self.v = candidates(n, B, torch.float32, device)
        self.nwd = (self.B + 63) // 64
        self.bits = [torch.zeros((max(n, 1), self.nwd), dtype=torch.int64, device=device) for _ in range(2)]
        self.unsat = torch.zeros((prob.n_inst, B), dtype=torch.int32, device=device)
        self.best = torch.zeros(prob.n_inst, dtype=torch.int32, device=device)
        self.noise = [candidates(n, B, torch.float32, device) for _ in range(2)] if noise_ring else None
        _abi.gs_reserve(prob, B, _abi.GS_F32)
        self.reset(seed, delta0)

    def reset(self, seed: int = 0, delta0: Optional[np.ndarray] = None) -> None:
        if delta0 is None:
            delta0 = synth.init_delta(self.n, self.B, seed)
        d = torch.from_numpy(np.ascontiguousarray(delta0[:, :self.B], dtype=np.float32))
        self.delta.copy_(d.to(self.device))
        self.m.zero_()
        self.v.zero_()
        self.t = 0
        self.cur = 0
        if self.noise is not None:
            _abi.gs_st_noise(self.prob, self.noise_seed, 1, self.noise[0])
        _abi.gs_st_sample(self.prob, self.delta, self.bits[0], seed=self.noise_seed, step=1,
                          noise=self.noise[0] if self.noise is not None else None)

    @property
    def bits_cur(self) -> torch.Tensor:
        """Hard assignment x_hat of the next step to run."""
        return self.bits[self.cur]

    def step(self, check: bool = True) -> None:
        """One training step (asynchronous on the current stream); with check, unsat / best hold
        the loss of this step's forward (the unsatisfied clauses of x_hat_t)."""
        self.t += 1
        if check:
            _abi.gs_check_bits(self.prob, self.bits[self.cur], self.B, self.unsat, self.best)
        ring = self.noise
        _abi.gs_st_step(self.prob, self.delta, self.m, self.v, self.bits[self.cur], self.bits[self.cur ^ 1],
                        self.t, seed=self.noise_seed, adam=self.adam,
                        noise=ring[self.cur] if ring is not None else None,
                        noise_next_out=ring[self.cur ^ 1] if ring is not None else None)
        self.cur ^= 1

    def state_dict(self) -> dict:
        """Logits, Adam moments, the hard assignment of the next step, its noise (ring), the step
        counter and the noise seed (host copies; the noise stream itself is a pure function of
        (seed, step), so nothing else is needed to continue bitwise)."""
        st = {"kind": "straight-through", "n": self.n, "B": self.B, "t": self.t, "noise_seed": self.noise_seed,
              "delta": self.delta.detach().cpu().clone(), "m": self.m.detach().cpu().clone(),
              "v": self.v.detach().cpu().clone(), "bits": self.bits[self.cur].detach().cpu().clone()}
        if self.noise is not None:
            st["noise"] = self.noise[self.cur].detach().cpu().clone()
        return st

    def load_state_dict(self, st: dict) -> None:
        if st.get("kind") != "straight-through" or st["n"] != self.n or st["B"] != self.B:
            raise ValueError("state does not match this engine (kind, n, B)")
        if (self.noise is not None) != ("noise" in st):
            raise ValueError("noise ring setting differs from the saved run")
        self.delta.copy_(st["delta"].to(self.device))
        self.m.copy_(st["m"].to(self.device))
        self.v.copy_(st["v"].to(self.device))
        self.cur = 0
        self.bits[0].copy_(st["bits"].to(self.device))
        if self.noise is not None:
            self.noise[0].copy_(st["noise"].to(self.device))
        self.t = int(st["t"])
        self.noise_seed = int(st["noise_seed"])

    def capture(self, steps: int, check: bool = True) -> torch.cuda.CUDAGraph:
        if steps % 2:
            raise ValueError("capture an even number of steps so the ping-pong buffers line up")
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                for _ in range(steps):
                    self.step(check)
        torch.cuda.current_stream().wait_stream(s)
        return g

    def run(self, steps: int, graph: bool = True, check: bool = True) -> None:
        if graph and steps >= 2:
            even = steps - (steps % 2)
            self.capture(even, check).replay()
            for _ in range(steps - even):
                self.step(check)
        else:
            for _ in range(steps):
                self.step(check)
