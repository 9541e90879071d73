"""Python front end of the CUDA engine: workspace and stream plumbing around include/fd.h.

PyTorch supplies device memory (the workspace is one uint8 tensor sized by
fd_workspace_bytes) and the CUDA stream; every step of the scheme runs in
libfd.so.  Problems are the plain dicts produced by `synth.problem`.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _lib as L

_DT = {"f64": L.FD_F64, "f32": L.FD_F32, "bf16": L.FD_BF16, "f16": L.FD_F16}
_TORCH = {L.FD_F64: torch.float64, L.FD_F32: torch.float32}


def make_problem(p: dict, max_steps: int | None = None, state: str = "f32", hist: str | None = None,
                 accum: str | None = None, kahan: bool = False, keep_tape: bool = False,
                 allow_unstable: bool = False, ckpt_every: int = 0, timeout_ms: int = 0,
                 inject_stall: bool = False, tile_threads: int = 0, chunk_terms: int = 0,
                 stage_rows: int = 0, stages: int = 0, ctas_per_sm: int = 0,
                 head_lags: int = 0, plain_state: bool = False, time_block: int = 0,
                 step_updates: bool = False, fma_far: bool = False,
                 closed_tau: float | None = None) -> L.FdProblem:
    """fd_problem for a synth-style problem dict.  closed_tau: closed-loop adaptive memory with
    that threshold (FD_FLAG_CLOSED_LOOP)."""
    s = L.FdProblem()
    s.ndim, s.nx, s.ny = p["ndim"], p["nx"], p["ny"]
    s.gamma, s.alpha, s.dt, s.dx = p["gamma"], p["alpha"], p["dt"], p["dx"]
    s.bc = p["bc"]
    for i in range(4):
        s.react[i] = p["react"][i]
    s.mem_mode, s.mem_L, s.mem_a = p["mem_mode"], p["mem_L"], p["mem_a"]
    s.adaptive_rule = p.get("adaptive_rule", 0)
    s.state_dtype = _DT[state]
    s.hist_dtype = _DT[hist or state]
    s.accum_dtype = _DT[accum or ("f64" if state == "f64" else "f32")]
    s.flags = ((L.FD_FLAG_KAHAN if kahan else 0) | (L.FD_FLAG_KEEP_TAPE if keep_tape else 0) |
               (L.FD_FLAG_ALLOW_UNSTABLE if allow_unstable else 0) |
               (L.FD_FLAG_INJECT_STALL if inject_stall else 0) |
               (L.FD_FLAG_PLAIN_STATE if plain_state else 0) |
               (L.FD_FLAG_STEP_UPDATES if step_updates else 0) |
               (L.FD_FLAG_FMA_FAR if fma_far else 0) |
               (L.FD_FLAG_CLOSED_LOOP if closed_tau is not None else 0))
    s.mem_tau = float(closed_tau) if closed_tau is not None else 0.0
    s.max_steps = int(max_steps if max_steps is not None else p["K"])
    s.ckpt_every, s.timeout_ms = ckpt_every, timeout_ms
    s.tile_threads, s.chunk_terms, s.stage_rows = tile_threads, chunk_terms, stage_rows
    s.stages, s.ctas_per_sm, s.head_lags = stages, ctas_per_sm, head_lags
    s.nz = p.get("nz", 1)
    s.time_block = time_block
    return s


def _require_cuda():
    if not torch.cuda.is_available():
        raise RuntimeError("the fractional-diffusion engine runs on a CUDA GPU only")
    L.lib()


GEOMETRY_KEYS = ("tile_threads", "chunk_terms", "stage_rows", "stages", "ctas_per_sm", "head_lags",
                 "time_block", "step_updates", "fma_far")


def tuned_geometry(p: dict, kw: dict) -> dict:
    """The autotuner's geometry for a handle with options kw, unless kw sets one itself.  A
    taped handle (adjoint) takes blocks of at most 8 steps, the blocked adjoint's limit."""
    if any(k in kw for k in GEOMETRY_KEYS) or kw.get("closed_tau") is not None:
        return {}  # explicit geometry, or closed-loop memory (per-step kernel, built-in geometry)
    from .autotune import lookup
    geo = lookup(p, kw.get("state", "f32"), kw.get("hist"), kw.get("kahan", False))
    if kw.get("keep_tape") and geo.get("time_block", 0) > 8:
        geo["time_block"] = 8
    return geo


class FRD:
    """One problem instance bound to a device workspace and a stream.

    Without explicit launch-geometry options the autotuner's table is consulted (`tuned=False`
    keeps the library's built-in heuristics)."""

    def __init__(self, p: dict, device: str | torch.device = "cuda", stream=None, tuned: bool = True,
                 **kw):
        _require_cuda()
        if tuned:
            kw.update(tuned_geometry(p, kw))
        self.problem = p
        self.prob = make_problem(p, **kw)
        self.device = torch.device(device)
        self.N = p["nx"] * p["ny"] * p.get("nz", 1)
        self.dtype = _TORCH[self.prob.state_dtype]
        self.ws_bytes = L.fd_workspace_bytes(self.prob)
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.h = L.fd_init(self.prob, self.ws.data_ptr(), self.ws_bytes, self.stream.cuda_stream)
        self._keep = []

    # -- state ------------------------------------------------------------------------------
    def _as_state(self, u) -> torch.Tensor:
        if isinstance(u, np.ndarray):
            u = torch.from_numpy(np.ascontiguousarray(u))
        u = u.reshape(-1)
        if u.device.type == "cuda":
            return u.to(self.dtype).contiguous()
        return u.to(self.dtype).contiguous()

    def set_state(self, u0):
        t = self._as_state(u0)
        self._keep = [t]
        L.fd_set_state(self.h, t.data_ptr())

    def step(self, n: int):
        L.fd_step(self.h, n)

    def run(self, n: int) -> torch.Tensor:
        out = torch.empty(self.N, dtype=self.dtype, device=self.device)
        L.fd_run(self.h, n, out.data_ptr())
        return out

    def state(self) -> torch.Tensor:
        out = torch.empty(self.N, dtype=self.dtype, device=self.device)
        L.fd_get_state(self.h, out.data_ptr())
        return out

    def save(self, device: bool = False) -> torch.Tensor:
        """Checkpoint at the current step (fd_save): a uint8 tensor in host memory, or on the
        handle's device with device=True."""
        n = L.fd_save_bytes(self.h)
        buf = torch.empty(n, dtype=torch.uint8, device=self.device if device else "cpu")
        L.fd_save(self.h, buf.data_ptr(), n)
        return buf

    def load(self, buf: torch.Tensor):
        """Resume from a checkpoint that save() wrote for the same problem and geometry (fd_load)."""
        buf = buf.contiguous()
        L.fd_load(self.h, buf.data_ptr(), buf.numel())

    @property
    def k(self) -> int:
        return L.fd_current_step(self.h)

    def status(self) -> int:
        return L.fd_get_status(self.h)

    def memory_terms(self) -> int:
        """Memory terms (lag, weight) used by the steps run so far, lag 0 included."""
        return L.fd_memory_terms(self.h)

    def error_info(self) -> dict:
        """Where a device wait gave up after a timeout (site and raw words)."""
        return L.fd_get_error_info(self.h)

    def geometry(self) -> dict:
        return L.fd_get_geometry(self.h)

    # -- adjoint ----------------------------------------------------------------------------
    def adjoint(self, dJ_duK) -> dict:
        g = self._as_state(dJ_duK)
        if g.device.type != "cuda":
            g = g.to(self.device)
        du0 = torch.empty(self.N, dtype=self.dtype, device=self.device)
        dgam, dalp, dr = L.fd_adjoint(self.h, g.data_ptr(), du0.data_ptr())
        return dict(du0=du0, dgamma=dgam, dalpha=dalp, dreact=dr)

    def close(self):
        if getattr(self, "h", None):
            L.fd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FRDBatch:
    """Many independent instances advanced by one persistent launch (replayed CUDA graph)."""

    def __init__(self, problems: list, device: str | torch.device = "cuda", stream=None,
                 tuned: bool = True, **kw):
        _require_cuda()
        if tuned and not any(k in kw for k in GEOMETRY_KEYS):
            from .autotune import lookup_batch
            kw.update(lookup_batch(problems, kw.get("state", "f32")))
        self.problems = problems
        self.device = torch.device(device)
        self.probs = [make_problem(p, **kw) for p in problems]
        self.dtype = _TORCH[self.probs[0].state_dtype]
        self.ws_bytes = L.fd_batch_workspace_bytes(self.probs)
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.b = L.fd_batch_init(self.probs, self.ws.data_ptr(), self.ws_bytes, self.stream.cuda_stream)
        self._keep = []

    def set_state(self, i: int, u0):
        t = torch.as_tensor(u0).reshape(-1).to(self.dtype).contiguous()
        self._keep.append(t)
        L.fd_batch_set_state(self.b, i, t.data_ptr())

    def run(self):
        L.fd_batch_run(self.b)

    def state(self, i: int) -> torch.Tensor:
        p = self.problems[i]
        out = torch.empty(p["nx"] * p["ny"] * p.get("nz", 1), dtype=self.dtype, device=self.device)
        L.fd_batch_get_state(self.b, i, out.data_ptr())
        return out

    def geometry(self, i: int) -> dict:
        return L.fd_batch_get_geometry(self.b, i)

    def status(self) -> int:
        s = L.fd_batch_get_status(self.b)
        self._keep = []
        return s

    def close(self):
        if getattr(self, "b", None):
            L.fd_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FRDFunction(torch.autograd.Function):
    """u^K = FRD(u0; gamma, alpha, react) with the reverse-time adjoint as its backward.

    forward(u0, gamma, alpha, react, cfg): cfg = dict(problem=<synth dict>, K=steps,
    state="f32"|"f64", ckpt_every=C, options=dict(...) of further FRD options such as
    time_block).  Gradients flow to u0, gamma, alpha and react (a length-4 tensor), for the
    full, short and adaptive memory of the problem.
    """

    @staticmethod
    def forward(ctx, u0, gamma, alpha, react, cfg):
        p = dict(cfg["problem"])
        p["gamma"] = float(gamma)
        p["alpha"] = float(alpha)
        p["react"] = [float(x) for x in torch.as_tensor(react).reshape(-1).tolist()]
        K = int(cfg["K"])
        solver = FRD(p, device=u0.device, max_steps=K, state=cfg.get("state", "f32"), keep_tape=True,
                     ckpt_every=int(cfg.get("ckpt_every", 200)), **cfg.get("options", {}))
        solver.set_state(u0.detach())
        uK = solver.run(K)
        ctx.solver = solver
        ctx.pdtype = torch.as_tensor(gamma).dtype if torch.is_tensor(gamma) else torch.float64
        return uK.reshape(u0.shape)

    @staticmethod
    def backward(ctx, grad):
        r = ctx.solver.adjoint(grad.reshape(-1).contiguous())
        ctx.solver.close()
        f64 = dict(dtype=torch.float64)
        return (r["du0"].reshape(grad.shape), torch.tensor(r["dgamma"], **f64),
                torch.tensor(r["dalpha"], **f64), torch.tensor(r["dreact"], **f64), None)
