"""torch.autograd.Function around the C ABI: the misfit J(m) of a batch of shots whose
backward is the hand-written adjoint (Eq. 2 exact, or Eq. 3 probed), for the isotropic
acoustic and the pseudo-acoustic TTI equations.

    loss = WaveMisfit.apply(m, problem)      # m: padded squared slowness (float32, CUDA)
    loss.backward()                          # m.grad = dJ/dm (probed or exact)

The variant is chosen per call: "probed" keeps r projections per shot (the method's
memory), "full" keeps the whole forward history, "checkpoint" stores states every
`ncheck` steps and recomputes, "auto" picks the first of full / checkpoint / probed whose
workspace fits in the free device memory.  Every step runs in libwp.so's kernels.

Each variant propagates forward once per loss evaluation: the probed forward keeps P_u
(and the residual) for the backward, while the exact variants run their whole adjoint-state
call (forward with history or checkpoints, then the adjoint with the imaging condition)
inside `forward` and keep only the gradient, so that the history never outlives the call
and no second forward is needed in `backward`.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import wp


@dataclasses.dataclass
class Problem:
    """A batch of shots on one grid: geometry, wavelet, observed data and probing."""
    ndim: int
    nx: int
    ny: int
    nz: int
    nbl: int
    h: float
    dt: float
    nt: int
    src: np.ndarray                 # (S, nsrc, 3) or (S, 3), metres
    rec: np.ndarray                 # (S, nrec, 3) or (nrec, 3)
    wavelet: torch.Tensor           # (nt,) CUDA float32
    d_obs: torch.Tensor             # (S, nt, nrec) CUDA float32
    Q: torch.Tensor | None = None   # (S, nt, r) CUDA float32 probing matrices
    scale: float | None = None      # estimator scale (default 1/r: Rademacher)
    Tb: int = 64
    variant: str = "auto"           # auto | probed | full | checkpoint
    ncheck: int = 64
    damp_v: float = 0.0
    last_variant: str = ""
    # pseudo-acoustic TTI: (eps, delta, theta, phi) CUDA float32 fields on the padded grid;
    # None for the isotropic equation
    thomsen: tuple | None = None

    def geometry(self):
        return wp.Geometry(self.src, self.rec)

    @property
    def fields(self) -> int:
        """Wavefields per shot (2 for TTI: the projections cover both)."""
        return 2 if self.thomsen is not None else 1


def _model(p: Problem, m: torch.Tensor) -> wp.Model:
    # wp_model validates m on a stream of its own that does not wait for torch's: let the
    # work that produced m (an optimiser step, say) finish first
    torch.cuda.current_stream(m.device).synchronize()
    kw = {}
    if p.thomsen is not None:
        kw = dict(eps=p.thomsen[0], delta=p.thomsen[1], theta=p.thomsen[2], phi=p.thomsen[3])
    return wp.Model(p.ndim, p.nx, p.ny, p.nz, p.nbl, p.h, p.h, p.h, p.dt, p.nt, m, p.damp_v, **kw)


def choose_variant(p: Problem, M: wp.Model, G: wp.Geometry) -> str:
    if p.variant != "auto":
        return p.variant
    free, _ = torch.cuda.mem_get_info()
    budget = 0.8 * free
    if wp.wp_workspace_bytes(M.handle, G.c, 0, 1, wp.WP_MODE_EXACT_FULL) < budget:
        return "full"
    if wp.wp_workspace_bytes(M.handle, G.c, 0, p.ncheck, wp.WP_MODE_EXACT_CHECKPOINT) < budget:
        return "checkpoint"
    return "probed"


class WaveMisfit(torch.autograd.Function):
    """J(m) = 1/2 sum |R u - d_obs|^2 over the shots of `problem`; backward = dJ/dm."""

    @staticmethod
    def forward(ctx, m: torch.Tensor, problem: Problem):
        m = m.detach().contiguous()
        M = _model(problem, m)
        G = problem.geometry()
        variant = choose_variant(problem, M, G)
        problem.last_variant = variant
        S, nt, nrec = problem.d_obs.shape
        N = M.N
        J = torch.zeros(1, dtype=torch.float64, device=m.device)
        ctx.problem, ctx.variant, ctx.m = problem, variant, m
        if variant == "probed":
            if problem.Q is None:
                raise ValueError("the probed variant needs a probing matrix Q")
            r = problem.Q.shape[-1]
            ws = wp.workspace(wp.wp_workspace_bytes(M.handle, G.c, r, problem.Tb, wp.WP_MODE_PROBED), m.device)
            RS = M.use_aligned_probes()   # P_u stays internal: kept in the contraction's layout
            Pu = torch.empty((S * problem.fields, r, RS), device=m.device)
            dsyn = torch.empty((S, nt, nrec), device=m.device)
            wp.wp_probe_forward(M.handle, G.c, problem.wavelet, problem.Q, r, problem.Tb, Pu, dsyn, ws)
            res = torch.empty_like(dsyn)
            rws = wp.workspace(wp.wp_residual_workspace_bytes(dsyn.numel()), m.device)
            wp.wp_residual(dsyn, problem.d_obs, res, dsyn.numel(), J, rws)
            ctx.saved = (Pu, res, ws)
        else:
            # forward + adjoint in one call: the misfit now, the gradient kept for backward
            mode = wp.WP_MODE_EXACT_FULL if variant == "full" else wp.WP_MODE_EXACT_CHECKPOINT
            nck = 1 if variant == "full" else problem.ncheck
            ws = wp.workspace(wp.wp_workspace_bytes(M.handle, G.c, 0, nck, mode), m.device)
            g = torch.empty(N, device=m.device)
            wp.wp_exact_gradient(M.handle, G.c, problem.wavelet, problem.d_obs, g, J, None, mode,
                                 nck, ws)
            wp.wp_stream_status(ws)
            del ws
            ctx.saved = (g,)
        M.close()
        return J.to(torch.float32).reshape(())

    @staticmethod
    def backward(ctx, grad_out):
        p, variant, m = ctx.problem, ctx.variant, ctx.m
        if variant != "probed":
            (g,) = ctx.saved
            return (grad_out.to(g.dtype) * g).reshape(m.shape), None
        M = _model(p, m)
        M.use_aligned_probes()   # the layout P_u was written in
        G = p.geometry()
        g = torch.empty(M.N, device=m.device)
        Pu, res, ws = ctx.saved
        r = p.Q.shape[-1]
        scale = p.scale if p.scale is not None else 1.0 / r
        wp.wp_adjoint_image(M.handle, G.c, res, p.Q, r, p.Tb, scale, Pu, g, None, ws)
        wp.wp_stream_status(ws)
        M.close()
        return (grad_out.to(g.dtype) * g).reshape(m.shape), None
