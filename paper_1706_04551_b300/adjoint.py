"""Gauge time series of the 2D step as a differentiable PyTorch function.

``gauge_series(H, eta0, ...)`` runs ``nsteps`` steps of fixed size dt through the C-ABI
(nh_step) and returns eta at the gauge cells after every step; its backward is the
hand-written adjoint of libnh (nh_step_taped / nh_adjoint_step) with checkpointed
recomputation: the state is kept every ``checkpoint`` steps in the forward pass, and each
segment is retaken with tapes before it is reversed.  Everything that computes runs in
libnh's CUDA kernels; this module moves arguments and device buffers (torch supplies the
memory) and adds the loss's gauge adjoints into eta_bar between reverse steps.
"""
from __future__ import annotations

import torch

from . import nh


class _Spec:
    def __init__(self, dx, dt, nsteps, gauges, precision, checkpoint, bc, params):
        self.dx, self.dt, self.nsteps = float(dx), float(dt), int(nsteps)
        self.gauges = [(int(i), int(j)) for i, j in gauges]
        self.precision, self.checkpoint = precision, int(checkpoint)
        self.bc, self.params = tuple(bc), dict(params)
        self.stats = {}


def _dtype(precision):
    return torch.float32 if precision == "fp32" else torch.float64


class GaugeRun(torch.autograd.Function):
    """eta at the gauges after steps 1..N as a function of (H, eta0, q1, q2)."""

    @staticmethod
    def forward(ctx, H, eta0, q1, q2, spec):
        dev = torch.device("cuda")
        td = _dtype(spec.precision)
        ny, nx = H.shape
        sim = nh.Sim(H.detach().double().cpu().numpy(), spec.dx, bc=spec.bc,
                     precision=spec.precision, **spec.params)
        e0 = eta0.detach().to(dev, td).contiguous().reshape(-1)
        a0 = q1.detach().to(dev, td).contiguous().reshape(-1)
        b0 = q2.detach().to(dev, td).contiguous().reshape(-1)
        sim.set_state(e0, a0, b0)
        gidx = torch.tensor([i * nx + j for i, j in spec.gauges], device=dev)
        gcells = gidx.to(torch.int32)
        ng = len(spec.gauges)
        series = torch.empty((spec.nsteps, ng), dtype=td, device=dev)
        nn = (nx + 1) * (ny + 1)
        cps = []
        prof = spec.stats.get("profile", False)
        if prof:
            sim.profile(True)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        for n in range(spec.nsteps):
            if n % spec.checkpoint == 0:
                cp = [torch.empty(nx * ny, dtype=td, device=dev) for _ in range(3)]
                cp += [torch.empty(nn, dtype=td, device=dev) for _ in range(2)]
                sim.get_state_into(*cp)
                cps.append(cp)
            sim.step(spec.dt)
            sim.gauges(gcells, series[n])   # one gather kernel on the handle's stream
        ev[1].record()
        torch.cuda.synchronize()
        spec.stats["forward_ms"] = ev[0].elapsed_time(ev[1])
        if prof:
            spec.stats["forward_kernels"] = sim.profile_read()
            sim.profile(True)
        ctx.sim, ctx.cps, ctx.spec, ctx.gidx = sim, cps, spec, gidx
        ctx.shape, ctx.hdev = (ny, nx), H.device
        return series.double().to(H.device)

    @staticmethod
    def backward(ctx, gout):
        sim, spec, gidx = ctx.sim, ctx.spec, ctx.gidx
        ny, nx = ctx.shape
        dev = torch.device("cuda")
        td = _dtype(spec.precision)
        nn = (nx + 1) * (ny + 1)
        g = gout.detach().to(dev, torch.float64)
        eb = torch.zeros(nx * ny, dtype=td, device=dev)
        ab = torch.zeros_like(eb)
        bb = torch.zeros_like(eb)
        wb = torch.zeros(nn, dtype=td, device=dev)
        Hb = torch.zeros_like(eb)
        tb = sim.tape_bytes()
        K = spec.checkpoint
        tape = torch.empty(min(K, spec.nsteps) * tb, dtype=torch.uint8, device=dev)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        for seg in reversed(range(len(ctx.cps))):
            n0 = seg * K
            n1 = min(n0 + K, spec.nsteps)
            sim.set_state(*ctx.cps[seg])
            for n in range(n0, n1):
                sim.step_taped(tape[(n - n0) * tb:(n - n0 + 1) * tb], spec.dt)
            for n in reversed(range(n0, n1)):
                eb.index_add_(0, gidx, g[n].to(td))
                sim.adjoint_step(tape[(n - n0) * tb:(n - n0 + 1) * tb], spec.dt, eb, ab, bb,
                                 wb, Hb)
        ev[1].record()
        torch.cuda.synchronize()
        spec.stats["backward_ms"] = ev[0].elapsed_time(ev[1])
        if spec.stats.get("profile", False):
            spec.stats["backward_kernels"] = sim.profile_read()
            sim.profile(False)
        sim.close()
        ctx.sim = None
        shape, hd = ctx.shape, ctx.hdev
        cvt = lambda t: t.reshape(shape).to(hd, torch.float64)
        return cvt(Hb), cvt(eb), cvt(ab), cvt(bb), None


def gauge_series(H, eta0, q1=None, q2=None, *, dx, dt, nsteps, gauges, precision="fp32",
                 checkpoint=100, bc=(nh.WALL,) * 4, stats=None, **params):
    """eta at `gauges` ((row, column) cells) after each of `nsteps` steps of size `dt`,
    differentiable with respect to H, eta0, q1, q2 (float64 torch tensors [ny][nx]).
    `params` are nh_params fields (tol, max_iter, solver, ...); friction and breaking are
    not allowed (the adjoint does not cover them).  If `stats` is a dict it receives the
    device times of the forward and backward passes (ms)."""
    if q1 is None:
        q1 = torch.zeros_like(eta0)
    if q2 is None:
        q2 = torch.zeros_like(eta0)
    spec = _Spec(dx, dt, nsteps, gauges, precision, checkpoint, bc, params)
    if stats is not None:
        spec.stats = stats
    return GaugeRun.apply(H, eta0, q1, q2, spec)


def misfit(series, target):
    """J = sum over steps and gauges of (eta - target)^2."""
    return ((series - target) ** 2).sum()


__all__ = ["gauge_series", "misfit", "GaugeRun"]
