"""Autotuning of launch parameters on a live run.

The tuned parameters change only speed, never results: the L2 prefetch distances of
the stream-collide kernel (of plain steps, and of the steps that also sum their
result), of the order-parameter kernel, and for the single-pass step its planes per
segment and prefetch distance in planes (lbm_set_tuning).  Each candidate is timed with
the library's CUDA-event kernel profile over a few steps of the run itself, so tuning
advances the simulation by (number of candidates) x (warm + steps) steps.
"""
from __future__ import annotations

from typing import Dict, Iterable, Optional

from . import lbm as L

# candidate distances as fractions of the default (one wave of resident blocks)
DEFAULT_FRACTIONS = (0.0, 0.33, 0.5, 0.67, 0.83, 1.0, 1.17)


def _time_kernel(ctx, kernel: int, steps: int, warm: int, sums: bool = False) -> float:
    """Mean duration (ms) of `kernel` over `steps` steps after `warm` untimed ones; with
    sums, steps that also sum their result (lbm_step_reduce_async, one step per call,
    back to back as a run that checks every step enqueues them)."""
    L.lbm_step(ctx, warm)
    if sums:
        # the whole step, timed on the context's stream: with its sums every step
        # launches two small reductions after the stream-collide pass, and the prefetch
        # distance that suits the pass alone need not suit the sequence
        import torch
        stream = torch.cuda.ExternalStream(ctx.stream) if ctx.stream else torch.cuda.default_stream()
        out = torch.zeros(8, dtype=torch.float64, device="cuda")
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record(stream)
        for _ in range(steps):
            L.lbm_step_reduce_async(ctx, 1, out.data_ptr())
        t1.record(stream)
        t1.synchronize()
        return t0.elapsed_time(t1) / steps
    L.lbm_profile(ctx, True)
    L.lbm_step(ctx, steps)
    ms, n = L.lbm_profile_read(ctx, kernel)
    L.lbm_profile(ctx, False)
    return ms / max(n, 1)


TUNED = (("prefetch_collide", L.LBM_TUNE_PREFETCH_COLLIDE, L.KERNEL_COLLIDE, False),
         ("prefetch_phi", L.LBM_TUNE_PREFETCH_PHI, L.KERNEL_PHI, False),
         ("prefetch_collide_sums", L.LBM_TUNE_PREFETCH_COLLIDE_SUMS, L.KERNEL_COLLIDE, True))


def autotune(ctx, steps: int = 16, warm: int = 2,
             fractions: Iterable[float] = DEFAULT_FRACTIONS) -> Dict[str, dict]:
    """Pick the fastest prefetch distance for k_collide (of plain steps and of summing
    steps) and k_phi; returns, per parameter, the chosen value and the mean kernel time
    of every candidate (ms)."""
    out = {}
    for name, param, kernel, sums in TUNED:
        base = L.lbm_get_tuning(ctx, param)
        cands = sorted({int(round(f * base)) for f in fractions})
        times = {}
        for v in cands:
            L.lbm_set_tuning(ctx, param, v)
            times[v] = _time_kernel(ctx, kernel, steps, warm, sums)
        best = min(times, key=times.get)
        L.lbm_set_tuning(ctx, param, best)
        out[name] = {"value": best, "default": base, "ms": {str(k): round(t, 5) for k, t in times.items()}}
    return out


def tuning_steps(steps: int = 16, warm: int = 2, fractions: Optional[Iterable[float]] = None) -> int:
    """Number of time steps autotune() advances the run by."""
    n = len(set(fractions or DEFAULT_FRACTIONS))
    return len(TUNED) * n * (steps + warm)


def autotune_fused(ctx, steps: int = 6, warm: int = 2,
                   segments: Iterable[int] = (0, 16, 32, 64),
                   prefetch: Iterable[int] = (0, 1, 2)) -> Dict[str, dict]:
    """For the single-pass step (LBM_TUNE_FUSED): pick the planes per segment and the L2
    prefetch distance in planes by timing the kernel on the live run."""
    times = {}
    for seg in segments:
        L.lbm_set_tuning(ctx, L.LBM_TUNE_FUSED_SEGMENT, seg)
        for pf in prefetch:
            L.lbm_set_tuning(ctx, L.LBM_TUNE_FUSED_PREFETCH, pf)
            times[(seg, pf)] = _time_kernel(ctx, L.KERNEL_COLLIDE, steps, warm)
    seg, pf = min(times, key=times.get)
    L.lbm_set_tuning(ctx, L.LBM_TUNE_FUSED_SEGMENT, seg)
    L.lbm_set_tuning(ctx, L.LBM_TUNE_FUSED_PREFETCH, pf)
    return {"fused_segment": {"value": L.lbm_get_tuning(ctx, L.LBM_TUNE_FUSED_SEGMENT)},
            "fused_prefetch": {"value": pf,
                               "ms": {f"{s}/{p}": round(t, 5) for (s, p), t in times.items()}}}
