"""Autotuner for the launch configuration of a workload.

Tile shape, the forward's pixels per thread and the number of records the
forward stages per shared-memory batch change only the schedule (the
per-pixel arithmetic and the gid-ascending traversal are the same), so the
fastest one can be picked by timing. K, tau_alpha and tau_K are method
parameters and never tuned. The search is coordinate-wise: every (tile
shape, pixels per thread) candidate at the default batch of 128 records,
then the other batch sizes for the best one. Results are cached per
workload signature.
"""
from __future__ import annotations

import torch

from . import binding as B

# (tile shape, forward pixels per thread) candidates compiled into the library.
CANDIDATES = [((16, 16), 1), ((16, 16), 2), ((32, 16), 1), ((32, 16), 2), ((16, 8), 1), ((16, 8), 2), ((8, 8), 1),
              ((8, 8), 2)]
# Records per shared-memory batch of the forward blend (the first is the default;
# 192 stages into two buffers instead of three).
BATCHES = (128, 192, 64, 32)

_cache: dict = {}


def signature(cameras, n_gaussians, params, backward: bool):
    res = tuple(sorted({(c.width, c.height) for c in cameras}))
    return (res, int(n_gaussians), int(params.K), bool(backward))


def _time(step_for_launch, launch, warmup, repeats):
    step = step_for_launch(launch)
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(repeats):
        step()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / repeats


def autotune(step_for_launch, key=None, candidates=CANDIDATES, batches=BATCHES, warmup=1, repeats=3,
             timer=_time):
    """step_for_launch(launch) -> callable running one step on the current
    stream with that launch configuration (the callable may allocate on its
    first use). Returns (best htgs_launch, {(tile, ppt, batch): ms}). A
    candidate whose step raises HTGSError (a shape the library does not
    support for this configuration) is skipped; timer(step_for_launch,
    launch, warmup, repeats) -> ms measures one candidate."""
    if key is not None and key in _cache:
        tile, ppt, batch = _cache[key][0]
        return B.c_launch(tile, ppt, smem_batch=batch), _cache[key][1]
    times = {}
    for tile, ppt in candidates:
        try:
            times[(tile, ppt, batches[0])] = timer(step_for_launch, B.c_launch(tile, ppt, smem_batch=batches[0]),
                                                   warmup, repeats)
        except B.HTGSError:
            continue
    if not times:
        raise B.HTGSError(B.HTGS_ERR_NOT_SUPPORTED, "autotune: no candidate launch ran")
    tile, ppt, _ = min(times, key=times.get)
    for batch in batches[1:]:
        try:
            times[(tile, ppt, batch)] = timer(step_for_launch, B.c_launch(tile, ppt, smem_batch=batch),
                                              warmup, repeats)
        except B.HTGSError:
            continue
    best = min(times, key=times.get)
    if key is not None:
        _cache[key] = (best, times)
    return B.c_launch(best[0], best[1], smem_batch=best[2]), times
