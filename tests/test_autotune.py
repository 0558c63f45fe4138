"""Host logic of the autotuner (no GPU: a fake timer stands in for the
CUDA-event timing). The search is coordinate-wise: every (tile shape, pixels
per thread) candidate at the first staging batch, then the other batches for
the fastest pair only; unsupported candidates are skipped; results are cached
per workload key."""
import pytest

from paper_2410_08129_gb300 import autotune as at
from paper_2410_08129_gb300 import binding as B


def _fake(ms_of, calls, unsupported=()):
    def timer(step_for_launch, launch, warmup, repeats):
        k = ((launch.tile_w, launch.tile_h), launch.px_per_thread, launch.smem_batch)
        calls.append(k)
        if k[:2] in unsupported:
            raise B.HTGSError(B.HTGS_ERR_NOT_SUPPORTED, "fake")
        return ms_of(k)
    return timer


def test_coordinate_search_picks_the_fastest():
    def ms(k):
        (tw, th), ppt, b = k
        base = {(32, 16): 1.0, (16, 16): 1.2}.get((tw, th), 2.0) + 0.3 * (ppt - 1)
        return base + {128: 0.05, 192: 0.02, 64: 0.0, 32: 0.1}[b]
    calls = []
    launch, times = at.autotune(lambda L: None, candidates=at.CANDIDATES, timer=_fake(ms, calls))
    assert ((launch.tile_w, launch.tile_h), launch.px_per_thread, launch.smem_batch) == ((32, 16), 1, 64)
    # every candidate at batch 128, then 192, 64 and 32 for the winner only
    assert calls[:len(at.CANDIDATES)] == [(t, p, 128) for t, p in at.CANDIDATES]
    assert calls[len(at.CANDIDATES):] == [((32, 16), 1, 192), ((32, 16), 1, 64), ((32, 16), 1, 32)]
    assert len(times) == len(at.CANDIDATES) + 3


def test_unsupported_candidates_are_skipped_and_results_cached():
    calls = []
    timer = _fake(lambda k: 1.0 if k[0] == (16, 8) else 3.0, calls, unsupported={((16, 16), 1), ((16, 16), 2)})
    key = ("unit-test", 1)
    at._cache.pop(key, None)
    launch, times = at.autotune(lambda L: None, key=key, timer=timer)
    assert (launch.tile_w, launch.tile_h) == (16, 8)
    assert all(k[0] != (16, 16) for k in times)
    n = len(calls)
    again, times2 = at.autotune(lambda L: None, key=key, timer=timer)
    assert len(calls) == n and times2 is times
    assert (again.tile_w, again.tile_h, again.px_per_thread, again.smem_batch) == \
        (launch.tile_w, launch.tile_h, launch.px_per_thread, launch.smem_batch)
    at._cache.pop(key, None)


def test_no_runnable_candidate_is_an_error():
    with pytest.raises(B.HTGSError) as e:
        at.autotune(lambda L: None, candidates=[((16, 16), 1)],
                    timer=_fake(lambda k: 1.0, [], unsupported={((16, 16), 1)}))
    assert e.value.status == B.HTGS_ERR_NOT_SUPPORTED
