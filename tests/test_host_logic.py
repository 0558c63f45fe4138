"""Host-side helpers of the Python layer (no GPU): the instance-capacity
growth after an overflow, the baked-record size and the launch structure."""
import os
import subprocess
import sys

import pytest

from paper_2410_08129_gb300 import binding as B
from paper_2410_08129_gb300.renderer import _grown_capacity


def test_capacity_grows_with_headroom_and_never_shrinks():
    assert _grown_capacity(1000, 10) == 1000 * 5 // 4 + 1024
    assert _grown_capacity(1000, 1 << 20) == 1 << 20            # never below the current capacity
    big = B.HTGS_MAX_CAPACITY - 10
    assert _grown_capacity(big, 1 << 20) == B.HTGS_MAX_CAPACITY  # clamped to the ABI's limit
    c = 1 << 16
    for needed in (70000, 300000, 5_000_000):                    # each growth covers what was needed
        c = _grown_capacity(needed, c)
        assert c >= needed


def test_capacity_beyond_the_limit_is_an_overflow():
    with pytest.raises(B.HTGSError) as e:
        _grown_capacity(B.HTGS_MAX_CAPACITY + 1, 1 << 20)
    assert e.value.status == B.HTGS_ERR_OVERFLOW


def test_launch_struct_fields():
    L = B.c_launch((32, 16), 2, smem_batch=64, test_lookback_stall=1)
    assert (L.tile_w, L.tile_h, L.px_per_thread, L.depth_bits, L.smem_batch, L.test_lookback_stall) == \
        (32, 16, 2, 0, 64, 1)
    assert B.c_launch().test_lookback_stall == 0
    assert all(e is None for e in B.c_launch().events)


def test_the_package_never_imports_the_oracle():
    """The product path (the package and its binding) has no route to the
    CPU oracle: importing every module leaves the oracle unloaded."""
    code = ("import sys, paper_2410_08129_gb300.binding, paper_2410_08129_gb300.renderer, "
            "paper_2410_08129_gb300.autotune, paper_2410_08129_gb300.scenes, paper_2410_08129_gb300.build; "
            "print(any(m == 'oracle' or m.startswith('oracle.') for m in sys.modules))")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=root, check=True)
    assert out.stdout.strip() == "False"
