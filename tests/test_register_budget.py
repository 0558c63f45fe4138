"""Register budget of the hot kernels, read from ptxas's resource report when
compiling for sm_103a (no GPU needed). Occupancy is set per kernel with
__launch_bounds__: the one-pixel-per-thread forward blend at K <= 8 runs four
CTAs of 256 threads (64 registers, where every spill measured slower on
GB300), and the adjoint blend is sized for three CTAs of 256 threads. These
tests keep those budgets from regressing unnoticed."""
import os
import re
import subprocess
import tempfile

import pytest

from paper_2410_08129_gb300 import build as build_mod

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2410_08129_gb300", "csrc")


def _resources(src):
    """{mangled kernel name: (registers, spill store bytes)} for one unit."""
    try:
        nvcc = build_mod._nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    with tempfile.TemporaryDirectory() as d:
        cmd = [nvcc] + build_mod._flags() + ["-Xptxas", "-v", "-c", os.path.join(CSRC, src), "-o",
                                              os.path.join(d, "x.o")]
        r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out, name, spill = {}, None, 0
    for line in r.stderr.splitlines():
        m = re.search(r"Compiling entry function '([^']+)'", line)
        if m:
            name = m.group(1)
        m = re.search(r"(\d+) bytes spill stores", line)
        if m and name:
            spill = int(m.group(1))
        m = re.search(r"Used (\d+) registers", line)
        if m and name:
            out[name] = (int(m.group(1)), spill)
            name, spill = None, 0
    return out


def _find(res, prefix, targs):
    # Itanium mangling of blend_fwd_kernel<8, 16, 16, 1, false> etc.
    keys = [k for k in res if prefix in k and targs in k]
    assert len(keys) == 1, (prefix, targs, keys)
    return res[keys[0]]


def test_forward_blend_budget():
    res = _resources("blend_k8.cu")
    for targs in ("ILi8ELi16ELi16ELi1ELb0E", "ILi8ELi32ELi16ELi1ELb0E"):   # K = 8, 16x16 and 32x16, 1 px/thread
        regs, spill = _find(res, "blend_fwd_kernel", targs)
        assert spill == 0 and regs <= 64, (targs, regs, spill)   # four resident CTAs of 256 threads
    regs, spill = _find(res, "blend_fwd_kernel", "ILi8ELi16ELi16ELi2ELb0E")  # 2 px/thread: 4 CTAs of 128
    assert spill == 0 and regs <= 128


def test_large_core_budgets():
    regs, spill = _find(_resources("blend_k16.cu"), "blend_fwd_kernel", "ILi16ELi16ELi16ELi1ELb0E")
    assert spill == 0 and regs <= 85      # three resident CTAs of 256 threads
    regs, spill = _find(_resources("blend_k32.cu"), "blend_fwd_kernel", "ILi32ELi16ELi16ELi1ELb0E")
    assert spill == 0 and regs <= 128     # two resident CTAs


def test_adjoint_blend_budget():
    res = _resources("blend_bwd.cu")
    for targs in ("ILi16ELi16ELb0ELb0E", "ILi32ELi16ELb0ELb0E"):
        regs, spill = _find(res, "blend_bwd_kernel", targs)
        assert regs <= 85 and spill <= 16, (targs, regs, spill)   # three resident CTAs of 256 threads
