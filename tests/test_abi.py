"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/htgs.h declares; host-only entry points validate arguments."""
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2410_08129_gb300 import build as build_mod
from paper_2410_08129_gb300 import scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(htgs_\w+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib_path():
    return build_mod.build()


def test_every_declared_symbol_is_exported(lib_path):
    declared = _declared()
    assert len(declared) >= 7
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (htgs_\w+)", out))
    missing = [n for n in declared if n not in exported]
    assert not missing, missing


def test_library_loads_and_host_entry_points_work(lib_path):
    from paper_2410_08129_gb300 import binding as B
    L = B.lib()
    for n in _declared():
        assert hasattr(L, n)
    _, cam, prm, tile = scenes.config1()
    fwd, saved = B.htgs_workspace_size(256, cam, prm, B.c_launch(tile), 1 << 16)
    assert fwd % 256 == 0 and saved == (7 + prm.K) * 64 * 64 * 4
    lay = B.htgs_workspace_layout(256, cam, prm, B.c_launch(tile), 1 << 16)
    assert lay.n_tiles == 16 and lay.tiles_x == 4 and lay.tile_bits == 4
    assert B.htgs_status_string(B.HTGS_ERR_OVERFLOW) != B.htgs_status_string(B.HTGS_OK)
    assert "unknown" not in B.htgs_status_string(B.HTGS_ERR_INTERNAL)


@pytest.mark.parametrize("bad", ["K", "capacity", "tile", "batch", "n", "alpha_max", "size", "cover"])
def test_host_side_argument_checks(lib_path, bad):
    from paper_2410_08129_gb300 import binding as B
    _, cam, prm, tile = scenes.config1()
    n, cap, launch = 256, 1 << 16, B.c_launch(tile)
    if bad == "K":
        prm = scenes.Params(K=33)
        expect = B.HTGS_ERR_NOT_SUPPORTED
    elif bad == "capacity":
        cap = 1 << 31
        expect = B.HTGS_ERR_INVALID_ARG
    elif bad == "tile":
        launch = B.c_launch((12, 12))
        expect = B.HTGS_ERR_NOT_SUPPORTED
    elif bad == "batch":
        launch = B.c_launch(tile, smem_batch=48)
        expect = B.HTGS_ERR_NOT_SUPPORTED
    elif bad == "n":
        n = -1
        expect = B.HTGS_ERR_INVALID_ARG
    elif bad == "cover":
        launch = B.c_launch(tile, tile_cover=2)
        expect = B.HTGS_ERR_INVALID_ARG
    elif bad == "alpha_max":
        prm = scenes.Params(alpha_max=1.0)
        expect = B.HTGS_ERR_INVALID_ARG
    else:
        cam = scenes.identity_camera(0, 10, 10.0)
        expect = B.HTGS_ERR_INVALID_ARG
    with pytest.raises(B.HTGSError) as e:
        B.htgs_workspace_size(n, cam, prm, launch, cap)
    assert e.value.status == expect


@pytest.mark.parametrize("batch,ok", [(0, True), (32, True), (64, True), (128, True), (192, True), (96, False),
                                      (256, False)])
def test_staging_batch_sizes(lib_path, batch, ok):
    """The forward stages 32, 64, 128 or 192 records per batch (0 means the
    default); any other count is refused on the host."""
    from paper_2410_08129_gb300 import binding as B
    _, cam, prm, tile = scenes.config1()
    launch = B.c_launch(tile, smem_batch=batch)
    if ok:
        assert B.htgs_workspace_size(256, cam, prm, launch, 1 << 16)[0] > 0
    else:
        with pytest.raises(B.HTGSError) as e:
            B.htgs_workspace_size(256, cam, prm, launch, 1 << 16)
        assert e.value.status == B.HTGS_ERR_NOT_SUPPORTED


def test_oracle_is_not_linked_into_the_library(lib_path):
    out = subprocess.run(["nm", "-D", lib_path], capture_output=True, text=True, check=True).stdout
    assert "og_" not in out
    deps = subprocess.run(["readelf", "-d", lib_path], capture_output=True, text=True, check=True).stdout
    assert "htgs_oracle" not in deps


def test_baked_record_size_matches_the_header():
    """HTGS_BAKED_FLOATS(deg) of include/htgs.h, evaluated as written, equals
    the binding's baked_floats: 12 floats of activated geometry, 3 (deg + 1)^2
    SH coefficients, rounded up to a multiple of 4."""
    from paper_2410_08129_gb300 import binding as B
    hdr = open(os.path.join(ROOT, "include", "htgs.h")).read()
    m = re.search(r"#define HTGS_BAKED_FLOATS\(deg\)\s+(.+)", hdr)
    assert m
    expr = m.group(1).strip().replace("/", "//")
    for deg in range(4):
        assert eval(expr, {"deg": deg}) == B.baked_floats(deg)
        assert B.baked_floats(deg) % 4 == 0 and B.baked_floats(deg) >= 12 + 3 * (deg + 1) ** 2
    assert B.baked_floats(3) * 4 == 240


def test_static_scratch_size_matches_the_header():
    from paper_2410_08129_gb300 import binding as B
    hdr = open(os.path.join(ROOT, "include", "htgs.h")).read()
    m = re.search(r"#define HTGS_STATIC_SCRATCH_BYTES \((\d+)u \* (\d+)u \* (\d+)u\)", hdr)
    assert m and int(m.group(1)) * int(m.group(2)) * int(m.group(3)) == B.HTGS_STATIC_SCRATCH_BYTES
