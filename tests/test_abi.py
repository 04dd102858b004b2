"""The C-ABI library builds, loads on a machine without a GPU, and exports every entry
point that include/gs.h declares (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^int\s+(gs_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_path():
    names = _declared()
    for need in ("gs_project", "gs_bin_sort", "gs_render_fwd", "gs_apply_ctf", "gs_loss",
                 "gs_render_bwd", "gs_step"):
        assert need in names


def test_library_exports_every_declared_symbol():
    from paper_2508_04929_b300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name
    from paper_2508_04929_b300 import _lib
    assert sorted(_lib.EXPORTED) == _declared()


def test_host_side_validation_without_gpu():
    """Size queries and argument checks run on the host; no kernel is launched."""
    from paper_2508_04929_b300 import _lib as L
    assert L.gs_tiles_per_image(L.config(256, tile=8)) == 1024
    assert L.gs_tiles_per_image(L.config(40, tile=16)) == 9
    with pytest.raises(L.GsError):
        L.gs_tiles_per_image(L.config(64, tile=12))
    with pytest.raises(L.GsError):
        L.gs_workspace_size(L.config(64, chunk=40), 1, 10)
    with pytest.raises(L.GsError):
        L.gs_workspace_size(L.config(4096, tile=8), 1, 10)  # 512 tiles per side > 64
    a = L.gs_workspace_size(L.config(64), 8, 2000, 0)
    b = L.gs_workspace_size(L.config(64), 8, 2000, 4096)
    assert b >= a + 4096 and a % 256 == 0
    # gs_project's output: 32-byte records, the 8-byte box plane, the 8-byte low-part plane
    assert L.gs_proj_size(128, 100_000) == 128 * 100_000 * 48
    assert L.gs_proj_size(0, 10) == 0
    with pytest.raises(L.GsError):
        L.gs_proj_size(-1, 10)


def test_binding_rejects_host_tensors_without_gpu():
    """Every device argument is checked before the call: a host (CPU) tensor raises
    ValueError instead of handing the kernels a host pointer."""
    torch = pytest.importorskip("torch")
    from paper_2508_04929_b300 import _lib as L
    cfg = L.config(64)
    with pytest.raises(ValueError, match="CUDA device memory"):
        L.gs_project(cfg, torch.zeros(10, 11), torch.zeros(2, 9), torch.zeros(1000, dtype=torch.uint8),
                     torch.zeros(1000, dtype=torch.uint8))
    with pytest.raises(ValueError, match="rows of 11"):
        L.gs_project(cfg, torch.zeros(10, 12), torch.zeros(2, 9), None, None)

