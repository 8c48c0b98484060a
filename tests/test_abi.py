"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
symbol that include/difuser_im.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "difuser_im.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(im_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("im_graph_load", "im_sketch_build", "im_select_seeds", "im_spread_mc"):
        assert n in names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2410_14047_gb300 import _build
    import paper_2410_14047_gb300 as im

    path = _build.build()
    L = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing
    assert sorted(im.EXPORTS) == _declared()
    im.load_library(path)


def test_bounds_checked_variant_builds_and_exports_every_declared_symbol():
    from paper_2410_14047_gb300 import _build

    L = ctypes.CDLL(_build.build_bounds())
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing


def test_status_strings_without_gpu():
    import paper_2410_14047_gb300 as im

    L = im.load_library()
    for code, name in im.STATUS.items():
        assert L.im_status_str(code).decode() == name


def test_ctx_create_without_gpu_fails_cleanly():
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2410_14047_gb300 as im

    L = im.load_library()
    h = ctypes.c_void_p()
    st = L.im_ctx_create(0, None, 0, None, ctypes.byref(h))
    assert st == -4  # IM_E_CUDA, no crash


def test_missing_library_fails_loudly(tmp_path):
    import paper_2410_14047_gb300 as im

    with pytest.raises(im.IMError):
        im.load_library(str(tmp_path / "nope.so"))
    assert str(tmp_path / "nope.so") not in im._libs
