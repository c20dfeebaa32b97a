"""The C-ABI library builds and exports every symbol include/rxgs.h declares.
No compute call: runs without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "rxgs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rxgs_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["rxgs_create", "rxgs_upload_scene", "rxgs_prepare", "rxgs_render",
              "rxgs_render_views", "rxgs_render_backward", "rxgs_sync"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2605_24290_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2605_24290_gb300 import rxgs
    assert set(declared_functions()) <= set(rxgs.SIGNATURES)


def test_default_options_without_gpu():
    from paper_2605_24290_gb300 import build, rxgs
    lib = ctypes.CDLL(build.build())
    o = rxgs.Options()
    lib.rxgs_default_options(ctypes.byref(o))
    assert (o.H, o.W, o.tile_h, o.tile_w) == (90, 360, 16, 16)
    assert o.q_max == 9.0 and abs(o.eps_T - 1e-4) < 1e-9


def test_context_refuses_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2605_24290_gb300 import rxgs
    with pytest.raises(RuntimeError):
        rxgs.Context()
