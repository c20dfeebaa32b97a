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


def test_film_packed_length_matches_the_binding_layout():
    """rxgs_film_param_count (host only) agrees with pack_film's layout and
    refuses sizes out of range."""
    import numpy as np
    from paper_2605_24290_gb300 import build, rxgs
    from paper_2605_24290_gb300 import synthetic as S
    lib = ctypes.CDLL(build.build())
    lib.rxgs_film_param_count.restype = ctypes.c_int64
    lib.rxgs_film_param_count.argtypes = [ctypes.c_int] * 4
    rng = np.random.default_rng(3)
    for F, dc, D, lmax in [(6, 16, 64, 9), (5, 16, 256, 4), (1, 0, 1, 0)]:
        p = S.draw_film(rng, lmax, F=F, dc=dc, D=D)
        flat = rxgs.pack_film(p)
        assert lib.rxgs_film_param_count(3 * F, dc, D, lmax) == flat.size
        assert rxgs.film_param_count(3 * F, dc, D, lmax) == flat.size
        back = rxgs.unpack_film(flat, 3 * F, dc, D, lmax)
        for k in rxgs.FILM_FIELDS:
            np.testing.assert_array_equal(back[k], p[k])
    for bad in [(0, 16, 64, 9), (33, 16, 64, 9), (18, 65, 64, 9), (18, 16, 257, 9),
                (18, 16, 64, 10), (18, -1, 64, 2)]:
        assert lib.rxgs_film_param_count(*bad) == 0


def test_film_packing_round_trip_with_torch():
    """pack_film / unpack_film keep every field, for numpy and torch."""
    torch = pytest.importorskip("torch")
    from paper_2605_24290_gb300 import rxgs
    import numpy as np
    from paper_2605_24290_gb300 import synthetic as S
    rng = np.random.default_rng(43)
    p = S.draw_film(rng, 3, F=2, dc=4, D=8)
    flat_np = rxgs.pack_film(p)
    flat_t = rxgs.pack_film({k: torch.from_numpy(v) for k, v in p.items()})
    assert isinstance(flat_t, torch.Tensor)
    np.testing.assert_array_equal(flat_t.numpy(), flat_np)
    back = rxgs.unpack_film(flat_t, *rxgs.film_sizes(p), 3)
    for k in rxgs.FILM_FIELDS:
        np.testing.assert_array_equal(back[k].numpy(), p[k])


def test_film_length_check_leaves_out_of_range_sizes_to_the_library():
    from paper_2605_24290_gb300 import rxgs
    n = rxgs.film_param_count(18, 16, 64, 9)
    rxgs.check_film_length(n, 18, 16, 64, 9)
    with pytest.raises(ValueError):
        rxgs.check_film_length(n - 1, 18, 16, 64, 9)
    rxgs.check_film_length(n, 18, 16, 300, 9)     # the library refuses hidden = 300
    rxgs.check_film_length(n, 18, 16, 64, 10)     # and lmax = 10
