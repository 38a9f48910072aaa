"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/*.h declares; argument checks that need no device work."""
import ctypes as C
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(spl_[A-Za-z0-9_]+)\s*\(",
                             src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1309_1114_gb300.build import build_library
    from paper_1309_1114_gb300 import splotch
    build_library()
    return splotch.load_library()


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("spl_create", "spl_destroy", "spl_load_particles", "spl_set_camera",
                 "spl_set_colormap", "spl_set_params", "spl_render", "spl_render_batch",
                 "spl_get_stats", "spl_error_string"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert missing == []


def test_binding_wraps_every_declared_symbol():
    from paper_1309_1114_gb300 import splotch
    missing = [n for n in declared_functions() if not callable(getattr(splotch, n, None))]
    assert missing == []


def test_host_side_argument_checks(lib):
    from paper_1309_1114_gb300 import splotch as S
    assert lib.spl_create(None, 0, None) == S.SPL_EINVAL
    assert lib.spl_default_params(None) == S.SPL_EINVAL
    assert lib.spl_destroy(None) == S.SPL_OK
    assert lib.spl_render(None, None, None) == S.SPL_EINVAL
    assert lib.spl_get_stats(None, None) == S.SPL_EINVAL
    q = S.spl_params()
    assert lib.spl_default_params(C.byref(q)) == S.SPL_OK
    assert (q.chi, q.r_sml, q.tile_px) == (3.0, 0.5, 32)
    assert lib.spl_error_string(S.SPL_EINVAL) == b"invalid argument"
    assert lib.spl_error_string(12345) == b"unknown status"
