"""CPU-side checks of the C ABI: the library builds, loads and exports every
function include/ebof.h declares; host-side helpers that need no device."""
import ctypes
import os
import re

import pytest

from tests.conftest import ROOT

HEADER = os.path.join(ROOT, "include", "ebof.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ebof_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("ebof_stream_create", "ebof_stream_destroy", "ebof_stream_reset",
                 "ebof_process_window", "ebof_process_windows", "ebof_stream_sync",
                 "ebof_status_string", "ebof_default_params", "ebof_alpha_from_dsat"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2112_10591_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_helpers_without_device():
    import paper_2112_10591_gb300 as eb
    p = eb.ebof_default_params(1280, 720)
    assert p.struct_size == ctypes.sizeof(eb.ebof_params)
    assert (p.levels, p.patch, p.stride, p.gn_iters) == (5, 12, 4, 12)
    p = eb.ebof_default_params(346, 260)
    assert (p.levels, p.patch, p.connectivity, p.n_d) == (3, 8, 8, 1)
    assert abs(p.alpha - 1.08) < 1e-6
    # Eq. 3: alpha = d_sat / ln 255
    assert abs(eb.ebof_alpha_from_dsat(6.0) - 1.0827835) < 1e-5
    assert eb.ebof_status_string(eb.EBOF_NO_PREVIOUS).startswith("first window")
    assert "invalid" in eb.ebof_status_string(eb.EBOF_ERR_INVALID_ARG)


def test_create_rejects_bad_params_before_touching_a_device():
    import paper_2112_10591_gb300 as eb
    bad = []
    for field, val in (("width", 0), ("height", 20000), ("connectivity", 6), ("n_d", -1),
                       ("alpha", 0.0), ("levels", 0), ("stride", 0), ("sor_omega", 2.0),
                       ("max_batch", 0), ("struct_size", 4), ("surface", 4),
                       ("surface", -1), ("d_sat", 0.0), ("d_sat", float("nan")),
                       ("storage", 2)):
        p = eb.ebof_default_params(64, 48)
        setattr(p, field, val)
        st, s = eb.ebof_stream_create(p, 0)
        bad.append((field, st))
        assert s is None
    assert all(st == eb.EBOF_ERR_INVALID_ARG for _, st in bad), bad
    p = eb.ebof_default_params(64, 48)
    p.patch = 20
    assert eb.ebof_stream_create(p, 0)[0] == eb.EBOF_ERR_UNSUPPORTED
    p = eb.ebof_default_params(64, 48)
    p.surface = 4
    assert eb.ebof_stream_device_bytes(p) == -1
    p.surface = eb.EBOF_SURFACE_LOG
    assert eb.ebof_stream_device_bytes(p) > 0
