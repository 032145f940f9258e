"""Host-side checks of the C ABI library (no GPU needed): it builds for
sm_103a, loads, and exports every entry point include/gbib.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gbib.h")


def declared_symbols():
    txt = open(HEADER).read()
    names = re.findall(r"^GBIB_API\s+[\w\s\*]*?\b(\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2408_14140_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_six_operators():
    syms = declared_symbols()
    for s in ("ib_interpolate", "ib_spread", "ib_multidirect_forcing",
              "particle_volume_integrals", "particle_force_torque", "particle_collide_update"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    for s in declared_symbols():
        assert hasattr(lib, s), s


def test_binding_covers_every_declared_symbol():
    from paper_2408_14140_gb300 import api
    assert sorted(api.EXPORTS) == declared_symbols()


def test_library_built_for_sm_103a():
    from paper_2408_14140_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_argument_errors_need_no_gpu(lib):
    """Argument validation happens on the host before any CUDA call."""
    lib.ib_interpolate.restype = ctypes.c_int
    lib.ib_last_error.restype = ctypes.c_char_p
    rc = lib.ib_interpolate(None, None, None, 0, None, 0, None, None)
    assert rc == -1
    assert b"ctx" in lib.ib_last_error()
