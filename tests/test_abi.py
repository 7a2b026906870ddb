"""CPU checks of the C ABI: the library loads and exports every function that
include/mapsq.h declares, and the binding covers each of them.  No device
call is made here."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]


def declared():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        names |= set(re.findall(r"^MAPSQ_API\s+[\w\s\*]+?\b(mapsq_\w+)\s*\(", text, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def built():
    from paper_1702_03484_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared()
    for required in ("mapsq_load_triples", "mapsq_scan_pattern", "mapsq_join", "mapsq_query"):
        assert required in names


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(built)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b(mapsq_\w+)\b", out))
    assert set(declared()) <= exported


def test_checked_build_exports_the_same_boundary(built):
    """libmapsq_checked.so (device bounds checks) exports the same calls and
    says which build it is, without any device call."""
    checked = os.path.join(os.path.dirname(built), "libmapsq_checked.so")
    lib = ctypes.CDLL(checked)
    assert not [n for n in declared() if not hasattr(lib, n)]
    lib.mapsq_build_info.restype = ctypes.c_char_p
    assert lib.mapsq_build_info() == b"sm_103a checked"
    plain = ctypes.CDLL(built)
    plain.mapsq_build_info.restype = ctypes.c_char_p
    assert plain.mapsq_build_info() == b"sm_103a"


def test_binding_covers_every_declared_symbol(built):
    from paper_1702_03484_gb300 import mapsq
    assert set(declared()) == set(mapsq._SIGNATURES)
    for n in declared():
        assert callable(getattr(mapsq, n)), n


def test_status_strings(built):
    from paper_1702_03484_gb300 import mapsq
    lib = mapsq.lib()
    assert lib.mapsq_strerror(0) == b"ok"
    assert lib.mapsq_strerror(-4) == b"memory budget exceeded"
    assert lib.mapsq_last_error(None) == b"no context"


def test_create_without_gpu_fails_cleanly(built):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1702_03484_gb300 import mapsq
    with pytest.raises(mapsq.MapsqError) as e:
        mapsq.mapsq_create(0)
    assert e.value.code == -1
