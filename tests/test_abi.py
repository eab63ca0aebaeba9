"""CPU checks of the C ABI: the library builds, loads, and exports every
function include/tnn.h declares; calls with invalid arguments fail with
TNN_EINVAL before touching a GPU; without a GPU, context creation reports
TNN_ENODEV.  No compute call runs here."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tnn.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[\w]+\s*\*?\s*(\w+)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "for")))


@pytest.fixture(scope="module")
def lib():
    from paper_1902_03070_gb300 import build
    path = build.build()
    return ctypes.CDLL(path), path


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["tsvd_dct_forward", "tsvd_dct_inverse", "tsvt_dct", "tprod_dct", "tnn_complete", "tdct3",
              "tnn_admm_iterate", "tnn_create", "tnn_destroy"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    _, path = lib
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if " T " in l)
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_binding_lists_the_same_symbols(lib):
    from paper_1902_03070_gb300 import tnn
    assert sorted(tnn.EXPORTS) == _declared()


def test_status_strings(lib):
    L, _ = lib
    L.tnn_status_string.restype = ctypes.c_char_p
    for s in range(7):
        assert L.tnn_status_string(s).startswith(b"TNN_")


def test_null_context_is_einval(lib):
    L, _ = lib
    from paper_1902_03070_gb300 import tnn
    sh = tnn.Shape(4, 4, 4)
    buf = (ctypes.c_double * 64)()
    assert L.tsvt_dct(None, buf, sh, ctypes.c_double(1.0), 0, buf, None, None) == tnn.EINVAL
    assert L.tdct3(None, buf, sh, 0, 0, 0, buf, None) == tnn.EINVAL
    assert L.tnn_create(None, 0) == tnn.EINVAL


def test_no_gpu_here_gives_enodev(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1902_03070_gb300 import tnn
    with pytest.raises(tnn.TnnError) as e:
        tnn.Context(0)
    assert e.value.status == tnn.ENODEV
