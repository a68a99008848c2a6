"""Host-side checks that need no GPU: the C-ABI library builds, loads and
exports every entry point the header declares; argument checks fail cleanly."""

import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vjb.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vjb_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1306_1467_gb300 import vjb
    return vjb.load_library()


def test_header_declares_the_paper_steps():
    names = _declared()
    for step in ("load_windows", "build_integral", "enumerate_haar", "train_round", "train_strong"):
        assert f"vjb_{step}" in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1306_1467_gb300 import vjb
    names = _declared()
    assert names, "no declarations parsed"
    for name in names:
        assert hasattr(lib, name), name
    # the binding wraps exactly the declared set
    assert sorted(vjb.SIGNATURES) == names


def test_null_context_is_rejected(lib):
    from paper_1306_1467_gb300 import vjb
    assert lib.vjb_build_integral(None) == vjb.EINVAL
    assert b"NULL" in lib.vjb_last_error()
    assert lib.vjb_train_round(None, None) == vjb.EINVAL
    cnt = C.c_int64(0)
    assert lib.vjb_enumerate_haar(None, C.byref(cnt), None) == vjb.EINVAL
    lib.vjb_destroy(None)  # accepted


def test_create_rejects_bad_arguments(lib):
    from paper_1306_1467_gb300 import vjb
    assert lib.vjb_create(None, 0, None) == vjb.EINVAL
    h = C.c_void_p()
    rc = lib.vjb_create(C.byref(h), -1, None)
    assert rc in (vjb.EINVAL, vjb.ECUDA)  # ECUDA where no driver is present
    assert not h.value


def test_library_is_built_for_sm103a():
    from paper_1306_1467_gb300 import build
    flags = build._flags(False)
    assert "arch=compute_103a,code=sm_103a" in flags
