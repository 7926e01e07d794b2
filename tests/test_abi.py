"""The C-ABI library builds, loads and exports every entry point that
include/lmfmm.h declares; host-only entry points behave (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lmfmm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lm_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("lm_create_medium", "lm_build_tree", "lm_apply", "lm_apply_adjoint", "lm_destroy_tree",
                 "lm_destroy_medium", "lm_last_error", "lm_status_string"):
        assert want in names


def test_library_exports_every_declared_symbol():
    import paper_1902_08250_gb300 as lm

    lib = ctypes.CDLL(lm.library_path())
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_entry_points():
    import paper_1902_08250_gb300 as lm

    lib = lm._lib
    assert lib.lm_status_string(1) == b"invalid argument"
    with pytest.raises(lm.LMError) as e:
        lm.create_medium(1.0, -1.5, 2.0, 1.0)
    assert e.value.status == 1
    with pytest.raises(lm.LMError):
        lm.create_medium(1.0, 1.5, 2.0, 0.0)
    with pytest.raises(lm.LMError):
        lm.create_medium(1.0, 1.5, float("nan"), 1.0)
    with pytest.raises(lm.LMError) as e:
        lm.create_medium(1.0, 1.5, 2.0, 1.0, p=1000)
    assert e.value.status == 1 and "p must be" in str(e.value)
    assert b"p must be" in lib.lm_last_error()
    m = lm.create_medium(1.0, 1.5, 2.0, 1.0, p=12)
    assert m.options["p"] == 12
    o = lm._Options()
    assert lib.lm_options_default(ctypes.byref(o)) == 0 and o.p == 20 and o.depth == -1
