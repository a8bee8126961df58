"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/nb.h declares.  No compute call runs here: these tests need no GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "nb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nb_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libnb():
    from paper_1312_1789_b300 import build, nb
    build.build()
    return nb.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("nb_create", "nb_set_particles", "nb_predict", "nb_force", "nb_correct", "nb_next_block",
                     "nb_energy", "nb_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(libnb):
    missing = [n for n in _declared() if not hasattr(libnb, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_1312_1789_b300 import nb
    assert sorted(nb.SIGNATURES) == _declared()


def test_version_string(libnb):
    assert b"sm_103a" in libnb.nb_version()


def test_create_rejects_bad_arguments_before_touching_the_device(libnb):
    h = C.c_void_p()
    assert libnb.nb_create(C.byref(h), 0, 6, 1e-4) == -1
    assert libnb.nb_create(C.byref(h), 16, 5, 1e-4) == -1
    assert libnb.nb_create(C.byref(h), 16, 6, -1.0) == -1
    assert libnb.nb_create(C.byref(h), 16, 6, float("nan")) == -1
    assert b"eps" in libnb.nb_last_error(None)
    assert not h.value


def test_null_context_is_rejected(libnb):
    assert libnb.nb_predict(None, 0.0) == -1
    assert libnb.nb_correct(None) == -1
    assert libnb.nb_set_graph(None, 4) == -1
    assert libnb.nb_autotune(None, 1) == -1
    assert libnb.nb_get_tuning(None, None, None, None, None) == -1
    assert libnb.nb_batch_set_graph(None, 2) == -1
    assert libnb.nb_set_tuning(None, 0, None, None) == -1
    assert libnb.nb_selftest_wait(None, C.c_double(0.1)) == -1
    assert libnb.nb_selftest_convert(None, 16, 1, None) == -1
    assert libnb.nb_get_nact_histogram(None, None, 0) == -1
    assert libnb.nb_fma_peak(None, 0, None) == -1
    libnb.nb_destroy(None)


def test_missing_library_fails_loudly(tmp_path):
    from paper_1312_1789_b300 import nb
    saved = nb._lib
    nb._lib = None
    try:
        with pytest.raises(ImportError):
            nb.lib(str(tmp_path / "libnb.so"))
    finally:
        nb._lib = saved


def test_binding_constants_match_the_header():
    from paper_1312_1789_b300 import nb
    src = open(os.path.join(ROOT, "include", "nb.h")).read()
    defs = dict(re.findall(r"#define\s+(NB_[A-Z_0-9]+)\s+\(?(-?\d+)\)?", src))
    shared = [k for k in defs if hasattr(nb, k)]
    assert {"NB_NACT_CLASSES", "NB_TUNE_MAX", "NB_NPHASES", "NB_JTILE", "NB_MIXED", "NB_ERR_TIMEOUT"} <= set(shared)
    for k in shared:
        assert getattr(nb, k) == int(defs[k]), k
