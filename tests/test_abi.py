"""The C-ABI library builds, loads and exports every entry point declared in include/*.h
(CPU only: no compute call is made without a GPU)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

import paper_1608_02227_gb300 as crgb
from paper_1608_02227_gb300 import _capi, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        names |= set(re.findall(r"CR_API\s+[\w\s\*]+?\b(cr_\w+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _capi.load()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("cr_create", "cr_dual_step", "cr_solve", "cr_primal", "cr_gap", "cr_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", _capi.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\sT\s(cr_\w+)$", out, flags=re.M))
    missing = _declared() - exported
    assert not missing, missing
    for n in _declared():
        assert hasattr(lib, n)


def test_binding_covers_the_header():
    assert _declared() <= set(_capi.symbols()) | set()
    assert set(_capi.symbols()) <= _declared()


def test_host_only_calls(lib):
    o = crgb.default_options()
    assert o.gamma == 1e-4 and o.precision == crgb.CR_FP32 and o.accelerate == 1
    assert lib.cr_version() >= 100
    assert lib.cr_strerror(0) == b"ok"
    assert lib.cr_strerror(1) == b"invalid argument"
    with pytest.raises(TypeError):
        crgb.default_options(no_such_option=1)
    # argument checks that return before any CUDA call
    assert lib.cr_checkpoint_bytes(None) == -1
    assert lib.cr_set_gamma(None, 1e-3) == 1
    assert lib.cr_checkpoint(None, None, 0) == 1
    assert lib.cr_restore(None, None, 0) == 1
    g = (ctypes.c_double * 1)(1e-3)
    assert lib.cr_solve_path(None, g, g, 1, 10, None) == 1
    assert lib.cr_solve_continuation(None, 0.1, 2.0, 0.1, 0.1, -1.0, 2, 10, None) == 1
    # memory an instance of the batched work-list needs (host arithmetic only)
    assert crgb.cr_batch_instance_bytes(1000, crgb.CR_MAX_N_BATCH + 1) == -1
    assert crgb.cr_batch_instance_bytes(1, 4) == -1
    b20, b40 = crgb.cr_batch_instance_bytes(1000, 20), crgb.cr_batch_instance_bytes(2000, 20)
    assert b20 >= 2 * 1000 * 1000 * 4 and b40 > 3 * b20  # the two N x N FP32 buffers dominate


def test_missing_library_fails_loudly(tmp_path):
    with pytest.raises(ImportError):
        _capi.load(str(tmp_path / "nope.so"))
