"""The C-ABI library builds, loads and exports every symbol of include/*.h
(CPU only: no compute call is made)."""
import ctypes
import glob
import os
import re

import pytest

from tests.conftest import ROOT


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(mochy_[a-z_0-9]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2310_15668_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_calls_of_the_boundary():
    need = {"mochy_project", "mochy_count_exact", "mochy_count_sampled", "mochy_randomize",
            "mochy_profile", "mochy_load", "mochy_create", "mochy_destroy",
            "mochy_count_exact_subset", "mochy_motif_pattern", "mochy_strerror"}
    assert need <= _declared()


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_export():
    from paper_2310_15668_gb300 import binding
    assert set(binding.EXPORTS) == _declared()


def test_strerror_without_gpu(lib):
    lib.mochy_strerror.restype = ctypes.c_char_p
    assert lib.mochy_strerror(0) == b"ok"
    assert b"device memory" in lib.mochy_strerror(-2)


def test_config_defaults_and_validation_without_gpu():
    """mochy_config_default fills every field of the header's struct (the
    binding's layout matches it), and mochy_create refuses a bad rest_path
    before it looks for a device."""
    from paper_2310_15668_gb300 import binding as B
    cfg = B.mochy_config()
    ctypes.memset(ctypes.byref(cfg), 0x5A, ctypes.sizeof(cfg))
    B.load_library().mochy_config_default(ctypes.byref(cfg))
    assert (cfg.theta, cfg.eps, cfg.hbm_budget_bytes, cfg.device) == (1, 1.0, 0, 0)
    assert (cfg.exact_kernel, cfg.dense_threshold, cfg.rest_path) == (0, 0, 0)
    for bad in (-1, 3):
        cfg.rest_path = bad
        with pytest.raises(B.MochyError) as e:
            B.mochy_create(cfg)
        assert e.value.code == -1 and "rest_path" in str(e.value)
