"""The C ABI library loads and exports every entry point include/pmace.h
declares; argument validation that happens before any device work is
checked here without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pmace.h")


@pytest.fixture(scope="module")
def binding():
    from paper_2111_14240_gb300 import build
    build.build()
    from paper_2111_14240_gb300 import pmace
    return pmace


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pmace_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["pmace_create", "pmace_iterate", "pmace_get_image", "pmace_residual",
                     "pmace_destroy", "pmace_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(binding):
    lib = ctypes.CDLL(binding._LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) == set(binding.EXPORTS)


def test_abi_version_and_status_strings(binding):
    assert binding.pmace_abi_version() == 2
    assert binding._lib.pmace_status_string(0) == b"ok"
    assert binding._lib.pmace_status_string(4) == b"unsupported size"


def _args(np_=32, J=4, n=64):
    probe = np.ones((np_, np_, 2), np.float32)
    offs = np.zeros((J, 2), np.int32)
    amps = np.ones((J, np_, np_), np.float32)
    return probe, offs, amps, n


def test_create_rejects_unsupported_probe_size(binding):
    probe, offs, amps, n = _args(np_=48)
    with pytest.raises(binding.PmaceError) as e:
        binding.pmace_create(n, n, 48, 4, 1.25, probe, offs, amps, inputs_on_device=False)
    assert e.value.status == binding.PMACE_ERR_UNSUPPORTED_SIZE
    assert "48" in binding.pmace_last_error(None)


def test_create_rejects_out_of_range_offsets(binding):
    probe, offs, amps, n = _args()
    offs[2] = (n - 31, 0)
    with pytest.raises(binding.PmaceError) as e:
        binding.pmace_create(n, n, 32, 4, 1.25, probe, offs, amps, inputs_on_device=False)
    assert e.value.status == binding.PMACE_ERR_INVALID_ARG
    assert "offset 2" in binding.pmace_last_error(None)


def test_create_rejects_bad_sizes_and_formats(binding):
    probe, offs, amps, n = _args()
    for bad in [dict(n1=0), dict(J=0), dict(n1=16), dict(kappa=float("nan")), dict(fmt=7),
                dict(fmt=1)]:
        kw = dict(n1=n, n2=n, J=4, kappa=1.25, fmt=0)
        kw.update(bad)
        with pytest.raises(binding.PmaceError) as e:
            binding.pmace_create(kw["n1"], kw["n2"], 32, kw["J"], kw["kappa"], probe, offs, amps,
                                 amp_format=kw["fmt"], inputs_on_device=False)
        assert e.value.status == binding.PMACE_ERR_INVALID_ARG, bad


def test_null_handle_calls_fail_cleanly(binding):
    step = binding.pmace_step(0.5, 0.5)
    assert binding._lib.pmace_iterate(None, 1, ctypes.byref(step), None) == binding.PMACE_ERR_INVALID_ARG
    out = (ctypes.c_double * 2)()
    assert binding._lib.pmace_residual(None, out, None) == binding.PMACE_ERR_INVALID_ARG
    binding._lib.pmace_destroy(None)   # no-op
