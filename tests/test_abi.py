"""The C ABI: libhmg.so builds for sm_103a, loads without a GPU, and exports every
symbol include/hmg.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


def _declared():
    src = open(os.path.join(ROOT, "include", "hmg.h")).read()
    return sorted(set(re.findall(r"\b(hmg_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1504_07499_gb300 import build, hmg
    build.build()
    return hmg.lib()


def test_header_declares_the_api():
    names = _declared()
    for n in ["hmg_create", "hmg_destroy", "hmg_voxelize", "hmg_solve", "hmg_submit", "hmg_poll"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1504_07499_gb300 import hmg
    for name in _declared():
        assert hasattr(lib, name), name
    assert sorted(hmg.EXPORTS) == _declared()


def test_version_and_error_without_gpu(lib):
    assert b"hmg" in lib.hmg_version()
    assert lib.hmg_last_error() is not None


def test_footprint_host_only(lib):
    from paper_1504_07499_gb300 import hmg
    a = hmg.hmg_footprint(256, hmg.HMG_FP32_BULK)
    b = hmg.hmg_footprint(256, hmg.HMG_FP64)
    assert a > b > 9 * 256 ** 3 * 8


def test_create_fails_cleanly_without_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1504_07499_gb300 import hmg
    with pytest.raises(hmg.HmgError):
        hmg.hmg_create(0)
