"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/rtm.h declares (no compute calls: no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_2001_06444_gb300 import build, rtm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rtm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|double|uint64_t|const char \*)\s*(rtm_\w+)\s*\(", src, re.M)))


def test_header_declarations_match_binding():
    assert _declared() == sorted(rtm.EXPORTS)


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name


def test_cfl_limit_closed_form():
    assert rtm.cfl_limit() == pytest.approx(2.0 / (2.0 * 2048.0 / 315.0) ** 0.5, rel=1e-15)


def test_no_device_means_loud_failure():
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(rtm.RTMError):
        rtm.Context(0)
