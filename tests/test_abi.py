"""The C-ABI library builds for sm_103a, loads without a GPU, exports every
symbol include/pic.h declares, and fails loudly (no CPU fallback) without a
GPU.  No compute call is made."""
import ctypes as C
import os
import re

import pytest

from paper_2104_00642_gb300 import build as B
from paper_2104_00642_gb300 import pic

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return C.CDLL(pic.LIB_PATH)


def _declared():
    src = open(os.path.join(ROOT, "include", "pic.h")).read()
    return sorted(set(re.findall(r"\b(pic_[a-z_]+)\s*\(", src)))


def test_header_and_binding_agree():
    assert _declared() == sorted(pic.EXPORTS)


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_create_without_gpu_fails_loudly_or_works():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(pic.PicError) as e:
        pic.pic_create(1, (16,), (0.1,), 0.05, [(-1.0, 1.0, 0.1, 10)])
    assert "PIC_ERR_CUDA" in str(e.value)


def test_argument_checks_run_before_device_use():
    # Courant violation and bad grids are rejected on the host
    with pytest.raises(pic.PicError) as e:
        pic.pic_create(1, (16,), (0.1,), 0.2, [(-1.0, 1.0, 0.1, 10)])
    assert "PIC_ERR_CFL" in str(e.value)
    with pytest.raises(pic.PicError) as e:
        pic.pic_create(1, (4,), (0.1,), 0.05, [(-1.0, 1.0, 0.1, 10)])
    assert "PIC_ERR_ARG" in str(e.value)
    with pytest.raises(pic.PicError) as e:
        pic.pic_create(4, (16,), (0.1,), 0.05, [])
    assert "PIC_ERR_ARG" in str(e.value)
