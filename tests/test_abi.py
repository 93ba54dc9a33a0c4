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


def test_struct_layouts_match_the_header(tmp_path):
    """Every struct of include/pic.h has the size and field offsets the
    binding's ctypes mirrors assume (compiled by gcc from the header alone),
    so a caller never passes a shorter or shifted struct."""
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("no gcc")
    structs = {"pic_grid": pic.pic_grid, "pic_species": pic.pic_species, "pic_options": pic.pic_options,
               "pic_laser": pic.pic_laser, "pic_diag": pic.pic_diag, "pic_qed": pic.pic_qed,
               "pic_field_view": pic.pic_field_view, "pic_mlp_train_opts": pic.pic_mlp_train_opts,
               "pic_mlp_report": pic.pic_mlp_report, "pic_mlp_info": pic.pic_mlp_info}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pic.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f in cls._fields_:
            lines.append(f'printf("{name} {f[0]} %zu\\n", offsetof({name}, {f[0]}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln:
            a, b, v = ln.split()
            got[(a, b)] = int(v)
    for name, cls in structs.items():
        assert got[(name, "size")] == C.sizeof(cls), name
        for f in cls._fields_:
            assert got[(name, f[0])] == getattr(cls, f[0]).offset, (name, f[0])


def test_options_of_another_size_are_refused():
    """pic_options.struct_size guards the layout: any other size is refused
    with PIC_ERR_ARG before anything is allocated."""
    L = pic.load_library()
    g = pic.pic_grid()
    g.dim, g.n[0], g.dx[0], g.order = 1, 16, 0.1, 2
    sp = (pic.pic_species * 1)()
    sp[0].q, sp[0].m, sp[0].w, sp[0].capacity = -1.0, 1.0, 0.1, 10
    o = pic.pic_options()
    o.struct_size = C.sizeof(pic.pic_options) - 8
    h = C.c_void_p()
    rc = L.pic_create(C.byref(g), 0.05, sp, 1, C.byref(o), C.byref(h))
    assert rc == -1 and not h.value
    assert b"struct_size" in L.pic_last_error(None)
