"""CPU checks of the C ABI: the library loads without a GPU and exports every
function include/rfa.h declares; the ctypes structures match the C layout."""
import os
import re
import subprocess

import pytest

import paper_1907_05709_b300 as rfa

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rfa.h")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rfa_[a-z_0-9]+)\s*\(", txt)))


def test_library_builds_and_loads():
    from paper_1907_05709_b300 import build
    build.build()
    L = rfa.lib()
    assert L is not None
    assert rfa.rfa_last_error() == ""


def test_exports_every_declared_symbol():
    names = declared_functions()
    assert "rfa_step" in names and "rfa_backward" in names and len(names) >= 21
    out = subprocess.check_output(["nm", "-D", "--defined-only", rfa.LIB_PATH]).decode()
    exported = set(re.findall(r" T (rfa_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    assert set(rfa.EXPORTED) == set(names)


def test_struct_layout_matches_header(tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "rfa.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu\\n", sizeof(rfa_tissue), '
                   'sizeof(rfa_needle), offsetof(rfa_needle, power_W), '
                   'offsetof(rfa_tissue, T_fixed_C), offsetof(rfa_needle, T_tip_C));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    vals = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    import ctypes
    assert vals == [ctypes.sizeof(rfa.rfa_tissue), ctypes.sizeof(rfa.rfa_needle),
                    rfa.rfa_needle.power_W.offset, rfa.rfa_tissue.T_fixed_C.offset,
                    rfa.rfa_needle.T_tip_C.offset]


def test_invalid_arguments_rejected_without_gpu():
    # argument checks run before any CUDA call
    with pytest.raises(rfa.RfaError) as e:
        rfa.rfa_create_grid(0, 4, 4, 1e-3, 0.05)
    assert e.value.status == 1
    with pytest.raises(rfa.RfaError) as e:
        rfa.rfa_create_grid(4, 4, 4, -1e-3, 0.05)
    assert e.value.status == 1
    with pytest.raises(rfa.RfaError) as e:
        rfa.rfa_create_grid(4, 4, 4, 1e-3, 0.05, state_prec=7)
    assert e.value.status == 1
    # setters check their grid before touching it
    with pytest.raises(rfa.RfaError) as e:
        rfa.rfa_set_potential_preconditioner(None, rfa.PRECOND_MULTIGRID)
    assert e.value.status == 1 and "null grid" in str(e.value)
