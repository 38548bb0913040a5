"""The Python binding restates include/bdis.h: its ctypes structures and its
constants must match what a C compiler makes of the header. A small C
program includes the header and prints every struct's size and field
offsets and every constant; the ctypes side must agree field by field.
(Host-side ABI; no GPU.)"""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2106_07136_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "bdis_image": _lib.BdisImage,
    "bdis_params": _lib.BdisParams,
    "bdis_patch_debug": _lib.BdisPatchDebug,
    "bdis_group": _lib.BdisGroup,
    "bdis_plan_choice": _lib.BdisPlanChoice,
    "bdis_timing": _lib.BdisTiming,
}

CONSTANTS = {
    "BDIS_OK": _lib.BDIS_OK, "BDIS_E_INVALID_ARG": _lib.BDIS_E_INVALID_ARG,
    "BDIS_E_NOMEM": _lib.BDIS_E_NOMEM, "BDIS_E_CUDA": _lib.BDIS_E_CUDA,
    "BDIS_E_TIMEOUT": _lib.BDIS_E_TIMEOUT, "BDIS_E_UNSUPPORTED": _lib.BDIS_E_UNSUPPORTED,
    "BDIS_U8": _lib.BDIS_U8, "BDIS_F32": _lib.BDIS_F32,
    "BDIS_FUSION_BDIS": _lib.BDIS_FUSION_BDIS, "BDIS_FUSION_DIS": _lib.BDIS_FUSION_DIS,
    "BDIS_PLAN_AUTOTUNE": _lib.BDIS_PLAN_AUTOTUNE,
    "BDIS_PLAN_SCALE_TO_WIDTH": _lib.BDIS_PLAN_SCALE_TO_WIDTH,
    "BDIS_STATIC_SCRATCH_BYTES": _lib.STATIC_SCRATCH_BYTES,
    "BDIS_ASYNC_SLOTS": _lib.ASYNC_SLOTS,
    "BDIS_TIMING_CLASSES": len(_lib.BdisTiming._fields_[0][1]()),
}


def probe_source():
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "bdis.h"', "int main(void) {"]
    for cname, cls in STRUCTS.items():
        lines.append(f'  printf("size {cname} %zu\\n", sizeof({cname}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("offset {cname}.{field} %zu\\n", offsetof({cname}, {field}));')
    for name in CONSTANTS:
        lines.append(f'  printf("const {name} %lld\\n", (long long)({name}));')
    lines += ["  return 0;", "}"]
    return "\n".join(lines) + "\n"


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "probe.c", d / "probe"
    src.write_text(probe_source())
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    table = {}
    for line in out.splitlines():
        kind, key, value = line.split()
        table[(kind, key)] = int(value)
    return table


@pytest.mark.parametrize("cname", list(STRUCTS))
def test_struct_layout_matches_the_header(c_layout, cname):
    cls = STRUCTS[cname]
    assert ctypes.sizeof(cls) == c_layout[("size", cname)], cname
    for field, _ in cls._fields_:
        assert getattr(cls, field).offset == c_layout[("offset", f"{cname}.{field}")], (cname, field)


def test_constants_match_the_header(c_layout):
    for name, value in CONSTANTS.items():
        assert value == c_layout[("const", name)], name
