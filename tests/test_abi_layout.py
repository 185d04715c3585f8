"""The Python binding's copies of the C ABI match the header: a small C
program compiled against include/paulinet.h prints the size and every field
offset of the structs the binding passes by pointer, and every enum value
the binding names; the ctypes structs and the binding's constants must agree
(runs without a GPU)."""

import ctypes
import os
import shutil
import subprocess

import pytest

from paper_1909_08423_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {"pn_system_desc": binding.SystemDesc, "pn_server_cfg": binding.ServerCfg, "pn_job": binding.Job,
           "pn_result": binding.Result}
ENUMS = {"PN_FP64": binding.PN_FP64, "PN_MIXED": binding.PN_MIXED, "PN_JOB_ELOC": binding.PN_JOB_ELOC,
         "PN_JOB_SWEEP": binding.PN_JOB_SWEEP, "PN_JOB_SCAN": binding.PN_JOB_SCAN,
         "PN_OPT_FUSED_SAMPLER": binding.PN_OPT_FUSED_SAMPLER, "PN_OPT_TENSOR_CORES": binding.PN_OPT_TENSOR_CORES,
         "PN_OPT_DRIFT": binding.PN_OPT_DRIFT, "PN_OPT_GUARD": binding.PN_OPT_GUARD,
         "PN_OPT_DET_TABLE": binding.PN_OPT_DET_TABLE}
ENUMS.update({name: code for code, name in binding.ERRORS.items()})


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include "include/paulinet.h"', "#include <stdio.h>", "#include <stddef.h>", "int main(void) {"]
    for sname, st in STRUCTS.items():
        lines.append(f'  printf("{sname} size %zu\\n", sizeof({sname}));')
        for field, _ in st._fields_:
            lines.append(f'  printf("{sname} {field} %zu\\n", offsetof({sname}, {field}));')
    for ename in ENUMS:
        lines.append(f'  printf("enum {ename} %d\\n", (int){ename});')
    lines += ["  return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c11", "-I", ROOT, str(src), "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    table = {}
    for line in out.splitlines():
        a, b, v = line.split()
        table[(a, b)] = int(v)
    return table


@pytest.mark.parametrize("sname", list(STRUCTS))
def test_struct_layout_matches_header(c_layout, sname):
    st = STRUCTS[sname]
    assert ctypes.sizeof(st) == c_layout[(sname, "size")]
    for field, _ in st._fields_:
        assert getattr(st, field).offset == c_layout[(sname, field)], field


def test_enum_values_match_header(c_layout):
    for ename, value in ENUMS.items():
        assert value == c_layout[("enum", ename)], ename
