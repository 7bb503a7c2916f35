"""The C header against the Python binding's mirror of it (no GPU needed).

`include/lks.h` is compiled as plain C11 (strict, warnings as errors) into a small
program that prints the size and field offsets of every structure the binding
mirrors with ctypes, and the values of the constants and enumerations the binding
restates.  A field added, removed, reordered or retyped on one side only would
shift the descriptor the library reads; this test fails instead.
"""
import ctypes as C
import os
import re
import shutil
import subprocess

import pytest

from paper_2411_03090_gb300 import lks

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {"lks_problem_desc": lks.Desc, "lks_stats": lks.Stats, "lks_batch_options": lks.BatchOptions,
           "lks_batch_stats": lks.BatchStats}

CONSTANTS = {
    "LKS_DESC_VERSION": lks.LKS_DESC_VERSION,
    "LKS_BATCH_VERSION": lks.LKS_BATCH_VERSION,
    "LKS_BATCH_TILE_CONFIGS": lks.LKS_BATCH_TILE_CONFIGS,
    "LKS_LATTICE_D3Q19": lks.LATTICE_D3Q19,
    "LKS_REAL_F32": lks.REAL["f32"], "LKS_REAL_F64": lks.REAL["f64"],
    "LKS_SNAP_F32": lks.SNAP["f32"], "LKS_SNAP_BF16": lks.SNAP["bf16"], "LKS_SNAP_F16": lks.SNAP["f16"],
    "LKS_PATH_AUTO": lks.PATH["auto"], "LKS_PATH_STEP": lks.PATH["step"],
    "LKS_PATH_RESIDENT": lks.PATH["resident"], "LKS_PATH_COLUMN": lks.PATH["column"],
    "LKS_OK": 0, "LKS_ERR_INVALID_ARG": 1, "LKS_ERR_WORKSPACE": 2, "LKS_ERR_CUDA": 3,
    "LKS_ERR_UNSTABLE": 4, "LKS_ERR_NOT_CONVERGED": 5, "LKS_ERR_TIMEOUT": 6, "LKS_ERR_STATE": 7,
}


def _program():
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "lks.h"', "int main(void) {"]
    for cname, py in STRUCTS.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f in py._fields_:
            lines.append(f'  printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    for name in CONSTANTS:
        lines.append(f'  printf("const {name} %lld\\n", (long long)({name}));')
    lines += ["  return 0;", "}"]
    return "\n".join(lines) + "\n"


@pytest.fixture(scope="module")
def layout(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("needs gcc")
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "abi.c", d / "abi"
    src.write_text(_program())
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I",
                    os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    table = {}
    for line in out.splitlines():
        a, b, v = line.split()
        table[(a, b)] = int(v)
    return table


@pytest.mark.parametrize("cname", sorted(STRUCTS))
def test_struct_layout_matches_the_binding(layout, cname):
    py = STRUCTS[cname]
    assert layout[(cname, "sizeof")] == C.sizeof(py)
    for f in py._fields_:
        assert layout[(cname, f[0])] == getattr(py, f[0]).offset, f[0]


def test_binding_mirrors_every_descriptor_field(layout):
    """Every member of lks_problem_desc has its ctypes field (the size check above
    would also catch a missing trailing member; this names the member)."""
    hdr = open(os.path.join(ROOT, "include", "lks.h")).read()
    body = hdr.split("typedef struct {", 1)[1].split("} lks_problem_desc;", 1)[0]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = set()
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        for part in decl.split(None, 1)[1].split(","):
            names.add(part.strip().split("[")[0])
    assert names == {f[0] for f in lks.Desc._fields_}


def test_constants_match_the_binding(layout):
    for name, val in CONSTANTS.items():
        assert layout[("const", name)] == val, name
