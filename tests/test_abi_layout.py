"""The ctypes binding lays out every struct of the C ABI as the C compiler does (CPU, no GPU).

A small C program is compiled against ``include/mfc.h`` with the host compiler and prints each
struct's size and each field's offset; the binding's ctypes structures must agree field by
field, so that a field added to the header (or reordered) without the binding fails here.
"""
import ctypes
import json
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
OUT = os.path.join(ROOT, "paper_1802_07525_gb300", "_build", "abi")

# C struct name -> name of the ctypes structure in paper_1802_07525_gb300.mfc
STRUCTS = {
    "mfc_lattice_desc": "LatticeDesc",
    "mfc_params": "Params",
    "mfc_solve_opts": "SolveOpts",
    "mfc_solve_result": "SolveResult",
    "mfc_launch": "Launch",
    "mfc_batch_opts": "BatchOpts",
    "mfc_batch_result": "BatchResult",
    "mfc_batch_stats": "BatchStats",
    "mfc_electro_params": "ElectroParams",
    "mfc_agent_params": "AgentParams",
    "mfc_agent_stats": "AgentStats",
    "mfc_electro_result": "ElectroResult",
}


def _c_layout(mfc):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "mfc.h"', "int main(void) {",
             '    printf("{");']
    first = True
    for cname, pyname in STRUCTS.items():
        fields = [f for f, _ in getattr(mfc, pyname)._fields_]
        sep = "" if first else ","
        first = False
        parts = ['\\"%s\\": {\\"size\\": %%zu' % cname]
        args = ["sizeof(%s)" % cname]
        for f in fields:
            parts.append('\\"%s\\": %%zu' % f)
            args.append("offsetof(%s, %s)" % (cname, f))
        lines.append('    printf("%s%s}", %s);' % (sep, ", ".join(parts), ", ".join(args)))
    lines += ['    printf("}\\n");', "    return 0;", "}"]
    os.makedirs(OUT, exist_ok=True)
    src = os.path.join(OUT, "abi_layout.c")
    exe = os.path.join(OUT, "abi_layout")
    with open(src, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe],
                   check=True, capture_output=True, text=True)
    return json.loads(subprocess.run([exe], check=True, capture_output=True, text=True).stdout)


def test_ctypes_structs_match_the_c_header():
    from paper_1802_07525_gb300 import mfc
    c = _c_layout(mfc)
    for cname, pyname in STRUCTS.items():
        cls = getattr(mfc, pyname)
        assert ctypes.sizeof(cls) == c[cname]["size"], cname
        for f, _ in cls._fields_:
            assert getattr(cls, f).offset == c[cname][f], (cname, f)
