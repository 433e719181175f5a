"""Host-side checks of the C-ABI library that need no GPU: it loads, exports
every entry point include/ebb.h declares, and its Python binding mirrors the
header's constants and structs."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ebb.h")


def _declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^(?:ebb_status_t|const char\*)\s+(ebb_\w+)\(", src, re.M)))


def _header_defines():
    src = open(HEADER).read()
    return {k: int(v, 0) for k, v in re.findall(r"#define\s+(EBB_\w+)\s+(0x[0-9a-fA-F]+|\d+)u?", src)}


@pytest.fixture(scope="module")
def abi():
    from paper_1506_07577_gb300 import build
    build.build()
    from paper_1506_07577_gb300 import abi as a
    return a


def test_library_exports_every_declared_symbol(abi):
    decl = _declared()
    assert len(decl) >= 13
    lib = ctypes.CDLL(abi.LIB_PATH)
    for name in decl:
        assert hasattr(lib, name), name
    assert sorted(abi.EXPORTED) == decl
    out = subprocess.run(["nm", "-D", "--defined-only", abi.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (ebb_\w+)", out))
    assert exported == set(decl)


def test_binding_constants_match_header(abi):
    for k, v in _header_defines().items():
        if k == "EBB_GB300_H":
            continue
        assert getattr(abi, k) == v, k
    src = open(HEADER).read()
    for name, val in re.findall(r"(EBB_(?:F32X4|F32|F64|I32|U8|STVK|NEOHOOKEAN|PREC_F64|PREC_F32|REDUCE_\w+))\s*=\s*(\d+)",
                                src):
        assert getattr(abi, name) == int(val), name


def test_struct_layouts_match_c_compiler(abi, tmp_path):
    """Compile a probe against include/ebb.h and compare every field offset
    and struct size with the ctypes mirror."""
    structs = {"ebb_map_opts_t": abi.ebb_map_opts_t, "ebb_step_params_t": abi.ebb_step_params_t,
               "ebb_cg_report_t": abi.ebb_cg_report_t, "ebb_autotune_cand_t": abi.ebb_autotune_cand_t,
               "ebb_autotune_report_t": abi.ebb_autotune_report_t, "ebb_relation_info_t": abi.ebb_relation_info_t}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ebb.h"', "int main(void){"]
    for sname, cls in structs.items():
        lines.append(f'printf("{sname} size %zu\\n", sizeof({sname}));')
        for fname, _ in cls._fields_:
            cname = "lambda" if fname == "lambda_" else fname
            lines.append(f'printf("{sname} {fname} %zu\\n", offsetof({sname}, {cname}));')
    lines.append("return 0;}")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    for line in filter(None, out):
        sname, what, val = line.split()
        cls = structs[sname]
        got = ctypes.sizeof(cls) if what == "size" else getattr(cls, what).offset
        assert got == int(val), line


def test_ctx_create_without_gpu_fails_cleanly(abi):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(abi.EbbError):
        abi.ebb_ctx_create(0, None)
