"""The C-ABI library builds, loads without a GPU and exports every entry point include/gipc.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "gipc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gipc_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2308_09400_gb300 import build as B
    if not os.path.exists(B.LIB) or any(os.path.getmtime(s) > os.path.getmtime(B.LIB) for s in B.sources()):
        B.build()
    return B.LIB


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for must in ("gipc_eval_stencils", "gipc_compute_eps_x", "gipc_create", "gipc_destroy", "gipc_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_entry_points() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header(libpath):
    from paper_2308_09400_gb300 import _abi
    assert set(declared_entry_points()) == set(_abi.SIGNATURES)


def test_host_side_argument_checks_need_no_gpu(libpath):
    """Invalid arguments are rejected on the host before any CUDA call."""
    from paper_2308_09400_gb300 import _abi
    L = _abi.lib()
    prm = _abi.BarrierParams(-1.0, 1e3, 0.1)
    st = L.gipc_eval_stencils(None, 10, None, 5, None, ctypes.byref(prm), 0, 0, None, None, None, None,
                              None, None)
    assert st == -1 and b"dhat" in L.gipc_last_error()
    prm = _abi.BarrierParams(1e-3, 1e3, 0.1)
    assert L.gipc_eval_stencils(None, 10, None, -1, None, ctypes.byref(prm), 0, 0, None, None, None,
                                None, None, None) == -1
    assert L.gipc_eval_stencils(None, 10, None, 0, None, ctypes.byref(prm), 0, 0, None, None, None,
                                None, None, None) == 0
    assert L.gipc_eval_stencils(None, 10, None, 3, None, ctypes.byref(prm), 7, 0, None, None, None,
                                None, None, None) == -1
    assert L.gipc_compute_eps_x(None, 3, None, -2, None, None) == -1


def test_ctypes_struct_layouts_match_the_header(tmp_path):
    """Field offsets and sizes of every ctypes struct equal the C compiler's for include/gipc.h."""
    from paper_2308_09400_gb300 import _abi
    structs = {"gipc_barrier_params": _abi.BarrierParams, "gipc_bsr": _abi.Bsr, "gipc_elements": _abi.Elements,
               "gipc_elastic_params": _abi.ElasticParams, "gipc_pcg_params": _abi.PcgParams,
               "gipc_kernel_time": _abi.KernelTime, "gipc_surface": _abi.Surface, "gipc_scene": _abi.Scene,
               "gipc_step_params": _abi.StepParams, "gipc_step_stats": _abi.StepStats,
               "gipc_scene_batch": _abi.SceneBatch, "gipc_spmv_tuning": _abi.SpmvTuning}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{os.path.join(ROOT, "include", "gipc.h")}"',
             'int main(void) {']
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            cf = {"lam": "lambda"}.get(f, f) if cname == "gipc_elastic_params" else f
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {cf}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    import subprocess
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        c, f, v = line.split()
        got[(c, f)] = int(v)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
