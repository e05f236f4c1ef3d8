"""C-ABI checks that need no GPU: the library builds for sm_103a, exports every
symbol include/rann_dd.h declares, the binding's struct layouts match the C
compiler's, and argument validation rejects bad descriptors before any CUDA
call."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rann_dd.h")


def header_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rann_dd_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2412_19207_gb300 import build
    build.build()
    import paper_2412_19207_gb300 as g
    return g.load_library()


def test_header_declares_the_method_entry_points():
    fns = header_functions()
    for name in ["rann_dd_create", "rann_dd_assemble", "rann_dd_pca", "rann_dd_setup_precond",
                 "rann_dd_solve_cg_as", "rann_dd_solve_gmres_ras", "rann_dd_eval", "rann_dd_destroy"]:
        assert name in fns


def test_library_exports_every_declared_symbol(lib):
    so = os.path.join(ROOT, "paper_2412_19207_gb300", "lib", "librann_dd.so")
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (rann_dd_\w+)", out))
    missing = [f for f in header_functions() if f not in exported]
    assert not missing, missing
    for f in header_functions():
        getattr(lib, f)


def test_binding_covers_the_header():
    import paper_2412_19207_gb300 as g
    assert sorted(g.SIGNATURES) == header_functions()


def test_struct_layouts_match_the_c_compiler():
    import paper_2412_19207_gb300 as g
    structs = [("rann_dd_desc", g.Desc), ("rann_dd_stats", g.Stats), ("rann_dd_pipeline", g.Pipeline),
               ("rann_dd_pipeline_out", g.PipelineOut)]
    prog = ['#include <stdio.h>', '#include <stddef.h>', '#include "rann_dd.h"', "int main(void){"]
    for cname, py in structs:
        prog.append(f'printf("%zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            prog.append(f'printf("%zu\\n", offsetof({cname}, {f}));')
    prog.append("return 0;}")
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "l.c")
        open(c, "w").write("\n".join(prog))
        exe = os.path.join(d, "l")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = [int(x) for x in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    want = []
    for _, py in structs:
        want.append(ctypes.sizeof(py))
        want += [getattr(py, f).offset for f, _ in py._fields_]
    assert vals == want


@pytest.mark.parametrize("field,value", [("dim", 4), ("neurons", 0), ("neurons", 2000), ("rho", 0.0),
                                         ("op", 7), ("layout", 5), ("g_kind", 3)])
def test_create_rejects_invalid_descriptors(lib, field, value):
    import rann_inputs as ri
    import paper_2412_19207_gb300 as g
    p = ri.config("poisson2d_2x2", small=True)
    d, keep = g.make_desc(p)
    setattr(d, field, value)
    h = ctypes.c_void_p()
    assert lib.rann_dd_create(ctypes.byref(d), None, ctypes.byref(h)) == g.EINVAL
    assert h.value is None
    assert lib.rann_dd_last_error().decode()


def test_paper_layout_needs_two_subdomains(lib):
    import rann_inputs as ri
    import paper_2412_19207_gb300 as g
    p = ri.example1_paper(sub=1)
    d, keep = g.make_desc(p)
    h = ctypes.c_void_p()
    assert lib.rann_dd_create(ctypes.byref(d), None, ctypes.byref(h)) == g.EINVAL


def test_null_handle_is_rejected(lib):
    import paper_2412_19207_gb300 as g
    assert lib.rann_dd_assemble(None) == g.EINVAL
    assert lib.rann_dd_pca(None, 0, 1e-3, None) == g.EINVAL
    assert lib.rann_dd_setup_precond(None, 1, 1) == g.EINVAL
    assert lib.rann_dd_profile_get(None, 0, None, None, None, None, None, None) == g.EINVAL
    assert lib.rann_dd_status_string(g.EORDER) == b"call out of order"


def test_missing_library_fails_loudly(tmp_path):
    import paper_2412_19207_gb300 as g
    saved = g._lib
    try:
        g._lib = None
        with pytest.raises(RuntimeError, match="no CPU fallback"):
            g.load_library(str(tmp_path / "nope.so"))
    finally:
        g._lib = saved


def test_product_path_never_touches_the_oracle():
    pkg = os.path.join(ROOT, "paper_2412_19207_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"\b(import|from)\s+oracle\b", src), f
                assert "rann_inputs" not in src or f == "__init__.py" and "rann_inputs.Problem" in src, f
