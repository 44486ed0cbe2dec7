"""The C-ABI library builds for sm_103a, loads, exports every entry point of
include/m1.h and rejects invalid grids on the host (no GPU needed)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2011_13926_gb300.build import build
    build()
    from paper_2011_13926_gb300 import m1
    return m1.load()


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "m1.h")).read()
    return sorted(set(re.findall(r"\b(m1_[a-z_0-9]+)\s*\(", txt)))


def test_exports_every_declared_symbol(lib):
    syms = header_symbols()
    assert "m1_implicit_step" in syms and "m1_init_grid" in syms
    for s in syms:
        assert hasattr(lib, s), s
    from paper_2011_13926_gb300 import m1
    assert set(m1.EXPORTED) <= set(syms)


def test_default_opts(lib):
    from paper_2011_13926_gb300 import default_opts, m1
    o = default_opts()
    assert o.newton_rtol == 1e-8 and o.restart == 30 and o.gmres_rtol == 1e-4 and o.precond == 1
    # the last fields of the struct: a layout mismatch with include/m1.h would garble them
    assert o.krylov == m1.KRYLOV_GMRES and o.pc_rebuild == 1 and o.line_search == 1 and o.refine_max == 4


@pytest.mark.parametrize("field,value", [("dim", 0), ("dim", 4), ("n", (0, 1, 1)), ("n", (4, 2, 1)),
                                         ("c", 0.0), ("periodic_one_side", None), ("hi", None)])
def test_init_rejects_bad_grids(lib, field, value):
    from paper_2011_13926_gb300 import m1
    d = m1.grid_desc(1, (8,))
    if field == "dim":
        d.dim = value
    elif field == "n":
        for a in range(3):
            d.n[a] = value[a]
    elif field == "c":
        d.c = value
    elif field == "periodic_one_side":
        d.bc[0][0] = 1
    elif field == "hi":
        d.hi[0] = d.lo[0]
    h = C.c_void_p()
    st = lib.m1_init_grid(C.byref(d), None, C.byref(h))
    assert st == m1.M1_ERR_ARG
    assert not h.value


def test_null_arguments(lib):
    from paper_2011_13926_gb300 import m1
    assert lib.m1_init_grid(None, None, None) == m1.M1_ERR_ARG
    assert lib.m1_destroy(None) == m1.M1_OK
    assert lib.m1_last_error(None) == b"null context"


def _c_struct_fields(header: str, name: str):
    """Field names, in order, of `typedef struct { ... } name;` in a C header: in each
    comma-separated declarator the last identifier once array brackets are removed."""
    import re
    src = re.sub(r"/\*.*?\*/", "", header, flags=re.S)
    m = re.search(r"typedef struct\s*\{([^{}]*)\}\s*" + re.escape(name) + r"\s*;", src)
    assert m, name
    fields = []
    for decl in m.group(1).split(";"):
        for d in decl.split(","):
            d = re.sub(r"\[[^\]]*\]", "", d).strip()
            if d:
                fields.append(re.findall(r"[A-Za-z_]\w*", d)[-1])
    return fields


@pytest.mark.parametrize("cname,pyname", [("m1_grid_desc", "GridDesc"), ("m1_solver_opts", "SolverOpts"),
                                          ("m1_step_info", "StepInfo"), ("m1_solve_info", "SolveInfo"),
                                          ("m1_stats_t", "Stats"), ("m1_batch_problem_info", "BatchProblemInfo"),
                                          ("m1_train_opts", "TrainOpts"), ("m1_train_info", "TrainInfo"),
                                          ("m1_device_fields", "DeviceFields")])
def test_ctypes_structs_mirror_the_header(cname, pyname):
    # the binding's ctypes structures must list the C structs' fields in the same order
    import os
    from paper_2011_13926_gb300 import m1
    header = open(os.path.join(os.path.dirname(__file__), "..", "include", "m1.h")).read()
    assert [f for f, _ in getattr(m1, pyname)._fields_] == _c_struct_fields(header, cname)
