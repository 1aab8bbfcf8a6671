"""The C-ABI library loads on a machine without a GPU and exports every entry
point that include/ldg.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built_lib():
    from paper_2205_07824_b300 import build
    return build.build()


def _declared():
    src = open(os.path.join(ROOT, "include", "ldg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ldg_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("ldg_create", "ldg_destroy", "ldg_residual", "ldg_jvp", "ldg_newton_gmres", "ldg_gmres",
              "ldg_set_time", "ldg_q", "ldg_interpolate", "ldg_project", "ldg_l2_error", "ldg_sizes",
              "ldg_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(built_lib):
    L = ctypes.CDLL(built_lib)
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing
    L.ldg_version.restype = ctypes.c_char_p
    assert b"sm_103a" in L.ldg_version()


def test_invalid_arguments_are_rejected_without_a_gpu(built_lib):
    L = ctypes.CDLL(built_lib)
    L.ldg_create.argtypes = [ctypes.c_void_p] * 6
    # null output / null descriptors: rejected before any CUDA call
    assert L.ldg_create(None, None, 2, None, None, None) == -1
    L.ldg_residual.argtypes = [ctypes.c_void_p] * 3
    assert L.ldg_residual(None, None, None) == -1
    L.ldg_destroy.argtypes = [ctypes.c_void_p]
    assert L.ldg_destroy(None) == 0


def _struct_fields(name):
    """Field names, in order, of `typedef struct { ... } name;` in include/ldg.h."""
    src = open(os.path.join(ROOT, "include", "ldg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    body = re.search(r"typedef struct \{([^}]*)\}\s*" + name + r"\s*;", src).group(1)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        # "type a, b" or "const double* mu": the names follow the type, separated by commas
        head, *rest = decl.split(",")
        fields.append(re.findall(r"[A-Za-z_][A-Za-z0-9_]*", head)[-1])
        fields += [r.strip().lstrip("*").strip() for r in rest]
    return fields


@pytest.mark.parametrize("cname,pyname", [("ldg_mesh_desc", "_Mesh"), ("ldg_model_desc", "_Model"),
                                          ("ldg_options", "_Options"), ("ldg_solve_report", "SolveReport"),
                                          ("ldg_train_opts", "TrainOpts"), ("ldg_train_report", "TrainReport")])
def test_binding_structs_follow_the_header(cname, pyname):
    """Every ctypes mirror in the binding has the header's fields in the header's order,
    so an option added to the C struct cannot silently shift the ones after it."""
    from paper_2205_07824_b300 import ldg
    py = [f for f, _ in getattr(ldg, pyname)._fields_]
    assert py == _struct_fields(cname)
