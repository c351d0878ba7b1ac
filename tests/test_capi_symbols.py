"""The C-ABI library builds, loads and exports every entry point that
include/fld.h declares; host-only calls behave as documented."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fld.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fld_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1403_8105_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("fld_create_grid", "fld_set_medium", "fld_set_source", "fld_solve", "fld_residual",
                     "fld_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_python_binding_wraps_every_symbol():
    import paper_1403_8105_gb300 as fld
    missing = [n for n in declared_functions() if not callable(getattr(fld, n, None))]
    assert not missing, missing


def test_default_params_and_status_strings():
    import paper_1403_8105_gb300 as fld
    p = fld.fld_default_params()
    assert p.limiter == fld.LIMITERS["lp"] and p.precision == fld.PRECISIONS["mixed"]
    assert p.tol == 1e-6 and p.local_iters == 2 and p.check_every >= 1
    assert p.anderson == 0 and p.nested == 0          # plain red-black SOR from the paper's start
    assert fld.fld_status_string(fld.FLD_ERR_DIVERGED) == "FLD_ERR_DIVERGED"
    assert fld.fld_status_string(99) == "FLD_ERR_UNKNOWN"
    # every status the header declares has its own name
    header = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "fld.h")).read()
    codes = {name: int(v) for name, v in re.findall(r"\b(FLD_(?:OK|ERR_\w+))\s*=\s*(\d+)", header)}
    assert len(codes) >= 9
    for name, v in codes.items():
        assert fld.fld_status_string(v) == name


def test_struct_layout_matches_header():
    # the ctypes mirror must list the same fields in the same order as fld.h
    import paper_1403_8105_gb300 as fld
    src = open(os.path.join(ROOT, "include", "fld.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    for cname, py in (("fld_solve_params", fld.SolveParams), ("fld_solve_result", fld.SolveResult)):
        body = re.search(r"typedef struct \{([^{}]*)\}\s*" + cname, src).group(1)
        fields = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            names = re.match(r"^(?:\w+\s+)+?(\w+(?:\s*,\s*\w+)*)$", decl).group(1)
            fields += [x.strip() for x in names.split(",")]
        assert [f for f, _ in py._fields_] == fields, cname


def test_create_grid_argument_checks_need_no_gpu():
    import paper_1403_8105_gb300 as fld
    with pytest.raises(fld.FldError) as e:
        fld.fld_create_grid(0, 4, 4, 0.25)
    assert e.value.status == fld.FLD_ERR_INVALID_ARG
    with pytest.raises(fld.FldError) as e:
        fld.fld_create_grid(4, 4, 4, -1.0)
    assert e.value.status == fld.FLD_ERR_INVALID_ARG
    # beyond the 32-bit offsets of the layout (2e9 padded elements per field):
    # rejected before anything is allocated
    for shape in ((1300, 1300, 1300), (2 ** 31 - 1, 1, 1), (1, 2 ** 31 - 1, 1), (4000, 4000, 200)):
        with pytest.raises(fld.FldError) as e:
            fld.fld_create_grid(*shape, 0.001)
        assert e.value.status == fld.FLD_ERR_INVALID_ARG, shape


def test_no_cpu_fallback_without_device():
    # Without a GPU the library refuses to create a grid instead of computing
    # anything on the host.
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1403_8105_gb300 as fld
    with pytest.raises(fld.FldError) as e:
        fld.fld_create_grid(4, 4, 4, 0.25)
    assert e.value.status == fld.FLD_ERR_NO_DEVICE


def test_server_checks_its_parameters_before_touching_a_device():
    # an out-of-range Anderson history or a bad blocking depth is refused while
    # the server checks its parameters, which happens before any device call
    import paper_1403_8105_gb300 as fld
    for bad, word in ((dict(anderson=17), "anderson"), (dict(anderson=4, scheme=1), "Anderson"),
                      (dict(temporal_depth=3), "temporal_depth"), (dict(fp64_verify=2), "fp64_verify"),
                      (dict(batch_launch=2), "batch_launch")):
        with pytest.raises(fld.FldError) as e:
            fld.fld_server_create(fld.params(**bad))
        assert e.value.status == fld.FLD_ERR_INVALID_ARG
        assert word in fld.fld_last_error()
