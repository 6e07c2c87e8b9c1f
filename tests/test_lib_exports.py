"""The C-ABI library loads without a GPU and exports every declared symbol."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1708_02845_gb300.build import build
    path = build()
    return ctypes.CDLL(path)


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dd_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("dd_create", "dd_destroy", "dd_load_mesh", "dd_poisson_kernel", "dd_distance", "dd_trace",
              "dd_trace_fields", "dd_query", "dd_last_error", "dd_check_mesh"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for n in declared_functions():
        assert hasattr(lib, n), n


def test_binding_covers_header():
    from paper_1708_02845_gb300 import dd
    for n in declared_functions():
        assert hasattr(dd, n), n
    assert dd.dd_version() == 100


def header_constants():
    """Every DD_ name given a value in dd.h: enum members and numeric #defines."""
    src = open(os.path.join(ROOT, "include", "dd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    vals = {}
    for name, v in re.findall(r"#define\s+(DD_[A-Z0-9_]+)\s+([-+0-9.eE]+)\s*$", src, flags=re.M):
        vals[name] = float(v)
    for body in re.findall(r"enum\s*\{(.*?)\}", src, flags=re.S):
        for name, v in re.findall(r"(DD_[A-Z0-9_]+)\s*=\s*(-?\d+)", body):
            vals[name] = int(v)
    return vals


def test_binding_constants_match_header():
    from paper_1708_02845_gb300 import dd
    vals = header_constants()
    assert len(vals) >= 26 and vals["DD_TILE_EXACT_BELOW"] == 0.25 and vals["DD_EBUDGET"] == -7
    for name, v in vals.items():
        assert hasattr(dd, name), name
        assert getattr(dd, name) == v, (name, getattr(dd, name), v)


def test_no_device_is_an_error_not_a_fallback():
    """Without a usable GPU the context cannot be created: dd_create reports
    an error status (no CPU path exists behind the boundary)."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1708_02845_gb300 import dd
    with pytest.raises(dd.DDError) as e:
        dd.dd_create(0)
    assert e.value.status in (dd.DD_ECUDA, dd.DD_EINVAL)
