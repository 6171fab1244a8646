"""Host-side checks of the C ABI library (no GPU calls)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "p2.h")


def _declared():
    with open(HEADER) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char \*)\s*\*?\s*(p2_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib_path():
    import __graft_entry__ as g
    g._build_module().build()
    return os.path.join(ROOT, "paper_1703_04219_gb300", "libp2.so")


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("p2_create", "p2_destroy", "p2_load_slices", "p2_init", "p2_iterate", "p2_fit",
              "p2_get_factors", "p2_set_factors", "p2_get_mttkrp", "p2_get_procrustes",
              "p2_stats", "p2_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(p2_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_binding_loads_and_names_match(lib_path):
    import paper_1703_04219_gb300 as p2
    assert sorted(p2.EXPORTED) == _declared()
    for n in p2.EXPORTED:
        assert hasattr(p2.lib, n)
    o = p2.p2_default_options(10)
    assert (o.R, o.use_graph, o.timing) == (10, 1, 0) and abs(o.rank_rtol - 1e-5) < 1e-20


def test_cpu_only_box_reports_cuda_error_not_crash(lib_path):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1703_04219_gb300 as p2
    with pytest.raises(p2.P2Error) as ei:
        p2.p2_create(p2.p2_default_options(4))
    assert ei.value.code in (p2.P2_ECUDA, p2.P2_EINVAL)
    bad = p2.p2_default_options(65)
    with pytest.raises(p2.P2Error) as ei:
        p2.p2_create(bad)
    assert ei.value.code == p2.P2_EINVAL
