"""The C-ABI library builds, loads and exports every symbol of include/ib.h (no GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ib.h")


def declared_symbols():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ib_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2309_03600_gb300 import build_lib
    if not os.path.exists(build_lib.OUT):
        build_lib.build()
    return build_lib.OUT


def test_header_declares_entry_points():
    syms = declared_symbols()
    for s in ["ib_build_stencils", "ib_forward", "ib_adjoint", "ib_forward_batch", "ib_table_free",
              "ib_table_stats", "ib_sync_status", "ib_last_error"]:
        assert s in syms


def test_library_exports_all_declared(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (ib_[a-z0-9_]+)", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing


def test_library_loads_without_gpu(libpath):
    from paper_2309_03600_gb300 import ib
    L = ib.load(libpath)
    assert ib.ib_version().startswith("ibwave")
    o = ib.ib_opts_default(8)
    assert o.space_order == 8 and o.min_order == 2 and o.eta_p < 0 and o.eta_v == 0.0
    for s in ib.EXPORTS:
        assert hasattr(L, s)


def test_binding_names_match_header():
    from paper_2309_03600_gb300 import ib
    assert sorted(ib.EXPORTS) == declared_symbols()
