"""The C ABI library loads and exports every entry point include/bamg.h declares
(no compute: runs without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_2606_24748_gb300 import bamg


def declared_symbols(root):
    names = set()
    inc = os.path.join(root, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            text = open(os.path.join(inc, f)).read()
            names |= set(re.findall(r"BAMG_API\s+[\w\s\*]+?\b(bamg_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def built(root):
    from paper_2606_24748_gb300.build import build
    return build()


def test_header_declares_the_boundary(root):
    names = declared_symbols(root)
    for required in ("bamg_bsr_create", "bamg_bsr_coo_preallocate", "bamg_bsr_coo_set_values",
                     "bamg_ptap_symbolic", "bamg_ptap_numeric", "bamg_mg_setup", "bamg_mg_update",
                     "bamg_vcycle", "bamg_cg_solve"):
        assert required in names


def test_library_exports_every_declared_symbol(root, built):
    L = ctypes.CDLL(built)
    missing = [n for n in sorted(declared_symbols(root)) if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_the_header(root, built):
    assert set(bamg.exported_symbols()) == declared_symbols(root)
    bamg.lib()


def test_opts_default_from_library(built):
    o = bamg.bamg_mg_opts_default()
    assert o.max_coarse_dofs == 2100 and o.cheb_degree == 2 and o.power_its == 15
    assert o.cheb_lower == pytest.approx(0.1) and o.cheb_upper == pytest.approx(1.1)
