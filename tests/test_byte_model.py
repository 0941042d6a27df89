"""The byte model reproduces the paper's blocked-vs-scalar byte accounting."""
import json
import os

import pytest

from paper_2606_24748_gb300 import bytes_model as bm


def golden(root):
    with open(os.path.join(root, "tests", "golden", "paper_byte_model.json")) as f:
        return json.load(f)


def test_block_and_scalar_bytes_per_3x3_block(root):
    g = golden(root)["block_3x3_fp64_int32"]
    assert bm.block_bytes(3, 3) == g["blocked"]["total_B"] == 76
    assert bm.scalar_csr_bytes(3, 3) == g["scalar_csr"]["total_B"] == 108
    assert bm.block_bytes(3, 3) / 9 == pytest.approx(g["blocked"]["per_scalar_nz_B"], abs=5e-3)
    assert bm.scalar_csr_bytes(3, 3) / 9 == g["scalar_csr"]["per_scalar_nz_B"]


def test_ratio_ceiling_and_saving(root):
    g = golden(root)
    ratio = bm.block_bytes(3, 3) / bm.scalar_csr_bytes(3, 3)
    assert ratio == pytest.approx(g["blocked_over_scalar_bytes"], abs=5e-3)
    assert 1 / ratio == pytest.approx(g["traffic_bound_ceiling"], abs=5e-3)
    assert 1 - ratio == pytest.approx(g["max_index_saving_fraction"], abs=5e-3)
    # the scalar SpGEMM moves a 12-byte value + index per 2-flop entry
    assert 2 / bm.scalar_csr_bytes(1, 1) == pytest.approx(g["scalar_spgemm_flop_per_byte"], abs=5e-3)


def test_spmv_bytes_formula_small_case():
    # 2 block rows, 3 blocks of 3x3, 2 block columns: values+idx, rowptr, x and y
    assert bm.spmv_bytes(3, 2, 2, 3, 3) == 3 * 76 + 4 * 3 + 8 * 6 + 8 * 6
    assert bm.spmv_flops(3, 3, 3) == 54
