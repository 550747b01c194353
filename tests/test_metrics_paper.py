"""The byte and work model reproduces the numbers printed for the paper's example.

Golden values: tests/golden/paper_tables.json (Table data_metrics,
Table data_sizes_input, Table data_sizes_output, cf and AI of the Results
chapter, Eq. ai_spgemm and Eq. ai_cf)."""
import json
import os

from paper_2105_14156_gb300 import metrics

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))


def test_input_csr_bytes():
    g = GOLD
    b = metrics.csr_bytes(g["dims"], g["nnz_a"], g["value_bytes"], g["index_bytes"], g["rowptr_bytes"])
    assert b == g["input_total_bytes"]
    assert g["index_bytes"] * g["nnz_a"] == g["input_column_index_bytes"]
    assert g["value_bytes"] * g["nnz_a"] == g["input_data_bytes"]
    assert g["rowptr_bytes"] * (g["dims"] + 1) == g["input_row_pointer_bytes"]


def test_output_csr_bytes():
    g = GOLD
    b = metrics.csr_bytes(g["dims"], g["nnz_c"], g["value_bytes"], g["index_bytes"], g["rowptr_bytes"])
    assert b == g["output_total_bytes"]


def test_arithmetic_intensity():
    g = GOLD
    b = g["index_bytes"] + g["value_bytes"]       # one element = 4 B index + 8 B value
    ai = metrics.arithmetic_intensity(g["nnz_a"], g["nnz_b"], g["nnz_c"], g["cf"], b)
    assert round(ai, 2) == g["ai"]
    assert ai <= g["cf"] / b
    products = round(g["cf"] * g["nnz_c"])
    assert abs(metrics.compression_factor(products, g["nnz_c"]) - g["cf"]) < 1e-6
