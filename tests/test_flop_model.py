"""The bench's flop model (the numerator of every GFLOP/s it reports), pinned
on two small cases computed by hand from its stated per-step counts."""
from __future__ import annotations

import importlib.util
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_flops", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_single_append_alpha_one():
    # one 4 x 3 block (s_1 = 3), A21 6 x 3 in one append, T 10 x 3 in one append
    # blocks 360 + row append 10 182 + U_row 72 + column append 4 722 + V 108 + apply 384
    F = _bench().flop_model(m=10, n=6, nnz_a21=5, nnz_t=7, m1=4, n1=3, m2=6, n2=3,
                            row_off=np.array([0, 4]), col_off=np.array([0, 3]), r=6, L=2, chunk=100)
    assert F == pytest.approx(15828.0)


def test_several_appends_start_from_s_largest_block_triplets():
    # three 1-column blocks (S = 3) but s = 2: with appends of 2 rows the row
    # phase starts at rank 2.  blocks 40 + row appends 3 092 + U_row 16 +
    # column appends 2 964.67 + V 36 + apply 192
    F = _bench().flop_model(m=10, n=6, nnz_a21=5, nnz_t=7, m1=4, n1=3, m2=6, n2=3,
                            row_off=np.array([0, 2, 3, 4]), col_off=np.array([0, 1, 2, 3]), r=3, L=2, chunk=2)
    assert F == pytest.approx(6340.0 + 2.0 / 3.0)


def test_pinv_threshold_report_hand_example():
    # m = n = 2^20: tau = 2^20 * 2^-52 * sigma_1 = 2^-32 for sigma_1 = 1
    b = _bench()
    tau = 2.0 ** -32
    S = np.array([1.0, 0.5, 5 * tau, 10 * tau, 10.5 * tau, tau, 0.0])
    rep = b.pinv_threshold_report(S, 1 << 20, 1 << 20)
    assert rep["tau"] == tau
    assert rep["sigma_at_or_below_tau"] == 2          # tau itself and 0
    assert rep["sigma_within_10x_tau"] == 2           # 5 tau and 10 tau
    assert b.pinv_threshold_report(np.zeros(0), 3, 4) == {"tau": 0.0, "sigma_at_or_below_tau": 0,
                                                           "sigma_within_10x_tau": 0}
