"""The resident-block schedule of the FP32 block Jacobi core SVD
(FASTPI_JACOBI_RESIDENT=1): every CTA keeps one of its two column blocks in
shared memory from round to round.  It visits the same block pairs in the
same rounds, with the same logical column order and the same arithmetic, so
the mixed factorization must be bit-for-bit identical to the default
schedule's.  The library's counters show that the resident schedule really ran
(core launches with it > 0 under the switch, none without it)."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import workloads
from gpu_common import binding

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["small", "medium"])
def test_resident_schedule_is_bit_identical(name, monkeypatch):
    fp = binding()
    w = workloads.make(name)
    cfg = w["cfg"]
    Yd = torch.from_numpy(w["Y"]).to("cuda:0")

    def run():
        h = fp.FastPI(w["m"], w["n"], w["rowptr"], w["col"], w["val"], device="cuda:0")
        fp.reset_counters()
        h.factor(cfg.r, cfg.k, "mixed", 256, 256)
        cnt = fp.counters()
        Z = h.apply(Yd).cpu().numpy()
        out = (h.S(), Z, h.info()["jacobi_sweeps_max"], cnt["core_resident_launches"], cnt["core32"]["launches"])
        h.close()
        return out

    monkeypatch.delenv("FASTPI_JACOBI_RESIDENT", raising=False)
    S0, Z0, sw0, res0, n0 = run()
    monkeypatch.setenv("FASTPI_JACOBI_RESIDENT", "1")
    S1, Z1, sw1, res1, n1 = run()
    assert n0 > 0 and n1 == n0
    assert res0 == 0, "the default schedule ran resident launches"
    assert res1 > 0, "the resident schedule never ran"
    assert np.array_equal(S0, S1)
    assert np.array_equal(Z0, Z1)
    assert sw0 == sw1
