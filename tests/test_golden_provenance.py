"""The stored oracle samples (tests/golden/sampled_*.json) still come from the oracle, in
IEEE binary128: each file records a 113-bit significand and holds 64 stations and 64 cells,
and a subset is recomputed live and must agree to the rounding of the stored doubles."""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_1912_06976_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("name,nf,nt", [("mag64", 2, 4), ("grav300", 0, 2), ("mag128", 1, 2)])
def test_golden_samples_recompute(name, nf, nt):
    g = json.load(open(os.path.join(HERE, "golden", f"sampled_{name}.json")))
    assert g["oracle_significand_bits"] == 113  # binary128: far-field entries keep their digits
    assert O.significand_bits() == 113
    assert len(g["forward_stations"]) == len(g["forward"]) == 64
    assert len(g["transpose_cells"]) == len(g["transpose"]) == 64
    w = W.WORKLOADS[name]
    geom = O.Geometry(w.sx, w.sy, w.nz, w.dx, w.dy, w.zplanes, w.pxl, w.pxr, w.pyl, w.pyr, w.kind,
                      w.incl_deg, w.decl_deg, w.F_nT)
    if nf:
        st = g["forward_stations"][:nf]
        got = O.forward(geom, W.model(name, g["model_seed"]), st)
        np.testing.assert_allclose(got, g["forward"][:nf], rtol=1e-14)
    cl = g["transpose_cells"][-nt:]
    got = O.transpose(geom, W.data(name, g["data_seed"]), cl)
    np.testing.assert_allclose(got, g["transpose"][-nt:], rtol=1e-14)
