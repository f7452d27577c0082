"""Writes tests/golden/sampled_<workload>.json: oracle values at sampled stations / cells.

For the workloads too large for the dense oracle to finish in seconds on every
machine (64x64x16 magnetic, 300x250x60 gravity, 128x128x32 magnetic), the
parity tests compare the GPU products at sampled outputs with values the CPU
oracle computes one by one.  This script calls only ``oracle`` (and the seeded
input generators) and stores those values; tests/test_golden_provenance.py
re-derives a subset live to show they still come from the oracle.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1912_06976_gb300 import workloads as W  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))

# (stations for d = G m, cells for m' = G^T d) per workload: 64 of each
SAMPLES = {"mag64": (64, 64), "grav300": (64, 64), "mag128": (64, 64)}


def geometry(w):
    return O.Geometry(w.sx, w.sy, w.nz, w.dx, w.dy, w.zplanes, w.pxl, w.pxr, w.pyl, w.pyr, w.kind,
                      w.incl_deg, w.decl_deg, w.F_nT)


def sample_indices(n, k, tag):
    """k distinct indices of range(n): the first, the last and k - 2 seeded others, sorted."""
    rng = np.random.default_rng((tag, 0x51))
    mid = rng.choice(np.arange(1, n - 1), size=k - 2, replace=False)
    return np.sort(np.concatenate([[0, n - 1], mid])).astype(np.int64)


def make(name):
    bits = O.significand_bits()
    if bits != 113:
        # far-field entries lose up to 1e-7 of their value in a 64-bit significand
        raise SystemExit(f"the oracle runs in a {bits}-bit significand; stored samples need binary128 (113)")
    w = W.WORKLOADS[name]
    geom = geometry(w)
    kf, kt = SAMPLES[name]
    tag = sum(ord(c) for c in name)
    fi = sample_indices(w.m, kf, tag)
    ti = sample_indices(w.n, kt, tag + 1)
    m = W.model(name, 0)
    d = W.data(name, 0)
    t0 = time.time()
    fwd = O.forward(geom, m, fi)
    tr = O.transpose(geom, d, ti)
    rec = {
        "workload": name,
        "model_seed": 0,
        "data_seed": 0,
        "forward_stations": fi.tolist(),
        "forward": [float(v) for v in fwd],
        "transpose_cells": ti.tolist(),
        "transpose": [float(v) for v in tr],
        "oracle_significand_bits": bits,
        "note": "d = G m at the listed stations and m' = G^T d at the listed cells, "
                "m = workloads.model(name, 0), d = workloads.data(name, 0), by oracle/gm_oracle.c in IEEE binary128",
    }
    path = os.path.join(HERE, f"sampled_{name}.json")
    with open(path, "w") as f:
        json.dump(rec, f, indent=1)
    print(f"{name}: {time.time() - t0:.1f} s -> {path}")


if __name__ == "__main__":
    for name in sys.argv[1:] or list(SAMPLES):
        make(name)
