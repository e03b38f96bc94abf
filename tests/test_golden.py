"""Stored expected values (written by tests/golden/make_golden.py from the
oracle) guard the seeded inputs and the oracle against silent drift."""
import json
import os

import numpy as np
import pytest

import graphgen as gg
import oracle
from tests.golden.make_golden import digest

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    with open(os.path.join(HERE, name)) as f:
        return json.load(f)


@pytest.mark.parametrize("name,make", [
    ("er1024_u32_src0.json", lambda: gg.tiny_er()),
    ("grid32_f32.json", lambda: gg.grid_f32(32, 0.01, nsrc=1, seed=0)),
])
def test_golden_inputs_and_oracle(name, make):
    rec = load(name)
    wl = make()
    assert digest(wl.row_ptr, wl.col, wl.weights) == rec["input_sha256"], "seeded generator drifted"
    dist, parent, pe = oracle.sssp(wl.row_ptr, wl.col, wl.weights, rec["source"])
    assert dist.view(np.uint32).tolist() == rec["dist_bits"]
    assert parent.tolist() == rec["parent"] and pe.tolist() == rec["parent_edge"]
