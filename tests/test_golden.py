"""The oracle reproduces its stored regression fixtures (tests/golden/).

The fixtures were written by tests/golden/make_golden.py, which calls only
the oracle; a change in the oracle's arithmetic shows up here first.
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def _cases():
    with open(os.path.join(HERE, "golden", "oracle_small.json")) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c["name"])
def test_oracle_matches_golden(case, oracle_mod):
    img = synth.make_scene(case["seed"], synth.scene512_u8_spec(case["sigma_d"], case["H"], case["W"]))
    r = oracle.detect(img, case["n"], case["tmin"], case["tmax"], threshold=case["threshold"],
                      overlap=case["overlap"], mode=case["mode"])
    assert (r.lo, r.hi) == (case["lo"], case["hi"])
    assert r.n_candidates == case["n_candidates"] and r.score == case["score"]
    want = np.array(case["candidates"], dtype=np.float64).reshape(-1, 5)
    got = np.stack([r.x, r.y, r.i, r.resp, r.keep.astype(np.int64)], 1).astype(np.float64)
    np.testing.assert_array_equal(got[:, [0, 1, 2, 4]], want[:, [0, 1, 2, 4]])
    np.testing.assert_allclose(got[:, 3], want[:, 3], rtol=1e-12, atol=0)
