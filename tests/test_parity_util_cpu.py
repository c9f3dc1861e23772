"""The parity helpers' 26-neighbour ambiguity at single items agrees with
the whole-stack map it stands in for at full size (ties and near-ties
planted by rounding to a coarse grid)."""
import numpy as np

from parity_util import ambiguous_26, ambiguous_26_at


def test_pointwise_26_ambiguity_matches_the_map():
    rng = np.random.default_rng(26)
    D = np.round(rng.normal(0.3, 0.2, size=(4, 19, 23)) * 20) / 20
    tol = np.array([0.01, 0.03, 0.0, 0.05])
    want = ambiguous_26(D, 0.3, tol)
    items = {(x, y, i) for i in range(4) for y in range(19) for x in range(23)}
    got = ambiguous_26_at(D, 0.3, tol, items)
    assert got == {(x, y, i) for x, y, i in items if want[i, y, x]}
    assert 0 < len(got) < len(items)
    assert ambiguous_26_at(D, 0.3, tol, set()) == set()
