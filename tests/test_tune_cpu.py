"""Host logic of the autotuner (no GPU): table keys and lookup, and the
candidate shapes it would compile and time for each kernel kind."""
import json

import pytest


@pytest.fixture(scope="module")
def tune():
    from paper_2108_12050_gb300 import _build, tune
    _build.build_lib()
    return tune


def test_ladder_keys_name_rule_response_and_kernel(tune):
    assert tune.ladder_key(16, 1.0, 12.0, 0) == "n16_t1-12_paper_tr4"
    assert tune.ladder_key(16, 1.0, 12.0, "local26") == "n16_t1-12_local26_tr4"
    assert tune.ladder_key(16, 1.0, 12.0, 0, response="log", tensor_cores=True) == \
        "n16_t1-12_paper_tr4_log_tc"
    assert tune.ladder_key(10, 0.5, 7.25, 0, truncate=3.0) == "n10_t0.5-7.25_paper_tr3"


def test_lookup_by_sm_count_with_fallback(tune, tmp_path, monkeypatch):
    table = {
        "n16_t1-12_paper_tr4_tc": {"152": {"shape": [352, 18, 4, 384, 3], "ms": 1.0},
                                   "any": {"shape": [320, 18, 4, 352, 3], "ms": 1.1}},
        "n16_t1-12_paper_tr4": {"148": {"shape": [288, 18, 4, 384, 3], "ms": 1.3}},
        "n4_t1-4_paper_tr4": {"152": {"shape": [1, 2, 3]}},       # malformed: ignored
    }
    path = tmp_path / "tuned.json"
    path.write_text(json.dumps(table))
    monkeypatch.setattr(tune, "TABLE", str(path))
    assert tune.lookup(16, 1.0, 12.0, 0, 152, tensor_cores=True) == [352, 18, 4, 384, 3, 1]
    assert tune.lookup(16, 1.0, 12.0, 0, 132, tensor_cores=True) == [320, 18, 4, 352, 3, 1]
    assert tune.lookup(16, 1.0, 12.0, 0, 148) == [288, 18, 4, 384, 3, 1]
    assert tune.lookup(16, 1.0, 12.0, 0, 152) is None            # no entry, no fallback
    assert tune.lookup(16, 1.0, 12.0, 1, 152) is None            # other rule
    assert tune.lookup(4, 1.0, 4.0, 0, 152) is None
    monkeypatch.setattr(tune, "TABLE", str(tmp_path / "missing.json"))
    assert tune.lookup(16, 1.0, 12.0, 0, 152, tensor_cores=True) is None


def test_ffma_candidates_are_balanced_shapes_of_the_ffma_menu(tune):
    from paper_2108_12050_gb300 import _native
    for kw in (dict(), dict(response="log")):
        menu = set(_native.tile_configs(n=16, t_min=1.0, t_max=12.0, nms=0, tensor_cores=False,
                                        **kw))
        cands = tune.candidates(16, 1.0, 12.0, 0, **kw)
        assert cands and len(set(cands)) == len(cands)
        for tx2, ty2, rb, nt, ng, item in cands:
            assert (tx2, ty2, rb, nt, ng, item) in menu
            assert 0.85 * nt <= tune.item_count(tx2, rb, item) <= nt


def test_item_counts():
    from paper_2108_12050_gb300 import tune
    assert tune.item_count(352, 4, 1) == 352
    assert tune.item_count(256, 8, 2) == 256
    assert tune.item_count(192, 4, 3) == 384


def test_width_candidates_fit_the_ffma_kernel(tune):
    from paper_2108_12050_gb300 import _native
    shapes = tune.width_candidates(16, 1.0, 12.0, 0, [312, 344], rbs=(2, 4), groups=(3,),
                                   items=(1, 2, 3))
    assert shapes and {s[0] for s in shapes} == {312, 344} and {s[5] for s in shapes} == {1, 2, 3}
    for s in shapes:
        assert s[3] % 32 == 0 and tune.item_count(s[0], s[2], s[5]) <= s[3]
        assert _native.chosen_tile(n=16, t_min=1.0, t_max=12.0, nms=0, tile_shape=s,
                                   tensor_cores=False) == s
