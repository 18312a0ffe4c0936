"""The run configuration: the paper's constants, a JSON round trip, and the
binding's constants agree with it."""
import json
import os

import pytest

from paper_2501_01677_b300.config import PgsagConfig

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_paper_constants_match_the_golden_fixture():
    with open(os.path.join(GOLDEN, "paper_constants.json")) as f:
        g = json.load(f)
    c = PgsagConfig()
    assert c.boundary_weight == g["boundary_weight"]["value"]
    assert c.lambda_gc == g["lambda_gc"]["value"]
    assert c.lambda_1_mvgeo == g["lambda_1_mvgeo"]["value"]
    assert c.lambda_2_mvrgb == g["lambda_2_mvrgb"]["value"]
    assert c.lambda_3_flatten == g["lambda_3_flatten"]["value"]
    assert c.lambda_4_ban == g["lambda_4_ban"]["value"]


def test_json_round_trip_and_unknown_keys(tmp_path):
    c = PgsagConfig(tile=(8, 8), objective="eq11", vote_tau=5)
    p = tmp_path / "cfg.json"
    c.save(str(p))
    d = PgsagConfig.load(str(p))
    assert d == c
    with pytest.raises(KeyError):
        PgsagConfig.from_json('{"no_such_key": 1}')


def test_binding_constants_agree():
    PgsagConfig().check_library()
