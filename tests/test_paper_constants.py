"""The planner's default parameters against the constants the paper prints
(tests/golden/paper_constants.txt, each with where the paper states it): the library's
defaults (cpp_params_default) and the oracle's defaults must both equal them."""
import math
import os

import oracle
from paper_2309_09102_gb300 import cppflow

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.txt")
TO_SI = {"mm": 1e-3, "cm": 1e-2, "deg": math.pi / 180.0, "-": 1.0}


def constants():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            name, value, unit, cite, param = [c.strip() for c in line.split("|")]
            rows.append((name, float(value), unit, cite, param))
    return rows


def test_fixture_is_complete_and_cited():
    rows = constants()
    assert len(rows) == 12
    assert all(cite.startswith(("§", "Table")) for _, _, _, cite, _ in rows)
    assert {p for *_, p in rows if p != "-"} == {"tau_pos", "tau_rot", "jump_max", "near_margin",
                                                "pen_limit", "pen_collide"}


def test_library_defaults_equal_the_papers_constants():
    p = cppflow.make_params()
    for name, value, unit, cite, param in constants():
        if param == "-":
            continue
        got = getattr(p, param)
        assert math.isclose(got, value * TO_SI[unit], rel_tol=1e-12), (name, got, cite)


def test_oracle_defaults_equal_the_papers_constants():
    p = oracle.make_params()
    for name, value, unit, cite, param in constants():
        if param == "-" or not hasattr(p, param):   # the oracle has no collision cost field
            continue
        got = getattr(p, param)
        assert math.isclose(got, value * TO_SI[unit], rel_tol=1e-12), (name, got, cite)
