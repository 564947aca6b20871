"""The oracle against the worked examples the paper prints (tests/golden/):
the single-upwind-neighbour solve of Eq. (5)-(7) and the causality example
of Fig. 4(b) (Sec. 2.2), with inputs that make the printed formulas exact."""
import json
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _num(v):
    return np.inf if v == "inf" else float(v)


def test_sec2_2_upwind_examples(oracle):
    data = json.load(open(os.path.join(GOLDEN, "sec2_2_upwind_examples.json")))
    assert data["cases"]
    for case in data["cases"]:
        nb = np.array([_num(v) for v in case["nb"]])
        kn = np.array(case["known"], np.uint8)
        t = oracle.local_solve(nb, kn, _num(case["Tc"]), tuple(case["h"]), case["F"])
        assert t == case["expected"], (case["name"], t)
