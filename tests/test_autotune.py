"""Autotuner: cache keys and selection on the CPU, one small tuning run on
the GPU whose chosen parameters must still give the oracle's solution."""
import math

import numpy as np
import pytest

from paper_1502_07303_gb300 import autotune
from paper_1502_07303_gb300 import workloads as wl


def test_keys_and_size_classes():
    assert autotune.size_class(256 ** 3) == 24
    assert autotune.size_class(1) == 0
    assert autotune.key("reinit", "f32", 2 ** 20) == "reinit/f32/20"


def test_select_best_skips_failures():
    t = [({"stride": 2.0}, None), ({"stride": 4.0}, 3.0), ({"stride": 8.0}, 2.5),
         ({"stride": math.inf}, float("nan"))]
    assert autotune.select_best(t) == ({"stride": 8.0}, 2.5)
    assert autotune.select_best([({}, None)]) is None


def test_cache_roundtrip(tmp_path):
    path = str(tmp_path / "tune.json")
    assert autotune.params_for("reinit", "float32", 1000, path=path) == {}
    cache = {autotune.key("reinit", "f32", 1000): {"stride": math.inf, "bucket": 4.0,
                                                     "exchange_passes": 2, "ctas": 0, "ms": 1.0}}
    autotune.save_cache(cache, path)
    got = autotune.params_for("reinit", "torch.float32", 1000, path=path)
    assert got == {"stride": math.inf, "bucket": 4.0, "exchange_passes": 2, "ctas": 0}
    assert set(got) <= set(autotune.PARAMS)
    assert autotune.params_for("reinit", "float64", 1000, path=path) == {}


def test_candidate_list():
    got = list(autotune.candidates(autotune.QUICK))
    assert got == [dict(c) for c in autotune.QUICK]
    assert {c["schedule"] for c in got} == {2, 3}
    assert all(set(c) <= set(autotune.PARAMS) for c in got)


def test_unset_parameters_come_from_the_cache(tmp_path):
    path = str(tmp_path / "tune.json")
    n = 100 ** 3
    autotune.save_cache({autotune.key("reinit", "f64", n): {"stride": 1.0, "bucket": 3.0,
                                                             "ahead": math.inf, "ms": 2.0}}, path)
    got = autotune.merge({"stride": 4.0, "bucket": 0.0}, "reinit", "float64", n, path=path)
    assert got == {"stride": 4.0, "bucket": 3.0, "ahead": math.inf}
    assert autotune.merge({"stride": 4.0}, "reinit", "float32", n, path=path) == {"stride": 4.0}


def test_candidate_grid():
    c = list(autotune.candidates({"schedule": [2], "stride": [2.0, 8.0], "bucket": [1.0],
                                  "exchange_passes": [1, 2], "ctas": [0], "ahead": [math.inf]}))
    assert len(c) == 4 and all(set(x) == set(autotune.PARAMS) for x in c)


@pytest.mark.gpu
def test_tune_small_problem_on_gpu(oracle, tmp_path):
    import torch
    from paper_1502_07303_gb300 import fmm
    from parity_util import compare
    p = wl.random_spheres(shape=(40, 40, 40), count=4, seed=21)
    path = str(tmp_path / "tune.json")
    search = {"schedule": [1, 3], "stride": [4.0, 16.0, math.inf], "bucket": [1.0, 4.0],
              "exchange_passes": [1, 2], "ctas": [0], "ahead": [math.inf]}
    best, ms, table = autotune.tune(p, torch.float64, search=search, reps=1, path=path)
    assert best is not None and ms > 0 and len(table) == 24
    assert autotune.params_for("reinit", torch.float64, p.n_points, path=path) == best
    phi = torch.as_tensor(p.phi0, dtype=torch.float64, device="cuda")
    with fmm.Solver(p.shape, p.h, dtype=torch.float64, **best) as s:
        T, G = s.reinit(phi)
    compare(T.cpu().numpy(), G.cpu().numpy(), oracle.solve_reinit(p.phi0, p.h), "f64")
