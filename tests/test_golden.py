"""Hand-worked examples under tests/golden/ (each file states the passage it
follows and the derivation), run through the oracle: the learned test, RES
and ADS on tiny indexes, and OPQ's dimension allocation."""
import json
import os

import numpy as np
import pytest

from oracle import pq, search

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
SEARCH_FILES = ["learned_worked_example.json", "res_worked_example.json", "ads_worked_example.json"]


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


@pytest.mark.parametrize("name", SEARCH_FILES)
def test_search_examples(name):
    g = _load(name)
    X = np.asarray(g["X"], dtype=np.float32)
    D = X.shape[1]
    idx = search.OracleIndex(X, np.zeros(D), np.eye(D), np.zeros((g["nlist"], D)),
                             np.asarray(g["assign"], np.int32), dtype="f64")
    if "members" in g:
        idx.members = np.asarray(g["members"], np.int64)
    if "var" in g:
        assert np.array_equal(idx.var, g["var"])      # the derivation's variances
    Q = np.asarray(g["Q"], np.float32)
    probes = np.asarray(g["probes"], np.int32)
    m1 = np.asarray(g["m1"]) if "m1" in g else None
    beta = np.asarray(g["beta"]) if "beta" in g else None
    for c in g["cases"]:
        kw = dict(mode=c["mode"], final_rel=g.get("final_rel", np.inf))
        if "tau" in c:
            kw["tau"] = np.asarray(c["tau"])
        for k in ("estimator", "res_m", "ads_eps0"):
            if k in c:
                kw[k] = c[k]
        ids, d, st = search.search(idx, Q, probes, g["nprobe"], g["K"], g["delta_d"], m1, beta, **kw)
        assert list(ids[0]) == c["ids"], c
        if "dists" in c:
            assert list(d[0][:len(c["dists"])]) == c["dists"], c
        assert list(st[0][:4]) == c["stats"], c


def test_opq_allocation_example():
    g = _load("opq_allocation_example.json")
    assert list(pq.eigen_allocation(np.asarray(g["var"]), g["m"])) == g["perm"]
