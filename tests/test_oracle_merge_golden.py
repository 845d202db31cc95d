"""Hand-worked pins of the fusion pipeline's merge and repeat rules (§IV-C),
no GPU.

``tests/golden/merge_hand_example.json`` holds short op streams whose block
boundaries were derived by hand from the rules of §IV-C: per-window Eq.
dp-recurrence, the greedy cross-window merge (union within the cap of the
merged mode, Gamma(a u b) <= Gamma(a) + Gamma(b)) and up to four repeats.
The oracle's ``fuse_pipeline`` must reproduce each one for every round limit
listed, and so must the library's host planner where it can express the case
(Gamma = 4^k, round limit 1..4).  Planted mistakes in a copy of the oracle's
merge (strict <, the merged mode as 'or', one cap for both modes, no
repeats, no chaining after a merge) each fail at least one case.
"""
import inspect
import json
import os

import numpy as np
import pytest

import oracle
import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "merge_hand_example.json")))
CASES = {c["name"]: c for c in GOLD["cases"]}


def _ops(case):
    ops = []
    for o in case["ops"]:
        k = len(o["t"])
        m = np.eye(1 << k, dtype=np.complex128)
        ops.append(W.Op(tuple(o["t"]), m, bool(o["diag"])))
    return ops


def _score(case):
    if case["score"] == "gamma":
        return None
    assert case["score"] == "width"
    return lambda w, diag, targets: float(w)


def _run(mod, case, rounds):
    return mod["fuse_pipeline"](_ops(case), case["kmax"], case["kmax_diag"], case["window"], rounds,
                                score=_score(case))


@pytest.mark.parametrize("name", sorted(CASES))
def test_oracle_reproduces_hand_worked_blocks(name):
    case = CASES[name]
    for rounds, want in case["expect_by_rounds"].items():
        assert _run(oracle.__dict__, case, int(rounds)) == want, (name, rounds)


@pytest.fixture(scope="module")
def q():
    import __graft_entry__
    __graft_entry__._build_module().build()
    import paper_2608_16940_gb300 as q
    return q


@pytest.mark.parametrize("name", sorted(n for n, c in CASES.items() if c["score"] == "gamma"))
def test_host_planner_reproduces_hand_worked_blocks(q, name):
    case = CASES[name]
    n = 1 + max(t for o in case["ops"] for t in o["t"])
    for rounds, want in case["expect_by_rounds"].items():
        if int(rounds) > 4:
            continue
        got = q.qsa_plan_circuit(_ops(case), n, q.make_opts(planner=q.QSA_PLAN_DP, kmax=case["kmax"],
                                                             kmax_diag=case["kmax_diag"], window=case["window"],
                                                             rounds=int(rounds)))
        assert got == want, (name, rounds)


def _mutant(old, new):
    """The oracle's merge and pipeline with one planted mistake, in a copy of
    the oracle's namespace (the oracle itself is untouched)."""
    src = inspect.getsource(oracle.merge_adjacent) + "\n" + inspect.getsource(oracle.fuse_pipeline)
    assert old in src, old
    ns = dict(oracle.__dict__)
    exec(compile(src.replace(old, new), "<mutant>", "exec"), ns)
    return ns


MUTANTS = {
    "strict_gamma": ('sc(merged) <= sc(cur) + sc(b)', 'sc(merged) < sc(cur) + sc(b)'),
    "mode_or": ('d = cur["diag"] and b["diag"]', 'd = cur["diag"] or b["diag"]'),
    "diag_cap_for_all": ("cap = kmax_diag if d else kmax", "cap = kmax_diag"),
    "dense_cap_for_all": ("cap = kmax_diag if d else kmax", "cap = kmax"),
    "no_repeats": ("for rnd in range(rounds):", "for rnd in range(1):"),
    "no_chaining": ("            cur = merged\n", "            out.append(merged)\n            cur = None\n"),
}


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_each_planted_mistake_fails_a_case(mutant):
    ns = _mutant(*MUTANTS[mutant])
    failed = [name for name, case in CASES.items()
              for rounds, want in case["expect_by_rounds"].items() if _run(ns, case, int(rounds)) != want]
    assert failed, mutant
