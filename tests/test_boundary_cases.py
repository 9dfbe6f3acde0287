"""Planted boundary draws (CPU): the golden cases and the parity rule.

tests/golden/boundary_cases.json holds two-node networks whose one skip draw
(or weight draw) sits next to an integer (tests/golden/plant_boundary_cases.py
explains the construction).  These tests pin what the cases claim with
arithmetic that does not go through the oracle's sampler: Python's libm for
the canonical FP64 expressions of Sec. 2.3 and Eq. 4, and 60-digit decimal
logarithms for the exact values.  They then check the oracle against them and
the parity rule of tests/parity.py on them.
"""
import json
import math
import os
from decimal import Decimal, getcontext

import numpy as np
import pytest

import oracle
from parity import check_sample

HERE = os.path.dirname(os.path.abspath(__file__))
getcontext().prec = 60


def load_cases():
    with open(os.path.join(HERE, "golden", "boundary_cases.json")) as f:
        doc = json.load(f)
    out = []
    for c in doc["cases"]:
        x = np.array([float.fromhex(v) for v in c["x"]])
        y = None if c["y"] is None else np.array([float.fromhex(v) for v in c["y"]])
        out.append((c, x, y))
    return out


CASES = load_cases()


def words(ctr):
    return oracle.philox(ctr, [0, 0])


def unit_open0(hi, lo):
    return float(((int(hi) << 32 | int(lo)) >> 11) + 1) * 2.0 ** -53


def canonical_q(model, x, y):
    if model == oracle.UBCM:
        z = x[0] * x[1]
        return z / (1.0 + z)
    A = (x[0] * y[0]) * (x[1] * y[1])
    c = y[0] * y[1]
    return A / ((1.0 - c) + A)


def ids(c):
    return f"{c[0]['kind']}-m{c[0]['model']}-s{c[0]['sample']}"


def test_cases_cover_both_models_and_kinds():
    kinds = {(c["kind"], c["model"]) for c, _, _ in CASES}
    for model in (oracle.UBCM, oracle.UECM):
        assert ("q_rounding", model) in kinds and ("skip_boundary", model) in kinds
    assert ("weight_boundary", oracle.UECM) in kinds
    zs = [c["z"] for c, _, _ in CASES if c["kind"] == "q_rounding"]
    assert min(zs) < 2.0 ** 16 and max(zs) > 2.0 ** 22  # both sides of the fast range's limit


@pytest.mark.parametrize("case", CASES, ids=ids)
def test_case_claims_hold(case):
    c, x, y = case
    s = c["sample"]
    w = words([0, 0, 0, s])
    U = unit_open0(w[1], w[0])
    q = canonical_q(c["model"], x, y)
    t = math.log(U) / math.log1p(-q)
    if c["kind"] == "q_rounding":
        assert t == float.fromhex(c["t_canonical"])
        # exact -ln U / ln(1 + z), z from the FP64 products the canonical q uses
        if c["model"] == oracle.UBCM:
            z = Decimal(x[0] * x[1])
        else:
            z = Decimal((x[0] * y[0]) * (x[1] * y[1])) / Decimal(1.0 - y[0] * y[1])
        ts = -Decimal(U).ln() / (1 + z).ln()
        m = c["m"]
        assert (t < m) != (ts < m), "the canonical and exact skips agree"
        assert (t < m) == c["canonical_edge"] and (ts < m) == c["exact_edge"]
        # both well away from the integer: not a boundary draw
        assert abs(t - m) > 16 * 2.0 ** -52 * m and abs(ts - m) > Decimal(2) ** -48 * m
    elif c["kind"] == "skip_boundary":
        assert abs(t - round(t)) <= 2 * (math.nextafter(t, math.inf) - t) and round(t) == c["m"]
    else:
        assert t < 0.5
        ww = words([0x80000000, 0, 0, s])
        Uw = unit_open0(ww[1], ww[0])
        tw = math.log(Uw) / math.log(y[0] * y[1])
        assert abs(tw - c["m"]) <= 2 * (math.nextafter(tw, math.inf) - tw)


def planted_edge(c, x):
    """The edge the planted draw proposes: (0, m) (node m is the candidate at t near m)."""
    return 0, c.get("m", 1) if c["kind"] == "q_rounding" else 1


@pytest.mark.parametrize("case", CASES, ids=ids)
def test_oracle_on_planted_cases(case):
    c, x, y = case
    (src, dst, w, counts, stats), log = oracle.boundary_draws(oracle.mh_sample, c["model"], x, y,
                                                               sample_begin=c["sample"], num_samples=1)
    u, v = planted_edge(c, x)
    present = bool(np.any((src == u) & (dst == v)))
    assert present == c["canonical_edge"]
    assert int(stats[3]) == c["boundary_draws"] == len(log)
    if len(log):
        kind = 1 if c["kind"] == "weight_boundary" else 0
        assert log.tolist() == [[c["sample"], 0, 0, kind, 0]]


def flipped(c, x, y):
    """The oracle's sample with the planted edge toggled (removed if present,
    else inserted first, where row 0's edges come)."""
    src, dst, w, counts, _ = oracle.mh_sample(c["model"], x, y, sample_begin=c["sample"], num_samples=1)
    u, v = planted_edge(c, x)
    hit = np.flatnonzero((src == u) & (dst == v))
    if len(hit):
        keep = np.ones(len(src), bool)
        keep[hit] = False
        return src[keep], dst[keep], None if w is None else w[keep], counts - len(hit)
    w2 = None if w is None else np.r_[np.int32(1), w].astype(np.int32)
    return (np.r_[np.int32(u), src].astype(np.int32), np.r_[np.int32(v), dst].astype(np.int32), w2, counts + 1)


@pytest.mark.parametrize("case", CASES, ids=ids)
def test_parity_rule_on_planted_cases(case):
    c, x, y = case
    kw = dict(sample_begin=c["sample"], num_samples=1)
    other = flipped(c, x, y)
    if c["kind"] == "q_rounding":
        # the sample a sampler deciding from ln(1 + z) would draw: not a boundary draw, so rejected
        with pytest.raises(AssertionError):
            check_sample(other, c["model"], x, y, **kw)
    elif c["kind"] == "skip_boundary":
        same, _ = check_sample(other, c["model"], x, y, **kw)  # traced to the logged draw
        assert not same
    else:
        src, dst, w, counts, _ = oracle.mh_sample(c["model"], x, y, **kw)
        same, _ = check_sample((src, dst, w + 1, counts), c["model"], x, y, **kw)  # weight off by one
        assert not same


def test_parity_rule_rejects_untraced_difference():
    rng = np.random.default_rng(12)
    x = np.exp(rng.normal(-1.5, 1.0, 300))
    src, dst, _, counts, stats = oracle.mh_sample(oracle.UBCM, x, num_samples=2)
    assert int(stats[3]) == 0 and len(src) > 10
    same, _ = check_sample((src, dst, None, counts), oracle.UBCM, x, num_samples=2)
    assert same
    e = len(src) // 3  # drop one edge of the first sample
    assert e < counts[0]
    dropped = (np.delete(src, e), np.delete(dst, e), None, counts - np.array([1, 0]))
    with pytest.raises(AssertionError, match="without a boundary draw"):
        check_sample(dropped, oracle.UBCM, x, num_samples=2)
