"""Planted mistakes in the CPU oracle must fail the pins (no GPU).

Each case edits a copy of oracle/mh_oracle.c (a dropped term, a wrong
operand, an off-by-one, a wrong bound), compiles it to a temporary library
and checks that the exact-enumeration, marginal or weight-law pin rejects it.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle
from tests.oracle_pins import enumeration_pvalue, marginal_zmax, weight_pvalue
from tests.test_oracle import UBCM_CASES, UECM_X, UECM_Y

SRC = os.path.join(os.path.dirname(oracle.__file__), "mh_oracle.c")

# (name, original text, replacement, which pin should catch it)
MUTATIONS = [
    ("skip_missing_plus_one", "int64_t j = pos + 1 + (int64_t)floor(t);", "int64_t j = pos + (int64_t)floor(t);",
     "ubcm"),
    ("accept_without_dividing_by_q", "if (V < p / q) {", "if (V < p) {", "ubcm"),
    ("first_candidate_without_skip", "double t = (q >= 1.0) ? 0.0 : log(U) / log1p(-q);",
     "double t = (q >= 1.0 || d == 1) ? 0.0 : log(U) / log1p(-q);", "ubcm"),
    ("sort_ascending", "if (a->key > b->key) return -1;\n    if (a->key < b->key) return 1;",
     "if (a->key > b->key) return 1;\n    if (a->key < b->key) return -1;", "ubcm"),
    ("ubcm_q_not_updated_to_p", "q = uecm ? prob_hat(g, i, j, c) : p;", "q = uecm ? prob_hat(g, i, j, c) : q * 0.5;",
     "ubcm"),
    ("uecm_q_from_p_not_phat", "q = uecm ? prob_hat(g, i, j, c) : p;", "q = p;", "uecm"),
    ("uecm_bound_from_head_y_only", "return g->ys[i] * g->ymax[a];", "return g->ys[i] * g->ys[a];", "uecm"),
    ("uecm_r_dropped_from_p", "return A / ((1.0 - r) + A);", "return A / (1.0 + A);", "uecm"),
    ("weight_log_of_one_minus_r", "double tw = log(Uw) / log(r);", "double tw = log(Uw) / log1p(-r);", "weight"),
    ("weight_missing_plus_one", "wt = 1 + (int32_t)floor(tw);", "wt = (int32_t)floor(tw);", "weight"),
]


def _compile(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation {name}: text not found"
    mutated = src.replace(old, new)
    c_path = tmp_path / f"{name}.c"
    so_path = tmp_path / f"{name}.so"
    c_path.write_text(mutated)
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so_path),
                    str(c_path), "-lm"], check=True)
    return oracle.load(str(so_path))


@pytest.mark.parametrize("name,old,new,pin", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(tmp_path, name, old, new, pin):
    lib = _compile(tmp_path, name, old, new)
    if pin == "ubcm":
        pvals = [enumeration_pvalue(oracle.UBCM, x, samples=20000, lib=lib, seg_target=T)
                 for x in UBCM_CASES for T in (2, 1 << 30)]
        assert min(pvals) < 1e-8
    elif pin == "uecm":
        p = min(enumeration_pvalue(oracle.UECM, UECM_X, UECM_Y, samples=40000, lib=lib, seg_target=T)
                for T in (2, 1 << 30))
        rng = np.random.default_rng(3)
        x = np.exp(rng.normal(-0.5, 1.2, 12))
        y = rng.uniform(0.1, 0.9, 12)
        z = marginal_zmax(oracle.UECM, x, y, lib=lib)
        assert p < 1e-8 or z > 8.0
    else:
        assert weight_pvalue(UECM_X, UECM_Y, lib=lib) < 1e-8


# Planted mistakes in the bipartite / directed walk (Sec. 2.6).
BIP_MUTATIONS = [
    ("directed_self_pair_not_excluded",
     "int64_t ex = directed ? (int64_t)B.rank_c[B.R.perm[i]] : -1;", "int64_t ex = -1;", "directed"),
    ("virtual_position_off_by_one", "return (ex >= 0 && v >= ex) ? v + 1 : v;",
     "return (ex >= 0 && v > ex) ? v + 1 : v;", "directed"),
    ("bipartite_bound_from_head_y_only", "return B->R.ys[i] * B->C.ymax[a];", "return B->R.ys[i] * B->C.ys[a];",
     "bipartite_uecm"),
]


@pytest.mark.parametrize("name,old,new,pin", BIP_MUTATIONS, ids=[m[0] for m in BIP_MUTATIONS])
def test_planted_bipartite_mistake_is_caught(tmp_path, name, old, new, pin):
    from tests.test_oracle_bipartite import DIR_XI, DIR_XO, DIR_YI, DIR_YO, bip_code_counts, bip_enumeration_pvalue
    lib = _compile(tmp_path, name, old, new)
    if pin == "directed":
        caught = False
        for model in (oracle.UBCM, oracle.UECM):
            yo, yi = (DIR_YO, DIR_YI) if model == oracle.UECM else (None, None)
            for T in (2, 1 << 30):
                src, dst, _, counts, _ = oracle.bip_sample(model, DIR_XO, yo, DIR_XI, yi, directed=True,
                                                           num_samples=20000, seg_target=T, lib=lib)
                hist = bip_code_counts(src, dst, counts, 3, 3, True)
                if hist[-1] > 0:
                    caught = True
                    continue
                if bip_enumeration_pvalue(model, DIR_XO, DIR_XI, yo, yi, directed=True, samples=20000,
                                          seg_target=T, lib=lib) < 1e-8:
                    caught = True
        assert caught
    else:
        # the - set in sorted order has y rising while a = x y falls, so in a
        # whole-row segment (T = 2^30) the head's y understates r_ij for every
        # later candidate and those pairs are proposed too rarely
        from tests.oracle_pins import alpha_of
        ym = np.array([0.1, 0.3, 0.5, 0.7, 0.9])
        xm = np.array([1.0, 0.8, 0.6, 0.4, 0.2]) / ym
        yp = np.array([0.95, 0.6])
        xp = np.array([1.0, 0.5]) / yp
        S = 20000
        src, dst, _, counts, _ = oracle.bip_sample(oracle.UECM, xp, yp, xm, ym, num_samples=S,
                                                   seg_target=1 << 30, lib=lib)
        ap, am, bp, bm = alpha_of(xp), alpha_of(xm), alpha_of(yp), alpha_of(ym)
        zmax = 0.0
        for (u, v) in oracle.bip_pair_list(2, 5):
            num = np.exp(-ap[u] - am[v] - bp[u] - bm[v])
            p = num / (1.0 - np.exp(-bp[u] - bm[v]) + num)
            f = ((src == u) & (dst == v)).sum() / S
            zmax = max(zmax, abs(f - p) / np.sqrt(p * (1 - p) / S))
        assert zmax > 6.0


# Planted mistakes in the oracle's Jacobian diagonal (Python): each must be
# rejected by the central-difference pin that the original passes.
JAC_MUTATIONS = [
    ("ds_dy_power_of_one_minus_r", "p * r / (y[i] * (1.0 - r) ** 2)", "p * r / (y[i] * (1.0 - r))"),
    ("dk_dy_missing_y", "math.fsum((p / (y[i] * D)).tolist())", "math.fsum((p / D).tolist())"),
    ("ds_dx_missing_one_minus_r", "math.fsum((dp_dx / (1.0 - r)).tolist())", "math.fsum(dp_dx.tolist())"),
    ("dk_dx_missing_one_minus_p", "dp_dx = p * (1.0 - p) / x[i]", "dp_dx = p / x[i]"),
]


def _mutant(func, old, new):
    import inspect
    import textwrap
    src = textwrap.dedent(inspect.getsource(func))
    assert src.count(old) == 1, old
    ns = dict(vars(oracle))
    exec(compile(src.replace(old, new), "<mutant>", "exec"), ns)
    return ns[func.__name__]


def _worst_jacobian_mismatch(jac, model):
    rng = np.random.default_rng(19)
    n = 12
    x = np.exp(rng.normal(-0.5, 1.0, n))
    y = rng.uniform(0.2, 0.9, n) if model == oracle.UECM else None
    diag = jac(model, x, y)
    worst = 0.0
    for i in range(n):
        for which, arr in (("x", x), ("y", y)):
            if arr is None:
                continue
            h = 1e-6 * arr[i]
            up, dn = arr.copy(), arr.copy()
            up[i] += h
            dn[i] -= h
            args = ((up, y), (dn, y)) if which == "x" else ((x, up), (x, dn))
            (kp, sp), (km, sm) = (oracle.expected_fwd(model, a, b, rows=[i]) for a, b in args)
            fd = [(kp[0] - km[0]) / (2 * h)] + ([(sp[0] - sm[0]) / (2 * h)] if y is not None else [])
            got = ([diag[0][i]] + ([diag[2][i]] if y is not None else [])) if which == "x" else \
                [diag[1][i], diag[3][i]]
            for f, g in zip(fd, got):
                worst = max(worst, abs(f - g) / max(1.0, abs(f)))
    return worst


def test_jacobian_diagonal_pin_accepts_the_oracle():
    for model in (oracle.UBCM, oracle.UECM):
        assert _worst_jacobian_mismatch(oracle.expected_jacobian_diag, model) < 1e-6


@pytest.mark.parametrize("name,old,new", JAC_MUTATIONS, ids=[m[0] for m in JAC_MUTATIONS])
def test_planted_mistake_in_the_jacobian_diagonal_is_caught(name, old, new):
    mutant = _mutant(oracle.expected_jacobian_diag, old, new)
    assert _worst_jacobian_mismatch(mutant, oracle.UECM) > 1e-3


# Planted mistakes in the oracle's gradient of the expected sums.
BWD_MUTATIONS = [
    ("upstream_k_of_j_dropped", "gk = g_k[i] + g_k[j]", "gk = g_k[i] + 0.0 * g_k[j]"),
    ("upstream_s_of_j_dropped", "gs = g_s[i] + g_s[j]", "gs = g_s[i] + 0.0 * g_s[j]"),
    ("dm_dx_missing_one_minus_r", "dm_dx = dp_dx / (1.0 - r)", "dm_dx = dp_dx"),
    ("dp_dy_wrong_denominator", "dp_dy = p / (y[i] * D)", "dp_dy = p / (y[i] * y[i])"),
]


def _worst_gradient_mismatch(bwd, model):
    rng = np.random.default_rng(8)
    n = 12
    x = np.exp(rng.normal(-0.5, 1.0, n))
    y = rng.uniform(0.2, 0.9, n) if model == oracle.UECM else None
    gk = rng.normal(size=n)
    gs = rng.normal(size=n) if y is not None else None

    def loss(xx, yy):
        k, s = oracle.expected_fwd(model, xx, yy)
        return float(np.dot(gk, k) + (np.dot(gs, s) if s is not None else 0.0))

    gx, gy = bwd(model, x, y, gk, gs)
    worst = 0.0
    for i in range(n):
        for arr, g in ((x, gx), (y, gy)):
            if arr is None:
                continue
            h = 1e-6 * arr[i]
            up, dn = arr.copy(), arr.copy()
            up[i] += h
            dn[i] -= h
            fd = ((loss(up, y) - loss(dn, y)) if arr is x else (loss(x, up) - loss(x, dn))) / (2 * h)
            worst = max(worst, abs(fd - g[i]) / max(1.0, abs(fd)))
    return worst


def test_gradient_pin_accepts_the_oracle():
    for model in (oracle.UBCM, oracle.UECM):
        assert _worst_gradient_mismatch(oracle.expected_bwd, model) < 1e-6


@pytest.mark.parametrize("name,old,new", BWD_MUTATIONS, ids=[m[0] for m in BWD_MUTATIONS])
def test_planted_mistake_in_the_gradient_is_caught(name, old, new):
    mutant = _mutant(oracle.expected_bwd, old, new)
    assert _worst_gradient_mismatch(mutant, oracle.UECM) > 1e-3
