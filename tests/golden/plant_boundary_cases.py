"""Writes tests/golden/boundary_cases.json: two-node networks whose first
skip draw (or first weight draw) is planted next to an integer boundary.

Test infrastructure.  Every stored value is an input (fitness values and a
sample index) or a property computed here from the paper's definitions with
Python's libm and exact decimal arithmetic; nothing comes from the CUDA
library.  Run from the repository root:  python tests/golden/plant_boundary_cases.py

Construction (Sec. 2.3 skip, Fig. 2; Eq. 4).  A two-node network has one
row (rank 0) with one segment [1, 2); its first draw d = 0 uses the Philox
counter {0, 0, 0, s} of sample s.  With q = p_01 the draw's skip is
t = log(U) / log1p(-q): the segment ends without an edge when t >= 1 and
otherwise proposes node 1, which is accepted (p/q = 1).  So the sample has an
edge exactly when t < 1.

  * "q-rounding" cases: z = x_0 x_1 (UBCM) or A / (1 - c) (UECM) between 2^11
    and about 2^30.  The canonical t divides by log1p(-fl(q)), and fl(q)
    differs from q = z / (1 + z) by up to 2^-53, which moves 1 - q by a
    relative z 2^-53.  z is chosen so that the canonical t and the exact
    t* = -ln U / ln(1 + z) lie on opposite sides of 1, both farther than
    8 ulp from it: a sampler that decides from ln(1 + z) instead of
    log1p(-fl(q)) gets the other sample.  Small U (about 1 / (1 + z)) is
    needed for t near 1, so the sample index s is searched for it.
  * "boundary" cases: the canonical t within 2 ulp of an integer (a skip
    draw), or the weight's log(U_w) / log(r) within 2 ulp of 2 (a weight
    draw of Eq. 4).  The oracle counts these draws as boundary draws.

The search over sample indices uses a numpy restatement of Philox4x32-10
(Salmon et al., SC'11); every chosen index is re-checked with the oracle's
own generator before it is stored.
"""
import json
import math
import os
import sys
from decimal import Decimal, getcontext

import numpy as np

sys.path.insert(0, os.path.abspath(os.path.join(os.path.dirname(__file__), "..", "..")))
import oracle  # noqa: E402

getcontext().prec = 60
M32 = np.uint64(0xFFFFFFFF)
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "boundary_cases.json")


def philox_np(c0, c1, c2, c3, k0, k1):
    """Philox4x32-10 on arrays (uint64 holding 32-bit words)."""
    c0, c1, c2, c3 = (np.asarray(v, np.uint64) for v in (c0, c1, c2, c3))
    k0, k1 = np.uint64(k0), np.uint64(k1)
    for rnd in range(10):
        if rnd:
            k0 = (k0 + np.uint64(0x9E3779B9)) & M32
            k1 = (k1 + np.uint64(0xBB67AE85)) & M32
        p0 = np.uint64(0xD2511F53) * c0
        p1 = np.uint64(0xCD9E8D57) * c2
        c0, c1, c2, c3 = (p1 >> np.uint64(32)) ^ c1 ^ k0, p1 & M32, (p0 >> np.uint64(32)) ^ c3 ^ k1, p0 & M32
    return c0, c1, c2, c3


def unit_open0(hi, lo):
    return float(((int(hi) << 32 | int(lo)) >> 11) + 1) * 2.0 ** -53


def small_u_samples(limit_log2=30, chunk=1 << 22, r1_max=1 << 14):
    """Sample indices s < 2^limit_log2 whose draw {0, 0, 0, s} has U < 2^-18."""
    hits = []
    for s0 in range(0, 1 << limit_log2, chunk):
        s = np.arange(s0, s0 + chunk, dtype=np.uint64)
        z = np.zeros_like(s)
        r0, r1, _, _ = philox_np(z, z, z, s, 0, 0)
        sel = np.flatnonzero(r1 < np.uint64(r1_max))
        hits += [(int(s[i]), unit_open0(r1[i], r0[i])) for i in sel]
    return hits


def oracle_u(s):
    w = oracle.philox([0, 0, 0, s], [0, 0])
    return unit_open0(w[1], w[0])


def exact_t(U, zexact):
    """-ln U / ln(1 + z) in 60-digit decimal arithmetic (U, z exact binary values)."""
    return -Decimal(U).ln() / (Decimal(1) + zexact).ln()


def ulp(v):
    return math.nextafter(v, math.inf) - v


def canonical_q(model, x0, x1, y0=None, y1=None):
    """q at the segment head in the oracle's expression order (Eq. 1; Eqs. 3, 5)."""
    if model == oracle.UBCM:
        z = x0 * x1
        return z / (1.0 + z)
    A = (x0 * y0) * (x1 * y1)
    c = y0 * y1  # two nodes: the suffix bound is r itself
    return A / ((1.0 - c) + A)


def z_exact(model, x0, x1, y0=None, y1=None):
    """The z with 1 - q = 1 / (1 + z) exactly, from the FP64 products the canonical q uses."""
    if model == oracle.UBCM:
        return Decimal(x0 * x1)
    A = (x0 * y0) * (x1 * y1)
    return Decimal(A) / Decimal(1.0 - y0 * y1)


def uecm_y(zt):
    """y_0, y_1 of a UECM case at z near zt: y_0 = 1/2 and y_1 = 1 - 2 delta, so
    c = y_0 y_1 = 1/2 - delta and 1 - c = 1/2 + delta exactly, with delta =
    0.49 ulp(A) for A = z (1 - c) near zt / 2.  Then fl((1 - c) + A) rounds A + 1/2
    + delta down by 0.49 ulp(A): when A lies just above a power of 2 that is
    almost one grid step (2^-53) of q, enough for fl(q) to cross the grid
    point next to 1 - U."""
    eA = math.floor(math.log2(zt / 2))
    delta = round(0.49 * 2.0 ** (eA - 52) / 2.0 ** -54) * 2.0 ** -54
    return 0.5, 1.0 - 2.0 * delta


def plant_q_rounding(model, U, m, ztarget):
    """x (and y) for which the canonical t and the exact t* straddle the integer m.

    m = 1: two nodes, the draw proposes node 1 or ends the segment.  m = 2:
    three nodes with x_1 = x_2 (equal p), the draw proposes node 2 or ends it.
    For m = 1 the q with 1 - q = U gives t = 1 exactly, so a straddle needs
    fl(q) to miss the exact q by more than one grid step of 2^-53.  The UBCM
    cannot: for z >= 1, 1 + z is exact and fl(q) = q rounded once, within half
    a step.  The UECM can, since fl((1 - c) + A) rounds too.  For m = 2 the
    boundary is not on that grid, so both models can."""
    E = -Decimal(U).ln()
    zt = float((E / m).exp() - 1)  # t* = m here
    # m = 2 needs no rounding of 1 - c; its third node pairs with the second at
    # r = y_1^2, which must stay well below 1 (weights of Eq. 4)
    y = (uecm_y(zt) if m == 1 else (0.6, 0.7)) if model == oracle.UECM else (None, None)
    p = math.ceil(math.log2(zt) / 2) + 1  # x0 = 2^p > x1
    x0 = 2.0 ** p
    ks = np.arange(-6000, 6001, dtype=np.float64)
    zk = zt * (1.0 + ks * 2.0 ** -46)
    if model == oracle.UBCM:
        x1s = zk / x0
    else:  # A / (1 - c) = zk with a = x y and c = y_0 y_1 (the suffix bound of two equal-y candidates)
        x1s = zk * (1.0 - y[0] * y[1]) / (x0 * y[0] * y[1])
    # prefilter in numpy (its log may differ from libm's in the last bit), then
    # decide every kept candidate with libm and 60-digit decimals
    if model == oracle.UBCM:
        zz = x0 * x1s
        qs = zz / (1.0 + zz)
        zex = zz
    else:
        A = (x0 * y[0]) * (x1s * y[1])
        qs = A / ((1.0 - y[0] * y[1]) + A)
        zex = A / (1.0 - y[0] * y[1])
    t_np = np.log(U) / np.log1p(-qs)
    ts_np = float(E) / np.log1p(zex)
    keep = np.flatnonzero((np.abs(t_np - m) < 1e-9) & (np.abs(ts_np - m) < 1e-9)
                          & (((t_np < m) != (ts_np < m)) | (np.abs(t_np - m) < 4e-16 * m) | (np.abs(ts_np - m) < 4e-16 * m)))
    best = None
    for i in keep:
        x1 = float(x1s[i])
        q = canonical_q(model, x0, x1, *y)
        if not (q < 1.0):
            continue
        t = math.log(U) / math.log1p(-q)
        ts = exact_t(U, z_exact(model, x0, x1, *y))
        if (t < m) == (ts < m):
            continue
        margin = min(abs(t - m), float(abs(ts - m)))
        if margin < 64 * ulp(float(m)):
            continue
        if best is None or margin > best[0]:
            best = (margin, x1, t, ts)
    if best is None:
        return None
    margin, x1, t, ts = best
    zex = z_exact(model, x0, x1, *y)
    xs = [x0, x1] if m == 1 else [x0, x1, x1]
    ys = None if y[0] is None else [y[0], y[1]] if m == 1 else [y[0], y[1], y[1]]
    return dict(kind="q_rounding", model=int(model), x=xs, y=ys, m=m, z=float(zex), t_canonical=t.hex(),
                t_exact=str(ts), canonical_edge=bool(t < m), exact_edge=bool(ts < m), boundary_draws=0,
                ztarget_log2=ztarget)


def plant_skip_boundary(model, U, m=1):
    """x with the canonical t within 2 ulp of the integer m (a boundary draw)."""
    E = -math.log(U)
    y = (0.5, 0.5) if model == oracle.UECM else (None, None)
    zt = math.expm1(E / m)
    x0 = 4.0 * max(1.0, math.sqrt(zt))
    for k in range(0, 400000):
        for sgn in (1, -1):
            zk = zt * (1.0 + sgn * k * 2.0 ** -52)
            x1 = zk / x0 if model == oracle.UBCM else zk * 0.75 / (x0 * 0.25)
            q = canonical_q(model, x0, x1, *y)
            t = math.log(U) / math.log1p(-q)
            if abs(t - m) <= 2 * ulp(float(m)):
                return dict(kind="skip_boundary", model=int(model), x=[x0, x1],
                            y=None if y[0] is None else list(y), t_canonical=t.hex(), m=m,
                            canonical_edge=bool(t < 1.0), boundary_draws=1)
    return None


def plant_weight_boundary(s, m=2):
    """UECM: the first edge's weight draw with log(U_w)/log(r) within 2 ulp of m."""
    w = oracle.philox([0x80000000, 0, 0, s], [0, 0])
    Uw = unit_open0(w[1], w[0])
    if not (Uw < 0.2):
        return None
    y0 = 0.5
    rt = math.exp(math.log(Uw) / m)
    for k in range(0, 400000):
        for sgn in (1, -1):
            y1 = rt / y0 * (1.0 + sgn * k * 2.0 ** -52)
            r = y0 * y1
            tw = math.log(Uw) / math.log(r)
            if abs(tw - m) <= 2 * ulp(float(m)):
                x = [300.0, 100.0]  # q close to 1: the skip draw proposes node 1
                U = oracle_u(s)
                q = canonical_q(oracle.UECM, x[0], x[1], y0, y1)
                t = math.log(U) / math.log1p(-q)
                if not (t < 0.5):
                    return None
                return dict(kind="weight_boundary", model=int(oracle.UECM), x=x, y=[y0, y1],
                            tw_canonical=tw.hex(), m=m, canonical_edge=True, boundary_draws=1)
    return None


def first_draw_u(count):
    s = np.arange(0, count, dtype=np.uint64)
    z = np.zeros_like(s)
    r0, r1, _, _ = philox_np(z, z, z, s, 0, 0)
    u = ((((r1 << np.uint64(32)) | r0) >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
    return s, u


def main():
    cache = sys.argv[sys.argv.index("--hits-cache") + 1] if "--hits-cache" in sys.argv else None
    if cache and os.path.exists(cache):
        hits = [(int(a), float(b)) for a, b in np.load(cache).tolist()]
    else:
        hits = small_u_samples()
        if cache:
            np.save(cache, np.array(hits, dtype=np.float64))
    hits.sort(key=lambda h: h[1])
    print(f"{len(hits)} sample indices with U < 2^-18; smallest U = 2^{math.log2(hits[0][1]):.1f}", flush=True)
    s_small, u_small = first_draw_u(1 << 22)
    cases = []
    # q-rounding cases.  m = 1 at z just above 2^zt (U in (2^-zt / 1.15, 2^-zt]),
    # m = 2 at z near 2^zt (U near 2^(-2 zt)).
    m1 = [(1, zt) for zt in (11, 13, 15, 17, 19, 21, 23, 25, 27, 29)]
    m2 = [(2, zt) for zt in (11, 12, 13, 14, 15)]
    for model in (oracle.UBCM, oracle.UECM):
        used = set()
        for m, zt in (m2 if model == oracle.UBCM else m1 + m2[:2]):
            if m == 1:  # z (and A = z (1 - c), about z / 2) just above a power of 2
                lo, hi = 2.0 ** -zt / 1.08, 2.0 ** -zt
            else:
                lo, hi = 2.0 ** (-2 * zt) / 1.5, 2.0 ** (-2 * zt) * 1.5
            cand = [h for h in hits if lo < h[1] <= hi]
            sel = np.flatnonzero((u_small > lo) & (u_small <= hi))
            cand += [(int(s_small[i]), float(u_small[i])) for i in sel]
            cand = [h for h in cand if h[0] not in used]
            for s, U in cand[:64]:
                assert U == oracle_u(s), "numpy Philox disagrees with the oracle's"
                c = plant_q_rounding(model, U, m, zt)
                if c is not None:
                    c["sample"] = s
                    used.add(s)
                    cases.append(c)
                    print(f"model {model} m {m} z ~ 2^{math.log2(c['z']):.2f} s = {s}: "
                          f"canonical edge {c['canonical_edge']}, exact edge {c['exact_edge']}", flush=True)
                    break
            else:
                print(f"model {model} m {m} z ~ 2^{zt}: no straddle among {len(cand[:64])} draws", flush=True)
    # boundary draws (the oracle counts them): skip draws near 1 and 2, a weight draw near 2
    for model in (oracle.UBCM, oracle.UECM):
        for s in range(100, 200):
            U = oracle_u(s)
            if not (0.05 < U < 0.5):
                continue
            c = plant_skip_boundary(model, U, m=1)
            if c is not None:
                c["sample"] = s
                cases.append(c)
                print(f"model {model} skip boundary s = {s}: t = {float.fromhex(c['t_canonical'])!r}")
                break
    for s in range(300, 400):
        c = plant_weight_boundary(s)
        if c is not None:
            c["sample"] = s
            cases.append(c)
            print(f"weight boundary s = {s}: tw = {float.fromhex(c['tw_canonical'])!r}")
            break
    for c in cases:
        c["x"] = [v.hex() for v in c["x"]]
        if c["y"] is not None:
            c["y"] = [v.hex() for v in c["y"]]
    doc = {
        "what": "two-node networks whose first skip or weight draw is planted next to an integer boundary; "
                "values are FP64 hex strings (float.fromhex); seed 0, network id 0, one sample at 'sample', "
                "segment length 32",
        "source": "tests/golden/plant_boundary_cases.py (Sec. 2.3 skip law, Fig. 2; Eq. 4)",
        "cases": cases,
    }
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=1)
    print(f"{len(cases)} cases -> {OUT}")


if __name__ == "__main__":
    main()
