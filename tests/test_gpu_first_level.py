"""The walk's first decision level (mh_debug_first_level) against FP64 (GPU).

The skip of a proposal is L = 1 + floor(t), t = ln U / ln(1 - q) (Sec. 2.3,
Fig. 2).  The walk's first level evaluates E = -ln U and lambda = -ln(1 - q)
= log1p(z) as pairs of FP32 numbers and decides floor(t) only when t lies
farther than t 2^-28 + 2^-22 from every integer.  Its error analysis claims
E within 2^-31.5 and lambda within 2^-31.3 (relative); these tests check the
claimed bounds on random and adversarial inputs (both sides of the series /
table switch, table points, powers of two, the whole-word normalisation of
U < 2^-8), and that every decided floor equals the FP64 floor of
log(U) / log1p(-q), also for t placed within a few margins of an integer.
"""
import numpy as np
import pytest
import torch

from paper_2509_13230_gb300 import _native as nat
from paper_2509_13230_gb300.sampler import _ptr

pytestmark = pytest.mark.gpu

E_BOUND = 2.0**-31.5
LAM_BOUND = 2.0**-31.3


def run(N, z, room):
    N = np.asarray(N, dtype=np.int64)
    z = np.asarray(z, dtype=np.float64)
    room = np.asarray(room, dtype=np.int32)
    n = len(N)
    dN, dz, dr = (torch.from_numpy(a).cuda() for a in (N, z, room))
    E = torch.empty(2 * n, dtype=torch.float32, device="cuda")
    lam = torch.empty(2 * n, dtype=torch.float32, device="cuda")
    fl = torch.empty(n, dtype=torch.int32, device="cuda")
    assert nat.mh_debug_first_level(_ptr(dN), _ptr(dz), _ptr(dr), n, _ptr(E), _ptr(lam), _ptr(fl), None) == nat.MH_OK
    torch.cuda.synchronize()
    E = E.cpu().numpy().astype(np.float64).reshape(n, 2)
    lam = lam.cpu().numpy().astype(np.float64).reshape(n, 2)
    return E[:, 0] + E[:, 1], lam[:, 0] + lam[:, 1], fl.cpu().numpy()


def neg_ln_u(N):
    N = np.asarray(N, dtype=np.int64)
    W = (1 << 53) - N
    U = N.astype(np.float64) * 2.0**-53  # exact: N <= 2^53
    return np.where(W < (1 << 44), -np.log1p(-W.astype(np.float64) * 2.0**-53), -np.log(U))


def z_df(z):
    """z rounded to a double-float, as the walk holds x_i x_j."""
    hi = z.astype(np.float32).astype(np.float64)
    return hi + (z - hi).astype(np.float32).astype(np.float64)


def canonical_floor(N, z, room):
    """The canonical FP64 skip: floor(log(U) / log1p(-q)), q = z / (1 + z), capped at room."""
    U = np.asarray(N, dtype=np.float64) * 2.0**-53
    q = z / (1.0 + z)
    t = np.log(U) / np.log1p(-q)
    return np.where(t >= room, room, np.floor(np.minimum(t, 2.0**40))).astype(np.int64), t


def special_N():
    out = [1, 2, 3, 5, (1 << 21) - 1, 1 << 21, (1 << 21) + 1, (1 << 44) - 1, 1 << 44, (1 << 44) + 1,
           (1 << 53) - 1, 1 << 53, (1 << 53) - (1 << 44), (1 << 53) - (1 << 44) - 1, (1 << 53) - (1 << 44) + 1,
           (1 << 53) - (1 << 21), (1 << 53) - (1 << 20)]
    for k in range(1, 54):
        for d in (-3, -1, 0, 1, 3):
            v = (1 << k) + d
            if 1 <= v <= 1 << 53:
                out.append(v)
            v = 3 * (1 << k) // 2 + d  # f near 1.5
            if 1 <= v <= 1 << 53:
                out.append(v)
    # table points c_k 2^e and their neighbours, at several exponents
    for e in (52, 45, 44, 30, 10):
        for k in range(0, 512, 7):
            c = (1.0 + k * 2.0**-9) if k < 256 else 0.5 * (1.0 + k * 2.0**-9)
            base = int(c * 2.0**e)
            for d in (-1, 0, 1):
                if 1 <= base + d <= 1 << 53:
                    out.append(base + d)
    return np.array(out, dtype=np.int64)


def special_z():
    out = [2.0**-100, 2.0**-60, 2.0**-30, 2.0**-10, np.nextafter(2.0**-9, 0), 2.0**-9, np.nextafter(2.0**-9, 1),
           1e-3, 0.5, 1.0, 2.0, 3.0, 1e3, 65535.0]
    for k in range(0, 512, 5):
        c = (1.0 + k * 2.0**-9) if k < 256 else 0.5 * (1.0 + k * 2.0**-9)
        for e in (0, 1, 3, 10):
            v = c * 2.0**e - 1.0
            for d in (-2.0**-40, 0.0, 2.0**-40):
                if 2.0**-9 <= v + d < 2.0**16:
                    out.append(v + d)
    return np.array(out, dtype=np.float64)


def test_first_level_error_bounds():
    rng = np.random.default_rng(11)
    n = 1 << 20
    N = np.concatenate([rng.integers(1, (1 << 53) + 1, n), (1 << 53) - rng.integers(0, 1 << 44, n // 4),
                        rng.integers(1, 1 << 44, n // 4), np.exp2(rng.uniform(0, 53, n // 4)).astype(np.int64),
                        special_N()])
    N = np.clip(N, 1, 1 << 53)
    z = np.concatenate([np.exp2(rng.uniform(-100, 15.99, len(N) - len(special_z()))), special_z()])
    E, lam, _ = run(N, z, np.zeros(len(N)))
    E_ref = neg_ln_u(N)
    lam_ref = np.log1p(z_df(z))
    e_err = np.where(E_ref > 0, np.abs(E - E_ref) / np.where(E_ref > 0, E_ref, 1.0), np.abs(E))  # U = 1: E = 0
    l_err = np.abs(lam - lam_ref) / lam_ref
    assert e_err.max() <= E_BOUND, (np.log2(e_err.max()), N[np.argmax(e_err)])
    assert l_err.max() <= LAM_BOUND, (np.log2(l_err.max()), z[np.argmax(l_err)])


def test_first_level_decisions_equal_fp64():
    rng = np.random.default_rng(12)
    n = 1 << 20
    # random draws over the walk's range of t: z from 2^-40 (skips of 10^12, past any segment) to 2^16
    N = rng.integers(1, (1 << 53) + 1, n)
    z = np.exp2(rng.uniform(-40, 15.99, n))
    room = rng.integers(0, 1 << 22, n)  # segments of up to 4 M candidates
    room[: n // 8] = rng.integers(0, 1 << 31, n // 8)
    _, _, fl = run(N, z, room)
    want, t = canonical_floor(N, z, room)
    dec = fl >= 0
    # fl >= room and the FP64 t >= room both end the segment
    assert np.array_equal(np.minimum(fl[dec], room[dec]), want[dec])
    # the level leaves to the next one only draws near an integer (or t tiny)
    margin = t * 2.0**-28 + 2.0**-22
    d = np.abs(t - np.rint(t))
    inside = t < room
    assert dec[(d > 4.0 * margin) & inside].all()
    expected = np.minimum(1.0, 2.0 * margin[inside]).sum()
    assert (~dec[inside]).sum() <= 2.0 * expected + 20


@pytest.mark.parametrize("offset_margins", [-8.0, -2.0, -0.5, 0.5, 2.0, 8.0])
def test_first_level_near_integers(offset_margins):
    """t placed a few margins from an integer m: decided floors equal FP64, and
    draws beyond two margins are decided."""
    rng = np.random.default_rng(13 + int(4 * (offset_margins + 8.0)))
    n = 1 << 18
    z = np.exp2(rng.uniform(-30, 8, n))
    q = z / (1.0 + z)
    lam = -np.log1p(-q)
    m = np.floor(np.exp2(rng.uniform(0, 22, n)))
    t_target = m + offset_margins * (m * 2.0**-28 + 2.0**-22)
    N = np.rint(np.exp(-t_target * lam) * 2.0**53)
    ok = (N >= 1) & (N <= 2.0**53)
    N, z, m = N[ok].astype(np.int64), z[ok], m[ok]
    room = np.full(len(N), (1 << 31) - 1)
    _, _, fl = run(N, z, room)
    want, t = canonical_floor(N, z, room)
    dec = fl >= 0
    assert np.array_equal(fl[dec], want[dec])
    dist = np.abs(t - np.rint(t))
    far = dist > 2.0 * (t * 2.0**-28 + 2.0**-22)
    assert dec[far].all()
    near = dist < 0.5 * (t * 2.0**-28)
    assert not dec[near].any()


def test_first_level_argument_errors():
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    assert nat.mh_debug_first_level(None, _ptr(x), _ptr(x), 4, _ptr(x), _ptr(x), _ptr(x), None) == nat.MH_ERR_ARG
    assert nat.mh_debug_first_level(_ptr(x), _ptr(x), _ptr(x), -1, _ptr(x), _ptr(x), _ptr(x), None) == nat.MH_ERR_ARG
    assert nat.mh_debug_first_level(None, None, None, 0, None, None, None, None) == nat.MH_OK
