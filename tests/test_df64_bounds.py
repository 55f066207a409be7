"""The error bounds of the mixed Kitaev stage's one-normalisation double-FP32
operations (df_fma, df_sub_dot2, df_dot2m, df_add_fast in
csrc/crbm_df64.cuh), which the stage's certified bound on log pi relies on
(Householder backward error, Sturm backward error), checked by exact
arithmetic: each FP32 operation restated with exact rationals and correct
rounding to the nearest float32 (ties to even), the fused multiply-add
rounded once, on random normalised double-FP32 operands -- including sums
that cancel -- against the exact rational result.
"""
from fractions import Fraction as Fr
import random

import pytest

U2 = Fr(1, 2 ** 48)      # (2^-24)^2


def f32(q: Fr) -> Fr:
    """q rounded to the nearest float32 (normal range), ties to even."""
    if q == 0:
        return Fr(0)
    s = -1 if q < 0 else 1
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fr(2) ** e > a:
        e -= 1
    # a in [2^e, 2^(e+1)): 24 significant bits -> unit 2^(e-23)
    scale = Fr(2) ** (e - 23)
    m = a / scale
    n = m.numerator // m.denominator
    r = m - n
    if r > Fr(1, 2) or (r == Fr(1, 2) and n % 2 == 1):
        n += 1
    return s * n * scale


def add(a, b): return f32(a + b)
def sub(a, b): return f32(a - b)
def mul(a, b): return f32(a * b)
def fma(a, b, c): return f32(a * b + c)


def two_sum(a, b):
    s = add(a, b)
    bb = sub(s, a)
    return s, add(sub(a, sub(s, bb)), sub(b, bb))


def fast_two_sum(a, b):
    s = add(a, b)
    return s, sub(b, sub(s, a))


def two_prod(a, b):
    p = mul(a, b)
    return p, fma(a, b, -p)


def df_fma(a, b, c):
    ph, pl = two_prod(a[0], b[0])
    t = add(fma(a[0], b[1], fma(a[1], b[0], pl)), c[1])
    sh, sl = two_sum(c[0], ph)
    return fast_two_sum(sh, add(sl, t))


def df_sub_dot2(a, x1, y1, x2, y2):
    p1h, p1l = two_prod(x1[0], y1[0])
    p2h, p2l = two_prod(x2[0], y2[0])
    c = fma(x1[0], y1[1], fma(x1[1], y1[0], fma(x2[0], y2[1], fma(x2[1], y2[0], add(p1l, p2l)))))
    s1h, s1l = two_sum(a[0], -p1h)
    s2h, s2l = two_sum(s1h, -p2h)
    return fast_two_sum(s2h, add(add(sub(a[1], c), s1l), s2l))


def df_dot2m(x1, y1, x2, y2):
    p1h, p1l = two_prod(x1[0], y1[0])
    p2h, p2l = two_prod(x2[0], y2[0])
    c = fma(x1[0], y1[1], fma(x1[1], y1[0], fma(-x2[0], y2[1], fma(-x2[1], y2[0], sub(p1l, p2l)))))
    sh, sl = two_sum(p1h, -p2h)
    return fast_two_sum(sh, add(sl, c))


def df_add_fast(a, b):
    sh, sl = two_sum(a[0], b[0])
    return fast_two_sum(sh, add(sl, add(a[1], b[1])))


def val(x):
    return x[0] + x[1]


def rand_df(rng, scale=1.0):
    """A normalised double-FP32 value: hi a float32, |lo| <= ulp(hi) / 2."""
    hi = f32(Fr(rng.uniform(-1.0, 1.0) * scale * 2.0 ** rng.randint(-6, 6)))
    if hi == 0:
        return (Fr(0), Fr(0))
    lo = f32(hi * Fr(rng.uniform(-1.0, 1.0)) * Fr(1, 2 ** 24))
    h2, l2 = fast_two_sum(hi, lo)
    return (h2, l2)


def near_negation(rng, x):
    """-x perturbed in its low part only: a sum with x cancels to ~2^-24 |x|."""
    return rand_df_near(rng, -val(x))


def rand_df_near(rng, q):
    hi = f32(q)
    lo = f32((q - hi) + q * Fr(rng.uniform(-1.0, 1.0)) * Fr(1, 2 ** 30))
    return fast_two_sum(hi, lo)


N_CASES = 1500


@pytest.mark.parametrize("cancel", [False, True])
def test_df_fma_bound(cancel):
    """|df_fma(a, b, c) - (a b + c)| <= 13 2^-48 |a b| + 3 2^-48 |c| (< 2^-44 (|a b| + |c|))."""
    rng = random.Random(11 + cancel)
    for _ in range(N_CASES):
        a, b = rand_df(rng), rand_df(rng)
        c = rand_df_near(rng, -val(a) * val(b)) if cancel else rand_df(rng)
        ab, cc = val(a) * val(b), val(c)
        err = abs(val(df_fma(a, b, c)) - (ab + cc))
        assert err <= U2 * (13 * abs(ab) + 3 * abs(cc)), (a, b, c, float(err))


@pytest.mark.parametrize("cancel", [False, True])
def test_df_sub_dot2_bound(cancel):
    """|df_sub_dot2(a, x1, y1, x2, y2) - (a - x1 y1 - x2 y2)| <= 2^-48 (6 |a| + 21 |x1 y1| + 23 |x2 y2|)."""
    rng = random.Random(21 + cancel)
    for _ in range(N_CASES):
        x1, y1, x2, y2 = (rand_df(rng) for _ in range(4))
        X, Y = val(x1) * val(y1), val(x2) * val(y2)
        a = rand_df_near(rng, X + Y) if cancel else rand_df(rng)
        A = val(a)
        err = abs(val(df_sub_dot2(a, x1, y1, x2, y2)) - (A - X - Y))
        assert err <= U2 * (6 * abs(A) + 21 * abs(X) + 23 * abs(Y)), float(err)


@pytest.mark.parametrize("cancel", [False, True])
def test_df_dot2m_bound(cancel):
    """|df_dot2m(x1, y1, x2, y2) - (x1 y1 - x2 y2)| <= 2^-48 (15 |x1 y1| + 17 |x2 y2|)."""
    rng = random.Random(31 + cancel)
    for _ in range(N_CASES):
        x1, y1, x2 = rand_df(rng), rand_df(rng), rand_df(rng)
        if cancel:     # x2 y2 ~ x1 y1: the Sturm recurrence near an eigenvalue
            y2 = rand_df_near(rng, val(x1) * val(y1) / val(x2)) if val(x2) != 0 else rand_df(rng)
        else:
            y2 = rand_df(rng)
        X, Y = val(x1) * val(y1), val(x2) * val(y2)
        err = abs(val(df_dot2m(x1, y1, x2, y2)) - (X - Y))
        assert err <= U2 * (15 * abs(X) + 17 * abs(Y)), float(err)


@pytest.mark.parametrize("cancel", [False, True])
def test_df_add_fast_bound(cancel):
    """|df_add_fast(a, b) - (a + b)| <= 3 2^-48 (|a| + |b|), and it is commutative
    (the warp butterflies give every lane the same sum)."""
    rng = random.Random(41 + cancel)
    for _ in range(N_CASES):
        a = rand_df(rng)
        b = near_negation(rng, a) if cancel else rand_df(rng)
        s = df_add_fast(a, b)
        assert s == df_add_fast(b, a)
        err = abs(val(s) - (val(a) + val(b)))
        assert err <= 3 * U2 * (abs(val(a)) + abs(val(b))), float(err)


def test_f32_rounding_matches_numpy():
    """The exact-rational rounding agrees with numpy's float32 conversion of
    values exactly representable in double (no double rounding there)."""
    np = pytest.importorskip("numpy")
    rng = random.Random(5)
    for _ in range(2000):
        x = rng.uniform(-1e3, 1e3)
        assert f32(Fr(x)) == Fr(float(np.float32(x)))
