"""The offset-grid sum that the double-word Wilson hop and the force kernel use
for their SU(3) products, restated in exact rational arithmetic on the host.

Method: for r = W h = A + iB with A = sum_b h_b.re W_b and B = sum_b h_b.im W_b,
sigma is the power of two 2^(e+2), where 2^e <= m < 2^(e+1) and
m = max|W.hi| * max(sum_b |h_b.re.hi|, sum_b |h_b.im.hi|) * (1 + 2^-19).
Every partial sum of exact high products is then below sigma/2.  A starts at
(1.5 sigma, 1.5 sigma) and B at (-1.5 sigma, 1.5 sigma).  Per product:
T' = fl(a.h b.h + T); d = fl(a.h b.h + (T - T')); c += d + a.h b.l + a.l b.h.

Checked here, on random links (SU(3) and general complex matrices with
components up to ~12) and spinors scaled by 2^-60 ... 2^60:
  * T - T' is exact (every accumulator lane stays in one binade; Sterbenz);
  * the high words of A + iB join exactly ((T0 + A.re) - (T0 + B.im) and
    (T0 + A.im) + (-T0 + B.re));
  * the double-word result agrees with the exact product to a few 1e-14.
The force kernel's outer products P_ba = sum_s v_sb conj(c_sa), nine entries
on one grid per part, are checked the same way.
FP32 rounding is emulated exactly with Python fractions (round to nearest
even, binary32 normal range), so no GPU is involved.
"""
import math
from fractions import Fraction

import numpy as np
import pytest


def rn32(x: Fraction) -> Fraction:
    """x rounded to the nearest binary32 value (ties to even), normal range."""
    if x == 0:
        return Fraction(0)
    s = -1 if x < 0 else 1
    a = abs(x)
    e = math.floor(math.log2(a.numerator) - math.log2(a.denominator))
    while Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    ulp = Fraction(2) ** (e - 23)
    q, r = divmod(a, ulp)
    if r > ulp / 2 or (r == ulp / 2 and q % 2 == 1):
        q += 1
    return s * q * ulp


def is_f32(x: Fraction) -> bool:
    return rn32(x) == x


def split_dw(v: float):
    """A double as a double-word pair (hi, lo) of binary32 values."""
    h = rn32(Fraction(v))
    return h, rn32(Fraction(v) - h)


def pow2_floor(m: Fraction) -> Fraction:
    e = math.floor(math.log2(m.numerator) - math.log2(m.denominator))
    p = Fraction(2) ** e
    while p > m:
        p /= 2
    while 2 * p <= m:
        p *= 2
    return p


def grid_matvec(W, h):
    """r = W h for one half-spinor colour vector, as the kernels compute it.
    W: 3x3 of ((re.h, re.l), (im.h, im.l)); h: 3 of the same.  Returns the
    three results as ((re.h, re.l), (im.h, im.l)) and asserts the exactness
    of every step the method relies on."""
    wmax = max(abs(W[a][b][k][0]) for a in range(3) for b in range(3) for k in range(2))
    wmax = rn32(wmax * rn32(Fraction(1) + Fraction(1, 2 ** 19)))
    sr = rn32(rn32(abs(h[0][0][0]) + abs(h[1][0][0])) + abs(h[2][0][0]))
    si = rn32(rn32(abs(h[0][1][0]) + abs(h[1][1][0])) + abs(h[2][1][0]))
    m = rn32(max(sr, si) * wmax)
    sigma = 4 * pow2_floor(m) if m > 0 else Fraction(2) ** -125
    t0 = rn32(Fraction(3, 2) * sigma)
    assert t0 == Fraction(3, 2) * sigma
    out = []
    for a in range(3):
        lanes = {}
        for which, start in ((0, (t0, t0)), (1, (-t0, t0))):  # A: multiplier h.re, B: h.im
            res = []
            for lane in (0, 1):  # lane 0: W.re, lane 1: W.im
                T, c = start[lane], Fraction(0)
                for b in range(3):
                    mh, ml = h[b][which]
                    wh, wl = W[a][b][lane]
                    Tn = rn32(mh * wh + T)
                    q = T - Tn
                    assert is_f32(q), "T - T' must be exact"
                    assert sigma <= abs(Tn) < 2 * sigma, "accumulator left its binade"
                    d = rn32(mh * wh + q)
                    t = d if b == 0 else rn32(c + d)
                    t = rn32(mh * wl + t)
                    c = rn32(ml * wh + t)
                    T = Tn
                res.append((T, c))
            lanes[which] = res
        (ATre, Acre), (ATim, Acim) = lanes[0]
        (BTre, Bcre), (BTim, Bcim) = lanes[1]
        hre, him = ATre - BTim, ATim + BTre  # i B = (-B.im, B.re)
        assert is_f32(hre) and is_f32(him), "the high words must join exactly"
        out.append(((hre, rn32(Acre - Bcim)), (him, rn32(Acim + Bcre))))
    return out


def su3(rng):
    z = (rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))) / np.sqrt(2)
    q, r = np.linalg.qr(z)
    q = q * (np.diag(r) / np.abs(np.diag(r)))
    return q / np.linalg.det(q) ** (1 / 3)


@pytest.mark.parametrize("links", ["su3", "general"])
@pytest.mark.parametrize("scale_exp", [-60, 0, 60])
def test_grid_matvec_exact_steps_and_error(links, scale_exp):
    rng = np.random.default_rng(1000 + scale_exp + (100 if links == "general" else 0))
    worst = 0.0
    for _ in range(6):
        Wc = su3(rng) if links == "su3" else 4.0 * (rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3)))
        hc = (rng.normal(size=3) + 1j * rng.normal(size=3)) * 2.0 ** scale_exp
        W = [[(split_dw(Wc[a, b].real), split_dw(Wc[a, b].imag)) for b in range(3)] for a in range(3)]
        h = [(split_dw(hc[b].real), split_dw(hc[b].imag)) for b in range(3)]
        got = grid_matvec(W, h)
        # exact product of the double-word inputs
        Wx = [[(W[a][b][0][0] + W[a][b][0][1], W[a][b][1][0] + W[a][b][1][1]) for b in range(3)] for a in range(3)]
        hx = [(h[b][0][0] + h[b][0][1], h[b][1][0] + h[b][1][1]) for b in range(3)]
        num = den = Fraction(0)
        for a in range(3):
            ere = sum(Wx[a][b][0] * hx[b][0] - Wx[a][b][1] * hx[b][1] for b in range(3))
            eim = sum(Wx[a][b][0] * hx[b][1] + Wx[a][b][1] * hx[b][0] for b in range(3))
            gre = got[a][0][0] + got[a][0][1]
            gim = got[a][1][0] + got[a][1][1]
            num += (gre - ere) ** 2 + (gim - eim) ** 2
            den += ere ** 2 + eim ** 2
        worst = max(worst, math.sqrt(float(num / den)))
    # a few 1e-14 typical; the kernels' gate per apply is 1e-12
    assert worst <= 3e-13, worst


def test_grid_matvec_zero_half_spinor():
    """h = 0: sigma falls to its floor 2^-125 (a normal binary32) and the
    result is exactly zero."""
    rng = np.random.default_rng(3)
    Wc = su3(rng)
    W = [[(split_dw(Wc[a, b].real), split_dw(Wc[a, b].imag)) for b in range(3)] for a in range(3)]
    zero = (Fraction(0), Fraction(0))
    got = grid_matvec(W, [(zero, zero)] * 3)
    assert all(v == Fraction(0) for r in got for part in r for v in part)


def grid_outer(v, c):
    """P_ba = sum_s v_sb conj(c_sa) for the two spins s of a force part, all
    nine entries on one grid: its bound is max|v.hi| times
    max_a max(|c_0a.re| + |c_1a.re|, |c_0a.im| + |c_1a.im|), raised by 2^-19.
    v, c: 2 x 3 of ((re.h, re.l), (im.h, im.l)).  Asserts the exact steps."""
    vm = max(abs(v[s][b][k][0]) for s in range(2) for b in range(3) for k in range(2))
    cm = max(max(rn32(abs(c[0][a][0][0]) + abs(c[1][a][0][0])), rn32(abs(c[0][a][1][0]) + abs(c[1][a][1][0])))
             for a in range(3))
    m = rn32(rn32(vm * cm) * rn32(Fraction(1) + Fraction(1, 2 ** 19)))
    sigma = 4 * pow2_floor(m) if m > 0 else Fraction(2) ** -125
    t0 = Fraction(3, 2) * sigma
    P = {}
    for a in range(3):
        for b in range(3):
            lanes = {}
            # A: multipliers Re c_sa (conj keeps it); B: multipliers -Im c_sa
            for which, start in ((0, (t0, t0)), (1, (-t0, t0))):
                res = []
                for lane in (0, 1):
                    T, acc = start[lane], Fraction(0)
                    for s in range(2):
                        mh, ml = c[s][a][which]
                        if which == 1:
                            mh, ml = -mh, -ml
                        wh, wl = v[s][b][lane]
                        Tn = rn32(mh * wh + T)
                        q = T - Tn
                        assert is_f32(q) and sigma <= abs(Tn) < 2 * sigma
                        d = rn32(mh * wh + q)
                        t = d if s == 0 else rn32(acc + d)
                        acc = rn32(ml * wh + rn32(mh * wl + t))
                        T = Tn
                    res.append((T, acc))
                lanes[which] = res
            (ATre, Acre), (ATim, Acim) = lanes[0]
            (BTre, Bcre), (BTim, Bcim) = lanes[1]
            hre, him = ATre - BTim, ATim + BTre
            assert is_f32(hre) and is_f32(him)
            P[b, a] = (hre + rn32(Acre - Bcim), him + rn32(Acim + Bcre))
    return P


@pytest.mark.parametrize("scale_exp", [-40, 0, 40])
def test_grid_outer_products_of_the_force(scale_exp):
    rng = np.random.default_rng(2000 + scale_exp)
    for _ in range(3):
        vc = (rng.normal(size=(2, 3)) + 1j * rng.normal(size=(2, 3))) * 2.0 ** scale_exp
        cc = rng.normal(size=(2, 3)) + 1j * rng.normal(size=(2, 3))
        v = [[(split_dw(vc[s, b].real), split_dw(vc[s, b].imag)) for b in range(3)] for s in range(2)]
        c = [[(split_dw(cc[s, a].real), split_dw(cc[s, a].imag)) for a in range(3)] for s in range(2)]
        P = grid_outer(v, c)
        num = den = Fraction(0)
        for a in range(3):
            for b in range(3):
                ere = eim = Fraction(0)
                for s in range(2):
                    vr, vi = v[s][b][0][0] + v[s][b][0][1], v[s][b][1][0] + v[s][b][1][1]
                    cr, ci = c[s][a][0][0] + c[s][a][0][1], c[s][a][1][0] + c[s][a][1][1]
                    ere += vr * cr + vi * ci  # v conj(c)
                    eim += vi * cr - vr * ci
                num += (P[b, a][0] - ere) ** 2 + (P[b, a][1] - eim) ** 2
                den += ere ** 2 + eim ** 2
        assert math.sqrt(float(num / den)) <= 3e-13
