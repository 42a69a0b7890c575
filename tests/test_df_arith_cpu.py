"""Error model of the double-float FFT arithmetic, on the CPU.

The residual updates run radix-8 decimation-in-frequency FFTs in double-float
arithmetic (pairs of FP32 numbers).  The update kernel uses unnormalised
additions and fused complex products; the exact residuals keep normalised
additions and products.  This file restates both arithmetics in numpy float32
(an FMA as the float64 product, exact for FP32 operands, plus the addend,
rounded once to FP32), runs the same pass structure (radix-8 passes from the
largest stride down, then one radix-2 or radix-4 pass, digit-reversed
spectrum, inverse as the adjoint) on a circular convolution of length P, and
checks the normwise errors against an FP64 FFT: both stay at a few u^2 log P
(u = 2^-24), and the cheaper arithmetic costs at most 1.6 times the error of
the normalised one.  It checks the error analysis, not the kernels; the
kernels are compared with each other in tests/test_sylv_gpu.py."""
import numpy as np
import pytest

f32 = np.float32
f64 = np.float64
U = 2.0 ** -24


def _fma(a, b, c):
    return (a.astype(f64) * b.astype(f64) + c.astype(f64)).astype(f32)


def _two_sum(a, b):
    s = a + b
    bb = s - a
    return s, (a - (s - bb)) + (b - bb)


def _fast_two_sum(a, b):
    s = a + b
    return s, b - (s - a)


def _neg(x):
    return (-x[0], -x[1])


class Normalised:
    """a complex value is (re.hi, re.lo, im.hi, im.lo)"""

    @staticmethod
    def add_r(x, y):
        s, e = _two_sum(x[0], y[0])
        return _fast_two_sum(s, e + (x[1] + y[1]))

    @staticmethod
    def mul_r(x, y):
        p = x[0] * y[0]
        e = _fma(x[0], y[0], -p)
        e = _fma(x[0], y[1], e)
        e = _fma(x[1], y[0], e)
        return _fast_two_sum(p, e)

    @classmethod
    def add(cls, a, b):
        return cls.add_r(a[0:2], b[0:2]) + cls.add_r(a[2:4], b[2:4])

    @classmethod
    def sub(cls, a, b):
        return cls.add_r(a[0:2], _neg(b[0:2])) + cls.add_r(a[2:4], _neg(b[2:4]))

    @classmethod
    def mul(cls, a, b):
        ar, ai, br, bi = a[0:2], a[2:4], b[0:2], b[2:4]
        re = cls.add_r(cls.mul_r(ar, br), _neg(cls.mul_r(ai, bi)))
        im = cls.add_r(cls.mul_r(ar, bi), cls.mul_r(ai, br))
        return re + im


class Fast(Normalised):
    @staticmethod
    def add_r(x, y):
        s, e = _two_sum(x[0], y[0])
        return s, e + (x[1] + y[1])

    @classmethod
    def mul(cls, a, b):
        arh, arl, aih, ail = a
        brh, brl, bih, bil = b
        p1, p2 = arh * brh, aih * bih
        e = _fma(arh, brh, -p1) - _fma(aih, bih, -p2)
        for x, y in ((arh, brl), (arl, brh), (-aih, bil), (-ail, bih)):
            e = _fma(x, y, e)
        s, t = _two_sum(p1, -p2)
        re = _fast_two_sum(s, t + e)
        q1, q2 = arh * bih, aih * brh
        f = _fma(arh, bih, -q1) + _fma(aih, brh, -q2)
        for x, y in ((arh, bil), (arl, bih), (aih, brl), (ail, brh)):
            f = _fma(x, y, f)
        s, t = _two_sum(q1, q2)
        im = _fast_two_sum(s, t + f)
        return re + im


_RS2 = 0.70710678118654752440
_RS2H = f32(_RS2)
_RS2L = f32(_RS2 - f64(_RS2H))


def _times_rsqrt2(x):
    p = x[0] * _RS2H
    e = _fma(x[0], np.full_like(x[0], _RS2H), -p)
    e = _fma(x[0], np.full_like(x[0], _RS2L), e)
    e = _fma(x[1], np.full_like(x[1], _RS2H), e)
    return _fast_two_sum(p, e)


def _mul_mi(a):
    return (a[2], a[3], -a[0], -a[1])


def _mul_w1(Ar, a):  # a e^{-i pi/4}
    re, im = a[0:2], a[2:4]
    return _times_rsqrt2(Ar.add_r(re, im)) + _times_rsqrt2(Ar.add_r(im, _neg(re)))


def _mul_w3(Ar, a):  # a e^{-3 i pi/4}
    re, im = a[0:2], a[2:4]
    return _times_rsqrt2(Ar.add_r(im, _neg(re))) + _neg(_times_rsqrt2(Ar.add_r(re, im)))


def _dft4(Ar, a0, a1, a2, a3):
    t0, t1 = Ar.add(a0, a2), Ar.sub(a0, a2)
    t2, t3 = Ar.add(a1, a3), _mul_mi(Ar.sub(a1, a3))
    return Ar.add(t0, t2), Ar.add(t1, t3), Ar.sub(t0, t2), Ar.sub(t1, t3)


def _dft8(Ar, v):
    e = _dft4(Ar, v[0], v[2], v[4], v[6])
    o = list(_dft4(Ar, v[1], v[3], v[5], v[7]))
    o[1], o[2], o[3] = _mul_w1(Ar, o[1]), _mul_mi(o[2]), _mul_w3(Ar, o[3])
    return [Ar.add(e[k], o[k]) for k in range(4)] + [Ar.sub(e[k], o[k]) for k in range(4)]


_REV3 = [0, 4, 2, 6, 1, 5, 3, 7]


def _split(z):
    rh = z.real.astype(f32)
    ih = z.imag.astype(f32)
    return [rh, (z.real - rh.astype(f64)).astype(f32), ih, (z.imag - ih.astype(f64)).astype(f32)]


def _join(c):
    return (c[0].astype(f64) + c[1].astype(f64)) + 1j * (c[2].astype(f64) + c[3].astype(f64))


def _take(c, idx):
    return tuple(x[idx] for x in c)


def _put(c, idx, v):
    for x, y in zip(c, v):
        x[idx] = y


def _conj(c):
    return (c[0], c[1], -c[2], -c[3])


def _forward(Ar, buf, logP, tw):
    """radix-8 DIF passes, then radix 2 or 4 at stride 1; digit-reversed output"""
    P, q = 1 << logP, logP // 3
    r = logP - 3 * q
    b = np.arange(P >> 3)
    ls = logP - 3
    for _ in range(q):
        j = b & ((1 << ls) - 1)
        base = ((b >> ls) << (ls + 3)) + j
        v = _dft8(Ar, [_take(buf, base + (m << ls)) for m in range(8)])
        tstep = j << (logP - ls - 3)
        _put(buf, base, v[0])
        for k in range(1, 8):
            _put(buf, base + (_REV3[k] << ls), Ar.mul(v[k], _take(tw, k * tstep)))
        ls -= 3
    if r == 1:
        i = 2 * np.arange(P >> 1)
        a, c = _take(buf, i), _take(buf, i + 1)
        _put(buf, i, Ar.add(a, c))
        _put(buf, i + 1, Ar.sub(a, c))
    elif r == 2:
        i = 4 * np.arange(P >> 2)
        a = _dft4(Ar, *(_take(buf, i + t) for t in range(4)))
        for slot, k in zip(range(4), (0, 2, 1, 3)):
            _put(buf, i + slot, a[k])


def _inverse(Ar, buf, logP, tw):
    """the adjoint of _forward without the 1/P factor; natural-order output"""
    P, q = 1 << logP, logP // 3
    r = logP - 3 * q
    if r == 1:
        i = 2 * np.arange(P >> 1)
        a, c = _take(buf, i), _take(buf, i + 1)
        _put(buf, i, Ar.add(a, c))
        _put(buf, i + 1, Ar.sub(a, c))
    elif r == 2:
        i = 4 * np.arange(P >> 2)
        a0, a2, a1, a3 = (_conj(_take(buf, i + t)) for t in range(4))
        out = _dft4(Ar, a0, a1, a2, a3)
        for t in range(4):
            _put(buf, i + t, _conj(out[t]))
    b = np.arange(P >> 3)
    ls = r
    for _ in range(q):
        j = b & ((1 << ls) - 1)
        base = ((b >> ls) << (ls + 3)) + j
        tstep = j << (logP - ls - 3)
        v = [_conj(_take(buf, base))]
        v += [Ar.mul(_conj(_take(buf, base + (_REV3[k] << ls))), _take(tw, k * tstep)) for k in range(1, 8)]
        v = _dft8(Ar, v)
        for m in range(8):
            _put(buf, base + (m << ls), _conj(v[m]))
        ls += 3


def _forward_f64(x, logP):
    """the same pass structure in complex128 (the spectrum's slot order)"""
    P, q = 1 << logP, logP // 3
    r = logP - 3 * q
    buf = x.astype(np.complex128).copy()
    w8 = np.exp(-2j * np.pi * np.outer(np.arange(8), np.arange(8)) / 8)
    w4 = np.exp(-2j * np.pi * np.outer(np.arange(4), np.arange(4)) / 4)
    tw = np.exp(-2j * np.pi * np.arange(P) / P)
    b = np.arange(P >> 3)
    ls = logP - 3
    for _ in range(q):
        j = b & ((1 << ls) - 1)
        base = ((b >> ls) << (ls + 3)) + j
        V = w8 @ np.stack([buf[base + (m << ls)] for m in range(8)])
        tstep = j << (logP - ls - 3)
        buf[base] = V[0]
        for k in range(1, 8):
            buf[base + (_REV3[k] << ls)] = V[k] * tw[k * tstep]
        ls -= 3
    if r == 1:
        i = 2 * np.arange(P >> 1)
        a, c = buf[i].copy(), buf[i + 1].copy()
        buf[i], buf[i + 1] = a + c, a - c
    elif r == 2:
        i = 4 * np.arange(P >> 2)
        A = w4 @ np.stack([buf[i + t] for t in range(4)])
        for slot, k in zip(range(4), (0, 2, 1, 3)):
            buf[i + slot] = A[k]
    return buf


def _convolution_error(Ar, logP, seed):
    P = 1 << logP
    N = P // 2
    rng = np.random.default_rng(seed)
    x = np.zeros(P, np.complex128)
    x[:N] = rng.standard_normal(N).astype(f32) + 1j * rng.standard_normal(N).astype(f32)
    g = np.zeros(P)
    g[:N + 1] = rng.standard_normal(N + 1) / np.arange(1, N + 2) ** 1.5
    tw = _split(np.exp(-2j * np.pi * np.arange(P) / P))
    ghat = _split(_forward_f64(g.astype(np.complex128), logP))
    buf = _split(x)
    _forward(Ar, buf, logP, tw)
    buf = list(Ar.mul(tuple(buf), tuple(ghat)))
    _inverse(Ar, buf, logP, tw)
    ref = np.fft.ifft(np.fft.fft(x) * np.fft.fft(g)) * P
    return np.linalg.norm(_join(buf) - ref) / np.linalg.norm(ref)


def test_slot_order_model_is_an_fft():
    # the FP64 model of the pass structure is the DFT with its outputs permuted:
    # an impulse at n = 1 has the distinct spectrum e^{-2 pi i k / P}, which names
    # the frequency k held by each slot; a random vector then matches np.fft there
    for logP in (11, 12, 13):
        P = 1 << logP
        e1 = np.zeros(P, np.complex128)
        e1[1] = 1.0
        k = np.rint(-np.angle(_forward_f64(e1, logP)) * P / (2 * np.pi)).astype(int) % P
        assert np.array_equal(np.sort(k), np.arange(P))
        x = np.random.default_rng(logP).standard_normal(P) + 1j * np.random.default_rng(P).standard_normal(P)
        ref = np.fft.fft(x)
        assert np.abs(_forward_f64(x, logP) - ref[k]).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("logP", [11, 13])
def test_fast_double_float_fft_error(logP):
    for seed in (1, 2):
        e_norm = _convolution_error(Normalised, logP, seed)
        e_fast = _convolution_error(Fast, logP, seed)
        assert e_norm <= 4 * U * U * logP * 8, e_norm
        assert e_fast <= 4 * U * U * logP * 8, e_fast
        assert e_fast <= 1.6 * e_norm, (e_fast, e_norm)
        # and far from FP32: the cheaper arithmetic keeps double-float accuracy
        assert e_fast <= 1e-13
