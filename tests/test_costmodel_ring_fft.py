"""Pin of the ring-FFT flop count that the folded angular map's roofline uses
(costmodel.ring_fft_flops).  A plain Python model replays the operation
sequence of the ring transforms -- the radix-2 decimation-in-time FFT of the
N/2 packed complex values with its special-cased butterflies, then the real
split (forward) or the Hermitian fold (inverse) -- counting every FP64
operation (an FMA as 2 flops).  The model must reproduce the plain cos/sin
sums it stands for (checked against numpy's FFT) and its count must equal the
closed form, so a change to either shows here."""
import numpy as np
import pytest

from paper_1804_09101_gb300 import costmodel


class Counter:
    def __init__(self):
        self.flops = 0

    def add(self, a, b):
        self.flops += 1
        return a + b

    def mul(self, a, b):
        self.flops += 1
        return a * b

    def fma(self, a, b, c):
        self.flops += 2
        return a * b + c


def _bitrev(j, bits):
    return int(format(j, "0%db" % bits)[::-1], 2) if bits else 0


def _fft(re, im, sign, c):
    """In-place radix-2 DIT FFT (input bit-reversed) with twiddle
    exp(sign 2 pi i j / (2 S)); trivial, +-i and (+-1 +- i)/sqrt 2 twiddles
    special-cased, a general butterfly as a + w b (two FMA chains) and
    2a - (a + w b)."""
    n = len(re)
    S = 1
    while S < n:
        for g in range(0, n, 2 * S):
            for j in range(S):
                a, b = g + j, g + j + S
                ar, ai, br, bi = re[a], im[a], re[b], im[b]
                if j == 0:
                    re[a], im[a], re[b], im[b] = c.add(ar, br), c.add(ai, bi), c.add(ar, -br), c.add(ai, -bi)
                elif 4 * j == 2 * S:
                    tr, ti = -sign * bi, sign * br
                    re[a], im[a], re[b], im[b] = c.add(ar, tr), c.add(ai, ti), c.add(ar, -tr), c.add(ai, -ti)
                elif 8 * j in (2 * S, 6 * S):
                    h = np.sqrt(0.5)
                    sr = 1 if 8 * j == 2 * S else -1
                    u, v = c.add(sr * br, -sign * bi), c.add(sr * bi, sign * br)
                    re[a], im[a] = c.fma(h, u, ar), c.fma(h, v, ai)
                    re[b], im[b] = c.fma(-h, u, ar), c.fma(-h, v, ai)
                else:
                    ang = sign * np.pi * j / S
                    wr, wi = np.cos(ang), np.sin(ang)
                    pr = c.fma(wr, br, c.fma(-wi, bi, ar))
                    pi = c.fma(wr, bi, c.fma(wi, br, ai))
                    re[a], im[a], re[b], im[b] = pr, pi, c.fma(2.0, ar, -pr), c.fma(2.0, ai, -pi)
        S *= 2


def _forward(x, c):
    N = len(x)
    n = N // 2
    bits = n.bit_length() - 1
    re, im = [0.0] * n, [0.0] * n
    for j in range(n):
        re[_bitrev(j, bits)], im[_bitrev(j, bits)] = x[2 * j], x[2 * j + 1]
    _fft(re, im, -1, c)
    re[0], im[0] = c.add(re[0], im[0]), 0.0
    for k in range(1, n // 2):
        ar, ai, br, bi = re[k], im[k], re[n - k], im[n - k]
        er, ei, dr, di = c.add(ar, br), c.add(ai, -bi), c.add(ar, -br), c.add(ai, bi)
        hc, hs = 0.5 * np.cos(2 * np.pi * k / N), 0.5 * np.sin(2 * np.pi * k / N)
        tr, ti = c.fma(hc, di, c.mul(-hs, dr)), c.fma(hc, dr, c.mul(hs, di))
        re[k], im[k] = c.fma(0.5, er, tr), c.fma(-0.5, ei, ti)
        re[n - k], im[n - k] = c.fma(0.5, er, -tr), c.fma(0.5, ei, ti)
    return np.array(re), np.array(im)


def _inverse(cc, ss, c):
    n = len(cc)
    N = 2 * n
    bits = n.bit_length() - 1
    zr, zi = [0.0] * n, [0.0] * n
    zr[0], zi[0] = cc[0], cc[0]
    zr[n // 2], zi[n // 2] = cc[n // 2], ss[n // 2]
    for m in range(1, n // 2):
        sr, si = c.add(cc[m], cc[n - m]), c.add(ss[n - m], -ss[m])
        dr, di = c.add(cc[m], -cc[n - m]), c.add(-ss[m], -ss[n - m])
        hc, hs = 0.5 * np.cos(2 * np.pi * m / N), 0.5 * np.sin(2 * np.pi * m / N)
        tr, ti = c.fma(hc, dr, c.mul(-hs, di)), c.fma(hc, di, c.mul(hs, dr))
        zr[m], zi[m] = c.fma(0.5, sr, -ti), c.fma(0.5, si, tr)
        zr[n - m], zi[n - m] = c.fma(0.5, sr, ti), c.fma(-0.5, si, tr)
    re, im = [0.0] * n, [0.0] * n
    for m in range(n):
        re[_bitrev(m, bits)], im[_bitrev(m, bits)] = zr[m], zi[m]
    _fft(re, im, +1, c)
    x = np.empty(N)
    x[0::2], x[1::2] = re, im
    return x


@pytest.mark.parametrize("nph", costmodel.FOLD_FFT_NPHI)
def test_ring_fft_model_is_the_cos_sin_sums_and_its_count_is_the_closed_form(nph):
    rng = np.random.default_rng(nph)
    n = nph // 2
    x = rng.standard_normal(nph)
    c = Counter()
    cr, ci = _forward(x, c)
    X = np.fft.rfft(x)                   # X_m = c_m - i s_m
    assert np.abs(cr - X.real[:n]).max() < 1e-13 * np.abs(x).sum()
    assert np.abs(ci[1:] + X.imag[1:n]).max() < 1e-13 * np.abs(x).sum()
    assert c.flops == costmodel.ring_fft_flops(nph)

    cc, ss = rng.standard_normal(n), rng.standard_normal(n)
    ss[0] = 0.0
    k = np.arange(nph)
    ref = sum(cc[m] * np.cos(2 * np.pi * m * k / nph) + ss[m] * np.sin(2 * np.pi * m * k / nph) for m in range(n))
    c = Counter()
    y = _inverse(cc, ss, c)
    assert np.abs(y - ref).max() < 1e-12 * (np.abs(cc).sum() + np.abs(ss).sum())
    assert c.flops == costmodel.ring_fft_flops(nph, forward=False)


def test_ring_fft_count_at_64_points():
    # per 64-point ring: 835 flops forward, 834 backward (569 and 568 FP64
    # instructions, an FMA being one instruction)
    assert (costmodel.ring_fft_flops(64), costmodel.ring_fft_flops(64, forward=False)) == (835, 834)
