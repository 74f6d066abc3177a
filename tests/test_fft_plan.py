"""The shared-memory FFT's formulation, checked on the CPU: a model of its passes
(bit-reversed input; each pass multiplies a group of 2^R elements by table twiddles
exp(2 pi i q0 rev_R(m) / (2^R h)) and then applies radix-2 stages with constant roots)
equals numpy's transform with the + sign, for the pass plans the kernels use; and the
padded layout's slot of element i0 + m h splits into a per-group base plus a per-m
constant, which the compile-time passes rely on."""
import numpy as np
import pytest

THREADS = 256


def _rev(x, bits):
    return int(format(x, "0%db" % bits)[::-1], 2) if bits else 0


def _plan(cn, logl, threads=THREADS):
    """(R, s) of every pass: R the largest of 2..4 with (L >> R) * cn >= threads, the
    remaining stages first."""
    r = 4
    while r > 2 and ((1 << logl) >> r) * cn < threads:
        r -= 1
    r = min(r, logl)
    lead = logl % r if r else 0
    out, s = [], 1
    while s <= logl:
        rr = lead if (s == 1 and lead) else r
        out.append((rr, s))
        s += rr
    return out


def _fft_model(z, cn=1):
    n = len(z)
    logn = n.bit_length() - 1
    buf = np.empty(n, complex)
    for j in range(n):
        buf[_rev(j, logn)] = z[j]
    for r, s in _plan(cn, logn):
        g_n, h = 1 << r, 1 << (s - 1)
        for g in range(n >> r):
            q0 = g & (h - 1)
            i0 = ((g >> (s - 1)) << (s - 1 + r)) + q0
            x = buf[[i0 + m * h for m in range(g_n)]].copy()
            for m in range(1, g_n):
                x[m] *= np.exp(2j * np.pi * q0 * _rev(m, r) / (g_n * h))
            for st in range(r):
                half = 1 << st
                for m in range(g_n):
                    if m & half:
                        continue
                    v = x[m + half] * np.exp(2j * np.pi * (m & (half - 1)) / (2 * half))
                    x[m], x[m + half] = x[m] + v, x[m] - v
            buf[[i0 + m * h for m in range(g_n)]] = x
    return buf


@pytest.mark.parametrize("n", [2, 4, 8, 32, 64, 128, 256, 512])
@pytest.mark.parametrize("cn", [1, 6, 16, 24])
def test_pass_model_equals_the_dft(n, cn):
    rng = np.random.Generator(np.random.PCG64(n * 31 + cn))
    z = rng.normal(size=n) + 1j * rng.normal(size=n)
    ref = np.fft.ifft(z) * n   # sum_j z_j exp(+2 pi i j l / n)
    assert np.abs(_fft_model(z, cn) - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("cn", [6, 12, 16, 24])
@pytest.mark.parametrize("logl", [6, 7, 8, 9])
@pytest.mark.parametrize("pad", [False, True])
def test_padded_slot_splits_into_group_base_and_constant(cn, logl, pad):
    sh = (logl - 5 if logl > 5 else 0) if pad else 31
    for r, s in _plan(cn, logl):
        h = 1 << (s - 1)
        for t in range(((1 << logl) >> r) * cn):
            c, g = t % cn, t // cn
            q0 = g & (h - 1)
            i0 = ((g >> (s - 1)) << (s - 1 + r)) + q0
            base = i0 * cn + c + (i0 >> sh)
            for m in range(1 << r):
                j = i0 + m * h
                assert j * cn + (j >> sh) + c == base + m * h * cn + ((m * h) >> sh)


def test_padded_bit_reversed_stores_hit_distinct_banks():
    """32 consecutive inputs stored at their bit-reversed slots of the padded layout fall
    on 32 different 8-byte bank pairs modulo 16 (two per bank pair for 32 lanes), for the
    pass-2 column counts."""
    for cn in (6, 12, 24):
        for logl in (6, 7, 8, 9):
            sh = logl - 5
            for t0 in range(0, 1 << logl, 32):
                slots = [_rev(t, logl) * cn + (_rev(t, logl) >> sh) for t in range(t0, t0 + 32)]
                banks = [x % 16 for x in slots]
                assert max(banks.count(b) for b in set(banks)) == 2
