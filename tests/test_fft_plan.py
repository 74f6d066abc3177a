"""The shared-memory FFT's formulation, checked on the CPU: a model of its passes
(bit-reversed input; each pass multiplies a group of 2^R elements by table twiddles
exp(2 pi i q0 rev_R(m) / (2^R h)) and then applies radix-2 stages with constant roots)
equals numpy's transform with the + sign, for the pass plans the kernels use; and the
padded layout's slot of element i0 + m h splits into a per-group base plus a per-m
constant, which the compile-time passes rely on; and the four-step pass 2's per-thread
index work (its unrolled tile copy and its output split into Z_l and Z_{N-l}) covers every
slot and every spectrum bin exactly once."""
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


# ---- four-step pass 2: the tile copy and the output split, modelled per thread

def _pass2_rows(n2, logn2, elem_bytes):
    """Rows per CTA as the host picks them: up to 4 within 96 KB of shared memory."""
    rows = 4
    while rows > 1 and elem_bytes * (n2 * 6 * rows + (n2 >> (logn2 - 5))) > 96 * 1024:
        rows >>= 1
    return rows


@pytest.mark.parametrize("rows", [1, 2, 4])
@pytest.mark.parametrize("logn2", [6, 7, 8, 9])
def test_pass2_copy_rounds_fill_every_slot_once(rows, logn2):
    """The unrolled copy rounds (col = cc * CPI + col0, CPI columns per round, the last
    round cut at Cn) put element j2 of every column into its bit-reversed padded slot
    exactly once, from row `l1` (side 0) or `N1 - l1` (side 1) of sequence `kind`, and
    zero-fill the columns of rows past N1 / 2."""
    n2, cn, sh = 1 << logn2, 6 * rows, logn2 - 5
    tpc = min(n2, THREADS)
    cpi, jpt = THREADS // tpc, n2 // tpc
    for logn1 in (logn2 - 1, logn2):
        n1 = 1 << logn1
        n = n1 * n2
        groups = (n1 // 2 + 1 + rows - 1) // rows
        for bx in sorted({0, 1, groups - 1}):
            r0 = bx * rows
            seen = {}
            for t in range(THREADS):
                col0 = 0 if cpi == 1 else t // tpc
                for cc in range((cn + cpi - 1) // cpi):
                    col = cc * cpi + col0
                    if cpi > 1 and col >= cn:
                        break
                    side, kind, r = col & 1, (col >> 1) % 3, col // 6
                    l1 = r0 + r
                    valid = l1 <= n1 // 2
                    row = ((n1 - l1) & (n1 - 1) if side else l1) if valid else 0
                    for u in range(jpt):
                        j = t % tpc + u * tpc
                        jr = _rev(j, logn2)
                        slot = jr * cn + (jr >> sh) + col
                        assert slot not in seen
                        seen[slot] = (kind * n + row * n2 + j, valid)
            want = {_rev(j, logn2) * cn + (_rev(j, logn2) >> sh) + col: (j, col)
                    for j in range(n2) for col in range(cn)}
            assert set(seen) == set(want)
            for slot, (j, col) in want.items():
                side, kind, r = col & 1, (col >> 1) % 3, col // 6
                l1 = r0 + r
                src, valid = seen[slot]
                assert valid == (l1 <= n1 // 2)
                if valid:
                    row = (n1 - l1) & (n1 - 1) if side else l1
                    assert src == kind * n + row * n2 + j


@pytest.mark.parametrize("logn", [13, 14, 15, 16, 17, 18])
@pytest.mark.parametrize("elem_bytes", [8, 16])
def test_pass2_writes_every_spectrum_bin_once_with_its_mirror(logn, elem_bytes):
    """Over all CTAs of a pixel pair, the output stage writes every l = 0 .. N/2 exactly
    once, as l = row + N1 l2 of the column it holds, and reads Z_{N-l} at row' + N1 l2m of
    the other side's column (row' = the mirror row), i.e. row' + N1 l2m = N - l mod N."""
    logn2 = (logn + 1) // 2
    logn1 = logn - logn2
    n1, n2, n = 1 << logn1, 1 << logn2, 1 << logn
    rows = _pass2_rows(n2, logn2, elem_bytes)
    groups = (n1 // 2 + 1 + rows - 1) // rows
    l2step = THREADS // (2 * rows)
    half = n // 2
    count = np.zeros(half + 1, np.int64)
    for bx in range(groups):
        r0 = bx * rows
        for t in range(THREADS):
            r, side = t % rows, (t // rows) & 1
            l1 = r0 + r
            if l1 > n1 // 2:
                continue
            l1p = (n1 - l1) & (n1 - 1)
            if side == 1 and l1p == l1:
                continue
            row = l1p if side else l1
            other = l1 if side else l1p
            for l2 in range(t // (2 * rows), n2, l2step):
                l = row + n1 * l2
                if l > half:
                    break
                l2m = (n2 - l2) & (n2 - 1) if row == 0 else n2 - 1 - l2
                assert (other + n1 * l2m) % n == (n - l) % n
                count[l] += 1
    assert (count == 1).all()
