"""The exact fixed-point sketch of the float-float basis, emulated on CPU in
IEEE float32 (numpy rounds every float32 operation to nearest, as the FP32
pipes do): a value v = hi + lo with |v| <= B is scaled by 2^(WB - E),
E = ilogb(1.0001 B) + 2, and split into three integer words by the
1.5 * 2^23 rounding trick with error-free two-sums between them.  The first
word is at most 2^(WB-1) in magnitude, the later ones (a rounding remainder
plus the low part carried along) below 1.2 * 2^(WB-1), which the word width
chosen for the bins leaves room for; the words reconstruct v to within
0.6 * 2^-2WB of the scaled unit (about 2^-61 of B at WB = 21), so integer
sums of words give the sketch to float64 accuracy, whatever the order of the
additions."""
import math

import numpy as np

F = np.float32
MAGIC = F(12582912.0)  # 1.5 * 2^23


def two_sum(a, b):
    s = F(a + b)
    bb = F(s - a)
    return s, F(F(a - F(s - bb)) + F(b - bb))


def fx_split(hi, lo, to_fixed, word, nw=3):
    h = F(hi * to_fixed)
    l = F(lo * to_fixed)
    q = []
    for w in range(nw):
        r = F(h + MAGIC)
        q.append(int(np.array(r, dtype=np.float32).view(np.int32)) - 0x4B400000)
        if w + 1 < nw:
            dh, dl = two_sum(F(h - F(r - MAGIC)), l)
            h, l = F(dh * word), F(dl * word)
    return q


def test_words_reconstruct_the_value_and_fit_their_bins():
    rng = np.random.default_rng(12)
    WB = 21
    word = F(2.0 ** WB)
    worst = 0.0
    for _ in range(4000):
        B = float(np.exp(rng.uniform(-40, 40)))
        v = rng.uniform(-1.0, 1.0) * B * rng.choice([1.0, 1e-3, 1e-9])
        hi = F(v)
        lo = F(v - float(hi))
        E = math.frexp(1.0001 * B)[1] + 1  # ilogb(x) + 2 with frexp's exponent = ilogb + 1
        to_fixed = F(2.0 ** (WB - E))
        q = fx_split(hi, lo, to_fixed, word)
        assert abs(q[0]) <= 2 ** (WB - 1) and all(abs(x) < 1.2 * 2 ** (WB - 1) for x in q[1:])
        scaled = (float(hi) + float(lo)) * 2.0 ** (WB - E)  # exact in float64 here
        rec = q[0] + q[1] * 2.0 ** -WB + q[2] * 2.0 ** (-2 * WB)
        worst = max(worst, abs(rec - scaled))
    assert worst < 0.6 * 2.0 ** (-2 * WB)


def test_word_sums_are_independent_of_the_order():
    """Integer sums of the words of many entries are exact, so any order of
    the atomics gives the same bin value; a float sum of the same values
    depends on the order."""
    rng = np.random.default_rng(13)
    WB, E = 21, 3
    to_fixed, word = F(2.0 ** (WB - E)), F(2.0 ** WB)
    vals = rng.uniform(-1.0, 1.0, 3000) * 3.9
    words = np.array([fx_split(F(v), F(v - float(F(v))), to_fixed, word) for v in vals], dtype=np.int64)
    sums = {tuple(words[rng.permutation(len(vals))].sum(axis=0)) for _ in range(5)}
    assert len(sums) == 1
    fsums = {float(np.sum(vals[rng.permutation(len(vals))].astype(np.float32))) for _ in range(20)}
    assert len(fsums) > 1
