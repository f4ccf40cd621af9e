"""The kernels' tables of exact constants, re-derived in 300-bit arithmetic:
2^(j/64) (the exponential), and 1/F and ln F = hi + lo at F = 1 + j/128 with
ln 2 = hi + lo (the logarithm). Each entry must be the double nearest its
exact value; each hi part must be the multiple of 2^-43 nearest ln F (ln 2),
so that m ln2_hi + lnF_hi is exact."""
import math
import os
import re

import mpmath as mp

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "paper_2403_05910_b300", "csrc", "xf_device.cuh")
HEX = r"-?0x[0-9a-fA-F.]+p[+-]\d+"


def _table(name):
    src = open(SRC).read()
    body = re.search(name + r"\[\d+\] = \{(.*?)\};", src, re.S).group(1)
    return [float.fromhex(t) for t in re.findall(HEX, body)]


def _nearest(v, exact):
    return abs(mp.mpf(v) - exact) <= mp.mpf(math.ulp(v) if v else 0.0) / 2


def _hi(exact):
    return mp.mpf(int(mp.nint(exact * 2 ** 43))) / 2 ** 43


def test_exp_table_holds_the_nearest_doubles():
    mp.mp.prec = 300
    e = _table("kExp2J64")
    assert len(e) == 64
    assert all(_nearest(v, mp.power(2, mp.mpf(j) / 64)) for j, v in enumerate(e))


def test_log_tables_hold_the_nearest_doubles_and_exact_hi_parts():
    mp.mp.prec = 300
    inv, hi, lo = _table("kInvF128"), _table("kLnF128Hi"), _table("kLnF128Lo")
    assert len(inv) == len(hi) == len(lo) == 129
    for j in range(129):
        F = mp.mpf(1) + mp.mpf(j) / 128
        assert _nearest(inv[j], 1 / F), j
        assert mp.mpf(hi[j]) == _hi(mp.log(F)), j
        assert _nearest(lo[j], mp.log(F) - mp.mpf(hi[j])) or lo[j] == 0.0, j
    coef = open(SRC).read().split("#define XF_LOG_COEF")[1].split("constexpr")[0]
    l2hi, l2lo = [float.fromhex(t) for t in re.findall(HEX, coef)]
    assert mp.mpf(l2hi) == _hi(mp.log(2))
    assert _nearest(l2lo, mp.log(2) - mp.mpf(l2hi))
