"""The table and constants of the device's table-driven exp (mc_device.cuh,
mc_exp2_table.inc), against 80-digit arithmetic: every entry is the correctly
rounded 2^(j/2048), the head of ln 2/2048 has at most 21 significant bits (so
that n times it is exact for |n| < 2^32), head plus tail is ln 2/2048 to within
half an ulp of the tail, and the kernel uses the generator's constants."""
import os
import re

import pytest

mpmath = pytest.importorskip("mpmath")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2212_02197_gb300", "csrc")


def _floats(text):
    return [float.fromhex(t) for t in re.findall(r"-?0x[0-9a-f.]+p[+-]\d+", text)]


def test_table_entries_are_correctly_rounded():
    mpmath.mp.dps = 80
    body = open(os.path.join(CSRC, "mc_exp2_table.inc")).read()
    rows = [ln for ln in body.splitlines() if not ln.startswith("//")]
    vals = _floats("\n".join(rows))
    assert len(vals) == 2048
    for j, v in enumerate(vals):
        exact = mpmath.power(2, mpmath.mpf(j) / 2048)
        err = abs(mpmath.mpf(v) - exact)
        half_ulp = mpmath.mpf(2) ** (-53)  # 1 <= 2^(j/2048) < 2: an ulp is 2^-52
        assert err <= half_ulp, j


def test_constants_split_and_match_the_kernel():
    mpmath.mp.dps = 80
    src = open(os.path.join(CSRC, "mc_device.cuh")).read()
    fn = src[src.index("double exp_table(double x)"):]
    fn = fn[:fn.index("\n}\n")]
    inv_l = float.fromhex(re.search(r"inv_l = (0x[0-9a-fp.+-]+);", fn).group(1))
    l_hi = float.fromhex(re.search(r"l_hi = (0x[0-9a-fp.+-]+);", fn).group(1))
    l_lo = float.fromhex(re.search(r"l_lo = (-?0x[0-9a-fp.+-]+);", fn).group(1))
    L = mpmath.log(2) / 2048
    assert abs(mpmath.mpf(inv_l) - 1 / L) <= mpmath.mpf(2) ** (11 - 53)   # half an ulp of 2954.6
    m, e = mpmath.frexp(mpmath.mpf(l_hi))
    assert mpmath.ldexp(m, 21) == mpmath.nint(mpmath.ldexp(m, 21))       # 21 significant bits
    # the tail is ln2/2048 - head rounded to nearest: within half its own ulp
    _, e_lo = mpmath.frexp(mpmath.mpf(l_lo))
    assert abs(mpmath.mpf(l_hi) + mpmath.mpf(l_lo) - L) <= mpmath.mpf(2) ** (e_lo - 54)
    hdr = open(os.path.join(CSRC, "mc_exp2_table.inc")).readline() + \
        open(os.path.join(CSRC, "mc_exp2_table.inc")).readlines()[1]
    assert [inv_l, l_hi, l_lo] == _floats(hdr)
