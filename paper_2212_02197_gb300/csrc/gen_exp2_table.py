"""Writes mc_exp2_table.inc: the correctly rounded doubles 2^(j/2048), j = 0..2047,
and the constants of the table-driven exp in mc_device.cuh (2048/ln 2, and
ln 2/2048 split into a head of 21 significant bits and a tail), computed in
80-digit arithmetic.

    python paper_2212_02197_gb300/csrc/gen_exp2_table.py
"""
import os

import mpmath

mpmath.mp.dps = 80
M = 2048


def rounded(v) -> float:
    """The double nearest to the mpmath value v (mpf -> float rounds to nearest)."""
    return float(mpmath.mpf(v))


def head(v, bits: int) -> float:
    """v rounded to `bits` significant bits (exact as a double)."""
    m, e = mpmath.frexp(v)
    return float(mpmath.ldexp(mpmath.nint(mpmath.ldexp(m, bits)), e - bits))


def constants():
    ln2 = mpmath.log(2)
    inv_l = rounded(M / ln2)
    l_hi = head(ln2 / M, 21)
    l_lo = rounded(ln2 / M - mpmath.mpf(l_hi))
    return inv_l, l_hi, l_lo


def table():
    return [rounded(mpmath.power(2, mpmath.mpf(j) / M)) for j in range(M)]


def main():
    inv_l, l_hi, l_lo = constants()
    t = table()
    lines = ["// Generated by gen_exp2_table.py: 2^(j/2048), j = 0..2047, correctly rounded.",
             f"// inv_l = {inv_l.hex()}, l_hi = {l_hi.hex()}, l_lo = {l_lo.hex()}"]
    for i in range(0, M, 4):
        lines.append("    " + ", ".join(v.hex() for v in t[i:i + 4]) + ",")
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "mc_exp2_table.inc")
    with open(out, "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
