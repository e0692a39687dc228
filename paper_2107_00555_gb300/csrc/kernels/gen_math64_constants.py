"""Writes the constant block of k_math64.cuh (run by hand after a change;
tests/test_capi_cpu.py checks that the header holds exactly this output).

Every constant is a mathematical quantity rounded to the nearest double,
computed here in 200-bit arithmetic and rounded once through an exact
rational:

* 2^(j/64), j = 0..63: the table of Tang's exp (ACM TOMS 15(2), 1989).
* 64/ln 2, and ln2/64 split into two doubles; 2/pi, and pi/2 split into
  three (Cody and Waite, 1980): each part is the rounding of what the
  previous parts leave, so the parts sum to the constant to about 106 or
  159 bits.
* 1/n! for the Taylor series of e^r - 1, sin r and cos r.
"""
from fractions import Fraction
import math

import mpmath

mpmath.mp.prec = 200


def to_fraction(x) -> Fraction:
    """The exact value of an mpf (or a Fraction) as a Fraction."""
    if isinstance(x, Fraction):
        return x
    man, exp = mpmath.mpf(x).man_exp
    return Fraction(man) * (Fraction(2) ** exp if exp >= 0 else Fraction(1, 2 ** -exp))


def rn(x) -> float:
    """Nearest double to x (CPython rounds a Fraction correctly, ties to even)."""
    return float(to_fraction(x))


def split(x, parts: int):
    out, rest = [], to_fraction(x)
    for _ in range(parts):
        h = rn(rest)
        out.append(h)
        rest -= Fraction(h)
    return out


def constants():
    ln2 = mpmath.log(2)
    pi = mpmath.pi
    c = {}
    c["DCP_M64_EXP_TAB"] = [rn(mpmath.power(2, mpmath.mpf(j) / 64)) for j in range(64)]
    c["DCP_M64_INV_L"] = [rn(64 / ln2)]
    c["DCP_M64_L"] = split(ln2 / 64, 2)
    c["DCP_M64_TWO_OVER_PI"] = [rn(2 / pi)]
    c["DCP_M64_PIO2"] = split(pi / 2, 3)
    c["DCP_M64_EXPM1_TAYLOR"] = [rn(Fraction(1, math.factorial(n))) for n in range(2, 6)]
    c["DCP_M64_SIN_TAYLOR"] = [rn(Fraction((-1) ** k, math.factorial(2 * k + 1))) for k in range(1, 9)]
    c["DCP_M64_COS_TAYLOR"] = [rn(Fraction((-1) ** k, math.factorial(2 * k))) for k in range(1, 9)]
    return c


def block() -> str:
    lines = ["// BEGIN generated by gen_math64_constants.py"]
    for name, vals in constants().items():
        body = ", ".join(v.hex() for v in vals)
        lines.append(f"#define {name} {body}")
    lines.append("// END generated by gen_math64_constants.py")
    return "\n".join(lines) + "\n"


if __name__ == "__main__":
    print(block(), end="")
