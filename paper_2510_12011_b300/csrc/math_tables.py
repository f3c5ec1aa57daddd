"""Regenerates the constants of the table-driven FP64 exp and log of the ionic kernels:
2^(j/2048) for j = 0..2047 as hi + lo pairs (the include file exp2_table.inc), the quadratic
coefficient of the exp's polynomial (kExpC2 in ionic_tp06.cuh), and for j = 0..127 the rounded
reciprocal c_j = fl(1/(1 + j/128)) with -ln(c_j) as a hi + lo pair (ionic_tp06.cuh).  Values
from mpmath at 60 digits, printed as C hex floating-point literals.

The exp's polynomial is r + c2 r^2 + r^3/6 on |r| <= a = ln2/4096.  Its error is dominated by
r^4/24; c2 = 1/2 + d takes the best multiple of r^2 off that term: r^4/24 - d r^2 on [0, a]
equioscillates (its value at r = a equals minus its interior extremum -6 d^2 at r^2 = 12 d) for
d = (sqrt(2) - 1) a^2 / 12.  That leaves a maximum error of 5.9e-18 against 3.4e-17 for 1/2.

The base-2 form used by the ionic kernel evaluates 2^r - 1 on |r| <= 2^-12 as
r (a1 + r (a2 + r a3)) with a1 = ln 2, a2 = c2 (ln 2)^2, a3 = (ln 2)^3 / 6: the same polynomial in
s = r ln 2 (maximum error 5.9e-18).

    python math_tables.py           print every table
    python math_tables.py --write   rewrite exp2_table.inc beside this file
"""
import os
import sys

import mpmath


def pair(v):
    hi = float(v)
    return hi, float(v - mpmath.mpf(hi))


def exp_quadratic():
    a = mpmath.log(2) / 4096
    return float(mpmath.mpf(1) / 2 + (mpmath.sqrt(2) - 1) * a * a / 12)


def exp2_coefficients():
    ln2 = mpmath.log(2)
    a = ln2 / 4096
    c2 = mpmath.mpf(1) / 2 + (mpmath.sqrt(2) - 1) * a * a / 12
    return float(ln2), float(c2 * ln2 ** 2), float(ln2 ** 3 / 6)


def exp_tables():
    return zip(*[pair(mpmath.mpf(2) ** (mpmath.mpf(j) / 2048)) for j in range(2048)])


def body(vals):
    return "\n".join("    " + ", ".join(v.hex() for v in vals[i:i + 3]) + "," for i in range(0, len(vals), 3))


def include_file():
    e_hi, e_lo = exp_tables()
    return ("// 2^(j/2048) = kExp2Hi[j] + kExp2Lo[j], j = 0..2047, each computed to 60 digits and split\n"
            "// into the nearest double and the rest; written by math_tables.py --write.\n"
            f"static __device__ const double kExp2Hi[2048] = {{\n{body(e_hi)}\n}};\n"
            f"static __device__ const double kExp2Lo[2048] = {{\n{body(e_lo)}\n}};\n")


def main():
    mpmath.mp.dps = 60
    if "--write" in sys.argv:
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "exp2_table.inc")
        with open(path, "w") as f:
            f.write(include_file())
        return
    e_hi, e_lo = exp_tables()
    inv = [float(1 / (mpmath.mpf(1) + mpmath.mpf(j) / 128)) for j in range(128)]
    l_hi, l_lo = zip(*[pair(-mpmath.log(mpmath.mpf(c))) for c in inv])
    print(f"kExpC2 = {exp_quadratic().hex()};")
    a1, a2, a3 = exp2_coefficients()
    print(f"kExp2A1 = {a1.hex()}, kExp2A2 = {a2.hex()}, kExp2A3 = {a3.hex()};")
    for name, vals in (("kExp2Hi", e_hi), ("kExp2Lo", e_lo), ("kLogInv", inv), ("kLogHi", l_hi),
                       ("kLogLo", l_lo)):
        print(f"{name} = {{\n{body(vals)}\n}};")


if __name__ == "__main__":
    main()
