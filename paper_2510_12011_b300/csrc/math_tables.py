"""Regenerates the constants of the table-driven FP64 exp and log in ionic_tp06.cuh:
2^(j/256) for j = 0..255 as hi + lo pairs; the cubic coefficient of the exp's polynomial; and
for j = 0..127 the rounded reciprocal c_j = fl(1/(1 + j/128)) with -ln(c_j) as a hi + lo pair.
Values from mpmath at 60 digits, printed as C hex floating-point literals.

The exp's polynomial is r + r^2/2 + c3 r^3 + r^4/24 on |r| <= a = ln2/512.  Its error is
dominated by r^5/120; c3 = 1/6 + k a^2/120 takes the best multiple of r^3 off that term, where
k solves the equioscillation condition of r^3 (r^2 - k a^2) on [0, a]: the value 1 - k at r = a
equals minus the interior extremum at r^2 = 3 k a^2 / 5, that is 1 - k = (2k/5)(3k/5)^(3/2).
That leaves a maximum error of 5.0e-18 (0.022 ulp of 1) against 3.8e-17 for the Taylor cubic.

    python math_tables.py
"""
import mpmath


def pair(v):
    hi = float(v)
    return hi, float(v - mpmath.mpf(hi))


def exp_cubic():
    k = mpmath.findroot(lambda k: 1 - k - (2 * k / 5) * (3 * k / 5) ** mpmath.mpf(1.5), 0.87)
    a = mpmath.log(2) / 512
    return float(mpmath.mpf(1) / 6 + k * a * a / 120)


def main():
    mpmath.mp.dps = 60
    e_hi, e_lo = zip(*[pair(mpmath.mpf(2) ** (mpmath.mpf(j) / 256)) for j in range(256)])
    inv = [float(1 / (mpmath.mpf(1) + mpmath.mpf(j) / 128)) for j in range(128)]
    l_hi, l_lo = zip(*[pair(-mpmath.log(mpmath.mpf(c))) for c in inv])
    print(f"kExpC3 = {exp_cubic().hex()};")
    for name, vals in (("kExp2Hi", e_hi), ("kExp2Lo", e_lo), ("kLogInv", inv), ("kLogHi", l_hi),
                       ("kLogLo", l_lo)):
        print(f"{name} = {{")
        for i in range(0, len(vals), 3):
            print("    " + ", ".join(v.hex() for v in vals[i:i + 3]) + ",")
        print("};")


if __name__ == "__main__":
    main()
