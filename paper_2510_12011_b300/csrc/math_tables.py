"""Regenerates the constant tables of the table-driven FP64 exp and log in ionic_tp06.cuh:
2^(j/64) for j = 0..63 as hi + lo pairs, and for j = 0..127 the rounded reciprocal
c_j = fl(1/(1 + j/128)) with -ln(c_j) as a hi + lo pair.  Values from mpmath at 60 digits,
printed as C hex floating-point literals.

    python math_tables.py
"""
import mpmath


def pair(v):
    hi = float(v)
    return hi, float(v - mpmath.mpf(hi))


def main():
    mpmath.mp.dps = 60
    e_hi, e_lo = zip(*[pair(mpmath.mpf(2) ** (mpmath.mpf(j) / 64)) for j in range(64)])
    inv = [float(1 / (mpmath.mpf(1) + mpmath.mpf(j) / 128)) for j in range(128)]
    l_hi, l_lo = zip(*[pair(-mpmath.log(mpmath.mpf(c))) for c in inv])
    for name, vals in (("kExp2Hi", e_hi), ("kExp2Lo", e_lo), ("kLogInv", inv), ("kLogHi", l_hi),
                       ("kLogLo", l_lo)):
        print(f"{name} = {{")
        for i in range(0, len(vals), 3):
            print("    " + ", ".join(v.hex() for v in vals[i:i + 3]) + ",")
        print("};")


if __name__ == "__main__":
    main()
