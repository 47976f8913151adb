"""Write gauss_cdt.inc: the library's inversion table for the encryption error.

Discrete Gaussian on the integers, sigma = 3.2 (sigma^2 = 256/25), cut at
|e| <= 19: P(e = k) is proportional to exp(-k^2 / (2 sigma^2)) =
exp(-25 k^2 / 512).  A 64-bit draw u maps to e = -19 + #{ j : u >= T_j } with
T_j = floor(2^64 * P(e <= -19 + j)), j = 0..37.

Each exp(-x) is summed exactly as a rational Taylor series with a rigorous
remainder bound, so every T_j is an exact floor (the script checks that the
bound cannot move it).  Run from the repository root or anywhere:
    python paper_2305_18396_gb300/csrc/gen_gauss_cdt.py
"""
from fractions import Fraction
from pathlib import Path

BOUND = 19
TERMS = 160


def exp_neg(x):
    """exp(-x) for rational x >= 0 as (value, error bound)."""
    s = Fraction(0)
    term = Fraction(1)
    for n in range(TERMS):
        s += term
        term = term * (-x) / (n + 1)
    # alternating series with terms decreasing in magnitude from here on
    assert abs(term) * 2 < Fraction(1, 2**200)
    return s, abs(term)


def table():
    rho, err = [], Fraction(0)
    for k in range(-BOUND, BOUND + 1):
        v, e = exp_neg(Fraction(25 * k * k, 512))
        rho.append(v)
        err += e
    total = sum(rho)
    out, acc = [], Fraction(0)
    for j in range(2 * BOUND):
        acc += rho[j]
        lo = (acc - err) / (total + err) * 2**64
        hi = (acc + err) / (total - err) * 2**64
        fl = lo.numerator // lo.denominator
        assert fl == hi.numerator // hi.denominator, "error bound straddles an integer"
        out.append(fl)
    return out


def main():
    lines = ["// Generated by gen_gauss_cdt.py -- do not edit.",
             "// T_j = floor(2^64 * P(e <= -19 + j)), discrete Gaussian sigma = 3.2, |e| <= 19."]
    for j, t in enumerate(table()):
        lines.append(f"0x{t:016x}ull,  // e <= {-BOUND + j}")
    Path(__file__).with_name("gauss_cdt.inc").write_text("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
