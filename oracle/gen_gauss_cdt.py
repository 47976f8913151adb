"""Write oracle/gauss_cdt.h: the oracle's inversion table for the encryption error.

The error of a fresh BFV ciphertext (Sec. 2.2) follows a discrete Gaussian on
the integers with sigma = 3.2, cut at |e| <= 19 (= floor(6 sigma)):

    P(e = k) = rho(k) / S,   rho(k) = exp(-k^2 / (2 sigma^2)),   S = sum_{|k|<=19} rho(k).

A 64-bit uniform draw u is mapped to e = -19 + #{ j : u >= T_j } with

    T_j = floor( 2^64 * sum_{k=-19}^{-19+j} P(e = k) ),   j = 0 .. 37.

The thresholds are evaluated with Python's `decimal` at 80 significant digits,
far more than the 20 digits that a 64-bit floor needs; the script refuses to
write a threshold whose 2^64-scaled value lies within 1e-40 of an integer.

Test infrastructure: run `python oracle/gen_gauss_cdt.py` to regenerate.
"""
from decimal import Decimal, getcontext
from pathlib import Path

SIGMA = Decimal("3.2")
BOUND = 19


def thresholds():
    getcontext().prec = 80
    two_sigma_sq = 2 * SIGMA * SIGMA
    rho = [(-(Decimal(k) * Decimal(k)) / two_sigma_sq).exp() for k in range(-BOUND, BOUND + 1)]
    total = sum(rho)
    scale = Decimal(2) ** 64
    out = []
    acc = Decimal(0)
    for j in range(2 * BOUND):
        acc += rho[j]
        v = acc / total * scale
        fl = int(v)  # v > 0, so int() is the floor
        frac = v - fl
        if frac < Decimal("1e-40") or frac > 1 - Decimal("1e-40"):
            raise ValueError(f"threshold {j} too close to an integer to floor reliably")
        out.append(fl)
    return out


def main():
    ts = thresholds()
    lines = [
        "/* Generated by oracle/gen_gauss_cdt.py -- do not edit.",
        " * Inversion table of the discrete Gaussian (sigma = 3.2, |e| <= 19):",
        " * T_j = floor(2^64 * P(e <= -19 + j)), j = 0..37. */",
        "#ifndef HE_ORACLE_GAUSS_CDT_H",
        "#define HE_ORACLE_GAUSS_CDT_H",
        f"#define OR_GAUSS_BOUND {BOUND}u",
        "static const unsigned long long OR_GAUSS_CDT[2 * OR_GAUSS_BOUND] = {",
    ]
    for j, t in enumerate(ts):
        lines.append(f"    0x{t:016x}ull, /* e <= {-BOUND + j} */")
    lines += ["};", "#endif", ""]
    Path(__file__).with_name("gauss_cdt.h").write_text("\n".join(lines))


if __name__ == "__main__":
    main()
