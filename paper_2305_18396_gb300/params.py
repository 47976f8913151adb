"""Parameter sets of the BFV scheme (Sec. 2.2) used by this library.

Primes q_l = c * 2^37 + 1 below 2^50: NTT-friendly for N <= 2^14 (q_l = 1 mod
2N) and q_l = 1 mod t for t = 2^37, so round(q m / t) is within one of
m (q - 1) / t.  N = 4096 uses the first two (q ~ 2^100), N = 8192 the first
three (q ~ 2^150); both stay under the 128-bit-security ceilings of the HE
standard for ternary secrets (109 and 218 bits).
"""
DEFAULT_PRIMES = (1125625028935681, 1125487589982209, 1123426005680129)
LOG2T = 37


def default_L(N):
    return 2 if N <= 4096 else 3
