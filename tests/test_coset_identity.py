"""The identity behind the coset form of the polynomial product, checked in plain Python
integers (no library, no oracle): for a of degree < D and any b, a b mod (x^N + 1) equals the
result of
  1. the first log2 G stages of the negacyclic NTT of b (Cooley-Tukey, twiddles
     psi^{brev(2^s + g)}): the residues b_g = b mod (x^D - zeta_g), G = N / D blocks;
  2. the zero-padded length-2D negacyclic NTT of a and of each b_g (twiddles: the first 2D
     entries of the length-N table), slot-wise products;
  3. the inverse length-2D transform (linear product c_g = lo + x^D hi), folded to
     lo + zeta_g hi with zeta_g = psi^{brev(G/2 + g/2)} for even g and its negative for odd g;
  4. the inverse of step 1.
This is the polynomial product of Algorithm 1 step 3 (NTT-based per the footnote of Sec.
3.1.3); the GPU's coset kernels follow these steps and their outputs are compared with the
oracle's in the GPU parity tests.  Here the steps are restated from their definitions and
compared with the schoolbook negacyclic product for every D from 2 to N/2.
"""
import functools
import random

import pytest

Q = 1125625028935681  # one of the library's primes (c 2^37 + 1)


@functools.lru_cache(maxsize=None)
def _pow(base, e):
    return pow(base, e, Q)


def _brev(x, bits):
    return int(format(x, f"0{bits}b")[::-1], 2) if bits else 0


def _psi(N):
    for g in range(2, 1000):
        w = pow(g, (Q - 1) // (2 * N), Q)
        if pow(w, N, Q) == Q - 1:
            return w
    raise AssertionError("no 2N-th root")


def _schoolbook(a, b, N):
    c = [0] * N
    for i, x in enumerate(a):
        if x:
            for j, y in enumerate(b):
                if i + j < N:
                    c[i + j] = (c[i + j] + x * y) % Q
                else:
                    c[i + j - N] = (c[i + j - N] - x * y) % Q
    return c


def _ct_stages(x, psi, logN, stages, length):
    """Cooley-Tukey stages 0 .. stages - 1 of a negacyclic NTT of `length` values, twiddle of
    stage s, group g: psi^{brev_logN(2^s + g)}."""
    x = list(x)
    for s in range(stages):
        t = length >> (s + 1)
        for g in range(1 << s):
            w = _pow(psi, _brev((1 << s) + g, logN))
            for j in range(g * 2 * t, g * 2 * t + t):
                u, v = x[j], x[j + t] * w % Q
                x[j], x[j + t] = (u + v) % Q, (u - v) % Q
    return x


def _gs_stages(x, psi, logN, stages, length):
    """Inverse of _ct_stages (Gentleman-Sande, stages in reverse order, halving each)."""
    x = list(x)
    ipsi, inv2 = pow(psi, Q - 2, Q), (Q + 1) // 2
    for s in reversed(range(stages)):
        t = length >> (s + 1)
        for g in range(1 << s):
            w = _pow(ipsi, _brev((1 << s) + g, logN))
            for j in range(g * 2 * t, g * 2 * t + t):
                u, v = x[j], x[j + t]
                x[j], x[j + t] = (u + v) * inv2 % Q, (u - v) * w % Q * inv2 % Q
    return x


def _coset_product(a, b, N, D):
    logN, logD = N.bit_length() - 1, D.bit_length() - 1
    G, logG = N // D, logN - logD
    psi = _psi(N)
    heads = _ct_stages(b, psi, logN, logG, N)
    a_hat = _ct_stages(a[:D] + [0] * D, psi, logN, logD + 1, 2 * D)
    out = []
    for g in range(G):
        b_hat = _ct_stages(heads[g * D:(g + 1) * D] + [0] * D, psi, logN, logD + 1, 2 * D)
        c = _gs_stages([x * y % Q for x, y in zip(a_hat, b_hat)], psi, logN, logD + 1, 2 * D)
        zeta = pow(psi, _brev(G // 2 + g // 2, logN), Q)
        if g & 1:
            zeta = Q - zeta
        out += [(c[u] + zeta * c[u + D]) % Q for u in range(D)]
    return _gs_stages(out, psi, logN, logG, N)


@pytest.mark.parametrize("N", [16, 64])
def test_coset_product_equals_negacyclic_product(N):
    rng = random.Random(N)
    D = 2
    while D <= N // 2:
        for support in sorted({1, D // 2 or 1, D}):  # a's nonzero coefficients: the lowest `support`
            a = [rng.randrange(Q) for _ in range(support)] + [0] * (N - support)
            b = [rng.randrange(Q) for _ in range(N)]
            assert _coset_product(a, b, N, D) == _schoolbook(a, b, N), (N, D, support)
        D *= 2


def test_fold_sign_matters():
    """A plausible slip -- folding every coset with +psi^{brev(G/2 + g/2)} -- breaks it."""
    N, D = 32, 8
    rng = random.Random(7)
    a = [rng.randrange(Q) for _ in range(D)] + [0] * (N - D)
    b = [rng.randrange(Q) for _ in range(N)]
    good = _coset_product(a, b, N, D)
    logN, G, psi = N.bit_length() - 1, N // D, _psi(N)
    heads = _ct_stages(b, psi, logN, 2, N)
    a_hat = _ct_stages(a[:D] + [0] * D, psi, logN, 4, 2 * D)
    out = []
    for g in range(G):
        b_hat = _ct_stages(heads[g * D:(g + 1) * D] + [0] * D, psi, logN, 4, 2 * D)
        c = _gs_stages([x * y % Q for x, y in zip(a_hat, b_hat)], psi, logN, 4, 2 * D)
        zeta = pow(psi, _brev(G // 2 + g // 2, logN), Q)  # sign of odd g dropped
        out += [(c[u] + zeta * c[u + D]) % Q for u in range(D)]
    assert _gs_stages(out, psi, logN, 2, N) != good
