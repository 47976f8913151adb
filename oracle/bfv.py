"""Protocol layer of the oracle: Algorithm 1 with the block split, on RNS-BFV.

Test infrastructure only.  Roles follow the footnote of Sec. 3.1.1
("Attention"): the client holds X (m x k) and the server holds W (k x n); in
Algorithm 1's notation the server's A = W^T (n x k) and the client's
B = X^T (k x m), so C = A B = (X W)^T and both parties transpose at decode.

Block split (Sec. 3.1.1 says only that larger matrices are split into
blocks): blocking (m_b, k_b, n_b) plays the role of Algorithm 1's (n, r, m)
with m_b * k_b * n_b <= N; block counts nI = ceil(n/n_b), nJ = ceil(k/k_b),
nLb = ceil(m/m_b); ragged edges are zero.  Block (I, J) of A is encoded with
pi_A, block (J, Lb) of B with pi_B, and output ciphertext (Lb, I) is
sum_J a_{I,J} * [[b_{Lb,J}]].

Layouts (all uint64, C order):
  input ciphertexts   [nLb * nJ][2][L][N]   index Lb * nJ + J, coefficient form
  output ciphertexts  [nLb * nI][2][L][N]   index Lb * nI + I, coefficient form
  shares              [m][n]                 values in Z_t
"""
import ctypes
import math

import numpy as np

from .core import lib, p32, p64, pi64

# Three ~50-bit primes q = c * 2^37 + 1 (so q = 1 mod 2N for N <= 2^14 and q = 1 mod t).
DEFAULT_PRIMES = (1125625028935681, 1125487589982209, 1123426005680129)
LOG2T = 37


class Params:
    """BFV parameters {N, t, q} of Sec. 2.2 with q = q_0 * ... * q_{L-1} (RNS)."""

    def __init__(self, N=4096, L=2, primes=None, log2t=LOG2T):
        primes = tuple(primes if primes is not None else DEFAULT_PRIMES[:L])
        if len(primes) != L:
            raise ValueError("need exactly L primes")
        if N < 2 or N & (N - 1):
            raise ValueError("N must be a power of two")
        self.N, self.L, self.log2t = N, L, log2t
        self.t = 1 << log2t
        self.q = primes
        for q in primes:
            if not lib.or_is_prime(q):
                raise ValueError(f"{q} is not prime")
            if (q - 1) % (2 * N):
                raise ValueError(f"{q} is not 1 mod 2N")
        self.psi = tuple(lib.or_primitive_2n_root(q, N) for q in primes)
        self.Q = math.prod(primes)
        self.q_arr = np.array(primes, dtype=np.uint64)
        self.psi_arr = np.array(self.psi, dtype=np.uint64)


def blocks(m, k, n, blk):
    m_b, k_b, n_b = blk
    return -(-n // n_b), -(-k // k_b), -(-m // m_b)


def check_blocking(N, blk):
    m_b, k_b, n_b = blk
    if min(blk) < 1 or m_b * k_b * n_b > N:
        raise ValueError("blocking needs m_b * k_b * n_b <= N")


# ---------------------------------------------------------------- encodings


def pack_input(X, blk, N):
    """pi_B of Algorithm 1 on B = X^T, per block (J, Lb):
    b_{J,Lb} = sum_{j<k_b, l<m_b} B[J k_b + j][Lb m_b + l] x^{l n_b k_b + j}.
    Returns [nLb * nJ][N] in Z_t."""
    check_blocking(N, blk)
    m_b, k_b, n_b = blk
    m, k = X.shape
    nJ, nLb = -(-k // k_b), -(-m // m_b)
    out = np.zeros((nLb, nJ, N), dtype=np.uint64)
    for Lb in range(nLb):
        for J in range(nJ):
            for l in range(min(m_b, m - Lb * m_b)):
                row = X[Lb * m_b + l, J * k_b : min(k, (J + 1) * k_b)]
                out[Lb, J, l * n_b * k_b : l * n_b * k_b + row.size] = row
    return out.reshape(nLb * nJ, N)


def encode_weights_coeff(W, blk, N):
    """pi_A of Algorithm 1 on A = W^T, per block (I, J):
    a_{I,J} = sum_{i<n_b, j<k_b} A[I n_b + i][J k_b + j] x^{i k_b + k_b - 1 - j}.
    Returns [nI][nJ][N] in Z_t."""
    check_blocking(N, blk)
    m_b, k_b, n_b = blk
    k, n = W.shape
    nI, nJ = -(-n // n_b), -(-k // k_b)
    out = np.zeros((nI, nJ, N), dtype=np.uint64)
    for I in range(nI):
        for J in range(nJ):
            for i in range(min(n_b, n - I * n_b)):
                for j in range(min(k_b, k - J * k_b)):
                    out[I, J, i * k_b + k_b - 1 - j] = W[J * k_b + j, I * n_b + i]
    return out


def decode_positions(m, n, blk):
    """pi_C^{-1} of Algorithm 1: C[i][l] sits at coefficient l n_b k_b + i k_b + k_b - 1
    of output (Lb, I).  Returns (ct index, coefficient) arrays of shape [m][n] for the
    (row, col) = (Lb m_b + l, I n_b + i) entry of X W."""
    m_b, k_b, n_b = blk
    nI = -(-n // n_b)
    rows = np.arange(m)[:, None]
    cols = np.arange(n)[None, :]
    Lb, l = rows // m_b, rows % m_b
    I, i = cols // n_b, cols % n_b
    ct = Lb * nI + I
    coef = l * n_b * k_b + i * k_b + k_b - 1
    return np.broadcast_to(ct, (m, n)), np.broadcast_to(coef, (m, n))


def unpack_output(dec, m, n, blk):
    """Client: its share of X W from the decrypted output polynomials [nLb*nI][N]."""
    ct, coef = decode_positions(m, n, blk)
    return dec[ct, coef].astype(np.uint64)


def centred_lift_residues(P, poly_t):
    """Lift Z_t coefficients to the centred range [-t/2, t/2) and reduce mod each q_l.
    poly_t [..., N] -> [..., L, N]."""
    v = poly_t.astype(object)
    half = P.t // 2
    out = np.empty(poly_t.shape[:-1] + (P.L, P.N), dtype=np.uint64)
    signed = np.where(poly_t >= half, v - P.t, v)
    for li, q in enumerate(P.q):
        out[..., li, :] = (signed % q).astype(np.uint64)
    return out


# ---------------------------------------------------------------- NTT helpers


def ntt_forward(P, a):
    """Negacyclic NTT of every polynomial of a[..., L, N] (copy)."""
    out = np.ascontiguousarray(a, dtype=np.uint64).copy()
    for li in range(P.L):
        part = np.ascontiguousarray(out[..., li, :])
        lib.or_ntt_forward(p64(part), P.N, P.q[li], P.psi[li], part.size // P.N)
        out[..., li, :] = part
    return out


def ntt_inverse(P, a):
    out = np.ascontiguousarray(a, dtype=np.uint64).copy()
    for li in range(P.L):
        part = np.ascontiguousarray(out[..., li, :])
        lib.or_ntt_inverse(p64(part), P.N, P.q[li], P.psi[li], part.size // P.N)
        out[..., li, :] = part
    return out


# ---------------------------------------------------------------- BFV test client


def keygen(P, seed):
    s = np.zeros(P.N, dtype=np.int64)
    lib.or_sample_ternary(seed, P.N, pi64(s))
    return s


def encrypt(P, s, plain, seed, obj0=0):
    """plain [cnt][N] in Z_t -> ciphertexts [cnt][2][L][N]; ciphertext j is object obj0 + j
    of the seed's random streams (so a slice of a larger batch can be encrypted alone)."""
    plain = np.ascontiguousarray(plain, dtype=np.uint64)
    cnt = plain.shape[0]
    ct = np.zeros((cnt, 2, P.L, P.N), dtype=np.uint64)
    s = np.ascontiguousarray(s, dtype=np.int64)
    lib.or_encrypt(P.N, P.L, p64(P.q_arr), p64(P.psi_arr), P.log2t, pi64(s), p64(plain), cnt, obj0, seed, p64(ct))
    return ct


def decrypt(P, s, ct):
    """Exact BFV decryption: m = round(t * [c0 + c1 s]_q / q) mod t, with the CRT and the
    rounding in Python big integers.  Returns (plain [cnt][N], noise budget bits [cnt]),
    the budget being floor(log2(q/2) - log2(max |t x - q round(t x / q)|))."""
    ct = np.ascontiguousarray(ct, dtype=np.uint64)
    cnt = ct.shape[0]
    x = np.zeros((cnt, P.L, P.N), dtype=np.uint64)
    lib.or_decrypt_residues(P.N, P.L, p64(P.q_arr), p64(P.psi_arr), pi64(np.ascontiguousarray(s)), p64(ct), cnt, p64(x))
    Q, t = P.Q, P.t
    crt = []
    for q in P.q:
        Mi = Q // q
        crt.append(Mi * pow(Mi, -1, q))
    plain = np.zeros((cnt, P.N), dtype=np.uint64)
    budget = np.zeros(cnt, dtype=np.int64)
    for j in range(cnt):
        cols = [list(map(int, x[j, li])) for li in range(P.L)]
        worst = 0
        row = []
        for i in range(P.N):
            xi = sum(c[i] * w for c, w in zip(cols, crt)) % Q
            r = (2 * t * xi + Q) // (2 * Q)
            w = abs(t * xi - Q * r)
            worst = max(worst, w)
            row.append(r % t)
        plain[j] = np.array(row, dtype=np.uint64)
        budget[j] = math.floor(math.log2(Q / 2) - math.log2(worst)) if worst else math.floor(math.log2(Q / 2))
    return plain, budget


def delta_residues(P, m):
    out = np.zeros(P.L, dtype=np.uint64)
    lib.or_delta_residues(p64(P.q_arr), P.L, P.log2t, int(m), p64(out))
    return out


# ---------------------------------------------------------------- server side


def mask_poly(P, seed, o):
    """The server's uniform share s of output ciphertext o (Algorithm 1, step 3)."""
    s = np.zeros(P.N, dtype=np.uint64)
    lib.or_sample_mask(seed, o, P.N, P.log2t, p64(s))
    return s


def matmul(P, ct_in, W, m, k, n, blk, mask_seed, sel=None):
    """Server evaluation of Algorithm 1 step 3 for output ciphertexts `sel`
    (default: all): [[c]] = sum_J a_{I,J} * [[b_{Lb,J}]], then c0 <- c0 - Delta(s).
    Returns [len(sel)][2][L][N] in coefficient form."""
    check_blocking(P.N, blk)
    nI, nJ, nLb = blocks(m, k, n, blk)
    sel = list(range(nLb * nI)) if sel is None else [int(o) for o in sel]
    I_list = sorted({o % nI for o in sel})
    Lb_list = sorted({o // nI for o in sel})
    I_pos = {I: p for p, I in enumerate(I_list)}
    Lb_pos = {Lb: p for p, Lb in enumerate(Lb_list)}
    if isinstance(ct_in, dict):  # only the input rows the selected outputs read: {Lb: [nJ][2][L][N]}
        cts = np.stack([np.ascontiguousarray(ct_in[Lb], dtype=np.uint64) for Lb in Lb_list])
        if cts.shape[1:] != (nJ, 2, P.L, P.N):
            raise ValueError(f"input rows must be {(nJ, 2, P.L, P.N)}, got {cts.shape[1:]}")
    else:
        ct_in = np.ascontiguousarray(ct_in, dtype=np.uint64)
        if ct_in.shape != (nLb * nJ, 2, P.L, P.N):
            raise ValueError(f"input ciphertexts must be {(nLb * nJ, 2, P.L, P.N)}, got {ct_in.shape}")
        cts = ct_in.reshape(nLb, nJ, 2, P.L, P.N)[Lb_list]

    # pi_A block I reads only columns I n_b .. I n_b + n_b - 1 of W: encode those alone
    n_b = blk[2]
    pt_t = np.concatenate([encode_weights_coeff(W[:, I * n_b:(I + 1) * n_b], blk, P.N) for I in I_list])
    pt_ntt = ntt_forward(P, centred_lift_residues(P, pt_t))          # [nI'][nJ][L][N]
    ct_ntt = ntt_forward(P, cts)                                     # [nLb'][nJ][2][L][N]

    sel_local = np.array([Lb_pos[o // nI] * len(I_list) + I_pos[o % nI] for o in sel], dtype=np.uint32)
    out = np.zeros((len(sel), 2, P.L, P.N), dtype=np.uint64)
    lib.or_ctpt_accumulate(P.N, P.L, p64(P.q_arr), p64(np.ascontiguousarray(pt_ntt)), p64(np.ascontiguousarray(ct_ntt)),
                           len(I_list), nJ, len(Lb_list), p32(sel_local), len(sel), p64(out))
    out = ntt_inverse(P, out)
    obj = np.array(sel, dtype=np.uint32)
    lib.or_apply_mask(P.N, P.L, p64(P.q_arr), P.log2t, mask_seed, p32(obj), len(sel), p64(out))
    return out


def unmask(P, mask_seed, m, n, blk):
    """Server: its share pi_C^{-1}(s) of X W, [m][n] in Z_t."""
    ct, coef = decode_positions(m, n, blk)
    cache = {}
    out = np.zeros((m, n), dtype=np.uint64)
    for o in np.unique(ct):
        cache[int(o)] = mask_poly(P, mask_seed, int(o))
    for r in range(m):
        for c in range(n):
            out[r, c] = cache[int(ct[r, c])][coef[r, c]]
    return out


def plain_matmul_mod_t(X, W, t):
    """Brute-force integer X W mod t (exact, Python integers)."""
    Xo = X.astype(object)
    Wo = W.astype(object)
    return (Xo.dot(Wo) % t).astype(np.uint64)


# ---------------------------------------------------------------- server-local share products


def share_matmul(X, W, bias=None, acc=None, log2t=37):
    """Sec. 3.1.1: the server's plaintext side of a linear layer, (acc + X W + bias) mod t,
    X [m][k], W [k][n], bias [n], acc [m][n] (each optional but X, W)."""
    X = np.ascontiguousarray(X, dtype=np.uint64)
    W = np.ascontiguousarray(W, dtype=np.uint64)
    m, k = X.shape
    k2, n = W.shape
    if k2 != k:
        raise ValueError("inner dimensions differ")
    out = np.zeros((m, n), dtype=np.uint64)
    b = None if bias is None else np.ascontiguousarray(bias, dtype=np.uint64).reshape(n)
    a = None if acc is None else np.ascontiguousarray(acc, dtype=np.uint64).reshape(m, n)
    null = ctypes.POINTER(ctypes.c_uint64)()
    lib.or_share_matmul(m, k, n, p64(X) if X.size else null, p64(W) if W.size else null,
                        null if b is None else p64(b), null if a is None else p64(a), log2t, p64(out))
    return out
