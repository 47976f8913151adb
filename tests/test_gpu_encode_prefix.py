"""The weight encoding's transform of sparse blocks, against the oracle, at every sparsity.

A weight block of Algorithm 1's encoding pi_A fills only its lowest n_b k_b coefficients,
so the first s0 butterfly stages of its forward transform (s0 the largest s with
n_b k_b <= N / 2^s) are copies: the encoder skips them, in registers when s0 equals the
first pass's stage count and otherwise by replicating the coefficients in shared memory,
running the stages up to the next pass boundary there and resuming the register passes.
The blockings below give every s0 from 0 to log2 N (m_b = 2^s0, with k_b n_b = N / 2^s0,
and a few with n_b k_b not a power of two), for every built transform radix; each
product's output ciphertexts (encoding, forward transforms, multiply-accumulate, inverse
transforms) must equal the oracle's.
"""
import numpy as np
import pytest

import oracle as O
from gpu_util import need_gpu, to_dev, to_np
from paper_2305_18396_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


def blockings(logN):
    out = []
    for s0 in range(logN + 1):
        a = logN - s0
        out.append((1 << s0, 1 << ((a + 1) // 2), 1 << (a // 2)))
    out += [(1 << (logN - 4), 3, 5), (1 << (logN - 7), 12, 10), (1 << (logN - 10), 31, 33)]
    return out


_STATE = {}


@pytest.fixture(scope="module")
def B():
    need_gpu()
    from paper_2305_18396_gb300 import binding

    return binding


def setup(B, N, L):
    if (N, L) not in _STATE:
        ctx, P = B.Context(N, L), O.Params(N, L)
        s = O.keygen(P, S.SEED_KEY)
        cases = []
        for i, blk in enumerate(blockings(N.bit_length() - 1)):
            m, k, n = 3, 2 * blk[1] + 1, blk[2] + 1  # ragged in k and n
            X = S.uniform_share((m, k), 10 + i)
            W = S.fixed_point_weights((k, n), 30 + i)
            ct = O.encrypt(P, s, O.pack_input(X, blk, N), 50 + i)
            cases.append((m, k, n, blk, W, ct, O.matmul(P, ct, W, m, k, n, blk, 70 + i)))
        _STATE[(N, L)] = (ctx, cases)
    return _STATE[(N, L)]


@pytest.mark.parametrize("N,L", [(4096, 2), (8192, 3)])
@pytest.mark.parametrize("logr", [3, 4, 5])
def test_sparse_weight_blocks_match_the_oracle(B, N, L, logr):
    ctx, cases = setup(B, N, L)
    ctx.set_ntt_radix(logr)
    try:
        for i, (m, k, n, blk, W, ct, want) in enumerate(cases):
            pt = B.he_encode_weights(ctx, to_dev(W), k, n, blk)
            out = B.he_matmul(ctx, to_dev(ct), pt, m, k, n, blk, 70 + i)
            assert np.array_equal(to_np(out).reshape(want.shape), want), blk
        B.he_device_status(ctx)
    finally:
        ctx.set_ntt_radix(4)
