"""Products through the ring's cosets (HE_MAC_COSET, the default engine's form for weight
blocks of at most N/2 coefficients) against the oracle and the integer engine.

Algorithm 1 step 3 computes, per output ciphertext, sum_J a_{I,J} [[b_{J,Lb}]] mod x^N + 1
and q_l; the coset form reaches the same polynomials by the first log2 G NTT stages, a
zero-padded length-2D transform per coset, the multiply-accumulate over 2D slots, the
inverse and a fold by each coset's root.  Every output must equal the oracle's Pi_MatMul
(and the integer engine's output) bit for bit.  The shapes cover the geometry's edges: the
smallest D (8) and the largest (N/2, two cosets), each transform form (D <= 32 per thread,
64 and 128 as register passes, larger in shared memory), ragged blocks, an odd number of k-blocks,
more than one exact accumulation round (> 128 k-blocks), many operand-row tiles, N = 4096
and 8192, full and compact (Sec. 3.1.3) outputs, and same-shape batches.
"""
import numpy as np
import pytest

import oracle as O
from gpu_util import need_gpu, to_dev, to_np
from paper_2305_18396_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

_CTX = {}


@pytest.fixture(scope="module")
def B():
    need_gpu()
    from paper_2305_18396_gb300 import binding

    return binding


def ctx_for(B, N, L, engine):
    key = (N, L, engine)
    if key not in _CTX:
        ctx = B.Context(N, L)
        ctx.set_mac_engine(engine)
        _CTX[key] = ctx
    return _CTX[key]


CASES = [  # (N, L, m, k, n, blocking); D = max(8, n_b k_b rounded up), G = N / D
    (4096, 2, 16, 64, 64, (16, 4, 4)),        # D 16, G 256, nJ 16, one stage
    (4096, 2, 5, 9, 7, (4, 1, 8)),            # D 8 (smallest), ragged everything
    (4096, 2, 20, 264, 200, (4, 8, 16)),      # D 128, nJ 33 (odd), 13 weight blocks
    (4096, 2, 18, 520, 1040, (2, 4, 8)),      # D 32, nJ 130 (two rounds), 130 weight blocks, 2304 rows
    (4096, 2, 40, 96, 300, (2, 16, 128)),     # D 2048 = N/2: two cosets
    (4096, 2, 24, 100, 160, (8, 8, 8)),       # D 64: register passes per coset half
    (8192, 3, 30, 200, 90, (16, 16, 16)),     # D 256: shared-memory transforms
    (8192, 3, 24, 300, 100, (8, 4, 32)),      # D 128, nJ 75, N = 8192, three primes
    (8192, 3, 512, 64, 512, (512, 4, 4)),     # a BERT-large attention product: D 16, G 512, 1024 rows
]


def _inputs(P, blk, m, k, n, seed):
    s = O.keygen(P, S.SEED_KEY)
    X = S.uniform_share((m, k), seed)
    W = S.fixed_point_weights((k, n), seed + 1)
    ct = O.encrypt(P, s, O.pack_input(X, blk, P.N), seed + 2)
    return s, X, W, ct


@pytest.mark.parametrize("N,L,m,k,n,blk", CASES)
def test_coset_products_equal_oracle_and_integer_engine(B, N, L, m, k, n, blk):
    P = O.Params(N, L)
    s, X, W, ct = _inputs(P, blk, m, k, n, 70 + m)
    cs = ctx_for(B, N, L, B.HE_MAC_COSET)
    im = ctx_for(B, N, L, B.HE_MAC_INTEGER)
    assert cs.uses_tensor_cores(k, blk)
    si_c, si_i = cs.sizes(m, k, n, blk), im.sizes(m, k, n, blk)
    D = max(8, 1 << (blk[1] * blk[2] - 1).bit_length())
    nI, nJ, nLb = O.blocks(m, k, n, blk)
    assert si_c["pt_words"] < si_i["pt_words"] or D == N // 2  # 2D slots per weight block instead of N
    outs = {}
    for name, ctx in (("coset", cs), ("int", im)):
        pt = B.he_encode_weights(ctx, to_dev(W), k, n, blk)
        outs[name] = to_np(B.he_matmul(ctx, to_dev(ct), pt, m, k, n, blk, 321))
        outs[name + "_c"] = to_np(B.he_matmul(ctx, to_dev(ct), pt, m, k, n, blk, 321, flags=B.HE_DROP_C0))
        B.he_device_status(ctx)
    assert np.array_equal(outs["coset"], outs["int"])
    assert np.array_equal(outs["coset_c"], outs["int_c"])
    total = nI * nLb
    if total <= 48:
        sel = list(range(total))
    else:  # the first and last weight blocks and row blocks, and one in the middle
        sel = sorted({0, nI - 1, nI * (nLb - 1), total - 1, (nLb // 2) * nI + nI // 2})
    want = O.matmul(P, ct, W, m, k, n, blk, 321, sel=sel)
    got = outs["coset"].reshape(total, 2, L, N)[sel]
    assert np.array_equal(got, want)
    kb, Nc = blk[1], N // blk[1]
    got_c = outs["coset_c"].reshape(total, L * (Nc + N))[sel]
    assert np.array_equal(got_c[:, L * Nc:].reshape(-1, L, N), want[:, 1])
    assert np.array_equal(got_c[:, :L * Nc].reshape(-1, L, Nc), want[:, 0, :, kb - 1::kb])


def test_coset_batch_and_decryption(B):
    """A same-shape batch of three products (each its own weights, inputs and mask seed
    mask_seed + b) equals the oracle; the client's decryption plus the server's mask share
    is X W mod t."""
    N, L = 4096, 2
    P = O.Params(N, L)
    ctx = ctx_for(B, N, L, B.HE_MAC_AUTO)
    m, k, n, blk = 30, 200, 72, (16, 8, 8)
    assert ctx.uses_tensor_cores(k, blk)
    s = O.keygen(P, S.SEED_KEY)
    Xs = [S.uniform_share((m, k), 110 + b) for b in range(3)]
    Ws = [S.fixed_point_weights((k, n), 120 + b) for b in range(3)]
    cts = [O.encrypt(P, s, O.pack_input(X, blk, N), 130 + b) for b, X in enumerate(Xs)]
    pt = B.he_encode_weights_batch(ctx, to_dev(np.stack(Ws)), k, n, blk, 3)
    out = to_np(B.he_matmul_batch(ctx, to_dev(np.stack(cts)), pt, m, k, n, blk, 3, 900))
    B.he_device_status(ctx)
    ow = ctx.sizes(m, k, n, blk)["out_words"]
    for b in range(3):
        want = O.matmul(P, cts[b], Ws[b], m, k, n, blk, 900 + b)
        got = out[b * ow:(b + 1) * ow]
        assert np.array_equal(got, want.reshape(-1)), b
        dec, budget = O.decrypt(P, s, want)
        assert np.min(budget) > 0
        client = O.unpack_output(dec, m, n, blk)
        server = O.unmask(P, 900 + b, m, n, blk)
        assert np.array_equal((client + server) % np.uint64(P.t), O.plain_matmul_mod_t(Xs[b], Ws[b], P.t))
