"""The tensor-core multiply-accumulate (exact balanced-digit split on tcgen05) against the
oracle and against the integer multiply-accumulate.

Algorithm 1 step 3 in the NTT domain must give the same output ciphertexts bit for bit
whichever engine sums the slot products.  The shapes cover the kernel's edges: a single
k-block, an odd number of k-blocks (padded operand rows), more than one exact accumulation
round (> 128 k-blocks), several 128-row weight tiles and 16-row ciphertext tiles with
ragged last tiles, compact output (Sec. 3.1.3), same-shape batches and a multi-product
launch that mixes tensor-core and integer products.  The oracle's inputs are its own
encryptions; small products are compared in full, larger ones on sampled outputs.
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


CASES = [  # (N, L, m, k, n, blocking)
    (4096, 2, 16, 64, 64, (8, 32, 16)),      # nJ 2
    (4096, 2, 5, 9, 7, (4, 1, 8)),           # nJ 9 (odd), ragged everything
    (4096, 2, 20, 264, 200, (4, 8, 16)),     # nJ 33, 13 weight blocks, 10 rows
    (4096, 2, 18, 520, 1040, (2, 4, 8)),     # nJ 130 (two rounds), 130 weight blocks (2 tiles), 18 rows (2 tiles)
    (8192, 3, 24, 300, 100, (8, 4, 32)),     # nJ 75 (odd), N = 8192, three primes
    (8192, 3, 64, 1024, 256, (8, 4, 16)),    # nJ 256, 16 weight blocks, 8 row-blocks (one full 16-row tile)
]


def _inputs(P, blk, m, k, n, seed):
    s = O.keygen(P, S.SEED_KEY)
    X = S.uniform_share((m, k), seed)
    W = S.fixed_point_weights((k, n), seed + 1)
    ct = O.encrypt(P, s, O.pack_input(X, blk, P.N), seed + 2)
    return s, X, W, ct


@pytest.mark.parametrize("N,L,m,k,n,blk", CASES)
def test_tensor_mac_equals_integer_mac_and_oracle(B, N, L, m, k, n, blk):
    P = O.Params(N, L)
    s, X, W, ct = _inputs(P, blk, m, k, n, 40 + m)
    tc = ctx_for(B, N, L, B.HE_MAC_TENSOR)
    im = ctx_for(B, N, L, B.HE_MAC_INTEGER)
    assert tc.uses_tensor_cores(k, blk) and not im.uses_tensor_cores(k, blk)
    outs = {}
    for name, ctx in (("tc", tc), ("int", im)):
        pt = B.he_encode_weights(ctx, to_dev(W), k, n, blk)
        outs[name] = to_np(B.he_matmul(ctx, to_dev(ct), pt, m, k, n, blk, 321))
        outs[name + "_c"] = to_np(B.he_matmul(ctx, to_dev(ct), pt, m, k, n, blk, 321, flags=B.HE_DROP_C0))
        B.he_device_status(ctx)
    assert np.array_equal(outs["tc"], outs["int"])
    assert np.array_equal(outs["tc_c"], outs["int_c"])
    nI, nJ, nLb = O.blocks(m, k, n, blk)
    total = nI * nLb
    if total <= 64:
        sel = list(range(total))
    else:  # both weight tiles, both row tiles, the ragged corners
        sel = sorted({0, nI - 1, 127 % nI, nI * (nLb - 1), total - 1, (nLb // 2) * nI + nI // 2})
    want = O.matmul(P, ct, W, m, k, n, blk, 321, sel=sel)
    got = outs["tc"].reshape(total, 2, L, N)[sel]
    assert np.array_equal(got, want)


def test_tensor_mac_batch_and_mixed_multi_launch(B):
    """Same-shape batch on the tensor cores (through the cosets, n_b k_b = 128); a
    multi-product launch with that product and one on the integer pipe (n_b k_b = N: no
    coset form; nJ 4) under the default engine."""
    N, L = 4096, 2
    P = O.Params(N, L)
    ctx = ctx_for(B, N, L, B.HE_MAC_AUTO)
    blk_t, blk_i = (8, 8, 16), (1, 64, 64)
    m, k, n = 24, 384, 96
    assert ctx.uses_tensor_cores(k, blk_t) and not ctx.uses_tensor_cores(256, blk_i)
    s, X, W, ct = _inputs(P, blk_t, m, k, n, 90)
    X2 = S.uniform_share((m, k), 95)
    ct2 = O.encrypt(P, s, O.pack_input(X2, blk_t, N), 96)
    W2 = S.fixed_point_weights((k, n), 97)
    pt = B.he_encode_weights_batch(ctx, to_dev(np.stack([W, W2])), k, n, blk_t, 2)
    out = to_np(B.he_matmul_batch(ctx, to_dev(np.stack([ct, ct2])), pt, m, k, n, blk_t, 2, 500))
    si = ctx.sizes(m, k, n, blk_t)
    for b, (c, w) in enumerate(((ct, W), (ct2, W2))):
        want = O.matmul(P, c, w, m, k, n, blk_t, 500 + b)
        assert np.array_equal(out[b * si["out_words"]:(b + 1) * si["out_words"]], want.reshape(-1)), b
    # mixed multi-product launch
    mi, ki, ni = 16, 256, 48
    _, Xi, Wi, cti = _inputs(P, blk_i, mi, ki, ni, 80)
    pti = B.he_encode_weights(ctx, to_dev(Wi), ki, ni, blk_i)
    pt1 = B.he_encode_weights(ctx, to_dev(W), k, n, blk_t)
    items = [dict(ct_in=to_dev(ct), pt=pt1, ct_out=ctx.empty(si["out_words_compact"]), m=m, k=k, n=n, blk=blk_t,
                  flags=B.HE_DROP_C0, mask_seed=600),
             dict(ct_in=to_dev(cti), pt=pti, ct_out=ctx.empty(ctx.sizes(mi, ki, ni, blk_i)["out_words"]), m=mi, k=ki,
                  n=ni, blk=blk_i, flags=0, mask_seed=601)]
    prods = B.make_products(items)
    ws = ctx.empty(B.he_multi_workspace_bytes(ctx, prods) // 8 + 1)
    B.he_matmul_multi(ctx, prods, ws)
    B.he_device_status(ctx)
    want_t = O.matmul(P, ct, W, m, k, n, blk_t, 600)
    kb, Nc = blk_t[1], N // blk_t[1]
    got_t = to_np(items[0]["ct_out"]).reshape(si["out_cts"], L * (Nc + N))
    assert np.array_equal(got_t[:, L * Nc:].reshape(-1, L, N), want_t[:, 1])
    assert np.array_equal(got_t[:, :L * Nc].reshape(-1, L, Nc), want_t[:, 0, :, kb - 1::kb])
    want_i = O.matmul(P, cti, Wi, mi, ki, ni, blk_i, 601)
    assert np.array_equal(to_np(items[1]["ct_out"]), want_i.reshape(-1))
