"""One BERT-base layer (seq 128, N=4096, L=2) in full against the oracle.

Every product of the layer -- QKV, attention-out, FFN1, FFN2 and all 12 heads' four
cross-term products (same-shape batches) -- runs through the library with the
default blockings; every output ciphertext must equal the oracle's bit for bit, and
the first and last output of each product decrypt, with the server's mask, to X W.
The oracle encrypts the inputs itself.
"""
import numpy as np
import pytest

import oracle as O
from gpu_util import need_gpu, to_dev, to_np
from paper_2305_18396_gb300 import synthetic as S
from paper_2305_18396_gb300 import workloads

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def env():
    need_gpu()
    from paper_2305_18396_gb300 import binding as B

    ctx, P = B.Context(4096, 2), O.Params(4096, 2)
    return B, ctx, P, O.keygen(P, S.SEED_KEY)


@pytest.mark.parametrize("prod", workloads.bert_layer_products(**workloads.BERT_BASE), ids=lambda p: p.name)
def test_bert_base_layer_in_full(env, prod):
    B, ctx, P, s = env
    m, k, n, cnt = prod.m, prod.k, prod.n, prod.count
    blk = ctx.default_blocking(m, k, n, prod.share_weights)
    nI, nJ, nLb = O.blocks(m, k, n, blk)
    si = ctx.sizes(m, k, n, blk)
    base = 1000 * sum(map(ord, prod.name))  # a fixed seed per product
    Xs = [S.uniform_share((m, k), base + b) for b in range(cnt)]
    if prod.share_weights:
        Ws = [S.uniform_share((k, n), base + 500 + b) for b in range(cnt)]
    else:
        Ws = [S.fixed_point_weights((k, n), base + 500 + b) for b in range(cnt)]
    cts = [O.encrypt(P, s, O.pack_input(X, blk, P.N), base + 900 + b) for b, X in enumerate(Xs)]
    pt = B.he_encode_weights_batch(ctx, to_dev(np.stack(Ws)), k, n, blk, cnt)
    out = to_np(B.he_matmul_batch(ctx, to_dev(np.stack(cts)), pt, m, k, n, blk, cnt, 77))
    out = out.reshape(cnt, nI * nLb, 2, P.L, P.N)
    m_b, k_b, n_b = blk
    for b in range(cnt):
        want = O.matmul(P, cts[b], Ws[b], m, k, n, blk, 77 + b)
        assert np.array_equal(out[b], want), (prod.name, b)
        if b in (0, cnt - 1):
            sel = [0, nI * nLb - 1]
            dec, budget = O.decrypt(P, s, want[sel])
            assert (budget > 0).all()
            for row, o in enumerate(sel):
                Lb, I = divmod(o, nI)
                ref = O.plain_matmul_mod_t(Xs[b][Lb * m_b:(Lb + 1) * m_b], Ws[b][:, I * n_b:(I + 1) * n_b], P.t)
                mask = O.mask_poly(P, 77 + b, o)
                for l in range(ref.shape[0]):
                    for i in range(ref.shape[1]):
                        pos = l * n_b * k_b + i * k_b + k_b - 1
                        assert (int(dec[row][pos]) + int(mask[pos])) % P.t == int(ref[l, i])
    assert si["out_words"] * cnt == out.size
