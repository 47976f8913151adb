"""Ciphertexts on the wire (Algorithm 1's exchange; Sec. 3.1.3, "Reducing the
communication cost"): he_ct_import / he_ct_export move the library's ciphertext layout
between host buffers and device memory, and the import rejects words that are not
residues of their prime.

A client's ciphertexts made by the oracle travel host -> device through he_ct_import,
the product runs on the device, and the result travels back through he_ct_export; the
words that arrive must equal the oracle's output bit for bit, in full and in compact form.
"""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import need_gpu
from paper_2305_18396_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    need_gpu()
    from paper_2305_18396_gb300 import binding

    return binding


def _host(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64).reshape(-1).copy())


@pytest.mark.parametrize("N,L,m,k,n,blk", [(4096, 2, 40, 96, 72, (8, 32, 16)), (8192, 3, 24, 64, 48, (8, 16, 32))])
def test_import_product_export_equals_oracle(B, N, L, m, k, n, blk):
    ctx = B.Context(N, L)
    P = O.Params(N, L)
    s = O.keygen(P, S.SEED_KEY)
    X = S.uniform_share((m, k), 31)
    W = S.fixed_point_weights((k, n), 32)
    ct = O.encrypt(P, s, O.pack_input(X, blk, N), 33)
    si = ctx.sizes(m, k, n, blk)
    ct_dev = B.he_ct_import(ctx, _host(ct), si["in_cts"])
    assert np.array_equal(B.he_ct_export(ctx, ct_dev, si["in_cts"]).numpy().view(np.uint64), ct.reshape(-1))
    pt = B.he_encode_weights(ctx, _host(W).to(ctx.device), k, n, blk)
    want = O.matmul(P, ct, W, m, k, n, blk, 34)
    full = B.he_matmul(ctx, ct_dev, pt, m, k, n, blk, 34)
    got = B.he_ct_export(ctx, full, si["out_cts"]).numpy().view(np.uint64)
    assert np.array_equal(got, want.reshape(-1))
    kb, Nc = blk[1], N // blk[1]
    comp = B.he_matmul(ctx, ct_dev, pt, m, k, n, blk, 34, flags=B.HE_DROP_C0)
    got = B.he_ct_export(ctx, comp, si["out_cts"], kb).numpy().view(np.uint64)
    assert got.size == B.wire_words(ctx, si["out_cts"], kb) == si["out_words_compact"]
    got = got.reshape(si["out_cts"], L * (Nc + N))
    assert np.array_equal(got[:, :L * Nc].reshape(-1, L, Nc), want[:, 0, :, kb - 1::kb])
    assert np.array_equal(got[:, L * Nc:].reshape(-1, L, N), want[:, 1])
    # the compact words re-imported are accepted and equal
    back = B.he_ct_import(ctx, _host(got), si["out_cts"], kb)
    assert torch.equal(back, comp[:back.numel()])
    ctx.close()


def test_import_rejects_words_not_below_their_prime(B):
    N, L = 4096, 2
    ctx = B.Context(N, L)
    P = O.Params(N, L)
    s = O.keygen(P, S.SEED_KEY)
    ct = O.encrypt(P, s, S.uniform_plaintexts(3, N, 5), 6)
    bad = ct.copy()
    bad[2, 1, 1, 17] = P.q[1]          # c1 of ciphertext 2, prime 1: exactly q_1
    bad[1, 0, 0, 5] = np.uint64(2**63)  # c0 of ciphertext 1, prime 0
    with pytest.raises(B.HEError) as e:
        B.he_ct_import(ctx, _host(bad), 3)
    msg = str(e.value)
    assert e.value.code == B.HE_EINVAL and "2 word(s)" in msg and "ciphertext 1, c0, prime 0" in msg
    edge = ct.copy()
    edge[0, 1, 1, 0] = P.q[1] - 1       # the largest residue is accepted
    dev = B.he_ct_import(ctx, _host(edge), 3)
    assert np.array_equal(dev.cpu().numpy().view(np.uint64), edge.reshape(-1))
    # compact form: c0 words are checked against their prime too
    kb = 8
    Nc = N // kb
    comp = np.zeros((1, L * (Nc + N)), dtype=np.uint64)
    comp[0, Nc + 3] = P.q[1]            # c0, prime 1
    with pytest.raises(B.HEError) as e:
        B.he_ct_import(ctx, _host(comp), 1, kb)
    assert "ciphertext 0, c0, prime 1" in str(e.value)
    rc = B.lib.he_ct_import(ctx.h, B._ptr(_host(comp)), 1, 3, B._ptr(ctx.empty(comp.size)), B._stream(None))
    assert rc == B.HE_EINVAL and "power of two" in B.lib.he_last_error().decode()  # k_b = 3
    ctx.close()
