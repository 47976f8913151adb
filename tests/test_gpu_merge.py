"""Requests that share a weight matrix, merged inside one multi-product launch.

Compact products (Sec. 3.1.3) with the same encoded weights, shape and blocking are run as
one product whose row-blocks are the requests' row-blocks back to back (each weight stage
of Algorithm 1 step 3 then serves every request's rows); each request keeps its own input
ciphertexts, output buffer, mask seed and output indices.  Every merged result must equal
the request's own he_matmul call bit for bit, on every multiply-accumulate engine, with a
mask seed read from device memory among them; sampled outputs are also compared with the
oracle's Pi_MatMul of the oracle's own encryptions.
"""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import need_gpu, to_dev, to_np
from paper_2305_18396_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    need_gpu()
    from paper_2305_18396_gb300 import binding

    return binding


@pytest.mark.parametrize("engine", ["coset", "tensor", "integer"])
def test_merged_requests_equal_their_own_calls_and_the_oracle(B, engine):
    N, L = 4096, 2
    ctx = B.Context(N, L)
    ctx.set_mac_engine({"coset": B.HE_MAC_COSET, "tensor": B.HE_MAC_TENSOR, "integer": B.HE_MAC_INTEGER}[engine])
    P = O.Params(N, L)
    s = O.keygen(P, S.SEED_KEY)
    mats = {"a": (384, 96, (4, 8, 16)), "b": (160, 200, (8, 4, 16))}  # k, n, blocking
    pts, Ws = {}, {}
    for i, (name, (k, n, blk)) in enumerate(mats.items()):
        Ws[name] = S.fixed_point_weights((k, n), 60 + i)
        pts[name] = B.he_encode_weights(ctx, to_dev(Ws[name]), k, n, blk)
    plan = [("a", 13), ("b", 40), ("a", 4), ("a", 29), ("b", 7), ("a", 16)]
    seeds = torch.tensor([777], dtype=torch.int64, device=ctx.device)
    items, reqs = [], []
    for r, (name, m) in enumerate(plan):
        k, n, blk = mats[name]
        X = S.uniform_share((m, k), 300 + r)
        ct = O.encrypt(P, s, O.pack_input(X, blk, N), 400 + r)
        si = ctx.sizes(m, k, n, blk)
        dev_seed = r == 3  # one request's mask seed is read from device memory
        items.append(dict(ct_in=to_dev(ct), pt=pts[name], ct_out=ctx.empty(si["out_words_compact"]), m=m, k=k, n=n,
                          blk=blk, flags=B.HE_DROP_C0 | (B.HE_SEED_DEVICE if dev_seed else 0),
                          mask_seed=seeds.data_ptr() if dev_seed else 500 + r))
        reqs.append((name, m, X, ct, 777 if dev_seed else 500 + r))
    prods = B.make_products(items)
    ws = ctx.empty(B.he_multi_workspace_bytes(ctx, prods) // 8 + 1)
    B.he_matmul_multi(ctx, prods, ws)
    B.he_device_status(ctx)
    for it, (name, m, X, ct, seed) in zip(items, reqs):
        k, n, blk = mats[name]
        alone = B.he_matmul(ctx, it["ct_in"], pts[name], m, k, n, blk, seed, flags=B.HE_DROP_C0)
        assert np.array_equal(to_np(it["ct_out"]), to_np(alone)), (name, m)
    for idx in (0, 4):  # one request of each matrix against the oracle
        name, m, X, ct, seed = reqs[idx]
        k, n, blk = mats[name]
        want = O.matmul(P, ct, Ws[name], m, k, n, blk, seed)
        kb, Nc = blk[1], N // blk[1]
        got = to_np(items[idx]["ct_out"]).reshape(want.shape[0], L * (Nc + N))
        assert np.array_equal(got[:, L * Nc:].reshape(-1, L, N), want[:, 1])
        assert np.array_equal(got[:, :L * Nc].reshape(-1, L, Nc), want[:, 0, :, kb - 1::kb])
    ctx.close()
