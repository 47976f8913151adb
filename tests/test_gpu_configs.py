"""Parity at the larger workload configurations, on sampled outputs.

* Full model stacks at N=8192 with three primes: every distinct product shape of a
  BERT-base layer at seq 128 and of a BERT-large layer at seq 512 (the layers of a stack
  repeat these shapes with other weights), run at full size with the library's default
  blocking.
* Batched form: 64 requests of mixed BERT-base / BERT-large layer matrices and sequence
  lengths uniform in [16, 512] in one multi-product launch at N=4096 (and 32 at N=8192):
  every result equals the request's own he_matmul, and sampled requests match the oracle.

The oracle cannot afford whole products at these sizes, so it evaluates a few output
ciphertexts (Algorithm 1 step 3 restricted to them).  Its inputs are its own: the test
encrypts the input rows those outputs read with the oracle (each at its object offset in
the batch) and writes them into the device buffer over the device's own encryption of
the same rows, after checking that the two are equal.  Each sampled output must match
bit for bit and decrypt, with the server's mask, to the corresponding block of X W mod t.
"""
import numpy as np
import pytest

import oracle as O
from gpu_util import need_gpu, to_dev, to_np
from paper_2305_18396_gb300 import synthetic as S
from paper_2305_18396_gb300 import workloads

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

_CTX = {}


@pytest.fixture(scope="module")
def B():
    need_gpu()
    from paper_2305_18396_gb300 import binding

    return binding


def ctx_for(B, N, L):
    if (N, L) not in _CTX:
        ctx, P = B.Context(N, L), O.Params(N, L)
        _CTX[(N, L)] = (ctx, P, B.he_keygen(ctx, S.SEED_KEY), O.keygen(P, S.SEED_KEY))
    return _CTX[(N, L)]


def oracle_rows(P, s, X, blk, nJ, Lb_list, enc_seed):
    """The oracle's encryption of input row-blocks Lb (ciphertexts Lb nJ .. Lb nJ + nJ - 1)."""
    m_b = blk[0]
    return {Lb: O.encrypt(P, s, O.pack_input(X[Lb * m_b:(Lb + 1) * m_b], blk, P.N), enc_seed, obj0=Lb * nJ)
            for Lb in Lb_list}


def plant_rows(ct_dev, rows, nJ, P):
    """Check the device's encryption of the rows equals the oracle's, then use the oracle's."""
    view = ct_dev.view(-1, 2, P.L, P.N)
    for Lb, r in rows.items():
        dev = to_np(view[Lb * nJ:(Lb + 1) * nJ])
        assert np.array_equal(dev.reshape(r.shape), r), f"device encryption of row-block {Lb}"
        view[Lb * nJ:(Lb + 1) * nJ] = to_dev(r).view(-1, 2, P.L, P.N)


def check_sampled(P, s, X, W, m, k, n, blk, mask_seed, rows, sel, got):
    """got: [len(sel)][2][L][N] from the device.  Bit-exact vs the oracle, then decrypt."""
    want = O.matmul(P, rows, W, m, k, n, blk, mask_seed, sel=sel)
    assert np.array_equal(got, want)
    check_decrypts(P, s, X, W, n, blk, mask_seed, sel, want)


def check_decrypts(P, s, X, W, n, blk, mask_seed, sel, want):
    """The oracle's outputs `want` of ciphertexts `sel` decrypt with a positive noise budget,
    and with the server's mask give the blocks of X W mod t."""
    dec, budget = O.decrypt(P, s, want)
    assert (budget > 0).all()
    m_b, k_b, n_b = blk
    nI = -(-n // n_b)
    for row, o in enumerate(sel):
        Lb, I = divmod(o, nI)
        r0, c0 = Lb * m_b, I * n_b
        ref = O.plain_matmul_mod_t(X[r0:r0 + m_b], W[:, c0:c0 + n_b], P.t)
        mask = O.mask_poly(P, mask_seed, o)
        for l in range(ref.shape[0]):
            for i in range(ref.shape[1]):
                pos = l * n_b * k_b + i * k_b + k_b - 1
                assert (int(dec[row][pos]) + int(mask[pos])) % P.t == int(ref[l, i]), (o, l, i)


def pick(total, seed, extra=1):
    rng = np.random.default_rng(seed)
    return sorted({0, total - 1, *map(int, rng.integers(0, total, extra))})


def stack_cases():
    out = []
    for tag, cfg in (("base", workloads.BERT_BASE), ("large", workloads.BERT_LARGE)):
        for p in workloads.bert_layer_products(**cfg, distinct_heads=1):
            out.append(pytest.param(p, id=f"{tag}-{p.name}-{p.m}x{p.k}x{p.n}"))
    return out


@pytest.mark.parametrize("prod", stack_cases())
def test_full_stack_products_n8192_sampled(B, prod):
    N, L = 8192, 3
    ctx, P, sk, s = ctx_for(B, N, L)
    m, k, n = prod.m, prod.k, prod.n
    blk = ctx.default_blocking(m, k, n, prod.share_weights)
    seed_x, seed_w = 100 + m + k, 200 + n
    X = S.uniform_share((m, k), seed_x)
    W = S.uniform_share((k, n), seed_w) if prod.share_weights else S.fixed_point_weights((k, n), seed_w)
    nI, nJ, nLb = O.blocks(m, k, n, blk)
    sel = pick(nI * nLb, 13)
    rows = oracle_rows(P, s, X, blk, nJ, sorted({o // nI for o in sel}), S.SEED_ENC)
    ct = B.he_encrypt(ctx, sk, B.he_pack_input(ctx, to_dev(X), m, k, blk), S.SEED_ENC)
    plant_rows(ct, rows, nJ, P)
    pt = B.he_encode_weights(ctx, to_dev(W), k, n, blk)
    out = B.he_matmul(ctx, ct, pt, m, k, n, blk, S.SEED_MASK)
    got = to_np(out).reshape(nI * nLb, 2, L, N)[sel]
    check_sampled(P, s, X, W, m, k, n, blk, S.SEED_MASK, rows, sel, got)
    B.he_device_status(ctx)


MATRICES = [("base.qkv", 768, 2304), ("base.ffn2", 3072, 768), ("large.out", 1024, 1024), ("large.ffn1", 1024, 4096)]


@pytest.mark.parametrize("N,L,count", [(4096, 2, 64), (8192, 3, 32)])
def test_batched_mixed_requests_one_launch(B, N, L, count):
    ctx, P, sk, s = ctx_for(B, N, L)
    rng = np.random.default_rng(21 + N)
    weights = {}
    for idx, (name, k, n) in enumerate(MATRICES):
        blk = ctx.default_blocking(128, k, n)
        W = S.fixed_point_weights((k, n), 700 + idx)
        weights[name] = (k, n, blk, W, B.he_encode_weights(ctx, to_dev(W), k, n, blk))
    sampled = set(map(int, rng.choice(count, 3, replace=False)))
    items, reqs = [], []
    for r in range(count):
        name = MATRICES[int(rng.integers(0, len(MATRICES)))][0]
        k, n, blk, W, pt = weights[name]
        m = int(rng.integers(16, 513))
        X = S.uniform_share((m, k), 5000 + r)
        ct = B.he_encrypt(ctx, sk, B.he_pack_input(ctx, to_dev(X), m, k, blk), 6000 + r)
        nI, nJ, nLb = O.blocks(m, k, n, blk)
        sel, rows = None, None
        if r in sampled:
            sel = pick(nI * nLb, r, extra=0)
            rows = oracle_rows(P, s, X, blk, nJ, sorted({o // nI for o in sel}), 6000 + r)
            plant_rows(ct, rows, nJ, P)
        si = ctx.sizes(m, k, n, blk)
        items.append(dict(ct_in=ct, pt=pt, ct_out=ctx.empty(si["out_words"]), m=m, k=k, n=n, blk=blk, flags=0,
                          mask_seed=7000 + r))
        reqs.append((name, m, X, sel, rows))
    prods = B.make_products(items)
    ws = ctx.empty(B.he_multi_workspace_bytes(ctx, prods) // 8 + 1)
    B.he_matmul_multi(ctx, prods, ws)
    B.he_device_status(ctx)
    for it, (name, m, X, sel, rows) in zip(items, reqs):
        k, n, blk, W, pt = weights[name]
        alone = B.he_matmul(ctx, it["ct_in"], pt, m, k, n, blk, it["mask_seed"])
        assert np.array_equal(to_np(it["ct_out"]), to_np(alone)), (name, m)
        if sel is not None:
            nI, nJ, nLb = O.blocks(m, k, n, blk)
            got = to_np(it["ct_out"]).reshape(nI * nLb, 2, L, N)[sel]
            check_sampled(P, s, X, W, m, k, n, blk, it["mask_seed"], rows, sel, got)
