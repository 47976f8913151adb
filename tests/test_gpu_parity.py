"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Everything here is exact integer work, so the bar is bit-exactness: every
ciphertext word, key word, packed coefficient and share must equal the
oracle's on the same seeded inputs.  Inputs come from the seeded generators
and the oracle's own encryption; nothing the GPU computes is fed to the
oracle.
"""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import need_gpu, to_dev, to_np
from paper_2305_18396_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

PARAMS = [(64, 2), (4096, 2), (8192, 3)]
_CTX = {}


@pytest.fixture(scope="module")
def B():
    need_gpu()
    from paper_2305_18396_gb300 import binding

    return binding


def ctx_for(B, N, L):
    if (N, L) not in _CTX:
        _CTX[(N, L)] = (B.Context(N, L), O.Params(N, L))
    return _CTX[(N, L)]


def _rand_residues(P, cnt, seed):
    rng = np.random.default_rng(seed)
    a = np.zeros((cnt, P.L, P.N), dtype=np.uint64)
    for li, q in enumerate(P.q):
        a[:, li] = rng.integers(0, q, size=(cnt, P.N), dtype=np.uint64)
    return a


def _pointwise(P, fa, fb):
    out = np.zeros_like(fa)
    for li, q in enumerate(P.q):
        out[:, li] = ((fa[:, li].astype(object) * fb[:, li].astype(object)) % q).astype(np.uint64)
    return out


# ------------------------------------------------------------------ NTT


@pytest.mark.parametrize("N,L", PARAMS)
def test_ntt_roundtrip_and_negacyclic_product(B, N, L):
    ctx, P = ctx_for(B, N, L)
    a = _rand_residues(P, 3, 1)
    b = _rand_residues(P, 3, 2)
    t = to_dev(a)
    B.he_ntt_forward(ctx, t)
    assert not np.array_equal(to_np(t, a.shape), a)
    B.he_ntt_inverse(ctx, t)
    assert np.array_equal(to_np(t, a.shape), a)
    c = B.he_poly_mul(ctx, to_dev(a), to_dev(b))
    want = O.ntt_inverse(P, _pointwise(P, O.ntt_forward(P, a), O.ntt_forward(P, b)))
    assert np.array_equal(to_np(c, a.shape), want)


def test_ntt_slot_order(B):
    """Slot j of the forward transform holds a(psi^{2 brev(j) + 1}) for the library's psi."""
    N, L = 4096, 2
    ctx, P = ctx_for(B, N, L)
    psi_gpu = ctx.params()["psi"]
    a = _rand_residues(P, 1, 3)
    t = to_dev(a)
    B.he_ntt_forward(ctx, t)
    got = to_np(t, a.shape)
    ref = O.ntt_forward(P, a)  # ref[k] = a(psi_oracle^{2k+1})
    logN = N.bit_length() - 1
    brev = np.array([int(format(j, f"0{logN}b")[::-1], 2) for j in range(N)])
    for li, q in enumerate(P.q):
        u = next(e for e in range(1, 2 * N, 2) if pow(P.psi[li], e, q) == psi_gpu[li])
        k = ((u * (2 * brev + 1)) % (2 * N) - 1) // 2
        assert np.array_equal(got[0, li], ref[0, li][k])


# ------------------------------------------------------------------ test client


@pytest.mark.parametrize("N,L", PARAMS)
def test_keygen_encrypt_decrypt_bit_exact(B, N, L):
    ctx, P = ctx_for(B, N, L)
    sk = B.he_keygen(ctx, S.SEED_KEY)
    s = O.keygen(P, S.SEED_KEY)
    coeff = sk.clone()
    B.he_ntt_inverse(ctx, coeff)
    want = np.stack([np.array([int(v) % q for v in s], dtype=np.uint64) for q in P.q])
    assert np.array_equal(to_np(coeff, (L, N)), want)

    plain = S.uniform_plaintexts(3, N, 17)
    ct = B.he_encrypt(ctx, sk, to_dev(plain), S.SEED_ENC)
    ct_or = O.encrypt(P, s, plain, S.SEED_ENC)
    assert np.array_equal(to_np(ct, ct_or.shape), ct_or)

    dec, budget = B.he_decrypt(ctx, sk, to_dev(ct_or), check_noise=True)
    dec_or, budget_or = O.decrypt(P, s, ct_or)
    assert np.array_equal(to_np(dec, (3, N)), plain)
    assert np.array_equal(dec_or, plain)
    # the library resolves the fraction to 2^-64, so its budget saturates at 63 bits
    assert np.all(np.abs(budget.cpu().numpy() - np.minimum(budget_or, 63)) <= 1)


def test_decrypt_reports_exhausted_noise(B):
    """A ciphertext with random c0 has no noise budget left: HE_ENOISE, host-side."""
    ctx, P = ctx_for(B, 4096, 2)
    sk = B.he_keygen(ctx, 1)
    junk = _rand_residues(P, 2, 9).reshape(1, 2, P.L, P.N)
    with pytest.raises(B.HEError) as e:
        B.he_decrypt(ctx, sk, to_dev(junk), check_noise=True)
    assert e.value.code == B.HE_ENOISE


def test_pack_unpack_unmask(B):
    ctx, P = ctx_for(B, 4096, 2)
    m, k, n, blk = 37, 70, 45, (8, 16, 32)
    X = S.uniform_share((m, k), 5)
    polys = B.he_pack_input(ctx, to_dev(X), m, k, blk)
    want = O.pack_input(X, blk, P.N)
    assert np.array_equal(to_np(polys, want.shape), want)
    nI, nJ, nLb = O.blocks(m, k, n, blk)
    dec = S.uniform_plaintexts(nLb * nI, P.N, 6)
    share = B.he_unpack_output(ctx, to_dev(dec), m, n, blk)
    assert np.array_equal(to_np(share, (m, n)), O.unpack_output(dec, m, n, blk))
    srv = B.he_unmask(ctx, 77, m, n, blk)
    assert np.array_equal(to_np(srv, (m, n)), O.unmask(P, 77, m, n, blk))


# ------------------------------------------------------------------ Algorithm 1 (server)


def _run_case(B, N, L, m, k, n, blk, W, X, mask_seed=5, host=False):
    ctx, P = ctx_for(B, N, L)
    s = O.keygen(P, S.SEED_KEY)
    ct_in = O.encrypt(P, s, O.pack_input(X, blk, N), S.SEED_ENC)
    pt = B.he_encode_weights(ctx, to_dev(W), k, n, blk)
    if host:
        ws = ctx.empty(B.matmul_host_workspace_words(ctx, m, k, n, blk))
        si = ctx.sizes(m, k, n, blk)
        out_host = torch.empty(si["out_words"], dtype=torch.int64).pin_memory()
        B.he_matmul_host(ctx, torch.from_numpy(ct_in.reshape(-1).view(np.int64)).pin_memory(), pt, m, k, n, blk,
                         mask_seed, out_host, ws)
        got = out_host.numpy().view(np.uint64)
    else:
        out = B.he_matmul(ctx, to_dev(ct_in), pt, m, k, n, blk, mask_seed)
        got = to_np(out)
    want = O.matmul(P, ct_in, W, m, k, n, blk, mask_seed)
    assert np.array_equal(got.reshape(want.shape), want)
    # end to end: client decrypts + server unmasks = X W mod t
    dec, budget = O.decrypt(P, s, want)
    client = O.unpack_output(dec, m, n, blk)
    server = to_np(B.he_unmask(ctx, mask_seed, m, n, blk), (m, n))
    assert np.array_equal((client + server) % np.uint64(P.t), O.plain_matmul_mod_t(X, W, P.t))
    assert (budget > 0).all()


MATMUL_CASES = [
    # (N, L, m, k, n, blocking, weights kind)
    (4096, 2, 16, 64, 64, (8, 32, 16), "fixed"),       # the single-product configuration
    (4096, 2, 9, 70, 37, (4, 32, 32), "fixed"),        # ragged in every dimension
    (4096, 2, 12, 40, 24, (4, 16, 64), "uniform"),     # share x share
    (8192, 3, 7, 33, 20, (8, 32, 32), "uniform"),
    (64, 2, 5, 6, 7, (2, 4, 8), "fixed"),              # N below one MAC thread block
    (4096, 2, 1, 1, 1, (1, 1, 1), "uniform"),          # degenerate 1 x 1 x 1
    (1024, 2, 1, 4096, 4, (1, 1, 4), "uniform"),       # 4096 k-blocks: accumulator headroom limit
]


@pytest.mark.parametrize("N,L,m,k,n,blk,kind", MATMUL_CASES)
def test_matmul_bit_exact(B, N, L, m, k, n, blk, kind):
    X = S.uniform_share((m, k), S.SEED_X)
    W = S.fixed_point_weights((k, n), S.SEED_W) if kind == "fixed" else S.uniform_share((k, n), S.SEED_W)
    _run_case(B, N, L, m, k, n, blk, W, X)


def test_matmul_host_buffers(B):
    X = S.uniform_share((16, 64), S.SEED_X)
    W = S.fixed_point_weights((64, 64), S.SEED_W)
    _run_case(B, 4096, 2, 16, 64, 64, (8, 32, 16), W, X, host=True)


def test_matmul_default_blocking_single_config(B):
    ctx, _ = ctx_for(B, 4096, 2)
    blk = ctx.default_blocking(16, 64, 64)
    X = S.uniform_share((16, 64), S.SEED_X)
    W = S.fixed_point_weights((64, 64), S.SEED_W)
    _run_case(B, 4096, 2, 16, 64, 64, blk, W, X)


def test_matmul_argument_errors(B):
    ctx, _ = ctx_for(B, 4096, 2)
    blk = (8, 32, 16)
    si = ctx.sizes(16, 64, 64, blk)
    ct = ctx.empty(si["in_words"])
    pt = ctx.empty(si["pt_words"])
    out = ctx.empty(si["out_words"])
    ws = ctx.empty(si["workspace_bytes"] // 8)
    rc = B.lib.he_matmul(ctx.h, B._ptr(ct), B._ptr(pt), 16, 64, 64, B._blk(blk), 1, 0, B._ptr(out), B._ptr(ws),
                         si["workspace_bytes"] - 8, B._stream(None))
    assert rc == B.HE_ENOMEM and "workspace" in B.lib.he_last_error().decode()
    with pytest.raises(B.HEError) as e:
        B.he_matmul(ctx, ct, pt, 16, 64, 64, (16, 32, 16), 1, out)
    assert e.value.code == B.HE_EINVAL
    with pytest.raises(B.HEError) as e:
        B.he_matmul(ctx, ct, pt, 16, 64, 64, blk, 1, out, flags=7)
    assert e.value.code == B.HE_EINVAL
    # empty product: valid no-op
    assert B.lib.he_matmul(ctx.h, None, None, 0, 64, 64, B._blk(blk), 1, 0, None, None, 0, None) == B.HE_OK


def test_launch_count_and_profile(B):
    ctx, _ = ctx_for(B, 4096, 2)
    X = S.uniform_share((16, 64), 1)
    W = S.fixed_point_weights((64, 64), 2)
    blk = (8, 32, 16)
    pt = B.he_encode_weights(ctx, to_dev(W), 64, 64, blk)
    polys = B.he_pack_input(ctx, to_dev(X), 16, 64, blk)
    sk = B.he_keygen(ctx, 3)
    ct = B.he_encrypt(ctx, sk, polys, 4)
    before = B.he_launch_count(ctx)
    B.he_profile_enable(ctx, True)
    B.he_matmul(ctx, ct, pt, 16, 64, 64, blk, 5)
    stats = B.he_profile_read(ctx)
    B.he_profile_enable(ctx, False)
    assert B.he_launch_count(ctx) - before == 3
    if ctx.uses_cosets(blk):  # n_b k_b = 512 <= N/2: the default engine's coset form
        assert set(stats) == {"coset_forward", "mac_tc", "coset_inverse"}
    else:
        assert set(stats) == {"ntt_forward", "mac", "intt_mask"}
    assert all(v["launches"] == 1 and v["total_ms"] > 0 for v in stats.values())


# ------------------------------------------------------------------ full-size layer products, sampled


def bert_layer_cases():
    from paper_2305_18396_gb300 import workloads

    return workloads.bert_layer_products(seq=128, hidden=768, ffn=3072, heads=12, distinct_heads=1)


@pytest.mark.parametrize("prod", bert_layer_cases(), ids=lambda p: p.name)
def test_bert_base_layer_products_sampled(B, prod):
    """Every distinct product shape of one BERT-base layer at seq 128 (N=4096, L=2), run at
    full size with the blocking the benchmark uses; sampled output ciphertexts must match the
    oracle bit for bit and decrypt (with the server's unmask) to X W mod t."""
    N, L = 4096, 2
    ctx, P = ctx_for(B, N, L)
    m, k, n = prod.m, prod.k, prod.n
    blk = ctx.default_blocking(m, k, n, prod.share_weights)
    X = S.uniform_share((m, k), S.SEED_X)
    W = S.uniform_share((k, n), S.SEED_W) if prod.share_weights else S.fixed_point_weights((k, n), S.SEED_W)
    s = O.keygen(P, S.SEED_KEY)
    ct_in = O.encrypt(P, s, O.pack_input(X, blk, N), S.SEED_ENC)
    pt = B.he_encode_weights(ctx, to_dev(W), k, n, blk)
    out = to_np(B.he_matmul(ctx, to_dev(ct_in), pt, m, k, n, blk, S.SEED_MASK))
    nI, nJ, nLb = O.blocks(m, k, n, blk)
    total = nI * nLb
    rng = np.random.default_rng(11)
    sel = sorted({0, total - 1, *map(int, rng.integers(0, total, 2))})
    want = O.matmul(P, ct_in, W, m, k, n, blk, S.SEED_MASK, sel=sel)
    got = out.reshape(total, 2, L, N)[sel]
    assert np.array_equal(got, want)
    dec, _ = O.decrypt(P, s, want)
    m_b, k_b, n_b = blk
    ref = O.plain_matmul_mod_t(X, W, P.t)
    for row, o in enumerate(sel):
        Lb, I = divmod(o, nI)
        mask = O.mask_poly(P, S.SEED_MASK, o)
        for l in range(min(m_b, m - Lb * m_b)):
            for i in range(min(n_b, n - I * n_b)):
                pos = l * n_b * k_b + i * k_b + k_b - 1
                assert (int(dec[row][pos]) + int(mask[pos])) % P.t == int(ref[Lb * m_b + l, I * n_b + i])


# ------------------------------------------------------------------ same-shape batches


@pytest.mark.parametrize("N,L,m,k,n,blk", [(4096, 2, 128, 64, 128, (64, 8, 8)), (1024, 2, 9, 30, 17, (4, 8, 8)),
                                           (256, 2, 5, 7, 3, (2, 4, 4))])
def test_matmul_batch_equals_single_calls_and_oracle(B, N, L, m, k, n, blk):
    ctx, P = ctx_for(B, N, L)
    batch = 3
    s = O.keygen(P, S.SEED_KEY)
    Xs = [S.uniform_share((m, k), 60 + b) for b in range(batch)]
    Ws = [S.uniform_share((k, n), 70 + b) for b in range(batch)]
    cts = [O.encrypt(P, s, O.pack_input(X, blk, N), 80 + b) for b, X in enumerate(Xs)]
    si = ctx.sizes(m, k, n, blk)
    pt = B.he_encode_weights_batch(ctx, to_dev(np.stack(Ws)), k, n, blk, batch)
    for b in range(batch):  # batched encode == single encodes
        single = B.he_encode_weights(ctx, to_dev(Ws[b]), k, n, blk)
        assert torch.equal(pt[b * si["pt_words"]:(b + 1) * si["pt_words"]], single)
    out = to_np(B.he_matmul_batch(ctx, to_dev(np.stack(cts)), pt, m, k, n, blk, batch, 500))
    ow = si["out_words"]
    for b in range(batch):
        single = to_np(B.he_matmul(ctx, to_dev(cts[b]), pt[b * si["pt_words"]:(b + 1) * si["pt_words"]], m, k, n,
                                   blk, 500 + b))
        assert np.array_equal(out[b * ow:(b + 1) * ow], single)
    want = O.matmul(P, cts[1], Ws[1], m, k, n, blk, 501)
    assert np.array_equal(out[ow:2 * ow].reshape(want.shape), want)


# ------------------------------------------------------------------ compact output (HE_DROP_C0)


@pytest.mark.parametrize("N,L,m,k,n,blk,batch", [
    (4096, 2, 16, 64, 64, (8, 32, 16), 1),
    (4096, 2, 9, 70, 37, (4, 32, 32), 1),
    (1024, 2, 7, 20, 9, (4, 8, 16), 2),
    (64, 2, 5, 6, 7, (2, 4, 8), 1),
    (8192, 3, 7, 33, 20, (8, 32, 32), 1),
    (4096, 2, 3, 5, 2, (1, 1, 1), 1),
    (4096, 2, 2, 300, 3, (1, 256, 16), 1),
    (4096, 2, 12, 40, 30, (4, 16, 8), 2),
    (4096, 2, 10, 9, 50, (8, 2, 64), 1),
    (8192, 3, 20, 50, 40, (16, 16, 32), 1),
])
def test_matmul_compact_c0(B, N, L, m, k, n, blk, batch):
    """With HE_DROP_C0 the output keeps c1 and c0 only at the decoded coefficients
    e = i k_b + k_b - 1 (Sec. 3.1.3); every kept word equals the oracle's full output, and
    the client's expand + decrypt + unpack plus the server's unmask give X W mod t."""
    ctx, P = ctx_for(B, N, L)
    s = O.keygen(P, S.SEED_KEY)
    Xs = [S.uniform_share((m, k), 90 + b) for b in range(batch)]
    Ws = [S.fixed_point_weights((k, n), 95 + b) for b in range(batch)]
    cts = [O.encrypt(P, s, O.pack_input(X, blk, N), 97 + b) for b, X in enumerate(Xs)]
    pt = B.he_encode_weights_batch(ctx, to_dev(np.stack(Ws)), k, n, blk, batch)
    out = B.he_matmul_batch(ctx, to_dev(np.stack(cts)), pt, m, k, n, blk, batch, 700, flags=B.HE_DROP_C0)
    si = ctx.sizes(m, k, n, blk)
    kb, out_cts, ow = blk[1], si["out_cts"], si["out_words_compact"]
    Nc = N // kb
    assert ow == out_cts * L * (Nc + N)
    got_all = to_np(out)
    sk = B.he_keygen(ctx, S.SEED_KEY)
    for b in range(batch):
        want = O.matmul(P, cts[b], Ws[b], m, k, n, blk, 700 + b)
        got = got_all[b * ow:(b + 1) * ow].reshape(out_cts, L * (Nc + N))
        assert np.array_equal(got[:, L * Nc:].reshape(out_cts, L, N), want[:, 1])
        assert np.array_equal(got[:, :L * Nc].reshape(out_cts, L, Nc), want[:, 0, :, kb - 1::kb])
        full = B.he_expand_compact(ctx, out[b * ow:(b + 1) * ow], out_cts, kb)
        dec, _ = B.he_decrypt(ctx, sk, full)
        client = to_np(B.he_unpack_output(ctx, dec, m, n, blk), (m, n))
        server = to_np(B.he_unmask(ctx, 700 + b, m, n, blk), (m, n))
        assert np.array_equal((client + server) % np.uint64(P.t), O.plain_matmul_mod_t(Xs[b], Ws[b], P.t))


# ------------------------------------------------------------------ failure detection


def test_bounded_wait_reports_timeout_and_context_survives(B):
    """A kernel wait that can never complete gives up after its limit, the host reads
    HE_ETIMEOUT through he_device_status, the flag clears, and the context keeps working."""
    ctx, P = ctx_for(B, 4096, 2)
    B.he_device_status(ctx)  # clean
    B.he_test_wait_timeout(ctx, 50)
    with pytest.raises(B.HEError) as e:
        B.he_device_status(ctx)
    assert e.value.code == B.HE_ETIMEOUT
    B.he_device_status(ctx)  # cleared
    X = S.uniform_share((16, 64), S.SEED_X)
    W = S.fixed_point_weights((64, 64), S.SEED_W)
    _run_case(B, 4096, 2, 16, 64, 64, (8, 32, 16), W, X)
    B.he_device_status(ctx)


# ------------------------------------------------------------------ multi-product launch


@pytest.mark.parametrize("N,L", [(4096, 2), (256, 2), (8192, 3)])
def test_matmul_multi_equals_single_calls(B, N, L):
    """Products of different shapes, blockings and output modes in one multi-product launch
    give exactly what their own he_matmul calls give (and one matches the oracle)."""
    ctx, P = ctx_for(B, N, L)
    s = O.keygen(P, S.SEED_KEY)
    sk = B.he_keygen(ctx, S.SEED_KEY)
    shapes = [(16, 64, 64, None, 0), (9, 70, 37, None, B.HE_DROP_C0), (128, 64, 128, None, B.HE_DROP_C0),
              (5, 7, 3, (1, 1, 1), 0), (33, 100, 20, None, 0), (0, 5, 5, (1, 1, 1), 0)]
    items, singles, oracle_case = [], [], None
    for idx, (m, k, n, blk, flags) in enumerate(shapes):
        blk = blk or ctx.default_blocking(max(m, 1), k, n)
        si = ctx.sizes(m, k, n, blk)
        X = S.uniform_share((m, k), 300 + idx)
        W = S.fixed_point_weights((k, n), 400 + idx)
        ct_in = B.he_encrypt(ctx, sk, B.he_pack_input(ctx, to_dev(X), m, k, blk), 500 + idx) if m else ctx.empty(1)
        pt = B.he_encode_weights(ctx, to_dev(W), k, n, blk)
        ow = si["out_words_compact"] if flags else si["out_words"]
        items.append(dict(ct_in=ct_in, pt=pt, ct_out=ctx.empty(max(ow, 1)), m=m, k=k, n=n, blk=blk, flags=flags,
                          mask_seed=600 + idx))
        if m:
            singles.append(to_np(B.he_matmul(ctx, ct_in, pt, m, k, n, blk, 600 + idx, flags=flags)))
        else:
            singles.append(None)
        if idx == 0:
            oracle_case = (X, W, m, k, n, blk)
    prods = B.make_products(items)
    ws = ctx.empty(max(B.he_multi_workspace_bytes(ctx, prods) // 8 + 1, 1))
    B.he_matmul_multi(ctx, prods, ws)
    for it, single in zip(items, singles):
        if single is not None:
            assert np.array_equal(to_np(it["ct_out"])[:single.size], single)
    X, W, m, k, n, blk = oracle_case
    ct_or = O.encrypt(P, s, O.pack_input(X, blk, N), 500)
    assert np.array_equal(to_np(items[0]["ct_in"]), ct_or.reshape(-1))
    want = O.matmul(P, ct_or, W, m, k, n, blk, 600)
    assert np.array_equal(to_np(items[0]["ct_out"]), want.reshape(-1))


def test_matmul_host_async_two_streams(B):
    """HE_ASYNC host-buffer calls on two streams (own workspaces) equal the device-buffer path."""
    ctx, P = ctx_for(B, 4096, 2)
    sk = B.he_keygen(ctx, 3)
    outs, refs, keep = [], [], []
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    for i, (m, k, n) in enumerate([(16, 64, 64), (40, 96, 48), (8, 256, 32)]):
        blk = ctx.default_blocking(m, k, n)
        X = S.uniform_share((m, k), 900 + i)
        W = S.fixed_point_weights((k, n), 910 + i)
        ct = B.he_encrypt(ctx, sk, B.he_pack_input(ctx, to_dev(X), m, k, blk), 920 + i)
        pt = B.he_encode_weights(ctx, to_dev(W), k, n, blk)
        flags = B.HE_DROP_C0 if i % 2 else B.HE_FLAGS_NONE
        refs.append(to_np(B.he_matmul(ctx, ct, pt, m, k, n, blk, 930 + i, flags=flags)))
        si = ctx.sizes(m, k, n, blk)
        ow = si["out_words_compact"] if flags else si["out_words"]
        host_in = ct.cpu().pin_memory()
        host_out = torch.zeros(ow, dtype=torch.int64).pin_memory()
        ws = ctx.empty(B.matmul_host_workspace_words(ctx, m, k, n, blk, flags))
        torch.cuda.synchronize()
        B.he_matmul_host(ctx, host_in, pt, m, k, n, blk, 930 + i, host_out, ws, flags=flags | B.HE_ASYNC,
                         stream=streams[i % 2])
        outs.append(host_out)
        keep += [host_in, ws]
    for s_ in streams:
        s_.synchronize()
    for o, r in zip(outs, refs):
        assert np.array_equal(o.numpy().view(np.uint64), r)


def test_matmul_multi_host_buffers(B):
    """he_matmul_multi_host (host ct_in / ct_out, pinned) equals he_matmul_multi on device
    buffers, synchronously and with HE_ASYNC calls on two streams."""
    ctx, P = ctx_for(B, 4096, 2)
    sk = B.he_keygen(ctx, 3)
    shapes = [(16, 64, 64, 0), (40, 96, 48, B.HE_DROP_C0), (9, 70, 37, B.HE_DROP_C0), (0, 5, 5, 0)]
    dev_items, host_items = [], []
    for i, (m, k, n, flags) in enumerate(shapes):
        blk = ctx.default_blocking(max(m, 1), k, n)
        si = ctx.sizes(m, k, n, blk)
        ow = si["out_words_compact"] if flags else si["out_words"]
        X = S.uniform_share((m, k), 40 + i)
        W = S.fixed_point_weights((k, n), 50 + i)
        ct = B.he_encrypt(ctx, sk, B.he_pack_input(ctx, to_dev(X), m, k, blk), 60 + i) if m else ctx.empty(1)
        pt = B.he_encode_weights(ctx, to_dev(W), k, n, blk)
        dev_items.append(dict(ct_in=ct, pt=pt, ct_out=ctx.empty(max(ow, 1)), m=m, k=k, n=n, blk=blk, flags=flags,
                              mask_seed=70 + i))
        host_items.append(dict(dev_items[-1], ct_in=ct.cpu().pin_memory(),
                               ct_out=torch.zeros(max(ow, 1), dtype=torch.int64).pin_memory()))
    prods = B.make_products(dev_items)
    B.he_matmul_multi(ctx, prods, ctx.empty(B.he_multi_workspace_bytes(ctx, prods) // 8 + 1))
    hprods = B.make_products(host_items)
    need = B.he_multi_host_workspace_bytes(ctx, hprods)
    B.he_matmul_multi_host(ctx, hprods, ctx.empty(need // 8 + 1))
    for d, h in zip(dev_items, host_items):
        if d["m"]:  # an empty product writes nothing
            assert np.array_equal(to_np(d["ct_out"]), h["ct_out"].numpy().view(np.uint64))
    # two asynchronous calls in flight on two streams, each with its own workspace and outputs
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = []
    for st in streams:
        items = [dict(h, ct_out=torch.zeros_like(h["ct_out"]).pin_memory()) for h in host_items]
        pr = B.make_products(items)
        ws = ctx.empty(need // 8 + 1)
        B.he_matmul_multi_host(ctx, pr, ws, flags=B.HE_ASYNC, stream=st)
        outs.append((items, pr, ws))
    for st in streams:
        st.synchronize()
    for items, _, _ in outs:
        for d, h in zip(dev_items, items):
            if d["m"]:
                assert np.array_equal(to_np(d["ct_out"]), h["ct_out"].numpy().view(np.uint64))


def test_multi_launch_keeps_each_clients_key(B):
    """Requests of three clients, each with its own secret key, in one multi-product launch
    (Sec. 3.1.1: the server's product needs no key): each client decrypts its own output
    with its own key, and with the server's mask share gets its X W mod t; another client's
    key does not."""
    ctx, P = ctx_for(B, 4096, 2)
    t = np.uint64(P.t)
    items, clients = [], []
    for c, (m, k, n, flags) in enumerate([(16, 64, 64, 0), (40, 96, 48, B.HE_DROP_C0), (9, 70, 37, 0)]):
        blk = ctx.default_blocking(m, k, n)
        sk = B.he_keygen(ctx, 1000 + c)
        X = S.uniform_share((m, k), 1100 + c)
        W = S.fixed_point_weights((k, n), 1200 + c)
        ct = B.he_encrypt(ctx, sk, B.he_pack_input(ctx, to_dev(X), m, k, blk), 1300 + c)
        pt = B.he_encode_weights(ctx, to_dev(W), k, n, blk)
        si = ctx.sizes(m, k, n, blk)
        items.append(dict(ct_in=ct, pt=pt, ct_out=ctx.empty(si["out_words_compact"] if flags else si["out_words"]),
                          m=m, k=k, n=n, blk=blk, flags=flags, mask_seed=1400 + c))
        clients.append((sk, X, W, blk, si, flags))
    prods = B.make_products(items)
    B.he_matmul_multi(ctx, prods, ctx.empty(B.he_multi_workspace_bytes(ctx, prods) // 8 + 1))
    for c, (it, (sk, X, W, blk, si, flags)) in enumerate(zip(items, clients)):
        m, n = it["m"], it["n"]
        out = it["ct_out"]
        if flags:
            out = B.he_expand_compact(ctx, out, si["out_cts"], blk[1])
        server = to_np(B.he_unmask(ctx, 1400 + c, m, n, blk), (m, n))
        want = O.plain_matmul_mod_t(X, W, P.t)
        dec, _ = B.he_decrypt(ctx, sk, out)
        client = to_np(B.he_unpack_output(ctx, dec, m, n, blk), (m, n))
        assert np.array_equal((client + server) % t, want), c
        other = clients[(c + 1) % len(clients)][0]
        dec_o, _ = B.he_decrypt(ctx, other, out)
        client_o = to_np(B.he_unpack_output(ctx, dec_o, m, n, blk), (m, n))
        assert not np.array_equal((client_o + server) % t, want), c
