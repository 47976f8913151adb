"""Continuous batching: every request's result is the same alone and in the mix, and
equals the oracle's.

Requests of different matrices and sequence lengths are served through the
continuous-batching loop (several multi-product launches in flight, admission by a
device-memory budget); each output must equal, bit for bit, the output of the same
request run alone through he_matmul.  With the clients' ciphertexts made by the oracle,
every served output (compact form, Sec. 3.1.3) must also equal the oracle's Pi_MatMul
(Algorithm 1 step 3 with the request's mask seed) word for word, and the client's
decryption plus the server's unmask must give X W mod t.
"""
import numpy as np
import pytest

from gpu_util import need_gpu, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    need_gpu()
    from paper_2305_18396_gb300 import binding as B
    from paper_2305_18396_gb300 import serving as SV

    ctx = B.Context(4096, 2)
    models = SV.make_models(ctx, [("a", 64, 64, 64), ("b", 128, 96, 40), ("c", 256, 32, 96)])
    return B, SV, ctx, models


@pytest.mark.parametrize("budget,slots", [(32 << 30, 2), (40 << 20, 1)])
def test_served_results_equal_alone(env, budget, slots):
    B, SV, ctx, models = env
    reqs = SV.make_requests(models, 24, rate=2000.0, seed=9, m_lo=1, m_hi=96)
    stats, done = SV.run_served(ctx, models, reqs, hbm_budget=budget, slots=slots)
    assert len(done) == len(reqs) and stats["launches"] >= 1
    by = {m.name: m for m in models}
    for r in done:
        mm = by[r.model]
        alone = B.he_matmul(ctx, mm.ct_pool, mm.pt, r.m, mm.k, mm.n, mm.blk, r.mask_seed, flags=B.HE_DROP_C0)
        assert np.array_equal(to_np(r.out), to_np(alone)), r.rid


def test_per_request_path_matches(env):
    B, SV, ctx, models = env
    reqs = SV.make_requests(models, 6, rate=5000.0, seed=10, m_lo=1, m_hi=64)
    stats, done = SV.run_per_request(ctx, models, reqs)
    by = {m.name: m for m in models}
    for r in done:
        mm = by[r.model]
        alone = B.he_matmul(ctx, mm.ct_pool, mm.pt, r.m, mm.k, mm.n, mm.blk, r.mask_seed, flags=B.HE_DROP_C0)
        assert np.array_equal(to_np(r.out), to_np(alone))
    assert stats["p99_ms"] >= stats["p50_ms"] > 0


def test_served_outputs_equal_oracle(env):
    """Models whose input pools the oracle encrypted: each served compact output equals the
    oracle's words, and decrypt + unpack + unmask gives X W mod t for the request's rows."""
    B, SV, ctx, _ = env
    import oracle as O
    from gpu_util import to_dev
    from paper_2305_18396_gb300 import synthetic as S

    N, L = ctx.N, ctx.L
    P = O.Params(N, L)
    s = O.keygen(P, 71)
    specs = [("p", 96, 80, 48), ("q", 64, 200, 40)]
    models, plain = [], {}
    for i, (name, k, n, max_m) in enumerate(specs):
        blk = ctx.default_blocking(128, k, n)
        W = S.fixed_point_weights((k, n), 300 + i)
        X = S.uniform_share((max_m, k), 400 + i)
        ct = O.encrypt(P, s, O.pack_input(X, blk, N), 500 + i)
        pt = B.he_encode_weights(ctx, to_dev(W), k, n, blk)
        models.append(SV.Model(name, k, n, blk, pt, to_dev(ct), max_m))
        plain[name] = (X, W, ct)
    reqs = SV.make_requests(models, 12, rate=3000.0, seed=12, m_lo=1, m_hi=48)
    stats, done = SV.run_served(ctx, models, reqs, slots=2)
    assert len(done) == len(reqs) and stats["failed"] == 0
    by = {m.name: m for m in models}
    for r in done:
        mm = by[r.model]
        X, W, ct = plain[r.model]
        nI, nJ, nLb = O.blocks(r.m, mm.k, mm.n, mm.blk)
        want = O.matmul(P, ct[:nLb * nJ], W, r.m, mm.k, mm.n, mm.blk, r.mask_seed)
        kb = mm.blk[1]
        Nc = N // kb
        got = to_np(r.out).reshape(nLb * nI, L * (Nc + N))
        assert np.array_equal(got[:, L * Nc:].reshape(-1, L, N), want[:, 1]), r.rid
        assert np.array_equal(got[:, :L * Nc].reshape(-1, L, Nc), want[:, 0, :, kb - 1::kb]), r.rid
        dec, budget = O.decrypt(P, s, want)
        assert (budget > 0).all()
        client = O.unpack_output(dec, r.m, mm.n, mm.blk)
        server = O.unmask(P, r.mask_seed, r.m, mm.n, mm.blk)
        assert np.array_equal((client + server) % np.uint64(P.t), O.plain_matmul_mod_t(X[:r.m], W, P.t)), r.rid
