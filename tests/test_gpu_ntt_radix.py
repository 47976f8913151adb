"""Every transform radix reproduces the oracle bit for bit; the radix tuner selects a built one.

The register-blocked transforms are built with 8, 16 and 32 values per thread at N = 4096
and 8192 (he_set_ntt_radix; 16 elsewhere).  For each radix the forward transform must put
the oracle's evaluations in the library's slot order and the inverse must undo it, and
the output ciphertexts of full-output and compact-output products, computed one by one and
in one multi-product launch, must equal the oracle's (these run the weight encoding, the
forward transforms, the multiply-accumulate and the inverse transforms of that radix).
The encoder skips its first transform pass when a weight block's nonzero coefficients fit
in N / 2^RS0 (RS0 = the stages of that pass).  The first case's blocks fill N/8 = 512
coefficients at N = 4096, where RS0 is 3 for 8 values per thread and 2 for 32 (skipped
pass) and 4 for 16 (full pass), so both paths are covered.
"""
import numpy as np
import pytest

import oracle as O
from gpu_util import need_gpu, to_dev, to_np
from paper_2305_18396_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

CASES = {  # (N, L): [(m, k, n, blocking, compact)]
    (4096, 2): [(16, 64, 64, (8, 32, 16), False), (9, 70, 37, (4, 32, 32), True)],
    (8192, 3): [(7, 33, 20, (8, 32, 32), False), (20, 50, 40, (16, 16, 32), True)],
}
_STATE = {}


@pytest.fixture(scope="module")
def B():
    need_gpu()
    from paper_2305_18396_gb300 import binding

    return binding


def setup(B, N, L):
    """Context, oracle parameters and, per case, the oracle's input and output (computed once)."""
    if (N, L) not in _STATE:
        ctx, P = B.Context(N, L), O.Params(N, L)
        s = O.keygen(P, S.SEED_KEY)
        cases = []
        for idx, (m, k, n, blk, compact) in enumerate(CASES[(N, L)]):
            X = S.uniform_share((m, k), 40 + idx)
            W = S.fixed_point_weights((k, n), 50 + idx)
            ct = O.encrypt(P, s, O.pack_input(X, blk, N), 60 + idx)
            cases.append((m, k, n, blk, compact, W, ct, 70 + idx, O.matmul(P, ct, W, m, k, n, blk, 70 + idx)))
        _STATE[(N, L)] = (ctx, P, cases)
    return _STATE[(N, L)]


def check_output(B, P, got, want, blk, compact, out_cts):
    L, N = P.L, P.N
    if not compact:
        assert np.array_equal(got.reshape(want.shape), want)
        return
    kb = blk[1]
    Nc = N // kb
    g = got.reshape(out_cts, L * (Nc + N))
    assert np.array_equal(g[:, L * Nc:].reshape(out_cts, L, N), want[:, 1])
    assert np.array_equal(g[:, :L * Nc].reshape(out_cts, L, Nc), want[:, 0, :, kb - 1::kb])


@pytest.mark.parametrize("N,L", list(CASES))
@pytest.mark.parametrize("logr", [3, 4, 5])
def test_radix_matches_oracle(B, N, L, logr):
    ctx, P, cases = setup(B, N, L)
    ctx.set_ntt_radix(logr)
    assert ctx.ntt_radix == logr
    try:
        # transforms: slot j of the forward transform is a(psi^(2 brev(j) + 1)), psi the library's
        rng = np.random.default_rng(5 + logr)
        a = np.stack([rng.integers(0, q, size=N, dtype=np.uint64) for q in P.q])[None]
        t = to_dev(a)
        B.he_ntt_forward(ctx, t)
        got = to_np(t, a.shape)
        ref = O.ntt_forward(P, a)
        psi_gpu = ctx.params()["psi"]
        logN = N.bit_length() - 1
        brev = np.array([int(format(j, f"0{logN}b")[::-1], 2) for j in range(N)])
        for li, q in enumerate(P.q):
            u = next(e for e in range(1, 2 * N, 2) if pow(P.psi[li], e, q) == psi_gpu[li])
            kidx = ((u * (2 * brev + 1)) % (2 * N) - 1) // 2
            assert np.array_equal(got[0, li], ref[0, li][kidx])
        B.he_ntt_inverse(ctx, t)
        assert np.array_equal(to_np(t, a.shape), a)

        # products one by one, then all in one multi-product launch
        items = []
        for m, k, n, blk, compact, W, ct, seed, want in cases:
            flags = B.HE_DROP_C0 if compact else 0
            si = ctx.sizes(m, k, n, blk)
            pt = B.he_encode_weights(ctx, to_dev(W), k, n, blk)
            ct_d = to_dev(ct)
            out = B.he_matmul(ctx, ct_d, pt, m, k, n, blk, seed, flags=flags)
            check_output(B, P, to_np(out), want, blk, compact, si["out_cts"])
            ow = si["out_words_compact"] if compact else si["out_words"]
            items.append(dict(ct_in=ct_d, pt=pt, ct_out=ctx.empty(ow), m=m, k=k, n=n, blk=blk, flags=flags,
                              mask_seed=seed))
        prods = B.make_products(items)
        B.he_matmul_multi(ctx, prods, ctx.empty(B.he_multi_workspace_bytes(ctx, prods) // 8 + 1))
        for it, (m, k, n, blk, compact, W, ct, seed, want) in zip(items, cases):
            check_output(B, P, to_np(it["ct_out"]), want, blk, compact, ctx.sizes(m, k, n, blk)["out_cts"])
        B.he_device_status(ctx)
    finally:
        ctx.set_ntt_radix(4)


def test_radix_tuner_selects_a_built_radix(B):
    ctx, P, cases = setup(B, 4096, 2)
    try:
        chosen, ms = ctx.autotune_ntt_radix()
        assert chosen in (3, 4, 5) and ctx.ntt_radix == chosen
        assert set(ms) == {3, 4, 5} and all(v > 0 for v in ms.values())
        best = min(ms, key=ms.get)  # the fastest, unless the default is within 5% of it
        assert chosen == best or (chosen == 4 and ms[best] > 0.95 * ms[4])
        assert chosen == 4 or ms[chosen] <= 0.95 * ms[4]
        m, k, n, blk, compact, W, ct, seed, want = cases[0]
        out = B.he_matmul(ctx, to_dev(ct), B.he_encode_weights(ctx, to_dev(W), k, n, blk), m, k, n, blk, seed)
        check_output(B, P, to_np(out), want, blk, compact, ctx.sizes(m, k, n, blk)["out_cts"])
    finally:
        ctx.set_ntt_radix(4)


def test_radix_not_built_is_rejected(B):
    ctx, _, _ = setup(B, 4096, 2)
    for bad in (0, 2, 6):
        with pytest.raises(B.HEError):
            ctx.set_ntt_radix(bad)
    assert ctx.ntt_radix == 4
    small = B.Context(1024, 2)
    small.set_ntt_radix(4)
    with pytest.raises(B.HEError):
        small.set_ntt_radix(3)
    chosen, ms = small.autotune_ntt_radix()
    assert chosen == 4 and set(ms) == {4}
    tiny = B.Context(64, 2)
    with pytest.raises(B.HEError):
        tiny.set_ntt_radix(5)
    assert tiny.autotune_ntt_radix() == (4, {})
