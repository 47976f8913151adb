"""The measured blocking choice (he_autotune_blocking).

It times the cost model's best candidates on pseudo-random data; the tests check its
contract (size query, scratch check, the returned blocking is one the model ranks among
its candidates, a positive time, at least as fast as the model's first choice within
timing noise) and that a product run with the tuned blocking still matches the oracle
bit for bit and decrypts to X W.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from gpu_util import need_gpu, to_dev, to_np
from paper_2305_18396_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    need_gpu()
    from paper_2305_18396_gb300 import binding as B

    return B, B.Context(4096, 2)


@pytest.mark.parametrize("m,k,n,wpc,flags,batch", [(128, 768, 768, False, 1, 1), (128, 64, 128, True, 1, 12),
                                                   (16, 64, 64, False, 0, 1)])
def test_autotune_contract(env, m, k, n, wpc, flags, batch):
    B, ctx = env
    blk, ms = ctx.autotune_blocking(m, k, n, wpc, flags, batch)
    assert ms > 0
    assert blk[0] * blk[1] * blk[2] <= ctx.N
    if flags:
        assert blk[1] & (blk[1] - 1) == 0
    # with one candidate the tuner times the model's own choice; the tuned one is no slower
    # (25% slack for timing noise)
    first, ms_model = ctx.autotune_blocking(m, k, n, wpc, flags, batch, candidates=1)
    assert first == ctx.default_blocking(m, k, n, wpc)
    assert ms <= ms_model * 1.25


def test_autotune_scratch_checks(env):
    B, ctx = env
    need = ctypes.c_size_t(0)
    b = B.Blocking()
    ms = ctypes.c_float(0)
    rc = B.lib.he_autotune_blocking(ctx.h, 64, 256, 128, 0, 0, 1, 4, None, 0, ctypes.byref(need), ctypes.byref(b),
                                    ctypes.byref(ms), None)
    assert rc == 0 and need.value > 0
    small = ctx.empty(16)
    rc = B.lib.he_autotune_blocking(ctx.h, 64, 256, 128, 0, 0, 1, 4, ctypes.c_void_p(small.data_ptr()), 128, None,
                                    ctypes.byref(b), ctypes.byref(ms), None)
    assert rc == 2  # HE_ENOMEM
    rc = B.lib.he_autotune_blocking(ctx.h, 64, 256, 128, 0, 8, 1, 4, None, 0, ctypes.byref(need), ctypes.byref(b),
                                    ctypes.byref(ms), None)
    assert rc == 1  # HE_EINVAL: unknown flags
    B.he_device_status(ctx)


def test_tuned_blocking_product_matches_oracle(env):
    B, ctx = env
    m, k, n = 24, 96, 40
    blk, _ = ctx.autotune_blocking(m, k, n)
    P = O.Params(4096, 2)
    X = S.uniform_share((m, k), 1)
    W = S.fixed_point_weights((k, n), 2)
    s = O.keygen(P, 3)
    ct_in = O.encrypt(P, s, O.pack_input(X, blk, P.N), 4)
    pt = B.he_encode_weights(ctx, to_dev(W), k, n, blk)
    got = to_np(B.he_matmul(ctx, to_dev(ct_in), pt, m, k, n, blk, 5))
    want = O.matmul(P, ct_in, W, m, k, n, blk, 5)
    assert np.array_equal(got, want.reshape(-1))
    dec, _ = O.decrypt(P, s, want)
    share = (O.unpack_output(dec, m, n, blk) + O.unmask(P, 5, m, n, blk)) % np.uint64(P.t)
    assert np.array_equal(share, O.plain_matmul_mod_t(X, W, P.t))
