"""Server-local share products (Sec. 3.1.1) on the GPU against the oracle.

he_share_matmul computes (acc + X W + bias) mod t; he_unmask_acc adds the server's mask
share of a Pi_MatMul (optionally transposed).  Both are exact integer work: the bar is
bit-exactness with the oracle's definition on the same seeded inputs.  The layer tests
assemble a fully connected layer and an attention product from the library's calls and
check the server's share against the oracle's, and client + server = the plain result.
"""
import numpy as np
import pytest

import oracle as O
from gpu_util import need_gpu, to_dev, to_np
from paper_2305_18396_gb300 import synthetic as S

pytestmark = pytest.mark.gpu
T = np.uint64(1 << 37)


@pytest.fixture(scope="module")
def env():
    need_gpu()
    from paper_2305_18396_gb300 import binding as B

    return B, B.Context(4096, 2), O.Params(4096, 2)


# sizes: single element, ragged tiles, split-k (small m n, long k), BERT-base FFN2 / QKV
@pytest.mark.parametrize("m,k,n", [(1, 1, 1), (5, 7, 3), (65, 17, 130), (16, 3000, 24), (128, 3072, 768),
                                   (128, 768, 2304), (200, 64, 1)])
def test_share_matmul_bit_exact(env, m, k, n):
    B, ctx, P = env
    X = S.uniform_share((m, k), 10 + m)
    W = S.uniform_share((k, n), 20 + n)
    bias = S.uniform_share((1, n), 30).reshape(n)
    acc = S.uniform_share((m, n), 40)
    want = O.share_matmul(X, W, bias, acc)
    got = B.he_share_matmul(ctx, to_dev(X), to_dev(W), m, k, n, bias=to_dev(bias), acc=to_dev(acc))
    assert np.array_equal(to_np(got, (m, n)), want)
    plain = B.he_share_matmul(ctx, to_dev(X), to_dev(W), m, k, n)
    assert np.array_equal(to_np(plain, (m, n)), O.share_matmul(X, W))


def test_share_matmul_edges(env):
    B, ctx, P = env
    m, n = 9, 11
    bias = S.uniform_share((1, n), 1).reshape(n)
    acc = S.uniform_share((m, n), 2)
    # k = 0: acc + bias
    got = B.he_share_matmul(ctx, None, None, m, 0, n, bias=to_dev(bias), acc=to_dev(acc))
    assert np.array_equal(to_np(got, (m, n)), (acc + bias) % T)
    # accumulate in place (acc aliases out), with the largest residues
    X = np.full((m, 33), int(T) - 1, dtype=np.uint64)
    W = np.full((33, n), int(T) - 1, dtype=np.uint64)
    buf = to_dev(acc)
    B.he_share_matmul(ctx, to_dev(X), to_dev(W), m, 33, n, acc=buf, out=buf)
    assert np.array_equal(to_np(buf, (m, n)), O.share_matmul(X, W, None, acc))
    # m = 0 or n = 0: nothing to do
    B.he_share_matmul(ctx, None, None, 0, 5, n)
    B.he_device_status(ctx)


@pytest.mark.parametrize("flags", [0, 4, 8, 12])
def test_unmask_acc(env, flags):
    B, ctx, P = env
    m, k, n, blk = 37, 64, 29, (8, 16, 16)
    base = S.uniform_share((n, m) if flags & 8 else (m, n), 7)
    buf = to_dev(base)
    B.he_unmask_acc(ctx, 99, m, n, blk, buf, flags=flags)
    share = O.unmask(P, 99, m, n, blk)
    if flags & 8:
        share = share.T
    want = (share + (base if flags & 4 else 0)) % T
    assert np.array_equal(to_np(buf, want.shape), want)
    # HE_UNMASK_ACCUMULATE alone on a zero buffer == he_unmask
    if flags == 0:
        assert np.array_equal(to_np(buf, (m, n)), to_np(B.he_unmask(ctx, 99, m, n, blk), (m, n)))


def test_fully_connected_layer_end_to_end(env):
    """Client: Pi_MatMul on its share, decrypted and unpacked on the device; server: its mask
    share + W<x>_1 + b, on the device.  Server share bit-exact vs the oracle's; the two
    shares sum to x W + b."""
    B, ctx, P = env
    m, k, n = 128, 768, 768
    blk = ctx.default_blocking(m, k, n)
    x0, x1 = S.uniform_share((m, k), 61), S.uniform_share((m, k), 62)
    W = S.fixed_point_weights((k, n), 63)
    b = S.uniform_share((1, n), 64).reshape(n)
    sk = B.he_keygen(ctx, 3)
    ct = B.he_encrypt(ctx, sk, B.he_pack_input(ctx, to_dev(x0), m, k, blk), 4)
    pt = B.he_encode_weights(ctx, to_dev(W), k, n, blk)
    out = B.he_matmul(ctx, ct, pt, m, k, n, blk, 5)
    dec, _ = B.he_decrypt(ctx, sk, out)
    y0 = to_np(B.he_unpack_output(ctx, dec, m, n, blk), (m, n))
    y1d = B.he_share_matmul(ctx, to_dev(x1), to_dev(W), m, k, n, bias=to_dev(b))
    B.he_unmask_acc(ctx, 5, m, n, blk, y1d)
    y1 = to_np(y1d, (m, n))
    assert np.array_equal(y1, O.share_matmul(x1, W, b, O.unmask(P, 5, m, n, blk)))
    x = (x0 + x1) % T
    assert np.array_equal((y0 + y1) % T, O.share_matmul(x, W, b))


def test_attention_server_share(env):
    """Server share of Z = X Y: <X>_1 <Y>_1 + mask share of cross term 1 + transposed mask
    share of cross term 2, assembled on the device, vs the oracle."""
    B, ctx, P = env
    m, k, n = 128, 64, 128
    X1, Y1 = S.uniform_share((m, k), 71), S.uniform_share((k, n), 72)
    blk1 = ctx.default_blocking(m, k, n, True)
    blk2 = ctx.default_blocking(n, k, m, True)
    z = B.he_share_matmul(ctx, to_dev(X1), to_dev(Y1), m, k, n)
    B.he_unmask_acc(ctx, 81, m, n, blk1, z, flags=B.HE_UNMASK_ACCUMULATE)
    B.he_unmask_acc(ctx, 82, n, m, blk2, z, flags=B.HE_UNMASK_ACCUMULATE | B.HE_UNMASK_TRANSPOSE)
    want = (O.share_matmul(X1, Y1) + O.unmask(P, 81, m, n, blk1) + O.unmask(P, 82, n, m, blk2).T) % T
    assert np.array_equal(to_np(z, (m, n)), want)


def test_share_matmul_batch_equals_items(env):
    """A batch of per-head sized products in one launch equals each item alone and the oracle."""
    B, ctx, P = env
    batch, m, k, n = 12, 128, 64, 128
    Xs = [S.uniform_share((m, k), 300 + b) for b in range(batch)]
    Ws = [S.uniform_share((k, n), 400 + b) for b in range(batch)]
    acc = S.uniform_share((batch * m, n), 500)
    got = B.he_share_matmul_batch(ctx, to_dev(np.stack(Xs)), to_dev(np.stack(Ws)), m, k, n, batch,
                                  acc=to_dev(acc))
    got = to_np(got, (batch, m, n))
    for b in range(batch):
        assert np.array_equal(got[b], O.share_matmul(Xs[b], Ws[b], None, acc[b * m:(b + 1) * m]))
    # split k across a batch (short outputs, long k), with a per-item bias
    batch, m, k, n = 3, 8, 2000, 16
    Xs = [S.uniform_share((m, k), 600 + b) for b in range(batch)]
    Ws = [S.uniform_share((k, n), 700 + b) for b in range(batch)]
    bias = S.uniform_share((batch, n), 800)
    got = to_np(B.he_share_matmul_batch(ctx, to_dev(np.stack(Xs)), to_dev(np.stack(Ws)), m, k, n, batch,
                                        bias=to_dev(bias)), (batch, m, n))
    for b in range(batch):
        assert np.array_equal(got[b], O.share_matmul(Xs[b], Ws[b], bias[b]))


@pytest.mark.parametrize("log2t", [20, 37, 40])
def test_share_matmul_other_plaintext_moduli(env, log2t):
    """t = 2^20 and 2^37 take the packed cross term, t = 2^40 the general one: both exact."""
    B, _, _ = env
    ctx = B.Context(1024, 2, log2t=log2t)
    t = 1 << log2t
    rng = np.random.default_rng(log2t)
    for m, k, n in [(33, 70, 65), (16, 1500, 8)]:
        X = rng.integers(0, t, size=(m, k), dtype=np.uint64)
        W = rng.integers(0, t, size=(k, n), dtype=np.uint64)
        X[0, :] = t - 1
        got = B.he_share_matmul(ctx, to_dev(X), to_dev(W), m, k, n)
        assert np.array_equal(to_np(got, (m, n)), O.share_matmul(X, W, log2t=log2t))
