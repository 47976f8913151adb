"""he_matmul_noalloc: the product for callers that cannot allocate device memory.

Some callers cannot hand the library a workspace -- e.g. a serving process whose
device memory is already reserved by another allocator, or a host program that is
not allowed to manage device memory.  he_matmul_noalloc uses a fixed scratch array
inside the library instead.  Its results must equal he_matmul's bit for bit (the
tolerance of every other parity test here), on consecutive calls that share that
scratch, and it must refuse products larger than the scratch.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from gpu_util import need_gpu, to_dev, to_np
from paper_2305_18396_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    need_gpu()
    from paper_2305_18396_gb300 import binding as B

    ctx = B.Context(4096, 2)
    sk = B.he_keygen(ctx, S.SEED_KEY)
    return B, ctx, sk


def _inputs(B, ctx, sk, m, k, n, seed):
    blk = ctx.default_blocking(m, k, n)
    X = S.uniform_share((m, k), seed)
    W = S.uniform_share((k, n), seed + 1)
    ct = B.he_encrypt(ctx, sk, B.he_pack_input(ctx, to_dev(X), m, k, blk), seed + 2)
    pt = B.he_encode_weights(ctx, to_dev(W), k, n, blk)
    return blk, ct, pt


def _noalloc(B, ctx, ct, pt, m, k, n, blk, seed):
    """Call the entry point through the C ABI with caller-owned input and output buffers."""
    out = ctx.empty(ctx.sizes(m, k, n, blk)["out_words"])
    rc = B.lib.he_matmul_noalloc(ctx.h, B._ptr(ct), B._ptr(pt), m, k, n, B._blk(blk), seed, 0, B._ptr(out),
                                 B._stream(None))
    assert rc == B.HE_OK, B.lib.he_last_error().decode()
    return out


def test_noalloc_matches_matmul_on_consecutive_calls(setup):
    """Shapes whose default blocking fits the scratch give he_matmul's words on two calls in a
    row; a shape whose default blocking does not (its workspace depends on the engine's
    layout) is refused."""
    B, ctx, sk = setup
    shapes = [(128, 64, 128), (16, 64, 64), (128, 256, 256), (128, 768, 768)]
    compared = 0
    for i, (m, k, n) in enumerate(shapes):
        blk, ct, pt = _inputs(B, ctx, sk, m, k, n, 40 + 10 * i)
        if ctx.sizes(m, k, n, blk)["workspace_bytes"] > B.HE_NOALLOC_SCRATCH_BYTES:
            out = ctx.empty(ctx.sizes(m, k, n, blk)["out_words"])
            rc = B.lib.he_matmul_noalloc(ctx.h, B._ptr(ct), B._ptr(pt), m, k, n, B._blk(blk), 99, 0, B._ptr(out),
                                         B._stream(None))
            assert rc == B.HE_EINVAL
            continue
        ref = to_np(B.he_matmul(ctx, ct, pt, m, k, n, blk, 99))
        first = to_np(_noalloc(B, ctx, ct, pt, m, k, n, blk, 99))
        second = to_np(_noalloc(B, ctx, ct, pt, m, k, n, blk, 99))
        assert np.array_equal(first, ref)
        assert np.array_equal(second, ref)
        compared += 1
    assert compared >= 2


def test_noalloc_compact_output_through_the_binding(setup):
    """HE_DROP_C0 through the Python wrapper: the same words as he_matmul with that flag, on
    two calls in a row."""
    B, ctx, sk = setup
    m, k, n = 64, 256, 192
    blk, ct, pt = _inputs(B, ctx, sk, m, k, n, 70)
    si = ctx.sizes(m, k, n, blk)
    assert si["workspace_bytes_compact"] <= B.HE_NOALLOC_SCRATCH_BYTES
    ref = to_np(B.he_matmul(ctx, ct, pt, m, k, n, blk, 7, flags=B.HE_DROP_C0))
    for _ in range(2):
        out = ctx.empty(si["out_words_compact"])
        B.he_matmul_noalloc(ctx, ct, pt, m, k, n, blk, 7, out, flags=B.HE_DROP_C0)
        assert np.array_equal(to_np(out), ref)


def test_noalloc_rejects_products_beyond_its_scratch(setup):
    B, ctx, sk = setup
    m, k, n = 128, 768, 2304  # the QKV product needs more scratch than the array holds
    blk = ctx.default_blocking(m, k, n)
    si = ctx.sizes(m, k, n, blk)
    assert si["workspace_bytes"] > B.HE_NOALLOC_SCRATCH_BYTES
    ct = ctx.empty(si["in_words"])
    pt = ctx.empty(si["pt_words"])
    out = ctx.empty(si["out_words"])
    rc = B.lib.he_matmul_noalloc(ctx.h, B._ptr(ct), B._ptr(pt), m, k, n, B._blk(blk), 1, 0, B._ptr(out),
                                 B._stream(None))
    assert rc == B.HE_EINVAL
    assert "scratch" in B.lib.he_last_error().decode()
