"""The transfer pipeline (he_pipe): multi-product launches from host buffers with the
uploads, kernels and downloads of consecutive submits overlapped on three streams.

Every submit's outputs must equal the same products run by he_matmul_multi from device
buffers, bit for bit, whatever the pipe depth and however many submits share a slot; a
submit of more than 64 products runs as consecutive launches; the per-submit work the
caller enqueues on the pipe's compute stream (encoding the server's share) is ordered with
the launches; sampled outputs equal the oracle's Pi_MatMul of the oracle's encryptions.
"""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import need_gpu, to_dev, to_np
from paper_2305_18396_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    need_gpu()
    from paper_2305_18396_gb300 import binding as B

    N, L = 4096, 2
    ctx, P = B.Context(N, L), O.Params(N, L)
    s = O.keygen(P, S.SEED_KEY)
    return B, ctx, P, s


def _case(B, ctx, P, s, shapes, seed0):
    """Products of the given (m, k, n, blocking, flags): oracle inputs on the host (pinned),
    weights encoded on the device."""
    out = []
    for i, (m, k, n, blk, flags) in enumerate(shapes):
        X = S.uniform_share((m, k), seed0 + 3 * i)
        W = S.fixed_point_weights((k, n), seed0 + 3 * i + 1)
        ct = O.encrypt(P, s, O.pack_input(X, blk, P.N), seed0 + 3 * i + 2)
        si = ctx.sizes(m, k, n, blk)
        ow = si["out_words_compact"] if flags & B.HE_DROP_C0 else si["out_words"]
        out.append(dict(m=m, k=k, n=n, blk=blk, flags=flags, W=W, ct=ct, ow=ow,
                        pt=B.he_encode_weights(ctx, to_dev(W), k, n, blk),
                        in_h=torch.from_numpy(np.ascontiguousarray(ct, dtype=np.uint64).view(np.int64).reshape(-1))
                        .pin_memory()))
    torch.cuda.synchronize()  # the pipe's streams do not wait for the encodings on this stream
    return out


def _items(prods, outs, seeds, host):
    return [dict(ct_in=p["in_h"] if host else p["in_h"].cuda(), pt=p["pt"], ct_out=o, m=p["m"], k=p["k"], n=p["n"],
                 blk=p["blk"], flags=p["flags"], mask_seed=sd) for p, o, sd in zip(prods, outs, seeds)]


@pytest.mark.parametrize("depth", [1, 2, 3])
def test_pipe_submits_equal_device_launches(env, depth):
    B, ctx, P, s = env
    shapes = [(16, 64, 64, (8, 32, 16), 0), (9, 70, 37, (4, 32, 32), B.HE_DROP_C0),
              (20, 264, 200, (4, 8, 16), B.HE_DROP_C0)]
    prods = _case(B, ctx, P, s, shapes, 100)
    pipe = B.Pipe(ctx, depth=depth)
    steps = 5
    outs = [[torch.empty(p["ow"], dtype=torch.int64).pin_memory() for p in prods] for _ in range(steps)]
    arrs = [B.make_products(_items(prods, outs[t], [1000 * t + i for i in range(len(prods))], True))
            for t in range(steps)]
    ws = ctx.empty(pipe.workspace_bytes(arrs[0]) // 8 + 1)
    for t in range(steps):
        pipe.submit(arrs[t], ws)
    pipe.wait()
    B.he_device_status(ctx)
    for t in range(steps):
        dev_out = [ctx.empty(p["ow"]) for p in prods]
        arr = B.make_products(_items(prods, dev_out, [1000 * t + i for i in range(len(prods))], False))
        B.he_matmul_multi(ctx, arr, ctx.empty(B.he_multi_workspace_bytes(ctx, arr) // 8 + 1))
        for i in range(len(prods)):
            assert np.array_equal(outs[t][i].numpy().view(np.uint64), to_np(dev_out[i])), (t, i)
    # one product of the last step against the oracle
    p = prods[0]
    want = O.matmul(P, p["ct"], p["W"], p["m"], p["k"], p["n"], p["blk"], 1000 * (steps - 1))
    assert np.array_equal(outs[steps - 1][0].numpy().view(np.uint64), want.reshape(-1))
    pipe.close()


def test_pipe_more_than_64_products_and_work_on_its_compute_stream(env):
    """70 products in one submit (two launches); the server's share re-encoded on the
    pipe's compute stream before each submit into the same buffer."""
    B, ctx, P, s = env
    m, k, n, blk = 8, 32, 16, (8, 32, 16)
    shapes = [(m, k, n, blk, B.HE_DROP_C0)] * 70
    prods = _case(B, ctx, P, s, shapes, 500)
    shares = [S.uniform_share((k, n), 900 + t) for t in range(3)]
    shares_dev = [to_dev(w) for w in shares]  # alive until the pipe has run (other streams read them)
    pt_step = ctx.empty(ctx.sizes(m, k, n, blk)["pt_words"])
    pipe = B.Pipe(ctx, depth=2)
    outs = [[torch.empty(p["ow"], dtype=torch.int64).pin_memory() for p in prods] for _ in range(3)]
    arrs = []
    for t in range(3):
        its = _items(prods, outs[t], [7 * t + i for i in range(70)], True)
        its[-1]["pt"] = pt_step  # the last product multiplies by the per-step share
        arrs.append(B.make_products(its))
    ws = ctx.empty(pipe.workspace_bytes(arrs[0]) // 8 + 1)
    torch.cuda.synchronize()
    for t in range(3):
        B.he_encode_weights(ctx, shares_dev[t], k, n, blk, pt=pt_step, stream=pipe.compute_stream)
        pipe.submit(arrs[t], ws)
    pipe.wait()
    B.he_device_status(ctx)
    for t in range(3):
        for i in (0, 63, 64, 69):
            p = prods[i]
            W = shares[t] if i == 69 else p["W"]
            want = O.matmul(P, p["ct"], W, m, k, n, blk, 7 * t + i)
            kb, Nc, L, N = blk[1], P.N // blk[1], P.L, P.N
            got = outs[t][i].numpy().view(np.uint64).reshape(want.shape[0], L * (Nc + N))
            assert np.array_equal(got[:, L * Nc:].reshape(-1, L, N), want[:, 1]), (t, i)
            assert np.array_equal(got[:, :L * Nc].reshape(-1, L, Nc), want[:, 0, :, kb - 1::kb]), (t, i)
    pipe.close()


def test_pipe_rejects_a_small_workspace_and_a_bad_depth(env):
    B, ctx, P, s = env
    prods = _case(B, ctx, P, s, [(16, 64, 64, (8, 32, 16), 0)], 700)
    with pytest.raises(B.HEError):
        B.Pipe(ctx, depth=0)
    pipe = B.Pipe(ctx, depth=2)
    out = torch.empty(prods[0]["ow"], dtype=torch.int64).pin_memory()
    arr = B.make_products(_items(prods, [out], [1], True))
    need = pipe.workspace_bytes(arr)
    with pytest.raises(B.HEError):
        pipe.submit(arr, ctx.empty(need // 8 - 64))
    pipe.close()


def test_pipe_moves_slices_of_one_host_array_in_one_copy_and_still_matches(env):
    """Inputs and outputs as adjacent slices of one pinned array each (the copies merge
    into one per direction), next to products with buffers of their own."""
    B, ctx, P, s = env
    m, k, n, blk = 12, 96, 40, (4, 8, 16)
    prods = _case(B, ctx, P, s, [(m, k, n, blk, B.HE_DROP_C0)] * 5, 800)
    iw = prods[0]["in_h"].numel()
    big_in = torch.empty(5 * iw, dtype=torch.int64).pin_memory()
    for i, p in enumerate(prods):
        big_in[i * iw:(i + 1) * iw].copy_(p["in_h"])
        p["in_h"] = big_in[i * iw:(i + 1) * iw]
    ow = prods[0]["ow"]
    big_out = torch.empty(5 * ow, dtype=torch.int64).pin_memory()
    outs = [big_out[i * ow:(i + 1) * ow] for i in range(5)]
    pipe = B.Pipe(ctx, depth=2)
    arr = B.make_products(_items(prods, outs, [40 + i for i in range(5)], True))
    ws = ctx.empty(pipe.workspace_bytes(arr) // 8 + 1)
    pipe.submit(arr, ws)
    pipe.wait()
    B.he_device_status(ctx)
    kb, Nc, L, N = blk[1], P.N // blk[1], P.L, P.N
    for i in (0, 4):
        p = prods[i]
        want = O.matmul(P, p["ct"], p["W"], m, k, n, blk, 40 + i)
        got = outs[i].numpy().view(np.uint64).reshape(want.shape[0], L * (Nc + N))
        assert np.array_equal(got[:, L * Nc:].reshape(-1, L, N), want[:, 1]), i
        assert np.array_equal(got[:, :L * Nc].reshape(-1, L, Nc), want[:, 0, :, kb - 1::kb]), i
    pipe.close()
