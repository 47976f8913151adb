"""CUDA-graph replay of a multi-product launch with per-replay mask seeds (HE_SEED_DEVICE).

The launch is captured once; each replay reads the products' mask seeds from device
words written before it.  Every replay must equal, bit for bit, the products' own
he_matmul calls with those seeds (which the parity tests tie to the oracle).
"""
import numpy as np
import pytest
import torch

from gpu_util import need_gpu, to_dev, to_np
from paper_2305_18396_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


def test_graph_replay_takes_fresh_seeds():
    need_gpu()
    from paper_2305_18396_gb300 import binding as B

    ctx = B.Context(4096, 2)
    sk = B.he_keygen(ctx, 3)
    shapes = [(16, 64, 64, 0), (40, 96, 48, B.HE_DROP_C0), (9, 70, 37, B.HE_DROP_C0)]
    seeds = torch.zeros(len(shapes), dtype=torch.int64, device=ctx.device)
    items, refs = [], []
    for i, (m, k, n, flags) in enumerate(shapes):
        blk = ctx.default_blocking(m, k, n)
        X = S.uniform_share((m, k), 10 + i)
        W = S.fixed_point_weights((k, n), 20 + i)
        ct = B.he_encrypt(ctx, sk, B.he_pack_input(ctx, to_dev(X), m, k, blk), 30 + i)
        pt = B.he_encode_weights(ctx, to_dev(W), k, n, blk)
        si = ctx.sizes(m, k, n, blk)
        ow = si["out_words_compact"] if flags else si["out_words"]
        items.append(dict(ct_in=ct, pt=pt, ct_out=ctx.empty(ow), m=m, k=k, n=n, blk=blk,
                          flags=flags | B.HE_SEED_DEVICE, mask_seed=seeds.data_ptr() + 8 * i))
        refs.append((ct, pt, m, k, n, blk, flags))
    prods = B.make_products(items)
    ws = ctx.empty(B.he_multi_workspace_bytes(ctx, prods) // 8 + 1)

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):  # warm-up outside the capture
        seeds.fill_(1)
        B.he_matmul_multi(ctx, prods, ws)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        B.he_matmul_multi(ctx, prods, ws)
    torch.cuda.synchronize()

    for trial in ([101, 102, 103], [7, 8, 9]):
        seeds.copy_(torch.tensor(trial, dtype=torch.int64))
        graph.replay()
        torch.cuda.synchronize()
        for it, (ct, pt, m, k, n, blk, flags), sd in zip(items, refs, trial):
            alone = B.he_matmul(ctx, ct, pt, m, k, n, blk, sd, flags=flags)
            assert np.array_equal(to_np(it["ct_out"]), to_np(alone)), (m, k, n, sd)
    B.he_device_status(ctx)


def test_seed_device_flag_rejected_without_address():
    need_gpu()
    from paper_2305_18396_gb300 import binding as B

    ctx = B.Context(4096, 2)
    m, k, n = 4, 8, 8
    blk = ctx.default_blocking(m, k, n)
    si = ctx.sizes(m, k, n, blk)
    item = dict(ct_in=ctx.empty(si["in_words"]), pt=ctx.empty(si["pt_words"]), ct_out=ctx.empty(si["out_words"]),
                m=m, k=k, n=n, blk=blk, flags=B.HE_SEED_DEVICE, mask_seed=0)
    prods = B.make_products([item])
    with pytest.raises(B.HEError):
        B.he_matmul_multi(ctx, prods, ctx.empty(1 << 20))
