"""The benchmark's step against the oracle, built exactly as bench.py builds it.

bench.Layer sets up the headline workload (one BERT-large encoder layer at seq 512, BFV
N = 8192, three primes): blockings chosen by the autotuner, the transform radix chosen by
its tuner, every product of the layer in one he_matmul_multi launch (Algorithm 1 step 3
for all 68 products), captured once as a CUDA graph and replayed with the step's mask
seeds read from device memory (HE_SEED_DEVICE), compact output (Sec. 3.1.3).

Every product of the layer is checked on sampled output ciphertexts: the oracle encrypts
the input rows those outputs read (at the same object indices and seed as the device),
the test verifies that the device encrypted them identically and plants the oracle's
words, replays the step, and compares the kept words with the oracle's Pi_MatMul of the
same rows, weights (or server shares) and mask seed; the oracle's output must decrypt,
with the server's mask, to the block of X W mod t.
"""
import numpy as np
import pytest

import bench
import oracle as O
from gpu_util import need_gpu, to_dev, to_np
from paper_2305_18396_gb300 import synthetic as S
from paper_2305_18396_gb300 import workloads
from test_gpu_configs import check_decrypts

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_bench_step_every_product_sampled_against_oracle():
    need_gpu()
    import torch

    from paper_2305_18396_gb300 import binding as B

    wl = bench.WORKLOADS[bench.DEFAULT_WORKLOAD]
    N, L = wl["N"], wl["L"]
    ctx = B.Context(N, L)
    ctx.autotune_ntt_radix()
    prods = workloads.bert_layer_products(**getattr(workloads, wl["model"]))
    layer = bench.Layer(B, ctx, prods, 0, False, B.HE_DROP_C0, tune=True, multi=True, graph=True)
    assert layer.products == 68 and len(layer.prod_chunks) == 2
    P = O.Params(N, L)
    s = O.keygen(P, S.SEED_KEY)  # bench's rank-0 client key
    rng = np.random.default_rng(77)
    checks = []
    for c in layer.calls:
        p, blk, si, cnt = c["p"], c["blk"], c["si"], c["cnt"]
        nI, nJ, nLb = O.blocks(p.m, p.k, p.n, blk)
        seed = 10_000 + c["idx"]  # bench's per-group input seed (rank 0)
        view = c["ct_in"].view(cnt, si["in_cts"], 2, L, N)
        for b in range(cnt):
            X = S.uniform_share((p.m, p.k), seed + b)
            if p.share_weights:
                W = S.uniform_share((p.k, p.n), seed + 500_000 + b)
            else:
                W = S.fixed_point_weights((p.k, p.n), seed + 500_000 + b)
            sel = sorted({int(rng.integers(0, nI * nLb)), nI * nLb - 1} if cnt == 1 else {int(rng.integers(0, nI * nLb))})
            rows = {}
            for Lb in sorted({o // nI for o in sel}):
                m_b = blk[0]
                r = O.encrypt(P, s, O.pack_input(X[Lb * m_b:(Lb + 1) * m_b], blk, N), seed + 900_000,
                              obj0=b * si["in_cts"] + Lb * nJ)
                dev = to_np(view[b, Lb * nJ:(Lb + 1) * nJ])
                assert np.array_equal(dev.reshape(r.shape), r), (p.name, b, Lb)
                view[b, Lb * nJ:(Lb + 1) * nJ] = to_dev(r).view(nJ, 2, L, N)
                rows[Lb] = r
            checks.append((c, b, X, W, sel, rows))
    layer.capture()
    step = 4242
    layer.step(step)  # graph replay: the step's seeds are written to the device words first
    torch.cuda.synchronize()
    B.he_device_status(ctx)
    for c, b, X, W, sel, rows in checks:
        p, blk, si = c["p"], c["blk"], c["si"]
        kb, Nc, ow = blk[1], N // blk[1], si["out"]
        assert ow == si["out_words_compact"]
        got = to_np(c["out"][b * ow:(b + 1) * ow]).reshape(si["out_cts"], L * (Nc + N))[sel]
        mask_seed = (step << 20) + c["idx"] + b
        want = O.matmul(P, rows, W, p.m, p.k, p.n, blk, mask_seed, sel=sel)
        assert np.array_equal(got[:, L * Nc:].reshape(-1, L, N), want[:, 1]), (p.name, b)
        assert np.array_equal(got[:, :L * Nc].reshape(-1, L, Nc), want[:, 0, :, kb - 1::kb]), (p.name, b)
        check_decrypts(P, s, X, W, p.n, blk, mask_seed, sel, want)
    ctx.close()
