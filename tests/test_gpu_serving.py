"""Continuous batching: every request's result is the same alone and in the mix.

Requests of different matrices and sequence lengths are served through the
continuous-batching loop (several multi-product launches in flight, admission by a
device-memory budget); each output must equal, bit for bit, the output of the same
request run alone through he_matmul.
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
