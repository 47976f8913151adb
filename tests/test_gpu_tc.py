"""Tensor-core building blocks on the GPU.

The tcgen05 descriptors (shared-memory matrix descriptor, instruction descriptor, TMEM
addressing of the accumulator) are checked against exact integer products: operands are
small integers (exact in bf16), so every f32 sum of at most 2^24 is exact and D = A B^T
must equal numpy's integer product element by element.  The operand ranges include the
balanced 8-bit digits an exact limb split of 50-bit residues would use.

The rate probes report the dense MMA rate of the two exact integer routes on this GPU
(tcgen05 bf16 -> f32; warp-level mma.sync s8 -> s32, the only 8-bit integer tensor
instruction sm_103a offers).
"""
import numpy as np
import pytest
import torch

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    need_gpu()
    from paper_2305_18396_gb300 import binding as B

    return B, B.Context(4096, 2)


@pytest.mark.parametrize("n,k,lo,hi", [(16, 16, -8, 8), (64, 64, -8, 8), (256, 32, -3, 3), (16, 128, -128, 127),
                                       (128, 256, -128, 127)])
def test_tcgen05_bf16_gemm_is_exact(env, n, k, lo, hi):
    B, ctx = env
    rng = np.random.default_rng(n * 1000 + k)
    a = rng.integers(lo, hi + 1, size=(128, k))
    b = rng.integers(lo, hi + 1, size=(n, k))
    A = torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16).cuda()
    Bm = torch.from_numpy(b.astype(np.float32)).to(torch.bfloat16).cuda()
    D = B.he_test_tc_gemm(ctx, A, Bm).cpu().numpy()
    want = a @ b.T
    assert np.abs(want).max() < 2**24
    assert np.array_equal(D.astype(np.int64), want)
    B.he_device_status(ctx)


def test_tensor_rate_probes(env):
    B, ctx = env
    bf16 = B.he_probe_tensor(ctx, 0)
    s8 = B.he_probe_tensor(ctx, 1)
    B.he_device_status(ctx)
    print(f"\ntcgen05 bf16 dense: {bf16 / 1e12:.1f} TFLOP/s; mma.sync s8: {s8 / 1e12:.1f} TOP/s")
    assert bf16 > 1e14 and s8 > 0
