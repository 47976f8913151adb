"""Seeded synthetic inputs shaped like the BERT workloads of Sec. 4.1.

This module holds no arithmetic of the homomorphic method: it only draws the
plaintext operands that both the CUDA path and the CPU oracle consume.  The
paper evaluates on GLUE text (Sec. 4.1); no dataset is used here -- the
operands are stand-ins with the value distributions of the method's inputs:

* client activations / shares: uniform in Z_t, t = 2^37 (an additive share of
  Sec. 2.2 is uniform);
* server weights: fixed point with f = 12 fractional bits (Sec. 2.2,
  "Encode(x) = x * 2^f"), round(N(0, 0.02) * 2^12) with ties away from zero,
  stored as signed values mod t;
* share x share operands (attention, Sec. 3.1.1): uniform in Z_t.
"""
import numpy as np

LOG2T = 37
FRAC_BITS = 12

# seeds used throughout the tests and the benchmark
SEED_X = 1
SEED_W = 2
SEED_KEY = 3
SEED_ENC = 4
SEED_MASK = 5


def uniform_share(shape, seed, log2t=LOG2T):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 1 << log2t, size=shape, dtype=np.uint64)


def fixed_point_weights(shape, seed, std=0.02, frac_bits=FRAC_BITS, log2t=LOG2T):
    rng = np.random.default_rng(seed)
    x = rng.normal(0.0, std, size=shape) * float(1 << frac_bits)
    r = np.sign(x) * np.floor(np.abs(x) + 0.5)  # round half away from zero
    r = r.astype(np.int64)
    return (r % (1 << log2t)).astype(np.uint64)


def uniform_plaintexts(cnt, N, seed, log2t=LOG2T):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 1 << log2t, size=(cnt, N), dtype=np.uint64)
