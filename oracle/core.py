"""ctypes loader for the C half of the oracle (he_oracle.c).

Test infrastructure only.  ``build_oracle()`` compiles he_oracle.c with gcc
into oracle/liboracle.so (rebuilt when the source or its table is newer).
"""
import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "he_oracle.c"
_HDR = _HERE / "gauss_cdt.h"
_SO = _HERE / "liboracle.so"

_u64p = ctypes.POINTER(ctypes.c_uint64)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u32p = ctypes.POINTER(ctypes.c_uint32)


def build_oracle(force=False):
    """Compile the oracle's C core (plain gcc, OpenMP over independent items)."""
    stale = (not _SO.exists()) or any(p.stat().st_mtime > _SO.stat().st_mtime for p in (_SRC, _HDR))
    if force or stale:
        tmp = _SO.with_suffix(f".so.{os.getpid()}.tmp")
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", str(_SRC), "-o", str(tmp)]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    build_oracle()
    so = ctypes.CDLL(str(_SO))
    u32, u64, sz = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_size_t
    sig = {
        "or_is_prime": (ctypes.c_int, [u64]),
        "or_primitive_2n_root": (u64, [u64, u32]),
        "or_ntt_forward": (None, [_u64p, u32, u64, u64, sz]),
        "or_ntt_inverse": (None, [_u64p, u32, u64, u64, sz]),
        "or_negacyclic_mul_schoolbook": (None, [_u64p, _u64p, _u64p, u32, u64]),
        "or_philox4x32_10": (None, [_u32p, _u32p, _u32p]),
        "or_sample_ternary": (None, [u64, u32, _i64p]),
        "or_sample_uniform": (None, [u64, u32, u32, u64, u32, _u64p]),
        "or_sample_gauss": (None, [u64, u32, u32, _i64p]),
        "or_gauss_from_draw": (ctypes.c_int64, [u64]),
        "or_sample_mask": (None, [u64, u32, u32, u32, _u64p]),
        "or_gauss_cdt": (None, [_u64p]),
        "or_gauss_bound": (u32, []),
        "or_delta_residues": (None, [_u64p, u32, u32, u64, _u64p]),
        "or_encrypt": (None, [u32, u32, _u64p, _u64p, u32, _i64p, _u64p, u32, u32, u64, _u64p]),
        "or_decrypt_residues": (None, [u32, u32, _u64p, _u64p, _i64p, _u64p, u32, _u64p]),
        "or_ctpt_accumulate": (None, [u32, u32, _u64p, _u64p, _u64p, u32, u32, u32, _u32p, u32, _u64p]),
        "or_apply_mask": (None, [u32, u32, _u64p, u32, u64, _u32p, u32, _u64p]),
        "or_max_primes": (ctypes.c_int, []),
        "or_share_matmul": (None, [u32, u32, u32, _u64p, _u64p, _u64p, _u64p, u32, _u64p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(so, name)
        fn.restype = res
        fn.argtypes = args
    return so


lib = _load()


def p64(a):
    """Pointer to a C-contiguous uint64 numpy array."""
    assert a.dtype == np.uint64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_u64p)


def pi64(a):
    assert a.dtype == np.int64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_i64p)


def p32(a):
    assert a.dtype == np.uint32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_u32p)
