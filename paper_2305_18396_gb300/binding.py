"""Thin Python binding of the C ABI in include/he_gb300.h (ctypes).

Argument marshalling only: every function checks that tensors live on the
context's device with the right size, passes their device pointers and the
current CUDA stream, and raises HEError on a non-zero status.  All arithmetic
runs in the CUDA kernels of libhe_gb300.so; there is no CPU fallback -- if the
library is missing, importing this module raises.

Tensors hold u64 words in torch.int64 storage (bit-identical to uint64;
numpy views with ``.view(np.uint64)``).
"""
import ctypes
from pathlib import Path

import torch

from . import build as _build

HE_OK, HE_EINVAL, HE_ENOMEM, HE_ECUDA, HE_ETIMEOUT, HE_ENOISE = range(6)
HE_FLAGS_NONE = 0
HE_DROP_C0 = 1
HE_ASYNC = 2
HE_MAC_AUTO, HE_MAC_INTEGER, HE_MAC_TENSOR, HE_MAC_COSET = 0, 1, 2, 3
_NAMES = {1: "HE_EINVAL", 2: "HE_ENOMEM", 3: "HE_ECUDA", 4: "HE_ETIMEOUT", 5: "HE_ENOISE"}


class HEError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class Blocking(ctypes.Structure):
    _fields_ = [("m_b", ctypes.c_uint32), ("k_b", ctypes.c_uint32), ("n_b", ctypes.c_uint32)]

    def as_tuple(self):
        return (self.m_b, self.k_b, self.n_b)


class SizeInfo(ctypes.Structure):
    _fields_ = [("nI", ctypes.c_uint32), ("nJ", ctypes.c_uint32), ("nLb", ctypes.c_uint32),
                ("in_cts", ctypes.c_uint64), ("out_cts", ctypes.c_uint64), ("pts", ctypes.c_uint64),
                ("in_words", ctypes.c_uint64), ("out_words", ctypes.c_uint64), ("pt_words", ctypes.c_uint64),
                ("packed_words", ctypes.c_uint64), ("workspace_bytes", ctypes.c_uint64),
                ("out_words_compact", ctypes.c_uint64), ("workspace_bytes_compact", ctypes.c_uint64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Product(ctypes.Structure):
    _fields_ = [("ct_in", ctypes.c_void_p), ("pt", ctypes.c_void_p), ("ct_out", ctypes.c_void_p),
                ("m", ctypes.c_uint32), ("k", ctypes.c_uint32), ("n", ctypes.c_uint32), ("blk", Blocking),
                ("flags", ctypes.c_uint32), ("mask_seed", ctypes.c_uint64)]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_uint64), ("total_ms", ctypes.c_double)]


LIB_PATH = _build.LIB


def _load():
    if not Path(LIB_PATH).exists():
        raise ImportError(f"CUDA library {LIB_PATH} is not built; run `python -m paper_2305_18396_gb300.build` "
                          "(or __graft_entry__.build()) -- there is no CPU fallback")
    so = ctypes.CDLL(str(LIB_PATH))
    P, u32, u64, i32, sz = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_size_t
    pB, pS = ctypes.POINTER(Blocking), ctypes.POINTER(SizeInfo)
    pu64, pu32, pi32 = ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_int32)
    sig = {
        "he_last_error": (ctypes.c_char_p, []),
        "he_params_init": (ctypes.c_int, [ctypes.POINTER(P), u32, u32, pu64, u32, ctypes.c_int]),
        "he_ctx_free": (ctypes.c_int, [P]),
        "he_get_params": (ctypes.c_int, [P, pu32, pu32, pu32, pu64, pu64]),
        "he_sizes": (ctypes.c_int, [P, u32, u32, u32, pB, pS]),
        "he_default_blocking": (ctypes.c_int, [P, u32, u32, u32, u32, pB]),
        "he_choose_blocking": (ctypes.c_int, [u32, u32, u32, u32, u32, u32, pB]),
        "he_keygen": (ctypes.c_int, [P, u64, P, P]),
        "he_encrypt": (ctypes.c_int, [P, P, P, u32, u64, P, P]),
        "he_decrypt": (ctypes.c_int, [P, P, P, u32, P, P, pi32, P]),
        "he_pack_input": (ctypes.c_int, [P, P, u32, u32, pB, P, P]),
        "he_unpack_output": (ctypes.c_int, [P, P, u32, u32, pB, P, P]),
        "he_encode_weights": (ctypes.c_int, [P, P, u32, u32, pB, P, P]),
        "he_matmul": (ctypes.c_int, [P, P, P, u32, u32, u32, pB, u64, u32, P, P, sz, P]),
        "he_matmul_host": (ctypes.c_int, [P, P, P, u32, u32, u32, pB, u64, u32, P, P, sz, P]),
        "he_matmul_batch_host": (ctypes.c_int, [P, P, P, u32, u32, u32, pB, u32, u64, u32, P, P, sz, P]),
        "he_matmul_noalloc": (ctypes.c_int, [P, P, P, u32, u32, u32, pB, u64, u32, P, P]),
        "he_matmul_batch": (ctypes.c_int, [P, P, P, u32, u32, u32, pB, u32, u64, u32, P, P, sz, P]),
        "he_matmul_multi": (ctypes.c_int, [P, u32, ctypes.POINTER(Product), P, sz, P]),
        "he_multi_workspace_bytes": (ctypes.c_int, [P, u32, ctypes.POINTER(Product), ctypes.POINTER(sz)]),
        "he_encode_weights_batch": (ctypes.c_int, [P, P, u32, u32, pB, u32, P, P]),
        "he_unmask": (ctypes.c_int, [P, u64, u32, u32, pB, P, P]),
        "he_unmask_acc": (ctypes.c_int, [P, u64, u32, u32, pB, u32, P, P]),
        "he_autotune_blocking": (ctypes.c_int, [P, u32, u32, u32, u32, u32, u32, u32, P, sz, ctypes.POINTER(sz), pB,
                                                ctypes.POINTER(ctypes.c_float), P]),
        "he_set_ntt_radix": (ctypes.c_int, [P, u32]),
        "he_set_mac_engine": (ctypes.c_int, [P, u32]),
        "he_get_mac_engine": (ctypes.c_int, [P, pu32]),
        "he_mac_uses_tensor_cores": (ctypes.c_int, [P, u32, pB, pu32]),
        "he_mac_uses_cosets": (ctypes.c_int, [P, pB, pu32]),
        "he_get_ntt_radix": (ctypes.c_int, [P, pu32]),
        "he_autotune_ntt_radix": (ctypes.c_int, [P, u32, P, sz, ctypes.POINTER(sz), ctypes.POINTER(ctypes.c_float),
                                                 pu32, P]),
        "he_share_matmul": (ctypes.c_int, [P, P, P, P, P, u32, u32, u32, P, P]),
        "he_share_matmul_batch": (ctypes.c_int, [P, P, P, P, P, u32, u32, u32, u32, P, P]),
        "he_matmul_multi_host": (ctypes.c_int, [P, u32, ctypes.POINTER(Product), u32, P, sz, P]),
        "he_pipe_create": (ctypes.c_int, [P, u32, ctypes.POINTER(P)]),
        "he_pipe_free": (ctypes.c_int, [P]),
        "he_pipe_compute_stream": (ctypes.c_int, [P, ctypes.POINTER(P)]),
        "he_pipe_submit": (ctypes.c_int, [P, u32, ctypes.POINTER(Product), P, sz]),
        "he_pipe_workspace_bytes": (ctypes.c_int, [P, u32, ctypes.POINTER(Product), ctypes.POINTER(sz)]),
        "he_pipe_wait": (ctypes.c_int, [P]),
        "he_multi_host_workspace_bytes": (ctypes.c_int, [P, u32, ctypes.POINTER(Product), ctypes.POINTER(sz)]),
        "he_expand_compact": (ctypes.c_int, [P, P, u32, u32, P, P]),
        "he_ct_export": (ctypes.c_int, [P, P, u32, u32, P, P]),
        "he_ct_import": (ctypes.c_int, [P, P, u32, u32, P, P]),
        "he_ntt_forward": (ctypes.c_int, [P, P, u32, P]),
        "he_ntt_inverse": (ctypes.c_int, [P, P, u32, P]),
        "he_poly_mul": (ctypes.c_int, [P, P, P, P, u32, P]),
        "he_gauss_cdt": (ctypes.c_int, [pu64, u32]),
        "he_profile_enable": (ctypes.c_int, [P, ctypes.c_int]),
        "he_profile_read": (ctypes.c_int, [P, ctypes.POINTER(KernelStat), u32, pu32]),
        "he_launch_count": (ctypes.c_int, [P, pu64]),
        "he_device_status": (ctypes.c_int, [P, P]),
        "he_test_wait_timeout": (ctypes.c_int, [P, u32, P]),
        "he_probe_mad_wide": (ctypes.c_int, [P, P, sz, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), P]),
        "he_probe_tensor": (ctypes.c_int, [P, u32, ctypes.POINTER(ctypes.c_double), P, sz, P]),
        "he_test_tc_gemm": (ctypes.c_int, [P, u32, u32, P, P, P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(so, name)
        fn.restype = res
        fn.argtypes = args
    return so


lib = _load()


def _check(code):
    if code != HE_OK:
        raise HEError(code, lib.he_last_error().decode())


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _blk(blk):
    return ctypes.byref(Blocking(*blk))


class Context:
    """Owns an he_ctx (parameters {N, t, q} of Sec. 2.2 and the NTT tables on `device`)."""

    def __init__(self, N=4096, L=2, primes=None, log2t=37, device=0):
        if primes is None:
            from .params import DEFAULT_PRIMES
            primes = DEFAULT_PRIMES[:L]
        arr = (ctypes.c_uint64 * L)(*primes)
        h = ctypes.c_void_p()
        _check(lib.he_params_init(ctypes.byref(h), N, L, arr, log2t, device))
        self.h = h
        self.N, self.L, self.log2t, self.device = N, L, log2t, torch.device("cuda", device)
        self.primes = tuple(primes)

    def close(self):
        if getattr(self, "h", None):
            lib.he_ctx_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- host-side queries
    def params(self):
        N, L, lt = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
        q, psi = (ctypes.c_uint64 * 3)(), (ctypes.c_uint64 * 3)()
        _check(lib.he_get_params(self.h, ctypes.byref(N), ctypes.byref(L), ctypes.byref(lt), q, psi))
        return {"N": N.value, "L": L.value, "log2t": lt.value, "q": list(q)[: L.value], "psi": list(psi)[: L.value]}

    def sizes(self, m, k, n, blk):
        si = SizeInfo()
        _check(lib.he_sizes(self.h, m, k, n, _blk(blk), ctypes.byref(si)))
        return si.as_dict()

    def default_blocking(self, m, k, n, weights_per_call=False):
        b = Blocking()
        _check(lib.he_default_blocking(self.h, m, k, n, 1 if weights_per_call else 0, ctypes.byref(b)))
        return b.as_tuple()

    def autotune_blocking(self, m, k, n, weights_per_call=False, flags=0, batch=1, candidates=0, stream=None):
        """Measured blocking (he_autotune_blocking): returns (blocking, ms per call)."""
        need = ctypes.c_size_t(0)
        b = Blocking()
        ms = ctypes.c_float(0)
        wpc = 1 if weights_per_call else 0
        _check(lib.he_autotune_blocking(self.h, m, k, n, wpc, flags, batch, candidates, None, 0,
                                        ctypes.byref(need), ctypes.byref(b), ctypes.byref(ms), _stream(stream)))
        if m and k and n:
            scratch = self.empty(max(need.value // 8 + 1, 1))
            _check(lib.he_autotune_blocking(self.h, m, k, n, wpc, flags, batch, candidates, _ptr(scratch),
                                            scratch.numel() * 8, None, ctypes.byref(b), ctypes.byref(ms),
                                            _stream(stream)))
            del scratch
        return b.as_tuple(), ms.value

    @property
    def ntt_radix(self):
        """log2 of the values per thread of the register-blocked transforms (he_get_ntt_radix)."""
        v = ctypes.c_uint32(0)
        _check(lib.he_get_ntt_radix(self.h, ctypes.byref(v)))
        return v.value

    def set_ntt_radix(self, log2_values):
        _check(lib.he_set_ntt_radix(self.h, log2_values))

    @property
    def mac_engine(self):
        """HE_MAC_AUTO, HE_MAC_INTEGER, HE_MAC_TENSOR or HE_MAC_COSET (he_get_mac_engine)."""
        v = ctypes.c_uint32(0)
        _check(lib.he_get_mac_engine(self.h, ctypes.byref(v)))
        return v.value

    def set_mac_engine(self, engine):
        """Set before encoding weights: the engine fixes their layout (he_set_mac_engine)."""
        _check(lib.he_set_mac_engine(self.h, engine))

    def uses_tensor_cores(self, k, blk):
        v = ctypes.c_uint32(0)
        _check(lib.he_mac_uses_tensor_cores(self.h, k, _blk(blk), ctypes.byref(v)))
        return bool(v.value)

    def uses_cosets(self, blk):
        v = ctypes.c_uint32(0)
        _check(lib.he_mac_uses_cosets(self.h, _blk(blk), ctypes.byref(v)))
        return bool(v.value)

    def autotune_ntt_radix(self, cnt=0, stream=None):
        """Measured transform radix (he_autotune_ntt_radix), selected for this context.
        Returns (log2 values per thread, {log2 values: ms per forward + inverse round trip})."""
        need = ctypes.c_size_t(0)
        ms = (ctypes.c_float * 3)()
        chosen = ctypes.c_uint32(0)
        _check(lib.he_autotune_ntt_radix(self.h, cnt, None, 0, ctypes.byref(need), ms, ctypes.byref(chosen),
                                         _stream(stream)))
        scratch = self.empty(max(need.value // 8, 1))
        _check(lib.he_autotune_ntt_radix(self.h, cnt, _ptr(scratch), scratch.numel() * 8, None, ms,
                                         ctypes.byref(chosen), _stream(stream)))
        del scratch
        return chosen.value, {r: ms[r - 3] for r in (3, 4, 5) if ms[r - 3] >= 0}

    # ---- allocation helpers (device memory comes from torch)
    def empty(self, words):
        return torch.empty(int(words), dtype=torch.int64, device=self.device)

    def _dev(self, t, words, name):
        if t.device != self.device or not t.is_contiguous() or t.dtype not in (torch.int64, torch.uint64):
            raise ValueError(f"{name} must be a contiguous int64/uint64 tensor on {self.device}")
        if t.numel() < words:
            raise ValueError(f"{name} needs at least {words} words, has {t.numel()}")
        return t


def he_choose_blocking(N, L, m, k, n, weights_per_call=False):
    """Host-only: the blocking the library picks for an (m x k) . (k x n) product."""
    b = Blocking()
    _check(lib.he_choose_blocking(N, L, m, k, n, 1 if weights_per_call else 0, ctypes.byref(b)))
    return b.as_tuple()


def he_params_init(N=4096, L=2, primes=None, log2_t=37, device=0):
    return Context(N, L, primes, log2_t, device)


def he_keygen(ctx, seed, sk=None, stream=None):
    sk = ctx.empty(ctx.L * ctx.N) if sk is None else ctx._dev(sk, ctx.L * ctx.N, "sk")
    _check(lib.he_keygen(ctx.h, seed, _ptr(sk), _stream(stream)))
    return sk


def he_encrypt(ctx, sk, plain, seed, ct=None, stream=None):
    cnt = plain.numel() // ctx.N
    ctx._dev(plain, cnt * ctx.N, "plain")
    ct = ctx.empty(cnt * 2 * ctx.L * ctx.N) if ct is None else ctx._dev(ct, cnt * 2 * ctx.L * ctx.N, "ct")
    _check(lib.he_encrypt(ctx.h, _ptr(ctx._dev(sk, ctx.L * ctx.N, "sk")), _ptr(plain), cnt, seed, _ptr(ct),
                          _stream(stream)))
    return ct


def he_decrypt(ctx, sk, ct, plain=None, noise_budget=None, check_noise=False, stream=None):
    """Returns (plain, noise_budget); with check_noise the call synchronizes and raises HE_ENOISE."""
    cnt = ct.numel() // (2 * ctx.L * ctx.N)
    ctx._dev(ct, cnt * 2 * ctx.L * ctx.N, "ct")
    plain = ctx.empty(cnt * ctx.N) if plain is None else ctx._dev(plain, cnt * ctx.N, "plain")
    if noise_budget is None:
        noise_budget = torch.empty(max(cnt, 1), dtype=torch.int32, device=ctx.device)
    mn = ctypes.c_int32()
    _check(lib.he_decrypt(ctx.h, _ptr(ctx._dev(sk, ctx.L * ctx.N, "sk")), _ptr(ct), cnt, _ptr(plain),
                          _ptr(noise_budget), ctypes.byref(mn) if check_noise else None, _stream(stream)))
    return plain, noise_budget[:cnt]


def he_pack_input(ctx, X, m, k, blk, polys=None, stream=None):
    si = ctx.sizes(m, k, 1, blk)
    ctx._dev(X, m * k, "X")
    polys = ctx.empty(si["packed_words"]) if polys is None else ctx._dev(polys, si["packed_words"], "polys")
    _check(lib.he_pack_input(ctx.h, _ptr(X), m, k, _blk(blk), _ptr(polys), _stream(stream)))
    return polys


def he_unpack_output(ctx, dec, m, n, blk, share=None, stream=None):
    si = ctx.sizes(m, 1, n, blk)
    ctx._dev(dec, si["out_cts"] * ctx.N, "dec")
    share = ctx.empty(m * n) if share is None else ctx._dev(share, m * n, "share")
    _check(lib.he_unpack_output(ctx.h, _ptr(dec), m, n, _blk(blk), _ptr(share), _stream(stream)))
    return share


def he_encode_weights(ctx, W, k, n, blk, pt=None, stream=None):
    si = ctx.sizes(1, k, n, blk)
    ctx._dev(W, k * n, "W")
    pt = ctx.empty(si["pt_words"]) if pt is None else ctx._dev(pt, si["pt_words"], "pt")
    _check(lib.he_encode_weights(ctx.h, _ptr(W), k, n, _blk(blk), _ptr(pt), _stream(stream)))
    return pt


def he_encode_weights_batch(ctx, W, k, n, blk, batch, pt=None, stream=None):
    si = ctx.sizes(1, k, n, blk)
    ctx._dev(W, batch * k * n, "W")
    words = batch * si["pt_words"]
    pt = ctx.empty(words) if pt is None else ctx._dev(pt, words, "pt")
    _check(lib.he_encode_weights_batch(ctx.h, _ptr(W), k, n, _blk(blk), batch, _ptr(pt), _stream(stream)))
    return pt


def _out_ws(si, flags):
    """(output words, workspace bytes) of one product for these flags."""
    if flags & HE_DROP_C0:
        return si["out_words_compact"], si["workspace_bytes_compact"]
    return si["out_words"], si["workspace_bytes"]


def he_matmul_batch(ctx, ct_in, pt, m, k, n, blk, batch, mask_seed, ct_out=None, workspace=None,
                    flags=HE_FLAGS_NONE, stream=None):
    """`batch` same-shape products back to back; item b is masked with seed mask_seed + b."""
    si = ctx.sizes(m, k, n, blk)
    ow, wb = _out_ws(si, flags)
    ctx._dev(ct_in, batch * si["in_words"], "ct_in")
    ctx._dev(pt, batch * si["pt_words"], "pt")
    ct_out = ctx.empty(batch * ow) if ct_out is None else ctx._dev(ct_out, batch * ow, "ct_out")
    ws_words = batch * ((wb + 7) // 8)
    workspace = ctx.empty(max(ws_words, 1)) if workspace is None else ctx._dev(workspace, ws_words, "workspace")
    _check(lib.he_matmul_batch(ctx.h, _ptr(ct_in), _ptr(pt), m, k, n, _blk(blk), batch, mask_seed, flags,
                               _ptr(ct_out), _ptr(workspace), workspace.numel() * 8, _stream(stream)))
    return ct_out


def make_products(items):
    """items: dicts with ct_in, pt, ct_out (device tensors), m, k, n, blk, flags, mask_seed.
    The returned descriptor array holds references to the tensors, so buffers made only for
    the call stay allocated while the array is alive."""
    arr = (Product * len(items))()
    arr._tensors = [(x["ct_in"], x["pt"], x["ct_out"]) for x in items]
    for a, x in zip(arr, items):
        a.ct_in, a.pt, a.ct_out = x["ct_in"].data_ptr(), x["pt"].data_ptr(), x["ct_out"].data_ptr()
        a.m, a.k, a.n = x["m"], x["k"], x["n"]
        a.blk = Blocking(*x["blk"])
        a.flags, a.mask_seed = x.get("flags", HE_FLAGS_NONE), x["mask_seed"]
    return arr


def he_multi_workspace_bytes(ctx, products):
    out = ctypes.c_size_t()
    _check(lib.he_multi_workspace_bytes(ctx.h, len(products), products, ctypes.byref(out)))
    return out.value


def he_matmul_multi(ctx, products, workspace, stream=None):
    """products: from make_products (keeps the descriptor array alive for the call)."""
    _check(lib.he_matmul_multi(ctx.h, len(products), products, _ptr(workspace), workspace.numel() * 8,
                               _stream(stream)))


def he_multi_host_workspace_bytes(ctx, products):
    out = ctypes.c_size_t()
    _check(lib.he_multi_host_workspace_bytes(ctx.h, len(products), products, ctypes.byref(out)))
    return out.value


def he_matmul_multi_host(ctx, products, workspace, flags=HE_FLAGS_NONE, stream=None):
    """products: from make_products with HOST (preferably pinned) ct_in / ct_out tensors."""
    _check(lib.he_matmul_multi_host(ctx.h, len(products), products, flags, _ptr(workspace), workspace.numel() * 8,
                                    _stream(stream)))


class Pipe:
    """Owns an he_pipe: multi-product launches from host buffers with uploads, kernels and
    downloads of consecutive submits overlapped on three streams, over `depth` slots of
    one device workspace."""

    def __init__(self, ctx, depth=3):
        h = ctypes.c_void_p()
        _check(lib.he_pipe_create(ctx.h, depth, ctypes.byref(h)))
        self.h, self.ctx, self.depth = h, ctx, depth
        st = ctypes.c_void_p()
        _check(lib.he_pipe_compute_stream(h, ctypes.byref(st)))
        self.compute_stream = torch.cuda.ExternalStream(st.value, device=ctx.device)

    def workspace_bytes(self, products):
        """Device workspace for submits of these products (depth slots)."""
        out = ctypes.c_size_t()
        _check(lib.he_pipe_workspace_bytes(self.h, len(products), products, ctypes.byref(out)))
        return out.value

    def submit(self, products, workspace):
        """products: from make_products with HOST (pinned) ct_in / ct_out tensors; keep them
        alive until wait()."""
        _check(lib.he_pipe_submit(self.h, len(products), products, _ptr(workspace), workspace.numel() * 8))

    def wait(self):
        _check(lib.he_pipe_wait(self.h))

    def close(self):
        if getattr(self, "h", None):
            lib.he_pipe_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def he_matmul(ctx, ct_in, pt, m, k, n, blk, mask_seed, ct_out=None, workspace=None, flags=HE_FLAGS_NONE,
              stream=None):
    si = ctx.sizes(m, k, n, blk)
    ow, wb = _out_ws(si, flags)
    ctx._dev(ct_in, si["in_words"], "ct_in")
    ctx._dev(pt, si["pt_words"], "pt")
    ct_out = ctx.empty(ow) if ct_out is None else ctx._dev(ct_out, ow, "ct_out")
    ws_words = (wb + 7) // 8
    workspace = ctx.empty(max(ws_words, 1)) if workspace is None else ctx._dev(workspace, ws_words, "workspace")
    _check(lib.he_matmul(ctx.h, _ptr(ct_in), _ptr(pt), m, k, n, _blk(blk), mask_seed, flags, _ptr(ct_out),
                         _ptr(workspace), workspace.numel() * 8, _stream(stream)))
    return ct_out


HE_NOALLOC_SCRATCH_BYTES = 32 << 20


def he_matmul_noalloc(ctx, ct_in, pt, m, k, n, blk, mask_seed, ct_out, flags=HE_FLAGS_NONE, stream=None):
    """he_matmul without a workspace: for callers that cannot allocate device memory.
    ct_out (out_words, or out_words_compact with HE_DROP_C0) must be provided by the
    caller; the library's fixed scratch is used instead."""
    si = ctx.sizes(m, k, n, blk)
    ow, _ = _out_ws(si, flags)
    ctx._dev(ct_in, si["in_words"], "ct_in")
    ctx._dev(pt, si["pt_words"], "pt")
    ctx._dev(ct_out, ow, "ct_out")
    _check(lib.he_matmul_noalloc(ctx.h, _ptr(ct_in), _ptr(pt), m, k, n, _blk(blk), mask_seed, flags, _ptr(ct_out),
                                 _stream(stream)))
    return ct_out


def matmul_host_workspace_words(ctx, m, k, n, blk, flags=HE_FLAGS_NONE):
    si = ctx.sizes(m, k, n, blk)
    ow, wb = _out_ws(si, flags)
    return (wb + 7) // 8 + si["in_words"] + ow


def he_matmul_host(ctx, ct_in_host, pt, m, k, n, blk, mask_seed, ct_out_host, workspace, flags=HE_FLAGS_NONE,
                   stream=None):
    """ct_in_host / ct_out_host: CPU tensors (pinned for asynchronous copies)."""
    si = ctx.sizes(m, k, n, blk)
    ow, _ = _out_ws(si, flags)
    for t, w, name in ((ct_in_host, si["in_words"], "ct_in_host"), (ct_out_host, ow, "ct_out_host")):
        if t.device.type != "cpu" or not t.is_contiguous() or t.numel() < w:
            raise ValueError(f"{name} must be a contiguous CPU tensor of >= {w} words")
    ctx._dev(workspace, matmul_host_workspace_words(ctx, m, k, n, blk, flags), "workspace")
    _check(lib.he_matmul_host(ctx.h, _ptr(ct_in_host), _ptr(ctx._dev(pt, si["pt_words"], "pt")), m, k, n, _blk(blk),
                              mask_seed, flags, _ptr(ct_out_host), _ptr(workspace), workspace.numel() * 8,
                              _stream(stream)))
    return ct_out_host


def he_expand_compact(ctx, ct_compact, cnt, k_b, ct_full=None, stream=None):
    """Client side of HE_DROP_C0: compact ciphertexts -> full ones (c0 zero off the kept coefficients)."""
    words = cnt * 2 * ctx.L * ctx.N
    ct_full = ctx.empty(words) if ct_full is None else ctx._dev(ct_full, words, "ct_full")
    _check(lib.he_expand_compact(ctx.h, _ptr(ct_compact), cnt, k_b, _ptr(ct_full), _stream(stream)))
    return ct_full


def wire_words(ctx, cnt, k_b=0):
    """Words of cnt ciphertexts in the wire format: full (k_b = 0) or compact (HE_DROP_C0 of a
    product with this k_b)."""
    return cnt * ctx.L * ((ctx.N // k_b if k_b else ctx.N) + ctx.N)


def _host(t, words, name):
    if t.device.type != "cpu" or not t.is_contiguous() or t.dtype not in (torch.int64, torch.uint64):
        raise ValueError(f"{name} must be a contiguous int64/uint64 CPU tensor")
    if t.numel() < words:
        raise ValueError(f"{name} needs at least {words} words, has {t.numel()}")
    return t


def he_ct_export(ctx, ct, cnt, k_b=0, host_buf=None, stream=None):
    """Device ciphertexts -> host wire format (a CPU tensor; pinned if host_buf is None)."""
    words = wire_words(ctx, cnt, k_b)
    ctx._dev(ct, words, "ct")
    host_buf = torch.empty(words, dtype=torch.int64).pin_memory() if host_buf is None else \
        _host(host_buf, words, "host_buf")
    _check(lib.he_ct_export(ctx.h, _ptr(ct), cnt, k_b, _ptr(host_buf), _stream(stream)))
    return host_buf


def he_ct_import(ctx, host_buf, cnt, k_b=0, ct=None, stream=None):
    """Host wire format -> device ciphertexts, every word checked to be below its prime."""
    words = wire_words(ctx, cnt, k_b)
    _host(host_buf, words, "host_buf")
    ct = ctx.empty(words) if ct is None else ctx._dev(ct, words, "ct")
    _check(lib.he_ct_import(ctx.h, _ptr(host_buf), cnt, k_b, _ptr(ct), _stream(stream)))
    return ct


def he_matmul_batch_host(ctx, ct_in_host, pt, m, k, n, blk, batch, mask_seed, ct_out_host, workspace,
                         flags=HE_FLAGS_NONE, stream=None):
    """Batched products with host (pinned) input/output buffers; see he_matmul_host."""
    si = ctx.sizes(m, k, n, blk)
    ow, _ = _out_ws(si, flags)
    for t, w, name in ((ct_in_host, batch * si["in_words"], "ct_in_host"), (ct_out_host, batch * ow, "ct_out_host")):
        if t.device.type != "cpu" or not t.is_contiguous() or t.numel() < w:
            raise ValueError(f"{name} must be a contiguous CPU tensor of >= {w} words")
    ctx._dev(workspace, batch * matmul_host_workspace_words(ctx, m, k, n, blk, flags), "workspace")
    _check(lib.he_matmul_batch_host(ctx.h, _ptr(ct_in_host), _ptr(ctx._dev(pt, batch * si["pt_words"], "pt")), m, k,
                                    n, _blk(blk), batch, mask_seed, flags, _ptr(ct_out_host), _ptr(workspace),
                                    workspace.numel() * 8, _stream(stream)))
    return ct_out_host


def he_unmask(ctx, mask_seed, m, n, blk, share=None, stream=None):
    share = ctx.empty(m * n) if share is None else ctx._dev(share, m * n, "share")
    _check(lib.he_unmask(ctx.h, mask_seed, m, n, _blk(blk), _ptr(share), _stream(stream)))
    return share


HE_SEED_DEVICE = 16
HE_UNMASK_ACCUMULATE = 4
HE_UNMASK_TRANSPOSE = 8


def he_unmask_acc(ctx, mask_seed, m, n, blk, out, flags=HE_UNMASK_ACCUMULATE, stream=None):
    """out (+)= the server's mask share of an (m x n) product, or its transpose into an n x m out."""
    ctx._dev(out, m * n, "out")
    _check(lib.he_unmask_acc(ctx.h, mask_seed, m, n, _blk(blk), flags, _ptr(out), _stream(stream)))
    return out


def he_share_matmul(ctx, X, W, m, k, n, bias=None, acc=None, out=None, stream=None):
    """Server-local share product: out = (acc + X W + bias) mod t, row-major device tensors."""
    return he_share_matmul_batch(ctx, X, W, m, k, n, 1, bias, acc, out, stream)


def he_share_matmul_batch(ctx, X, W, m, k, n, batch, bias=None, acc=None, out=None, stream=None):
    """`batch` same-shape share products laid back to back (item b at b m k, b k n, b n, b m n)."""
    out = ctx.empty(batch * m * n) if out is None else ctx._dev(out, batch * m * n, "out")
    if not m or not n or not batch:
        return out
    if k:
        ctx._dev(X, batch * m * k, "X")
        ctx._dev(W, batch * k * n, "W")
    if bias is not None:
        ctx._dev(bias, batch * n, "bias")
    if acc is not None:
        ctx._dev(acc, batch * m * n, "acc")
    _check(lib.he_share_matmul_batch(ctx.h, _ptr(X) if k else None, _ptr(W) if k else None,
                                     None if bias is None else _ptr(bias), None if acc is None else _ptr(acc),
                                     m, k, n, batch, _ptr(out), _stream(stream)))
    return out


def he_ntt_forward(ctx, polys, stream=None):
    cnt = polys.numel() // (ctx.L * ctx.N)
    _check(lib.he_ntt_forward(ctx.h, _ptr(ctx._dev(polys, cnt * ctx.L * ctx.N, "polys")), cnt, _stream(stream)))
    return polys


def he_ntt_inverse(ctx, polys, stream=None):
    cnt = polys.numel() // (ctx.L * ctx.N)
    _check(lib.he_ntt_inverse(ctx.h, _ptr(ctx._dev(polys, cnt * ctx.L * ctx.N, "polys")), cnt, _stream(stream)))
    return polys


def he_poly_mul(ctx, a, b, c=None, stream=None):
    cnt = a.numel() // (ctx.L * ctx.N)
    words = cnt * ctx.L * ctx.N
    c = ctx.empty(words) if c is None else ctx._dev(c, words, "c")
    _check(lib.he_poly_mul(ctx.h, _ptr(ctx._dev(a, words, "a")), _ptr(ctx._dev(b, words, "b")), _ptr(c), cnt,
                           _stream(stream)))
    return c


def he_gauss_cdt():
    out = (ctypes.c_uint64 * 38)()
    _check(lib.he_gauss_cdt(out, 38))
    return list(out)


def he_profile_enable(ctx, on=True):
    _check(lib.he_profile_enable(ctx.h, 1 if on else 0))


def he_profile_read(ctx):
    buf = (KernelStat * 32)()
    n = ctypes.c_uint32()
    _check(lib.he_profile_read(ctx.h, buf, 32, ctypes.byref(n)))
    return {buf[i].name.decode(): {"launches": buf[i].launches, "total_ms": buf[i].total_ms} for i in range(n.value)}


def he_device_status(ctx, stream=None):
    """Raises HEError(HE_ETIMEOUT) if a kernel's bounded wait expired since the last check."""
    _check(lib.he_device_status(ctx.h, _stream(stream)))


def he_test_wait_timeout(ctx, limit_ms=100, stream=None):
    _check(lib.he_test_wait_timeout(ctx.h, limit_ms, _stream(stream)))


def he_probe_mad_wide(ctx, stream=None):
    """(mad.wide.u32 operations/s, per SM per clock) measured on the context's GPU."""
    sms = torch.cuda.get_device_properties(ctx.device).multi_processor_count
    scratch = ctx.empty(sms * 2048)
    ops, per = ctypes.c_double(), ctypes.c_double()
    _check(lib.he_probe_mad_wide(ctx.h, _ptr(scratch), scratch.numel(), ctypes.byref(ops), ctypes.byref(per),
                                 _stream(stream)))
    return ops.value, per.value


def he_probe_tensor(ctx, kind, stream=None):
    """Dense tensor MMA rate (ops/s) on the context's GPU: kind 0 tcgen05 bf16 -> f32, kind 1
    mma.sync s8 -> s32."""
    sms = torch.cuda.get_device_properties(ctx.device).multi_processor_count
    scratch = torch.empty(4 * sms, dtype=torch.int32, device=ctx.device)
    ops = ctypes.c_double()
    _check(lib.he_probe_tensor(ctx.h, kind, ctypes.byref(ops), _ptr(scratch), scratch.numel(), _stream(stream)))
    return ops.value


def he_test_tc_gemm(ctx, A, B, stream=None):
    """A: (128, k), B: (n, k) torch.bfloat16 CUDA tensors; returns D = A B^T as (128, n)
    float32, computed by tcgen05."""
    assert A.is_cuda and B.is_cuda and A.is_contiguous() and B.is_contiguous()
    assert A.dtype == torch.bfloat16 and B.dtype == torch.bfloat16
    n, k = B.shape
    assert A.shape == (128, k)
    D = torch.empty((128, n), dtype=torch.float32, device=A.device)
    _check(lib.he_test_tc_gemm(ctx.h, n, k, _ptr(A), _ptr(B), _ptr(D), _stream(stream)))
    return D


def he_launch_count(ctx):
    v = ctypes.c_uint64()
    _check(lib.he_launch_count(ctx.h, ctypes.byref(v)))
    return v.value
