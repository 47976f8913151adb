"""Host-side checks of the C ABI library (no GPU needed): the library loads,
exports every entry point its header declares, validates arguments before
touching a device, and its host-only helpers behave."""
import re
from pathlib import Path

import numpy as np
import pytest

ROOT = Path(__file__).resolve().parent.parent


@pytest.fixture(scope="module")
def B():
    from paper_2305_18396_gb300 import build

    build.build()
    from paper_2305_18396_gb300 import binding

    return binding


def declared_symbols():
    names = set()
    for h in (ROOT / "include").glob("*.h"):
        names |= set(re.findall(r"^HE_API\s+[^(]*?\b(he_\w+)\s*\(", h.read_text(), re.M))
    return names


def test_every_declared_symbol_is_exported(B):
    names = declared_symbols()
    assert len(names) >= 20
    for n in sorted(names):
        assert hasattr(B.lib, n), n


def test_params_init_rejects_bad_parameters_without_gpu(B):
    import ctypes

    q_ok = (1125625028935681, 1125487589982209)
    cases = [
        (4096, 2, q_ok, 37, "ok-shape"),
        (3000, 2, q_ok, 37, "N not a power of two"),
        (16384, 2, q_ok, 37, "N too large"),
        (4096, 4, q_ok + (1, 1), 37, "L too large"),
        (4096, 2, (q_ok[0], q_ok[0]), 37, "repeated prime"),
        (4096, 2, (q_ok[0], q_ok[0] + 2 * 4096 * 2), 37, "composite"),
        (4096, 2, q_ok, 60, "t too large"),
        (4096, 1, (65537,), 37, "q below t"),
        (4096, 1, (562949953216513,), 37, "prime 1 mod 2N but not 1 mod 2^32"),
    ]
    for N, L, q, lt, why in cases:
        if why == "ok-shape":
            continue
        arr = (ctypes.c_uint64 * len(q))(*q)
        h = ctypes.c_void_p()
        rc = B.lib.he_params_init(ctypes.byref(h), N, L, arr, lt, 0)
        assert rc == B.HE_EINVAL, why
        assert h.value is None
        assert B.lib.he_last_error().decode()


def test_choose_blocking_properties(B):
    from paper_2305_18396_gb300 import workloads

    for N, L in ((4096, 2), (8192, 3), (1024, 2)):
        for p in workloads.bert_layer_products(distinct_heads=1, **workloads.BERT_BASE):
            mb, kb, nb = B.he_choose_blocking(N, L, p.m, p.k, p.n)
            assert mb * kb * nb <= N
            for v in (mb, kb, nb):
                assert v & (v - 1) == 0
    assert B.he_choose_blocking(4096, 2, 1, 1, 1) == (1, 1, 1)
    assert B.he_choose_blocking(4096, 2, 16, 64, 64)[0] * 64 >= 16  # covers the rows
    with pytest.raises(B.HEError):
        B.he_choose_blocking(3000, 2, 4, 4, 4)


def test_library_gauss_table_matches_oracle(B):
    """The library's inversion table is generated independently of the oracle's; both are
    exact floors of the same quantity and must agree word for word."""
    from oracle.core import lib, p64

    t = np.zeros(38, dtype=np.uint64)
    lib.or_gauss_cdt(p64(t))
    assert B.he_gauss_cdt() == [int(x) for x in t]


def test_binding_refuses_missing_library(tmp_path, monkeypatch):
    """No CPU fallback: a missing library is an ImportError."""
    import importlib
    import sys

    import paper_2305_18396_gb300.build as build

    monkeypatch.setattr(build, "LIB", tmp_path / "missing.so")
    saved = sys.modules.pop("paper_2305_18396_gb300.binding", None)
    try:
        with pytest.raises(ImportError):
            importlib.import_module("paper_2305_18396_gb300.binding")
    finally:
        sys.modules.pop("paper_2305_18396_gb300.binding", None)
        if saved is not None:
            sys.modules["paper_2305_18396_gb300.binding"] = saved


def test_wire_format_calls_reject_a_null_context_without_gpu(B):
    import ctypes

    buf = (ctypes.c_uint64 * 4)()
    for fn in (B.lib.he_ct_export, B.lib.he_ct_import):
        assert fn(None, buf, 1, 0, buf, None) == B.HE_EINVAL
        assert "ctx" in B.lib.he_last_error().decode()


def test_pipe_calls_reject_null_arguments_without_gpu(B):
    import ctypes

    h = ctypes.c_void_p()
    assert B.lib.he_pipe_create(None, 3, ctypes.byref(h)) == B.HE_EINVAL
    assert B.lib.he_pipe_submit(None, 1, None, None, 0) == B.HE_EINVAL
    assert "pipe" in B.lib.he_last_error().decode()
    assert B.lib.he_pipe_wait(None) == B.HE_EINVAL
    out = ctypes.c_void_p()
    assert B.lib.he_pipe_compute_stream(None, ctypes.byref(out)) == B.HE_EINVAL
    sz = ctypes.c_size_t()
    assert B.lib.he_pipe_workspace_bytes(None, 0, None, ctypes.byref(sz)) == B.HE_EINVAL
    assert B.lib.he_pipe_free(None) == B.HE_OK


def test_cost_model_fills_ciphertexts_with_rows_in_the_coset_form(B):
    """Coset products store 2D residues per weight block whatever m_b is, so the cost model
    packs a whole sequence into each ciphertext (m_b = m) for the BERT-large products at
    N = 8192 and keeps n_b k_b = N / m_b (every coefficient used)."""
    from paper_2305_18396_gb300 import workloads

    for p in workloads.bert_layer_products(distinct_heads=1, **workloads.BERT_LARGE):
        mb, kb, nb = B.he_choose_blocking(8192, 3, p.m, p.k, p.n)
        if p.m == 512:
            assert mb == 512, (p.name, mb, kb, nb)
        assert mb * kb * nb == 8192, (p.name, mb, kb, nb)
        assert kb * nb <= 4096  # n_b k_b <= N/2: the coset form applies
