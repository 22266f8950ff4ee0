"""The C-ABI library builds, loads without a GPU, and exports every symbol include/hbsd.h declares."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hbsd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hbsd_[A-Za-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1308_2445_gb300 import build_lib, hbsd
    if not os.path.exists(build_lib.LIB):
        build_lib.build()
    return hbsd.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("hbsd_create", "hbsd_solve", "hbsd_destroy", "hbsd_update_H", "hbsd_status_string",
                 "hbsd_spmm_pair", "hbsd_precond_apply", "hbsd_minres", "hbsd_gram", "hbsd_rayleigh_ritz",
                 "hbsd_update", "hbsd_residual"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(lib):
    from paper_1308_2445_gb300 import hbsd
    assert set(_declared()) <= set(hbsd.exported_symbols())


def test_status_strings_and_defaults(lib):
    from paper_1308_2445_gb300 import hbsd
    assert lib.hbsd_status_string(0) == b"ok"
    assert lib.hbsd_status_string(-3).startswith(b"H - sigma_bar S")
    o = hbsd.options_default()
    assert (o.tau1, o.tau2, o.eta, o.max_minres, o.max_outer, o.m0) == (0.1, 0.1, 0.25, 20, 1000, -1)


def test_create_rejects_bad_input_without_gpu(lib):
    # argument validation happens before any CUDA call
    from paper_1308_2445_gb300 import hbsd
    import ctypes as C
    h = C.c_void_p()
    rc = lib.hbsd_create(None, None, None, None, None, C.byref(h))
    assert rc == hbsd.HBSD_ERR_ARG
    assert b"required" in lib.hbsd_last_error()
    # a 2 x 2 diagonal pair, then one defect at a time
    rp = (C.c_int64 * 3)(0, 1, 2)
    ci = (C.c_int32 * 2)(0, 1)
    ci_bad = (C.c_int32 * 2)(0, 2)
    ci_other = (C.c_int32 * 2)(1, 0)
    hv = (C.c_double * 2)(1.0, 2.0)
    sv = (C.c_double * 2)(1.0, 1.0)
    dn = (C.c_int32 * 2)(0, 0)
    lb = hbsd.hbsd_local_blocks(dof_node=C.cast(dn, C.POINTER(C.c_int32)))
    lb.grid[:] = [1, 1, 1]
    o = hbsd.options_default()
    o.sigma_bar = -1.0

    def csr(n, nnz, row_ptr, col_idx, val):
        return hbsd.hbsd_csr(n=n, nnz=nnz, row_ptr=C.cast(row_ptr, C.POINTER(C.c_int64)) if row_ptr else None,
                             col_idx=C.cast(col_idx, C.POINTER(C.c_int32)), val=C.cast(val, C.POINTER(C.c_double)),
                             is_complex=0)

    S = csr(2, 2, rp, ci, sv)
    for H, words in ((csr(2, 2, None, ci, hv), b"NULL CSR array"),      # checked before row_ptr is read
                     (csr(2, 3, rp, ci, hv), b"same n and nnz"),
                     (csr(2, 2, rp, ci_other, hv), b"one sparsity pattern")):
        assert lib.hbsd_create(C.byref(H), C.byref(S), C.byref(lb), C.byref(o), None, C.byref(h)) == hbsd.HBSD_ERR_ARG
        assert words in lib.hbsd_last_error(), lib.hbsd_last_error()
    Sb = csr(2, 2, rp, ci_bad, sv)
    Hb = csr(2, 2, rp, ci_bad, hv)
    assert lib.hbsd_create(C.byref(Hb), C.byref(Sb), C.byref(lb), C.byref(o), None, C.byref(h)) == hbsd.HBSD_ERR_ARG
    assert b"column index out of range" in lib.hbsd_last_error()
    H = csr(2, 2, rp, ci, hv)
    o.sigma_bar = float("nan")
    assert lib.hbsd_create(C.byref(H), C.byref(S), C.byref(lb), C.byref(o), None, C.byref(h)) == hbsd.HBSD_ERR_ARG
    assert b"sigma_bar" in lib.hbsd_last_error()
    o.sigma_bar = -1.0
    o.precond = 9
    assert lib.hbsd_create(C.byref(H), C.byref(S), C.byref(lb), C.byref(o), None, C.byref(h)) == hbsd.HBSD_ERR_ARG
    assert h.value is None


def test_library_start_block_generator_matches_inputs(lib):
    # the library draws the same SplitMix64 / Box-Muller normals as the shared input module
    import numpy as np
    from paper_1308_2445_gb300 import hbsd, pufe_inputs as pi
    for seed, count in ((1, 19 * 646), (5, 1001), (123456789, 8)):
        a = hbsd.seed_normals(seed, pi.STREAM_X0, count)
        b = pi.normal(seed, pi.STREAM_X0, count)
        assert np.allclose(a, b, rtol=1e-14, atol=1e-14)


def test_server_host_bookkeeping_without_gpu():
    # the request loop's argument checks and ticket bookkeeping run on the host; with an explicit
    # memory budget, creating and destroying a server makes no CUDA call
    from paper_1308_2445_gb300 import hbsd
    lib = hbsd.lib()
    o = hbsd.hbsd_server_opts()
    lib.hbsd_server_opts_default(ctypes.byref(o))
    assert o.max_slots == 4 and o.hbm_budget_bytes == 0
    o.max_slots = 0
    h = ctypes.c_void_p()
    assert lib.hbsd_server_create(ctypes.byref(o), ctypes.byref(h)) == hbsd.HBSD_ERR_ARG
    o.max_slots = 2
    o.hbm_budget_bytes = 1 << 30
    assert lib.hbsd_server_create(ctypes.byref(o), ctypes.byref(h)) == hbsd.HBSD_OK
    r = hbsd.hbsd_result()
    assert lib.hbsd_poll(h, ctypes.c_uint64(7), ctypes.byref(r)) == hbsd.HBSD_ERR_ARG      # unknown ticket
    rq = hbsd.hbsd_request()
    rq.session_id = 3
    rq.nev = 4
    rq.tol = 1e-8
    lam = (ctypes.c_double * 4)()
    t = ctypes.c_uint64(0)
    assert lib.hbsd_submit(h, ctypes.byref(rq), lam, None, ctypes.byref(t)) == hbsd.HBSD_ERR_ARG  # no session 3
    rq.nev = 0
    assert lib.hbsd_submit(h, ctypes.byref(rq), lam, None, ctypes.byref(t)) == hbsd.HBSD_ERR_ARG  # nev < 1
    rq.nev, rq.session_id = 4, -1
    assert lib.hbsd_submit(h, ctypes.byref(rq), lam, None, ctypes.byref(t)) == hbsd.HBSD_ERR_ARG  # no problem
    assert lib.hbsd_session_release(h, ctypes.c_int64(0)) == hbsd.HBSD_ERR_ARG
    lib.hbsd_server_destroy(h)


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    # no CPU fallback: with the shared library absent every call raises
    from paper_1308_2445_gb300 import hbsd
    monkeypatch.setattr(hbsd, "_lib", None)
    monkeypatch.setattr(hbsd, "LIB_PATH", str(tmp_path / "libhbsd.so"))
    with pytest.raises(RuntimeError, match="missing"):
        hbsd.lib()
    with pytest.raises(RuntimeError, match="missing"):
        hbsd.options_default()


def test_step_entry_points_refuse_a_short_leading_dimension(lib):
    # checked before any device work: a row-major block of q columns needs ld >= q
    from paper_1308_2445_gb300 import hbsd
    import ctypes as C
    buf = (C.c_double * 64)()
    p = C.cast(buf, C.POINTER(C.c_double))
    n, q = 8, 4
    assert lib.hbsd_update(p, 3, n, q, p, 2, None) == hbsd.HBSD_ERR_ARG
    assert b"leading dimension" in lib.hbsd_last_error()
    assert lib.hbsd_update_df64(p, 3, n, q, p, 2, None) == hbsd.HBSD_ERR_ARG
    assert lib.hbsd_gram(p, q, p, 2, p, q, n, q, p, p, None) == hbsd.HBSD_ERR_ARG
    assert b"leading dimension" in lib.hbsd_last_error()
    assert lib.hbsd_gram_df64(p, q, p, q, p, 1, n, q, p, p, None) == hbsd.HBSD_ERR_ARG
    assert lib.hbsd_gram_noalloc(p, 2, p, q, p, q, n, q, p, p, None) == hbsd.HBSD_ERR_ARG
    # k > q is refused as before
    assert lib.hbsd_update(p, q, n, q, p, q + 1, None) == hbsd.HBSD_ERR_ARG
    assert b"bad arguments" in lib.hbsd_last_error()


def test_server_admission_refuses_a_problem_beyond_its_budget_without_gpu():
    # the footprint estimate of a new problem (matrix, factor at the measured fill, solve blocks)
    # is checked against the budget at submission, on the host: a real 8^3 problem and its complex
    # (Bloch) twin, whose real pencil is twice as large, against a 64 MiB budget
    from paper_1308_2445_gb300 import hbsd, pufe_inputs as pi
    sv = hbsd.Server(max_slots=1, hbm_budget_bytes=64 << 20)
    for p in (pi.small_case(1), pi.generate(8, 2, 2, 0.25, 4, kpt=(0.5 * np.pi, 0.5 * np.pi, 0.5 * np.pi))):
        with pytest.raises(hbsd.HbsdError) as e:
            sv.submit(16, 1e-8, problem=p, want_vectors=False)
        assert e.value.code == hbsd.HBSD_ERR_OOM
    sv.close()
