"""hbsd_gram_noalloc: the allocation-free Gram for callers that must not allocate device memory
(a serving loop whose per-request path may not call cudaMalloc/cudaFree, which can synchronise
the whole device; a host whose own pool owns all device memory).  Checked through the C ABI
against hbsd_gram on two calls in a row, with the tolerance of the other Gram tests."""
import ctypes as C
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1308_2445_gb300 import build_lib
    if not os.path.exists(build_lib.LIB):
        build_lib.build()


def _block(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    n, k = a.shape
    t = torch.zeros(n, k + (k % 2), dtype=torch.float64, device="cuda")[:, :k]
    t.copy_(torch.from_numpy(a))
    return t


def _gram(fn, Z, ZH, ZS):
    q = Z.shape[1]
    HR = torch.full((q, q), float("nan"), dtype=torch.float64, device="cuda")
    SR = torch.full((q, q), float("nan"), dtype=torch.float64, device="cuda")
    rc = fn(Z.data_ptr(), Z.stride(0), ZH.data_ptr(), ZH.stride(0), ZS.data_ptr(), ZS.stride(0),
            Z.shape[0], q, HR.data_ptr(), SR.data_ptr(), None)
    assert rc == 0
    torch.cuda.synchronize()
    return HR.cpu().numpy(), SR.cpu().numpy()


def test_noalloc_gram_matches_gram_on_consecutive_calls():
    from paper_1308_2445_gb300 import hbsd, pufe_inputs as pi
    lib = hbsd.lib()
    # q = 135 and 71 keep hbsd_gram's row chunks; q = 400 and 1024 make the static scratch cut
    # the chunk count (1 chunk at q = 1024, the largest q it holds)
    for call, (n, q) in enumerate([(47620, 135), (4000, 71), (47620, 135), (20000, 400), (4096, 1024),
                                   (4096, 1024)]):
        Z = _block(pi.seed_normal_block(10 + call, n, q))
        ZH = _block(pi.seed_normal_block(20 + call, n, q))
        ZS = _block(pi.seed_normal_block(30 + call, n, q))
        HRa, SRa = _gram(lib.hbsd_gram, Z, ZH, ZS)
        HRb, SRb = _gram(lib.hbsd_gram_noalloc, Z, ZH, ZS)
        for a, b in ((HRa, HRb), (SRa, SRb)):
            assert np.isfinite(b).all()
            assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


def test_noalloc_gram_rejects_sizes_beyond_its_scratch():
    from paper_1308_2445_gb300 import hbsd
    lib = hbsd.lib()
    # leading dimensions that fit q = 1025, so only the scratch limit can refuse the call; it is
    # refused on the host before any launch (nothing is read or written)
    t = torch.zeros(4, 1026, dtype=torch.float64, device="cuda")
    p = t.data_ptr()
    rc = lib.hbsd_gram_noalloc(p, 1026, p, 1026, p, 1026, 4, 1025, p, p, None)
    assert rc == hbsd.HBSD_ERR_ARG
    assert b"exceeds the static scratch" in lib.hbsd_last_error()
    # the same refusal with a leading dimension below q: the scratch limit is reported first
    rc = lib.hbsd_gram_noalloc(p, 2, p, 2, p, 2, 4, 1025, p, p, None)
    assert rc == hbsd.HBSD_ERR_ARG
    assert b"exceeds the static scratch" in lib.hbsd_last_error()
