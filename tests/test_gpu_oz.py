"""Steps 10-11 on the tensor cores (hbsd_update_oz): Y = [Z0 Z1] W from exact bf16 slices of the
FP64 operands, checked against the FP64 product with the bound of the method (fixed point against
each row's and column's largest entry, per block), on ragged sizes, with the two blocks' rows at
very different magnitudes, and with the second block empty."""
import numpy as np
import pytest

from paper_1308_2445_gb300 import pufe_inputs as pi

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import os
    from paper_1308_2445_gb300 import build_lib
    if not os.path.exists(build_lib.LIB):
        build_lib.build()


def dev(a, pad=2):
    a = np.ascontiguousarray(a, dtype=np.float64)
    n, k = a.shape
    t = torch.zeros(n, k + (-k) % pad, dtype=torch.float64, device="cuda")[:, :k]
    t.copy_(torch.from_numpy(a))
    return t


def run(Z0, Z1, W, k):
    from paper_1308_2445_gb300 import hbsd
    n, q0 = Z0.shape
    q1 = 0 if Z1 is None else Z1.shape[1]
    a, w = dev(Z0), torch.from_numpy(np.ascontiguousarray(W)).cuda()
    b = dev(Z1) if q1 else None
    Y = dev(np.full((n, k), np.nan))
    rc = hbsd.lib().hbsd_update_oz(a.data_ptr(), a.stride(0), q0, b.data_ptr() if q1 else None,
                                   b.stride(0) if q1 else 0, q1, n, w.data_ptr(), k, Y.data_ptr(), Y.stride(0), None)
    assert rc == 0, hbsd.lib().hbsd_last_error()
    torch.cuda.synchronize()
    return Y.cpu().numpy()


def bound(Zs, Ws):
    """Error bound of the method, summed over the blocks g: truncating an entry to 48 bits of its
    row's (or column's) scale 2^E < 2 max costs below 2^-47 max, hence
    2^-47 (max|Z_g(i,:)| |W_g(:,j)|_1 + |Z_g(i,:)|_1 max|W_g(:,j)|); the dropped digit products of
    weight 2^-54 and below add under 2^-49.4 max|Z_g(i,:)| max|W_g(:,j)| per term, q_g terms.
    Stated with a factor 2 of room: 2^-46 (...) + q_g 2^-48 max max."""
    out = 0.0
    for Z, W in zip(Zs, Ws):
        rmax = np.abs(Z).max(axis=1)[:, None]
        cmax = np.abs(W).max(axis=0)[None, :]
        out = out + 2.0 ** -46 * (rmax * np.abs(W).sum(axis=0)[None, :] + np.abs(Z).sum(axis=1)[:, None] * cmax)
        out = out + Z.shape[1] * 2.0 ** -48 * rmax * cmax
    return out


@pytest.mark.parametrize("n,q0,q1,k", [(1000, 19, 16, 16), (5000, 85, 64, 85), (3001, 282, 256, 282),
                                       (700, 135, 0, 71), (130, 640, 520, 300)])
def test_update_oz_against_fp64(n, q0, q1, k):
    Z0 = pi.seed_normal_block(q0 + 3, n, q0) * np.logspace(-4, 4, q0)
    Z1 = pi.seed_normal_block(q1 + 5, n, q1) if q1 else None
    W = pi.seed_normal_block(k + 7, q0 + q1, k)
    Y = run(Z0, Z1, W, k)
    ref = Z0 @ W[:q0] + (Z1 @ W[q0:] if q1 else 0.0)
    b = bound([Z0] + ([Z1] if q1 else []), [W[:q0]] + ([W[q0:]] if q1 else []))
    err = np.abs(Y - ref)
    assert np.isfinite(Y).all()
    assert np.all(err <= b), float((err / b).max())
    # typical accuracy: FP64-class relative to the entries' own size
    rel = err / (np.abs(Z0) @ np.abs(W[:q0]) + (np.abs(Z1) @ np.abs(W[q0:]) if q1 else 0.0))
    assert np.median(rel) <= 1e-14


def test_update_oz_blocks_of_very_different_magnitude():
    """Rows of the second block 1e10 times larger, its coefficients 1e10 times smaller (directions
    with large components along the near-null space of S, small weights): each block keeps its own
    scale, so the first block's part is computed as accurately as on its own."""
    n, q0, q1, k = 2000, 71, 57, 71
    Z0 = pi.seed_normal_block(11, n, q0)
    Z1 = pi.seed_normal_block(12, n, q1) * 1e10
    W = pi.seed_normal_block(13, q0 + q1, k)
    W[q0:] *= 1e-10
    Y = run(Z0, Z1, W, k)
    ref = Z0 @ W[:q0] + Z1 @ W[q0:]
    scale = np.abs(Z0) @ np.abs(W[:q0]) + np.abs(Z1) @ np.abs(W[q0:])
    assert np.all(np.abs(Y - ref) <= bound([Z0, Z1], [W[:q0], W[q0:]]))
    # the first block's own part is not swamped: errors stay far below its terms' size
    assert np.median(np.abs(Y - ref) / scale) <= 1e-14


def test_update_oz_edge_values():
    """Zeros, signs, subnormal-range and widely spread magnitudes in one row pass through the
    identity to the fixed-point accuracy of the row's largest entry (2^-47 of it)."""
    v = np.array([0.0, -0.0, 1.0, -1.0, 2.0 ** 100, -(2.0 ** -100), 1e30, -1e-28, 3.141592653589793,
                  1.0 + 2.0 ** -40, 1e-39, -1e-300, 5e-324, -1e-35, 7.0, -7.5])
    q = v.size
    Z = v[None, :].copy()
    Y = run(Z, None, np.eye(q), q)[0]
    assert np.all(np.abs(Y - v) <= 2.0 ** -46 * np.abs(v).max())
    assert Y[0] == 0.0 and Y[4] == 2.0 ** 100
