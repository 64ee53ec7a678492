"""FP64-class products of FP64 matrices on the tensor cores (the digit split: 42-bit fixed-point
digits per column / row exponent, 7 BF16 slices, 28 exact products) against numpy FP64.

  C = A^T B over K chunks with a ragged tail and several K splits (the adjoint's Zh^T W);
  C = X L^-1 with the device model's factor (the adjoint's Zh L^-1), across a row-chunk border.

Bound per element: K 2^-38 max|A_:i| max|B_:j| (rounding to 42 bits is 2^-43 of the column's
power-of-two scale per operand; the dropped levels 7..12 add under 2^-40), and the median error
relative to sum_k |a_ki b_kj| must stay below 1e-10 (FP32-class products sit near 1e-7; with row
scales spread over 10^4 the column exponent, not the entry, sets the digits' resolution)."""
import numpy as np
import pytest
from scipy.linalg import solve_triangular

import workloads
from gpu_util import model_of, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


@pytest.fixture(scope="module")
def g():
    import paper_2512_12442_gb300 as g
    return g


def _wide(rng, rows, cols):
    """Normal entries with column scales 10^U(-3,3) and row scales 10^U(-2,2); one zero column."""
    a = rng.standard_normal((rows, cols))
    a *= 10.0 ** rng.uniform(-3, 3, cols)[None, :]
    a *= 10.0 ** rng.uniform(-2, 2, rows)[:, None]
    a[:, 3] = 0.0
    return a


@pytest.mark.parametrize("K,nc,kchunk,nsplit", [(70000, 200, 32768, 7), (1000, 64, 0, 19), (37, 500, 0, 3)])
def test_mul_tn_vs_numpy(torch, g, K, nc, kchunk, nsplit):
    rng = np.random.default_rng(K + nc)
    A, B = _wide(rng, K, nc), _wide(rng, K, nc)
    C = g.gpr_oz_mul_tn_test(torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda"), kchunk, nsplit)
    C = C.cpu().numpy()
    ref = A.T @ B
    err = np.abs(C - ref)
    bound = K * 2.0 ** -38 * np.outer(np.abs(A).max(0), np.abs(B).max(0))
    assert np.all(err <= bound), float(np.max(err / np.maximum(bound, 1e-300)))
    mag = np.abs(A).T @ np.abs(B)
    rel = err[mag > 0] / mag[mag > 0]
    assert np.median(rel) < 1e-10, float(np.median(rel))
    assert np.all(C[:, 3] == 0.0) and np.all(C[3, :] == 0.0)


@pytest.mark.parametrize("rows", [3000, 230000])
def test_mul_linv_vs_numpy(torch, g, rows):
    """X L^-1 for the m=500 field's factor; 230000 rows cross the 1.5 GB digit-chunk border."""
    w = workloads.config5()
    M = model_of(w)
    L = g.gpr_model_export(M)["L"]
    Linv = solve_triangular(L, np.eye(L.shape[0]), lower=True)
    rng = np.random.default_rng(rows)
    X = _wide(rng, rows, w.m)
    Z = g.gpr_oz_mul_linv_test(M, torch.tensor(X, device="cuda")).cpu().numpy()
    ref = X @ Linv
    err = np.abs(Z - ref)
    mag = np.abs(X) @ np.abs(Linv)
    bound = w.m * 2.0 ** -38 * np.outer(np.abs(X).max(1), np.abs(Linv).max(0)) + 1e-11 * mag
    assert np.all(err <= bound), float(np.max(err / np.maximum(bound, 1e-300)))
    rel = err[mag > 0] / mag[mag > 0]
    assert np.median(rel) < 1e-10, float(np.median(rel))
