"""The reduction's block Jacobi (lattice_sum_jacobi_eig) on its own.

Claim under test: one run of the block Jacobi diagonalises a symmetric
matrix (with the rotation floor above E's FP32 noise, as in the reduction). The diagonal is an FP32 hi/lo pair, and E and the rotation
accumulator are FP32. With tol = 1e-7, against bounds taken from that
FP32 representation accumulated over tens of sweeps (the pipeline's
second run, on the nearly diagonal U^T H U, is what reaches FP64 level):
- the eigenvalues come out within 4e-6 of ||H||: each eigenvalue gathers the
  roundings (2^-24 of ||H|| each) of the sweeps x k rotations that touch its
  row, a random sum of about sqrt(13 x 488) 2^-24 = 5e-6 of ||H|| at the
  largest size here (measured: up to 1.1e-6);
- the accumulated rotation V = I + F is orthogonal within 1e-4;
- H V = V diag(D) holds within 1e-5 ||H||.
The grid form, with the matrices in global memory, performs the same
rounds with the same arithmetic as the cluster form, with the matrix in
shared memory. Where both apply they give bitwise the same D and V.

Inputs: H = Q diag(lambda) Q^T with Q a seeded random orthogonal matrix.
lambda is either graded (1 down to 1e-10, like the compressed Gram matrices
of the truncation step) or holds clustered pairs. The reference is
numpy.linalg.eigh in FP64.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1411_1994_gb300 import build as B  # noqa: E402
from paper_1411_1994_gb300 import lattice_sum as L  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    B.build()
    L.lib()


def _matrix(k, seed, spectrum="graded"):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((k, k)))
    if spectrum == "graded":
        lam = 10.0 ** np.linspace(0.0, -10.0, k)
    else:   # clustered pairs
        base = 10.0 ** np.linspace(0.0, -6.0, (k + 1) // 2)
        lam = np.sort(np.concatenate([base, base * (1 + 1e-9)])[:k])[::-1]
    H = (Q * lam) @ Q.T
    return 0.5 * (H + H.T), np.sort(lam)[::-1]


def _run(H, form, tol=1e-7):
    # the floor sits above the FP32 noise of E (entries rounded to 2^-24 of |H_ij| <= ||H||),
    # as the reduction's resolution floor does
    floor = 1e-8 * float(np.abs(H).max())
    D, V, sweeps = L.jacobi_eig(torch.from_numpy(H).cuda(), tol=tol, abs_floor=floor, form=form)
    return D.cpu().numpy(), V.cpu().numpy(), sweeps


@pytest.mark.parametrize("k,spectrum", [(40, "graded"), (185, "graded"), (200, "clustered"), (17, "graded"), (208, "graded")])
def test_grid_form_equals_cluster_form(k, spectrum):
    H, _ = _matrix(k, 100 + k, spectrum)
    D1, V1, s1 = _run(H, 1)
    D2, V2, s2 = _run(H, 2)
    assert np.array_equal(D1, D2)
    assert np.array_equal(V1, V2)
    # the grid form confirms convergence by one empty sweep, the cluster form by a scan
    assert s2 in (s1, s1 + 1), (s1, s2)


@pytest.mark.parametrize("k,spectrum", [(300, "graded"), (488, "graded"), (333, "clustered")])
def test_grid_form_large(k, spectrum):
    H, lam = _matrix(k, 200 + k, spectrum)
    D, V, sweeps = _run(H, 2)
    norm = np.abs(lam).max()
    assert np.max(np.abs(np.sort(D)[::-1] - lam)) <= 4e-6 * norm
    assert np.max(np.abs(V.T @ V - np.eye(k))) <= 1e-4
    assert np.max(np.abs(H @ V - V * D)) <= 1e-5 * norm
    assert 1 <= sweeps <= 30


def test_bad_arguments():
    H = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(Exception):
        L.jacobi_eig(H, tol=0.0)
    with pytest.raises(Exception):
        L.jacobi_eig(H, form=3)
    big = torch.zeros((600, 600), dtype=torch.float64, device="cuda")
    with pytest.raises(Exception):
        L.jacobi_eig(big, form=1)   # beyond the cluster form's shared memory
