"""The one-sided (Hestenes) Jacobi of the non-squaring route
(lattice_sum_svd_rows) against independent references.

Def. 4.1 truncates by the singular values of each side matrix; the FP64 path
takes them by plane rotations of pairs of rows of B = Q^T A_w, never forming
B B^T. Such rotations keep each singular value to the relative accuracy of its
row (Demmel & Veselic, SIAM J. Matrix Anal. Appl. 13, 1992): for B = D W with
D diagonal and W well conditioned, sigma_k is good to about u cond(W)
relative, however graded D is. The tests pin:
  * plain random matrices: the sorted singular values against LAPACK's SVD
    (numpy) to 1e-14 sqrt(C) of sigma_1; M orthogonal; M B with orthogonal rows;
  * graded matrices B = D W (row scales down to 1e-14): every singular value to
    1e-12 relative against a different algorithm with the same guarantee:
    two-sided cyclic Jacobi, written here, on the Gram matrix D (W W^T) D,
    whose entries are formed from correctly rounded dot products (exact
    products by Veltkamp/Dekker splitting, summed by math.fsum), so that each
    entry carries only its own relative rounding;
  * rank-deficient B (repeated and zero rows) and argument errors.
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


def run(Bh):
    sig2, M, sweeps, rots = L.svd_rows(torch.from_numpy(Bh).cuda())
    return sig2.cpu().numpy(), M.cpu().numpy(), sweeps, rots


@pytest.mark.parametrize("m,C", [(40, 96), (173, 408), (64, 64), (7, 300)])
def test_plain_random_against_lapack(m, C):
    rng = np.random.default_rng(m * 1000 + C)
    Bh = rng.standard_normal((m, C))
    sig2, M, sweeps, rots = run(Bh)
    s = np.sort(np.sqrt(sig2))[::-1]
    ref = np.linalg.svd(Bh, compute_uv=False)
    assert np.max(np.abs(s - ref)) <= 1e-14 * ref[0] * np.sqrt(C), np.max(np.abs(s - ref))
    assert np.max(np.abs(M @ M.T - np.eye(m))) < 1e-14 * np.sqrt(m)
    # the rows of M B mutually orthogonal; this check forms M B in FP64, whose rounding
    # (u ||M_i|| ||B|| per row) sets the floor: u m sigma_1 / sigma_i in the cosine
    R = M @ Bh
    G = R @ R.T
    d = np.sqrt(np.diag(G))
    off = np.abs(G / np.outer(d, d) - np.eye(m))
    assert off.max() < 1e-15 * m * ref[0] / ref[-1], (off.max(), ref[0] / ref[-1])
    assert sweeps <= 12 and rots[-1] <= rots[0]


def two_product(a, b):
    """a * b = p + e exactly (Veltkamp split, Dekker's product), elementwise."""
    f = 134217729.0   # 2^27 + 1
    p = a * b
    ca, cb = f * a, f * b
    ah = ca - (ca - a)
    al = a - ah
    bh = cb - (cb - b)
    bl = b - bh
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return p, e


def exact_gram(W):
    """W W^T with each entry the correctly rounded dot product."""
    import math
    m = W.shape[0]
    A = np.empty((m, m))
    for i in range(m):
        for j in range(i, m):
            p, e = two_product(W[i], W[j])
            A[i, j] = A[j, i] = math.fsum(np.concatenate([p, e]))
    return A


def two_sided_jacobi_eigenvalues(H, sweeps=40):
    """Eigenvalues of a symmetric positive definite H by cyclic two-sided Jacobi: for each
    pair (p, q) the rotation that zeroes H[p, q]; stop when every |H[p, q]| <= u sqrt(H[p, p]
    H[q, q]). Relative accuracy on graded H = D A D (Demmel & Veselic 1992)."""
    import math
    H = H.copy()
    m = H.shape[0]
    u = 2.0 ** -53
    for _ in range(sweeps):
        rotated = False
        for p in range(m - 1):
            for q in range(p + 1, m):
                hpq = H[p, q]
                if abs(hpq) <= u * math.sqrt(H[p, p] * H[q, q]):
                    continue
                rotated = True
                theta = (H[q, q] - H[p, p]) / (2.0 * hpq)
                t = math.copysign(1.0, theta) / (abs(theta) + math.sqrt(1.0 + theta * theta))
                c = 1.0 / math.sqrt(1.0 + t * t)
                s = t * c
                hp, hq = H[p].copy(), H[q].copy()
                H[p], H[q] = c * hp - s * hq, s * hp + c * hq
                hp, hq = H[:, p].copy(), H[:, q].copy()
                H[:, p], H[:, q] = c * hp - s * hq, s * hp + c * hq
        if not rotated:
            break
    return np.diag(H).copy()


@pytest.mark.parametrize("m,C,decades", [(40, 120, 14), (60, 200, 12)])
def test_graded_rows_relative_accuracy(m, C, decades):
    """B = D W, W random m x C, D = diag(10^(-decades k / m)) (largest first, rows in a
    shuffled order): every singular value, down to 10^-decades of the largest, to 1e-12
    relative against two-sided Jacobi on the correctly rounded graded Gram matrix."""
    rng = np.random.default_rng(decades * 7 + m)
    W = rng.standard_normal((m, C))
    d = 10.0 ** (-decades * rng.permutation(m) / m)
    Bh = d[:, None] * W
    sig2, M, sweeps, rots = run(Bh)
    s = np.sort(np.sqrt(sig2))[::-1]
    H = d[:, None] * exact_gram(W) * d[None, :]
    ref = np.sqrt(np.sort(two_sided_jacobi_eigenvalues(H))[::-1])
    assert np.all(np.abs(s - ref) <= 1e-12 * ref), float(np.max(np.abs(s - ref) / ref))
    assert np.max(np.abs(M @ M.T - np.eye(m))) < 1e-14 * np.sqrt(m)


def test_rank_deficient_rows():
    rng = np.random.default_rng(3)
    W = rng.standard_normal((10, 50))
    Bh = np.vstack([W, W[:3] * 2.0, np.zeros((2, 50))])
    sig2, M, sweeps, rots = run(Bh)
    s = np.sort(np.sqrt(np.maximum(sig2, 0.0)))[::-1]
    ref = np.linalg.svd(Bh, compute_uv=False)
    assert np.max(np.abs(s - ref)) <= 1e-13 * ref[0]
    assert np.sum(s > 1e-12 * s[0]) == 10


def test_bad_arguments():
    x = torch.zeros((3, 4), dtype=torch.float64, device="cuda")
    import ctypes as C
    for m, Cc, tol in ((0, 4, 1e-15), (3, 0, 1e-15), (3, 4, 0.0)):
        rc = L.lib().lattice_sum_svd_rows(C.c_void_p(x.data_ptr()), m, Cc, C.c_double(tol), 0,
                                          C.c_void_p(x.data_ptr()), C.c_void_p(x.data_ptr()), None, None, None)
        assert rc == L.LS_ERR_ARG
