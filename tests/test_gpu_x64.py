"""The FP64-grade tensor-core product (lattice_sum_gemm_nt), which carries the
reduction's dense FP64 contractions (Gram matrices, CholeskyQR, FP64
projection), checked on its own.

Claim under test: every row is scaled by a power of two and written as eight
balanced base-128 digits (integers in [-64, 64], exact in BF16); the digit
products of one level, summed over K <= 512, stay below 2^24 and so
accumulate exactly in FP32 on the tensor cores; the result is then good to
about 2^-53 sum_k |a_k||b_k|, as an FP64 dot product is.

1. Random matrices spanning several K chunks and ragged tiles, against the
   correctly rounded dot products (math.fsum of the exact FP64 products):
   |error| <= 4 * 2^-53 * sum_k |a_k||b_k| element by element.
2. Adversarial digits: every entry equal to x* whose digits are
   (-63, -64, ..., -64), so that the highest level's partial sums reach
   2^24 - 32768 at K = 512 (the edge of exact FP32 accumulation). The
   product K x*^2 must come out as the correctly rounded value up to one ulp;
   a tensor core that dropped low bits of those sums would miss it by ~2^-24.
3. Signs and zero rows: a zero row gives an exact zero; negated operands give
   the negated result within the error bound (balanced digits of -x are not
   always the negated digits of x, so the dropped terms below 2^-56 may
   differ).
"""
import math
from fractions import Fraction

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1411_1994_gb300 import build as B  # noqa: E402
from paper_1411_1994_gb300 import lattice_sum as L  # noqa: E402

pytestmark = pytest.mark.gpu
U = 2.0 ** -53


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    B.build()
    L.lib()


@pytest.mark.parametrize("M,N,K", [(130, 70, 1100), (7, 200, 64), (256, 128, 512), (1, 1, 1)])
def test_random_against_correctly_rounded(M, N, K):
    rng = np.random.default_rng(M * 1000 + N + K)
    # graded rows (magnitudes over 12 decades) like the reduction's operands
    A = rng.standard_normal((M, K)) * (10.0 ** rng.uniform(-6, 6, size=(M, 1)))
    Bm = rng.standard_normal((N, K)) * (10.0 ** rng.uniform(-6, 6, size=(N, 1)))
    D = L.gemm_nt(torch.from_numpy(A).cuda(), torch.from_numpy(Bm).cuda()).cpu().numpy()
    # reference: the exact dot product correctly rounded (Fractions) on a sample of entries;
    # elsewhere fsum of the FP64-rounded products (within u sum |a b| of it)
    ref = np.empty((M, N))
    absdot = np.abs(A) @ np.abs(Bm).T
    for m in range(M):
        for n in range(N):
            if (m + n) % 97 == 0:
                ref[m, n] = float(sum(Fraction(a) * Fraction(b) for a, b in zip(A[m], Bm[n])))
            else:
                ref[m, n] = math.fsum(A[m] * Bm[n])
    err = np.abs(D - ref)
    assert np.all(err <= 4 * U * absdot + 1e-300), float(np.max(err / np.maximum(absdot, 1e-300)))


def x_star():
    digits = [-63] + [-64] * 7
    v = sum(Fraction(d, 128 ** (i + 1)) for i, d in enumerate(digits))
    x = float(v)
    assert Fraction(x) == v   # exactly representable: the low digits are multiples of 64
    return x


@pytest.mark.parametrize("K", [512, 1024, 1536])
def test_adversarial_digits_exact_accumulation(K):
    x = x_star()
    A = np.full((128, K), x)
    Bm = np.full((64, K), x)
    D = L.gemm_nt(torch.from_numpy(A).cuda(), torch.from_numpy(Bm).cuda()).cpu().numpy()
    exact = float(K * Fraction(x) * Fraction(x))
    ulp = math.ulp(exact)
    assert np.all(np.abs(D - exact) <= ulp), float(np.max(np.abs(D - exact)) / ulp)


def test_zero_rows_and_sign_symmetry():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((40, 300))
    Bm = rng.standard_normal((33, 300))
    A[3] = 0.0
    Bm[7] = 0.0
    tA, tB = torch.from_numpy(A).cuda(), torch.from_numpy(Bm).cuda()
    D = L.gemm_nt(tA, tB).cpu().numpy()
    assert np.all(D[3] == 0.0) and np.all(D[:, 7] == 0.0)
    Dn = L.gemm_nt(-tA, tB).cpu().numpy()
    assert np.all(np.abs(Dn + D) <= 4 * U * (np.abs(A) @ np.abs(Bm).T))


def test_bad_arguments():
    assert L.lib().lattice_sum_gemm_nt(None, None, 4, 4, 8, None, None) == L.LS_ERR_ARG
    with pytest.raises(ValueError):
        L.gemm_nt(torch.zeros((4, 8), dtype=torch.float64, device="cuda"),
                  torch.zeros((4, 9), dtype=torch.float64, device="cuda"))
