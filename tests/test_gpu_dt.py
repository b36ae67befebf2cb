"""The mixed slab evaluation's tensor-core product (lattice_sum_gemm_nt_mixed),
checked on its own.

Claim under test:
- Operand rows (FP64) are scaled by 2^(6-E), where max|x| lies in
  [2^(E-1), 2^E).
- Each scaled row is written as d0 + d1 2^-7 + t1 + t2, with d0, d1 nearest
  integers in [-64, 64] and t1, t2 11-bit rests (FP16, scaled by 2^9).
  This is good to 2^-30 of a digit unit.
- On the tensor cores, the level-0 products (d0 d0) and the level-1 products
  (d0 d1 + d1 d0) 2^-7 accumulate EXACTLY in FP32 for K <= 2048; for K up to
  4096 the two level-1 products take one accumulator each and stay exact.
- The products below them go to a third accumulator, at 2^-14 of the
  result or less. Its adds truncate, so it drifts in one direction by about
  half an ulp of its running sum per MMA: on random data (a running sum
  growing like sqrt(k)) that error grows like K^1.5.
- The dropped products are below 2^-30 of max|a| max|b| per term.

1. Random matrices (graded row magnitudes, ragged M, N, several k-blocks, K up
   to 4096), FP64 output, against the FP64 product: every entry's error is at
   most (2^-28 sqrt(K) + 2^-37 K^1.5) * max|a_m| * max|b_n|. The first term is
   a wide margin over the dropped terms' random sum (about 2^-34 sqrt(K)); the
   second is twice the drift of the third accumulator measured at K = 2081
   and 4096 (2^-22.4 and 2^-21.0 of max|a| max|b|).
2. Exact accumulation of the leading levels: entries (128 d0 + d1) / 2^13
   with integer digits, so the tails vanish. Every level's sums are then
   integers below 2^24 in their units, and at K = 2048 the level-1 sums
   reach 2^24 (at K = 4096 each of the two level-1 accumulators does). The
   result must equal the exact integer product bit for bit.
   A tensor core that dropped low bits of any level would miss it.
3. Exact cancellation: a_k = x (-1)^k, b_k = x gives exactly zero (every part
   cancels term by term at even K).
4. The tile width changes only the grouping of outputs, not any output's
   sequence of products: results are bitwise equal for tile widths 32..128.
5. Zero rows give exact zeros. The FP32 output is the exact sum rounded once,
   so it is the FP64 output rounded to FP32 (within half an FP32 ulp).
"""
import math

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


def _graded(rng, rows, K, decades=6):
    return rng.standard_normal((rows, K)) * (10.0 ** rng.uniform(-decades / 2, decades / 2, size=(rows, 1)))


def _run(A, Bm, **kw):
    return L.gemm_nt_mixed(torch.from_numpy(A).cuda(), torch.from_numpy(Bm).cuda(), **kw).cpu().numpy()


@pytest.mark.parametrize("M,N,K", [(130, 70, 33), (300, 77, 512), (129, 257, 1000), (64, 40, 2048), (1, 1, 1),
                                   (97, 50, 2081), (40, 33, 4096)])
def test_random_within_bound(M, N, K):
    rng = np.random.default_rng(M * 7919 + N * 31 + K)
    A = _graded(rng, M, K)
    Bm = _graded(rng, N, K)
    ref = A @ Bm.T
    scale = np.abs(A).max(axis=1)[:, None] * np.abs(Bm).max(axis=1)[None, :]
    D = _run(A, Bm, dtype=torch.float64)
    ratio = np.abs(D - ref) / (scale * (2.0 ** -28 * math.sqrt(K) + 2.0 ** -37 * K ** 1.5))
    assert ratio.max() <= 1.0, math.log2(ratio.max())


@pytest.mark.parametrize("lo", [32, -63])
def test_leading_levels_exact(lo):
    """Entries (128 d0 + d1) / 2^13 with d0 in [lo, 63] (a 63 in every row, so E = 0 and
    the digits are d0, d1) and d1 in [-63, 63]: the product is a multiple of 2^-26 that
    the tensor cores must produce exactly. With lo = 32 the level-0 sums climb to about
    2^23 and the level-1 sums to 2^23.6."""
    K = 2048
    rng = np.random.default_rng(64 + lo)
    Ia = 128 * rng.integers(lo, 64, size=(130, K)) + rng.integers(-63, 64, size=(130, K))
    Ib = 128 * rng.integers(lo, 64, size=(40, K)) + rng.integers(-63, 64, size=(40, K))
    Ia[:, 0] = 128 * 63
    Ib[:, 0] = 128 * 63
    exact = (Ia @ Ib.T).astype(np.float64) / 2.0 ** 26    # integers below 2^48: exact in FP64
    D = _run(Ia / 2.0 ** 13, Ib / 2.0 ** 13, dtype=torch.float64)
    assert np.array_equal(D, exact), np.abs(D - exact).max()


def test_leading_levels_exact_four_accumulators():
    """K = 4096 with d0 and d1 both in [32, 63]: each level-1 product sum (d0 d1 and d1 d0)
    climbs to about 2^23.1 on its own and their total above 2^24, so one shared FP32
    accumulator could not hold it exactly; with one accumulator each the product is exact."""
    K = 4096
    rng = np.random.default_rng(4096)
    Ia = 128 * rng.integers(32, 64, size=(130, K)) + rng.integers(32, 64, size=(130, K))
    Ib = 128 * rng.integers(32, 64, size=(40, K)) + rng.integers(32, 64, size=(40, K))
    Ia[:, 0] = 128 * 63
    Ib[:, 0] = 128 * 63
    lvl1 = (Ia // 128) @ (Ib % 128).T
    assert lvl1.max() > 2 ** 23 and 2 * lvl1.min() > 2 ** 24     # the sums the test relies on
    exact = (Ia @ Ib.T).astype(np.float64) / 2.0 ** 26
    D = _run(Ia / 2.0 ** 13, Ib / 2.0 ** 13, dtype=torch.float64)
    assert np.array_equal(D, exact), np.abs(D - exact).max()


def test_exact_cancellation():
    K = 1024
    x = 0.7654321
    sign = np.where(np.arange(K) % 2 == 0, 1.0, -1.0)
    A = np.tile(x * sign, (5, 1))
    Bm = np.full((9, K), x)
    D = _run(A, Bm, dtype=torch.float64)
    assert np.all(D == 0.0), np.abs(D).max()


def test_tile_width_bitwise_invariant():
    rng = np.random.default_rng(5)
    A = _graded(rng, 200, 300)
    Bm = _graded(rng, 300, 300)
    outs = [_run(A, Bm, dtype=torch.float64, tile_n=t) for t in (32, 64, 128)]
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


def test_zero_rows_and_f32_output():
    rng = np.random.default_rng(9)
    A = _graded(rng, 150, 96)
    Bm = _graded(rng, 70, 96)
    A[3] = 0.0
    Bm[11] = 0.0
    D64 = _run(A, Bm, dtype=torch.float64)
    D32 = _run(A, Bm, dtype=torch.float32)
    assert np.all(D64[3] == 0.0) and np.all(D64[:, 11] == 0.0)
    assert np.all(D32[3] == 0.0) and np.all(D32[:, 11] == 0.0)
    half_ulp = np.spacing(np.abs(D64).astype(np.float32)).astype(np.float64) / 2
    assert np.all(np.abs(D32.astype(np.float64) - D64) <= half_ulp * (1 + 2.0 ** -20))


def test_bad_arguments():
    A = torch.zeros((4, 4200), dtype=torch.float64, device="cuda")
    with pytest.raises(Exception):
        L.gemm_nt_mixed(A, A)                       # K above 4096 with FP32 output
    A = torch.zeros((4, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(Exception):
        L.gemm_nt_mixed(A, A, tile_n=256)
