"""lattice_sum_eval_slab_noalloc: slab values with no device allocation.

It exists for callers that cannot allocate device memory when they evaluate
(an application that reserved all of its device memory in one arena at
start-up, a latency-critical loop that must not wait on the allocator). Its
scratch is a static device array inside the library. The tests call it
through the C ABI, twice in a row (the second call finds the first call's
contents in the array), and compare it with

  * lattice_sum_eval_slab on the same Tucker factors (the existing entry
    point), within the FP64 tolerance the other parity tests use, and
  * the oracle's Tucker evaluation (Eq. Tucker_singePot) of the factors read
    back to the host, so that the check does not rest on the library alone;

and, with random Tucker factors large enough that one slab fills most of the
array, the chunked form (one slab per chunk: later chunks write at an output
offset and reuse the array) against the oracle's evaluation. The file is
collected last and passes both alone and after the other tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import lattice_oracle as O  # noqa: E402
from paper_1411_1994_gb300 import build as B  # noqa: E402
from paper_1411_1994_gb300 import lattice_sum as L  # noqa: E402
from paper_1411_1994_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def reduced():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    B.build()
    wl = W.small_case(L=(4, 3, 3), N=72, frac_vac=0.1, frac_imp=0.05, eps=1e-7)
    s, _ = O.fit_t_scale(wl.R, wl.sinc_step, wl.r_min, O.default_r_max(wl))
    ls = L.LatticeSum.from_workload(wl, s, L.LS_FP64)
    ls.add_defects(wl.defects)
    ls.rhosvd_reduce(wl.eps)
    yield wl, ls
    ls.close()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matches_eval_slab_and_oracle_twice(reduced):
    wl, ls = reduced
    Z, core, ranks = ls.factors()
    # the factors read back: Z_l as [r_l][N] rows, the core as [r0][r1][r2]
    Zh = [ls.read(L.LS_READ_BASIS, a).reshape(ranks[a], wl.N).T for a in range(3)]
    Bh = ls.read(L.LS_READ_CORE).reshape(ranks)
    for zs in ([0, 7, wl.N // 2, wl.N - 1], [3, 3, 40, 11, 65]):
        ref = ls.eval_slab_torch(zs).cpu().numpy()
        orc = np.stack([O.tucker_slab(Zh, Bh, z) for z in zs])
        for dtype, code in ((torch.float64, L.LS_OUT_F64), (torch.float32, L.LS_OUT_F32)):
            out = torch.full((len(zs), wl.N, wl.N), float("nan"), dtype=dtype, device="cuda")
            L.eval_slab_noalloc(Z, core, ranks, wl.N, zs, out.data_ptr(), code)
            torch.cuda.synchronize()
            got = out.double().cpu().numpy()
            tol = 1e-12 if dtype == torch.float64 else 1e-6
            assert np.all(np.isfinite(got))
            assert rel(got, ref) <= tol
            assert rel(got, orc) <= tol


def test_noalloc_chunked_against_oracle():
    """r = (1024, 1024, 8), N = 2048: one slab takes 8 (r0 r1 + r0 N) bytes = 25 MB of the
    32 MiB array, so three slabs run as three chunks."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    B.build()
    r, N = (1024, 1024, 8), 2048
    rng = np.random.default_rng(2048)
    Zh = [np.linalg.qr(rng.standard_normal((N, r[a])))[0] for a in range(3)]
    Bh = rng.standard_normal(r)
    Zd = [torch.from_numpy(np.ascontiguousarray(Zh[a].T)).cuda() for a in range(3)]
    Bd = torch.from_numpy(Bh).cuda()
    zs = [5, N - 1, 1000]
    orc = np.stack([O.tucker_slab(Zh, Bh, z) for z in zs])
    for _ in range(2):
        out = torch.full((len(zs), N, N), float("nan"), dtype=torch.float64, device="cuda")
        L.eval_slab_noalloc([z.data_ptr() for z in Zd], Bd.data_ptr(), list(r), N, zs, out.data_ptr())
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert rel(got, orc) <= 1e-12
        del out


def test_noalloc_rejects_oversized_request(reduced):
    wl, ls = reduced
    Z, core, ranks = ls.factors()
    big_n = 1 << 20                       # r0 * N doubles per slab exceed the static scratch
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    with pytest.raises(L.LatticeSumError) as ei:
        L.eval_slab_noalloc(Z, core, ranks, big_n, [0], out.data_ptr())
    assert ei.value.code == L.LS_ERR_ARG
    with pytest.raises(L.LatticeSumError) as ei:
        L.eval_slab_noalloc(Z, core, ranks, wl.N, [wl.N], out.data_ptr())
    assert ei.value.code == L.LS_ERR_ARG
