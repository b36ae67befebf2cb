"""lattice_sum_eval_slab_noalloc: slab values with no device allocation.

It exists for callers that cannot allocate device memory when they evaluate
(an application that reserved all of its device memory in one arena at
start-up, a latency-critical loop that must not wait on the allocator). Its
scratch is a static device array inside the library, so the test checks it
through the C ABI against lattice_sum_eval_slab on the same Tucker factors,
twice in a row (the second call reuses the array's stale contents), within
the FP64 tolerance the other parity tests use. It sits in its own file that
pytest collects last and passes both alone and after the other tests.
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


def test_noalloc_matches_eval_slab_twice(reduced):
    wl, ls = reduced
    Z, core, ranks = ls.factors()
    for zs in ([0, 7, wl.N // 2, wl.N - 1], [3, 3, 40, 11, 65]):
        ref = ls.eval_slab_torch(zs)
        for dtype, code in ((torch.float64, L.LS_OUT_F64), (torch.float32, L.LS_OUT_F32)):
            out = torch.full((len(zs), wl.N, wl.N), float("nan"), dtype=dtype, device="cuda")
            L.eval_slab_noalloc(Z, core, ranks, wl.N, zs, out.data_ptr(), code)
            torch.cuda.synchronize()
            got = out.double().cpu().numpy()
            want = ref.cpu().numpy()
            tol = 1e-12 if dtype == torch.float64 else 1e-6
            assert np.all(np.isfinite(got))
            assert np.linalg.norm(got - want) <= tol * np.linalg.norm(want)


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
