"""Failure paths, driven without faulting the GPU.

The library reports failures as status codes (include/lattice_sum.h): a device
allocation that fails gives LS_ERR_OOM, an iteration that hits its sweep limit
LS_ERR_NOCONVERGE, and a bounded device-side wait that runs out LS_ERR_TIMEOUT
(the kernel ends and the context stays usable). These tests make each happen
on purpose, in the permitted forms: an allocation failure injected on the host
(lattice_sum_test_fail_alloc), a sweep cap too small for the matrix, and the
cooperative kernels' bounded group barrier with a short limit and a partner
CTA that never arrives (lattice_sum_test_bounded_wait). After each, the
library must still reduce a fresh context correctly.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import lattice_oracle as O  # noqa: E402
from paper_1411_1994_gb300 import build as B  # noqa: E402
from paper_1411_1994_gb300 import lattice_sum as L  # noqa: E402
from paper_1411_1994_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    B.build()
    L.lib()
    yield
    L.test_fail_alloc(-1)


WL = W.small_case(L=(3, 2, 2), frac_vac=0.2, frac_imp=0.1, eps=1e-6)


def scale():
    return O.fit_t_scale(WL.R, WL.sinc_step, WL.r_min, O.default_r_max(WL))[0]


def still_works():
    """A fresh context reduces to the oracle's ranks and Tucker values."""
    s = scale()
    ls = L.LatticeSum.from_workload(WL, s)
    ls.add_defects(WL.defects)
    info = ls.rhosvd_reduce(WL.eps)
    t, w = O.sinc_quadrature(WL.R, WL.sinc_step, s)
    g = O.generating_vectors(WL.N, WL.box_lo, WL.box_hi, t, w)
    cols, tcol, xi = O.canonical_terms(WL.N, WL.box_lo, WL.box_hi, g, WL.blocks, WL.defects)
    res = O.rhosvd(cols, tcol, xi, WL.eps)
    assert info["r"] == list(res["r"])
    out = ls.eval_slab_torch(WL.slabs).cpu().numpy()
    ref = np.stack([O.tucker_slab(res["Z"], res["B"], z) for z in WL.slabs])
    assert np.linalg.norm(out - ref) <= 1e-12 * np.linalg.norm(ref)
    ls.close()


@pytest.mark.parametrize("at", [0, 3, 17, 40])
def test_allocation_failure_in_reduce_returns_oom(at):
    s = scale()
    ls = L.LatticeSum.from_workload(WL, s)
    ls.add_defects(WL.defects)
    L.test_fail_alloc(at)
    with pytest.raises(L.LatticeSumError) as ei:
        ls.rhosvd_reduce(WL.eps)
    L.test_fail_alloc(-1)
    assert ei.value.code == L.LS_ERR_OOM, ei.value
    ls.close()
    still_works()


def test_allocation_failure_in_create_returns_oom():
    L.test_fail_alloc(0)
    with pytest.raises(L.LatticeSumError) as ei:
        L.LatticeSum.from_workload(WL, scale())
    L.test_fail_alloc(-1)
    assert ei.value.code == L.LS_ERR_OOM
    still_works()


def test_sweep_cap_returns_noconverge():
    """A graded random symmetric matrix needs several Jacobi sweeps; a cap of one sweep
    ends the block Jacobi (both forms) and the one-sided Jacobi with LS_ERR_NOCONVERGE."""
    rng = np.random.default_rng(1)
    k = 40
    Qm = np.linalg.qr(rng.standard_normal((k, k)))[0]
    H = (Qm * np.geomspace(1.0, 1e-6, k)) @ Qm.T
    Hd = torch.from_numpy(H).cuda()
    for form in (1, 2):
        with pytest.raises(L.LatticeSumError) as ei:
            L.jacobi_eig(Hd, tol=1e-10, form=form, max_sweeps=1)
        assert ei.value.code == L.LS_ERR_NOCONVERGE
        D, V, sweeps = L.jacobi_eig(Hd, tol=1e-10, form=form)
        assert sweeps > 1
    Bm = torch.from_numpy(rng.standard_normal((30, 80))).cuda()
    with pytest.raises(L.LatticeSumError) as ei:
        L.svd_rows(Bm, max_sweeps=1)
    assert ei.value.code == L.LS_ERR_NOCONVERGE
    sig2, M, sweeps, rots = L.svd_rows(Bm)
    assert sweeps > 1
    still_works()


def test_bounded_wait_runs_out_and_returns_timeout():
    # both CTAs arrive: the barrier completes
    assert L.test_bounded_wait(0, 1 << 16) == L.LS_OK
    # the partner never arrives: the wait gives up after the limit (about a millisecond)
    assert L.test_bounded_wait(1, 1 << 12) == L.LS_ERR_TIMEOUT
    assert "ran out" in L.lib().lattice_sum_last_error(None).decode()
    still_works()
