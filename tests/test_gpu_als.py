"""ALS refinement on the GPU (lattice_sum_als_refine, Thm A.1(a)-(b)) against
the oracle's als_refine, which is pinned against HOOI on the explicit tensor.

Both start from the RHOSVD at the same ranks (bases equal to FP64 rounding)
and apply the same alternating update (leading left singular vectors of B_l),
so the core norms after each sweep agree to 1e-12 relative and the refined
Tucker tensors to 1e-10 relative on slabs (each step's subspace is determined
to u sigma_1 / gap; the history is the first quantity to check). The history
never decreases, and it starts at the RHOSVD core norm.
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


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CASES = [W.small_case(L=(3, 3, 2), frac_vac=0.2, frac_imp=0.1, eps=1e-3),
         W.small_case(L=(4, 3, 2), N=64, frac_vac=0.15, frac_imp=0.1, eps=1e-4),
         W.small_case(L=(5, 4, 3), N=56, R=16, frac_vac=0.1, eps=3e-3)]


@pytest.mark.parametrize("wl", CASES, ids=lambda w: w.name)
def test_als_matches_oracle(wl):
    s, _ = O.fit_t_scale(wl.R, wl.sinc_step, wl.r_min, O.default_r_max(wl))
    t, w = O.sinc_quadrature(wl.R, wl.sinc_step, s)
    g = O.generating_vectors(wl.N, wl.box_lo, wl.box_hi, t, w)
    cols, tcol, xi = O.canonical_terms(wl.N, wl.box_lo, wl.box_hi, g, wl.blocks, wl.defects)
    res = O.rhosvd(cols, tcol, xi, wl.eps)
    Zo, core_o, hist_o = O.als_refine(cols, tcol, xi, res["Z"], sweeps=3)
    ls = L.LatticeSum.from_workload(wl, s)
    ls.add_defects(wl.defects)
    info = ls.rhosvd_reduce(wl.eps)
    assert info["r"] == list(res["r"])
    hist, info2 = ls.als_refine(3)
    assert info2["r"] == info["r"] and info2["sweeps"] == [3, 3, 3]
    assert np.all(np.abs(np.array(hist) - np.array(hist_o)) <= 1e-12 * hist_o[0]), (hist, hist_o)
    assert all(b >= a * (1 - 1e-14) for a, b in zip(hist, hist[1:])), hist
    out = ls.eval_slab_torch(wl.slabs).cpu().numpy()
    ref = np.stack([O.tucker_slab(Zo, core_o, z) for z in wl.slabs])
    assert rel(out, ref) <= 1e-10, rel(out, ref)
    # the refined bases stay orthonormal and the core is their projection
    for a in range(3):
        Z = ls.read(L.LS_READ_BASIS, a).reshape(info["r"][a], wl.N)
        assert np.max(np.abs(Z @ Z.T - np.eye(Z.shape[0]))) < 1e-13
    assert abs(np.linalg.norm(ls.read(L.LS_READ_CORE)) - hist[-1]) <= 1e-12 * hist[-1]
    ls.close()


def test_als_zero_sweeps_keeps_the_reduction():
    wl = CASES[0]
    s, _ = O.fit_t_scale(wl.R, wl.sinc_step, wl.r_min, O.default_r_max(wl))
    ls = L.LatticeSum.from_workload(wl, s)
    ls.add_defects(wl.defects)
    ls.rhosvd_reduce(wl.eps)
    before = ls.eval_slab_torch(wl.slabs).cpu().numpy()
    hist, _ = ls.als_refine(0)
    after = ls.eval_slab_torch(wl.slabs).cpu().numpy()
    assert len(hist) == 1 and abs(hist[0] - np.linalg.norm(ls.read(L.LS_READ_CORE))) <= 1e-12 * hist[0]
    assert rel(after, before) <= 1e-13
    ls.close()


def test_als_mixed_context_on_the_non_squaring_route():
    wl = CASES[1]
    s, _ = O.fit_t_scale(wl.R, wl.sinc_step, wl.r_min, O.default_r_max(wl))
    a = L.LatticeSum.from_workload(wl, s)
    a.add_defects(wl.defects)
    a.rhosvd_reduce(wl.eps)
    ha, _ = a.als_refine(2)
    b = L.LatticeSum.from_workload(wl, s, L.LS_MIXED, flags=L.LS_FLAG_SVD_ONESIDED)
    b.add_defects(wl.defects)
    b.rhosvd_reduce(wl.eps)
    hb, _ = b.als_refine(2)
    # the start is each path's own core (the mixed core to its tensor-core accuracy); the ALS
    # steps themselves run in FP64 on both and give the same norms
    assert abs(ha[0] - hb[0]) <= 1e-7 * ha[0]
    assert np.allclose(ha[1:], hb[1:], rtol=1e-12, atol=0)
    sa, sb = a.eval_slab_torch(wl.slabs).cpu().numpy(), b.eval_slab_torch(wl.slabs).cpu().numpy()
    assert rel(sb, sa) <= 1e-7
    a.close()
    b.close()


def test_als_needs_the_range_bases():
    wl = CASES[0]
    s, _ = O.fit_t_scale(wl.R, wl.sinc_step, wl.r_min, O.default_r_max(wl))
    ls = L.LatticeSum.from_workload(wl, s, L.LS_MIXED)   # Gram route: no range bases kept
    ls.add_defects(wl.defects)
    with pytest.raises(L.LatticeSumError) as ei:
        ls.als_refine(1)
    assert ei.value.code == L.LS_ERR_STATE                # before the reduction
    ls.rhosvd_reduce(wl.eps)
    with pytest.raises(L.LatticeSumError) as ei:
        ls.als_refine(1)
    assert ei.value.code == L.LS_ERR_STATE
    ls.close()
