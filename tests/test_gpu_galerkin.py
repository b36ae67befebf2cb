"""The Galerkin matrix of the reduced potential in a rank-one basis
(lattice_sum_galerkin, Eq. nuc_pot) against the oracle.

v_km = <G_k (.) G_m, T> is a contraction of FP64 data through FP64-grade
products (error about 2^-53 sum |a||b| per product), so it agrees with the
oracle's evaluation of the same Tucker factors (read back) to 1e-12 of the
largest entry; against the oracle's own reduction at the same ranks it
inherits the FP64 path's 1e-12. For one unit charge and s-type Gaussians,
h^3 V approaches the closed-form nuclear-attraction integrals at second
order in h (within 2e-3 at N = 128).
"""
import math

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


def basis_for(wl, nb, seed):
    x = O.cell_centres(wl.N, wl.box_lo, wl.box_hi)
    rng = np.random.default_rng(seed)
    half = 0.4 * (wl.box_hi - wl.box_lo)
    cen = rng.uniform(-half, half, (nb, 3))
    alph = rng.uniform(0.2, 2.0, nb)
    return [np.exp(-alph[:, None] * (x[None, :] - cen[:, l:l + 1]) ** 2) for l in range(3)]


@pytest.mark.parametrize("wl,nb,prec", [(W.small_case(L=(3, 2, 2), frac_vac=0.2, frac_imp=0.1, eps=1e-6), 7, L.LS_FP64),
                                        (W.config2(), 24, L.LS_FP64),
                                        (W.config2(), 24, L.LS_MIXED)],
                         ids=["small_fp64", "c2_fp64", "c2_mixed"])
def test_galerkin_matches_oracle(wl, nb, prec):
    s, _ = O.fit_t_scale(wl.R, wl.sinc_step, wl.r_min, O.default_r_max(wl))
    ls = L.LatticeSum.from_workload(wl, s, prec)
    ls.add_defects(wl.defects)
    info = ls.rhosvd_reduce(wl.eps)
    basis = basis_for(wl, nb, 3)
    V = ls.galerkin([torch.from_numpy(b).cuda() for b in basis]).cpu().numpy()
    Z = [ls.read(L.LS_READ_BASIS, a).reshape(info["r"][a], wl.N).T for a in range(3)]
    Bc = ls.read(L.LS_READ_CORE).reshape(info["r"])
    ref = O.galerkin_matrix(Z, Bc, basis)
    assert np.max(np.abs(V - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert np.array_equal(V, V.T)
    if prec == L.LS_FP64:
        # against the oracle's own reduction (same ranks): the FP64 path's 1e-12
        t, w = O.sinc_quadrature(wl.R, wl.sinc_step, s)
        g = O.generating_vectors(wl.N, wl.box_lo, wl.box_hi, t, w)
        cols, tcol, xi = O.canonical_terms(wl.N, wl.box_lo, wl.box_hi, g, wl.blocks, wl.defects)
        res = O.rhosvd(cols, tcol, xi, wl.eps)
        assert info["r"] == list(res["r"])
        ref2 = O.galerkin_matrix(res["Z"], res["B"], basis)
        assert np.max(np.abs(V - ref2)) <= 1e-12 * np.max(np.abs(ref2))
    ls.close()


def test_galerkin_nuclear_attraction_of_one_charge():
    from scipy.special import erf
    wl = W.small_case(L=(1, 1, 1), N=128, R=24, eps=1e-10, sinc_step=0.25)
    s, _ = O.fit_t_scale(wl.R, wl.sinc_step, 0.02, O.default_r_max(wl))
    ls = L.LatticeSum.from_workload(wl, s)
    ls.rhosvd_reduce(wl.eps)
    x = O.cell_centres(wl.N, wl.box_lo, wl.box_hi)
    h = x[1] - x[0]
    a = O.charged_centres(wl.N, wl.box_lo, wl.box_hi, wl.blocks, wl.defects)[0][0]
    rng = np.random.default_rng(0)
    alph = rng.uniform(0.8, 2.0, 4)
    cen = a + rng.uniform(-1.0, 1.0, (4, 3))
    basis = [np.exp(-alph[:, None] * (x[None, :] - cen[:, l:l + 1]) ** 2) for l in range(3)]
    V = ls.galerkin([torch.from_numpy(b).cuda() for b in basis]).cpu().numpy() * h ** 3
    A = np.zeros((4, 4))
    for k in range(4):
        for m in range(4):
            p = alph[k] + alph[m]
            mu = alph[k] * alph[m] / p
            P = (alph[k] * cen[k] + alph[m] * cen[m]) / p
            tt = p * float(np.sum((P - a) ** 2))
            F0 = 1.0 if tt < 1e-14 else 0.5 * math.sqrt(math.pi / tt) * erf(math.sqrt(tt))
            A[k, m] = 2.0 * math.pi / p * math.exp(-mu * float(np.sum((cen[k] - cen[m]) ** 2))) * F0
    assert np.max(np.abs(V - A) / np.abs(A)) < 2e-3
    ls.close()


def test_galerkin_argument_errors():
    wl = W.small_case(L=(2, 2, 2), eps=1e-6)
    s, _ = O.fit_t_scale(wl.R, wl.sinc_step, wl.r_min, O.default_r_max(wl))
    ls = L.LatticeSum.from_workload(wl, s)
    b = [torch.zeros((2, wl.N), dtype=torch.float64, device="cuda") for _ in range(3)]
    with pytest.raises(L.LatticeSumError) as ei:
        ls.galerkin(b)
    assert ei.value.code == L.LS_ERR_STATE
    ls.close()
