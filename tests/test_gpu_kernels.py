"""The other kernels of Sec. 2.3 through the C ABI against the FP64 oracle:
Yukawa exp(-kappa r)/r (Eq. LalpYukawa), Slater exp(-kappa r) (Eq.
LalpSlater) and the dipole 1/r^3 (Eq. LalpPoly at n = 3/2); and Galerkin
reference vectors (cell averages, Eq. galten) for the Newton and Yukawa
kernels.

Only the reference vectors change (the quadrature weights follow each
kernel's Laplace-Gauss density and the nodes start at q = 1); the rest of the
path is the one the Newton kernel takes. Tolerances are those of the Newton
parity tests: reference and canonical vectors to 1e-13 of each vector's
maximum (the same closed forms in FP64), term maps and charges bit-exact, the
RHOSVD within the Thm A.1(d) bound at the free eps-rank and to the Gram
route's accuracy at a forced common rank; the mixed path within eps; slab
values against the direct screened sum within the rule's error.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import lattice_oracle as O  # noqa: E402
from paper_1411_1994_gb300 import build as B  # noqa: E402
from paper_1411_1994_gb300 import lattice_sum as L  # noqa: E402
from paper_1411_1994_gb300 import workloads as W  # noqa: E402

import test_gpu_parity as P  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    B.build()
    L.lib()


YUK, SLA, DIP = L.LS_KERNEL_YUKAWA, L.LS_KERNEL_SLATER, L.LS_KERNEL_DIPOLE
CASES = [W.small_case(L=(3, 2, 2), frac_vac=0.2, frac_imp=0.1, eps=1e-7, kappa=0.6),
         W.small_case(L=(5, 3, 2), N=70, frac_vac=0.1, eps=1e-6, kappa=1.2),
         W.small_case(L=(4, 4, 4), N=64, R=20, frac_vac=0.15, frac_imp=0.05, eps=1e-6, kappa=0.3),
         W.small_case(L=(3, 2, 2), frac_vac=0.2, frac_imp=0.1, eps=1e-7, kappa=0.8, kernel=SLA),
         W.small_case(L=(4, 4, 4), N=64, R=20, frac_vac=0.15, frac_imp=0.05, eps=1e-6, kappa=1.5, kernel=SLA),
         W.small_case(L=(3, 2, 2), frac_vac=0.2, frac_imp=0.1, eps=1e-7, kernel=DIP),
         W.small_case(L=(4, 4, 4), N=64, R=20, frac_vac=0.15, frac_imp=0.05, eps=1e-6, kernel=DIP),
         W.small_case(L=(3, 2, 2), frac_vac=0.2, frac_imp=0.1, eps=1e-7, galerkin=True),
         W.small_case(L=(4, 4, 4), N=64, R=20, frac_vac=0.15, frac_imp=0.05, eps=1e-6, kappa=0.5, galerkin=True)]


def scale_for(wl):
    s, _ = O.fit_t_scale(wl.R, wl.sinc_step, wl.r_min, O.default_r_max(wl), kappa=wl.kappa, kernel=wl.kernel)
    return s


@pytest.mark.parametrize("wl", CASES, ids=lambda w: w.name)
def test_kernel_vectors_and_terms_match_oracle(wl):
    s = scale_for(wl)
    t, w = O.sinc_quadrature(wl.R, wl.sinc_step, s, wl.kappa, wl.kernel)
    g = O.generating_vectors(wl.N, wl.box_lo, wl.box_hi, t, w, wl.galerkin)
    cols, tcol, xi = O.canonical_terms(wl.N, wl.box_lo, wl.box_hi, g, wl.blocks, wl.defects)
    ls = P.gpu_ctx(wl, s)
    gg = ls.read(L.LS_READ_GENVEC).reshape(wl.R, 2 * wl.N)
    assert np.all(np.abs(gg - g) <= 1e-13 * np.abs(g).max(1, keepdims=True))
    # the collocated Newton rule's vectors are not these (the kernel's weights or the cell
    # averages are applied)
    tn, wn = O.sinc_quadrature(wl.R, wl.sinc_step, s)
    gn = O.generating_vectors(wl.N, wl.box_lo, wl.box_hi, tn, wn)
    assert np.max(np.abs(gg - gn)) > 1e-3 * np.abs(gn).max()
    for a in range(3):
        c = ls.read(L.LS_READ_COLUMNS, a).reshape(-1, wl.N)
        assert c.shape == cols[a].shape
        assert np.all(np.abs(c - cols[a]) <= 1e-13 * np.abs(cols[a]).max(1, keepdims=True))
    assert np.array_equal(ls.read(L.LS_READ_TERMS).reshape(-1, 3), tcol)
    assert np.array_equal(ls.read(L.LS_READ_XI), xi)
    ls.close()


@pytest.mark.parametrize("wl", CASES, ids=lambda w: w.name)
def test_kernel_fp64_reduction_matches_oracle(wl):
    s = scale_for(wl)
    P.check_reduction(wl, s)
    P.forced_rank_parity(wl, s)


@pytest.mark.parametrize("wl", CASES[0:2] + CASES[3:4] + CASES[5:6] + CASES[8:9], ids=lambda w: w.name)
def test_kernel_mixed_within_eps(wl):
    s = scale_for(wl)
    orc = P.oracle_run(wl, s)
    ls = P.gpu_ctx(wl, s, L.LS_MIXED)
    ls.rhosvd_reduce(wl.eps)
    out = ls.eval_slab_torch(wl.slabs).cpu().numpy()
    ref = np.stack([O.canonical_slab(orc["ncols"], orc["tcol"], orc["xin"], z) for z in wl.slabs])
    assert P.rel(out, ref) <= wl.eps, P.rel(out, ref)
    ls.close()


@pytest.mark.parametrize("wl", [CASES[2], CASES[4], CASES[6]], ids=lambda w: w.name)
def test_kernel_slabs_against_direct_sum(wl):
    """Slab values of the FP64 path vs sum_s Z_s p(d_s) over the snapped
    centres, at points at least r_min from every centre: within tau * sum_s
    |Z_s| m(d_s) (tau: the rule's error measured against m = 1/r, 1 or 1/r^3)
    plus the truncation bound."""
    s = scale_for(wl)
    ls = P.gpu_ctx(wl, s)
    info = ls.rhosvd_reduce(wl.eps)
    z = [wl.N // 2, wl.N // 3, 5]
    out = ls.eval_slab_torch(z).cpu().numpy()
    xs = O.cell_centres(wl.N, wl.box_lo, wl.box_hi)
    centres, charges = O.charged_centres(wl.N, wl.box_lo, wl.box_hi, wl.blocks, wl.defects)
    t, w = O.sinc_quadrature(wl.R, wl.sinc_step, s, wl.kappa, wl.kernel)
    tau = float(np.max(O.quadrature_rel_error(t, w, np.geomspace(wl.r_min, O.default_r_max(wl), 6000),
                                              wl.kappa, wl.kernel)))
    rng = np.random.default_rng(11)
    for k, zz in enumerate(z):
        ij = rng.integers(0, wl.N, size=(3000, 2))
        pts = np.stack([xs[ij[:, 0]], xs[ij[:, 1]], np.full(len(ij), xs[zz])], 1)
        bf, absbf, dmin, _ = O.brute_force(pts, centres, charges, kappa=wl.kappa, kernel=wl.kernel)
        keep = dmin >= wl.r_min
        if wl.kernel == SLA:
            scale = np.full(int(keep.sum()), np.abs(charges).sum())
        elif wl.kernel == DIP:
            scale = absbf[keep]
        else:
            scale = O.brute_force(pts, centres, charges)[1][keep]
        val = out[k][ij[keep, 0], ij[keep, 1]]
        assert np.all(np.abs(val - bf[keep]) <= tau * scale * 1.01 + info["bound_abs"])
    ls.close()


def test_kernel_rejects_bad_parameters():
    wl = CASES[0]
    for kernel, kappa in ((YUK, -0.1), (YUK, float("nan")), (YUK, 1e4), (SLA, 0.0), (SLA, 1e4), (DIP, 0.5),
                          (7, 0.0)):
        with pytest.raises(L.LatticeSumError) as ei:
            L.LatticeSum(wl.N, wl.box_lo, wl.box_hi, wl.R, wl.sinc_step, 10.0, wl.blocks, kappa=kappa,
                         kernel=kernel)
        assert ei.value.code == L.LS_ERR_ARG
