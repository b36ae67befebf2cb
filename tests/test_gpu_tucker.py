"""The Tucker-reference variant on the GPU (LS_FLAG_TUCKER_REF) against the
oracle: the reference Tucker tensor (RHOSVD of the canonical reference on the
doubled grid), the Tucker lattice sum with defects (Thm 3.1(B), Sec. 4.1) and
its generalized RHOSVD (Thm 4.3), all through the C ABI.

Tolerances: the reference Tucker vectors are singular vectors of the R unit
reference vectors; any backward-stable SVD (LAPACK's, the GPU's one-sided
Jacobi) determines them only to about delta_t = 2 u sigma_1 / gap (Wedin's
bound, gap the smallest separation of a kept singular value from its
neighbours), computed here from the oracle's own spectrum (3e-12 to 1e-11 at
the thresholds used). Everything downstream inherits it: with
tol = max(1e-12, delta_t), the reference vectors agree up to sign to tol, the
vectors of the lattice sum to tol of each vector's maximum, the side-matrix
singular values to tol sigma_1 (ranks exactly), the Thm 4.3 quantities to
tol, and the Tucker result to tol relative on slabs. The bound the GPU
reports dominates the error against the untruncated sum.
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
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def cases():
    a = W.small_case(L=(4, 3, 3), N=40, frac_vac=0.15, frac_imp=0.1, eps=1e-6)
    a.defects = list(a.defects) + [W.Defect(W.DEFECT_SITES, 0, (1, 1, 0), (2, 2, 2), charge=1.3),
                                   W.Defect(W.DEFECT_POINT, pos=(0.37, -1.1, 0.5), charge=0.7)]
    b = W.small_case(L=(4, 4, 4), N=64, R=20, frac_vac=0.1, frac_imp=0.05, eps=1e-7)
    c = W.small_case(L=(3, 2, 2), N=48, frac_vac=0.2, eps=1e-5)
    return [(a, 1e-5), (b, 1e-5), (c, 1e-4)]


def oracle(wl, ref_eps, s, ranks=None):
    t, w = O.sinc_quadrature(wl.R, wl.sinc_step, s)
    g = O.generating_vectors(wl.N, wl.box_lo, wl.box_hi, t, w)
    tt, b, sig = O.reference_tucker(g, ref_eps)
    terms = O.tucker_terms(wl.N, wl.box_lo, wl.box_hi, tt, b, wl.blocks, wl.defects)
    res = O.tucker_sum_rhosvd(terms, wl.eps, ranks=ranks)
    gp = (tt.T @ (tt @ g.T)).T
    cols, tcol, xi = O.canonical_terms(wl.N, wl.box_lo, wl.box_hi, gp, wl.blocks, wl.defects)
    # Wedin's bound on the reference singular vectors: 2 u sigma_1 / (smallest gap of a kept value)
    r = tt.shape[0]
    sg = np.concatenate([sig, [0.0]])
    gap = min(min(sg[k - 1] - sg[k] if k > 0 else np.inf, sg[k] - sg[k + 1]) for k in range(r))
    tol = max(1e-12, 2.0 * 2.0 ** -53 * sig[0] / gap)
    return dict(g=g, tt=tt, b=b, terms=terms, res=res, cols=cols, tcol=tcol, xi=xi, tol=tol)


def gpu(wl, s, ref_eps, precision=L.LS_FP64):
    ls = L.LatticeSum.from_workload(wl, s, precision, flags=L.LS_FLAG_TUCKER_REF, ref_eps=ref_eps)
    ls.add_defects(wl.defects)
    return ls


@pytest.mark.parametrize("k", [0, 1, 2])
def test_tucker_reference_and_vectors_match_oracle(k):
    wl, ref_eps = cases()[k]
    s, _ = O.fit_t_scale(wl.R, wl.sinc_step, wl.r_min, O.default_r_max(wl))
    orc = oracle(wl, ref_eps, s)
    ls = gpu(wl, s, ref_eps)
    tg = ls.read(L.LS_READ_TUCKER_REF).reshape(-1, 2 * wl.N)
    assert tg.shape == orc["tt"].shape
    # the same singular vectors up to sign
    tol = orc["tol"]
    d = np.abs(np.sum(tg * orc["tt"], axis=1))
    assert np.all(np.abs(d - 1.0) <= tol), (d, tol)
    # the canonical vectors of the projected reference, assembled and windowed
    for a in range(3):
        c = ls.read(L.LS_READ_COLUMNS, a).reshape(-1, wl.N)
        assert c.shape == orc["cols"][a].shape
        assert np.all(np.abs(c - orc["cols"][a]) <= tol * np.abs(orc["cols"][a]).max(1, keepdims=True))
    ls.close()


@pytest.mark.parametrize("k", [0, 1, 2])
def test_tucker_sum_reduction_matches_oracle(k):
    wl, ref_eps = cases()[k]
    s, _ = O.fit_t_scale(wl.R, wl.sinc_step, wl.r_min, O.default_r_max(wl))
    orc = oracle(wl, ref_eps, s)
    res = orc["res"]
    tol = orc["tol"]
    # free eps rank
    ls = gpu(wl, s, ref_eps)
    info = ls.rhosvd_reduce(wl.eps)
    assert list(info["r"]) == list(res["r"]), (info["r"], res["r"])
    for a in range(3):
        sg = ls.read(L.LS_READ_SIGMA, a)
        so = res["sigma"][a]
        n = min(len(sg), len(so))
        kk = so[:n] > 1e-11 * so[0]
        assert np.all(np.abs(sg[:n][kk] - so[:n][kk]) <= tol * so[0]), (a, float(np.max(np.abs(sg[:n][kk] - so[:n][kk]))))
        assert abs(info["sigma_discarded"][a] - res["d"][a]) <= tol * so[0]
    assert abs(info["xi_norm"] - res["Bhat"]) <= tol * res["Bhat"]
    assert abs(info["bound_abs"] - res["bound"]) <= tol * res["bound"] + 1e-13 * res["Bhat"]
    out = ls.eval_slab_torch(wl.slabs).cpu().numpy()
    ref = np.stack([O.tucker_slab(res["Z"], res["B"], z) for z in wl.slabs])
    assert rel(out, ref) <= tol, (rel(out, ref), tol)
    # the Thm 4.3 bound dominates the error against the untruncated Tucker sum
    full = np.stack([O.canonical_slab(orc["cols"], orc["tcol"], orc["xi"], z) for z in wl.slabs])
    assert np.linalg.norm(out - full) <= info["bound_abs"] * (1 + 1e-9)
    ls.close()


def test_tucker_sum_mixed_precision_within_eps():
    wl, ref_eps = cases()[1]
    s, _ = O.fit_t_scale(wl.R, wl.sinc_step, wl.r_min, O.default_r_max(wl))
    orc = oracle(wl, ref_eps, s)
    ls = gpu(wl, s, ref_eps, L.LS_MIXED)
    info = ls.rhosvd_reduce(wl.eps)
    assert list(info["r"]) == list(orc["res"]["r"])
    out = ls.eval_slab_torch(wl.slabs).cpu().numpy()
    ref = np.stack([O.tucker_slab(orc["res"]["Z"], orc["res"]["B"], z) for z in wl.slabs])
    assert rel(out, ref) <= 1e-7 + orc["tol"], rel(out, ref)
    ls.close()


def test_tucker_flag_argument_errors():
    wl, _ = cases()[2]
    s = 6.0
    for flags, ref_eps in ((L.LS_FLAG_TUCKER_REF, 0.0), (L.LS_FLAG_TUCKER_REF | L.LS_FLAG_SVD_GRAM, 1e-6)):
        with pytest.raises(L.LatticeSumError) as ei:
            L.LatticeSum.from_workload(wl, s, L.LS_FP64, flags=flags, ref_eps=ref_eps)
        assert ei.value.code == L.LS_ERR_ARG
    # a canonical context has no reference Tucker vectors
    ls = L.LatticeSum.from_workload(wl, s)
    with pytest.raises(L.LatticeSumError) as ei:
        ls.read(L.LS_READ_TUCKER_REF)
    ls.close()
