"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances, derived from the arithmetic:
  * reference vectors, assembled and defect vectors (steps a0, a, b): both
    sides evaluate the same closed forms in FP64; the only difference is the
    last bit of exp(), amplified by the exponent size, so 1e-13 relative to
    each vector's maximum.
  * term maps and charges: integer / copied data, bit-exact.
  * RHOSVD (step c) on the FP64 path: the oracle takes the SVD of the side
    matrix (dgesdd), the GPU the non-squaring route (a basis of the side
    matrix's range from two deflated Gram passes, then one-sided Jacobi on
    Q^T A_w). Both are backward stable: singular values agree to a few u
    sigma_1 (the test allows 1e-13 sigma_1), ranks agree exactly, and at a
    common rank the truncated Tucker tensors agree to u sigma_1 / gap relative;
    the test allows 1e-12 relative on slabs (the relative error the FP64 path
    is held to).
  * at the free eps-rank both results must satisfy the Thm A.1(d) bound
    against the untruncated canonical tensor.
  * the Gram route (LS_FLAG_SVD_GRAM, the mixed path's) squares the singular
    values: sigma_k^2 to 1e3 u sigma_1^2, checked separately.
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
U = 2.0 ** -53


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    B.build()
    L.lib()


def scale_for(wl):
    s, _ = O.fit_t_scale(wl.R, wl.sinc_step, wl.r_min, O.default_r_max(wl))
    return s


def gpu_ctx(wl, s, precision=L.LS_FP64, defects=True, flags=0):
    ls = L.LatticeSum.from_workload(wl, s, precision, flags=flags)
    if defects:
        ls.add_defects(wl.defects)
    return ls


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# ---------------------------------------------------------------------------
# steps (a0), (a), (b): bit-level agreement of the canonical vectors
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("wl", [W.small_case(L=(3, 2, 2), frac_vac=0.2, frac_imp=0.1),
                                W.small_case(L=(5, 1, 3), N=50, frac_vac=0.3),
                                W.config1(), W.config2()], ids=lambda w: w.name)
def test_vectors_and_terms_match_oracle(wl):
    s = scale_for(wl)
    t, w = O.sinc_quadrature(wl.R, wl.sinc_step, s)
    g = O.generating_vectors(wl.N, wl.box_lo, wl.box_hi, t, w)
    cols, tcol, xi = O.canonical_terms(wl.N, wl.box_lo, wl.box_hi, g, wl.blocks, wl.defects)
    ls = gpu_ctx(wl, s)
    gg = ls.read(L.LS_READ_GENVEC).reshape(wl.R, 2 * wl.N)
    assert np.all(np.abs(gg - g) <= 1e-13 * np.abs(g).max(1, keepdims=True))
    for a in range(3):
        c = ls.read(L.LS_READ_COLUMNS, a).reshape(-1, wl.N)
        assert c.shape == cols[a].shape
        assert np.all(np.abs(c - cols[a]) <= 1e-13 * np.abs(cols[a]).max(1, keepdims=True))
    assert np.array_equal(ls.read(L.LS_READ_TERMS).reshape(-1, 3), tcol)
    assert np.array_equal(ls.read(L.LS_READ_XI), xi)
    ls.close()


def test_point_and_cluster_defects_match_oracle():
    L3 = (6, 5, 4)
    lo, hi = W.box_for(L3)
    blk = W.centred_block(L3)
    defects = [W.Defect(W.DEFECT_SITES, 0, (1, 1, 1), (3, 3, 2), charge=0.0),
               W.Defect(W.DEFECT_SITES, 0, (0, 2, 0), (2, 2, 2), charge=1.4),
               W.Defect(W.DEFECT_POINT, pos=(0.37, -1.21, 0.5), charge=0.8),
               W.Defect(W.DEFECT_POINT, pos=(lo, hi, 0.0), charge=-0.3),   # on the box corner
               W.Defect(W.DEFECT_SITES, 0, (5, 4, 3), (1, 1, 1), charge=2.0)]
    wl = W.Workload("pc", 40, lo, hi, 10, 0.35, 1e-7, [blk], defects, r_min=0.5)
    s = 6.0
    t, w = O.sinc_quadrature(wl.R, wl.sinc_step, s)
    g = O.generating_vectors(wl.N, lo, hi, t, w)
    cols, tcol, xi = O.canonical_terms(wl.N, lo, hi, g, wl.blocks, defects)
    ls = gpu_ctx(wl, s)
    for a in range(3):
        c = ls.read(L.LS_READ_COLUMNS, a).reshape(-1, wl.N)
        assert np.all(np.abs(c - cols[a]) <= 1e-13 * np.abs(cols[a]).max(1, keepdims=True))
    assert np.array_equal(ls.read(L.LS_READ_TERMS).reshape(-1, 3), tcol)
    assert np.array_equal(ls.read(L.LS_READ_XI), xi)


# ---------------------------------------------------------------------------
# step (c) RHOSVD and step (d) slabs
# ---------------------------------------------------------------------------

def oracle_run(wl, s, eps=None, ranks=None):
    t, w = O.sinc_quadrature(wl.R, wl.sinc_step, s, wl.kappa, wl.kernel)
    g = O.generating_vectors(wl.N, wl.box_lo, wl.box_hi, t, w, wl.galerkin)
    cols, tcol, xi = O.canonical_terms(wl.N, wl.box_lo, wl.box_hi, g, wl.blocks, wl.defects)
    res = O.rhosvd(cols, tcol, xi, wl.eps if eps is None else eps, ranks=ranks)
    ncols, _, xin = O.normalise_terms(cols, tcol, xi)
    return dict(cols=cols, ncols=ncols, tcol=tcol, xi=xi, xin=xin, res=res)


def check_reduction(wl, s, precision=L.LS_FP64, slabs=None, fp_tol=None, flags=0):
    orc = oracle_run(wl, s)
    res = orc["res"]
    ls = gpu_ctx(wl, s, precision, flags=flags)
    info = ls.rhosvd_reduce(wl.eps)
    slabs = slabs or wl.slabs
    gram = precision == L.LS_MIXED or (flags & L.LS_FLAG_SVD_GRAM)
    for a in range(3):
        sg = ls.read(L.LS_READ_SIGMA, a)
        so = res["sigma"][a]
        n = min(len(sg), len(so))
        if gram:
            # squared singular values to the Gram route's absolute accuracy
            assert np.all(np.abs(sg[:n] ** 2 - so[:n] ** 2) <= 1e3 * U * so[0] ** 2 * max(n, 1)), a
        else:
            # the non-squaring route: singular values to a few u sigma_1, over the range its
            # residual pass resolves (above ~1e-13 sigma_1; below it the energy joins the tail)
            k = so > 1e-11 * so[0]
            k[n:] = False
            assert np.all(np.abs(sg[:n][k[:n]] - so[:n][k[:n]]) <= 1e-13 * so[0]), \
                (a, float(np.max(np.abs(sg[:n][k[:n]] - so[:n][k[:n]]))))
            # and the discarded tail (sum_{k>r} s_k^2)^(1/2) to the same absolute accuracy
            assert abs(info["sigma_discarded"][a] - res["d"][a]) <= 1e-12 * so[0], \
                (a, info["sigma_discarded"][a], res["d"][a])
        # orthonormal Tucker vectors
        Z = ls.read(L.LS_READ_BASIS, a).reshape(info["r"][a], wl.N)
        assert np.max(np.abs(Z @ Z.T - np.eye(Z.shape[0]))) < 1e-13
    if gram:
        # ranks: equal up to the eps-boundary ambiguity of the squared spectrum
        assert all(abs(info["r"][a] - res["r"][a]) <= 2 for a in range(3)), (info["r"], res["r"])
    else:
        assert list(info["r"]) == list(res["r"]), (info["r"], res["r"])
    # term weights with the vector norms folded in
    assert np.allclose(ls.read(L.LS_READ_XI), orc["xin"], rtol=1e-13, atol=0)
    assert abs(info["xi_norm"] - np.linalg.norm(orc["xin"])) <= 1e-12 * info["xi_norm"]
    # free eps-rank: Thm A.1(d) bound against the untruncated canonical tensor
    out = ls.eval_slab_torch(slabs).cpu().numpy()
    err2 = 0.0
    for k, z in enumerate(slabs):
        can = O.canonical_slab(orc["ncols"], orc["tcol"], orc["xin"], z)
        err2 += float(np.sum((out[k] - can) ** 2))
        if fp_tol is not None:
            assert rel(out[k], can) <= fp_tol
    assert math.sqrt(err2) <= info["bound_abs"] * (1 + 1e-6) + 1e-12 * np.abs(out).max()
    ls.close()
    return info, res


def forced_rank_parity(wl, s, precision=L.LS_FP64, tol=1e-12):
    """At the oracle's ranks (forced), the FP64 path's Tucker tensor equals the
    oracle's to `tol` relative on every seeded slab, and so does the core's
    Frobenius norm (projector-invariant: the bases may differ by rotations
    inside degenerate singular values)."""
    orc = oracle_run(wl, s)
    r_or = orc["res"]["r"]
    res = orc["res"]
    ls = gpu_ctx(wl, s, precision)
    info = ls.rhosvd_reduce(wl.eps, forced_ranks=r_or)
    assert list(info["r"]) == list(r_or), (info["r"], r_or)
    out = ls.eval_slab_torch(wl.slabs).cpu().numpy()
    worst = 0.0
    for k, z in enumerate(wl.slabs):
        ref = O.tucker_slab(res["Z"], res["B"], z)
        worst = max(worst, rel(out[k], ref))
    assert worst <= tol, (worst, tol)
    core = ls.read(L.LS_READ_CORE)
    assert abs(np.linalg.norm(core) - np.linalg.norm(res["B"])) <= tol * np.linalg.norm(res["B"])
    ls.close()
    return worst


def test_config1_fp64_end_to_end():
    wl = W.config1()
    s = scale_for(wl)
    info, res = check_reduction(wl, s)
    # defect-free lattice: exact canonical rank R (Thm 3.1) -> r <= R
    assert max(info["r"]) <= wl.R


def test_config1_fp64_forced_rank():
    wl = W.config1()
    forced_rank_parity(wl, scale_for(wl))


def test_config1_fp64_against_brute_force():
    """Slab values against the direct sum of 1/|x - a| within the quadrature
    tolerance plus the truncation bound."""
    wl = W.config1()
    s = scale_for(wl)
    ls = gpu_ctx(wl, s)
    info = ls.rhosvd_reduce(wl.eps)
    z = [64, 128, 200]
    out = ls.eval_slab_torch(z).cpu().numpy()
    xs = O.cell_centres(wl.N, wl.box_lo, wl.box_hi)
    centres, charges = O.charged_centres(wl.N, wl.box_lo, wl.box_hi, wl.blocks, wl.defects)
    t, w = O.sinc_quadrature(wl.R, wl.sinc_step, s)
    tau = float(np.max(O.quadrature_rel_error(t, w, np.geomspace(wl.r_min, O.default_r_max(wl), 6000))))
    rng = np.random.default_rng(5)
    for k, zz in enumerate(z):
        ij = rng.integers(0, wl.N, size=(3000, 2))
        pts = np.stack([xs[ij[:, 0]], xs[ij[:, 1]], np.full(len(ij), xs[zz])], 1)
        bf, absbf, dmin, _ = O.brute_force(pts, centres, charges)
        keep = dmin >= wl.r_min
        val = out[k][ij[keep, 0], ij[keep, 1]]
        assert np.all(np.abs(val - bf[keep]) <= tau * absbf[keep] * 1.01 + info["bound_abs"])


def test_config2_fp64_end_to_end():
    wl = W.config2()
    check_reduction(wl, scale_for(wl))


def test_config2_fp64_slab_accuracy():
    """16^3 lattice with defects, eps = 1e-6, on 16 of its seeded slabs: the
    FP64 path takes the oracle's ranks by itself and reproduces the oracle's
    Tucker values to 1e-12 relative, and the untruncated canonical tensor to
    within eps (the oracle's own truncation error is 8.5e-8 here)."""
    wl = W.config2()
    s = scale_for(wl)
    orc = oracle_run(wl, s)
    ls = gpu_ctx(wl, s)
    info = ls.rhosvd_reduce(wl.eps)
    assert info["r"] == list(orc["res"]["r"])
    z = wl.slabs[:16]
    out = ls.eval_slab_torch(z).cpu().numpy()
    ref_t = np.stack([O.tucker_slab(orc["res"]["Z"], orc["res"]["B"], zz) for zz in z])
    ref_c = np.stack([O.canonical_slab(orc["ncols"], orc["tcol"], orc["xin"], zz) for zz in z])
    assert rel(out, ref_t) < 1e-12, rel(out, ref_t)
    assert rel(out, ref_c) < wl.eps, rel(out, ref_c)
    assert rel(out, ref_c) < 1.5 * rel(ref_t, ref_c) + 1e-12
    ls.close()


def test_config2_fp64_forced_rank():
    wl = W.config2()
    forced_rank_parity(wl, scale_for(wl))


@pytest.mark.parametrize("wl", [W.small_case(L=(3, 2, 2), frac_vac=0.2, frac_imp=0.1, eps=1e-6),
                                W.small_case(L=(1, 1, 1), N=33, eps=1e-10),
                                W.small_case(L=(7, 3, 2), N=70, frac_vac=0.1, eps=1e-5)],
                         ids=lambda w: f"{w.name}_eps{w.eps:g}")
def test_small_cases_fp64(wl):
    s = scale_for(wl)
    check_reduction(wl, s)
    forced_rank_parity(wl, s)


@pytest.mark.parametrize("eps", [1e-8, 1e-10, 1e-12])
def test_small_eps_reduces_without_error(eps):
    """eps far below the Gram route's resolution sqrt(8 u T): the non-squaring
    route keeps the oracle's ranks and its Tucker values (the 4x4x4 lattice's
    singular values fall to ~1e-14 sigma_1, so eps = 1e-12 keeps nearly all)."""
    wl = W.small_case(L=(4, 4, 4), N=64, frac_vac=0.1, eps=eps)
    s = scale_for(wl)
    check_reduction(wl, s)
    forced_rank_parity(wl, s)


def test_gram_route_still_available():
    """LS_FLAG_SVD_GRAM puts an FP64 context on the Gram route (the mixed path's):
    at eps = 1e-6 it meets its own resolution-based checks and the Thm A.1(d)
    bound."""
    wl = W.small_case(L=(3, 2, 2), frac_vac=0.2, frac_imp=0.1, eps=1e-6)
    check_reduction(wl, scale_for(wl), flags=L.LS_FLAG_SVD_GRAM)


@pytest.mark.parametrize("cls", ["B", "C"])
def test_skewed_lattices_fp64(cls):
    """Sec. 4.4 classes (B) and (C): a parallelogram lattice and a lattice
    skewed in two directions (unions of rectangular blocks), with vacancies
    placed at skewed sites as point charges: the full reduction checks."""
    L3 = (6, 5, 3)
    a2 = (0.5, 1.0, 0.0)
    a3 = (0.0, 0.0, 1.0) if cls == "B" else (0.3, 0.25, 1.0)
    origin = (-4.0, -2.6, -1.2)
    blocks = W.skewed_lattice_blocks(L3, 1.0, a2, a3, origin)
    defects = [W.Defect(W.DEFECT_POINT, pos=tuple(origin[d] + i * (1.0 if d == 0 else 0.0) + j * a2[d] + k * a3[d]
                                                  for d in range(3)), charge=-1.0)
               for (i, j, k) in ((1, 1, 0), (4, 2, 1), (2, 4, 2))]
    wl = W.Workload("skew" + cls, 56, -8.0, 8.0, 16, 0.3, 1e-6, blocks, defects, r_min=0.5, slabs=[28, 20])
    s = scale_for(wl)
    check_reduction(wl, s)
    forced_rank_parity(wl, s)


def test_cubic_lattice_modes_are_equivalent():
    """A defect-free cubic centred lattice is symmetric under axis
    permutations: equal spectra in all modes and symmetric slabs."""
    wl = W.config1()
    ls = gpu_ctx(wl, scale_for(wl))
    info = ls.rhosvd_reduce(wl.eps)
    s = [ls.read(L.LS_READ_SIGMA, a) for a in range(3)]
    assert np.allclose(s[0], s[1], rtol=0, atol=1e-12 * s[0][0]) and np.allclose(s[0], s[2], rtol=0, atol=1e-12 * s[0][0])
    out = ls.eval_slab_torch([100]).cpu().numpy()[0]
    assert rel(out, out.T) < 1e-12
    assert rel(out, out[::-1, ::-1]) < 1e-10    # reflection about the box centre


def test_f32_output_matches_f64():
    wl = W.config1()
    ls = gpu_ctx(wl, scale_for(wl))
    ls.rhosvd_reduce(wl.eps)
    a = ls.eval_slab_torch([3, 77, 255]).cpu().numpy()
    b = ls.eval_slab_torch([3, 77, 255], dtype=torch.float32).cpu().numpy()
    assert np.max(np.abs(a - b) / np.abs(a).max()) < 1e-7


# ---------------------------------------------------------------------------
# call order and argument errors through the C ABI
# ---------------------------------------------------------------------------

def test_call_order_and_argument_errors():
    wl = W.small_case()
    s = scale_for(wl)
    ls = gpu_ctx(wl, s)
    out = torch.empty((1, wl.N, wl.N), dtype=torch.float64, device="cuda")
    with pytest.raises(L.LatticeSumError) as ei:
        ls.eval_slab([0], out.data_ptr())
    assert ei.value.code == L.LS_ERR_STATE
    with pytest.raises(L.LatticeSumError) as ei:
        ls.add_defects([W.Defect(W.DEFECT_SITES, 3, (0, 0, 0))])
    assert ei.value.code == L.LS_ERR_ARG
    with pytest.raises(L.LatticeSumError) as ei:
        ls.add_defects([W.Defect(W.DEFECT_SITES, 0, (2, 1, 1), (2, 1, 1))])
    assert ei.value.code == L.LS_ERR_ARG
    with pytest.raises(L.LatticeSumError) as ei:
        ls.rhosvd_reduce(0.0)
    assert ei.value.code == L.LS_ERR_ARG
    ls.rhosvd_reduce(1e-6)
    with pytest.raises(L.LatticeSumError) as ei:
        ls.rhosvd_reduce(1e-6)
    assert ei.value.code == L.LS_ERR_STATE
    with pytest.raises(L.LatticeSumError) as ei:
        ls.add_defects([W.Defect(W.DEFECT_SITES, 0, (0, 0, 0))])
    assert ei.value.code == L.LS_ERR_STATE
    with pytest.raises(L.LatticeSumError) as ei:
        ls.eval_slab([wl.N], out.data_ptr())
    assert ei.value.code == L.LS_ERR_ARG
    ls.eval_slab([0], out.data_ptr())
    torch.cuda.synchronize()
    ls.close()
