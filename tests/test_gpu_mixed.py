"""GPU parity of the mixed-precision path (tcgen05 contractions with exact
head accumulation, FP64 orthogonalisation) against the FP64 path and the FP64
oracle.

Tolerances, from the arithmetic of the tensor-core contractions: every
operand row is scaled by a power of two and written as two exact 7-bit
digits and two 11-bit tails (FP16); the digit products accumulate exactly in
FP32 (two levels), the products below them in a third accumulator at 2^-14
of the result or less. A contraction is then good to ~2^-30 of
sum |a_k b_k|; with the cancellation of the core contraction the tests allow
1e-7 relative against the FP64 path for projections, the core and slabs, and
the configuration's eps (1e-6) for the final slab values against the FP64
oracle, as the precision target requires. The measured tile-width choice
(lattice_sum_tune_eval) changes no result bit.
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


def scale_for(wl):
    s, _ = O.fit_t_scale(wl.R, wl.sinc_step, wl.r_min, O.default_r_max(wl))
    return s


def run(wl, s, prec, forced=None, flags=0):
    ls = L.LatticeSum.from_workload(wl, s, prec, flags=flags)
    ls.add_defects(wl.defects)
    info = ls.rhosvd_reduce(wl.eps, forced_ranks=forced)
    return ls, info


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("wl", [W.small_case(L=(3, 2, 2), frac_vac=0.2, frac_imp=0.1, eps=1e-6),
                                W.small_case(L=(5, 3, 2), N=50, frac_vac=0.2, eps=1e-6),
                                W.config2()], ids=lambda w: w.name)
def test_mixed_contractions_match_fp64_path(wl):
    s = scale_for(wl)
    # the FP64 path on the mixed path's singular-value route (the Gram route): the same
    # pre-compression and eps rule; the mixed path stops its eigen-solver after the first Jacobi
    # run (Rayleigh quotients of the FP64 re-projection), so the bases agree as subspaces, and
    # the contractions are compared through basis-free quantities
    a, ia = run(wl, s, L.LS_FP64, flags=L.LS_FLAG_SVD_GRAM)
    b, ib = run(wl, s, L.LS_MIXED)
    assert ib["r"] == ia["r"]
    for m in range(3):
        Za = a.read(L.LS_READ_BASIS, m).reshape(ia["r"][m], wl.N)
        Zb = b.read(L.LS_READ_BASIS, m).reshape(ib["r"][m], wl.N)
        pa, pb = a.read(L.LS_READ_PROJ, m).reshape(ia["r"][m], -1), b.read(L.LS_READ_PROJ, m).reshape(ib["r"][m], -1)
        # the projected side matrices Z^T P (the columns' components in the subspace)
        assert rel(Zb.T @ pb, Za.T @ pa) < 1e-7, (m, rel(Zb.T @ pb, Za.T @ pa))
    ca, cb = a.read(L.LS_READ_CORE), b.read(L.LS_READ_CORE)
    assert abs(np.linalg.norm(cb) - np.linalg.norm(ca)) < 1e-7 * np.linalg.norm(ca)
    z = wl.slabs[:8]
    sa = a.eval_slab_torch(z).cpu().numpy()
    sb = b.eval_slab_torch(z).cpu().numpy()
    assert rel(sb, sa) < 1e-7, rel(sb, sa)
    a.close()
    b.close()


def test_mixed_slabs_meet_eps_against_oracle():
    """16^3 lattice with defects, eps = 1e-6: relative L2 error of the mixed
    slabs (FP32 output) against the untruncated FP64 canonical tensor of the
    oracle is within eps, on the 64 seeded slabs."""
    wl = W.config2()
    s = scale_for(wl)
    t, w = O.sinc_quadrature(wl.R, wl.sinc_step, s)
    g = O.generating_vectors(wl.N, wl.box_lo, wl.box_hi, t, w)
    cols, tcol, xi = O.canonical_terms(wl.N, wl.box_lo, wl.box_hi, g, wl.blocks, wl.defects)
    ncols, _, xin = O.normalise_terms(cols, tcol, xi)
    ls, info = run(wl, s, L.LS_MIXED)
    out = ls.eval_slab_torch(wl.slabs, dtype=torch.float32).cpu().numpy().astype(np.float64)
    num = den = 0.0
    worst = 0.0
    for k, zz in enumerate(wl.slabs):
        ref = O.canonical_slab(ncols, tcol, xin, zz)
        num += float(np.sum((out[k] - ref) ** 2))
        den += float(np.sum(ref ** 2))
        worst = max(worst, float(np.max(np.abs(out[k] - ref))))
    err = math.sqrt(num / den)
    assert err <= wl.eps, err
    # the largest pointwise error, relative to the largest value: also within eps
    assert worst <= wl.eps * float(np.max(np.abs(out))), worst
    ls.close()


@pytest.mark.parametrize("wl", [W.config2(), W.small_case(L=(4, 3, 2), N=64, frac_vac=0.15, frac_imp=0.1, eps=1e-6)],
                         ids=lambda w: w.name)
def test_mixed_against_fp64_path_at_common_ranks(wl):
    """The mixed path (Gram route, tensor-core contractions) against the FP64
    path (non-squaring route, FP64 contractions) at the FP64 path's ranks:
    the Gram route's subspace and the contractions together stay within
    1e-7 of the FP64 result on slabs, far inside eps."""
    s = scale_for(wl)
    a, ia = run(wl, s, L.LS_FP64)
    b, ib = run(wl, s, L.LS_MIXED, forced=ia["r"])
    assert ib["r"] == ia["r"]
    z = wl.slabs[:8]
    sa = a.eval_slab_torch(z).cpu().numpy()
    sb = b.eval_slab_torch(z).cpu().numpy()
    assert rel(sb, sa) < 1e-7, rel(sb, sa)
    a.close()
    b.close()


def test_mixed_context_on_the_non_squaring_route():
    """LS_FLAG_SVD_ONESIDED on a mixed context: its ranks and bases are the FP64
    path's (same route), and its slabs agree with them to the contractions'
    accuracy."""
    wl = W.small_case(L=(3, 2, 2), frac_vac=0.2, frac_imp=0.1, eps=1e-8)
    s = scale_for(wl)
    a, ia = run(wl, s, L.LS_FP64)
    b, ib = run(wl, s, L.LS_MIXED, flags=L.LS_FLAG_SVD_ONESIDED)
    assert ib["r"] == ia["r"]
    for m in range(3):
        assert np.array_equal(a.read(L.LS_READ_BASIS, m), b.read(L.LS_READ_BASIS, m))
    z = wl.slabs
    assert rel(b.eval_slab_torch(z).cpu().numpy(), a.eval_slab_torch(z).cpu().numpy()) < 1e-7
    a.close()
    b.close()


def test_mixed_single_site_and_ragged_tiles():
    """Degenerate ranks (a single site, r = 1 per mode possible) and sizes that
    leave ragged tensor-core tiles in every dimension."""
    for wl in (W.small_case(L=(1, 1, 1), N=33, eps=1e-6), W.small_case(L=(7, 3, 2), N=70, frac_vac=0.1, eps=1e-5)):
        s = scale_for(wl)
        a, ia = run(wl, s, L.LS_FP64, flags=L.LS_FLAG_SVD_GRAM)
        b, ib = run(wl, s, L.LS_MIXED)
        assert ib["r"] == ia["r"]
        z = [0, wl.N // 2, wl.N - 1]
        sa = a.eval_slab_torch(z).cpu().numpy()
        sb = b.eval_slab_torch(z).cpu().numpy()
        assert rel(sb, sa) < 1e-7, (wl.name, rel(sb, sa))
        a.close()
        b.close()


def test_tuned_evaluation_is_bitwise_the_plain_one():
    wl = W.config2()
    s = scale_for(wl)
    ls, _ = run(wl, s, L.LS_MIXED)
    zs = [int(z) for z in wl.slabs[:16]]
    plain = ls.eval_slab_torch(zs, dtype=torch.float32).cpu().numpy()
    out = torch.empty((len(zs), wl.N, wl.N), dtype=torch.float32, device="cuda")
    rep = ls.tune_eval(zs, out)
    assert set(rep) == {"M", "T", "S"}, rep
    for name, r in rep.items():
        assert r["tile_n"] in (32, 64, 128) and len(r["ms"]) == 3 and min(r["ms"]) > 0.0, (name, r)
    assert np.array_equal(out.cpu().numpy(), plain)
    # later evaluations take the kept widths and still agree bit for bit
    again = ls.eval_slab_torch(zs, dtype=torch.float32).cpu().numpy()
    assert np.array_equal(again, plain)
    ls.close()


def test_tune_rejects_fp64_context():
    wl = W.small_case(L=(3, 2, 2), eps=1e-6)
    s = scale_for(wl)
    ls, _ = run(wl, s, L.LS_FP64)
    out = torch.empty((1, wl.N, wl.N), dtype=torch.float64, device="cuda")
    with pytest.raises(L.LatticeSumError):
        ls.tune_eval([wl.N // 2], out)
    ls.close()
