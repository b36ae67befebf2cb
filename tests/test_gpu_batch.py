"""The batched form (lattice_sum_batch_reduce) against individual reductions
and the oracle: every item of a small seeded batch of uneven lattices (sizes,
grids, ranks, defect fractions drawn like the 256-item batch workload, scaled
down so that the oracle finishes in seconds) must give the ranks and slab
values of its own lattice_sum_rhosvd_reduce, and stay within eps of the
untruncated canonical tensor."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import lattice_oracle as O  # noqa: E402
from paper_1411_1994_gb300 import build as B  # noqa: E402
from paper_1411_1994_gb300 import lattice_sum as L  # noqa: E402
from paper_1411_1994_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


def small_batch(n=6):
    out = []
    for j in range(n):
        rng = W.SplitMix64(7000 + j)
        Ls = tuple(2 + rng.below(5) for _ in range(3))
        N = (48, 64, 80)[rng.below(3)]
        R = (12, 14, 16)[rng.below(3)]
        f = 0.3 * rng.uniform()
        lo, hi = W.box_for(Ls)
        blocks = [W.centred_block(Ls)]
        defects = W.point_defects(rng, blocks, f * 5 / 7, f * 2 / 7)
        out.append(W.Workload(f"b{j}", N, lo, hi, R, 0.3, 1e-6, blocks, defects, r_min=0.5, slabs=[N // 2, 5]))
    return out


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    B.build()
    L.lib()


# 6 lattices: 18 eigen-problems, each in an 8-CTA cluster (all fit on the GPU at once); 8
# lattices: 24, more than 8-CTA clusters can hold side by side on 152 SMs, so the launch takes
# 4-CTA clusters, while each individual reduction (3 problems) keeps 8-CTA ones
@pytest.mark.parametrize("n", [6, 8])
@pytest.mark.parametrize("precision", [L.LS_FP64, L.LS_MIXED])
def test_batch_matches_individual_reductions(precision, n):
    wls = small_batch(n)
    scales = [O.fit_t_scale(w.R, w.sinc_step, w.r_min, O.default_r_max(w))[0] for w in wls]
    batch = []
    for w, s in zip(wls, scales):
        c = L.LatticeSum.from_workload(w, s, precision)
        c.add_defects(w.defects)
        batch.append(c)
    infos = L.batch_reduce(batch, 1e-6)
    for w, s, c, info in zip(wls, scales, batch, infos):
        one = L.LatticeSum.from_workload(w, s, precision)
        one.add_defects(w.defects)
        i1 = one.rhosvd_reduce(1e-6)
        assert info["r"] == i1["r"], (w.name, info["r"], i1["r"])
        a = c.eval_slab_torch(w.slabs).cpu().numpy()
        b = one.eval_slab_torch(w.slabs).cpu().numpy()
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b), w.name
        t, wq = O.sinc_quadrature(w.R, w.sinc_step, s)
        g = O.generating_vectors(w.N, w.box_lo, w.box_hi, t, wq)
        cols, tcol, xi = O.canonical_terms(w.N, w.box_lo, w.box_hi, g, w.blocks, w.defects)
        ncols, _, xin = O.normalise_terms(cols, tcol, xi)
        ref = np.stack([O.canonical_slab(ncols, tcol, xin, z) for z in w.slabs])
        assert np.linalg.norm(a - ref) <= w.eps * np.linalg.norm(ref), w.name
        one.close()
        c.close()


def test_batch_rejects_bad_input():
    w = small_batch(1)[0]
    s = O.fit_t_scale(w.R, w.sinc_step, w.r_min, O.default_r_max(w))[0]
    c = L.LatticeSum.from_workload(w, s)
    with pytest.raises(L.LatticeSumError) as ei:
        L.batch_reduce([c, c], 1e-6)
    assert ei.value.code == L.LS_ERR_ARG
    c.rhosvd_reduce(1e-6)
    with pytest.raises(L.LatticeSumError) as ei:
        L.batch_reduce([c], 1e-6)
    assert ei.value.code == L.LS_ERR_STATE
    c.close()
