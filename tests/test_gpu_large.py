"""Full-size parity on the two large configurations, run as bench.py runs them
(create, add_defects, rhosvd_reduce, then slabs).

The step-shaped lattice (a 48x48x24 and a 24^3 block,
3% vacancies, N = 4096, R = 28, eps = 1e-6): the configuration of the
precision comparison, run as bench.py runs it (create, add_defects,
rhosvd_reduce, then slabs), for both arithmetic paths.

The oracle cannot reduce this size in seconds (its core alone is an einsum
of ~7e12 flop), but it can compute single grid rows of the untruncated
canonical tensor exactly (Eq. Can_LatticeSum_full): for fixed (x, z) the row
over y is sum_t xi_t a0[c0(t)][x] a2[c2(t)][z] a1[c1(t)][:], i.e. a weight
per distinct mode-1 vector followed by one product with the mode-1 side
matrix. The sampled rows (16 rows in each of 8 seeded z-slabs, 524288
values) must lie within eps of those values in relative L2 (the Frobenius
error of the Tucker result is bounded by Thm A.1(d); random rows estimate
the relative Frobenius error), and the reported bound must dominate the
observed error on the samples.

The 256^3 lattice with 1000 3x3x3 defect clusters (N = 16384, R = 32,
eps = 1e-6; C ~ 8000 columns and ranks ~ 2200 per mode, a core of ~1.1e10
entries) runs the mixed path only and is checked the same way on 4 of its
slabs (8 rows each, 524288 values).
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


@pytest.fixture(scope="module")
def step_lattice():
    wl = W.config3()
    s, _ = O.fit_t_scale(wl.R, wl.sinc_step, wl.r_min, O.default_r_max(wl))
    t, w = O.sinc_quadrature(wl.R, wl.sinc_step, s)
    g = O.generating_vectors(wl.N, wl.box_lo, wl.box_hi, t, w)
    cols, tcol, xi = O.canonical_terms(wl.N, wl.box_lo, wl.box_hi, g, wl.blocks, wl.defects)
    ncols, _, xin = O.normalise_terms(cols, tcol, xi)
    return wl, s, ncols, tcol, xin


def canonical_row(ncols, tcol, xin, x, z):
    """Row (x, :, z) of sum_t xin_t a0[c0][x] a1[c1][:] a2[c2][z]."""
    wt = xin * ncols[0][tcol[:, 0], x] * ncols[2][tcol[:, 2], z]
    coef = np.bincount(tcol[:, 1], weights=wt, minlength=ncols[1].shape[0])
    return coef @ ncols[1]


@pytest.mark.parametrize("precision", [L.LS_FP64, L.LS_MIXED], ids=["fp64", "mixed"])
def test_step_lattice_sampled_rows_within_eps(step_lattice, precision):
    wl, s, ncols, tcol, xin = step_lattice
    ls = L.LatticeSum.from_workload(wl, s, precision)
    ls.add_defects(wl.defects)
    info = ls.rhosvd_reduce(wl.eps)
    assert info["T"] == tcol.shape[0]
    assert all(c == n.shape[0] for c, n in zip(info["C"], ncols))
    assert all(1 <= r <= c for r, c in zip(info["r"], info["C"]))
    rng = np.random.default_rng(4096)
    zs = [int(z) for z in wl.slabs[:8]]
    slabs = ls.eval_slab_torch(zs).cpu().numpy()
    num = den = 0.0
    for k, z in enumerate(zs):
        for x in rng.choice(wl.N, size=16, replace=False):
            ref = canonical_row(ncols, tcol, xin, int(x), z)
            num += float(np.sum((slabs[k, int(x)] - ref) ** 2))
            den += float(np.sum(ref ** 2))
    err = math.sqrt(num / den)
    assert err <= wl.eps, err
    # the absolute Thm A.1(d) bound dominates the absolute error on the samples
    assert math.sqrt(num) <= info["bound_abs"], (math.sqrt(num), info["bound_abs"])
    ls.close()


@pytest.fixture(scope="module")
def cluster_lattice():
    wl = W.config5()
    s, _ = O.fit_t_scale(wl.R, wl.sinc_step, wl.r_min, O.default_r_max(wl))
    t, w = O.sinc_quadrature(wl.R, wl.sinc_step, s)
    g = O.generating_vectors(wl.N, wl.box_lo, wl.box_hi, t, w)
    cols, tcol, xi = O.canonical_terms(wl.N, wl.box_lo, wl.box_hi, g, wl.blocks, wl.defects)
    ncols, _, xin = O.normalise_terms(cols, tcol, xi)
    return wl, s, ncols, tcol, xin


def test_cluster_lattice_sampled_rows_within_eps(cluster_lattice):
    wl, s, ncols, tcol, xin = cluster_lattice
    ls = L.LatticeSum.from_workload(wl, s, L.LS_MIXED)
    ls.add_defects(wl.defects)
    info = ls.rhosvd_reduce(wl.eps)
    assert info["T"] == tcol.shape[0]
    assert all(c == n.shape[0] for c, n in zip(info["C"], ncols))
    assert all(1 <= r <= c for r, c in zip(info["r"], info["C"]))
    rng = np.random.default_rng(16384)
    zs = [int(z) for z in wl.slabs[:4]]
    slabs = ls.eval_slab_torch(zs)
    num = den = 0.0
    for k, z in enumerate(zs):
        xs = [int(x) for x in rng.choice(wl.N, size=8, replace=False)]
        rows = slabs[k, xs].cpu().numpy()
        for i, x in enumerate(xs):
            ref = canonical_row(ncols, tcol, xin, x, z)
            num += float(np.sum((rows[i] - ref) ** 2))
            den += float(np.sum(ref ** 2))
    del slabs
    err = math.sqrt(num / den)
    assert err <= wl.eps, err
    assert math.sqrt(num) <= info["bound_abs"], (math.sqrt(num), info["bound_abs"])
    ls.close()
