"""Pins of the FP64 oracle to things other than itself (no GPU needed).

Each test checks the oracle against a closed form, an exact identity of the
paper, brute-force 1/|x - a| sums, or the paper's RHOSVD error bound. They are
chosen so that a plausible slip (a dropped factor in a weight, a shifted
window index, a transposed projection, a wrong rank rule) fails one of them.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import lattice_oracle as O
from paper_1411_1994_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _terms(wl, s=None):
    if s is None:
        s, _ = O.fit_t_scale(wl.R, wl.sinc_step, wl.r_min, O.default_r_max(wl))
    t, w = O.sinc_quadrature(wl.R, wl.sinc_step, s)
    g = O.generating_vectors(wl.N, wl.box_lo, wl.box_hi, t, w)
    cols, tcol, xi = O.canonical_terms(wl.N, wl.box_lo, wl.box_hi, g, wl.blocks, wl.defects)
    return s, t, w, g, cols, tcol, xi


# --- (a0) quadrature: Sec. 2.1, Eqs. laplace / hM / sinc_Newt ---------------

def test_fine_sinc_rule_reproduces_inverse_distance():
    """With a fine step and many nodes the rule must reproduce the closed form
    1/r = (2/sqrt(pi)) int exp(-r^2 t^2) dt to ~machine precision: any wrong
    factor in t_q or w_q (the 2, the cosh, sqrt(pi), the halved q=0 weight)
    leaves an O(1) error."""
    t, w = O.sinc_quadrature(400, 0.05, 10.0)
    r = np.geomspace(0.05, 50.0, 2000)
    assert np.max(O.quadrature_rel_error(t, w, r)) < 1e-12


def test_gaussian_integral_identity():
    """Laplace-Gauss identity at one r, by an independent trapezoid rule in t
    (not in u): (2/sqrt(pi)) int_0^T exp(-r^2 t^2) dt -> 1/r."""
    r = 0.7
    tt = np.linspace(0.0, 40.0, 400001)
    f = np.exp(-(r * tt) ** 2)
    integral = (2.0 / math.sqrt(math.pi)) * np.trapezoid(f, tt)
    t, w = O.sinc_quadrature(400, 0.05, 10.0)
    approx = float(np.sum(w * np.exp(-(t * r) ** 2)))
    assert abs(integral - 1.0 / r) < 1e-10
    assert abs(approx - integral) < 1e-10


def test_sinc_error_decays_with_rank():
    """Eq. (sinc_conv): the error decays (exponentially in sqrt(M)) with the
    number of nodes at a fixed, well-chosen step."""
    r = np.geomspace(0.25, 20.0, 500)
    errs = []
    for R in (12, 18, 24, 30):
        s, _ = O.fit_t_scale(R, 0.25, 0.25, 20.0)
        t, w = O.sinc_quadrature(R, 0.25, s)
        errs.append(float(np.max(O.quadrature_rel_error(t, w, r))))
    assert all(a > 3 * b for a, b in zip(errs, errs[1:])), errs


def test_fitted_scale_error_holds_on_dense_grid():
    """The error reported by the scale fit holds on a 10x denser r-grid (to
    within 20%), and for the 4x4x4 configuration (R=24, h=0.25) it is below
    1e-7 on [0.25, sqrt(3) b]."""
    wl = W.config1()
    rmax = O.default_r_max(wl)
    s, e = O.fit_t_scale(wl.R, wl.sinc_step, wl.r_min, rmax)
    t, w = O.sinc_quadrature(wl.R, wl.sinc_step, s)
    dense = np.max(O.quadrature_rel_error(t, w, np.geomspace(wl.r_min, rmax, 6000)))
    assert dense < 1.2 * e
    assert dense < 1e-7


def test_fitted_scale_is_a_local_minimum():
    """Sec. 2.1 chooses the quadrature so that the kernel is reproduced to a tolerance; the
    oracle's fit takes the scale s that minimises the largest relative error on its r-grid. The
    returned error is the error at the returned s, and moving s by 0.1 %, 1 % or 3 % either way
    gives no smaller error on the same grid (a search that kept the wrong half of a bracket, or
    returned a bracket end, fails this)."""
    for R, h, r0, r1 in ((24, 0.25, 0.25, 20.0), (28, 0.25, 0.25, 48.5), (20, 0.3, 0.5, 30.0)):
        s, e = O.fit_t_scale(R, h, r0, r1)
        r = np.geomspace(r0, r1, 600)

        def err(sc):
            t, w = O.sinc_quadrature(R, h, sc)
            return float(np.max(O.quadrature_rel_error(t, w, r)))

        assert err(s) == e
        for f in (0.97, 0.99, 0.999, 1.001, 1.01, 1.03):
            assert err(s * f) >= e * (1.0 - 1e-12), (R, f, err(s * f), e)


# --- (a0) the Yukawa kernel: Sec. 2.3, Eq. LalpYukawa ----------------------

def test_yukawa_laplace_gauss_identity_and_reading():
    """By a plain trapezoid rule in t: (2/sqrt(pi)) int exp(-kappa^2/(4 t^2))
    exp(-r^2 t^2) dt = exp(-kappa r)/r, the identity the oracle's weights use;
    the exponent kappa^2/t^2 as printed integrates to exp(-2 kappa r)/r."""
    tt = np.linspace(1e-9, 40.0, 800001)
    for kappa, r in ((0.8, 0.7), (1.5, 2.0), (0.3, 5.0)):
        quarter = (2.0 / math.sqrt(math.pi)) * np.trapezoid(np.exp(-kappa ** 2 / (4 * tt ** 2) - (r * tt) ** 2), tt)
        printed = (2.0 / math.sqrt(math.pi)) * np.trapezoid(np.exp(-kappa ** 2 / tt ** 2 - (r * tt) ** 2), tt)
        assert abs(quarter - math.exp(-kappa * r) / r) <= 1e-12 * math.exp(-kappa * r) / r + 1e-15
        assert abs(printed - math.exp(-2 * kappa * r) / r) <= 1e-12 * math.exp(-2 * kappa * r) / r + 1e-15


def test_fine_sinc_rule_reproduces_yukawa():
    """A fine rule reproduces exp(-kappa r)/r to ~machine precision relative to
    the kernel itself; a dropped screening factor, a wrong 1/4 or keeping the
    zero-weight node t_0 = 0 leaves an O(1) error somewhere on the range."""
    for kappa in (0.4, 0.8, 2.0):
        t, w = O.sinc_quadrature(400, 0.05, 10.0, kappa)
        assert t[0] > 0.0 and np.all(w >= 0.0) and np.all(np.diff(t) > 0.0)
        r = np.geomspace(0.05, 20.0, 2000)
        approx = np.exp(-np.outer(r * r, t * t)) @ w
        assert np.max(np.abs(approx / (np.exp(-kappa * r) / r) - 1.0)) < 1e-11
        assert np.max(O.quadrature_rel_error(t, w, r, kappa)) < 1e-12
    # kappa = 0 is the Newton rule, bit for bit
    t0, w0 = O.sinc_quadrature(24, 0.25, 13.0, 0.0)
    t1, w1 = O.sinc_quadrature(24, 0.25, 13.0)
    assert np.array_equal(t0, t1) and np.array_equal(w0, w1)


def test_yukawa_fitted_scale_error_holds_on_dense_grid():
    """For the 16^3 lattice's rank and range (R = 24, h = 0.25, r in
    [0.25, sqrt(3) b]) and kappa = 0.5 the fitted rule's error relative to 1/r
    is below 1e-6 and holds on a 10x denser grid."""
    wl = W.config2()
    rmax = O.default_r_max(wl)
    s, e = O.fit_t_scale(wl.R, wl.sinc_step, wl.r_min, rmax, kappa=0.5)
    t, w = O.sinc_quadrature(wl.R, wl.sinc_step, s, 0.5)
    dense = np.max(O.quadrature_rel_error(t, w, np.geomspace(wl.r_min, rmax, 6000), 0.5))
    assert dense < 1.2 * e
    assert dense < 1e-6


def test_yukawa_lattice_against_brute_force():
    """A defected lattice with the Yukawa kernel: canonical tensor values at
    sampled grid points vs the direct sum of Z exp(-kappa d)/d over the snapped
    centres, within tau * sum |Z|/d (tau: the rule's error relative to 1/r)."""
    wl = W.small_case(L=(4, 3, 3), N=60, R=20, frac_vac=0.2, frac_imp=0.1, kappa=0.6)
    rmax = O.default_r_max(wl)
    s, _ = O.fit_t_scale(wl.R, wl.sinc_step, wl.r_min, rmax, kappa=wl.kappa)
    t, w = O.sinc_quadrature(wl.R, wl.sinc_step, s, wl.kappa)
    g = O.generating_vectors(wl.N, wl.box_lo, wl.box_hi, t, w)
    cols, tcol, xi = O.canonical_terms(wl.N, wl.box_lo, wl.box_hi, g, wl.blocks, wl.defects)
    xs = O.cell_centres(wl.N, wl.box_lo, wl.box_hi)
    rng = np.random.default_rng(4)
    idx = rng.integers(0, wl.N, size=(20000, 3))
    centres, charges = O.charged_centres(wl.N, wl.box_lo, wl.box_hi, wl.blocks, wl.defects)
    bf, _, dmin, _ = O.brute_force(xs[idx], centres, charges, kappa=wl.kappa)
    _, abs_newton, _, _ = O.brute_force(xs[idx], centres, charges)
    keep = dmin >= wl.r_min
    tens = (xi[:, None] * cols[0][tcol[:, 0]][:, idx[keep, 0]] * cols[1][tcol[:, 1]][:, idx[keep, 1]]
            * cols[2][tcol[:, 2]][:, idx[keep, 2]]).sum(0)
    tau = float(np.max(O.quadrature_rel_error(t, w, np.geomspace(wl.r_min, rmax, 6000), wl.kappa)))
    err = np.abs(tens - bf[keep])
    assert np.all(err <= tau * abs_newton[keep] * 1.001 + 1e-13)
    # the screening is real: the Newton sum differs by far more than that
    nb, _, _, _ = O.brute_force(xs[idx[keep]], centres, charges)
    assert np.min(np.abs(nb - bf[keep]) - err) > 0.0


# --- (a0) Slater and dipole kernels: Sec. 2.3, Eqs. LalpSlater, LalpPoly ---

def test_slater_and_dipole_transforms():
    """By trapezoid rules: Eq. LalpSlater as printed, exp(-2 sqrt(k rho)) =
    sqrt(k/pi) int t^-3/2 exp(-k/t) exp(-rho t) dt, and the Laplace-Gauss forms
    the oracle's weights use: exp(-kappa r) = (kappa/sqrt(pi)) int t^-2
    exp(-kappa^2/(4 t^2)) exp(-r^2 t^2) dt and 1/r^3 = (4/sqrt(pi)) int t^2
    exp(-r^2 t^2) dt (Eq. LalpPoly at n = 3/2, Gamma(3/2) = sqrt(pi)/2)."""
    tt = np.linspace(1e-9, 60.0, 1200001)
    for kappa, r in ((0.8, 0.7), (1.5, 2.0)):
        k = kappa * kappa / 4.0
        printed = math.sqrt(k / math.pi) * np.trapezoid(tt ** -1.5 * np.exp(-k / tt - r * r * tt), tt)
        assert abs(printed - math.exp(-2.0 * math.sqrt(k) * r)) < 1e-9
        gauss = (kappa / math.sqrt(math.pi)) * np.trapezoid(tt ** -2 * np.exp(-kappa ** 2 / (4 * tt ** 2) - (r * tt) ** 2), tt)
        assert abs(gauss - math.exp(-kappa * r)) < 1e-12
    for r in (0.6, 1.3, 3.0):
        dip = (4.0 / math.sqrt(math.pi)) * np.trapezoid(tt ** 2 * np.exp(-(r * tt) ** 2), tt)
        assert abs(dip * r ** 3 - 1.0) < 1e-12


@pytest.mark.parametrize("kernel,kappa", [(O.SLATER, 0.8), (O.SLATER, 2.0), (O.DIPOLE, 0.0)])
def test_fine_sinc_rule_reproduces_slater_and_dipole(kernel, kappa):
    """A fine rule reproduces exp(-kappa r) and 1/r^3 to ~machine precision
    relative to the kernel: a wrong power of t or prefactor leaves an O(1)
    error."""
    t, w = O.sinc_quadrature(400, 0.05, 10.0, kappa, kernel)
    assert t[0] > 0.0 and np.all(w >= 0.0)
    r = np.geomspace(0.05, 20.0, 2000)
    approx = np.exp(-np.outer(r * r, t * t)) @ w
    assert np.max(np.abs(approx / O.kernel_value(r, kappa, kernel) - 1.0)) < 1e-12
    assert np.max(O.quadrature_rel_error(t, w, r, kappa, kernel)) < 1e-12
    with pytest.raises(ValueError):
        O.sinc_quadrature(20, 0.3, 10.0, 0.0 if kernel == O.SLATER else 0.5, kernel)


@pytest.mark.parametrize("kernel,kappa", [(O.SLATER, 0.7), (O.DIPOLE, 0.0)])
def test_slater_and_dipole_lattices_against_brute_force(kernel, kappa):
    """Defected lattices with the Slater and dipole kernels: canonical tensor
    values at sampled grid points vs the direct sum of Z p(d), within
    tau * sum |Z| m(d) (m: the scale the rule's error tau is measured against,
    1 for Slater and 1/d^3 for the dipole)."""
    wl = W.small_case(L=(4, 3, 3), N=60, R=20, frac_vac=0.2, frac_imp=0.1, kappa=kappa, kernel=kernel)
    rmax = O.default_r_max(wl)
    s, _ = O.fit_t_scale(wl.R, wl.sinc_step, wl.r_min, rmax, kappa=kappa, kernel=kernel)
    t, w = O.sinc_quadrature(wl.R, wl.sinc_step, s, kappa, kernel)
    g = O.generating_vectors(wl.N, wl.box_lo, wl.box_hi, t, w)
    cols, tcol, xi = O.canonical_terms(wl.N, wl.box_lo, wl.box_hi, g, wl.blocks, wl.defects)
    xs = O.cell_centres(wl.N, wl.box_lo, wl.box_hi)
    rng = np.random.default_rng(6)
    idx = rng.integers(0, wl.N, size=(20000, 3))
    centres, charges = O.charged_centres(wl.N, wl.box_lo, wl.box_hi, wl.blocks, wl.defects)
    bf, absbf, dmin, _ = O.brute_force(xs[idx], centres, charges, kappa=kappa, kernel=kernel)
    keep = dmin >= wl.r_min
    if kernel == O.SLATER:
        scale = np.full(int(keep.sum()), np.abs(charges).sum())
    else:
        scale = absbf[keep]
    tens = (xi[:, None] * cols[0][tcol[:, 0]][:, idx[keep, 0]] * cols[1][tcol[:, 1]][:, idx[keep, 1]]
            * cols[2][tcol[:, 2]][:, idx[keep, 2]]).sum(0)
    tau = float(np.max(O.quadrature_rel_error(t, w, np.geomspace(wl.r_min, rmax, 6000), kappa, kernel)))
    err = np.abs(tens - bf[keep])
    assert np.all(err <= tau * scale * 1.001 + 1e-13)
    assert np.max(err / np.abs(bf[keep]).max()) < 1e-4


# --- (a0) Galerkin reference vectors: Eq. galten ----------------------------

def test_galerkin_cell_average_matches_composite_rule():
    """Cell averages of exp(-t^2 x^2) against a 400-panel composite
    Gauss-Legendre rule, over t from 0 to 300 (both of the oracle's branches)
    and cells on both sides of 0."""
    xg, wg = np.polynomial.legendre.leggauss(16)

    def composite(t, a, b, n=400):
        e = np.linspace(a, b, n + 1)
        m, hh = 0.5 * (e[1:] + e[:-1]), 0.5 * (e[1:] - e[:-1])
        return float(np.sum(wg[None, :] * np.exp(-(t * (m[:, None] + hh[:, None] * xg[None, :])) ** 2)
                            * hh[:, None])) / (b - a)
    for t in (0.0, 1e-4, 0.02, 0.5, 3.0, 30.0, 300.0):
        for a, b in ((-0.3, -0.2), (0.0, 0.1), (0.2, 0.3), (2.0, 2.1), (-5.1, -5.0), (-0.1, 0.0)):
            ref = composite(t, a, b)
            v = O.gaussian_cell_average(t, a, b)
            assert abs(v - ref) <= 1e-13 * abs(ref) + 1e-300, (t, a, b, v, ref)


def test_galerkin_vectors_telescope_and_approach_collocation():
    """h sum_j p_q[j] over the doubled grid is w_q^(1/3) int_-b^b exp(-t^2 x^2)
    dx = w_q^(1/3) sqrt(pi)/t erf(t b) (b = N h); and on a fine grid the cell
    average differs from the collocated value by the midpoint-rule term
    (h^2/24) d^2/dx^2 exp(-t^2 x^2), which a cell shifted by any fraction of h
    would turn into an O(h) difference."""
    N, lo, hi = 40, -3.0, 3.0
    h = (hi - lo) / N
    t, w = O.sinc_quadrature(12, 0.3, 8.0)
    g = O.generating_vectors(N, lo, hi, t, w, galerkin=True)
    for q in range(len(t)):
        exact = 2 * N * h if t[q] == 0.0 else math.sqrt(math.pi) / t[q] * math.erf(t[q] * N * h)
        assert abs(h * g[q].sum() - np.cbrt(w[q]) * exact) <= 1e-13 * np.cbrt(w[q]) * exact
    N2 = 4000
    h2 = (hi - lo) / N2
    tq = np.array([0.7, 1.3])
    wq = np.ones(2)
    gg = O.generating_vectors(N2, lo, hi, tq, wq, galerkin=True)
    gc = O.generating_vectors(N2, lo, hi, tq, wq)
    x = (np.arange(2 * N2) - N2 + 0.5) * h2
    for q in range(2):
        f2 = (4 * tq[q] ** 4 * x * x - 2 * tq[q] ** 2) * np.exp(-(tq[q] * x) ** 2)
        sel = np.abs(f2) > 1e-3
        ratio = (gg[q] - gc[q])[sel] / (h2 * h2 / 24 * f2[sel])
        assert np.all(np.abs(ratio - 1.0) < 1e-3)


# --- generating vectors and windows: Eqs. master_pot, sub_tens -------------

def test_reference_tensor_reproduces_kernel():
    """sum_q prod_l p_q[j_l] = sum_q w_q exp(-t_q^2 |x|^2) ~ 1/|x| on the
    doubled grid (Eq. sinc_general): pins the cube root of the weights and
    the doubled-grid coordinates."""
    wl = W.small_case()
    s, t, w, g, *_ = _terms(wl)
    N = wl.N
    h = O.mesh_size(N, wl.box_lo, wl.box_hi)
    rng = np.random.default_rng(0)
    j = rng.integers(0, 2 * N, size=(4000, 3))
    x = (j - N + 0.5) * h
    r = np.sqrt((x * x).sum(1))
    keep = (r >= wl.r_min) & (r <= O.default_r_max(wl))
    val = (g[:, j[keep, 0]] * g[:, j[keep, 1]] * g[:, j[keep, 2]]).sum(0)
    tau = float(np.max(O.quadrature_rel_error(t, w, np.geomspace(wl.r_min, O.default_r_max(wl), 4000))))
    assert np.max(np.abs(val * r[keep] - 1.0)) <= 1.05 * tau
    # the reference vectors are symmetric about the centre of the doubled box
    assert np.array_equal(g, g[:, ::-1])


def test_window_centre_at_origin_is_index_set_I0():
    """A centre at the box centre (vertex N/2) restricts the reference vector
    to the middle N entries (index set I_0 of Sec. 3.1)."""
    N = 16
    g = np.arange(2 * N, dtype=float)[None, :]
    assert np.array_equal(O.window(g[0], N // 2, N), np.arange(N // 2, N // 2 + N, dtype=float))


def test_shifted_window_is_potential_of_shifted_centre():
    """sum_q prod_l (W_m g_q)[i_l] ~ 1/|x_i - a_m| for a centre at an
    off-centre vertex (brute force): an off-by-one in the window index gives
    an error of order h/r, far above the quadrature tolerance."""
    wl = W.small_case()
    s, t, w, g, *_ = _terms(wl)
    N = wl.N
    h = O.mesh_size(N, wl.box_lo, wl.box_hi)
    m = (7, 30, 41)
    a = np.array([wl.box_lo + mm * h for mm in m])
    win = [np.array([O.window(g[q], m[l], N) for q in range(wl.R)]) for l in range(3)]
    xs = O.cell_centres(N, wl.box_lo, wl.box_hi)
    rng = np.random.default_rng(1)
    idx = rng.integers(0, N, size=(3000, 3))
    pts = xs[idx]
    r = np.sqrt(((pts - a) ** 2).sum(1))
    keep = r >= wl.r_min
    val = (win[0][:, idx[keep, 0]] * win[1][:, idx[keep, 1]] * win[2][:, idx[keep, 2]]).sum(0)
    tau = float(np.max(O.quadrature_rel_error(t, w, np.geomspace(wl.r_min, O.default_r_max(wl), 4000))))
    assert np.max(np.abs(val * r[keep] - 1.0)) <= 1.05 * tau


def test_snap_is_nearest_vertex():
    N, lo, hi = 256, -6.0, 6.0
    h = (hi - lo) / N
    for pos in (-1.5, -0.5, 0.5, 1.5, 5.99, -6.0):
        m = O.snap(pos, N, lo, hi)
        assert abs(lo + m * h - pos) <= 0.5 * h + 1e-12
    assert [O.snap(p, N, lo, hi) for p in (-1.5, -0.5, 0.5, 1.5)] == [96, 117, 139, 160]
    with pytest.raises(ValueError):
        O.snap(6.2, N, lo, hi)


# --- (a) Thm 3.1(A): assembled sum == full site-by-site sum -----------------

def test_assembled_sum_equals_sitewise_full_tensor():
    """Thm 3.1(A) and rule (conc2sum): the rank-R tensor of 1D-assembled
    vectors equals the sum over all L^3 shifted reference tensors, to
    roundoff."""
    wl = W.small_case(L=(3, 2, 4))
    s, t, w, g, cols, tcol, xi = _terms(wl)
    assert len(xi) == wl.R           # defect-free lattice: rank R (Thm 3.1)
    full = O.full_tensor_sitewise(wl.N, wl.box_lo, wl.box_hi, g, wl.blocks, wl.defects)
    tens = O.full_from_canonical(cols, tcol, xi)
    assert np.linalg.norm(tens - full) <= 1e-13 * np.linalg.norm(full)


def test_single_site_lattice_is_the_reference_window():
    """Special case L = 1: the assembled vector is the window itself."""
    wl = W.small_case(L=(1, 1, 1))
    s, t, w, g, cols, tcol, xi = _terms(wl)
    m = O.snap(wl.blocks[0].origin[0], wl.N, wl.box_lo, wl.box_hi)
    for q in range(wl.R):
        assert np.array_equal(cols[0][q], O.window(g[q], m, wl.N))


def test_config1_against_brute_force():
    """4x4x4 lattice (N=256): tensor values at sampled grid points vs the
    direct sum of 1/|x - a| over the snapped centres, with the rigorous bound
    |err| <= tau * sum_s |Z_s| / |x - a_s| (each term carries the relative
    quadrature error tau, Eq. sinc_conv)."""
    wl = W.config1()
    s, t, w, g, cols, tcol, xi = _terms(wl)
    xs = O.cell_centres(wl.N, wl.box_lo, wl.box_hi)
    rng = np.random.default_rng(2)
    idx = rng.integers(0, wl.N, size=(20000, 3))
    centres, charges = O.charged_centres(wl.N, wl.box_lo, wl.box_hi, wl.blocks, wl.defects)
    bf, absbf, dmin, dmax = O.brute_force(xs[idx], centres, charges)
    keep = dmin >= wl.r_min
    tens = (xi[:, None] * cols[0][tcol[:, 0]][:, idx[keep, 0]] * cols[1][tcol[:, 1]][:, idx[keep, 1]]
            * cols[2][tcol[:, 2]][:, idx[keep, 2]]).sum(0)
    tau = float(np.max(O.quadrature_rel_error(t, w, np.geomspace(wl.r_min, O.default_r_max(wl), 6000))))
    err = np.abs(tens - bf[keep])
    assert np.all(err <= tau * absbf[keep] * 1.001 + 1e-13)
    assert np.max(err / np.abs(bf[keep])) < 1e-7


# --- (b) defects and sub-lattices: Sec. 4.1, 4.4 ----------------------------

def _canon_full(wl, blocks=None, defects=None, s=None):
    blocks = wl.blocks if blocks is None else blocks
    defects = wl.defects if defects is None else defects
    t, w = O.sinc_quadrature(wl.R, wl.sinc_step, s)
    g = O.generating_vectors(wl.N, wl.box_lo, wl.box_hi, t, w)
    cols, tcol, xi = O.canonical_terms(wl.N, wl.box_lo, wl.box_hi, g, blocks, defects)
    return O.full_from_canonical(cols, tcol, xi), (cols, tcol, xi), g


def test_vacating_every_site_gives_zero():
    wl = W.small_case(L=(3, 2, 2))
    s = 8.0
    base, *_ = _canon_full(wl, s=s, defects=[])
    b = wl.blocks[0]
    vac = [W.Defect(W.DEFECT_SITES, 0, (i, j, k)) for i in range(b.L[0])
           for j in range(b.L[1]) for k in range(b.L[2])]
    full, *_ = _canon_full(wl, defects=vac, s=s)
    assert np.linalg.norm(full) <= 1e-13 * np.linalg.norm(base)
    # one 3x2x2 "cluster" vacancy does the same with a single rank-R term
    full2, (cols, tcol, xi), _ = _canon_full(wl, defects=[W.Defect(W.DEFECT_SITES, 0, (0, 0, 0), b.L)], s=s)
    assert len(xi) == 2 * wl.R
    assert np.linalg.norm(full2) <= 1e-13 * np.linalg.norm(base)


def test_block_split_is_the_same_tensor():
    """Class (A) of Sec. 4.4: a 4x3x2 block equals the union of a 2x3x2 and a
    2x3x2 block."""
    L = (4, 3, 2)
    wl = W.small_case(L=L)
    s = 8.0
    whole, *_ = _canon_full(wl, s=s)
    halves = [W.centred_block((2, 3, 2), L, (0, 0, 0)), W.centred_block((2, 3, 2), L, (2, 0, 0))]
    split, (cols, tcol, xi), _ = _canon_full(wl, blocks=halves, s=s)
    assert len(xi) == 2 * wl.R
    assert np.linalg.norm(split - whole) <= 1e-13 * np.linalg.norm(whole)


def test_remove_and_readd_is_identity():
    wl = W.small_case(L=(3, 2, 2))
    s = 8.0
    base, *_ = _canon_full(wl, s=s, defects=[])
    b = wl.blocks[0]
    site = (1, 1, 0)
    pos = tuple(b.origin[a] + site[a] * b.spacing[a] for a in range(3))
    d = [W.Defect(W.DEFECT_SITES, 0, site), W.Defect(W.DEFECT_POINT, pos=pos, charge=1.0)]
    full, *_ = _canon_full(wl, defects=d, s=s)
    assert np.linalg.norm(full - base) <= 1e-13 * np.linalg.norm(base)


def test_impurity_replaces_charge():
    """An impurity of charge Z' at a site equals the lattice plus (Z'-1) times
    that site's reference tensor (reading: the charge is replaced)."""
    wl = W.small_case(L=(2, 2, 2))
    s = 8.0
    base, _, g = _canon_full(wl, s=s, defects=[])
    d = [W.Defect(W.DEFECT_SITES, 0, (1, 0, 1), charge=1.7)]
    full, *_ = _canon_full(wl, defects=d, s=s)
    b = wl.blocks[0]
    m = [O.snap(b.origin[a] + (1, 0, 1)[a] * b.spacing[a], wl.N, wl.box_lo, wl.box_hi) for a in range(3)]
    one = sum(np.einsum("i,j,k->ijk", O.window(g[q], m[0], wl.N), O.window(g[q], m[1], wl.N),
                        O.window(g[q], m[2], wl.N)) for q in range(wl.R))
    assert np.linalg.norm(full - base - 0.7 * one) <= 1e-13 * np.linalg.norm(base)


def test_defected_lattice_sitewise_identity():
    """Defected lattice (vacancies + impurities): the canonical terms equal the
    site-by-site sum with the modified charges (Eq. Can_LatticeSum_full)."""
    wl = W.small_case(L=(3, 3, 2), frac_vac=0.2, frac_imp=0.1)
    s, t, w, g, cols, tcol, xi = _terms(wl)
    full = O.full_tensor_sitewise(wl.N, wl.box_lo, wl.box_hi, g, wl.blocks, wl.defects)
    tens = O.full_from_canonical(cols, tcol, xi)
    assert len(xi) == wl.R * (1 + len(wl.defects))
    assert np.linalg.norm(tens - full) <= 1e-13 * np.linalg.norm(full)


def test_regular_vacancy_sublattice_has_rank_2R():
    """Sec. 4.4 (Fig. 4.5): vacancies on a regular tensor sub-lattice keep the
    canonical rank at 2R -- the sub-lattice is one negative block. The 6x6x1
    block of a 12x12x1 lattice (every second site) as 36 single vacancies
    and as one block of charge -1 with spacing 2 give the same tensor."""
    L = (12, 12, 1)
    lo, hi = W.box_for(L)
    wl = W.Workload("sub", 64, lo, hi, 16, 0.3, 1e-8, [W.centred_block(L)], [], r_min=0.5)
    s = 8.0
    vac = [W.Defect(W.DEFECT_SITES, 0, (2 * i, 2 * j, 0)) for i in range(6) for j in range(6)]
    full_vac, (c1, t1, x1), _ = _canon_full(wl, defects=vac, s=s)
    b = wl.blocks[0]
    sub = W.Block((6, 6, 1), b.origin, (2.0, 2.0, 1.0), -1.0)
    full_blk, (c2, t2, x2), _ = _canon_full(wl, blocks=[b, sub], defects=[], s=s)
    assert len(x2) == 2 * wl.R
    assert np.linalg.norm(full_vac - full_blk) <= 1e-13 * np.linalg.norm(full_blk)


# --- (b) non-rectangular lattices, Sec. 4.4 classes (B) and (C) -----------

def _skewed_sites(L, a1, a2, a3, origin):
    return np.array([[origin[d] + i * (a1 if d == 0 else 0.0) + j * a2[d] + k * a3[d] for d in range(3)]
                     for k in range(L[2]) for j in range(L[1]) for i in range(L[0])])


@pytest.mark.parametrize("cls", ["B", "C"])
def test_skewed_lattice_against_brute_force(cls):
    """A parallelogram lattice (class B) and a lattice skewed in two
    directions (class C), summed as unions of rectangular blocks: canonical
    tensor values at sampled grid points vs the direct sum of 1/|x - a| over
    the sites generated from the lattice vectors themselves, within tau sum
    |Z|/d; and the directional ranks the paper states: distinct x-vectors grow
    like L[1] (B) or L[1] L[2] (C), while class B has only R distinct z-vectors."""
    L = (5, 4, 3)
    a2 = (0.5, 1.0, 0.0)
    a3 = (0.0, 0.0, 1.0) if cls == "B" else (0.3, 0.25, 1.0)
    origin = (-3.2, -2.1, -1.05)
    blocks = W.skewed_lattice_blocks(L, 1.0, a2, a3, origin)
    assert len(blocks) == (L[1] if cls == "B" else L[1] * L[2])
    lo, hi = -8.0, 8.0
    wl = W.Workload("skew" + cls, 64, lo, hi, 16, 0.3, 1e-8, blocks, [], r_min=0.5)
    s, t, w, g, cols, tcol, xi = _terms(wl)
    sites = _skewed_sites(L, 1.0, a2, a3, origin)
    N, h = wl.N, O.mesh_size(wl.N, lo, hi)
    centres = np.array([[lo + h * O.snap(p[d], N, lo, hi) for d in range(3)] for p in sites])
    uniq, counts = np.unique(centres, axis=0, return_counts=True)
    xs = O.cell_centres(N, lo, hi)
    rng = np.random.default_rng(8)
    idx = rng.integers(0, N, size=(20000, 3))
    bf, absbf, dmin, _ = O.brute_force(xs[idx], uniq, counts.astype(np.float64))
    keep = dmin >= wl.r_min
    tens = (xi[:, None] * cols[0][tcol[:, 0]][:, idx[keep, 0]] * cols[1][tcol[:, 1]][:, idx[keep, 1]]
            * cols[2][tcol[:, 2]][:, idx[keep, 2]]).sum(0)
    tau = float(np.max(O.quadrature_rel_error(t, w, np.geomspace(wl.r_min, O.default_r_max(wl), 6000))))
    assert np.all(np.abs(tens - bf[keep]) <= tau * absbf[keep] * 1.001 + 1e-13)
    nblk = len(blocks)
    assert cols[0].shape[0] == wl.R * nblk
    if cls == "B":
        # every block sums the same z-windows: R distinct z-vectors (stored per block)
        assert np.unique(cols[2], axis=0).shape[0] == wl.R


# --- (c) RHOSVD: Def. 4.1, Lemma 4.2, Thm A.1 -------------------------------

def test_truncation_rank_rule():
    sig = np.array([1.0, 1e-3, 1e-6, 1e-9])
    total = math.sqrt(np.sum(sig ** 2))
    assert O.truncation_rank(sig, 1e-2) == 1
    assert O.truncation_rank(sig, 1.5e-6 / total) == 2
    assert O.truncation_rank(sig, 0.5e-6 / total) == 3
    assert O.truncation_rank(sig, 1e-12) == 4


@pytest.fixture(scope="module")
def defected_small():
    wl = W.small_case(L=(3, 3, 2), frac_vac=0.2, frac_imp=0.1, eps=1e-6)
    s, t, w, g, cols, tcol, xi = _terms(wl)
    full = O.full_from_canonical(cols, tcol, xi)
    return wl, cols, tcol, xi, full


def test_rhosvd_dedup_equals_explicit_side_matrices(defected_small):
    """The weighted distinct-column SVD has the same singular values, ranks
    and result as the SVD of the explicit concatenated side matrix."""
    wl, cols, tcol, xi, full = defected_small
    a = O.rhosvd(cols, tcol, xi, 1e-6)
    ecols, etcol, exi = O.explicit_terms(cols, tcol, xi)
    b = O.rhosvd(ecols, etcol, exi, 1e-6)
    for l in range(3):
        n = len(a["sigma"][l])
        assert np.allclose(a["sigma"][l], b["sigma"][l][:n], rtol=0, atol=1e-12 * a["sigma"][l][0])
        assert np.all(b["sigma"][l][n:] <= 1e-12 * a["sigma"][l][0])
    assert a["r"] == b["r"]
    ta, tb = O.full_from_tucker(a["Z"], a["B"]), O.full_from_tucker(b["Z"], b["B"])
    assert np.linalg.norm(ta - tb) <= 1e-12 * np.linalg.norm(tb)


def test_rhosvd_singular_value_trace(defected_small):
    """With unit-length canonical vectors, sum_k sigma_k^2 = trace(A A^T) =
    number of terms, in every mode."""
    wl, cols, tcol, xi, full = defected_small
    res = O.rhosvd(cols, tcol, xi, 1e-6)
    for l in range(3):
        assert abs(np.sum(res["sigma"][l] ** 2) - len(xi)) <= 1e-10 * len(xi)


@pytest.mark.parametrize("eps", [1e-2, 1e-4, 1e-6, 1e-8])
def test_rhosvd_error_within_thm_A1d_bound(defected_small, eps):
    """Thm A.1(d): ||A - A0|| <= ||xi|| sum_l (sum_{k>r_l} sigma_{l,k}^2)^(1/2)
    on the full tensor; Z_l orthonormal."""
    wl, cols, tcol, xi, full = defected_small
    res = O.rhosvd(cols, tcol, xi, eps)
    approx = O.full_from_tucker(res["Z"], res["B"])
    err = np.linalg.norm(full - approx)
    assert err <= res["bound"] * (1 + 1e-9) + 1e-14 * np.linalg.norm(full)
    for Z in res["Z"]:
        assert np.max(np.abs(Z.T @ Z - np.eye(Z.shape[1]))) < 1e-13


def test_rhosvd_core_is_orthogonal_projection(defected_small):
    """Thm A.1(c): the RHOSVD tensor is the orthogonal projection
    A x1 Z1 Z1^T x2 Z2 Z2^T x3 Z3 Z3^T, computed here by explicit mode products
    on the full tensor (not through the canonical core)."""
    wl, cols, tcol, xi, full = defected_small
    res = O.rhosvd(cols, tcol, xi, 1e-4)
    P = [Z @ Z.T for Z in res["Z"]]
    proj = np.einsum("ia,abc->ibc", P[0], full)
    proj = np.einsum("jb,ibc->ijc", P[1], proj)
    proj = np.einsum("kc,ijc->ijk", P[2], proj)
    approx = O.full_from_tucker(res["Z"], res["B"])
    assert np.linalg.norm(proj - approx) <= 1e-12 * np.linalg.norm(full)
    # a transposed mode (core indices in the wrong order) would not match
    bad = np.einsum("abc,ib,ja,kc->ijk", res["B"], res["Z"][0], res["Z"][1], res["Z"][2]) \
        if res["r"][0] == res["r"][1] else None
    if bad is not None:
        assert np.linalg.norm(bad - proj) > 1e-6 * np.linalg.norm(full)


def test_rhosvd_tiny_eps_reproduces_tensor(defected_small):
    wl, cols, tcol, xi, full = defected_small
    res = O.rhosvd(cols, tcol, xi, 1e-15)
    approx = O.full_from_tucker(res["Z"], res["B"])
    assert np.linalg.norm(full - approx) <= 1e-12 * np.linalg.norm(full)


def test_defect_free_lattice_needs_at_most_rank_R():
    """Thm 3.1: a perfect lattice is an exact rank-R canonical tensor, so
    every side matrix has rank <= R and the RHOSVD is exact at r_l <= R."""
    wl = W.small_case(L=(3, 2, 2))
    s, t, w, g, cols, tcol, xi = _terms(wl)
    res = O.rhosvd(cols, tcol, xi, 1e-15)
    assert max(res["r"]) <= wl.R
    full = O.full_from_canonical(cols, tcol, xi)
    assert np.linalg.norm(full - O.full_from_tucker(res["Z"], res["B"])) <= 1e-12 * np.linalg.norm(full)


# --- ALS refinement after RHOSVD: Thm A.1(a)-(c) ------------------------------

def _hooi_full(T, Z0, sweeps):
    """HOOI on the explicit N^3 tensor by mode unfoldings: for mode l, the
    leading left singular vectors of the mode-l unfolding of T x_m Y_m^T x_n
    Y_n^T. Written on the full tensor, apart from the canonical route."""
    Z = [np.array(z) for z in Z0]
    norms = []
    for _ in range(sweeps):
        for l in range(3):
            Y = T
            for a in range(3):
                if a != l:
                    Y = np.moveaxis(np.tensordot(Y, Z[a], axes=([a], [0])), -1, a)
            U, _, _ = np.linalg.svd(np.moveaxis(Y, l, 0).reshape(T.shape[l], -1), full_matrices=False)
            Z[l] = U[:, :Z[l].shape[1]]
        core = np.einsum("ijk,ia,jb,kc->abc", T, Z[0], Z[1], Z[2])
        norms.append(float(np.linalg.norm(core)))
    return Z, norms


def test_als_matches_full_tensor_hooi_and_improves_on_rhosvd():
    """From the RHOSVD start, ALS on the canonical terms and HOOI on the
    explicit tensor give the same core norms sweep by sweep; the norms do not
    decrease (Thm A.1(a): ALS ascends the dual objective), the error
    ||A - A_r||^2 = ||A||^2 - ||mu||^2 holds against the explicit tensor, and
    the refined error is at most the RHOSVD error."""
    wl = W.small_case(L=(3, 2, 2), N=24, R=10, frac_vac=0.3, frac_imp=0.2, eps=1e-3)
    s, t, w, g, cols, tcol, xi = _terms(wl)
    res = O.rhosvd(cols, tcol, xi, wl.eps, ranks=(4, 3, 3))
    Z, core, hist = O.als_refine(cols, tcol, xi, res["Z"], sweeps=4)
    full = O.full_from_canonical(cols, tcol, xi)
    _, norms_full = _hooi_full(full, res["Z"], 4)
    assert np.allclose(hist[1:], norms_full, rtol=1e-10, atol=0)
    assert all(b >= a * (1 - 1e-13) for a, b in zip(hist, hist[1:]))
    for a in range(3):
        assert np.max(np.abs(Z[a].T @ Z[a] - np.eye(Z[a].shape[1]))) < 1e-12
    approx = np.einsum("abc,ia,jb,kc->ijk", core, Z[0], Z[1], Z[2])
    err2 = float(np.sum((full - approx) ** 2))
    assert abs(err2 - (np.sum(full ** 2) - hist[-1] ** 2)) <= 1e-9 * np.sum(full ** 2)
    rh = np.einsum("abc,ia,jb,kc->ijk", res["B"], res["Z"][0], res["Z"][1], res["Z"][2])
    assert err2 <= float(np.sum((full - rh) ** 2)) * (1 + 1e-12)
    assert hist[-1] > hist[0]


def test_als_fixed_point_at_exact_rank():
    """A defect-free lattice has exact Tucker rank <= R (Thm 3.1): with the
    RHOSVD bases of that rank the core already holds the whole norm, and ALS
    keeps it there."""
    wl = W.small_case(L=(3, 2, 2), N=24, R=8, eps=1e-12)
    s, t, w, g, cols, tcol, xi = _terms(wl)
    res = O.rhosvd(cols, tcol, xi, 1e-14)
    Z, core, hist = O.als_refine(cols, tcol, xi, res["Z"], sweeps=2)
    full = O.full_from_canonical(cols, tcol, xi)
    assert abs(hist[0] - np.linalg.norm(full)) <= 1e-12 * np.linalg.norm(full)
    assert abs(hist[-1] - hist[0]) <= 1e-12 * hist[0]


def test_als_refuses_a_start_rank_it_cannot_keep():
    """One ALS step takes r_l leading singular vectors of the N x (r_m r_n) matrix B_l
    (Thm A.1(b)); a start with r_l > r_m r_n cannot keep its rank, and the oracle says so
    instead of returning a basis with fewer columns."""
    wl = W.small_case(L=(3, 2, 2), N=24, R=10, frac_vac=0.3, frac_imp=0.2, eps=1e-3)
    s, t, w, g, cols, tcol, xi = _terms(wl)
    rng = np.random.default_rng(7)
    Z0 = [np.linalg.qr(rng.standard_normal((wl.N, k)))[0] for k in (5, 2, 2)]
    with pytest.raises(ValueError):
        O.als_refine(cols, tcol, xi, Z0, sweeps=1)
    Z0[0] = Z0[0][:, :4]   # r_0 = r_1 r_2 is allowed
    Z, core, hist = O.als_refine(cols, tcol, xi, Z0, sweeps=1)
    assert [z.shape[1] for z in Z] == [4, 2, 2]


# --- (d) slabs ---------------------------------------------------------------

def test_slab_evaluation_matches_full_tensors(defected_small):
    wl, cols, tcol, xi, full = defected_small
    res = O.rhosvd(cols, tcol, xi, 1e-6)
    approx = O.full_from_tucker(res["Z"], res["B"])
    for i3 in (0, 5, wl.N // 2, wl.N - 1):
        assert np.allclose(O.tucker_slab(res["Z"], res["B"], i3), approx[:, :, i3], rtol=0,
                           atol=1e-13 * np.abs(approx).max())
        assert np.allclose(O.canonical_slab(cols, tcol, xi, i3), full[:, :, i3], rtol=0,
                           atol=1e-13 * np.abs(full).max())


# --- printed values of the paper ---------------------------------------------

def test_paper_rank_claims_fixture():
    """Golden fixture of the paper's printed rank statements; the 2R claim of
    Sec. 4.4 is checked in test_regular_vacancy_sublattice_has_rank_2R, the
    rank-R claim of Thm 3.1 in test_assembled_sum_equals_sitewise_full_tensor."""
    with open(os.path.join(GOLDEN, "paper_claims.json")) as f:
        claims = json.load(f)
    assert claims["thm_3_1_rank_factor"] == 1
    assert claims["sec_4_4_sublattice_rank_factor_max"] == 2


# --- Tucker-reference variant: Thm 3.1(B), Sec. 4.1, Thm 4.3 ----------------

@pytest.fixture(scope="module")
def tucker_small():
    """A 4x3x3 lattice with vacancies, impurities, a 2x2x2 cluster and an off-lattice
    charge; reference Tucker tensor at eps_ref = 1e-7."""
    wl = W.small_case(L=(4, 3, 3), N=40, frac_vac=0.15, frac_imp=0.1, eps=1e-6)
    defects = list(wl.defects) + [W.Defect(W.DEFECT_SITES, 0, (1, 1, 0), (2, 2, 2), charge=1.3),
                                  W.Defect(W.DEFECT_POINT, pos=(0.37, -1.1, 0.5), charge=0.7)]
    s, t, w, g, cols, tcol, xi = _terms(wl)
    tt, b, sig = O.reference_tucker(g, 1e-7)
    terms = O.tucker_terms(wl.N, wl.box_lo, wl.box_hi, tt, b, wl.blocks, defects)
    return wl, defects, g, tt, b, sig, terms


def test_reference_tucker_within_thm_A1d_bound():
    """The reference Tucker tensor (RHOSVD of the reference canonical tensor on the
    doubled grid) is within the Thm A.1(d) bound of the canonical reference tensor,
    its vectors are orthonormal, and a tiny threshold reproduces it."""
    wl = W.small_case(L=(1, 1, 1), N=20, R=12, eps=1e-6)
    s, t, w, g, cols, tcol, xi = _terms(wl)
    P = np.einsum("qi,qj,qk->ijk", g, g, g)
    for eps_ref in (1e-3, 1e-6, 1e-10):
        tt, b, sig = O.reference_tucker(g, eps_ref)
        assert np.max(np.abs(tt @ tt.T - np.eye(tt.shape[0]))) < 1e-13
        T = np.einsum("abc,ai,bj,ck->ijk", b, tt, tt, tt)
        r = tt.shape[0]
        d = math.sqrt(float(np.sum(sig[r:] ** 2)))
        xi = np.sqrt((g * g).sum(1)) ** 3
        assert np.linalg.norm(P - T) <= np.linalg.norm(xi) * 3 * d * (1 + 1e-9) + 1e-14 * np.linalg.norm(P)
    tt, b, sig = O.reference_tucker(g, 1e-15)
    T = np.einsum("abc,ai,bj,ck->ijk", b, tt, tt, tt)
    assert np.linalg.norm(P - T) <= 1e-12 * np.linalg.norm(P)


def test_tucker_lattice_sum_sitewise_identity(tucker_small):
    """Thm 3.1(B) and Eq. (Tuck_LatticeSum_full): the assembled Tucker block terms plus
    the shifted reference Tucker defect terms equal the site-by-site sum of shifted
    reference Tucker tensors with the net charges (an exact identity)."""
    wl, defects, g, tt, b, sig, terms = tucker_small
    A = O.tucker_full(terms)
    S = O.reference_tucker_full(wl.N, wl.box_lo, wl.box_hi, tt, b, wl.blocks, defects)
    assert np.linalg.norm(A - S) <= 1e-13 * np.linalg.norm(S)


def test_tucker_lattice_sum_near_canonical_sum(tucker_small):
    """The Tucker lattice sum differs from the canonical one (the same lattice and
    defects) by at most the reference approximation error times the sum of |charges|."""
    wl, defects, g, tt, b, sig, terms = tucker_small
    cols, tcol, xi = O.canonical_terms(wl.N, wl.box_lo, wl.box_hi, g, wl.blocks, defects)
    C = O.full_from_canonical(cols, tcol, xi)
    A = O.tucker_full(terms)
    P = np.einsum("qi,qj,qk->ijk", g, g, g)
    Tref = np.einsum("abc,ai,bj,ck->ijk", b, tt, tt, tt)
    pos, z = O.charged_centres(wl.N, wl.box_lo, wl.box_hi, wl.blocks, defects)
    assert np.linalg.norm(A - C) <= np.sum(np.abs(z)) * np.linalg.norm(P - Tref) * (1 + 1e-9)


@pytest.mark.parametrize("eps", [1e-2, 1e-4, 1e-6, 1e-8])
def test_tucker_sum_within_thm43_bound(tucker_small, eps):
    """Thm 4.3(a): ||U_hat - U_r|| <= |B_hat| sum_l (sum_{k>r_l} sigma_{l,k}^2)^(1/2),
    on the full tensor; the bases orthonormal."""
    wl, defects, g, tt, b, sig, terms = tucker_small
    full = O.tucker_full(terms)
    res = O.tucker_sum_rhosvd(terms, eps)
    approx = O.full_from_tucker(res["Z"], res["B"])
    err = np.linalg.norm(full - approx)
    assert err <= res["bound"] * (1 + 1e-9) + 1e-14 * np.linalg.norm(full), (err, res["bound"])
    for Z in res["Z"]:
        assert np.max(np.abs(Z.T @ Z - np.eye(Z.shape[1]))) < 1e-13
    # the orthogonal projection of U_hat onto the bases, by explicit mode products
    P = [Z @ Z.T for Z in res["Z"]]
    proj = np.einsum("ia,jb,kc,abc->ijk", P[0], P[1], P[2], full, optimize=True)
    assert np.linalg.norm(proj - approx) <= 1e-12 * np.linalg.norm(full)


def test_tucker_sum_tiny_eps_reproduces(tucker_small):
    wl, defects, g, tt, b, sig, terms = tucker_small
    full = O.tucker_full(terms)
    res = O.tucker_sum_rhosvd(terms, 1e-15)
    assert np.linalg.norm(full - O.full_from_tucker(res["Z"], res["B"])) <= 1e-12 * np.linalg.norm(full)


def test_tucker_sum_of_rank_one_terms_is_the_canonical_rhosvd(defected_small):
    """Sec. 4.1: the RHOSVD of a canonical sum is the special case of the generalized
    scheme for rank-one Tucker tensors. Each canonical term as a Tucker term (side
    matrices the term's three vectors, core its charge): the same singular values,
    ranks, result and bound as ``rhosvd``."""
    wl, cols, tcol, xi, full = defected_small
    terms = [([cols[a][tcol[t, a]][:, None] for a in range(3)], np.array([[[xi[t]]]]), None)
             for t in range(len(xi))]
    for eps in (1e-3, 1e-6):
        a = O.tucker_sum_rhosvd(terms, eps)
        c = O.rhosvd(cols, tcol, xi, eps)
        assert a["r"] == c["r"]
        for l in range(3):
            n = len(c["sigma"][l])
            assert np.allclose(a["sigma"][l][:n], c["sigma"][l], rtol=0, atol=1e-12 * c["sigma"][l][0])
        ta, tc = O.full_from_tucker(a["Z"], a["B"]), O.full_from_tucker(c["Z"], c["B"])
        assert np.linalg.norm(ta - tc) <= 1e-12 * np.linalg.norm(tc)
        assert abs(a["bound"] - c["bound"]) <= 1e-10 * c["bound"]


def test_tucker_core_as_canonical_sum(tucker_small):
    """The core of Thm 4.3 written as a canonical sum: the reference core is
    b = sum_q h_q^(x3) with h_q = Z_ref^T g_q, so each term's projection
    sum_s B_s x_l (Z_l^T F_s) equals the canonical core (Thm A.1(c)) of the lattice
    sum whose reference vectors are the projected g'_q = Z_ref Z_ref^T g_q, with the
    same bases Z_l (the form the CUDA path contracts)."""
    wl, defects, g, tt, b, sig, terms = tucker_small
    res = O.tucker_sum_rhosvd(terms, 1e-6)
    gp = (tt.T @ (tt @ g.T)).T                     # rows g'_q
    cols, tcol, xi = O.canonical_terms(wl.N, wl.box_lo, wl.box_hi, gp, wl.blocks, defects)
    P = [res["Z"][a].T @ cols[a].T for a in range(3)]
    Bc = O.core_tensor(P, tcol, xi)
    assert np.linalg.norm(Bc - res["B"]) <= 1e-12 * np.linalg.norm(res["B"])
    # and |B_hat|^2 = ||b||^2 sum_s charge_s^2 prod_l |F_{s,l}|_F^2 with
    # ||b||^2 = sum_{q,q'} (h_q . h_q')^3, h_q = Z_ref^T g_q (the form the CUDA path uses)
    h = tt @ g.T
    b2 = float(np.sum((h.T @ h) ** 3))
    assert abs(b2 - float(np.sum(b * b))) <= 1e-12 * b2
    R = g.shape[0]
    bh2 = sum(xi[s_idx * R] ** 2 * b2 * np.prod([np.linalg.norm(F[a]) ** 2 for a in range(3)])
              for s_idx, (F, core, keys) in enumerate(terms))
    assert abs(math.sqrt(bh2) - res["Bhat"]) <= 1e-12 * res["Bhat"]


# --- Galerkin matrix of the Tucker potential, Eq. (nuc_pot) ----------------------

def _gaussian_basis(x, centres, alphas):
    return [np.exp(-alphas[:, None] * (x[None, :] - centres[:, l:l + 1]) ** 2) for l in range(3)]


def test_galerkin_matrix_equals_full_tensor_definition(defected_small):
    """The 1D Hadamard/scalar-product form equals the sum over the full grid of
    T g_k g_m, for a non-symmetric Tucker tensor (a defected lattice)."""
    wl, cols, tcol, xi, full = defected_small
    res = O.rhosvd(cols, tcol, xi, 1e-6)
    T = O.full_from_tucker(res["Z"], res["B"])
    x = O.cell_centres(wl.N, wl.box_lo, wl.box_hi)
    rng = np.random.default_rng(11)
    basis = _gaussian_basis(x, rng.uniform(-2.0, 2.0, (5, 3)), rng.uniform(0.3, 2.0, 5))
    V = O.galerkin_matrix(res["Z"], res["B"], basis)
    Vf = O.galerkin_matrix_full(T, basis)
    assert np.max(np.abs(V - Vf)) <= 1e-12 * np.max(np.abs(Vf))
    assert np.max(np.abs(V - V.T)) <= 1e-13 * np.max(np.abs(V))


def test_galerkin_matrix_of_constant_potential_is_overlap_product():
    """T = 1 everywhere (Z_l = ones / sqrt(N), core N^(3/2)): v_km is the product over
    the modes of the 1D overlaps sum_i g_k^l(i) g_m^l(i)."""
    N = 40
    x = np.linspace(-3.0, 3.0, N)
    rng = np.random.default_rng(5)
    basis = _gaussian_basis(x, rng.uniform(-1.0, 1.0, (4, 3)), rng.uniform(0.5, 3.0, 4))
    Z = [np.ones((N, 1)) / math.sqrt(N) for _ in range(3)]
    B = np.array([[[N ** 1.5]]])
    V = O.galerkin_matrix(Z, B, basis)
    S = [basis[l] @ basis[l].T for l in range(3)]
    assert np.max(np.abs(V - S[0] * S[1] * S[2])) <= 1e-12 * np.max(np.abs(V))


def test_galerkin_matrix_converges_to_gaussian_nuclear_attraction():
    """A single unit charge and s-type Gaussians exp(-alpha |x - A|^2): h^3 v_km tends to
    the closed-form nuclear attraction integral (2 pi / p) exp(-mu |A - B|^2)
    F0(p |P - C|^2), F0(t) = (1/2) sqrt(pi/t) erf(sqrt t) (p = alpha + beta,
    mu = alpha beta / p, P = (alpha A + beta B)/p), at second order in h: the midpoint
    rule on the collocated potential."""
    from scipy.special import erf
    errs = []
    for N in (64, 128):
        wl = W.small_case(L=(1, 1, 1), N=N, R=24, eps=1e-10, sinc_step=0.25)
        s, _ = O.fit_t_scale(wl.R, wl.sinc_step, 0.02, O.default_r_max(wl))
        s, t, w, g, cols, tcol, xi = _terms(wl, s)
        res = O.rhosvd(cols, tcol, xi, 1e-10)
        x = O.cell_centres(wl.N, wl.box_lo, wl.box_hi)
        h = x[1] - x[0]
        a = O.charged_centres(wl.N, wl.box_lo, wl.box_hi, wl.blocks, wl.defects)[0][0]
        rng = np.random.default_rng(0)
        alph = rng.uniform(0.8, 2.0, 4)
        cen = a + rng.uniform(-1.0, 1.0, (4, 3))
        V = O.galerkin_matrix(res["Z"], res["B"], _gaussian_basis(x, cen, alph)) * h ** 3
        A = np.zeros((4, 4))
        for k in range(4):
            for m in range(4):
                p = alph[k] + alph[m]
                mu = alph[k] * alph[m] / p
                P = (alph[k] * cen[k] + alph[m] * cen[m]) / p
                tt = p * float(np.sum((P - a) ** 2))
                F0 = 1.0 if tt < 1e-14 else 0.5 * math.sqrt(math.pi / tt) * erf(math.sqrt(tt))
                A[k, m] = 2.0 * math.pi / p * math.exp(-mu * float(np.sum((cen[k] - cen[m]) ** 2))) * F0
        errs.append(float(np.max(np.abs(V - A) / np.abs(A))))
    assert errs[1] < 2e-3, errs
    assert 3.5 < errs[0] / errs[1] < 4.5, errs
