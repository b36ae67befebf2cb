"""Plain FP64 CPU oracle for the assembled lattice sum with defects and RHOSVD.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import or call this
module: only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline leg use it. It shares no code with the CUDA library; the only common
ground is the seeded workload description (block sizes, defect lists), which
holds none of the method's arithmetic.

Every function below is written from the paper (Khoromskaia & Khoromskij,
"Tucker tensor method for fast grid-based summation of long-range potentials
on 3D lattices with defects", arXiv 1411.1994) and cites the passage it
follows. Where the paper is silent or garbled, the reading used is stated in
the docstring. The code is deliberately slow and literal: explicit loops over
lattice sites, LAPACK SVD (numpy.linalg.svd -> dgesdd) for the RHOSVD, and
matrix products only where the definition is a contraction.

Parity status: every function here is pinned by the CPU tests
(tests/test_oracle_pins.py) to closed forms, exact identities, brute-force
1/|x-a| (and exp(-kappa |x-a|)/|x-a|) sums or the paper's error bound --
except ``fit_t_scale``, whose optimality is not pinned (only the error it
reports is, by recomputation on a denser r-grid).

Kernels (Sec. 2.3, Eqs. LalpSlater, LalpYukawa, LalpNewt, LalpPoly), all as a
Laplace-Gauss integral p(r) = int_0^inf a(t) exp(-r^2 t^2) dt, so that they
share the sinc rule and differ only in the quadrature weights:
  YUKAWA (0): exp(-kappa r)/r, a = (2/sqrt(pi)) exp(-kappa^2/(4 t^2));
              kappa = 0 is the Newton kernel 1/r;
  SLATER (1): exp(-kappa r), a = (kappa/sqrt(pi)) t^-2 exp(-kappa^2/(4 t^2));
  DIPOLE (2): 1/r^3, a = (4/sqrt(pi)) t^2 (kappa = 0).
"""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple

import numpy as np

YUKAWA, SLATER, DIPOLE = 0, 1, 2   # kernel families (YUKAWA with kappa = 0: Newton)

SITES = 0   # a defect that replaces the charge of a box of lattice sites
POINT = 1   # a defect that adds a charge at an arbitrary position


# ---------------------------------------------------------------------------
# (a0) quadrature and generating vectors, Sec. 2.1
# ---------------------------------------------------------------------------

def sinc_quadrature(R: int, sinc_step: float, t_scale: float,
                    kappa: float = 0.0, kernel: int = YUKAWA) -> Tuple[np.ndarray, np.ndarray]:
    """Nodes t_q and weights w_q of the rank-R separable expansion of the
    kernel: 1/r for kappa = 0, exp(-kappa r)/r for kappa > 0.

    Sec. 2.1, Eqs. (laplace), (hM), (sinc_Newt): 1/r = (2/sqrt(pi)) int_0^inf
    exp(-r^2 t^2) dt, discretised by a sinc rule with nodes on a uniform
    u-grid. Reading (the printed rule t_k = k h_M does not converge over the
    needed range of r): substitute t = sinh(u)/s, whose integrand
    cosh(u)/s * exp(-r^2 sinh(u)^2 / s^2) is even in u, take the sinc rule
    u_k = k*h, k = -M..M, and merge the equal +k and -k terms. That leaves
    R = M + 1 distinct Gaussians, q = 0..R-1:
        t_q = sinh(q h) / s,
        w_0 = h / (s sqrt(pi)),  w_q = 2 h cosh(q h) / (s sqrt(pi))  (q >= 1).

    Yukawa (Sec. 2.3, Eq. LalpYukawa with rho = r^2): the Laplace-Gauss form
    exp(-kappa r)/r = (2/sqrt(pi)) int_0^inf exp(-kappa^2/(4 t^2)) exp(-r^2 t^2) dt.
    Reading: the printed exponent kappa^2/t^2 gives exp(-2 kappa r)/r; the
    factor 1/4 is the one for which the identity holds (a pinned test
    integrates both). The same sinc rule applies with each weight multiplied
    by exp(-kappa^2/(4 t_q^2)); that factor is 0 at t_0 = 0, so the R nodes
    are q = 1..R, each weight 2 h cosh(q h)/(s sqrt(pi)) exp(-kappa^2/(4 t_q^2)).

    Slater exp(-kappa r) (Eq. LalpSlater with its parameter kappa_S = kappa^2/4
    and rho = r^2, then t -> t^2): a(t) = (kappa/sqrt(pi)) t^-2
    exp(-kappa^2/(4 t^2)). Dipole 1/r^3 (Eq. LalpPoly extended to n = 3/2 with
    Gamma(3/2) = sqrt(pi)/2, then t -> t^2): a(t) = (4/sqrt(pi)) t^2. Both
    vanish at t = 0, so again q = 1..R, with w_q = 2 h cosh(q h)/s * a(t_q) / 2
    (the merged +q and -q terms of the rule for (1/2) int_R a(t(u)) t'(u) du).
    """
    if kappa < 0.0:
        raise ValueError("kappa must be >= 0")
    if kernel in (SLATER, DIPOLE):
        if (kernel == SLATER) != (kappa > 0.0):
            raise ValueError("the Slater kernel needs kappa > 0, the dipole kernel kappa = 0")
        q = np.arange(R, dtype=np.float64) + 1.0
        u = q * sinc_step
        t = np.sinh(u) / t_scale
        if kernel == SLATER:
            a = (kappa / math.sqrt(math.pi)) / (t * t) * np.exp(-(kappa * kappa) / (4.0 * t * t))
        else:
            a = (4.0 / math.sqrt(math.pi)) * t * t
        w = sinc_step * np.cosh(u) / t_scale * a
        return t, w
    q = np.arange(R, dtype=np.float64) + (1.0 if kappa > 0.0 else 0.0)
    u = q * sinc_step
    t = np.sinh(u) / t_scale
    w = 2.0 * sinc_step * np.cosh(u) / (t_scale * math.sqrt(math.pi))
    if kappa > 0.0:
        w = w * np.exp(-(kappa * kappa) / (4.0 * t * t))
    else:
        w[0] = sinc_step / (t_scale * math.sqrt(math.pi))
    return t, w


def kernel_value(r, kappa: float = 0.0, kernel: int = YUKAWA):
    """The kernel p(r): exp(-kappa r)/r (1/r at kappa = 0), exp(-kappa r), or 1/r^3
    (Sec. 2.3)."""
    r = np.asarray(r, dtype=np.float64)
    if kernel == SLATER:
        return np.exp(-kappa * r)
    if kernel == DIPOLE:
        return 1.0 / (r * r * r)
    return np.exp(-kappa * r) / r


def quadrature_rel_error(t: np.ndarray, w: np.ndarray, r: np.ndarray, kappa: float = 0.0,
                         kernel: int = YUKAWA) -> np.ndarray:
    """r |sum_q w_q exp(-t_q^2 r^2) - p(r)|: the error of the separable
    expansion of the kernel p at distances r, relative to 1/r (Sec. 2.1, Eq.
    sinc_conv bounds the absolute error by C/a e^(-beta sqrt(M)) for r >= a).
    For the Newton kernel this is the relative error |r sum - 1|. For the
    Yukawa kernel it is the error relative to the unscreened 1/r: the relative
    error of exp(-kappa r)/r itself, many decades down at large kappa r, is
    neither reachable with a few terms nor felt in a lattice sum. Slater: the
    absolute error (the kernel is 1 at r = 0); dipole: the relative error
    |r^3 sum - 1|."""
    r = np.asarray(r, dtype=np.float64)
    s = np.exp(-np.outer(r * r, t * t)) @ w
    if kernel == SLATER:
        return np.abs(s - np.exp(-kappa * r))
    if kernel == DIPOLE:
        return np.abs(r * r * r * s - 1.0)
    return np.abs(r * s - np.exp(-kappa * r))


def fit_t_scale(R: int, sinc_step: float, r_min: float, r_max: float,
                n_r: int = 600, kappa: float = 0.0, kernel: int = YUKAWA) -> Tuple[float, float]:
    """Scale s of the substitution t = sinh(u)/s that minimises the maximum
    relative error of the expansion over [r_min, r_max] (Sec. 2.1: M, and here
    s, are chosen so that the kernel is reproduced to a tolerance; the paper's
    C_0 plays the role of s). Coarse log-scan then golden-section refinement.
    For kappa > 0, s is at most sinh(h) sqrt(2400)/kappa, so that no weight's
    screening factor exp(-kappa^2/(4 t_q^2)) falls below e^-600.
    Returns (s, max relative error on the fitting grid)."""
    r = np.geomspace(r_min, r_max, n_r)

    def err(log_s):
        t, w = sinc_quadrature(R, sinc_step, math.exp(log_s), kappa, kernel)
        return float(np.max(quadrature_rel_error(t, w, r, kappa, kernel)))

    hi = math.log(1e5)
    if kappa > 0.0:
        # keep the first node's screening factor representable: kappa^2/(4 t_1^2) <= 600
        hi = min(hi, math.log(math.sinh(sinc_step) * math.sqrt(2400.0) / kappa))
    grid = np.linspace(math.log(1e-2), hi, 241)
    vals = [err(x) for x in grid]
    i = int(np.argmin(vals))
    a, b = grid[max(i - 1, 0)], grid[min(i + 1, len(grid) - 1)]
    gr = (math.sqrt(5.0) - 1.0) / 2.0
    c, d = b - gr * (b - a), a + gr * (b - a)
    fc, fd = err(c), err(d)
    for _ in range(60):
        if fc < fd:
            b, d, fd = d, c, fc
            c = b - gr * (b - a)
            fc = err(c)
        else:
            a, c, fc = c, d, fd
            d = a + gr * (b - a)
            fd = err(d)
    x = 0.5 * (a + b)
    return math.exp(x), err(x)


def mesh_size(N: int, box_lo: float, box_hi: float) -> float:
    """h = b/n for the uniform grid on the box (Sec. 2.1)."""
    return (box_hi - box_lo) / N


def cell_centres(N: int, box_lo: float, box_hi: float) -> np.ndarray:
    """Collocation points x_i = box_lo + (i + 1/2) h, i = 0..N-1 (reading:
    cell-centred collocation instead of the Galerkin integral of Eq. galten)."""
    h = mesh_size(N, box_lo, box_hi)
    return box_lo + (np.arange(N, dtype=np.float64) + 0.5) * h


def snap(pos: float, N: int, box_lo: float, box_hi: float) -> int:
    """Vertex index m of the grid vertex nearest to ``pos`` (vertex m sits at
    box_lo + m h). Sec. 3.1 places each centre on a grid point and allows
    off-grid centres with O(h) error (footnote to Eq. sub_tens); reading: snap
    to the nearest vertex, so that no collocation point coincides with a
    centre."""
    h = mesh_size(N, box_lo, box_hi)
    m = math.floor((pos - box_lo) / h + 0.5)
    if m < 0 or m > N:
        raise ValueError(f"centre {pos} outside the box")
    return int(m)


_GL_X, _GL_W = np.polynomial.legendre.leggauss(24)


def gaussian_cell_average(t: float, a: float, b: float) -> float:
    """(1/(b - a)) int_a^b exp(-t^2 x^2) dx. Where t (b - a) <= 10 the integrand
    is smooth on the cell on the scale of its width and a 24-point
    Gauss-Legendre rule gives it to rounding (degree 47, error of order
    (t (b - a)/2)^48 / 48!). Wider cells (a narrow Gaussian) never straddle 0
    (cell ends are multiples of h), so the error-function form (sqrt(pi) /
    (2 t (b - a))) (erfc(t a) - erfc(t b)) (mirrored for a cell below 0) has
    no cancellation there: erfc(t a) exceeds erfc(t b) by a factor of at
    least e^100."""
    if t == 0.0:
        return 1.0
    if t * (b - a) <= 10.0:
        mid, half = 0.5 * (a + b), 0.5 * (b - a)
        x = mid + half * _GL_X
        return 0.5 * float(np.sum(_GL_W * np.exp(-(t * x) ** 2)))
    if a >= 0.0:
        d = math.erfc(t * a) - math.erfc(t * b)
    else:
        d = math.erfc(-t * b) - math.erfc(-t * a)
    return math.sqrt(math.pi) / (2.0 * t * (b - a)) * d


def generating_vectors(N: int, box_lo: float, box_hi: float,
                       t: np.ndarray, w: np.ndarray, galerkin: bool = False) -> np.ndarray:
    """Canonical vectors of the reference tensor on the doubled grid,
    Eq. (master_pot): p_q[j] = w_q^(1/3) exp(-t_q^2 xt_j^2) on the 2N cell
    centres xt_j = (j - N + 1/2) h of [-b, b] (collocation reading). The same
    vectors serve all three modes (Eq. sinc_general). Shape (R, 2N).

    galerkin: Eq. (galten) with piecewise-constant basis functions, each entry
    the integral of the Gaussian over its cell [(j - N) h, (j - N + 1) h].
    Reading: divided by the cell width, i.e. cell averages, so that the tensor
    holds cell averages of the kernel (Eq. galten divided by h^3) on the same
    scale as the collocated values."""
    h = mesh_size(N, box_lo, box_hi)
    if galerkin:
        g = np.empty((len(t), 2 * N))
        for q in range(len(t)):
            c = np.cbrt(w[q])
            for j in range(2 * N):
                g[q, j] = c * gaussian_cell_average(float(t[q]), (j - N) * h, (j - N + 1) * h)
        return g
    xt = (np.arange(2 * N, dtype=np.float64) - N + 0.5) * h
    return np.cbrt(w)[:, None] * np.exp(-np.outer(t * t, xt * xt))


def window(gq: np.ndarray, m: int, N: int) -> np.ndarray:
    """Shift-and-window operator W_m of Eq. (sub_tens) applied to one doubled-
    grid vector: the restriction to the box of the reference vector centred on
    vertex m, (W_m g)[i] = g[i - m + N], i = 0..N-1. (The printed index range
    i+n/2 : i+3n/2 has n+1 entries; this is the reading for a centre at a
    vertex and cell-centred collocation.)"""
    return gq[N - m: 2 * N - m].copy()


# ---------------------------------------------------------------------------
# (a) assembled lattice sum, Thm 3.1(A); (b) defects, Sec. 4.1 and 4.4
# ---------------------------------------------------------------------------

def block_vertex_indices(block, N: int, box_lo: float, box_hi: float) -> List[List[int]]:
    """Per mode, the vertex index of every lattice site of a rectangular block
    (site k at origin + k * spacing, snapped)."""
    out = []
    for a in range(3):
        out.append([snap(block.origin[a] + k * block.spacing[a], N, box_lo, box_hi)
                    for k in range(block.L[a])])
    return out


def assembled_vector(gq: np.ndarray, ms: Sequence[int], N: int) -> np.ndarray:
    """sum_k W_{m_k} g_q, one 1D sum per mode and rank index (Thm 3.1(A),
    Eq. EwaldTensorGl), by an explicit loop over the sites."""
    v = np.zeros(N)
    for m in ms:
        v += window(gq, m, N)
    return v


def defect_charge(defect, blocks) -> float:
    """Weight xi of a defect term: a SITES defect replaces the block's charge
    by ``defect.charge`` (vacancy: 0, so xi = -Z; impurity Z': xi = Z' - Z),
    Eq. (Can_LatticeSum_full); a POINT defect adds its charge."""
    if defect.kind == SITES:
        return defect.charge - blocks[defect.block].charge
    return defect.charge


def canonical_terms(N, box_lo, box_hi, g, blocks, defects):
    """All canonical terms of the defected lattice sum, deduplicated by window.

    Sec. 4.1, Eq. (Can_LatticeSum_full): P_hat = P_0 + sum_s P_s, where P_0 is
    the assembled rank-R sum of each rectangular block (Thm 3.1(A); a union of
    blocks is class (A) of Sec. 4.4) and each defect P_s is a shifted rank-R
    reference tensor scaled by its charge change (a cluster of sites sums its
    windows per mode, class (D)). Returns

      cols : 3 arrays (C_l, N) -- distinct canonical vectors per mode (each
             block's assembled vectors, then one vector per distinct defect
             window set and rank index),
      tcol : (T, 3) int -- the column of each term in each mode,
      xi   : (T,) float -- the weight of each term (charges, not yet
             including the vector norms).

    Terms are ordered block-major then defect-major, rank index q fastest.
    """
    R = g.shape[0]
    nb = len(blocks)
    bidx = [block_vertex_indices(b, N, box_lo, box_hi) for b in blocks]
    cols = [[] for _ in range(3)]
    keys = [dict() for _ in range(3)]
    tcol, xi = [], []
    for bi, b in enumerate(blocks):
        for q in range(R):
            for a in range(3):
                cols[a].append(assembled_vector(g[q], bidx[bi][a], N))
            tcol.append([bi * R + q] * 3)
            xi.append(b.charge)

    def defect_windows(d, a):
        if d.kind == SITES:
            return tuple(bidx[d.block][a][d.site[a] + e] for e in range(d.extent[a]))
        return (snap(d.pos[a], N, box_lo, box_hi),)

    for d in defects:
        base = []
        for a in range(3):
            key = defect_windows(d, a)
            if key not in keys[a]:
                keys[a][key] = len(keys[a])
                for q in range(R):
                    cols[a].append(assembled_vector(g[q], key, N))
            base.append(nb * R + keys[a][key] * R)
        z = defect_charge(d, blocks)
        for q in range(R):
            tcol.append([base[0] + q, base[1] + q, base[2] + q])
            xi.append(z)
    return ([np.array(c) for c in cols], np.array(tcol, dtype=np.int64),
            np.array(xi, dtype=np.float64))


def explicit_terms(cols, tcol, xi):
    """The same terms with one explicit vector per term and mode (no sharing):
    the paper's concatenated side matrices, Eq. (SideMTuckS)."""
    return [cols[a][tcol[:, a]] for a in range(3)], np.arange(len(xi))[:, None].repeat(3, 1), xi


# ---------------------------------------------------------------------------
# full-tensor and brute-force references (Thm 3.1 proof; Eq. EwaldSumE)
# ---------------------------------------------------------------------------

def full_tensor_sitewise(N, box_lo, box_hi, g, blocks, defects) -> np.ndarray:
    """The full N^3 tensor sum_sites Z_s W_s P_R, built site by site as in the
    first line of the proof of Thm 3.1 (Eq. fullsum before the 1D
    reduction): every charged site contributes its own shifted rank-R
    reference tensor. Small N only."""
    R = g.shape[0]
    charges = {}
    for bi, b in enumerate(blocks):
        idx = block_vertex_indices(b, N, box_lo, box_hi)
        for k1 in range(b.L[0]):
            for k2 in range(b.L[1]):
                for k3 in range(b.L[2]):
                    key = (idx[0][k1], idx[1][k2], idx[2][k3])
                    charges[key] = charges.get(key, 0.0) + b.charge
    for d in defects:
        if d.kind == SITES:
            b = blocks[d.block]
            idx = block_vertex_indices(b, N, box_lo, box_hi)
            for e1 in range(d.extent[0]):
                for e2 in range(d.extent[1]):
                    for e3 in range(d.extent[2]):
                        key = (idx[0][d.site[0] + e1], idx[1][d.site[1] + e2],
                               idx[2][d.site[2] + e3])
                        charges[key] = charges.get(key, 0.0) + d.charge - b.charge
        else:
            key = tuple(snap(d.pos[a], N, box_lo, box_hi) for a in range(3))
            charges[key] = charges.get(key, 0.0) + d.charge
    T = np.zeros((N, N, N))
    for (m1, m2, m3), z in charges.items():
        if z == 0.0:
            continue
        for q in range(R):
            T += z * np.einsum("i,j,k->ijk", window(g[q], m1, N), window(g[q], m2, N),
                               window(g[q], m3, N))
    return T


def charged_centres(N, box_lo, box_hi, blocks, defects):
    """(positions (K,3), charges (K,)) of all net charges, at their snapped
    vertex positions: the centres a_nu and charges Z_nu of Eq. (EwaldSumE)
    with the defects applied."""
    h = mesh_size(N, box_lo, box_hi)
    charges = {}
    for b in blocks:
        idx = block_vertex_indices(b, N, box_lo, box_hi)
        for k1 in range(b.L[0]):
            for k2 in range(b.L[1]):
                for k3 in range(b.L[2]):
                    key = (idx[0][k1], idx[1][k2], idx[2][k3])
                    charges[key] = charges.get(key, 0.0) + b.charge
    for d in defects:
        if d.kind == SITES:
            b = blocks[d.block]
            idx = block_vertex_indices(b, N, box_lo, box_hi)
            for e1 in range(d.extent[0]):
                for e2 in range(d.extent[1]):
                    for e3 in range(d.extent[2]):
                        key = (idx[0][d.site[0] + e1], idx[1][d.site[1] + e2],
                               idx[2][d.site[2] + e3])
                        charges[key] = charges.get(key, 0.0) + d.charge - b.charge
        else:
            key = tuple(snap(d.pos[a], N, box_lo, box_hi) for a in range(3))
            charges[key] = charges.get(key, 0.0) + d.charge
    keys = [k for k, z in charges.items() if z != 0.0]
    pos = box_lo + h * np.array(keys, dtype=np.float64).reshape(-1, 3)
    z = np.array([charges[k] for k in keys], dtype=np.float64)
    return pos, z


def brute_force(points: np.ndarray, centres: np.ndarray, charges: np.ndarray, kappa: float = 0.0,
                kernel: int = YUKAWA):
    """Direct sum sum_nu Z_nu p(|x - a_nu|) (Eq. EwaldSumE; p = 1/r, or
    exp(-kappa r)/r) at the given points; also returns sum_nu |Z_nu| p(|x - a_nu|)
    and the minimum and maximum distance to a centre, which bound the
    quadrature error."""
    points = np.atleast_2d(points)
    val = np.zeros(len(points))
    absval = np.zeros(len(points))
    dmin = np.full(len(points), np.inf)
    dmax = np.zeros(len(points))
    for c0 in range(0, len(centres), 256):
        c = centres[c0:c0 + 256]
        d = np.sqrt(((points[:, None, :] - c[None, :, :]) ** 2).sum(-1))
        pd = kernel_value(d, kappa, kernel)
        val += (charges[c0:c0 + 256] * pd).sum(1)
        absval += (np.abs(charges[c0:c0 + 256]) * pd).sum(1)
        dmin = np.minimum(dmin, d.min(1))
        dmax = np.maximum(dmax, d.max(1))
    return val, absval, dmin, dmax


# ---------------------------------------------------------------------------
# (c) RHOSVD, Def. 4.1, Thm A.1, Sec. 4.3 (Eq. SideMTuckS)
# ---------------------------------------------------------------------------

def truncation_rank(sigma: np.ndarray, eps: float) -> int:
    """Smallest r with (sum_{k>r} sigma_k^2)^(1/2) <= eps (sum_k sigma_k^2)^(1/2).
    Sec. 4.3 lets a threshold eps replace the fixed rank; reading: relative
    Frobenius norm of the (column-normalised) side matrix, per mode."""
    s2 = np.asarray(sigma, dtype=np.float64) ** 2
    tail = np.concatenate([np.cumsum(s2[::-1])[::-1], [0.0]])   # tail[r] = sum_{k>=r}
    total = tail[0]
    for r in range(len(s2) + 1):
        if math.sqrt(tail[r]) <= eps * math.sqrt(total):
            return max(r, 1) if len(s2) else 0
    return len(s2)


def normalise_terms(cols, tcol, xi):
    """Eq. (CP_form): canonical vectors of unit length, the norms moved into
    the weights xi_nu. Returns (normalised cols, norms, xi)."""
    norms = [np.sqrt((c * c).sum(1)) for c in cols]
    xin = xi.copy()
    for a in range(3):
        xin = xin * norms[a][tcol[:, a]]
    ncols = [cols[a] / norms[a][:, None] for a in range(3)]
    return ncols, norms, xin


def rhosvd(cols, tcol, xi, eps, ranks=None, core=True):
    """Reduced HOSVD of the canonical tensor sum_nu xi_nu a1 (x) a2 (x) a3.

    Def. 4.1 and Thm A.1(c),(d): for each mode, the SVD of the side matrix
    A^(l) (columns = the normalised canonical vectors of every term, Eq.
    SideMTuckS), Z_l = the leading r_l left singular vectors; the core is the
    projection mu = sum_nu xi_nu (Z1^T a1_nu) (x) (Z2^T a2_nu) (x) (Z3^T a3_nu).

    ``cols`` may hold each distinct vector once (``tcol`` maps terms to
    columns). The side matrix with repeated columns has A A^T = sum_c count_c
    a_c a_c^T, so its left singular vectors and values are those of the
    distinct columns scaled by sqrt(count) -- an identity, not an
    approximation (pinned in the tests against the explicit side matrix).

    Returns a dict: Z (3 x (N, r_l)), sigma (3 arrays), r, d (discarded
    (sum_{k>r} sigma^2)^(1/2) per mode), xi (normalised weights), P (3 x
    (r_l, C_l)), B (r1, r2, r3) core, bound = ||xi||_2 * sum_l d_l (Thm A.1(d)).
    ``ranks`` forces the ranks instead of the eps rule.
    """
    ncols, norms, xin = normalise_terms(cols, tcol, xi)
    out = {"Z": [], "sigma": [], "r": [], "d": [], "P": [], "xi": xin, "norms": norms}
    for a in range(3):
        count = np.bincount(tcol[:, a], minlength=len(ncols[a])).astype(np.float64)
        Aw = (ncols[a] * np.sqrt(count)[:, None]).T          # (N, C) weighted side matrix
        U, S, _ = np.linalg.svd(Aw, full_matrices=False)
        r = truncation_rank(S, eps) if ranks is None else int(ranks[a])
        Z = U[:, :r]
        out["Z"].append(Z)
        out["sigma"].append(S)
        out["r"].append(r)
        out["d"].append(math.sqrt(float(np.sum(S[r:] ** 2))))
        out["P"].append(Z.T @ ncols[a].T)                  # (r, C): Z^T a_c
    out["bound"] = float(np.linalg.norm(xin)) * sum(out["d"])
    if core:
        out["B"] = core_tensor(out["P"], tcol, xin)
    return out


def core_tensor(P, tcol, xi, chunk=512) -> np.ndarray:
    """mu[i,j,k] = sum_nu xi_nu P1[i,c1(nu)] P2[j,c2(nu)] P3[k,c3(nu)]
    (Thm A.1(c), core in canonical form), summed in chunks of terms."""
    r1, r2, r3 = P[0].shape[0], P[1].shape[0], P[2].shape[0]
    B = np.zeros((r1, r2 * r3))
    for s in range(0, len(xi), chunk):
        sl = slice(s, s + chunk)
        p1 = P[0][:, tcol[sl, 0]] * xi[sl]
        kr = (P[1][:, None, tcol[sl, 1]] * P[2][None, :, tcol[sl, 2]]).reshape(r2 * r3, -1)
        B += p1 @ kr.T
    return B.reshape(r1, r2, r3)


def als_refine(cols, tcol, xi, Z0, sweeps: int = 3, chunk: int = 512):
    """ALS refinement of a rank-(r1, r2, r3) Tucker approximation of the
    canonical tensor sum_nu xi_nu a1 (x) a2 (x) a3 (Thm A.1(a)-(c)).

    Thm A.1(a): the best rank-r Tucker approximation maximises ||mu||^2, mu =
    sum_nu xi_nu (Y1^T a1_nu) (x) (Y2^T a2_nu) (x) (Y3^T a3_nu), over
    orthonormal Y_l; (b) the maximiser is found by ALS from the RHOSVD start.
    One ALS step for mode l, with the other two bases fixed, maximises
    ||Y_l^T B_l||_F for the N x (r_m r_n) matrix B_l = sum_nu xi_nu a_l,nu
    (x) vec((Y_m^T a_m,nu) (x) (Y_n^T a_n,nu)), so Y_l = its r_l leading left
    singular vectors (an SVD of B_l). (c) The core is the projection with the
    final bases. ``cols`` are the terms' vectors (normalised inside, norms
    moved into xi, as in ``rhosvd``), ``Z0`` the starting bases.

    Returns (Z, core, history), history[s] = ||mu|| after sweep s (history[0]:
    the start). ||A - A_r||^2 = ||A||^2 - ||mu||^2 for orthonormal bases, so
    a non-decreasing history is a non-increasing error."""
    ncols, _, xin = normalise_terms(cols, tcol, xi)
    Z = [np.array(z, dtype=np.float64) for z in Z0]
    r = [z.shape[1] for z in Z]
    # B_l has min(N, r_m r_n) singular vectors: a start whose rank r_l exceeds that would leave
    # Y_l with fewer columns than asked (the step could not keep the rank)
    for l in range(3):
        m, n = [a for a in range(3) if a != l]
        if r[l] > min(ncols[l].shape[1], r[m] * r[n]):
            raise ValueError(f"als_refine: rank {r[l]} of mode {l} exceeds min(N, r_m r_n) = "
                             f"{min(ncols[l].shape[1], r[m] * r[n])}")

    def core_of(Z):
        return core_tensor([Z[a].T @ ncols[a].T for a in range(3)], tcol, xin)
    history = [float(np.linalg.norm(core_of(Z)))]
    for _ in range(sweeps):
        for l in range(3):
            m, n = [a for a in range(3) if a != l]
            Pm, Pn = Z[m].T @ ncols[m].T, Z[n].T @ ncols[n].T
            N = ncols[l].shape[1]
            B = np.zeros((N, r[m] * r[n]))
            for s0 in range(0, len(xin), chunk):
                sl = slice(s0, s0 + chunk)
                al = ncols[l][tcol[sl, l]].T * xin[sl]                       # (N, terms)
                kr = (Pm[:, None, tcol[sl, m]] * Pn[None, :, tcol[sl, n]]).reshape(r[m] * r[n], -1)
                B += al @ kr.T
            U, _, _ = np.linalg.svd(B, full_matrices=False)
            Z[l] = U[:, :r[l]]
        history.append(float(np.linalg.norm(core_of(Z))))
    return Z, core_of(Z), history


# ---------------------------------------------------------------------------
# Tucker-reference variant: Thm 3.1(B), Sec. 4.1 (Eqs. Tuck_LatticeKi,
# Tuck_LatticeSum_full), Thm 4.3 (Tucker-Sum-to-Tucker)
# ---------------------------------------------------------------------------

def reference_tucker(g: np.ndarray, eps_ref: float):
    """The rank-r "reference" Tucker tensor of Eq. (TuckRef_sum) on the doubled
    grid. Reading: the paper obtains it from the canonical reference tensor
    (its Table 2.1 uses an ALS Can-to-Tucker); here it is the RHOSVD of the
    reference canonical tensor P = sum_q g_q (x) g_q (x) g_q (Def. 4.1, Thm
    A.1(c)): the side matrix has the unit vectors g_q/|g_q| as columns (Eq.
    CP_form), Z = its leading left singular vectors at the relative threshold
    eps_ref (same rule as the lattice sum), and the core b = sum_q
    (Z^T g_q) (x) (Z^T g_q) (x) (Z^T g_q). The three modes share g, so they
    share Z.

    Returns (t, b, sigma): t (r, 2N) the reference Tucker vectors as rows,
    b (r, r, r), sigma the singular values of the side matrix."""
    norms = np.sqrt((g * g).sum(1))
    U, S, _ = np.linalg.svd((g / norms[:, None]).T, full_matrices=False)
    r = truncation_rank(S, eps_ref)
    Z = U[:, :r]
    h = Z.T @ g.T                               # (r, R): Z^T g_q
    b = np.einsum("iq,jq,kq->ijk", h, h, h)
    return Z.T.copy(), b, S


def tucker_terms(N, box_lo, box_hi, t, b, blocks, defects):
    """The lattice sum with defects as a sum of Tucker tensors, Sec. 4.1:
    U_hat = U_0 + sum_s U_s (Eq. Tuck_LatticeSum_full).

    * each rectangular block contributes its assembled Tucker tensor (Thm
      3.1(B), Eq. Tuck_LatticeSum): mode-l side matrix sum_k W_{m_k} t_m (one
      1D window sum per Tucker vector and mode), core = charge * b;
    * each defect contributes the shifted reference Tucker tensor
      (Eq. Tuck_LatticeKi): side matrix W_m t_m at its vertex (a cluster of
      sites: the sum of its windows per mode), core = (charge change) * b;
      a POINT defect: its charge times b at its snapped vertex.

    Returns a list of (F, core, keys): F = 3 arrays (N, r) of side matrices,
    core (r, r, r), keys = per mode the tuple of window vertices (terms with
    equal keys share a side matrix)."""
    r = t.shape[0]
    terms = []
    bidx = [block_vertex_indices(bl, N, box_lo, box_hi) for bl in blocks]

    def side(ms):
        F = np.zeros((N, r))
        for m in ms:
            for k in range(r):
                F[:, k] += window(t[k], m, N)
        return F

    for bi, bl in enumerate(blocks):
        keys = [("block", bi, a) for a in range(3)]
        terms.append(([side(bidx[bi][a]) for a in range(3)], bl.charge * b, keys))
    for d in defects:
        if d.kind == SITES:
            ms = [tuple(bidx[d.block][a][d.site[a] + e] for e in range(d.extent[a])) for a in range(3)]
        else:
            ms = [(snap(d.pos[a], N, box_lo, box_hi),) for a in range(3)]
        terms.append(([side(ms[a]) for a in range(3)], defect_charge(d, blocks) * b, [("win",) + ms[a] for a in range(3)]))
    return terms


def tucker_full(terms) -> np.ndarray:
    """The full tensor sum_s core_s x1 F1 x2 F2 x3 F3 of a list of Tucker terms (small N)."""
    N = terms[0][0][0].shape[0]
    T = np.zeros((N, N, N))
    for F, core, _ in terms:
        T += np.einsum("abc,ia,jb,kc->ijk", core, F[0], F[1], F[2], optimize=True)
    return T


def reference_tucker_full(N, box_lo, box_hi, t, b, blocks, defects) -> np.ndarray:
    """The same lattice sum built site by site from shifted reference Tucker
    tensors, sum_sites Z_s W_s T_ref (Eq. WindowTuck_sum), before any 1D
    agglomeration (the identity Thm 3.1(B) asserts). Small N only."""
    pos, z = charged_centres(N, box_lo, box_hi, blocks, defects)
    h = mesh_size(N, box_lo, box_hi)
    T = np.zeros((N, N, N))
    for p, q in zip(pos, z):
        m = [int(round((p[a] - box_lo) / h)) for a in range(3)]
        F = [np.stack([window(t[k], m[a], N) for k in range(t.shape[0])], 1) for a in range(3)]
        T += q * np.einsum("abc,ia,jb,kc->ijk", b, F[0], F[1], F[2], optimize=True)
    return T


def tucker_sum_rhosvd(terms, eps, ranks=None):
    """Generalized RHOSVD of a sum of Tucker tensors, Thm 4.3 (Tucker-Sum-to-
    Tucker), Sec. 4.3 (Eq. SideMTuckS).

    Reading. Thm 4.3 takes the Tucker tensors of the sum as orthogonal (Sec.
    4.1); what its bound uses is that every side matrix has spectral norm at
    most 1, so that a projection error in one mode is not amplified by the
    other two. The assembled block vectors (Thm 3.1(B); the paper notes they
    lose orthogonality) and cluster windows do not have it, and
    orthonormalising them (Gram-Schmidt) is ill-conditioned: windowed and
    assembled Tucker vectors are nearly dependent (condition numbers of 1e6 -
    1e7 on small lattices), so the orthonormal basis is known only to about
    u * cond. Here each term's side matrix F_l is scaled to unit Frobenius norm
    (which bounds its spectral norm by 1) and the scale is moved into its core:
    F_l -> F_l / |F_l|_F, B_s -> B_s prod_l |F_l|_F. For rank-one terms with
    unit vectors this is the RHOSVD of a canonical sum (Thm A.1), which the
    paper names as the special case of the generalized scheme.

    The agglomerated side matrix of mode l concatenates the scaled side
    matrices of all terms (Eq. SideMTuckS; a side matrix shared by k terms
    enters k times, or once with weight sqrt(k): the same left singular vectors
    and values). Its truncated SVD gives Z_l (the eps rule of
    ``truncation_rank``, or forced ``ranks``); the core is the projection
    sum_s B_s x_l (Z_l^T F_s) of the sum itself. The bound of Thm 4.3(a) is
    |B_hat| sum_l (sum_{k > r_l} sigma_{l,k}^2)^(1/2) with
    |B_hat|^2 = sum_s ||B_s||^2 prod_l |F_{s,l}|_F^2.

    Returns a dict: Z (3 x (N, r_l)), sigma, r, d, B (core), bound, Bhat."""
    out = {"Z": [], "sigma": [], "r": [], "d": []}
    scale = [[float(np.linalg.norm(F[a])) for a in range(3)] for F, _, _ in terms]
    for a in range(3):
        side = np.concatenate([F[a] / sc[a] for (F, _, _), sc in zip(terms, scale)], axis=1)
        U, S, _ = np.linalg.svd(side, full_matrices=False)
        r = truncation_rank(S, eps) if ranks is None else int(ranks[a])
        out["Z"].append(U[:, :r])
        out["sigma"].append(S)
        out["r"].append(r)
        out["d"].append(math.sqrt(float(np.sum(S[r:] ** 2))))
    B = np.zeros(tuple(out["r"]))
    Bhat2 = 0.0
    for (F, core, _), sc in zip(terms, scale):
        P = [out["Z"][a].T @ F[a] for a in range(3)]
        B += np.einsum("abc,ia,jb,kc->ijk", core, P[0], P[1], P[2], optimize=True)
        Bhat2 += float(np.sum(core * core)) * (sc[0] * sc[1] * sc[2]) ** 2
    out["B"] = B
    out["Bhat"] = math.sqrt(Bhat2)
    out["bound"] = out["Bhat"] * sum(out["d"])
    return out


# ---------------------------------------------------------------------------
# (d) evaluation on slabs (n-mode products, Eq. Tucker_singePot)
# ---------------------------------------------------------------------------

def tucker_slab(Z, B, i3: int) -> np.ndarray:
    """Values of the Tucker tensor B x1 Z1 x2 Z2 x3 Z3 on the slab i3
    (Eq. Tucker_singePot): (B x3 Z3[i3,:]) then Z1 M Z2^T. Shape (N, N),
    first index = mode 1."""
    M = B @ Z[2][i3]                 # (r1, r2)
    return Z[0] @ M @ Z[1].T


def canonical_slab(cols, tcol, xi, i3: int) -> np.ndarray:
    """Values of the untruncated canonical tensor sum_nu xi_nu a1 (x) a2 (x) a3
    on the slab i3: A1 diag(xi * a3[i3]) A2^T (Eq. CP_form)."""
    w = xi * cols[2][tcol[:, 2], i3]
    return (cols[0][tcol[:, 0]].T * w) @ cols[1][tcol[:, 1]]


def full_from_tucker(Z, B) -> np.ndarray:
    """The full tensor B x1 Z1 x2 Z2 x3 Z3 (small N only)."""
    return np.einsum("abc,ia,jb,kc->ijk", B, Z[0], Z[1], Z[2], optimize=True)


def full_from_canonical(cols, tcol, xi) -> np.ndarray:
    """The full tensor sum_nu xi_nu a1 (x) a2 (x) a3 (small N only)."""
    return np.einsum("n,ni,nj,nk->ijk", xi, cols[0][tcol[:, 0]], cols[1][tcol[:, 1]],
                     cols[2][tcol[:, 2]], optimize=True)


# ---------------------------------------------------------------------------
# Galerkin matrix of the Tucker potential in a rank-one basis, Eq. (nuc_pot)
# ---------------------------------------------------------------------------

def galerkin_matrix(Z, B, basis) -> np.ndarray:
    """v_km = <G_k (.) G_m, T> (Eq. nuc_pot) for rank-one basis functions
    G_k = g_k^1 (x) g_k^2 (x) g_k^3 (``basis[l]``: (nb, N), row k = g_k^l) and
    the Tucker tensor T = B x1 Z1 x2 Z2 x3 Z3: the Hadamard product of two
    rank-one tensors is rank one, (g_k^l (.) g_m^l) per mode, so the scalar
    product is the core contracted with the three 1D projections
    Z_l^T (g_k^l (.) g_m^l). The grid inner product, without the cell volume
    h^3 (times h^3 it is the midpoint rule for the integral of v g_k g_m).
    Returns V (nb, nb)."""
    M = [np.einsum("ki,mi,ia->kma", basis[l], basis[l], Z[l], optimize=True) for l in range(3)]
    return np.einsum("abc,kma,kmb,kmc->km", B, M[0], M[1], M[2], optimize=True)


def galerkin_matrix_full(T, basis) -> np.ndarray:
    """The same matrix from the definition on the full N^3 tensor: the sum over
    all grid points of T times g_k g_m (small N only)."""
    nb = basis[0].shape[0]
    V = np.zeros((nb, nb))
    for k in range(nb):
        for m in range(nb):
            w = [basis[l][k] * basis[l][m] for l in range(3)]
            V[k, m] = np.einsum("ijl,i,j,l->", T, w[0], w[1], w[2])
    return V


# ---------------------------------------------------------------------------
# whole pipeline (a) + (b) + (c), as timed for the CPU baseline
# ---------------------------------------------------------------------------

def pipeline(wl, t_scale: float, core: bool = True, ranks=None):
    """Quadrature -> generating vectors -> assembled and defect terms ->
    RHOSVD, for a workload description (N, box, R, sinc step, blocks,
    defects, eps; kappa for the Yukawa kernel). Returns (terms, rhosvd result)."""
    t, w = sinc_quadrature(wl.R, wl.sinc_step, t_scale, getattr(wl, "kappa", 0.0), getattr(wl, "kernel", YUKAWA))
    g = generating_vectors(wl.N, wl.box_lo, wl.box_hi, t, w, getattr(wl, "galerkin", False))
    cols, tcol, xi = canonical_terms(wl.N, wl.box_lo, wl.box_hi, g, wl.blocks, wl.defects)
    res = rhosvd(cols, tcol, xi, wl.eps, ranks=ranks, core=core)
    return {"t": t, "w": w, "g": g, "cols": cols, "tcol": tcol, "xi": xi}, res


def default_r_max(wl) -> float:
    """Largest centre-to-point distance inside the cubic box: sqrt(3) b."""
    return math.sqrt(3.0) * (wl.box_hi - wl.box_lo)
