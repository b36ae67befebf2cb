"""Seeded synthetic workloads for the lattice-sum path.

This module only *describes* inputs: lattice blocks (sizes, origins, spacing,
charges), defect lists, grid sizes, quadrature rank and truncation threshold.
It holds none of the method's arithmetic (no quadrature, no snapping to the
grid, no window sums, no SVD), so that the CUDA path and the CPU oracle can
both consume exactly the same inputs without sharing any computation.

Random choices use SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written out here so that the
defect lists are identical on every machine and Python version.

Geometry conventions (the paper leaves them open):
  * every lattice has spacing 1.0 and unit charges;
  * sites of an L1 x L2 x L3 lattice are centred on the origin: site k along
    an axis sits at (k - (L_max - 1)/2) * spacing, where L_max is the extent of
    the bounding lattice (so sub-blocks of a union stay aligned);
  * the cubic box is [-b/2, b/2] with b = (L_max - 1) * spacing + 9 * spacing
    (the 4x4x4 case then has the box [-6, 6] of the small configuration).

Defect semantics (Sec. 4.1, Eq. Can_LatticeSum_full): a defect *replaces* the
charge of a set of lattice sites. A vacancy gives the new charge 0, an
impurity a new charge Z' drawn uniformly from [0.5, 1.5]. A cluster defect is
a 3x3x3 box of sites with one new charge (class D of Sec. 4.4). A point
defect adds a charge at an arbitrary position (off-lattice impurity, Sec. 4.4).
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Tuple

MASK64 = (1 << 64) - 1

DEFECT_SITES = 0   # replace the charge of a box of lattice sites of one block
DEFECT_POINT = 1   # add a charge at an arbitrary position


class SplitMix64:
    """SplitMix64 generator; ``uniform()`` returns a double in [0, 1)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def below(self, n: int) -> int:
        """Integer uniform in [0, n) (n small, bias < 2^-40)."""
        return int(self.uniform() * n)


@dataclasses.dataclass(frozen=True)
class Block:
    """A rectangular L[0] x L[1] x L[2] lattice; site k along axis a sits at
    origin[a] + k * spacing[a]; every site carries ``charge``."""
    L: Tuple[int, int, int]
    origin: Tuple[float, float, float]
    spacing: Tuple[float, float, float]
    charge: float = 1.0

    @property
    def nsites(self) -> int:
        return self.L[0] * self.L[1] * self.L[2]


@dataclasses.dataclass(frozen=True)
class Defect:
    """DEFECT_SITES: sites block[site[a] : site[a] + extent[a]] get charge
    ``charge`` (0 = vacancy). DEFECT_POINT: a charge ``charge`` is added at
    ``pos``."""
    kind: int
    block: int = 0
    site: Tuple[int, int, int] = (0, 0, 0)
    extent: Tuple[int, int, int] = (1, 1, 1)
    pos: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    charge: float = 0.0


@dataclasses.dataclass
class Workload:
    name: str
    N: int
    box_lo: float
    box_hi: float
    R: int
    sinc_step: float
    eps: float
    blocks: List[Block]
    defects: List[Defect]
    r_min: float = 0.25     # distance below which the quadrature is not asked to hold
    slabs: Optional[List[int]] = None   # z-indices to evaluate
    kappa: float = 0.0      # kernel parameter: Yukawa exp(-kappa r)/r (0: Newton 1/r), Slater exp(-kappa r)
    kernel: int = 0         # 0: Yukawa/Newton, 1: Slater, 2: dipole 1/r^3
    galerkin: bool = False  # reference vectors as cell averages (Eq. galten) instead of collocation

    @property
    def n_sites(self) -> int:
        return sum(b.nsites for b in self.blocks)

    @property
    def n_vacated(self) -> int:
        n = 0
        for d in self.defects:
            if d.kind == DEFECT_SITES and d.charge == 0.0:
                n += d.extent[0] * d.extent[1] * d.extent[2]
        return n

    @property
    def units(self) -> int:
        """Charged lattice sites represented in the result (sites minus
        vacated sites; impurities count once)."""
        return self.n_sites - self.n_vacated


def centred_block(L, L_max=None, k0=(0, 0, 0), spacing=1.0, charge=1.0) -> Block:
    """Block of L sites starting at site index k0 of a centred bounding
    lattice of extent L_max per axis."""
    if L_max is None:
        L_max = L
    origin = tuple((k0[a] - (L_max[a] - 1) / 2.0) * spacing for a in range(3))
    return Block(tuple(int(x) for x in L), origin, (spacing,) * 3, charge)


def skewed_lattice_blocks(L, a1: float, a2, a3, origin=(0.0, 0.0, 0.0), charge=1.0) -> List[Block]:
    """Sec. 4.4 classes (B) and (C): the lattice of sites origin + i (a1, 0, 0)
    + j a2 + k a3, 0 <= i < L[0], 0 <= j < L[1], 0 <= k < L[2], with the first
    lattice vector along x, as a union of rectangular blocks (class A input).
    Class (B), a3 = (0, 0, d3) and a2 skewed in the (x, y) plane (a
    parallelogram lattice): one L[0] x 1 x L[2] block per j, so the summation
    stays agglomerated in two indices and the rank grows like L[1]. Class (C),
    a3 skewed as well: one L[0] x 1 x 1 block per (j, k), rank growing like
    L[1] L[2]."""
    a2, a3 = tuple(float(x) for x in a2), tuple(float(x) for x in a3)
    blocks = []
    if a3[0] == 0.0 and a3[1] == 0.0:
        for j in range(L[1]):
            o = tuple(origin[d] + j * a2[d] for d in range(3))
            blocks.append(Block((int(L[0]), 1, int(L[2])), o, (float(a1), 1.0, a3[2]), charge))
    else:
        for k in range(L[2]):
            for j in range(L[1]):
                o = tuple(origin[d] + j * a2[d] + k * a3[d] for d in range(3))
                blocks.append(Block((int(L[0]), 1, 1), o, (float(a1), 1.0, 1.0), charge))
    return blocks


def box_for(L_max, spacing=1.0) -> Tuple[float, float]:
    b = (max(L_max) - 1) * spacing + 9.0 * spacing
    return -b / 2.0, b / 2.0


def _sample_sites(rng: SplitMix64, L, count: int) -> List[Tuple[int, int, int]]:
    """``count`` distinct sites of an L[0] x L[1] x L[2] lattice (partial
    Fisher-Yates over the linear index, x fastest)."""
    n = L[0] * L[1] * L[2]
    perm = list(range(n))
    out = []
    for i in range(count):
        j = i + rng.below(n - i)
        perm[i], perm[j] = perm[j], perm[i]
        lin = perm[i]
        out.append((lin % L[0], (lin // L[0]) % L[1], lin // (L[0] * L[1])))
    return out


def point_defects(rng: SplitMix64, blocks: List[Block], frac_vac: float, frac_imp: float,
                  imp_lo=0.5, imp_hi=1.5) -> List[Defect]:
    """round(f * #sites) vacancies and impurities at distinct sites of the
    union of ``blocks`` (vacancies first, then impurities)."""
    nsites = sum(b.nsites for b in blocks)
    nv = int(round(frac_vac * nsites))
    ni = int(round(frac_imp * nsites))
    # sample over the union by linear index, then map back to (block, site)
    perm = list(range(nsites))
    picks = []
    for i in range(nv + ni):
        j = i + rng.below(nsites - i)
        perm[i], perm[j] = perm[j], perm[i]
        picks.append(perm[i])
    out = []
    for i, lin in enumerate(picks):
        b = 0
        while lin >= blocks[b].nsites:
            lin -= blocks[b].nsites
            b += 1
        L = blocks[b].L
        site = (lin % L[0], (lin // L[0]) % L[1], lin // (L[0] * L[1]))
        if i < nv:
            out.append(Defect(DEFECT_SITES, b, site, (1, 1, 1), charge=0.0))
        else:
            z = imp_lo + (imp_hi - imp_lo) * rng.uniform()
            out.append(Defect(DEFECT_SITES, b, site, (1, 1, 1), charge=z))
    return out


def cluster_defects(rng: SplitMix64, L, count: int, size=3) -> List[Defect]:
    """``count`` non-overlapping size^3 clusters with corners uniform in
    [0, L - size] per axis; each is a vacancy cluster with probability 1/2,
    otherwise an impurity cluster with one charge uniform in [0.5, 1.5]."""
    taken = set()
    out = []
    tries = 0
    while len(out) < count:
        tries += 1
        if tries > 1000 * count:
            raise RuntimeError("cannot place clusters")
        c = tuple(rng.below(L[a] - size + 1) for a in range(3))
        cells = {(c[0] + i, c[1] + j, c[2] + k)
                 for i in range(size) for j in range(size) for k in range(size)}
        vac = rng.uniform() < 0.5
        z = 0.0 if vac else 0.5 + rng.uniform()
        if cells & taken:
            continue
        taken |= cells
        out.append(Defect(DEFECT_SITES, 0, c, (size,) * 3, charge=z))
    return out


def config1() -> Workload:
    """4x4x4 lattice, box [-6,6], N=256, R=24, h=0.25, eps=1e-8, no defects."""
    L = (4, 4, 4)
    lo, hi = box_for(L)
    return Workload("c1_4x4x4_N256_R24", 256, lo, hi, 24, 0.25, 1e-8,
                    [centred_block(L)], [], slabs=list(range(0, 256, 8)))


def config2(seed=1002) -> Workload:
    """16^3 lattice, N=1024, R=24, 5% vacancies + 2% impurities, eps=1e-6,
    64 random z-slabs."""
    L = (16, 16, 16)
    lo, hi = box_for(L)
    blocks = [centred_block(L)]
    rng = SplitMix64(seed)
    defects = point_defects(rng, blocks, 0.05, 0.02)
    slabs = sorted(set(rng.below(1024) for _ in range(200)))[:64]
    return Workload("c2_16x16x16_N1024_R24_defects", 1024, lo, hi, 24, 0.25, 1e-6,
                    blocks, defects, slabs=slabs)


def config3(seed=1003) -> Workload:
    """Step-shaped union of a 48x48x24 block (z sites 0..23) and a 24x24x24
    block (x,y sites 0..23, z sites 24..47) of a centred 48^3 bounding lattice,
    3% vacancies, N=4096, R=28, eps=1e-6."""
    Lmax = (48, 48, 48)
    lo, hi = box_for(Lmax)
    blocks = [centred_block((48, 48, 24), Lmax, (0, 0, 0)),
              centred_block((24, 24, 24), Lmax, (0, 0, 24))]
    rng = SplitMix64(seed)
    defects = point_defects(rng, blocks, 0.03, 0.0)
    slabs = sorted(set(rng.below(4096) for _ in range(100)))[:16]
    return Workload("c3_step_48x48x24+24x24x24_N4096_R28", 4096, lo, hi, 28, 0.25, 1e-6,
                    blocks, defects, slabs=slabs)


def config4_item(j: int) -> Workload:
    """Item j of the batch: L uniform in 8..48 per axis, defect fraction
    uniform in [0, 0.1] split 5:2 vacancy:impurity, N in {512,1024,2048},
    R in {20,24,28}, eps=1e-6."""
    rng = SplitMix64(4000 + j)
    L = tuple(8 + rng.below(41) for _ in range(3))
    f = 0.1 * rng.uniform()
    N = (512, 1024, 2048)[rng.below(3)]
    R = (20, 24, 28)[rng.below(3)]
    lo, hi = box_for(L)
    blocks = [centred_block(L)]
    defects = point_defects(rng, blocks, f * 5.0 / 7.0, f * 2.0 / 7.0)
    return Workload(f"c4_item{j}_{L[0]}x{L[1]}x{L[2]}_N{N}_R{R}", N, lo, hi, R, 0.25, 1e-6,
                    blocks, defects, slabs=[N // 2])


def config4(n_items=256) -> List[Workload]:
    return [config4_item(j) for j in range(n_items)]


def config5(seed=1005) -> Workload:
    """256^3 lattice, N=16384, R=32, 1000 3x3x3 defect clusters, eps=1e-6."""
    L = (256, 256, 256)
    lo, hi = box_for(L)
    rng = SplitMix64(seed)
    defects = cluster_defects(rng, L, 1000)
    slabs = sorted(set(rng.below(16384) for _ in range(400)))[:128]
    return Workload("c5_256^3_N16384_R32_clusters", 16384, lo, hi, 32, 0.25, 1e-6,
                    [centred_block(L)], defects, slabs=slabs)


def small_case(L=(3, 2, 2), N=48, R=16, eps=1e-8, frac_vac=0.0, frac_imp=0.0, seed=7,
               sinc_step=0.3, kappa=0.0, kernel=0, galerkin=False) -> Workload:
    """A tiny workload whose full N^3 tensor fits in memory (tests)."""
    lo, hi = box_for(L)
    blocks = [centred_block(L)]
    rng = SplitMix64(seed)
    defects = point_defects(rng, blocks, frac_vac, frac_imp) if (frac_vac or frac_imp) else []
    kname = {0: "yukawa", 1: "slater", 2: "dipole"}[kernel]
    name = f"small_{L[0]}x{L[1]}x{L[2]}_N{N}_R{R}" + (f"_{kname}{kappa:g}" if (kappa or kernel) else "")
    name += "_galerkin" if galerkin else ""
    return Workload(name, N, lo, hi, R, sinc_step, eps, blocks, defects, r_min=0.5,
                    slabs=[N // 2, N // 3], kappa=kappa, kernel=kernel, galerkin=galerkin)


CONFIGS = {"c1": config1, "c2": config2, "c3": config3, "c5": config5}
