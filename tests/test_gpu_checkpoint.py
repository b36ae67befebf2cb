"""Checkpoints of a reduced context and the reference-vector cache.

- LatticeSum.save / load_checkpoint: the .npz round trip returns the Tucker
  vectors, core, ranks and singular values bit for bit as lattice_sum_read
  gives them, and the restored factors evaluated on the GPU
  (lattice_sum_eval_slab_noalloc on their device copies) give the context's
  own slabs (lattice_sum_eval_slab) within the FP64 tolerance of the other
  parity tests, and the oracle's Tucker evaluation (Eq. Tucker_singePot) of
  the saved factors.
- LS_FLAG_CACHE_GENVEC: the reference vectors g_q of Sec. 2.2, "computed once
  and stored for multiple use": a context that finds them in the cache holds
  bit for bit the vectors of a context that computed them, and the two
  reductions agree bit for bit; lattice_sum_cache_clear reports the entries.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import lattice_oracle as O  # noqa: E402
from paper_1411_1994_gb300 import build as B  # noqa: E402
from paper_1411_1994_gb300 import lattice_sum as L  # noqa: E402
from paper_1411_1994_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wl():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    B.build()
    w = W.small_case(L=(4, 3, 3), N=72, frac_vac=0.1, frac_imp=0.05, eps=1e-7)
    s, _ = O.fit_t_scale(w.R, w.sinc_step, w.r_min, O.default_r_max(w))
    return w, s


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_checkpoint_round_trip(wl, tmp_path):
    w, s = wl
    ls = L.LatticeSum.from_workload(w, s, L.LS_FP64)
    ls.add_defects(w.defects)
    info = ls.rhosvd_reduce(w.eps)
    path = str(tmp_path / "tucker.npz")
    ls.save(path, extra={"workload": w.name})
    ck = L.load_checkpoint(path)
    assert ck.ranks == list(info["r"])
    assert ck.params["N"] == w.N and ck.params["t_scale"] == s and ck.extra["workload"] == w.name
    for l in range(3):
        assert np.array_equal(ck.Z[l], ls.read(L.LS_READ_BASIS, l).reshape(ck.ranks[l], w.N))
        assert np.array_equal(ck.sigma[l], ls.read(L.LS_READ_SIGMA, l))
    assert np.array_equal(ck.core.ravel(), ls.read(L.LS_READ_CORE))
    # the same read into a caller's pinned buffer (what the e2e timing does)
    pinned = torch.empty(int(np.prod(ck.ranks)), dtype=torch.float64, pin_memory=True)
    assert ls.read_into(L.LS_READ_CORE, 0, pinned) == pinned.numel() * 8
    assert np.array_equal(pinned.numpy(), ck.core.ravel())
    with pytest.raises(L.LatticeSumError):
        ls.read_into(L.LS_READ_CORE, 0, torch.empty(3, dtype=torch.float64))
    zs = [0, 5, w.N // 2, w.N - 1]
    ref = ls.eval_slab_torch(zs).cpu().numpy()
    got = ck.eval_slab_torch(zs)
    torch.cuda.synchronize()
    got = got.cpu().numpy()
    orc = np.stack([O.tucker_slab([z.T for z in ck.Z], ck.core, zz) for zz in zs])
    assert rel(got, ref) <= 1e-12
    assert rel(got, orc) <= 1e-12
    ls.close()


def test_checkpoint_refuses_unreduced_context(wl, tmp_path):
    w, s = wl
    with L.LatticeSum.from_workload(w, s, L.LS_FP64) as ls:
        with pytest.raises(L.LatticeSumError):
            ls.save(str(tmp_path / "x.npz"))


def test_genvec_cache_hit_is_bitwise(wl):
    w, s = wl
    L.cache_clear()
    res = []
    for flags in (0, L.LS_FLAG_CACHE_GENVEC, L.LS_FLAG_CACHE_GENVEC):   # computed, stored, found
        ls = L.LatticeSum.from_workload(w, s, L.LS_FP64, flags=flags)
        g = ls.read(L.LS_READ_GENVEC)
        ls.add_defects(w.defects)
        ls.rhosvd_reduce(w.eps)
        res.append((g, ls.read(L.LS_READ_CORE), [ls.read(L.LS_READ_BASIS, l) for l in range(3)]))
        ls.close()
    for g, core, Z in res[1:]:
        assert np.array_equal(g, res[0][0])
        assert np.array_equal(core, res[0][1])
        assert all(np.array_equal(a, b) for a, b in zip(Z, res[0][2]))
    assert L.cache_clear() == 1    # one key: the second cached context found the first one's entry
    assert L.cache_clear() == 0
