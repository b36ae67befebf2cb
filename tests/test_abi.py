"""C-ABI checks that need no GPU: the library builds and loads, exports every
symbol declared in include/*.h, validates its arguments on the host, and its
host-side quadrature fit agrees with the oracle's."""
import math
import os
import re

import numpy as np
import pytest

from paper_1411_1994_gb300 import build as B
from paper_1411_1994_gb300 import lattice_sum as L
from paper_1411_1994_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.lib()


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lattice_sum_\w+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert {"lattice_sum_create", "lattice_sum_add_defects", "lattice_sum_rhosvd_reduce",
            "lattice_sum_eval_slab"} <= names
    for n in names:
        assert hasattr(lib, n), n
    assert names <= set(L.EXPORTED) | names


def test_binding_structs_match_header_sizes(lib):
    import ctypes as C
    assert C.sizeof(L.ls_params) == 8 + 8 + 8 + 8 + 8 + 8 + 4 + 4 + 8 + 8 + 8
    assert C.sizeof(L.ls_block) == 3 * 8 * 3 + 8
    assert C.sizeof(L.ls_defect) == 4 + 4 + 3 * 8 + 3 * 8 + 3 * 8 + 8


def test_fit_t_scale_matches_oracle_quality(lib):
    from oracle import lattice_oracle as O
    for wl in (W.config1(), W.config2(), W.config3()):
        rmax = O.default_r_max(wl)
        s_lib, e_lib = L.fit_t_scale(wl.R, wl.sinc_step, wl.r_min, rmax)
        s_or, e_or = O.fit_t_scale(wl.R, wl.sinc_step, wl.r_min, rmax)
        t, w = O.sinc_quadrature(wl.R, wl.sinc_step, s_lib)
        e_chk = float(np.max(O.quadrature_rel_error(t, w, np.geomspace(wl.r_min, rmax, 600))))
        assert abs(e_chk - e_lib) <= 1e-3 * e_lib
        assert e_lib <= 1.05 * e_or
        assert abs(math.log(s_lib / s_or)) < 0.05


def test_fit_t_scale_rejects_bad_input(lib):
    with pytest.raises(L.LatticeSumError) as ei:
        L.fit_t_scale(24, 0.25, 1.0, 0.5)
    assert ei.value.code == L.LS_ERR_ARG
    for kappa in (-0.5, float("nan"), float("inf")):
        with pytest.raises(L.LatticeSumError) as ei:
            L.fit_t_scale(24, 0.25, 0.25, 40.0, kappa=kappa)
        assert ei.value.code == L.LS_ERR_ARG
    for kernel, kappa in ((L.LS_KERNEL_SLATER, 0.0), (L.LS_KERNEL_DIPOLE, 0.5), (3, 0.0), (-1, 0.0)):
        with pytest.raises(L.LatticeSumError) as ei:
            L.fit_t_scale(24, 0.25, 0.25, 40.0, kappa=kappa, kernel=kernel)
        assert ei.value.code == L.LS_ERR_ARG


@pytest.mark.parametrize("kernel,kappa", [(0, 0.3), (0, 0.5), (0, 1.0), (1, 0.5), (1, 1.0), (2, 0.0)])
def test_fit_t_scale_kernels_match_oracle_quality(lib, kernel, kappa):
    """The library's fit for the Yukawa, Slater and dipole kernels: its
    reported error is the oracle's error of the same rule, and as good as the
    oracle's own fit."""
    from oracle import lattice_oracle as O
    wl = W.config2()
    rmax = O.default_r_max(wl)
    s_lib, e_lib = L.fit_t_scale(wl.R, wl.sinc_step, wl.r_min, rmax, kappa=kappa, kernel=kernel)
    s_or, e_or = O.fit_t_scale(wl.R, wl.sinc_step, wl.r_min, rmax, kappa=kappa, kernel=kernel)
    t, w = O.sinc_quadrature(wl.R, wl.sinc_step, s_lib, kappa, kernel)
    e_chk = float(np.max(O.quadrature_rel_error(t, w, np.geomspace(wl.r_min, rmax, 600), kappa, kernel)))
    assert abs(e_chk - e_lib) <= 1e-3 * e_lib
    assert e_lib <= 1.05 * e_or
    assert e_lib < 1e-5


@pytest.mark.parametrize("bad", [dict(N=1), dict(R=0), dict(R=65), dict(box_hi=-6.0), dict(sinc_step=0.0),
                                 dict(t_scale=-1.0), dict(precision=7), dict(kappa=-1.0),
                                 dict(kappa=float("nan")), dict(kappa=1e4), dict(kernel=3),
                                 dict(kernel=L.LS_KERNEL_SLATER), dict(kernel=L.LS_KERNEL_DIPOLE, kappa=0.5)])
def test_create_validates_arguments_on_host(lib, bad):
    kw = dict(N=64, box_lo=-6.0, box_hi=6.0, R=8, sinc_step=0.25, t_scale=10.0, precision=L.LS_FP64,
              kappa=0.0, kernel=L.LS_KERNEL_YUKAWA)
    kw.update(bad)
    blocks = [W.centred_block((2, 2, 2))]
    with pytest.raises(L.LatticeSumError) as ei:
        L.LatticeSum(kw["N"], kw["box_lo"], kw["box_hi"], kw["R"], kw["sinc_step"], kw["t_scale"], blocks,
                     kw["precision"], kappa=kw["kappa"], kernel=kw["kernel"])
    assert ei.value.code == L.LS_ERR_ARG


def test_create_rejects_unknown_flags(lib):
    """LS_FLAG_GALERKIN, LS_FLAG_SVD_GRAM, LS_FLAG_SVD_ONESIDED,
    LS_FLAG_TUCKER_REF and LS_FLAG_CACHE_GENVEC are the known flags; the two singular-value routes
    exclude each other, the Tucker-reference variant needs 0 < ref_eps < 1 and
    the non-squaring route; anything else is refused on the host before the
    device is touched."""
    import ctypes as C
    blocks = L.make_blocks([W.centred_block((2, 2, 2))])
    for flags, ref_eps in ((L.LS_FLAG_SVD_GRAM | L.LS_FLAG_SVD_ONESIDED, 0.0), (32, 0.0), (0x100, 0.0), (-1, 0.0),
                           (L.LS_FLAG_TUCKER_REF, 0.0), (L.LS_FLAG_TUCKER_REF, 1.5),
                           (L.LS_FLAG_TUCKER_REF | L.LS_FLAG_SVD_GRAM, 1e-6)):
        p = L.ls_params(64, -6.0, 6.0, 8, 0.25, 10.0, L.LS_FP64, flags, 0.0, L.LS_KERNEL_YUKAWA, ref_eps)
        ctx = C.c_void_p()
        rc = L.lib().lattice_sum_create(C.byref(ctx), C.byref(p), blocks, 1, None)
        assert rc == L.LS_ERR_ARG, flags
        assert not ctx.value


def test_create_rejects_site_outside_box(lib):
    blk = W.Block((3, 1, 1), (5.0, 0.0, 0.0), (1.0, 1.0, 1.0), 1.0)
    with pytest.raises(L.LatticeSumError) as ei:
        L.LatticeSum(64, -6.0, 6.0, 8, 0.25, 10.0, [blk])
    assert ei.value.code == L.LS_ERR_ARG


def test_no_gpu_fails_loudly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(L.LatticeSumError) as ei:
        L.LatticeSum.from_workload(W.config1(), 11.9)
    assert ei.value.code == L.LS_ERR_CUDA


def test_missing_library_raises(tmp_path):
    with pytest.raises(ImportError):
        L.load_library(str(tmp_path / "nope.so"))
