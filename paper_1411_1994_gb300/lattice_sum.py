"""Thin ctypes binding of the lattice-sum C ABI (include/lattice_sum.h).

Argument marshalling only: every step of the path runs in the CUDA library.
PyTorch is used for device memory (output slabs) and streams. If the shared
library is missing or cannot be loaded, importing this module raises: there
is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "liblattice_sum.so")

LS_OK, LS_ERR_ARG, LS_ERR_OOM, LS_ERR_CUDA, LS_ERR_NOCONVERGE, LS_ERR_STATE, LS_ERR_TIMEOUT = 0, -1, -2, -3, -4, -5, -6
LS_FP64, LS_MIXED = 0, 1
LS_FLAG_GALERKIN = 1   # reference vectors as cell averages (Eq. galten) instead of collocation
LS_FLAG_SVD_GRAM = 2       # singular values from the FP64 Gram matrix (default of LS_MIXED)
LS_FLAG_SVD_ONESIDED = 4   # singular values without squaring (default of LS_FP64)
LS_FLAG_TUCKER_REF = 8     # Tucker-reference variant (Thm 3.1(B), Thm 4.3), threshold ref_eps
LS_FLAG_CACHE_GENVEC = 16  # reference vectors from / into the process-wide device cache
LS_KERNEL_YUKAWA, LS_KERNEL_SLATER, LS_KERNEL_DIPOLE = 0, 1, 2   # exp(-kappa r)/r (1/r at kappa = 0), exp(-kappa r), 1/r^3
LS_DEFECT_SITES, LS_DEFECT_POINT = 0, 1
LS_OUT_F64, LS_OUT_F32 = 0, 1
(LS_READ_GENVEC, LS_READ_COLUMNS, LS_READ_NORMS, LS_READ_TERMS, LS_READ_XI, LS_READ_SIGMA,
 LS_READ_BASIS, LS_READ_PROJ, LS_READ_CORE, LS_READ_TUCKER_REF) = range(10)

EXPORTED = ("lattice_sum_fit_t_scale", "lattice_sum_fit_t_scale_kernel", "lattice_sum_create", "lattice_sum_add_defects",
            "lattice_sum_rhosvd_reduce", "lattice_sum_eval_slab", "lattice_sum_get_factors",
            "lattice_sum_read", "lattice_sum_profile", "lattice_sum_profile_report",
            "lattice_sum_eval_slab_noalloc", "lattice_sum_batch_reduce", "lattice_sum_gemm_nt",
            "lattice_sum_gemm_nt_mixed", "lattice_sum_jacobi_eig", "lattice_sum_svd_rows", "lattice_sum_tune_eval",
            "lattice_sum_test_fail_alloc", "lattice_sum_test_bounded_wait", "lattice_sum_galerkin",
            "lattice_sum_als_refine", "lattice_sum_cache_clear", "lattice_sum_destroy",
            "lattice_sum_last_error")


class ls_params(C.Structure):
    _fields_ = [("N", C.c_int64), ("box_lo", C.c_double), ("box_hi", C.c_double), ("R", C.c_int32),
                ("sinc_step", C.c_double), ("t_scale", C.c_double), ("precision", C.c_int32),
                ("flags", C.c_int32), ("kappa", C.c_double), ("kernel", C.c_int32), ("ref_eps", C.c_double)]


class ls_block(C.Structure):
    _fields_ = [("L", C.c_int64 * 3), ("origin", C.c_double * 3), ("spacing", C.c_double * 3),
                ("charge", C.c_double)]


class ls_defect(C.Structure):
    _fields_ = [("kind", C.c_int32), ("block", C.c_int32), ("site", C.c_int64 * 3),
                ("extent", C.c_int64 * 3), ("pos", C.c_double * 3), ("charge", C.c_double)]


class ls_tucker_info(C.Structure):
    _fields_ = [("r", C.c_int32 * 3), ("C", C.c_int32 * 3), ("T", C.c_int64),
                ("sigma_discarded", C.c_double * 3), ("sigma_total", C.c_double * 3),
                ("xi_norm", C.c_double), ("bound_abs", C.c_double), ("sweeps", C.c_int32 * 3),
                ("rotations", C.c_int64 * 3), ("pivots", C.c_int32 * 3)]

    def as_dict(self):
        return {"r": list(self.r), "C": list(self.C), "T": int(self.T),
                "sigma_discarded": list(self.sigma_discarded), "sigma_total": list(self.sigma_total),
                "xi_norm": self.xi_norm, "bound_abs": self.bound_abs, "sweeps": list(self.sweeps),
                "rotations": list(self.rotations), "pivots": list(self.pivots)}


class LatticeSumError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"lattice_sum error {code}: {msg}")
        self.code = code


def load_library(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"lattice-sum CUDA library not built ({path}); run __graft_entry__.build()")
    lib = C.CDLL(path)
    P = C.POINTER
    lib.lattice_sum_fit_t_scale.argtypes = [C.c_int32, C.c_double, C.c_double, C.c_double, P(C.c_double),
                                            P(C.c_double)]
    lib.lattice_sum_fit_t_scale_kernel.argtypes = [C.c_int32, C.c_double, C.c_int32, C.c_double, C.c_double,
                                                   C.c_double, P(C.c_double), P(C.c_double)]
    lib.lattice_sum_create.argtypes = [P(C.c_void_p), P(ls_params), P(ls_block), C.c_int32, C.c_void_p]
    lib.lattice_sum_add_defects.argtypes = [C.c_void_p, P(ls_defect), C.c_int64]
    lib.lattice_sum_rhosvd_reduce.argtypes = [C.c_void_p, C.c_double, P(C.c_int32), P(ls_tucker_info)]
    lib.lattice_sum_eval_slab.argtypes = [C.c_void_p, P(C.c_int64), C.c_int32, C.c_void_p, C.c_int32]
    lib.lattice_sum_get_factors.argtypes = [C.c_void_p, P(C.c_void_p), P(C.c_void_p), P(C.c_int32)]
    lib.lattice_sum_read.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_int64, P(C.c_int64)]
    lib.lattice_sum_profile.argtypes = [C.c_int32]
    lib.lattice_sum_profile_report.argtypes = [C.c_char_p, C.c_int64, P(C.c_int64)]
    lib.lattice_sum_eval_slab_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                                  P(C.c_int32), C.c_int64, P(C.c_int64), C.c_int32,
                                                  C.c_void_p, C.c_int32, C.c_void_p]
    lib.lattice_sum_batch_reduce.argtypes = [P(C.c_void_p), C.c_int32, C.c_double, P(ls_tucker_info)]
    lib.lattice_sum_gemm_nt.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_void_p,
                                        C.c_void_p]
    lib.lattice_sum_gemm_nt_mixed.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_void_p,
                                              C.c_int32, C.c_int32, C.c_void_p]
    lib.lattice_sum_jacobi_eig.argtypes = [C.c_void_p, C.c_int32, C.c_double, C.c_double, C.c_int32, C.c_int32,
                                           C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.lattice_sum_test_fail_alloc.argtypes = [C.c_int64]
    lib.lattice_sum_test_bounded_wait.argtypes = [C.c_int32, C.c_int64, C.c_void_p]
    lib.lattice_sum_svd_rows.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_double, C.c_int32, C.c_void_p,
                                         C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.lattice_sum_cache_clear.argtypes = []
    lib.lattice_sum_destroy.argtypes = [C.c_void_p]
    lib.lattice_sum_destroy.restype = None
    lib.lattice_sum_last_error.argtypes = [C.c_void_p]
    lib.lattice_sum_last_error.restype = C.c_char_p
    for name in EXPORTED:
        if name not in ("lattice_sum_destroy", "lattice_sum_last_error"):
            getattr(lib, name).restype = C.c_int
    return lib


_LIB: Optional[C.CDLL] = None


def lib() -> C.CDLL:
    global _LIB
    if _LIB is None:
        _LIB = load_library()
    return _LIB


def _check(rc, ctx=None):
    if rc != LS_OK:
        msg = lib().lattice_sum_last_error(ctx).decode(errors="replace")
        raise LatticeSumError(rc, msg)


def profile(enable: bool):
    """Start (clearing the trace) or stop the library's per-step event tracing."""
    _check(lib().lattice_sum_profile(1 if enable else 0))


def profile_report() -> dict:
    """Per-step device times, kernel-launch count and copy bytes since the
    last ``profile(True)``."""
    import json
    need = C.c_int64()
    _check(lib().lattice_sum_profile_report(None, 0, C.byref(need)))
    buf = C.create_string_buffer(need.value + 64)
    _check(lib().lattice_sum_profile_report(buf, need.value + 64, None))
    return json.loads(buf.value.decode())


def eval_slab_noalloc(Z, core, ranks, N, z_index, out_ptr, out_dtype=LS_OUT_F64, stream=None):
    """Slab values from caller-owned Tucker factors (device pointers) with no
    device allocation inside the library."""
    r = (C.c_int32 * 3)(*[int(x) for x in ranks])
    z = (C.c_int64 * max(len(z_index), 1))(*[int(x) for x in z_index])
    _check(lib().lattice_sum_eval_slab_noalloc(C.c_void_p(Z[0]), C.c_void_p(Z[1]), C.c_void_p(Z[2]),
                                               C.c_void_p(core), r, int(N), z, len(z_index),
                                               C.c_void_p(out_ptr), out_dtype,
                                               C.c_void_p(stream) if stream else None))


def cache_clear() -> int:
    """lattice_sum_cache_clear: frees the reference-vector cache; returns the entries freed."""
    rc = lib().lattice_sum_cache_clear()
    if rc < 0:
        _check(rc)
    return rc


def batch_reduce(contexts, eps: float):
    """RHOSVD of several LatticeSum contexts in one call (the batched form);
    returns their info dicts."""
    n = len(contexts)
    arr = (C.c_void_p * n)(*[c.ctx.value for c in contexts])
    infos = (ls_tucker_info * n)()
    rc = lib().lattice_sum_batch_reduce(arr, n, float(eps), infos)
    if rc != LS_OK:
        raise LatticeSumError(rc, lib().lattice_sum_last_error(None).decode(errors="replace"))
    out = []
    for c, inf in zip(contexts, infos):
        c.info = inf.as_dict()
        out.append(c.info)
    return out


def gemm_nt(A, B):
    """D = A B^T for float64 CUDA tensors (A: M x K, B: N x K) in the library's FP64-grade
    exact-slice tensor-core arithmetic (lattice_sum_gemm_nt)."""
    import torch
    A = A.contiguous()
    B = B.contiguous()
    M, K = A.shape
    N, K2 = B.shape
    if K2 != K or A.dtype != torch.float64 or B.dtype != torch.float64:
        raise ValueError("gemm_nt: A (M x K) and B (N x K) must be float64 with the same K")
    D = torch.empty((M, N), dtype=torch.float64, device=A.device)
    _check(lib().lattice_sum_gemm_nt(C.c_void_p(A.data_ptr()), C.c_void_p(B.data_ptr()), C.c_int64(M),
                                     C.c_int64(N), C.c_int64(K), C.c_void_p(D.data_ptr()), None))
    return D


def gemm_nt_mixed(A, B, dtype=None, tile_n: int = 0):
    """D = A B^T for float64 CUDA tensors (A: M x K, B: N x K; K <= 4096 for float32 output) in the mixed slab
    evaluation's tensor-core arithmetic (lattice_sum_gemm_nt_mixed): two exact digits and two
    11-bit tails (FP16), the two leading levels accumulated exactly; `tile_n` 32/64/128 (0 = by size);
    D in `dtype` (torch.float32 or torch.float64, default float32)."""
    import torch
    A = A.contiguous()
    B = B.contiguous()
    M, K = A.shape
    N, K2 = B.shape
    if K != K2 or A.dtype != torch.float64 or B.dtype != torch.float64:
        raise ValueError("gemm_nt_mixed: A (M x K) and B (N x K) must be float64 with the same K")
    dtype = dtype or torch.float32
    D = torch.empty((M, N), dtype=dtype, device=A.device)
    _check(lib().lattice_sum_gemm_nt_mixed(C.c_void_p(A.data_ptr()), C.c_void_p(B.data_ptr()), C.c_int64(M),
                                           C.c_int64(N), C.c_int64(K), C.c_void_p(D.data_ptr()),
                                           C.c_int32(LS_OUT_F32 if dtype == torch.float32 else LS_OUT_F64),
                                           C.c_int32(tile_n), None))
    return D


def jacobi_eig(H, tol: float = 1e-7, abs_floor: float = 0.0, form: int = 2, max_sweeps: int = 0):
    """One run of the block Jacobi (lattice_sum_jacobi_eig) on a symmetric float64 CUDA tensor:
    returns (diagonal, V = I + F, sweeps); form 1 = cluster (shared memory), 2 = grid;
    max_sweeps 0 = the default limit (60)."""
    import torch
    H = H.contiguous()
    k = H.shape[0]
    D = torch.empty(k, dtype=torch.float64, device=H.device)
    V = torch.empty((k, k), dtype=torch.float64, device=H.device)
    sw = C.c_int32()
    _check(lib().lattice_sum_jacobi_eig(C.c_void_p(H.data_ptr()), C.c_int32(k), C.c_double(tol),
                                        C.c_double(abs_floor), C.c_int32(form), C.c_int32(max_sweeps),
                                        C.c_void_p(D.data_ptr()), C.c_void_p(V.data_ptr()), C.byref(sw), None))
    return D, V, sw.value


def svd_rows(B, tol: float = None, max_sweeps: int = 0):
    """One-sided Jacobi on the rows of a float64 CUDA tensor B (m x C) (lattice_sum_svd_rows):
    returns (squared row norms after convergence, rotation M, sweeps, rotations per sweep)."""
    import torch
    B = B.contiguous()
    m, Cc = B.shape
    if tol is None:
        tol = 8.0 * 2.0 ** -53 * Cc ** 0.5
    sig2 = torch.empty(m, dtype=torch.float64, device=B.device)
    M = torch.empty((m, m), dtype=torch.float64, device=B.device)
    sw = C.c_int32()
    rot = (C.c_int64 * 64)()
    _check(lib().lattice_sum_svd_rows(C.c_void_p(B.data_ptr()), C.c_int32(m), C.c_int32(Cc), C.c_double(tol),
                                      C.c_int32(max_sweeps), C.c_void_p(sig2.data_ptr()), C.c_void_p(M.data_ptr()), C.byref(sw), rot, None))
    return sig2, M, sw.value, [int(rot[k]) for k in range(sw.value)]


def test_fail_alloc(n: int):
    """lattice_sum_test_fail_alloc: the n-th context allocation from now fails (n < 0: off)."""
    _check(lib().lattice_sum_test_fail_alloc(C.c_int64(int(n))))


def test_bounded_wait(absent: int, spin_limit: int):
    """lattice_sum_test_bounded_wait: the return code (LS_OK or LS_ERR_TIMEOUT) of the probe."""
    return int(lib().lattice_sum_test_bounded_wait(C.c_int32(int(absent)), C.c_int64(int(spin_limit)), None))


def fit_t_scale(R: int, sinc_step: float, r_min: float, r_max: float, kappa: float = 0.0,
                kernel: int = LS_KERNEL_YUKAWA):
    s, e = C.c_double(), C.c_double()
    if kappa == 0.0 and kernel == LS_KERNEL_YUKAWA:
        _check(lib().lattice_sum_fit_t_scale(R, sinc_step, r_min, r_max, C.byref(s), C.byref(e)))
    else:
        _check(lib().lattice_sum_fit_t_scale_kernel(R, sinc_step, kernel, kappa, r_min, r_max, C.byref(s),
                                                    C.byref(e)))
    return s.value, e.value


def make_blocks(blocks) -> C.Array:
    arr = (ls_block * len(blocks))()
    for i, b in enumerate(blocks):
        arr[i].L[:] = [int(x) for x in b.L]
        arr[i].origin[:] = [float(x) for x in b.origin]
        arr[i].spacing[:] = [float(x) for x in b.spacing]
        arr[i].charge = float(b.charge)
    return arr


def make_defects(defects) -> C.Array:
    arr = (ls_defect * max(len(defects), 1))()
    for i, d in enumerate(defects):
        arr[i].kind = int(d.kind)
        arr[i].block = int(d.block)
        arr[i].site[:] = [int(x) for x in d.site]
        arr[i].extent[:] = [int(x) for x in d.extent]
        arr[i].pos[:] = [float(x) for x in d.pos]
        arr[i].charge = float(d.charge)
    return arr


_READ_DTYPE = {LS_READ_TERMS: np.int32}


class LatticeSum:
    """One lattice-sum context: create -> add_defects -> rhosvd_reduce ->
    eval_slab, each a direct call of the C ABI."""

    def __init__(self, N, box_lo, box_hi, R, sinc_step, t_scale, blocks, precision=LS_FP64, stream=None,
                 kappa=0.0, kernel=LS_KERNEL_YUKAWA, galerkin=False, flags=0, ref_eps=0.0):
        self._lib = lib()
        p = ls_params(int(N), float(box_lo), float(box_hi), int(R), float(sinc_step), float(t_scale),
                      int(precision), (LS_FLAG_GALERKIN if galerkin else 0) | int(flags), float(kappa), int(kernel),
                      float(ref_eps))
        self._blocks = make_blocks(blocks)
        ctx = C.c_void_p()
        rc = self._lib.lattice_sum_create(C.byref(ctx), C.byref(p), self._blocks, len(blocks),
                                          C.c_void_p(stream) if stream else None)
        if rc != LS_OK:
            raise LatticeSumError(rc, self._lib.lattice_sum_last_error(None).decode(errors="replace"))
        self.ctx = ctx
        self.N = int(N)
        self.info = None
        # what the context was created from (a checkpoint records it)
        self.params = {"N": int(N), "box_lo": float(box_lo), "box_hi": float(box_hi), "R": int(R),
                       "sinc_step": float(sinc_step), "t_scale": float(t_scale), "precision": int(precision),
                       "flags": int(p.flags), "kappa": float(kappa), "kernel": int(kernel), "ref_eps": float(ref_eps)}

    @classmethod
    def from_workload(cls, wl, t_scale, precision=LS_FP64, stream=None, flags=0, ref_eps=0.0):
        return cls(wl.N, wl.box_lo, wl.box_hi, wl.R, wl.sinc_step, t_scale, wl.blocks, precision, stream,
                   getattr(wl, "kappa", 0.0), getattr(wl, "kernel", LS_KERNEL_YUKAWA), getattr(wl, "galerkin", False),
                   flags, ref_eps)

    def add_defects(self, defects):
        """lattice_sum_add_defects for a sequence of Defect descriptions, or for an ls_defect
        array already built by make_defects (reused across calls without re-marshalling)."""
        if len(defects) == 0:
            return
        arr = defects if isinstance(defects, C.Array) else make_defects(defects)
        _check(self._lib.lattice_sum_add_defects(self.ctx, arr, len(defects)), self.ctx)

    def rhosvd_reduce(self, eps: float, forced_ranks: Optional[Sequence[int]] = None) -> dict:
        info = ls_tucker_info()
        fr = (C.c_int32 * 3)(*[int(x) for x in forced_ranks]) if forced_ranks is not None else None
        _check(self._lib.lattice_sum_rhosvd_reduce(self.ctx, float(eps), fr, C.byref(info)), self.ctx)
        self.info = info.as_dict()
        return self.info

    def eval_slab(self, z_index: Sequence[int], out_ptr: int, out_dtype=LS_OUT_F64):
        z = (C.c_int64 * max(len(z_index), 1))(*[int(x) for x in z_index])
        _check(self._lib.lattice_sum_eval_slab(self.ctx, z, len(z_index), C.c_void_p(out_ptr), out_dtype),
               self.ctx)

    def tune_eval(self, z_index, out) -> dict:
        """lattice_sum_tune_eval into the float32/float64 CUDA tensor `out` (len(z_index) x N x N):
        the evaluation with its products' tile widths measured and kept; returns the report."""
        import json
        import torch
        z = (C.c_int64 * max(len(z_index), 1))(*[int(x) for x in z_index])
        buf = C.create_string_buffer(4096)
        _check(self._lib.lattice_sum_tune_eval(self.ctx, z, len(z_index), C.c_void_p(out.data_ptr()),
                                               LS_OUT_F32 if out.dtype == torch.float32 else LS_OUT_F64, buf,
                                               C.c_int64(len(buf))), self.ctx)
        return json.loads(buf.value.decode())

    def eval_slab_torch(self, z_index, dtype=None, out=None):
        import torch
        dtype = dtype or torch.float64
        n = len(z_index)
        if out is None:
            out = torch.empty((n, self.N, self.N), dtype=dtype, device="cuda")
        self.eval_slab(z_index, out.data_ptr(), LS_OUT_F32 if dtype == torch.float32 else LS_OUT_F64)
        return out

    def read(self, what: int, mode: int = 0) -> np.ndarray:
        need = C.c_int64()
        _check(self._lib.lattice_sum_read(self.ctx, what, mode, None, 0, C.byref(need)), self.ctx)
        dt = _READ_DTYPE.get(what, np.float64)
        arr = np.empty(need.value // np.dtype(dt).itemsize, dtype=dt)
        _check(self._lib.lattice_sum_read(self.ctx, what, mode, arr.ctypes.data_as(C.c_void_p), need.value,
                                          None), self.ctx)
        return arr

    def read_into(self, what: int, mode: int, out) -> int:
        """lattice_sum_read into a caller-owned host array (numpy, or a CPU torch tensor, e.g. in
        pinned memory so that the copy runs at the link's DMA rate); returns the bytes read."""
        need = C.c_int64()
        _check(self._lib.lattice_sum_read(self.ctx, what, mode, None, 0, C.byref(need)), self.ctx)
        if hasattr(out, "data_ptr"):
            ptr, size = out.data_ptr(), out.numel() * out.element_size()
        else:
            ptr, size = out.ctypes.data, out.nbytes
        if size < need.value:
            raise LatticeSumError(LS_ERR_ARG, f"read_into: {size} bytes given, {need.value} needed")
        _check(self._lib.lattice_sum_read(self.ctx, what, mode, C.c_void_p(ptr), need.value, None), self.ctx)
        return need.value

    def als_refine(self, sweeps: int):
        """lattice_sum_als_refine: returns (history of ||core|| (sweeps + 1 values), info)."""
        hist = (C.c_double * (int(sweeps) + 1))()
        info = ls_tucker_info()
        _check(self._lib.lattice_sum_als_refine(self.ctx, int(sweeps), hist, C.byref(info)), self.ctx)
        self.info = info.as_dict()
        return [hist[i] for i in range(int(sweeps) + 1)], self.info

    def galerkin(self, basis):
        """lattice_sum_galerkin for three float64 CUDA tensors (nb x N), row k = g_k^l; returns the
        nb x nb Galerkin matrix (a float64 CUDA tensor)."""
        import torch
        basis = [b.contiguous() for b in basis]
        nb = basis[0].shape[0]
        V = torch.empty((nb, nb), dtype=torch.float64, device=basis[0].device)
        ptrs = (C.c_void_p * 3)(*[b.data_ptr() for b in basis])
        _check(self._lib.lattice_sum_galerkin(self.ctx, ptrs, nb, C.c_void_p(V.data_ptr())), self.ctx)
        return V

    def factors(self):
        Z = (C.c_void_p * 3)()
        core = C.c_void_p()
        r = (C.c_int32 * 3)()
        _check(self._lib.lattice_sum_get_factors(self.ctx, Z, C.byref(core), r), self.ctx)
        return [Z[i] for i in range(3)], core.value, list(r)

    def save(self, path: str, extra: Optional[dict] = None):
        """Checkpoint of a reduced context as a .npz file: the Tucker vectors Z_l ([r_l][N] each),
        the core ([r0][r1][r2]), the ranks, the singular values of each mode, the creation
        parameters and the reduction's info (JSON), and `extra` (JSON) if given. Everything is
        read back through lattice_sum_read; load_checkpoint restores it."""
        import json
        if self.info is None:
            raise LatticeSumError(LS_ERR_STATE, "save: the context is not reduced")
        ranks = [int(x) for x in self.info["r"]]
        arrays = {f"Z{l}": self.read(LS_READ_BASIS, l).reshape(ranks[l], self.N) for l in range(3)}
        arrays["core"] = self.read(LS_READ_CORE).reshape(ranks)
        for l in range(3):
            arrays[f"sigma{l}"] = self.read(LS_READ_SIGMA, l)
        arrays["ranks"] = np.asarray(ranks, dtype=np.int32)
        meta = {"format": "lattice_sum.tucker.v1", "params": self.params, "info": self.info, "extra": extra or {}}
        arrays["meta"] = np.frombuffer(json.dumps(meta).encode(), dtype=np.uint8)
        np.savez(path, **arrays)

    def close(self):
        if getattr(self, "ctx", None):
            self._lib.lattice_sum_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Checkpoint:
    """A Tucker result restored from LatticeSum.save: Z (three [r_l][N] arrays), core
    ([r0][r1][r2]), ranks, sigma (per mode), params, info and extra (dicts). Its slabs are
    evaluated on the GPU from device copies of the factors (eval_slab_torch)."""

    def __init__(self, arrays, meta):
        self.Z = [np.ascontiguousarray(arrays[f"Z{l}"]) for l in range(3)]
        self.core = np.ascontiguousarray(arrays["core"])
        self.ranks = [int(x) for x in arrays["ranks"]]
        self.sigma = [arrays[f"sigma{l}"] for l in range(3)]
        self.params = meta["params"]
        self.info = meta["info"]
        self.extra = meta.get("extra", {})
        self.N = int(self.params["N"])
        self._dev = None

    def device_factors(self):
        """The factors as float64 CUDA tensors (made once): ([Z0, Z1, Z2], core)."""
        import torch
        if self._dev is None:
            self._dev = ([torch.from_numpy(z).cuda() for z in self.Z], torch.from_numpy(self.core).cuda())
        return self._dev

    def eval_slab_torch(self, z_index, dtype=None, out=None):
        """Slabs z_index of the restored Tucker tensor (len x N x N, float64 or float32 CUDA
        tensor), through lattice_sum_eval_slab_noalloc on the device copies of the factors;
        its scratch limit applies (one slab's r0 (r1 + N) doubles)."""
        import torch
        dtype = dtype or torch.float64
        Z, core = self.device_factors()
        if out is None:
            out = torch.empty((len(z_index), self.N, self.N), dtype=dtype, device="cuda")
        eval_slab_noalloc([z.data_ptr() for z in Z], core.data_ptr(), self.ranks, self.N, z_index, out.data_ptr(),
                          LS_OUT_F32 if dtype == torch.float32 else LS_OUT_F64,
                          torch.cuda.current_stream().cuda_stream)
        return out


def load_checkpoint(path: str) -> Checkpoint:
    """Restores a checkpoint written by LatticeSum.save."""
    import json
    with np.load(path) as f:
        arrays = {k: f[k] for k in f.files}
    meta = json.loads(arrays.pop("meta").tobytes().decode())
    if meta.get("format") != "lattice_sum.tucker.v1":
        raise ValueError(f"{path}: not a lattice-sum Tucker checkpoint")
    return Checkpoint(arrays, meta)
