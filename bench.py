#!/usr/bin/env python
"""Throughput of the lattice-sum hot path on GB300: lattice potentials summed
per second, one step = create (reference vectors + assembled lattice sums) +
add_defects + rhosvd_reduce on one seeded synthetic workload. The default is
the workload the metric is quoted on: the step-shaped lattice (a 48x48x24 and
a 24^3 block, 3% vacancies, N = 4096, R = 28, eps = 1e-6), mixed path against
the plain FP64 GPU path on the same inputs.

Prints ONE JSON line (rank 0). ``--impl reference`` times the FP64 CPU
oracle on the host cores instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1411_1994_gb300 import workloads as W  # noqa: E402

METRIC = "lattice potentials summed/s (build+RHOSVD), mixed vs FP64 GPU at 1e-6 rel err"
FP64_PEAK_TFLOPS_DERIVED = 152 * 2 * 2 * 2.070e9 / 1e12   # SMs x DFMA/clk x flops x max clock
FP32_PEAK_TFLOPS_DERIVED = 152 * 128 * 2 * 2.070e9 / 1e12  # SMs x FFMA/clk x flops x max clock


def max_over_ranks(x, dist, device):
    """The largest of a per-rank number over all ranks of the process group (the slowest rank's
    time); x itself without one."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, units_per_rank, seconds_per_step):
    """Units of all ranks per second: every rank (one GPU each) runs its own replica of the
    workload, so the job processes world x units in the slowest rank's step time."""
    return world * units_per_rank / seconds_per_step


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="c3", choices=["c1", "c2", "c3", "c4", "c5"])
    ap.add_argument("--batch-items", type=int, default=256, help="c4: configurations in the batch")
    ap.add_argument("--batch-wave", type=int, default=32, help="c4: contexts reduced per batch_reduce call")
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--no-compare", action="store_true", help="skip the FP64-path comparison run")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    return ap.parse_args()


def load_peaks():
    """HBM GB/s and dense BF16 TFLOP/s: the measured figures of MEASURED_PEAKS.json, else the
    fallback figures of an earlier GB300 measurement (6800 GB/s, 1900 TFLOP/s burst), marked so."""
    try:
        p = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        if p.get("hbm_gbs") and p.get("bf16_tflops"):
            p["source"] = "measured (MEASURED_PEAKS.json)"
            return p
    except Exception:
        pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "source": "fallback (no MEASURED_PEAKS.json): 6.8 TB/s, 1.9 PFLOP/s bf16 burst"}


def workload(name):
    return {"c1": W.config1, "c2": W.config2, "c3": W.config3, "c5": W.config5}[name]()


def config_of(wl, args, extra=None):
    cfg = {"workload": wl.name, "N": wl.N, "R": wl.R, "eps": wl.eps, "sites": wl.n_sites,
           "defects": len(wl.defects), "units_per_step": wl.units, "box": [wl.box_lo, wl.box_hi],
           "path": args.precision, "l2": "flushed between steps (512 MB write outside the per-step events)"}
    if extra:
        cfg.update(extra)
    return cfg


# ---------------------------------------------------------------------------
# CPU oracle (baseline leg and --impl reference)
# ---------------------------------------------------------------------------

def oracle_step(wl, s):
    from oracle import lattice_oracle as O
    O.pipeline(wl, s, core=True)


# the oracle's core einsum is run in full below this many flops (2 r0 r1 r2 T); above it, on a
# sample of the terms and extrapolated (its time is linear in the number of terms)
FULL_CORE_FLOPS = 4e11
CORE_SAMPLE_TERMS = 1024
GRAM_SAMPLE_ROWS = 2048


def oracle_sample(wl, s, ranks=None):
    """One bounded oracle step on the host cores, as the CPU baseline of the workload.

    Small workloads: the whole oracle pipeline (quadrature, per-site window sums, dgesdd
    RHOSVD, core einsum). Where the core einsum is too large for a bounded sample (the step
    lattice: 2 r^3 T ~ 1.4e13 flop), everything but the core is timed in full and the core on
    its first CORE_SAMPLE_TERMS terms, scaled to all T terms. The 256^3 lattice: (a) + (b)
    (quadrature, window sums, normalisation) and the Gram matrix of mode 0 on a
    GRAM_SAMPLE_ROWS-row slice are timed; the rest is extrapolated at that product's rate:
    per mode the R-SVD of the N x C side matrix (6 N C^2 + 20 C^3 flop), the projection
    (2 N r C), and the core (2 r0 r1 r2 T), with r the ranks of the GPU reduction.

    Returns (seconds for one whole step, measured seconds, description of the sample)."""
    from oracle import lattice_oracle as O
    t0 = time.perf_counter()
    t, w = O.sinc_quadrature(wl.R, wl.sinc_step, s, wl.kappa, wl.kernel)
    g = O.generating_vectors(wl.N, wl.box_lo, wl.box_hi, t, w, wl.galerkin)
    cols, tcol, xi = O.canonical_terms(wl.N, wl.box_lo, wl.box_hi, g, wl.blocks, wl.defects)
    T = len(xi)
    C = [c.shape[0] for c in cols]
    if wl.N >= 16384:
        ncols, _, _ = O.normalise_terms(cols, tcol, xi)
        t1 = time.perf_counter()
        a = np.ascontiguousarray(ncols[0][:, :GRAM_SAMPLE_ROWS])
        a @ a.T
        t2 = time.perf_counter()
        rate = 2.0 * GRAM_SAMPLE_ROWS * C[0] ** 2 / (t2 - t1)
        r = ranks or [min(c, 1) for c in C]
        rest = sum(6.0 * wl.N * c * c + 20.0 * c ** 3 + 2.0 * wl.N * rr * c for c, rr in zip(C, r))
        rest += 2.0 * r[0] * r[1] * r[2] * T
        total = (t1 - t0) + rest / rate
        how = (f"extrapolated: (a)+(b) timed ({t1 - t0:.2f} s), Gram of mode 0 on {GRAM_SAMPLE_ROWS} of "
               f"{wl.N} rows timed ({t2 - t1:.2f} s, {rate / 1e9:.1f} GFLOP/s); per mode 6NC^2+20C^3 "
               f"(R-SVD) + 2NrC (projection) and 2 r0 r1 r2 T (core) at that rate, r = {r} from the GPU")
        return total, t2 - t0, how
    res = O.rhosvd(cols, tcol, xi, wl.eps, core=False)
    r = res["r"]
    core_flops = 2.0 * r[0] * r[1] * r[2] * T
    if core_flops <= FULL_CORE_FLOPS:
        O.core_tensor(res["P"], tcol, res["xi"])
        t2 = time.perf_counter()
        return t2 - t0, t2 - t0, "full oracle pipeline (quadrature, per-site window sums, dgesdd RHOSVD, core einsum)"
    t1 = time.perf_counter()
    n = min(CORE_SAMPLE_TERMS, T)
    O.core_tensor(res["P"], tcol[:n], res["xi"][:n])
    t2 = time.perf_counter()
    total = (t1 - t0) + (t2 - t1) * T / n
    how = (f"(a)+(b)+(c1)+(c2) timed in full ({t1 - t0:.2f} s: quadrature, per-site window sums, dgesdd "
           f"RHOSVD, projections); core einsum timed on {n} of {T} terms ({t2 - t1:.2f} s) and scaled to "
           f"all terms (extrapolated, ranks {r})")
    return total, t2 - t0, how


def time_oracle(wl, s, budget_s, ranks=None):
    """Bounded oracle samples for budget_s seconds of host time (at least one)."""
    totals, measured, how = [], 0.0, ""
    t_end = time.perf_counter() + budget_s
    while not totals or time.perf_counter() < t_end:
        tot, m, how = oracle_sample(wl, s, ranks)
        totals.append(tot)
        measured += m
        if len(totals) >= 50:
            break
    return totals, measured, how


def cores_used():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_reference_batch(args):
    """The oracle on the batch of config 4: each step a bounded sample (~15 s) of the items,
    taken in order and continued from step to step; units and time summed over the sample."""
    from oracle import lattice_oracle as O
    items = W.config4(args.batch_items)
    nxt = 0

    def sample(budget_s):
        nonlocal nxt
        units, secs, n = 0, 0.0, 0
        while secs < budget_s and n < len(items):
            w = items[nxt % len(items)]
            s, _ = O.fit_t_scale(w.R, w.sinc_step, w.r_min, O.default_r_max(w))
            t0 = time.perf_counter()
            oracle_step(w, s)
            secs += time.perf_counter() - t0
            units += w.units
            nxt += 1
            n += 1
        return units, secs, n

    for _ in range(args.warmup):
        sample(3.0)
    tot_u, tot_s, tot_n = 0, 0.0, 0
    for _ in range(args.steps):
        u, t, n = sample(15.0)
        tot_u, tot_s, tot_n = tot_u + u, tot_s + t, tot_n + n
    value = tot_u / tot_s
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "potentials/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded)",
            "config": {"workload": f"c4_batch{len(items)}_L8-48_N512-2048_R20-28", "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "potentials/s", "cores": cores_used(), "kind": "oracle",
                             "sample": f"{tot_n} of the {len(items)} batch items over {args.steps} steps "
                                       "(full oracle pipelines, in order)"},
            "e2e": {"value": value, "unit": "potentials/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    if args.workload == "c4":
        return run_reference_batch(args)
    wl = workload(args.workload)
    from oracle import lattice_oracle as O
    s, _ = O.fit_t_scale(wl.R, wl.sinc_step, wl.r_min, O.default_r_max(wl))
    for _ in range(args.warmup):
        oracle_sample(wl, s)
    totals, how = [], ""
    for _ in range(args.steps):
        tot, _, how = oracle_sample(wl, s)
        totals.append(tot)
    ms = 1e3 * sum(totals) / len(totals)
    value = wl.units / (ms / 1e3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "potentials/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
            "config": config_of(wl, args, {"l2": "n/a (CPU)", "path": "fp64 oracle (CPU)"}),
            "cpu_baseline": {"value": value, "unit": "potentials/s", "cores": cores_used(), "kind": "oracle",
                             "sample": f"{args.steps} samples of {wl.name}, each: {how}"},
            "e2e": {"value": value, "unit": "potentials/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def oracle_errors(wl, s, zs, xs, rows):
    """Error of each path's Tucker result against the oracle on sampled grid rows: row (x, :, z)
    of the untruncated canonical tensor sum_t xi_t a0[c0(t)] (x) a1[c1(t)] (x) a2[c2(t)] is exact
    in the oracle's terms (Eq. Can_LatticeSum_full), one weighted sum of mode-1 vectors per row.
    Reports the relative L2 error over the sampled values, the largest absolute error, and that
    error relative to the largest sampled value."""
    from oracle import lattice_oracle as O
    t, w = O.sinc_quadrature(wl.R, wl.sinc_step, s, wl.kappa, wl.kernel)
    g = O.generating_vectors(wl.N, wl.box_lo, wl.box_hi, t, w, wl.galerkin)
    cols, tcol, xi = O.canonical_terms(wl.N, wl.box_lo, wl.box_hi, g, wl.blocks, wl.defects)
    ncols, _, xin = O.normalise_terms(cols, tcol, xi)
    ref = []
    for z, xx in zip(zs, xs):
        part = []
        for x in xx:
            wt = xin * ncols[0][tcol[:, 0], x] * ncols[2][tcol[:, 2], z]
            part.append(np.bincount(tcol[:, 1], weights=wt, minlength=ncols[1].shape[0]) @ ncols[1])
        ref.append(np.stack(part))
    ref = np.stack(ref)
    out = {"reference": "oracle: exact rows of the untruncated canonical tensor (FP64)",
           "points": int(ref.size), "slabs": list(zs), "rows_per_slab": len(xs[0]), "eps": wl.eps}
    for name, got in rows.items():
        d = got - ref
        out[name] = {"rel_l2": float(np.linalg.norm(d) / np.linalg.norm(ref)),
                     "max_abs": float(np.abs(d).max()),
                     "max_rel_to_max": float(np.abs(d).max() / np.abs(ref).max())}
    return out


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        try:
            with open(self.path) as f:
                for ln in f:
                    p = [x.strip() for x in ln.split(",")]
                    if len(p) >= 9:
                        rows.append(p)
            os.unlink(self.path)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        loaded = [x for x in sm if mx and x >= 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# roofline of the dominant step
# ---------------------------------------------------------------------------

# what the mixed path computes in: FP64-grade (exact BF16 slices, 2^-53) Gram, CholeskyQR2 and
# projection; the eigen-solver's rotations in FP32 (hi/lo FP32 diagonal) with the eigenvalues
# taken as Rayleigh quotients of an FP64-grade re-projection; core and slabs as BF16x-split
# (two exact digits + two tails, FP16) tensor-core products with FP32 accumulation
MIXED_DTYPE = ("f64-grade Gram/CholeskyQR2/projection (exact bf16 slices) + f32 Jacobi with f64-grade "
               "Rayleigh quotients + fp16 digit+tail tensor-core core and slabs (f32 acc)")


def step_flops(name, info, N):
    """Algorithmic FP64 / tensor flops of one pipeline step (all three modes): a
    symmetric product (Gram matrix) counts its N C^2 distinct multiply-adds
    once, a triangular one (L^{-1} Y) its N r^2 / 2."""
    C, r, T, k = info["C"], info["r"], info["T"], info["pivots"]
    if name == "gram":
        return sum(1.0 * N * c * (c + 1) for c in C)
    if name == "pchol":
        # k pivot steps of C dot products of length <= k, then H = L^T L (k x k, length C)
        return sum(1.0 * C[a] * k[a] ** 2 + 1.0 * C[a] * k[a] * (k[a] + 1) for a in range(3))
    if name == "basis":
        # Vg = L U (C x k x k), Y = Vg^T A_w (r x C x N)
        return sum(2.0 * C[a] * k[a] ** 2 + 2.0 * N * C[a] * r[a] for a in range(3))
    if name == "cholqr2":
        # two passes: G = Y Y^T, Cholesky, triangular inverse, L^{-1} Y
        return sum(2 * (1.0 * N * r[a] * (r[a] + 1) + 2.0 * r[a] ** 3 / 3.0 + 1.0 * N * r[a] ** 2) for a in range(3))
    if name == "project":
        return sum(2.0 * N * r[a] * C[a] for a in range(3))
    if name == "core":
        # two exact steps: grouped step 1 (2 r1 r2 T) + dense step 2 (2 r0 r1 r2 C0)
        return 2.0 * r[1] * r[2] * T + 2.0 * r[0] * r[1] * r[2] * C[0]
    if name == "jacobi":
        # each applied rotation of the k x k matrix H = L^T L updates two rows and two columns
        # (~2 k entries x 3 flop x 2) and two columns of the accumulated rotation (2 k x 3 flop);
        # the rotations run in FP32 (the FP64 re-projection products are not counted)
        return sum(18.0 * k[a] * info["rotations"][a] for a in range(3))
    return None


def traffic_record(step, profiles_dir=None, sources_dir=None):
    """DRAM bytes per launch of the step's kernel from the committed ncu summary under profiles/
    (a `traffic_record:` line: step | kernel | sources | sha256 of the sources | bytes), taken only
    while the sources hash as they did when the counters were captured; else None."""
    import glob
    import hashlib
    here = os.path.dirname(os.path.abspath(__file__))
    profiles_dir = profiles_dir or os.path.join(here, "profiles")
    sources_dir = sources_dir or os.path.join(here, "paper_1411_1994_gb300", "csrc")
    for path in sorted(glob.glob(os.path.join(profiles_dir, "*.md"))):
        for line in open(path):
            if not line.startswith("traffic_record:"):
                continue
            parts = [x.strip() for x in line[len("traffic_record:"):].split("|")]
            if len(parts) != 5 or parts[0] != step:
                continue
            h = hashlib.sha256()
            for f in parts[2].split("+"):
                src = os.path.join(sources_dir, f)
                if not os.path.exists(src):
                    return None
                h.update(open(src, "rb").read())
            return float(parts[4]) if h.hexdigest() == parts[3] else None
    return None


def roofline(report, info, N, steps, precision, peaks):
    st = report.get("steps", {})
    if not st:
        return None
    # names with a dot are parts of another step (reported, not ranked)
    name = max((k for k in st if "." not in k), key=lambda k: st[k]["ms"])
    ms_launch = st[name]["ms"] / max(st[name]["launches"], 1)
    launches_per_step = st[name]["launches"] / max(steps, 1)
    fl = step_flops(name, info, N)
    out = {"kernel": name, "ms_per_launch": ms_launch, "launches_per_step": launches_per_step}
    if fl is None:
        out.update({"bound": "latency", "achieved": None, "peak": None, "unit": None, "frac": None, "traffic": None})
        return out
    achieved = fl / launches_per_step / (ms_launch * 1e-3) / 1e12
    tensor = precision == "mixed" and name in ("project", "core")
    if name == "jacobi":
        peak = FP32_PEAK_TFLOPS_DERIVED
        out.update({"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "traffic": traffic_record(name),
                    "traffic_source": "k_jacobi_gblk, one ncu capture (profiles/k_jacobi_gblk_c3.md), bytes per launch",
                    "peak_source": "derived: 152 SMs x 128 FFMA/clk x 2 flop x 2.07 GHz (FP32 on CUDA cores; "
                                   "an FFMA probe measured 73 TFLOP/s); the rotations are sequential rounds, "
                                   "so this step is bound by latency, not by this peak"})
    elif not tensor:
        peak = FP64_PEAK_TFLOPS_DERIVED
        out.update({"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "traffic": None,
                    "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (FP64 on CUDA cores; "
                                   "a DFMA probe measured 1.255 TFLOP/s)"})
    else:
        peak = peaks.get("bf16_tflops")
        out.update({"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak if peak else None, "traffic": None,
                    "peak_source": f"bf16 burst, {peaks.get('source')}; the digit MMAs per k16 step "
                                   "of the exact split products are counted as overhead, not as work"})
    return out


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_batch(args, torch, B, L):
    """The batched form (config 4): one step reduces every seeded configuration of the batch,
    lattice_sum_batch_reduce over waves of contexts (mixed path), against the same items
    reduced one at a time on the FP64 path."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    B.build()
    items = W.config4(args.batch_items)
    units = sum(w.units for w in items)
    scale = {}
    for w in items:
        key = (w.R, w.sinc_step, w.r_min, w.box_hi - w.box_lo)
        if key not in scale:
            scale[key] = L.fit_t_scale(w.R, w.sinc_step, w.r_min, math.sqrt(3.0) * (w.box_hi - w.box_lo))[0]
    s_of = [scale[(w.R, w.sinc_step, w.r_min, w.box_hi - w.box_lo)] for w in items]
    stream = torch.cuda.Stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    # each item's defect list as the C ABI takes it, built once (host input data)
    defects_c = [L.make_defects(w.defects) if w.defects else [] for w in items]

    def step(batched):
        infos = []
        for j0 in range(0, len(items), args.batch_wave):
            ctxs = []
            for j, (w, s) in enumerate(zip(items[j0:j0 + args.batch_wave], s_of[j0:j0 + args.batch_wave])):
                c = L.LatticeSum.from_workload(w, s, L.LS_MIXED if batched else L.LS_FP64, stream=stream.cuda_stream)
                c.add_defects(defects_c[j0 + j])
                ctxs.append(c)
            if batched:
                infos += L.batch_reduce(ctxs, items[0].eps)
            else:
                infos += [c.rhosvd_reduce(w.eps) for c, w in zip(ctxs, items[j0:j0 + args.batch_wave])]
            for c in ctxs:
                c.close()
        return infos

    def timed(batched, sample_clocks):
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                step(batched)
        torch.cuda.synchronize()
        clocks = ClockSampler(local) if sample_clocks else None
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        L.profile(True)
        if clocks:
            clocks.start()
        with torch.cuda.stream(stream):
            for k in range(args.steps):
                flush.fill_(k & 0xFF)
                ev[k][0].record(stream)
                infos = step(batched)
                ev[k][1].record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop() if clocks else None
        L.profile(False)
        rep = L.profile_report()
        total_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), dist, "cuda")
        ms = total_ms / args.steps
        return {"value": whole_job_rate(world, units, ms / 1e3), "ms_per_step": ms, "infos": infos, "report": rep,
                "clocks": clk}

    head = timed(True, True)
    seq = None if args.no_compare else timed(False, False)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    rs = [i["r"] for i in head["infos"]]
    line = {
        "metric": METRIC, "value": head["value"], "unit": "potentials/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": MIXED_DTYPE,
        "data": "synthetic (seeded)",
        "config": {"workload": f"c4_batch{len(items)}_L8-48_N512-2048_R20-28", "items": len(items),
                   "units_per_step": units, "wave": args.batch_wave, "eps": items[0].eps,
                   "l2": "flushed between steps (512 MB write outside the per-step events)",
                   "parallelism": f"replicas x{world}", "rank_range": [min(min(r) for r in rs), max(max(r) for r in rs)],
                   "columns_range": [min(min(i["C"]) for i in head["infos"]), max(max(i["C"]) for i in head["infos"])]},
        "gpu_launches": int(head["report"].get("kernel_launches", 0)),
        "clocks": head["clocks"],
        "steps_ms": {k: v["ms"] / args.steps for k, v in head["report"].get("steps", {}).items()},
    }
    if seq is not None:
        line["fp64_sequential"] = {"value": seq["value"], "ms_per_step": seq["ms_per_step"]}
        line["batched_over_sequential_fp64"] = head["value"] / seq["value"]
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "c4":
        import torch
        from paper_1411_1994_gb300 import build as B
        from paper_1411_1994_gb300 import lattice_sum as L
        if not torch.cuda.is_available():
            raise SystemExit("bench.py needs a CUDA GPU")
        return run_batch(args, torch, B, L)
    import torch
    from paper_1411_1994_gb300 import build as B
    from paper_1411_1994_gb300 import lattice_sum as L

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    B.build()
    wl = workload(args.workload)
    # the 256^3 workload: its core is ~87 GB (FP64) and its FP64-path core ~7e14 DFMA, so it
    # runs the mixed path alone, reads no factors back to the host and evaluates its 128
    # slabs in chunks of 16 (17 GB of FP32 output at a time)
    large = args.workload == "c5"
    if large:
        args.no_compare = True
    s, _ = L.fit_t_scale(wl.R, wl.sinc_step, wl.r_min, math.sqrt(3.0) * (wl.box_hi - wl.box_lo))
    stream = torch.cuda.Stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    peaks = load_peaks()

    # the defect list as the C ABI takes it, built once (host input data, like the workload)
    defects_c = L.make_defects(wl.defects) if wl.defects else []

    def step(prec):
        ls = L.LatticeSum.from_workload(wl, s, prec, stream=stream.cuda_stream)
        ls.add_defects(defects_c)
        info = ls.rhosvd_reduce(wl.eps)
        ls.close()
        return info

    def timed(prec, sample_clocks):
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                info = step(prec)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        clocks = ClockSampler(local) if sample_clocks else None
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        L.profile(True)
        if clocks:
            clocks.start()
        t_wall = time.perf_counter()
        with torch.cuda.stream(stream):
            for k in range(args.steps):
                flush.fill_(k & 0xFF)
                ev[k][0].record(stream)
                info = step(prec)
                ev[k][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t_wall
        clk = clocks.stop() if clocks else None
        L.profile(False)
        report = L.profile_report()
        total_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), dist, "cuda")
        if dist:
            dist.barrier()
        ms = total_ms / args.steps
        return {"value": whole_job_rate(world, wl.units, ms / 1e3), "ms_per_step": ms, "info": info, "report": report,
                "clocks": clk, "wall": wall}

    def e2e(prec):
        """Same metric through the public API with host inputs and the Tucker factors read back
        into pinned host buffers (allocated once, before the timed steps, at the sizes of an
        untimed first run)."""
        ls = L.LatticeSum.from_workload(wl, s, prec, stream=stream.cuda_stream)
        ls.add_defects(defects_c)
        r = ls.rhosvd_reduce(wl.eps)["r"]
        ls.close()
        host = [torch.empty(int(r[a]) * wl.N, dtype=torch.float64, pin_memory=True) for a in range(3)]
        host.append(torch.empty(int(r[0]) * int(r[1]) * int(r[2]), dtype=torch.float64, pin_memory=True))
        times = []
        L.profile(True)
        for k in range(max(3, args.steps // 2)):
            flush.fill_(k & 0xFF)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ls = L.LatticeSum.from_workload(wl, s, prec, stream=stream.cuda_stream)
            ls.add_defects(defects_c)
            ls.rhosvd_reduce(wl.eps)
            for a in range(3):
                ls.read_into(L.LS_READ_BASIS, a, host[a])
            ls.read_into(L.LS_READ_CORE, 0, host[3])
            ls.close()
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        L.profile(False)
        rep = L.profile_report()
        n = len(times)
        mean_s = max_over_ranks(sum(times) / n, dist, "cuda")
        return {"value": whole_job_rate(world, wl.units, mean_s), "unit": "potentials/s",
                "h2d_bytes_per_step": int(rep["h2d_bytes"] // n), "d2h_bytes_per_step": int(rep["d2h_bytes"] // n)}

    def eval_timing(prec):
        """Step (d) on its own: the workload's slabs from one reduced context, FP32 output on the
        mixed path (FP64 on the FP64 path), CUDA events on the library stream after warm-up; then
        one traced pass for the split between the small products and the slab product."""
        zs = list(wl.slabs or [wl.N // 2])
        f32 = prec == L.LS_MIXED
        ls = L.LatticeSum.from_workload(wl, s, prec, stream=stream.cuda_stream)
        ls.add_defects(wl.defects)
        info = ls.rhosvd_reduce(wl.eps)
        r0, r1, r2 = info["r"]
        chunk = 16 if large else len(zs)
        out = torch.empty((chunk, wl.N, wl.N), dtype=torch.float32 if f32 else torch.float64, device="cuda")
        reps, warm = (2, 1) if large else (5, 3)
        # the products' tile widths, measured once on the first chunk (outside the timing)
        tune = None
        if prec == L.LS_MIXED:
            first = zs[:chunk]
            with torch.cuda.stream(stream):
                tune = ls.tune_eval(first, out[:len(first)])

        def all_slabs():
            for c0 in range(0, len(zs), chunk):
                part = zs[c0:c0 + chunk]
                ls.eval_slab_torch(part, dtype=out.dtype, out=out[:len(part)])

        with torch.cuda.stream(stream):
            for _ in range(warm):
                all_slabs()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                all_slabs()
            e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        L.profile(True)
        with torch.cuda.stream(stream):
            for _ in range(reps):
                all_slabs()
        torch.cuda.synchronize()
        L.profile(False)
        steps = L.profile_report().get("steps", {})
        ls.close()
        ns, N = len(zs), wl.N
        pts = ns * N * N
        written = pts * out.element_size()
        hbm = peaks.get("hbm_gbs")
        bf16 = peaks.get("bf16_tflops")
        # algorithmic flops per slab: 2 r0 r1 r2 (M) + 2 N r0 r1 (T) + 2 N^2 r0 (S)
        flops = ns * (2.0 * r0 * r1 * r2 + 2.0 * N * r0 * r1 + 2.0 * N * N * r0)
        res = {"slabs": ns, "N": N, "ranks": [r0, r1, r2], "dtype": "f32" if f32 else "f64", "ms": ms,
               "tile_n_tuned": tune,
               "points_per_s": pts / (ms * 1e-3), "bytes_written": written,
               "write_gbs": written / (ms * 1e-3) / 1e9, "algorithmic_tflops": flops / (ms * 1e-3) / 1e12,
               "steps_ms": {k: v["ms"] / reps for k, v in steps.items() if k.startswith("eval")}}
        sl = steps.get("eval.slab")
        if sl and f32:
            # the slab product S_s = T_s x1 Z0 alone: its flops, its writes, and the tensor-pipe
            # work of its 11 FP16 products a k-step (the split form's overhead, not counted as work)
            t = sl["ms"] / reps * 1e-3
            fl = ns * 2.0 * N * N * r0
            ach = fl / t / 1e12
            res["slab_product"] = {
                "kernel": "k_dt_gemm (S_s = T_s x1 Z0)", "ms": t * 1e3, "launches": sl["kernels"] / reps,
                "achieved_tflops": ach, "bf16_peak_tflops": bf16, "frac_of_measured_bf16": ach / bf16 if bf16 else None,
                "products_per_kstep": 11, "tensor_pipe_frac": 11 * ach / bf16 if bf16 else None,
                "write_gbs": written / t / 1e9, "frac_of_measured_hbm": written / t / 1e9 / hbm if hbm else None}
        return res

    def gpu_rows(prec, zs, xs):
        """Rows xs[k] of slab zs[k] of the path's Tucker result, FP64 output, on the host."""
        ls = L.LatticeSum.from_workload(wl, s, prec, stream=stream.cuda_stream)
        ls.add_defects(defects_c)
        ls.rhosvd_reduce(wl.eps)
        got = []
        with torch.cuda.stream(stream):
            for z, xx in zip(zs, xs):
                sl = ls.eval_slab_torch([z])
                got.append(sl[0, xx].cpu().numpy())
                del sl
        torch.cuda.synchronize()
        ls.close()
        return np.stack(got)

    head_prec = L.LS_MIXED if args.precision == "mixed" else L.LS_FP64
    head = timed(head_prec, True)
    head_e2e = None if large else e2e(head_prec)
    head_eval = eval_timing(head_prec)
    other = None
    agreement = None
    if args.precision == "mixed" and not args.no_compare:
        other = timed(L.LS_FP64, False)
        # accuracy of the mixed path against the FP64 path at the same ranks (outside the timed region)
        a = L.LatticeSum.from_workload(wl, s, L.LS_FP64)
        a.add_defects(wl.defects)
        ia = a.rhosvd_reduce(wl.eps)
        b = L.LatticeSum.from_workload(wl, s, L.LS_MIXED)
        b.add_defects(wl.defects)
        b.rhosvd_reduce(wl.eps, forced_ranks=ia["r"])
        z = (wl.slabs or [wl.N // 2])[:8]
        sa = a.eval_slab_torch(z)
        sb = b.eval_slab_torch(z)
        agreement = float(torch.linalg.norm(sb - sa) / torch.linalg.norm(sa))
        a.close()
        b.close()

    # sampled grid rows of each path's Tucker result (FP64 output), for the error against the
    # oracle's exact rows of the untruncated canonical tensor (outside every timed region)
    acc_z = [int(z) for z in (wl.slabs or [wl.N // 2])[:(4 if large else 8)]]
    rng = np.random.default_rng(wl.N)
    acc_x = [[int(x) for x in rng.choice(wl.N, size=(8 if large else 16), replace=False)] for _ in acc_z]
    rows = {args.precision: gpu_rows(head_prec, acc_z, acc_x)}
    if other is not None:
        rows["fp64"] = gpu_rows(L.LS_FP64, acc_z, acc_x)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    info = head["info"]
    cpu = None
    error_vs_oracle = None
    if not args.no_cpu_baseline and world == 1:
        totals, measured, how = time_oracle(wl, s, args.cpu_seconds, ranks=info["r"])
        mean_s = statistics.mean(totals)
        cpu = {"value": wl.units / mean_s, "unit": "potentials/s", "cores": cores_used(), "kind": "oracle",
               "sample": f"{len(totals)} samples of {wl.name} on the host cores ({measured:.1f} s of host time; "
                         f"{mean_s:.2f} s per step), each: {how}"}
        error_vs_oracle = oracle_errors(wl, s, acc_z, acc_x, rows)
    line = {
        "metric": METRIC, "value": head["value"], "unit": "potentials/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": ("f64 (Gram, CholeskyQR2, projection: f64-grade exact bf16 slices; singular values: f64 "
                  "one-sided Jacobi; core and slabs: f64 CUDA cores)") if args.precision == "fp64" else MIXED_DTYPE,
        "data": "synthetic (seeded)",
        "config": config_of(wl, args, {"parallelism": f"replicas x{world}", "ranks": info["r"],
                                       "columns": info["C"], "terms": info["T"], "jacobi_sweeps": info["sweeps"]}),
        "roofline": roofline(head["report"], info, wl.N, args.steps, args.precision, peaks),
        "cpu_baseline": cpu,
        "e2e": head_e2e,
        "gpu_launches": int(head["report"].get("kernel_launches", 0)),
        "clocks": head["clocks"],
        "steps_ms": {k: v["ms"] / args.steps for k, v in head["report"].get("steps", {}).items()},
        "wall_s_timed_region": head["wall"],
        "eval_slab": head_eval,
    }
    if large:
        line["large_case_note"] = ("mixed path only (the FP64-path core is ~7e14 DFMA); no e2e read-back of the "
                                   "~87 GB core; the CPU baseline is an extrapolation from a timed sample (see "
                                   "cpu_baseline.sample); slabs evaluated 16 at a time")
    if error_vs_oracle is not None:
        line["error_vs_oracle"] = error_vs_oracle
    if other is not None:
        line["fp64_path"] = {"value": other["value"], "ms_per_step": other["ms_per_step"],
                             "steps_ms": {k: v["ms"] / args.steps for k, v in other["report"].get("steps", {}).items()}}
        line["mixed_over_fp64"] = head["value"] / other["value"]
        line["mixed_vs_fp64_slab_rel_l2"] = agreement
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
