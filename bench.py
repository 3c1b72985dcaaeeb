#!/usr/bin/env python3
"""Time-to-solution of preconditioned block BiCGGR (arXiv:0907.3261) on one or more GB300s.

Workload (the paper's lattice, Sec. 3.1, with synthetic links in place of its configurations):
16^3 x 32 periodic lattice, links SU3proj(1 + 0.2 G) (seed 0), c_SW = 1.0, kappa = 0.134, L = 12
Z4-noise sources (seed 1 + rank), Jacobi j = 12 (the paper's recommended L = 12, j >= 12, Sec. 3.3),
X_0 = 0, R~_0 = R_0, tolerance 1e-12 on the recursive residual and then on the true residual.
One step = one complete solve through the C-ABI.  By default the Jacobi sweeps run in double-float
arithmetic (FP32 operator, spinors as FP32 pairs) and so do the direction recurrences, while the
products with A, the X and R updates, the L x L solves and the true residual stay FP64
(--precision df_dirs; fp64 is the plain FP64 method, df double-float sweeps only, mixed FP32 sweeps,
bf16 FP32 sweeps on BF16-stored blocks).  The run also times the other forms on the same workload
for comparison.  kappa = 0.134
is the largest value of the 0.001-step sweep from 0.115 at which the L = 1, j = 0 solve still
converges (660 iterations); at 0.135 it no longer does.

Prints one JSON line on stdout.  --impl reference times the FP64 oracle on the host cores instead.
With torchrun each rank solves its own sources (independent problems, no collective on the data
path); the timing is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DIMS = (16, 16, 16, 32)
L_RHS = 12
J_JACOBI = 12
KAPPA = 0.134
CSW = 1.0
LINK_EPS = 0.2
TOL = 1e-12
# Outer iterations the FP64 method takes on this workload (L = 12, j = 12, kappa = 0.134): used
# only by the reference arm, whose oracle cannot finish the solve within a bench run, to
# extrapolate its measured outer iterations.
WORKLOAD_ITERS = 36

PRECISIONS = {"fp64": 0, "mixed": 1, "bf16": 3, "df": 4, "df_dirs": 5}   # bbicggr_opts.precision
FORM_NAMES = {"fp64": "plain FP64 Jacobi", "mixed": "mixed: FP32 Jacobi preconditioner",
              "bf16": "mixed: Jacobi preconditioner on BF16-stored blocks",
              "df": "mixed: double-float Jacobi preconditioner (FP32 pairs, FP32 operator)",
              "df_dirs": "mixed: double-float preconditioner and direction recurrences"}
# FP32 lane operations (a packed FP32x2 instruction is two) per site and RHS of one double-float
# sweep, counting a split product (FP32 operator entry x FP32-pair value, added into a sum with
# two-sum) as 11, the first product of a sum as 3 and a two-sum addition as 8.  Each of the 8 hops: 12 additions for the projection, the link
# times two half-spinors (6 sums of 3 complex products: 6 x (2 x 3 + 2 x 11) + 12 x 4 x 11) and 24
# additions into the sums; the row-2 rebuild of the 8 links (30 each); the two 6x6 blocks (12 rows
# of 1 real and 5 complex products: 6 + 5 x 44 or 28 + 4 x 44 + 22 = 226); U + kappa H (24 split
# products) and normalising the 24 stored reals (3 each).  This counts the emulation's work, not
# the method's: it sets the secondary (ALU) roofline of the double-float sweep only.
DF_OPS = 8 * (12 * 8 + 6 * (2 * 3 + 2 * 11) + 12 * 4 * 11 + 24 * 8) + 8 * 30 + 12 * 226 \
    + 24 * 11 + 24 * 3
# The same count for the grid-sum sweep (the DF tile's staged = 2): per lane a product costs 5
# operations (4 for the first of a sum) and each complex product sum is combined with 4 lane
# operations per lane pair.  Each hop: the projection (12 x 8), six complex outputs of two
# three-term lane-pair sums (6 x (2 x 2 x 14 + 8)), 16 for the grid's bound and the 24 additions
# into the site sums (24 x 8); the row-2 rebuild (8 x 30); the twelve clover rows of two six-term
# lane-pair sums (12 x (2 x 2 x 29 + 8)) and 30 for their bounds; U + kappa H and the stores.
DF_OPS_GRID = 8 * (12 * 8 + 6 * (2 * 2 * 14 + 8) + 16 + 24 * 8) + 8 * 30 \
    + 12 * (2 * 2 * 29 + 8) + 30 + 24 * 11 + 24 * 3
# FP64-pipe operations per site and RHS of the FP32-lane form of the FP64 stencils
# (csrc/dslash_x3.cu, wd_set_apply_form 1): the spin projections (8 hops x 12 real FMAs), joining
# the three levels of the 24 hopping sums (2 adds each), the 24 final FMAs with kappa, and the two
# Hermitian 6x6 site blocks (6 real x complex products and 15 complex entries used twice, 4 FMAs per
# complex product: 2 x (12 + 120)).  The hopping products themselves run on the FP32 lanes: 288
# packed lane-pair products of 24 operations (48 lane operations), 48 row combinations of ~38 lane
# operations, 96 exact three-way splits of ~15 and the joins' 360 bit-field operations.
X3_FP64_OPS = 8 * 12 + 24 * 2 + 24 + 2 * (12 + 120)
X3_FP32_OPS = 288 * 48 + 48 * 38 + 96 * 15 + 360
METRIC = "time-to-solution at true resid 1e-12 for L RHS; Dslash HBM GB/s vs peak"
FLOP_APPLY = 1824          # flop per site per RHS of A (1320 hopping + 504 clover)
FLOP_JACOBI = 1872         # flop per site per RHS of one Jacobi sweep A_D^{-1}(U + kappa H G)


def alu_peaks(sm_count: int, sm_mhz: float):
    """Derived ALU peaks of the device: FP32 lane operations/s (128 FP32 lanes per SM per clock)
    and FP64 flop/s (2 FP64 FMAs per SM per clock, 2 flop each), from its SM count and the SM
    clock sampled during the timed region."""
    hz = sm_mhz * 1e6
    return {"fp32_lane_tops": sm_count * 128 * hz / 1e12, "fp64_tflops": sm_count * 4 * hz / 1e12}


def algorithmic_bytes(kind: str, L: int, real_bytes: int = 8, link_reals: int = 18,
                      op_real_bytes: int = 0) -> int:
    """Minimum DRAM bytes per site: 4 links of `link_reals` reals (each link serves two sites),
    one packed 2x(6x6) clover or inverse block, and the spinors (reals of `real_bytes`) read or
    written once.  The links and clover blocks have reals of `op_real_bytes` (default: as the
    spinors)."""
    op_real_bytes = op_real_bytes or real_bytes
    links = 4 * link_reals * op_real_bytes
    clov = 72 * op_real_bytes
    spinor = 24 * real_bytes * L
    if kind == "dslash_apply":
        return links + clov + 2 * spinor
    if kind == "dslash_jacobi":
        return links + clov + 3 * spinor
    raise ValueError(kind)


def source_seed(rank: int) -> int:
    """Each rank solves its own independent sources."""
    return 1 + rank


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Largest value over all ranks (timings); the value itself without a process group."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


# ---------------------------------------------------------------- clocks during the timed region
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200", "-i",
                                       gpu_id], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.strip().split(", ") for r in self.f.read().splitlines() if r.strip()]
        self.f.close()
        os.unlink(self.f.name)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_id_for_smi(torch, dev) -> str:
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(dev.index or 0)


# ---------------------------------------------------------------- traffic from committed ncu summaries
# The source files each profiled kernel class is compiled from (with the shared headers): its
# recorded DRAM traffic stays valid while these are unchanged.
KERNEL_SOURCES = {
    ("dslash_jacobi_lp", "df"): ["sweep_df.cu", "common.cuh", "elem.cuh", "internal.h"],
    ("dslash_jacobi_lp", "fp32"): ["sweep_lp.cuh", "sweep_f32.cu", "sweep_lp.cu", "common.cuh",
                                   "elem.cuh", "internal.h"],
    ("dslash_apply", "fp64"): ["dslash_x3.cu", "dslash.cu", "common.cuh", "spin.cuh", "internal.h"],
}


def csrc_sha(files=None) -> str:
    """Hash of the library sources (all of csrc/, or the given file names in it)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_0907_3261_gb300", "csrc")
    names = sorted(files) if files else sorted(os.listdir(d))
    for name in names:
        if name.endswith((".cu", ".cuh", ".h")):
            h.update(open(os.path.join(d, name), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_class: str, precision: str):
    """DRAM bytes per launch recorded in profiles/*.md as
    ``bench-traffic: <class> <precision> <bytes> <sources sha>`` (the hash of the class's
    KERNEL_SOURCES); None if absent or stale."""
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return None
    sha = csrc_sha(KERNEL_SOURCES.get((kernel_class, precision)))
    for name in os.listdir(pdir):
        if not name.endswith((".md", ".txt")):
            continue
        for line in open(os.path.join(pdir, name)):
            m = re.match(r"\s*bench-traffic:\s*(\S+)\s+(\S+)\s+(\d+)\s+(\S+)", line)
            if m and m.group(1) == kernel_class and m.group(2) == precision:
                return int(m.group(3)) if m.group(4) == sha else None
    return None


# ---------------------------------------------------------------- oracle timing (host cores)
# The C++ oracle (oracle/cpp/oracle.cpp: plain FP64, full 4x4 spin and 12x12 site matrices, the
# algorithm box as written, OpenMP over sites) timed on the host cores.  c1 and c2 are solved in
# full; the headline workload, which takes the oracle an hour or more, is timed as its set-up, the
# start of the algorithm box (R_0, F_0 = M R_0, W_0) and measured outer iterations, and
# extrapolated to the iteration count of the FP64 method.
SMALL_CONFIGS = {
    "c1": dict(dims=(4, 4, 4, 4), L=4, j=4, kappa=0.115, eps=0.3, sources="point"),
    "c2": dict(dims=(8, 8, 8, 16), L=12, j=12, kappa=0.13, eps=0.2, sources="z4"),
}


def small_sources(cfg):
    from paper_0907_3261_gb300 import inputs as I
    if cfg["sources"] == "point":
        return I.point_sources(cfg["dims"], cfg["L"])
    return I.z4_noise(cfg["dims"], cfg["L"], seed=1)


def oracle_full_solve(cfg, threads):
    """Wall seconds and outcome of a complete C++-oracle solve of a small config."""
    from oracle import cpp
    from paper_0907_3261_gb300 import inputs as I
    used = cpp.set_threads(threads)
    links = I.random_links(cfg["dims"], cfg["eps"], seed=0)
    B = small_sources(cfg)
    t0 = time.perf_counter()
    X, st, k, restarts, mvm, tr = cpp.CppOracle(links, cfg["dims"], cfg["kappa"], CSW).solve(
        B, cfg["j"])
    sec = time.perf_counter() - t0
    return {"seconds": round(sec, 4), "threads": used, "status": st,
            "iters": k, "mvm_per_column": mvm, "max_true_resid": float(tr.max()),
            "gflops": round(solve_flop(cfg, mvm) / sec / 1e9, 2)}


def solve_flop(cfg, mvm_per_column):
    """Stencil flop of a solve: the paper's #MVM count per column times L RHS times 1824 flop per
    site and RHS (each Jacobi step counted as one MVM, as Table 1 counts them)."""
    import numpy as np
    return mvm_per_column * cfg["L"] * int(np.prod(cfg["dims"])) * FLOP_APPLY


class OracleSample:
    """The headline workload on the C++ oracle, one outer iteration at a time (all host cores)."""

    def __init__(self, threads):
        from oracle import cpp
        from paper_0907_3261_gb300 import inputs as I
        self.threads = cpp.set_threads(threads)
        links = I.random_links(DIMS, LINK_EPS, seed=0)
        self.B = I.z4_noise(DIMS, L_RHS, seed=source_seed(0))
        t0 = time.perf_counter()
        self.s = cpp.Stepper(links, DIMS, KAPPA, CSW)
        self.t_setup = time.perf_counter() - t0
        t0 = time.perf_counter()
        self.s.start(self.B, J_JACOBI)
        self.t_start = time.perf_counter() - t0
        self.steps = []

    def step(self):
        from oracle import cpp
        if self.s.status != cpp.RUNNING:         # converged within the sample: begin again
            self.s.start(self.B, J_JACOBI)
        t0 = time.perf_counter()
        self.s.step()
        self.steps.append(time.perf_counter() - t0)
        return self.steps[-1]

    def true_residual_seconds(self):
        t0 = time.perf_counter()
        self.s.result(true_resid=True)
        return time.perf_counter() - t0

    def extrapolate(self, k, t_iter, t_true):
        """Set-up + start + k outer iterations + the true residual at exit."""
        return self.t_setup + self.t_start + k * t_iter + t_true

    def close(self):
        self.s.close()


def cpu_baseline(k_fp64: int):
    """The oracle on the host cores: c1 (single thread and all cores) and c2 solved in full, the
    headline workload extrapolated per measured outer iteration to the FP64 method's k."""
    cores = os.cpu_count() or 1
    small = {"c1_single_thread": oracle_full_solve(SMALL_CONFIGS["c1"], 1),
             "c1_all_cores": oracle_full_solve(SMALL_CONFIGS["c1"], cores),
             "c2_all_cores": oracle_full_solve(SMALL_CONFIGS["c2"], cores)}
    smp = OracleSample(cores)
    t_iter = smp.step()
    t_true = smp.true_residual_seconds()
    value = smp.extrapolate(k_fp64, t_iter, t_true)
    smp.close()
    return {"value": round(value, 2), "unit": "s", "cores": cores, "threads": smp.threads,
            "kind": "oracle",
            "sample": (f"C++ oracle on {cores} host cores: set-up {smp.t_setup:.2f}s, start of the "
                       f"algorithm box (R_0, F_0 = M R_0, W_0) {smp.t_start:.2f}s and one measured "
                       f"outer iteration {t_iter:.2f}s on the full workload, extrapolated to "
                       f"k={k_fp64} outer iterations (the FP64 method's count) plus the true "
                       f"residual {t_true:.2f}s"),
            "extrapolated": True, "measured_outer_iteration_s": round(t_iter, 3),
            "full_solves": small}


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    cores = os.cpu_count() or 1
    smp = OracleSample(cores)
    for step in range(args.warmup + args.steps):
        t = smp.step()
        log(f"reference step {step}: one outer iteration {t:.2f}s")
    t_iter = statistics.mean(smp.steps[args.warmup:])
    t_true = smp.true_residual_seconds()
    value = smp.extrapolate(WORKLOAD_ITERS, t_iter, t_true)
    smp.close()
    sample = (f"C++ oracle on {cores} host cores: set-up {smp.t_setup:.2f}s, start (R_0, F_0, W_0) "
              f"{smp.t_start:.2f}s, one outer iteration per step ({t_iter:.2f}s mean over "
              f"{args.steps} steps), extrapolated to k={WORKLOAD_ITERS} outer iterations plus the "
              f"true residual")
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 2), "unit": "s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(value * 1e3, 1), "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config(args),
           "measured_s_per_step": round(t_iter, 3),
           "cpu_baseline": {"value": round(value, 2), "unit": "s", "cores": cores,
                            "threads": smp.threads, "kind": "oracle", "sample": sample,
                            "extrapolated": True},
           "e2e": {"value": round(value, 2), "unit": "s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def config(args):
    return {"workload": f"clover Wilson-Dirac {DIMS[0]}^3x{DIMS[3]}, L={L_RHS} Z4 sources, "
                        f"Jacobi j={J_JACOBI}, kappa={KAPPA}, c_SW={CSW}, "
                        f"links SU3proj(1+{LINK_EPS}G), true resid <= {TOL}",
            "lattice": list(DIMS), "L": L_RHS, "j": J_JACOBI, "kappa": KAPPA, "csw": CSW,
            "tol": TOL, "precision": args.precision,
            "parallelism": f"independent solves x{args.gpus}",
            "l2": "working set 13 blocks x 302 MB > L2 (no flush needed)"}


# ---------------------------------------------------------------- 24 solves in one graph
BATCH_LATTICES = [(8, 8, 8, 8), (12, 12, 12, 24), (16, 16, 16, 32), (32, 32, 32, 64)]
BATCH_L = [1, 3, 7, 12]


def batch_jobs():
    """24 solves: every lattice with every L, and the two smaller lattices once more; kappa spread
    evenly over [0.115, 0.124]."""
    combos = [(d, L) for d in BATCH_LATTICES for L in BATCH_L]
    combos += [(d, L) for d in BATCH_LATTICES[:2] for L in BATCH_L]
    return [(d, L, 0.115 + 0.009 * i / (len(combos) - 1)) for i, (d, L) in enumerate(combos)]


# Preconditioner mixes of the batch (--batch-mix).  The kappa stay well below the critical one,
# where FP32 sweeps keep block BiCGGR converging; precision 2 adds the double-float direction
# recurrences.  "stated" is the mixed-precision plus learned-preconditioner batch: the 8^4 jobs use
# the gauge-covariant network (FP32 activations; trained in this run on 16 other 8^4
# configurations, outside the timed region) with j = 8 FP64 Jacobi as its fallback, every other
# job FP32 sweeps with double-float directions.
BATCH_J = 8
BATCH_MIXES = {
    "stated": "8^4 jobs: learned 4-layer network (FP32 activations, FP64-Jacobi j=8 fallback); "
              "others: Jacobi j=8 in FP32 with double-float direction recurrences",
    "jacobi": "Jacobi j=8 in FP32 with double-float direction recurrences",
    "df": "Jacobi j=8 in double-float with double-float direction recurrences",
}
NET_TRAIN_SEEDS = list(range(1, 17))
NET_TRAIN_KAPPA = 0.12
NET_TRAIN_STEPS = 600


def train_batch_network(wd, I, torch, dev):
    """The learned preconditioner of the stated mix, trained on (r, A^-1 r) pairs that the plain
    solver generates on 16 8^4 configurations other than the batch's (seeds 1-16)."""
    from paper_0907_3261_gb300 import train_net as T
    t0 = time.perf_counter()
    pairs = T.make_pairs(wd, I, torch, BATCH_LATTICES[0], NET_TRAIN_KAPPA, CSW, NET_TRAIN_SEEDS,
                         12, LINK_EPS, 12, dev)
    net = wd.wd_net_create(4, 4, I.network_weights(4, 4, seed=7, noise=0.01))
    hist = T.train(wd, net, pairs, NET_TRAIN_STEPS, 3e-3, log_every=0)
    torch.cuda.synchronize()
    return net, {"configs": len(NET_TRAIN_SEEDS), "kappa": NET_TRAIN_KAPPA,
                 "steps": NET_TRAIN_STEPS, "loss_first": round(hist[0], 4),
                 "loss_last": round(hist[-1], 4), "seconds": round(time.perf_counter() - t0, 2)}


def batch_job_options(mix, d, net):
    if mix == "df":
        return dict(precision=5)
    if mix == "stated" and d == BATCH_LATTICES[0]:
        return dict(precision=0, net=net)
    return dict(precision=2)


def batch_workload(args):
    """Time for 24 independent solves launched as one CUDA graph (device-side iteration control,
    fallback and restarts), against the same 24 solves run one after another with host-side
    control."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_0907_3261_gb300 as wd
    from paper_0907_3261_gb300 import inputs as I
    dev = torch.device("cuda", 0)
    mix = args.batch_mix
    net, training = (train_batch_network(wd, I, torch, dev) if mix == "stated" else (None, None))
    links = {d: torch.from_numpy(I.random_links(d, LINK_EPS, seed=0)).to(dev) for d in BATCH_LATTICES}
    jobs = []
    for n, (d, L, kappa) in enumerate(batch_jobs()):
        ctx = wd.wd_create(links[d], d, kappa, CSW)
        B = torch.from_numpy(I.z4_noise(d, L, seed=100 + n)).to(dev)
        jobs.append(dict(ctx=ctx, B=B, X=torch.zeros_like(B), j=BATCH_J, tol=TOL,
                         **batch_job_options(mix, d, net)))
    del links
    site_rhs = sum(int(np.prod(d)) * L for d, L, _ in batch_jobs())

    def run_graph():
        for jb in jobs:
            jb["X"].zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        infos = wd.bbicggr_solve_batch(jobs)
        return time.perf_counter() - t0, infos

    def run_sequential():
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        infos = []
        for jb in jobs:
            jb["X"].zero_()
            kw = {k: jb[k] for k in ("j", "tol", "precision", "net") if k in jb}
            infos.append(wd.bbicggr_solve(jb["ctx"], jb["B"], jb["X"], **kw)[1])
        torch.cuda.synchronize()
        return time.perf_counter() - t0, infos

    for _ in range(args.warmup):
        run_graph()
    tg = [run_graph() for _ in range(args.steps)]
    ts = [run_sequential() for _ in range(max(1, args.steps // 2))]
    g_s = statistics.mean(t for t, _ in tg)
    s_s = statistics.mean(t for t, _ in ts)
    infos = tg[-1][1]
    ok = all(i["status"] == wd.WD_OK for i in infos)
    same = all(a["iters"] == b["iters"] and a["fallbacks"] == b["fallbacks"]
               for a, b in zip(infos, ts[-1][1]))
    out = {"metric": "time for 24 independent solves (one CUDA graph)", "value": round(g_s, 4),
           "unit": "s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(g_s * 1e3, 2), "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64+f32+df32x2", "data": "synthetic",
           "config": {"workload": "batch24: lattices 8^4, 12^3x24, 16^3x32, 32^3x64 x L in {1,3,7,12} "
                                  "(+ 8^4 and 12^3x24 again), kappa 0.115..0.124, true resid <= 1e-12",
                      "mix": mix, "preconditioners": BATCH_MIXES[mix],
                      "jobs": len(jobs), "site_rhs_total": site_rhs},
           "sequential_host_controlled_s": round(s_s, 4),
           "speedup_vs_sequential": round(s_s / g_s, 3),
           "solves": {"status": "ok" if ok else "FAILED",
                      "same_as_sequential": same,
                      "jobs": [{"dims": "x".join(map(str, d)), "L": L, "kappa": round(kappa, 5),
                                "precond": "network" if jb.get("net") is not None else
                                           f"jacobi p{jb['precision']}",
                                "iters": i["iters"], "fallbacks": i["fallbacks"],
                                "true_resid": float(f"{i['max_true_resid']:.3e}")}
                               for (d, L, kappa), jb, i in zip(batch_jobs(), jobs, infos)],
                      "max_true_resid": max(i["max_true_resid"] for i in infos)}}
    if training:
        out["network_training"] = training
    print(json.dumps(out), flush=True)
    return 0 if ok else 1


# ---------------------------------------------------------------- the FP64 method on 8^3 x 16
GRID_DIMS = (8, 8, 8, 16)
GRID_L = [1, 2, 4, 8, 12]
GRID_J = [0, 4, 8, 12, 16]
GRID_SCAN_MAXIT = 2000


def grid8_workload(args):
    """The plain FP64 method on an 8^3 x 16 lattice: kappa rises from 0.115 in steps of 0.001 until
    the L = 1, j = 0 solve first needs more than 2000 iterations; then every L in {1, 2, 4, 8, 12}
    with every j in {0, 4, 8, 12, 16} is solved at three kappa of the scan (the first, the middle
    and the last that converged within 2000 iterations), with its outer iterations, #MVM per
    column, time to solution and true residual.  Times are medians of --steps solves after one
    untimed solve."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_0907_3261_gb300 as wd
    from paper_0907_3261_gb300 import inputs as I
    dev = torch.device("cuda", 0)
    links = torch.from_numpy(I.random_links(GRID_DIMS, LINK_EPS, seed=0)).to(dev)
    Bs = {L: torch.from_numpy(I.z4_noise(GRID_DIMS, L, seed=1)).to(dev) for L in GRID_L}
    scan = []
    kappa = 0.115
    while True:
        ctx = wd.wd_create(links, GRID_DIMS, kappa, CSW)
        _, info = wd.bbicggr_solve(ctx, Bs[1], j=0, tol=TOL, maxit=GRID_SCAN_MAXIT)
        scan.append({"kappa": round(kappa, 3), "iters": info["iters"],
                     "status": info["status_name"]})
        if info["status"] != wd.WD_OK or info["iters"] > GRID_SCAN_MAXIT or kappa > 0.2:
            break
        kappa += 0.001
    ok_kappas = [r["kappa"] for r in scan if r["status"] == "WD_OK"]
    picks = sorted({ok_kappas[0], ok_kappas[len(ok_kappas) // 2], ok_kappas[-1]})
    rows = []
    for kappa in picks:
        ctx = wd.wd_create(links, GRID_DIMS, kappa, CSW)
        for L in GRID_L:
            for j in GRID_J:
                X = torch.zeros_like(Bs[L])
                wd.bbicggr_solve(ctx, Bs[L], X, j=j, tol=TOL, maxit=20000)
                times = []
                for _ in range(args.steps):
                    X.zero_()
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    _, info = wd.bbicggr_solve(ctx, Bs[L], X, j=j, tol=TOL, maxit=20000)
                    torch.cuda.synchronize()
                    times.append(time.perf_counter() - t0)
                rows.append({"kappa": kappa, "L": L, "j": j, "status": info["status_name"],
                             "iters": info["iters"], "mvm_per_col": info["mvm_paper"] // L,
                             "tts_s": round(statistics.median(times), 5),
                             "true_resid": float(f"{info['max_true_resid']:.3e}")})
    ok = all(r["status"] == "WD_OK" for r in rows)
    out = {"metric": "time-to-solution grid, plain FP64 method, 8^3x16", "unit": "s",
           "n_gpus": 1, "steps": args.steps, "dtype": "f64", "data": "synthetic",
           "higher_is_better": False,
           "config": {"workload": "8^3x16, links SU3proj(1+0.2G) seed 0, c_SW 1.0, Z4 sources "
                                  "seed 1, tol 1e-12, L in {1,2,4,8,12} x j in {0,4,8,12,16}"},
           "kappa_scan": scan, "kappa_picked": picks, "grid": rows,
           "status": "ok" if ok else "FAILED"}
    print(json.dumps(out), flush=True)
    return 0 if ok else 1


# ---------------------------------------------------------------- the learned preconditioner
NET_LAYERS, NET_HIDDEN = 4, 4


def net_flop(layers: int, hidden: int) -> int:
    """Flop per site and RHS of one network application: every layer transports each input channel
    along the 8 hops (4 spins x a 3x3 complex link: 36 complex multiply-adds, 288 flop) and mixes
    every (output, input) channel pair in each of the 9 directions (a 4x4 complex spin matrix on 3
    colours: 48 complex multiply-adds, 384 flop)."""
    from paper_0907_3261_gb300 import inputs as I
    ch = I.network_channels(layers, hidden)
    pairs = zip(ch[:-1], ch[1:])
    return sum(cin * 8 * 288 + cin * cout * 9 * 384 for cin, cout in pairs)


def net_workload(args):
    """One application G = N(R) of the learned gauge-covariant preconditioner (4 layers, channels
    1-4-4-4-1) on the bench lattice (16^3 x 32, L = 12, the bench's links), with weights from the
    seeded initialisation plus noise 0.1; FP32 activations (the value) and BF16 activations.
    One application converts R to the FP32 channel layout, runs the 4 layer kernels and converts
    back (6 launches), moving ~4.8 GB of activations and blocks, far more than L2."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_0907_3261_gb300 as wd
    from paper_0907_3261_gb300 import inputs as I
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    links = torch.from_numpy(I.random_links(DIMS, LINK_EPS, seed=0)).to(dev)
    ctx = wd.wd_create(links, DIMS, KAPPA, CSW)
    net = wd.wd_net_create(NET_LAYERS, NET_HIDDEN,
                           I.network_weights(NET_LAYERS, NET_HIDDEN, seed=0, noise=0.1))
    R = torch.from_numpy(I.z4_noise(DIMS, L_RHS, seed=1)).to(dev)
    G = torch.empty_like(R)
    stream = torch.cuda.current_stream(dev)
    times = {}
    clocks = None
    for bf16 in (False, True):
        for _ in range(args.warmup):
            wd.wd_net_apply(ctx, net, R, G, bf16=bf16, stream=stream)
        torch.cuda.synchronize(dev)
        sampler = ClockSampler(gpu_id_for_smi(torch, dev)) if not bf16 else None
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            wd.wd_net_apply(ctx, net, R, G, bf16=bf16, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if sampler is not None:
            clocks = sampler.stop()
        times["bf16" if bf16 else "fp32"] = e0.elapsed_time(e1) / args.steps
    ok = bool(torch.isfinite(G).all().item())
    V = 1
    for d in DIMS:
        V *= d
    flop = net_flop(NET_LAYERS, NET_HIDDEN) * V * L_RHS
    props = torch.cuda.get_device_properties(dev)
    mhz = (clocks or {}).get("sm_mhz") or 2070.0
    peak = 2 * alu_peaks(props.multi_processor_count, mhz)["fp32_lane_tops"]   # FMA = 2 flop
    achieved = flop / (times["fp32"] * 1e-3) / 1e12
    out = {"metric": "learned preconditioner application time (16^3x32, L=12)",
           "value": round(times["fp32"], 4), "unit": "ms", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(times["fp32"], 4),
           "higher_is_better": False, "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "network application: 4 layers, channels 1-4-4-4-1, 16^3x32, "
                                  "L=12, activations > L2",
                      "flop_per_site_rhs": net_flop(NET_LAYERS, NET_HIDDEN)},
           "bf16_activations_ms": round(times["bf16"], 4),
           "gpu_launches": (NET_LAYERS + 2) * args.steps,
           "roofline": {"bound": "alu", "achieved": round(achieved, 2), "peak": round(peak, 2),
                        "unit": "TFLOP/s", "frac": round(achieved / peak, 3), "traffic": None,
                        "peak_kind": "derived: SMs x 128 FP32 lanes x 2 flop x sampled SM clock"},
           "clocks": clocks, "status": "ok" if ok else "FAILED"}
    print(json.dumps(out), flush=True)
    return 0 if ok else 1


def gpu_small_solves(wd, I, dev, prec):
    """The same c1 and c2 solves on the GPU (default form), for the side-by-side baseline."""
    import torch
    out = {}
    for name, cfg in SMALL_CONFIGS.items():
        links = torch.from_numpy(I.random_links(cfg["dims"], cfg["eps"], seed=0)).to(dev)
        ctx = wd.wd_create(links, cfg["dims"], cfg["kappa"], CSW)
        B = torch.from_numpy(small_sources(cfg)).to(dev)
        wd.bbicggr_solve(ctx, B, j=cfg["j"], tol=TOL, precision=prec)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        _, info = wd.bbicggr_solve(ctx, B, j=cfg["j"], tol=TOL, precision=prec)
        torch.cuda.synchronize(dev)
        sec = time.perf_counter() - t0
        out[name] = {"seconds": round(sec, 5), "iters": info["iters"],
                     "max_true_resid": info["max_true_resid"],
                     "gflops": round(solve_flop(cfg, info["mvm_paper"] // cfg["L"]) / sec / 1e9, 2)}
        wd.wd_destroy(ctx)
    return out


# ---------------------------------------------------------------- GB300 arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="df_dirs", choices=list(PRECISIONS),
                    help="fp64: the plain FP64 method; mixed: FP32 Jacobi "
                         "preconditioner with the FP64 outer method; bf16: the preconditioner's "
                         "blocks stored in BF16, FP32 arithmetic; df: double-float (FP32-pair) "
                         "preconditioner arithmetic; df_dirs (the default): df and double-float "
                         "direction recurrences")
    ap.add_argument("--fp32-tile", default="",
                    help="fix the FP32 sweep tile 'rhs_per_thread,block,min_blocks[,staged]' instead of "
                         "autotuning it (reproducible profiling)")
    ap.add_argument("--bf16-tile", default="", help="the same for the BF16-storage sweep")
    ap.add_argument("--df-tile", default="",
                    help="the same for the double-float sweep (e.g. 1,128,0,2: packed, grid sums); "
                         "a run under a profiler should fix it, since the profiler's per-launch "
                         "overhead misleads the autotuner's timings")
    ap.add_argument("--link-reals", type=int, default=0, choices=[0, 12, 18],
                    help="link format of the low-precision sweeps (0: the library's choice)")
    ap.add_argument("--no-other-form", action="store_true",
                    help="skip timing the other precision forms on the same workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-mix", default="stated", choices=list(BATCH_MIXES),
                    help="preconditioners of the batch24 workload")
    ap.add_argument("--workload", default="tts", choices=["tts", "batch24", "grid8", "net16"],
                    help="tts: the time-to-solution line; batch24: 24 solves in one CUDA graph; "
                         "grid8: the FP64 method's kappa scan and L x j grid on 8^3x16; net16: "
                         "one application of the learned preconditioner on 16^3x32, L = 12")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return reference_arm(args)
    if args.workload == "batch24":
        return batch_workload(args)
    if args.workload == "grid8":
        return grid8_workload(args)
    if args.workload == "net16":
        return net_workload(args)

    import numpy as np
    import torch
    rank, world, local = dist_env()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if dist:
        dist.barrier()
    import paper_0907_3261_gb300 as wd
    from paper_0907_3261_gb300 import inputs as I
    prec = PRECISIONS[args.precision]

    links = torch.from_numpy(I.random_links(DIMS, LINK_EPS, seed=0)).to(dev)
    Bh = torch.from_numpy(I.z4_noise(DIMS, L_RHS, seed=source_seed(rank))).pin_memory()
    B = Bh.to(dev)
    ctx = wd.wd_create(links, DIMS, KAPPA, CSW)
    if args.fp32_tile:
        wd.wd_set_tile(ctx, L_RHS, *[int(v) for v in args.fp32_tile.split(",")], precision=1)
    if args.bf16_tile:
        wd.wd_set_tile(ctx, L_RHS, *[int(v) for v in args.bf16_tile.split(",")], precision=3)
    if args.df_tile:
        wd.wd_set_tile(ctx, L_RHS, *[int(v) for v in args.df_tile.split(",")], precision=4)
    if args.link_reals:
        wd.wd_set_link_reals(ctx, args.link_reals)
    link_reals = wd.wd_link_reals(ctx)
    X = torch.zeros_like(B)
    stream = torch.cuda.current_stream(dev)

    def solve():
        X.zero_()
        return wd.bbicggr_solve(ctx, B, X, j=J_JACOBI, tol=TOL, precision=prec, stream=stream)[1]

    for w in range(args.warmup):
        info = solve()
        log(f"[rank {rank}] warmup {w}: {info['status_name']} k={info['iters']} "
            f"{info['seconds']:.3f}s true={info['max_true_resid']:.2e}")

    def maxr(v: float) -> float:
        return max_over_ranks(v, dist, dev)

    # ---- device-timed region: inputs resident in HBM
    wd.wd_profile_reset(ctx)
    wd.wd_profile_enable(ctx, True)
    sampler = ClockSampler(gpu_id_for_smi(torch, dev))
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    infos = [solve() for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    wd.wd_profile_enable(ctx, False)
    prof = wd.wd_profile_read(ctx)
    ms_total = maxr(e0.elapsed_time(e1))
    ms_step = ms_total / args.steps
    ok = all(i["status"] == wd.WD_OK and i["max_true_resid"] <= TOL for i in infos)
    X_main = X.clone()   # this form's solution, compared per column with the FP64 form's below
    # how far the recursive residual R (R -= zeta W + Y) drifted from B - A X over the solve, per
    # column relative to ||b||, with B - A X from the library's FP64 stencil (outside the timing)
    R_rec = wd.wd_copy_residual(ctx, torch.empty_like(B))
    R_true = B - wd.wd_apply(ctx, X_main)
    gap = ((R_rec - R_true).reshape(-1, L_RHS).norm(dim=0) / B.reshape(-1, L_RHS).norm(dim=0))
    residual_gap = float(gap.max().item())
    del R_rec, R_true

    # ---- end to end through the C-ABI with pinned host buffers.  Every step gets its own X0 = 0
    # host buffer, prepared before the timed region like B; inside it are the copies of B and X0
    # in, the solve, and the copy of X out.  Preparing a buffer includes its first transfer: the
    # first DMA from freshly pinned memory maps its pages (~35 ms for 302 MB on this host, against
    # ~1.5 ms for every later transfer), which is a cost of allocating the buffer, not of a step.
    Xhs = [torch.zeros(B.shape, dtype=torch.complex128).pin_memory() for _ in range(args.steps)]
    X.zero_()
    for Xh in Xhs:                        # first transfers both ways (the buffers stay zero)
        X.copy_(Xh, non_blocking=True)
        Xh.copy_(X, non_blocking=True)
    torch.cuda.synchronize(dev)
    Bn = Bh.numpy()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for Xh in Xhs:
        _, ie = wd.bbicggr_solve(ctx, Bn, Xh.numpy(), j=J_JACOBI, tol=TOL, precision=prec)
        ok = ok and ie["status"] == wd.WD_OK
    e2e_s = maxr((time.perf_counter() - t0) / args.steps)
    del Xhs
    block = B.numel() * 16

    # ---- the host link alone: pinned host <-> device copies of one block, for comparison with
    # the part of e2e that the copies take
    def copy_gbs(src, dst, reps=5):
        dst.copy_(src, non_blocking=True)     # the first transfer maps freshly pinned pages
        torch.cuda.synchronize(dev)
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for _ in range(reps):
            dst.copy_(src, non_blocking=True)
        c1.record(stream)
        torch.cuda.synchronize(dev)
        return reps * src.numel() * src.element_size() / (c0.elapsed_time(c1) / 1e3) / 1e9
    Xh_pinned = torch.empty(B.shape, dtype=torch.complex128).pin_memory()
    host_link = {"pinned_h2d_gbs": round(copy_gbs(Bh, X), 1),
                 "pinned_d2h_gbs": round(copy_gbs(X, Xh_pinned), 1)}
    del Xh_pinned

    # ---- the other precision forms on the same workload, for comparison (not the value)
    others = []
    col_diff = None
    for oname, oprec in ([] if args.no_other_form else list(PRECISIONS.items())):
        if oprec == prec:
            continue

        def solve_other():
            X.zero_()
            return wd.bbicggr_solve(ctx, B, X, j=J_JACOBI, tol=TOL, precision=oprec,
                                    stream=stream)[1]
        solve_other()
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        io = [solve_other() for _ in range(2)]
        f1.record(stream)
        torch.cuda.synchronize(dev)
        to = maxr(f0.elapsed_time(f1) / 2 / 1e3)
        ok = ok and all(i["status"] == wd.WD_OK for i in io)
        if oprec == 0:   # ||X - X_fp64|| / ||X_fp64|| per column
            Xf = X.reshape(-1, L_RHS)
            col_diff = ((X_main.reshape(-1, L_RHS) - Xf).norm(dim=0) / Xf.norm(dim=0)).tolist()
        others.append({"form": FORM_NAMES[oname], "precision": oname,
                       "value": round(to, 6), "unit": "s", "iters": io[-1]["iters"],
                       "fallbacks": io[-1]["fallbacks"],
                       "max_true_resid": max(i["max_true_resid"] for i in io),
                       "ratio_to_value": round(to / (ms_step / 1e3), 3)})

    # ---- roofline of the dominant kernel class, and of every stencil class.  The primary figure
    # is the metric's: algorithmic DRAM bytes per launch (each spinor, link and clover block read
    # or written once) over the CUDA-event launch time, against the measured HBM copy peak.  The
    # roofline that binds the kernel on this GPU is given beside it (FP64 pipe or FP32 lanes).
    V = int(np.prod(DIMS))
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    hbm_source = ("MEASURED_PEAKS.json hbm_gbs (measured copy)" if "hbm_gbs" in peaks
                  else "fallback 6800 GB/s")
    props = torch.cuda.get_device_properties(dev)
    sm_count = int(props.multi_processor_count)
    clock_mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 2070.0
    alu = alu_peaks(sm_count, clock_mhz)
    alu_source = f"derived: {sm_count} SMs at the sampled median {clock_mhz:.0f} MHz"
    sweep_prec = {"fp64": "fp64", "mixed": "fp32", "bf16": "bf16", "df": "df",
                  "df_dirs": "df"}[args.precision]
    df_tile = wd.wd_tuned_tile(ctx, L_RHS, precision=4) if sweep_prec == "df" else None
    per_kernel = {}
    stencil_form = wd.wd_get_apply_form(ctx)
    for cls in ("dslash_jacobi_lp", "dslash_jacobi", "dslash_apply"):
        n, ms = prof.get(cls, (0, 0.0))
        if not n:
            continue
        # the FP32-lane form launches an exponent pre-pass with each FP64 stencil
        per_launch = 2 if stencil_form == 1 and cls in ("dslash_apply", "dslash_jacobi") else 1
        n //= per_launch
        avg_s = ms / n / 1e3
        kprec = sweep_prec if cls == "dslash_jacobi_lp" else "fp64"
        f32 = kprec in ("fp32", "bf16")
        flop_unit = FLOP_APPLY if cls == "dslash_apply" else FLOP_JACOBI
        kind = "dslash_apply" if cls == "dslash_apply" else "dslash_jacobi"
        if f32:   # spinors FP32 or BF16; links and A_D^{-1} FP32
            per_site = algorithmic_bytes(kind, L_RHS, 4 if kprec == "fp32" else 2, link_reals, 4)
        elif kprec == "df":   # spinors as FP32 pairs; links and A_D^{-1} FP32
            per_site = algorithmic_bytes(kind, L_RHS, 8, link_reals, 4)
        else:
            per_site = algorithmic_bytes(kind, L_RHS, 8)
        nbytes = per_site * V
        tflops = flop_unit * V * L_RHS / avg_s / 1e12
        gbs = nbytes / avg_s / 1e9
        fig = {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm_peak, "unit": "GB/s",
               "frac": round(gbs / hbm_peak, 4), "peak_source": hbm_source,
               "algorithmic_bytes_per_site": per_site, "units_per_launch": f"{V} sites x L={L_RHS}",
               "tflops": round(tflops, 3)}
        if kprec == "df":
            ops = DF_OPS_GRID if df_tile and df_tile[3] == 2 else DF_OPS
            tops = ops * V * L_RHS / avg_s / 1e12
            fig["binding_roofline"] = {
                "bound": "alu", "achieved": round(tops, 3), "peak": round(alu["fp32_lane_tops"], 2),
                "unit": "T FP32 lane ops/s", "frac": round(tops / alu["fp32_lane_tops"], 4),
                "peak_source": alu_source + " x 128 FP32 lanes", "fp32_ops_per_site_rhs": ops}
        elif not f32 and stencil_form == 1:
            # the FP32-lane form: FP64 pipe and FP32 lanes both carry work; the FP64 pipe is the
            # busier one (ncu)
            ops64 = X3_FP64_OPS * V * L_RHS / avg_s / 1e12
            ops32 = X3_FP32_OPS * V * L_RHS / avg_s / 1e12
            fig["binding_roofline"] = {
                "bound": "alu", "achieved": round(ops64, 4), "peak": round(alu["fp64_tflops"] / 2, 4),
                "unit": "T FP64-pipe ops/s", "frac": round(ops64 / (alu["fp64_tflops"] / 2), 4),
                "peak_source": alu_source + " x 2 FP64 lanes/clk", "fp64_ops_per_site_rhs": X3_FP64_OPS,
                "fp32_lane_ops_per_site_rhs": X3_FP32_OPS,
                "fp32_lane_frac": round(ops32 / alu["fp32_lane_tops"], 4),
                "form": "hopping sums on the FP32 lanes (wd_set_apply_form 1)"}
        elif not f32:
            fig["binding_roofline"] = {
                "bound": "alu", "achieved": round(tflops, 4), "peak": round(alu["fp64_tflops"], 4),
                "unit": "TFLOP/s", "frac": round(tflops / alu["fp64_tflops"], 4),
                "peak_source": alu_source + " x 2 FP64 FMA/clk"}
        fig.update({"kernel": cls, "precision": kprec,
                    "traffic": ncu_traffic(cls, kprec),
                    "algorithmic_bytes_per_launch": nbytes, "flop_per_site_rhs": flop_unit,
                    "avg_launch_ms": round(avg_s * 1e3, 4), "launches": n,
                    "kernels_per_launch": per_launch, "total_ms": round(ms, 2)})
        per_kernel[cls] = fig
    dom = max(per_kernel, key=lambda k: per_kernel[k]["total_ms"])
    roofline = dict(per_kernel[dom])
    roofline["stencil_kernels"] = per_kernel

    launches = sum(n for k, (n, _) in prof.items())
    tile = (wd.wd_tuned_tile(ctx, L_RHS, precision={1: 1, 2: 1, 3: 3, 4: 4, 5: 4}[prec])
            if prec else None)
    out = {"metric": METRIC, "value": round(ms_step / 1e3, 6), "unit": "s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 3),
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": {0: "f64", 1: "f64+f32", 3: "f64+f32(bf16 storage)", 4: "f64+df32x2",
                     5: "f64+df32x2"}[prec],
           "data": "synthetic",
           "config": dict(config(args), sweep_tile=tile, link_reals=link_reals),
           "roofline": roofline,
           "e2e": {"value": round(e2e_s, 6), "unit": "s", "h2d_bytes_per_step": 2 * block,
                   "d2h_bytes_per_step": block, "host_link": host_link},
           "gpu_launches": launches, "clocks": clocks,
           "solve": {"status": "ok" if ok else "FAILED", "iters": infos[-1]["iters"],
                     "mvm_paper": infos[-1]["mvm_paper"],
                     "max_true_resid": max(i["max_true_resid"] for i in infos),
                     "restarts": infos[-1]["restarts"],
                     "fallbacks": infos[-1]["fallbacks"],
                     "true_resid_per_column": [float(f"{v:.3e}") for v in infos[-1]["true_resid"]],
                     "recursive_vs_true_residual_gap": float(f"{residual_gap:.3e}"),
                     "rel_diff_vs_fp64_per_column": (None if col_diff is None else
                                                     [float(f"{v:.3e}") for v in col_diff])},
           "kernels": {k: {"launches": n, "ms": round(ms, 3)} for k, (n, ms) in prof.items() if n or ms}}
    if others:
        out["other_forms"] = others
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle runs the plain FP64 method: extrapolate to that method's iteration count
        k = infos[-1]["iters"] if prec == 0 else next(
            (o["iters"] for o in others if o["precision"] == "fp64"), WORKLOAD_ITERS)
        out["cpu_baseline"] = cpu_baseline(k)
        out["cpu_baseline"]["gpu_full_solves"] = gpu_small_solves(wd, I, dev, prec)
    if rank == 0:
        print(json.dumps(out), flush=True)
    wd.wd_destroy(ctx)
    if dist:
        dist.destroy_process_group()
    return 0 if ok else 1


if __name__ == "__main__":
    sys.exit(main())
