"""Benchmark: one Green iteration of treecode-accelerated Green Iteration on GB300.

A step is one pass of the whole hot path over one synthetic Li workload
(hydrogenic Li, adaptive mesh of ~309k points, 2 occupied orbitals plus the
Hartree sum, treecode degree 8, theta 0.7, leaf size 2000, FP32C):
  tree + batches + interaction lists + work items   (tagi_tree_build)
  field forming, anterpolation, near/far kernel,
  SS epilogue, eigenvalue update, Gram-Schmidt,
  normalisation, residuals, Hartree energy           (tagi_green_step)
with inputs resident in HBM.  The metric is treecode interactions per second:
one interaction = one (target, source-or-proxy, field) kernel evaluation,
counted from the interaction lists.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank solves its own independent workload (seed = rank):
weak scaling, no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "treecode kernel interactions/s at rel err 1e-6"
UNIT = "interactions/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tagi", choices=["tagi", "reference"])
    ap.add_argument("--no-plain", action="store_true", help="skip the FP64 plain-form comparison step")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-loop", action="store_true", help="skip the Green Iteration loop and SCF legs")
    ap.add_argument("--workload", default="li", choices=["li", "li-small", "co", "c6h6"],
                    help="li: the benchmark workload (309k points); li-small: tol_m 1e-3 mesh (99k) for "
                         "profiling; co (1.72M points, 7 orbitals + Hartree) and c6h6 (4.57M points, 21 orbitals "
                         "+ Hartree): the larger configurations, Green steps only")
    ap.add_argument("--profile-case", action="store_true",
                    help="build one tree and run two Green steps, nothing timed (for ncu captures)")
    ap.add_argument("--scf-steps", type=int, default=0,
                    help="c6h6: run this many SCF steps (Algorithm 1) from the aufbau start after the timed Green "
                         "steps, and report s per SCF step and Green iterations per step")
    ap.add_argument("--gi-max-iter", type=int, default=60, help="c6h6 SCF: Green Iteration steps per SCF step at most")
    ap.add_argument("--tol-m", type=float, default=None, help="co/c6h6: adaptive mesh tolerance (default: the "
                                                                "workload's, about 1.7M and 4.6M points)")
    ap.add_argument("--autotune", action="store_true",
                    help="pick degree, theta, leaf size and the work-item segment length with the autotuner "
                         "(quadrature-weighted error <= 1e-6) before the timed steps, and time that choice")
    return ap.parse_args()


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


WORKLOAD = "li"
SCF_START = False  # c6h6: the aufbau start of the SCF workload instead of seeded orbitals
TOL_M = None


def make_workload(seed):
    from paper_2003_01833_gb300 import workloads as W

    kw = {} if TOL_M is None else {"tol_m": TOL_M}
    if WORKLOAD == "co":
        return W.carbon_monoxide(seed=1 + seed, **kw)
    if WORKLOAD == "c6h6":
        return W.benzene_scf(**kw) if SCF_START else W.benzene(seed=2 + seed, **kw)
    return W.lithium(seed=seed, tol_m=1e-3) if WORKLOAD == "li-small" else W.lithium(seed=seed)


def kernel_traffic():
    """DRAM bytes per launch of k_interact32 on the benchmark workload, from
    the ncu capture summarised in profiles/, if that capture was taken on the
    current source of the kernel (else None)."""
    import hashlib

    src = os.path.join(ROOT, "paper_2003_01833_gb300", "csrc", "interact.cu")
    rec = os.path.join(ROOT, "profiles", "k_interact32_li309k_traffic.txt")
    if not os.path.exists(rec):
        return None
    digest = hashlib.sha256(open(src, "rb").read()).hexdigest()
    vals = dict(line.split()[:2] for line in open(rec) if line.strip() and not line.startswith("#"))
    if vals.get("interact_cu_sha256") != digest:
        return None
    return float(vals["dram_bytes_per_launch"])


def kernel_pipes():
    """ncu pipe utilisation of k_interact32 (small-case capture) from
    profiles/, while it was taken on the current source of the kernel."""
    import hashlib

    src = os.path.join(ROOT, "paper_2003_01833_gb300", "csrc", "interact.cu")
    rec = os.path.join(ROOT, "profiles", "k_interact32_li99k_pipes.txt")
    if not os.path.exists(rec):
        return None
    vals = dict(line.split()[:2] for line in open(rec) if line.strip() and not line.startswith("#"))
    if vals.pop("interact_cu_sha256", None) != hashlib.sha256(open(src, "rb").read()).hexdigest():
        return None
    return {k: float(v) for k, v in vals.items()}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ roofline model
# Thread instructions issued per pair in the FP32C kernel are counted from the
# source of tile_near / tile_far / tile_far_tensor (FP32 pipe + MUFU;
# shared-memory loads, the self-pair mask, the two-float folds and loop
# overhead excluded), see kernel_work.
ISSUE_PER_SM_CLK = 128  # 4 schedulers x 32 lanes, one warp instruction each per clock
# ex2.approx per SM per clock: measured live by tagi_unit_rates (the value
# below, from the same measurement on a GB300, serves only when none is given)
XU_EX2_PER_SM_CLK = 30.1
TF32_PER_BF16 = 1.1 / 2.25  # nominal dense tf32 : bf16 tensor throughput of the GB300


def kernel_work(info, ny, hh):
    """Work of one k_interact32 launch, summed over its pairs: FP32-pipe plus
    MUFU instructions per pair as counted from the kernel source, and MUFU
    work in ex2 units (rsqrt = 2).  Per pair:
      near (record path): 10 geometry (3 differences, r^2 in 3, rsqrt, r,
        r (w_hi + w_lo) in 2), 6 per Yukawa field, 5 for the Hartree field
        (2 where the entry leaves out the Gaussian, list flag bit2);
      far: 4 geometry on the tensor grid (degrees 6 and 8: one difference, one
        FMA, rsqrt, r), else 8; 5 per Yukawa field; Hartree 5 (1 without
        the Gaussian)."""
    tensor = info["degree"] in (6, 8)
    nn, nfar = info["near_pairs"], info["far_pairs"]
    nng, nfg = (info["near_pairs_nogauss"], info["far_pairs_nogauss"]) if hh else (0, 0)
    near_g, near_ng = 10 + 6 * ny + (5 if hh else 0), 10 + 6 * ny + (2 if hh else 0)
    geo = 4 if tensor else 8
    far_g, far_ng = geo + 5 * ny + (5 if hh else 0), geo + 5 * ny + (1 if hh else 0)
    instr = (nn - nng) * near_g + nng * near_ng + (nfar - nfg) * far_g + nfg * far_ng
    xu = (nn + nfar) * (2 + ny) + ((nn - nng) + (nfar - nfg)) * (1 if hh else 0)
    return instr, xu


def roofline(info, nfields_y, hh, kernel_ms, clk_mhz, sms, xu_rate=XU_EX2_PER_SM_CLK):
    """ALU roofline of k_interact32: the tighter of the issue bound (128
    instructions per SM per clock) and the MUFU bound (measured ex2 rate).
    Fields go to the kernel in launch groups of up to 8 (the Hartree field
    joins the last group when it fits), each group with its own geometry."""
    instr = xu = 0
    o = 0
    while o < nfields_y or (hh and o == nfields_y):
        g = min(8, nfields_y - o)
        g_hh = hh and o + g == nfields_y and g < 8
        i1, x1 = kernel_work(info, g, g_hh)
        instr += i1
        xu += x1
        o += g + (1 if g_hh else 0)
        if g_hh or (g == 0 and not hh):
            break
    nf = nfields_y + (1 if hh else 0)
    inter = (info["near_pairs"] + info["far_pairs"]) * nf
    f = clk_mhz * 1e6
    peak_issue = sms * ISSUE_PER_SM_CLK * f * inter / instr
    peak_xu = sms * xu_rate * f * inter / xu
    achieved = inter / (kernel_ms * 1e-3)
    return achieved, min(peak_issue, peak_xu), {"issue_bound": peak_issue, "mufu_bound": peak_xu,
                                                "instr_per_interaction": instr / inter,
                                                "mufu_ex2_units_per_interaction": xu / inter}


def measured_peaks():
    """MEASURED_PEAKS.json (driver-written) or None."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(p))
    except (OSError, ValueError):
        return None


def anterp_line(info, ncols, prof, steps, clk_mhz, sms):
    """Anterpolation of the step's fields (a4) on the tensor cores (3xTF32):
    algorithmic 2 P N_S flops per column summed over the approximated
    clusters, over the phase time, against the tf32 tensor peak (the measured
    bf16 peak x the nominal tf32 : bf16 ratio); the split precision executes 3x
    the algorithmic flops.  Also against the FP32 FMA peak, the bound of a
    SIMT form."""
    ms = prof["anterp"][0] / max(1, steps)
    flops = 2.0 * info["n_proxies"] * info["ant_points"] * ncols
    achieved = flops / (ms * 1e-3)
    fma_peak = sms * 128 * 2 * clk_mhz * 1e6
    mp = measured_peaks()
    bf16 = (mp or {}).get("bf16_tflops") or 1900.0
    tf32 = bf16 * TF32_PER_BF16 * 1e12
    return {"ms_per_step": ms, "algorithmic_flops": flops, "achieved_tflops": achieved / 1e12,
            "tf32_peak_tflops": tf32 / 1e12, "frac_tf32": achieved / tf32, "frac_tf32_executed": 3 * achieved / tf32,
            "tf32_peak_source": ("of measured: MEASURED_PEAKS.json bf16_tflops" if mp else "of fallback: 1.9 PFLOP/s")
                                + " x 1.1/2.25 nominal",
            "fp32_fma_peak_tflops": fma_peak / 1e12, "frac_fp32_fma": achieved / fma_peak,
            "note": "phase = charge split and tiling, 3xTF32 tcgen05 contraction with two-float folds, per-cluster "
                    "reduction; the basis rows are cached with the tree"}


# ------------------------------------------------------------------ oracle legs
def workload_name(wl):
    """The workload string both arms print in config.workload."""
    if wl.name == "Li":
        head = f"Li atom (hydrogenic Z=3, adaptive mesh p=4, tol_m {wl.meta.get('tol_m', 3e-7):g}): {wl.n} points, "
    else:
        head = f"{wl.name}, adaptive mesh p=4: {wl.n} points, "
    return head + f"{wl.psi.shape[0]} orbitals + Hartree, degree {wl.degree}, theta {wl.theta}, leaf {wl.leaf_size}"


def nucleus_batches(ot, xyz, nuclei, count=50):
    """Leaves holding the `count` mesh points nearest each nucleus: where the
    singularity subtraction cancels the most (f_i/k^2 >> |u_i|)."""
    leaf_of = np.empty(xyz.shape[1], dtype=np.int64)
    for c in ot.leaves:
        leaf_of[ot.points(c)] = c
    out = set()
    for R in nuclei:
        r = np.sqrt(((xyz - np.asarray(R, float)[:, None]) ** 2).sum(0))
        out.update(int(c) for c in leaf_of[np.argsort(r)[:count]])
    return sorted(out)


class OracleSample:
    """The float64 oracle treecode (as it stands, OpenMP over batches) on a
    bounded sample of a workload's target batches, all fields: the sample
    holds at least 2 batches per thread (so the dynamic batch schedule keeps
    every core busy) and always the batches that meet at the nuclei.  The
    oracle anterpolates every cluster on each call; that cost is timed once
    on its own (a call with no batch) and charged to a sample in proportion
    to its share of the batches, as a full run would amortise it."""

    def __init__(self, wl, nthreads=0, nuclei=((0.0, 0.0, 0.0),)):
        import oracle

        self.oracle = oracle
        self.wl = wl
        self.threads = oracle.threads(nthreads if nthreads > 0 else len(os.sched_getaffinity(0)))
        m = wl.mesh
        self.ot = ot = oracle.Tree(m.xyz, wl.leaf_size)
        b, c, k = ot.lists(wl.theta, wl.degree)
        P = (wl.degree + 1) ** 3
        self.size = ot.end - ot.begin
        self.per_batch = {}
        for bb, cc, kk in zip(b, c, k):
            self.per_batch[bb] = self.per_batch.get(bb, 0) + (P if kk == 1 else int(self.size[cc]))
        self.leaves = np.array(ot.leaves)
        self.nuc = nucleus_batches(ot, m.xyz, nuclei)
        self.fields = [(0, wl.k[o], wl.f[o]) for o in range(wl.psi.shape[0])] + [(1, wl.alpha, wl.rho)]
        self.t_ant = 0.0
        for kern, par, f in self.fields:
            ts = time.time()
            ot.treecode_batches(wl.theta, wl.degree, kern, par, f, m.w, [])
            self.t_ant += time.time() - ts

    def run(self, nbatch, seed=0, with_nucleus=True):
        """Time the sample; returns (interactions/s, description, the oracle's
        results per field restricted to the sample's targets, the targets,
        the nucleus targets)."""
        wl, ot = self.wl, self.ot
        rng = np.random.default_rng(seed)
        nuc = list(self.nuc) if with_nucleus else []
        rest = np.array([c for c in self.leaves if c not in set(nuc)])
        rng.shuffle(rest)
        nb = int(min(len(self.leaves), max(nbatch, len(nuc) + 1)))
        pick = np.array(nuc + list(rest[:nb - len(nuc)]))
        t_b, outs = 0.0, []
        for kern, par, f in self.fields:
            ts = time.time()
            outs.append(ot.treecode_batches(wl.theta, wl.degree, kern, par, f, wl.mesh.w, pick))
            t_b += time.time() - ts
        nf = len(self.fields)
        t_b -= self.t_ant  # every call re-anterpolated the whole tree; charged below by share
        inter = sum(self.per_batch[x] * int(self.size[x]) for x in pick) * nf
        share = len(pick) / len(self.leaves)
        desc = (f"{len(pick)} of {len(self.leaves)} target batches ({len(nuc)} at the nucleus, the rest "
                f"seeded) x {nf} fields of this workload on {self.threads} threads: {t_b:.2f} s of batch work + "
                f"{share:.3f} x {self.t_ant:.2f} s whole-tree anterpolation")
        pts = np.concatenate([ot.points(c) for c in pick])
        nuc_pts = np.concatenate([ot.points(c) for c in nuc]) if nuc else np.zeros(0, dtype=np.int64)
        return inter / (t_b + share * self.t_ant), desc, outs, pts, nuc_pts


def rel_err_vs_oracle(gpu_fields, outs, w, pts, nuc_pts, other_scale=None):
    """Relative L2 error of the GPU's fields against the oracle treecode at
    the same (n, theta), on the sample's targets: unweighted (over mesh
    points) and quadrature-weighted, for the nucleus batches and for the
    other sampled batches.  With other_scale (batches outside the nucleus
    set in the whole tree / those sampled) also a stratified estimate over
    the whole mesh: the nucleus batches are all in the sample, the others a
    seeded random sample of theirs."""
    res = {}
    other = np.setdiff1d(pts, nuc_pts)
    names = [f"psi{o}" for o in range(len(outs) - 1)] + ["hartree"]
    for name, g, ref in zip(names, gpu_fields, outs):
        row, sums = {}, {}
        for label, idx in (("nucleus", nuc_pts), ("other", other)):
            d = g[idx] - ref[idx]
            sums[label] = (np.sum(d * d), np.sum(ref[idx] ** 2), np.sum(d * d * w[idx]), np.sum(ref[idx] ** 2 * w[idx]))
            row[label] = {"plain": float(np.sqrt(sums[label][0] / sums[label][1])),
                          "weighted": float(np.sqrt(sums[label][2] / sums[label][3]))}
        if other_scale is not None:
            a, b = sums["nucleus"], sums["other"]
            tot = [a[i] + other_scale * b[i] for i in range(4)]
            row["whole_mesh_estimate"] = {"plain": float(np.sqrt(tot[0] / tot[1])),
                                          "weighted": float(np.sqrt(tot[2] / tot[3]))}
        res[name] = row
    return res


def run_reference(args):
    rank, world, local = dist_info()
    if rank != 0:
        return
    wl = make_workload(1)
    smp = OracleSample(wl)
    rates, desc = [], ""
    for i in range(args.warmup + args.steps):
        rate, desc, *_ = smp.run(2 * smp.threads, seed=i)
        if i >= args.warmup:
            rates.append(rate)
    v = float(np.mean(rates))
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": workload_name(wl), "model": "oracle treecode (float64 CPU)"},
           "cpu_baseline": {"kind": "oracle", "value": v, "unit": UNIT, "cores": smp.threads, "sample": desc},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------ ranks
def combine_ranks(ms, interactions, world, device):
    """Replicas: every rank times its own workload.  Returns the slowest
    rank's step time and the interactions of all ranks together (the
    whole-job rate is their ratio).  Uses whatever process group is open."""
    if world <= 1:
        return float(ms), float(interactions)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    tot = torch.tensor([float(interactions)], dtype=torch.float64, device=device)
    dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    return float(t.item()), float(tot.item())


# ------------------------------------------------------------------ GPU arm
def graph_replay(T, args, wl, xyz, w, params, veff, rho, vh, psi0, flush, inter, dev):
    """Time whole Green iterations replayed from a captured CUDA graph on a
    tree built once.  Capture needs a created stream, so this runs on one."""
    import torch

    nw = wl.psi.shape[0]
    side = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(side):
        h = T.tagi_tree_build(xyz, w, params)
        psi_g = psi0.clone()
        eps_g = torch.tensor(wl.eps, device=dev)
        res_g = torch.empty(nw, dtype=torch.float64, device=dev)
        eh_g = torch.empty(1, dtype=torch.float64, device=dev)
        g = T.tagi_green_graph_create(h, veff, wl.vshift, psi_g, eps_g, res_g, rho=rho, vh=vh, eh=eh_g)
        eps0 = eps_g.clone()
        times = []
        for i in range(args.warmup + args.steps):
            # the same first iteration every time (the synthetic start is not
            # an eigenstate; repeated iterations would walk away from it)
            psi_g.copy_(psi0)
            eps_g.copy_(eps0)
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(side)
            T.tagi_green_graph_launch(g)
            e1.record(side)
            torch.cuda.synchronize()
            if i >= args.warmup:
                times.append(e0.elapsed_time(e1))
        T.tagi_green_graph_check(g)
        T.tagi_green_graph_destroy(g)
        T.tagi_tree_destroy(h)
    ms = float(np.median(times))
    return {"ms_per_green_iteration": ms, "interactions_per_s": inter / (ms * 1e-3), "replays": len(times),
            "statistic": "median of the timed replays (CUDA events, L2 flushed before each)",
            "note": "tree built once; each replay is one whole Green iteration (a3-a8) from a CUDA graph"}


def gi_loop(T, wl, xyz, w, params, veff, psi0, tol_gi=1e-5, max_iter=80):
    """Green Iteration to tol_gi from the seeded start on one tree (Algorithm
    2), with Anderson mixing of eigenpairs (beta 0.5, 5 past pairs) and
    without; wall-clock seconds per loop, steps, and convolved orbital-steps."""
    import torch

    out = {"tol_gi": tol_gi, "max_iter": max_iter, "beta": 0.5, "history": 5}
    h = T.tagi_tree_build(xyz, w, params)
    try:
        for name, kw in (("mixed", {}), ("plain", {"mix_tol": 0.0})):
            psi = psi0.clone()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            try:
                r = T.tagi_green_iterate(h, veff, wl.vshift, psi, wl.eps, tol_gi, max_iter, **kw)
            except T.TagiError as e:
                out[name] = {"error": str(e)}
                continue
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            out[name] = {"s": dt, "steps": r["steps"], "converged": r["n_converged"],
                         "field_steps": r["field_steps"], "iters": [int(x) for x in r["iters"]],
                         "eps": [float(x) for x in r["eps"]], "ms_per_step": 1e3 * dt / max(1, r["steps"])}
    finally:
        T.tagi_tree_destroy(h)
    return out


KT_200K = 200.0 * 3.166811563e-6  # k_B T at 200 K in Ha (Section 6)
# Table timings (Section 6): E_TAGI minus its error against the DFT-FE
# reference (Ha per atom times the atoms), i.e. the reference energy
E_REF = {"Li": -7.334051 - 4.59e-4, "C6H6": -230.193158 + 12 * 3.64e-4}
E_REF_LI = E_REF["Li"]


def scf_loop(T, wl, xyz, w, params, max_steps=30, tol_scf=1e-4, store_output=False, gi_max_iter=100):
    """SCF iteration (Algorithm 1) from the superposition density to
    ||rho_out - rho_in||_w < tol_scf on one tree: wall-clock seconds per SCF
    step, Green Iteration steps per SCF step, and the converged energy.
    store_output: converged orbitals keep their Green step's output rather
    than its input (Algorithm 2's rule)."""
    import torch

    dev = xyz.device
    h = T.tagi_tree_build(xyz, w, params)
    out = {"tol_scf": tol_scf, "kT_ha": KT_200K, "tol_gi": "3e-3 -> 1e-5 over 4 steps (Section 6)",
           "gi_store_output": bool(store_output)}
    try:
        with T.Scf(h, wl.n_elec, kT=KT_200K, e_zz=wl.e_zz, gi_store_output=store_output,
                   gi_max_iter=gi_max_iter) as scf:
            rho = torch.tensor(wl.rho, device=dev)
            psi = torch.tensor(wl.psi, device=dev)
            vx = torch.tensor(wl.vext, device=dev)
            eps = wl.eps
            times, res, gis, energies = [], [], [], []
            for _ in range(max_steps):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rep = scf.step(vx, wl.vshift, rho, psi, eps)
                torch.cuda.synchronize()
                times.append(time.perf_counter() - t0)
                eps = rep["eps"]
                res.append(rep["residual"])
                gis.append(rep["gi"]["steps"])
                energies.append(rep["e_total"])
                if rep["residual"] < tol_scf:
                    break
        ref = E_REF.get(wl.name)
        out.update({"steps": len(times), "converged": res[-1] < tol_scf, "s_total": float(sum(times)),
                    "s_per_scf_step": float(np.mean(times)), "s_per_step_each": times, "gi_steps": gis,
                    "s_per_green_iteration": float(sum(times)) / max(1, sum(gis)), "residuals": res,
                    "energies": energies, "e_total": energies[-1], "eps": [float(x) for x in eps],
                    "e_ref_paper": ref, "error_ha": energies[-1] - ref if ref is not None else None,
                    "gi_max_iter": gi_max_iter})
    except T.TagiError as e:
        out["error"] = str(e)
    finally:
        T.tagi_tree_destroy(h)
    return out


def profile_case(args):
    """One tree and two Green steps, nothing else: the command ncu wraps."""
    import torch

    import paper_2003_01833_gb300.tagi as T

    wl = make_workload(1)
    dev = torch.device("cuda", 0)
    t = lambda a: torch.tensor(a, device=dev)
    with T.Tree(t(wl.mesh.xyz), t(wl.mesh.w), theta=wl.theta, degree=wl.degree, leaf_size=wl.leaf_size,
                prec=T.TAGI_FP32C) as tr:
        vh = torch.empty(wl.n, dtype=torch.float64, device=dev)
        for _ in range(2):
            psi = t(wl.psi)
            eps, res, eh = T.tagi_green_step(tr.handle, t(wl.veff), wl.vshift, psi, wl.eps, rho=t(wl.rho), vh=vh)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": WORKLOAD, "n": wl.n, "eps": [float(x) for x in eps]}))


def main():
    global WORKLOAD, SCF_START, TOL_M
    args = parse()
    WORKLOAD = args.workload
    SCF_START = WORKLOAD == "c6h6" and args.scf_steps > 0
    TOL_M = args.tol_m if WORKLOAD in ("co", "c6h6") else None
    if args.profile_case:
        profile_case(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    import torch

    import paper_2003_01833_gb300.tagi as T

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    T.lib()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    wl = make_workload(seed=1 + rank)
    n = wl.n
    nw = wl.psi.shape[0]
    xyz = torch.tensor(wl.mesh.xyz, device=dev)
    w = torch.tensor(wl.mesh.w, device=dev)
    veff = torch.tensor(wl.veff, device=dev)
    rho = torch.tensor(wl.rho, device=dev)
    psi0 = torch.tensor(wl.psi, device=dev)
    psi = psi0.clone()
    vh = torch.empty(n, dtype=torch.float64, device=dev)
    tuned = None
    if args.autotune:
        from paper_2003_01833_gb300 import autotune as A

        t0 = time.perf_counter()
        best, trials, ref = A.autotune(xyz, w, torch.tensor(wl.f, device=dev), list(wl.k), rho=rho, tol=1e-6,
                                       norm="weighted", **A.grid_for(n))
        tuned = {"norm": "weighted", "tol": 1e-6, "reference": list(ref), "trials": len(trials),
                 "seconds": time.perf_counter() - t0,
                 "choice": None if best is None else {"degree": best.degree, "theta": best.theta,
                                                      "leaf_size": best.leaf_size, "segment": best.segment,
                                                      "conv_ms": best.conv_ms, "err_weighted": best.err_weighted,
                                                      "err_l2": best.err_l2}}
        if best is not None:
            wl.degree, wl.theta, wl.leaf_size = best.degree, best.theta, best.leaf_size
    seg = tuned["choice"]["segment"] if tuned and tuned["choice"] else 0
    params = T.make_params(theta=wl.theta, degree=wl.degree, leaf_size=wl.leaf_size, prec=T.TAGI_FP32C, segment=seg)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > L2 (129 MB)
    stream = torch.cuda.current_stream()

    def step(psi_buf):
        h = T.tagi_tree_build(xyz, w, params)
        psi_buf.copy_(psi0)
        eps, res, eh = T.tagi_green_step(h, veff, wl.vshift, psi_buf, wl.eps, rho=rho, vh=vh)
        return h, eps, res, eh

    # ---- warm-up
    for _ in range(args.warmup):
        h, *_ = step(psi)
        T.tagi_tree_destroy(h)
    torch.cuda.synchronize()

    # ---- timed steps (device resident inputs), L2 flushed before each step
    T.tagi_profile_enable(True)
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    times = []
    info = None
    launches0 = T.tagi_kernel_launches()
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h, eps, res, eh = step(psi)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        if info is None:
            info = T.tagi_tree_info(h)
        T.tagi_tree_destroy(h)
    launches = (T.tagi_kernel_launches() - launches0 - 0) / args.steps
    barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    prof = {g: T.tagi_profile_read(g) for g in T.PROFILE_GROUPS}
    T.tagi_profile_enable(False)
    ms = float(np.mean(times))
    nf = nw + 1
    inter = (info["near_pairs"] + info["far_pairs"]) * nf
    t_max, inter_all = combine_ranks(ms, inter, world, dev)
    value = inter_all / (t_max * 1e-3)

    # ---- Green iterations replayed from a captured CUDA graph (fixed tree)
    graph = graph_replay(T, args, wl, xyz, w, params, veff, rho, vh, psi0, flush, inter, dev) if rank == 0 else None

    # ---- Green Iteration to convergence (fixed V_eff), with and without mixing
    loop = gi_loop(T, wl, xyz, w, params, veff, psi0) if (rank == 0 and not args.no_loop and
                                                          WORKLOAD in ("li", "li-small")) else None
    scf = scf_loop(T, wl, xyz, w, params) if (rank == 0 and not args.no_loop and WORKLOAD == "li") else None
    scf_so = scf_loop(T, wl, xyz, w, params, store_output=True) if scf is not None else None
    if rank == 0 and SCF_START:
        # config 4: C6H6 SCF steps from the aufbau start (stored Green step
        # outputs, c34), the s per SCF step of the metric
        scf = scf_loop(T, wl, xyz, w, params, max_steps=args.scf_steps, store_output=True,
                       gi_max_iter=args.gi_max_iter)
    lithium = WORKLOAD in ("li", "li-small")  # the other workloads time Green steps only

    # ---- end to end through the public API: pinned host inputs -> device,
    # step, results -> host, all inside the timed region
    hx = torch.tensor(wl.mesh.xyz).pin_memory()
    hw = torch.tensor(wl.mesh.w).pin_memory()
    hv = torch.tensor(wl.veff).pin_memory()
    hr = torch.tensor(wl.rho).pin_memory()
    hp = torch.tensor(wl.psi).pin_memory()
    out_psi = torch.empty_like(hp).pin_memory()
    out_vh = torch.empty(n, dtype=torch.float64).pin_memory()
    dx, dw, dv, dr, dp = (torch.empty_like(a, device=dev) for a in (hx, hw, hv, hr, hp))
    dvh = torch.empty(n, dtype=torch.float64, device=dev)
    e2e_times = []
    for i in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for d_, h_ in ((dx, hx), (dw, hw), (dv, hv), (dr, hr), (dp, hp)):
            d_.copy_(h_, non_blocking=True)
        hh = T.tagi_tree_build(dx, dw, params)
        T.tagi_green_step(hh, dv, wl.vshift, dp, wl.eps, rho=dr, vh=dvh)
        out_psi.copy_(dp, non_blocking=True)
        out_vh.copy_(dvh, non_blocking=True)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e_times.append(time.perf_counter() - t0)
        T.tagi_tree_destroy(hh)
    e2e_s = float(np.mean(e2e_times))
    h2d = 8 * n * (3 + 1 + 1 + 1 + nw)
    d2h = 8 * n * (nw + 1)

    # ---- plain FP64 form: one orbital per launch, same tree, no graph.  One
    # warm-up and three timed Green iterations on a tree built once, beside
    # the FP32C eager Green iteration timed the same way.
    plain = None
    if not args.no_plain and rank == 0 and lithium:
        def time_steps(prm, count, warm):
            hh = T.tagi_tree_build(xyz, w, prm)
            ts, res = [], None
            for i in range(warm + count):
                pb = psi0.clone()
                flush.zero_()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                r = T.tagi_green_step(hh, veff, wl.vshift, pb, wl.eps, rho=rho, vh=vh)
                e1.record(stream)
                torch.cuda.synchronize()
                if i >= warm:
                    ts.append(e0.elapsed_time(e1))
                res = (pb, r)
            T.tagi_tree_destroy(hh)
            return ts, res
        pp = T.make_params(theta=wl.theta, degree=wl.degree, leaf_size=wl.leaf_size, prec=T.TAGI_FP64)
        t64, (psi64, (eps64, _, eh64)) = time_steps(pp, 3, 1)
        t32, (psi32, (eps32, _, eh32)) = time_steps(params, 10, 3)
        a, b = psi32.cpu().numpy(), psi64.cpu().numpy()
        rel = [float(np.linalg.norm(a[o] - b[o]) / np.linalg.norm(b[o])) for o in range(nw)]
        p_ms, f_ms = float(np.median(t64)), float(np.median(t32))
        plain = {"s_per_green_iteration_fp64_plain": p_ms * 1e-3, "plain_times_ms": t64,
                 "s_per_green_iteration_fp32c_eager": f_ms * 1e-3,
                 "speedup_vs_plain": p_ms / f_ms,
                 "speedup_vs_plain_graph": p_ms / graph["ms_per_green_iteration"] if graph else None,
                 "statistic": "median of 3 plain (after 1 warm-up) and of 10 FP32C (after 3) Green iterations "
                              "on a tree built once, CUDA events, L2 flushed before each",
                 "fp32c_vs_fp64_psi_rel_l2": rel, "fp32c_vs_fp64_eps_abs": [float(x) for x in np.abs(eps32 - eps64)],
                 "fp32c_vs_fp64_eh_abs": abs(eh32 - eh64)}
        if scf is not None and "gi_steps" in scf:
            gi = float(np.mean(scf["gi_steps"]))
            plain["s_per_scf_step_fp64_plain_estimate"] = gi * p_ms * 1e-3
            plain["scf_estimate_note"] = (f"estimate, not measured: {gi:.1f} Green iterations per SCF step (the "
                                          "FP32C SCF leg) x the measured plain s per Green iteration")
            plain["speedup_vs_plain_per_scf_step_estimate"] = gi * p_ms * 1e-3 / scf["s_per_scf_step"]

    if rank != 0:
        return
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    k_ms, k_cnt = prof["interact"]
    k_ms_per_step = k_ms / max(1, args.steps)
    clk_mhz = clk.get("sm_mhz") or 1900.0
    rates = T.tagi_unit_rates()
    achieved, peak, bounds = roofline(info, nw, True, k_ms_per_step, clk_mhz, sms, xu_rate=rates["ex2"])
    cpu, rel_err = None, None
    if not args.no_cpu and lithium:
        # the fields of the step's convolutions on the GPU, for the error
        # against the oracle on the oracle's own sample
        hh = T.tagi_tree_build(xyz, w, params)
        ug = torch.empty((nw, n), dtype=torch.float64, device=dev)
        T.tagi_fields_conv(hh, torch.tensor(wl.f, device=dev), list(wl.k), ug, rho=rho, vh=vh)
        torch.cuda.synchronize()
        gpu_fields = list(ug.cpu().numpy()) + [vh.cpu().numpy()]
        T.tagi_tree_destroy(hh)
        smp = OracleSample(wl)
        nb_sample = 2 * smp.threads
        rate, desc, outs, pts, nuc_pts = smp.run(nb_sample, seed=0)
        n_other = len(smp.leaves) - len(smp.nuc)
        rel_err = rel_err_vs_oracle(gpu_fields, outs, wl.mesh.w, pts, nuc_pts,
                                    other_scale=n_other / max(1, nb_sample - len(smp.nuc)))
        smp1 = OracleSample(wl, nthreads=1)
        rate1, desc1, *_ = smp1.run(2, seed=1, with_nucleus=False)
        smp.oracle.threads(smp.threads)
        cpu = {"value": rate, "unit": UNIT, "cores": smp.threads, "kind": "oracle", "sample": desc,
               "value_1_core": rate1, "sample_1_core": desc1}
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32c", "data": "synthetic",
        "config": {"workload": workload_name(wl), "segment": seg or 8192,
                   "step": "tree+lists+items, fields, anterpolation, near/far kernel, SS epilogue, "
                           "eps update, MGS, residuals, E_H",
                   "interactions_per_step": inter, "near_pairs": info["near_pairs"], "far_pairs": info["far_pairs"],
                   "l2": "flushed (256 MB write) before each timed step", "parallelism": f"replicas x{world}"},
        "s_per_green_iteration": t_max * 1e-3,
        "phases_ms_per_step": {g: prof[g][0] / max(1, args.steps) for g in prof},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "interactions/s",
                     "frac": achieved / peak, "traffic": kernel_traffic() if WORKLOAD == "li" else None,
                     "kernel": "k_interact32 (near/far)", **bounds,
                     "ncu_small_case_pct": kernel_pipes() if lithium else None,
                     "unit_rates_per_sm_clk": rates,
                     "peak_model": f"min(issue: {sms} SMs x 128 instr/clk, MUFU: {sms} SMs x "
                                   f"{rates['ex2']:.1f} ex2/clk measured live by tagi_unit_rates) x {clk_mhz:.0f} MHz "
                                   "(measured clock) over the per-interaction counts; not MEASURED_PEAKS.json "
                                   "(HBM and bf16 tensor peaks do not bound this kernel)"},
        "rel_err_vs_oracle": rel_err,
        "autotune": tuned,
        "clocks": clk,
        "e2e": {"value": inter_all / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "s_per_step": e2e_s},
        "gpu_launches": launches,
        "anterpolation": anterp_line(info, nf, prof, args.steps, clk_mhz, sms),
        "graph_replay": graph,
        "scf_store_output": scf_so,
        "green_iteration_loop": loop,
        "scf": scf,
        "plain_fp64": plain,
        "cpu_baseline": cpu,
    }
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
