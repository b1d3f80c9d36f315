"""Choice of the treecode parameters -- interpolation degree n, MAC theta and
leaf size N_L (Section 5) -- and of the near/far kernel's work-item segment
length (sources per item: a tile shape of the kernel) under an error bar, for
one mesh and one set of fields.

Every candidate builds its tree and runs the one-pass convolution of the
fields (tagi_fields_conv, the work of a Green iteration on a tree built once).
Its error is the relative L2 norm per field against a tight reference
configuration evaluated in the plain float64 form (or, on meshes where that
form is too slow, the FP32C form at the tight configuration, whose own error
is ~1e-7), in one of two norms: the
plain one over mesh points, or the quadrature-weighted one that Green
Iteration's convergence test uses.  The choice is the candidate with the
shortest convolution time whose largest error in the chosen norm stays below
the bar.  Host logic over the library's calls: every evaluation runs the CUDA
path.

Next to a nucleus the singularity subtraction cancels f_i/k^2 of up to ~10^3
times the result, so the float32 kernel sums of the FP32C form carry errors
of ~1e-5 at the few mesh points there whatever (n, theta, N_L) is; the plain
norm then finds no candidate within 1e-6 on all-electron meshes while the
weighted norm, in which those points have tiny volume, does.
"""
from __future__ import annotations

import math
import time
from dataclasses import asdict, dataclass

import numpy as np

from . import tagi as T


@dataclass
class Trial:
    degree: int
    theta: float
    leaf_size: int
    segment: int
    build_ms: float
    conv_ms: float
    max_rel_err: float
    interactions: int
    err_l2: float = float("nan")
    err_weighted: float = float("nan")

    def ok(self, tol: float) -> bool:
        return bool(np.isfinite(self.max_rel_err) and self.max_rel_err <= tol)


def select(trials, tol):
    """The trial with the shortest convolution time among those within tol
    (None if there is none)."""
    good = [t for t in trials if t.ok(tol)]
    return min(good, key=lambda t: t.conv_ms) if good else None


def _conv(tree, f, k, rho, u, vh):
    T.tagi_fields_conv(tree.handle, f, k, u, rho=rho, vh=vh)


def _measure(xyz, w, f, k, rho, degree, theta, leaf_size, prec, reps, segment=0):
    import torch

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tree = T.Tree(xyz, w, theta=theta, degree=degree, leaf_size=leaf_size, prec=prec, segment=segment)
    torch.cuda.synchronize()
    build_ms = 1e3 * (time.perf_counter() - t0)
    try:
        n = xyz.shape[1]
        u = torch.empty((f.shape[0], n), dtype=torch.float64, device=xyz.device)
        vh = torch.empty(n, dtype=torch.float64, device=xyz.device) if rho is not None else None
        _conv(tree, f, k, rho, u, vh)  # warm-up (the only run when reps is 0)
        times = []
        stream = torch.cuda.current_stream()
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _conv(tree, f, k, rho, u, vh)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        info = T.tagi_tree_info(tree.handle)
        nf = f.shape[0] + (1 if rho is not None else 0)
        inter = (info["near_pairs"] + info["far_pairs"]) * nf
        rows = [u[o].cpu().numpy() for o in range(f.shape[0])]
        if rho is not None:
            rows.append(vh.cpu().numpy())
        return build_ms, float(np.median(times)) if times else math.nan, rows, inter
    finally:
        tree.close()


def rel_errors(rows, ref_rows, w):
    """Largest relative error over the fields, plain and quadrature-weighted
    L2 norms (w: host quadrature weights)."""
    l2 = max(float(np.linalg.norm(a - r) / np.linalg.norm(r)) for a, r in zip(rows, ref_rows))
    wt = max(float(np.sqrt(np.sum((a - r) ** 2 * w) / np.sum(r * r * w))) for a, r in zip(rows, ref_rows))
    return l2, wt


def autotune(xyz, w, f, k, rho=None, tol=1e-6, norm="l2", degrees=(6, 8), thetas=(0.5, 0.6, 0.7, 0.8),
             leaf_sizes=(1000, 2000, 4000), segments=(8192,), reference=(8, 0.4, 2000), prec=None, prec_ref=None,
             reps=3):
    """xyz (3, n), w (n,), f (nf, n), rho (n,) or None: float64 CUDA tensors;
    k: nf decay rates; norm: "l2" or "weighted".  The candidates run in prec
    (FP32C by default), the reference in prec_ref (the plain float64 form by
    default).  Returns (best Trial or None, all trials, reference
    configuration)."""
    if norm not in ("l2", "weighted"):
        raise ValueError("norm must be 'l2' or 'weighted'")
    prec = T.TAGI_FP32C if prec is None else prec
    prec_ref = T.TAGI_FP64 if prec_ref is None else prec_ref
    _, _, ref_rows, _ = _measure(xyz, w, f, k, rho, reference[0], reference[1], reference[2], prec_ref, 0)
    wh = w.cpu().numpy()
    trials = []
    for n in degrees:
        for th in thetas:
            for nl in leaf_sizes:
                for sg in segments:
                    b_ms, c_ms, rows, inter = _measure(xyz, w, f, k, rho, n, th, nl, prec, reps, sg)
                    l2, wt = rel_errors(rows, ref_rows, wh)
                    trials.append(Trial(n, th, nl, sg, b_ms, c_ms, l2 if norm == "l2" else wt, int(inter), l2, wt))
    return select(trials, tol), trials, reference


def grid_for(n):
    """The search grid for an n-point mesh: the full grid (with segment
    lengths 4096, 8192 and 16384) up to 400,000 points; above that a
    narrower one and the FP32C form as the reference (the plain float64 form
    takes minutes per convolution there)."""
    if n <= 400_000:
        return {"segments": (4096, 8192, 16384)}
    return {"degrees": (6, 8), "thetas": (0.6, 0.7, 0.8), "leaf_sizes": (2000, 4000), "segments": (8192, 16384),
            "prec_ref": T.TAGI_FP32C, "reps": 2}


def report(best, trials, reference, tol, norm="l2"):
    """JSON-ready summary."""
    return {"tol": tol, "norm": norm,
            "reference": {"degree": reference[0], "theta": reference[1], "leaf_size": reference[2]},
            "best": asdict(best) if best else None, "trials": [asdict(t) for t in trials]}


def main(argv=None):
    """python -m paper_2003_01833_gb300.autotune [--workload li|li-small|h]
    prints one JSON object: the trials and the choice."""
    import argparse
    import json

    import torch

    from . import workloads as W

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="li-small", choices=["li", "li-small", "h", "co"])
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--norm", default="l2", choices=["l2", "weighted"])
    a = ap.parse_args(argv)
    wl = {"li": lambda: W.lithium(), "li-small": lambda: W.lithium(tol_m=1e-3),
          "h": lambda: W.hydrogen_adaptive(), "co": lambda: W.carbon_monoxide()}[a.workload]()
    dev = lambda x: torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")
    best, trials, ref = autotune(dev(wl.mesh.xyz), dev(wl.mesh.w), dev(wl.f), list(wl.k), rho=dev(wl.rho),
                                 tol=a.tol, norm=a.norm, **grid_for(wl.n))
    out = report(best, trials, ref, a.tol, a.norm)
    out["workload"] = {"name": wl.name, "points": int(wl.n), "fields": int(len(wl.k)) + 1}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
