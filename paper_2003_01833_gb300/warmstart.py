"""Learned warm start for SCF runs of molecules: a small per-point MLP that
predicts the converged orbital from features of the geometry (distances to
the nuclei and the superposed atomic Slater orbitals), and a second one that
predicts the eigenvalue from the bond length.  Both are trained on converged
orbitals that this solver's own SCF iteration (Algorithm 1 with Green
Iteration) produces for perturbed geometries; the plain superposition of
atomic orbitals stays the fallback, and plain Green Iteration measures the
prediction: the SCF run from the predicted start is compared with the run
from the superposition start.

The orbital model predicts a relative correction y(x) of the normalised
superposition start s(x): psi_warm = s (1 + y), normalised.  Its training
target is t = psi* / s - 1 and its loss the quadrature-weighted
sum_p w_p s_p^2 (y_p - t_p)^2, which is the squared orbital error
||psi_warm - psi*||_w^2 before normalisation.

The data set of H2 runs: `h2_bond_lengths` (32 seeded bond lengths in
[1, 2] Bohr), meshes from `workloads.hydrogen_molecule`.  The network has 64
hidden units by default (the tensor-core kernels; 32 selects the SIMT ones).

Measure: an SCF run ends when ||rho_out - rho_in||_w < tol_scf and the
total energy has settled, |E_k - E_{k-1}| < 1e-6 Ha; the steps, Green
iterations and wall time until the energy first settles are reported for
both starts.
"""
from __future__ import annotations

import time

import numpy as np

from . import workloads as W

KT_200K = 200.0 * 3.166811563e-6  # k_B T at 200 K in Ha (Section 6)


def _dev(torch, a, device="cuda"):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=device)


E_TOL = 1e-6  # Ha: the total energy has settled when successive SCF steps differ by less


def scf_run(wl, psi0=None, eps0=None, rho0=None, tol_scf=1e-4, max_steps=40, prec=None, store_output=True,
            e_tol=E_TOL):
    """SCF iteration on the device from (psi0, eps0, rho0) (the workload's
    superposition start where None) until ||rho_out - rho_in||_w < tol_scf.
    Returns the converged orbitals (host), eigenvalues, energy and the cost:
    SCF steps and Green iterations.

    store_output: converged orbitals keep their Green step's output.  With
    Algorithm 2's rule (the step input) an orbital whose first step in an SCF
    iteration moves it by less than tol_gi is not updated at all, the density
    residual then falls by mixing alone, and runs from different starts end
    at energies up to ~1e-4 Ha apart; keeping the output makes every SCF
    iteration follow V_eff[rho_in], so both starts reach one fixed point."""
    import torch

    from . import tagi as T

    prec = T.TAGI_FP32C if prec is None else prec
    m = wl.mesh
    psi0 = wl.psi if psi0 is None else psi0
    eps = np.array(wl.eps if eps0 is None else eps0, dtype=np.float64)
    rho0 = wl.rho if rho0 is None else rho0
    hist = []
    t0 = time.perf_counter()
    with T.Tree(_dev(torch, m.xyz), _dev(torch, m.w), theta=wl.theta, degree=wl.degree, leaf_size=wl.leaf_size,
                prec=prec) as tr, T.Scf(tr.handle, wl.n_elec, kT=KT_200K, e_zz=wl.e_zz,
                                        gi_store_output=store_output) as scf:
        rho, psi, vx = _dev(torch, rho0), _dev(torch, psi0), _dev(torch, wl.vext)
        rep = None
        error = None
        settled = None  # (steps, Green iterations, seconds) when |dE| < e_tol first held
        for _ in range(max_steps):
            try:
                rep = scf.step(vx, wl.vshift, rho, psi, eps)
            except T.TagiError as e:  # e.g. eps + V_shift >= 0 (Section 3.3): the run has failed
                error = str(e)
                break
            eps = rep["eps"]
            hist.append({"residual": rep["residual"], "e_total": rep["e_total"], "gi_steps": rep["gi"]["steps"],
                         "eps": [float(e) for e in eps], "seconds": time.perf_counter() - t0})
            if settled is None and len(hist) > 1 and abs(hist[-1]["e_total"] - hist[-2]["e_total"]) < e_tol:
                settled = (len(hist), int(sum(h["gi_steps"] for h in hist)), hist[-1]["seconds"])
            if rep["residual"] < tol_scf and settled is not None:
                break
        psi_h = psi.cpu().numpy()
        rho_h = rho.cpu().numpy()
    torch.cuda.synchronize()
    ok = error is None and rep is not None and rep["residual"] < tol_scf
    return {"psi": psi_h, "rho": rho_h, "eps": np.array(eps), "e_total": rep["e_total"] if rep else float("nan"),
            "converged": bool(ok), "error": error,
            "scf_steps": len(hist), "gi_steps": int(sum(h["gi_steps"] for h in hist)), "history": hist,
            "seconds": time.perf_counter() - t0,
            "energy_settled": None if settled is None else {"scf_steps": settled[0], "gi_steps": settled[1],
                                                            "seconds": settled[2], "e_tol": e_tol}}


def generate(bond_lengths, tol_m=3e-6, tol_scf=1e-4, log=print):
    """Converged H2 runs from the superposition start, one per bond length.
    Returns a list of records (R, n, mesh weight sum, psi* as float32, eps*,
    E, cost)."""
    out = []
    for R in bond_lengths:
        wl = W.hydrogen_molecule(float(R), tol_m=tol_m)
        r = scf_run(wl, tol_scf=tol_scf)
        psi = r["psi"][0]
        if np.sum(psi * wl.psi[0] * wl.mesh.w) < 0:  # the sign of an eigenvector is free
            psi = -psi
        rec = {"R": float(R), "n": wl.n, "w_sum": float(np.sum(wl.mesh.w)), "psi": psi.astype(np.float32),
               "eps": float(r["eps"][0]), "e_total": float(r["e_total"]), "converged": bool(r["converged"]),
               "scf_steps": r["scf_steps"], "gi_steps": r["gi_steps"], "seconds": r["seconds"]}
        log(f"R {R:.4f} n {wl.n} eps {rec['eps']:.6f} E {rec['e_total']:.6f} scf {rec['scf_steps']} "
            f"gi {rec['gi_steps']} {rec['seconds']:.2f} s")
        out.append(rec)
    return out


def save(records, path):
    np.savez_compressed(path, **{f"{k}_{i}": np.asarray(v) for i, r in enumerate(records) for k, v in r.items()},
                        count=len(records))


def load(path):
    z = np.load(path)
    keys = ("R", "n", "w_sum", "psi", "eps", "e_total", "converged", "scf_steps", "gi_steps", "seconds")
    return [{k: (z[f"{k}_{i}"] if k == "psi" else z[f"{k}_{i}"].item()) for k in keys} for i in range(int(z["count"]))]


# ---------------------------------------------------------------- training
def _nuclei(wl):
    return np.asarray(wl.meta["nuclei"], dtype=np.float64)


def _midpoint_features(T, torch, nuclei):
    """Features at the midpoint of the two nuclei: a function of the bond
    length alone, the eigenvalue model's input."""
    mid = _dev(torch, (0.5 * (nuclei[0] + nuclei[1])).reshape(3, 1))
    return T.tagi_mlp_features(mid, nuclei)


def cosine_lr(lr0, steps):
    return lambda k: 0.5 * lr0 * (1.0 + np.cos(np.pi * (k - 1) / steps))


def train(records, train_idx, steps=3000, lr=3e-3, seed=0, tol_m=3e-6, hidden=64, log=print):
    """Trains the orbital model on the converged runs records[i], i in
    train_idx (full-batch Adam on the device, cosine step size), and the
    eigenvalue model on their eigenvalues.  Returns (orbital Mlp, eigenvalue
    Mlp, info)."""
    import torch

    from . import tagi as T

    feats, targets, wts, mids, eps = [], [], [], [], []
    G = len(train_idx)
    for i in train_idx:
        r = records[i]
        wl = W.hydrogen_molecule(r["R"], tol_m=tol_m)
        if wl.n != r["n"]:
            raise RuntimeError(f"mesh of R = {r['R']} has {wl.n} points, the record {r['n']}")
        s = wl.psi[0]
        feats.append(T.tagi_mlp_features(_dev(torch, wl.mesh.xyz), _nuclei(wl)))
        targets.append(torch.tensor((r["psi"].astype(np.float64) / s - 1.0).astype(np.float32), device="cuda"))
        wts.append(torch.tensor((wl.mesh.w * s * s / G).astype(np.float32), device="cuda"))
        mids.append(_midpoint_features(T, torch, _nuclei(wl)))
        eps.append(r["eps"])
    feat, target, wt = torch.cat(feats), torch.cat(targets), torch.cat(wts)
    del feats, targets, wts
    orb = T.Mlp(W.mlp_init(seed, hidden=hidden), hidden=hidden)
    sched = cosine_lr(lr, steps)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = []
    for k in range(1, steps + 1):
        want = k == 1 or k % 500 == 0 or k == steps
        L = orb.train_step(feat, target, wt, sched(k), want_loss=want)
        if want:
            losses.append((k, L))
    torch.cuda.synchronize()
    t_orb = time.perf_counter() - t0
    # eigenvalue model: one "point" per geometry
    mfeat = torch.cat(mids)
    et = torch.tensor(np.array(eps, dtype=np.float32), device="cuda")
    ew = torch.full((G,), 1.0 / G, dtype=torch.float32, device="cuda")
    eig = T.Mlp(W.mlp_init(seed + 1, hidden=hidden), hidden=hidden)
    for k in range(1, steps + 1):
        eig.train_step(mfeat, et, ew, sched(k))
    e_loss = eig.gradient(mfeat, et, ew)[0]
    info = {"points": int(feat.shape[0]), "geometries": G, "steps": steps, "lr": lr, "losses": losses,
            "hidden": hidden,
            "seconds": t_orb, "ms_per_step": 1e3 * t_orb / steps, "eig_rms": float(np.sqrt(e_loss)),
            "R_range": [min(records[i]["R"] for i in train_idx), max(records[i]["R"] for i in train_idx)]}
    log(f"trained on {info['points']} points of {G} geometries: loss {losses[0][1]:.3e} -> {losses[-1][1]:.3e}, "
        f"{info['ms_per_step']:.2f} ms per step; eigenvalue rms {info['eig_rms']:.2e}")
    return orb, eig, info


def predict(orb, eig, wl, R_range=None):
    """Warm start (psi, eps, rho) for the workload wl, or None when the
    geometry lies outside the trained range or the prediction is not usable
    (the superposition start then stays)."""
    import torch

    from . import tagi as T

    R = wl.meta["R"]
    if R_range is not None and not (R_range[0] <= R <= R_range[1]):
        return None
    feat = T.tagi_mlp_features(_dev(torch, wl.mesh.xyz), _nuclei(wl))
    psi = orb.warm_start(feat, _dev(torch, wl.psi[0]), _dev(torch, wl.mesh.w)).cpu().numpy()
    e = float(eig.forward(_midpoint_features(T, torch, _nuclei(wl))).cpu().numpy()[0])
    if not (np.all(np.isfinite(psi)) and np.isfinite(e) and e + wl.vshift < 0.0):
        return None
    return psi, e, wl.n_elec * psi * psi


def evaluate(orb, eig, records, test_idx, R_range=None, tol_m=3e-6, tol_scf=1e-4, log=print):
    """SCF runs of the held-out geometries from the superposition start and
    from the predicted start; the converged runs measure both starts."""
    rows = []
    for i in test_idx:
        r = records[i]
        wl = W.hydrogen_molecule(r["R"], tol_m=tol_m)
        w = wl.mesh.w
        ref = r["psi"].astype(np.float64)
        base = scf_run(wl, tol_scf=tol_scf)
        pred = predict(orb, eig, wl, R_range)
        if pred is None:
            warm, used = base, False
            e_pred, err_pred = float("nan"), float("nan")
        else:
            psi, e_pred, rho = pred
            warm, used = scf_run(wl, psi0=psi[None], eps0=[e_pred], rho0=rho, tol_scf=tol_scf), True
            err_pred = float(np.sqrt(np.sum((psi - ref) ** 2 * w)))
        row = {"R": r["R"], "n": wl.n, "used_prediction": used,
               "orbital_error": {"superposition": float(np.sqrt(np.sum((wl.psi[0] - ref) ** 2 * w))),
                                 "predicted": err_pred},
               "eps": {"converged": r["eps"], "predicted": e_pred, "superposition_guess": float(wl.eps[0])},
               "scf_steps": {"superposition": base["scf_steps"], "predicted": warm["scf_steps"]},
               "green_iterations": {"superposition": base["gi_steps"], "predicted": warm["gi_steps"]},
               "seconds": {"superposition": base["seconds"], "predicted": warm["seconds"]},
               "e_total": {"superposition": base["e_total"], "predicted": warm["e_total"]},
               "energy_settled": {"superposition": base["energy_settled"], "predicted": warm["energy_settled"]},
               "converged": bool(base["converged"] and warm["converged"]),
               "errors": {"superposition": base["error"], "predicted": warm["error"]}}
        log(f"R {r['R']:.4f}: orbital error {row['orbital_error']['superposition']:.3e} -> {err_pred:.3e}; "
            f"SCF steps {base['scf_steps']} -> {warm['scf_steps']}, Green iterations {base['gi_steps']} -> "
            f"{warm['gi_steps']}; E {base['e_total']:.7f} / {warm['e_total']:.7f}")
        rows.append(row)
    return rows


# ------------------------------------------------------ CO: a density model
# The orbital model needs one well-defined target per orbital; CO's 1pi
# levels are a degenerate pair that an SCF run may return in any rotation.
# The density is unique, and Algorithm 1 starts from rho_in, so for CO the
# network predicts the density: its amplitude sqrt(rho / N_e) as a relative
# correction of the normalised superposition amplitude s = sqrt(rho_sup / N_e)
# (the same kernels as the orbital model), rho_warm = N_e psi_warm^2.  The
# features take the nuclei in list order (C first), so a point's features
# tell the two atoms apart.  The orbitals keep the aufbau start.
def generate_co(bond_lengths, tol_m=3e-6, tol_scf=1e-5, log=print):
    """Converged CO runs from the superposition density and the aufbau
    orbitals, one per bond length: records (R, n, rho* as float32, E, cost)."""
    out = []
    for R in bond_lengths:
        wl = W.carbon_monoxide_scf(tol_m=tol_m, R=float(R))
        r = scf_run(wl, tol_scf=tol_scf, max_steps=60)
        rec = {"R": float(R), "n": wl.n, "w_sum": float(np.sum(wl.mesh.w)), "psi": r["rho"].astype(np.float32),
               "eps": float(r["eps"][6]), "e_total": float(r["e_total"]), "converged": bool(r["converged"]),
               "scf_steps": r["scf_steps"], "gi_steps": r["gi_steps"], "seconds": r["seconds"]}
        log(f"CO R {R:.4f} n {wl.n} E {rec['e_total']:.7f} scf {rec['scf_steps']} gi {rec['gi_steps']} "
            f"{rec['seconds']:.2f} s" + ("" if rec["converged"] else f" not converged ({r['error'] or 'step limit'})"))
        out.append(rec)
    return out


# decay rates of the first two CO features: the Slater 1s exponents of C and
# O (the nuclei in list order), so that those features resolve the two cores
CO_FEATURE_RATES = (W.ATOM_Z["C"] - 0.30, W.ATOM_Z["O"] - 0.30)


def _co_amplitudes(wl):
    """(s, features) of a CO workload: the normalised superposition amplitude
    and the list-order features with the 1s decay rates of C and O."""
    import torch

    from . import tagi as T

    s = np.sqrt(np.maximum(wl.rho, 0.0) / wl.n_elec)
    feat = T.tagi_mlp_features(_dev(torch, wl.mesh.xyz), wl.meta["nuclei"], ordered=True, scale=CO_FEATURE_RATES)
    return s, feat


def train_co(records, train_idx, steps=3000, lr=3e-3, seed=0, tol_m=3e-6, hidden=64, log=print):
    """The density model on the converged runs records[i], i in train_idx:
    target t = sqrt(rho* / rho_sup) - 1, with rho = N_e s^2 (1 + y)^2 the
    predicted density.  The loss is the density error to first order in
    y - t: sum w (2 N_e s^2 (1 + t))^2 (y - t)^2 ~ ||rho - rho*||_w^2, the
    norm the held-out comparison reports."""
    import torch

    from . import tagi as T

    feats, targets, wts = [], [], []
    G = len(train_idx)
    for i in train_idx:
        r = records[i]
        wl = W.carbon_monoxide_scf(tol_m=tol_m, R=r["R"])
        if wl.n != r["n"]:
            raise RuntimeError(f"mesh of R = {r['R']} has {wl.n} points, the record {r['n']}")
        s, feat = _co_amplitudes(wl)
        rho_c = np.maximum(r["psi"].astype(np.float64), 0.0)  # the converged density of the record
        # the target, bounded where both densities vanish (its weight is ~0 there)
        t = np.clip(np.sqrt(rho_c / np.maximum(wl.rho, 1e-300)) - 1.0, -1.0, 100.0)
        feats.append(feat)
        targets.append(torch.tensor(t.astype(np.float32), device="cuda"))
        # (2 N_e s^2 (1 + t))^2 = 4 rho_sup rho*: finite wherever the target is large
        wts.append(torch.tensor((wl.mesh.w * 4.0 * np.maximum(wl.rho, 0.0) * rho_c / G).astype(np.float32),
                                device="cuda"))
    feat, target, wt = torch.cat(feats), torch.cat(targets), torch.cat(wts)
    del feats, targets, wts
    model = T.Mlp(W.mlp_init(seed, hidden=hidden), hidden=hidden)
    sched = cosine_lr(lr, steps)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = []
    for k in range(1, steps + 1):
        want = k == 1 or k % 500 == 0 or k == steps
        L = model.train_step(feat, target, wt, sched(k), want_loss=want)
        if want:
            losses.append((k, L))
    torch.cuda.synchronize()
    t_tr = time.perf_counter() - t0
    info = {"points": int(feat.shape[0]), "geometries": G, "steps": steps, "lr": lr, "losses": losses,
            "hidden": hidden, "seconds": t_tr, "ms_per_step": 1e3 * t_tr / steps,
            "R_range": [min(records[i]["R"] for i in train_idx), max(records[i]["R"] for i in train_idx)]}
    log(f"CO density model: {info['points']} points of {G} geometries, loss {losses[0][1]:.3e} -> "
        f"{losses[-1][1]:.3e}, {info['ms_per_step']:.2f} ms per step")
    return model, info


def predict_co(model, wl, R_range=None):
    """rho_warm = N_e psi_warm^2 for a CO workload, or None outside the
    trained range or when not usable (the superposition density stays)."""
    import torch

    R = wl.meta["R"]
    if R_range is not None and not (R_range[0] <= R <= R_range[1]):
        return None
    s, feat = _co_amplitudes(wl)
    psi = model.warm_start(feat, _dev(torch, s), _dev(torch, wl.mesh.w)).cpu().numpy()
    if not np.all(np.isfinite(psi)):
        return None
    return wl.n_elec * psi * psi


def evaluate_co(model, records, test_idx, R_range=None, tol_m=3e-6, tol_scf=1e-5, log=print):
    """SCF runs of the held-out CO geometries from the superposition density
    and from the predicted one (the same aufbau orbitals)."""
    rows = []
    for i in test_idx:
        r = records[i]
        wl = W.carbon_monoxide_scf(tol_m=tol_m, R=r["R"])
        w = wl.mesh.w
        ref = r["psi"].astype(np.float64)
        base = scf_run(wl, tol_scf=tol_scf, max_steps=60)
        rho = predict_co(model, wl, R_range)
        used = rho is not None
        warm = scf_run(wl, rho0=rho, tol_scf=tol_scf, max_steps=60) if used else base
        err = lambda x: float(np.sqrt(np.sum((x - ref) ** 2 * w)))
        row = {"R": r["R"], "n": wl.n, "used_prediction": used,
               "density_error": {"superposition": err(wl.rho), "predicted": err(rho) if used else float("nan")},
               "scf_steps": {"superposition": base["scf_steps"], "predicted": warm["scf_steps"]},
               "green_iterations": {"superposition": base["gi_steps"], "predicted": warm["gi_steps"]},
               "seconds": {"superposition": base["seconds"], "predicted": warm["seconds"]},
               "e_total": {"superposition": base["e_total"], "predicted": warm["e_total"]},
               "energy_settled": {"superposition": base["energy_settled"], "predicted": warm["energy_settled"]},
               "converged": bool(base["converged"] and warm["converged"]),
               "errors": {"superposition": base["error"], "predicted": warm["error"]}}
        es = row["energy_settled"]
        log(f"CO R {r['R']:.4f}: density error {row['density_error']['superposition']:.3e} -> "
            f"{row['density_error']['predicted']:.3e}; SCF steps {base['scf_steps']} -> {warm['scf_steps']}; "
            f"to |dE| < 1e-6: {es['superposition']} -> {es['predicted']}; E {base['e_total']:.7f} / "
            f"{warm['e_total']:.7f}")
        rows.append(row)
    return rows


def split(count=32):
    """Held-out geometries: every fourth bond length in sorted order."""
    test = list(range(1, count, 4))
    return [i for i in range(count) if i not in test], test


def split_converged(records):
    """split() over the records whose SCF converged (the others are left
    out): (train, test) indices into records, in sorted order."""
    usable = [i for i, r in enumerate(records) if r["converged"]]
    tr_u, te_u = split(len(usable))
    return [usable[i] for i in tr_u], [usable[i] for i in te_u]


def profile_case(steps=3, hidden=64):
    """The kernels of the warm start on one H2 mesh (R = 1.4 Bohr, 192,000
    points): features, `steps` training steps against a smooth synthetic
    target, inference and the warm start.  The command ncu wraps; prints
    the measured ms per training step."""
    import torch

    from . import tagi as T

    wl = W.hydrogen_molecule(1.4)
    s = wl.psi[0]
    feat = T.tagi_mlp_features(_dev(torch, wl.mesh.xyz), _nuclei(wl))
    r = np.sqrt((wl.mesh.xyz ** 2).sum(0))
    target = torch.tensor((0.2 * np.tanh(r - 1.0)).astype(np.float32), device="cuda")
    wt = torch.tensor((wl.mesh.w * s * s).astype(np.float32), device="cuda")
    with T.Mlp(W.mlp_init(0, hidden=hidden), hidden=hidden) as m:
        m.train_step(feat, target, wt, 1e-3)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            m.train_step(feat, target, wt, 1e-3)
        torch.cuda.synchronize()
        ms = 1e3 * (time.perf_counter() - t0) / steps
        m.forward(feat)
        m.warm_start(feat, _dev(torch, s), _dev(torch, wl.mesh.w))
        torch.cuda.synchronize()
    print(f"profile case: {wl.n} points, H = {hidden}, {ms:.3f} ms per training step")


def main(argv=None):
    """python -m paper_2003_01833_gb300.warmstart [--data file.npz] [--steps K]
    runs the H2 data set (or loads it), trains both models, evaluates the
    held-out geometries and prints one JSON object.  --profile-case runs
    only the kernels on one mesh (the command ncu wraps)."""
    import argparse
    import json

    ap = argparse.ArgumentParser()
    ap.add_argument("--data", default=None, help="npz from a previous run (else generated here)")
    ap.add_argument("--save", default=None, help="write the generated data set here")
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--hidden", type=int, default=64, choices=[32, 64])
    ap.add_argument("--molecule", default="h2", choices=["h2", "co"])
    ap.add_argument("--profile-case", action="store_true")
    a = ap.parse_args(argv)
    if a.profile_case:
        profile_case(hidden=a.hidden)
        return
    import sys

    log = lambda m: print(m, file=sys.stderr, flush=True)
    if a.molecule == "co":
        main_co(a, log)
        return
    Rs = W.h2_bond_lengths()
    t0 = time.perf_counter()
    records = load(a.data) if a.data else generate(Rs, log=log)
    t_gen = time.perf_counter() - t0
    if a.save and not a.data:
        save(records, a.save)
    tr, te = split(len(records))
    orb, eig, info = train(records, tr, steps=a.steps, lr=a.lr, hidden=a.hidden, log=log)
    rows = evaluate(orb, eig, records, te, R_range=info["R_range"], log=log)
    orb.close()
    eig.close()
    tot = lambda key, k: int(sum(r[key][k] for r in rows))
    settled = lambda k, f: (sum(r["energy_settled"][k][f] for r in rows)
                            if all(r["energy_settled"][k] for r in rows) else None)
    out = {"data": {"molecule": "H2", "geometries": len(records), "bond_lengths": [r["R"] for r in records],
                    "points": [r["n"] for r in records], "seconds": t_gen,
                    "all_converged": all(bool(r["converged"]) for r in records)},
           "train": info, "test": rows,
           "totals": {"scf_steps": {"superposition": tot("scf_steps", "superposition"),
                                    "predicted": tot("scf_steps", "predicted")},
                      "green_iterations": {"superposition": tot("green_iterations", "superposition"),
                                           "predicted": tot("green_iterations", "predicted")},
                      "max_energy_difference": max(abs(r["e_total"]["superposition"] - r["e_total"]["predicted"])
                                                   for r in rows),
                      "to_energy_settled_1e-6_ha": {
                          k: {"scf_steps": settled(k, "scf_steps"), "green_iterations": settled(k, "gi_steps"),
                              "seconds": settled(k, "seconds")} for k in ("superposition", "predicted")}}}
    print(json.dumps(out))


def main_co(a, log):
    import json

    Rs = W.co_bond_lengths()
    t0 = time.perf_counter()
    records = load(a.data) if a.data else generate_co(Rs, log=log)
    t_gen = time.perf_counter() - t0
    if a.save and not a.data:
        save(records, a.save)
    tr, te = split_converged(records)
    model, info = train_co(records, tr, steps=a.steps, lr=a.lr, hidden=a.hidden, log=log)
    rows = evaluate_co(model, records, te, R_range=info["R_range"], log=log)
    model.close()
    both = [r for r in rows if r["converged"]]
    tot = lambda key, k: int(sum(r[key][k] for r in both))
    settled = lambda k, f: (sum(r["energy_settled"][k][f] for r in both)
                            if all(r["energy_settled"][k] for r in both) else None)
    out = {"data": {"molecule": "CO", "geometries": len(records), "bond_lengths": [r["R"] for r in records],
                    "points": [r["n"] for r in records], "seconds": t_gen,
                    "all_converged": all(bool(r["converged"]) for r in records),
                    "converged": [bool(r["converged"]) for r in records]},
           "train": info, "test": rows,
           "totals": {"rows": len(both),
                      "scf_steps": {"superposition": tot("scf_steps", "superposition"),
                                    "predicted": tot("scf_steps", "predicted")},
                      "green_iterations": {"superposition": tot("green_iterations", "superposition"),
                                           "predicted": tot("green_iterations", "predicted")},
                      "max_energy_difference": max((abs(r["e_total"]["superposition"] - r["e_total"]["predicted"])
                                                    for r in both), default=None),
                      "to_energy_settled_1e-6_ha": {
                          k: {"scf_steps": settled(k, "scf_steps"), "green_iterations": settled(k, "gi_steps"),
                              "seconds": settled(k, "seconds")} for k in ("superposition", "predicted")}}}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
