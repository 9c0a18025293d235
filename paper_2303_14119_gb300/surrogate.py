"""Surface-charge surrogate of the 1D2V flashover model.

A small network maps the parameters of a run -- applied field E_y (Sec. 2),
SEE yield delta_max, A_max and emission temperature T_se (Eqs. 8-15),
injected current J (Eq. 7) and gap h_max -- to the run's surface-charge
history sigma(t) (Eq. 18) sampled at N_PROFILE times over HORIZON seconds,
and to log10 of its saturation time (the convergence test of Sec. 2).  It is
trained on runs of the batched solver (fk_batch_*), with the network's
forward, backward and Adam kernels on the tensor cores (fk_mlp_*), and used
to warm-start the surface charge of new runs and to triage sweep points.
The paper has no surrogate; its error is always measured against the solver.

``python -m paper_2303_14119_gb300.surrogate --out DIR`` runs the whole
pipeline (data, training, evaluation, warm starts) and writes a JSON report.
The data can also be solved in parts, ``--solve-part I/P`` per call, and the
part files merged by ``--data A.npz,B.npz,...``; a batch steps every run
exactly as stepping it alone, so the labels do not depend on the split.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import fk, synth

N_PROFILE = 64
HORIZON = 1.25e-9          # s of physical time per run
SIGMA_SCALE = 1e-4         # C/m^2: profile targets are sigma / SIGMA_SCALE
T_UNIT = 1e-9              # s: the time target is log10(t_sat / T_UNIT)
T_CENSOR = 2.0 * HORIZON   # time label of runs that do not saturate within HORIZON
WIDTH, DEPTH = 256, 3
N_FEATURES = 6
FEATURES = ("log10 |E_y| (V/m)", "delta_max", "A_max / 100 eV", "T_se (eV)",
            "log10 J (A/m^2)", "h_max / 10 um")


def features(runs):
    return np.array([[math.log10(-p["Ey"]), p["delta_max"], p["A_max"] / 100.0, p["T_se"],
                      math.log10(p["J"]), p["h_max"] / 1e-5] for p in runs], dtype=np.float64)


def make_grid(p, precision, stream, history_capacity=16384):
    g = fk.Grid(p["nx"], p["nv1"], p["nv2"], p["h_max"], -p["v1_span"], p["v1_span"],
                -p["v2_span"], p["v2_span"], cfl=p["cfl"], precision=precision,
                history_capacity=history_capacity, stream=stream)
    g.set_fields(p["Ey"])
    g.set_see(p["delta_max"], p["A_max"], p["k_s"], p["T_se"])
    g.set_source(p["J"], p["x_lo"], p["x_hi"], p["T_fe"])
    return g


def solve(runs, horizon=HORIZON, sample_every=5000, sigma0=None, precision=fk.FK_F32,
          stream=None, autotune=True):
    """Run every description from f = 0 (and sigma = sigma0[i], default 0)
    for at least `horizon` seconds of physical time, all in one batch.
    Returns per run: dt, the sampled (step, sigma) history, the first
    saturated step (-1 if none) and the final status."""
    grids, status0 = [], []
    for q, p in enumerate(runs):
        g = make_grid(p, precision, stream)
        st = fk.FK_OK
        if sigma0 is not None and sigma0[q] != 0.0:
            try:
                g.set_surface_charge(float(sigma0[q]))
            except fk.FkError as e:  # the warm-start field breaks the CFL bound
                st = e.status
        grids.append(g)
        status0.append(st)
    dt = np.array([g.info()["dt"] for g in grids])
    total = int(np.ceil(horizon / dt.min()))
    t0 = time.perf_counter()
    with fk.Batch(grids, stream) as b:
        done = b.autotune(2) if autotune else 0
        steps, sig = [], []
        s0, st0, _, _ = b.scalars()
        steps.append(st0.copy())
        sig.append(s0.copy())
        while done < total:
            k = min(sample_every, total - done)
            b.step(k)
            done += k
            s, st, _, _ = b.scalars()
            steps.append(st.copy())
            sig.append(s.copy())
        _, _, sat, status = b.scalars()
    seconds = time.perf_counter() - t0
    for g in grids:
        g.close()
    status = np.where(np.array(status0) != fk.FK_OK, np.array(status0), status)
    return dict(dt=dt, steps=np.array(steps), sigma=np.array(sig), sat_step=sat,
                status=status, seconds=seconds, batch_steps=total,
                cells=float(sum(p["nx"] * p["nv1"] * p["nv2"] for p in runs)))


def solve_to_saturation(runs, max_steps, sigma0=None, sample_every=5000, precision=fk.FK_F32,
                        stream=None, autotune=True):
    """Like solve(), but stops once every run has passed the convergence test
    of Sec. 2 (or after max_steps batch steps): the runs of a finer grid,
    whose horizon would cost several times their saturation time.  The
    history after a run's saturation is flat to the test's tolerance, so
    labels() extends each sampled history with its last value."""
    grids, status0 = [], []
    for q, p in enumerate(runs):
        g = make_grid(p, precision, stream)
        st = fk.FK_OK
        if sigma0 is not None and sigma0[q] != 0.0:
            try:
                g.set_surface_charge(float(sigma0[q]))
            except fk.FkError as e:  # the warm-start field breaks the CFL bound
                st = e.status
        grids.append(g)
        status0.append(st)
    dt = np.array([g.info()["dt"] for g in grids])
    t0 = time.perf_counter()
    with fk.Batch(grids, stream) as b:
        done = b.autotune(2) if autotune else 0
        steps, sig = [], []
        s0, st0, _, _ = b.scalars()
        steps.append(st0.copy())
        sig.append(s0.copy())
        while done < max_steps:
            k = min(sample_every, max_steps - done)
            b.step(k)
            done += k
            s, st, sat, status = b.scalars()
            steps.append(st.copy())
            sig.append(s.copy())
            live = (status == fk.FK_OK) & (np.array(status0) == fk.FK_OK)
            if np.all((sat >= 0) | ~live):
                break
        _, _, sat, status = b.scalars()
    seconds = time.perf_counter() - t0
    for g in grids:
        g.close()
    status = np.where(np.array(status0) != fk.FK_OK, np.array(status0), status)
    return dict(dt=dt, steps=np.array(steps), sigma=np.array(sig), sat_step=sat,
                status=status, seconds=seconds, batch_steps=done,
                cells=float(sum(p["nx"] * p["nv1"] * p["nv2"] for p in runs)))


def labels(res, horizon=HORIZON):
    """Targets of each run: sigma at t_k = (k + 1) horizon / N_PROFILE
    (linear interpolation of the sampled history, C/m^2), the saturation
    time (T_CENSOR if not saturated within the horizon), and whether the run
    stayed valid (no sticky error)."""
    n = res["dt"].size
    tk = (np.arange(N_PROFILE) + 1) * horizon / N_PROFILE
    prof = np.zeros((n, N_PROFILE))
    tsat = np.full(n, T_CENSOR)
    ok = res["status"] == fk.FK_OK
    for q in range(n):
        t = res["steps"][:, q] * res["dt"][q]
        prof[q] = np.interp(tk, t, res["sigma"][:, q])
        if res["sat_step"][q] >= 0:
            ts = res["sat_step"][q] * res["dt"][q]
            if ts <= horizon:
                tsat[q] = ts
    return prof, tsat, ok


def targets(prof, tsat):
    return np.concatenate([prof / SIGMA_SCALE, np.log10(tsat / T_UNIT)[:, None]], axis=1)


class Surrogate:
    """The network plus the normalisation of its inputs and outputs."""

    def __init__(self, max_batch=512, seed=0, stream=None):
        self.net = fk.Mlp(N_FEATURES, WIDTH, DEPTH, N_PROFILE + 1, max_batch, stream=stream)
        rng = np.random.default_rng(seed)
        dims = [N_FEATURES] + [WIDTH] * DEPTH + [N_PROFILE + 1]
        parts = []
        for q in range(len(dims) - 1):
            parts.append(rng.normal(0.0, math.sqrt(2.0 / dims[q]), dims[q + 1] * dims[q]))
            parts.append(np.zeros(dims[q + 1]))
        self.net.set_params(np.concatenate(parts))
        self.x_mean = np.zeros(N_FEATURES)
        self.x_std = np.ones(N_FEATURES)
        self.y_mean = np.zeros(N_PROFILE + 1)
        self.y_std = np.ones(N_PROFILE + 1)
        # the time output counts as much as a quarter of the profile
        self.w = np.ones(N_PROFILE + 1)
        self.w[-1] = N_PROFILE / 4.0

    def fit(self, runs, Y, epochs=300, lr=1e-3, batch=256, seed=0):
        X = features(runs)
        self.x_mean, self.x_std = X.mean(0), X.std(0) + 1e-12
        self.y_mean, self.y_std = Y.mean(0), Y.std(0) + 1e-12
        Xn = (X - self.x_mean) / self.x_std
        Yn = (Y - self.y_mean) / self.y_std
        return self.net.train(Xn, Yn, self.w, batch=batch, epochs=epochs, lr=lr, seed=seed)

    def predict(self, runs):
        """(sigma profile [n][N_PROFILE] in C/m^2, saturation time [n] in s)."""
        Xn = (features(runs) - self.x_mean) / self.x_std
        Y = self.net.forward(Xn).astype(np.float64) * self.y_std + self.y_mean
        return Y[:, :N_PROFILE] * SIGMA_SCALE, T_UNIT * 10.0 ** Y[:, N_PROFILE]

    def save(self, path, **extra):
        """Weights and normalisation; `extra` arrays (e.g. the held-out
        labels the network was evaluated on) are stored beside them."""
        np.savez(path, params=self.net.get_params(), x_mean=self.x_mean, x_std=self.x_std,
                 y_mean=self.y_mean, y_std=self.y_std, w=self.w,
                 meta=json.dumps(dict(n_profile=N_PROFILE, horizon=HORIZON,
                                      sigma_scale=SIGMA_SCALE, width=WIDTH, depth=DEPTH,
                                      features=FEATURES)), **extra)

    @classmethod
    def load(cls, path, max_batch=512, stream=None):
        d = np.load(path)
        s = cls(max_batch=max_batch, stream=stream)
        s.net.set_params(d["params"])
        for k in ("x_mean", "x_std", "y_mean", "y_std", "w"):
            setattr(s, k, d[k])
        return s

    def close(self):
        self.net.close()


def evaluate(sur, runs, prof, tsat, ok):
    """Errors of the surrogate against solver labels on valid runs."""
    pp, pt = sur.predict(runs)
    pp, pt, prof, tsat = pp[ok], pt[ok], prof[ok], tsat[ok]
    nrm = np.maximum(np.linalg.norm(prof, axis=1), 1e-30)
    rel_prof = np.linalg.norm(pp - prof, axis=1) / nrm
    rel_end = np.abs(pp[:, -1] - prof[:, -1]) / np.maximum(np.abs(prof[:, -1]), 1e-30)
    sat_true = tsat < T_CENSOR
    sat_pred = pt < HORIZON
    lt = np.abs(np.log10(pt[sat_true]) - np.log10(tsat[sat_true])) if sat_true.any() else np.zeros(0)
    return {
        "runs": int(ok.sum()),
        "profile_rel_l2": {"median": float(np.median(rel_prof)), "p90": float(np.percentile(rel_prof, 90))},
        "sigma_end_rel": {"median": float(np.median(rel_end)), "p90": float(np.percentile(rel_end, 90))},
        "saturated_fraction": float(sat_true.mean()),
        "triage_accuracy": float((sat_true == sat_pred).mean()),
        "log10_tsat_abs_err": {"median": float(np.median(lt)) if lt.size else None,
                               "p90": float(np.percentile(lt, 90)) if lt.size else None},
    }


def warm_start(sur, runs, prof_cold, res_cold, horizon=HORIZON, stream=None, precision=fk.FK_F32):
    """Re-run `runs` from the surrogate's saturated surface charge (its
    sigma at the end of the horizon) and compare with the cold runs: steps
    to saturation and the surface charge at the end of the horizon."""
    pp, _ = sur.predict(runs)
    res_w = solve(runs, horizon=horizon, sigma0=pp[:, -1], stream=stream, precision=precision)
    prof_w, _, ok_w = labels(res_w, horizon)
    sat_c = np.where(res_cold["sat_step"] >= 0, res_cold["sat_step"], np.iinfo(np.int64).max)
    sat_w = np.where(res_w["sat_step"] >= 0, res_w["sat_step"], np.iinfo(np.int64).max)
    both = (res_cold["sat_step"] >= 0) & (res_w["sat_step"] >= 0) & ok_w
    end_err = np.abs(prof_w[:, -1] - prof_cold[:, -1]) / np.maximum(np.abs(prof_cold[:, -1]), 1e-30)
    saved = (sat_c - sat_w)[both]
    return {
        "runs": len(runs),
        "cold_saturated": int((res_cold["sat_step"] >= 0).sum()),
        "warm_saturated": int((res_w["sat_step"] >= 0).sum()),
        "warm_valid": int(ok_w.sum()),
        "steps_to_saturation_cold": {"median": float(np.median(sat_c[both])) if both.any() else None,
                                     "sum": int(sat_c[both].sum()) if both.any() else 0},
        "steps_to_saturation_warm": {"median": float(np.median(sat_w[both])) if both.any() else None,
                                     "sum": int(sat_w[both].sum()) if both.any() else 0},
        "steps_saved_fraction": float(saved.sum() / sat_c[both].sum()) if both.any() else None,
        "runs_faster": int((saved > 0).sum()),
        "sigma_end_rel_diff_warm_vs_cold": {
            "median": float(np.median(end_err[ok_w])) if ok_w.any() else None,
            "p90": float(np.percentile(end_err[ok_w], 90)) if ok_w.any() else None},
        "seconds": res_w["seconds"],
    }


def fine_points(ok, sat_step, tsat, n_train, n_fine_train, n_fine_test):
    """Indices of the parameter points solved on the fine grid: the first
    n_fine_train training draws and the first n_fine_test held-out draws
    whose coarse run is valid and saturates within the horizon."""
    good = ok & (sat_step >= 0) & (tsat < HORIZON)
    tr = np.flatnonzero(good[:n_train])[:n_fine_train]
    te = n_train + np.flatnonzero(good[n_train:])[:n_fine_test]
    return tr, te


def fine_solve(runs, idx, nx, nv, max_steps, stream=None):
    """Cold runs of the draws idx on an nx x nv x nv grid, to saturation."""
    fine = [dict(runs[q], nx=nx, nv1=nv, nv2=nv) for q in idx]
    res = solve_to_saturation(fine, max_steps, stream=stream)
    prof, tsat, ok = labels(res)
    ok = ok & (res["sat_step"] >= 0)  # a label needs the saturated charge
    return fine, res, prof, tsat, ok


def fine_tune(sur, runs, Y, epochs=200, lr=2e-4, batch=64, seed=1):
    """Continue training the network on the fine-grid labels, keeping the
    input and output normalisation of its coarse training."""
    Xn = (features(runs) - sur.x_mean) / sur.x_std
    Yn = (Y - sur.y_mean) / sur.y_std
    sur.net.set_params(sur.net.get_params())  # fresh Adam state
    return sur.net.train(Xn, Yn, sur.w, batch=batch, epochs=epochs, lr=lr, seed=seed)


def fine_warm_start_vs_cold(sur, fine_runs, cold, max_steps, stream=None):
    """Warm starts of fine-grid runs from the network's end-of-horizon
    charge, to saturation, against their stored cold runs (cold: sat_step
    and the saturated charge sigma_sat of each run)."""
    pp, pt = sur.predict(fine_runs)
    res = solve_to_saturation(fine_runs, max_steps, sigma0=pp[:, -1], stream=stream)
    prof_w, _, ok_w = labels(res)
    warm = res["sat_step"]
    cs, cw = cold["sat_step"], warm
    both = (cs >= 0) & (cw >= 0) & ok_w
    end_c = cold["sigma_sat"]
    # the charge each warm run saturates at (flat from its saturated step on)
    end_w = prof_w[:, -1]
    return {
        "runs": len(fine_runs), "grid": [fine_runs[0]["nx"], fine_runs[0]["nv1"], fine_runs[0]["nv2"]],
        "warm_valid": int(ok_w.sum()), "warm_saturated": int((cw >= 0).sum()),
        "sat_step_cold": [int(x) for x in cs], "sat_step_warm": [int(x) for x in cw],
        "steps_saved_fraction": float(1.0 - cw[both].sum() / cs[both].sum()) if both.any() else None,
        "runs_faster": int(((cs - cw) > 0)[both].sum()),
        "sigma_warm_start": [float(x) for x in pp[:, -1]],
        "sigma_sat_cold": [float(x) for x in end_c],
        "sigma_sat_warm": [float(x) for x in end_w],
        "start_rel_err": [float(abs(a - c) / max(abs(c), 1e-30)) for a, c in zip(pp[:, -1], end_c)],
        "sigma_sat_rel_diff_warm_vs_cold": [float(abs(a - c) / max(abs(c), 1e-30))
                                            for a, c in zip(end_w, end_c)],
        "batch_steps": int(res["batch_steps"]), "solver_seconds": res["seconds"],
    }


DATA_KEYS = ("prof", "tsat", "ok", "status", "sat_step", "dt")


def part_slice(n, part):
    """Indices of part "I/P" of n runs: the I-th of P contiguous,
    nearly equal slices."""
    i, p = (int(v) for v in part.split("/"))
    if not 0 <= i < p:
        raise ValueError("part must be I/P with 0 <= I < P")
    return np.array_split(np.arange(n), p)[i]


def save_data(path, idx, runs, res, prof, tsat, ok):
    """Labels of the runs with indices idx (runs: all draws), with the
    solver's cost."""
    np.savez(path, idx=idx, X=features([runs[q] for q in idx]), prof=prof, tsat=tsat, ok=ok,
             status=res["status"], sat_step=res["sat_step"], dt=res["dt"],
             seconds=res["seconds"], batch_steps=res["batch_steps"], cells=res["cells"])


def load_data(paths, runs):
    """Merge data files (whole sets or parts) into the labels of all runs
    in draw order; every run must be covered exactly once and by the same
    draw.  The solver cost adds up over the parts (cell_steps: cells x batch
    steps)."""
    n = len(runs)
    X = features(runs)
    seen = np.zeros(n, dtype=bool)
    out = {}
    seconds = cell_steps = 0.0
    batch_steps = 0
    for path in paths:
        d = np.load(path)
        idx = d["idx"] if "idx" in d.files else np.arange(len(d["X"]))
        if idx.size and (idx.min() < 0 or idx.max() >= n):
            raise ValueError("%s: run indices outside the %d draws" % (path, n))
        if seen[idx].any():
            raise ValueError("%s: runs covered twice" % path)
        # the same draws up to the last bit: the transcendental functions of
        # the draws and features may round differently on another machine
        if not np.allclose(d["X"], X[idx], rtol=1e-12, atol=0.0):
            raise ValueError("%s was made from other draws" % path)
        seen[idx] = True
        for k in DATA_KEYS:
            if k not in out:
                out[k] = np.zeros((n,) + d[k].shape[1:], dtype=d[k].dtype)
            out[k][idx] = d[k]
        seconds += float(d["seconds"])
        cell_steps += float(d["cells"]) * int(d["batch_steps"])
        batch_steps = max(batch_steps, int(d["batch_steps"]))
    if not seen.all():
        raise ValueError("%d of %d runs have no data" % (int((~seen).sum()), n))
    out.update(seconds=seconds, batch_steps=batch_steps, cell_steps=cell_steps)
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--n-train", type=int, default=4096)
    ap.add_argument("--n-test", type=int, default=512)
    ap.add_argument("--seed", type=int, default=11)
    ap.add_argument("--epochs", type=int, default=300)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--horizon", type=float, default=HORIZON)
    ap.add_argument("--out", default="surrogate_out")
    ap.add_argument("--data", default=None,
                    help="comma-separated data files of earlier runs of the same draws, whole "
                         "or parts (skips the solver runs)")
    ap.add_argument("--solve-part", default=None, metavar="I/P",
                    help="only solve part I of P of the draws and save its data_partIofP.npz")
    ap.add_argument("--no-warm", action="store_true", help="skip the warm-start runs")
    ap.add_argument("--fine-nx", type=int, default=512)
    ap.add_argument("--fine-nv", type=int, default=128)
    ap.add_argument("--fine-solve", default=None, metavar="NTR,NTE",
                    help="with --data: solve NTR training and NTE held-out points (valid, "
                         "saturating on the coarse grid) cold on the fine grid to saturation and "
                         "save data_fine_NXxNVxNV.npz")
    ap.add_argument("--fine-data", default=None, metavar="FILE",
                    help="with --data: after the coarse training, fine-tune the network on the "
                         "training points of FILE (from --fine-solve), evaluate it on its held-out "
                         "points and warm-start their fine-grid runs")
    ap.add_argument("--fine-max-steps", type=int, default=1600000)
    ap.add_argument("--fine-epochs", type=int, default=200)
    ap.add_argument("--fine-lr", type=float, default=2e-4)
    args = ap.parse_args(argv)
    import torch
    torch.cuda.set_stream(torch.cuda.Stream())
    stream = torch.cuda.current_stream().cuda_stream
    os.makedirs(args.out, exist_ok=True)
    runs = synth.surrogate_runs(args.n_train + args.n_test, args.seed)
    if args.solve_part:
        idx = part_slice(len(runs), args.solve_part)
        res = solve([runs[q] for q in idx], horizon=args.horizon, stream=stream)
        prof, tsat, ok = labels(res, args.horizon)
        i, p = args.solve_part.split("/")
        path = os.path.join(args.out, "data_part%sof%s.npz" % (i, p))
        save_data(path, idx, runs, res, prof, tsat, ok)
        print(json.dumps({"part": args.solve_part, "runs": int(idx.size), "valid": int(ok.sum()),
                          "solver_seconds": res["seconds"], "batch_steps": res["batch_steps"],
                          "file": path}))
        return
    if args.data:
        try:
            d = load_data(args.data.split(","), runs)
        except ValueError as e:
            raise SystemExit("--data: %s" % e)
        res = {k: d[k] for k in ("status", "sat_step", "dt")}
        res.update(seconds=d["seconds"], batch_steps=d["batch_steps"], cell_steps=d["cell_steps"])
        prof, tsat, ok = d["prof"], d["tsat"], d["ok"]
    else:
        res = solve(runs, horizon=args.horizon, stream=stream)
        res["cell_steps"] = res["cells"] * res["batch_steps"]
        prof, tsat, ok = labels(res, args.horizon)
        save_data(os.path.join(args.out, "data.npz"), np.arange(len(runs)), runs, res, prof,
                  tsat, ok)
    grid_tag = "%dx%dx%d" % (args.fine_nx, args.fine_nv, args.fine_nv)
    if args.fine_solve:
        ntr, nte = (int(v) for v in args.fine_solve.split(","))
        itr, ite = fine_points(ok, res["sat_step"], tsat, args.n_train, ntr, nte)
        idx = np.concatenate([itr, ite])
        fine, fres, fprof, ftsat, fok = fine_solve(runs, idx, args.fine_nx, args.fine_nv,
                                                   args.fine_max_steps, stream)
        path = os.path.join(args.out, "data_fine_%s.npz" % grid_tag)
        np.savez(path, idx_train=itr, idx_test=ite, prof=fprof, tsat=ftsat, ok=fok,
                 status=fres["status"], sat_step=fres["sat_step"], dt=fres["dt"],
                 sigma_sat=fprof[:, -1], seconds=fres["seconds"], batch_steps=fres["batch_steps"],
                 cells=fres["cells"])
        print(json.dumps({"fine_solve": grid_tag, "train": int(itr.size), "test": int(ite.size),
                          "saturated": int((fres["sat_step"] >= 0).sum()), "valid": int(fok.sum()),
                          "batch_steps": int(fres["batch_steps"]),
                          "solver_seconds": fres["seconds"], "file": path}))
        return
    tr = np.arange(args.n_train)
    te = np.arange(args.n_train, args.n_train + args.n_test)
    tr_ok = tr[ok[tr]]
    sur = Surrogate(max_batch=512, seed=args.seed, stream=stream)
    t0 = time.perf_counter()
    hist = sur.fit([runs[q] for q in tr_ok], targets(prof[tr_ok], tsat[tr_ok]),
                   epochs=args.epochs, lr=args.lr, batch=args.batch, seed=args.seed)
    train_s = time.perf_counter() - t0
    coarse_tag = "%dx%dx%d" % (runs[0]["nx"], runs[0]["nv1"], runs[0]["nv2"])
    sur.save(os.path.join(args.out, "surrogate_%s.npz" % coarse_tag), seed=args.seed,
             n_train=args.n_train, n_test=args.n_test, test_prof=prof[te], test_tsat=tsat[te],
             test_ok=ok[te], test_sat_step=res["sat_step"][te], test_dt=res["dt"][te])
    test_runs = [runs[q] for q in te]
    ev_test = evaluate(sur, test_runs, prof[te], tsat[te], ok[te])
    ev_train = evaluate(sur, [runs[q] for q in tr], prof[tr], tsat[tr], ok[tr])
    # warm starts of the held-out runs that saturated when started cold
    ws = None
    if not args.no_warm:
        ws_idx = te[ok[te] & (res["sat_step"][te] >= 0)]
        sub = {k: (v[ws_idx] if isinstance(v, np.ndarray) and v.ndim == 1 else v)
               for k, v in res.items()}
        ws = warm_start(sur, [runs[q] for q in ws_idx], prof[ws_idx], sub, args.horizon, stream)
    report = {
        "data": {"runs": len(runs), "valid": int(ok.sum()),
                 "invalid_status": {str(int(s)): int((res["status"] == s).sum())
                                    for s in np.unique(res["status"]) if s != fk.FK_OK},
                 "grid": [runs[0]["nx"], runs[0]["nv1"], runs[0]["nv2"]],
                 "horizon_s": args.horizon, "batch_steps": res["batch_steps"],
                 "solver_seconds": res["seconds"],
                 "cell_updates_per_s": res["cell_steps"] / res["seconds"]},
        "training": {"epochs": args.epochs, "lr": args.lr, "batch": args.batch,
                     "samples": int(tr_ok.size), "seconds": train_s,
                     "loss_first": float(hist[0]), "loss_last": float(hist[-1])},
        "train_eval": ev_train,
        "test_eval": ev_test,
        "warm_start": ws,
    }
    if args.fine_data:
        fd = np.load(args.fine_data)
        itr, ite = fd["idx_train"], fd["idx_test"]
        ntr = itr.size
        fprof, ftsat, fok = fd["prof"], fd["tsat"], fd["ok"]
        fine_tr = [dict(runs[q], nx=args.fine_nx, nv1=args.fine_nv, nv2=args.fine_nv) for q in itr]
        fine_te = [dict(runs[q], nx=args.fine_nx, nv1=args.fine_nv, nv2=args.fine_nv) for q in ite]
        # before fine-tuning: the coarse network on the fine held-out points
        ev_fine_before = evaluate(sur, fine_te, fprof[ntr:], ftsat[ntr:], fok[ntr:])
        keep = np.flatnonzero(fok[:ntr])
        t0 = time.perf_counter()
        fh = fine_tune(sur, [fine_tr[q] for q in keep], targets(fprof[keep], ftsat[keep]),
                       epochs=args.fine_epochs, lr=args.fine_lr, seed=args.seed + 1)
        tune_s = time.perf_counter() - t0
        ev_fine = evaluate(sur, fine_te, fprof[ntr:], ftsat[ntr:], fok[ntr:])
        sur.save(os.path.join(args.out, "surrogate_%s.npz" % grid_tag), seed=args.seed,
                 n_train=args.n_train, n_test=args.n_test, fine_idx_train=itr, fine_idx_test=ite,
                 test_prof=fprof[ntr:], test_tsat=ftsat[ntr:], test_ok=fok[ntr:],
                 test_sat_step=fd["sat_step"][ntr:], test_dt=fd["dt"][ntr:],
                 grid=np.array([args.fine_nx, args.fine_nv, args.fine_nv]))
        sel = np.flatnonzero(fok[ntr:])
        cold = {"sat_step": fd["sat_step"][ntr:][sel], "sigma_sat": fd["sigma_sat"][ntr:][sel]}
        fws = fine_warm_start_vs_cold(sur, [fine_te[q] for q in sel], cold, args.fine_max_steps,
                                      stream)
        report["fine"] = {
            "grid": [args.fine_nx, args.fine_nv, args.fine_nv],
            "train_points": int(ntr), "train_valid": int(keep.size),
            "test_points": int(ite.size), "test_valid": int(fok[ntr:].sum()),
            "cold_solver_seconds": float(fd["seconds"]), "cold_batch_steps": int(fd["batch_steps"]),
            "fine_tune": {"epochs": args.fine_epochs, "lr": args.fine_lr, "seconds": tune_s,
                          "loss_first": float(fh[0]), "loss_last": float(fh[-1])},
            "test_eval_coarse_network": ev_fine_before,
            "test_eval_fine_tuned": ev_fine,
            "warm_start": fws,
        }
    with open(os.path.join(args.out, "report.json"), "w") as fh_:
        json.dump(report, fh_, indent=1)
    print(json.dumps(report))
    sur.close()


if __name__ == "__main__":
    main()
