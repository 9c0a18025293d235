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

    def save(self, path):
        np.savez(path, params=self.net.get_params(), x_mean=self.x_mean, x_std=self.x_std,
                 y_mean=self.y_mean, y_std=self.y_std, w=self.w,
                 meta=json.dumps(dict(n_profile=N_PROFILE, horizon=HORIZON,
                                      sigma_scale=SIGMA_SCALE, width=WIDTH, depth=DEPTH,
                                      features=FEATURES)))

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


def fine_warm_start(weights, n_runs=4, nx=512, nv=128, horizon=HORIZON, stream=None,
                    precision=fk.FK_F32):
    """Warm starts on a finer grid than the network was trained on: the
    first n_runs held-out parameter points of `weights` whose coarse run
    saturated, solved on nx x nv x nv cold and from the network's
    end-of-horizon charge, all in one batch."""
    d = np.load(weights)
    n_train, n_test, seed = int(d["n_train"]), int(d["n_test"]), int(d["seed"])
    held = synth.surrogate_runs(n_train + n_test, seed)[n_train:]
    sel = np.flatnonzero(d["test_ok"] & (d["test_sat_step"] >= 0) & (d["test_tsat"] < HORIZON))
    sel = sel[:n_runs]
    runs = [dict(held[q], nx=nx, nv1=nv, nv2=nv) for q in sel]
    sur = Surrogate.load(weights, stream=stream)
    pp, pt = sur.predict(runs)
    sur.close()
    sigma0 = np.concatenate([np.zeros(len(runs)), pp[:, -1]])
    res = solve(runs + runs, horizon=horizon, sigma0=sigma0, stream=stream, precision=precision)
    prof, _, ok = labels(res, horizon)
    n = len(runs)
    cold, warm = res["sat_step"][:n], res["sat_step"][n:]
    end_c, end_w = prof[:n, -1], prof[n:, -1]
    both = (cold >= 0) & (warm >= 0)
    return {
        "grid": [nx, nv, nv], "runs": n, "held_out_index": [int(q) for q in sel],
        "cells_per_run": nx * nv * nv, "batch_steps": res["batch_steps"],
        "solver_seconds": res["seconds"], "valid": [bool(x) for x in ok],
        "sat_step_cold": [int(x) for x in cold], "sat_step_warm": [int(x) for x in warm],
        "steps_saved_fraction": float(1.0 - warm[both].sum() / cold[both].sum()) if both.any() else None,
        "sigma_end_cold": [float(x) for x in end_c], "sigma_end_warm": [float(x) for x in end_w],
        "sigma_warm_start": [float(x) for x in pp[:, -1]],
        "sigma_end_rel_diff": [float(abs(w - c) / max(abs(c), 1e-30)) for w, c in zip(end_w, end_c)],
        "predicted_tsat_s": [float(x) for x in pt],
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
    ap.add_argument("--fine", default=None, metavar="WEIGHTS",
                    help="only run fine-grid warm starts with these trained weights")
    ap.add_argument("--fine-runs", type=int, default=4)
    ap.add_argument("--fine-nx", type=int, default=512)
    ap.add_argument("--fine-nv", type=int, default=128)
    args = ap.parse_args(argv)
    import torch
    torch.cuda.set_stream(torch.cuda.Stream())
    stream = torch.cuda.current_stream().cuda_stream
    os.makedirs(args.out, exist_ok=True)
    if args.fine:
        rep = fine_warm_start(args.fine, args.fine_runs, args.fine_nx, args.fine_nv, args.horizon,
                              stream)
        with open(os.path.join(args.out, "fine_report.json"), "w") as fh:
            json.dump(rep, fh, indent=1)
        print(json.dumps(rep))
        return
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
    tr = np.arange(args.n_train)
    te = np.arange(args.n_train, args.n_train + args.n_test)
    tr_ok = tr[ok[tr]]
    sur = Surrogate(max_batch=512, seed=args.seed, stream=stream)
    t0 = time.perf_counter()
    hist = sur.fit([runs[q] for q in tr_ok], targets(prof[tr_ok], tsat[tr_ok]),
                   epochs=args.epochs, lr=args.lr, batch=args.batch, seed=args.seed)
    train_s = time.perf_counter() - t0
    sur.save(os.path.join(args.out, "surrogate.npz"))
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
    with open(os.path.join(args.out, "report.json"), "w") as fh:
        json.dump(report, fh, indent=1)
    print(json.dumps(report))
    sur.close()


if __name__ == "__main__":
    main()
