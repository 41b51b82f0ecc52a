"""Training data, training and evaluation of the learned parameter selector.

The selector (C ABI: gmres_matrix_features, gmres_mlp_*, gmres_select_params) maps 16 cheap
features of A to one of 32 GMRES-IR configurations:

    class c = (im * 4 + id) * 2 + ip,   m = (25, 50, 100, 200)[im],
                                        poly degree = (0, 10, 25, 40)[id],
                                        inner storage = (FP32, FP16)[ip],

each with the inner tolerance (1e-2, 1e-4 or 1e-6) that was best for that class on the
training matrices.  The fixed default -- m 50, no polynomial, FP32, inner tolerance 1e-4 --
is the fallback and the yardstick.  Everything here drives the library through its C ABI:

    sweep()        times every (class, tolerance) on each matrix with this solver
    fit()          per-class tolerances, labels (fastest class per matrix), feature
                   normalisation, and full-batch Adam training on the GPU (gmres_mlp_train)
    evaluate()     held-out time ratio of the selected configuration against the default

    python -m paper_2109_01232_b300.selector sweep --count 128 --first 0 --last 64 --out a.npz
    python -m paper_2109_01232_b300.selector sweep --count 128 --first 64 --out b.npz
    python -m paper_2109_01232_b300.selector merge a.npz b.npz     # -> selector_sweep.npz
    python -m paper_2109_01232_b300.selector fit                   # -> selector_model.npz
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

M_VALUES = (25, 50, 100, 200)
DEGREES = (0, 10, 25, 40)
PRECS = ("fp32", "fp16")
TOLS = (1e-2, 1e-4, 1e-6)
N_CLASSES = len(M_VALUES) * len(DEGREES) * len(PRECS)
DEFAULT = dict(m=50, degree=0, prec="fp32", inner_rtol=1e-4)
TIMEOUT_FACTOR = 3.0  # a configuration slower than 3x the default counts as a failure
DEFAULT_CAP = 20000   # iterations of the default run (a longer default counts as not converged)
HERE = os.path.dirname(os.path.abspath(__file__))
MODEL_PATH = os.path.join(HERE, "selector_model.npz")
SWEEP_PATH = os.path.join(HERE, "selector_sweep.npz")


def class_index(im: int, idg: int, ip: int) -> int:
    return (im * len(DEGREES) + idg) * len(PRECS) + ip


def class_config(c: int) -> tuple[int, int, str]:
    ip = c % len(PRECS)
    idg = (c // len(PRECS)) % len(DEGREES)
    im = c // (len(PRECS) * len(DEGREES))
    return M_VALUES[im], DEGREES[idg], PRECS[ip]


DEFAULT_CLASS = class_index(M_VALUES.index(DEFAULT["m"]), DEGREES.index(DEFAULT["degree"]),
                            PRECS.index(DEFAULT["prec"]))


def _solve_time(g, torch, plan, bt, x, rtol, tol, max_iters):
    plan.set_tolerances(rtol, tol, max_iters)
    x.zero_()
    r = plan.solve(bt, x)
    return (r.t_solve_ms if r.status == g.OK else np.inf), r.iters


def sweep(descs, rtol: float = 1e-10, log=print, checkpoint: str | None = None,
          tol_index=None, n_hi: float = 2e5):
    """For each matrix descriptor (gen.selector_matrices with this n_hi): features, the
    default's time and the device time (ms) of every (class, tolerance), inf for a failure or
    a timeout.  tol_index (one tolerance index per class, e.g. a trained model's) restricts
    each class to that tolerance (the others stay inf), a third of the runs for large
    matrices.  With `checkpoint`, the matrices done so far are saved there after each one."""
    import torch

    import gen
    import paper_2109_01232_b300 as g
    F = np.zeros((len(descs), 16), np.float32)
    T = np.full((len(descs), N_CLASSES, len(TOLS)), np.inf)
    It = np.zeros((len(descs), N_CLASSES, len(TOLS)), np.int64)
    T0 = np.zeros(len(descs))
    for k, desc in enumerate(descs):
        t_start = time.time()
        p = gen.build_selector_matrix(desc)
        A = g.DeviceCSR.from_problem(p)
        F[k] = g.matrix_features(A)
        bt = torch.ones(p.n, dtype=torch.float64, device="cuda")
        x = torch.zeros_like(bt)
        plan = g.Plan(A, "ir", restart_m=DEFAULT["m"], inner_prec=DEFAULT["prec"], rtol=rtol,
                      inner_rtol=DEFAULT["inner_rtol"], max_iters=DEFAULT_CAP)
        _solve_time(g, torch, plan, bt, x, rtol, DEFAULT["inner_rtol"], DEFAULT_CAP)  # warm-up
        t0, it0 = _solve_time(g, torch, plan, bt, x, rtol, DEFAULT["inner_rtol"], DEFAULT_CAP)
        if not np.isfinite(t0):  # the default did not converge: time its capped run instead
            plan.set_tolerances(rtol, DEFAULT["inner_rtol"], DEFAULT_CAP)
            x.zero_()
            t_ref = plan.solve(bt, x).t_solve_ms
        else:
            t_ref = t0
        plan.close()
        T0[k] = t0
        for c in range(N_CLASSES):
            m, d, prec = class_config(c)
            try:
                plan = g.Plan(A, "ir", restart_m=m, inner_prec=prec, poly_degree=d, rtol=rtol,
                              max_iters=m, seed=desc["seed"])
            except g.GmresError:
                continue  # e.g. a polynomial set-up that broke down: the class fails here
            # iteration cap from the time of one cycle, so no run lasts much over the timeout
            plan.set_tolerances(rtol, TOLS[0], m)
            x.zero_()
            rp_ = plan.solve(bt, x)
            per_it = rp_.t_solve_ms / max(rp_.iters, 1)
            cap = int(min(DEFAULT_CAP, max(m, 1.2 * TIMEOUT_FACTOR * t_ref / max(per_it, 1e-6)) + m))
            for it_, tol in enumerate(TOLS):
                if tol_index is not None and it_ != int(tol_index[c]):
                    continue
                t, its = _solve_time(g, torch, plan, bt, x, rtol, tol, cap)
                if t > TIMEOUT_FACTOR * t_ref:
                    t = np.inf
                T[k, c, it_] = t
                It[k, c, it_] = its
            plan.close()
        log(f"[{k + 1}/{len(descs)}] n={p.n} dim={desc['dim']} pe={desc['peclet']:.3g} "
            f"an={desc['anisotropy']:.3g} default {t0:.1f} ms ({it0} it), best "
            f"{np.min(T[k]):.1f} ms, {time.time() - t_start:.1f} s")
        if checkpoint:
            save(checkpoint, _sweep_dict(F, T, It, T0, descs, k + 1, n_hi))
    return _sweep_dict(F, T, It, T0, descs, len(descs), n_hi)


def _sweep_dict(F, T, It, T0, descs, done: int, n_hi: float) -> dict:
    """desc_index / desc_n_hi identify each matrix: gen.selector_matrices(count > index,
    n_hi=desc_n_hi)[desc_index]."""
    return dict(features=F[:done], times=T[:done], iters=It[:done], default_ms=T0[:done],
                desc_index=np.array([d["index"] for d in descs[:done]]),
                desc_seed=np.array([d["seed"] for d in descs[:done]]),
                desc_n_hi=np.full(done, n_hi), desc_n=np.array([d["side"] ** d["dim"]
                                                                for d in descs[:done]]))


def descriptor(data: dict, k: int) -> dict:
    """The corpus descriptor of matrix k of a sweep."""
    import gen
    idx = int(data["desc_index"][k])
    n_hi = float(data["desc_n_hi"][k]) if "desc_n_hi" in data else float(data.get("n_hi", 2e5))
    return gen.selector_matrices(count=idx + 1, n_hi=n_hi)[idx]


def live_evaluate(data: dict, model: dict, idx, rtol: float = 1e-10, reps: int = 2,
                  log=None) -> dict:
    """Re-solve the matrices idx with the selector's choice (gmres_select_params through
    Selector.choose, on the GPU-computed features) and with the default, from b = ones,
    x0 = 0: device time of each (median of `reps` after a warm-up), status and relres."""
    import torch

    import gen
    import paper_2109_01232_b300 as g
    sel = g.Selector(model)
    rows = []
    for k in idx:
        desc = descriptor(data, k)
        p = gen.build_selector_matrix(desc)
        A = g.DeviceCSR.from_problem(p)
        bt = torch.ones(p.n, dtype=torch.float64, device="cuda")
        x = torch.zeros_like(bt)
        ps, cls, conf = sel.choose(A)
        chosen = dict(restart_m=int(ps.restart_m), inner_prec=int(ps.inner_prec),
                      poly_degree=int(ps.poly_degree), inner_rtol=float(ps.inner_rtol))
        out = {}
        for name, prm in (("default", dict(restart_m=DEFAULT["m"], inner_prec=DEFAULT["prec"],
                                           poly_degree=DEFAULT["degree"],
                                           inner_rtol=DEFAULT["inner_rtol"])),
                          ("selected", chosen)):
            plan = g.Plan(A, "ir", rtol=rtol, max_iters=DEFAULT_CAP, seed=desc["seed"], **prm)
            ts, r = [], None
            for _ in range(reps + 1):
                x.zero_()
                r = plan.solve(bt, x)
                ts.append(r.t_solve_ms)
            plan.close()
            out[name] = dict(ms=float(np.median(ts[1:])), status=r.status_name, iters=r.iters,
                             relres=r.relres)
        row = dict(index=int(k), n=p.n, chosen=chosen, cls=cls, confidence=conf, **out)
        rows.append(row)
        if log:
            log(row)
    ok_def = [r for r in rows if r["default"]["status"] == "OK"]
    ratio = [r["selected"]["ms"] / r["default"]["ms"] for r in ok_def
             if r["selected"]["status"] == "OK"]
    lost = sum(1 for r in ok_def if r["selected"]["status"] != "OK")
    return dict(rows=rows, geomean_ratio=float(np.exp(np.mean(np.log(ratio)))) if ratio else None,
                lost_convergence=lost, n=len(rows),
                converged_default=len(ok_def),
                converged_selected=sum(1 for r in rows if r["selected"]["status"] == "OK"))


def split(n: int, held_out: int, seed: int = 4999):
    perm = np.random.Generator(np.random.PCG64(seed)).permutation(n)
    return np.sort(perm[held_out:]), np.sort(perm[:held_out])


CORPUS_N_HI, CORPUS_COUNT, CORPUS_HELD_OUT = 4e6, 400, 80


def corpus_split(data: dict, held_out: int = CORPUS_HELD_OUT, seed: int = 4999):
    """Train / held-out positions of a sweep that holds the whole configured corpus
    (gen.selector_matrices(400, n_hi=4e6)): the held-out matrices are the corpus indices
    permutation(400)[:80] of PCG64(seed); every other swept matrix trains, except a matrix of
    another corpus drawn from the same seed as a held-out one (same dimension, Peclet
    number, anisotropy and wind at another size), which is left out of both."""
    nh, di, ds = data["desc_n_hi"], data["desc_index"], data["desc_seed"]
    conf = nh == CORPUS_N_HI
    if sorted(di[conf].tolist()) != list(range(CORPUS_COUNT)):
        raise ValueError("the sweep does not hold every matrix of the configured corpus")
    held_idx = np.random.Generator(np.random.PCG64(seed)).permutation(CORPUS_COUNT)[:held_out]
    te = np.flatnonzero(conf & np.isin(di, held_idx))
    held_seeds = ds[te]
    tr = np.flatnonzero(~np.isin(np.arange(len(nh)), te) & ~(~conf & np.isin(ds, held_seeds)))
    return tr, te


def _ratio(times, t0):
    """Time relative to the default; failures count as the timeout factor."""
    r = times / t0
    return np.where(np.isfinite(r), r, TIMEOUT_FACTOR)


def fit(data: dict, train_idx, epochs: int = 1000, lr: float = 3e-3, seed: int = 4242,
        min_confidence: float = 0.0):
    """Per-class tolerances, labels and GPU training (gmres_mlp_train) on train_idx."""
    import gen
    import paper_2109_01232_b300 as g
    T, T0, F = data["times"][train_idx], data["default_ms"][train_idx], data["features"][train_idx]
    # each class keeps the tolerance with the smallest geometric-mean time ratio to the
    # default, over the training matrices on which the default converges
    ok = np.isfinite(T0)
    tol_idx = np.zeros(N_CLASSES, int)
    for c in range(N_CLASSES):
        gm = [np.exp(np.mean(np.log(_ratio(T[ok, c, t], T0[ok])))) for t in range(len(TOLS))]
        tol_idx[c] = int(np.argmin(gm))
    # labels: the fastest class on every training matrix that some class solves (also where
    # the default does not converge)
    Tc = np.stack([T[:, c, tol_idx[c]] for c in range(N_CLASSES)], axis=1)
    solved = np.isfinite(Tc).any(axis=1)
    T, T0, F, Tc = T[solved], T0[solved], F[solved], Tc[solved]
    labels = np.argmin(np.where(np.isfinite(Tc), Tc, np.inf), axis=1)
    mean = F.mean(axis=0)
    std = F.std(axis=0)
    scale = np.where(std > 1e-6, 1.0 / np.maximum(std, 1e-6), 0.0).astype(np.float32)
    X = ((F - mean) * scale).astype(np.float32)
    params, losses = g.mlp_train(gen.mlp_init(seed), X, labels, epochs, lr)
    cm = np.array([class_config(c)[0] for c in range(N_CLASSES)], np.int32)
    cd = np.array([class_config(c)[1] for c in range(N_CLASSES)], np.int32)
    cp = np.array([g.PREC[class_config(c)[2]] for c in range(N_CLASSES)], np.int32)
    ct = np.array([TOLS[tol_idx[c]] for c in range(N_CLASSES)], np.float64)
    return dict(params=params, feat_mean=mean.astype(np.float32), feat_scale=scale,
                class_m=cm, class_degree=cd, class_prec=cp, class_inner_rtol=ct,
                min_confidence=np.float32(min_confidence), train_labels=labels.astype(np.int32),
                train_losses=losses, tol_index=tol_idx)


def predict(model: dict, F) -> tuple[np.ndarray, np.ndarray]:
    """Chosen class (or -1 = default) and confidence for feature rows F (GPU forward)."""
    import paper_2109_01232_b300 as g
    X = ((np.asarray(F, np.float32) - model["feat_mean"]) * model["feat_scale"]).astype(np.float32)
    P = g.mlp_forward(model["params"], X)
    c = P.argmax(axis=1)
    conf = P.max(axis=1)
    c = np.where(conf >= float(model["min_confidence"]), c, -1)
    return c, conf


def evaluate(data: dict, model: dict, idx) -> dict:
    """Time of the selected configuration relative to the default on the matrices idx."""
    c, conf = predict(model, data["features"][idx])
    T, T0 = data["times"][idx], data["default_ms"][idx]
    chosen = np.array([T0[k] if c[k] < 0 else T[k, c[k], model["tol_index"][c[k]]]
                       for k in range(len(idx))])
    ok_def = np.isfinite(T0)
    r = _ratio(chosen[ok_def], T0[ok_def])
    # the best any single class could do with its stored tolerance (the oracle choice)
    best = np.array([min(T[k, cc, model["tol_index"][cc]] for cc in range(N_CLASSES))
                     for k in range(len(idx))])
    return dict(geomean_ratio=float(np.exp(np.mean(np.log(r)))),
                converged_selected=int(np.isfinite(chosen).sum()),
                converged_default=int(ok_def.sum()), n=len(idx),
                best_possible_geomean=float(np.exp(np.mean(np.log(_ratio(best[ok_def], T0[ok_def]))))),
                chosen=c)


def save(path: str, d: dict):
    np.savez_compressed(path, **{k: np.asarray(v) for k, v in d.items()})


def load(path: str) -> dict:
    with np.load(path) as f:
        return {k: f[k] for k in f.files}


def main(argv=None):
    sys.path.insert(0, os.path.dirname(HERE))
    import gen
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    s1 = sub.add_parser("sweep")
    s1.add_argument("--count", type=int, default=128)
    s1.add_argument("--n-hi", type=float, default=2e5)
    s1.add_argument("--first", type=int, default=0, help="sweep matrices [first, last) only")
    s1.add_argument("--last", type=int, default=None)
    s1.add_argument("--n-range", type=float, nargs=2, default=None,
                    help="only the matrices with lo <= N <= hi")
    s1.add_argument("--max", type=int, default=None, help="at most this many matrices")
    s1.add_argument("--tols-from", default=None,
                    help="a model whose per-class tolerance each class is restricted to")
    s1.add_argument("--out", default=SWEEP_PATH)
    s3 = sub.add_parser("merge")
    s3.add_argument("parts", nargs="+")
    s3.add_argument("--out", default=SWEEP_PATH)
    s4 = sub.add_parser("live")
    s4.add_argument("--sweep", default=SWEEP_PATH)
    s4.add_argument("--model", default=MODEL_PATH)
    s4.add_argument("--n-max", type=float, default=2e6)
    s2 = sub.add_parser("fit")
    s2.add_argument("--sweep", default=SWEEP_PATH)
    s2.add_argument("--held-out", type=float, default=0.2,
                    help="share held out when the sweep lacks part of the configured corpus")
    s2.add_argument("--out", default=MODEL_PATH)
    a = ap.parse_args(argv)
    if a.cmd == "sweep":
        descs = gen.selector_matrices(count=a.count, n_hi=a.n_hi)[a.first:a.last]
        if a.n_range:
            descs = [d for d in descs if a.n_range[0] <= d["side"] ** d["dim"] <= a.n_range[1]]
        descs = descs[:a.max]
        tol_index = load(a.tols_from)["tol_index"] if a.tols_from else None
        data = sweep(descs, checkpoint=a.out, tol_index=tol_index, n_hi=a.n_hi)
        save(a.out, data)
    elif a.cmd == "merge":
        parts = [load(q) for q in a.parts]
        for q in parts:  # sweeps written before desc_n_hi existed carry one n_hi for all
            if "desc_n_hi" not in q:
                q["desc_n_hi"] = np.full(len(q["default_ms"]), float(q.get("n_hi", 2e5)))
            if "desc_n" not in q:
                d0 = gen.selector_matrices(count=int(q["desc_index"].max()) + 1,
                                           n_hi=float(q["desc_n_hi"][0]))
                q["desc_n"] = np.array([d0[i]["side"] ** d0[i]["dim"] for i in q["desc_index"]])
        keys = [k for k in parts[0] if k != "n_hi"]
        data = {k: np.concatenate([q[k] for q in parts]) for k in keys}
        order = np.lexsort((data["desc_index"], data["desc_n_hi"]))
        data = {k: v[order] for k, v in data.items()}
        save(a.out, data)
    elif a.cmd == "live":
        data, model = load(a.sweep), load(a.model)
        idx = [int(k) for k in model["held_out"] if data["desc_n"][k] <= a.n_max]
        res = live_evaluate(data, model, idx, log=print)
        print({k: v for k, v in res.items() if k != "rows"})
    else:
        data = load(a.sweep)
        n = len(data["default_ms"])
        try:
            tr, te = corpus_split(data)
        except ValueError:
            tr, te = split(n, int(round(a.held_out * n)))
        model = fit(data, tr)
        model["held_out"] = te
        res = evaluate(data, model, te)
        print({k: v for k, v in res.items() if k != "chosen"})
        save(a.out, model)


if __name__ == "__main__":
    main()
