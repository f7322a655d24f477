"""Learned temperature seed: data from plain Monte Carlo iterations, training
on the library's own network kernels, and seeded versus plain convergence.

For every cloud the Monte Carlo path gives T1 (temperatures after iteration 0:
background and point sources only) and the converged T (dust re-emission
iterated with frozen random numbers until max |dT| < tol).  The network maps
(log T1, log rho), normalised, to log T - log T1.  A seeded run replaces the
start T1 by T1 exp(prediction); the Monte Carlo iterations then continue to
the same fixed point, so they remain both the fallback and the measure of the
seed's error.
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import inputs as I

T_MIN, T_MAX = 2.7, 3000.0


def _ctx_for(w, soc):
    ctx = soc.Context(0, w.seed)
    ctx.dust_upload(w.dust.nu, w.dust.kabs, w.dust.ksca, w.dust.g)
    cid = ctx.grid_upload(w.clouds[0])
    ctx.sources_upload(cid, w.bg_I[0], w.ps_pos[0], w.ps_L[0])
    return ctx, cid


def iteration0(ctx, cid, w, T):
    """Constant sources once: T <- T1 (kept in the context for reuse)."""
    return ctx.iterate(cid, T, n_background=w.n_bg[0], n_point=w.n_ps[0], max_iter=0)


def iterate_from(ctx, cid, T_start, T_out, max_iter, tol):
    """Dust iterations from T_start, reusing iteration 0's absorption."""
    return ctx.iterate(cid, T_out, n_per_cell=1, max_iter=max_iter, dT_tol=tol, T_seed=T_start, reuse_constant=True)


def simulate_cloud(w, max_iter=60, tol=0.1):
    """(T1, T_converged, plain-run info) for one cloud, on the GPU."""
    import torch
    from . import soc
    ctx, cid = _ctx_for(w, soc)
    n = w.clouds[0].n_cells
    T1 = torch.empty(n, dtype=torch.float32, device="cuda")
    iteration0(ctx, cid, w, T1)
    T = torch.empty_like(T1)
    r = iterate_from(ctx, cid, T1, T, max_iter, tol)
    torch.cuda.synchronize()
    out = (T1.cpu().numpy(), T.cpu().numpy(), r)
    ctx.close()
    return out


def features(T1, rho, side, stats):
    """Network input (side^3 x 2, normalised log T1 and log rho)."""
    lt = (np.log(np.clip(T1, T_MIN, T_MAX)) - stats["lt_mean"]) / stats["lt_std"]
    lr = (np.log(np.maximum(rho, 1e-30)) - stats["lr_mean"]) / stats["lr_std"]
    return np.stack([lt, lr], axis=-1).reshape(side, side, side, 2).astype(np.float32)


def make_dataset(seeds, side=64, max_iter=60, tol=0.1, log=print):
    """Plain-MC inputs and targets for the given cloud seeds."""
    T1s, Ts, rhos, info = [], [], [], []
    for s in seeds:
        w = I.config_c4(int(s), side=side)
        t0 = time.perf_counter()
        T1, T, r = simulate_cloud(w, max_iter, tol)
        T1s.append(T1); Ts.append(T); rhos.append(w.clouds[0].rho.copy())
        info.append(dict(seed=int(s), iterations=r["iterations"], converged=r["converged"],
                         seconds=time.perf_counter() - t0, **w.extra))
        log(f"cloud {s}: {r['iterations']} iterations, converged={r['converged']}, max T {T.max():.1f} K")
    return np.array(T1s), np.array(Ts), np.array(rhos), info


def norm_stats(T1, rho):
    lt = np.log(np.clip(T1, T_MIN, T_MAX))
    lr = np.log(np.maximum(rho, 1e-30))
    return dict(lt_mean=float(lt.mean()), lt_std=float(lt.std() + 1e-12),
                lr_mean=float(lr.mean()), lr_std=float(lr.std() + 1e-12))


def init_params(seed=0):
    """He-style initial weights in the packed layout of soc_unet_set_params."""
    rng = np.random.default_rng(seed)
    layers = [(16, 16), (16, 16), (16, 32), (32, 32), (32, 64), (64, 64), (64, 128), (128, 128),
              (192, 64), (64, 64), (96, 32), (32, 32), (48, 16), (16, 16), (16, 16)]
    out = []
    for k, (cin, cout) in enumerate(layers):
        w = rng.normal(0.0, np.sqrt(2.0 / (27 * cin)), size=(cout, 27, cin))
        if k == len(layers) - 1:
            w *= 0.1
            w[1:] = 0.0
        out += [w.ravel(), np.zeros(cout)]
    return np.concatenate(out).astype(np.float32)


def train(X, Y, side, epochs=30, batch=4, lr=1e-3, seed=0, log=print):
    """Adam on MSE of the normalised residual (Y is already normalised, so a
    constant predictor scores 1); the learning rate decays linearly to 10 %.
    Returns the trained net and the loss history."""
    import torch
    from . import soc
    net = soc.UNet(batch, side)
    net.set_params(init_params(seed))
    rng = np.random.default_rng(seed)
    n = X.shape[0]
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    hist = []
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.from_numpy(Y).cuda()
    for ep in range(epochs):
        perm = rng.permutation(n)
        tot = 0.0
        for b0 in range(0, n - batch + 1, batch):
            idx = torch.from_numpy(perm[b0:b0 + batch]).cuda()
            xb = Xd.index_select(0, idx).contiguous()
            yb = Yd.index_select(0, idx).contiguous()
            net.backward(xb, yb, loss=loss)
            net.adam(lr * (1.0 - 0.9 * ep / max(1, epochs - 1)))
            tot += loss.item()
        hist.append(tot / max(1, n // batch))
        log(f"epoch {ep}: loss {hist[-1]:.5f}")
    return net, hist


def predict_seed(net, T1, rho, side, stats):
    """T1 exp(prediction), clamped to the solver's range."""
    import torch
    x = torch.from_numpy(np.repeat(features(T1, rho, side, stats)[None], net.batch, axis=0)).cuda()
    pred = torch.empty((net.batch, side, side, side), dtype=torch.float32, device="cuda")
    net.forward(x, pred)
    p = pred[0].reshape(-1) * stats["y_std"] + stats["y_mean"]
    return torch.clamp(torch.from_numpy(T1).cuda() * torch.exp(p), T_MIN, T_MAX).contiguous()


def compare(net, seeds, side, stats, max_iter=60, tol=0.1, log=print):
    """Wall time to max |dT| < tol for plain and learned-seeded iteration on
    the given (held-out) clouds; both start with the same iteration 0."""
    import torch
    from . import soc
    rows = []
    # one untimed forward: loads the network's kernels before the timed runs
    w0 = I.config_c4(int(seeds[0]), side=side)
    predict_seed(net, np.full(w0.clouds[0].n_cells, 10.0, np.float32), w0.clouds[0].rho, side, stats)
    torch.cuda.synchronize()
    for s in seeds:
        w = I.config_c4(int(s), side=side)
        res = {}
        for mode in ("plain", "learned"):
            ctx, cid = _ctx_for(w, soc)
            n = w.clouds[0].n_cells
            T1 = torch.empty(n, dtype=torch.float32, device="cuda")
            T = torch.empty_like(T1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            iteration0(ctx, cid, w, T1)
            if mode == "learned":
                seed_T = predict_seed(net, T1.cpu().numpy(), w.clouds[0].rho, side, stats)
            else:
                seed_T = T1
            r = iterate_from(ctx, cid, seed_T, T, max_iter, tol)
            torch.cuda.synchronize()
            res[mode] = dict(seconds=time.perf_counter() - t0, iterations=r["iterations"],
                             converged=r["converged"], T=T.cpu().numpy())
            ctx.close()
        d = float(np.abs(res["plain"]["T"] - res["learned"]["T"]).max())
        rows.append(dict(seed=int(s), plain_s=res["plain"]["seconds"], learned_s=res["learned"]["seconds"],
                         plain_iters=res["plain"]["iterations"], learned_iters=res["learned"]["iterations"],
                         plain_converged=res["plain"]["converged"], learned_converged=res["learned"]["converged"],
                         max_abs_T_difference=d))
        log(json.dumps(rows[-1]))
    return rows


def seed_bound(seeds, side=64, max_iter=60, tol=0.1, other_seed=7, log=print):
    """What any seed can gain here: dust iterations to max |dT| < tol from
    (a) the run's own converged T (a perfect predictor), (b) the converged T
    of an independent Monte Carlo realisation of the same cloud (context
    seed `other_seed`: a prediction as good as the method's own answer but
    without this run's frozen noise) and (c) T1 (the plain start)."""
    import torch
    from . import soc
    rows = []
    for s in seeds:
        w = I.config_c4(int(s), side=side)
        n = w.clouds[0].n_cells
        runs = {}
        for cseed in (w.seed, other_seed):
            ctx = soc.Context(0, cseed)
            ctx.dust_upload(w.dust.nu, w.dust.kabs, w.dust.ksca, w.dust.g)
            cid = ctx.grid_upload(w.clouds[0])
            ctx.sources_upload(cid, w.bg_I[0], w.ps_pos[0], w.ps_L[0])
            T1 = torch.empty(n, dtype=torch.float32, device="cuda")
            T = torch.empty_like(T1)
            iteration0(ctx, cid, w, T1)
            iterate_from(ctx, cid, T1, T, max_iter, tol)
            runs[cseed] = (ctx, cid, T1, T)
        ctx, cid, T1, T = runs[w.seed]
        T_other = runs[other_seed][3]
        row = dict(seed=int(s))
        for name, start in (("own_converged", T), ("other_realisation", T_other), ("T1", T1)):
            out = torch.empty_like(T1)
            row[name + "_iters"] = iterate_from(ctx, cid, start.contiguous(), out, max_iter, tol)["iterations"]
        d = (T_other - T).double()
        row["realisations_max_abs_dT_K"] = float(d.abs().max().item())
        row["realisations_rms_rel_dT"] = float(((T_other.double() / T.double() - 1) ** 2).mean().sqrt().item())
        for c in runs.values():
            c[0].close()
        rows.append(row)
        log(json.dumps(row))
    return rows


def run(side=64, n_train=160, n_test=20, epochs=60, max_iter=60, tol=0.1, lr=2e-3, log=print):
    """The whole comparison: data from the plain Monte Carlo path (training
    clouds), training, then plain against learned-seeded runs to max|dT| <
    tol on the test clouds.  Returns the summary (times in seconds)."""
    t0 = time.perf_counter()
    train_seeds = np.arange(1000, 1000 + n_train)
    test_seeds = np.arange(2000, 2000 + n_test)
    T1, T, rho, info = make_dataset(train_seeds, side, max_iter, tol, log=log)
    t_data = time.perf_counter() - t0
    stats = norm_stats(T1, rho)
    X = np.stack([features(T1[i], rho[i], side, stats) for i in range(len(train_seeds))])
    Y = (np.log(np.clip(T, T_MIN, T_MAX)) - np.log(np.clip(T1, T_MIN, T_MAX))).reshape(-1, side, side, side)
    stats["y_mean"] = float(Y.mean())
    stats["y_std"] = float(Y.std() + 1e-12)
    Y = ((Y - stats["y_mean"]) / stats["y_std"]).astype(np.float32)
    t1 = time.perf_counter()
    net, hist = train(X, Y, side, epochs=epochs, lr=lr, log=log)
    t_train = time.perf_counter() - t1
    rows = compare(net, test_seeds, side, stats, max_iter, tol, log=log)
    summary = dict(side=side, n_train=n_train, n_test=n_test, epochs=epochs, tol_K=tol,
                   data_seconds=t_data, train_seconds=t_train, loss_history=hist, train_info=info,
                   test=rows, norm=stats,
                   plain_total_s=sum(r["plain_s"] for r in rows), learned_total_s=sum(r["learned_s"] for r in rows),
                   plain_iters_mean=float(np.mean([r["plain_iters"] for r in rows])),
                   learned_iters_mean=float(np.mean([r["learned_iters"] for r in rows])))
    return summary


def main():
    ap = argparse.ArgumentParser(description="learned temperature seed: data, training, comparison")
    ap.add_argument("--side", type=int, default=64)
    ap.add_argument("--train", type=int, default=160)
    ap.add_argument("--test", type=int, default=20)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--max-iter", type=int, default=60)
    ap.add_argument("--tol", type=float, default=0.1)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--out", default="learned_seed.json")
    ap.add_argument("--bound", action="store_true",
                    help="only measure what an ideal seed can gain on the test clouds (no training)")
    a = ap.parse_args()
    if a.bound:
        rows = seed_bound(np.arange(2000, 2000 + a.test), a.side, a.max_iter, a.tol)
        keys = ["own_converged_iters", "other_realisation_iters", "T1_iters"]
        print(json.dumps({k: float(np.mean([r[k] for r in rows])) for k in keys}))
        return
    summary = run(a.side, a.train, a.test, a.epochs, a.max_iter, a.tol, a.lr)
    os.makedirs(os.path.dirname(a.out) or ".", exist_ok=True)
    with open(a.out, "w") as f:
        json.dump(summary, f, indent=1)
    print(json.dumps({k: v for k, v in summary.items() if k not in ("loss_history", "train_info", "test")}))


if __name__ == "__main__":
    main()
