"""Train the learned preconditioner network and compare it with j-step Jacobi.

Pairs (r, e = A^{-1} r) come from the plain solver itself (FP64 Jacobi block BiCGGR) on seeded
synthetic gauge configurations; the network is trained on the training configurations with the
library's own forward/backward/Adam kernels and evaluated, as M in block BiCGGR, on held-out
configurations against Jacobi (FP64 and FP32 sweeps) and against no preconditioner.

    python -m paper_0907_3261_gb300.train_net --steps 600 --out weights.npz
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np


def make_pairs(wd, I, torch, dims, kappa, csw, seeds, L, eps, j_data, dev):
    """(ctx, R, E) per configuration: Z4 sources and their solutions from the FP64 solver."""
    pairs = []
    for s in seeds:
        links = torch.from_numpy(I.random_links(dims, eps, seed=s)).to(dev)
        ctx = wd.wd_create(links, dims, kappa, csw)
        R = torch.from_numpy(I.z4_noise(dims, L, seed=1000 + s)).to(dev)
        E, info = wd.bbicggr_solve(ctx, R, j=j_data, tol=1e-10)
        if info["status"] != wd.WD_OK:
            raise RuntimeError(f"training data solve failed on seed {s}: {info['status_name']}")
        pairs.append((ctx, R, E))
    return pairs


def train(wd, net, pairs, steps, lr, log_every=100):
    hist = []
    for step in range(steps):
        ctx, R, E = pairs[step % len(pairs)]
        loss, _ = wd.wd_net_loss_grad(ctx, net, R, E, want_grad=False)
        wd.wd_net_adam_step(net, lr * (0.1 ** (step / max(steps, 1))))
        hist.append(loss)
        if log_every and step % log_every == 0:
            print(f"step {step}: loss {loss:.4e}", file=sys.stderr, flush=True)
    return hist


def held_out_loss(wd, net, pairs):
    return float(np.mean([wd.wd_net_loss_grad(c, net, R, E, want_grad=False)[0]
                          for c, R, E in pairs]))


def compare(wd, I, torch, net, dims, kappa, csw, seeds, L, eps, j, dev, maxit=3000):
    """Iterations and time of block BiCGGR with each preconditioner on held-out configurations:
    FP64, FP32 and double-float Jacobi (the last with double-float direction recurrences), the
    network with FP64 or double-float direction recurrences, and no preconditioner."""
    rows = []
    for s in seeds:
        links = torch.from_numpy(I.random_links(dims, eps, seed=s)).to(dev)
        ctx = wd.wd_create(links, dims, kappa, csw)
        B = torch.from_numpy(I.z4_noise(dims, L, seed=2000 + s)).to(dev)
        row = {"seed": s}
        for name, kw in (("jacobi_fp64", dict(j=j)), ("jacobi_fp32", dict(j=j, precision=1)),
                         ("jacobi_df_dirs", dict(j=j, precision=5)),
                         ("network", dict(j=j, net=net)),
                         ("network_df_dirs", dict(j=j, net=net, precision=2)),
                         ("none", dict(j=0))):
            wd.bbicggr_solve(ctx, B, maxit=maxit, **kw)                  # warm-up (autotuning)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, info = wd.bbicggr_solve(ctx, B, maxit=maxit, **kw)
            torch.cuda.synchronize()
            row[name] = {"status": info["status_name"], "iters": info["iters"],
                         "seconds": time.perf_counter() - t0,
                         "true_resid": info["max_true_resid"], "fallbacks": info["fallbacks"]}
        rows.append(row)
        wd.wd_destroy(ctx)
    return rows


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", default="8,8,8,8")
    ap.add_argument("--kappa", type=float, default=0.13)
    ap.add_argument("--csw", type=float, default=1.0)
    ap.add_argument("--eps", type=float, default=0.2)
    ap.add_argument("--L", type=int, default=12)
    ap.add_argument("--j", type=int, default=12)
    ap.add_argument("--layers", type=int, default=4)
    ap.add_argument("--hidden", type=int, default=4)
    ap.add_argument("--train-seeds", type=int, default=16)
    ap.add_argument("--test-seeds", type=int, default=4)
    ap.add_argument("--steps", type=int, default=600)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--eval-dims", default="", help="also evaluate on this lattice (e.g. 16,16,16,32)")
    ap.add_argument("--out", default="")
    args = ap.parse_args(argv)
    import torch
    import paper_0907_3261_gb300 as wd
    from paper_0907_3261_gb300 import inputs as I
    dev = torch.device("cuda", torch.cuda.current_device())
    dims = tuple(int(x) for x in args.dims.split(","))
    tr = list(range(args.train_seeds))
    te = list(range(args.train_seeds, args.train_seeds + args.test_seeds))
    t0 = time.perf_counter()
    pairs = make_pairs(wd, I, torch, dims, args.kappa, args.csw, tr, args.L, args.eps, args.j, dev)
    test_pairs = make_pairs(wd, I, torch, dims, args.kappa, args.csw, te, args.L, args.eps, args.j, dev)
    t_data = time.perf_counter() - t0
    net = wd.wd_net_create(args.layers, args.hidden,
                           I.network_weights(args.layers, args.hidden, seed=7, noise=0.01))
    loss0 = held_out_loss(wd, net, test_pairs)
    t0 = time.perf_counter()
    hist = train(wd, net, pairs, args.steps, args.lr)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    loss1 = held_out_loss(wd, net, test_pairs)
    summary = {"dims": dims, "kappa": args.kappa, "layers": args.layers, "hidden": args.hidden,
               "train_configs": len(tr), "test_configs": len(te), "steps": args.steps,
               "data_seconds": t_data, "train_seconds": t_train,
               "train_loss_first": hist[0], "train_loss_last": hist[-1],
               "held_out_loss_before": loss0, "held_out_loss_after": loss1,
               "held_out": compare(wd, I, torch, net, dims, args.kappa, args.csw, te, args.L,
                                   args.eps, args.j, dev)}
    if args.eval_dims:
        ed = tuple(int(x) for x in args.eval_dims.split(","))
        summary["transfer"] = compare(wd, I, torch, net, ed, args.kappa, args.csw, [0], args.L,
                                      args.eps, args.j, dev)
    if args.out:
        w = wd.wd_net_get_weights(net)
        np.savez(args.out, *w, layers=args.layers, hidden=args.hidden)
    print(json.dumps(summary))
    return summary


if __name__ == "__main__":
    main()
