"""Training of the learned far-field correction on the GPU.

The training set is generated by the library itself: for seeded meshes it
builds the cluster tree, samples admissible (target leaf, cluster) pairs at
an opening angle and labels them with the direct sums over the members
(``tp_far_sample_pairs``).  The network is then trained with the library's
own BF16 tensor-core forward/backward kernels and AdamW (``tp_far_train``).

    python -m paper_2509_22110_gb300.far_train --out far_model.bin

defaults to the full configuration: 50 level-7 SH-deformed spheres (seeds
1000-1049), about 40,000 pairs per mesh (2 M pairs) at theta = 0.25.
"""

from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import _tp, meshgen


def sample_meshes(ctx, seeds, level, theta, pairs_per_mesh, seed=0, log=print, leaf=16):
    """Append sampled, labelled pairs of each mesh (tree leaves of up to `leaf`
    triangles) to the context's training set."""
    import torch

    total = 0
    for s in seeds:
        V, F = meshgen.sh_deformed_sphere(level, 12, 0.05, int(s))
        Vd = torch.tensor(V, device="cuda")
        Fd = torch.tensor(F, device="cuda")
        _tp.tp_mesh_upload(ctx, Vd, Fd)
        _tp.tp_tree_build(ctx, int(leaf), 30)
        n_far = _tp.tp_far_sample_pairs(ctx, theta, 1.0, 0, 0)
        keep = min(1.0, pairs_per_mesh / max(1, n_far))
        added = _tp.tp_far_sample_pairs(ctx, theta, keep, seed * 1000003 + int(s), int(pairs_per_mesh * 1.2) + 16)
        total += added
        if log:
            log(f"mesh seed {s}: {n_far} admissible pairs, kept {added}")
    return total


def train(ctx, steps, batch=4096, lr=2e-3, lr_min=1e-4, wd=1e-4, seed=0, chunk=50, log=print):
    """Cosine-decayed AdamW; returns the list of (step, loss)."""
    hist = []
    done = 0
    while done < steps:
        n = min(chunk, steps - done)
        frac = done / max(1, steps)
        cur = lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * frac))
        loss = _tp.tp_far_train(ctx, n, batch, cur, wd, seed + done)
        done += n
        hist.append((done, loss))
        if log and (done % (chunk * 10) == 0 or done == steps):
            log(f"step {done}: loss {loss:.5f} (lr {cur:.2e})")
    return hist


def keep_channels(ctx, channels):
    """Zero the output rows of the channels not listed, so their factor is exp(0) = 1."""
    P, N = _tp.tp_far_get_params(ctx)
    w4 = 64 * 24 + 64 + 2 * (64 * 64 + 64)
    b4 = w4 + 7 * 64
    for c in range(7):
        if c not in channels:
            P[w4 + c * 64: w4 + (c + 1) * 64] = 0.0
            P[b4 + c] = 0.0
    _tp.tp_far_set_params(ctx, P, N)


def evaluate(ctx, seeds, level, thetas, log=print, bh_leaves=(), bh_thetas=(), leaf=16):
    """Energy and gradient errors of plain Barnes-Hut, of the learned correction
    and of the learned correction of the energy channels only
    (TP_LEARNED_ENERGY), against the direct sum (FP32 pair terms, FP64
    accumulation), with the device time of each evaluation (tree build
    included), on held-out meshes.  The tree has leaves of up to `leaf`
    triangles (the size the model was trained with); for every size in bh_leaves plain Barnes-Hut is evaluated again on a tree
    with leaves of that size, at the opening angles bh_thetas (rows
    "bh_leaf<size>")."""
    import torch

    rows = []
    for s in seeds:
        V, F = meshgen.sh_deformed_sphere(level, 12, 0.05, int(s))
        Vd = torch.tensor(V, device="cuda")
        Fd = torch.tensor(F, device="cuda")
        _tp.tp_mesh_upload(ctx, Vd, Fd)
        gd = torch.zeros_like(Vd)
        ed = _tp.tp_gradient(ctx, gd, _tp.tp_params_default())
        td = _tp.tp_get_stats(ctx)["ms_total"]
        _tp.tp_tree_build(ctx, int(leaf), 30)
        tb_ms = _tp.tp_get_stats(ctx)["ms_total"]
        for th in thetas:
            for name, mode, flags in (("bh", _tp.TP_BH, 0), ("learned", _tp.TP_LEARNED, 0),
                                      ("learned_energy", _tp.TP_LEARNED, _tp.TP_LEARNED_ENERGY)):
                g = torch.zeros_like(Vd)
                e = _tp.tp_gradient(ctx, g, _tp.tp_params_default(mode=mode, theta=th, flags=flags))
                st = _tp.tp_get_stats(ctx)
                rows.append(dict(seed=int(s), theta=th, mode=name,
                                 energy_err=abs(e - ed) / abs(ed),
                                 grad_err=float(torch.linalg.norm(g - gd) / torch.linalg.norm(gd)),
                                 ms_eval=st["ms_total"] + tb_ms, ms_direct=td,
                                 far_terms=st["far_terms"], learned_terms=st["learned_terms"]))
                if log:
                    r = rows[-1]
                    log(f"seed {s} theta {th} {r['mode']:14s}: energy err {r['energy_err']:.3e} grad err "
                        f"{r['grad_err']:.3e} {r['ms_eval']:.2f} ms (direct {td:.2f} ms)")
        for bl in bh_leaves:
            for th in bh_thetas:
                _tp.tp_tree_build(ctx, int(bl), 30)
                tb = _tp.tp_get_stats(ctx)["ms_total"]
                g = torch.zeros_like(Vd)
                e = _tp.tp_gradient(ctx, g, _tp.tp_params_default(mode=_tp.TP_BH, theta=th))
                st = _tp.tp_get_stats(ctx)
                rows.append(dict(seed=int(s), theta=th, mode=f"bh_leaf{int(bl)}",
                                 energy_err=abs(e - ed) / abs(ed),
                                 grad_err=float(torch.linalg.norm(g - gd) / torch.linalg.norm(gd)),
                                 ms_eval=st["ms_total"] + tb, ms_direct=td,
                                 far_terms=st["far_terms"], learned_terms=0))
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default="far_model.bin")
    ap.add_argument("--level", type=int, default=7)
    ap.add_argument("--leaf", type=int, default=16, help="cluster leaf size of the trees (training and evaluation)")
    ap.add_argument("--seeds", type=int, nargs=2, default=[1000, 1050])
    ap.add_argument("--pairs-per-mesh", type=int, default=40000)
    ap.add_argument("--theta", type=float, nargs="+", default=[0.25],
                    help="opening angles to sample training pairs at (pairs-per-mesh each)")
    ap.add_argument("--channels", type=int, nargs="+", default=list(range(7)),
                    help="output channels kept in the saved model (others predict factor 1)")
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--init-seed", type=int, default=1234, help="seed of the network's initial weights")
    ap.add_argument("--train-seed", type=int, default=0, help="seed of the minibatch order")
    ap.add_argument("--eval-seeds", type=int, nargs=2, default=None)
    ap.add_argument("--eval-thetas", type=float, nargs="+", default=[0.25, 0.5])
    ap.add_argument("--summary", default=None, help="write the evaluation rows as JSON here")
    ap.add_argument("--bh-leaves", type=int, nargs="*", default=[],
                    help="also evaluate plain Barnes-Hut on trees with these leaf sizes (at --bh-thetas)")
    ap.add_argument("--bh-thetas", type=float, nargs="*", default=[])
    ap.add_argument("--eval-only", default=None, metavar="MODEL",
                    help="skip training: load this model file and evaluate it on --eval-seeds")
    args = ap.parse_args()
    import torch

    ctx = _tp.tp_create(0, torch.cuda.current_stream().cuda_stream)
    if args.eval_only:
        if not args.eval_seeds:
            ap.error("--eval-only needs --eval-seeds")
        _tp.tp_far_model_load(ctx, args.eval_only)
        rows = evaluate(ctx, range(*args.eval_seeds), args.level, args.eval_thetas, log=None,
                        bh_leaves=args.bh_leaves, bh_thetas=args.bh_thetas, leaf=args.leaf)
        summ = {}
        for th in args.eval_thetas:
            for mode in ("bh", "learned", "learned_energy"):
                rs = [r for r in rows if r["theta"] == th and r["mode"] == mode]
                summ[f"{mode}@{th}"] = {k: {"min": float(np.min([r[k] for r in rs])),
                                            "mean": float(np.mean([r[k] for r in rs])),
                                            "max": float(np.max([r[k] for r in rs]))}
                                        for k in ("energy_err", "grad_err", "ms_eval")}
        for bl in args.bh_leaves:
            for th in args.bh_thetas:
                rs = [r for r in rows if r["theta"] == th and r["mode"] == f"bh_leaf{bl}"]
                summ[f"bh_leaf{bl}@{th}"] = {k: {"min": float(np.min([r[k] for r in rs])),
                                                   "mean": float(np.mean([r[k] for r in rs])),
                                                   "max": float(np.max([r[k] for r in rs]))}
                                               for k in ("energy_err", "grad_err", "ms_eval")}
        print(json.dumps(summ))
        if args.summary:
            with open(args.summary, "w") as f:
                json.dump({"model": args.eval_only, "eval": summ, "rows": rows}, f, indent=1)
        _tp.tp_destroy(ctx)
        return
    t0 = time.time()
    _tp.tp_far_model_init(ctx, args.init_seed)
    _tp.tp_far_dataset_reset(ctx)
    n = 0
    for th in args.theta:
        n += sample_meshes(ctx, range(*args.seeds), args.level, th, args.pairs_per_mesh, seed=int(th * 1000),
                           leaf=args.leaf)
    t1 = time.time()
    _tp.tp_far_fit_normalisation(ctx)
    hist = train(ctx, args.steps, args.batch, args.lr, seed=args.train_seed)
    t2 = time.time()
    if sorted(args.channels) != list(range(7)):
        keep_channels(ctx, args.channels)
    _tp.tp_far_model_save(ctx, args.out)
    print(f"{n} pairs in {t1 - t0:.1f} s; {args.steps} steps in {t2 - t1:.1f} s; final loss {hist[-1][1]:.5f}; "
          f"saved {args.out}")
    if args.eval_seeds:
        rows = evaluate(ctx, range(*args.eval_seeds), args.level, args.eval_thetas, leaf=args.leaf)
        summ = {}
        for th in args.eval_thetas:
            for mode in ("bh", "learned", "learned_energy"):
                rs = [r for r in rows if r["theta"] == th and r["mode"] == mode]
                summ[f"{mode}@{th}"] = {k: float(np.mean([r[k] for r in rs])) for k in
                                        ("energy_err", "grad_err", "ms_eval", "ms_direct")}
        print(json.dumps(summ))
        if args.summary:
            with open(args.summary, "w") as f:
                json.dump({"train": {"pairs": n, "steps": args.steps, "final_loss": hist[-1][1],
                                     "level": args.level, "seeds": args.seeds, "theta": args.theta,
                                     "channels": args.channels},
                           "eval": summ, "rows": rows}, f, indent=1)
    _tp.tp_destroy(ctx)


if __name__ == "__main__":
    main()
