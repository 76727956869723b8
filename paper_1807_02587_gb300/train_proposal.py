"""Train the pose-proposal network on the GPU and save its parameters.

    python -m paper_1807_02587_gb300.train_proposal --pairs 100000 --out <file.npz>

Training pairs: SO(3)-uniform poses of synthetic plane/box/sphere scenes
(``synth.so3_scene_set``: each scene sampled twice, ``--per-scene`` poses of
the second sample), generated on the host in a spawn process pool, labelled
on the GPU by the plain method from five starts (``proposal.label_pairs``),
labels checked against the ground truth.  The network then trains with Adam
on the GPU (``proposal.train``) and is evaluated on held-out SO(3) pairs
against the plain method from the identity.  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import time
from concurrent.futures import ProcessPoolExecutor

import numpy as np

DEFAULT_OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "proposal_mlp.npz")


def _chunk(args):
    """Host-side generation of one chunk (runs in a worker process)."""
    from paper_1807_02587_gb300 import synth
    seed, n_scenes, per_scene, n = args
    sc = synth.so3_scene_set(seed, n_scenes, per_scene, n)
    tgts = [[synth.apply(sc["T"][i, j], sc["tgt_base"][i].astype(np.float64)).astype(np.float32)
             for j in range(per_scene)] for i in range(n_scenes)]
    return sc["src"], tgts, sc["T"]


def _pairset(chunk):
    from paper_1807_02587_gb300 import proposal as P
    src, tgts, T = chunk
    clouds, src_of, tgt_of, Ts = [], [], [], []
    for i in range(len(src)):
        si = len(clouds)
        clouds.append(src[i])
        for j, t in enumerate(tgts[i]):
            tgt_of.append(len(clouds))
            src_of.append(si)
            clouds.append(t)
            Ts.append(T[i, j])
    return P.PairSet(clouds, src_of, tgt_of, np.array(Ts))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--pairs", type=int, default=100000)
    ap.add_argument("--per-scene", type=int, default=8)
    ap.add_argument("--points", type=int, default=8000, help="points per training cloud")
    ap.add_argument("--chunk-scenes", type=int, default=250)
    ap.add_argument("--label-depth", type=int, default=3)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--w-t", type=float, default=1.0)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--workers", type=int, default=max(1, min(16, (os.cpu_count() or 2) - 1)))
    ap.add_argument("--test-pairs", type=int, default=256)
    ap.add_argument("--test-points", type=int, default=50000)
    ap.add_argument("--out", default=DEFAULT_OUT)
    args = ap.parse_args(argv)

    n_scenes = max(1, args.pairs // args.per_scene)
    jobs = [(args.seed * 1000003 + 7919 * c, min(args.chunk_scenes, n_scenes - c * args.chunk_scenes),
             args.per_scene, args.points)
            for c in range((n_scenes + args.chunk_scenes - 1) // args.chunk_scenes)]
    t0 = time.perf_counter()
    # the workers start before the first CUDA call (spawn: no CUDA state is inherited)
    pool = ProcessPoolExecutor(max_workers=args.workers, mp_context=mp.get_context("spawn"))
    window = 2 * args.workers  # chunks in flight: bounds host memory
    futures = [pool.submit(_chunk, j) for j in jobs[:window]]

    import torch
    from paper_1807_02587_gb300 import binding as B
    from paper_1807_02587_gb300 import proposal as P

    Xs, Ls, Ks, label_stats = [], [], [], []
    label_s = 0.0
    for k in range(len(jobs)):
        ps = _pairset(futures[k].result())
        futures[k] = None
        if k + window < len(jobs):
            futures.append(pool.submit(_chunk, jobs[k + window]))
        X, L, keep, st = P.label_pairs(ps, depth=args.label_depth, iters=30)
        label_s += st["seconds"]
        Xs.append(X)
        Ls.append(L)
        Ks.append(keep)
        label_stats.append(st["label_within_tol"])
        del ps
    pool.shutdown()
    X = torch.cat(Xs)
    L = torch.cat(Ls)
    keep = np.concatenate(Ks)
    gen_s = time.perf_counter() - t0

    net = B.Mlp(args.batch)
    B.hgmm_mlp_set_params(net.handle, P.init_params(args.seed))
    t1 = time.perf_counter()
    last = P.train(net, X, L, keep, epochs=args.epochs, batch=args.batch, lr=args.lr, w_t=args.w_t,
                   seed=args.seed)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t1
    params = B.hgmm_mlp_get_params(net.handle)
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    np.savez_compressed(args.out, params=params)

    ts = P.so3_test_pairs(args.seed + 777, args.test_pairs, args.test_points)
    res = P.evaluate(net, ts, depth=4, iters=30)
    out = {"train_pairs": int(keep.shape[0]), "train_rows_kept": int(keep.sum()),
           "label_within_1deg": float(np.mean(label_stats)), "gen_and_label_s": gen_s,
           "label_gpu_s": label_s, "train_s": train_s, "epochs": args.epochs, "batch": args.batch,
           "final_loss": last, "out": args.out, **res}
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
