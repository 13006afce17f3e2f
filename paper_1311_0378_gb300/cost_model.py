"""Training and use of the learned cost model (the scheduler's analogue of the
paper's performance-aware task scheduling, Sec. IV: per-task cost estimates
decide how and in which order tasks run).

Pipeline (every step on the GPU goes through the C ABI):
  1. tiles from the seeded generator (the uneven-size law: H, W in
     {256..4096 step 256}, blob density uniform in [0, 1/1000], radius 3..20,
     h-dome / fill-holes markers 50/50, 8-connectivity);
  2. labels measured by the method itself: each tile reconstructed alone with
     variant A (scan pairs to stability, no queue) and variant B (k scan pairs
     then the queue), device time from CUDA events -> log(ms);
  3. features: recon_features (16-bin histogram of I - J, blob-pixel and
     zero-marker fractions, log sizes);
  4. training: recon_mlp_train (the library's forward / backward / Adam
     kernels) on standardised targets;
  5. the weights, target normalisation and variant ids go to a small file that
     recon_sched_set_model installs for RECON_FLAG_LEARNED batches.
The model never touches pixel values: it only picks each tile's variant and
the packing order (decreasing predicted cost).
"""
from __future__ import annotations

import json
import os
import struct
import time
from typing import List, Sequence, Tuple

import numpy as np

import paper_1311_0378_gb300 as rc

MODEL_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cost_model.bin")
MAGIC = b"RCM1"


def save(path: str, theta: np.ndarray, norm: Sequence[float], variants: Tuple[int, int], meta: dict) -> None:
    head = json.dumps(meta).encode()
    with open(path, "wb") as f:
        f.write(MAGIC)
        f.write(struct.pack("<iii", variants[0], variants[1], len(head)))
        f.write(np.asarray(norm, np.float32).tobytes())
        f.write(np.asarray(theta, np.float32).tobytes())
        f.write(head)


def load(path: str = MODEL_PATH):
    with open(path, "rb") as f:
        if f.read(4) != MAGIC:
            raise ValueError("not a cost model file: " + path)
        va, vb, nh = struct.unpack("<iii", f.read(12))
        norm = np.frombuffer(f.read(16), np.float32).copy()
        theta = np.frombuffer(f.read(4 * rc.RECON_MLP_NPARAMS), np.float32).copy()
        meta = json.loads(f.read(nh).decode())
    return theta, norm, (va, vb), meta


def install(ctx, path: str = MODEL_PATH) -> dict:
    theta, norm, (va, vb), meta = load(path)
    rc.check(rc.recon_sched_set_model(ctx, theta, norm, va, vb), "recon_sched_set_model")
    return meta


def label_chunk(ctx, specs, seed, variants, torch, dev):
    """Features and per-variant log device times of one chunk of tiles."""
    import synth
    n = len(specs)
    Ih = [torch.empty((s.H, s.W), dtype=torch.uint8).pin_memory() for s in specs]
    Jh = [torch.empty((s.H, s.W), dtype=torch.uint8).pin_memory() for s in specs]
    synth.generate_into(specs, seed, [x.data_ptr() for x in Ih], [x.data_ptr() for x in Jh])
    Id = [x.to(dev, non_blocking=True) for x in Ih]
    J0 = [x.to(dev, non_blocking=True) for x in Jh]
    Jd = [x.clone() for x in J0]
    torch.cuda.synchronize()
    tiles = [(a.data_ptr(), b.data_ptr(), s.H, s.W, s.W, s.conn) for a, b, s in zip(Id, Jd, specs)]
    feat = torch.zeros((n, rc.RECON_NFEAT), dtype=torch.float32, device=dev)
    rc.check(rc.recon_features(ctx, tiles, feat.data_ptr()), "recon_features")
    ms = np.zeros((n, len(variants)))
    work = []
    for t in range(n):
        for v, var in enumerate(variants):
            Jd[t].copy_(J0[t])
            torch.cuda.synchronize()
            rc.check(rc.recon_batch_ex(ctx, [tiles[t]], [var], None), "label run")
            ms[t, v] = rc.recon_last_kernel_ms(ctx)
            work.append(rc.recon_get_work(ctx, 1)[0])
    return feat.cpu().numpy(), np.log(np.maximum(ms, 1e-4)), work


def build_dataset(ctx, specs, seed, variants, chunk=64):
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    X, Y = [], []
    for s in range(0, len(specs), chunk):
        f, y, _ = label_chunk(ctx, specs[s:s + chunk], seed, variants, torch, dev)
        X.append(f)
        Y.append(y)
    return np.concatenate(X), np.concatenate(Y)


def train(ctx, X: np.ndarray, Y: np.ndarray, epochs=200, batch=256, lr=2e-3, seed=0):
    """Trains on the GPU; returns (theta fp32, norm, per-epoch losses)."""
    import torch
    mean, std = Y.mean(axis=0), Y.std(axis=0) + 1e-6
    T = (Y - mean) / std
    rng = np.random.default_rng(seed)
    theta = init_params(rng)
    dth = torch.from_numpy(theta).cuda()
    dX = torch.from_numpy(X.astype(np.float32)).cuda()
    dT = torch.from_numpy(T.astype(np.float32)).cuda()
    torch.cuda.synchronize()
    st, losses = rc.recon_mlp_train(ctx, dth.data_ptr(), dX.data_ptr(), dT.data_ptr(), len(X), epochs, batch,
                                    lr, seed)
    rc.check(st, "recon_mlp_train")
    norm = [float(mean[0]), float(std[0]), float(mean[1]), float(std[1])]
    return dth.cpu().numpy(), norm, losses


def init_params(rng) -> np.ndarray:
    """He-uniform weights, zero biases, flat fp32 layout of the C ABI."""
    sizes = [(64, 20), (64,), (64, 64), (64,), (2, 64), (2,)]
    out = []
    for s in sizes:
        if len(s) == 2:
            b = np.sqrt(6.0 / s[1])
            out.append(rng.uniform(-b, b, size=s).ravel())
        else:
            out.append(np.zeros(s))
    return np.concatenate(out).astype(np.float32)


def main():
    import argparse
    import torch
    import synth
    ap = argparse.ArgumentParser(description="train the learned cost model")
    ap.add_argument("--tiles", type=int, default=20000)
    ap.add_argument("--epochs", type=int, default=200)
    ap.add_argument("--out", default=MODEL_PATH)
    ap.add_argument("--queue-k", type=int, default=1)
    args = ap.parse_args()
    w = synth.workload("train20k")
    specs = list(w.tiles[:args.tiles])
    ctx = rc.recon_init(0, 0, 0)
    variants = (-1, args.queue_k)
    t0 = time.time()
    X, Y = build_dataset(ctx, specs, w.seed, variants)
    t1 = time.time()
    theta, norm, losses = train(ctx, X, Y, epochs=args.epochs)
    t2 = time.time()
    pick_b = float(np.mean(Y[:, 1] < Y[:, 0]))
    meta = {"tiles": len(specs), "workload": w.name, "seed": w.seed, "variants": list(variants),
            "label": "log device ms of the tile reconstructed alone", "epochs": args.epochs,
            "final_loss": losses[-1], "first_loss": losses[0], "label_seconds": round(t1 - t0, 1),
            "train_seconds": round(t2 - t1, 1), "fraction_b_faster": pick_b}
    save(args.out, theta, norm, variants, meta)
    np.savez_compressed(os.path.splitext(args.out)[0] + "_data.npz", X=X, Y=Y)
    rc.recon_free(ctx)
    print(json.dumps(meta))


if __name__ == "__main__":
    main()
