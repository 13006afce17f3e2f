"""Training and use of the learned cost model (the scheduler's analogue of the
paper's performance-aware task scheduling, Sec. IV: per-task cost estimates
decide how and in which order tasks run).

Pipeline (every step on the GPU goes through the C ABI):
  1. tiles from the seeded generator (the uneven-size law: H, W in
     {256..4096 step 256}, blob density uniform in [0, 1/1000], radius 3..20,
     h-dome / fill-holes markers 50/50, 8-connectivity);
  2. labels measured by the method itself: each tile reconstructed alone with
     variant A (scan pairs to stability, no queue) and variant B (k scan pairs
     then the queue); the label is the log of the work the kernel reports for
     the tile -- the summed time CTAs spent on its blocks -- because inside a
     batch the tiles share the GPU, so work, not a tile's latency alone,
     decides the makespan;
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


CKPT_MAGIC = b"RCK1"


def save_checkpoint(path: str, theta: np.ndarray, adam_mv: np.ndarray, state: dict) -> None:
    """Training checkpoint: magic, header length, a JSON header (state: step,
    epoch, norm, seed, lr, batch, variants, ...), then theta and Adam's two
    moment vectors as flat fp32. Written to a temporary file, then renamed."""
    head = json.dumps(state).encode()
    tmp = path + ".tmp"
    with open(tmp, "wb") as f:
        f.write(CKPT_MAGIC)
        f.write(struct.pack("<i", len(head)))
        f.write(head)
        f.write(np.asarray(theta, np.float32).tobytes())
        f.write(np.asarray(adam_mv, np.float32).tobytes())
    os.replace(tmp, path)


def load_checkpoint(path: str):
    """Returns (theta, adam_mv, state) of a checkpoint written by save_checkpoint."""
    n = rc.RECON_MLP_NPARAMS
    with open(path, "rb") as f:
        if f.read(4) != CKPT_MAGIC:
            raise ValueError("not a cost-model training checkpoint: " + path)
        (nh,) = struct.unpack("<i", f.read(4))
        state = json.loads(f.read(nh).decode())
        theta = np.frombuffer(f.read(4 * n), np.float32).copy()
        mv = np.frombuffer(f.read(8 * n), np.float32).copy()
    if theta.size != n or mv.size != 2 * n:
        raise ValueError("truncated checkpoint: " + path)
    return theta, mv, state


def train_resumable(ctx, X: np.ndarray, Y: np.ndarray, epochs=200, batch=256, lr=2e-3, seed=0,
                    checkpoint: str = None, every: int = 50, resume: str = None):
    """GPU training with checkpoints every `every` epochs (and at the end) to
    `checkpoint`; `resume` continues from a checkpoint (its theta, Adam state,
    step, epoch and output normalisation). Returns (theta, norm, losses of the
    epochs run here)."""
    import torch
    if resume:
        theta, mv, state = load_checkpoint(resume)
        norm, step, epoch0 = state["norm"], state["step"], state["epoch"]
        seed, lr, batch = state["seed"], state["lr"], state["batch"]
    else:
        mean, std = Y.mean(axis=0), Y.std(axis=0) + 1e-6
        norm = [float(mean[0]), float(std[0]), float(mean[1]), float(std[1])]
        theta = init_params(np.random.default_rng(seed))
        mv = np.zeros(2 * rc.RECON_MLP_NPARAMS, np.float32)
        step, epoch0 = 0, 0
    T = (Y - np.array([norm[0], norm[2]])) / np.array([norm[1], norm[3]])
    dth = torch.from_numpy(np.ascontiguousarray(theta)).cuda()
    dmv = torch.from_numpy(np.ascontiguousarray(mv)).cuda()
    dX = torch.from_numpy(X.astype(np.float32)).cuda()
    dT = torch.from_numpy(T.astype(np.float32)).cuda()
    torch.cuda.synchronize()
    losses = []
    epoch = epoch0
    while epoch < epochs:
        k = min(every if every > 0 else epochs, epochs - epoch)
        st, step, ls = rc.recon_mlp_train_resume(ctx, dth.data_ptr(), dmv.data_ptr(), step, epoch, dX.data_ptr(),
                                                 dT.data_ptr(), len(X), k, batch, lr, seed)
        rc.check(st, "recon_mlp_train_resume")
        epoch += k
        losses += ls
        if checkpoint:
            save_checkpoint(checkpoint, dth.cpu().numpy(), dmv.cpu().numpy(),
                            {"step": step, "epoch": epoch, "epochs": epochs, "norm": norm, "seed": seed,
                             "lr": lr, "batch": batch, "samples": int(len(X))})
    return dth.cpu().numpy(), norm, losses


def install(ctx, path: str = MODEL_PATH) -> dict:
    theta, norm, (va, vb), meta = load(path)
    rc.check(rc.recon_sched_set_model(ctx, theta, norm, va, vb), "recon_sched_set_model")
    return meta


class Arena:
    """Pinned host and device buffers reused across chunks of tiles."""

    def __init__(self, torch, dev, max_px):
        self.h = torch.empty(2 * max_px, dtype=torch.uint8).pin_memory()
        self.d = torch.empty(3 * max_px, dtype=torch.uint8, device=dev)
        self.max_px = max_px


def label_chunk(ctx, specs, seed, variants, torch, arena):
    """Features and per-variant log device times of one chunk of tiles, each
    tile reconstructed alone (J restored from its pristine copy every run)."""
    import synth
    n = len(specs)
    px = [s.H * s.W for s in specs]
    off = np.concatenate([[0], np.cumsum(px)]).astype(np.int64)
    tot = int(off[-1])
    assert tot <= arena.max_px
    hI, hJ = arena.h[:tot], arena.h[tot:2 * tot]
    synth.generate_into(specs, seed, [hI.data_ptr() + int(o) for o in off[:-1]],
                        [hJ.data_ptr() + int(o) for o in off[:-1]])
    dI, dJ0, dJ = arena.d[:tot], arena.d[tot:2 * tot], arena.d[2 * tot:3 * tot]
    dI.copy_(hI, non_blocking=True)
    dJ0.copy_(hJ, non_blocking=True)
    dJ.copy_(dJ0)
    torch.cuda.synchronize()
    tiles = [(dI.data_ptr() + int(off[t]), dJ.data_ptr() + int(off[t]), s.H, s.W, s.W, s.conn)
             for t, s in enumerate(specs)]
    feat = torch.zeros((n, rc.RECON_NFEAT), dtype=torch.float32, device=dI.device)
    rc.check(rc.recon_features(ctx, tiles, feat.data_ptr()), "recon_features")
    work = np.zeros((n, len(variants)))
    ms = np.zeros((n, len(variants)))
    for t in range(n):
        a, b = int(off[t]), int(off[t + 1])
        for v, var in enumerate(variants):
            dJ[a:b].copy_(dJ0[a:b])
            torch.cuda.synchronize()
            rc.check(rc.recon_batch_ex(ctx, [tiles[t]], [var], None), "label run")
            ms[t, v] = rc.recon_last_kernel_ms(ctx)
            work[t, v] = rc.recon_get_work(ctx, 1)[0]["busy_ns"] * 1e-6   # CTA-milliseconds
    return feat.cpu().numpy(), np.log(np.maximum(work, 1e-4)), np.log(np.maximum(ms, 1e-4))


def build_dataset(ctx, specs, seed, variants, chunk_px=1 << 30):
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    arena = Arena(torch, dev, max(chunk_px, max(s.H * s.W for s in specs)))
    X, Y, Yms = [], [], []
    i = 0
    while i < len(specs):
        j, acc = i, 0
        while j < len(specs) and acc + specs[j].H * specs[j].W <= arena.max_px:
            acc += specs[j].H * specs[j].W
            j += 1
        f, y, yms = label_chunk(ctx, specs[i:j], seed, variants, torch, arena)
        X.append(f)
        Y.append(y)
        Yms.append(yms)
        i = j
    return np.concatenate(X), np.concatenate(Y), np.concatenate(Yms)


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


def evaluate(ctx, model_path, workload="eval1000", reps=3):
    """Learned vs plain schedule on one batch: device time of the persistent
    launch, and byte equality of the two outputs."""
    import torch
    import synth
    w = synth.workload(workload)
    specs = list(w.tiles)
    tot = sum(s.H * s.W for s in specs)
    dev = torch.device("cuda", torch.cuda.current_device())
    hI = torch.empty(tot, dtype=torch.uint8).pin_memory()
    hJ = torch.empty(tot, dtype=torch.uint8).pin_memory()
    off = np.concatenate([[0], np.cumsum([s.H * s.W for s in specs])]).astype(np.int64)
    synth.generate_into(specs, w.seed, [hI.data_ptr() + int(o) for o in off[:-1]],
                        [hJ.data_ptr() + int(o) for o in off[:-1]])
    dI = hI.to(dev)
    dJ0 = hJ.to(dev)
    dJ = dJ0.clone()
    torch.cuda.synchronize()
    tiles = [(dI.data_ptr() + int(off[t]), dJ.data_ptr() + int(off[t]), s.H, s.W, s.W, s.conn)
             for t, s in enumerate(specs)]
    install(ctx, model_path)
    st, var, order, pred = rc.recon_sched_plan_batch(ctx, tiles)
    rc.check(st, "plan")

    def timed(fn):
        out = []
        for r in range(reps + 1):
            dJ.copy_(dJ0)
            torch.cuda.synchronize()
            fn()
            rc.check(rc.recon_sync(ctx), "sync")
            if r:
                out.append(rc.recon_last_kernel_ms(ctx))
        return float(np.median(out))

    ms_plain = timed(lambda: rc.check(rc.recon_batch(ctx, tiles), "plain"))
    R_plain = dJ.clone()
    ms_learned = timed(lambda: rc.check(rc.recon_batch_ex(ctx, tiles, var, order), "learned"))
    same = bool(torch.equal(R_plain, dJ))
    return {"workload": workload, "tiles": len(specs), "pixels": tot, "plain_ms": ms_plain,
            "learned_ms": ms_learned, "plain_mpix_s": tot / ms_plain / 1e3, "learned_mpix_s": tot / ms_learned / 1e3,
            "gain": ms_plain / ms_learned, "outputs_identical": same,
            "variant_a_fraction": float(np.mean(np.array(var) != load(model_path)[2][1]))}


def main():
    import argparse
    import torch
    import synth
    ap = argparse.ArgumentParser(description="train the learned cost model")
    ap.add_argument("--tiles", type=int, default=20000)
    ap.add_argument("--epochs", type=int, default=200)
    ap.add_argument("--out", default=MODEL_PATH)
    ap.add_argument("--queue-k", type=int, default=1)
    ap.add_argument("--scan-variant", type=int, default=1 + 256 * 32,
                    help="variant A: 1 scan pair, then keep scanning while a pair raises >= 2048 px")
    ap.add_argument("--eval", action="store_true", help="then compare learned vs plain on eval1000")
    ap.add_argument("--eval-only", action="store_true", help="only evaluate the model at --out")
    ap.add_argument("--data", help="reuse a labelled dataset (.npz written by an earlier run) instead of labelling")
    ap.add_argument("--checkpoint", help="write a training checkpoint here every --checkpoint-every epochs")
    ap.add_argument("--checkpoint-every", type=int, default=50)
    ap.add_argument("--resume", help="continue training from this checkpoint")
    args = ap.parse_args()
    w = synth.workload("train20k")
    specs = list(w.tiles[:args.tiles])
    ctx = rc.recon_init(0, 0, 0)
    if args.eval_only:
        print(json.dumps(evaluate(ctx, args.out)), flush=True)
        rc.recon_free(ctx)
        return
    variants = (args.scan_variant, args.queue_k)
    t0 = time.time()
    if args.data:
        d = np.load(args.data)
        X, Y, Yms = d["X"], d["Y"], d["Yms"]
    else:
        X, Y, Yms = build_dataset(ctx, specs, w.seed, variants)
    t1 = time.time()
    if args.checkpoint or args.resume:
        theta, norm, losses = train_resumable(ctx, X, Y, epochs=args.epochs, checkpoint=args.checkpoint,
                                              every=args.checkpoint_every, resume=args.resume)
    else:
        theta, norm, losses = train(ctx, X, Y, epochs=args.epochs)
    t2 = time.time()
    pick_b = float(np.mean(Y[:, 1] < Y[:, 0]))
    meta = {"tiles": len(specs), "workload": w.name, "seed": w.seed, "variants": list(variants),
            "label": "log CTA-busy milliseconds (work) of the tile reconstructed alone", "epochs": args.epochs,
            "final_loss": losses[-1] if losses else None, "first_loss": losses[0] if losses else None,
            "label_seconds": round(t1 - t0, 1),
            "train_seconds": round(t2 - t1, 1), "fraction_b_faster": pick_b}
    save(args.out, theta, norm, variants, meta)
    if not args.data:
        np.savez_compressed(os.path.splitext(args.out)[0] + "_data.npz", X=X, Y=Y, Yms=Yms)
    print(json.dumps(meta), flush=True)
    if args.eval:
        print(json.dumps(evaluate(ctx, args.out)), flush=True)
    rc.recon_free(ctx)


if __name__ == "__main__":
    main()
