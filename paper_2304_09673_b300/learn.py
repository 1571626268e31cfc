"""Learned relaxation factor: dataset recording, training and weights I/O.

The network (6 -> 32 -> 32 -> 1, see include/st.h "learned relaxation
factor") is trained on step records of the plain synchronized tracer
(st_trace_record) over seeded synthetic scenes, with the library's own FP32
gradient kernel (st_mlp_grad) and Adam update (st_mlp_adam).  Inference in
the tracer uses the BF16 tensor-core path (ST_STEP_LEARNED).

    python -m paper_2304_09673_b300.learn --out paper_2304_09673_b300/weights/relax_mlp.npz
"""
from __future__ import annotations

import argparse
import json
import math
import time
from pathlib import Path

import numpy as np

from . import scenegen as sg
from . import st

WEIGHTS = Path(__file__).resolve().parent / "weights" / "relax_mlp.npz"
TRAIN_SEEDS = range(10000, 10200)     # 200 training scenes
TEST_SEEDS = range(20000, 20010)      # held-out scenes


def init_params(seed: int = 0) -> np.ndarray:
    """He-style random initialisation of the FP32 parameter vector."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(scale=math.sqrt(2.0 / 6), size=(32, 6))
    W2 = rng.normal(scale=math.sqrt(2.0 / 32), size=(32, 32))
    w3 = rng.normal(scale=math.sqrt(1.0 / 32), size=32)
    return np.concatenate([W1.ravel(), np.zeros(32), W2.ravel(), np.zeros(32), w3, [0.0]]).astype(np.float32)


def training_scene(seed: int):
    """One training scene: N uniform in [1000, 4000], depth <= min(20, ceil(log2 N) + 4)."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1000, 4001))
    depth = min(20, math.ceil(math.log2(n)) + 4)
    return sg.make_scene(n, depth, seed)


def record(scenes, cam, opts, ray_stride: int = 331, cap_per_scene: int = 200000, tile: int = 16):
    """Step records (float32 [n, 8]) of the plain tracer over the scenes."""
    import torch
    out = []
    W, H = cam.width, cam.height
    dev = torch.device("cuda")
    depth = torch.empty(H * W, dtype=torch.float32, device=dev)
    normal = torch.empty(H * W * 3, dtype=torch.float32, device=dev)
    evals = torch.empty(H * W, dtype=torch.int32, device=dev)
    flags = torch.empty(H * W, dtype=torch.uint8, device=dev)
    recs = torch.empty(cap_per_scene * 8, dtype=torch.float32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    for scene in scenes:
        h = st.st_scene_create(scene)
        try:
            tiles = st.st_build_tiles(h, cam, tile)
            cnt.zero_()
            st.st_trace_record(h, cam, tiles, opts, depth, normal, evals, flags, recs, cnt, ray_stride)
            n = min(int(cnt.item()), cap_per_scene)
            out.append(recs[: n * 8].view(n, 8).cpu().numpy().copy())
        finally:
            st.st_scene_destroy(h)
    return np.concatenate(out) if out else np.zeros((0, 8), np.float32)


def train(records: np.ndarray, epochs: int = 12, batch: int = 65536, lr: float = 3e-3, seed: int = 0,
          val_frac: float = 0.05, log=print, tensor_cores: bool = True):
    """Adam on the asymmetric squared error; returns (params, history).
    Gradients from the BF16 tensor-core kernel (st_mlp_grad_bf16) unless
    tensor_cores is False (the FP32 kernel, st_mlp_grad)."""
    grad_fn = st.st_mlp_grad_bf16 if tensor_cores else st.st_mlp_grad
    import torch
    dev = torch.device("cuda")
    rng = np.random.default_rng(seed)
    perm = rng.permutation(len(records))
    n_val = max(1, int(val_frac * len(records)))
    val, tr = records[perm[:n_val]], records[perm[n_val:]]
    Xt = torch.tensor(tr[:, :6], device=dev)
    yt = torch.tensor(tr[:, 6], device=dev)
    Xv = torch.tensor(val[:, :6], device=dev)
    yv = torch.tensor(val[:, 6], device=dev)
    params = torch.tensor(init_params(seed), device=dev)
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    grad = torch.zeros_like(params)
    loss = torch.zeros(1, device=dev)
    step = 0
    hist = []
    n = Xt.shape[0]
    n_batches = max(1, n // batch)
    total_steps = epochs * n_batches
    for ep in range(epochs):
        order = torch.randperm(n, device=dev)
        tl = 0.0
        for b in range(n_batches):
            idx = order[b * batch:(b + 1) * batch]
            xb = Xt[idx].contiguous()
            yb = yt[idx].contiguous()
            grad.zero_()
            loss.zero_()
            grad_fn(params, xb, yb, grad, loss)
            step += 1
            cur_lr = lr * 0.5 * (1 + math.cos(math.pi * step / total_steps))
            st.st_mlp_adam(params, grad, m, v, step, cur_lr, grad_scale=1.0 / len(idx))
            tl += float(loss.item()) / len(idx)
        grad.zero_()
        loss.zero_()
        grad_fn(params, Xv, yv, grad, loss)
        vl = float(loss.item()) / Xv.shape[0]
        hist.append(dict(epoch=ep, train_loss=tl / n_batches, val_loss=vl))
        log(f"epoch {ep}: train {tl / n_batches:.5f} val {vl:.5f}")
    return params.cpu().numpy(), hist


def save(params: np.ndarray, path: Path, meta: dict) -> None:
    path = Path(path)
    path.parent.mkdir(parents=True, exist_ok=True)
    np.savez(path, params=np.asarray(params, np.float32), version=np.array([1]))
    path.with_suffix(".json").write_text(json.dumps(meta, indent=1, sort_keys=True))


def load(path: Path = WEIGHTS) -> np.ndarray:
    d = np.load(path)
    p = np.asarray(d["params"], np.float32)
    if p.size != st.MLP_PARAMS:
        raise ValueError("weights file has %d parameters" % p.size)
    return p


def packed_device(params: np.ndarray):
    """Packed BF16 weights as a CUDA uint8 tensor (for st_trace_opts.mlp)."""
    import torch
    return torch.tensor(st.st_mlp_pack(params), device="cuda")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=str(WEIGHTS))
    ap.add_argument("--scenes", type=int, default=200)
    ap.add_argument("--stride", type=int, default=331)
    ap.add_argument("--epochs", type=int, default=12)
    ap.add_argument("--max-new", type=int, default=24)
    ap.add_argument("--width", type=int, default=1920)
    ap.add_argument("--height", type=int, default=1080)
    args = ap.parse_args()
    import torch
    torch.cuda.set_device(0)
    cam = sg.default_camera(args.width, args.height)
    opts = st.make_opts(max_new_per_turn=args.max_new)
    t0 = time.time()
    seeds = list(TRAIN_SEEDS)[: args.scenes]
    recs = []
    for i in range(0, len(seeds), 20):
        recs.append(record([training_scene(s) for s in seeds[i:i + 20]], cam, opts, args.stride))
        print(f"recorded {sum(len(r) for r in recs)} records from {min(i + 20, len(seeds))} scenes "
              f"({time.time() - t0:.1f} s)", flush=True)
    records = np.concatenate(recs)
    t1 = time.time()
    params, hist = train(records, epochs=args.epochs)
    meta = dict(records=int(len(records)), scenes=len(seeds), seeds=[seeds[0], seeds[-1]], stride=args.stride,
                resolution=[args.width, args.height], max_new_per_turn=args.max_new,
                label_mean=float(records[:, 6].mean()), history=hist, record_seconds=t1 - t0,
                train_seconds=time.time() - t1)
    save(params, Path(args.out), meta)
    print(json.dumps(dict(out=args.out, records=len(records), final=hist[-1])))


if __name__ == "__main__":
    main()
