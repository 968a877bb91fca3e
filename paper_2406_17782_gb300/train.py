"""Train the encoder and decoder on data generated by the reference kernel
(Sec. 5.1-5.2), then measure the neural frame's error.

  python -m paper_2406_17782_gb300.train --out weights.ckpt [--queries 16777216 --steps 40000]

Data: `--queries` training queries over 32 parameter sets x 8 weaves (256
materials), half frame-like and half drawn from the paper's Table 2; targets
are the four components of the reference integral at 64 x 32 = 2048 samples
(the paper's data sample count).  Training: Adam, batch 65536, learning rate
1e-3 decayed by cosine to 1e-5, all in the library's kernels
(fabric_train_step); the dataset is shuffled once per epoch and batches are
contiguous slices of it.  Initial weights U(+-1/sqrt(fan_in)); loss Eq. 11
(--loss eq11) or, by default, its rendered-space option.  Evaluation: RMSE
of the 1920 x 1080 frame of eight weaves as lit by a unit directional light
(f_P <wi.n_s> per RGB channel) against the reference integral at 32 x 32 =
1024 samples (independent seed).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

from .api import Fabric, GBuffer  # noqa: E402


def generate_dataset(fab: Fabric, mats, n_queries: int, spp=(64, 32), seed: int = 0xDA7A, chunk: int = 1 << 22,
                     frame_share: float = 0.0):
    """Queries (device G-buffer) and target components [n, 4] from the
    reference kernel over the training material table.  A share
    `frame_share` of the queries uses only the first parameter set (the
    frame's eight materials, indices 0..7)."""
    n_frame = int(n_queries * frame_share)
    q = W.training_queries(n_queries - n_frame, len(mats), stream="train-data")
    if n_frame:
        qf = W.training_queries(n_frame, W.N_PATTERNS, stream="train-data-frame")
        q = {k: np.concatenate([q[k], qf[k]]) for k in q}
    g = GBuffer.from_numpy(q)
    fab.set_materials(mats)
    target = torch.empty((n_queries, 4), dtype=torch.float32, device=fab.device)
    rgb = torch.empty((min(chunk, n_queries), 3), dtype=torch.float32, device=fab.device)
    for s in range(0, n_queries, chunk):
        e = min(n_queries, s + chunk)
        sub = GBuffer(*(getattr(g, k)[s:e] for k in ("u", "v", "radius", "wi", "wo", "material")))
        fab.shade_reference(sub, spp[0], spp[1], seed + s, out_rgb=rgb[: e - s], out_comps=target[s:e])
    fab.sync_status()
    return g, target


def epoch_seed(seed: int, epoch: int) -> int:
    """The permutation seed of one epoch's shuffle."""
    return (seed << 32) + epoch


def train(fab: Fabric, mats, g: GBuffer, target: torch.Tensor, steps: int, batch: int = 65536,
          lr0: float = 1e-3, lr1: float = 1e-5, log_every: int = 1000, seed: int = 1, verbose: bool = True,
          paper: bool = False):
    """Adam with a cosine-decayed learning rate over shuffled epochs of the
    dataset; `paper` trains the paper's decoder structure
    (fabric_paper_train_step) instead of the workload's network."""
    step_fn = fab.paper_train_step if paper else fab.train_step
    fab.set_train_materials(mats)
    per_epoch = g.n // batch
    if per_epoch < 1:
        raise ValueError(f"the dataset ({g.n} points) is smaller than one batch ({batch})")
    losses = []
    t0 = time.time()
    # each epoch a shuffled copy of the dataset (fabric_shuffle_dataset),
    # written over the previous epoch's in stream order
    gs, ts = fab.shuffle_dataset(g, target, epoch_seed(seed, 0))
    if not paper:
        # one native call per epoch (fabric_train_steps: the same steps,
        # learning rates and results as the per-step loop below)
        all_loss = torch.empty(max(1, steps), dtype=torch.float64, device=fab.device)
        step = 0
        while step < steps:
            if step > 0:
                gs, ts = fab.shuffle_dataset(g, target, epoch_seed(seed, step // per_epoch), out=(gs, ts))
            n = min(per_epoch, steps - step)
            fab.train_steps(gs, ts, batch, n, step, max(1, steps), lr0, lr1, loss_out=all_loss[step:step + n])
            for m in range((step // log_every + 1) * log_every, step + n + 1, log_every):
                mean = float(all_loss[m - log_every:m].mean().item())
                losses.append((m, mean))
                if verbose:
                    lr = lr1 + 0.5 * (lr0 - lr1) * (1.0 + math.cos(math.pi * (m - 1) / max(1, steps)))
                    print(f"step {m:7d}  loss {mean:.5f}  lr {lr:.2e}  {time.time() - t0:6.1f}s", flush=True)
            step += n
        fab.sync_status()
        return losses
    loss_buf = torch.empty(log_every, dtype=torch.float64, device=fab.device)
    for step in range(steps):
        k = step % per_epoch
        if k == 0 and step > 0:
            gs, ts = fab.shuffle_dataset(g, target, epoch_seed(seed, step // per_epoch), out=(gs, ts))
        sl = slice(k * batch, (k + 1) * batch)
        bg = GBuffer(*(getattr(gs, f)[sl] for f in ("u", "v", "radius", "wi", "wo", "material")))
        lr = lr1 + 0.5 * (lr0 - lr1) * (1.0 + math.cos(math.pi * step / max(1, steps)))
        step_fn(bg, ts[sl], lr, loss_out=loss_buf[step % log_every])
        if (step + 1) % log_every == 0:
            mean = float(loss_buf.mean().item())
            losses.append((step + 1, mean))
            if verbose:
                print(f"step {step + 1:7d}  loss {mean:.5f}  lr {lr:.2e}  {time.time() - t0:6.1f}s", flush=True)
    fab.sync_status()
    return losses


def _errors(fab, a, gt, g):
    """Frame errors of `a` against `gt` ([n, 3] RGB): `rmse_fp` / `rel_l2_fp`
    on the linear f_P values, unclamped, over all pixels and channels;
    `rmse_tm` on the tone-mapped x / (1 + x); `rmse` / `rel_l2` on the frame
    lit by a unit directional light along wi (f_P <wi . n_s>)."""
    n = gt.numel()
    raw = fab.error_stats(a, gt).cpu().numpy()
    tm = fab.error_stats(a / (1.0 + a), gt / (1.0 + gt)).cpu().numpy()
    lit = fab.error_stats(a, gt, weights=g.wi[:, 2], group=3, weight_stride=3).cpu().numpy()
    return {"rmse": math.sqrt(lit[0] / n), "rel_l2": math.sqrt(lit[0] / lit[1]),
            "rmse_fp": math.sqrt(raw[0] / n), "rel_l2_fp": math.sqrt(raw[0] / raw[1]), "max_abs_fp": float(raw[2]),
            "rmse_tm": math.sqrt(tm[0] / n)}


def frame_rmse(fab: Fabric, precision: str = "fp16", gt_spp=(32, 32), ref_spps=(1, 2, 4, 8, 16), gbuf=None,
               paper: bool = False, paper_fp32: bool = False):
    """Error of the neural 1080p frame, and of the reference at lower sample
    counts, against the reference at gt_spp (see _errors for the metrics;
    the paper's results are direct-lit renders, Sec. 6, the scope's metric is
    the linear f_P).  The ground truth's own Monte Carlo noise is estimated
    from a second, independent ground-truth frame: `gt_noise_*` is its RMS
    deviation from the integral (half the mean squared difference of the
    two, per metric).  `gbuf`: a host G-buffer of the frame's materials
    (default: the 1080p frame); `paper`: shade with the paper's decoder
    structure instead of the workload's network (on tensor cores at
    `precision`, or in FP32 with `paper_fp32`, which runs every ablation)."""
    mats = W.frame_materials()
    fab.set_materials(mats)
    g = GBuffer.from_numpy(W.frame_gbuffer() if gbuf is None else gbuf)
    gt, _ = fab.shade_reference(g, gt_spp[0], gt_spp[1], 0x6721)
    out = {}
    if paper and paper_fp32:
        nrgb, _ = fab.paper_shade_fp32(g, fab.paper_encode_params(mats))
    elif paper:
        nrgb, _ = fab.paper_shade_neural(g, fab.paper_encode_params(mats), precision)
    else:
        nrgb, _ = fab.shade_neural(g, fab.encode_params(mats), precision)
    out["neural"] = _errors(fab, nrgb, gt, g)
    for s in ref_spps:
        r, _ = fab.shade_reference(g, s, s, 0x1234)
        out[f"reference_{s * s}spp"] = _errors(fab, r, gt, g)
    gt2, _ = fab.shade_reference(g, gt_spp[0], gt_spp[1], 0x9E37)
    two = _errors(fab, gt2, gt, g)
    out["gt_noise_fp"] = two["rmse_fp"] / math.sqrt(2.0)
    out["gt_noise"] = two["rmse"] / math.sqrt(2.0)
    lit = fab.error_stats(gt, torch.zeros_like(gt), weights=g.wi[:, 2], group=3, weight_stride=3).cpu().numpy()
    out["gt_rms"] = math.sqrt(float(lit[0]) / gt.numel())      # sum (gt w)^2 over the frame
    raw = fab.error_stats(gt, torch.zeros_like(gt)).cpu().numpy()
    out["gt_rms_fp"] = math.sqrt(float(raw[0]) / gt.numel())
    fab.sync_status()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--queries", type=int, default=1 << 24)
    ap.add_argument("--steps", type=int, default=40000)
    ap.add_argument("--batch", type=int, default=65536)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--spp", type=int, nargs=2, default=[64, 32])
    ap.add_argument("--frame-share", type=float, default=0.5)
    ap.add_argument("--report", default=None)
    ap.add_argument("--loss", default="rendered", choices=["eq11", "rendered"])
    args = ap.parse_args(argv)
    fab = Fabric(0)
    fab.set_params(W.decoder_init(weight_bound="small"), W.encoder_init(weight_bound="small"))
    fab.set_train_loss(args.loss)
    mats = W.training_materials(32)
    t = time.time()
    g, target = generate_dataset(fab, mats, args.queries, tuple(args.spp), frame_share=args.frame_share)
    torch.cuda.synchronize()
    t_data = time.time() - t
    print(f"data: {args.queries} queries x {args.spp[0] * args.spp[1]} spp in {t_data:.2f}s", flush=True)
    t = time.time()
    losses = train(fab, mats, g, target, args.steps, args.batch, args.lr)
    torch.cuda.synchronize()
    t_train = time.time() - t
    fab.checkpoint_save(args.out)
    rm = frame_rmse(fab)
    report = {"queries": args.queries, "data_spp": args.spp[0] * args.spp[1], "data_seconds": t_data,
              "steps": args.steps, "batch": args.batch, "lr": args.lr, "frame_share": args.frame_share,
              "train_seconds": t_train, "losses": losses, "rmse": rm}
    print(json.dumps(rm, indent=1))
    if args.report:
        json.dump(report, open(args.report, "w"), indent=1)


if __name__ == "__main__":
    main()
