"""Run one kernel of the library a few times on the standard 1080p workload,
for profilers (ncu) and quick timing:

  python -m paper_2406_17782_gb300.profile_case reference [--spp 16] [--reps 3]
  python -m paper_2406_17782_gb300.profile_case decoder [--precision fp16] [--reps 3]
  python -m paper_2406_17782_gb300.profile_case train [--batch 65536] [--train-precision fp32|bf16] [--reps 3]
  python -m paper_2406_17782_gb300.profile_case error [--elements 33554432] [--reps 3]
  python -m paper_2406_17782_gb300.profile_case batched [--precision fp16] [--reps 3]
  python -m paper_2406_17782_gb300.profile_case paper [--width 128] [--precision fp16] [--reps 3]
  python -m paper_2406_17782_gb300.profile_case paper-train [--width 128] [--batch 65536] [--reps 3]
  python -m paper_2406_17782_gb300.profile_case reference --spp 16 --visibility

The workload is the 1920 x 1080 G-buffer of eight weave materials (random-init
networks); the training case uses a batch of queries over 256 training
materials with targets from the reference kernel at 4 x 4 samples; the error
case reduces two arrays of uniform random floats (2^25 elements each by
default, 268 MB together: more than L2); the batched case shades the 4K
view plus 256 ragged segments through one plan (one launch per call); the
paper cases run the paper's decoder structure (random-init, width 64 or
128) on the 1080p G-buffer, or its FP32 training step.  Prints the
mean time per launch (CUDA events) as one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

from .api import Fabric, GBuffer  # noqa: E402


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["reference", "decoder", "train", "error", "batched", "paper", "paper-train"])
    ap.add_argument("--width", type=int, default=128, choices=[64, 128])
    ap.add_argument("--spp", type=int, default=16, help="samples per axis (reference)")
    ap.add_argument("--precision", default="fp16")
    ap.add_argument("--batch", type=int, default=65536)
    ap.add_argument("--train-precision", default="fp32", choices=["fp32", "bf16"])
    ap.add_argument("--elements", type=int, default=1 << 25, help="array length (error)")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--visibility", action="store_true", help="the reference with the proposed visibility model")
    args = ap.parse_args(argv)
    fab = Fabric(0)
    mats = W.frame_materials()
    fab.set_materials(mats)
    fab.set_params(W.decoder_init(), W.encoder_init())
    if args.case == "batched":
        segs_host, n_b = W.batched_4k()
        keep = []
        for h in segs_host:
            g = GBuffer.from_numpy(h)
            keep.append((g, torch.empty((g.n, 3), dtype=torch.float32, device=fab.device), None))
        fab.prepare_neural(fab.encode_params(mats), args.precision)
        plan = fab.plan(keep)
        fn = lambda: plan.shade(args.precision)
        points = n_b
    elif args.case == "error":
        ea = torch.rand(args.elements, device=fab.device)
        eb = torch.rand(args.elements, device=fab.device)
        out = torch.empty(3, dtype=torch.float64, device=fab.device)
        fn = lambda: fab.error_stats(ea, eb, out=out)
        points = args.elements
    elif args.case in ("paper", "paper-train"):
        fab.paper_set_params(args.width, W.paper_decoder_init(args.width), W.paper_encoder_init())
        if args.case == "paper":
            g = GBuffer.from_numpy(W.frame_gbuffer())
            rgb = torch.empty((g.n, 3), dtype=torch.float32, device=fab.device)
            fab.paper_prepare(fab.paper_encode_params(mats), args.precision)
            fn = lambda: fab.paper_shade_prepared(g, args.precision, out_rgb=rgb)
        else:
            tm = W.training_materials(32)
            q = W.training_queries(args.batch, len(tm), stream="profile-train")
            g = GBuffer.from_numpy(q)
            target = torch.empty((args.batch, 4), dtype=torch.float32, device=fab.device)
            fab.set_materials(tm)
            fab.shade_reference(g, 4, 4, 3, out_comps=target)
            fab.set_train_materials(tm)
            fn = lambda: fab.paper_train_step(g, target, 1e-3)
        points = g.n
    elif args.case == "train":
        tm = W.training_materials(32)
        q = W.training_queries(args.batch, len(tm), stream="profile-train")
        g = GBuffer.from_numpy(q)
        target = torch.empty((args.batch, 4), dtype=torch.float32, device=fab.device)
        fab.set_materials(tm)
        fab.shade_reference(g, 4, 4, 3, out_comps=target)
        fab.set_train_materials(tm)
        fab.set_train_precision(args.train_precision)
        fn = lambda: fab.train_step(g, target, 1e-3)
        points = g.n
    else:
        g = GBuffer.from_numpy(W.frame_gbuffer())
        rgb = torch.empty((g.n, 3), dtype=torch.float32, device=fab.device)
        if args.case == "reference":
            fab.set_visibility(args.visibility)
            fn = lambda: fab.shade_reference(g, args.spp, args.spp, 11, out_rgb=rgb)
        else:
            fab.prepare_neural(fab.encode_params(mats), args.precision)
            fn = lambda: fab.shade_neural_prepared(g, args.precision, out_rgb=rgb)
        points = g.n
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    fab.sync_status()
    print(json.dumps({"case": args.case, "ms_per_launch": e0.elapsed_time(e1) / args.reps, "reps": args.reps,
                      "points": points}))


if __name__ == "__main__":
    main()
