"""Train the warm-start U-Net and write its weights.

Training data (generated by the method itself, nothing is read from disk):
template pools of the nested-label and blob families at 128^3, velocity pools
band-limited to |k| <= 6 with max |v| in [0.3, 1.2], N(0, 0.02^2) noise on
both images; every pair is the advection of a template by a velocity with the
library's SL transport.  100 templates x 200 velocities give 20,000 distinct
pairs; 5,000 Adam steps of batch 4 draw 20,000 of them.  The loss is the
velocity misfit plus the transport mismatch, whose gradient comes from the
hand-written SL adjoint (see warmstart.train).

    python -m paper_2209_08189_gb300.train_warmstart --out paper_2209_08189_gb300/weights/unet_warmstart_128.npz

With --pc-head the network also predicts the coarse preconditioner weight
(a fourth output channel, see warmstart.train; --pc-target scale: the
per-pair constant of warmstart.pc_scale_target, fit: the least-squares fit
of the data term): starting from --init (the velocity network's weights; the
new head row starts at w = 1), the velocity loss and wpc times the weight
loss are trained together on pairs drawn the same way:

    python -m paper_2209_08189_gb300.train_warmstart --pc-head --steps 1500 \
        --init paper_2209_08189_gb300/weights/unet_warmstart_128.npz \
        --out paper_2209_08189_gb300/weights/unet_warmstart_pc_128.npz

Prints one JSON line with the training record.  Needs a CUDA GPU.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DEFAULT_OUT = os.path.join(ROOT, "paper_2209_08189_gb300", "weights", "unet_warmstart_128.npz")


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_OUT)
    ap.add_argument("--n", type=int, default=128, help="training grid points per axis")
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--templates", type=int, default=100)
    ap.add_argument("--velocities", type=int, default=200)
    ap.add_argument("--kmax", type=int, default=6)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--pc-head", action="store_true", help="also learn the coarse preconditioner weight")
    ap.add_argument("--wpc", type=float, default=1.0, help="weight of the preconditioner-weight fit loss")
    ap.add_argument("--pc-probes", type=int, default=2, help="probe fields per sample and step (--pc-target fit)")
    ap.add_argument("--pc-target", default="scale", choices=["scale", "fit"],
                    help="target of the preconditioner weight (see warmstart.train)")
    ap.add_argument("--pc-grid", type=int, default=None,
                    help="grid of the scale target (--pc-target scale; default the training grid)")
    ap.add_argument("--init", default=None, help="start from these weights (a velocity-only file is extended)")
    args = ap.parse_args(argv)

    import torch
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import __graft_entry__ as entry
    entry.build()
    from paper_2209_08189_gb300 import net, warmstart
    if not torch.cuda.is_available():
        raise SystemExit("training needs a CUDA GPU")
    st = torch.cuda.current_stream().cuda_stream
    t0 = time.perf_counter()
    src = warmstart.PairSource(args.n, n_templates=args.templates, n_velocities=args.velocities,
                               kmax=(args.kmax, args.kmax), vmax=(0.3, 1.2), noise=0.02, seed=args.seed)
    t_pool = time.perf_counter() - t0
    u = net.UNet(seed=args.seed, stream=st, pc_head=args.pc_head)
    init_meta = None
    if args.init:
        init_meta, state = net.UNet.read_weights(args.init)
        if args.pc_head and not init_meta.get("pc_head", False):
            # keep the new head row (small weights, bias at softplus^-1(1))
            hw, hb = (x.cpu().numpy() for x in (u.p["head"]["w"], u.p["head"]["b"]))
            hw[:3], hb[:3] = state["head"]
            state["head"] = (hw, hb)
        u.load_state(state)
    t0 = time.perf_counter()
    hist = warmstart.train(u, src, steps=args.steps, batch=args.batch, lr=1e-3 if not args.init else 2e-4,
                           lr_final=1e-4 if not args.init else 2e-5, wv=1.0, wm=1.0,
                           log_every=max(1, args.steps // 20), wpc=args.wpc if args.pc_head else 0.0,
                           pc_probes=args.pc_probes, pc_target=args.pc_target, pc_grid=args.pc_grid)
    t_train = time.perf_counter() - t0
    src.ctx.close()
    record = {"grid": args.n, "steps": args.steps, "batch": args.batch, "pairs_drawn": args.steps * args.batch,
              "distinct_pairs": args.templates * args.velocities, "kmax": args.kmax, "vmax": [0.3, 1.2],
              "noise": 0.02, "params": u.num_params(), "pool_s": t_pool, "train_s": t_train,
              "pc_head": args.pc_head, "wpc": args.wpc if args.pc_head else 0.0,
              "pc_probes": args.pc_probes if args.pc_head else 0,
              "pc_target": args.pc_target if args.pc_head else None,
              "pc_grid": (args.pc_grid or args.n) if args.pc_head else None,
              "init": {"file": os.path.basename(args.init), "training": (init_meta or {}).get("training")}
              if args.init else None,
              "history": [{"step": h[0], "Lv": h[1], "mismatch_rel": h[2], "s": h[3], "Lpc": h[4]} for h in hist]}
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    u.save_weights(args.out, meta={"n_net": args.n, "training": {k: v for k, v in record.items()
                                                                 if k != "history"}})
    record["out"] = args.out
    record["bytes"] = os.path.getsize(args.out)
    print(json.dumps(record))


if __name__ == "__main__":
    main()
