"""Train the coarse propagator G to step the fine operator over one slice.

Sec. 3.2 asks for G(U_n; Theta) ~ F(t_n, t_{n+1}, U_n).  Trajectories come from
the library's own fine propagator; the loss is the m-step unrolled mean squared
error  sum_{j=1..m} mean |G^j(U_t) - U_{t+j}|^2  over random windows; gradients
come from cnn_backward (through the unrolled chain) and the update from
cnn_adam_step.  Every step of the arithmetic runs in the library's kernels; torch
only holds buffers and gathers batches.

    python -m paper_2510_07672_gb300.train --out weights.npz     # the 256^2 mass-conserving G
    python -m paper_2510_07672_gb300.train --workload large --out weights.npz
        # the 1 -> 64 x 8 G of the 1024^2 classic problem, trained on periodic
        # 128^2 crops with the same grid spacing h = 1/1024 (eps, dt and the
        # 500-step slice as in the large problem): the network is a local,
        # translation-invariant stencil of radius 8 cells, so it only sees the
        # discrete operator on h = 1/1024, whatever the domain size
"""
from __future__ import annotations

import argparse
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def make_trajectories(fp, ics, slices: int, steps: int):
    """U[r][0..slices] with U[r][j+1] = F(U[r][j]) (c = steps fine steps)."""
    import torch

    from . import abi
    R, n = ics.shape[0], ics.shape[-1]
    traj = torch.empty((R, slices + 1, n, n), dtype=torch.float32, device=ics.device)
    traj[:, 0] = ics
    cur = ics.contiguous().clone()
    nxt = torch.empty_like(cur)
    for j in range(slices):
        abi.ac_fine_propagate_slices(fp, steps, cur, nxt)
        traj[:, j + 1] = nxt
        cur, nxt = nxt, cur
    return traj


def train_coarse(net, traj, iters: int, batch: int, unroll: int, lr: float, seed: int = 0, log_every: int = 0,
                 lr_final: float | None = None, fine=None, perturb: float = 0.0):
    """Adam on the unrolled MSE.  Returns the list of per-iteration losses.

    With `fine` (FineParams and steps per slice) and perturb > 0, each window
    starts from a perturbed state U_t + delta instead, with targets produced by
    the fine propagator from that state: Parareal applies G to iterates that
    are off the fine trajectory, and its correction converges only as fast as
    G's response to such deviations matches F's.  delta mixes a slice increment
    of another trajectory (smooth, realistic spectrum) and white noise, with
    relative size up to `perturb`."""
    import numpy as np
    import torch

    from . import abi
    R, S1, n, _ = traj.shape
    S = S1 - 1
    dev = traj.device
    rng = np.random.default_rng(seed)
    ws = [net.new_workspace(n, batch) for _ in range(unroll)]
    xs = [torch.empty((batch, n, n), dtype=torch.float32, device=dev) for _ in range(unroll + 1)]
    tg = [torch.empty((batch, n, n), dtype=torch.float32, device=dev) for _ in range(unroll)]
    gbuf = [torch.empty((batch, n, n), dtype=torch.float32, device=dev) for _ in range(2)]
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    scratch = torch.empty(64, dtype=torch.float64, device=dev)
    scale = 1.0 / (batch * n * n * unroll)
    losses = []
    for it in range(iters):
        if lr_final is not None and iters > 1:
            cur_lr = lr * (lr_final / lr) ** (it / (iters - 1))
        else:
            cur_lr = lr
        r = torch.as_tensor(rng.integers(0, R, batch), device=dev)
        t = torch.as_tensor(rng.integers(0, S - unroll + 1, batch), device=dev)
        xs[0].copy_(traj[r, t])
        if fine is not None and perturb > 0:
            fp, steps = fine
            r2 = torch.as_tensor(rng.integers(0, R, batch), device=dev)
            t2 = torch.as_tensor(rng.integers(0, S, batch), device=dev)
            amp = torch.as_tensor(rng.uniform(0, perturb, (batch, 1, 1)), dtype=torch.float32, device=dev)
            rms = xs[0].pow(2).mean(dim=(1, 2), keepdim=True).sqrt()
            smooth = traj[r2, t2 + 1] - traj[r2, t2]
            smooth = smooth / smooth.pow(2).mean(dim=(1, 2), keepdim=True).sqrt().clamp_min(1e-12)
            white = torch.randn_like(xs[0])
            mix = torch.as_tensor(rng.uniform(0, 1, (batch, 1, 1)), dtype=torch.float32, device=dev)
            xs[0].add_(amp * rms * (mix * smooth + (1 - mix) * white))
            prev = xs[0]
            for j in range(unroll):
                abi.ac_fine_propagate_slices(fp, steps, prev, tg[j])
                prev = tg[j]
        else:
            for j in range(unroll):
                tg[j].copy_(traj[r, t + j + 1])
        for j in range(unroll):
            net.forward_train(xs[j], ws[j], out=xs[j + 1])
        # backward through the chain: g_j = dL/dx_{j+1} (+ what flows back from step j+2)
        g_cur = gbuf[0]
        for j in reversed(range(unroll)):
            abi.mse_loss_grad(xs[j + 1], tg[j], scale, grad=g_cur, grad_accumulate=j < unroll - 1, loss=loss,
                              scratch=scratch, accumulate=j < unroll - 1)
            g_next = gbuf[1] if g_cur is gbuf[0] else gbuf[0]
            net.backward(xs[j], g_cur, ws[j], grad_in=g_next if j > 0 else None, accumulate=j < unroll - 1)
            g_cur = g_next
        net.adam(lr=cur_lr)
        losses.append(float(loss.item()))
        if log_every and (it % log_every == 0 or it == iters - 1):
            print(f"iter {it:5d}  loss {losses[-1]:.4e}  lr {cur_lr:.2e}", flush=True)
    return losses


def main():
    import numpy as np
    import torch

    import acpr_inputs as I
    from . import abi

    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--ics", type=int, default=32)
    ap.add_argument("--iters", type=int, default=3000)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--unroll", type=int, default=2)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--lr-final", type=float, default=1e-4)
    ap.add_argument("--seed0", type=int, default=5000)
    ap.add_argument("--perturb", type=float, default=0.05)
    ap.add_argument("--init", default=None, help="start from these weights (.npz)")
    ap.add_argument("--workload", default="mass256", choices=["mass256", "large"])
    ap.add_argument("--crop", type=int, default=128, help="large: crop size (grid spacing stays 1/1024)")
    ap.add_argument("--slices", type=int, default=0, help="trajectory length in slices (0: the workload's)")
    args = ap.parse_args()
    W = I.MASS_F32_256 if args.workload == "mass256" else I.LARGE_F32_1024
    n = W.n if args.workload == "mass256" else args.crop
    length = W.length * n / W.n
    slices = args.slices or W.slices
    fp = abi.FineParams(n, W.eps, W.S, W.dt, variant=W.variant, precision=abi.AC_F32, length=length)
    ics = torch.tensor(np.stack([I.random_field(n, seed=args.seed0 + i, zero_mean=W.zero_mean)
                                 for i in range(args.ics)]), dtype=torch.float32, device="cuda")
    t0 = time.time()
    traj = make_trajectories(fp, ics, slices, W.steps)
    torch.cuda.synchronize()
    t1 = time.time()
    wt, bs = W.weights()
    if args.init:
        z = np.load(args.init)
        wt, bs = z["w"], z["b"]
    net = abi.TrainableCoarseNet(W.layers, W.channels, wt.astype(np.float32), bs.astype(np.float32), act=W.act,
                                 mass_fix=W.mass_fix)
    losses = train_coarse(net, traj, args.iters, args.batch, args.unroll, args.lr, log_every=200,
                          lr_final=args.lr_final, fine=(fp, W.steps), perturb=args.perturb)
    torch.cuda.synchronize()
    t2 = time.time()
    np.savez(args.out, w=net.w.cpu().numpy(), b=net.b.cpu().numpy(), layers=W.layers, channels=W.channels,
             act=W.act, workload=W.name, iters=args.iters, batch=args.batch, unroll=args.unroll, lr=args.lr,
             final_loss=losses[-1], first_loss=losses[0], perturb=args.perturb, ics=args.ics, mass_fix=W.mass_fix,
             seed0=args.seed0, crop=n, length=length, slices=slices,
             losses=np.asarray(losses[:: max(1, len(losses) // 200)]))
    print(f"trajectories {t1 - t0:.1f} s, training {t2 - t1:.1f} s, loss {losses[0]:.3e} -> {losses[-1]:.3e}")


if __name__ == "__main__":
    main()
