"""Small single-kernel cases for profiling with ncu.

    python -m paper_2510_07672_gb300.profile_cases fine   # ac_fine_propagate_slices, 512 x 256^2, 20 steps
    python -m paper_2510_07672_gb300.profile_cases conv   # cnn_coarse_step, 16 x 256^2, 1-32x6-1 gelu bf16, mass shift
    python -m paper_2510_07672_gb300.profile_cases big    # ac_fine_propagate_slices, 16 x 1024^2, 2 steps
    python -m paper_2510_07672_gb300.profile_cases acnn   # acnn_forward (fused), 512 x 256^2, C = 4, 2 blocks
    python -m paper_2510_07672_gb300.profile_cases fine3d # ac_fine3d_propagate, 16 x 128^3, 1 step (5 passes)

Each case runs its call twice (a warm-up launch, then the one to capture) and
exits 0, so `ncu -s <warm-up launches> -c 1` captures a warm launch.  Inputs
are the benchmark's seeded synthetic fields.
"""
from __future__ import annotations

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(case: str) -> None:
    import numpy as np
    import torch

    import acpr_inputs as I
    import paper_2510_07672_gb300 as G

    W = I.MASS_F32_256
    if case == "fine":
        u = torch.tensor(np.stack([I.random_field(W.n, seed=s, zero_mean=True) for s in range(512)]),
                         dtype=torch.float32, device="cuda")
        fp = G.FineParams(W.n, W.eps, W.S, W.dt, variant=W.variant, precision=G.AC_F32)
        out = torch.empty_like(u)
        for _ in range(2):
            G.ac_fine_propagate_slices(fp, 20, u, out)
    elif case == "conv":
        wt, bs = W.weights()
        net = G.CoarseNet(W.layers, W.channels, wt.astype(np.float32), bs.astype(np.float32), act=W.act,
                          precision=G.AC_F32, mass_fix=W.mass_fix)
        u = torch.tensor(W.ics(), dtype=torch.float32, device="cuda")
        for _ in range(2):
            G.cnn_coarse_step(net, u)
    elif case == "big":
        n = 1024
        u = torch.tensor(np.stack([I.random_field(n, seed=s) for s in range(16)]), dtype=torch.float32,
                         device="cuda")
        fp = G.FineParams(n, 0.004, 2.0, 2e-5, variant=G.AC_CLASSIC, precision=G.AC_F32)
        out = torch.empty_like(u)
        for _ in range(2):
            G.ac_fine_propagate_slices(fp, 2, u, out)
    elif case == "acnn":
        w, b = I.acnn_weights(4, 2, seed=0)
        net = G.Acnn(4, 2, w, b, mass_fix=1, limiter=1, precision=G.AC_F32)
        u = torch.tensor(np.stack([I.random_field(W.n, seed=s, zero_mean=True) for s in range(512)]),
                         dtype=torch.float32, device="cuda")
        out = torch.empty_like(u)
        for _ in range(2):
            net(u, out=out)
    elif case == "fine3d":
        n = 128
        u = torch.tensor(np.stack([(-0.9 + 1.8 * I.uniform01(7000 + f, I.STREAM_IC, n ** 3)).reshape(n, n, n)
                                   for f in range(16)]), dtype=torch.float32, device="cuda")
        fp = G.FineParams(n, 0.02, 2.0, 1e-4, variant=G.AC_MASS_CONSERVING, precision=G.AC_F32)
        out = torch.empty_like(u)
        for _ in range(2):
            G.ac_fine3d_propagate(fp, 1, u, out)
    else:
        raise SystemExit(f"unknown case {case!r} (fine | conv | big | acnn | fine3d)")
    torch.cuda.synchronize()
    print(f"{case}: ok")


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "fine")
