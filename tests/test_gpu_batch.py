"""GPU tests of batching: problems of uneven slice counts and
steps in one handle, CUDA-graph replay of the iterations, several grid sizes
solved together on separate streams, and the fine-kernel autotuner.

Every field's arithmetic is independent of which other fields share a launch
(the fine kernel owns a field per cluster, the conv stack per pixel and per
field), so batched results must equal single-problem results bit for bit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import acpr_inputs as I
import paper_2510_07672_gb300 as G

pytestmark = pytest.mark.gpu


def make_net(C=16, L=4, seed=0, act=1):
    w, b = I.cnn_weights(L, C, seed=seed, sigma=0.05)
    return G.CoarseNet(L, C, w.astype(np.float32), b.astype(np.float32), act=act, precision=G.AC_F32)


def fields(n, seeds):
    return torch.tensor(np.stack([I.random_field(n, seed=s) for s in seeds]), dtype=torch.float32, device="cuda")


def test_uneven_problems_match_single_problem_solves():
    n = 64
    fp = G.FineParams(n, 2.5 / n, 2.0, 5e-5, variant=G.AC_CLASSIC, precision=G.AC_F32)
    net = make_net()
    s = [3, 5, 4]
    c = [20, 35, 10]
    u0 = fields(n, [1, 2, 3])
    pr = G.Parareal(fp, net, u0, s, c)
    its, _ = pr.solve(tol=0.0, kmax=max(s))
    assert its == s  # every problem runs to k = s_p, where it is exact
    U = pr.trajectory()
    for p in range(3):
        one = G.Parareal(fp, net, u0[p:p + 1].contiguous(), s[p], c[p])
        one.solve(tol=0.0, kmax=s[p])
        ref = one.trajectory()[0]
        assert torch.equal(U[p, : s[p] + 1], ref), p
        assert torch.count_nonzero(U[p, s[p] + 1:]) == 0
        # exact at k = s_p: the sequential fine solve with the same kernel
        seq = [u0[p:p + 1]]
        for j in range(s[p]):
            seq.append(G.ac_fine_propagate_slices(fp, c[p], seq[-1]))
        assert torch.equal(ref, torch.cat(seq))


def test_graph_replay_matches_direct_launches():
    n = 64
    fp = G.FineParams(n, 0.04, 2.0, 5e-5, variant=G.AC_MASS_CONSERVING, precision=G.AC_F32)
    w, b = I.cnn_weights(6, 32, seed=1)
    net = G.CoarseNet(6, 32, w.astype(np.float32), b.astype(np.float32), act=1, precision=G.AC_F32, mass_fix=1)
    u0 = fields(n, [4, 5])
    res = []
    for graphs in (False, True, True):  # the second graph run replays cached graphs
        pr = G.Parareal(fp, net, u0, 6, 25)
        pr.enable_graphs(graphs)
        pr.enable_timing(True)
        incs = []
        pr.iterate()
        for k in range(1, 7):
            l2, mx = pr.iterate()
            incs.append(l2)
        res.append((pr.trajectory(), incs))
        if graphs:
            pr.reset(u0)
            n0 = G.ac_launch_count()
            pr.iterate()
            for k in range(1, 7):
                l2, _ = pr.iterate()
                assert l2 == incs[k - 1]
            assert torch.equal(pr.trajectory(), res[-1][0])
            assert G.ac_launch_count() - n0 > 6 * 7  # replays count their kernels
            st = pr.stats()
            assert st["fine_ms"] > 0 and st["coarse_ms"] > 0 and st["increment_ms"] > 0
    assert torch.equal(res[0][0], res[1][0])
    assert res[0][1] == res[1][1]


def test_solve_many_sizes_on_streams():
    nets = make_net()
    handles, streams, singles = [], [], []
    for n, s, c, seeds in ((64, [4, 3], [30, 15], [7, 8]), (128, [3], [12], [9])):
        fp = G.FineParams(n, 2.5 / n, 2.0, 5e-5, precision=G.AC_F32)
        u0 = fields(n, seeds)
        handles.append(G.Parareal(fp, nets, u0, s, c))
        streams.append(torch.cuda.Stream())
        one = G.Parareal(fp, nets, u0, s, c)
        one.solve(tol=1e-6, kmax=max(s))
        singles.append(one.trajectory())
    out = G.parareal_solve_many(handles, streams, tol=1e-6, kmax=4)
    torch.cuda.synchronize()
    for h, ref in zip(handles, singles):
        assert torch.equal(h.trajectory(), ref)
    assert [len(o[0]) for o in out] == [2, 1]


def test_parareal_1024_exact_at_k_equals_s():
    """One 1024^2 problem (the two-pass fine path inside Parareal): at k = s the
    trajectory is the sequential fine solve bit for bit."""
    n, s, c = 1024, 3, 4
    fp = G.FineParams(n, 0.004, 2.0, 2e-5, precision=G.AC_F32)
    net = make_net(C=16, L=3)
    u0 = fields(n, [11])
    pr = G.Parareal(fp, net, u0, s, c)
    its, _ = pr.solve(tol=0.0, kmax=s)
    assert its == [s]
    seq = [u0]
    for j in range(s):
        seq.append(G.ac_fine_propagate_slices(fp, c, seq[-1]))
    assert torch.equal(pr.trajectory()[0], torch.cat(seq))


def test_uneven_grid_sizes_together_match_oracle():
    """Three handles of classic problems on 128^2, 256^2 and 512^2 grids
    (eps = 2.5 h, uneven slice counts and steps), iterated together by
    ac_parareal_solve_many on three streams with CUDA graphs, to k = 2: one
    problem of each grid size against the oracle's Algorithm 2 at the same k
    (float64 fine solves, the conv with the same bf16 roundings).  The
    bound is the float32 fine error 2e-5 sqrt(c) per slice times the slices
    the error is carried through, with a factor 2 for its growth along the
    sweep (the G here, N(0, 0.05^2) weights with 16 channels, adds bf16 flips
    far below that).  Measured on GB300 at 512^2: 1.9e-4 against 3.8e-4."""
    import os
    import oracle as O
    w, b = I.cnn_weights(4, 16, seed=0, sigma=0.05)
    w32, b32 = w.astype(np.float32), b.astype(np.float32)
    net = G.CoarseNet(4, 16, w32, b32, act=1, precision=G.AC_F32)
    spec = O.CnnSpec(4, 16, w32.astype(np.float64), b32.astype(np.float64), act=1, bf16=1)
    cases = [(128, [4, 3], [30, 20]), (256, [3, 5], [20, 10]), (512, [3, 2], [10, 15])]
    handles, streams, inputs = [], [], []
    for n, sl, st in cases:
        fp = G.FineParams(n, 2.5 / n, 2.0, 5e-5, variant=G.AC_CLASSIC, precision=G.AC_F32)
        u0 = fields(n, [100 + n + i for i in range(len(sl))])
        h = G.Parareal(fp, net, u0, sl, st)
        h.enable_graphs(True)
        handles.append(h)
        streams.append(torch.cuda.Stream())
        inputs.append((fp, u0, sl, st))
    G.parareal_solve_many(handles, streams, tol=0.0, kmax=2, allow_unconverged=True)
    torch.cuda.synchronize()
    with O.threads(os.cpu_count() or 1):
        for h, (fp, u0, sl, st) in zip(handles, inputs):
            n = fp.n
            U = h.trajectory()[0].double().cpu().numpy()
            ref = O.parareal(O.params(n, 2.5 / n, 2.0, 5e-5, 0), spec, sl[0], st[0], kmax=min(2, sl[0]), tol=0.0,
                             u0=u0[0].double().cpu().numpy())
            err = np.abs(U[: sl[0] + 1] - ref["U"]).max()
            print(f"n={n}: max-abs {err:.2e}")
            assert err < 2 * 2e-5 * np.sqrt(st[0]) * sl[0], n
