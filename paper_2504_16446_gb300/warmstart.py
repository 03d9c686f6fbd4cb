"""Learned warm start for the L-BFGS reconstruction (library side).

A small 3-D convolutional network (tt.WarmStartNet: 4 layers of 3x3x3
convolutions, 15 -> 32 -> 32 -> 32 -> 15 channels, bfloat16 activations,
tensor-core kernels) maps the first back-projected gradient g0 = grad L(0) of
a reconstruction to a starting coefficient volume.  It is trained on
phantoms paired with their plain L-BFGS reconstructions, which the plain
method itself produces.  The zero-start plain solve remains the fallback
and the judge: the warm start is used only if its loss is below L(0).

Scale: the network is bias-free and ReLU is positively homogeneous, so the
input is normalised by its RMS and the output scale is fixed at inference by
the exact minimiser of the loss along the predicted direction u:
L(alpha u) = alpha^2 |Au|^2 - 2 alpha <Au, I> + L(0).  The solver starts
there through tt_lbfgs_create_ray, which needs one gradient evaluation, at
u: with g0 = grad L(0) = -2 A^T I it knows <Au, I> = -<u, g0>/2, |Au|^2 from
L(u), and the loss and gradient at the minimiser as combinations of those at
0 and u.  (warm_start() below is the two-loss form of the same scaling.)

Running this module (``python -m paper_2504_16446_gb300.warmstart``) trains
on the 64^3 ellipsoid workload and tests on held-out 128^3 phantoms (l_max 4,
240 projections of 128 x 128 x 16 segments), printing one JSON line with the
iterations and wall time to a 1e-3 excess loss for the zero-start FP32
solve, the warm-started FP32 solve and the warm-started bfloat16-storage
solve.  ``--save-weights weights/wsnet_ell64_15to15.npy`` writes the trained
weights that the benchmark loads (``load_net``).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np
import torch

from . import synth, tt


def phantom_data(h: tt.Handle, st, n_ell: int, seed: int, mean_counts: float = 1e4):
    """(I, c_true): Poisson data of a seeded ellipsoid phantom (GPU forward model)."""
    ph = synth.ellipsoid_phantom(st.shape[0], st.ell_max, n_ell, seed)
    dirs = torch.as_tensor(ph.dirs.reshape(-1, 3), dtype=torch.float32, device="cuda")
    amps = torch.as_tensor(ph.amps.reshape(-1, st.ell_max // 2 + 1), dtype=torch.float32, device="cuda")
    c_true = tt.zonal_to_sh(st.ell_max, dirs, amps).reshape(st.volume_shape).contiguous()
    clean = h.project(c_true)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    scale = mean_counts / float(clean.mean())
    I = (torch.poisson(clean.clamp(min=0) * scale, generator=gen) / scale).contiguous()
    return I, c_true


def plain_solve(h: tt.Handle, I, iters: int, c0=None):
    """Plain FP32 L-BFGS (m = 10) from c0 (zero by default): (c, loss)."""
    opt = tt.LBFGS(h, c0, I, None, m=10, log=False)
    for _ in range(iters):
        _, _, st = opt.step()
        if st != tt.TT_OK:
            break
    c = opt.get()[0]
    loss = opt.loss
    opt.close()
    return c, loss


def warm_start(net: tt.WarmStartNet, h: tt.Handle, I, g0, L0: float):
    """(c0, loss): alpha * net(g0 / rms(g0)) with the loss-minimising alpha, or
    zero when that does not beat L(0).  Along u the loss is the quadratic
    L(alpha u) = alpha^2 |Au|^2 - 2 alpha <Au, I> + L0, so L(u) and L(2u) fix
    it and its minimum L0 - <Au, I>^2 / |Au|^2 is the loss at c0."""
    s_in = float(g0.pow(2).mean().sqrt())
    u = net.forward(g0, s_in, 1.0).contiguous()
    L1, _ = h.gradient_residual(u, I, None, want_grad=False)
    L2, _ = h.gradient_residual((2.0 * u).contiguous(), I, None, want_grad=False)
    quad = 0.5 * (L2 - 2.0 * L1 + L0)          # |Au|^2
    lin = 0.5 * (L0 + quad - L1)               # <Au, I>
    if not quad > 0:
        return torch.zeros_like(u), L0
    Lw = L0 - lin * lin / quad
    if not Lw < L0:
        return torch.zeros_like(u), L0
    return ((lin / quad) * u).contiguous(), Lw


def warm_lbfgs(net: tt.WarmStartNet, h: tt.Handle, I, g0, L0: float, m: int = 10, log: bool = False) -> tt.LBFGS:
    """L-BFGS state at the loss minimiser along u = net(g0 / rms(g0)) (one
    gradient evaluation, at u); at zero when that ray does not lower the loss
    (the zero start is the fallback)."""
    s_in = math.sqrt(h.l2_norm(g0, want_grad=False)[0] / g0.numel())
    u = net.forward(g0, s_in, 1.0).contiguous()
    return tt.LBFGS.from_ray(h, u, g0, L0, I, None, m=m, log=log)


def warm_solve_to(net: tt.WarmStartNet, h: tt.Handle, I, L0ref: float, Lstar: float, target: float,
                  max_iter: int):
    """The whole warm-started solve on handle h, timed from scratch: the
    evaluation at zero that gives the network its input g0, the inference,
    the ray start and L-BFGS until (L - L*)/(L0 - L*) <= target (L0, L* the
    FP32 reference values).  Returns (iterations, evaluations -- both
    starting ones included --, seconds, seconds to the started state,
    L(start)/L0, alpha)."""
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    L0, g0 = h.gradient_residual(None, I, None)    # at c = 0: the back-projection of the data
    opt = warm_lbfgs(net, h, I, g0, L0)          # returns after a host synchronisation
    t_start = time.perf_counter() - t0
    L_start, alpha = opt.loss, opt.alpha
    it, ev = 0, 2
    while (opt.loss - Lstar) > target * (L0ref - Lstar) and it < max_iter:
        _, ne, st = opt.step()
        it += 1
        ev += ne
        if st != tt.TT_OK:
            break
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    opt.close()
    return it, ev, dt, t_start, L_start / L0, alpha


def iterations_to(h: tt.Handle, I, c0, L0: float, Lstar: float, target: float, max_iter: int):
    """(iterations, evaluations, seconds) of L-BFGS from c0 (None: from zero,
    whose first evaluation skips the forward projection) until
    (L - L*)/(L0 - L*) <= target."""
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    opt = tt.LBFGS(h, c0, I, None, m=10, log=False)
    it, ev = 0, 1
    while (opt.loss - Lstar) > target * (L0 - Lstar) and it < max_iter:
        _, ne, st = opt.step()
        it += 1
        ev += ne
        if st != tt.TT_OK:
            break
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    opt.close()
    return it, ev, dt


def conv_timing(n: int = 128, reps: int = 20):
    """Device time of the network's forward convolutions on an n^3 volume
    (tensor-core kernels): per layer shape, the standalone float-output form
    (tt_conv3d_bf16) and the form the network's layers run (tt_conv3d_bf16_act:
    bfloat16 output, ReLU fused for the 32-channel outputs), ms per launch and
    the dense-equivalent TFLOP/s."""
    import ctypes
    lib = tt.load()
    out = {}
    for cin, cout in ((16, 32), (32, 32), (32, 16)):
        gen = torch.Generator(device="cuda")
        gen.manual_seed(cin * 100 + cout)
        x = torch.randn((n, n, n, cin), device="cuda", generator=gen).to(torch.bfloat16)
        w = (0.1 * torch.randn((27, cout, cin), device="cuda", generator=gen)).to(torch.bfloat16)
        y32 = torch.empty((n, n, n, cout), device="cuda", dtype=torch.float32)
        y16 = torch.empty((n, n, n, cout), device="cuda", dtype=torch.bfloat16)
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        relu = 1 if cout == 32 else 0

        def run_f32():
            st = lib.tt_conv3d_bf16(n, n, n, cin, cout, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(w.data_ptr()),
                                    0, ctypes.c_void_p(y32.data_ptr()), stream)
            if st != tt.TT_OK:
                raise tt.TTError(st, "tt_conv3d_bf16", lib.tt_last_error().decode())

        def run_act():
            st = lib.tt_conv3d_bf16_act(n, n, n, cin, cout, ctypes.c_void_p(x.data_ptr()),
                                        ctypes.c_void_p(w.data_ptr()), relu, ctypes.c_void_p(y16.data_ptr()), stream)
            if st != tt.TT_OK:
                raise tt.TTError(st, "tt_conv3d_bf16_act", lib.tt_last_error().decode())

        row = {}
        for name, run in (("f32_out", run_f32), ("bf16_out" + ("_relu" if relu else ""), run_act)):
            for _ in range(3):
                run()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                run()
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1) / reps
            row[name] = {"ms": ms, "tflops": 2.0 * n ** 3 * 27 * cin * cout / (ms * 1e9)}
        out[f"{cin}->{cout}"] = row
    return out


WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "wsnet_ell64_15to15.npy")


def train(n_train: int = 512, epochs: int = 6, target_iters: int = 60, lr: float = 1e-3, seed0: int = 100,
          lr_final: float | None = None):
    """Trains the network on n_train seeded 6-ellipsoid phantoms of the 64^3
    workload (l_max 4, 120 projections of 64x64 x 16 segments): input g0 =
    grad L(0), target = plain L-BFGS after target_iters iterations.  The
    Adam step size is lr throughout, or with lr_final given, decays from lr
    to lr_final along a half cosine over the epochs.  Returns (net, info)."""
    st_tr = synth.workload("ell64")
    h_tr = tt.Handle(st_tr, "f32")
    t0 = time.perf_counter()
    data = []
    for s in range(n_train):
        I, _ = phantom_data(h_tr, st_tr, 6, seed0 + s)
        _, g0 = h_tr.gradient_residual(None, I, None)
        cstar, _ = plain_solve(h_tr, I, target_iters)
        data.append((g0, cstar, float(g0.pow(2).mean().sqrt()), float(cstar.pow(2).mean().sqrt())))
        del I
    t_data = time.perf_counter() - t0
    net = tt.WarmStartNet(15, 15, seed=0)
    t0 = time.perf_counter()
    losses = []
    for epoch in range(epochs):
        lr_e = lr
        if lr_final is not None and epochs > 1:
            lr_e = lr_final + 0.5 * (lr - lr_final) * (1.0 + math.cos(math.pi * epoch / (epochs - 1)))
        order = np.random.default_rng(epoch).permutation(len(data))
        ep = [net.train_step(data[i][0], data[i][1], data[i][2], lr_e, out_scale=data[i][3]) for i in order]
        losses.append(float(np.mean(ep)))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    h_tr.close()
    info = {"workload": "64^3, l_max 4, 120 x 64x64 x 16, 6-ellipsoid phantoms, seeds %d.." % seed0,
            "samples": n_train, "epochs": epochs, "target_iters": target_iters, "lr": lr, "lr_final": lr_final,
            "data_seconds": t_data, "train_seconds": t_train, "epoch_mean_loss": losses}
    return net, info


def load_net(path: str = WEIGHTS) -> tt.WarmStartNet:
    """The network with weights saved by ``--save-weights`` (float32 .npy)."""
    return tt.WarmStartNet(15, 15, weights=np.load(path))


def held_out_test(net: tt.WarmStartNet, n_test: int = 32, ref_iters: int = 150, seed0: int = 5000):
    """Time to (L - L*)/(L0 - L*) <= 1e-3 on n_test held-out 128^3 phantoms
    (l_max 4, 240 projections of 128 x 128 x 16 segments; L* = plain FP32
    L-BFGS after ref_iters iterations): zero-start FP32, warm-started FP32 and
    warm-started bfloat16-storage solves.  Every row is timed from scratch:
    the zero start's first evaluation is the one at zero inside
    tt_lbfgs_create; a warm row's time includes its own evaluation at zero
    (the network's input), the inference and the ray start.  Returns
    (summary, per-sample rows)."""
    st = synth.workload("ell128c16")
    h32 = tt.Handle(st, "f32")
    h16 = tt.Handle(st, "bf16")
    # one untimed warm-started solve first, on the first test phantom: the
    # first call in a process loads kernels and grows the allocator's pools
    # (reported apart from the per-phantom times)
    I, _ = phantom_data(h32, st, 6, seed0)
    L0, _ = h32.gradient_residual(None, I, None, want_grad=False)
    t_first = warm_solve_to(net, h16, I, L0, 0.0, 1e-3, 3)[2]
    del I
    rows = []
    for s in range(n_test):
        I, _ = phantom_data(h32, st, 6, seed0 + s)
        L0, _ = h32.gradient_residual(None, I, None, want_grad=False)
        _, Lstar = plain_solve(h32, I, ref_iters)
        zero = iterations_to(h32, I, None, L0, Lstar, 1e-3, ref_iters)
        warm = warm_solve_to(net, h32, I, L0, Lstar, 1e-3, ref_iters)
        warm16 = warm_solve_to(net, h16, I, L0, Lstar, 1e-3, ref_iters)
        rows.append({"seed": seed0 + s, "L0": L0, "L_star": Lstar, "L_warm_over_L0": warm[4],
                     "alpha": warm[5], "zero_f32": zero, "warm_f32": warm, "warm_bf16": warm16})
        del I
    h32.close()
    h16.close()

    def agg(key, i):
        return float(np.mean([r[key][i] for r in rows]))

    def warm_row(key):
        return {"iterations": agg(key, 0), "evals": agg(key, 1), "seconds": agg(key, 2),
                "warm_start_seconds": agg(key, 3)}

    summary = {"workload": "128^3, l_max 4, 240 x 128x128 x 16, 6-ellipsoid phantoms, held-out seeds %d.." % seed0,
               "samples": n_test, "criterion": f"(L - L*)/(L0 - L*) <= 1e-3, L* after {ref_iters} iterations",
               "timing": "each row from scratch: the zero row includes its evaluation at zero; a warm row its "
                         "evaluation at zero (the network's input), inference and ray start (one evaluation at "
                         "the network's output), in warm_start_seconds",
               "mean_L_warm_over_L0": float(np.mean([r["L_warm_over_L0"] for r in rows])),
               "zero_f32": {"iterations": agg("zero_f32", 0), "evals": agg("zero_f32", 1),
                            "seconds": agg("zero_f32", 2)},
               "warm_f32": warm_row("warm_f32"),
               "warm_bf16": warm_row("warm_bf16"),
               "fewer_iterations_in": int(sum(r["warm_bf16"][0] < r["zero_f32"][0] for r in rows)),
               "first_call_seconds": t_first}
    return summary, rows


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--conv-timing", type=int, default=0, metavar="N",
                    help="only time the forward convolutions on an N^3 volume and exit")
    ap.add_argument("--train", type=int, default=512)
    ap.add_argument("--test", type=int, default=32)
    ap.add_argument("--epochs", type=int, default=100)
    ap.add_argument("--target-iters", type=int, default=60, help="plain L-BFGS iterations of a training target")
    ap.add_argument("--ref-iters", type=int, default=150, help="L-BFGS iterations defining L* of a test phantom")
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--lr-final", type=float, default=5e-5,
                    help="decay the step size from --lr to this value along a half cosine (0 or less: constant)")
    ap.add_argument("--save-weights", default="", metavar="PATH",
                    help="write the trained weights (float32 .npy) to PATH")
    ap.add_argument("--load-weights", default="", metavar="PATH",
                    help="skip training: test the network with these weights")
    args = ap.parse_args(argv)
    if args.conv_timing:
        print(json.dumps({"experiment": "forward convolution timing", "volume": f"{args.conv_timing}^3",
                          "layers": conv_timing(args.conv_timing)}))
        return
    if args.load_weights:
        net, info = load_net(args.load_weights), {"weights": args.load_weights}
    else:
        net, info = train(args.train, args.epochs, args.target_iters, args.lr,
                          lr_final=args.lr_final if args.lr_final > 0 else None)
    if args.save_weights:
        os.makedirs(os.path.dirname(os.path.abspath(args.save_weights)), exist_ok=True)
        np.save(args.save_weights, net.weights())
    summary, rows = held_out_test(net, args.test, args.ref_iters)
    print(json.dumps({"experiment": "learned warm start", "train": info, "test": summary, "per_sample": rows}))


if __name__ == "__main__":
    main()
