"""Learned warm start: tensor-core convolution kernels and the network's
training gradients against the FP64 oracle, and what the trained network
gains over the zero-start solve.

The kernels take bfloat16 operands and accumulate in float, so the oracle is
fed the same bfloat16 values (FP64 sums): tolerance 1e-5 relative L2 for
one convolution and its weight gradient.  The whole network keeps its
activations and propagated gradients in bfloat16; against the oracle with
the same roundings the weight gradient agrees to 2e-2 (a rounding that
lands on the other side of a bfloat16 tie changes one element by 2^-8), and
against the unrounded FP64 network to 8e-2.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle.convnet import conv3d, conv3d_backward, network_backward, network_forward
from oracle.lbfgs import LBFGS as OracleLBFGS
from paper_2504_16446_gb300 import synth, tt

pytestmark = pytest.mark.gpu


def bf16_bits(a):
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)
    return ((u + (((u >> 16) & 1) + 0x7FFF)) >> 16).astype(np.uint16)


def bf16_round(a):
    return (bf16_bits(a).astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("cin,cout", [(16, 32), (32, 32), (32, 16), (16, 16)])
@pytest.mark.parametrize("shape", [(5, 7, 37), (2, 4, 32), (9, 3, 20), (1, 2, 1), (3, 9, 61)])
def test_conv_kernels_match_oracle(cin, cout, shape):
    rng = np.random.default_rng(cin + cout + shape[2])
    x = bf16_round(rng.normal(size=shape + (cin,)))
    w = bf16_round(rng.normal(size=(27, cout, cin)) * 0.2)
    dy = bf16_round(rng.normal(size=shape + (cout,)))
    lib = tt.load()
    xd = torch.as_tensor(bf16_bits(x).view(np.int16), device="cuda")
    wd = torch.as_tensor(bf16_bits(w).view(np.int16), device="cuda")
    dyd = torch.as_tensor(bf16_bits(dy).view(np.int16), device="cuda")
    y = torch.empty(shape + (cout,), dtype=torch.float32, device="cuda")
    dw = torch.zeros((27, cout, cin), dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert lib.tt_conv3d_bf16(*shape, cin, cout, xd.data_ptr(), wd.data_ptr(), 0, y.data_ptr(), s) == 0
    assert lib.tt_conv3d_wgrad_bf16(*shape, cin, cout, xd.data_ptr(), dyd.data_ptr(), dw.data_ptr(), s) == 0
    w5 = w.reshape(3, 3, 3, cout, cin)
    assert rel_l2(y.cpu().numpy(), conv3d(x, w5)) <= 1e-5
    _, dw_ref = conv3d_backward(x, w5, dy)
    assert rel_l2(dw.cpu().numpy(), dw_ref.reshape(27, cout, cin)) <= 1e-5


@pytest.mark.parametrize("cin,cout,relu", [(16, 32, 1), (32, 32, 1), (32, 32, 0), (32, 16, 0), (16, 32, 0)])
@pytest.mark.parametrize("shape", [(5, 7, 37), (9, 3, 20)])
def test_hidden_layer_form_matches_oracle(cin, cout, relu, shape):
    """bfloat16 output (ReLU fused or not), the network's hidden layers: each
    element is the FP32 accumulation rounded once to bfloat16, so it is
    within one bfloat16 unit (at most 2^-7 relative, plus the FP32 sum's
    error near zero) of the oracle's FP64 value rounded the same way, and
    within 2^-8 relative L2 (half a unit) of the unrounded one."""
    rng = np.random.default_rng(cin + 3 * cout + relu + shape[2])
    x = bf16_round(rng.normal(size=shape + (cin,)))
    w = bf16_round(rng.normal(size=(27, cout, cin)) * 0.2)
    lib = tt.load()
    xd = torch.as_tensor(bf16_bits(x).view(np.int16), device="cuda")
    wd = torch.as_tensor(bf16_bits(w).view(np.int16), device="cuda")
    y = torch.full(shape + (cout,), -1, dtype=torch.int16, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert lib.tt_conv3d_bf16_act(*shape, cin, cout, xd.data_ptr(), wd.data_ptr(), relu, y.data_ptr(), s) == 0
    got = (y.cpu().numpy().view(np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    ref = conv3d(x, w.reshape(3, 3, 3, cout, cin))
    if relu:
        ref = np.maximum(ref, 0.0)
    ref_b = bf16_round(ref)
    # one bfloat16 unit (at most 2^-7 of the value: 8 significant bits),
    # plus the FP32 accumulation's own error near zero
    assert np.all(np.abs(got - ref_b) <= 2.0 ** -7 * np.abs(ref_b) + 1e-5 * np.abs(ref).max())
    assert rel_l2(got, ref) <= 2.0 ** -8
    if relu:
        assert np.all(got >= 0.0)


def test_hidden_layer_form_rejects_uncompiled_pairs():
    lib = tt.load()
    x = torch.zeros((2, 2, 2, 16), dtype=torch.int16, device="cuda")
    w = torch.zeros((27, 16, 16), dtype=torch.int16, device="cuda")
    y = torch.zeros((2, 2, 2, 16), dtype=torch.int16, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert lib.tt_conv3d_bf16_act(2, 2, 2, 16, 16, x.data_ptr(), w.data_ptr(), 0, y.data_ptr(), s) == tt.TT_UNSUPPORTED


def test_network_gradient_matches_oracle():
    k_in, k_out = 15, 15
    shape = (6, 5, 21)
    rng = np.random.default_rng(4)
    x = rng.normal(size=shape + (k_in,)).astype(np.float32)
    tgt = rng.normal(size=shape + (k_out,)).astype(np.float32)
    scale = 1.7
    net = tt.WarmStartNet(k_in, k_out, seed=3)
    w_flat = net.weights().astype(np.float64)
    loss, g = net.gradient(torch.as_tensor(x, device="cuda"), torch.as_tensor(tgt, device="cuda"), scale)
    shapes = tt.WarmStartNet.layer_shapes(k_in, k_out)
    ws, off = [], 0
    for shp in shapes:
        n = int(np.prod(shp))
        ws.append(w_flat[off:off + n].reshape(shp))
        off += n
    count = np.prod(shape) * k_out
    for rnd, tol in ((bf16_round, 2e-2), (lambda a: a, 8e-2)):
        acts = network_forward(x / scale, ws, rnd)
        ref_loss = float(np.sum((acts[-1] - tgt / scale) ** 2) / count)
        grads = network_backward(acts, ws, 2 * (acts[-1] - tgt / scale) / count, rnd)
        ref = np.concatenate([gg.ravel() for gg in grads])
        assert abs(loss - ref_loss) <= tol * ref_loss
        assert rel_l2(g, ref) <= tol, rel_l2(g, ref)


def test_training_steps_reduce_the_loss():
    rng = np.random.default_rng(5)
    shape = (8, 8, 32)
    x = torch.as_tensor(rng.normal(size=shape + (15,)).astype(np.float32), device="cuda")
    # a target that a 3^3 convolution can represent: a fixed random linear filter of x
    w_t = rng.normal(size=(3, 3, 3, 15, 15)) * 0.05
    tgt = torch.as_tensor(conv3d(x.cpu().numpy(), w_t).astype(np.float32), device="cuda")
    net = tt.WarmStartNet(15, 15, seed=1)
    losses = [net.train_step(x, tgt, 1.0, 3e-3) for _ in range(100)]
    assert losses[-1] < 0.3 * losses[0], (losses[0], losses[-1])


def _solve_iters(h, I, c0, L0, Lstar, target=1e-3, max_iter=200):
    opt = tt.LBFGS(h, c0, I, None, m=10)
    it = 0
    while (opt.loss - Lstar) > target * (L0 - Lstar) and it < max_iter:
        _, _, st = opt.step()
        it += 1
        if st != tt.TT_OK:
            break
    return it


def test_warm_start_gains_over_zero_start():
    """Small version of the learned warm start: train on 24 phantoms of 24^3
    (the ellipsoid generator) paired with their plain L-BFGS reconstructions,
    then compare iterations to a 1e-3 excess loss on 4 held-out phantoms.
    The zero-start solve is the fallback (used when the warm start has a
    higher loss than zero) and the judge of the final loss."""
    n, L = 24, 4
    base = synth.workload("ell64")
    idx = np.arange(0, base.S, 4)
    st = synth.Setup(shape=(n, n, n), nj=n, nk=n, ell_max=L, inner_angle=base.inner_angle[idx],
                     outer_angle=base.outer_angle[idx], seg_start=base.seg_start, seg_end=base.seg_end,
                     j_offset=base.j_offset[idx], k_offset=base.k_offset[idx])
    h = tt.Handle(st, "f32")
    z = torch.zeros(st.volume_shape, dtype=torch.float32, device="cuda")

    def sample(seed):
        ph = synth.ellipsoid_phantom(n, L, 6, seed)
        dirs = torch.as_tensor(ph.dirs.reshape(-1, 3), dtype=torch.float32, device="cuda")
        amps = torch.as_tensor(ph.amps.reshape(-1, L // 2 + 1), dtype=torch.float32, device="cuda")
        c_true = tt.zonal_to_sh(L, dirs, amps).reshape(st.volume_shape)
        clean = h.project(c_true)
        gen = torch.Generator(device="cuda")
        gen.manual_seed(seed)
        scale = 1e4 / float(clean.mean())
        I = (torch.poisson(clean.clamp(min=0) * scale, generator=gen) / scale).contiguous()
        L0, g0 = h.gradient_residual(z, I, None)
        opt = tt.LBFGS(h, z, I, None, m=10)
        for _ in range(60):
            opt.step()
        Lstar = opt.loss
        cstar = opt.get()[0]
        s_in = float(g0.pow(2).mean().sqrt())
        s_out = float(cstar.pow(2).mean().sqrt())
        return I, g0, cstar, s_in, s_out, L0, Lstar

    train = [sample(100 + s) for s in range(24)]
    # output scale at inference: the training set's mean ratio of solution to gradient scale
    kappa = float(np.mean([so / si for _, _, _, si, so, _, _ in train]))
    net = tt.WarmStartNet(15, 15, seed=0)
    for epoch in range(40):
        for I, g0, cstar, si, so, _, _ in train:
            net.train_step(g0, cstar, si, 1e-3, out_scale=kappa * si)
    iters_zero, iters_warm, loss_ratio = [], [], []
    for s in range(4):
        I, g0, cstar, si, so, L0, Lstar = sample(900 + s)
        c0 = net.forward(g0, si, kappa * si).contiguous()
        Lw, _ = h.gradient_residual(c0, I, None, want_grad=False)
        loss_ratio.append(Lw / L0)
        if Lw >= L0:
            c0 = z
        iters_zero.append(_solve_iters(h, I, z, L0, Lstar))
        iters_warm.append(_solve_iters(h, I, c0, L0, Lstar))
    print("zero-start iterations", iters_zero, "warm-start iterations", iters_warm,
          "L(c0)/L(0)", [round(r, 4) for r in loss_ratio])
    assert max(loss_ratio) < 0.5
    assert sum(iters_warm) < sum(iters_zero)


def test_warm_start_scaling_reports_the_loss_at_its_result():
    """warmstart.warm_start scales the network's output u by the exact
    minimiser of the loss along it, from the losses at u and 2u (the squared
    loss is a quadratic in the scale); the loss it reports for the scaled
    start equals the library's loss there, and lies below L(0)."""
    from paper_2504_16446_gb300 import warmstart
    st = synth.small_setup(n=(16, 16, 16), nj=16, nk=16, ell_max=4, n_proj=12, n_seg=8, seed=21, offsets=False)
    h = tt.Handle(st, "f32")
    ph = synth.ellipsoid_phantom(16, 4, 3, 77)
    dirs = torch.as_tensor(ph.dirs.reshape(-1, 3), dtype=torch.float32, device="cuda")
    amps = torch.as_tensor(ph.amps.reshape(-1, 3), dtype=torch.float32, device="cuda")
    c_true = tt.zonal_to_sh(4, dirs, amps).reshape(st.volume_shape).contiguous()
    I = h.project(c_true)
    z = torch.zeros(st.volume_shape, dtype=torch.float32, device="cuda")
    L0, g0 = h.gradient_residual(z, I, None)
    net = tt.WarmStartNet(15, 15, seed=5)
    c0, Lw = warmstart.warm_start(net, h, I, g0, L0)
    assert float(c0.abs().max()) > 0 and Lw < L0
    L_true, _ = h.gradient_residual(c0, I, None, want_grad=False)
    assert abs(L_true - Lw) <= 1e-4 * L0


def test_ray_started_solver_agrees_with_the_two_loss_scaling():
    """warmstart.warm_lbfgs (one evaluation at u through tt_lbfgs_create_ray)
    starts where warmstart.warm_start's two-loss scaling puts c0, with the
    same loss."""
    from paper_2504_16446_gb300 import warmstart
    st = synth.small_setup(n=(16, 16, 16), nj=16, nk=16, ell_max=4, n_proj=12, n_seg=8, seed=23, offsets=False)
    h = tt.Handle(st, "f32")
    ph = synth.ellipsoid_phantom(16, 4, 3, 79)
    dirs = torch.as_tensor(ph.dirs.reshape(-1, 3), dtype=torch.float32, device="cuda")
    amps = torch.as_tensor(ph.amps.reshape(-1, 3), dtype=torch.float32, device="cuda")
    I = h.project(tt.zonal_to_sh(4, dirs, amps).reshape(st.volume_shape).contiguous())
    z = torch.zeros(st.volume_shape, dtype=torch.float32, device="cuda")
    L0, g0 = h.gradient_residual(z, I, None)
    net = tt.WarmStartNet(15, 15, seed=6)
    c0, Lw = warmstart.warm_start(net, h, I, g0, L0)
    opt = warmstart.warm_lbfgs(net, h, I, g0, L0)
    x, _, f = opt.get()
    assert opt.alpha != 0.0
    assert float((x - c0).norm() / c0.norm()) <= 1e-4
    assert abs(f - Lw) <= 1e-4 * L0
    f1, _, status = opt.step()
    assert status == tt.TT_OK and f1 < f
