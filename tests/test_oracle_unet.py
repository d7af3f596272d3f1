"""Pins of the FP64 reference U-Net (oracle/unet_ref.py).

Each building block is checked against a direct, loop-level restatement of its
definition ("U-Net with temporal conditioning", Methods) on tiny inputs, and the
assembled network against invariants its structure implies: a group
normalisation after the first convolution removes an input scale, and one after
the bottleneck's decoder block removes the scale of the deepest conditioning
factor, but not that of the shallow ones.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
from oracle import unet_ref as U
from paper_2312_05410_gb300 import inputs as I  # noqa: E402


def test_bf16_rounding_matches_the_format():
    # spacing at 1 is 2^-7; ties go to the even significand
    cases = {1.0: 1.0, 1.0 + 2**-8: 1.0, 1.0 + 3 * 2**-8: 1.0 + 2**-6, 1.0 + 2**-7: 1.0 + 2**-7,
             -2.5: -2.5, 3.0e38: 2.9975e38, 1e-40: 9.99995e-41}
    for x, want in cases.items():
        got = float(U.bf16(np.float32(x)))
        assert got == pytest.approx(want, rel=2**-8), (x, got)
    assert float(U.bf16(np.float32(1.0 + 2**-8))) == 1.0
    assert float(U.bf16(np.float32(1.0 + 3 * 2**-8))) == 1.0 + 2**-6
    # against an independent implementation of the same rounding
    x = np.random.default_rng(0).standard_normal(10000).astype(np.float32) * 100
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(U.bf16(x), ref)


def test_conv3x3_is_zero_padded_cross_correlation():
    g = np.random.default_rng(1)
    x = U.bf16(g.standard_normal((1, 2, 5, 6)))
    w = g.standard_normal((3, 2, 3, 3)).astype(np.float32)
    wb = U.bf16(w)
    got = U.conv3x3(torch.tensor(x), w).numpy()
    ref = np.zeros((1, 3, 5, 6))
    for co in range(3):
        for i in range(5):
            for j in range(6):
                s = 0.0
                for ci in range(2):
                    for m in range(3):
                        for n in range(3):
                            ii, jj = i + m - 1, j + n - 1
                            if 0 <= ii < 5 and 0 <= jj < 6:
                                s += x[0, ci, ii, jj] * wb[co, ci, m, n]
                ref[0, co, i, j] = s
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)


def test_transposed_conv_scatters_each_pixel_into_a_2x2_block():
    g = np.random.default_rng(2)
    x = U.bf16(g.standard_normal((1, 3, 2, 3)))
    w = g.standard_normal((3, 2, 2, 2)).astype(np.float32)
    wb = U.bf16(w)
    got = U.up(torch.tensor(x), w).numpy()
    ref = np.zeros((1, 2, 4, 6))
    for co in range(2):
        for i in range(2):
            for j in range(3):
                for di in range(2):
                    for dj in range(2):
                        ref[0, co, 2 * i + di, 2 * j + dj] = sum(x[0, ci, i, j] * wb[ci, co, di, dj] for ci in range(3))
    np.testing.assert_array_equal(got, U.bf16(ref))


def test_group_norm_and_pooling_follow_their_definitions():
    g = np.random.default_rng(3)
    y = g.standard_normal((2, 8, 4, 4)) * 3 + 1
    gamma = g.standard_normal(8)
    beta = g.standard_normal(8)
    t = torch.tensor(y)
    mean, var = U.group_stats(t, 4)
    got = U.group_norm(t, mean, var, gamma, beta, 4).numpy()
    for n in range(2):
        for gi in range(4):
            v = y[n, 2 * gi:2 * gi + 2]
            m, s2 = v.mean(), ((v - v.mean()) ** 2).mean()
            for k in range(2):
                c = 2 * gi + k
                want = (y[n, c] - m) / math.sqrt(s2 + U.EPS) * gamma[c] + beta[c]
                np.testing.assert_allclose(got[n, c], want, rtol=1e-12, atol=1e-12)
    p = U.down(t).numpy()
    np.testing.assert_array_equal(p, y.reshape(2, 8, 2, 2, 2, 2).max(axis=(3, 5)))


def test_gelu_is_the_tanh_form_and_close_to_the_erf_form():
    for u in np.linspace(-6, 6, 61):
        want = 0.5 * u * (1 + math.tanh(math.sqrt(2 / math.pi) * (u + 0.044715 * u**3)))
        assert float(U.gelu(torch.tensor(u))) == pytest.approx(want, rel=1e-14, abs=1e-15)
        assert abs(want - 0.5 * u * (1 + math.erf(u / math.sqrt(2)))) < 1e-3


def test_mlp_basis_matches_a_loop_restatement():
    W = I.unet_weights(5)
    tau = 0.37
    w0, b0, w1, b1, w2, b2 = (W[k].astype(np.float64).tolist() for k in
                              ("mlp_w0", "mlp_b0", "mlp_w1", "mlp_b1", "mlp_w2", "mlp_b2"))
    h0 = [math.sin(w0[k][0] * tau + b0[k]) for k in range(U.FDIM)]
    h1 = [math.sin(sum(w1[k][j] * h0[j] for j in range(U.FDIM)) + b1[k]) for k in range(U.FDIM)]
    f = [sum(w2[k][j] * h1[j] for j in range(U.FDIM)) + b2[k] for k in range(U.FDIM)]
    np.testing.assert_allclose(U.basis(W, tau), f, rtol=1e-12, atol=1e-12)
    s = U.scales(W, tau)
    assert [v.shape[0] for v in s] == list(U.CH)
    np.testing.assert_allclose(s[2], W["proj3"].astype(np.float64) @ np.array(f), rtol=1e-12)


def _net_input(seed=4, n=2, h=32, w=32):
    """Three look-back frames of (phi, c, rho) that drift apart a little, then the dt plane."""
    g = np.random.default_rng(seed)
    x = np.empty((n, U.IN_CH, h, w))
    phi = np.tanh(g.standard_normal((n, h, w)))
    c = 0.5 + 0.2 * g.standard_normal((n, h, w))
    for f in range(U.LB):
        pf_ = np.tanh(np.arctanh(np.clip(phi, -0.99, 0.99)) + 0.3 * f)
        x[:, 3 * f] = pf_
        x[:, 3 * f + 1] = c + 0.1 * f * g.standard_normal((n, h, w))
        x[:, 3 * f + 2] = 0.5 * (1 - pf_)
    x[:, -1] = 0.25
    return x


def _newest(x):
    k = 3 * (U.LB - 1)
    return x[:, k:k + 3]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_network_shapes_and_the_residual_output():
    W = I.unet_weights(0)
    taps = {}
    x = _net_input()
    y = U.forward(W, x, 0.25, taps)
    assert y.shape == (2, 3, 32, 32)
    assert taps["z4"].shape == (2, 256, 4, 4) and taps["d1"].shape == (2, 32, 32, 32)
    np.testing.assert_allclose(y, _newest(x).astype(np.float32) + taps["inc"].numpy() * W["out_gamma"][None, :, None, None]
                               + W["out_beta"][None, :, None, None], rtol=1e-12, atol=1e-12)
    # with a zero output affine the jump is the identity on the FP32 fields
    W0 = dict(W, out_gamma=np.zeros(3, np.float32), out_beta=np.zeros(3, np.float32))
    np.testing.assert_array_equal(U.forward(W0, x, 0.25), _newest(x).astype(np.float32).astype(np.float64))


def test_network_invariants_of_the_normalisation_and_conditioning():
    """Invariants of the predicted increment (the output before the residual affine)."""
    W = I.unet_weights(0)
    x = _net_input()
    taps = {}
    U.forward(W, x, 0.25, taps)
    y = taps["inc"].numpy()

    def inc(Wd, xd, tau):
        t = {}
        U.forward(Wd, xd, tau, t)
        return t["inc"].numpy()
    # the first convolution is linear and GN follows it: an input scale of 2 (exact in BF16) drops out
    x2 = x.copy()
    x2 *= 2.0
    assert _rel(inc(W, x2, 0.25), y) < 1e-2
    # the bottleneck block sees only zc4 and normalises it: scaling W_4 changes nothing
    W4 = dict(W, proj4=W["proj4"] * 2.0)
    assert _rel(inc(W4, x, 0.25), y) < 1e-2
    # the shallow skip zc1 is concatenated with d1 before the block: scaling W_1 changes the output
    W1 = dict(W, proj1=W["proj1"] * 2.0)
    assert _rel(inc(W1, x, 0.25), y) > 0.05
    # the jump length enters through the basis: another tau gives another prediction
    assert _rel(inc(W, x, 0.75), y) > 0.05
    # every look-back frame enters the prediction: replacing the oldest or the middle frame by the newest
    # one (a stationary history) moves the increment
    for f in range(U.LB - 1):
        xs = x.copy()
        xs[:, 3 * f:3 * f + 3] = _newest(x)
        assert _rel(inc(W, xs, 0.25), y) > 0.05, f


def test_flop_count_matches_the_layer_shapes():
    # 256^2: encoder 377 M (10 input planes) + 3 x 604 M, decoder 1208 M + 3 x 2416 M, up-sampling
    # 3 x 268 M, output 113 M
    want = 377.5e6 + 3 * 604.0e6 + 1208.0e6 + 3 * 2416.0e6 + 3 * 268.4e6 + 113.2e6
    assert U.flops_per_sample(256, 256) == pytest.approx(want, rel=1e-3)


def test_training_network_is_the_reference_network():
    """The network that train_unet.py fits (PyTorch operations, FP32, no BF16 storage) and the FP64
    reference network that the inference kernels are tested against are the same function: their
    increments agree to 1 % (the BF16 storage of the reference), while a conditioning factor scaled by 2
    or a reversed channel order in the last block moves it by 30 % and more."""
    from paper_2312_05410_gb300 import train_unet as T
    net = T.make_model(0)
    W = {k: v.detach().numpy().copy() for k, v in net.p.items()}
    x = _net_input()
    with torch.no_grad():
        y = net(torch.tensor(x, dtype=torch.float32), 0.25).double().numpy()
    ref = U.forward(W, x, 0.25)
    base = _newest(x).astype(np.float32).astype(np.float64)
    assert _rel(y - base, ref - base) < 3e-2
    assert _rel(U.forward(dict(W, proj1=W["proj1"] * 2.0), x, 0.25) - base, ref - base) > 0.1
    assert _rel(U.forward(dict(W, dec1=W["dec1"][:, ::-1].copy()), x, 0.25) - base, ref - base) > 0.1
