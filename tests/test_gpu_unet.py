"""Tensor-core U-Net kernels against the FP64 reference U-Net (oracle/unet_ref.py).

The convolutions take BF16 operands, whose products are exact, and sum them in FP32
in tensor memory. Against the FP64 sum of the same BF16 values, each stored BF16
result therefore differs by at most
- one BF16 unit in the last place (the two sums may round to neighbouring values),
- plus the FP32 accumulation error.

The accumulation error is bounded by (K/4) 2^-24 sum|x w|. The tensor core rounds
to FP32 at most once per 4 products (K = taps x input channels), and cancellation
makes sum|x w| the relevant scale near zero. A missing or misplaced tap would
change a result by about sum|x w| / 9, thousands of times this bound.
"""
import numpy as np
import pytest

from oracle import unet_ref as U
from paper_2312_05410_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pf(cuda_ok):
    from paper_2312_05410_gb300 import build as B
    B.build()
    from paper_2312_05410_gb300 import pf as mod
    return mod


def ulp_bf16(x):
    a = np.abs(np.asarray(x, dtype=np.float64))
    e = np.floor(np.log2(np.maximum(a, 2.0 ** -126)))
    return 2.0 ** (e - 7)


def bound(ref, absdot, k):
    return ulp_bf16(ref) + (k / 4.0) * 2.0 ** -24 * absdot


def nhwc_dev(x_nchw):
    return torch.as_tensor(np.ascontiguousarray(np.transpose(x_nchw, (0, 2, 3, 1))), dtype=torch.float32).to(
        "cuda", torch.bfloat16)


def to_nchw(t):
    return np.transpose(t.float().cpu().numpy(), (0, 3, 1, 2)).astype(np.float64)


@pytest.mark.parametrize("n,h,w,cin,cout", [(2, 32, 32, 64, 128), (1, 16, 64, 32, 64), (1, 8, 256, 128, 32),
                                            (3, 8, 16, 256, 256), (1, 4, 32, 96, 64),
                                            (2, 8, 256, 64, 32), (1, 6, 384, 64, 64), (1, 1, 128, 64, 32),
                                            (2, 8, 128, 128, 64), (1, 3, 256, 128, 32), (2, 8, 128, 32, 64)])
def test_conv3x3_within_one_bf16_ulp_of_the_fp64_sum(pf, n, h, w, cin, cout):
    g = np.random.default_rng(n * 1000 + cin + cout)
    x = U.bf16(g.standard_normal((n, cin, h, w)))
    wt = (g.standard_normal((cout, cin, 3, 3)) / np.sqrt(9 * cin)).astype(np.float32)
    groups = 8
    out, part = pf.conv3x3_bf16(nhwc_dev(x), pf.conv_weight_layout(wt), groups)
    torch.cuda.synchronize()
    got = to_nchw(out)
    ref = U.conv3x3(torch.tensor(x), wt).numpy()
    absdot = U.conv3x3(torch.tensor(np.abs(x)), np.abs(U.bf16(wt))).numpy()
    tol = bound(ref, absdot, 9 * cin)
    assert np.all(np.abs(got - ref) <= tol), float(np.max(np.abs(got - ref) / tol))
    # group sums and sums of squares of the FP32 results, per 128-pixel tile
    p = part.cpu().numpy().astype(np.float64)
    cg = cout // groups
    tot = p.sum(axis=(2, 3))
    for i in range(n):
        for gi in range(groups):
            v = ref[i, gi * cg:(gi + 1) * cg]
            np.testing.assert_allclose(tot[i, gi, 0], v.sum(), rtol=1e-4, atol=1e-3)
            np.testing.assert_allclose(tot[i, gi, 1], (v * v).sum(), rtol=1e-4)


@pytest.mark.parametrize("n,h,w,cin,cout", [(2, 16, 256, 64, 32), (1, 5, 128, 64, 64), (3, 2, 512, 64, 32),
                                            (2, 8, 128, 128, 64), (1, 4, 256, 128, 32), (2, 6, 128, 32, 64),
                                            (1, 3, 256, 32, 32)])
def test_halo_staging_gives_the_same_sums_as_per_tap_staging(pf, n, h, w, cin, cout):
    """32-, 64- and 128-channel tiles on 128-pixel rows take the halo path by default (128 -> 64 as two
    column tiles of 32); the per-tap path adds the same products in the same order (tap by tap, then
    channel block, 16 channels at a time), so the two agree bit for bit, group sums included."""
    g = np.random.default_rng(h * w + cin + cout)
    x = nhwc_dev(U.bf16(g.standard_normal((n, cin, h, w))))
    wd = pf.conv_weight_layout((g.standard_normal((cout, cin, 3, 3)) / (3 * np.sqrt(cin))).astype(np.float32))
    assert pf.conv_halo(True) is True
    a, pa = pf.conv3x3_bf16(x, wd, 8)
    prev = pf.conv_halo(False)
    try:
        b, pb = pf.conv3x3_bf16(x, wd, 8)
    finally:
        pf.conv_halo(prev)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert torch.equal(pa, pb)


def test_conv3x3_writes_only_its_channel_slice(pf):
    g = np.random.default_rng(9)
    x = U.bf16(g.standard_normal((1, 64, 16, 16)))
    wt = (g.standard_normal((32, 64, 3, 3)) / 24).astype(np.float32)
    buf = torch.full((1, 16, 16, 96), 7.0, dtype=torch.bfloat16, device="cuda")
    pf.conv3x3_bf16(nhwc_dev(x), pf.conv_weight_layout(wt), 8, out=buf, out_coff=32)
    torch.cuda.synchronize()
    b = buf.float().cpu().numpy()
    assert np.all(b[..., :32] == 7.0) and np.all(b[..., 64:] == 7.0)
    ref = U.conv3x3(torch.tensor(x), wt).numpy()
    absdot = U.conv3x3(torch.tensor(np.abs(x)), np.abs(U.bf16(wt))).numpy()
    got = np.transpose(b[..., 32:64], (0, 3, 1, 2))
    assert np.all(np.abs(got - ref) <= bound(ref, absdot, 9 * 64))


@pytest.mark.parametrize("n,h,w,cin,cout", [(2, 16, 16, 256, 128), (1, 32, 32, 128, 64), (2, 64, 64, 64, 32)])
def test_transposed_conv_within_one_bf16_ulp(pf, n, h, w, cin, cout):
    g = np.random.default_rng(h + cin)
    x = U.bf16(g.standard_normal((n, cin, h, w)))
    wt = (g.standard_normal((cin, cout, 2, 2)) / np.sqrt(cin)).astype(np.float32)
    out = pf.tconv2x2_bf16(nhwc_dev(x), pf.tconv_weight_layout(wt))
    torch.cuda.synchronize()
    got = to_nchw(out)
    import torch.nn.functional as F
    ref = F.conv_transpose2d(torch.tensor(x), torch.tensor(U.bf16(wt)), stride=2).numpy()
    absdot = F.conv_transpose2d(torch.tensor(np.abs(x)), torch.tensor(np.abs(U.bf16(wt))), stride=2).numpy()
    tol = bound(ref, absdot, cin)
    assert np.all(np.abs(got - ref) <= tol), float(np.max(np.abs(got - ref) / tol))


def test_unsupported_shapes_are_rejected(pf):
    x = torch.zeros((1, 10, 10, 64), dtype=torch.bfloat16, device="cuda")
    w = torch.zeros((9, 32, 64), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(pf.PFError) as e:
        pf.conv3x3_bf16(x, w, 8)                    # 100 pixels: not a whole number of 128-pixel tiles
    assert e.value.code == pf.PF_ERR_ARG
    x = torch.zeros((1, 16, 16, 64), dtype=torch.bfloat16, device="cuda")
    w48 = torch.zeros((9, 48, 64), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(pf.PFError) as e:
        pf.conv3x3_bf16(x, w48, 8)                  # 48 output channels: not a width the kernel is built for
    assert e.value.code == pf.PF_ERR_ARG
    with pytest.raises(pf.PFError) as e:
        pf.conv3x3_bf16(x, w, 4)                    # the statistics are taken over 8 groups
    assert e.value.code == pf.PF_ERR_ARG


def _lookback_states(n, H, base_seed=0):
    """Three look-back frames per run: films of growing thickness and drifting composition (oldest first)."""
    import oracle as O
    from paper_2312_05410_gb300 import inputs as I
    p = O.with_dt(I.default_params())
    return [[I.film_state(I.FilmSpec(H, H, 40.0 + 10 * k + 4 * f, seed=base_seed + k, c_inc=0.45 + 0.05 * f), p)
             for f in range(3)] for k in range(n)]


def _unet_case(pf, n=2, H=128, seed=0, tau=0.5):
    """A jump of n runs with two pushed look-back frames, and the reference network on the same input."""
    from paper_2312_05410_gb300 import inputs as I
    W = I.unet_weights(seed)
    frames = _lookback_states(n, H)
    fields = [[tuple(pf.device_fields(fr)) for fr in run] for run in frames]
    net = pf.UNet(W, n, H, H)
    net.frame([run[0] for run in fields])
    net.frame([run[1] for run in fields])
    cur = [run[2] for run in fields]
    net.jump(cur, tau)
    net.sync()
    x = np.stack([np.concatenate([np.stack(fr) for fr in run] + [np.full((1, H, H), tau)]) for run in frames])
    taps = {}
    ref = U.forward(W, x, tau, taps)
    states = [run[2] for run in frames]
    return net, cur, ref, taps, x, states


def _layer_report(net, taps):
    pairs = [("zc1", "cat1", 0, 32), ("d1", "cat1", 32, 64), ("zc2", "cat2", 0, 64), ("d2", "cat2", 64, 128),
             ("zc3", "cat3", 0, 128), ("d3", "cat3", 128, 256), ("zc4", "zc4", 0, 256), ("h1", "h1", 0, 32)]
    rep = {}
    for tap, buf, c0, c1 in pairs:
        got = to_nchw(net.buffer(buf)[..., c0:c1])
        ref = taps[tap].numpy()
        d = np.abs(got - ref)
        rep[tap] = (float(np.mean(d > ulp_bf16(ref))), float(np.linalg.norm(got - ref) / np.linalg.norm(ref)))
    return rep


def test_unet_jump_matches_the_reference_network(pf):
    net, fields, ref, taps, x, states = _unet_case(pf)
    rep = _layer_report(net, taps)
    print("per-layer (fraction beyond 1 BF16 ulp, relative L2):", rep)
    for tap, (_, rel) in rep.items():
        assert rel <= 1e-2, (tap, rel)
    for i, f in enumerate(fields):
        for q, name in enumerate(("phi", "c", "rho")):
            got = f[q][:, :128].cpu().numpy().astype(np.float64)
            e = np.linalg.norm(got - ref[i, q]) / np.linalg.norm(ref[i, q])
            # the increment alone (the output convolution's affine result), against the reference's
            base = np.asarray(states[i][q], dtype=np.float32).astype(np.float64)
            di = np.linalg.norm((got - base) - (ref[i, q] - base)) / np.linalg.norm(ref[i, q] - base)
            print(f"run {i} {name}: relative L2 {e:.3e}, of the increment {di:.3e}")
            assert e <= 2e-2, (i, name, e)
            assert di <= 5e-2, (i, name, di)
    net.close()


def test_lookback_frames_enter_the_jump(pf):
    """The jump reads the pushed frames: with no frame pushed it equals the jump whose frames are the
    current fields themselves (bit for bit), and pushing other frames changes its result; reset_frames
    forgets them."""
    from paper_2312_05410_gb300 import inputs as I
    W = I.unet_weights(6)
    frames = _lookback_states(2, 128, base_seed=30)
    out = {}
    for mode in ("none", "current", "history", "reset"):
        fields = [[tuple(pf.device_fields(fr)) for fr in run] for run in frames]
        net = pf.UNet(W, 2, 128, 128)
        cur = [run[2] for run in fields]
        if mode == "current":
            net.frame(cur)
            net.frame(cur)
        elif mode in ("history", "reset"):
            net.frame([run[0] for run in fields])
            net.frame([run[1] for run in fields])
            if mode == "reset":
                net.reset_frames()
        net.jump(cur, 0.5)
        net.sync()
        out[mode] = [t.clone() for f in cur for t in f]
        net.close()
    for a, b in zip(out["none"], out["current"]):
        assert torch.equal(a, b)
    for a, b in zip(out["none"], out["reset"]):
        assert torch.equal(a, b)
    assert any(not torch.equal(a, b) for a, b in zip(out["none"], out["history"]))


def test_jump_is_the_same_with_halo_and_per_tap_staging(pf):
    """A whole jump at 256^2 (every halo form: 32, 64 and 128 input channels, the two-column-tile split,
    the output layer) against the same jump with every convolution staged per tap: bit for bit."""
    from paper_2312_05410_gb300 import inputs as I2
    import oracle as O
    W = I2.unet_weights(3)
    p = O.with_dt(I2.default_params())
    states = [I2.film_state(I2.FilmSpec(256, 256, 60.0, seed=20 + k), p) for k in range(2)]
    out = []
    prev = pf.conv_halo(True)
    try:
        for on in (True, False):
            pf.conv_halo(on)
            fields = [tuple(pf.device_fields(st)) for st in states]
            net = pf.UNet(W, 2, 256, 256)
            net.jump(fields, 0.5)
            net.sync()
            out.append([[t.clone() for t in f] for f in fields] + [net.buffer("h1").clone()])
            net.close()
    finally:
        pf.conv_halo(prev)
    a, b = out
    assert torch.equal(a[-1], b[-1])
    for fa, fb in zip(a[:-1], b[:-1]):
        for x, y in zip(fa, fb):
            assert torch.equal(x, y)


def test_plausibility_check_flags_out_of_range_runs(pf):
    from paper_2312_05410_gb300 import inputs as I2
    import oracle as O
    W = I2.unet_weights(1)
    W["out_gamma"][:] = 0.0
    W["out_beta"][:] = 0.0                      # zero increment: the jump is the identity
    p = O.with_dt(I2.default_params())
    st = [I2.film_state(I2.FilmSpec(128, 128, 50.0, seed=9 + k), p) for k in range(2)]
    fields = [tuple(pf.device_fields(s)) for s in st]
    before = [tuple(t.clone() for t in f) for f in fields]
    net = pf.UNet(W, 2, 128, 128)
    net.jump(fields, 0.5)
    net.sync()
    for f, b in zip(fields, before):
        for x, y in zip(f, b):
            assert torch.equal(x, y)
    assert net.check() == [True, True]
    fields[1][1][5, 7] = float("nan")
    assert net.check() == [True, False]
    fields[1][1][5, 7] = 0.5
    fields[0][0][0, 0] = 3.0
    assert net.check() == [False, True]
    net.close()


def test_hybrid_with_rejected_jumps_is_exactly_the_dns(pf):
    """Seeded untrained weights make every jump implausible: each one must be undone and replaced by the DNS
    stretch, so the hybrid result (pf_hybrid_run) equals plain DNS bit for bit."""
    import oracle as O
    from paper_2312_05410_gb300 import inputs as I2
    ms = []
    for m in I2.hybrid_members(2, 128, seed=7):
        p = O.with_dt(I2.default_params(v_mag=m["v_mag"]))
        ms.append((p, *I2.film_state(m["spec"], p)))
    ens = pf.Ensemble(ms)
    ens.set_tile(0)
    net = pf.UNet(I2.unet_weights(0), 2, 128, 128, stream=ens.stream)
    st = pf.Hybrid(ens, net, dns_stretch=200, jump_steps=200, frame_every=100).run(1200)
    assert st == {"jumps": 0, "fallbacks": 3, "dns_steps": 1200}
    hyb = [tuple(t.clone() for t in run) for run in ens.fields]
    ens.close()
    ref = pf.Ensemble(ms)
    ref.set_tile(0)
    ref.step(1200)
    for a, b in zip(hyb, ref.fields):
        for x, y in zip(a, b):
            assert torch.equal(x, y)
    ref.close()
    net.close()


def test_hybrid_with_identity_jumps_skips_the_jumped_steps(pf):
    """A zero output affine makes each jump the identity: the hybrid (pf_hybrid_run) then equals DNS of the
    stretches only."""
    import oracle as O
    from paper_2312_05410_gb300 import inputs as I2
    ms = []
    for m in I2.hybrid_members(2, 128, seed=8):
        p = O.with_dt(I2.default_params(v_mag=m["v_mag"]))
        ms.append((p, *I2.film_state(m["spec"], p)))
    W = I2.unet_weights(0)
    W["out_gamma"][:] = 0.0
    W["out_beta"][:] = 0.0
    ens = pf.Ensemble(ms)
    ens.set_tile(0)
    net = pf.UNet(W, 2, 128, 128, stream=ens.stream)
    st = pf.Hybrid(ens, net, dns_stretch=100, jump_steps=300, frame_every=50).run(800)
    assert st == {"jumps": 2, "fallbacks": 0, "dns_steps": 200}
    hyb = [tuple(t.clone() for t in run) for run in ens.fields]
    ens.close()
    ref = pf.Ensemble(ms)
    ref.set_tile(0)
    ref.step(200)
    for a, b in zip(hyb, ref.fields):
        for x, y in zip(a, b):
            assert torch.equal(x, y)
    ref.close()
    net.close()


def test_committed_weights_drive_the_hybrid_close_to_dns(pf):
    """The trained look-back surrogate shipped with the package, through pf_hybrid_run on two runs of the
    benchmark's 256^2 batch for 3 cycles: every jump passes the plausibility gate, and the fields stay within
    the measured per-cycle drift of plain DNS (phi and rho within 0.5 %, c within 2 %; the 16-run benchmark
    measured phi 0.08 %, c 0.5 % after 2 cycles)."""
    import os
    import oracle as O
    from paper_2312_05410_gb300 import inputs as I2
    path = os.path.join(os.path.dirname(pf.__file__), "weights", "unet_lb3_hybrid256.npz")
    with np.load(path) as z:
        W = {k: z[k] for k in z.files}
    assert W["enc1"].shape == (32, 10, 3, 3)
    ms = []
    for m in I2.hybrid_members(16, 256, seed=5)[:2]:
        p = O.with_dt(I2.default_params(v_mag=m["v_mag"]))
        ms.append((p, *I2.film_state(m["spec"], p)))
    hyb = pf.Ensemble(ms)
    hyb.set_tile(1)
    net = pf.UNet(W, 2, 256, 256, stream=hyb.stream)
    st = pf.Hybrid(hyb, net).run(12000)
    assert st == {"jumps": 3, "fallbacks": 0, "dns_steps": 6000}
    dns = pf.Ensemble(ms)
    dns.set_tile(1)
    dns.step(12000)
    torch.cuda.synchronize()
    for q, tol in ((0, 5e-3), (1, 2e-2), (2, 5e-3)):
        num = sum(float(((a[q][:, :256] - b[q][:, :256]) ** 2).sum()) for a, b in zip(hyb.fields, dns.fields))
        den = sum(float((b[q][:, :256] ** 2).sum()) for b in dns.fields)
        err = (num / den) ** 0.5
        print(f"field {q}: relative L2 against DNS after 3 cycles {err:.2e}")
        assert err <= tol, (q, err)
    net.close()
    hyb.close()
    dns.close()


def test_hybrid_dns_lead_in_runs_the_solver_alone_first(pf):
    """dns_lead: the first steps are DNS only, counted in total_steps.  With identity jumps the hybrid equals
    DNS of the lead-in plus the stretches; a lead-in at least as long as the run is plain DNS; a negative
    one is refused."""
    import oracle as O
    from paper_2312_05410_gb300 import inputs as I2
    ms = []
    for m in I2.hybrid_members(2, 128, seed=8):
        p = O.with_dt(I2.default_params(v_mag=m["v_mag"]))
        ms.append((p, *I2.film_state(m["spec"], p)))
    W = I2.unet_weights(0)
    W["out_gamma"][:] = 0.0
    W["out_beta"][:] = 0.0
    for lead, total, expect, dns_steps in ((300, 1100, {"jumps": 2, "fallbacks": 0, "dns_steps": 500}, 500),
                                           (1200, 1100, {"jumps": 0, "fallbacks": 0, "dns_steps": 1100}, 1100)):
        ens = pf.Ensemble(ms)
        ens.set_tile(0)
        net = pf.UNet(W, 2, 128, 128, stream=ens.stream)
        st = pf.Hybrid(ens, net, dns_stretch=100, jump_steps=300, frame_every=50, dns_lead=lead).run(total)
        assert st == expect, (lead, st)
        hyb = [tuple(t.clone() for t in run) for run in ens.fields]
        with pytest.raises(pf.PFError):
            pf.Hybrid(ens, net, dns_stretch=100, jump_steps=300, frame_every=50, dns_lead=-1).run(total)
        net.close()
        ens.close()
        ref = pf.Ensemble(ms)
        ref.set_tile(0)
        ref.step(dns_steps)
        for a, b in zip(hyb, ref.fields):
            for x, y in zip(a, b):
                assert torch.equal(x, y)
        ref.close()


def test_hybrid_lead_in_with_the_committed_weights_is_dns_then_the_cycles(pf):
    """With the trained surrogate, a lead-in of L steps gives bit for bit what L DNS steps followed by a
    hybrid run without lead-in give (no look-back frame is taken during the lead-in)."""
    import os
    import oracle as O
    from paper_2312_05410_gb300 import inputs as I2
    path = os.path.join(os.path.dirname(pf.__file__), "weights", "unet_lb3_hybrid256.npz")
    with np.load(path) as z:
        W = {k: z[k] for k in z.files}
    ms = []
    for m in I2.hybrid_members(16, 256, seed=5)[:2]:
        p = O.with_dt(I2.default_params(v_mag=m["v_mag"]))
        ms.append((p, *I2.film_state(m["spec"], p)))
    out = []
    for split in (False, True):
        ens = pf.Ensemble(ms)
        ens.set_tile(1)
        net = pf.UNet(W, 2, 256, 256, stream=ens.stream)
        if split:
            ens.step(3000)
            st = pf.Hybrid(ens, net).run(9000)
        else:
            st = pf.Hybrid(ens, net, dns_lead=3000).run(12000)
        assert st["jumps"] == 2 and st["fallbacks"] == 0, st
        torch.cuda.synchronize()
        out.append([tuple(t.clone() for t in run) for run in ens.fields])
        net.close()
        ens.close()
    for a, b in zip(*out):
        for x, y in zip(a, b):
            assert torch.equal(x, y)
