"""The code against the numbers the paper prints (tests/golden/paper_values.txt).

The fixture holds the paper's own figures, each with the passage that states it: the
constants of its GELU and of its time-basis MLP, the shape of its training dataset, and
its hybrid solver's headline results (reported beside ours, not a target of a test).
"""
import inspect
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
from oracle import unet_ref as U  # noqa: E402
from paper_2312_05410_gb300 import inputs as I  # noqa: E402
from paper_2312_05410_gb300 import train_unet as T  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")


def paper_values():
    vals = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            k, v = (s.strip() for s in line.split("=", 1))
            nums = [float(t) for t in v.split()]
            vals[k] = nums[0] if len(nums) == 1 else nums
    return vals


def test_fixture_is_complete_and_self_consistent():
    P = paper_values()
    assert P["gelu_tanh_scale"] == pytest.approx(math.sqrt(2 / math.pi), rel=1e-15)
    for k in ("gelu_cubic_coefficient", "mlp_hidden_layers", "mlp_hidden_width", "dataset_grid",
              "dataset_snapshots", "hybrid_s2_rel_l2", "hybrid_speedup"):
        assert k in P, k


def test_oracle_gelu_uses_the_printed_constants():
    P = paper_values()
    for u in np.linspace(-5, 5, 41):
        want = 0.5 * u * (1 + math.tanh(P["gelu_tanh_scale"] * (u + P["gelu_cubic_coefficient"] * u ** 3)))
        assert float(U.gelu(torch.tensor(u, dtype=torch.float64))) == pytest.approx(want, rel=1e-14, abs=1e-15)


def test_time_basis_has_the_printed_depth_and_width():
    P = paper_values()
    assert U.FDIM == P["mlp_hidden_width"] == I.UNET_FDIM
    W = I.unet_weights(0)
    # input layer (1 -> width), hidden-to-hidden layers, output layer: 2 sin layers in between
    hidden = [k for k in W if k.startswith("mlp_w")]
    assert len(hidden) - 1 == P["mlp_hidden_layers"]
    assert W["mlp_w0"].shape == (U.FDIM, 1) and W["mlp_w1"].shape == (U.FDIM, U.FDIM)
    # sin after each of the two hidden layers: a zero-weight network gives f = w2 sin(w1 sin(b0) + b1) + b2
    tau = 0.3
    w0, b0, w1, b1, w2, b2 = (W[k].astype(np.float64) for k in
                              ("mlp_w0", "mlp_b0", "mlp_w1", "mlp_b1", "mlp_w2", "mlp_b2"))
    f = w2 @ np.sin(w1 @ np.sin(w0[:, 0] * tau + b0) + b1) + b2
    np.testing.assert_allclose(U.basis(W, tau), f, rtol=1e-12, atol=1e-12)


def test_training_data_has_the_printed_shape():
    P = paper_values()
    d = inspect.signature(T.generate).parameters
    assert [d["side"].default] * 2 == P["dataset_grid"]
    # a trajectory holds the paper's 50 equally spaced snapshots one jump (2000 steps) apart, and the
    # midpoints between them, which the look-back frames (1000 steps apart) need
    every, snaps = d["every"].default, d["snapshots"].default
    jump = 2 * every
    assert snaps * every == P["dataset_snapshots"] * jump
    assert snaps == 2 * P["dataset_snapshots"]


def test_paper_shaped_parameter_ranges():
    """The headline 512^2 film sits inside the paper's sweep: its deposition rate at the low end of the
    printed range, normal incidence at the top of the angle range, and a 50 % incident composition."""
    P = paper_values()
    lo, hi = P["dataset_rate_range"]
    alo, ahi = P["dataset_angle_range_deg"]
    p = I.default_params(**I.PAPER_512["params"])
    assert lo <= p["v_mag"] <= hi
    assert alo <= p["v_angle_deg"] <= ahi
    assert I.PAPER_512["spec"].c_inc == P["dataset_phase_fraction"]
