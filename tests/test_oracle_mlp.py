"""Pins of the learned-proposal oracle (oracle/mlp.py)."""
import math

import numpy as np
import pytest

import synth
from oracle import mlp


def test_bf16_rounding_matches_definition():
    # exactly representable values stay; halfway cases round to even
    vals = np.array([1.0, -2.5, 1.0 + 2 ** -7, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 0.0, 3e38])
    got = mlp.bf16(vals)
    assert got[0] == 1.0 and got[1] == -2.5 and got[2] == 1.0 + 2 ** -7
    assert got[3] == 1.0                     # tie -> even (down)
    assert got[4] == 1.0 + 2 ** -6           # tie -> even (up)
    rng = np.random.default_rng(0)
    a = rng.normal(0, 10, 10000)
    r = mlp.bf16(a)
    assert np.all(np.abs(r - a) <= np.abs(a) * 2 ** -8 + 1e-300)
    assert np.all(mlp.bf16(r) == r)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    p = rng.normal(0, 0.2, mlp.n_params())
    f = rng.normal(0, 1, (40, 6))
    lab = rng.integers(-1, 64, 40)
    loss, g = mlp.loss_and_grad(p, f, lab, round_bf16=False)
    idx = rng.choice(p.shape[0], 60, replace=False)
    h = 1e-6
    for t in idx:
        e = np.zeros_like(p); e[t] = h
        lp, _ = mlp.loss_and_grad(p + e, f, lab, round_bf16=False)
        lm, _ = mlp.loss_and_grad(p - e, f, lab, round_bf16=False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[t]) <= 1e-6 * max(1.0, abs(fd)) + 1e-8, t


def test_softmax_and_loss_closed_forms():
    p = np.zeros(mlp.n_params())
    W1, b1, W2, b2, W3, b3 = mlp.unpack(p)
    b3[:] = np.log(np.arange(1, 65))           # zero weights: logits are the bias
    f = np.ones((3, 6))
    logits, prob, _ = mlp.forward(p, f, round_bf16=False)
    assert np.allclose(prob[0], np.arange(1, 65) / np.arange(1, 65).sum(), rtol=1e-13)
    loss, g = mlp.loss_and_grad(p, f, np.array([63, 63, -1]), round_bf16=False)
    assert math.isclose(loss, -math.log(64 / 2080), rel_tol=1e-12)


def test_adam_first_step_moves_by_lr():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    p1, m, v = mlp.adam(p, np.zeros(3), np.zeros(3), g, 1, lr=0.01)
    # bias-corrected first step: m_hat = g, v_hat = g^2 -> step lr * sign(g)
    assert np.allclose(p1, p - 0.01 * np.sign(g), atol=1e-9)


def test_region_labels_follow_the_vote_bins():
    g = synth.geometry_of("event100_256")
    rho = np.array([-g["rho_max"] * 0.999, g["rho_max"] * 0.999, 0.0, 2 * g["rho_max"]])
    d0 = np.array([0.0, 19.0, -20.0, 0.0])
    reg = mlp.region_of(g, rho, d0)
    # d0 = 0 sits in bin 64 (block 4); rho just above -max is row 0 (block 0)
    assert reg.tolist() == [0 * 8 + 4, 7 * 8 + 7, 4 * 8 + 0, -1]


def test_mask_halo_and_fallback():
    g = synth.geometry_of("event100_256")
    mask = 1 << (3 * 8 + 5)                    # rho block 3, d0 block 5
    inside, halo = mlp.cell_allowed(g, mask)
    assert inside.sum() == 32 * 16
    assert halo.sum() == 34 * 18
    assert halo[95, 79] and halo[128, 96] and not halo[129, 80]
    mass = np.full(64, 1 / 64)
    assert mlp.region_mask(mass, 0.01, 0.5) == (1 << 64) - 1   # all pass -> fallback all
    mass2 = np.zeros(64); mass2[[1, 9]] = 0.5
    assert mlp.region_mask(mass2, 0.1, 0.5) == (1 << 1) | (1 << 9)


def test_mask_growth_and_empty_event():
    mass = np.zeros(64); mass[0 * 8 + 0] = 0.5; mass[4 * 8 + 7] = 0.5
    m = mlp.region_mask(mass, 0.1, 1.0, grow=True)
    want = {0, 1, 8, 9, 3 * 8 + 6, 3 * 8 + 7, 4 * 8 + 6, 4 * 8 + 7, 5 * 8 + 6, 5 * 8 + 7}
    assert m == sum(1 << r for r in want)
    assert mlp.region_mask(np.zeros(64), 0.1, 0.5, n_hits=0) == (1 << 64) - 1


def test_parameters_are_rounded_like_the_bf16_copy():
    # a bias just off a BF16 value is used as its rounding
    p = np.zeros(mlp.n_params())
    b3 = mlp.unpack(p)[5]
    b3[0] = 1.0 + 2 ** -10
    logits, _, _ = mlp.forward(p, np.zeros((1, 6)))
    assert logits[0, 0] == 1.0
    logits, _, _ = mlp.forward(p, np.zeros((1, 6)), round_bf16=False)
    assert logits[0, 0] == 1.0 + 2 ** -10


def test_masked_event_keeps_exactly_the_inside_peaks():
    import oracle
    g = synth.geometry_of("single_64")
    ev = synth.make_event(synth.CONFIGS["single_64"]["gen"], 5)
    full = oracle.run_event(g, ev.x, ev.y, ev.z)
    pk = full["peaks"]
    # a mask made of the regions of every other peak
    regs = sorted({int(p[0]) * 8 // 64 * 8 + int(p[1]) * 8 // 64 for p in pk[::2]})
    mask = sum(1 << r for r in regs)
    m = mlp.masked_event(g, ev.x, ev.y, ev.z, mask, acc=full["acc"])
    inside = [(p[0] * 8 // 64) * 8 + p[1] * 8 // 64 in regs for p in pk]
    assert np.array_equal(m["peaks"], pk[np.array(inside, bool)])
    assert m["count"] == sum(inside) and m["count"] >= (len(pk) + 1) // 2
    # every mask bit set reproduces the full event
    allm = mlp.masked_event(g, ev.x, ev.y, ev.z, (1 << 64) - 1, acc=full["acc"])
    assert np.array_equal(allm["assign"], full["assign"])
    assert np.array_equal(allm["zres"], full["zres"])
    assert allm["votes"] == full["stats"]["votes"]


# ------------------------------------------------ hand-computed pins of the network
def _features_pin(features):
    """features() at hand-placed hits; every expected value is exact in BF16.
    (0, -55) lies at azimuth -pi/2, which fixes the sign of the azimuth; z is
    a quarter of the z scale 110 sinh 2.5 (a float32 product, so the quarter
    divides back exactly)."""
    zs = np.float32(110.0) * np.float32(math.sinh(2.5))
    x = np.array([110.0, 0.0, -27.5], np.float32)
    y = np.array([0.0, -55.0, 0.0], np.float32)
    z = np.array([0.0, zs * np.float32(0.25), -zs], np.float32)
    lay = np.array([9, 0, 3])
    want = np.array([[1.0, 0.0, 0.0, 1.0, 0.0, 1.0],
                     [0.0, -0.5, 0.25, 0.5, -0.5, 0.0],
                     [-0.25, 0.0, -1.0, 0.25, 1.0, 0.333984375]])   # bf16(float32(3 / 9))
    return np.array_equal(features(x, y, z, lay), want)


def _dyadic_params():
    """Parameters with a few dyadic entries (exact in BF16): hidden units
    that go negative (so each ReLU matters) and an asymmetric W2 (so a
    transposed layer shows)."""
    p = np.zeros(mlp.n_params())
    W1, b1, W2, b2, W3, b3 = mlp.unpack(p)
    W1[0, 0] = 1.0                  # u0 = f0
    W1[0, 1] = -1.0                 # u1 = -f0 (negative for f0 > 0)
    W1[1, 2] = 0.5; b1[2] = 0.25    # u2 = f1 / 2 + 1/4
    W2[0, 0] = 1.0; W2[1, 0] = 2.0; W2[2, 0] = -1.0   # v0 = h0 + 2 h1 - h2
    W2[0, 1] = -1.0                                    # v1 = -h0
    W2[2, 2] = 1.0; b2[2] = 0.5                        # v2 = h2 + 1/2
    W2[1, 3] = 4.0                                     # v3 = 4 h1 (row 1 != column 1)
    W3[0, 0] = 1.0                                     # logit0 = w0
    W3[2, 1] = 2.0                                     # logit1 = 2 w2
    W3[1, 2] = 1.0                                     # logit2 = w1
    W3[0, 3] = -1.0; b3[3] = 1.0                       # logit3 = 1 - w0
    W3[3, 4] = 1.0                                     # logit4 = w3
    return p


def _forward_pin(forward):
    """Two hits by hand.  Hit A (f0 = 1, f1 = 1/2): u = (1, -1, 1/2) ->
    h1 = (1, 0, 1/2); v = (1/2, -1, 1, 0) -> h2 = (1/2, 0, 1, 0); logits
    (1/2, 2, 0, 1/2, 0, 0 ...).  Hit B (f0 = -1/2, f1 = -1/2): u = (-1/2,
    1/2, 0) -> h1 = (0, 1/2, 0); v = (1, 0, 1/2, 2) -> h2 = (1, 0, 1/2, 2);
    logits (1, 1, 0, 0, 2, 0 ...).  The other 59 logits are 0."""
    f = np.array([[1.0, 0.5, 0.0, 0.0, 0.0, 0.0],
                  [-0.5, -0.5, 0.0, 0.0, 0.0, 0.0]])
    logits, prob, _ = forward(_dyadic_params(), f)
    want = np.zeros((2, 64))
    want[0, :5] = [0.5, 2.0, 0.0, 0.5, 0.0]
    want[1, :5] = [1.0, 1.0, 0.0, 0.0, 2.0]
    if not np.array_equal(logits, want):
        return False
    e = np.exp(want - want.max(axis=1, keepdims=True))
    return np.allclose(prob, e / e.sum(axis=1, keepdims=True), rtol=1e-15, atol=0)


def test_features_at_hand_placed_hits():
    assert _features_pin(mlp.features)


def test_forward_pass_by_hand_through_both_relus():
    assert _forward_pin(mlp.forward)
    assert _forward_pin(lambda p, f: mlp.forward(p, f, round_bf16=False))


def test_planted_network_mistakes_fail_the_pins():
    """A copy of the oracle's forward pass or features with one step wrong --
    a ReLU dropped, W2 used transposed, x scaled by 1/100, the azimuth's sign
    flipped -- fails the hand-computed pins."""
    def forward_variant(no_relu1=False, no_relu2=False, w2_t=False):
        def fwd(p, f):
            W1, b1, W2, b2, W3, b3 = mlp.unpack(mlp.bf16(np.asarray(p, np.float64)))
            a1 = f @ W1 + b1
            h1 = mlp.bf16(a1 if no_relu1 else np.maximum(a1, 0.0))
            a2 = h1 @ (W2.T if w2_t else W2) + b2
            h2 = mlp.bf16(a2 if no_relu2 else np.maximum(a2, 0.0))
            logits = h2 @ W3 + b3
            z = logits - logits.max(axis=1, keepdims=True)
            e = np.exp(z)
            return logits, e / e.sum(axis=1, keepdims=True), None
        return fwd

    assert _forward_pin(forward_variant())                 # the copy itself is right
    assert not _forward_pin(forward_variant(no_relu1=True))
    assert not _forward_pin(forward_variant(no_relu2=True))
    assert not _forward_pin(forward_variant(w2_t=True))

    def features_variant(scale=110.0, az_sign=1.0):
        def feat(x, y, z, layer):
            f = mlp.features(x, y, z, layer).copy()
            f[:, 0] = mlp.bf16(np.asarray(x, np.float32) / np.float32(scale))
            f[:, 4] = az_sign * f[:, 4]
            return f
        return feat

    assert _features_pin(features_variant())
    assert not _features_pin(features_variant(scale=100.0))
    assert not _features_pin(features_variant(az_sign=-1.0))
