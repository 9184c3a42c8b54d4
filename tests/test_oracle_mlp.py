"""Pins of the oracle's DP PSF network (Sec. 3.2: five hidden layers of 512
ReLU neurons, 2 ks^2 linear outputs, clamped and sum-normalised jointly at
inference).

The pins use networks whose every layer is a signed, scaled permutation (one
non-zero weight per row), so the value of each neuron follows one path back
to one input and can be computed by hand: h_l[j] = max(s_l[j] c_l[j]
h_{l-1}[pi_l[j]] + b_l[j], 0).  The expected outputs are evaluated with that
scalar path walk, never with a matrix product, and the cases are chosen so
that a plausible slip in the oracle fails one of them:
  * a transposed hidden weight gathers from pi^-1 instead of pi (the
    permutations are not involutions);
  * a dropped or repeated layer changes the product of the per-neuron scales
    along each path (the scales differ per neuron, so the normalisation does
    not cancel them);
  * a missing ReLU lets a neuron negated at layer l come back positive after a
    second negation at layer l+1, and keeps a neuron that a negative bias
    should have zeroed;
  * a wrong input order reads another component of p;
  * a missing output clamp or a separate (per-plane) normalisation changes
    the normalised outputs.
Each planted variant of the network is evaluated beside the oracle to show
that the pins tell them apart.
"""
import numpy as np
import pytest

import oracle as O

HID = 512
N_LAYERS = 6  # input layer + 4 hidden-to-hidden + output


def _perm_no_fixed_involution(rng, n):
    """A permutation with no fixed point whose inverse differs from it."""
    while True:
        p = rng.permutation(n)
        if np.all(p != np.arange(n)) and np.any(p[p] != np.arange(n)):
            return p


def perm_net(rng, ks, negate_pairs=(), neg_bias=(), pos_bias=(), out_neg=()):
    """Signed scaled-permutation network.  Returns (weights, biases, path)
    where path describes each layer as (src index per neuron, sign, scale)."""
    n_out = 2 * ks * ks
    W, B, path = [], [], []
    # layer 0: neuron j reads input j % 3
    src0 = np.arange(HID) % 3
    sgn0 = np.ones(HID)
    sc0 = 1.0 + (np.arange(HID) % 5) * 0.25
    w0 = np.zeros((HID, 3))
    w0[np.arange(HID), src0] = sgn0 * sc0
    W.append(w0)
    B.append(np.zeros(HID))
    path.append((src0, sgn0, sc0))
    for l in range(1, 5):
        src = _perm_no_fixed_involution(rng, HID)
        sgn = np.ones(HID)
        sc = 1.0 + rng.integers(0, 7, size=HID) * 0.125
        w = np.zeros((HID, HID))
        w[np.arange(HID), src] = sgn * sc
        W.append(w)
        B.append(np.zeros(HID))
        path.append((src, sgn, sc))
    # output layer: output k reads hidden neuron q[k]
    q = rng.choice(HID, size=n_out, replace=False)
    sgn5 = np.ones(n_out)
    sc5 = 1.0 + (np.arange(n_out) % 3) * 0.5
    w5 = np.zeros((n_out, HID))
    w5[np.arange(n_out), q] = sgn5 * sc5
    W.append(w5)
    B.append(np.zeros(n_out))
    path.append((q, sgn5, sc5))

    def trace_back(k):
        """Neuron index of each hidden layer 0..4 on the path of output k."""
        idx = [0] * 5
        j = q[k]
        for l in range(4, -1, -1):
            idx[l] = j
            if l > 0:
                j = path[l][0][j]
        return idx

    # a negation at layer l followed by one at layer l + 1 on the path of k
    for k, l in negate_pairs:
        idx = trace_back(k)
        for ll in (l, l + 1):
            j = idx[ll]
            W[ll][j, path[ll][0][j]] *= -1
            path[ll][1][j] = -1
    # a negative bias larger than the pre-activation zeroes the neuron
    for k, l, b in neg_bias:
        B[l][trace_back(k)[l]] = b
    for k, l, b in pos_bias:
        B[l][trace_back(k)[l]] = b
    for k in out_neg:
        W[5][k, q[k]] *= -1
        path[5][1][k] = -1
    return W, B, path


def walk(W, B, path, p, relu=True):
    """Expected unnormalised outputs by walking each output's path with
    scalar arithmetic (layer by layer, neuron by neuron)."""
    out = []
    for x in np.asarray(p, np.float64):
        h = [float(v) for v in x]
        for l in range(5):
            src, sgn, sc = path[l]
            nh = []
            for j in range(HID):
                v = sgn[j] * sc[j] * h[src[j]] + B[l][j]
                nh.append(max(v, 0.0) if relu else v)
            h = nh
        q, sgn5, sc5 = path[5]
        out.append([sgn5[k] * sc5[k] * h[q[k]] + B[5][k] for k in range(len(q))])
    return np.array(out)


def normalise(o):
    o = np.maximum(o, 0.0)
    s = o.sum(axis=1, keepdims=True)
    return np.divide(o, s, out=np.zeros_like(o), where=s > 0)


# ---------------------------------------------------------------------------
# planted mistakes (evaluated beside the oracle; they must fail the pins)
# ---------------------------------------------------------------------------
def net_variant(W, B, p, ks, kind):
    h = np.asarray(p, np.float64)
    for l in range(5):
        if kind == "four_layers" and l == 3:
            continue
        w = W[l].T if (kind == "transposed" and 1 <= l <= 4) else W[l]
        h = h @ w.T + B[l]
        if not (kind == "no_relu" and l in (1, 2, 3)):
            h = np.maximum(h, 0.0)
    o = h @ W[5].T + B[5]
    if kind == "no_clamp":
        s = o.sum(axis=1, keepdims=True)
        return (o / s).reshape(-1, 2, ks, ks)
    if kind == "separate_norm":
        o = np.maximum(o, 0.0).reshape(-1, 2, ks * ks)
        return (o / o.sum(axis=2, keepdims=True)).reshape(-1, 2, ks, ks)
    return normalise(o).reshape(-1, 2, ks, ks)


INPUTS = np.array([[0.30, 0.70, 0.45],
                   [0.95, 0.05, 0.60],
                   [0.10, 0.20, 0.85]])


def test_positive_permutation_path_all_layers():
    """All signs +1, zero biases, positive inputs: every output is the
    product of its path's scales times one input component."""
    rng = np.random.default_rng(11)
    ks = 3
    W, B, path = perm_net(rng, ks)
    exp = normalise(walk(W, B, path, INPUTS)).reshape(-1, 2, ks, ks)
    got = O.mlp_psf(W, B, INPUTS, ks)
    np.testing.assert_allclose(got, exp, rtol=1e-13, atol=0)
    for kind in ("transposed", "four_layers"):
        bad = net_variant(W, B, INPUTS, ks, kind)
        assert np.max(np.abs(bad - exp)) > 1e-3, kind


def test_relu_zeroes_negated_and_biased_neurons():
    """Negated at hidden layer l and again at l + 1: ReLU zeroes the neuron
    at l, so the path's output is 0 (without the ReLU it would come back
    positive).  A negative bias larger than the pre-activation also zeroes
    it; a positive bias adds to it."""
    rng = np.random.default_rng(12)
    ks = 3
    negate = [(0, 1), (3, 2), (7, 3), (11, 1)]
    neg_bias = [(5, 2, -1e3), (13, 4, -1e3)]
    pos_bias = [(2, 1, 0.5), (9, 3, 0.25)]
    W, B, path = perm_net(rng, ks, negate_pairs=negate, neg_bias=neg_bias,
                          pos_bias=pos_bias)
    raw = walk(W, B, path, INPUTS)
    exp = normalise(raw).reshape(-1, 2, ks, ks)
    got = O.mlp_psf(W, B, INPUTS, ks)
    np.testing.assert_allclose(got, exp, rtol=1e-13, atol=0)
    flat = got.reshape(len(INPUTS), -1)
    for k in [k for k, _ in negate] + [k for k, _, _ in neg_bias]:
        assert np.all(flat[:, k] == 0.0), k
    for k, _, _ in pos_bias:
        assert np.all(flat[:, k] > 0.0)
    # the walk without ReLU brings the doubly negated paths back
    raw_lin = walk(W, B, path, INPUTS, relu=False)
    assert np.all(raw_lin[:, [k for k, _ in negate]] > 0)
    bad = net_variant(W, B, INPUTS, ks, "no_relu")
    assert np.max(np.abs(bad - exp)) > 1e-3


def test_input_layer_relu_and_component_order():
    """Layer 0 neuron j reads input j % 3: a negative input component
    zeroes every path that starts from it, the others keep theirs."""
    rng = np.random.default_rng(13)
    ks = 5
    W, B, path = perm_net(rng, ks)
    p = np.array([[0.4, -0.8, 0.9], [-0.5, 0.3, -0.2]])
    exp = normalise(walk(W, B, path, p))
    got = O.mlp_psf(W, B, p, ks).reshape(2, -1)
    np.testing.assert_allclose(got, exp, rtol=1e-13, atol=0)
    # which input each output traces back to
    q = path[5][0]
    start = np.empty(len(q), int)
    for k in range(len(q)):
        j = q[k]
        for l in range(4, 0, -1):
            j = path[l][0][j]
        start[k] = path[0][0][j]
    assert np.all(got[0, start == 1] == 0) and np.all(got[0, start != 1] > 0)
    assert np.all(got[1, start == 1] > 0) and np.all(got[1, start != 1] == 0)
    # swapping two input components changes the map
    assert np.max(np.abs(O.mlp_psf(W, B, p[:, [1, 0, 2]], ks).reshape(2, -1) - got)) > 1e-3


def test_output_clamp_joint_normalisation_and_layout():
    """Negative output weights are clamped to 0 before the sum; the sum runs
    over L and R together; output k lands at [k // ks^2][(k % ks^2) // ks]
    [k % ks]."""
    rng = np.random.default_rng(14)
    ks = 3
    out_neg = [1, 4, 10, 17]
    W, B, path = perm_net(rng, ks, out_neg=out_neg)
    raw = walk(W, B, path, INPUTS)
    exp = normalise(raw)
    got = O.mlp_psf(W, B, INPUTS, ks)
    np.testing.assert_allclose(got.reshape(len(INPUTS), -1), exp, rtol=1e-13, atol=0)
    for k in range(2 * ks * ks):
        side, r, c = k // (ks * ks), (k % (ks * ks)) // ks, k % ks
        np.testing.assert_allclose(got[:, side, r, c], exp[:, k], rtol=1e-13, atol=0)
    assert np.all(got.reshape(len(INPUTS), -1)[:, out_neg] == 0)
    np.testing.assert_allclose(got.sum(axis=(1, 2, 3)), 1.0, rtol=1e-13)
    for kind in ("no_clamp", "separate_norm"):
        bad = net_variant(W, B, INPUTS, ks, kind)
        assert np.max(np.abs(bad - got)) > 1e-3, kind


def test_mlp_biases_only_closed_form():
    """Zero weights: every point predicts ReLU(b_5) / sum ReLU(b_5); an
    all-negative output layer predicts the zero PSF."""
    rng = np.random.default_rng(1)
    ks = 5
    shapes = [(HID, 3)] + [(HID, HID)] * 4 + [(2 * ks * ks, HID)]
    w = [np.zeros(s) for s in shapes]
    b = [rng.normal(0, 0.05, size=s[0]) for s in shapes]
    p = rng.uniform(-1, 1, size=(4, 3))
    got = O.mlp_psf(w, b, p, ks)
    r = np.maximum(b[5], 0)
    np.testing.assert_allclose(got, np.broadcast_to((r / r.sum()).reshape(2, ks, ks), got.shape),
                               rtol=1e-14)
    b[5] = -np.abs(b[5])
    assert np.all(O.mlp_psf(w, b, p, ks) == 0)


def test_hidden_biases_propagate_through_every_layer():
    """Zero weights except a chain of unit weights from hidden layer 0 to
    the output: the output is the bias of layer 0 carried through four unit
    links plus each later bias, e.g. ((((b0 + b1) + b2) + b3) + b4) + b5."""
    ks = 1
    shapes = [(HID, 3)] + [(HID, HID)] * 4 + [(2, HID)]
    w = [np.zeros(s) for s in shapes]
    b = [np.zeros(s[0]) for s in shapes]
    chain = [7, 300, 41, 499, 128]
    for l in range(1, 5):
        w[l][chain[l], chain[l - 1]] = 1.0
    w[5][0, chain[4]] = 1.0
    vals = [0.5, 0.25, 0.125, 0.0625, 0.03125]
    for l in range(5):
        b[l][chain[l]] = vals[l]
    b[5][:] = [0.1, 0.3]
    p = np.array([[0.2, -0.4, 0.9]])
    got = O.mlp_psf(w, b, p, ks).reshape(-1)
    o0 = sum(vals) + 0.1
    np.testing.assert_allclose(got, [o0 / (o0 + 0.3), 0.3 / (o0 + 0.3)], rtol=1e-14)


def test_mlp_inputs_normalisation():
    H, W = 4, 6
    d = np.full((H, W), 0.5)
    d[1, 2] = 20.0
    p = O.mlp_inputs(d, 0.5, 20.0).reshape(H, W, 3)
    np.testing.assert_allclose(p[0, 0, :2], [-(W - 1) / W, -(H - 1) / H])
    np.testing.assert_allclose(p[-1, -1, :2], [(W - 1) / W, (H - 1) / H])
    np.testing.assert_allclose(p[:, :, 0].mean(), 0, atol=1e-15)
    assert p[0, 0, 2] == -1.0 and p[1, 2, 2] == 1.0
