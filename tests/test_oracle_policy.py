"""Pins of the policy-side oracle (no GPU)."""
import math

import numpy as np
import pytest

from oracle import policy as op


def test_exp32_error_bound_and_special_values():
    """Cody-Waite + degree-7 Taylor: within 2 float32 ulps of e^x on [-80, 0];
    exact at 0; non-decreasing; 0 below the cut-off."""
    x = np.linspace(-80.0, 0.0, 200001).astype(np.float32)
    y = op.exp32(x).astype(np.float64)
    ref = np.exp(x.astype(np.float64))
    ulp = np.spacing(ref.astype(np.float32)).astype(np.float64)
    assert np.max(np.abs(y - ref) / ulp) <= 2.0
    assert op.exp32(np.float32(0.0)) == np.float32(1.0)
    assert np.all(np.diff(y) >= 0)
    assert op.exp32(np.float32(-80.5)) == 0.0


def test_sampler_single_valid_action_and_masking():
    rng = np.random.default_rng(0)
    N, K = 1000, 24
    logits = rng.normal(size=(N, K)).astype(np.float32)
    valid = np.zeros((N, K), bool)
    valid[np.arange(N), rng.integers(0, K, N)] = True
    u = rng.random(N).astype(np.float32)
    a = op.sample32(logits, valid, u)
    assert valid[np.arange(N), a].all()
    valid = rng.random((N, K)) < 0.3
    valid[:, 5] = True
    a = op.sample32(logits, valid, u)
    assert valid[np.arange(N), a].all()


def test_sampler_frequencies_match_softmax():
    """Inverse CDF on the masked softmax: empirical frequencies of one logit
    row over a fine grid of u equal the softmax probabilities."""
    K = 7
    logits = np.array([[0.3, -1.0, 2.0, 0.0, 1.5, -3.0, 0.7]], np.float32)
    valid = np.array([[1, 1, 1, 0, 1, 1, 1]], bool)
    n = 200000
    u = ((np.arange(n) + 0.5) / n).astype(np.float32)
    a = op.sample32(np.repeat(logits, n, 0), np.repeat(valid, n, 0), u)
    freq = np.bincount(a, minlength=K) / n
    z = np.exp(logits[0].astype(np.float64)) * valid[0]
    assert np.allclose(freq, z / z.sum(), atol=2e-5)


def test_logp_entropy_closed_forms():
    K = 6
    logits = np.zeros((3, K))
    valid = np.ones((3, K), bool)
    valid[1, 3:] = False
    valid[2, :] = False
    valid[2, 4] = True
    lp, ent = op.logp_entropy64(logits, valid, np.array([0, 1, 4]))
    assert lp == pytest.approx([-math.log(6), -math.log(3), 0.0])
    assert ent == pytest.approx([math.log(6), math.log(3), 0.0])


def test_mlp_hand_worked_example():
    """2 -> 2 -> 2 -> 2 network evaluated by hand (ReLU clips the second
    hidden unit of layer one to zero)."""
    w = dict(W1=np.array([[1.0, -1.0], [2.0, 0.0]]), b1=np.array([0.0, 1.0]),
             W2=np.eye(2), b2=np.array([-1.0, 0.5]),
             W3=np.array([[1.0, 2.0], [3.0, 4.0]]), b3=np.array([0.0, -1.0]),
             V1=np.array([[1.0, 0.0], [0.0, -1.0]]), c1=np.array([0.0, 0.0]),
             V2=np.array([[2.0, 1.0], [1.0, 1.0]]), c2=np.array([0.0, -10.0]),
             V3=np.array([[0.5], [7.0]]), c3=np.array([0.25]))
    x = np.array([[1.0, 1.0], [-1.0, 0.0]])
    logits, value = op.mlp64(w, x)
    # row 0: h1 = relu([3, 0]) = [3, 0]; h2 = relu([2, 0.5]); logits = [2 + 1.5, 4 + 2 - 1]
    # row 1: h1 = relu([-1, 2]) = [0, 2]; h2 = relu([-1, 2.5]) = [0, 2.5]; logits = [7.5, 9]
    assert logits.tolist() == [[3.5, 5.0], [7.5, 9.0]]
    # value row 0: g1 = relu([1, -1]) = [1, 0]; g2 = relu([2, 1 - 10]) = [2, 0]; v = 1 + 0.25
    # value row 1: g1 = relu([-1, 0]) = [0, 0]; g2 = relu([0, -10]) = 0; v = 0.25
    assert value.tolist() == [1.25, 0.25]
