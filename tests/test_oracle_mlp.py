"""Pins of the float64 surrogate-network reference (oracle/mlp_oracle.py), independent of
its own formulas: bfloat16 rounding against torch's conversion and hand-made ties, the tanh
GELU against the exact (erf) GELU and finite differences, and the layer-by-layer gradient
against central finite differences of the loss."""
import math

import numpy as np
import pytest

from oracle import mlp_oracle as M


def test_bf16_rounding_ties_and_library():
    torch = pytest.importorskip("torch")
    assert M.bf16(1.0) == 1.0
    assert M.bf16(1.0 + 2.0**-8) == 1.0               # tie between 1 and 1 + 2^-7: even
    assert M.bf16(1.0 + 3 * 2.0**-8) == 1.0 + 2.0**-6  # tie: rounds to the even neighbour
    assert M.bf16(1.0 + 2.0**-8 + 2.0**-20) == 1.0 + 2.0**-7
    x = np.random.default_rng(3).normal(0, 10, 10000).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).double().numpy()
    assert np.array_equal(M.bf16(x), ref)


def test_gelu_tanh_form_and_derivative():
    z = np.linspace(-6, 6, 1201)
    exact = 0.5 * z * (1.0 + np.array([math.erf(v / math.sqrt(2.0)) for v in z]))
    assert np.max(np.abs(M.gelu(z) - exact)) < 1e-3  # accuracy of the tanh form
    h = 1e-6
    fd = (M.gelu(z + h) - M.gelu(z - h)) / (2 * h)
    assert np.max(np.abs(M.gelu_grad(z) - fd)) < 1e-8


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(7)
    p = rng.normal(0, 0.1, M.N_PARAMS)
    x = rng.normal(0, 1, (5, M.N_IN))
    t = rng.normal(0, 1, (5, M.N_OUT))
    g, L = M.gradients(p, x, t)
    assert abs(L - M.loss(p, x, t)) < 1e-15
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in M.SHAPES])
    idx = np.concatenate([rng.integers(offs[k], offs[k + 1], 6) for k in range(len(M.SHAPES))])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (M.loss(p + e, x, t) - M.loss(p - e, x, t)) / (2 * h)
        assert abs(g[i] - fd) <= 1e-7 * max(1.0, abs(fd)) + 1e-9, (i, g[i], fd)


def test_flat_layout_round_trip():
    p = np.arange(M.N_PARAMS, dtype=np.float64)
    assert np.array_equal(M.flatten(M.unflatten(p)), p)
    assert M.N_PARAMS == 256 * 7 + 256 + 256 * 256 + 256 + 192 * 256 + 192
