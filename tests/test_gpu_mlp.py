"""The surrogate network's tensor-core kernels against the float64 reference
(oracle/mlp_oracle.py), element by element, stage by stage.

Every kernel stage is checked on the inputs it actually consumed (read back with
pic_mlp_get_activations), against the reference's definition of that stage in float64:
  - each product (Z1, Z2, Y, dW1, dW2, dW3 and the dZ products) within the FP32 accumulation
    bound K u |A||B|^T + u |C| (u = 2^-24, K terms), as the GEMM test;
  - each BF16 rounding point (X, H1, H2, dYh, dZ2h, dZ1h) bit for bit, except where the
    stage's FP32 value and the reference's lie on two sides of a BF16 rounding midpoint within
    the FP32 error of the element-wise function (GELU by tanhf): there, one BF16 step;
  - bias gradients (column sums in row order) and the loss within their summation bounds.
Since every stage passes element-wise on its own inputs, the chain equals the reference
network up to those rounding allowances; the whole chain is also compared with the
reference's end-to-end outputs and gradients in norm.  Batches: 1, 130 and 1024 rows
forward, 128, 384 and 1024 rows for gradients (the backward pass needs multiples of 128).
"""
import numpy as np
import pytest

from oracle import mlp_oracle as M
from paper_2109_04469_gb300 import pic

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
U = 2.0**-24
C = np.sqrt(2.0 / np.pi)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2109_04469_gb300 import build as B

    B.build()
    assert torch.cuda.is_available()


@pytest.fixture(scope="module")
def net():
    n = pic.Mlp(1024, seed=11)
    yield n
    n.close()


def _data(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, (n, M.N_IN)).astype(np.float32)
    t = rng.normal(0, 1, (n, M.N_OUT)).astype(np.float32)
    return x, t


def _params(seed):
    rng = np.random.default_rng(seed)
    return rng.normal(0, 0.08, M.N_PARAMS).astype(np.float32)


def _step(v):
    return 2.0 ** (np.floor(np.log2(np.maximum(np.abs(v), 2.0**-126))) - 7)


def _check_product(name, got, A, B, bias=None, extra=0.0):
    """got ~ A @ B (+ bias) within K u |A||B| + u |result| (+ u |bias| + extra)."""
    ref = A @ B + (0.0 if bias is None else bias)
    bound = A.shape[1] * U * (np.abs(A) @ np.abs(B)) + U * np.abs(ref) + extra + 1e-30
    if bias is not None:
        bound = bound + U * np.abs(bias)
    err = np.abs(got - ref)
    assert np.all(err <= bound), (name, float((err / bound).max()),
                                  np.unravel_index(np.argmax(err / bound), err.shape))
    return ref


def _check_rounding(name, got, exact, tol):
    """got = bf16(FP32 value) where `exact` is the float64 value of the same function of the
    same inputs and tol bounds the FP32 evaluation error: equal to bf16(exact), or one BF16
    step away where the FP32 value may lie across a midpoint."""
    want = M.bf16(exact)
    ambiguous = M.bf16(exact - 2 * tol) != M.bf16(exact + 2 * tol)
    diff = np.abs(got - want)
    assert np.all((diff == 0) | (ambiguous & (diff <= _step(exact) * 1.0001))), \
        (name, int(np.count_nonzero(diff)), int(np.count_nonzero(ambiguous)))
    assert np.mean(ambiguous) < 0.01, (name, float(np.mean(ambiguous)))
    return int(np.count_nonzero(diff))


def _gelu_err(z):
    a = C * (z + 0.044715 * z**3)
    t = np.tanh(a)
    return 4.0 * U * (np.abs(z) * (2.0 + 2.0 * np.abs(t) + 2.0 * np.abs(a) * (1.0 - t * t))
                      + 3.0 * np.abs(0.5 * z * (1.0 + t)) + 1e-30)


def _gelu_grad_err(z):
    a = C * (z + 0.044715 * z**3)
    t = np.tanh(a)
    big = 0.5 * np.abs(z) * C * (1.0 + 0.134145 * z * z)
    dt = 4.0 * np.abs(t) + 4.0 * np.abs(a) * (1.0 - t * t) + 1.0
    return 4.0 * U * (2.0 + dt + big * (2.0 * np.abs(t) * dt + 4.0 * (1.0 - t * t) + 1.0))


def _forward_stages(net, p, x):
    n = x.shape[0]
    q = M.unflatten(p.astype(np.float64))
    W1, W2, W3 = M.bf16(q["W1"]), M.bf16(q["W2"]), M.bf16(q["W3"])
    A = {k: net.activations(k, n) for k in ("X", "Z1", "H1", "Z2", "H2", "Y")}
    assert np.array_equal(A["X"][:, :M.N_IN], M.bf16(x)) and not np.any(A["X"][:, M.N_IN:])
    _check_product("Z1", A["Z1"], A["X"][:, :M.N_IN], W1.T, q["b1"])
    flips = _check_rounding("H1", A["H1"], M.gelu(A["Z1"]), _gelu_err(A["Z1"]))
    _check_product("Z2", A["Z2"], A["H1"], W2.T, q["b2"])
    flips += _check_rounding("H2", A["H2"], M.gelu(A["Z2"]), _gelu_err(A["Z2"]))
    _check_product("Y", A["Y"], A["H2"], W3.T, q["b3"])
    return A, (W1, W2, W3), flips


@pytest.mark.parametrize("n", [1, 130, 1024])
def test_forward_stages_element_wise(net, n):
    p = _params(n)
    net.set_params(p)
    x, _ = _data(n, n + 1)
    y = net.forward(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    A, _, flips = _forward_stages(net, p, x)
    assert np.array_equal(y.cpu().numpy().astype(np.float64), A["Y"])
    # end to end against the reference network (rounding allowances only)
    ref, _ = M.forward(p.astype(np.float64), x, bf16_points=True)
    assert np.abs(A["Y"] - ref).max() <= 5e-3 * max(1.0, np.abs(ref).max()), flips


@pytest.mark.parametrize("n", [128, 384, 1024])
def test_gradient_stages_element_wise(net, n):
    p = _params(3 * n + 1)
    net.set_params(p)
    x, t = _data(n, 4 * n)
    g, loss = net.gradients(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    A, (W1, W2, W3), _ = _forward_stages(net, p, x)
    B = {k: net.activations(k, n) for k in ("dY", "dYh", "dZ2", "dZ2h", "dZ1", "dZ1h")}
    tt = t.astype(np.float64)
    # loss (per-row double sums of FP32 differences) and dY = 2 (Y - T) / (n 192) in FP32
    d = A["Y"] - tt
    assert abs(loss - np.mean(d * d)) <= 1e-6 * np.mean(d * d)
    s = 2.0 / (n * M.N_OUT)
    assert np.all(np.abs(B["dY"] - s * d) <= 4 * U * np.abs(s * d) + 1e-45)
    assert np.array_equal(B["dYh"], M.bf16(B["dY"]))  # one rounding of the same FP32 value
    gr = M.unflatten(g.astype(np.float64))
    # dW3 = dYh^T H2, db3 = column sums of dY
    _check_product("dW3", gr["W3"], B["dYh"].T, A["H2"])
    _check_product("db3", gr["b3"][None, :], np.ones((1, n)), B["dY"])
    # dZ2 = (dYh W3) GELU'(Z2), then its BF16 copy
    P2 = B["dYh"] @ W3
    D2 = M.gelu_grad(A["Z2"])
    bound = (M.N_OUT * U * (np.abs(B["dYh"]) @ np.abs(W3))) * np.abs(D2) + \
        np.abs(P2) * _gelu_grad_err(A["Z2"]) + 2 * U * np.abs(P2 * D2) + 1e-45
    assert np.all(np.abs(B["dZ2"] - P2 * D2) <= bound), float((np.abs(B["dZ2"] - P2 * D2) / bound).max())
    assert np.array_equal(B["dZ2h"], M.bf16(B["dZ2"]))
    _check_product("dW2", gr["W2"], B["dZ2h"].T, A["H1"])
    _check_product("db2", gr["b2"][None, :], np.ones((1, n)), B["dZ2"])
    P1 = B["dZ2h"] @ W2
    D1 = M.gelu_grad(A["Z1"])
    bound = (256 * U * (np.abs(B["dZ2h"]) @ np.abs(W2))) * np.abs(D1) + \
        np.abs(P1) * _gelu_grad_err(A["Z1"]) + 2 * U * np.abs(P1 * D1) + 1e-45
    assert np.all(np.abs(B["dZ1"] - P1 * D1) <= bound), float((np.abs(B["dZ1"] - P1 * D1) / bound).max())
    assert np.array_equal(B["dZ1h"], M.bf16(B["dZ1"]))
    _check_product("dW1", gr["W1"], B["dZ1h"].T, A["X"][:, :M.N_IN])
    _check_product("db1", gr["b1"][None, :], np.ones((1, n)), B["dZ1"])
    # end to end against the reference (rounding-point flips only)
    ref, lr = M.gradients(p.astype(np.float64), x, t, bf16_points=True)
    assert abs(loss - lr) <= 1e-4 * lr
    assert np.linalg.norm(g - ref) <= 2e-2 * np.linalg.norm(ref)


def test_initial_parameters_in_bounds():
    net = pic.Mlp(256, seed=5)
    p = M.unflatten(net.params().astype(np.float64))
    for name, (fi, fo) in (("W1", (7, 256)), ("W2", (256, 256)), ("W3", (256, 192))):
        a = np.sqrt(6.0 / (fi + fo))
        assert np.all(np.abs(p[name]) <= a) and np.std(p[name]) > 0.4 * a
    assert not np.any(p["b1"]) and not np.any(p["b2"]) and not np.any(p["b3"])
    net.close()


def test_activations_need_a_backward_pass():
    net = pic.Mlp(256, seed=5)
    x = torch.zeros(3, 7, device="cuda")
    net.forward(x)
    net.activations("Y", 3)
    with pytest.raises(pic.PicError):
        net.activations("dY", 3)
    with pytest.raises(pic.PicError):
        net.activations("Y", 4)  # more rows than the last call had
    net.close()


def test_training_fits_a_smooth_map():
    """Targets from a fixed smooth function of the inputs; Adam must cut the loss by 20x."""
    rng = np.random.default_rng(21)
    x = rng.uniform(-1, 1, (1024, M.N_IN)).astype(np.float32)
    freq = rng.normal(0, 1, (M.N_IN, M.N_OUT))
    t = np.sin(x @ freq).astype(np.float32)
    net = pic.Mlp(1024, seed=2)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    first = net.train_step(xd, td, 2e-3)
    for _ in range(400):
        net.train_step(xd, td, 2e-3, want_loss=False)
    last = net.train_step(xd, td, 2e-3)
    assert last < first / 20, (first, last)
