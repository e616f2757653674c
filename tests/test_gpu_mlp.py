"""The surrogate network's tensor-core kernels against the float64 reference
(oracle/mlp_oracle.py) with BF16 rounding at the same points: forward outputs, the loss and
every parameter gradient, and an Adam training run that fits a smooth synthetic map.

Tolerances: the reference rounds to BF16 where the kernels do, so the remaining differences
are FP32 accumulation order and the odd activation rounding the other way across a BF16
boundary (one BF16 step, 2^-8 relative, in a few elements), a few 1e-3 of the scale."""
import numpy as np
import pytest

from oracle import mlp_oracle as M
from paper_2109_04469_gb300 import pic

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2109_04469_gb300 import build as B

    B.build()
    assert torch.cuda.is_available()


def _data(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, (n, M.N_IN)).astype(np.float32)
    t = rng.normal(0, 1, (n, M.N_OUT)).astype(np.float32)
    return x, t


def test_initial_parameters_in_bounds():
    net = pic.Mlp(256, seed=5)
    p = M.unflatten(net.params().astype(np.float64))
    for name, (fi, fo) in (("W1", (7, 256)), ("W2", (256, 256)), ("W3", (256, 192))):
        a = np.sqrt(6.0 / (fi + fo))
        assert np.all(np.abs(p[name]) <= a) and np.std(p[name]) > 0.4 * a
    assert not np.any(p["b1"]) and not np.any(p["b2"]) and not np.any(p["b3"])


@pytest.mark.parametrize("n", [1, 130, 256])
def test_forward_matches_reference(n):
    net = pic.Mlp(256, seed=11)
    rng = np.random.default_rng(n)
    p = (rng.normal(0, 0.08, M.N_PARAMS)).astype(np.float32)
    net.set_params(p)
    x, _ = _data(n, n + 1)
    y = net.forward(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    ref, _ = M.forward(p.astype(np.float64), x, bf16_points=True)
    err = np.abs(y.cpu().numpy() - ref)
    assert err.max() <= 5e-3 * max(1.0, np.abs(ref).max()), err.max()


def test_gradients_match_reference():
    net = pic.Mlp(256, seed=3)
    rng = np.random.default_rng(9)
    p = (rng.normal(0, 0.08, M.N_PARAMS)).astype(np.float32)
    net.set_params(p)
    x, t = _data(256, 4)
    g, loss = net.gradients(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    gr, lr = M.gradients(p.astype(np.float64), x, t, bf16_points=True)
    assert abs(loss - lr) <= 1e-4 * lr
    off = 0
    for name, shp in M.SHAPES:
        k = int(np.prod(shp))
        a, b = g[off:off + k].astype(np.float64), gr[off:off + k]
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        assert rel < 2e-2, (name, rel)
        off += k


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
