"""The surrogate pipeline end to end on the GPU: a scan of settings run by the FP32 ensemble
(the plain method), the network trained on it by the tensor-core kernels, and judged on
held-out settings by the plain method's own profiles.  What the network gains: profiles of
unseen settings closer than the best constant guess (the training mean), at a tiny fraction
of the cost of running them, and the §3.5 accuracy flags of unseen settings."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2109_04469_gb300 import build as B

    B.build()
    assert torch.cuda.is_available()


def test_surrogate_learns_the_scan_and_beats_the_mean():
    from paper_2109_04469_gb300 import surrogate as S

    settings = S.sample_settings(384, seed=11)
    X, Y, D, pic_s = S.run_scan(settings, warm_cycles=0.5, avg_cycles=0.5)
    assert X.shape == (384, 7) and Y.shape == (384, 192) and np.all(np.isfinite(Y))
    tr, te = np.arange(320), np.arange(320, 384)
    sur = S.Surrogate(batch_max=512, seed=4)
    losses = sur.fit(X[tr], Y[tr], epochs=300)
    assert losses[-1] < losses[0] / 4
    t = time.perf_counter()
    P = sur.predict(X[te])
    net_s = time.perf_counter() - t
    err = S.profile_error(P, Y[te])
    base = S.profile_error(np.repeat(Y[tr].mean(axis=0, keepdims=True), len(te), 0), Y[te])
    print("held-out profile error: network mean %.3f median %.3f | training mean %.3f"
          % (err.mean(), np.median(err), base.mean()))
    assert err.mean() < 0.8 * base.mean()
    assert net_s * len(settings) / len(te) < pic_s / 100  # per setting, >100x cheaper
    pf = S.accuracy_flags([settings[i] for i in te], P)
    gf = S.pic_flags([D[i] for i in te])
    agree = (pf == gf).mean(axis=0)
    print("flag agreement (omega_pe dt > 0.2, dx > lambda_D):", agree)
    assert agree[0] >= 0.75
