"""Checkpoint / resume (the paper's runs converge over thousands of RF periods, §3): a handle
resumed from a checkpoint continues bit for bit as the saved handle does, in both
precisions, and foreign, damaged or truncated checkpoints are refused without touching the
handle."""
import numpy as np
import pytest

from paper_2109_04469_gb300 import pic, workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2109_04469_gb300 import build as B

    B.build()
    assert torch.cuda.is_available()


def _cfg(prec, **kw):
    c = workloads.params("ccp_5pa_150v_128c", refl_e=0.2, gamma_see=0.1, **kw)
    c["precision"] = prec
    return c


def _same(a, b):
    for s in (0, 1):
        pa, pb = a.particles(s), b.particles(s)
        for k in ("x", "vx", "vy", "vz", "id"):
            assert np.array_equal(pa[k], pb[k]), (s, k)
    assert a.step_state() == b.step_state()
    ga, gb = a.grid(), b.grid()
    for k in ("Ce", "Ci", "phi", "E"):
        assert np.array_equal(ga[k], gb[k]), k
    aa, ab = a.accum(), b.accum()
    for k in ("acc_e", "acc_i", "eepf", "fedf_e", "fedf_i", "counters", "steps"):
        assert np.array_equal(np.asarray(aa[k]), np.asarray(ab[k])), k


@pytest.mark.parametrize("prec", [pic.PIC_FP64, pic.PIC_FP32])
def test_resume_continues_bit_for_bit(prec):
    a = pic.Simulation(_cfg(prec))
    a.step(40)
    ck = a.checkpoint()
    assert bytes(ck[:8]) == b"PICCKPT1"
    a.step(35)
    assert a.sync() == 0
    # a second handle: another initial load size and a larger capacity are allowed
    b = pic.Simulation(_cfg(prec, init_per_species=100, capacity_per_species=80000))
    b.restore(ck)
    assert b.step_state()[0] == 40
    b.step(35)
    assert b.sync() == 0
    _same(a, b)


def test_foreign_damaged_and_truncated_checkpoints_are_refused():
    a = pic.Simulation(_cfg(pic.PIC_FP32))
    a.step(5)
    ck = a.checkpoint()
    b = pic.Simulation(_cfg(pic.PIC_FP32, n_cells=100))  # other physics
    with pytest.raises(pic.PicError):
        b.restore(ck)
    c = pic.Simulation(_cfg(pic.PIC_FP64))  # other precision
    with pytest.raises(pic.PicError):
        c.restore(ck)
    d = pic.Simulation(_cfg(pic.PIC_FP32))
    before = d.particles(0)
    bad = ck.copy()
    bad[0] ^= 0xFF
    with pytest.raises(pic.PicError):
        d.restore(bad)
    with pytest.raises(pic.PicError):
        d.restore(ck[: len(ck) - 1])
    small = pic.Simulation(_cfg(pic.PIC_FP32, capacity_per_species=1024, init_per_species=100))
    with pytest.raises(pic.PicError):  # counts beyond its capacity
        small.restore(ck)
    after = d.particles(0)
    assert all(np.array_equal(before[k], after[k]) for k in before)
