"""Ensembles of FP32 simulations (one launch per step) against the same simulations advanced
one by one with pic_step.

The compaction rule fixes every particle slot and the deposit is an integer sum, so the
schedule of the ensemble (owner size, grid, graph or not) cannot change a result: members must
match their single runs bit for bit (particles, ids, counts, fields, accumulators), whatever
the schedule, and stop exactly at their target steps (the paper's scans run different
numbers of steps per setting, §3)."""
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


# four different discharges around the 5 Pa base case (§3 scans: pressure, voltage, N_t,
# cells, weight, R, gamma), each its own seed stream
MEMBERS = [
    dict(n_cells=64, init_per_species=4000),
    dict(n_cells=100, pressure_pa=10.0, v_rf_amp_v=250.0, steps_per_rf=800, refl_e=0.3,
         gamma_see=0.2, init_per_species=6000, weight=1.5e5),
    dict(n_cells=200, pressure_pa=2.0, v_rf_amp_v=100.0, steps_per_rf=1500, refl_e=0.5,
         gamma_see=0.1, init_per_species=3000),
    dict(n_cells=128, pressure_pa=20.0, v_rf_amp_v=400.0, steps_per_rf=2000, refl_e=0.1,
         gamma_see=0.4, init_per_species=8000, weight=4e5),
]


def _cfg(i):
    c = workloads.params("ccp_5pa_150v_128c", **MEMBERS[i])
    c.update(precision=pic.PIC_FP32, instance=i, capacity_per_species=40000)
    return c


_STREAM = []


def _members():
    """The members, on one non-default stream (a graph is recorded only there: the legacy
    default stream cannot be captured, and the ensemble then launches directly)."""
    if not _STREAM:
        _STREAM.append(torch.cuda.Stream())
    with torch.cuda.stream(_STREAM[0]):
        return [pic.Simulation(_cfg(i)) for i in range(len(MEMBERS))]


def _same(a, b, where):
    for s in (0, 1):
        pa, pb = a.particles(s), b.particles(s)
        for k in ("x", "vx", "vy", "vz", "id"):
            assert np.array_equal(pa[k], pb[k]), (where, s, k)
    assert a.step_state() == b.step_state(), where
    ga, gb = a.grid(), b.grid()
    for k in ("Ce", "Ci", "phi", "E"):
        assert np.array_equal(ga[k], gb[k]), (where, k)
    aa, ab = a.accum(), b.accum()
    for k in ("acc_e", "acc_i", "eepf", "fedf_e", "fedf_i", "counters", "steps"):
        assert np.array_equal(np.asarray(aa[k]), np.asarray(ab[k])), (where, k)


def test_members_match_single_runs_bit_for_bit():
    ens_sims, solo = _members(), _members()
    ens = pic.Ensemble(ens_sims, [10**9] * len(ens_sims))
    assert ens.info()["graph"] == 1
    ens.step(60)
    assert ens.sync() == 0
    for s in solo:
        s.step(60)
        assert s.sync() == 0
    for i, (a, b) in enumerate(zip(ens_sims, solo)):
        assert a.step_state()[0] == 60
        _same(a, b, f"member {i}")
    ens.close()


def test_crowded_lists_match_an_ensemble_member():
    """A 2 mm gap with 2 keV electrons: nearly every electron leaves within the first steps,
    so a particle block's hole list outgrows its first warp's range and the single run packs
    its warps' lists in barrier-separated rounds.  The ensemble's owners need no packing, so
    the two runs agree bit for bit only if the packed lists keep particle order."""
    def cfg():
        c = workloads.params("ccp_5pa_150v_128c", gap_m=0.002, init_te_ev=2000.0, refl_e=0.5,
                             gamma_see=0.3, init_per_species=40000)
        c.update(precision=pic.PIC_FP32, instance=9, capacity_per_species=60000)
        return c

    if not _STREAM:
        _STREAM.append(torch.cuda.Stream())
    with torch.cuda.stream(_STREAM[0]):
        a, b = pic.Simulation(cfg()), pic.Simulation(cfg())
    ens = pic.Ensemble([a], [10**9])
    ens.step(6)
    assert ens.sync() == 0
    b.step(6)
    assert b.sync() == 0
    ne, _ = b.counts()
    assert ne < 20000  # most electrons left: the lists were crowded
    _same(a, b, "crowded")
    ens.close()


def test_uneven_targets_stop_each_member():
    targets = [60, 25, 0, 45]
    ens_sims, solo = _members(), _members()
    ens = pic.Ensemble(ens_sims, targets)
    ens.step(70)
    assert ens.sync() == 0
    for i, (a, b, t) in enumerate(zip(ens_sims, solo, targets)):
        b.step(t)
        b.sync()
        assert a.step_state()[0] == t
        _same(a, b, f"member {i}")
    ens.close()


@pytest.mark.parametrize("unit,bps,graph", [(256, 1, False), (1024, 2, True), (4000, 1, True)])
def test_schedule_does_not_change_results(unit, bps, graph):
    ref_sims, sims = _members(), _members()
    ref = pic.Ensemble(ref_sims, [10**9] * len(ref_sims))
    ens = pic.Ensemble(sims, [10**9] * len(sims))
    bps = min(bps, 2)
    try:
        ens.configure(unit, bps, graph)
    except pic.PicError:
        ens.configure(unit, 1, graph)
    info = ens.info()
    assert info["unit"] == unit and info["graph"] == int(graph)
    ref.step(40)
    ens.step(40)
    assert ref.sync() == 0 and ens.sync() == 0
    for i, (a, b) in enumerate(zip(ref_sims, sims)):
        _same(a, b, f"member {i}")
    ref.close()
    ens.close()


def test_autotune_picks_a_schedule_and_keeps_results():
    ens_sims, solo = _members(), _members()
    ens = pic.Ensemble(ens_sims, [10**9] * len(ens_sims))
    unit, bps = ens.autotune(2)
    assert unit in (4000, 8000, 16000) and bps in (1, 2)
    assert ens.info()["unit"] == unit
    ens.step(5)
    assert ens.sync() == 0
    n = ens_sims[0].step_state()[0]
    assert n > 5
    for s in solo:
        s.step(n)
    for i, (a, b) in enumerate(zip(ens_sims, solo)):
        _same(a, b, f"member {i}")
    ens.close()


def test_bad_members_are_rejected():
    fp64 = pic.Simulation(dict(_cfg(0), precision=pic.PIC_FP64))
    with pytest.raises(pic.PicError):
        pic.Ensemble([fp64], [10])
    s = pic.Simulation(_cfg(0))
    with pytest.raises(pic.PicError):
        pic.Ensemble([s, s], [10, 10])


def test_members_on_the_default_stream_launch_directly():
    sims = [pic.Simulation(_cfg(i)) for i in (0, 2)]  # legacy default stream
    solo = [pic.Simulation(_cfg(i)) for i in (0, 2)]
    ens = pic.Ensemble(sims, [10**9, 10**9])
    assert ens.info()["graph"] == 0
    ens.step(20)
    assert ens.sync() == 0
    for a, b in zip(sims, solo):
        b.step(20)
        _same(a, b, "default stream")
    ens.close()


def test_handles_of_different_grids_coexist():
    """Kernels are shared by all handles: a handle made later for a smaller grid must not
    lower the shared-memory limit a larger grid needs (both precisions)."""
    for prec in (pic.PIC_FP32, pic.PIC_FP64):
        big = pic.Simulation(dict(_cfg(2), precision=prec))    # 200 cells
        small = pic.Simulation(dict(_cfg(0), precision=prec))  # 64 cells, made later
        for sim in (big, small, big):
            sim.step(3)
            assert sim.sync() == 0



def test_bounded_waits_report_timeouts():
    """Failure detection without a fault: a bulk-copy barrier nothing completes and a grid
    barrier expecting a block that does not exist both give up and report PIC_ERR_TIMEOUT,
    and the context stays usable afterwards."""
    assert pic.selftest_waits() == (-6, -6)
    sim = pic.Simulation(_cfg(0))
    sim.step(3)
    assert sim.sync() == 0
