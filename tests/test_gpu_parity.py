"""GPU FP64 path vs the FP64 oracle through the C-ABI, on identical seeds.

Bar: the CUDA FP64 path follows the same step contract with the same operation order, so
particle states, charge counts, fields and accumulators are compared exactly; the stated
floating-point tolerance (1e-12 relative to each quantity's scale) is checked as well so a
failure reports its size.  Integer work (deposit counts, ids, order after compaction,
histograms, counters) must be bit-exact.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2109_04469_gb300 import pic, workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

REL_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2109_04469_gb300 import build as B

    B.build()
    O.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _pair(cfg):
    return pic.Simulation(cfg), O.OracleSim(cfg)


def _compare_particles(sim, ref, s, L, where=""):
    g, r = sim.particles(s), ref.particles(s)
    assert len(g["x"]) == len(r["x"]), f"{where} species {s}: count {len(g['x'])} vs {len(r['x'])}"
    assert np.array_equal(g["id"], r["id"]), f"{where} species {s}: ids/order differ"
    vscale = max(1.0, float(np.max(np.abs(r["vx"]))) if len(r["vx"]) else 1.0)
    report = {}
    for k in ("x", "vx", "vy", "vz"):
        scale = L if k == "x" else vscale
        d = np.abs(g[k] - r[k])
        report[k] = (int(np.count_nonzero(g[k] != r[k])), float(d.max() / scale) if len(d) else 0.0)
        assert report[k][1] <= REL_TOL, f"{where} species {s} {k}: {report[k]}"
    return report


def _compare_all(sim, ref, cfg, where=""):
    rep = [_compare_particles(sim, ref, s, cfg["gap_m"], where) for s in (0, 1)]
    ref.solve_field()  # the GPU solves the field of the current step at the end of a step
    gg, rg = sim.grid(), ref.grid()
    assert np.array_equal(gg["Ce"], rg["Ce"]) and np.array_equal(gg["Ci"], rg["Ci"]), where
    assert np.array_equal(gg["phi"], rg["phi"]) and np.array_equal(gg["E"], rg["E"]), where
    ga, ra = sim.accum(), ref.accum()
    assert ga["steps"] == ra["steps"]
    for k in ("eepf", "fedf_e", "fedf_i", "counters"):
        assert np.array_equal(ga[k], ra[k]), (where, k, ga[k], ra[k])
    for k in ("acc_e", "acc_i"):
        assert np.array_equal(ga[k], ra[k]), (where, k)
    return rep


def test_initial_load_and_deposit_bit_exact():
    for n in (1, 1023, 1025, 10_000):
        cfg = workloads.params("ccp_5pa_150v_128c", init_per_species=n,
                               capacity_per_species=max(n, 4096))
        sim, ref = _pair(cfg)
        rep = _compare_all(sim, ref, cfg, f"load n={n}")
        assert all(v[0] == 0 for r in rep for v in r.values()), rep
        sim.close()


def test_field_bit_exact():
    cfg = workloads.params("ccp_5pa_150v_128c")
    sim, ref = _pair(cfg)
    for step in (0, 137, 500, 999):
        sim.set_step(step)
        ref.set_step(step)
        sim.solve_field()
        ref.solve_field()
        g, r = sim.grid(), ref.grid()
        assert np.array_equal(g["phi"], r["phi"]) and np.array_equal(g["E"], r["E"]), step
    sim.close()


@pytest.mark.parametrize("nc", [2, 3, 401, 1024, 4096])
def test_deposit_and_field_random_positions(nc):
    cfg = workloads.params("ccp_5pa_150v_128c", n_cells=nc, init_per_species=0,
                           capacity_per_species=50_000)
    sim, ref = _pair(cfg)
    rng = np.random.default_rng(nc)
    n = 40_001
    L = cfg["gap_m"]
    for s in (0, 1):
        x = rng.uniform(0, L, n)
        x[:3] = [0.0, L, L * (1 - 2**-52)]
        v = rng.normal(0, 1e5, (3, n))
        ids = np.arange(n, dtype=np.uint32)
        sim.set_particles(s, x, v[0], v[1], v[2], ids, n)
        ref.set_particles(s, x, v[0], v[1], v[2], ids, n)
    sim.solve_field()
    ref.solve_field()
    g, r = sim.grid(), ref.grid()
    for k in ("Ce", "Ci", "phi", "E"):
        assert np.array_equal(g[k], r[k]), k
    assert int(g["Ce"].sum()) == n * 2**32
    sim.close()


@pytest.mark.parametrize("variant", [dict(), dict(refl_e=0.2, gamma_see=0.1),
                                     dict(refl_e=1.0, gamma_see=1.0)])
def test_200_steps_parity(variant):
    cfg = workloads.params("ccp_5pa_150v_128c", **variant)
    sim, ref = _pair(cfg)
    done = 0
    for upto in (1, 10, 50, 100, 200):
        sim.step(upto - done)
        ref.step(upto - done)
        done = upto
        assert sim.sync() == 0
        _compare_all(sim, ref, cfg, f"{variant} step {upto}")
    d_g, d_r = sim.diag(), ref.diag()
    for k in ("n_e", "n_i", "eepf", "fedf_i"):
        assert np.allclose(d_g[k], d_r[k], rtol=1e-13, atol=0), k
    for k in ("ion_flux", "omega_pe_dt", "lambda_d", "cfl_max", "p_coll_e", "p_coll_i"):
        assert abs(d_g[k] - d_r[k]) <= 1e-12 * abs(d_r[k]), k
    # a sum over the electrons in another order: rounding differences only
    assert abs(d_g["mean_energy_e_ev"] - d_r["mean_energy_e_ev"]) <= 1e-11 * d_r["mean_energy_e_ev"]
    assert d_g["return_code"] == int(d_r["unstable"])
    sim.close()


def test_high_collisionality_parity():
    # 100 Pa: electron P_max ~ 0.6 per step at this dt: most particles take the MCC branch
    cfg = workloads.params("ccp_5pa_150v_128c", pressure_pa=100.0, steps_per_rf=400,
                           init_per_species=5000, capacity_per_species=20_000,
                           refl_e=0.3, gamma_see=0.2)
    sim, ref = _pair(cfg)
    sim.step(60)
    ref.step(60)
    _compare_all(sim, ref, cfg, "100 Pa")
    assert ref.accum()["counters"][8] > 0
    sim.close()


def test_capacity_overflow_matches_oracle():
    cfg = workloads.params("ccp_5pa_150v_128c", pressure_pa=100.0, steps_per_rf=400,
                           init_per_species=3000, capacity_per_species=3010, v_rf_amp_v=0.0,
                           init_te_ev=40.0)
    sim, ref = _pair(cfg)
    sim.step(5)
    ref.step(5)
    assert ref.status & 1
    assert sim.status() == -3
    _compare_all(sim, ref, cfg, "capacity")
    sim.close()


def test_empty_population():
    cfg = workloads.params("ccp_5pa_150v_128c", init_per_species=0, capacity_per_species=64)
    sim, ref = _pair(cfg)
    sim.step(3)
    ref.step(3)
    _compare_all(sim, ref, cfg, "empty")
    ref.solve_field()  # the GPU has already solved the field of the current step
    g = sim.grid()
    assert np.array_equal(g["phi"], ref.grid()["phi"]) and np.array_equal(g["E"], ref.grid()["E"])
    sim.close()


def test_constant_rate_tables_parity():
    cfg = workloads.params("ccp_5pa_150v_128c", v_rf_amp_v=0.0, init_te_ev=30.0)
    sim, ref = _pair(cfg)
    F = np.zeros((O.XS_NODES, 4))
    F[:, 0], F[:, 1], F[:, 2] = 0.2, 0.5, 0.7
    sim.override_table(0, F, 3e9)
    ref.override_table(0, F, 3e9)
    sim.step(5)
    ref.step(5)
    _compare_all(sim, ref, cfg, "const table")
    sim.close()


def test_full_size_workload_parity():
    """The 2e6-per-species production workload (1 Pa, 300 V, 400 cells, R = 0.2, gamma = 0.1)
    in the launch configuration the benchmark times: 3 steps, every particle compared."""
    cfg = workloads.params("ccp_1pa_300v_400c")
    sim, ref = _pair(cfg)
    sim.step(3)
    ref.step(3)
    rep = _compare_all(sim, ref, cfg, "full size")
    print(rep)
    sim.close()
