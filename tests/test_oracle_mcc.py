"""Pins of the oracle's null-collision Monte Carlo step (§2 step 6; §3.1 one event per step;
§3.5 P_coll = 1 - exp(-nu_max dt); readings C-7..C-10, C-13, C-XS)."""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O

QE, ME, KB = 1.602176634e-19, 9.1093837015e-31, 1.380649e-23
MI = 39.948 * 1.66053906660e-27
XS = O.XS_NODES


def _sim(**kw):
    cfg = dict(gap_m=1.0, pressure_pa=5.0, v_rf_amp_v=0.0, steps_per_rf=1000, n_cells=64,
               weight=0.0, init_per_species=0, capacity_per_species=600_000)
    cfg.update(kw)
    return O.OracleSim(cfg)


def _electrons_at(s, eps_ev, n, seed=0):
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    sp = np.sqrt(np.asarray(eps_ev) * 2 * QE / ME) * np.ones(n)
    v = d * sp[:, None]
    x = rng.uniform(0.4, 0.6, n)
    s.set_particles(0, x, v[:, 0], v[:, 1], v[:, 2], np.arange(n, dtype=np.uint32), n)
    return x, v


def _const_table(f1, f2, f3):
    F = np.zeros((XS, 4))
    F[:, 0], F[:, 1], F[:, 2] = f1, f2, f3
    return F


def _eps(v):
    return 0.5 * ME * np.sum(v * v, axis=-1) / QE


def _v(p):
    return np.stack([p["vx"], p["vy"], p["vz"]], axis=1)


def test_candidate_and_process_rates_binomial():
    s = _sim()
    dt = s.derived()["dt"]
    pmax = 0.3
    s.override_table(0, _const_table(0.2, 0.5, 0.7), -math.log(1 - pmax) / dt)
    n = 100_000
    _electrons_at(s, 100.0, n)
    s.step(1)
    c = s.accum()["counters"].astype(float)
    cand = c[11]
    assert abs(cand - n * pmax) <= 4 * math.sqrt(n * pmax * (1 - pmax))
    for k, p in ((6, 0.2), (7, 0.3), (8, 0.2)):
        assert abs(c[k] - cand * p) <= 4 * math.sqrt(cand * p * (1 - p))
    assert s.count(0) == n + int(c[8]) and s.count(1) == int(c[8])


def test_excitation_removes_exactly_threshold():
    s = _sim()
    s.override_table(0, _const_table(0.0, 1.0, 1.0), 1e30)  # every electron is a candidate
    n = 5000
    rng = np.random.default_rng(1)
    eps = rng.uniform(11.6, 200.0, n)
    eps[:100] = rng.uniform(0.1, 11.5, 100)  # below threshold: null
    _, v = _electrons_at(s, eps, n, seed=1)
    s.step(1)
    p = s.particles(0)
    e2 = _eps(_v(p))
    assert np.array_equal(_v(p)[:100], v[:100])
    assert np.allclose(e2[100:], eps[100:] - 11.55, rtol=1e-12, atol=1e-12)
    assert int(s.accum()["counters"][7]) == n - 100


def test_ionization_energy_sharing_and_births():
    s = _sim()
    s.override_table(0, _const_table(0.0, 0.0, 1.0), 1e30)
    n = 20000
    rng = np.random.default_rng(2)
    eps = rng.uniform(16.0, 300.0, n)
    x, v = _electrons_at(s, eps, n, seed=2)
    s.step(1)
    pe, pi = s.particles(0), s.particles(1)
    assert s.count(0) == 2 * n and s.count(1) == n
    e_prim = _eps(_v(pe)[:n])
    e_new = _eps(_v(pe)[n:])
    assert np.allclose(e_prim, 0.5 * (eps - 15.76), rtol=1e-12)
    assert np.allclose(e_new, 0.5 * (eps - 15.76), rtol=1e-12)
    # births sit at the primary's position after the push (x^{n+1})
    assert np.array_equal(pe["x"][n:], pe["x"][:n]) and np.array_equal(pi["x"], pe["x"][:n])
    assert np.allclose(pe["x"][:n], x + v[:, 0] * s.derived()["dt"], rtol=1e-14)
    assert np.array_equal(pe["id"][n:], np.arange(n, 2 * n)) and np.array_equal(pi["id"], np.arange(n))
    sig = math.sqrt(KB * 300.0 / MI)
    for c in ("vx", "vy", "vz"):
        assert stats.kstest(pi[c] / sig, "norm").pvalue > 1e-3
    # charge of the births is deposited at birth: counts match the populations exactly
    g = s.grid()
    assert int(g["Ce"].sum()) == 2 * n * 2**32 and int(g["Ci"].sum()) == n * 2**32


def test_elastic_energy_loss_and_isotropy():
    s = _sim()
    s.override_table(0, _const_table(1.0, 1.0, 1.0), 1e30)
    n = 40000
    _, v = _electrons_at(s, 10.0, n, seed=3)
    s.step(1)
    v2 = _v(s.particles(0))
    ratio = _eps(v2) / _eps(v)
    mr2 = 2 * ME / MI
    assert np.all(ratio <= 1 + 1e-12) and np.all(ratio >= 1 - 2 * mr2 - 1e-12)
    cosx = np.sum(v * v2, axis=1) / (np.linalg.norm(v, axis=1) * np.linalg.norm(v2, axis=1))
    assert stats.kstest(cosx, "uniform", args=(-1, 2)).pvalue > 1e-3
    assert abs(np.mean(ratio) - (1 - mr2)) < 5 * mr2 / math.sqrt(3 * n)


@pytest.mark.parametrize("eps", [0.5, 5.0, 20.0, 100.0])
def test_null_collision_rate_is_summed_frequency(eps):
    """The real-collision probability per step equals P_max nu_T(eps) / nu_max, with nu_T the
    summed collision frequency of the closed-form cross sections."""
    s = _sim(pressure_pa=5.0)
    d = s.derived()
    n = 200_000
    _electrons_at(s, eps, n, seed=4)
    s.step(1)
    c = s.accum()["counters"].astype(float)
    ng = d["ng"]
    v = math.sqrt(eps * 2 * QE / ME)
    nus = [ng * O.sigma_e(m, eps) * v for m in range(3)]
    for k, nu in zip((6, 7, 8), nus):
        p = d["pmax_e"] * nu / d["numax_e"]
        assert abs(c[k] - n * p) <= 4 * math.sqrt(n * p * (1 - p)) + 1, (k, c[k], n * p)


def test_table_nodes_equal_closed_forms():
    s = _sim(pressure_pa=10.0)
    d = s.derived()
    Fe, Fi = s.table(0), s.table(1)
    rng = np.random.default_rng(5)
    for k in rng.integers(1, XS, 200):
        eps = k / 100.0
        v = math.sqrt(eps * d["spd2_e"])
        nu = [d["ng"] * O.sigma_e(m, eps) * v for m in range(3)]
        assert abs(Fe[k, 2] * d["numax_e"] - sum(nu)) <= 1e-13 * sum(nu) + 1e-300
        assert abs(Fe[k, 0] * d["numax_e"] - nu[0]) <= 1e-13 * nu[0]
        nui = [d["ng"] * O.sigma_g_i(m, eps, d["spd2_rel"]) for m in range(2)]
        assert abs(Fi[k, 1] * d["numax_i"] - sum(nui)) <= 1e-13 * sum(nui)
    assert Fe[:, 2].max() == 1.0 and Fi[:, 1].max() == 1.0
    # thresholds of §3.1: no inelastic process below 11.55 / 15.76 eV
    assert np.all(Fe[:1156, 1] == Fe[:1156, 0]) and np.all(Fe[:1577, 2] == Fe[:1577, 1])
    # P_coll of §3.5
    assert d["pmax_e"] == 1.0 - math.exp(-d["numax_e"] * d["dt"])


def test_ion_maxwellian_relaxation():
    """Cold ions in a field-free gas relax to the gas Maxwellian at T_g."""
    s = _sim(pressure_pa=100.0, steps_per_rf=10, gap_m=1.0)
    n = 20000
    x = np.random.default_rng(6).uniform(0.45, 0.55, n)
    z = np.zeros(n)
    s.set_particles(1, x, z, z, z, np.arange(n, dtype=np.uint32), n)
    s.step(300)
    p = s.particles(1)
    sig = math.sqrt(KB * 300.0 / MI)
    for c in ("vx", "vy", "vz"):
        assert stats.kstest(p[c] / sig, "norm").pvalue > 1e-3, c
    T = MI * np.mean(p["vx"] ** 2 + p["vy"] ** 2 + p["vz"] ** 2) / (3 * KB)
    assert abs(T / 300.0 - 1) < 5 * math.sqrt(2 / (3 * n))
    c = s.accum()["counters"]
    assert c[9] > 0 and c[10] > 0  # both ion processes occurred


def test_at_most_one_event_per_particle_step():
    """§3.1: one collision at most per particle and step: real events <= candidates <= N."""
    s = _sim(pressure_pa=200.0)
    n = 50000
    _electrons_at(s, 50.0, n, seed=7)
    s.step(1)
    c = s.accum()["counters"]
    assert c[6] + c[7] + c[8] <= c[11] <= n
