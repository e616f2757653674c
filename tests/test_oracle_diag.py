"""Pins of the oracle's diagnostics (§3.1 EEPF normalisation, §3.4 FEDF normalisation and ion
flux, §3.5 criteria) and whole-loop invariants of the cycle of §2."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2109_04469_gb300 import workloads

QE, ME, EPS0 = 1.602176634e-19, 9.1093837015e-31, 8.8541878128e-12


def test_eepf_of_a_maxwellian_is_exponential():
    """A Maxwellian at T has EEPF proportional to exp(-eps/T) (§3.1 normalisation)."""
    T = 3.0
    cfg = dict(gap_m=0.025, pressure_pa=0.0, v_rf_amp_v=0.0, steps_per_rf=1000, n_cells=8,
               weight=0.0, init_per_species=0, capacity_per_species=400_000,
               f_rf_hz=1e15, eepf_bins=300, eepf_emax_ev=30.0)
    s = O.OracleSim(cfg)
    n = 400_000
    rng = np.random.default_rng(0)
    v = rng.normal(0, math.sqrt(T * QE / ME), (n, 3))
    x = 0.0125 + rng.uniform(-0.4, 0.4, n) * (0.025 / 8)  # inside the centre window
    s.set_particles(0, x, v[:, 0], v[:, 1], v[:, 2], np.arange(n, dtype=np.uint32), n)
    s.step(1)
    d = s.diag()
    e, f = d["eepf_energy"], d["eepf"]
    de = e[1] - e[0]
    assert abs(np.sum(np.sqrt(e) * f) * de - 1.0) < 1e-12
    sel = (e > 1.0) & (e < 15.0)
    slope = np.polyfit(e[sel], np.log(f[sel]), 1, w=np.sqrt(f[sel]))[0]
    assert abs(slope * T + 1.0) < 0.03
    assert abs(d["te_center_ev"] / T - 1) < 0.01
    assert int(d["counters"][13]) == n


def _short_cfg0_run(steps, **over):
    cfg = workloads.params("ccp_5pa_150v_128c", **over)
    s = O.OracleSim(cfg)
    s.step(steps)
    return s


def test_whole_cycle_invariants():
    """Charge counts always equal the populations x 2^32 (deposit at x^{n+1} plus births),
    ids stay unique and the id counter advances by the births."""
    s = O.OracleSim(workloads.params("ccp_5pa_150v_128c", refl_e=0.3, gamma_see=0.2))
    for _ in range(6):
        s.step(50)
        g = s.grid()
        for sp, key in ((0, "Ce"), (1, "Ci")):
            p = s.particles(sp)
            assert int(g[key].sum()) == s.count(sp) * 2**32
            assert len(np.unique(p["id"])) == len(p["id"])
            assert np.all((p["x"] >= 0) & (p["x"] <= 0.025))
    c = s.accum()["counters"]
    births_e = int(c[8] + c[5])
    assert s.next_id(0) == 10_000 + births_e
    assert s.next_id(1) == 10_000 + int(c[8])
    lost_e = int(c[0] + c[1])
    assert s.count(0) == 10_000 + births_e - lost_e
    assert s.count(1) == 10_000 + int(c[8]) - int(c[2] + c[3])
    assert s.status == 0


def test_diagnostics_normalisations_and_criteria():
    s = _short_cfg0_run(600, gamma_see=0.1)
    d = s.diag()
    e, f = d["eepf_energy"], d["eepf"]
    assert abs(np.sum(np.sqrt(e) * f) * (e[1] - e[0]) - 1.0) < 1e-12
    for sp in ("e", "i"):
        fe = d[f"fedf_{sp}"]
        assert abs(np.sum(fe) * (d["fedf_energy"][1] - d["fedf_energy"][0]) - 1.0) < 1e-12
    # the time-averaged density integrates to the time-averaged population (C-5 volumes)
    dx = 0.025 / 128
    w = np.full(129, dx)
    w[0] = w[-1] = dx / 2
    acc = s.accum()
    mean_pop_e = acc["acc_e"].sum() / 2**32 / acc["steps"]
    assert abs(np.sum(d["n_e"] * w) * 1e-4 / 2.5e5 - mean_pop_e) < 1e-9 * mean_pop_e
    # criteria of §3.5 from the centre density / temperature (C-19, C-20)
    wpe = math.sqrt(d["n_e_center"] * QE * QE / (EPS0 * ME))
    assert abs(d["omega_pe_dt"] - wpe * s.derived()["dt"]) < 1e-12 * d["omega_pe_dt"]
    lam = math.sqrt(EPS0 * d["te_center_ev"] / (d["n_e_center"] * QE))
    assert abs(d["lambda_d"] / lam - 1) < 1e-12
    assert abs(d["n_debye"] - d["n_e_center"] * 1e-4 * lam / 2.5e5) < 1e-9 * d["n_debye"]
    assert 0 < d["p_coll_e"] < 0.06 and 0 < d["p_coll_i"] < 0.01
    assert 0.05 < d["omega_pe_dt"] < 0.3  # ~0.13 expected at 1e15 m^-3


# ---------------------------------------------------------------------------------------
# Diagnostics whose answers are fixed by construction: the test sets the populations,
# positions and velocities, so every expected value below follows from those choices and
# the parameters alone (nothing is read back from the oracle's own intermediate results).
def _quiet_sim(**kw):
    cfg = dict(gap_m=0.025, pressure_pa=0.0, v_rf_amp_v=0.0, steps_per_rf=1000, n_cells=64,
               weight=1e3, init_per_species=0, capacity_per_species=100_000,
               f_rf_hz=13.56e6, refl_e=0.0, gamma_see=0.0)
    cfg.update(kw)
    return O.OracleSim(cfg), cfg


def _put(s, sp, x, vx=None, vy=None, vz=None):
    n = len(x)
    z = np.zeros(n)
    s.set_particles(sp, np.asarray(x, float), z if vx is None else vx, z if vy is None else vy,
                    z if vz is None else vz, np.arange(n, dtype=np.uint32), n)


def test_ion_flux_of_hand_set_impacts():
    """Γ of §3.4 (Fig. 11), reading C-21: K ions set to cross x = 0 and M ions set to cross
    x = L within one step give Γ_left = K W / (A T) and Γ_right = M W / (A T) over an averaging
    time T = steps x Δt; Γ is their mean."""
    s, c = _quiet_sim()
    L, nc, W, A = c["gap_m"], c["n_cells"], c["weight"], 1e-4
    dt = 1.0 / (c["f_rf_hz"] * c["steps_per_rf"])
    dx = L / nc
    K, M, stay = 37, 53, 100
    x = np.concatenate([np.full(K, 0.2 * dx), np.full(M, L - 0.2 * dx),
                        np.linspace(0.4 * L, 0.6 * L, stay)])
    vx = np.concatenate([np.full(K, -0.5 * dx / dt), np.full(M, 0.5 * dx / dt), np.zeros(stay)])
    _put(s, 1, x, vx)
    steps = 5
    s.step(steps)
    d = s.diag()
    assert d["steps"] == steps
    assert int(d["counters"][2]) == K and int(d["counters"][3]) == M
    assert s.count(1) == stay
    T = steps * dt
    want_l, want_r = K * W / (A * T), M * W / (A * T)
    assert abs(d["ion_flux_left"] / want_l - 1) < 1e-13
    assert abs(d["ion_flux_right"] / want_r - 1) < 1e-13
    assert abs(d["ion_flux"] / (0.5 * (want_l + want_r)) - 1) < 1e-13


def test_courant_number_of_hand_set_velocities():
    """max |vx| Δt / Δx over the electrons (§3.5): hand-set velocities in a gap with no field
    (ions on the electrons' positions, so ρ = 0, and no drive), before and after one step."""
    s, c = _quiet_sim(n_cells=50)
    L, nc = c["gap_m"], c["n_cells"]
    dt = 1.0 / (c["f_rf_hz"] * c["steps_per_rf"])
    dx = L / nc
    x = np.linspace(0.3 * L, 0.7 * L, 7)
    vx = np.array([1e5, -3.7e6, 2e6, 0.0, 5e5, -1e6, 3.6e6])
    _put(s, 0, x, vx)
    _put(s, 1, x)
    want = 3.7e6 * dt / dx
    assert abs(s.diag()["cfl_max"] / want - 1) < 1e-13
    s.step(1)
    assert np.array_equal(s.particles(0)["vx"], vx)  # no field acted on them
    assert abs(s.diag()["cfl_max"] / want - 1) < 1e-13


def test_centre_density_temperature_and_debye_criteria_closed_form():
    """Readings C-19, C-20 and the criteria of §3.5 on a quiet load whose centre density and
    temperature are known exactly.  65 cells put L/2 half-way between nodes 32 and 33;
    8 electrons per cell left of the centre and 16 from cell 32 on, at offsets (2i+1)/2k of
    a cell, give node densities 8, 12 (node 32) and 16 (node 33 on) x W/(A Δx), hence
    n(L/2) = 14 W/(A Δx).  Electrons have vx = 0 and |v| set for 3 eV each, so they stay put
    (ions on the same positions: no field) and the centre EEPF's mean energy is 3 eV:
    k T_e = 2 eV.  Then λ_D = sqrt(ε0 k T_e / (n e²)), N_D = n A λ_D / W, and
    ω_pe Δt = sqrt(n e² / (ε0 m_e)) Δt (centre) and with the largest node density (peak)."""
    nc = 65
    s, c = _quiet_sim(n_cells=nc, weight=1e5, eepf_bins=60, eepf_emax_ev=30.0)
    L, W, A = c["gap_m"], c["weight"], 1e-4
    dt = 1.0 / (c["f_rf_hz"] * c["steps_per_rf"])
    dx = L / nc
    xs = []
    for j in range(nc):
        k = 8 if j < 32 else 16
        xs.append((j + (2 * np.arange(k) + 1) / (2 * k)) * dx)
    x = np.concatenate(xs)
    rng = np.random.default_rng(7)
    phi_dir = rng.uniform(0, 2 * np.pi, len(x))
    speed = math.sqrt(2 * 3.0 * QE / ME)
    _put(s, 0, x, np.zeros(len(x)), speed * np.cos(phi_dir), speed * np.sin(phi_dir))
    _put(s, 1, x)
    s.step(1)
    d = s.diag()
    unit = W / (A * dx)
    want_node = np.where(np.arange(nc + 1) < 32, 8.0, 16.0) * unit
    want_node[32] = 12.0 * unit
    assert np.max(np.abs(d["n_e"] / want_node - 1)) < 1e-8
    n_c, Te = 14.0 * unit, 2.0
    assert abs(d["n_e_center"] / n_c - 1) < 1e-8
    assert int(d["counters"][13]) == 16  # the 16 electrons of cell 32 are the EEPF window
    assert abs(d["te_center_ev"] - Te) < 1e-12
    lam = math.sqrt(EPS0 * Te / (n_c * QE))
    assert abs(d["lambda_d"] / lam - 1) < 1e-8
    assert abs(d["dx_over_lambda_d"] / (dx / lam) - 1) < 1e-8
    assert abs(d["n_debye"] / (n_c * A * lam / W) - 1) < 1e-8
    assert abs(d["omega_pe_dt"] / (math.sqrt(n_c * QE**2 / (EPS0 * ME)) * dt) - 1) < 1e-8
    assert abs(d["omega_pe_dt_max"] / (math.sqrt(16.0 * unit * QE**2 / (EPS0 * ME)) * dt) - 1) \
        < 1e-8


def _hot_electrons(eps_ev, n=2000, **kw):
    """n electrons with |v| set for eps_ev each (isotropic directions) on ions at the same
    positions (no field), one step taken; returns the diagnostics."""
    s, c = _quiet_sim(**kw)
    L = c["gap_m"]
    rng = np.random.default_rng(11)
    x = rng.uniform(0.45 * L, 0.55 * L, n)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    speed = np.sqrt(2 * np.asarray(eps_ev, float) * QE / ME)
    v = d * (speed[:, None] if np.ndim(speed) else speed)
    _put(s, 0, x, v[:, 0], v[:, 1], v[:, 2])
    _put(s, 1, x)
    s.step(1)
    return s.diag()


def test_mean_electron_energy_of_a_hand_set_population():
    """The runaway check's mean kinetic energy: half the electrons at 5 eV and half at 7 eV
    give 6 eV (a field-free step leaves the speeds unchanged)."""
    eps = np.where(np.arange(2000) % 2 == 0, 5.0, 7.0)
    d = _hot_electrons(eps, steps_per_rf=100000)
    assert abs(d["mean_energy_e_ev"] - 6.0) < 1e-9
    assert not d["unstable"]


@pytest.mark.parametrize("eps,vrf,want", [(50.0, 0.0, False), (150.0, 0.0, True),
                                          (150.0, 300.0, False), (400.0, 300.0, True)])
def test_runaway_energy_flag(eps, vrf, want):
    """A mean electron energy above max(e |V_rf|, 100 eV) flags the run as unstable.  The
    electrons sit in the middle of the gap, where a drive of 300 V does not change their
    energy in one step by more than a fraction of an eV."""
    d = _hot_electrons(eps, v_rf_amp_v=vrf, steps_per_rf=100000)
    assert abs(d["mean_energy_e_ev"] / eps - 1) < 1e-2
    assert d["unstable"] is want


@pytest.mark.parametrize("wdt,want", [(1.5, False), (2.5, True)])
def test_stability_flag_from_omega_pe_dt(wdt, want):
    """§3.5: leapfrog is unstable for ω_pe Δt > 2.  A quiet, neutral, cold load of density
    n = (wdt / Δt)² ε0 m_e / e² (8 electrons per cell on 8 ions per cell) reports that ω_pe Δt
    after one step, and the flag follows it."""
    nc, L, A, f, Nt = 64, 0.025, 1e-4, 13.56e6, 1000
    dt = 1.0 / (f * Nt)
    n = (wdt / dt) ** 2 * EPS0 * ME / QE**2
    dx = L / nc
    W = n * A * dx / 8
    s, c = _quiet_sim(n_cells=nc, weight=W)
    x = np.concatenate([(j + (2 * np.arange(8) + 1) / 16) * dx for j in range(nc)])
    _put(s, 0, x)
    _put(s, 1, x)
    s.step(1)
    d = s.diag()
    assert abs(d["omega_pe_dt"] / wdt - 1) < 1e-8
    assert d["unstable"] is want
