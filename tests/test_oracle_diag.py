"""Pins of the oracle's diagnostics (§3.1 EEPF normalisation, §3.4 FEDF normalisation and ion
flux, §3.5 criteria) and whole-loop invariants of the cycle of §2."""
import math

import numpy as np

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
