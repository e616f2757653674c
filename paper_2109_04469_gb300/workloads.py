"""Named synthetic workloads (parameter sets only; no arithmetic of the method).

The physical setting follows §2 and Table 1 of arXiv 2109.04469 (argon, 13.56 MHz,
300 K, 1 cm^2 nominal electrode area).  The sizes are the synthetic stand-ins for the
paper's base cases: the paper's Phelps cross sections and converged runs are not
available, so the initial state is a uniform Maxwellian load (reading C-22).
"""
from __future__ import annotations

COMMON = dict(
    gas_temp_k=300.0, f_rf_hz=13.56e6, area_m2=1e-4, init_te_ev=3.0, see_energy_ev=1.0,
    seed=1, instance=0, eepf_bins=500, eepf_emax_ev=50.0, fedf_bins=500, fedf_emax_ev=500.0,
)

# 2.5 cm gap, 128 cells, 5 Pa, 150 V, dt = T_RF/1000, 1e4 + 1e4 superparticles,
# W = 2.5e5 (initial density 1e15 m^-3), R = 0, gamma = 0; 10 RF cycles.
CCP_5PA_150V_128C = dict(
    COMMON, gap_m=0.025, pressure_pa=5.0, v_rf_amp_v=150.0, steps_per_rf=1000, n_cells=128,
    weight=2.5e5, refl_e=0.0, gamma_see=0.0, init_per_species=10_000,
    capacity_per_species=65_536, rf_cycles=10,
)

# 2.5 cm gap, 400 cells, 1 Pa, 300 V, dt = T_RF/3000, 2e6 superparticles per species,
# W = 1250 (initial density 1e15 m^-3), R = 0.2, gamma = 0.1.
CCP_1PA_300V_400C = dict(
    COMMON, gap_m=0.025, pressure_pa=1.0, v_rf_amp_v=300.0, steps_per_rf=3000, n_cells=400,
    weight=1250.0, refl_e=0.2, gamma_see=0.1, init_per_species=2_000_000,
    capacity_per_species=3_000_000, rf_cycles=500,
)

# 3 cm gap, 1024 cells, 20 Pa, 500 V, dt = T_RF/4000, 5e7 superparticles per species,
# W chosen for an initial density of 1e16 m^-3; R = 0.2, gamma = 0.2.
CCP_20PA_500V_1024C = dict(
    COMMON, gap_m=0.03, pressure_pa=20.0, v_rf_amp_v=500.0, steps_per_rf=4000, n_cells=1024,
    weight=600.0, refl_e=0.2, gamma_see=0.2, init_per_species=50_000_000,
    capacity_per_species=60_000_000, rf_cycles=200,
)

WORKLOADS = {
    "ccp_5pa_150v_128c": CCP_5PA_150V_128C,
    "ccp_1pa_300v_400c": CCP_1PA_300V_400C,
    "ccp_20pa_500v_1024c": CCP_20PA_500V_1024C,
}


def params(name: str, **overrides) -> dict:
    """The C-ABI parameter dict of a named workload (run-length keys removed)."""
    d = dict(WORKLOADS[name])
    d.pop("rf_cycles", None)
    d.update(overrides)
    return d
