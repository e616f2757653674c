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


def ensemble_members(n: int = 64, seed: int = 2109, rf_cycles: float = 2.0,
                     per_run=(2.5e5, 4.0e6), growth: float = 3.5) -> list[tuple[dict, int]]:
    """A parameter scan in the manner of §3: n uneven FP32 simulations on a Latin hypercube
    over pressure 1-20 Pa (log), voltage 100-500 V, N_t 500-4000 (log), cells 100-800 (log),
    weight giving `per_run` superparticles per simulation (both species, log; a 16x spread at
    the default), R 0-0.7 and gamma 0-0.4.  2.5 cm gap, initial density 1e15 m^-3.  Each entry
    is (parameters, target step index = rf_cycles x N_t): the members run uneven step
    counts.  Capacity is `growth` x the initial population (+4096): the fastest-ionizing
    members grow about 2.4x in their first 45 steps from the uniform load, and 3.5 x 2e6
    stays within the ensemble launch's bound on a member's capacity (about 7.6e6)."""
    import numpy as np

    rng = np.random.default_rng(seed)
    d = 7
    # Latin hypercube: one stratum per member and dimension, strata shuffled per dimension
    u = (np.argsort(rng.random((d, n)), axis=1) + rng.random((d, n))) / n

    def logu(x, a, b):
        return float(np.exp(np.log(a) + x * (np.log(b) - np.log(a))))

    out = []
    gap, dens, area = 0.025, 1e15, COMMON["area_m2"]
    for i in range(n):
        nt = int(round(logu(u[2, i], 500, 4000)))
        cells = int(round(logu(u[3, i], 100, 800)))
        per_species = int(logu(u[4, i], per_run[0], per_run[1]) / 2)
        c = dict(COMMON, gap_m=gap, pressure_pa=logu(u[0, i], 1.0, 20.0),
                 v_rf_amp_v=100.0 + 400.0 * float(u[1, i]), steps_per_rf=nt, n_cells=cells,
                 weight=dens * area * gap / per_species, refl_e=0.7 * float(u[5, i]),
                 gamma_see=0.4 * float(u[6, i]), init_per_species=per_species,
                 capacity_per_species=int(per_species * growth) + 4096, instance=i)
        out.append((c, int(rf_cycles * nt)))
    return out
