"""pic_diag on hand-set states whose answers are fixed by construction (§3.4 ion flux, §3.5
Courant number, centre density and temperature, Debye length, ω_pe Δt, the instability flag),
and failure detection through the C-ABI without a GPU fault: a NaN velocity injected through
pic_set_particles is reported as PIC_ERR_NONFINITE by the next step's sync, in both
precisions, and the context keeps working.

The injected NaN is safe by construction: every index the kernels form from a position or an
energy is clamped or range-tested before use (cell indices clamped to [0, N_c - 1], table,
EEPF and FEDF bins guarded by an ordered comparison that fails for NaN), so a NaN particle
only carries NaN arithmetic and sets the sticky status.

FP64 handles follow the oracle's formulas with the same constants; FP32 handles store the
state in FP32 cell units, so their diagnostics agree to FP32 rounding (relative 1e-6).
"""
import math

import numpy as np
import pytest

from paper_2109_04469_gb300 import pic

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

QE, ME, EPS0 = 1.602176634e-19, 9.1093837015e-31, 8.8541878128e-12
PREC = [(pic.PIC_FP64, 1e-12), (pic.PIC_FP32, 1e-6)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2109_04469_gb300 import build as B

    B.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _quiet(prec, **kw):
    cfg = dict(gap_m=0.025, pressure_pa=0.0, v_rf_amp_v=0.0, steps_per_rf=1000, n_cells=64,
               weight=1e3, init_per_species=0, capacity_per_species=100_000, f_rf_hz=13.56e6,
               refl_e=0.0, gamma_see=0.0, precision=prec)
    cfg.update(kw)
    return pic.Simulation(cfg), cfg


def _put(sim, sp, x, vx=None, vy=None, vz=None):
    n = len(x)
    z = np.zeros(n)
    sim.set_particles(sp, np.asarray(x, float), z if vx is None else vx,
                      z if vy is None else vy, z if vz is None else vz,
                      np.arange(n, dtype=np.uint32), n)


@pytest.mark.parametrize("prec,tol", PREC)
def test_ion_flux_of_hand_set_impacts(prec, tol):
    sim, c = _quiet(prec)
    L, nc, W, A = c["gap_m"], c["n_cells"], c["weight"], 1e-4
    dt = 1.0 / (c["f_rf_hz"] * c["steps_per_rf"])
    dx = L / nc
    K, M, stay = 37, 53, 100
    x = np.concatenate([np.full(K, 0.2 * dx), np.full(M, L - 0.2 * dx),
                        np.linspace(0.4 * L, 0.6 * L, stay)])
    vx = np.concatenate([np.full(K, -0.5 * dx / dt), np.full(M, 0.5 * dx / dt), np.zeros(stay)])
    _put(sim, 1, x, vx)
    sim.step(5)
    d = sim.diag()
    assert d["steps_averaged"] == 5 and d["count_i"] == stay
    assert int(d["counters"][2]) == K and int(d["counters"][3]) == M
    T = 5 * dt
    assert abs(d["ion_flux_left"] / (K * W / (A * T)) - 1) < 1e-13
    assert abs(d["ion_flux_right"] / (M * W / (A * T)) - 1) < 1e-13
    assert abs(d["ion_flux"] / (0.5 * (K + M) * W / (A * T)) - 1) < 1e-13
    sim.close()


@pytest.mark.parametrize("prec,tol", PREC)
def test_courant_number_of_hand_set_velocities(prec, tol):
    sim, c = _quiet(prec, n_cells=50)
    L, nc = c["gap_m"], c["n_cells"]
    dt = 1.0 / (c["f_rf_hz"] * c["steps_per_rf"])
    x = np.linspace(0.3 * L, 0.7 * L, 7)
    _put(sim, 0, x, np.array([1e5, -3.7e6, 2e6, 0.0, 5e5, -1e6, 3.6e6]))
    _put(sim, 1, x)
    want = 3.7e6 * dt / (L / nc)
    assert abs(sim.diag()["cfl_max"] / want - 1) < tol
    sim.step(1)
    assert abs(sim.diag()["cfl_max"] / want - 1) < tol
    sim.close()


@pytest.mark.parametrize("prec,tol", PREC)
def test_centre_density_temperature_and_debye_criteria(prec, tol):
    """65 cells, 8 electrons per cell left of L/2 and 16 from cell 32 on, at offsets (2i+1)/2k:
    n(L/2) = 14 W/(A Δx); vx = 0 and 3 eV each: k T_e = 2 eV (see the oracle's pin)."""
    nc = 65
    sim, c = _quiet(prec, n_cells=nc, weight=1e5, eepf_bins=60, eepf_emax_ev=30.0)
    L, W, A = c["gap_m"], c["weight"], 1e-4
    dt = 1.0 / (c["f_rf_hz"] * c["steps_per_rf"])
    dx = L / nc
    x = np.concatenate([(j + (2 * np.arange(8 if j < 32 else 16) + 1) / (16 if j < 32 else 32))
                        * dx for j in range(nc)])
    rng = np.random.default_rng(7)
    ang = rng.uniform(0, 2 * np.pi, len(x))
    sp = math.sqrt(2 * 3.0 * QE / ME)
    _put(sim, 0, x, np.zeros(len(x)), sp * np.cos(ang), sp * np.sin(ang))
    _put(sim, 1, x)
    sim.step(1)
    d = sim.diag()
    unit = W / (A * dx)
    n_c = 14.0 * unit
    assert abs(d["n_e_center"] / n_c - 1) < max(tol, 1e-8)
    assert int(d["counters"][13]) == 16
    assert abs(d["te_center_ev"] - 2.0) < 2.0 * max(tol, 1e-12)
    lam = math.sqrt(EPS0 * 2.0 / (n_c * QE))
    assert abs(d["lambda_d"] / lam - 1) < max(tol, 1e-8)
    assert abs(d["n_debye"] / (n_c * A * lam / W) - 1) < max(tol, 1e-8)
    assert abs(d["omega_pe_dt"] / (math.sqrt(n_c * QE**2 / (EPS0 * ME)) * dt) - 1) < max(tol, 1e-8)
    assert abs(d["mean_energy_e_ev"] - 3.0) < 3.0 * max(tol, 1e-12)
    assert d["return_code"] == 0
    sim.close()


@pytest.mark.parametrize("prec,tol", PREC)
@pytest.mark.parametrize("wdt,want", [(1.5, 0), (2.5, 1)])
def test_unstable_warning_from_omega_pe_dt(prec, tol, wdt, want):
    """§3.5: a quiet neutral load with ω_pe Δt = 2.5 makes pic_diag return PIC_WARN_UNSTABLE
    (1); at 1.5 it returns PIC_OK."""
    nc, L, A, f, Nt = 64, 0.025, 1e-4, 13.56e6, 1000
    dt = 1.0 / (f * Nt)
    dx = L / nc
    W = (wdt / dt) ** 2 * EPS0 * ME / QE**2 * A * dx / 8
    sim, _ = _quiet(prec, n_cells=nc, weight=W)
    x = np.concatenate([(j + (2 * np.arange(8) + 1) / 16) * dx for j in range(nc)])
    _put(sim, 0, x)
    _put(sim, 1, x)
    sim.step(1)
    d = sim.diag()
    assert abs(d["omega_pe_dt"] / wdt - 1) < max(tol, 1e-8)
    assert d["return_code"] == want
    sim.close()


@pytest.mark.parametrize("prec,tol", PREC)
@pytest.mark.parametrize("eps,vrf,want", [(50.0, 0.0, 0), (150.0, 0.0, 1), (400.0, 300.0, 1)])
def test_unstable_warning_from_runaway_energy(prec, tol, eps, vrf, want):
    """A mean electron energy above max(e |V_rf|, 100 eV) makes pic_diag return
    PIC_WARN_UNSTABLE."""
    sim, c = _quiet(prec, v_rf_amp_v=vrf, steps_per_rf=100000)
    L = c["gap_m"]
    n = 2000
    rng = np.random.default_rng(11)
    x = rng.uniform(0.45 * L, 0.55 * L, n)
    dvec = rng.normal(size=(n, 3))
    dvec /= np.linalg.norm(dvec, axis=1, keepdims=True)
    v = dvec * math.sqrt(2 * eps * QE / ME)
    _put(sim, 0, x, v[:, 0], v[:, 1], v[:, 2])
    _put(sim, 1, x)
    sim.step(1)
    d = sim.diag()
    assert abs(d["mean_energy_e_ev"] / eps - 1) < 1e-2
    assert d["return_code"] == want
    sim.close()


@pytest.mark.parametrize("prec", [pic.PIC_FP64, pic.PIC_FP32])
def test_nan_velocity_is_reported_as_nonfinite(prec):
    """Failure detection without a fault: one electron of 5000 is given vx = NaN through
    pic_set_particles; the particle pass flags it, pic_sync (and pic_step, pic_diag) then
    return PIC_ERR_NONFINITE, and the context stays usable."""
    sim, c = _quiet(prec, v_rf_amp_v=150.0, pressure_pa=5.0)
    L = c["gap_m"]
    n = 5000
    rng = np.random.default_rng(3)
    x = rng.uniform(0.1 * L, 0.9 * L, n)
    v = rng.normal(0, 1e6, (3, n))
    v[0, 1234] = np.nan
    _put(sim, 0, x, v[0], v[1], v[2])
    _put(sim, 1, x)
    sim.step(3)
    assert sim.status() == -4
    with pytest.raises(pic.PicError) as e:
        sim.sync()
    assert e.value.code == -4
    with pytest.raises(pic.PicError) as e:
        sim.diag()
    assert e.value.code == -4
    sim.close()
    # the context keeps working: a fresh handle steps cleanly
    ok, _ = _quiet(prec, v_rf_amp_v=150.0, pressure_pa=5.0, init_per_species=2000)
    ok.step(5)
    assert ok.sync() == 0
    ok.close()
