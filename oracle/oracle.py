"""ctypes wrapper of the plain FP64 CPU oracle (pic_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py``.  The product path never imports this module.

The oracle follows the six-step PIC/MCC cycle of §2 (steps 1-6) of Vass, Palla & Hartmann,
arXiv 2109.04469, in plain loops over particles in array order.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pic_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")

XS_NODES = 100001
N_COUNTERS = 16
COUNTER_NAMES = (
    "e_abs_left", "e_abs_right", "i_abs_left", "i_abs_right", "e_reflected", "see_emitted",
    "e_elastic", "e_excitation", "e_ionization", "i_isotropic", "i_charge_transfer",
    "e_candidates", "i_candidates", "eepf_samples", "eepf_esum_fx20", "births_dropped",
)
DERIVED_NAMES = (
    "dt", "dx", "ng", "numax_e", "numax_i", "pmax_e", "pmax_i", "efac", "rfac", "qm_dt_e",
    "qm_dt_i", "emfac_e", "spd2_e", "emfac_rel", "spd2_rel", "sig_e", "sig_i", "v_see", "mr2",
)

_lock = threading.Lock()
_lib = None


class OrcParams(C.Structure):
    _fields_ = [
        ("gap_m", C.c_double), ("pressure_pa", C.c_double), ("gas_temp_k", C.c_double),
        ("v_rf_amp_v", C.c_double), ("f_rf_hz", C.c_double),
        ("steps_per_rf", C.c_int32), ("n_cells", C.c_int32),
        ("weight", C.c_double), ("refl_e", C.c_double), ("gamma_see", C.c_double),
        ("area_m2", C.c_double), ("init_te_ev", C.c_double), ("see_energy_ev", C.c_double),
        ("init_per_species", C.c_int64), ("capacity_per_species", C.c_int64),
        ("seed", C.c_uint64), ("instance", C.c_uint32),
        ("eepf_bins", C.c_int32), ("eepf_emax_ev", C.c_double),
        ("fedf_bins", C.c_int32), ("fedf_emax_ev", C.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile pic_oracle.c with gcc (no FMA contraction) into oracle/_build/."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.c_void_p
            dp = C.POINTER(C.c_double)
            L.orc_create.restype = P
            L.orc_create.argtypes = [C.POINTER(OrcParams)]
            L.orc_destroy.argtypes = [P]
            L.orc_step.restype = C.c_int
            L.orc_step.argtypes = [P, C.c_int64]
            L.orc_count.restype = C.c_int64
            L.orc_count.argtypes = [P, C.c_int]
            L.orc_next_id.restype = C.c_uint32
            L.orc_next_id.argtypes = [P, C.c_int]
            L.orc_step_index.restype = C.c_uint32
            L.orc_step_index.argtypes = [P]
            L.orc_status.restype = C.c_int
            L.orc_status.argtypes = [P]
            L.orc_get_particles.restype = C.c_int64
            L.orc_get_particles.argtypes = [P, C.c_int, P, P, P, P, P, C.c_int64]
            L.orc_set_particles.restype = C.c_int
            L.orc_set_particles.argtypes = [P, C.c_int, P, P, P, P, P, C.c_int64, C.c_uint32]
            L.orc_set_step.argtypes = [P, C.c_uint32]
            L.orc_solve_field.argtypes = [P]
            L.orc_get_grid.argtypes = [P, P, P, P, P]
            L.orc_get_accum.restype = C.c_int64
            L.orc_get_accum.argtypes = [P, P, P, P, P, P, P]
            L.orc_reset_averages.argtypes = [P]
            L.orc_get_derived.argtypes = [P, P]
            L.orc_override_table.argtypes = [P, C.c_int, P, C.c_double]
            L.orc_get_table.argtypes = [P, C.c_int, P]
            L.orc_set_counts.argtypes = [P, P, P]
            L.orc_thomas_phi.argtypes = [P, C.c_double, P]
            L.orc_philox4x32_10.argtypes = [P, P, P]
            L.orc_log.restype = C.c_double
            L.orc_log.argtypes = [C.c_double]
            L.orc_uniform_pair.argtypes = [C.c_uint64, C.c_uint32, C.c_int, C.c_int,
                                           C.c_uint32, C.c_uint32, C.c_uint32, dp]
            L.orc_sigma_e.restype = C.c_double
            L.orc_sigma_e.argtypes = [C.c_int, C.c_double]
            L.orc_sigma_g_i.restype = C.c_double
            L.orc_sigma_g_i.argtypes = [C.c_int, C.c_double, C.c_double]
            L.orc_sample_dirs.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_int64, P]
            L.orc_sample_gauss.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_int64, P]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.c_void_p)


DEFAULTS = dict(
    gas_temp_k=300.0, f_rf_hz=13.56e6, area_m2=1e-4, init_te_ev=3.0, see_energy_ev=1.0,
    refl_e=0.0, gamma_see=0.0, seed=1, instance=0, eepf_bins=500, eepf_emax_ev=50.0,
    fedf_bins=500, fedf_emax_ev=500.0,
)


def make_params(cfg: dict) -> OrcParams:
    d = dict(DEFAULTS)
    d.update(cfg)
    p = OrcParams()
    for name, _ in OrcParams._fields_:
        setattr(p, name, d[name])
    return p


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return o


def own_log(x: float) -> float:
    return lib().orc_log(float(x))


def uniform_pair(seed, instance, species, purpose, pid, step, block):
    out = (C.c_double * 2)()
    lib().orc_uniform_pair(seed, instance, species, purpose, pid, step, block, out)
    return out[0], out[1]


def sigma_e(proc: int, eps: float) -> float:
    return lib().orc_sigma_e(proc, eps)


def sigma_g_i(proc: int, eps: float, spd2_rel: float) -> float:
    return lib().orc_sigma_g_i(proc, eps, spd2_rel)


def sample_dirs(n, seed=1, instance=0, id0=0) -> np.ndarray:
    out = np.zeros((n, 3))
    lib().orc_sample_dirs(seed, instance, id0, n, _ptr(out))
    return out


def sample_gauss(n, seed=1, instance=0, id0=0) -> np.ndarray:
    out = np.zeros((n, 2))
    lib().orc_sample_gauss(seed, instance, id0, n, _ptr(out))
    return out


class OracleSim:
    """One oracle simulation (FP64, single thread)."""

    def __init__(self, cfg: dict):
        self.cfg = dict(DEFAULTS)
        self.cfg.update(cfg)
        self._p = make_params(self.cfg)
        self._h = lib().orc_create(C.byref(self._p))
        if not self._h:
            raise ValueError("oracle rejected the parameters")
        self.nx = self.cfg["n_cells"] + 1

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def step(self, n: int = 1) -> int:
        return lib().orc_step(self._h, int(n))

    def count(self, s: int) -> int:
        return lib().orc_count(self._h, s)

    def next_id(self, s: int) -> int:
        return lib().orc_next_id(self._h, s)

    @property
    def step_index(self) -> int:
        return lib().orc_step_index(self._h)

    @property
    def status(self) -> int:
        return lib().orc_status(self._h)

    def set_step(self, n: int):
        lib().orc_set_step(self._h, n)

    def particles(self, s: int) -> dict:
        n = self.count(s)
        out = {k: np.zeros(n) for k in ("x", "vx", "vy", "vz")}
        out["id"] = np.zeros(n, dtype=np.uint32)
        lib().orc_get_particles(self._h, s, _ptr(out["x"]), _ptr(out["vx"]), _ptr(out["vy"]),
                                _ptr(out["vz"]), _ptr(out["id"]), n)
        return out

    def set_particles(self, s: int, x, vx, vy, vz, ids, next_id: int):
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (x, vx, vy, vz)]
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
        rc = lib().orc_set_particles(self._h, s, *[_ptr(a) for a in arrs], _ptr(ids),
                                     len(ids), next_id)
        if rc != 0:
            raise ValueError("capacity exceeded")

    def set_counts(self, Ce, Ci):
        Ce = np.ascontiguousarray(Ce, dtype=np.int64)
        Ci = np.ascontiguousarray(Ci, dtype=np.int64)
        assert Ce.shape == (self.nx,) and Ci.shape == (self.nx,)
        lib().orc_set_counts(self._h, _ptr(Ce), _ptr(Ci))

    def thomas_phi(self, V: float) -> np.ndarray:
        """Potential of the current counts by the Thomas algorithm (pin of the field solve)."""
        out = np.zeros(self.nx)
        lib().orc_thomas_phi(self._h, float(V), _ptr(out))
        return out

    def solve_field(self):
        lib().orc_solve_field(self._h)

    def grid(self) -> dict:
        g = dict(Ce=np.zeros(self.nx, np.int64), Ci=np.zeros(self.nx, np.int64),
                 phi=np.zeros(self.nx), E=np.zeros(self.nx))
        lib().orc_get_grid(self._h, _ptr(g["Ce"]), _ptr(g["Ci"]), _ptr(g["phi"]), _ptr(g["E"]))
        return g

    def accum(self) -> dict:
        c = self.cfg
        a = dict(acc_e=np.zeros(self.nx), acc_i=np.zeros(self.nx),
                 eepf=np.zeros(c["eepf_bins"], np.uint64),
                 fedf_e=np.zeros(c["fedf_bins"], np.uint64),
                 fedf_i=np.zeros(c["fedf_bins"], np.uint64),
                 counters=np.zeros(N_COUNTERS, np.uint64))
        a["steps"] = lib().orc_get_accum(self._h, _ptr(a["acc_e"]), _ptr(a["acc_i"]),
                                         _ptr(a["eepf"]), _ptr(a["fedf_e"]), _ptr(a["fedf_i"]),
                                         _ptr(a["counters"]))
        return a

    def reset_averages(self):
        lib().orc_reset_averages(self._h)

    def derived(self) -> dict:
        out = np.zeros(len(DERIVED_NAMES))
        lib().orc_get_derived(self._h, _ptr(out))
        return dict(zip(DERIVED_NAMES, out.tolist()))

    def table(self, s: int) -> np.ndarray:
        F = np.zeros((XS_NODES, 4))
        lib().orc_get_table(self._h, s, _ptr(F))
        return F

    def override_table(self, s: int, F: np.ndarray, numax: float):
        F = np.ascontiguousarray(F, dtype=np.float64)
        assert F.shape == (XS_NODES, 4)
        lib().orc_override_table(self._h, s, _ptr(F), float(numax))

    def diag(self) -> dict:
        """Physical diagnostics from the raw accumulators (§3.1, §3.4, §3.5; C-18..C-21)."""
        pe = self.particles(0)
        return derived_diagnostics(self.cfg, self.accum(), self.derived(),
                                   self.count(0), self.count(1), pe["vx"], pe["vy"], pe["vz"])


# physical constants (CODATA 2018) used by the derived diagnostics
_QE, _ME, _EPS0 = 1.602176634e-19, 9.1093837015e-31, 8.8541878128e-12
# floor of the runaway-energy threshold (eV) of the instability flag, for undriven runs
RUNAWAY_FLOOR_EV = 100.0


def derived_diagnostics(cfg, acc, der, n_e, n_i, vx_e, vy_e=None, vz_e=None) -> dict:
    """Densities, EEPF, FEDFs, ion flux and the stability/accuracy criteria of §3.5, and the
    instability flag: ω_pe Δt above the leapfrog bound 2 (§3.5), or a runaway in which the
    electrons' mean kinetic energy exceeds the largest energy the drive can give them,
    e |V_rf| (at least RUNAWAY_FLOOR_EV)."""
    nc = cfg["n_cells"]
    steps = acc["steps"]
    W, A, dx, dt = cfg["weight"], cfg["area_m2"], der["dx"], der["dt"]
    out = dict(steps=steps, n_e_count=n_e, n_i_count=n_i, counters=acc["counters"])
    dens_fac = W / ((A * dx) * 4294967296.0)
    vol = np.ones(nc + 1)
    vol[0] = vol[-1] = 0.5  # C-5: half cells at the electrodes
    for s in ("e", "i"):
        out[f"n_{s}"] = (acc[f"acc_{s}"] / max(steps, 1)) * dens_fac / vol
    # EEPF, normalised so that sum sqrt(eps) f d eps = 1 (§3.1)
    bins, emax = cfg["eepf_bins"], cfg["eepf_emax_ev"]
    de = emax / bins
    centers = (np.arange(bins) + 0.5) * de
    h = acc["eepf"].astype(np.float64)
    tot = h.sum()
    out["eepf_energy"] = centers
    out["eepf"] = h / (np.sqrt(centers) * de * tot) if tot > 0 else np.zeros(bins)
    # flux-energy distributions, normalised so that sum f d eps = 1 (§3.4)
    fb, fmax = cfg["fedf_bins"], cfg["fedf_emax_ev"]
    fde = fmax / fb
    out["fedf_energy"] = (np.arange(fb) + 0.5) * fde
    for s in ("e", "i"):
        hf = acc[f"fedf_{s}"].astype(np.float64)
        out[f"fedf_{s}"] = hf / (fde * hf.sum()) if hf.sum() > 0 else np.zeros(fb)
    cn = acc["counters"].astype(np.float64)
    T = steps * dt
    if T > 0:
        gl, gr = cn[2] * W / (A * T), cn[3] * W / (A * T)
    else:
        gl = gr = 0.0
    out["ion_flux_left"], out["ion_flux_right"] = gl, gr
    out["ion_flux"] = 0.5 * (gl + gr)  # C-21
    # centre density and temperature (C-19)
    xc = 0.5 * nc
    j = int(np.floor(xc))
    f = xc - j
    ne = out["n_e"]
    n_c = (1 - f) * ne[j] + f * ne[min(j + 1, nc)]
    mean_eps = (cn[14] / 1048576.0) / cn[13] if cn[13] > 0 else 0.0
    te_ev = (2.0 / 3.0) * mean_eps
    out["n_e_center"], out["te_center_ev"] = n_c, te_ev
    wpe = np.sqrt(max(n_c, 0.0) * _QE * _QE / (_EPS0 * _ME))
    out["omega_pe_dt"] = wpe * dt
    out["omega_pe_dt_max"] = np.sqrt(max(ne.max(), 0.0) * _QE * _QE / (_EPS0 * _ME)) * dt
    out["p_coll_e"], out["p_coll_i"] = der["pmax_e"], der["pmax_i"]
    lam = np.sqrt(_EPS0 * te_ev / (n_c * _QE)) if n_c > 0 and te_ev > 0 else float("inf")
    out["lambda_d"] = lam
    out["dx_over_lambda_d"] = dx / lam
    out["n_debye"] = n_c * A * lam / W if np.isfinite(lam) else float("inf")  # C-20
    out["cfl_max"] = (np.abs(vx_e).max() * dt / dx) if len(vx_e) else 0.0
    if vy_e is not None and len(vx_e):
        v2 = np.asarray(vx_e) ** 2 + np.asarray(vy_e) ** 2 + np.asarray(vz_e) ** 2
        out["mean_energy_e_ev"] = float(np.mean(v2)) * (0.5 * _ME / _QE)
    else:
        out["mean_energy_e_ev"] = 0.0
    runaway = max(abs(cfg["v_rf_amp_v"]), RUNAWAY_FLOOR_EV)
    out["unstable"] = bool(out["omega_pe_dt_max"] > 2.0 or
                           not (out["mean_energy_e_ev"] <= runaway))
    return out
