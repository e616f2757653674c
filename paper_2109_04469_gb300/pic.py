"""ctypes binding of libpic.so (C-ABI in include/pic.h).

Argument marshalling only: every step of the PIC/MCC cycle (arXiv 2109.04469 §2 steps 1-6)
runs in the library's CUDA kernels.  PyTorch provides the device workspace (one uint8
tensor) and the CUDA stream.  There is no CPU fallback: if the library is missing or no
GPU is present, construction raises.
"""
from __future__ import annotations

import ctypes as C
import os
import re
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libpic.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "pic.h")

PIC_FP64, PIC_FP32 = 0, 1
N_COUNTERS = 16
XS_NODES = 100001
ERRORS = {
    -1: "PIC_ERR_PARAM", -2: "PIC_ERR_CUDA", -3: "PIC_ERR_CAPACITY", -4: "PIC_ERR_NONFINITE",
    -5: "PIC_ERR_WORKSPACE", -6: "PIC_ERR_TIMEOUT", -7: "PIC_ERR_SCRATCH",
    1: "PIC_WARN_UNSTABLE",
}


class PicParams(C.Structure):
    _fields_ = [
        ("gap_m", C.c_double), ("pressure_pa", C.c_double), ("gas_temp_k", C.c_double),
        ("v_rf_amp_v", C.c_double), ("f_rf_hz", C.c_double),
        ("steps_per_rf", C.c_int32), ("n_cells", C.c_int32),
        ("weight", C.c_double), ("refl_e", C.c_double), ("gamma_see", C.c_double),
        ("area_m2", C.c_double), ("init_te_ev", C.c_double), ("see_energy_ev", C.c_double),
        ("init_per_species", C.c_int64), ("capacity_per_species", C.c_int64),
        ("seed", C.c_uint64), ("instance", C.c_uint32), ("precision", C.c_int32),
        ("eepf_bins", C.c_int32), ("eepf_emax_ev", C.c_double),
        ("fedf_bins", C.c_int32), ("fedf_emax_ev", C.c_double),
    ]


_DP = C.POINTER(C.c_double)


class PicDiagOut(C.Structure):
    _fields_ = [
        ("n_x", C.c_int32), ("eepf_bins", C.c_int32), ("fedf_bins", C.c_int32),
        ("n_e", _DP), ("n_i", _DP), ("eepf_energy", _DP), ("eepf", _DP),
        ("fedf_energy", _DP), ("fedf_e", _DP), ("fedf_i", _DP),
        ("counters", C.c_uint64 * N_COUNTERS),
        ("steps_averaged", C.c_int64), ("count_e", C.c_int64), ("count_i", C.c_int64),
        ("ion_flux_left", C.c_double), ("ion_flux_right", C.c_double), ("ion_flux", C.c_double),
        ("n_e_center", C.c_double), ("te_center_ev", C.c_double),
        ("omega_pe_dt", C.c_double), ("omega_pe_dt_max", C.c_double),
        ("p_coll_e", C.c_double), ("p_coll_i", C.c_double), ("cfl_max", C.c_double),
        ("lambda_d", C.c_double), ("dx_over_lambda_d", C.c_double), ("n_debye", C.c_double),
        ("mean_energy_e_ev", C.c_double),
        ("status", C.c_int32),
    ]


# pic_diag_out's scalar fields (everything but the array pointers, their lengths and the
# counters)
_DIAG_SCALARS = tuple(n for n, _ in PicDiagOut._fields_
                      if n not in ("n_e", "n_i", "eepf_energy", "eepf", "fedf_energy", "fedf_e",
                                   "fedf_i", "n_x", "eepf_bins", "fedf_bins", "counters"))


_lock = threading.Lock()
_lib = None


def declared_functions() -> list[str]:
    """Names of the entry points declared in include/pic.h."""
    src = open(HEADER).read()
    return re.findall(r"^\s*(?:int|void|const char\*)\s+(pic_\w+)\s*\(", src, re.M)


def lib() -> C.CDLL:
    """Load libpic.so (raises if it was not built: the product has no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build()")
            L = C.CDLL(LIB_PATH)
            P, i64, u32 = C.c_void_p, C.c_int64, C.c_uint32
            sig = {
                "pic_workspace_bytes": (C.c_int, [C.POINTER(PicParams), C.POINTER(C.c_size_t)]),
                "pic_init": (C.c_int, [C.POINTER(PicParams), P, C.c_size_t, P, C.POINTER(P)]),
                "pic_step": (C.c_int, [P, i64]),
                "pic_sync": (C.c_int, [P]),
                "pic_step_profiled": (C.c_int, [P, i64, P]),
                "pic_diag": (C.c_int, [P, C.POINTER(PicDiagOut)]),
                "pic_get_particles": (C.c_int, [P, C.c_int, P, P, P, P, P, i64, C.POINTER(i64)]),
                "pic_set_particles": (C.c_int, [P, C.c_int, P, P, P, P, P, i64, u32]),
                "pic_counts": (C.c_int, [P, C.POINTER(i64), C.POINTER(i64)]),
                "pic_counts_async": (C.c_int, [P, P]),
                "pic_get_grid": (C.c_int, [P, P, P, P, P]),
                "pic_solve_field": (C.c_int, [P]),
                "pic_get_accum": (C.c_int, [P, P, P, P, P, P, P, C.POINTER(i64)]),
                "pic_reset_averages": (C.c_int, [P]),
                "pic_set_step": (C.c_int, [P, u32]),
                "pic_get_step": (C.c_int, [P, C.POINTER(u32), C.POINTER(u32), C.POINTER(u32)]),
                "pic_override_table": (C.c_int, [P, C.c_int, P, C.c_double]),
                "pic_get_derived": (C.c_int, [P, P]),
                "pic_fp64_rate": (C.c_int, [P, P]),
                "pic_free": (None, [P]),
                "pic_strerror": (C.c_char_p, [C.c_int]),
                "pic_last_cuda_error": (C.c_char_p, []),
                "pic_tc_gemm_bf16": (C.c_int, [P, P, P, C.c_int32, C.c_int32, C.c_int32, P]),
                "pic_mlp_num_params": (C.c_int, []),
                "pic_mlp_workspace_bytes": (C.c_int, [C.c_int32, C.POINTER(C.c_size_t)]),
                "pic_mlp_init": (C.c_int, [C.c_int32, C.c_uint64, P, C.c_size_t, P, C.POINTER(P)]),
                "pic_mlp_get_params": (C.c_int, [P, P]),
                "pic_mlp_set_params": (C.c_int, [P, P]),
                "pic_mlp_forward": (C.c_int, [P, P, C.c_int32, P]),
                "pic_mlp_gradients": (C.c_int, [P, P, P, C.c_int32, P, C.POINTER(C.c_float)]),
                "pic_mlp_train_step": (C.c_int, [P, P, P, C.c_int32, C.c_float, C.POINTER(C.c_float)]),
                "pic_mlp_get_activations": (C.c_int, [P, C.c_int32, C.c_int32, P]),
                "pic_mlp_free": (None, [P]),
                "pic_checkpoint_bytes": (C.c_int, [P, C.POINTER(C.c_size_t)]),
                "pic_checkpoint_save": (C.c_int, [P, P, C.c_size_t]),
                "pic_checkpoint_load": (C.c_int, [P, P, C.c_size_t]),
                "pic_ensemble_workspace_bytes": (C.c_int, [C.c_int, C.POINTER(C.c_size_t)]),
                "pic_ensemble_create": (C.c_int, [P, C.c_int, P, P, C.c_size_t, C.POINTER(P)]),
                "pic_ensemble_step": (C.c_int, [P, i64]),
                "pic_ensemble_sync": (C.c_int, [P]),
                "pic_ensemble_configure": (C.c_int, [P, C.c_int32, C.c_int32, C.c_int32]),
                "pic_ensemble_autotune": (C.c_int, [P, C.c_int32, P]),
                "pic_ensemble_info": (C.c_int, [P, P]),
                "pic_ensemble_free": (None, [P]),
                "pic_selftest_waits": (C.c_int, [P, C.c_size_t, P, P]),
                "pic_field_solve_static": (C.c_int, [P, P, C.c_int32, C.c_double, C.c_double,
                                                     C.c_double, C.c_double, P, P, P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


class PicError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        msg = lib().pic_strerror(code).decode() if _lib else ERRORS.get(code, str(code))
        if _lib and code == -2:
            msg += ": " + lib().pic_last_cuda_error().decode()
        super().__init__(f"{what}: {ERRORS.get(code, code)} ({msg})")


def _check(code: int, what: str, allow_warn: bool = True) -> int:
    if code < 0 or (code > 0 and not allow_warn):
        raise PicError(code, what)
    return code


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.c_void_p)


DEFAULTS = dict(
    gas_temp_k=300.0, f_rf_hz=13.56e6, area_m2=1e-4, init_te_ev=3.0, see_energy_ev=1.0,
    refl_e=0.0, gamma_see=0.0, seed=1, instance=0, precision=PIC_FP64, eepf_bins=500,
    eepf_emax_ev=50.0, fedf_bins=500, fedf_emax_ev=500.0,
)


def make_params(cfg: dict) -> PicParams:
    d = dict(DEFAULTS)
    d.update(cfg)
    p = PicParams()
    for name, _ in PicParams._fields_:
        setattr(p, name, d[name])
    return p


def workspace_bytes(cfg: dict) -> int:
    p = make_params(cfg)
    n = C.c_size_t(0)
    _check(lib().pic_workspace_bytes(C.byref(p), C.byref(n)), "pic_workspace_bytes")
    return n.value


class Simulation:
    """One simulation on the current CUDA device and torch's current stream."""

    def __init__(self, cfg: dict, stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("libpic needs a CUDA device; there is no CPU path")
        self.cfg = dict(DEFAULTS)
        self.cfg.update(cfg)
        self._p = make_params(self.cfg)
        nbytes = workspace_bytes(self.cfg)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        _check(lib().pic_init(C.byref(self._p), C.c_void_p(self.workspace.data_ptr()), nbytes,
                              C.c_void_p(self.stream.cuda_stream), C.byref(h)), "pic_init")
        self._h = h
        self.nx = self.cfg["n_cells"] + 1

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            lib().pic_free(h)
            self._h = None

    def __del__(self):
        self.close()

    def step(self, n: int = 1) -> int:
        return _check(lib().pic_step(self._h, int(n)), "pic_step")

    def step_profiled(self, n: int, ms: np.ndarray) -> int:
        """n steps with per-launch CUDA-event times added to ms[0] (particle pass) and ms[1]
        (compaction with the next field solve beside it)."""
        assert ms.dtype == np.float64 and ms.shape == (2,)
        return _check(lib().pic_step_profiled(self._h, int(n), _ptr(ms)), "pic_step_profiled")

    def sync(self) -> int:
        return _check(lib().pic_sync(self._h), "pic_sync")

    def status(self) -> int:
        return lib().pic_sync(self._h)

    def counts(self) -> tuple[int, int]:
        a, b = C.c_int64(), C.c_int64()
        _check(lib().pic_counts(self._h, C.byref(a), C.byref(b)), "pic_counts")
        return a.value, b.value

    def checkpoint(self) -> np.ndarray:
        """The whole state at the current step boundary, as a host byte array."""
        nb = C.c_size_t(0)
        _check(lib().pic_checkpoint_bytes(self._h, C.byref(nb)), "pic_checkpoint_bytes")
        buf = np.zeros(nb.value, dtype=np.uint8)
        _check(lib().pic_checkpoint_save(self._h, _ptr(buf), nb.value), "pic_checkpoint_save")
        return buf

    def restore(self, buf: np.ndarray) -> None:
        """Resume from a checkpoint of a simulation with the same parameters."""
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        _check(lib().pic_checkpoint_load(self._h, _ptr(buf), buf.nbytes), "pic_checkpoint_load")

    def counts_async(self, out) -> None:
        """Enqueue a copy of the two counts into `out` (a pinned host int64 tensor of 2)."""
        import torch

        if out.dtype != torch.int64 or out.numel() < 2 or out.is_cuda or not out.is_contiguous():
            raise ValueError("counts_async: a contiguous host int64 tensor of 2 expected")
        _check(lib().pic_counts_async(self._h, C.c_void_p(out.data_ptr())), "pic_counts_async")

    def step_state(self) -> tuple[int, int, int]:
        s, e, i = C.c_uint32(), C.c_uint32(), C.c_uint32()
        _check(lib().pic_get_step(self._h, C.byref(s), C.byref(e), C.byref(i)), "pic_get_step")
        return s.value, e.value, i.value

    def particles(self, s: int) -> dict:
        n = self.counts()[s]
        out = {k: np.zeros(n) for k in ("x", "vx", "vy", "vz")}
        out["id"] = np.zeros(n, dtype=np.uint32)
        got = C.c_int64()
        _check(lib().pic_get_particles(self._h, s, _ptr(out["x"]), _ptr(out["vx"]),
                                       _ptr(out["vy"]), _ptr(out["vz"]), _ptr(out["id"]), n,
                                       C.byref(got)), "pic_get_particles")
        return out

    def set_particles(self, s: int, x, vx, vy, vz, ids, next_id: int):
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (x, vx, vy, vz)]
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
        _check(lib().pic_set_particles(self._h, s, *[_ptr(a) for a in arrs], _ptr(ids),
                                       len(ids), next_id), "pic_set_particles")

    def grid(self) -> dict:
        g = dict(Ce=np.zeros(self.nx, np.int64), Ci=np.zeros(self.nx, np.int64),
                 phi=np.zeros(self.nx), E=np.zeros(self.nx))
        _check(lib().pic_get_grid(self._h, _ptr(g["Ce"]), _ptr(g["Ci"]), _ptr(g["phi"]),
                                  _ptr(g["E"])), "pic_get_grid")
        return g

    def solve_field(self):
        _check(lib().pic_solve_field(self._h), "pic_solve_field")

    def accum(self) -> dict:
        c = self.cfg
        a = dict(acc_e=np.zeros(self.nx), acc_i=np.zeros(self.nx),
                 eepf=np.zeros(c["eepf_bins"], np.uint64),
                 fedf_e=np.zeros(c["fedf_bins"], np.uint64),
                 fedf_i=np.zeros(c["fedf_bins"], np.uint64),
                 counters=np.zeros(N_COUNTERS, np.uint64))
        st = C.c_int64()
        _check(lib().pic_get_accum(self._h, _ptr(a["acc_e"]), _ptr(a["acc_i"]), _ptr(a["eepf"]),
                                   _ptr(a["fedf_e"]), _ptr(a["fedf_i"]), _ptr(a["counters"]),
                                   C.byref(st)), "pic_get_accum")
        a["steps"] = st.value
        return a

    def reset_averages(self):
        _check(lib().pic_reset_averages(self._h), "pic_reset_averages")

    def set_step(self, n: int):
        _check(lib().pic_set_step(self._h, n), "pic_set_step")

    def override_table(self, s: int, F: np.ndarray, numax: float):
        F = np.ascontiguousarray(F, dtype=np.float64)
        assert F.shape == (XS_NODES, 4)
        _check(lib().pic_override_table(self._h, s, _ptr(F), float(numax)), "pic_override_table")

    def derived(self) -> dict:
        out = np.zeros(7)
        _check(lib().pic_get_derived(self._h, _ptr(out)), "pic_get_derived")
        return dict(zip(("dt", "dx", "ng", "numax_e", "numax_i", "pmax_e", "pmax_i"),
                        out.tolist()))

    _DIAG_ARRAYS = ("n_e", "n_i", "eepf_energy", "eepf", "fedf_energy", "fedf_e", "fedf_i")

    def diag(self) -> dict:
        d = getattr(self, "_diag_out", None)
        if d is None:  # one output struct per simulation, its array lengths set once
            c = self.cfg
            d = self._diag_out = PicDiagOut()
            d.n_x, d.eepf_bins, d.fedf_bins = self.nx, c["eepf_bins"], c["fedf_bins"]
            n = (self.nx, self.nx, c["eepf_bins"], c["eepf_bins"], c["fedf_bins"],
                 c["fedf_bins"], c["fedf_bins"])
            self._diag_cuts = [int(v) for v in np.cumsum((0,) + n)]
        cuts = self._diag_cuts
        # fresh arrays every call (the caller may keep them), all seven in one buffer that
        # pic_diag fills completely
        buf = np.empty(cuts[-1])
        base = buf.ctypes.data
        out = {}
        for i, k in enumerate(self._DIAG_ARRAYS):
            out[k] = buf[cuts[i]:cuts[i + 1]]
            setattr(d, k, C.cast(base + 8 * cuts[i], _DP))
        rc = _check(lib().pic_diag(self._h, C.byref(d)), "pic_diag")
        for name in _DIAG_SCALARS:
            out[name] = getattr(d, name)
        out["counters"] = np.array(d.counters, dtype=np.uint64)
        out["return_code"] = rc
        return out


def fp64_rate(stream=None) -> tuple[float, float]:
    """Measured FP64 operations per second of the device: (separate multiply + add, fused
    multiply-add), from pic_fp64_rate."""
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    out = np.zeros(2)
    _check(lib().pic_fp64_rate(C.c_void_p(s.cuda_stream), _ptr(out)), "pic_fp64_rate")
    return float(out[0]), float(out[1])


FIELD_STATIC_MAX_CELLS = 65536


def field_solve_static(charge_e, charge_i, n_cells: int, gap_m: float, weight: float,
                       area_m2: float, v_left: float, phi, efield, stream=None) -> int:
    """pic_field_solve_static on CUDA tensors: int64 charge counts [n_cells + 1] in, float64
    phi and E [n_cells + 1] out, enqueued on `stream` (default: torch's current stream).
    Allocates no device memory; calls that may run at the same time on one device race on
    the library's static scratch array.  Returns the C-ABI code, raising on errors."""
    import torch

    for t, dt in ((charge_e, torch.int64), (charge_i, torch.int64), (phi, torch.float64),
                  (efield, torch.float64)):
        if t.dtype != dt or not t.is_cuda or not t.is_contiguous() or t.numel() < n_cells + 1:
            raise ValueError("field_solve_static: contiguous CUDA tensors of n_cells + 1 "
                             "int64 (charges) and float64 (phi, efield) elements expected")
    s = stream if stream is not None else torch.cuda.current_stream()
    return _check(lib().pic_field_solve_static(
        C.c_void_p(charge_e.data_ptr()), C.c_void_p(charge_i.data_ptr()), int(n_cells),
        float(gap_m), float(weight), float(area_m2), float(v_left),
        C.c_void_p(phi.data_ptr()), C.c_void_p(efield.data_ptr()), C.c_void_p(s.cuda_stream)),
        "pic_field_solve_static")


class Ensemble:
    """PIC_FP32 simulations advanced together, one launch per step (pic_ensemble_*).

    `sims` are Simulation objects on one stream; `targets[i]` is the step index at which
    member i stops.  Members keep every single-run method (diag, particles, grid, ...)."""

    def __init__(self, sims, targets):
        import torch

        self.sims = list(sims)
        n = len(self.sims)
        nb = C.c_size_t(0)
        _check(lib().pic_ensemble_workspace_bytes(n, C.byref(nb)), "pic_ensemble_workspace_bytes")
        self.workspace = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
        hs = (C.c_void_p * n)(*[s._h.value for s in self.sims])
        tg = np.ascontiguousarray(targets, dtype=np.int64)
        if tg.shape != (n,):
            raise ValueError("one target step per member")
        h = C.c_void_p()
        _check(lib().pic_ensemble_create(hs, n, _ptr(tg), C.c_void_p(self.workspace.data_ptr()),
                                         nb.value, C.byref(h)), "pic_ensemble_create")
        self._h = h

    def step(self, n: int = 1) -> int:
        return _check(lib().pic_ensemble_step(self._h, int(n)), "pic_ensemble_step")

    def sync(self) -> int:
        return _check(lib().pic_ensemble_sync(self._h), "pic_ensemble_sync")

    def configure(self, unit: int, blocks_per_sm: int, graph: bool = True):
        _check(lib().pic_ensemble_configure(self._h, int(unit), int(blocks_per_sm), int(graph)),
               "pic_ensemble_configure")

    def autotune(self, trial_steps: int = 3) -> tuple[int, int]:
        out = np.zeros(2, dtype=np.int32)
        _check(lib().pic_ensemble_autotune(self._h, int(trial_steps), _ptr(out)),
               "pic_ensemble_autotune")
        return int(out[0]), int(out[1])

    def info(self) -> dict:
        out = np.zeros(5, dtype=np.int32)
        _check(lib().pic_ensemble_info(self._h, _ptr(out)), "pic_ensemble_info")
        return dict(zip(("unit", "blocks_per_sm", "grid", "graph", "smem_bytes"),
                        (int(v) for v in out)))

    def close(self):
        if getattr(self, "_h", None):
            lib().pic_ensemble_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tc_gemm_bf16(a, b, c, stream=None) -> int:
    """pic_tc_gemm_bf16 on CUDA tensors: a [m, k] and b [n, k] torch.bfloat16, c [m, n]
    torch.float32 (all contiguous); c = a @ b.T with FP32 accumulation."""
    import torch

    m, k = a.shape
    n = b.shape[0]
    if (a.dtype != torch.bfloat16 or b.dtype != torch.bfloat16 or c.dtype != torch.float32
            or b.shape[1] != k or tuple(c.shape) != (m, n)
            or not all(t.is_cuda and t.is_contiguous() for t in (a, b, c))):
        raise ValueError("tc_gemm_bf16: contiguous CUDA bf16 a[m,k], b[n,k] and fp32 c[m,n]")
    s = stream if stream is not None else torch.cuda.current_stream()
    return _check(lib().pic_tc_gemm_bf16(C.c_void_p(a.data_ptr()), C.c_void_p(b.data_ptr()),
                                         C.c_void_p(c.data_ptr()), m, n, k,
                                         C.c_void_p(s.cuda_stream)), "pic_tc_gemm_bf16")


class Mlp:
    """The surrogate network on the library's tensor-core kernels (pic_mlp_*): x [n, 7] ->
    y [n, 192]; CUDA float32 tensors in, out."""

    def __init__(self, batch_max: int = 1024, seed: int = 1, stream=None):
        import torch

        nb = C.c_size_t(0)
        _check(lib().pic_mlp_workspace_bytes(batch_max, C.byref(nb)), "pic_mlp_workspace_bytes")
        self.workspace = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.batch_max = batch_max
        self.n_params = lib().pic_mlp_num_params()
        h = C.c_void_p()
        _check(lib().pic_mlp_init(batch_max, seed, C.c_void_p(self.workspace.data_ptr()),
                                  nb.value, C.c_void_p(self.stream.cuda_stream), C.byref(h)),
               "pic_mlp_init")
        self._h = h

    @staticmethod
    def _dev(t, cols):
        import torch

        if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous() or t.shape[-1] != cols:
            raise ValueError(f"contiguous CUDA float32 tensor [n, {cols}] expected")
        return C.c_void_p(t.data_ptr())

    def params(self) -> np.ndarray:
        out = np.zeros(self.n_params, dtype=np.float32)
        _check(lib().pic_mlp_get_params(self._h, _ptr(out)), "pic_mlp_get_params")
        return out

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.shape == (self.n_params,)
        _check(lib().pic_mlp_set_params(self._h, _ptr(p)), "pic_mlp_set_params")

    def forward(self, x):
        import torch

        n = x.shape[0]
        y = torch.empty((n, 192), dtype=torch.float32, device="cuda")
        _check(lib().pic_mlp_forward(self._h, self._dev(x, 7), n, self._dev(y, 192)),
               "pic_mlp_forward")
        return y

    def gradients(self, x, t) -> tuple[np.ndarray, float]:
        g = np.zeros(self.n_params, dtype=np.float32)
        loss = C.c_float(0.0)
        _check(lib().pic_mlp_gradients(self._h, self._dev(x, 7), self._dev(t, 192), x.shape[0],
                                       _ptr(g), C.byref(loss)), "pic_mlp_gradients")
        return g, loss.value

    def train_step(self, x, t, lr: float, want_loss: bool = True):
        loss = C.c_float(0.0)
        _check(lib().pic_mlp_train_step(self._h, self._dev(x, 7), self._dev(t, 192), x.shape[0],
                                        float(lr), C.byref(loss) if want_loss else None),
               "pic_mlp_train_step")
        return loss.value if want_loss else None

    ACTS = {"X": (0, 16, True), "Z1": (1, 256, False), "H1": (2, 256, True),
            "Z2": (3, 256, False), "H2": (4, 256, True), "Y": (5, 192, False),
            "dY": (6, 192, False), "dYh": (7, 192, True), "dZ2": (8, 256, False),
            "dZ2h": (9, 256, True), "dZ1": (10, 256, False), "dZ1h": (11, 256, True)}

    def activations(self, name: str, n: int) -> np.ndarray:
        """An intermediate array of the last call (pic_mlp_get_activations), first n rows, as
        float64 (BF16 arrays decoded exactly)."""
        which, cols, is_bf16 = self.ACTS[name]
        buf = np.zeros((n, cols), dtype=np.uint16 if is_bf16 else np.float32)
        _check(lib().pic_mlp_get_activations(self._h, which, n, _ptr(buf)),
               "pic_mlp_get_activations")
        if is_bf16:
            return (buf.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
        return buf.astype(np.float64)

    def close(self):
        if getattr(self, "_h", None):
            lib().pic_mlp_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def selftest_waits(stream=None) -> tuple[int, int]:
    """Run the bounded-wait self-test; returns the codes of the bulk-copy barrier and the grid
    barrier waits (PIC_ERR_TIMEOUT, -6, when each gave up as designed)."""
    import torch

    nb = C.c_size_t(0)
    _check(lib().pic_ensemble_workspace_bytes(1, C.byref(nb)), "pic_ensemble_workspace_bytes")
    ws = torch.empty(nb.value + 256, dtype=torch.uint8, device="cuda")
    s = stream if stream is not None else torch.cuda.current_stream()
    codes = np.zeros(2, dtype=np.int32)
    _check(lib().pic_selftest_waits(C.c_void_p(ws.data_ptr()), nb.value + 256,
                                    C.c_void_p(s.cuda_stream), _ptr(codes)), "pic_selftest_waits")
    return int(codes[0]), int(codes[1])

