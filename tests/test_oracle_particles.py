"""Pins of the oracle's particle steps: linear deposit (§2 step 1, reading C-14), gather and
leapfrog (§2 steps 3-4), surfaces (§2 step 5, readings C-11, C-12) and compaction (C-15)."""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O

QE, ME, EPS0 = 1.602176634e-19, 9.1093837015e-31, 8.8541878128e-12
MI = 39.948 * 1.66053906660e-27


def _sim(**kw):
    cfg = dict(gap_m=0.025, pressure_pa=0.0, v_rf_amp_v=0.0, steps_per_rf=1000, n_cells=64,
               weight=0.0, init_per_species=0, capacity_per_species=200_000)
    cfg.update(kw)
    return O.OracleSim(cfg)


def _set(s, sp, x, vx=None, vy=None, vz=None, ids=None, next_id=None):
    n = len(x)
    z = np.zeros(n)
    ids = np.arange(n, dtype=np.uint32) if ids is None else ids
    s.set_particles(sp, x, z if vx is None else vx, z if vy is None else vy,
                    z if vz is None else vz, ids, n if next_id is None else next_id)


# ------------------------------------------------------------------------------ deposit
def test_deposit_charge_conservation_exact():
    s = _sim(n_cells=400)
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 0.025, 100_000)
    x[:5] = [0.0, 0.025, 0.0125, 1e-300, 0.025 * (1 - 2**-52)]
    _set(s, 0, x)
    assert int(s.grid()["Ce"].sum()) == len(x) * 2**32


def test_deposit_brute_force_exact_fractions():
    """L = 1 m and 4 cells make x/dx exact, so the hand computation with fractions is exact,
    including the round-half-to-even ties of the 32-bit fixed point."""
    s = _sim(gap_m=1.0, n_cells=4)
    tie = 0.25 * (2 * 12345 + 1) / 2**33  # f * 2^32 = 12345.5 -> 12346 (even)
    tie2 = 0.25 * (2 * 12346 + 1) / 2**33  # 12346.5 -> 12346 (even)
    x = np.array([0.0, 0.25, 0.3, 0.999, 1.0, 0.5 + tie, 0.75 + tie2])
    _set(s, 0, x)
    got = s.grid()["Ce"]
    want = [0] * 5
    for xi in x:
        xn = Fraction(float(xi)) * 4
        j = min(int(math.floor(xn)), 3)
        f = xn - j
        t = f * 2**32
        wr = round(t)  # Python's round is half-to-even on Fractions
        want[j] += 2**32 - wr
        want[j + 1] += wr
    assert list(got) == want
    # the two ties on their own: 12345.5 -> 12346 and 12346.5 -> 12346
    for xt, j, wr in ((0.5 + tie, 2, 12346), (0.75 + tie2, 3, 12346)):
        _set(s, 0, np.array([xt]))
        c = s.grid()["Ce"]
        assert c[j] == 2**32 - wr and c[j + 1] == wr


def test_deposit_first_moment():
    """Linear weighting conserves the first moment: sum_j w_j x_j = x (to 2^-32 of a cell)."""
    s = _sim(n_cells=17)
    rng = np.random.default_rng(2)
    for xi in rng.uniform(0, 0.025, 50):
        _set(s, 1, np.array([xi]))
        C = s.grid()["Ci"].astype(np.float64)
        xm = float(np.sum(C * np.arange(18) * (0.025 / 17)) / 2**32)
        assert abs(xm - xi) <= (0.025 / 17) * 2**-31


# -------------------------------------------------------------------------------- push
def test_field_free_ballistic_motion():
    s = _sim()
    rng = np.random.default_rng(3)
    x0 = rng.uniform(0.01, 0.015, 1000)
    vx = rng.normal(0, 1e4, 1000)
    vy, vz = rng.normal(0, 1e4, (2, 1000))
    _set(s, 1, x0, vx, vy, vz)
    s.step(50)
    p = s.particles(1)
    dt = s.derived()["dt"]
    assert np.array_equal(p["vx"], vx) and np.array_equal(p["vy"], vy)
    assert np.max(np.abs(p["x"] - (x0 + 50 * vx * dt))) <= 1e-15 * 0.025 * 60


def test_uniform_field_leapfrog_exact_parabola():
    """With a constant field (N_t = 1 so V is constant, no charge) leapfrog started from
    v^{-1/2} = v0 - a dt/2 reproduces x0 + v0 t + a t^2/2 at every node in time."""
    V, L = 40.0, 0.025
    s = _sim(steps_per_rf=1, v_rf_amp_v=V, f_rf_hz=1e9)
    dt = s.derived()["dt"]
    a = QE * (V / L) / MI  # ions are pushed towards x = L
    x0 = np.array([0.001, 0.002, 0.004])
    v0 = np.array([0.0, 100.0, -50.0])
    _set(s, 1, x0, v0 - 0.5 * a * dt)
    for n in range(1, 200):
        s.step(1)
        t = n * dt
        want = x0 + v0 * t + 0.5 * a * t * t
        assert np.max(np.abs(s.particles(1)["x"] - want)) <= 1e-12 * L, n


def _cold_plasma_run(wdt, steps, nc=64, n_per=64 * 64, with_sim=False):
    """Electrons on a uniform ion background, displaced by xi = delta sin(2 pi x / L);
    grounded electrodes.  Returns the electrons' mean displacement projection per step (and
    the simulation itself with with_sim)."""
    L = 0.01
    f = 13.56e6
    n0 = 1e15
    wpe = math.sqrt(n0 * QE * QE / (EPS0 * ME))
    dt = wdt / wpe
    Nt = 1.0 / (f * dt)
    W = n0 * L * 1e-4 / n_per
    s = _sim(gap_m=L, n_cells=nc, steps_per_rf=1, v_rf_amp_v=0.0, weight=W,
             f_rf_hz=1.0 / (dt * 1.0))
    dt_sim = s.derived()["dt"]
    assert abs(dt_sim - dt) <= 1e-12 * dt
    x_eq = (np.arange(n_per) + 0.5) * (L / n_per)
    delta = 0.02 * L / n_per * 50
    xe = x_eq + delta * np.sin(2 * np.pi * x_eq / L)
    _set(s, 1, x_eq.copy())
    _set(s, 0, xe)
    proj = []
    basis = np.sin(2 * np.pi * x_eq / L)
    for _ in range(steps):
        s.step(1)
        p = s.particles(0)
        if len(p["x"]) != n_per:  # an unstable run has thrown electrons out of the gap
            break
        order = np.argsort(p["id"])
        xi = p["x"][order] - x_eq
        proj.append(float(np.dot(xi, basis)))
    del Nt
    if with_sim:
        return np.array(proj), wpe, dt, s
    return np.array(proj), wpe, dt


@pytest.mark.parametrize("wdt", [0.2, 1.0, 1.8])
def test_cold_plasma_oscillation_leapfrog_frequency(wdt):
    """Leapfrog on a harmonic oscillator has numerical frequency 2 asin(w dt / 2) / dt and is
    stable for w dt < 2 (§3.5, the textbook analysis the paper quotes)."""
    steps = int(12 * 2 * math.pi / wdt)
    y, wpe, dt = _cold_plasma_run(wdt, steps)
    # frequency from zero crossings of the mode amplitude
    zc = np.where(np.sign(y[:-1]) != np.sign(y[1:]))[0]
    # sub-step crossing times by linear interpolation
    t = zc + y[zc] / (y[zc] - y[zc + 1])
    half_periods = np.diff(t)
    w_meas = math.pi / (np.mean(half_periods) * dt)
    w_theory = 2 * math.asin(wdt / 2) / dt
    assert abs(w_meas / w_theory - 1) < 0.01, (w_meas / wpe, w_theory / wpe)
    assert np.max(np.abs(y)) < 3 * np.max(np.abs(y[: int(2 * math.pi / wdt) + 2]))


@pytest.mark.parametrize("wdt", [0.3, 1.2])
def test_reported_omega_pe_dt_matches_the_measured_oscillation(wdt):
    """The criterion ω_pe Δt that the diagnostics report (§3.5, reading C-19: from the
    time-averaged density at L/2) against the plasma frequency the simulation itself
    oscillates at: a measured numerical frequency Ω gives ω_pe Δt = 2 sin(Ω Δt / 2) (the
    leapfrog dispersion relation inverted).  A wrong constant, density scale or centre
    interpolation in the diagnostic would miss the measured value."""
    steps = int(10 * 2 * math.pi / wdt)
    y, _, dt, s = _cold_plasma_run(wdt, steps, with_sim=True)
    assert len(y) == steps
    zc = np.where(np.sign(y[:-1]) != np.sign(y[1:]))[0]
    t = zc + y[zc] / (y[zc] - y[zc + 1])
    omega = math.pi / (np.mean(np.diff(t)) * dt)
    measured = 2 * math.sin(omega * dt / 2)
    d = s.diag()
    assert abs(d["omega_pe_dt"] / measured - 1) < 0.005, (d["omega_pe_dt"], measured)


def test_cold_plasma_unstable_beyond_two():
    y, _, _ = _cold_plasma_run(2.3, 60)
    assert np.max(np.abs(y)) > 50 * abs(y[0])
    y2, _, _ = _cold_plasma_run(1.9, 60)
    assert np.max(np.abs(y2)) < 5 * abs(y2[0])


# --------------------------------------------------------------------------- surfaces
def _wall_sim(R=0.0, gamma=0.0, **kw):
    return _sim(refl_e=R, gamma_see=gamma, **kw)


def _beam(n, speed, seed=0, L=0.025):
    """particles at random positions all moving fast enough to hit a wall in one step"""
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.3 * L, 0.7 * L, n)
    sign = np.where(rng.uniform(size=n) < 0.5, -1.0, 1.0)
    return x, sign * speed


def test_full_reflection_conserves_electrons():
    s = _wall_sim(R=1.0)
    dt = s.derived()["dt"]
    x, vx = _beam(5000, 0.8 * 0.025 / dt)
    _set(s, 0, x, vx)
    s.step(1)
    c = s.accum()["counters"]
    p = s.particles(0)
    assert s.count(0) == 5000
    assert int(c[4]) == int(np.sum(np.abs(vx) * dt > np.minimum(x, 0.025 - x)))
    assert int(c[0] + c[1]) == 0
    assert np.all((p["x"] > 0) & (p["x"] < 0.025))
    assert int(s.grid()["Ce"].sum()) == 5000 * 2**32


def test_no_reflection_removes_all_hits():
    s = _wall_sim(R=0.0)
    dt = s.derived()["dt"]
    x, vx = _beam(5000, 0.8 * 0.025 / dt, seed=1)
    hit = np.abs(vx) * dt >= np.where(vx < 0, x, 0.025 - x)
    _set(s, 0, x, vx)
    s.step(1)
    c = s.accum()["counters"]
    assert s.count(0) == 5000 - hit.sum()
    assert int(c[0]) == int(np.sum(hit & (vx < 0))) and int(c[1]) == int(np.sum(hit & (vx > 0)))
    assert set(s.particles(0)["id"].tolist()) == set(np.nonzero(~hit)[0].tolist())


def test_gamma_one_emits_one_electron_per_ion():
    s = _wall_sim(gamma=1.0, see_energy_ev=2.0)
    dt = s.derived()["dt"]
    x, vx = _beam(3000, 0.9 * 0.025 / dt, seed=2)
    _set(s, 1, x, vx)
    s.step(1)
    c = s.accum()["counters"]
    hits = int(c[2] + c[3])
    assert hits > 0 and int(c[5]) == hits
    assert s.count(0) == hits and s.count(1) == 3000 - hits
    p = s.particles(0)
    left = p["x"] == 0.0
    right = p["x"] == 0.025
    assert np.all(left | right)
    assert int(left.sum()) == int(c[2])
    assert np.all(p["vx"][left] > 0) and np.all(p["vx"][right] < 0)
    speed = np.sqrt(p["vx"] ** 2 + p["vy"] ** 2 + p["vz"] ** 2)
    assert np.allclose(speed, math.sqrt(2.0 * 2 * QE / ME), rtol=1e-13)
    assert sorted(p["id"].tolist()) == list(range(hits))


@pytest.mark.parametrize("R,gamma", [(0.4, 0.3)])
def test_binomial_surface_rates(R, gamma):
    s = _wall_sim(R=R, gamma=gamma)
    dt = s.derived()["dt"]
    xe, ve = _beam(20000, 0.9 * 0.025 / dt, seed=3)
    xi, vi = _beam(20000, 0.9 * 0.025 / dt, seed=4)
    _set(s, 0, xe, ve)
    _set(s, 1, xi, vi)
    s.step(1)
    c = s.accum()["counters"].astype(float)
    e_hits = c[0] + c[1] + c[4]
    i_hits = c[2] + c[3]
    for k, n, p in ((c[4], e_hits, R), (c[5], i_hits, gamma)):
        assert abs(k - n * p) <= 4 * math.sqrt(n * p * (1 - p))


def test_compaction_rule_invariants():
    """Holes are filled by births in rank order, then by tail survivors (reading C-15)."""
    s = _wall_sim(gamma=1.0)
    dt = s.derived()["dt"]
    n = 1000
    rng = np.random.default_rng(5)
    x = rng.uniform(0.3, 0.7, n) * 0.025
    vx = np.where(rng.uniform(size=n) < 0.3, 0.9 * 0.025 / dt, 0.0)  # 30% hit the right wall
    _set(s, 1, x, vx)
    _set(s, 0, x[:10].copy(), ids=np.arange(10, dtype=np.uint32) + 500, next_id=510)
    s.step(1)
    hit = vx > 0
    H = int(hit.sum())
    pi = s.particles(1)
    # ions: no births, H holes; tail survivors fill the holes below N - H in order
    N2 = n - H
    assert s.count(1) == N2
    holes = np.nonzero(hit)[0]
    expect = np.arange(n)
    low_holes = holes[holes < N2]
    tail = np.array([t for t in range(N2, n) if not hit[t]])
    assert len(low_holes) == len(tail)
    expect[low_holes] = tail
    assert np.array_equal(pi["id"], expect[:N2].astype(np.uint32))
    # electrons: 10 survivors, then H gamma-electrons appended with ids 510.. in ion order
    pe = s.particles(0)
    assert s.count(0) == 10 + H
    assert np.array_equal(pe["id"][:10], np.arange(500, 510))
    assert np.array_equal(pe["id"][10:], np.arange(510, 510 + H))


def test_one_step_brute_force_small():
    """Tiny whole step (no gas): a dense numpy solve and hand-written gather/push agree with
    the oracle to rounding."""
    L, nc, V, W, A = 0.02, 4, 50.0, 3e6, 1e-4
    s = _sim(gap_m=L, n_cells=nc, steps_per_rf=8, v_rf_amp_v=V, weight=W, f_rf_hz=1.25e10)
    xe = np.array([0.003, 0.011, 0.0175])
    xi = np.array([0.0049, 0.0151])
    ve = np.array([1e5, -2e5, 3e4])
    vi = np.array([300.0, -100.0])
    _set(s, 0, xe, ve)
    _set(s, 1, xi, vi)
    s.step(1)
    dx = L / nc
    dt = s.derived()["dt"]

    def counts(xs):
        c = np.zeros(nc + 1)
        for x in xs:
            j = min(int(x // dx), nc - 1)
            f = x / dx - j
            c[j] += 1 - f
            c[j + 1] += f
        return c

    q = counts(xi) - counts(xe)
    vol = np.full(nc + 1, dx)
    vol[0] = vol[-1] = dx / 2
    rho = QE * W * q / (A * vol)
    K = 2 * np.eye(nc - 1) - np.eye(nc - 1, k=1) - np.eye(nc - 1, k=-1)
    b = rho[1:nc] * dx * dx / EPS0
    b[0] += V  # V(t_0) = V cos 0
    phi = np.concatenate([[V], np.linalg.solve(K, b), [0.0]])
    E = np.empty(nc + 1)
    E[1:nc] = (phi[:-2] - phi[2:]) / (2 * dx)
    E[0] = (phi[0] - phi[1]) / dx - rho[0] * dx / (2 * EPS0)
    E[nc] = (phi[nc - 1] - phi[nc]) / dx + rho[nc] * dx / (2 * EPS0)

    def push(xs, vs, qm):
        out = []
        for x, v in zip(xs, vs):
            j = min(int(x // dx), nc - 1)
            f = x / dx - j
            v2 = v + qm * ((1 - f) * E[j] + f * E[j + 1]) * dt
            out.append((x + v2 * dt, v2))
        return np.array(out)

    pe, pi = push(xe, ve, -QE / ME), push(xi, vi, QE / MI)
    ge, gi = s.particles(0), s.particles(1)
    assert np.allclose(ge["x"], pe[:, 0], rtol=1e-12, atol=0)
    assert np.allclose(ge["vx"], pe[:, 1], rtol=1e-10, atol=0)
    assert np.allclose(gi["x"], pi[:, 0], rtol=1e-12, atol=0)
    assert np.allclose(gi["vx"], pi[:, 1], rtol=1e-10, atol=0)
