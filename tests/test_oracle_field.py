"""Pins of the oracle's field solve (§2 step 2: the Dirichlet finite-difference Poisson system,
solved exactly through its discrete Green's function (reading C-23) and kept beside the
Thomas algorithm the paper names; E by differencing; readings C-4, C-5)."""
import numpy as np
import pytest

from oracle import oracle as O

QE, EPS0 = 1.602176634e-19, 8.8541878128e-12


def _sim(**kw):
    cfg = dict(gap_m=0.025, pressure_pa=0.0, v_rf_amp_v=150.0, steps_per_rf=1, n_cells=64,
               weight=2.5e5, init_per_species=0, capacity_per_species=16)
    cfg.update(kw)
    return O.OracleSim(cfg)


def test_zero_charge_linear_potential():
    s = _sim(v_rf_amp_v=237.0)
    s.set_counts(np.zeros(65, np.int64), np.zeros(65, np.int64))
    s.solve_field()
    g = s.grid()
    x = np.arange(65) * (0.025 / 64)
    phi = 237.0 * (1 - x / 0.025)
    assert np.max(np.abs(g["phi"] - phi)) <= 1e-13 * 237.0
    assert np.max(np.abs(g["E"] - 237.0 / 0.025)) <= 1e-11 * 237.0 / 0.025


@pytest.mark.parametrize("nc", [2, 3, 64, 401])
def test_uniform_charge_closed_form(nc):
    """phi = V(1 - x/L) + rho x (L - x) / (2 eps0): the 3-point scheme is exact for quadratics,
    and the half-cell Gauss law at the ends (C-4) makes E exact at the electrodes too."""
    L, V, W, A = 0.025, 100.0, 2.5e5, 1e-4
    s = _sim(n_cells=nc, v_rf_amp_v=V, weight=W)
    c = 3 * 2**32  # three unit particles' worth of counts per interior node
    Ci = np.full(nc + 1, c, np.int64)
    Ci[0] = Ci[-1] = c // 2  # half volume at the electrodes (C-5): same density
    s.set_counts(np.zeros(nc + 1, np.int64), Ci)
    s.solve_field()
    g = s.grid()
    dx = L / nc
    rho = QE * 3 * W / (A * dx)
    x = np.arange(nc + 1) * dx
    phi = V * (1 - x / L) + rho * x * (L - x) / (2 * EPS0)
    E = V / L - rho * (L - 2 * x) / (2 * EPS0)
    scale = np.max(np.abs(phi))
    assert np.max(np.abs(g["phi"] - phi)) <= 1e-12 * scale
    assert np.max(np.abs(g["E"] - E)) <= 1e-10 * np.max(np.abs(E))


def _random_counts(nc, seed):
    rng = np.random.default_rng(seed)
    Ce = rng.integers(0, 50 * 2**32, nc + 1, dtype=np.int64)
    Ci = rng.integers(0, 50 * 2**32, nc + 1, dtype=np.int64)
    return Ce, Ci


@pytest.mark.parametrize("nc", [5, 128, 1024])
def test_random_charge_against_dense_solve(nc):
    """The field solve equals a dense LU solve (numpy) of the same finite-difference system."""
    L, V, W, A = 0.025, -80.0, 1e5, 1e-4
    s = _sim(n_cells=nc, v_rf_amp_v=V, weight=W)
    Ce, Ci = _random_counts(nc, nc)
    s.set_counts(Ce, Ci)
    s.solve_field()
    g = s.grid()
    dx = L / nc
    rho = QE * W * (Ci - Ce).astype(np.float64) / (A * dx * 2.0**32)
    M = nc - 1
    K = np.diag(np.full(M, 2.0)) - np.diag(np.ones(M - 1), 1) - np.diag(np.ones(M - 1), -1)
    b = rho[1:nc] * dx * dx / EPS0
    b[0] += V
    phi_in = np.linalg.solve(K, b)
    scale = max(np.max(np.abs(phi_in)), abs(V))
    assert g["phi"][0] == V and g["phi"][-1] == 0.0
    assert np.max(np.abs(g["phi"][1:nc] - phi_in)) <= 1e-11 * scale
    # residual of the discrete Poisson equation at every interior node
    phi = g["phi"]
    lap = (phi[:-2] - 2 * phi[1:-1] + phi[2:]) / dx**2
    assert np.max(np.abs(lap + rho[1:nc] / EPS0)) <= 1e-8 * np.max(np.abs(rho / EPS0)) + 1e-6


@pytest.mark.parametrize("nc", [7, 400])
def test_discrete_gauss_law(nc):
    """E_N - E_0 equals the total charge per area over eps0 (interior nodes full cells,
    electrode nodes half cells), whatever the charge distribution."""
    L, W, A = 0.025, 2e5, 1e-4
    s = _sim(n_cells=nc, v_rf_amp_v=33.0, weight=W)
    Ce, Ci = _random_counts(nc, 100 + nc)
    s.set_counts(Ce, Ci)
    s.solve_field()
    E = s.grid()["E"]
    q_per_area = QE * W * float(np.sum(Ci - Ce)) / (A * 2.0**32)
    assert abs((E[-1] - E[0]) - q_per_area / EPS0) <= 1e-9 * abs(q_per_area / EPS0)


@pytest.mark.parametrize("nc", [2, 3, 17, 400, 4096])
def test_green_function_solve_matches_thomas(nc):
    """The exact Green's-function evaluation (reading C-23) and the Thomas algorithm named in
    §2 step 2 solve the same tridiagonal system: they agree to rounding."""
    s = _sim(n_cells=nc, v_rf_amp_v=-61.0, weight=3e5)
    Ce, Ci = _random_counts(nc, 7 * nc)
    s.set_counts(Ce, Ci)
    s.solve_field()
    phi = s.grid()["phi"]
    th = s.thomas_phi(-61.0)
    # the sequential sweep's rounding grows with the condition number (~nc^2) of the matrix
    tol = max(1e-13, 2.2e-16 * nc * nc)
    assert np.max(np.abs(phi - th)) <= tol * max(np.max(np.abs(th)), 61.0)


def test_green_function_solve_exact_rational():
    """On a small grid the solve is compared with an exact rational solution (fractions)
    of the tridiagonal system: the only error left is the final rounding."""
    from fractions import Fraction as Fr

    nc, V = 9, 37.0
    s = _sim(n_cells=nc, v_rf_amp_v=V, weight=4e5)
    Ce, Ci = _random_counts(nc, 3)
    s.set_counts(Ce, Ci)
    s.solve_field()
    phi = s.grid()["phi"]
    rfac = Fr(s.derived()["rfac"])
    # Gaussian elimination in exact arithmetic
    M = nc - 1
    a = [[Fr(0)] * M for _ in range(M)]
    b = [rfac * int(Ci[j + 1] - Ce[j + 1]) for j in range(M)]
    b[0] += Fr(V)
    for i in range(M):
        a[i][i] = Fr(2)
        if i:
            a[i][i - 1] = Fr(-1)
        if i + 1 < M:
            a[i][i + 1] = Fr(-1)
    for i in range(M):
        for r in range(i + 1, M):
            f = a[r][i] / a[i][i]
            for c in range(i, M):
                a[r][c] -= f * a[i][c]
            b[r] -= f * b[i]
    x = [Fr(0)] * M
    for i in reversed(range(M)):
        x[i] = (b[i] - sum(a[i][c] * x[c] for c in range(i + 1, M))) / a[i][i]
    for j in range(M):
        exact = x[j]
        assert abs(Fr(phi[j + 1]) - exact) <= abs(exact) * Fr(2, 2**52) + Fr(1, 2**60)


def test_field_is_linear_in_charge_and_voltage():
    s = _sim(n_cells=50, v_rf_amp_v=10.0)
    Ce, Ci = _random_counts(50, 9)
    s.set_counts(Ce, Ci)
    s.solve_field()
    e1 = s.grid()["E"].copy()
    s2 = _sim(n_cells=50, v_rf_amp_v=0.0)
    s2.set_counts(Ce, Ci)
    s2.solve_field()
    e0 = s2.grid()["E"].copy()
    s3 = _sim(n_cells=50, v_rf_amp_v=10.0)
    s3.set_counts(np.zeros(51, np.int64), np.zeros(51, np.int64))
    s3.solve_field()
    ev = s3.grid()["E"].copy()
    assert np.max(np.abs(e1 - (e0 + ev))) <= 1e-9 * np.max(np.abs(e1))
