"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test ties one oracle function to something other than itself: a
closed form, an invariant, a worked value printed with the paper's
workloads, a published known-answer vector, or brute force.  A dropped term,
a flipped sign or a shifted stagger in the oracle fails at least one of
them.  (Ngirmang et al., arXiv 2501.07465; equation labels as in the paper.)
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")
QE = 1.602176634e-19
ME = 9.1093837015e-31
EPS0 = 8.8541878128e-12
C = 299792458.0
KB = 1.380649e-23
HBAR = 1.054571817e-34


def _rows(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------------------
# random numbers and the Fermi-Dirac loader (Sec. 2)
# ---------------------------------------------------------------------------

def test_philox_known_answers():
    for r in _rows("philox4x32_10_kat.txt"):
        v = [int(x, 16) for x in r]
        out = O.philox(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_fermi_energy_exponent_is_two_thirds():
    """Sec. 2 prints (3 pi^2 N)^(3/2); the workloads' (n, E_F) pairs fix 2/3."""
    for n, ef, tol in _rows("fermi_energy_configs.txt"):
        got = O.fermi_energy(float(n), ME) / QE
        assert abs(got - float(ef)) / float(ef) < float(tol)
        wrong = HBAR ** 2 / (2 * ME) * (3 * math.pi ** 2 * float(n)) ** 1.5 / QE
        assert wrong / float(ef) > 1e10


def _stratified(n):
    return (np.arange(n) + 0.5) / n


def test_fd_zero_temperature_mean_energy_3d():
    """T -> 0: <E> = (3/5) E_F for the 3D Fermi sphere."""
    EF = 5.5 * QE
    p = O.fd_invert(False, ME, EF, 0.0, 0.0, _stratified(200000))
    E = p ** 2 / (2 * ME)
    assert abs(E.mean() / EF - 0.6) < 1e-6


def test_fd_zero_temperature_mean_energy_2d_dirac():
    """T -> 0, 2D Dirac disc: <E> = (2/3) E_F with E = v_F p."""
    EF, vF = 0.2 * QE, 1e6
    p = O.fd_invert(True, 0.0, EF, 0.0, vF, _stratified(200000))
    assert abs((vF * p).mean() / EF - 2.0 / 3.0) < 1e-6


def test_fd_finite_temperature_sommerfeld_3d():
    """mu fixed at E_F: <E> = (3/5) mu [1 + (pi^2/2)(kT/mu)^2] + O((kT/mu)^4),
    and <E^2> = (3/7) mu^2 [1 + (4 pi^2 / 3)(kT/mu)^2] + O((kT/mu)^4)."""
    EF, T = 5.5 * QE, 300.0
    p = O.fd_invert(False, ME, EF, T, 0.0, _stratified(400000))
    E = p ** 2 / (2 * ME)
    t = KB * T / EF
    assert abs(E.mean() / (0.6 * EF * (1 + math.pi ** 2 / 2 * t * t)) - 1) < 2e-7
    # second moment: num int E^{5/2} f ~ (2/7)mu^{7/2}(1 + (35/8) pi^2/6 t^2 ...)
    m2 = (3.0 / 7.0) * EF ** 2 * (1 + (35.0 / 24.0 - 1.0 / 8.0) * math.pi ** 2 * t * t)
    assert abs((E ** 2).mean() / m2 - 1) < 2e-7
    # and the finite-temperature shift is resolved (it is 6.7e-5 here)
    assert abs(E.mean() / (0.6 * EF) - 1) > 5e-5


def test_fd_finite_temperature_2d_polylog():
    """2D Dirac sheet at moderate mu/kT: <E> = 2 kT Li_3(-e^eta) / Li_2(-e^eta)
    (complete Fermi-Dirac integrals; the mu + 40 kT cut is e^-40 small)."""
    mp = pytest.importorskip("mpmath")
    EF, T, vF = 0.2 * QE, 300.0, 1e6
    p = O.fd_invert(True, 0.0, EF, T, vF, _stratified(400000))
    eta = EF / (KB * T)
    z = -mp.e ** eta
    exact = 2 * KB * T * float(mp.polylog(3, z) / mp.polylog(2, z))
    assert abs((vF * p).mean() / exact - 1) < 1e-6


def test_fd_loader_structure():
    """Positions uniform per material cell, isotropic direction, |v| = v_F
    for Dirac, v = 0 for bound, ids in material-cell order."""
    n = (6, 5, 4)
    mask = np.zeros((4, 5, 6), np.uint8)
    mask[1:3, 1:4, 2:5] = 1
    cell, off, v = O.fd_load(3, n, mask, O.KIND_FREE, ME, 5.5 * QE, 300.0, 0.0, 4, False, 7, 0)
    assert cell.size == mask.sum() * 4
    assert np.all(mask.ravel()[cell] == 1)
    assert np.all(np.diff(cell) >= 0)
    assert np.all((off >= 0) & (off < 1))
    cell, off, v = O.fd_load(3, n, mask, O.KIND_DIRAC, 0.01 * ME, 0.2 * QE, 300.0, 1e6, 4,
                             False, 7, 1)
    assert np.allclose(np.linalg.norm(v, axis=1), 1e6, rtol=1e-14)
    assert np.all(v[:, 2] == 0)
    cell, off, v = O.fd_load(3, n, mask, O.KIND_BOUND, ME, 0, 0, 0, 8, True, 7, 2)
    assert np.all(v == 0)
    assert set(np.round(off[:, 0], 12)) == {0.25, 0.75}
    # isotropy of a large free sample: <v_a> ~ 0 and <v_a^2> equal per axis
    n2 = (16, 16, 16)
    cell, off, v = O.fd_load(3, n2, None, O.KIND_FREE, ME, 5.5 * QE, 300.0, 0.0, 8, False, 3, 0)
    s2 = (v ** 2).mean(axis=0)
    assert np.all(np.abs(s2 / s2.mean() - 1) < 0.02)
    assert np.all(np.abs(v.mean(axis=0)) < 0.01 * math.sqrt(s2.mean()))


def test_fd_loader_quiet_needs_perfect_power():
    with pytest.raises(ValueError):
        O.fd_load(2, (4, 4, 1), None, O.KIND_FREE, ME, 5.5 * QE, 300.0, 0.0, 8, True, 1, 0)


# ---------------------------------------------------------------------------
# pushers (Appendix A, Sec. 5)
# ---------------------------------------------------------------------------

RNG = np.random.default_rng(20250107)


def test_boris_pure_B_conserves_speed_and_rotates_2atan_b():
    q, m, dt = -QE, ME, 1e-16
    for _ in range(50):
        v = RNG.normal(size=3) * 1e6
        B = RNG.normal(size=3) * 50.0
        v1 = O.push_free(v, np.zeros(3), B, q, m, dt)
        assert abs(np.linalg.norm(v1) / np.linalg.norm(v) - 1) < 1e-14
        bhat = B / np.linalg.norm(B)
        vp0 = v - bhat * (v @ bhat)
        vp1 = v1 - bhat * (v1 @ bhat)
        ang = math.atan2(np.linalg.norm(np.cross(vp0, vp1)), vp0 @ vp1)
        b = abs(q) * dt * np.linalg.norm(B) / (2 * m)
        assert abs(ang - 2 * math.atan(b)) < 1e-12
        assert abs(v1 @ bhat - v @ bhat) < 1e-9 * np.linalg.norm(v)


def test_boris_pure_E_is_linear_kick():
    q, m, dt = -QE, ME, 1e-17
    v = np.array([1e5, -2e5, 3e5])
    E = np.array([1e9, 2e9, -5e8])
    v1 = O.push_free(v, E, np.zeros(3), q, m, dt)
    assert np.allclose(v1, v + q / m * E * dt, rtol=1e-14, atol=0)


def test_boris_ExB_drift_direction():
    """Time-averaged velocity in crossed fields is E x B / B^2 (fixes the sign
    of the v x B rotation)."""
    q, m = -QE, ME
    E = np.array([0.0, 1e6, 0.0])
    B = np.array([0.0, 0.0, 10.0])
    wc = QE * 10.0 / ME
    dt = 0.02 / wc
    v = np.zeros(3)
    acc = np.zeros(3)
    nsteps = int(round(2 * math.pi / (wc * dt))) * 20
    for _ in range(nsteps):
        v = O.push_free(v, E, B, q, m, dt)
        acc += v
    drift = np.cross(E, B) / (B @ B)
    assert np.allclose(acc / nsteps, drift, atol=0.01 * np.linalg.norm(drift))


def test_bound_push_reproduces_taflove_recurrence():
    """Eliminating v gives x_{n+1} - 2x_n + x_{n-1} = dt^2 [(q/m)E_n - w0^2 x_n
    - gamma (x_{n+1} - x_{n-1})/(2 dt)] (Eq. taflove, read with dt^2)."""
    q, m, dt = -QE, ME, 4.81e-19
    w0 = np.array([4.7e15, 3.1e15, 6.0e15])
    g = np.array([1e14, 1e14, 1e14])
    v, D = np.zeros(3), np.zeros(3)
    xs, Es = [D.copy()], []
    for n in range(400):
        E = RNG.normal(size=3) * 1e9
        Es.append(E)
        v, D = O.push_bound(v, D, E, np.zeros(3), q, m, dt, w0, g)
        xs.append(D.copy())
    xs = np.array(xs)
    for n in range(1, 399):
        lhs = xs[n + 1] - 2 * xs[n] + xs[n - 1]
        rhs = dt * dt * (q / m * Es[n] - w0 ** 2 * xs[n] - g * (xs[n + 1] - xs[n - 1]) / (2 * dt))
        scale = dt * dt * np.abs(q / m * Es[n]).max()
        assert np.all(np.abs(lhs - rhs) < 1e-9 * scale)


def test_bound_driven_amplitude_matches_discrete_closed_form():
    """E = E0 cos(w t_n): the steady state is Re[X e^{-i w t_n}] with
    X = (q/m) E0 dt^2 / (w0^2 dt^2 - 4 sin^2(w dt/2) - i gamma dt sin(w dt)),
    which tends to the Lorentz response of Eq. lordielectric as dt -> 0."""
    q, m = -QE, ME
    w0, gam = 4.709e15, 2e14
    w = 3.6e15
    dt = 0.04 / w
    E0 = 1e8
    v, D = np.zeros(3), np.zeros(3)
    nsteps = int(70 / (gam * dt))
    xs = []
    for n in range(nsteps):
        E = np.array([E0 * math.cos(w * n * dt), 0, 0])
        v, D = O.push_bound(v, D, E, np.zeros(3), q, m, dt, [w0] * 3, [gam] * 3)
        xs.append(D[0])
    X = q / m * E0 * dt ** 2 / (w0 ** 2 * dt ** 2 - 4 * math.sin(w * dt / 2) ** 2
                                - 1j * gam * dt * math.sin(w * dt))
    # D after the push of step n is x_{n+1}
    for n in range(nsteps - 200, nsteps):
        pred = (X * np.exp(-1j * w * (n + 1) * dt)).real
        assert abs(xs[n] - pred) < 1e-9 * abs(X)
    cont = q / m * E0 / (w0 ** 2 - w ** 2 - 1j * gam * w)
    assert abs(X / cont - 1) < 0.01


def test_bound_anisotropic_gamma():
    """Diagonal damping gamma = (g_x, g_y, g_z) (the general 3x3 solve).
    With B = 0 the axes decouple and each follows Eq. taflove with its own
    w0 and gamma; with B the rotation step keeps the discrete energy balance
    |v+|^2 - |v-|^2 = -sum_a g_a dt/2 (v+_a + v-_a)^2 (the magnetic term
    does no work), v- and v+ the velocities around it."""
    q, m, dt = -QE, ME, 4.81e-19
    w0 = np.array([4.7e15, 3.1e15, 6.0e15])
    g = np.array([1e14, 4e14, 2.5e13])
    v, D = np.zeros(3), np.zeros(3)
    xs, Es = [D.copy()], []
    for n in range(400):
        E = RNG.normal(size=3) * 1e9
        Es.append(E)
        v, D = O.push_bound(v, D, E, np.zeros(3), q, m, dt, w0, g)
        xs.append(D.copy())
    xs = np.array(xs)
    for n in range(1, 399):
        lhs = xs[n + 1] - 2 * xs[n] + xs[n - 1]
        rhs = dt * dt * (q / m * Es[n] - w0 ** 2 * xs[n] - g * (xs[n + 1] - xs[n - 1]) / (2 * dt))
        scale = dt * dt * np.abs(q / m * Es[n]).max()
        assert np.all(np.abs(lhs - rhs) < 1e-9 * scale)
    # energy balance of the rotation step: E = 0 and D = 0 make the two
    # kicks vanish, so v- = v and v+ = the pushed v
    dt2 = 1e-16
    g2 = np.array([3e14, 1e13, 8e14])
    for _ in range(50):
        v0 = RNG.normal(size=3) * 1e6
        B = RNG.normal(size=3) * 2e3
        v1, _ = O.push_bound(v0, np.zeros(3), np.zeros(3), B, q, m, dt2, [0] * 3, g2)
        lhs = v1 @ v1 - v0 @ v0
        rhs = -np.sum(g2 * dt2 / 2 * (v1 + v0) ** 2)
        assert abs(lhs - rhs) < 1e-12 * (v0 @ v0)
        assert abs(rhs) > 1e-4 * (v0 @ v0)


def test_bound_binding_tensor_is_rotation_covariant():
    """A full symmetric binding tensor Omega^2 = R diag(w^2) R^T: pushing D
    with it under a random drive E_n equals pushing R^T D with the diagonal
    tensor under R^T E_n and rotating back (isotropic damping, B = 0, so the
    rotation commutes with the scheme); a transposed or misplaced
    off-diagonal entry breaks this."""
    q, m, dt = -QE, ME, 4.81e-19
    w = np.array([4.7e15, 3.1e15, 6.0e15])
    a, b = 0.7, -0.4
    Rz = np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]])
    Rx = np.array([[1, 0, 0], [0, math.cos(b), -math.sin(b)], [0, math.sin(b), math.cos(b)]])
    R = Rz @ Rx
    W2 = R @ np.diag(w ** 2) @ R.T
    omega0 = np.sqrt(np.diag(W2))
    off = np.array([W2[0, 1], W2[0, 2], W2[1, 2]])
    g = np.array([2e14] * 3)
    v, D = np.zeros(3), np.zeros(3)
    vr, Dr = np.zeros(3), np.zeros(3)
    for n in range(300):
        E = RNG.normal(size=3) * 1e9
        v, D = O.push_bound_tensor(v, D, E, np.zeros(3), q, m, dt, omega0, off, g)
        vr, Dr = O.push_bound(vr, Dr, R.T @ E, np.zeros(3), q, m, dt, w, g)
        np.testing.assert_allclose(D, R @ Dr, rtol=0, atol=1e-9 * np.abs(D).max())
        np.testing.assert_allclose(v, R @ vr, rtol=0, atol=1e-9 * np.abs(v).max())


def test_bound_push_reduces_to_boris_when_unbound():
    """gamma = 0, w0 = 0: the gyrotropic solve equals the Boris rotation."""
    q, m, dt = -QE, ME, 1e-16
    for _ in range(50):
        v = RNG.normal(size=3) * 1e6
        E = RNG.normal(size=3) * 1e9
        B = RNG.normal(size=3) * 100
        vb, _ = O.push_bound(v, np.zeros(3), E, B, q, m, dt, [0, 0, 0], [0, 0, 0])
        vf = O.push_free(v, E, B, q, m, dt)
        assert np.allclose(vb, vf, rtol=1e-13, atol=1e-13 * np.linalg.norm(vf))


def test_bound_damping_factor():
    """E = 0, w0 = 0: each step multiplies |v| by (1 - g dt/2)/(1 + g dt/2)
    (Eq. modborisrotsol); with B the component along b obeys the same."""
    q, m, dt, g = -QE, ME, 1e-16, 3e14
    f = (1 - g * dt / 2) / (1 + g * dt / 2)
    v = np.array([1e5, 2e5, -3e5])
    v1, _ = O.push_bound(v, np.zeros(3), np.zeros(3), np.zeros(3), q, m, dt, [0] * 3, [g] * 3)
    assert np.allclose(v1, f * v, rtol=1e-14)
    B = np.array([20.0, -10.0, 40.0])
    bh = B / np.linalg.norm(B)
    v2, _ = O.push_bound(v, np.zeros(3), np.zeros(3), B, q, m, dt, [0] * 3, [g] * 3)
    assert abs(v2 @ bh - f * (v @ bh)) < 1e-12 * np.linalg.norm(v)
    # across b the damped rotation scales |v_perp| by sqrt((c^2 + b^2)/(a^2 + b^2)),
    # a = 1 + g dt/2, c = 1 - g dt/2, b = |q| dt |B| / (2m)
    a, cc = 1 + g * dt / 2, 1 - g * dt / 2
    b = QE * dt * np.linalg.norm(B) / (2 * m)
    vp, v2p = v - bh * (v @ bh), v2 - bh * (v2 @ bh)
    pred = math.sqrt((cc * cc + b * b) / (a * a + b * b))
    assert abs(np.linalg.norm(v2p) / np.linalg.norm(vp) - pred) < 1e-12


def test_dirac_speed_is_vF():
    q, m, dt, vF = -QE, 0.0176 * ME, 1e-18, 1e6
    for _ in range(100):
        phi = RNG.uniform(0, 2 * math.pi)
        v = vF * np.array([math.cos(phi), math.sin(phi), 0.0])
        E = RNG.normal(size=3) * 1e8
        B = RNG.normal(size=3) * 10
        v1 = O.push_dirac(v, E, B, q, m, dt, vF)
        assert abs(np.linalg.norm(v1) / vF - 1) < 1e-12
        assert v1[2] == 0.0
    v = np.array([vF, 0, 0])
    assert np.allclose(O.push_dirac(v, np.zeros(3), np.zeros(3), q, m, dt, vF), v, rtol=1e-15)


def test_dirac_turns_toward_force():
    """A transverse E turns the direction by the Boris kick of mass m_d and
    never changes the speed (Sec. 5: infinite longitudinal mass)."""
    q, m, dt, vF = -QE, 0.0176 * ME, 1e-18, 1e6
    v = np.array([vF, 0, 0])
    E = np.array([0, 1e7, 0])
    v1 = O.push_dirac(v, E, np.zeros(3), q, m, dt, vF)
    dvy = q / m * E[1] * dt
    assert abs(v1[1] - vF * dvy / math.hypot(vF, dvy)) < 1e-9 * vF


# ---------------------------------------------------------------------------
# grid: gather, deposit, Yee (Sec. 4.1)
# ---------------------------------------------------------------------------

def _grid3(n=(8, 7, 6), bc=(0, 0, 0), **kw):
    g = dict(dims=3, n=n, d=(1e-9, 1.1e-9, 0.9e-9), dt=1e-18, bc=bc, pml_cells=0)
    g.update(kw)
    return g


def test_gather_is_exact_for_linear_fields_on_the_stagger():
    """CIC reproduces a field that is linear in position exactly when the
    nodes sit at the Yee stagger; a misplaced half cell breaks this."""
    s = O.OracleSim(**_grid3(bc=(1, 1, 1), pml_cells=0))
    nz, ny, nx = s.shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    stagE = [(0.5, 0, 0), (0, 0.5, 0), (0, 0, 0.5)]
    stagB = [(0, 0.5, 0.5), (0.5, 0, 0.5), (0.5, 0.5, 0)]
    coef = np.array([[1.0, 2.0, -3.0, 0.5], [2.0, -1.0, 0.25, 1.5], [-1.0, 0.5, 1.0, -2.0]])
    for c in range(3):
        a = coef[c]
        sx, sy, sz = stagE[c]
        s.set_field(c, a[0] + a[1] * (i + sx) + a[2] * (j + sy) + a[3] * (k + sz))
        sx, sy, sz = stagB[c]
        s.set_field(3 + c, 2 * a[0] + a[1] * (i + sx) - a[2] * (j + sy) + a[3] * (k + sz))
    s.step(0)
    # B^n is computed inside a step; with E linear, curl E is constant, so
    # check E directly and B through a zero-E copy
    for _ in range(20):
        X = RNG.uniform([1.5, 1.5, 1.5], [5.4, 4.4, 3.4])
        E, _ = s.gather(X)
        for c in range(3):
            a = coef[c]
            assert abs(E[c] - (a[0] + a[1] * X[0] + a[2] * X[1] + a[3] * X[2])) < 1e-12


def test_esirkepov_satisfies_continuity_exactly():
    """(rho(X1) - rho(X0))/dt + div J = 0 at every node, for moves with and
    without cell crossings, in 3D and 2D3V, across periodic edges."""
    for dims in (3, 2):
        n = (6, 5, 4) if dims == 3 else (6, 5, 1)
        g = dict(dims=dims, n=n, d=(1e-9, 1.3e-9, 0.8e-9), dt=1e-17, bc=(0, 0, 0))
        for trial in range(30):
            s = O.OracleSim(**g)
            X0 = RNG.uniform(0, 1, 3) * np.array(n)
            dX = RNG.uniform(-0.9, 0.9, 3)
            if trial % 3 == 0:
                dX *= 0.05
            if dims == 2:
                dX[2] = 0
            X1 = X0 + dX
            qw = -QE * 1e3
            s.deposit_one(X0, X1, qw, vz=2e5)
            Jx, Jy, Jz = s.J(0), s.J(1), s.J(2)
            V = 1e-9 * 1.3e-9 * 0.8e-9
            r0 = _rho_cic(dims, n, X0, qw / V)
            r1 = _rho_cic(dims, n, X1, qw / V)
            div = (Jx - np.roll(Jx, 1, axis=2)) / 1e-9 + (Jy - np.roll(Jy, 1, axis=1)) / 1.3e-9
            if dims == 3:
                div += (Jz - np.roll(Jz, 1, axis=0)) / 0.8e-9
            res = (r1 - r0) / 1e-17 + div
            assert np.abs(res).max() < 1e-12 * np.abs(r0).max() / 1e-17
            # total current = charge x velocity (for a straight move)
            vel = dX * np.array([1e-9, 1.3e-9, 0.8e-9]) / 1e-17
            assert abs(Jx.sum() * V - qw * vel[0]) < 1e-12 * abs(qw) * 1e8 + 1e-12 * abs(qw * vel[0])
            assert abs(Jy.sum() * V - qw * vel[1]) < 1e-12 * abs(qw) * 1e8 + 1e-12 * abs(qw * vel[1])
            if dims == 2:
                assert abs(Jz.sum() * V - qw * 2e5) < 1e-12 * abs(qw * 2e5)
            s.close()


def _rho_tsc(dims, n, X, qv):
    """Brute force: TSC weights of every node (periodic) for a point charge;
    the quadratic B-spline is 3/4 - d^2 below 1/2, (3/2 - d)^2 / 2 below 3/2."""
    nx, ny, nz = n
    out = np.zeros((nz, ny, nx))
    for k in range(nz if dims == 3 else 1):
        for j in range(ny):
            for i in range(nx):
                w = 1.0
                for a, idx in enumerate((i, j, k)[:dims]):
                    L = n[a]
                    d = (X[a] - idx) % L
                    d = min(d, L - d)
                    w *= 0.75 - d * d if d < 0.5 else (0.5 * (1.5 - d) ** 2 if d < 1.5 else 0.0)
                out[k, j, i] = qv * w
    return out


def test_tsc_weights_hand_computed():
    """A unit E_x at the single node (3.5, 3, 3) gathered at (3.8, 3.3,
    2.6) with TSC: offsets 0.3, 0.3, -0.4 give 0.66 x 0.66 x 0.59; the
    nodes one further out give (3/2 - 1.3)^2 / 2 = 0.02 along x."""
    s = O.OracleSim(**_grid3(bc=(0, 0, 0)))
    s.set_shape_order(2)
    Ex = np.zeros(s.shape)
    Ex[3, 3, 3] = 1.0
    s.set_field(0, Ex)
    E, _ = s.gather(np.array([3.8, 3.3, 2.6]))
    assert E[0] == pytest.approx(0.66 * 0.66 * 0.59, rel=1e-13)
    E, _ = s.gather(np.array([4.8, 3.3, 2.6]))  # x offset 1.3 from the node
    assert E[0] == pytest.approx(0.02 * 0.66 * 0.59, rel=1e-12)
    E, _ = s.gather(np.array([5.1, 3.3, 2.6]))  # 1.6: beyond the support
    assert E[0] == 0.0


def test_tsc_gather_is_exact_for_linear_fields():
    """TSC, like CIC, reproduces fields linear in position when the nodes
    sit at the Yee stagger."""
    s = O.OracleSim(**_grid3(bc=(1, 1, 1), pml_cells=0))
    s.set_shape_order(2)
    nz, ny, nx = s.shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    stagE = [(0.5, 0, 0), (0, 0.5, 0), (0, 0, 0.5)]
    coef = np.array([[1.0, 2.0, -3.0, 0.5], [2.0, -1.0, 0.25, 1.5], [-1.0, 0.5, 1.0, -2.0]])
    for c in range(3):
        a = coef[c]
        sx, sy, sz = stagE[c]
        s.set_field(c, a[0] + a[1] * (i + sx) + a[2] * (j + sy) + a[3] * (k + sz))
    for _ in range(20):
        X = RNG.uniform([2.1, 2.1, 2.1], [5.0, 4.0, 3.0])
        E, _ = s.gather(X)
        for c in range(3):
            a = coef[c]
            assert abs(E[c] - (a[0] + a[1] * X[0] + a[2] * X[1] + a[3] * X[2])) < 1e-12


def test_tsc_esirkepov_satisfies_continuity_exactly():
    """With TSC shapes: (rho(X1) - rho(X0))/dt + div J = 0 at every node
    against brute-force TSC charge densities, for moves with and without
    crossings of the nearest node, in 3D and 2D3V, across periodic edges;
    total current = charge x velocity."""
    for dims in (3, 2):
        n = (7, 6, 5) if dims == 3 else (7, 6, 1)
        g = dict(dims=dims, n=n, d=(1e-9, 1.3e-9, 0.8e-9), dt=1e-17, bc=(0, 0, 0))
        for trial in range(20):
            s = O.OracleSim(**g)
            s.set_shape_order(2)
            X0 = RNG.uniform(0, 1, 3) * np.array(n)
            dX = RNG.uniform(-0.9, 0.9, 3)
            if trial % 3 == 0:
                dX *= 0.05
            if dims == 2:
                dX[2] = 0
            X1 = X0 + dX
            qw = -QE * 1e3
            s.deposit_one(X0, X1, qw, vz=2e5)
            Jx, Jy, Jz = s.J(0), s.J(1), s.J(2)
            V = 1e-9 * 1.3e-9 * 0.8e-9
            r0 = _rho_tsc(dims, n, X0, qw / V)
            r1 = _rho_tsc(dims, n, X1, qw / V)
            div = (Jx - np.roll(Jx, 1, axis=2)) / 1e-9 + (Jy - np.roll(Jy, 1, axis=1)) / 1.3e-9
            if dims == 3:
                div += (Jz - np.roll(Jz, 1, axis=0)) / 0.8e-9
            res = (r1 - r0) / 1e-17 + div
            assert np.abs(res).max() < 1e-12 * np.abs(r0).max() / 1e-17
            vel = dX * np.array([1e-9, 1.3e-9, 0.8e-9]) / 1e-17
            assert abs(Jx.sum() * V - qw * vel[0]) < 1e-12 * abs(qw) * 1e8 + 1e-12 * abs(qw * vel[0])
            assert abs(Jy.sum() * V - qw * vel[1]) < 1e-12 * abs(qw) * 1e8 + 1e-12 * abs(qw * vel[1])
            if dims == 2:
                assert abs(Jz.sum() * V - qw * 2e5) < 1e-12 * abs(qw * 2e5)
            s.close()


def _rho_cic(dims, n, X, qv):
    """Brute force: CIC weights of every node (periodic) for a point charge."""
    nx, ny, nz = n
    out = np.zeros((nz, ny, nx))
    for k in range(nz if dims == 3 else 1):
        for j in range(ny):
            for i in range(nx):
                w = 1.0
                for a, idx in enumerate((i, j, k)[:dims]):
                    L = n[a]
                    d = (X[a] - idx) % L
                    d = min(d, L - d)
                    w *= max(0.0, 1 - d)
                out[k, j, i] = qv * w
    return out


def _plane_wave_check(axis, pol, nsteps=200):
    """Vacuum eigenmode of the Yee scheme: with sin^2(w dt/2)/(c dt)^2 =
    sin^2(k d/2)/d^2 the discrete wave E_pol = cos(k x - w t) stays a pure
    travelling wave, B = E / c rotated by the propagation direction."""
    n = [4, 4, 4]
    n[axis] = 32
    d = [1e-9, 1e-9, 1e-9]
    dt = 0.5 * 1e-9 / (C * math.sqrt(3))
    g = dict(dims=3, n=n, d=d, dt=dt, bc=(0, 0, 0))
    s = O.OracleSim(**g)
    kk = 2 * math.pi * 3 / (n[axis] * d[axis])
    w = 2 / dt * math.asin(C * dt / d[axis] * math.sin(kk * d[axis] / 2))
    nz, ny, nx = s.shape
    idx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    pos = [idx[2], idx[1], idx[0]][axis].astype(float)
    bcomp = 3 - axis - pol  # the remaining axis
    sign = 1.0 if (axis, pol, bcomp) in ((0, 1, 2), (1, 2, 0), (2, 0, 1)) else -1.0
    E = np.cos(kk * pos * d[axis])  # E_pol sits at an integer position along `axis`
    s.set_field(pol, E)
    # B_bcomp sits at a half position along `axis`, time n - 1/2
    Bv = sign / C * np.cos(kk * (pos + 0.5) * d[axis] + w * dt / 2)
    s.set_field(3 + bcomp, Bv)
    s.step(nsteps)
    E1 = s.field(pol)
    pred = np.cos(kk * pos * d[axis] - w * nsteps * dt)
    assert np.abs(E1 - pred).max() < 1e-9
    B1 = s.field(3 + bcomp)
    predB = sign / C * np.cos(kk * (pos + 0.5) * d[axis] - w * (nsteps - 0.5) * dt)
    assert np.abs(B1 - predB).max() < 1e-9 / C
    for c in range(3):
        if c != pol:
            assert np.abs(s.field(c)).max() < 1e-12


def test_yee_plane_waves_follow_numerical_dispersion():
    for axis, pol in ((0, 1), (0, 2), (1, 2), (1, 0), (2, 0), (2, 1)):
        _plane_wave_check(axis, pol)


def _eigenmode(axis, pol, nsteps):
    """The vacuum Yee eigenmode of _plane_wave_check, stepped nsteps times;
    returns (sim, grid positions along `axis`, k, w, B component, sign)."""
    n = [4, 4, 4]
    n[axis] = 32
    d = [1e-9, 1e-9, 1e-9]
    dt = 0.5 * 1e-9 / (C * math.sqrt(3))
    s = O.OracleSim(dims=3, n=n, d=d, dt=dt, bc=(0, 0, 0))
    kk = 2 * math.pi * 3 / (n[axis] * d[axis])
    w = 2 / dt * math.asin(C * dt / d[axis] * math.sin(kk * d[axis] / 2))
    nz, ny, nx = s.shape
    idx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    pos = [idx[2], idx[1], idx[0]][axis].astype(float)
    bcomp = 3 - axis - pol
    sign = 1.0 if (axis, pol, bcomp) in ((0, 1, 2), (1, 2, 0), (2, 0, 1)) else -1.0
    s.set_field(pol, np.cos(kk * pos * d[axis]))
    s.set_field(3 + bcomp, sign / C * np.cos(kk * (pos + 0.5) * d[axis] + w * dt / 2))
    s.step(nsteps)
    return s, pos, kk, w, bcomp, sign, d[axis], dt


def test_gather_B_is_the_integer_step_average_of_the_eigenmode():
    """B at integer time for the gather (Sec. 4.1: E on integer steps, B on
    half steps): B^n = B^{n-1/2} - (dt/2) curl E^n must equal the mean of the
    eigenmode's half-step values B^{n-1/2} and B^{n+1/2}, i.e.
    cos(w dt / 2) times the travelling wave at t_n.  The last step's gather
    used n = nsteps - 1; both the stored B^n and the B a particle gathers
    (linear interpolation along the wave between the B nodes) are checked.
    A sign or a factor 2 wrong in the half-step correction moves B^n to
    B^{n-1/2} + (dt/2) curl E^n or to B^{n+1/2}."""
    nsteps = 37
    for axis, pol in ((0, 1), (0, 2), (1, 2), (1, 0), (2, 0), (2, 1)):
        s, pos, kk, w, bcomp, sign, da, dt = _eigenmode(axis, pol, nsteps)
        tn = (nsteps - 1) * dt
        amp = sign / C * math.cos(w * dt / 2)
        pred = amp * np.cos(kk * (pos + 0.5) * da - w * tn)
        Bn = s.field(9 + bcomp)
        assert np.abs(Bn - pred).max() < 1e-10 / C, (axis, pol)
        # the other components of B^n vanish with the wave's
        for c in range(3):
            if c != bcomp:
                assert np.abs(s.field(9 + c)).max() < 1e-14 / C
        # a particle gathers B^n: along the wave the B node sits at m + 1/2
        for _ in range(10):
            X = RNG.uniform([0.0, 0.0, 0.0], [4.0, 4.0, 4.0])
            X[axis] = RNG.uniform(2.0, 29.0)
            _, B = s.gather(X)
            m0 = math.floor(X[axis] - 0.5)
            f = X[axis] - 0.5 - m0
            node = lambda m: amp * math.cos(kk * (m + 0.5) * da - w * tn)
            want = (1 - f) * node(m0) + f * node(m0 + 1)
            assert abs(B[bcomp] - want) < 1e-10 / C, (axis, pol, X)
        s.close()


def test_diag_energies_hand_computed():
    """orc_diag's sums (Sec. 2: energy as a derived quantity): the kinetic
    energy sum(m w |v|^2 / 2) of a few hand-placed particles of two species
    with different masses and weights; the field energy of uniform E and B
    (eps0 |E|^2 V / 2 and |B|^2 V / (2 mu0) per cell); and of the standing
    wave E_y = E0 cos(k x) with an integer number of wavelengths on the grid,
    whose cell sum is exactly eps0 E0^2 V N / 4."""
    g = _grid3(n=(8, 6, 4), bc=(0, 0, 0))
    V = g["d"][0] * g["d"][1] * g["d"][2]
    N = 8 * 6 * 4
    mu0 = 1.0 / (EPS0 * C * C)
    s = O.OracleSim(**g)
    X = np.array([[1.2, 2.5, 0.5], [3.7, 0.1, 2.9], [6.0, 5.5, 1.0]])
    V1 = np.array([[1e5, -2e5, 3e5], [0.0, 0.0, -4e5], [2.5e5, 1e5, 0.0]])
    V2 = np.array([[-3e4, 7e4, 1e4], [5e4, 0.0, 2e4]])
    s.add_species(O.KIND_FREE, -QE, ME, 3.0, X, V1)
    s.add_species(O.KIND_FREE, QE, 7.0 * ME, 0.25, X[:2], V2)
    E0 = (2.0e7, -1.0e7, 5.0e6)
    B0 = (0.3, 0.0, -0.2)
    for c in range(3):
        s.set_field(c, np.full(s.shape, E0[c]))
        s.set_field(3 + c, np.full(s.shape, B0[c]))
    d = s.diag()
    k1 = 0.5 * ME * 3.0 * (1e10 + 4e10 + 9e10 + 16e10 + 6.25e10 + 1e10)
    k2 = 0.5 * 7.0 * ME * 0.25 * (9e8 + 49e8 + 1e8 + 25e8 + 4e8)
    assert abs(d["kinetic"][0] / k1 - 1) < 1e-14
    assert abs(d["kinetic"][1] / k2 - 1) < 1e-14
    uE = 0.5 * EPS0 * (4e14 + 1e14 + 0.25e14) * V * N
    uB = 0.5 / mu0 * (0.09 + 0.04) * V * N
    assert abs(d["field_E"] / uE - 1) < 1e-13
    assert abs(d["field_B"] / uB - 1) < 1e-13
    s.close()
    s = O.OracleSim(**g)
    i = np.arange(8)
    for c in range(6):
        s.set_field(c, np.zeros(s.shape))
    s.set_field(1, np.broadcast_to(3e7 * np.cos(2 * math.pi * 2 * i / 8), s.shape))
    d = s.diag()
    assert abs(d["field_E"] / (EPS0 * 9e14 * V * N / 4) - 1) < 1e-13
    assert d["field_B"] == 0.0
    s.close()


def test_dt_limit_closed_forms():
    d = [0.5e-9] * 3
    assert abs(O.dt_limit(3, d, 0, 0) - d[0] / (C * math.sqrt(3))) < 1e-30
    assert abs(O.dt_limit(2, d, 0, 0) - d[0] / (C * math.sqrt(2))) < 1e-30
    big = 1e22
    assert abs(O.dt_limit(3, d, big, 0) * big / 2 - 1) < 1e-6
    assert abs(O.dt_limit(3, d, 0, big) * big / 2 - 1) < 1e-6


# ---------------------------------------------------------------------------
# material boundary (Sec. 3) and whole-step invariants
# ---------------------------------------------------------------------------

def test_reflection_hand_computed():
    for r in _rows("reflection_single.txt"):
        v = [float(x) for x in r]
        g = dict(dims=3, n=(8, 8, 8), d=(1e-9, 1e-9, 1e-9), dt=1e-17, bc=(0, 0, 0))
        s = O.OracleSim(**g)
        mask = np.zeros((8, 8, 8), np.uint8)
        mask[:, :, :5] = 1
        s.set_mask(mask)
        s.add_species(O.KIND_FREE, -QE, ME, 1.0, [v[0:3]], [v[3:6]])
        s.step(1)
        X, V, _, nr = s.species(0)
        assert np.allclose(X[0], v[6:9], atol=1e-12)
        assert np.allclose(V[0], v[9:12], rtol=1e-12)
        assert nr == int(v[12])


def _sphere_setup(seed=5, n=12, with_bound=True, bg=1, bc=(1, 1, 1), order=1):
    g = dict(dims=3, n=(n, n, n), d=(0.5e-9,) * 3, dt=0.5 * 0.5e-9 / (C * math.sqrt(3)),
             bc=bc, pml_cells=2 if bc[0] else 0)
    s = O.OracleSim(**g)
    s.set_shape_order(order)
    kk, jj, ii = np.meshgrid(*(np.arange(n),) * 3, indexing="ij")
    r = np.sqrt((ii + 0.5 - n / 2) ** 2 + (jj + 0.5 - n / 2) ** 2 + (kk + 0.5 - n / 2) ** 2)
    mask = (r < n / 2 - 2.5).astype(np.uint8)
    s.set_mask(mask)
    cell, off, v = O.fd_load(3, (n, n, n), mask, O.KIND_FREE, ME, 5.5 * QE, 300.0, 0.0, 8,
                             False, seed, 0)
    cz, rem = np.divmod(cell, n * n)
    cy, cx = np.divmod(rem, n)
    X = np.stack([cx, cy, cz], 1) + off
    V = v * 40.0  # hot enough that many particles hit the wall in a few steps
    w = 5.9e28 * (0.5e-9) ** 3 / 8
    s.add_species(O.KIND_FREE, -QE, ME, w, X, V, bg=bg)
    if with_bound:
        cellb, offb, vb = O.fd_load(3, (n, n, n), mask, O.KIND_BOUND, ME, 0, 0, 0, 8, True,
                                    seed, 1)
        cz, rem = np.divmod(cellb, n * n)
        cy, cx = np.divmod(rem, n)
        Xb = np.stack([cx, cy, cz], 1) + offb
        Vb = RNG.normal(size=Xb.shape) * 1e5
        s.add_species(O.KIND_BOUND, -QE, ME, 0.5 * w, Xb, Vb, omega0=[4.709e15] * 3,
                      gamma=[1e14] * 3, bg=bg)
    return s, mask


def test_reflection_conserves_count_and_keeps_particles_inside():
    s, mask = _sphere_setup(with_bound=False)
    n0 = s.species(0)[0].shape[0]
    for _ in range(10):
        s.step(5)
        X, V, _, nr = s.species(0)
        assert X.shape[0] == n0
        c = np.floor(X).astype(int)
        assert np.all(mask[c[:, 2], c[:, 1], c[:, 0]] == 1)
    assert nr > 0
    assert np.array_equal(s.cell_counts(0).sum(), n0)


@pytest.mark.parametrize("order", [1, 2])
def test_gauss_law_is_preserved_by_the_step(order):
    """Charge-conserving deposit + Yee: div E - rho/eps0 stays at its initial
    value (zero here: quiet ions at the loaded positions, E = 0).  Periodic
    walls: the CPML layer is not a charge-conserving medium.  Order 2: the
    free electrons deposit and gather with TSC, the bound ones with CIC."""
    s, _ = _sphere_setup(with_bound=True, bg=1, bc=(0, 0, 0), order=order)
    d0 = s.diag()
    qscale = QE * 5.9e28 / 8 / EPS0  # charge density of one macro-particle / eps0
    assert d0["gauss_max"] < 1e-12 * qscale
    for _ in range(4):
        s.step(5)
        d = s.diag()
        assert d["gauss_max"] < 1e-10 * qscale
    assert d["field_E"] > 0


# ---------------------------------------------------------------------------
# source and absorbing layer
# ---------------------------------------------------------------------------

def _source_run(nsteps, probe_off=20):
    n = (160, 2, 1)
    d = (1e-9, 1e-9, 1e-9)
    dt = 0.5 * 1e-9 / (C * math.sqrt(2))
    lam = 40e-9
    w = 2 * math.pi * C / lam
    tau = 1.2e-16
    t0 = 1.5 * tau
    g = dict(dims=2, n=n, d=d, dt=dt, bc=(1, 0, 0), pml_cells=16, src=True, inc_axis=0,
             pol_axis=1, src_index=40, E0=1e8, omega=w, tau=tau, t0=t0)
    s = O.OracleSim(**g)
    trace = []
    for _ in range(nsteps):
        s.step(1)
        trace.append(s.field(1)[0, 0, 40 + probe_off])
    return s, np.array(trace), g


def test_soft_source_launches_E0_pulse():
    """The current sheet J = -2 E0 g(t) / (eta0 dx) radiates E_pol = E0 g(t -
    x/c) on both sides (the field of an infinite sheet is -eta0 K / 2)."""
    s, trace, g = _source_run(900)
    dt = g["dt"]
    t = (np.arange(900) + 1) * dt
    delay = 20 * 1e-9 / C
    tt = t - delay - g["t0"]
    pred = 1e8 * np.exp(-2 * math.log(2) * tt ** 2 / g["tau"] ** 2) * np.sin(g["omega"] * tt)
    assert np.abs(trace - pred).max() < 0.03 * 1e8
    s.close()


def test_cpml_absorbs_the_pulse():
    """Parity unpinned for the absorption coefficient: only the decay of the
    field energy after the pulse has entered the layers is checked."""
    s, trace, g = _source_run(2200)
    Ey = s.field(1)
    assert np.abs(Ey).max() < 2e-3 * 1e8
    s.close()


# ---------------------------------------------------------------------------
# collective physics (closed forms of the plasma)
# ---------------------------------------------------------------------------

def _fit_frequency(t, y, w_guess):
    """Least-squares fit of y = a cos(w t) + b sin(w t) + c over w."""
    best = None
    for w in np.linspace(0.8 * w_guess, 1.2 * w_guess, 4001):
        A = np.stack([np.cos(w * t), np.sin(w * t), np.ones_like(t)], 1)
        coef, res, *_ = np.linalg.lstsq(A, y, rcond=None)
        r = np.sum((A @ coef - y) ** 2)
        if best is None or r < best[0]:
            best = (r, w)
    return best[1]


@pytest.mark.slow
def test_langmuir_frequency():
    """Periodic 2D3V electron plasma with a 1% density ripple oscillates at
    w_p = sqrt(n e^2 / (eps0 m)) (Bohm-Gross shift (3/5) k^2 v_F^2 included)."""
    n0 = 8.5e28
    nx, ny = 64, 4
    dx = 0.1e-9
    dt = 0.5 * dx / (C * math.sqrt(2))
    g = dict(dims=2, n=(nx, ny, 1), d=(dx, dx, dx), dt=dt, bc=(0, 0, 0))
    s = O.OracleSim(**g)
    cell, off, v = O.fd_load(2, (nx, ny, 1), None, O.KIND_FREE, ME, 7.0 * QE, 300.0, 0.0, 16,
                             True, 11, 0)
    cy, cx = np.divmod(cell, nx)
    X = np.stack([cx, cy, np.zeros_like(cx)], 1) + off
    k = 2 * math.pi / (nx * dx)
    A = 0.01
    X[:, 0] = X[:, 0] - A / (k * dx) * np.sin(k * X[:, 0] * dx)
    w = n0 * dx ** 3 / 16
    s.add_species(O.KIND_FREE, -QE, ME, w, X, v, bg=2)
    i = np.arange(nx)
    Ex = -(QE * n0 * A / (EPS0 * k)) * np.sin(k * (i + 0.5) * dx)
    s.set_field(0, np.broadcast_to(Ex, (1, ny, nx)))
    wp = math.sqrt(n0 * QE ** 2 / (EPS0 * ME))
    nsteps = int(2.2 * 2 * math.pi / (wp * dt))
    t, y = [], []
    for it in range(nsteps // 10):
        s.step(10)
        E = s.field(0)[0].mean(axis=0)
        y.append(2 / nx * np.sum(E * np.sin(k * (i + 0.5) * dx)))
        t.append((it + 1) * 10 * dt)
    wfit = _fit_frequency(np.array(t), np.array(y), wp)
    vF = math.sqrt(2 * 7.0 * QE / ME)
    wbg = math.sqrt(wp ** 2 + 0.6 * k ** 2 * vF ** 2)
    assert abs(wfit / wp - 1) < 0.01
    assert abs(wfit / wbg - 1) < 0.01


def sheet_plasmon_closed_form(ns, q, m_pl, Lz, vF):
    """2D plasmon of a sheet of carriers (density ns, plasmon mass m_pl per
    carrier, Sec. 5) in vacuum: w^2 = ns e^2 kappa g / (2 eps0 m_pl), kappa =
    sqrt(q^2 - w^2 / c^2) (the field's decay rate off the sheet, equal to q
    without retardation).  On a grid periodic in z with period Lz the sheet's
    images multiply the field at the sheet by coth(kappa Lz / 2).  Carriers
    that all move at v_F in uniformly spread directions answer a wave of
    phase velocity w / q with the factor g(s) = 2 (1/sqrt(1 - s^2) - 1) / s^2,
    s = q v_F / w (collisionless response of a ring of velocities; 1 + 3 s^2
    / 4 for small s).  Solved by fixed-point iteration."""
    w2 = ns * QE ** 2 * q / (2 * EPS0 * m_pl)
    for _ in range(60):
        kap = math.sqrt(q * q - w2 / C ** 2)
        s2 = (q * vF) ** 2 / w2
        g = 2 * (1 / math.sqrt(1 - s2) - 1) / s2
        w2 = ns * QE ** 2 * kap / math.tanh(kap * Lz / 2) * g / (2 * EPS0 * m_pl)
    return math.sqrt(w2)


def sheet_plasmon_particles(nx, ny, k0, q, dx, vF, ppc_side=4, drift=0.1):
    """Quiet start of a Dirac sheet in the node plane z = k0: a
    ppc_side x ppc_side lattice per cell, the carriers' in-plane directions
    evenly spaced (so every cell carries no current), each direction then
    tilted toward +x by drift * cos(q x) and renormalised to v_F.  Only the
    part transverse to the direction survives the renormalisation, so the
    sheet starts with a current ~ (drift / 2) v_F cos(q x) and no charge
    ripple (Gauss's law holds with E = 0)."""
    ppc = ppc_side * ppc_side
    a, b = np.meshgrid(np.arange(ppc_side), np.arange(ppc_side), indexing="ij")
    a, b = a.ravel(), b.ravel()
    th = 2 * math.pi * (a * ppc_side + b + 0.5) / ppc
    X, Vv = [], []
    for j in range(ny):
        for i in range(nx):
            x = i + (a + 0.5) / ppc_side
            ux = np.cos(th) + drift * np.cos(q * x * dx)
            uy = np.sin(th)
            nrm = np.hypot(ux, uy)
            X.append(np.stack([x, j + (b + 0.5) / ppc_side, np.full(ppc, float(k0))], 1))
            Vv.append(np.stack([vF * ux / nrm, vF * uy / nrm, np.zeros(ppc)], 1))
    return np.concatenate(X), np.concatenate(Vv), ppc


@pytest.mark.slow
@pytest.mark.parametrize("mode", [1, 2])
def test_sheet_plasmon_frequency(mode):
    """Dirac carriers of a sheet (Sec. 5) pushed with the averaged transverse
    mass m_d = p_F / (2 v_F) oscillate collectively with the plasmon mass
    m_pl = 2 m_d = p_F / v_F: the ringing of the sheet's in-plane E at
    q = 2 pi mode / L_x matches the 2D plasmon closed form within 1 %, at two
    wavenumbers.  (Using m_d itself as the plasmon mass, or pushing without
    the renormalisation, is off by sqrt(2).)"""
    nx, ny, nz = 64, 2, 32
    dx = 10e-9
    dt = 0.5 * dx / (C * math.sqrt(3))
    ns, EF, vF = 4e17, 0.2 * QE, 1e6
    pF = EF / vF
    md, mpl = pF / (2 * vF), pF / vF
    q = 2 * math.pi * mode / (nx * dx)
    w = sheet_plasmon_closed_form(ns, q, mpl, nz * dx, vF)
    k0 = nz // 2
    X, Vv, ppc = sheet_plasmon_particles(nx, ny, k0, q, dx, vF)
    s = O.OracleSim(dims=3, n=(nx, ny, nz), d=(dx, dx, dx), dt=dt, bc=(0, 0, 0))
    s.add_species(O.KIND_DIRAC, -QE, md, ns * dx * dx / ppc, X, Vv, vF=vF, bg=1)
    nsteps = int(1.5 * 2 * math.pi / (w * dt))
    every = max(1, nsteps // 300)
    xi = (np.arange(nx) + 0.5) * dx
    t, y = [], []
    for it in range(nsteps // every):
        s.step(every)
        y.append(np.sum(s.field(0)[k0].mean(axis=0) * np.cos(q * xi)))
        t.append((it + 1) * every * dt)
    _, V1, _, _ = s.species(0)
    assert np.abs(np.linalg.norm(V1, axis=1) / vF - 1).max() < 1e-12
    wfit = _fit_frequency(np.array(t), np.array(y), w)
    assert abs(wfit / w - 1) < 0.01, (mode, wfit, w)
    s.close()


@pytest.mark.slow
def test_bound_medium_longitudinal_resonance():
    """Uniform Lorentz medium (periodic) with a k-mode displacement rings at
    w_L = sqrt(w0^2 + w_pb^2 - gamma^2/4) and decays as exp(-gamma t / 2)."""
    nb = 0.5 * 5.9e28
    nx, ny = 32, 2
    dx = 0.5e-9
    dt = 0.5 * dx / (C * math.sqrt(2))
    w0, gam = 4.709e15, 1e14
    g = dict(dims=2, n=(nx, ny, 1), d=(dx, dx, dx), dt=dt, bc=(0, 0, 0))
    s = O.OracleSim(**g)
    cell, off, v = O.fd_load(2, (nx, ny, 1), None, O.KIND_BOUND, ME, 0, 0, 0, 16, True, 3, 0)
    cy, cx = np.divmod(cell, nx)
    X = np.stack([cx, cy, np.zeros_like(cx)], 1) + off
    k = 2 * math.pi / (nx * dx)
    D = np.zeros_like(X)
    D[:, 0] = 1e-12 * np.sin(k * X[:, 0] * dx)
    w = nb * dx ** 3 / 16
    s.add_species(O.KIND_BOUND, -QE, ME, w, X, v, D=D, omega0=[w0] * 3, gamma=[gam] * 3, bg=1)
    i = np.arange(nx)
    # Gauss-consistent start: E = -P / eps0 with P = n_b q D
    Ex = -nb * (-QE) * 1e-12 * np.sin(k * (i + 0.5) * dx) / EPS0
    s.set_field(0, np.broadcast_to(Ex, (1, ny, nx)))
    wpb2 = nb * QE ** 2 / (EPS0 * ME)
    wL = math.sqrt(w0 ** 2 + wpb2 - gam ** 2 / 4)
    nsteps = int(3 * 2 * math.pi / (wL * dt))
    t, y = [], []
    i = np.arange(nx)
    for it in range(nsteps // 5):
        s.step(5)
        E = s.field(0)[0].mean(axis=0)
        y.append(2 / nx * np.sum(E * np.sin(k * (i + 0.5) * dx)))
        t.append((it + 1) * 5 * dt)
    t, y = np.array(t), np.array(y)
    wfit = _fit_frequency(t, y * np.exp(gam * t / 2), wL)
    assert abs(wfit / wL - 1) < 0.01
    # decay: envelope ratio over the run
    A = np.stack([np.cos(wL * t), np.sin(wL * t)], 1)
    half = len(t) // 2
    a1 = np.linalg.lstsq(A[:half], y[:half], rcond=None)[0]
    a2 = np.linalg.lstsq(A[half:], y[half:], rcond=None)[0]
    ratio = np.linalg.norm(a2) / np.linalg.norm(a1)
    pred = math.exp(-gam / 2 * (t[half:].mean() - t[:half].mean()))
    assert abs(ratio / pred - 1) < 0.05


def test_dielectric_half_space_fresnel():
    """Eq. consteps with eps = eps0 eps_r: a plane-wave pulse in vacuum meeting
    a half-space of eps_r = 4 (n = 2) at normal incidence reflects with
    r = (1 - n) / (1 + n) = -1/3 and transmits t = 2 / (1 + n) = 2/3 (Fresnel;
    the medium has no dispersion, so the whole pulse scales by r and t).  The
    pulse is smooth on the grid (80 cells per wavelength)."""
    nx = 1200
    n = (nx, 2, 1)
    d = (1e-9, 1e-9, 1e-9)
    dt = 0.5 * 1e-9 / (C * math.sqrt(2))
    lam = 80e-9
    tau = 0.25e-15
    g = dict(dims=2, n=n, d=d, dt=dt, bc=(1, 0, 0), pml_cells=16, src=True, inc_axis=0,
             pol_axis=1, src_index=40, E0=1e8, omega=2 * math.pi * C / lam, tau=tau,
             t0=3 * tau)
    s = O.OracleSim(**g)
    eps = np.ones((1, 2, nx))
    eps[..., 700:] = 4.0
    s.set_permittivity(eps)
    pa, pb = 200, 800
    nsteps = int((3 * tau * C / 1e-9 + 1560) / (C * dt / 1e-9))
    ta, ea, eb = [], [], []
    for it in range(nsteps):
        s.step(1)
        E = s.field(1)[0, 0]
        ta.append((it + 1) * dt)
        ea.append(E[pa])
        eb.append(E[pb])
    t, ea, eb = np.array(ta), np.abs(ea), np.abs(eb)
    split = 3 * tau + (pa - 40 + 500) * 1e-9 / C  # between incident and reflected at probe A
    inc = ea[t < split].max()
    ref = ea[t > split].max()
    tra = eb.max()
    assert abs(ref / inc - 1 / 3) < 0.02 / 3
    assert abs(tra / inc - 2 / 3) < 0.02 * 2 / 3
    s.close()


def test_gauss_law_holds_for_D_in_a_dielectric():
    """With a permittivity the step preserves the discrete Gauss law for
    D = eps0 eps_r E (Eq. consteps): starting neutral (ions at the loaded
    positions, E = 0), div(eps_r E) - rho/eps0 stays at roundoff while
    electrons move through and out of a dielectric slab."""
    rng = np.random.default_rng(17)
    n = (12, 10, 8)
    d = (1e-9, 1e-9, 1e-9)
    dt = 0.5 * 1e-9 / (C * math.sqrt(3))
    s = O.OracleSim(dims=3, n=n, d=d, dt=dt, bc=(0, 0, 0))
    eps = np.ones((8, 10, 12))
    eps[:, :, 4:9] = 3.0
    s.set_permittivity(eps)
    npart = 400
    X = rng.random((npart, 3)) * np.array(n)
    V = rng.normal(size=(npart, 3)) * 3e6
    w = 5.9e28 * 1e-27 / 4
    s.add_species(O.KIND_FREE, -QE, ME, w, X, V, bg=1)
    qscale = QE * w / 1e-27 / EPS0  # charge density of one macro-particle / eps0
    assert s.diag()["gauss_max"] < 1e-12 * qscale
    for _ in range(4):
        s.step(5)
        dg = s.diag()
        assert dg["gauss_max"] < 1e-10 * qscale
    assert dg["field_E"] > 0
    s.close()


@pytest.mark.slow
def test_lorentz_half_space_reflection_spectrum():
    """Sec. 4, Eq. lordielectric: the oracle's bound species, deposit and Yee
    update together make a medium whose reflection spectrum is Fresnel's with
    eps(omega) = 1 + w_pb^2 / (w0^2 - w^2 - i gamma w) (discrete form):
    within 1 % over w = 0.34 .. 0.66 w0 (the setup of the GPU test of the
    same name)."""
    from tests import pairs as PR
    grid, mask, sp, steps, prm = PR.lorentz_half_space_case()
    g = dict(grid)
    src = g.pop("src")
    g.update(src=True, **src)
    s = O.OracleSim(**g)
    s.set_mask(mask)
    n = grid["n"]
    cell, off, v = O.fd_load(2, n, mask, O.KIND_BOUND, ME, 0.0, 0.0, 0.0, sp["ppc"], True,
                             sp["seed"], 0)
    cy, cx = np.divmod(cell, n[0])
    X = np.stack([cx, cy, np.zeros_like(cx)], 1) + off
    w = sp["density"] * np.prod(grid["d"]) / sp["ppc"]
    s.add_species(O.KIND_BOUND, -QE, ME, w, X, v, D=np.zeros_like(X), omega0=sp["omega0"],
                  gamma=sp["gamma"], bg=1)
    trace = np.zeros(steps)
    for it in range(steps):
        s.step(1)
        trace[it] = s.field(1)[0, 0, 100]
    s.close()
    err, band = PR.lorentz_reflection_error(trace, **prm)
    assert band.min() < 0.36 * prm["w0"] and band.max() > 0.64 * prm["w0"]
    assert err < 0.01, err


# ---------------------------------------------------------------------------
# particle boundary variants (Sec. 3): work-function barrier, open edges,
# diffusive reflection
# ---------------------------------------------------------------------------

def _slab_sim(n=(24, 4, 4), lo=6, hi=14, dims=3, d=(0.45e-9, 0.5e-9, 0.4e-9), axis=0):
    dt = 0.5 * min(d[:dims]) / (C * math.sqrt(dims))
    s = O.OracleSim(dims=dims, n=n, d=d, dt=dt, bc=(0, 0, 0), pml_cells=0)
    m = np.zeros(s.shape, np.uint8)
    sl = [slice(None)] * 3
    sl[2 - axis] = slice(lo, hi)
    m[tuple(sl)] = 1
    s.set_mask(m)
    return s, m


@pytest.mark.parametrize("dims,axis", [(3, 0), (3, 1), (3, 2), (2, 0), (2, 1)])
def test_work_function_planar_barrier_closed_form(dims, axis):
    """A planar surface: the node potential steps 0 -> -W/2 -> -W (vacuum
    fraction 0, 1/2, 1), so E along the normal is W / (2 d) on the two half
    nodes beside each face (sign: pushing electrons back into the slab) and
    zero elsewhere; the tangential components vanish."""
    n = [10, 10, 10 if dims == 3 else 1]
    s, _ = _slab_sim(n=tuple(n), lo=3, hi=7, dims=dims, axis=axis)
    d = (0.45e-9, 0.5e-9, 0.4e-9)
    W = 4.3
    E = s.work_function_field(W)
    for c in range(3):
        if c != axis:
            assert np.all(E[c] == 0.0)
    line = np.moveaxis(E[axis], 2 - axis, -1).reshape(-1, n[axis])
    want = np.zeros(n[axis])
    # face at 3 (vacuum below): an electron there is pushed up, E < 0
    want[2] = want[3] = -W / (2 * d[axis])
    # face at 7 (vacuum above): pushed down, E > 0
    want[6] = want[7] = W / (2 * d[axis])
    for row in line:
        np.testing.assert_allclose(row, want, rtol=1e-14, atol=0)


def test_work_function_corner_and_gradient_invariants():
    """A material cube in vacuum: hand-computed values at an outer corner
    (node vacuum fraction 7/8) and edge (3/4), and the field is a discrete
    gradient: its Yee curl vanishes everywhere."""
    d = (0.45e-9, 0.5e-9, 0.4e-9)
    s = O.OracleSim(dims=3, n=(9, 8, 7), d=d, dt=1e-19, bc=(0, 1, 0), pml_cells=1)
    m = np.zeros(s.shape, np.uint8)
    m[2:5, 2:6, 3:7] = 1          # z in [2,5), y in [2,6), x in [3,7)
    s.set_mask(m)
    W = 3.0
    ex, ey, ez = s.work_function_field(W)
    # E_x of cell (2, 2, 2) sits between nodes (2,2,2) (vacuum fraction 1,
    # outside the cube) and (3,2,2) (the cube's corner: 7/8)
    assert ex[2, 2, 2] == pytest.approx(W * (7 / 8 - 1) / d[0], rel=1e-14)
    # E_x of cell (3, 3, 2): node (3,3,2) on an edge (3/4) -> (4,3,2) on a face (1/2)
    assert ex[2, 3, 3] == pytest.approx(W * (1 / 2 - 3 / 4) / d[0], rel=1e-14)
    # E_z of cell (4, 4, 4): nodes (4,4,4) inside (0) -> (4,4,5) on the top face (1/2)
    assert ez[4, 4, 4] == pytest.approx(W * (1 / 2 - 0) / d[2], rel=1e-14)
    # the Yee curl of a gradient is zero (interior cells)
    scale = W / min(d)
    cxy = (ey[:, :-1, 1:] - ey[:, :-1, :-1]) / d[0] - (ex[:, 1:, :-1] - ex[:, :-1, :-1]) / d[1]
    cyz = (ez[:-1, 1:, :] - ez[:-1, :-1, :]) / d[1] - (ey[1:, :-1, :] - ey[:-1, :-1, :]) / d[2]
    czx = (ex[1:, :, :-1] - ex[:-1, :, :-1]) / d[2] - (ez[:-1, :, 1:] - ez[:-1, :, :-1]) / d[0]
    for cc in (cxy, cyz, czx):
        assert np.abs(cc).max() < 1e-12 * scale / min(d)


def test_external_field_gather_is_exact_for_linear_fields():
    """The external field is interpolated on the E stagger like E itself: a
    field linear in position (sampled at the E nodes) is reproduced exactly
    while the Maxwell E stays zero."""
    d = (1e-9, 1.1e-9, 0.9e-9)
    s = O.OracleSim(dims=3, n=(8, 7, 6), d=d, dt=1e-18, bc=(0, 0, 0), pml_cells=0)
    kk, jj, ii = np.meshgrid(np.arange(6), np.arange(7), np.arange(8), indexing="ij")
    coef = [(1.0, -2.0, 0.5, 3.0), (-0.7, 0.3, 1.1, -2.0), (0.2, 0.9, -1.3, 1.0)]
    stag = [(0.5, 0, 0), (0, 0.5, 0), (0, 0, 0.5)]
    E = []
    for c in range(3):
        a, b, e, f = coef[c]
        E.append(1e6 * (a * (ii + stag[c][0]) + b * (jj + stag[c][1]) + e * (kk + stag[c][2]) + f))
    s.set_external_field(E)
    for X in ([2.3, 3.7, 2.1], [4.9, 1.2, 3.5], [3.5, 3.5, 2.5]):
        Eg, Bg = s.gather(np.array(X))
        for c in range(3):
            a, b, e, f = coef[c]
            assert Eg[c] == pytest.approx(1e6 * (a * X[0] + b * X[1] + e * X[2] + f), rel=1e-12)
        assert np.all(Bg == 0.0)
    assert np.all(s.field(0) == 0.0)


def _wall_run(K_over_W, W=4.0, vt=(3e4, -2e4)):
    s, _ = _slab_sim()
    s.set_external_field(s.work_function_field(W))
    s.set_particle_bc(open_edges=True)
    v0 = math.sqrt(2 * K_over_W * W * QE / ME)
    s.add_species(O.KIND_FREE, -QE, ME, 1e-12, [[10.3, 1.5, 2.2]], [[v0, vt[0], vt[1]]])
    for _ in range(400):
        s.step(50)
        X, V, _, nr = s.species(0)
        if X[0, 0] > 18.0 or (X[0, 0] < 10.3 and V[0, 0] < 0):
            return X[0], V[0], nr
    raise AssertionError("particle neither escaped nor came back")


@pytest.mark.parametrize("K_over_W", [0.5, 0.9, 1.1, 2.0])
def test_potential_wall_reflects_below_W_and_takes_W_above(K_over_W):
    """An electron meeting the work-function barrier of height W with normal
    kinetic energy K (open edges, negligible weight): K < W -> it turns back
    with its normal speed; K > W -> it leaves with normal energy K - W.  The
    tangential velocity is untouched (the barrier field is along the
    normal)."""
    W = 4.0
    X, V, nr = _wall_run(K_over_W, W)
    Kx = 0.5 * ME * V[0] ** 2 / (W * QE)
    if K_over_W < 1:
        assert V[0] < 0 and X[0] < 14
        assert Kx == pytest.approx(K_over_W, rel=1e-5)
    else:
        assert V[0] > 0 and X[0] > 18
        assert Kx == pytest.approx(K_over_W - 1.0, rel=1e-4)
    np.testing.assert_allclose(V[1:], [3e4, -2e4], rtol=1e-8)
    assert nr == 0


def _outgoing(n_part, seed, dims=3, kind=O.KIND_FREE, vF=1e6):
    """Particles just inside the face x = 14 of the slab, all crossing it in
    the first step; (X, V) in cell units and m/s."""
    rng = np.random.default_rng(seed)
    d0 = 0.45e-9
    dt = 0.5 * min((0.45e-9, 0.5e-9, 0.4e-9)[:dims]) / (C * math.sqrt(dims))
    # transverse offsets in [0.25, 0.75): only the x face is crossed
    yz = rng.integers(0, 4, (n_part, 2)) + 0.25 + 0.5 * rng.random((n_part, 2))
    if kind == O.KIND_DIRAC:
        th = rng.uniform(-1.2, 1.2, n_part)
        V = np.column_stack([vF * np.cos(th), vF * np.sin(th), np.zeros(n_part)])
    else:
        V = rng.normal(size=(n_part, 3)) * 2e5
        V[:, 0] = 0.1 * d0 / dt * (1.0 + rng.random(n_part))
    # the face is reached 5 % to 95 % into the first step
    x0 = 14.0 - (0.05 + 0.9 * rng.random(n_part)) * V[:, 0] * dt / d0
    X = np.column_stack([x0, yz[:, 0], yz[:, 1] if dims == 3 else np.zeros(n_part)])
    return X, V


def test_open_edges_let_particles_leave():
    """Open edges: a particle that crosses the material surface is not
    reflected and moves ballistically (E = B = 0, negligible weight); with
    the default rule the same particles are all reflected."""
    X0, V0 = _outgoing(200, 3)
    for open_edges in (True, False):
        s, _ = _slab_sim()
        s.set_particle_bc(open_edges=open_edges)
        s.add_species(O.KIND_FREE, -QE, ME, 1e-12, X0, V0)
        s.step(1)
        X, V, _, nr = s.species(0)
        ballistic = X0 + V0 * s.dt / np.array([0.45e-9, 0.5e-9, 0.4e-9])
        if open_edges:
            assert nr == 0
            np.testing.assert_allclose(X, ballistic, rtol=0, atol=1e-9)
            np.testing.assert_allclose(V, V0, rtol=1e-9)
        else:
            assert nr == len(X0)
            assert np.all(X[:, 0] < 14.0)


def test_diffuse_probability_zero_is_specular():
    """p = 0 takes no draw: the step is the specular rule bit for bit."""
    X0, V0 = _outgoing(300, 4)
    out = []
    for p in (None, 0.0):
        s, _ = _slab_sim()
        if p is not None:
            s.set_particle_bc(p_diffuse=p, seed=77)
        s.add_species(O.KIND_FREE, -QE, ME, 1e-12, X0, V0)
        s.step(3)
        out.append(s.species(0))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert out[0][3] == out[1][3] == len(X0)


def _diffuse_once(n_part, p, seed, dims=3, kind=O.KIND_FREE, vF=1e6, key=1234):
    X0, V0 = _outgoing(n_part, seed, dims, kind, vF)
    n = (24, 4, 4) if dims == 3 else (24, 4, 1)
    s, _ = _slab_sim(n=n, dims=dims)
    s.set_particle_bc(p_diffuse=p, seed=key)
    if kind == O.KIND_DIRAC:
        s.add_species(kind, -QE, 0.1 * ME, 1e-12, X0, V0, vF=vF)
    else:
        s.add_species(kind, -QE, ME, 1e-12, X0, V0)
    s.step(1)
    X, V, _, nr = s.species(0)
    return s, X0, V0, X, V, nr


def test_diffuse_reflection_follows_lambert_law_3d():
    """p = 1: every reflection re-emits the particle with its speed into the
    material side with Lambert's cosine law: cos(theta) to the inward normal
    has density 2 cos(theta) sin(theta), so E[cos] = 2/3 and E[cos^2] = 1/2,
    and the azimuth about the normal is uniform.  Positions are mirrored about
    the face as in the specular rule."""
    N = 20000
    s, X0, V0, X, V, nr = _diffuse_once(N, 1.0, 5)
    assert nr == N
    sp0 = np.linalg.norm(V0, axis=1)
    np.testing.assert_allclose(np.linalg.norm(V, axis=1), sp0, rtol=1e-12)
    ct = -V[:, 0] / sp0
    assert np.all(ct > 0)
    assert abs(ct.mean() - 2 / 3) < 4 * math.sqrt(1 / 18 / N)
    assert abs((ct ** 2).mean() - 0.5) < 4 * math.sqrt(1 / 12 / N)
    ph = np.arctan2(V[:, 2], V[:, 1])
    for f in (np.cos(ph), np.sin(ph), np.cos(2 * ph)):
        assert abs(f.mean()) < 4 * math.sqrt(0.5 / N)
    X1 = X0 + V0 * s.dt / np.array([0.45e-9, 0.5e-9, 0.4e-9])
    np.testing.assert_allclose(X[:, 0], 28.0 - X1[:, 0], atol=1e-12)
    np.testing.assert_allclose(X[:, 1:], X1[:, 1:], atol=1e-12)


def test_diffuse_reflection_of_dirac_carriers_is_2d_lambert():
    """Dirac carriers of a 2D sheet: the diffuse direction stays in the sheet
    (v_z = 0, |v| = v_F) with the 2D cosine law, density cos(theta) / 2 on
    (-pi/2, pi/2): E[cos] = pi/4, E[cos^2] = 2/3, E[sin] = 0."""
    N = 20000
    vF = 1e6
    s, X0, V0, X, V, nr = _diffuse_once(N, 1.0, 6, dims=2, kind=O.KIND_DIRAC, vF=vF)
    assert nr == N
    assert np.all(V[:, 2] == 0.0)
    np.testing.assert_allclose(np.hypot(V[:, 0], V[:, 1]), vF, rtol=1e-12)
    ct = -V[:, 0] / vF
    assert np.all(ct >= 0)
    var = 2 / 3 - (math.pi / 4) ** 2
    assert abs(ct.mean() - math.pi / 4) < 4 * math.sqrt(var / N)
    assert abs((ct ** 2).mean() - 2 / 3) < 4 * math.sqrt(4 / 45 / N)
    assert abs((V[:, 1] / vF).mean()) < 4 * math.sqrt(1 / 3 / N)


def test_diffuse_fraction_and_draw_layout():
    """p = 0.3: particle j of species 0 at step 0 reflects diffusely exactly
    when the first word of Philox(key = seed, counter = (j, 0, 0,
    0x44494655)) gives u = (w >> 8) / 2^24 < p (p in FP32), and the diffuse
    share is p within the binomial error."""
    N = 20000
    p, key = 0.3, 987654321987
    s, X0, V0, X, V, nr = _diffuse_once(N, p, 7, key=key)
    spec = np.column_stack([-V0[:, 0], V0[:, 1], V0[:, 2]])
    diffuse = ~np.all(V == spec, axis=1)
    want = np.zeros(N, bool)
    for j in range(N):
        w = O.philox([j, 0, 0, 0x44494655], [key & 0xFFFFFFFF, key >> 32])
        want[j] = (int(w[0]) >> 8) / 16777216.0 < float(np.float32(p))
    assert np.array_equal(diffuse, want)
    assert abs(diffuse.mean() - p) < 4 * math.sqrt(p * (1 - p) / N)


# ---------------------------------------------------------------------------
# kinetic-energy histogram (the relaxation study of Sec. 2)
# ---------------------------------------------------------------------------

def test_energy_histogram_bin_edges():
    """Hand-computed: m = 2 kg, so E = |v|^2 J; bins of width 1 J up to 4 J,
    half-open [b, b+1), E >= 4 J in the overflow entry."""
    s = O.OracleSim(dims=3, n=(4, 4, 4), d=(1e-9,) * 3, dt=1e-18, bc=(0, 0, 0))
    V = [[0, 0, 0], [1, 0, 0], [1, 1, 1], [2, 0, 0], [0, 1.9999, 0], [0, 0, 1.5],
         [1, 1, 0], [3, 0, 0], [0.5, 0.5, 0.5]]
    # E = 0, 1, 3, 4, 3.9996, 2.25, 2, 9, 0.75
    s.add_species(O.KIND_FREE, -QE, 2.0, 1.0, [[1.5, 1.5, 1.5]] * len(V), V)
    h = s.energy_histogram(0, 4.0, 4)
    assert h.tolist() == [2, 1, 2, 2, 2]


def test_energy_histogram_of_the_T0_fermi_sea():
    """The T = 0 loader fills the Fermi sphere uniformly, so the fraction of
    particles with E < x is (x / E_F)^(3/2): every bin holds
    N ((b / E_F)^1.5 - (a / E_F)^1.5) within 4.5 sigma, nothing lies above
    E_F, and the counts sum to N."""
    EF = 5.53 * QE
    n = (12, 12, 12)
    cell, off, v = O.fd_load(3, n, None, O.KIND_FREE, ME, EF, 0.0, 0.0, 64, False, 17, 0)
    X = np.column_stack(np.unravel_index(cell, (n[2], n[1], n[0]))[::-1]) + off
    s = O.OracleSim(dims=3, n=n, d=(0.2e-9,) * 3, dt=1e-19, bc=(0, 0, 0))
    s.add_species(O.KIND_FREE, -QE, ME, 1.0, X, v)
    N = len(cell)
    nb = 24
    h = s.energy_histogram(0, 1.2 * EF, nb).astype(np.int64)
    assert h.sum() == N
    edges = np.linspace(0, 1.2, nb + 1)
    cdf = np.minimum(edges, 1.0) ** 1.5
    want = N * np.diff(cdf)
    assert np.all(h[:nb][edges[1:] > 1.0 + 1e-12] == 0) and h[nb] == 0
    inside = edges[1:] <= 1.0 + 1e-12
    assert np.all(np.abs(h[:nb][inside] - want[inside]) <= 4.5 * np.sqrt(want[inside]) + 1)
