"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: the DFT definition
and numpy's FFT, the Clifford algebra of the Dirac matrices, scipy's dense matrix
exponential, exact free-particle evolution, unitarity, second-order convergence of the
Strang splitting, the standing-wave structure of the beam of Sec. II.A (zero at t = 0,
parity in y, plane-wave limit, Coulomb gauge to leading order in epsilon), gauge and
frame invariances, and the x-reflection symmetry behind Table II.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from paper_2307_01571_gb300 import workloads as W

NAT = W.NATURAL


def _pauli():
    sx = np.array([[0, 1], [1, 0]], complex)
    sy = np.array([[0, -1j], [1j, 0]], complex)
    sz = np.array([[1, 0], [0, -1]], complex)
    return sx, sy, sz


# --------------------------------------------------------------------------- FFT
@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32, 64])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft_equals_direct_dft(n, sign):
    rng = np.random.default_rng(n)
    a = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    j = np.arange(n)
    dft = np.exp(sign * 2j * np.pi * np.outer(j, j) / n) @ a   # O(N^2) definition
    got = oracle.fft1d(a, sign)
    assert np.max(np.abs(got - dft)) <= 1e-13 * max(1.0, np.max(np.abs(dft)))


def test_fft_matches_numpy_parseval_roundtrip():
    rng = np.random.default_rng(1)
    a = rng.standard_normal(1024) + 1j * rng.standard_normal(1024)
    f = oracle.fft1d(a, -1)
    assert np.allclose(f, np.fft.fft(a), rtol=0, atol=1e-11)
    assert abs(np.sum(np.abs(f) ** 2) / 1024 - np.sum(np.abs(a) ** 2)) < 1e-10
    assert np.allclose(oracle.fft1d(f, 1) / 1024, a, rtol=0, atol=1e-13)


def test_fft_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        oracle.fft1d(np.ones(6), -1)


def test_fft2d_matches_numpy_per_component():
    psi = W.random_spinor(16, 8, 3)
    got = oracle.fft2d(psi, -1)
    for c in range(4):
        assert np.allclose(got[:, :, c], np.fft.fft2(psi[:, :, c]), rtol=0, atol=1e-13)
    back = oracle.fft2d(got, 1) / (16 * 8)
    assert np.allclose(back, psi, rtol=0, atol=1e-15)


# ------------------------------------------------------------- Dirac algebra
def test_dirac_matrices_standard_representation_and_clifford():
    ax, ay, b = oracle.dirac_matrices()
    sx, sy, _ = _pauli()
    z = np.zeros((2, 2))
    assert np.array_equal(ax, np.block([[z, sx], [sx, z]]))
    assert np.array_equal(ay, np.block([[z, sy], [sy, z]]))
    assert np.array_equal(b, np.diag([1, 1, -1, -1]).astype(complex))
    I4 = np.eye(4)
    for A in (ax, ay, b):
        assert np.allclose(A, A.conj().T)
        assert np.allclose(A @ A, I4)
    assert np.allclose(ax @ ay + ay @ ax, 0)
    assert np.allclose(ax @ b + b @ ax, 0)
    assert np.allclose(ay @ b + b @ ay, 0)


def _H0(u, pix, piy):
    ax, ay, b = oracle.dirac_matrices()
    return u.c * (ax * pix + ay * piy) + b * u.m * u.c ** 2


def _E(u, pix, piy):
    return math.sqrt((u.m * u.c ** 2) ** 2 + u.c ** 2 * (pix ** 2 + piy ** 2))


@pytest.mark.parametrize("units", [NAT, W.ATOMIC])
def test_H0_squared_is_E_squared(units):
    rng = np.random.default_rng(2)
    for _ in range(5):
        pix, piy = rng.standard_normal(2) * units.m * units.c
        H = _H0(units, pix, piy)
        E2 = _E(units, pix, piy) ** 2
        assert np.max(np.abs(H @ H - E2 * np.eye(4))) <= 1e-13 * E2


# --------------------------------------------------- closed-form exponentials
@pytest.mark.parametrize("units", [NAT, W.ATOMIC])
@pytest.mark.parametrize("amag", [0.0, 1e-12, 1e-3, 0.1, 0.4, 3.0])
def test_potential_factor_equals_expm(units, amag):
    ax_m, ay_m, _ = oracle.dirac_matrices()
    rng = np.random.default_rng(int(amag * 1000) + 7)
    phi = rng.uniform(0, 2 * np.pi)
    ax, ay = amag * math.cos(phi), amag * math.sin(phi)
    tau = 0.025 * units.hbar / (units.m * units.c ** 2)
    V = -units.m * units.c ** 2 * (ax_m * ax + ay_m * ay)        # V = -q alpha.A
    ref = sla.expm(-1j * tau * V / units.hbar)
    M = oracle.potential_factor(units, ax, ay, tau)
    assert np.max(np.abs(M - ref)) <= 1e-14
    assert np.allclose(M.conj().T @ M, np.eye(4), atol=1e-14)
    # (alpha.a)^2 = |a|^2 used by the closed form
    G = ax_m * ax + ay_m * ay
    assert np.allclose(G @ G, amag ** 2 * np.eye(4), atol=1e-15)


@pytest.mark.parametrize("units", [NAT, W.ATOMIC])
def test_kinetic_factor_equals_expm(units):
    rng = np.random.default_rng(5)
    dt = 0.05 * units.hbar / (units.m * units.c ** 2)
    for pix, piy in [(0.0, 0.0), *(rng.standard_normal(2) * units.m * units.c for _ in range(6))]:
        ref = sla.expm(-1j * dt * _H0(units, pix, piy) / units.hbar)
        M = oracle.kinetic_factor(units, pix, piy, dt)
        assert np.max(np.abs(M - ref)) <= 1e-14
        assert np.allclose(M.conj().T @ M, np.eye(4), atol=1e-14)


# ------------------------------------------------------------------ bispinors
@pytest.mark.parametrize("units", [NAT, W.ATOMIC])
@pytest.mark.parametrize("basis", [0, 1])
def test_spinor_u_is_normalised_positive_energy_eigenvector(units, basis):
    rng = np.random.default_rng(11)
    sx, sy, sz = _pauli()
    for pix, piy in [(0.0, 0.0), (-0.1 * units.m * units.c, units.m * units.c),
                     *(rng.standard_normal(2) * units.m * units.c for _ in range(4))]:
        H = _H0(units, pix, piy)
        E = _E(units, pix, piy)
        up = oracle.spinor_u(units, pix, piy, 1, basis)
        um = oracle.spinor_u(units, pix, piy, -1, basis)
        for v in (up, um):
            assert np.allclose(H @ v, E * v, atol=1e-12 * E)
            assert abs(np.vdot(v, v) - 1) < 1e-14
            # lower components = c sigma.pi / (E + mc^2) times upper (Eq. Spinors_of_Dirac_equation)
            low = units.c * (sx * pix + sy * piy) @ v[:2] / (E + units.m * units.c ** 2)
            assert np.allclose(v[2:], low, atol=1e-15)
        assert abs(np.vdot(up, um)) < 1e-14
        # upper components are eigenvectors of sigma_x (x basis) or sigma_z (z basis)
        s = sx if basis == 0 else sz
        assert np.allclose(s @ up[:2], up[:2]) and np.allclose(s @ um[:2], -um[:2])
        # completeness with the negative-energy eigenvectors of H0
        w, vecs = np.linalg.eigh(H)
        neg = vecs[:, w < 0]
        phi = rng.standard_normal(4) + 1j * rng.standard_normal(4)
        tot = abs(np.vdot(up, phi)) ** 2 + abs(np.vdot(um, phi)) ** 2 + np.sum(
            np.abs(neg.conj().T @ phi) ** 2)
        assert abs(tot - np.vdot(phi, phi).real) < 1e-13 * np.vdot(phi, phi).real


def test_spinor_u_at_rest_is_x_polarised():
    up = oracle.spinor_u(NAT, 0.0, 0.0, 1, 0)
    um = oracle.spinor_u(NAT, 0.0, 0.0, -1, 0)
    s = 1 / math.sqrt(2)
    assert np.allclose(up, [s, s, 0, 0]) and np.allclose(um, [s, -s, 0, 0])


# ---------------------------------------------------------------------- field
def _gauss_field(eps=0.05, longitudinal=1, a0=0.1, phase0=0.0, env_T=0.0, kind=W.GAUSS):
    k = 0.1
    return W.Field(kind=kind, longitudinal=longitudinal, a0=a0, k_L=k, epsilon=eps, env_T=env_T,
                   phase0=phase0)


def test_standing_wave_vanishes_at_t0():
    for kind in (W.PLANE, W.GAUSS):
        f = _gauss_field(kind=kind)
        rng = np.random.default_rng(0)
        for x, y in rng.uniform(-300, 300, (20, 2)):
            ax, ay = oracle.field_a(NAT, f, x, y, 0.0)
            assert abs(ax) < 1e-15 and abs(ay) < 1e-15


def test_beam_on_focal_plane_closed_form():
    """At x = 0: w = w0, no Gouy or curvature phase, the two beams' A_x cancel and
    A_y = -2 a0 exp(-y^2/w0^2) sin(omega t)."""
    f = _gauss_field(eps=0.04)
    w0 = 1 / (f.k_L * f.epsilon)
    for y in (-2 * w0, -0.3 * w0, 0.0, 0.7 * w0, 1.5 * w0):
        for t in (3.0, 17.0, 40.0):
            ax, ay = oracle.field_a(NAT, f, 0.0, y, t)
            assert abs(ax) < 1e-15
            ref = -2 * f.a0 * math.exp(-y * y / w0 ** 2) * math.sin(NAT.c * f.k_L * t)
            assert abs(ay - ref) < 1e-15


def test_beam_parity_in_y():
    f = _gauss_field(eps=0.05)
    rng = np.random.default_rng(4)
    for x, y, t in zip(rng.uniform(-200, 200, 10), rng.uniform(0, 60, 10), rng.uniform(0, 50, 10)):
        axp, ayp = oracle.field_a(NAT, f, x, y, t)
        axm, aym = oracle.field_a(NAT, f, x, -y, t)
        assert abs(axp + axm) < 1e-15 and abs(ayp - aym) < 1e-15   # A_x odd, A_y even


def test_beam_plane_wave_limit_and_nodes():
    fp = _gauss_field(kind=W.PLANE)
    fg = _gauss_field(eps=1e-7)
    k = fp.k_L
    rng = np.random.default_rng(6)
    for x, y, t in zip(rng.uniform(-100, 100, 10), rng.uniform(-30, 30, 10), rng.uniform(1, 50, 10)):
        a1 = oracle.field_a(NAT, fp, x, y, t)
        a2 = oracle.field_a(NAT, fg, x, y, t)
        assert abs(a1[1] - a2[1]) < 1e-5 * fp.a0 and abs(a2[0]) < 1e-5 * fp.a0
        # plane wave: standing wave with nodes where cos(k x) = 0
        assert abs(a1[1] + 2 * fp.a0 * math.sin(NAT.c * k * t) * math.cos(k * x)) < 1e-14
    xn = 0.5 * math.pi / k
    assert abs(oracle.field_a(NAT, fp, xn, 0.0, 7.0)[1]) < 1e-15


def test_envelope_and_phase0():
    f = _gauss_field(kind=W.PLANE, env_T=100.0)
    assert oracle.field_a(NAT, f, 1.0, 0.0, 150.0) == (0.0, 0.0)
    a_half = oracle.field_a(NAT, f, 0.0, 0.0, 50.0)[1]
    a_cw = oracle.field_a(NAT, _gauss_field(kind=W.PLANE), 0.0, 0.0, 50.0)[1]
    assert abs(a_half - a_cw) < 1e-15        # sin^2(pi/2) = 1 at the envelope centre
    f2 = _gauss_field(kind=W.PLANE, phase0=0.5 * math.pi)
    assert abs(oracle.field_a(NAT, f2, 0.0, 0.0, 0.0)[1] + 2 * f2.a0) < 1e-15


def _divergence_ratio(eps):
    """max |div A| / max |d_y A_y| over points inside the beam (central differences)."""
    f = _gauss_field(eps=eps, a0=1.0)
    k = f.k_L
    w0 = 1 / (k * eps)
    h = 1e-3 / k
    worst_div, scale = 0.0, 0.0
    for xs in (-0.4, 0.13, 0.55):
        for ys in (-1.1, -0.35, 0.6, 1.3):
            for t in (2.0, 9.0):
                x, y = xs * w0, ys * w0
                dAx = (oracle.field_a(NAT, f, x + h, y, t)[0] - oracle.field_a(NAT, f, x - h, y, t)[0]) / (2 * h)
                dAy = (oracle.field_a(NAT, f, x, y + h, t)[1] - oracle.field_a(NAT, f, x, y - h, t)[1]) / (2 * h)
                worst_div = max(worst_div, abs(dAx + dAy))
                scale = max(scale, abs(dAy))
    return worst_div / scale


def test_beam_is_coulomb_gauge_to_leading_order():
    """The longitudinal component makes div A vanish at leading order in epsilon
    (Sec. II.A: both components in Coulomb gauge); with it switched off the residual
    is of the size of d_y A_y itself."""
    r1, r2 = _divergence_ratio(0.04), _divergence_ratio(0.02)
    assert r1 < 0.01 and 3.5 < r1 / r2 < 4.5     # residual is O(epsilon^2) relative
    f = _gauss_field(eps=0.04, a0=1.0, longitudinal=0)
    w0 = 1 / (f.k_L * 0.04)
    h = 1e-3 / f.k_L
    x, y, t = 0.1 * w0, 0.6 * w0, 9.0
    dAy = (oracle.field_a(NAT, f, x, y + h, t)[1] - oracle.field_a(NAT, f, x, y - h, t)[1]) / (2 * h)
    assert abs(dAy) > 0.1 * abs(oracle.field_a(NAT, f, x, y, t)[1]) / w0


# ------------------------------------------------------- dense whole-step pin
def _dense_step(u, g, f, psi, t0, dt):
    """exp(-i dt/2 H_V(t1)) exp(-i dt H_K) exp(-i dt/2 H_V(t0)) on the flattened grid,
    built from dense matrices: H_V block-diagonal in position, H_K = F^dag diag(H0 - v p_y) F
    with F the unitary DFT (numpy) and momenta from numpy.fft.fftfreq."""
    ax_m, ay_m, _ = oracle.dirac_matrices()
    nx, ny = g.nx, g.ny
    dx, dy = (g.x_max - g.x_min) / nx, (g.y_max - g.y_min) / ny
    P = nx * ny
    I4 = np.eye(4)

    def HV(t):
        H = np.zeros((4 * P, 4 * P), complex)
        for iy in range(ny):
            for ix in range(nx):
                ax, ay = oracle.field_a(u, f, g.x_min + ix * dx, g.y_min + iy * dy + f.box_vy * t, t)
                i = (iy * nx + ix) * 4
                H[i:i + 4, i:i + 4] = -u.m * u.c ** 2 * (ax_m * ax + ay_m * ay)
        return H

    px = 2 * np.pi * u.hbar * np.fft.fftfreq(nx, d=dx)
    py = 2 * np.pi * u.hbar * np.fft.fftfreq(ny, d=dy)
    D = np.zeros((4 * P, 4 * P), complex)
    for ky in range(ny):
        for kx in range(nx):
            i = (ky * nx + kx) * 4
            D[i:i + 4, i:i + 4] = _H0(u, px[kx] + f.p_shift_x, py[ky] + f.p_shift_y) - f.box_vy * py[ky] * I4
    Fy = np.fft.fft(np.eye(ny)) / math.sqrt(ny)
    Fx = np.fft.fft(np.eye(nx)) / math.sqrt(nx)
    F = np.kron(np.kron(Fy, Fx), I4)
    HK = F.conj().T @ D @ F
    U = sla.expm(-0.5j * dt * HV(t0 + dt) / u.hbar) @ sla.expm(-1j * dt * HK / u.hbar) @ \
        sla.expm(-0.5j * dt * HV(t0) / u.hbar)
    return (U @ psi.reshape(-1)).reshape(psi.shape)


@pytest.mark.parametrize("nx,ny,kind,vy", [(4, 4, W.GAUSS, 0.0), (8, 4, W.GAUSS, 0.7),
                                           (4, 8, W.PLANE, 0.0), (8, 8, W.GAUSS, 0.5)])
def test_step_equals_dense_exponentials(nx, ny, kind, vy):
    u = NAT
    g = W.Grid(nx, ny, -3.0 * nx, 3.0 * nx, -2.0 * ny + 1.0, 2.0 * ny + 1.0)
    f = W.Field(kind=kind, longitudinal=1 if kind == W.GAUSS else 0, a0=0.4, k_L=0.3,
                epsilon=0.1 if kind == W.GAUSS else 0.0, phase0=0.7, p_shift_x=0.05,
                p_shift_y=0.6, box_vy=vy)
    psi = W.random_spinor(nx, ny, 7 + nx + ny)
    t0, dt = 3.3, 0.4
    ref = _dense_step(u, g, f, psi, t0, dt)
    got = oracle.step(u, g, f, psi, t0, dt, 1)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


# ------------------------------------------------------------- free particle
@pytest.mark.parametrize("vy", [0.0, 0.6])
def test_free_plane_wave_is_exact_eigenstate(vy):
    u = NAT
    nx, ny = 32, 16
    g = W.Grid(nx, ny, -40.0, 40.0, -20.0, 20.0)
    f = W.Field(kind=W.NONE, p_shift_x=0.0, p_shift_y=1.0, box_vy=vy)
    kx, ky = 3, ny - 2
    pix, piy = oracle.momentum(g, u, f, kx, ky)
    px, py = pix - f.p_shift_x, piy - f.p_shift_y
    us = oracle.spinor_u(u, pix, piy, 1, 0)
    x = g.x_min + np.arange(nx) * (g.x_max - g.x_min) / nx
    y = g.y_min + np.arange(ny) * (g.y_max - g.y_min) / ny
    wave = np.exp(1j * (px * (x[None, :] - g.x_min) + py * (y[:, None] - g.y_min)) / u.hbar)
    psi0 = wave[:, :, None] * us[None, None, :]
    dt, n = 0.05, 2000
    got = oracle.step(u, g, f, psi0, 0.0, dt, n)
    T = n * dt
    E = _E(u, pix, piy)
    ref = psi0 * np.exp(-1j * (E - vy * py) * T / u.hbar)
    assert np.max(np.abs(got - ref)) <= 1e-12


# ---------------------------------------------------- unitarity, convergence
def test_norm_conserved_gaussian_beam():
    wl = W.small(32, 32, W.GAUSS, units=NAT, a0=0.4)
    psi = oracle.init_packet(wl.units, wl.grid, wl.field, wl.packet)
    spec = W.default_obs_spec(wl.units, wl.field, wl.packet)
    n0 = oracle.observe(wl.units, wl.grid, wl.field, spec, psi, 0.0)["norm"]
    assert abs(n0 - 1) < 1e-13
    out = oracle.step(wl.units, wl.grid, wl.field, psi, 0.0, wl.dt, 200)
    n1 = oracle.observe(wl.units, wl.grid, wl.field, spec, out, 200 * wl.dt)["norm"]
    assert abs(n1 - n0) < 1e-12


def test_strang_splitting_is_second_order():
    u = NAT
    g = W.Grid(16, 16, -40.0, 40.0, -40.0, 40.0)
    f = W.Field(kind=W.GAUSS, longitudinal=1, a0=0.6, k_L=0.3, epsilon=0.08, phase0=0.2,
                p_shift_y=0.5, box_vy=0.3)
    psi = W.random_spinor(16, 16, 9)
    T = 2.0
    ref = oracle.step(u, g, f, psi, 0.0, T / 256, 256)
    errs = []
    for n in (8, 16, 32):
        errs.append(np.linalg.norm(oracle.step(u, g, f, psi, 0.0, T / n, n) - ref))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.6 < r1 < 4.4 and 3.6 < r2 < 4.4, (errs, r1, r2)


# ------------------------------------------------------ gauge / frame readings
def test_gauge_shift_equals_shifted_packet():
    """A constant gauge shift of m c along y (the paper's A_m) equals an unshifted run whose
    packet sits at p_y = m c, with momentum densities related by an index shift."""
    u = NAT
    nx, ny, N = 16, 64, 16
    Ly = 2 * np.pi * u.hbar * N / (u.m * u.c)     # m c = N momentum cells
    g = W.Grid(nx, ny, -60.0, 60.0, -Ly / 2, Ly / 2)
    common = dict(kind=W.PLANE, a0=0.3, k_L=2 * np.pi / 60.0, phase0=0.4, box_vy=0.0)
    fa = W.Field(p_shift_y=u.m * u.c, **common)
    fb = W.Field(p_shift_y=0.0, **common)
    dp = 2 * np.pi / Ly
    pk = W.Packet(0.0, u.m * u.c, 0.0, 0.0, 2 * dp, 1, 0)
    out = []
    for f in (fa, fb):
        psi = oracle.init_packet(u, g, f, pk)
        psi = oracle.step(u, g, f, psi, 0.0, 0.2, 50)
        out.append(oracle.momentum_density(u, g, f, psi))
    # kinetic momentum of (a) at canonical index j equals (b) at canonical index j + N
    a, b = out
    assert np.max(np.abs(a - np.roll(b, -N, axis=0))) < 1e-12


def test_moving_frame_leaves_free_momentum_density_unchanged():
    u = NAT
    wl = W.small(16, 16, W.NONE, units=u)
    g = wl.grid
    res = []
    for vy in (0.0, 0.7):
        f = W.Field(kind=W.NONE, p_shift_y=1.0, box_vy=vy)
        psi = oracle.init_packet(u, g, f, wl.packet)
        res.append(oracle.momentum_density(u, g, f, oracle.step(u, g, f, psi, 0.0, 0.05, 100)))
    assert np.max(np.abs(res[0] - res[1])) < 1e-14


def test_x_reflection_symmetry_of_diffraction():
    """Plane-wave standing wave and a packet with p_x = 0: the momentum-space densities at
    +p_x and -p_x agree (the left/right symmetry of Table II).  The field is weak enough that
    the Nyquist column, which has no mirror partner on the grid, stays empty."""
    u = NAT
    nx, ny = 64, 16
    k = 0.1
    L = 4 * 2 * np.pi / k
    g = W.Grid(nx, ny, -L / 2, L / 2, -10 * np.pi / k, 10 * np.pi / k)
    f = W.Field(kind=W.PLANE, a0=0.03, k_L=k, p_shift_y=1.0)
    pk = W.Packet(0.0, 1.0, 0.0, 0.0, k / 4, 1, 0)
    psi = oracle.init_packet(u, g, f, pk)
    psi = oracle.step(u, g, f, psi, 0.0, 0.5, 200)
    md = oracle.momentum_density(u, g, f, psi)
    assert md[:, nx // 2, 0].sum() < 1e-16
    mirrored = md[:, (-np.arange(nx)) % nx, :]
    assert np.max(np.abs(md - mirrored)) < 1e-13 * md.max()
    assert md[:, 8, 0].sum() > 1e-3        # population diffracted to +2 hbar k_L


# ----------------------------------------------------------------- observables
def test_packet_and_observables_against_numpy():
    wl = W.small(32, 16, W.PLANE, units=NAT)
    u, g, f, pk = wl.units, wl.grid, wl.field, wl.packet
    psi = oracle.init_packet(u, g, f, pk)
    md = oracle.momentum_density(u, g, f, psi)
    dxdy = (g.x_max - g.x_min) / g.nx * (g.y_max - g.y_min) / g.ny
    # Parseval: the cell probabilities sum to the norm
    assert abs(md[:, :, 0].sum() - np.sum(np.abs(psi) ** 2) * dxdy) < 1e-13
    # the packet is pure u^+ : |c+|^2 = |phi|^2 cell by cell, |c-|^2 = 0
    assert np.allclose(md[:, :, 1], md[:, :, 0], atol=1e-15) and md[:, :, 2].max() < 1e-28
    # windows: brute force with numpy momenta
    spec = W.default_obs_spec(u, f, pk)
    psi2 = oracle.step(u, g, f, psi, 0.0, 0.5, 40)
    md2 = oracle.momentum_density(u, g, f, psi2)
    ob = oracle.observe(u, g, f, spec, psi2, 20.0)
    px = 2 * np.pi * np.fft.fftfreq(g.nx, d=(g.x_max - g.x_min) / g.nx) + f.p_shift_x
    py = 2 * np.pi * np.fft.fftfreq(g.ny, d=(g.y_max - g.y_min) / g.ny) + f.p_shift_y
    dpx, dpy = px[1] - px[0], py[1] - py[0]

    def win(cx, cy):
        mx = np.abs(np.round((px - cx) / dpx)) <= math.floor(spec.half_width / dpx + 1e-9)
        my = np.abs(np.round((py - cy) / dpy)) <= math.floor(spec.half_width / dpy + 1e-9)
        return my[:, None] & mx[None, :]

    wi, wd = win(spec.p_in_x, spec.p_in_y), win(spec.p_diff_x, spec.p_diff_y)
    assert abs(ob["pop_in"] - md2[:, :, 0][wi].sum()) < 1e-14
    assert abs(ob["pop_diff"] - md2[:, :, 0][wd].sum()) < 1e-14
    assert abs(ob["cm_diff"] - md2[:, :, 2][wd].sum()) < 1e-14
    assert abs(ob["cp_in"] - md2[:, :, 1][wi].sum()) < 1e-14
    assert abs(ob["max_diff"] - md2[:, :, 0][wd].max()) < 1e-16
    it = np.argmin(np.abs(px - spec.target_x)); jt = np.argmin(np.abs(py - spec.target_y))
    assert ob["p_target"] == md2[jt, it, 0] and ob["cm_target"] == md2[jt, it, 2]
    dens = oracle.density_x(g, psi2)
    assert np.allclose(dens, np.sum(np.abs(psi2) ** 2, axis=(0, 2)) * (g.y_max - g.y_min) / g.ny,
                       atol=1e-15)


# ----------------------------------------------------------------- initial packet
# Eq. (Density_distribution_of_Gaussian_wave_packet), Sec. II.C: the momentum amplitude
# is exp(-|pi - p0|^2 / (4 sigma_p^2)) times a position phase exp(-i r0.p / hbar), and
# phi = u^s rho.  These pins check the packet through moments computed here with numpy
# momenta and positions (not the oracle's): the sampled Gaussian |rho|^2 on a grid with
# dp = sigma_p / 2 has mean p0 and standard deviation sigma_p up to Poisson-summation
# terms of order exp(-2 pi^2 sigma_p^2 / dp^2) = e^-79.
def _moment_grid(n=64, sig=0.02, frac_x=0.3, frac_y=0.45):
    dp = sig / 2
    L = 2 * math.pi / dp
    return W.Grid(n, n, -frac_x * L, (1 - frac_x) * L, -frac_y * L, (1 - frac_y) * L), L, dp


def _axis_momenta(g, f):
    px = 2 * np.pi * np.fft.fftfreq(g.nx, d=(g.x_max - g.x_min) / g.nx) + f.p_shift_x
    py = 2 * np.pi * np.fft.fftfreq(g.ny, d=(g.y_max - g.y_min) / g.ny) + f.p_shift_y
    return px, py


@pytest.mark.parametrize("spin", [1, -1])
@pytest.mark.parametrize("basis", [0, 1])
def test_packet_momentum_mean_and_width(spin, basis):
    sig = 0.02
    g, L, dp = _moment_grid(sig=sig)
    f = W.Field(kind=W.NONE, p_shift_x=0.013, p_shift_y=0.7)
    # p0 off the grid points on both axes, kinetic (pi = p + p_shift)
    pk = W.Packet(0.013 + 3.3 * dp, 0.7 - 5.6 * dp, 0.1 * L, -0.2 * L, sig, spin, basis)
    psi = oracle.init_packet(NAT, g, f, pk)
    md = oracle.momentum_density(NAT, g, f, psi, basis=basis)
    px, py = _axis_momenta(g, f)
    w = md[:, :, 0] / md[:, :, 0].sum()
    wx, wy = w.sum(0), w.sum(1)
    mx, my = (wx * px).sum(), (wy * py).sum()
    sx = math.sqrt((wx * (px - mx) ** 2).sum())
    sy = math.sqrt((wy * (py - my) ** 2).sum())
    assert abs(mx - pk.p0x) < 1e-12 and abs(my - pk.p0y) < 1e-12
    assert abs(sx / sig - 1) < 1e-10 and abs(sy / sig - 1) < 1e-10
    # the amplitude itself is the sampled Gaussian, cell by cell
    gauss = np.exp(-((py[:, None] - pk.p0y) ** 2 + (px[None, :] - pk.p0x) ** 2) / (2 * sig ** 2))
    assert np.max(np.abs(w - gauss / gauss.sum())) < 1e-13
    # a pure u^s packet: all of |phi|^2 is in the spin-s projection, none in the other
    mine, other = (1, 2) if spin == 1 else (2, 1)
    assert np.max(np.abs(md[:, :, mine] - md[:, :, 0])) < 1e-14 * md[:, :, 0].max()
    assert md[:, :, other].max() < 1e-26


@pytest.mark.parametrize("spin,basis", [(1, 0), (-1, 0), (1, 1), (-1, 1)])
@pytest.mark.parametrize("fx,fy", [(0.5, 0.5), (0.3, 0.45)])
def test_packet_position_centre(spin, basis, fx, fy):
    """With p0 = 0 and no momentum shift, u^s(-p) = beta u^s(p), so |psi|^2 is exactly
    symmetric about r0: its mean is r0, on a centred and on an off-centre box."""
    sig = 0.02
    g, L, dp = _moment_grid(sig=sig, frac_x=fx, frac_y=fy)
    f = W.Field(kind=W.NONE)
    dx = L / g.nx
    r0x, r0y = g.x_min + 29 * dx, g.y_min + 35 * dx
    pk = W.Packet(0.0, 0.0, r0x, r0y, sig, spin, basis)
    psi = oracle.init_packet(NAT, g, f, pk)
    dens = np.sum(np.abs(psi) ** 2, axis=2)
    x = g.x_min + np.arange(g.nx) * dx
    y = g.y_min + np.arange(g.ny) * dx
    w = dens / dens.sum()
    assert abs((w.sum(0) * x).sum() - r0x) < 1e-9 * L
    assert abs((w.sum(1) * y).sum() - r0y) < 1e-9 * L
    # spatial width hbar / (2 sigma_p) per axis of the scalar Gaussian (the spinor
    # structure adds a relative correction of order (sigma_p / m c)^2)
    sx = math.sqrt((w.sum(0) * (x - r0x) ** 2).sum())
    assert abs(sx / (1.0 / (2 * sig)) - 1) < 1e-3


def test_packet_position_phase_translates_exactly():
    """Moving r0 by whole grid cells (mx, my) moves the state by exactly that cyclic shift:
    the position phase exp(-i r0.p/hbar) with the grid's own momenta is a discrete
    translation.  A wrong sign or scale of the phase breaks this."""
    sig = 0.02
    g, L, dp = _moment_grid(sig=sig)
    f = W.Field(kind=W.NONE, p_shift_x=0.01, p_shift_y=0.5)
    dx = L / g.nx
    a = W.Packet(0.01 + 2.2 * dp, 0.5 - 1.7 * dp, 0.05 * L, 0.1 * L, sig, 1, 0)
    mx, my = 7, -5
    b = W.Packet(a.p0x, a.p0y, a.r0x + mx * dx, a.r0y + my * dx, sig, 1, 0)
    pa = oracle.init_packet(NAT, g, f, a)
    pb = oracle.init_packet(NAT, g, f, b)
    assert np.max(np.abs(pb - np.roll(pa, (my, mx), axis=(0, 1)))) < 1e-12 * np.max(np.abs(pa))


def test_study_definitions():
    from paper_2307_01571_gb300 import studies
    w3, w4 = studies.e3(), studies.e4()
    assert len(w3) == 12 and len(w4) == 8
    for w in w3:
        e, kn = w.extra["eps"], w.extra["k_nat"]
        lam = 2 * math.pi / w.field.k_L
        assert abs(w.field.k_L - kn) < 1e-15 and abs(w.field.epsilon - e) < 1e-15
        assert abs((w.grid.x_max - w.grid.x_min) - 80 * lam) < 1e-9 * lam
        assert abs(w.nsteps * w.dt - 280 * lam * math.sqrt(2)) < w.dt
    assert sorted({w.field.longitudinal for w in w4}) == [0, 1]
    # the slope fit recovers an exact power law
    x = np.array([1.0, 2.0, 5.0, 10.0])
    assert abs(studies.fit_slope(x, 3.0 * x ** 2) - 2.0) < 1e-12


def test_openmp_timing_variant_equals_plain_oracle():
    """The OpenMP build (rows, columns and grid points on threads; the timing variant of
    the CPU baseline) computes exactly what the plain build computes."""
    wl = W.small(64, 32, W.GAUSS, units=NAT, a0=0.3, nsteps=4)
    u, g, f, pk = wl.units, wl.grid, wl.field, wl.packet
    psi = W.random_spinor(64, 32, 4)
    oracle.use_openmp(False)
    a = oracle.step(u, g, f, psi, 0.0, wl.dt, 4)
    try:
        oracle.use_openmp(True)
        b = oracle.step(u, g, f, psi, 0.0, wl.dt, 4)
    finally:
        oracle.use_openmp(False)
    assert np.array_equal(a, b)
