"""Pins of the oracle's time step (Eq. 1-8, 13, 14 and the boundary rules).

Each check compares the oracle with something other than itself: textbook
special cases (BGK with Guo forcing, the Hermite equilibrium), closed forms
(the force of a plane-wave psi, an exact streaming shift), invariants (mass,
momentum, uniform rest state) and the coexistence densities of Eq. 9 solved
by quadrature, which the scheme reproduces in the regime where Eq. 9 holds.
"""
import numpy as np
import pytest

from oracle import d2q9, thermo

EX, EY = d2q9.EX, d2q9.EY
OPP = [0, 3, 4, 1, 2, 7, 8, 5, 6]
W_EQ = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def hermite_feq(rho, vx, vy):
    """Textbook second-order D2Q9 equilibrium in velocity space."""
    eu = EX * vx + EY * vy
    return W_EQ * rho * (1 + 3 * eu + 4.5 * eu ** 2 - 1.5 * (vx * vx + vy * vy))


def guo_source(vx, vy, Fx, Fy):
    """Textbook Guo forcing term w_a [3 (e_a - v) + 9 (e_a . v) e_a] . F."""
    eu = EX * vx + EY * vy
    return W_EQ * (3 * ((EX - vx) * Fx + (EY - vy) * Fy) + 9 * eu * (EX * Fx + EY * Fy))


# ------------------------------------------------------------------ moments

def test_moment_matrix_orthogonal_and_inverse():
    M, Minv = d2q9.moment_matrix()
    # orthogonal rows (Sec. 2.1), norms of the standard D2Q9 moment basis
    assert np.allclose(M @ M.T, np.diag([9, 36, 36, 6, 12, 6, 12, 4, 4]), atol=0, rtol=0)
    assert np.allclose(Minv @ M, np.eye(9), atol=1e-15)


def test_equilibrium_projects_to_eq4():
    # M f_eq(Hermite) reproduces m_eq of Eq. 4; oracle_feq = M^-1 m_eq
    # reproduces the Hermite equilibrium.
    M, _ = d2q9.moment_matrix()
    rng = np.random.default_rng(1)
    for _ in range(20):
        rho = rng.uniform(0.01, 0.5)
        vx, vy = rng.uniform(-0.1, 0.1, 2)
        fe = hermite_feq(rho, vx, vy)
        assert np.allclose(d2q9.feq(rho, vx, vy), fe, rtol=0, atol=1e-15)
        v2 = vx * vx + vy * vy
        eq4 = rho * np.array([1, -2 + 3 * v2, 1 - 3 * v2, vx, -vx, vy, -vy, vx * vx - vy * vy, vx * vy])
        assert np.allclose(M @ fe, eq4, rtol=0, atol=1e-15)


def test_guo_forcing_projects_to_eq8():
    # (I - Lambda/2) S = M F' (text under Eq. 3): the velocity-space Guo term
    # maps to Eq. 8 in moment space.
    M, _ = d2q9.moment_matrix()
    rng = np.random.default_rng(2)
    for _ in range(20):
        vx, vy, Fx, Fy = rng.uniform(-0.1, 0.1, 4)
        vF = vx * Fx + vy * Fy
        eq8 = np.array([0, 6 * vF, -6 * vF, Fx, -Fx, Fy, -Fy, 2 * (vx * Fx - vy * Fy), vx * Fy + vy * Fx])
        assert np.allclose(M @ guo_source(vx, vy, Fx, Fy), eq8, rtol=0, atol=1e-15)


@pytest.mark.parametrize("tau", [0.51, 0.6, 1.0, 1.7])
def test_srt_limit_is_bgk_with_guo_forcing(tau):
    # All rates 1/tau and eps = 0: Eq. 3 with Eq. 8 is BGK with Guo's forcing.
    L = d2q9.Lattice(1, 1, T=0.07, s=[1 / tau] * 9, eps=0.0)
    rng = np.random.default_rng(3)
    for _ in range(25):
        f = W_EQ * rng.uniform(0.05, 0.45) * (1 + 0.05 * rng.uniform(-1, 1, 9))
        Fx, Fy = rng.uniform(-1e-3, 1e-3, 2)
        psi = rng.uniform(0.1, 0.6)
        rho = f.sum()
        vx = (np.dot(EX, f) + 0.5 * Fx) / rho
        vy = (np.dot(EY, f) + 0.5 * Fy) / rho
        expect = f - (f - hermite_feq(rho, vx, vy)) / tau + (1 - 0.5 / tau) * guo_source(vx, vy, Fx, Fy)
        got = L.collide_node(f, Fx, Fy, psi)
        assert np.allclose(got, expect, rtol=0, atol=1e-15)


def test_li_term_keeps_conserved_moments_and_scales_with_eps():
    # Eq. 14 changes only the two energy moments; it leaves mass and
    # momentum alone and is linear in eps.
    M, _ = d2q9.moment_matrix()
    s = [1.0, 1.1, 1.1, 1.0, 1.1, 1.0, 1.1, 1 / 0.6, 1 / 0.6]
    rng = np.random.default_rng(4)
    f = W_EQ * 0.3 * (1 + 0.02 * rng.uniform(-1, 1, 9))
    Fx, Fy, psi = 2e-3, -1e-3, 0.4
    base = d2q9.Lattice(1, 1, T=0.07, s=s, eps=0.0).collide_node(f, Fx, Fy, psi)
    d1 = M @ (d2q9.Lattice(1, 1, T=0.07, s=s, eps=1.0).collide_node(f, Fx, Fy, psi) - base)
    d2 = M @ (d2q9.Lattice(1, 1, T=0.07, s=s, eps=2.0).collide_node(f, Fx, Fy, psi) - base)
    for k in (0, 3, 4, 5, 6, 7, 8):
        assert abs(d1[k]) < 1e-16 and abs(d2[k]) < 1e-16
    assert d1[1] > 0 > d1[2]
    assert np.allclose(d2[1:3], 2 * d1[1:3], rtol=1e-12)


# ------------------------------------------------------------------ force, Eq. 7

@pytest.mark.parametrize("kx,ky", [(1, 0), (0, 2), (1, 1), (2, 3)])
def test_force_of_plane_wave_psi(kx, ky):
    # psi = A + B sin(k . x): sum_a w_a psi(x + e_a) e_a = B cos(k . x) sum_a w_a sin(k . e_a) e_a,
    # which for w_axis = 1/3, w_diag = 1/12 is
    # B cos(k.x) ((2/3) sin kx + (1/3) sin kx cos ky, (2/3) sin ky + (1/3) sin ky cos kx).
    nx, ny, G = 24, 18, -1.0
    L = d2q9.Lattice(nx, ny, G=G)
    kxv, kyv = 2 * np.pi * kx / nx, 2 * np.pi * ky / ny
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    th = kxv * x + kyv * y
    A, B = 0.5, 0.1
    psi = A + B * np.sin(th)
    Fx, Fy = L.force_from_psi(psi)
    gx = B * np.cos(th) * (2 / 3 * np.sin(kxv) + 1 / 3 * np.sin(kxv) * np.cos(kyv))
    gy = B * np.cos(th) * (2 / 3 * np.sin(kyv) + 1 / 3 * np.sin(kyv) * np.cos(kxv))
    assert np.allclose(Fx, -G * psi * gx, rtol=0, atol=1e-15)
    assert np.allclose(Fy, -G * psi * gy, rtol=0, atol=1e-15)


def test_force_next_to_wall_uses_own_psi():
    nx, ny = 6, 5
    solid = np.zeros((ny, nx), np.uint8)
    solid[0, :] = 1
    L = d2q9.Lattice(nx, ny, G=-1.0, solid=solid)
    psi = np.full((ny, nx), 0.3)
    psi[1, :] = 0.5
    Fx, Fy = L.force_from_psi(psi)
    # at y = 1: downward neighbours are solid -> psi(node) = 0.5; upward are 0.3
    # g_y = (1/3)(0.3 - 0.5) + (1/12)(0.3 + 0.3 - 0.5 - 0.5)
    gy = (0.3 - 0.5) / 3 + (0.6 - 1.0) / 12
    assert np.allclose(Fy[1], 0.5 * gy, atol=1e-16)
    assert np.allclose(Fx[1], 0.0, atol=1e-16)
    assert np.all(Fx[0] == 0) and np.all(Fy[0] == 0)


# ------------------------------------------------------------------ streaming

@pytest.mark.parametrize("walls", [False, True])
def test_one_step_is_exact_shift_without_collision(walls):
    # Uniform rho gives F = 0 exactly; with all rates 0 the collision is the
    # identity (up to M^-1 M rounding), so one step is Eq. 5: a pure shift by
    # e_a, with reflection at solid nodes.
    nx, ny = 7, 6
    solid = None
    if walls:
        solid = np.zeros((ny, nx), np.uint8)
        solid[0, :] = 1
        solid[ny - 1, :] = 1
    L = d2q9.Lattice(nx, ny, T=0.07, s=[0.0] * 9, eps=0.0, solid=solid)
    rng = np.random.default_rng(5)
    rho0 = 0.3
    dev = rng.uniform(-1e-3, 1e-3, (9, ny, nx))
    dev -= dev.mean(axis=0, keepdims=True)        # sum over a of the deviation is 0
    f0 = W_EQ[:, None, None] * rho0 + dev
    L.f[:] = f0
    L.step(1)
    expect = np.zeros_like(f0)
    for a in range(9):
        for y in range(ny):
            for x in range(nx):
                if solid is not None and solid[y, x]:
                    expect[a, y, x] = f0[a, y, x]
                    continue
                xt, yt = (x + EX[a]) % nx, (y + EY[a]) % ny
                if solid is not None and solid[yt, xt]:
                    expect[OPP[a], y, x] = f0[a, y, x]
                else:
                    expect[a, yt, xt] = f0[a, y, x]
    assert np.allclose(L.f, expect, rtol=0, atol=1e-15)


# ------------------------------------------------------------------ invariants

def _droplet_lattice(nx, ny, tr, eps, tau, walls=False, R=10.0):
    Tc, _, _ = thermo.critical_point()
    rg, rl, _ = thermo.maxwell(tr * Tc)
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    r = np.hypot(x - (nx - 1) / 2, y - (ny - 1) / 2)
    rho = 0.5 * (rl + rg) - 0.5 * (rl - rg) * np.tanh(2 * (r - R) / 3.0)
    solid = None
    if walls:
        solid = np.zeros((ny, nx), np.uint8)
        solid[0, :] = 1
        solid[ny - 1, :] = 1
    s = [1.0, 1.1, 1.1, 1.0, 1.1, 1.0, 1.1, 1 / tau, 1 / tau]
    L = d2q9.Lattice(nx, ny, T=tr * Tc, s=s, eps=eps, solid=solid)
    L.init(rho)
    return L


def test_uniform_rest_state_is_fixed_point():
    L = d2q9.Lattice(9, 7, T=0.6 * 0.0943287, s=[1, 1.1, 1.1, 1, 1.1, 1, 1.1, 1.5, 1.5], eps=1.86)
    L.init(np.full((7, 9), 0.35))
    f0 = L.f.copy()
    L.step(50)
    assert np.allclose(L.f, f0, rtol=0, atol=1e-15)
    rho, ux, uy, p = L.moments()
    assert np.all(ux == 0) and np.all(uy == 0)


@pytest.mark.parametrize("walls", [False, True])
def test_mass_conserved(walls):
    L = _droplet_lattice(40, 36, 0.7, 1.86, 0.6, walls=walls)
    m0 = L.mass()
    L.step(400)
    assert L.flags == 0
    assert abs(L.mass() / m0 - 1) < 1e-13


def test_momentum_conserved_periodic():
    # sum_x F = 0 by the pairwise antisymmetry of Eq. 7, and the collision
    # sends j to j + F (Eq. 3 with Eq. 6), so total momentum is invariant.
    L = _droplet_lattice(40, 36, 0.7, 1.86, 0.6)
    # give the droplet a uniform drift
    rho, _, _, _ = L.moments()
    L.init(rho, np.full_like(rho, 0.01), np.full_like(rho, -0.005))
    def mom():
        return (np.tensordot(EX, L.f, 1).sum(), np.tensordot(EY, L.f, 1).sum())
    p0 = mom()
    L.step(300)
    p1 = mom()
    scale = L.mass()
    assert abs(p1[0] - p0[0]) < 1e-13 * scale and abs(p1[1] - p0[1]) < 1e-13 * scale


def _stratified_at_rest(nx, ny, along_x):
    """Walls on two opposite edges, a density that varies only across them
    (a diffuse interface with a trend), at rest."""
    Tc, _, _ = thermo.critical_point()
    rg, rl, _ = thermo.maxwell(0.6 * Tc)
    n = nx if along_x else ny
    k = np.arange(n, dtype=float)
    prof = 0.5 * (rl + rg) + 0.5 * (rl - rg) * np.tanh((k - 0.4 * n) / 3.0) + 0.002 * k
    rho = np.tile(prof, (ny, 1)) if along_x else np.tile(prof[:, None], (1, nx))
    solid = np.zeros((ny, nx), np.uint8)
    if along_x:
        solid[:, 0] = solid[:, nx - 1] = 1
    else:
        solid[0, :] = solid[ny - 1, :] = 1
    L = d2q9.Lattice(nx, ny, T=0.6 * Tc, s=[1, 1.1, 1.1, 1, 1.1, 1, 1.1, 1.25, 1.25], eps=1.86, solid=solid)
    L.init(rho)
    return L, prof


@pytest.mark.parametrize("along_x", [False, True])
def test_total_momentum_at_rest_is_half_the_wall_reaction(along_x):
    # At rest j = 0, so the total is sum F / 2. For a field that varies only
    # across the channel, Eq. 7 gives F_n(k) = -G psi_k (psi_{k+1} - psi_{k-1})
    # / 2 (axis weight 1/3 plus two diagonals of 1/12), a wall neighbour
    # taking psi_k. The sum over the fluid layers telescopes to
    # -G (psi_last^2 - psi_first^2) / 2 per line, so the total momentum along
    # the normal is -G * lines * (psi_last^2 - psi_first^2) / 4 and zero along
    # the walls.
    nx, ny = (24, 7) if along_x else (7, 24)
    L, prof = _stratified_at_rest(nx, ny, along_x)
    lines = ny if along_x else nx
    n = len(prof)
    psi_first, f1 = L.psi(prof[1])
    psi_last, f2 = L.psi(prof[n - 2])
    assert f1 == 0 and f2 == 0
    G = -1.0
    normal = -G * lines * (psi_last ** 2 - psi_first ** 2) / 4
    px, py = L.momentum()
    along, across = (px, py) if along_x else (py, px)
    assert abs(normal) > 1e-3
    assert along == pytest.approx(normal, rel=1e-12)
    assert abs(across) < 1e-15 * abs(normal)


def test_total_momentum_of_a_uniform_drift():
    # uniform density: F = 0, and f_eq(rho, u) carries j = rho u (Eq. 4)
    nx, ny, rho0, ux, uy = 11, 6, 0.31, 0.013, -0.021
    L = d2q9.Lattice(nx, ny, T=0.6 * 0.0943287, s=[1, 1.1, 1.1, 1, 1.1, 1, 1.1, 1.5, 1.5], eps=1.86)
    L.init(np.full((ny, nx), rho0), np.full((ny, nx), ux), np.full((ny, nx), uy))
    px, py = L.momentum()
    assert px == pytest.approx(nx * ny * rho0 * ux, rel=1e-13)
    assert py == pytest.approx(nx * ny * rho0 * uy, rel=1e-13)


def test_total_momentum_is_invariant_without_walls():
    L = _droplet_lattice(40, 36, 0.7, 1.86, 0.6)
    rho, _, _, _ = L.moments()
    L.init(rho, np.full_like(rho, 0.01), np.full_like(rho, -0.005))
    p0 = L.momentum()
    L.step(200)
    p1 = L.momentum()
    scale = L.mass()
    assert abs(p0[0] - 0.01 * scale) < 1e-3 * abs(p0[0])   # the drift, up to F/2 of the droplet
    assert abs(p1[0] - p0[0]) < 1e-13 * scale and abs(p1[1] - p0[1]) < 1e-13 * scale


def test_pressure_eq10_equals_eos_eq15():
    # With psi from Eq. 13, the LB pressure of Eq. 10 is the CS EOS (Sec. 2.2).
    Tc, _, _ = thermo.critical_point()
    L = d2q9.Lattice(1, 1, T=0.6 * Tc)
    for rho in (1e-4, 0.01, 0.1, 0.3, 0.45):
        psi, fl = L.psi(rho)
        assert fl == 0
        p = L.lib.oracle_pressure(__import__("ctypes").byref(L.p), rho, psi)
        assert p == pytest.approx(thermo.p_eos(rho, 0.6 * Tc), rel=1e-12, abs=1e-17)


def test_psi_clamp_flag_above_root():
    Tc, _, _ = thermo.critical_point()
    L = d2q9.Lattice(1, 1, T=0.5 * Tc)
    r0 = thermo.psi_root(0.5 * Tc)
    assert L.psi(r0 - 1e-3)[1] == 0
    psi, fl = L.psi(r0 + 1e-3)
    assert psi == 0.0 and fl == d2q9.FLAG_PSI_CLAMPED


# ------------------------------------------------------------------ Eq. 9 coexistence

def _slab(tr, eps, tau, nx=128, ny=2, steps=40000):
    Tc, _, _ = thermo.critical_point()
    rg, rl, _ = thermo.maxwell(tr * Tc)
    x = np.arange(nx, dtype=float)
    prof = rg + 0.5 * (rl - rg) * (np.tanh(2 * (x - nx / 4) / 5) - np.tanh(2 * (x - 3 * nx / 4) / 5))
    s = [1.0, 1.1, 1.1, 1.0, 1.1, 1.0, 1.1, 1 / tau, 1 / tau]
    L = d2q9.Lattice(nx, ny, T=tr * Tc, s=s, eps=eps)
    L.init(np.tile(prof, (ny, 1)))
    L.step(steps)
    rho, ux, _, _ = L.moments()
    assert L.flags == 0
    return rho[0, 0], rho[0, nx // 2], np.abs(ux).max()


@pytest.mark.slow
def test_flat_interface_eps0_matches_eq9():
    # Standard forcing (Eq. 14 with eps = 0 is Eq. 8). At 0.9 Tc the interface
    # is wide and Eq. 9 with eps = 0 predicts the coexistence densities.
    Tc, _, _ = thermo.critical_point()
    rg9, rl9, _ = thermo.lb_coexistence(0.9 * Tc, 0.0)
    rg, rl, umax = _slab(0.9, 0.0, 0.6, steps=30000)
    assert umax < 1e-4
    assert rg == pytest.approx(rg9, rel=1e-3)
    assert rl == pytest.approx(rl9, rel=1e-4)


@pytest.mark.slow
def test_flat_interface_li_term_matches_eq9():
    # Li's term with eps = 1 at 0.7 Tc: Eq. 9 gives rho_g = 3.11e-3; the same
    # quadrature at eps = 0.75 or 1.33 gives 1.0e-3 and 6.0e-3, so a wrong
    # factor or sign in Eq. 14 fails by a wide margin.
    Tc, _, _ = thermo.critical_point()
    rg9, rl9, _ = thermo.lb_coexistence(0.7 * Tc, 1.0)
    rg, rl, _ = _slab(0.7, 1.0, 0.6, steps=60000)
    assert rg == pytest.approx(rg9, rel=0.02)
    assert rl == pytest.approx(rl9, rel=5e-4)


def test_y_uniform_field_evolves_as_the_one_row_lattice():
    # A field that depends on x only stays y-uniform, and each of its rows
    # equals the run of the same row alone on an nx x 1 periodic lattice
    # (there every y-neighbour is the node itself): bit for bit, since every
    # node sees the same operands in the same order.
    Tc, _, _ = thermo.critical_point()
    rg, rl, _ = thermo.maxwell(0.7 * Tc)
    nx = 64
    x = np.arange(nx, dtype=float)
    prof = rg + 0.5 * (rl - rg) * (np.tanh(2 * (x - 16) / 4) - np.tanh(2 * (x - 48) / 4))
    ux = 0.01 * np.sin(2 * np.pi * x / nx)
    s = [1.0, 1.1, 1.1, 1.0, 1.1, 1.0, 1.1, 1 / 0.7, 1 / 0.7]
    runs = []
    for ny in (1, 6):
        L = d2q9.Lattice(nx, ny, T=0.7 * Tc, s=s, eps=1.86)
        L.init(np.tile(prof, (ny, 1)), np.tile(ux, (ny, 1)), np.zeros((ny, nx)))
        L.step(50)
        runs.append(L.moments())
    for a, b in zip(runs[0], runs[1]):
        for row in b:
            assert np.array_equal(row, a[0])


# ------------------------------------------------------------------ read-out velocity (Eq. 6)

def test_readout_velocity_hand_computed_three_node_row():
    # A 3 x 1 periodic row with given populations and psi of Eq. 12 at e = 0,
    # psi = exp(-1/rho), worked out by hand: every y-neighbour of a node is
    # the node's own row, so in Eq. 7 the axis term gives
    # (1/3)(psi_{i+1} - psi_{i-1}) and the four diagonals (1/12) * 2 times the
    # same difference, g_x = (psi_{i+1} - psi_{i-1}) / 2, g_y = 0, and
    # F = -G psi_i g. Eq. 6: v = (sum_a e_a f_a + F/2) / rho. A dropped or
    # doubled F/2 misses by |F_x| / (2 rho) > 1e-2 here.
    rng = np.random.default_rng(66)
    nx, G = 3, -1.0
    f = rng.uniform(0.05, 0.15, size=(9, 1, nx)) * np.array([1.0, 3.0, 8.0])
    L = d2q9.Lattice(nx, 1, G=G, eps=0.0, eos="psi_exp")
    L.f[:] = f
    rho, ux, uy, _ = L.moments()
    r = f[:, 0, :].sum(axis=0)
    psi = np.exp(-1.0 / r)
    jx = (f[1] - f[3] + f[5] - f[6] - f[7] + f[8])[0]
    jy = (f[2] - f[4] + f[5] + f[6] - f[7] - f[8])[0]
    for i in range(nx):
        gx = 0.5 * (psi[(i + 1) % nx] - psi[(i - 1) % nx])
        Fx = -G * psi[i] * gx
        assert abs(Fx) / (2 * r[i]) > 1e-2
        assert rho[0, i] == pytest.approx(r[i], rel=1e-15)
        assert ux[0, i] == pytest.approx((jx[i] + 0.5 * Fx) / r[i], rel=1e-13, abs=1e-16)
        assert uy[0, i] == pytest.approx(jy[i] / r[i], rel=1e-13, abs=1e-16)


@pytest.mark.parametrize("tr,eps", [(0.8, 1.0), (0.7, 1.86)])
def test_readout_velocity_vanishes_at_steady_flat_interface(tr, eps):
    # At a steady, mirror-symmetric flat interface the discrete mass flux
    # through every link is zero, which makes the post-collision momentum the
    # negative of the pre-collision one, j* = -j. The collision sends j to
    # j + F (Eq. 3 with Eq. 6), so j = -F/2 and the velocity of Eq. 6,
    # (j + F/2)/rho, is zero to rounding, while j/rho alone (a dropped F/2)
    # or (j + F)/rho (a doubled one) is |F|/(2 rho), about 0.1 in the vapour.
    Tc, _, _ = thermo.critical_point()
    rg, rl, _ = thermo.maxwell(tr * Tc)
    nx = 64
    x = np.arange(nx, dtype=float)
    prof = rg + 0.5 * (rl - rg) * (np.tanh(2 * (x - nx / 4) / 5) - np.tanh(2 * (x - 3 * nx / 4) / 5))
    s = [1.0, 1.1, 1.1, 1.0, 1.1, 1.0, 1.1, 1 / 0.6, 1 / 0.6]
    L = d2q9.Lattice(nx, 1, T=tr * Tc, s=s, eps=eps)
    L.init(prof[None, :])
    L.step(20000)
    assert L.flags == 0
    rho, ux, uy, _ = L.moments()
    jx = np.tensordot(EX, L.f, 1)
    assert np.abs(jx / rho).max() > 0.05
    assert np.abs(ux).max() < 1e-9
    assert np.abs(uy).max() < 1e-15


def test_threaded_sweeps_are_bitwise_serial():
    # The sweeps update nodes independently, so running them on several
    # threads gives the serial result bit for bit (walls included).
    runs = []
    for n in (1, 4):
        if not d2q9.set_threads(n) and n > 1:
            pytest.skip("oracle built without OpenMP")
        L = _droplet_lattice(45, 37, 0.7, 1.86, 0.6, walls=True)
        L.step(30)
        runs.append((L.f.copy(), L.flags))
    d2q9.set_threads(1)
    assert np.array_equal(runs[0][0], runs[1][0]) and runs[0][1] == runs[1][1]
