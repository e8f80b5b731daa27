"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints (tests/golden/paper_values.json), closed forms and integral
identities of the thin-film Green's tensor, a point-dipole limit, thin-film
demagnetisation limits, an independent FFT convolution, exact gradient
identities of a quadratic energy, integrator convergence orders, the
Boltzmann law of a single macrospin, and NVIDIA's own Philox4x32-10 generator.
"""
import ctypes
import ctypes.util
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate, stats

import ndsynth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
MU0 = 4e-7 * math.pi
KB = 1.380649e-23
MAT = GOLD["material"]
A, MS, GAMMA, A_CELL = MAT["A_J_per_m"], MAT["Ms_A_per_m"], MAT["gamma_per_T_s"], MAT["a_m"]


def close(x, g):
    return abs(x - g["value"]) <= g["rel_tol"] * abs(g["value"])


# ------------------------------------------------------------------ units

def test_units_match_printed_values(O):
    lam, B0, t0, J, c = O.units(A, MS, A_CELL, 5e-9, GAMMA)
    assert close(lam * 1e9, GOLD["lambda_ex_nm"])
    assert close(MU0 * MS, GOLD["mu0_Ms_T"])
    assert close(B0, GOLD["B0_T"])
    assert close(t0 * 1e12, GOLD["t0_ps"])
    assert close(GAMMA * B0 / 1e12, GOLD["f0_THz"])
    assert close(1e-7 * GAMMA * MS / 1e9, GOLD["cgs_freq_GHz"])
    assert close(J * 1e21, GOLD["J_L5nm_zJ"])
    assert close(KB * 300 * 1e21, GOLD["kT_300K_zJ"])
    assert close(O.scaled_temperature(300.0, A, 5e-9), GOLD["Tscaled_L5nm_300K"])
    assert close(KB * 300 / (A * A_CELL), GOLD["kT_300K_over_Aa"])
    # B0 has the two printed forms J/(L a^2 Ms) and (lambda^2/a^2) mu0 Ms
    assert B0 == pytest.approx(J / (5e-9 * A_CELL ** 2 * MS), rel=1e-14)
    assert B0 == pytest.approx(lam ** 2 / A_CELL ** 2 * MU0 * MS, rel=1e-14)
    assert c == pytest.approx(A_CELL ** 2 / lam ** 2, rel=1e-15)


def test_noise_variance_formula(O):
    # sigma_s^2 = 2 alpha T dtau (FD theorem integrated over one step)
    assert O.sigma_s(0.01, 0.015931, 0.0133) ** 2 == pytest.approx(2 * 0.01 * 0.015931 * 0.0133, rel=1e-14)


# ----------------------------------------------------- Green's tensor

RNG = np.random.default_rng(7)
DISPL = [(x, y) for x, y in RNG.uniform(-40e-9, 40e-9, (40, 2))] + [(2e-9, 0.0), (0.0, 2e-9), (2e-9, 2e-9)]


@pytest.mark.parametrize("L", [1e-9, 5e-9, 20e-9])
def test_green_trace_vanishes_off_origin(O, L):
    for x, y in DISPL:
        g = O.green(x, y, L)
        scale = np.abs(g).max()
        assert abs(g[0] + g[1] + g[3]) <= 1e-13 * scale


@pytest.mark.parametrize("L,a", [(5e-9, 2e-9), (10e-9, 2e-9), (1e-9, 2e-9), (20e-9, 3e-9)])
def test_self_factors_sum_to_one_and_signs(O, L, a):
    Nx, Nz = O.self_factors(L, a)
    assert 2 * Nx + Nz == pytest.approx(1.0, abs=1e-15)
    assert 0 < Nx < 0.5 and 0 < Nz < 1          # G_xx(0) = -Nx < 0 (sign reading)
    ro = a / math.sqrt(math.pi)
    # thin-cell (L << r_o) and long-cell (L >> r_o) limits of a cylinder
    if L / ro < 1.5:
        assert Nz > Nx
    if L / ro > 8:
        assert Nx == pytest.approx(0.5, abs=0.07)


def test_green_symmetries(O):
    L = 5e-9
    for x, y in DISPL:
        g = O.green(x, y, L)
        gs = O.green(y, x, L)
        assert g[1] == pytest.approx(gs[0], rel=1e-13, abs=1e-30)       # G_yy(x,y) = G_xx(y,x)
        gm = O.green(-x, y, L)
        assert gm[2] == pytest.approx(-g[2], rel=1e-13, abs=1e-30)      # G_xy odd in x
        assert gm[0] == pytest.approx(g[0], rel=1e-13, abs=1e-30)       # G_xx even in x
        assert O.green(x, -y, L)[2] == pytest.approx(-g[2], rel=1e-13, abs=1e-30)
        assert g[3] < 0                                                 # G_zz always negative


def test_green_far_field_is_point_dipole(O):
    # field of a point dipole of moment M L dA:  (L/(4 pi r^5)) (3 r r - r^2 I)
    L = 5e-9
    for ang in np.linspace(0.1, 2 * np.pi, 7):
        r = 70 * L
        x, y = r * np.cos(ang), r * np.sin(ang)
        g = O.green(x, y, L)
        pre = L / (4 * np.pi * r ** 5)
        dip = np.array([pre * (2 * x * x - y * y), pre * (2 * y * y - x * x), pre * 3 * x * y, -L / (4 * np.pi * r ** 3)])
        scale = L / (4 * np.pi * r ** 3)
        assert np.max(np.abs(g - dip)) <= 2e-3 * scale


@pytest.mark.parametrize("L,a", [(5e-9, 2e-9), (10e-9, 2e-9)])
def test_green_infinite_film_identities(O, L, a):
    """A uniform infinite film: the continuum integral of the kernel outside the
    cell disc r_o plus the self term gives h_z = -m_z and h_x = 0."""
    Nx, Nz = O.self_factors(L, a)
    ro = a / math.sqrt(math.pi)

    # integrate in u = r/L; G has units 1/m^2, so G L^2 is dimensionless
    def gzz(u):
        return O.green(u * L, 0.0, L)[3] * L * L * 2 * math.pi * u

    def gxx_ang(u):  # angular average of G_xx: (G_xx(r,0) + G_xx(0,r))/2
        return 0.5 * (O.green(u * L, 0.0, L)[0] + O.green(0.0, u * L, L)[0]) * L * L * 2 * math.pi * u

    u0 = ro / L
    Izz = integrate.quad(gzz, u0, 50, limit=400, epsabs=1e-13)[0] + integrate.quad(gzz, 50, np.inf, limit=400, epsabs=1e-13)[0]
    Ixx = integrate.quad(gxx_ang, u0, 50, limit=400, epsabs=1e-13)[0] + integrate.quad(gxx_ang, 50, np.inf, limit=400, epsabs=1e-13)[0]
    assert Izz - Nz == pytest.approx(-1.0, abs=1e-8)
    assert Ixx - Nx == pytest.approx(0.0, abs=1e-8)


# ------------------------------------------------------- demag field

def fft_convolution_field(O, model, m):
    """Independent route: zero-padded circular convolution with numpy's FFT of
    the oracle's kernel table, P >= 2D-1 (exact linear convolution)."""
    D, a, L = model.D, model.a, model.L
    P = 1
    while P < 2 * D - 1:
        P *= 2
    G = np.zeros((4, P, P))
    Nx, Nz = O.self_factors(L, a)
    for dy in range(-(D - 1), D):
        for dx in range(-(D - 1), D):
            if dx == 0 and dy == 0:
                g = np.array([-Nx, -Nx, 0.0, -Nz])
            else:
                g = O.green(dx * a, dy * a, L) * a * a
            G[:, dy % P, dx % P] = g
    Gh = np.fft.fft2(G)
    mm = np.zeros((3, P, P))
    mm[:, :D, :D] = m * model.mask
    Mh = np.fft.fft2(mm)
    H = np.empty_like(Mh)
    H[0] = Gh[0] * Mh[0] + Gh[2] * Mh[1]
    H[1] = Gh[2] * Mh[0] + Gh[1] * Mh[1]
    H[2] = Gh[3] * Mh[2]
    h = np.real(np.fft.ifft2(H))[:, :D, :D]
    return h * model.mask


@pytest.mark.parametrize("R,L", [(6e-9, 5e-9), (13e-9, 3e-9), (16e-9, 10e-9)])
def test_direct_sum_equals_fft_convolution(O, R, L):
    model = O.Model(R, L)
    m = ndsynth.random_unit_vectors(model.D, seed=3) * model.mask
    h = model.demag(m)
    hf = fft_convolution_field(O, model, m)
    assert np.linalg.norm(h - hf) <= 1e-12 * np.linalg.norm(hf)


def test_single_source_brute_force(O):
    """One source cell: the field at every other cell is a^2 G(r_i - r_j) m_j,
    and at the source itself -N m (tiny-input brute force)."""
    model = O.Model(8e-9, 5e-9)
    D, a = model.D, model.a
    js, is_ = D // 2, D // 2 - 1
    m = np.zeros((3, D, D))
    m[:, js, is_] = [0.3, -0.5, 0.8]
    h = model.demag(m)
    for j in range(D):
        for i in range(D):
            if not model.mask[j, i]:
                assert np.all(h[:, j, i] == 0)
                continue
            if (j, i) == (js, is_):
                exp = [-model.Nx * 0.3, -model.Nx * -0.5, -model.Nz * 0.8]
            else:
                g = O.green((i - is_) * a, (j - js) * a, model.L) * a * a
                exp = [g[0] * 0.3 + g[2] * -0.5, g[2] * 0.3 + g[1] * -0.5, g[3] * 0.8]
            assert np.allclose(h[:, j, i], exp, rtol=1e-13, atol=1e-16)


def test_thin_film_limits(O):
    """A large thin disk: uniform m_z gives h_z ~ -1 inside (minus the finite
    size correction); uniform in-plane m gives a small h_x inside."""
    R, L = 60e-9, 6e-9
    model = O.Model(R, L)
    D = model.D
    c = D // 2
    mz = np.zeros((3, D, D)); mz[2] = model.mask
    hz = model.demag(mz)[2, c - 1:c + 1, c - 1:c + 1].mean()
    # continuum value at the centre: -1 + int_R^inf L / (s (s + r)) dr
    # (integrated in u = r/L; the lattice sum differs from the continuum by O(a/L) near the origin)
    corr = integrate.quad(lambda u: 1.0 / (math.hypot(u, 1.0) * (math.hypot(u, 1.0) + u)), R / L, np.inf)[0]
    assert hz == pytest.approx(-1.0 + corr, abs=0.03)
    assert hz < -0.85
    mx = np.zeros((3, D, D)); mx[0] = model.mask
    hx = model.demag(mx)[0, c - 1:c + 1, c - 1:c + 1].mean()
    assert -0.08 < hx < 0.0


# ---------------------------------------------------- field and energy

def test_energy_gradient_is_minus_field(O):
    """E/J is a quadratic form plus a linear term, so the central difference is
    exact up to rounding: dE/dm_i = -J b_i (Eq. Bi from Eq. Hmm)."""
    model = O.Model(10e-9, 5e-9, hext=(2e4, -1e4, 3e4))
    m = ndsynth.random_unit_vectors(model.D, seed=11) * model.mask
    b = model.field(m)
    h = 1e-4
    rng = np.random.default_rng(0)
    cells = [tuple(x) for x in np.argwhere(model.mask)]
    for idx in rng.choice(len(cells), 12, replace=False):
        j, i = cells[idx]
        for k in range(3):
            mp = m.copy(); mp[k, j, i] += h
            mm = m.copy(); mm[k, j, i] -= h
            g = (model.energy(mp) - model.energy(mm)) / (2 * h)
            assert g == pytest.approx(-b[k, j, i], rel=1e-7, abs=1e-9)


def test_exchange_of_uniform_state(O):
    """Uniform in-plane state: the exchange part of b_i counts the in-disk
    neighbours, and the pair sum equals the number of neighbour pairs."""
    model = O.Model(12e-9, 5e-9)
    D, M = model.D, model.mask.astype(bool)
    m = np.zeros((3, D, D)); m[0] = M
    ex, _ = model.field_parts(m)
    nb = np.zeros((D, D))
    pad = np.pad(M, 1)
    nb = pad[:-2, 1:-1].astype(int) + pad[2:, 1:-1] + pad[1:-1, :-2] + pad[1:-1, 2:]
    assert np.array_equal(ex[0], nb * M)
    pairs = int((M[:, :-1] & M[:, 1:]).sum() + (M[:-1, :] & M[1:, :]).sum())
    assert model.pair_count() == pairs
    hM = model.demag(m)
    assert model.energy(m) == pytest.approx(-(pairs + model.c * 0.5 * (hM[0] * m[0]).sum()), rel=1e-14)


# -------------------------------------------------------------- RK4

def test_rk4_conserves_energy_and_norm(O):
    """alpha = 0: energy to better than 12 digits (Sec. III.A) at dtau = 0.04,
    starting, as the paper does, from a vortex cleaned of spin waves by a damped
    pre-phase."""
    model = O.Model(12e-9, 5e-9, alpha=0.1)
    m0 = model.rk4(model.init_vortex(3e-9, 1e-9), 2500, 0.04)
    model.set_alpha(0.0)
    E0 = model.energy(m0)
    m = m0
    for _ in range(4):
        m = model.rk4(m, 250, 0.04)
        assert abs(model.energy(m) - E0) <= 1e-12 * abs(E0)
    n = np.sqrt((m ** 2).sum(0))[model.mask.astype(bool)]
    assert np.max(np.abs(n - 1)) < 1e-14
    assert np.linalg.norm(m - m0) > 1e-3 * np.linalg.norm(m0)   # the vortex moved


def test_rk4_damping_decreases_energy(O):
    model = O.Model(10e-9, 5e-9, alpha=0.05)
    m = ndsynth.random_unit_vectors(model.D, seed=5) * model.mask
    E = model.energy(m)
    for _ in range(10):
        m = model.rk4(m, 5, 0.04)
        En = model.energy(m)
        assert En < E
        E = En


def test_rk4_is_fourth_order(O):
    model = O.Model(8e-9, 5e-9, alpha=0.1, hext=(0, 0, 5e4))
    m0 = ndsynth.random_unit_vectors(model.D, seed=2) * model.mask
    T = 0.64
    ref = model.rk4(m0, 256, T / 256)
    e1 = np.linalg.norm(model.rk4(m0, 8, T / 8) - ref)
    e2 = np.linalg.norm(model.rk4(m0, 16, T / 16) - ref)
    assert 11 < e1 / e2 < 22   # 2^4 = 16


# -------------------------------------------------------------- Heun

def test_heun_deterministic_is_second_order(O):
    model = O.Model(8e-9, 5e-9, alpha=0.1, hext=(0, 0, 5e4))
    m0 = ndsynth.random_unit_vectors(model.D, seed=2) * model.mask
    T = 0.32
    ref = model.rk4(m0, 512, T / 512)
    e1 = np.linalg.norm(model.heun(m0, 16, T / 16, 0.0, 0) - ref)
    e2 = np.linalg.norm(model.heun(m0, 32, T / 32, 0.0, 0) - ref)
    assert 3.0 < e1 / e2 < 5.5  # 2^2 = 4


def test_heun_noise_is_reused_in_corrector_and_counter_based(O):
    model = O.Model(8e-9, 5e-9, alpha=0.02)
    m0 = ndsynth.random_unit_vectors(model.D, seed=9) * model.mask
    a = model.heun(m0, 6, 0.01, 0.05, seed=42, step0=100)
    b = model.heun(model.heun(m0, 2, 0.01, 0.05, seed=42, step0=100), 4, 0.01, 0.05, seed=42, step0=102)
    assert np.array_equal(a, b)          # resuming at step0 is bit-identical
    c = model.heun(m0, 6, 0.01, 0.05, seed=43, step0=100)
    assert not np.allclose(a, c)


@pytest.mark.slow
def test_macrospin_boltzmann(O):
    """One cell in a field along z: the stationary m_z distribution of the
    paper's Langevin equation (noise in the precession and damping terms,
    <b_s b_s> = 2 alpha T) is Boltzmann at T (1 + alpha^2) -- the Fokker-Planck
    diffusion tensor of that equation is (1 + alpha^2) alpha T times the
    tangent projector -- with energy -J c [h m_z + (N_x - N_z) m_z^2 / 2]."""
    alpha, hz, Ts, dtau = 1.0, 5.0, 0.5, 0.005
    model = O.Model(1e-9, 5e-9, alpha=alpha, hext=(0, 0, hz * MS))
    assert model.D == 1 and model.C == 1
    c, Nx, Nz = model.c, model.Nx, model.Nz

    def moments(T):
        f = lambda z: np.exp((c * hz * z + 0.5 * c * (Nx - Nz) * z * z) / T)
        Z = integrate.quad(f, -1, 1)[0]
        return integrate.quad(lambda z: z * f(z), -1, 1)[0] / Z

    zs = []
    for s in range(6):
        v = np.zeros((3, 1, 1)); v[2] = 1.0
        v = model.heun(v, 4000, dtau, Ts, seed=1000 + s)
        for blk in range(120):
            v = model.heun(v, 1500, dtau, Ts, seed=1000 + s, step0=4000 + 1500 * blk)
            zs.append(v[2, 0, 0])
    zs = np.array(zs)
    err = zs.std() / np.sqrt(len(zs))
    pred = moments(Ts * (1 + alpha ** 2))
    wrong = moments(Ts)
    assert abs(zs.mean() - pred) < 4 * err + 0.01
    assert abs(zs.mean() - wrong) > 4 * err


# ----------------------------------------------------- Philox + normals

def _curand():
    for name in ("libcurand.so.10", "libcurand.so", ctypes.util.find_library("curand")):
        if not name:
            continue
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    return None


def test_philox_matches_curand_host_generator(O):
    """NVIDIA's host Philox4x32-10 generator (an independent implementation):
    its n-th block of four words is Philox(counter = (0, 0, n, 0), key = seed)."""
    cr = _curand()
    if cr is None:
        pytest.skip("libcurand not available")
    for seed in (0, 0x123456789ABCDEF0, 2 ** 64 - 1):
        gen = ctypes.c_void_p()
        if cr.curandCreateGeneratorHost(ctypes.byref(gen), 161) != 0:
            pytest.skip("curand host generator unavailable")
        try:
            assert cr.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
            n = 4 * 64
            out = np.zeros(n, dtype=np.uint32)
            assert cr.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
        finally:
            cr.curandDestroyGenerator(gen)
        key = (seed & 0xFFFFFFFF, seed >> 32)
        mine = np.concatenate([O.philox4x32_10((0, 0, blk, 0), key) for blk in range(64)])
        assert np.array_equal(out, mine)


def test_thermal_normals_are_standard_normal(O):
    w = O.normals_block(seed=12345, step=7, ncell=400000).ravel()
    n = w.size
    assert abs(w.mean()) < 5 / np.sqrt(n)
    assert abs(w.var() - 1) < 5 * np.sqrt(2 / n)
    assert abs(stats.kurtosis(w, fisher=False) - 3) < 5 * np.sqrt(24 / n)
    assert stats.kstest(w, "norm").pvalue > 1e-4
    w2 = O.normals_block(seed=12345, step=8, ncell=400000).ravel()
    assert abs(np.corrcoef(w, w2)[0, 1]) < 5 / np.sqrt(n)
    ww = w.reshape(-1, 3)
    assert abs(np.corrcoef(ww[:, 0], ww[:, 1])[0, 1]) < 5 / np.sqrt(n / 3)
    assert abs(np.corrcoef(ww[:, 0], ww[:, 2])[0, 1]) < 5 / np.sqrt(n / 3)


# ----------------------------------------------------- vortex + core

def test_init_vortex_sense_and_core_estimator(O):
    model = O.Model(30e-9, 5e-9)
    X0 = (3.3e-9, -1.7e-9)
    m = model.init_vortex(*X0)
    st, xc, rv = model.vortex_core(m)
    assert st == 0
    assert np.allclose(xc, X0, atol=1e-13)       # Gaussian core sampled on the grid: centroid is X0
    assert np.hypot(*(rv - np.array(X0))) < model.a
    # counter-clockwise circulation (chirality +1): right of the core m ~ +y, above it m ~ -x
    x, y = model.cell_centres()
    j, i = np.unravel_index(np.argmin((x - X0[0] - 10e-9) ** 2 + (y - X0[1]) ** 2), x.shape)
    assert m[1, j, i] > 0.95
    j, i = np.unravel_index(np.argmin((x - X0[0]) ** 2 + (y - X0[1] - 10e-9) ** 2), x.shape)
    assert m[0, j, i] < -0.95
    assert m[2].max() > 0.5 and m[2].min() >= 0   # polarity +1
    assert np.allclose((m ** 2).sum(0)[model.mask.astype(bool)], 1.0)


def test_core_reports_no_vortex_for_uniform_state(O):
    model = O.Model(20e-9, 5e-9)
    m = np.zeros((3, model.D, model.D)); m[0] = model.mask
    st, _, _ = model.vortex_core(m)
    assert st == 1


# ------------------------------------------------ constrained relaxation

@pytest.mark.slow
def test_relaxation_fixed_point_and_kF_consistency(O):
    """Relax at X = 0 and X = 2a on a small disk: converged states satisfy the
    constraint and the torque condition, the centre is the minimum, and k_F from
    the energy difference (Eq. Ux) matches k_F from the Lagrange multiplier
    (envelope theorem: dU/dX = J lambda_x sum_W m_z^2 / a)."""
    model = O.Model(30e-9, 10e-9)    # the 4 lambda_ex window must sit inside the disk
    a = model.a
    out = {}
    for X in (0.0, 2 * a):
        m0 = model.init_vortex(X, 0.0)
        r = model.relax(m0, (X, 0.0), tol=1e-9, max_iter=20000)
        assert r["status"] == 0, r["iters"]
        C = model.constraint(r["m"], (X, 0.0))
        assert np.max(np.abs(C)) < 1e-6
        assert r["U"] < model.energy(m0)
        out[X] = r
    assert abs(out[0.0]["lam"]).max() < 1e-6
    U0, U1 = out[0.0]["U"], out[2 * a]["U"]
    kF = O.kF_from_energies(U0 * model.J, U1 * model.J, 2 * a)
    assert kF > 0
    m1 = out[2 * a]["m"]
    x, y = model.cell_centres()
    W = ((x - 2 * a) ** 2 + y ** 2 < (4 * model.lambda_ex) ** 2) & model.mask.astype(bool)
    S = (m1[2][W] ** 2).sum()
    dUdX = model.J * out[2 * a]["lam"][0] * S / a
    kF_lagrange = dUdX / (2 * a)
    assert kF == pytest.approx(kF_lagrange, rel=0.03)
    st, xc, _ = model.vortex_core(m1)
    assert st == 0 and abs(xc[0] - 2 * a) < 0.1 * a and abs(xc[1]) < 0.05 * a


def test_relax_sweep_reduces_constraint_violation(O):
    model = O.Model(16e-9, 10e-9)
    X = (2.5e-9, 1.0e-9)
    m = model.init_vortex(0.0, 0.0)      # core deliberately off the target
    lam = np.zeros(2)
    c0 = np.abs(model.constraint(m, X)).max()
    for _ in range(30):
        m, lam, res = model.relax_sweep(m, X, lam)
    assert np.abs(model.constraint(m, X)).max() < 0.05 * c0


# ------------------------------------------------ closed-form physics

def test_statistics_closed_forms(O):
    kT = KB * 300.0
    for case in GOLD["rrms_predictions"]["cases"]:
        kF = case["kF_A_per_a"] * A / A_CELL
        nm = 1e-9   # integrate in nanometres
        rr = integrate.quad(lambda u: (u * nm) ** 2 * O.p_r(u * nm, kF, kT) * nm, 0, 200)[0]
        assert math.sqrt(rr) * 1e9 == pytest.approx(case["rrms_nm"], abs=GOLD["rrms_predictions"]["abs_tol_nm"])
        assert rr == pytest.approx(2 * kT / kF, rel=1e-9)
        assert integrate.quad(lambda u: O.p_r(u * nm, kF, kT) * nm, 0, 200)[0] == pytest.approx(1.0, abs=1e-9)
        rmax = math.sqrt(kT / kF)
        assert O.p_r(rmax, kF, kT) == pytest.approx(math.exp(-0.5) / rmax, rel=1e-12)
        assert O.p_r(rmax * 1.01, kF, kT) < O.p_r(rmax, kF, kT) > O.p_r(rmax * 0.99, kF, kT)


def test_thiele_linear_fit_coefficients(O):
    lam, B0, t0, J, c = O.units(A, MS, A_CELL, 10e-9, GAMMA)
    coeff = lam ** 2 / (8 * A_CELL ** 2)                     # kF = coeff mu0 Ms^2 L^2/R
    assert coeff == pytest.approx(GOLD["kF_linear_coeff"]["value"], rel=GOLD["kF_linear_coeff"]["rel_tol"])
    L, R = 10e-9, 60e-9
    kF = 0.25 * L ** 2 / R * A / A_CELL ** 2
    Om = abs(O.omega_G(kF, A_CELL, L, A, 1))
    assert Om / (L / R) == pytest.approx(GOLD["OmegaG_coeff"]["value"], rel=GOLD["OmegaG_coeff"]["rel_tol"])
    w = GAMMA * B0 * Om
    assert w / (GAMMA * MU0 * MS * L / R) == pytest.approx(GOLD["omegaG_coeff"]["value"], rel=GOLD["omegaG_coeff"]["rel_tol"])
    f = w / (2 * math.pi)
    assert f / (1e-7 * GAMMA * MS * L / R) == pytest.approx(GOLD["fG_coeff"]["value"], rel=GOLD["fG_coeff"]["rel_tol"])
    # omega_G = -kF/G in physical units is the same number
    G = O.gyrovector(L, MS, GAMMA, 1)
    assert abs(kF / G) == pytest.approx(w, rel=1e-12)


def test_gyrotropic_mass(O):
    g = GOLD["mG_R100nm_kg"]
    R, L = g["R_m"], 10e-9
    kF = GOLD["kF_linear_coeff"]["value"] * MU0 * MS ** 2 * L ** 2 / R
    G = O.gyrovector(L, MS, GAMMA, 1)
    assert G ** 2 / kF == pytest.approx(g["value"], rel=g["rel_tol"])


# ------------------------------------------- pins of the sampled field, <m>

def test_field_at_equals_the_full_field(O):
    """The sampled direct sum (used for the largest grids) equals the full
    field at those cells: same Green's table, component order and exchange."""
    model = O.Model(20e-9, 5e-9, hext=(1.5e4, -2.5e4, 3.5e4))
    m = ndsynth.random_unit_vectors(model.D, seed=31) * model.mask
    full = model.field(m)
    inside = np.flatnonzero(model.mask.ravel())
    cells = np.concatenate([inside[ndsynth.sample_indices(len(inside), 40, seed=4)], inside[:3], inside[-3:],
                            np.flatnonzero(model.mask.ravel() == 0)[:2]])     # two outside cells read as zero
    got = model.field_at(m, cells)
    ref = np.stack([full[:, c // model.D, c % model.D] for c in cells])
    assert np.abs(got - ref).max() <= 1e-14 * np.abs(full).max()
    assert np.all(got[-2:] == 0)


def test_mean_m_is_the_average_over_disk_cells(O):
    model = O.Model(17e-9, 5e-9)
    m = ndsynth.random_unit_vectors(model.D, seed=8)        # nonzero outside the disk too
    m = m * model.mask
    inside = model.mask.astype(bool)
    ref = np.array([m[k][inside].mean() for k in range(3)])
    assert np.allclose(model.mean_m(m), ref, rtol=0, atol=1e-15)
    # a uniform state averages to itself
    u = np.zeros((3, model.D, model.D)); u[1] = model.mask
    assert np.allclose(model.mean_m(u), [0.0, 1.0, 0.0], atol=1e-15)


def _two_vortex_state(model, c1, c2, core1, core2):
    """In-plane angle winding +1 around each of two plaquette centres c1, c2
    (cell units, relative to the grid centre); m_z = 0.05 everywhere except the
    four corners of the two plaquettes, which carry core1 and core2."""
    D = model.D
    idx = np.arange(D) - 0.5 * (D - 1)
    x, y = np.meshgrid(idx, idx, indexing="xy")
    phi = np.arctan2(y - c1[1], x - c1[0]) + np.arctan2(y - c2[1], x - c2[0]) + 0.5 * np.pi
    mz = np.full((D, D), 0.05)
    for c, v in ((c1, core1), (c2, core2)):
        i0, j0 = int(round(c[0] + 0.5 * (D - 1) - 0.5)), int(round(c[1] + 0.5 * (D - 1) - 0.5))
        mz[j0:j0 + 2, i0:i0 + 2] = v
    sp = np.sqrt(1 - mz ** 2)
    m = np.stack([sp * np.cos(phi), sp * np.sin(phi), mz]) * model.mask
    return m


def test_core_tie_break_picks_the_largest_corner_mz2(O):
    """Two plaquettes of winding +1 (Sec. IV's vorticity centre, tie-break of
    the reading): the one whose corners carry the larger sum of m_z^2 wins;
    on an exact tie the first in row-major order (smaller y, then x) wins."""
    model = O.Model(30e-9, 5e-9)
    a = model.a
    c1, c2 = (-4.0, -3.0), (5.0, 4.0)                 # plaquette centres (half-integer grid offsets)
    for core1, core2, want in ((0.6, 0.8, c2), (0.8, 0.6, c1), (0.7, 0.7, c1)):
        m = _two_vortex_state(model, c1, c2, core1, core2)
        st, xc, rv = model.vortex_core(m)
        assert st == 0
        assert np.allclose(rv, np.array(want) * a, atol=1e-15), (core1, core2, rv / a)
    # the same pair placed on one row: the smaller x is first
    c3, c4 = (-5.0, 2.0), (6.0, 2.0)
    st, xc, rv = model.vortex_core(_two_vortex_state(model, c3, c4, 0.7, 0.7))
    assert st == 0 and np.allclose(rv, np.array(c3) * a, atol=1e-15)


# ------------------------------------------------ rotational-speed law

def test_speed_law_of_the_rotational_velocity(O):
    """Sec. VI: f(V) = beta m_G V exp(-beta m_G V^2/2) with m_G = G^2/k_F is
    p(r) mapped by V = |omega_G| r, omega_G = k_F/G; V_rms = sqrt(2 k_F kT)/G,
    so <V^2> = 2kT/m_G.  Checked by quadrature and against the oracle's own
    p(r) and gyrovector, for the paper's two r_rms examples."""
    kT = KB * 300.0
    for case in GOLD["rrms_predictions"]["cases"]:
        kF = case["kF_A_per_a"] * A / A_CELL
        L = case["L_nm"] * 1e-9
        G = O.gyrovector(L, MS, GAMMA, 1)
        mG = O.gyro_mass(G, kF)
        assert mG == pytest.approx(G * G / kF, rel=1e-15)
        w = kF / G
        vrms = math.sqrt(2 * kF * kT) / G
        s = vrms   # integrate in units of V_rms
        norm = integrate.quad(lambda u: O.f_V(u * s, mG, kT) * s, 0, 40)[0]
        v2 = integrate.quad(lambda u: (u * s) ** 2 * O.f_V(u * s, mG, kT) * s, 0, 40)[0]
        assert norm == pytest.approx(1.0, abs=1e-10)
        assert v2 == pytest.approx(2 * kT / mG, rel=1e-9)
        assert math.sqrt(v2) == pytest.approx(vrms, rel=1e-9)
        # f(V) = p(V/omega)/omega, p the oracle's radial law (Eq. pr)
        for u in (0.1, 0.7, 1.0, 2.3):
            V = u * vrms
            assert O.f_V(V, mG, kT) == pytest.approx(O.p_r(V / w, kF, kT) / w, rel=1e-12)
        vmax = math.sqrt(kT / mG)
        assert O.f_V(vmax, mG, kT) == pytest.approx(math.exp(-0.5) / vmax, rel=1e-12)
        # V_rms = |omega_G| r_rms with the paper's r_rms (Sec. VI)
        assert vrms / w * 1e9 == pytest.approx(case["rrms_nm"], abs=GOLD["rrms_predictions"]["abs_tol_nm"])


# ---------------------------------------------- gyration frequency fit

def test_omega_from_track_recovers_circular_motion(O):
    """The Omega_G estimator on exact tracks: clockwise and counter-clockwise
    circles over several turns, an off-centre start, and a shrinking spiral."""
    dtau = 0.7
    tau = np.arange(900) * dtau
    for om, r0, phase in ((-3.06e-3, 4e-9, 0.3), (2.5e-3, 1e-9, -2.9), (-0.02, 6e-9, 3.1)):
        x, y = r0 * np.cos(om * tau + phase), r0 * np.sin(om * tau + phase)
        assert O.omega_from_track(x, y, dtau) == pytest.approx(om, rel=1e-10)
        rr = r0 * np.exp(-1e-4 * tau)
        x, y = rr * np.cos(om * tau + phase), rr * np.sin(om * tau + phase)
        assert O.omega_from_track(x, y, dtau) == pytest.approx(om, rel=1e-10)
    # a slowly modulated angular speed: the least-squares slope is the mean rate
    th = -3e-3 * tau + 0.2 * np.sin(2 * np.pi * tau / tau[-1])
    slope = np.polyfit(tau, th, 1)[0]
    assert O.omega_from_track(np.cos(th), np.sin(th), dtau) == pytest.approx(slope, rel=1e-10)


# --------------------------------------------------- power spectrum

def test_power_spectrum_parseval_and_pure_tone(O):
    """The averaged periodogram (Sec. V's thermal power spectra): the one-sided
    sum times the bin width equals each window's mean square after its mean is
    removed (Parseval), and a tone at bin k0 puts dt W A^2 / 2 in that bin and
    nothing elsewhere."""
    W, dt = 256, 2.5e-12
    rng = np.random.default_rng(3)
    x = rng.standard_normal(3 * W + 17) + 0.4
    psd, nw = O.power_spectrum(x, W, dt)
    assert nw == 3
    win = x[:3 * W].reshape(3, W)
    ms = np.mean([np.mean((w - w.mean()) ** 2) for w in win])
    assert psd.sum() / (W * dt) == pytest.approx(ms, rel=1e-12)
    k0, amp = 19, 0.37
    t = np.arange(2 * W)
    tone = amp * np.cos(2 * np.pi * k0 * t / W + 0.8) + 5.0      # the constant is removed per window
    psd, nw = O.power_spectrum(tone, W, dt)
    assert nw == 2
    assert psd[k0] == pytest.approx(dt * W * amp ** 2 / 2, rel=1e-12)
    others = np.delete(psd, k0)
    assert others.max() <= 1e-20 * psd[k0] + 1e-40
    assert O.power_spectrum(x[:W - 1], W, dt)[1] == 0


# ------------------------------------------- user Green's table (Sec. II.B)

def test_set_green_with_the_closed_form_table_changes_nothing(O):
    model = O.Model(14e-9, 5e-9, hext=(0, 1e4, 0))
    m = ndsynth.random_unit_vectors(model.D, seed=12) * model.mask
    b0 = model.field(m)
    model.set_green(model.quarter_table())
    assert np.array_equal(model.field(m), b0)


def test_set_green_extends_a_quarter_table_by_symmetry(O):
    """A single source cell at the centre of an odd grid sees the table itself:
    h^M(dx, dy) = table(|dx|, |dy|) for xx, yy, zz and sign(dx) sign(dy) times it
    for xy (zero on the axes), so an arbitrary quarter table is reproduced in
    every quadrant with the tensor's parities."""
    model = O.Model(9e-9, 5e-9)                       # D = 9, centre cell (4, 4)
    D = model.D
    assert D % 2 == 1
    rng = np.random.default_rng(5)
    q = rng.standard_normal((4, D, D))
    model.set_green(q)
    c = D // 2
    for comp in range(3):
        m = np.zeros((3, D, D)); m[comp, c, c] = 1.0
        hM = model.demag(m)
        for j in range(D):
            for i in range(D):
                if not model.mask[j, i]:
                    continue
                dx, dy = i - c, j - c
                qq = q[:, abs(dy), abs(dx)]
                s = np.sign(dx) * np.sign(dy)
                if comp == 0:     # m = x: h = (Gxx, Gxy, 0)
                    want = (qq[0], s * qq[2], 0.0)
                elif comp == 1:   # m = y: h = (Gxy, Gyy, 0)
                    want = (s * qq[2], qq[1], 0.0)
                else:             # m = z: h = (0, 0, Gzz)
                    want = (0.0, 0.0, qq[3])
                assert np.allclose(hM[:, j, i], want, rtol=0, atol=1e-15), (comp, i, j)


def test_set_green_scaling_zz_halves_the_perpendicular_demag(O):
    model = O.Model(14e-9, 5e-9)
    m = ndsynth.random_unit_vectors(model.D, seed=13) * model.mask
    hM = model.demag(m)
    q = model.quarter_table()
    q[3] *= 0.5
    model.set_green(q)
    h2 = model.demag(m)
    assert np.array_equal(h2[:2], hM[:2])
    assert np.array_equal(h2[2], 0.5 * hM[2])


# ------------------------------------------ variants: mask and field pulses

def _shapes(D):
    """Cell sets of the D x D grid: the full square, an ellipse, an annulus."""
    idx = np.arange(D) - 0.5 * (D - 1)
    x, y = np.meshgrid(idx, idx, indexing="xy")
    r = 0.5 * D
    return {"square": np.ones((D, D), np.uint8),
            "ellipse": ((x / r) ** 2 + (y / (0.55 * r)) ** 2 <= 1).astype(np.uint8),
            "annulus": ((x * x + y * y <= r * r) & (x * x + y * y >= (0.4 * r) ** 2)).astype(np.uint8)}


def test_set_mask_with_the_disk_mask_changes_nothing(O):
    model = O.Model(14e-9, 5e-9, hext=(0, 2e4, 0))
    m = ndsynth.random_unit_vectors(model.D, seed=3) * model.mask
    b0, E0, C0 = model.field(m), model.energy(m), model.C
    model.set_mask(model.mask.copy())
    assert model.C == C0
    assert np.array_equal(model.field(m), b0) and model.energy(m) == E0


@pytest.mark.parametrize("shape", ["square", "ellipse", "annulus"])
def test_masked_direct_sum_equals_fft_convolution(O, shape):
    """Any cell set: the direct sum over the new mask equals the independent
    FFT convolution restricted to it, the exchange counts neighbours inside it
    only, and the energy gradient is still -b (Eq. Hmm, Eq. Bi)."""
    model = O.Model(13e-9, 4e-9)
    mk = _shapes(model.D)[shape]
    model.set_mask(mk)
    assert model.C == int(mk.sum()) and np.array_equal(model.mask, mk)
    m = ndsynth.random_unit_vectors(model.D, seed=17) * mk
    ref = fft_convolution_field(O, model, m)
    hM = model.demag(m)
    assert np.linalg.norm(hM - ref) <= 1e-12 * np.linalg.norm(ref)
    u = np.zeros((3, model.D, model.D)); u[0] = mk
    ex, _ = model.field_parts(u)
    pad = np.pad(mk, 1).astype(int)
    nb = pad[:-2, 1:-1] + pad[2:, 1:-1] + pad[1:-1, :-2] + pad[1:-1, 2:]
    assert np.array_equal(ex[0], nb * mk)
    # dE/dm_i = -b_i: central difference of the quadratic energy at one cell
    j, i = np.argwhere(mk)[len(np.argwhere(mk)) // 3]
    b = model.field(m)
    for c in range(3):
        e = np.zeros_like(m); e[c, j, i] = 1e-3
        g = (model.energy(m + e) - model.energy(m - e)) / 2e-3
        assert g == pytest.approx(-b[c, j, i], rel=1e-9, abs=1e-12)


def test_field_schedule_of_the_static_value_changes_nothing(O):
    model = O.Model(10e-9, 5e-9, alpha=0.05, hext=(1e4, 0, -2e4))
    m0 = model.init_vortex(1e-9, 0.0)
    dtau = 0.02
    r0, h0 = model.rk4(m0, 7, dtau), model.heun(m0, 7, dtau, 0.01, 3, 5)
    model.set_schedule(np.tile([1e4, 0, -2e4], (20, 1)))
    assert np.array_equal(model.rk4(m0, 7, dtau), r0)
    assert np.array_equal(model.heun(m0, 7, dtau, 0.01, 3, 5), h0)
    model.set_schedule(None)
    assert np.array_equal(model.rk4(m0, 7, dtau), r0)


def test_field_pulse_precesses_a_macrospin_by_the_closed_form_angle(O):
    """One cell (D = 1), alpha = 0, field along z: m_z is conserved and the
    in-plane angle turns at d(phi)/d(tau) = -(a^2/lambda^2)(h_z + (N_x - N_z) m_z)
    (m x b with the cell's self field -N m).  A pulse h1 for n1 steps, then
    h0, turns it by the sum of the two rates times their durations; RK4 with
    the schedule reproduces that to its own accuracy."""
    a = 2e-9
    model = O.Model(0.5 * a, 5e-9, a=a, hext=(0, 0, 3e4))
    assert model.D == 1 and model.C == 1
    Ms = model.Ms
    th = 0.7
    m0 = np.array([np.sin(th), 0.0, np.cos(th)]).reshape(3, 1, 1)
    n1, n2, dtau, H1 = 300, 500, 0.01, 9e4
    hs = np.zeros((n1, 3)); hs[:, 2] = H1
    model.set_schedule(hs)
    out = model.rk4(m0, n1 + n2, dtau)
    c, mz = model.c, np.cos(th)
    rate = lambda H: -c * (H / Ms + (model.Nx - model.Nz) * mz)
    phi = rate(H1) * n1 * dtau + rate(3e4) * n2 * dtau
    assert out[2, 0, 0] == pytest.approx(mz, abs=1e-12)
    got = math.atan2(out[1, 0, 0], out[0, 0, 0])
    assert abs((got - phi + math.pi) % (2 * math.pi) - math.pi) < 1e-9
    # the same run split in two calls, the second starting at step n1 + 100
    mid = model.rk4(m0, n1 + 100, dtau, step0=0)
    assert np.allclose(model.rk4(mid, n2 - 100, dtau, step0=n1 + 100), out, atol=1e-14)
