"""Pins of the oracle against facts that do not come from the oracle itself:
hand values, analytic cell averages, the Jiang-Shu integral definition of the
smoothness indicators, symmetries, exact solutions, conservation, and the
paper's printed Tables 1 and 2.  CPU only."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import exact
from paper_2405_12301_gb300 import inputs as I


# ----------------------------------------------------------------- physics
def test_pressure_and_flux_hand_values():
    """U = (1, 0, 0, 0, 2.5), gamma = 1.4: p = 0.4 * 2.5 = 1, F = (0, 1, 0, 0, 0)."""
    c = O.Cfg(dim=3, n=(4, 4, 4))
    q = np.array([1.0, 0.0, 0.0, 0.0, 2.5])
    assert O.pressure(c, q) == pytest.approx(1.0, abs=1e-15)
    for d in range(3):
        f = O.flux(c, q, d)
        want = np.zeros(5)
        want[1 + d] = 1.0
        np.testing.assert_allclose(f, want, atol=1e-15)


def test_flux_moving_state_hand_values():
    """rho = 2, (u, v, w) = (3, -1, 0.5), p = 4: by hand, rho E = p/0.4 + rho |u|^2 / 2
    = 10 + 10.25 = 20.25; F = (6, 22, -6, 3, 3 * 24.25), G = (-2, -6, 6, -1, -24.25)."""
    c = O.Cfg(dim=3, n=(4, 4, 4))
    q = np.array([2.0, 6.0, -2.0, 1.0, 20.25])
    assert O.pressure(c, q) == pytest.approx(4.0, rel=1e-14)
    np.testing.assert_allclose(O.flux(c, q, 0), [6.0, 22.0, -6.0, 3.0, 72.75], rtol=1e-14)
    np.testing.assert_allclose(O.flux(c, q, 1), [-2.0, -6.0, 6.0, -1.0, -24.25], rtol=1e-14)
    np.testing.assert_allclose(O.flux(c, q, 2), [1.0, 3.0, -1.0, 4.5, 12.125], rtol=1e-14)
    # |u| + a = sqrt(10.25) + sqrt(1.4 * 4 / 2)
    assert O.wavespeed(c, q) == pytest.approx(math.sqrt(10.25) + math.sqrt(2.8), rel=1e-14)


# ---------------------------------------------------------------- WENO5-JS
def _cell_averages(coeffs, centres, h):
    """Exact cell averages of the polynomial sum_k coeffs[k] x^k."""
    P = np.polynomial.Polynomial(coeffs).integ()
    return (P(centres + h / 2) - P(centres - h / 2)) / h


@pytest.mark.parametrize("eps", [1e-6, 1e-2, 1.0, 1e6])
def test_weno_exact_for_quadratic_cell_averages(eps):
    """Every candidate is exact for cell averages of a degree <= 2 polynomial, so
    the reconstruction at x_{i+1/2} is exact for any weights."""
    rng = np.random.default_rng(1)
    for _ in range(20):
        co = rng.normal(size=3)
        h = rng.uniform(0.01, 0.5)
        xc = np.arange(-2, 3) * h
        v = _cell_averages(co, xc, h)
        want = np.polynomial.Polynomial(co)(h / 2)
        np.testing.assert_allclose(O.weno5_candidates(v), [want] * 3, rtol=1e-12, atol=1e-12)
        assert O.weno5(v, eps) == pytest.approx(want, rel=1e-12, abs=1e-12)


def test_weno_linear_weights_exact_for_quartic_cell_averages():
    """With eps -> infinity the weights become d = (3/10, 3/5, 1/10) and the scheme is
    the fifth-order upwind reconstruction: exact for degree <= 4 cell averages."""
    rng = np.random.default_rng(2)
    for _ in range(20):
        co = rng.normal(size=5)
        h = rng.uniform(0.05, 0.5)
        xc = np.arange(-2, 3) * h
        v = _cell_averages(co, xc, h)
        want = np.polynomial.Polynomial(co)(h / 2)
        np.testing.assert_allclose(O.weno5_weights(v, 1e30), [0.3, 0.6, 0.1], rtol=1e-12)
        assert O.weno5(v, 1e30) == pytest.approx(want, rel=1e-11, abs=1e-11)


def test_beta_matches_jiang_shu_integral_definition():
    """beta_r = sum_{l=1,2} dx^(2l-1) int_cell (d^l p_r / dx^l)^2 dx, p_r the quadratic
    whose cell averages over S_r(i) equal v (computed here by polynomial algebra)."""
    rng = np.random.default_rng(3)
    h = 1.0
    for _ in range(20):
        v = rng.normal(size=5)  # cells i-2..i+2 centred at -2..2
        beta = O.weno5_beta(v)
        for r in range(3):
            cells = [-r, -r + 1, -r + 2]          # S_r(i) = {i-r, ..., i-r+2}
            A = np.zeros((3, 3))
            for row, c in enumerate(cells):
                for k in range(3):
                    mono = np.zeros(k + 1)
                    mono[k] = 1.0
                    A[row, k] = _cell_averages(mono, np.array([float(c)]), h)[0]
            co = np.linalg.solve(A, v[[c + 2 for c in cells]])
            p = np.polynomial.Polynomial(co)
            b = 0.0
            for l in (1, 2):
                dl = p.deriv(l)
                sq = (dl * dl).integ()
                b += h ** (2 * l - 1) * (sq(0.5) - sq(-0.5))
            assert beta[r] == pytest.approx(b, rel=1e-11, abs=1e-12)


def test_weights_linear_data_and_constant_data():
    """Linear data: all beta equal, omega = d exactly.  Constant data: beta = 0."""
    for eps in (1e-6, 1e-2):
        w = O.weno5_weights(np.array([1.0, 1.5, 2.0, 2.5, 3.0]), eps)
        np.testing.assert_allclose(w, [0.3, 0.6, 0.1], rtol=1e-14)
    np.testing.assert_allclose(O.weno5_beta(np.full(5, 7.25)), [0, 0, 0], atol=0)
    assert O.weno5(np.full(5, 7.25), 1e-6) == pytest.approx(7.25, rel=1e-15)


def test_weights_scale_with_inverse_square_of_beta_plus_eps():
    """alpha_r = d_r / (beta_r + eps)^2: with beta_0 = 0 and beta_1 = beta_2 > 0, the ratio
    omega_1 / omega_0 equals (d_1 / d_0) (eps / (beta_1 + eps))^2, i.e. slope 2 in eps."""
    # v chosen so that S_0 = {i, i+1, i+2} is constant and S_1, S_2 see a kink
    v = np.array([0.0, 0.0, 1.0, 1.0, 1.0])
    beta = O.weno5_beta(v)
    assert beta[0] == 0.0
    r = []
    for eps in (1e-8, 2e-8, 4e-8):
        w = O.weno5_weights(v, eps)
        r.append(w[1] / w[0])
        assert w[1] / w[0] == pytest.approx(2.0 * (eps / (beta[1] + eps)) ** 2, rel=1e-10)
    assert math.log(r[1] / r[0], 2) == pytest.approx(2.0, abs=1e-6)


def test_weno_eno_property_at_a_step():
    """At a step between i and i+1 the weights select the smooth stencil S_2."""
    v = np.array([0.0, 0.0, 0.0, 1.0, 1.0])
    w = O.weno5_weights(v, 1e-6)
    assert w[2] > 1 - 1e-10
    assert abs(O.weno5(v, 1e-6)) < 1e-10


# ----------------------------------------------------------------- residual
def test_free_stream_gives_zero_residual():
    for dim in (1, 2, 3):
        n = (12, 10, 8)[:dim]
        c = O.Cfg(dim=dim, n=n, bc=((O.TRANSMISSIVE, O.PERIODIC),) * 3)
        rho = np.full(c.shape[1:], 1.3)
        vel = [np.full(c.shape[1:], 0.7 - 0.2 * d) for d in range(dim)]
        U = I.conserved(dim, rho, vel, np.full(c.shape[1:], 2.1))
        R, _ = O.residual(c, U)
        assert np.abs(R).max() < 1e-12


def test_periodic_residual_telescopes():
    """sum_i R_i = 0: every interface flux enters two cells with opposite signs."""
    for dim, n in ((1, (64,)), (2, (24, 20)), (3, (12, 10, 8))):
        c = O.Cfg(dim=dim, n=n)
        U = I.random_state(dim, n, seed=5 + dim, jumps=True)
        R, _ = O.residual(c, U)
        scale = np.abs(R).max(axis=(1, 2, 3))
        s = R.sum(axis=(1, 2, 3))
        assert np.all(np.abs(s) <= 1e-13 * scale * R[0].size)


def test_mass_equation_is_the_scalar_scheme():
    """With u = 1 and p = 1 the continuity flux is rho, so the density component of the
    Euler residual equals the scalar LF-WENO5 residual of f(rho) = rho with the same alpha."""
    n = (48,)
    ce = O.Cfg(dim=1, n=n, lo=(0.0,), hi=(2.0,))
    U = I.density_wave(1, n)
    Re, a = O.residual(ce, U)
    cs = O.Cfg(dim=1, n=n, lo=(0.0,), hi=(2.0,), model=O.ADVECT)
    Rs = O.residual_dirs(cs, U[:1], a)
    np.testing.assert_allclose(Re[0], Rs[0], rtol=0, atol=1e-14)


def test_mirror_symmetry_pins_the_minus_reconstruction():
    """Reflecting x -> -x (rho u -> -rho u) must reflect the residual.  This holds only if
    the f(-) reconstruction is the mirror image of the f(+) one."""
    n = (40,)
    c = O.Cfg(dim=1, n=n)
    U = I.random_state(1, n, seed=11, jumps=True)
    M = U[:, :, :, ::-1].copy()
    M[1] *= -1
    R, _ = O.residual(c, U)
    Rm, _ = O.residual(c, M)
    Rm = Rm[:, :, :, ::-1]
    Rm[1] *= -1
    np.testing.assert_allclose(Rm, R, rtol=0, atol=1e-12 * np.abs(R).max())


def test_residual_is_fifth_order_for_smooth_data():
    """With linear weights the residual approximates -dF/dx at fifth order."""
    errs = []
    for N in (20, 40, 80):
        c = O.Cfg(dim=1, n=(N,), lo=(0.0,), hi=(2.0,), eps=1e30)
        U = I.density_wave(1, (N,))
        R, a = O.residual(c, U)
        x = c.centres(0)
        # -d(rho u)/dx with u = 1: -0.2 pi cos(pi x)
        errs.append(np.abs(R[0, 0, 0] + 0.2 * np.pi * np.cos(np.pi * x)).max())
    orders = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert orders[-1] > 4.8, orders


def test_2d_uniform_in_y_equals_1d():
    n1 = (32,)
    c1 = O.Cfg(dim=1, n=n1, bc=((O.TRANSMISSIVE, O.TRANSMISSIVE),))
    U1 = I.random_state(1, n1, seed=21, jumps=True)
    R1, _ = O.residual(c1, U1)
    ny = 6
    c2 = O.Cfg(dim=2, n=(32, ny), bc=((O.TRANSMISSIVE, O.TRANSMISSIVE), (O.PERIODIC, O.PERIODIC)))
    U2 = np.zeros(c2.shape)
    U2[0] = U1[0]
    U2[1] = U1[1]
    U2[3] = U1[2]
    R2, _ = O.residual(c2, U2)
    for j in range(ny):
        np.testing.assert_allclose(R2[0, 0, j], R1[0, 0, 0], atol=1e-13)
        np.testing.assert_allclose(R2[1, 0, j], R1[1, 0, 0], atol=1e-13)
        np.testing.assert_allclose(R2[3, 0, j], R1[2, 0, 0], atol=1e-13)
        assert np.abs(R2[2, 0, j]).max() < 1e-13


def test_quadrant_problem_transpose_symmetry():
    """The quadrant data are symmetric under (x, y, u, v) -> (y, x, v, u); so is R."""
    n = (32, 32)
    c = O.Cfg(dim=2, n=n, bc=((O.TRANSMISSIVE, O.TRANSMISSIVE),) * 3)
    U = I.quadrant_riemann(n)
    T = U[:, :, :, :].transpose(0, 1, 3, 2)[[0, 2, 1, 3]]
    np.testing.assert_array_equal(T, U)
    R, _ = O.residual(c, U)
    RT = R.transpose(0, 1, 3, 2)[[0, 2, 1, 3]]
    np.testing.assert_allclose(RT, R, rtol=0, atol=1e-13 * np.abs(R).max())


def test_reflective_wall_mirror_equals_doubled_periodic_domain():
    """A symmetry plane at x = 0 and x = L equals a periodic domain of length 2L whose
    right half is the mirror image (rho u negated) of the left half."""
    N = 24
    U = I.random_state(1, (N,), seed=31)
    cr = O.Cfg(dim=1, n=(N,), hi=(1.0,), bc=((O.REFLECTIVE, O.REFLECTIVE),))
    R, a = O.residual(cr, U)
    D = np.concatenate([U, U[:, :, :, ::-1]], axis=3)
    D[1, :, :, N:] *= -1
    cp = O.Cfg(dim=1, n=(2 * N,), hi=(2.0,))
    Rp = O.residual_dirs(cp, D, a)
    np.testing.assert_allclose(R, Rp[:, :, :, :N], rtol=0, atol=1e-13 * np.abs(R).max())


# ------------------------------------------------------------------ runs
def test_density_wave_converges_at_fifth_order():
    """1D advected density wave to t = 2 with dt = min(0.5 h / alpha, h^(5/3))."""
    errs = []
    Ns = (32, 64, 128, 256)
    for N in Ns:
        c = O.Cfg(dim=1, n=(N,), lo=(0.0,), hi=(2.0,))
        U, steps, t = O.run(c, I.density_wave(1, (N,)), 2.0, cfl=0.5, dt_coef=1.0)
        assert t == pytest.approx(2.0, abs=1e-14)
        ex = exact.density_wave_rho(c.centres(0), 2.0, 1)
        errs.append(np.abs(U[0, 0, 0] - ex).mean())
    orders = [math.log2(errs[k] / errs[k + 1]) for k in range(len(Ns) - 1)]
    assert orders[-1] >= 4.8, (errs, orders)


def test_periodic_run_conserves_mass_momentum_energy():
    n = (24, 20)
    c = O.Cfg(dim=2, n=n)
    U0 = I.random_state(2, n, seed=41, jumps=True)
    U, steps, t = O.run(c, U0, 0.05, cfl=0.5)
    s0, s1 = O.sums(c, U0), O.sums(c, U)
    scale = np.abs(U0).sum(axis=(1, 2, 3))
    assert np.all(np.abs(s1 - s0) <= 1e-13 * scale), (s1 - s0) / scale


def test_riemann_solver_satisfies_jump_conditions():
    """The exact solver's Sod star state satisfies Rankine-Hugoniot across the right
    shock and isentropy + Riemann invariant across the left rarefaction."""
    g = 1.4
    L, R = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    ps, us = exact.star_state(L, R, g)
    # right shock: mass and momentum flux continuity in the shock frame
    g1 = (g - 1) / (g + 1)
    rs = R[0] * (ps / R[2] + g1) / (g1 * ps / R[2] + 1)
    S = (rs * us - R[0] * R[1]) / (rs - R[0])
    assert rs * (us - S) == pytest.approx(R[0] * (R[1] - S), rel=1e-12)
    assert rs * (us - S) ** 2 + ps == pytest.approx(R[0] * (R[1] - S) ** 2 + R[2], rel=1e-12)
    E = lambda rho, u, p: p / (g - 1) + 0.5 * rho * u * u
    # energy: F_E(U*) - F_E(U_R) = S (E* - E_R), F_E = u (E + p)
    lhs = us * (E(rs, us, ps) + ps) - R[1] * (E(*R) + R[2])
    assert lhs == pytest.approx(S * (E(rs, us, ps) - E(*R)), rel=1e-10)
    # left rarefaction: p / rho^gamma and u + 2a/(gamma-1) constant
    rl = L[0] * (ps / L[2]) ** (1 / g)
    al, asl = math.sqrt(g * L[2] / L[0]), math.sqrt(g * ps / rl)
    assert L[1] + 2 * al / (g - 1) == pytest.approx(us + 2 * asl / (g - 1), rel=1e-12)
    # textbook values for Sod (Toro, Table 4.3): p* = 0.30313, u* = 0.92745
    assert ps == pytest.approx(0.30313, abs=5e-5)
    assert us == pytest.approx(0.92745, abs=5e-5)


def test_sod_shock_tube_against_exact_solution():
    """Sec. 5.5 set-up in 1D (T = 0.2, CFL 0.5, transmissive ends): L1 error falls with
    N, and the density stays within the initial bounds up to a small overshoot."""
    errs = []
    for N in (100, 200, 400):
        c = O.Cfg(dim=1, n=(N,), bc=((O.TRANSMISSIVE, O.TRANSMISSIVE),))
        U, steps, t = O.run(c, I.sod(1, (N,)), 0.2, cfl=0.5)
        x = c.centres(0)
        ex = exact.riemann_sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), (x - 0.5) / 0.2)
        errs.append(np.abs(U[0, 0, 0] - ex[0]).mean())
        assert U[0].max() < 1.0 * 1.02 and U[0].min() > 0.125 * 0.98
    assert errs[0] > errs[1] > errs[2]
    assert math.log2(errs[0] / errs[2]) / 2 > 0.6, errs


def _l2(err, h, dim):
    return math.sqrt(h ** dim * float((err ** 2).sum()))


@pytest.mark.parametrize("N,want", [(10, 1.47e-2), (20, 6.11e-4), (40, 1.88e-5)])
def test_table1_linear_advection(N, want):
    """Table 1 (Sec. 5.1), full-tensor column: u0 = sin(2 pi (x+y+z)) on [0,1]^3,
    periodic, dt = h^(5/3), T = 0.1, eps = dx^2, alpha = max|f'| = 1, cell-centred grid.
    The oracle reproduces the printed L2 errors to their three digits."""
    h = 1.0 / N
    c = O.Cfg(dim=3, n=(N, N, N), model=O.ADVECT, eps=h * h)
    U, steps, t = O.run(c, I.scalar_sine(3, (N, N, N)), 0.1, cfl=0.0, dt_coef=1.0)
    X = [c.centres(d) for d in range(3)]
    Z, Y, Xg = np.meshgrid(X[2], X[1], X[0], indexing="ij")
    ex = np.sin(2 * np.pi * (Xg + Y + Z - 3 * 0.1))
    e = _l2(U[0] - ex, h, 3)
    assert e == pytest.approx(want, rel=0.005), e


def _burgers_exact(s, T):
    u = 0.5 + 0.5 * np.sin(2 * np.pi * s)
    for _ in range(100):  # Newton on g(u) = u - u0(s - 3 u T), characteristics of u_t + 3 u u_s = 0
        arg = 2 * np.pi * (s - 3 * u * T)
        g = u - 0.5 - 0.5 * np.sin(arg)
        dg = 1 + 0.5 * np.cos(arg) * 2 * np.pi * 3 * T
        u = u - g / dg
    return u


@pytest.mark.parametrize("N,want", [(10, 6.90e-3), (20, 5.99e-4)])
def test_table2_burgers_reading(N, want):
    """Table 2 (Sec. 5.2), full-tensor column: u0 = 0.5 + 0.5 sin(2 pi (x+y+z)),
    T = 1/(12 pi), dt = h^(5/3), eps = dx^2.  The printed errors are reproduced within
    10% only when the LF constant sums the three directional speeds, alpha = 3 max|u|;
    with alpha = max|u| the errors come out 1.6-2.3x smaller.  This records that reading
    (the Euler path takes alpha = max(|u| + a), Sec. 4.3, which Table 1 does not test)."""
    h = 1.0 / N
    T = 1.0 / (12.0 * np.pi)
    c = O.Cfg(dim=3, n=(N, N, N), model=O.BURGERS, eps=h * h)
    X = [c.centres(d) for d in range(3)]
    Z, Y, Xg = np.meshgrid(X[2], X[1], X[0], indexing="ij")
    s = Xg + Y + Z
    U = I.scalar_sine(3, (N, N, N), offset=0.5, amp=0.5)
    t = 0.0
    L = lambda V: O.residual_dirs(c, V, 3.0 * np.abs(V).max())
    while t < T - 1e-15:
        dt = min(h ** (5.0 / 3.0), T - t)
        U1 = U + dt * L(U)
        U2 = 0.75 * U + 0.25 * (U1 + dt * L(U1))
        U = U / 3.0 + 2.0 / 3.0 * (U2 + dt * L(U2))
        t += dt
    e = _l2(U[0] - _burgers_exact(s, T), h, 3)
    assert e == pytest.approx(want, rel=0.10), e
    U1, _, _ = O.run(c, I.scalar_sine(3, (N, N, N), offset=0.5, amp=0.5), T, cfl=0.0, dt_coef=1.0)
    e1 = _l2(U1[0] - _burgers_exact(s, T), h, 3)
    assert 1.4 < want / e1 < 2.5, e1


# --------------------------------------------------------- TT pointwise path
def test_tt_full_matches_einsum_contraction():
    rng = np.random.default_rng(7)
    n, r = (5, 6, 4), (3, 2)
    cores = [rng.normal(size=(n[0], 1, r[0])).astype(np.float32),
             rng.normal(size=(n[1], r[0], r[1])).astype(np.float32),
             rng.normal(size=(n[2], r[1], 1)).astype(np.float32)]
    X = O.tt_full(n, r, cores)
    want = np.einsum("ia,jab,kb->kji", cores[0][:, 0, :].astype(np.float64),
                     cores[1].astype(np.float64), cores[2][:, :, 0].astype(np.float64))
    np.testing.assert_allclose(X, want, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("bc", [O.PERIODIC, O.TRANSMISSIVE, O.REFLECTIVE])
def test_cross_eval_equals_full_grid_residual(bc):
    """Pointwise evaluation from TT cores equals the full-grid residual of the FP64
    tensor built from the same cores, at the sampled fibers, for every sweep mode and
    flux direction."""
    inst = I.tt_instance(seed=3, n=[10, 12, 9], r=[3, 4], device="cpu")
    n, r, cores = inst["n"], inst["r"], inst["cores"]
    h = [1.0 / n[0], 1.0 / n[1], 1.0 / n[2]]
    bcs = ((bc, bc),) * 3
    cfg = O.Cfg(dim=3, n=tuple(n), hi=(1.0, 1.0, 1.0), bc=bcs)
    U = np.stack([O.tt_full(n, r, cores[f]) for f in range(5)])
    alpha = O.alpha_max(cfg, U) * 1.05
    for fd in range(3):
        Rf = O.residual_dirs(cfg, U, alpha, 1 << fd)
        for mode in range(3):
            left, right = I.cross_index_sets(100 + 3 * fd + mode, n, r, mode)
            out = O.cross_eval(n, r, cores, h, alpha, 1.4, 1e-6, bcs, mode, fd, left, right)
            for li in range(left.shape[0]):
                for ri in range(right.shape[0]):
                    for i in range(n[mode]):
                        ix = list(left[li]) + [i] + list(right[ri])
                        want = Rf[:, ix[2], ix[1], ix[0]]
                        got = out[:, li, i, ri]
                        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(Rf).max())


# ---------------------------------------------------------------- inflow
def _inflow_state(rho, u, p, dim, gamma=1.4):
    vel = [u] + [0.0] * (dim - 1)
    return [rho] + [rho * v for v in vel] + [p / (gamma - 1) + 0.5 * rho * sum(v * v for v in vel)]


def test_inflow_ghosts_equal_a_padded_domain():
    """An inflow side holds the given state in its three ghost layers: the residual
    equals that of a domain extended by three cells of that state (transmissive
    beyond them), restricted to the original cells."""
    N = 40
    U = I.random_state(1, (N,), seed=51, jumps=True)
    qin = _inflow_state(1.3, 0.4, 1.1, 1)
    cfg = O.Cfg(dim=1, n=(N,), bc=((O.INFLOW, O.TRANSMISSIVE),),
                bc_state=[[qin, [0] * 3], [[0] * 3] * 2, [[0] * 3] * 2])
    a = O.alpha(cfg, U)
    R = O.residual_dirs(cfg, U, a)
    pad = np.concatenate([np.array(qin)[:, None, None, None] * np.ones((3, 1, 1, 3)), U], axis=3)
    cp = O.Cfg(dim=1, n=(N + 3,), hi=((N + 3) / N,), bc=((O.TRANSMISSIVE, O.TRANSMISSIVE),))
    Rp = O.residual_dirs(cp, pad, a)
    np.testing.assert_allclose(R, Rp[:, :, :, 3:], rtol=0, atol=1e-13 * np.abs(R).max())


def test_inflow_of_the_interior_state_keeps_a_free_stream():
    n = (16, 12)
    qs = _inflow_state(1.2, 0.7, 0.9, 2)
    st = [[qs, qs], [qs, qs], [[0] * 4] * 2]
    cfg = O.Cfg(dim=2, n=n, bc=((O.INFLOW, O.INFLOW), (O.INFLOW, O.INFLOW)), bc_state=st)
    U = np.ascontiguousarray(np.broadcast_to(np.array(qs)[:, None, None, None], cfg.shape))
    R, _ = O.residual(cfg, U)
    assert np.abs(R).max() < 1e-12


# ------------------------------------------- boundary, alpha and dt branches
def _edge_pad(U, axis, k=3):
    """U with k copies of its first and last cell along `axis` (numpy axis of the
    [f][z][y][x] layout) prepended and appended, built by hand."""
    lo = np.take(U, [0], axis=axis)
    hi = np.take(U, [U.shape[axis] - 1], axis=axis)
    return np.concatenate([lo] * k + [U] + [hi] * k, axis=axis)


@pytest.mark.parametrize("dim", [1, 2])
def test_transmissive_ghosts_equal_a_padded_periodic_domain(dim):
    """A transmissive side copies its edge cell into all three ghost layers (the
    zero-order extrapolation read into Sec. 4.5's ghost fill).  The residual must
    equal that of the state padded by hand with three copies of each edge cell,
    on a periodic domain six cells wider per direction, restricted to the
    original cells: their stencils reach at most three cells beyond the edge, so
    the wrap-around of the padded domain never enters.  The state's edge cells
    differ from their neighbours, so a clamp to the second cell or a mirror fill
    changes the answer."""
    n = (40,) if dim == 1 else (28, 22)
    U = I.random_state(dim, n, seed=61, jumps=True)
    for d in range(dim):
        ax = 3 - d
        edge = np.take(U, [0, 1, 2], axis=ax)
        assert np.abs(np.diff(edge, axis=ax)).mean() > 1e-4
    cfg = O.Cfg(dim=dim, n=n, bc=((O.TRANSMISSIVE, O.TRANSMISSIVE),) * 3)
    a = O.alpha(cfg, U)
    R = O.residual_dirs(cfg, U, a)
    P = U
    for d in range(dim):
        P = _edge_pad(P, 3 - d)
    h = [cfg.spacing(d) for d in range(dim)]
    cp = O.Cfg(dim=dim, n=tuple(m + 6 for m in n), hi=tuple((m + 6) * hd for m, hd in zip(n, h)))
    Rp = O.residual_dirs(cp, np.ascontiguousarray(P), a)
    inner = Rp[..., 3:3 + n[0]] if dim == 1 else Rp[:, :, 3:3 + n[1], 3:3 + n[0]]
    np.testing.assert_allclose(R, inner, rtol=0, atol=1e-13 * np.abs(R).max())
    # the same state with a clamp to the second cell would not pass
    Q = U.copy()
    Q[..., 0] = Q[..., 1]
    assert np.abs(O.residual_dirs(cfg, Q, a) - R).max() > 1e-6 * np.abs(R).max()


def _speed_cells():
    """(rho, u, v, w, p) of three cells whose direction-wise speeds |u_d| + a peak
    in different cells, and a quiet cell (a = 1, at rest).  With gamma = 1.4:
      A: rho 1.4,  p 1, a = 1, u = (2, 0.5, -0.25)  -> |u_d| + a = (3, 1.5, 1.25)
      B: rho 0.35, p 1, a = 2, u = (0.5, -1.5, 0)   -> (2.5, 3.5, 2)
      C: rho 1.4,  p 1, a = 1, u = (0, 0.1, -3)     -> (1, 1.1, 4)
    so max_d = (3, 3.5, 4) by hand, and max(|u| + a) = 1 + sqrt(9.01) (cell C)."""
    return [(1.4, 2.0, 0.5, -0.25, 1.0), (0.35, 0.5, -1.5, 0.0, 1.0), (1.4, 0.0, 0.1, -3.0, 1.0)], \
        (1.4, 0.0, 0.0, 0.0, 1.0)


def _state_with_cells(n, cells, quiet):
    rho = np.full(n[::-1], quiet[0])
    vel = [np.full(n[::-1], quiet[1 + d]) for d in range(3)]
    p = np.full(n[::-1], quiet[4])
    spots = [(0, 0, 1), (1, 2, 0), (2, 1, 3)]  # (z, y, x) of A, B, C
    for (k, j, i), c in zip(spots, cells):
        rho[k, j, i] = c[0]
        for d in range(3):
            vel[d][k, j, i] = c[1 + d]
        p[k, j, i] = c[4]
    return I.conserved(3, rho, vel, p)


def test_per_direction_alpha_hand_values():
    """Eq. (lax-friedrichs) read per direction: alpha_d = max over cells of
    |u_d| + a.  Hand values (3, 3.5, 4) from three cells whose peaks sit in
    different cells and need the absolute value (B's v and C's w are negative);
    the global reading gives 1 + sqrt(9.01) in every direction."""
    cells, quiet = _speed_cells()
    n = (4, 3, 4)
    U = _state_with_cells(n, cells, quiet)
    cpd = O.Cfg(dim=3, n=n, alpha_mode=O.ALPHA_PER_DIR)
    np.testing.assert_allclose(O.alpha(cpd, U), [3.0, 3.5, 4.0], rtol=1e-15)
    cg = O.Cfg(dim=3, n=n)
    np.testing.assert_allclose(O.alpha(cg, U), [1.0 + math.sqrt(9.01)] * 3, rtol=1e-15)
    assert O.alpha_max(cpd, U) == pytest.approx(1.0 + math.sqrt(9.01), rel=1e-15)


def test_per_direction_alpha_routes_alpha_y_to_the_y_splitting():
    """A 2D state varying only in y with u = 0: in per-direction mode the y
    splitting must take alpha_y = max(|v| + a), which is the 1D alpha of the
    same profile along x, so the residual equals the 1D residual of (rho, rho v,
    rho E) (rho E is the same since u = 0).  alpha_x = max(a) is smaller, so
    handing it to the y direction would change the result."""
    ny = 36
    W = I.random_state(1, (ny,), seed=71, jumps=True)
    rho = W[0]
    v = W[1] / rho + 0.8
    U1 = I.conserved(1, rho, [v], 0.4 * (W[2] - 0.5 * W[1] ** 2 / rho))
    c1 = O.Cfg(dim=1, n=(ny,))
    R1, a1 = O.residual(c1, U1)
    nx = 4
    c2 = O.Cfg(dim=2, n=(nx, ny), alpha_mode=O.ALPHA_PER_DIR)
    U2 = np.zeros(c2.shape)
    for f_src, f_dst in ((0, 0), (1, 2), (2, 3)):
        U2[f_dst, 0] = U1[f_src, 0, 0][:, None]
    a2 = O.alpha(c2, U2)
    assert a2[1] == a1[0] and a2[0] < 0.8 * a2[1]
    R2, _ = O.residual(c2, U2)
    for i in range(nx):
        np.testing.assert_allclose(R2[0, 0, :, i], R1[0, 0, 0], rtol=0, atol=1e-13 * np.abs(R1).max())
        np.testing.assert_allclose(R2[2, 0, :, i], R1[1, 0, 0], rtol=0, atol=1e-13 * np.abs(R1).max())
        np.testing.assert_allclose(R2[3, 0, :, i], R1[2, 0, 0], rtol=0, atol=1e-13 * np.abs(R1).max())
        assert np.abs(R2[1, 0, :, i]).max() < 1e-13 * np.abs(R1).max()


def test_cfl_dt_hand_value_on_an_anisotropic_grid():
    """Eq. (cfl-other): dt = lambda h / max(|u| + a) with h the smallest spacing.
    Grid spacings (0.25, 0.125, 0.5): h = 0.125 is the y spacing, so neither the
    first nor the largest spacing passes; max(|u| + a) = 1 + sqrt(9.01) from
    cell C (the per-direction maximum 4 would not pass either)."""
    cells, quiet = _speed_cells()
    n = (4, 4, 4)
    U = _state_with_cells(n, cells, quiet)
    cfg = O.Cfg(dim=3, n=n, hi=(1.0, 0.5, 2.0))
    want = 0.4 * 0.125 / (1.0 + math.sqrt(9.01))
    assert O.cfl_dt(cfg, U, 0.4) == pytest.approx(want, rel=1e-15)
    # the run takes that dt for its first step
    _, steps, t = O.run(cfg, U, 1.0, cfl=0.4, max_steps=1)
    assert steps == 1 and t == pytest.approx(want, rel=1e-15)
    # convergence-study rule: dt = min(CFL dt, c h^(5/3)), (1/8)^(5/3) = 1/32
    _, steps, t = O.run(cfg, U, 1.0, cfl=0.4, dt_coef=0.01, max_steps=1)
    assert steps == 1 and t == pytest.approx(0.01 / 32.0, rel=1e-14)
    # the last step is shortened to land on t_end exactly
    _, steps, t = O.run(cfg, U, 1.5 * want, cfl=0.4)
    assert steps == 2 and t == 1.5 * want
