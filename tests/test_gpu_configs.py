"""The workloads end to end on the GPU: whole runs against the oracle, L1
errors against the exact solution, and measured convergence orders, in FP64
and FP32-bulk.  GPU only; each test prints the numbers it checks.

Convergence runs take dt = min(0.5 h / alpha, h^(5/3)) (alpha of the initial
state, constant for the advected wave), the paper's practice for order
studies (Sec. 5.1); the CFL-0.5 run is checked separately."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import exact
from paper_2405_12301_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_12301_gb300 import build, weno
    build.build()
    weno.lib()
    return weno


def gpu_run(W, cfg, U0, t_end, precision, dt=0.0, graph_steps=32):
    s = W.Solver(cfg.dim, cfg.n[:cfg.dim], cfg.lo[:cfg.dim], cfg.hi[:cfg.dim], gamma=cfg.gamma, eps_weno=cfg.eps,
                 cfl=0.5, bc=cfg.bc, precision=precision)
    Ud = torch.from_numpy(np.ascontiguousarray(U0)).cuda()
    s.set_time(0.0)
    steps = s.run(Ud, t_end, dt=dt, graph_steps=graph_steps)
    t, _ = s.time()
    out = Ud.cpu().numpy()
    s.close()
    assert t == t_end
    return out, steps


def rel_field_err(a, b):
    err = 0.0
    for f in range(b.shape[0]):
        scale = np.maximum(np.abs(b[f]), np.abs(b[f]).max())
        err = max(err, float((np.abs(a[f] - b[f]) / scale).max()))
    return err


def wave_dt(dim, N):
    h = 2.0 / N
    alpha = dim ** 0.5 + math.sqrt(1.4 / 0.8)  # |u| + max a of the wave (rho >= 0.8, p = 1)
    return min(0.5 * h / alpha, h ** (5.0 / 3.0))


def test_1d_wave_n256_cfl05_run_matches_oracle(W):
    """Config 1: N = 256, CFL 0.5 to t = 2, FP64: the GPU run equals the oracle's."""
    cfg = O.Cfg(dim=1, n=(256,), lo=(0.0,), hi=(2.0,))
    U0 = I.density_wave(1, (256,))
    Uref, steps, _ = O.run(cfg, U0, 2.0, cfl=0.5)
    Ug, gsteps = gpu_run(W, cfg, U0, 2.0, W.FP64)
    assert gsteps == steps
    assert rel_field_err(Ug, Uref) <= 1e-10
    l1 = np.abs(Ug[0, 0, 0] - exact.density_wave_rho(cfg.centres(0), 2.0, 1)).mean()
    print("1D N=256 CFL 0.5: L1(rho) = %.3e after %d steps" % (l1, steps))


def test_1d_convergence_sweep_fifth_order(W):
    """Config 1: N = 32..512; the order over the finest pairs is at least 4.8."""
    errs = []
    Ns = (32, 64, 128, 256, 512)
    for N in Ns:
        cfg = O.Cfg(dim=1, n=(N,), lo=(0.0,), hi=(2.0,))
        Ug, _ = gpu_run(W, cfg, I.density_wave(1, (N,)), 2.0, W.FP64, dt=wave_dt(1, N))
        errs.append(np.abs(Ug[0, 0, 0] - exact.density_wave_rho(cfg.centres(0), 2.0, 1)).mean())
    orders = [math.log2(errs[k] / errs[k + 1]) for k in range(len(Ns) - 1)]
    print("1D L1:", ["%.3e" % e for e in errs], "orders:", ["%.2f" % o for o in orders])
    assert min(orders[-2:]) >= 4.8


def test_2d_wave_fp64_and_fp32_bulk_orders(W):
    """Config 2: 2D density wave on [0,2)^2 to t = 2, 64^2..512^2, FP64 and FP32-bulk:
    L1 errors, orders, and the FP32-bulk gate (within 1.1x of FP64 wherever FP64 is
    at least 10x the FP32 floor)."""
    rows = []
    for N in (64, 128, 256, 512):
        cfg = O.Cfg(dim=2, n=(N, N), lo=(0.0, 0.0), hi=(2.0, 2.0))
        U0 = I.density_wave(2, (N, N))
        ex = I.density_wave(2, (N, N), t=2.0)[0]
        u64, _ = gpu_run(W, cfg, U0, 2.0, W.FP64, dt=wave_dt(2, N))
        u32, _ = gpu_run(W, cfg, U0, 2.0, W.FP32_BULK, dt=wave_dt(2, N))
        e64 = np.abs(u64[0] - ex).mean()
        e32 = np.abs(u32[0] - ex).mean()
        floor = np.abs(u32[0] - u64[0]).mean()
        rows.append((N, e64, e32, floor))
        if e64 >= 10 * floor:
            assert e32 <= 1.1 * e64, (N, e64, e32, floor)
    for k in range(len(rows) - 1):
        print("2D N=%d: L1 fp64 %.3e fp32-bulk %.3e floor %.3e, order fp64 %.2f" % (
            rows[k][0], rows[k][1], rows[k][2], rows[k][3], math.log2(rows[k][1] / rows[k + 1][1])))
    print("2D N=%d: L1 fp64 %.3e fp32-bulk %.3e floor %.3e" % rows[-1])
    orders = [math.log2(rows[k][1] / rows[k + 1][1]) for k in range(len(rows) - 1)]
    assert orders[-1] >= 4.8


def test_2d_wave_1024_cfl05_fp64_and_fp32_bulk(W):
    """Config 2 at 1024^2 with the CFL-0.5 step to t = 2 (the h^(5/3) rule would take
    ~66k steps here): FP64 and FP32-bulk take the same number of steps, and the
    FP32-bulk L1 error is within 1.1x of FP64 plus the floor (the L1 distance of
    the two runs), both printed."""
    N = 1024
    cfg = O.Cfg(dim=2, n=(N, N), lo=(0.0, 0.0), hi=(2.0, 2.0))
    U0 = I.density_wave(2, (N, N))
    ex = I.density_wave(2, (N, N), t=2.0)[0]
    u64, s64 = gpu_run(W, cfg, U0, 2.0, W.FP64)
    u32, s32 = gpu_run(W, cfg, U0, 2.0, W.FP32_BULK)
    e64 = np.abs(u64[0] - ex).mean()
    e32 = np.abs(u32[0] - ex).mean()
    floor = np.abs(u32[0] - u64[0]).mean()
    print("2D N=1024 CFL 0.5: %d steps; L1 fp64 %.3e fp32-bulk %.3e floor %.3e" % (s64, e64, e32, floor))
    assert s32 == s64
    assert e32 <= 1.1 * e64 + floor


def test_fp32_bulk_and_fp64_runs_take_the_same_steps(W):
    """Both precisions take dt = lambda h / alpha from their own state's alpha
    (FP32-bulk forms the wavespeeds in FP32, the max and dt in FP64); the two
    alphas differ at the FP32 rounding level, so the step sequences to t = 2
    have the same length and both land on t_end."""
    for N in (64, 256):
        cfg = O.Cfg(dim=2, n=(N, N), lo=(0.0, 0.0), hi=(2.0, 2.0))
        U0 = I.density_wave(2, (N, N))
        _, s64 = gpu_run(W, cfg, U0, 2.0, W.FP64)
        _, s32 = gpu_run(W, cfg, U0, 2.0, W.FP32_BULK)
        _, sref, _ = O.run(cfg, U0, 2.0, cfl=0.5) if N == 64 else (None, s64, None)
        print("N=%d: steps fp64 %d, fp32-bulk %d, oracle %d" % (N, s64, s32, sref))
        assert s32 == s64 == sref


def test_2d_quadrant_256_run_matches_oracle(W):
    """Config 3 at the oracle's size: 256^2, transmissive, to t = 0.3, FP64 equals
    the oracle to 1e-10; FP32-bulk stays within a bounded distance of FP64, and the
    conservation sums are reported."""
    n = (256, 256)
    T = O.TRANSMISSIVE
    cfg = O.Cfg(dim=2, n=n, bc=((T, T), (T, T)))
    U0 = I.quadrant_riemann(n)
    Uref, steps, _ = O.run(cfg, U0, 0.3, cfl=0.5)
    u64, gsteps = gpu_run(W, cfg, U0, 0.3, W.FP64)
    assert gsteps == steps
    assert rel_field_err(u64, Uref) <= 1e-10
    u32, _ = gpu_run(W, cfg, U0, 0.3, W.FP32_BULK)
    d = np.abs(u32[0] - u64[0]).mean() / np.abs(u64[0]).mean()
    print("quadrant 256^2: %d steps; FP32-bulk vs FP64 L1(rho)/mean = %.2e; sums0 %s sums_fp64 %s" % (
        steps, d, np.round(O.sums(cfg, U0), 6), np.round(O.sums(cfg, u64), 6)))
    assert d < 1e-4


def test_3d_wave_to_half_time(W):
    """Config 4: 3D density wave on [0,2)^3 to t = 0.5 with CUDA-graph-captured steps:
    FP64 at 32^3 equals the oracle to 1e-10; FP32-bulk at 256^3 reaches the
    accuracy of the scheme (L1 of rho against the exact wave)."""
    n = (32, 32, 32)
    cfg = O.Cfg(dim=3, n=n, lo=(0, 0, 0), hi=(2.0, 2.0, 2.0))
    U0 = I.density_wave(3, n)
    Uref, steps, _ = O.run(cfg, U0, 0.5, cfl=0.5)
    u64, gsteps = gpu_run(W, cfg, U0, 0.5, W.FP64)
    assert gsteps == steps
    assert rel_field_err(u64, Uref) <= 1e-10
    N = 256
    n = (N, N, N)
    cfg = O.Cfg(dim=3, n=n, lo=(0, 0, 0), hi=(2.0, 2.0, 2.0))
    u32, st = gpu_run(W, cfg, I.density_wave(3, n), 0.5, W.FP32_BULK)
    ex = I.density_wave(3, n, t=0.5)[0]
    l1 = np.abs(u32[0] - ex).mean()
    print("3D 256^3 FP32-bulk to t=0.5: %d steps, L1(rho) = %.3e" % (st, l1))
    assert l1 < 1e-6


def test_3d_384_cube_run_to_half_time(W):
    """Config 4 at 384^3: FP32-bulk, CUDA-graph-captured steps to t = 0.5; the L1
    error of rho against the exact wave is the scheme's (below the 256^3 run's)."""
    N = 384
    n = (N, N, N)
    cfg = O.Cfg(dim=3, n=n, lo=(0, 0, 0), hi=(2.0, 2.0, 2.0))
    u32, st = gpu_run(W, cfg, I.density_wave(3, n), 0.5, W.FP32_BULK)
    ex = I.density_wave(3, n, t=0.5)[0]
    l1 = np.abs(u32[0] - ex).mean()
    print("3D 384^3 FP32-bulk to t=0.5: %d steps, L1(rho) = %.3e" % (st, l1))
    assert l1 < 1e-6


def test_2d_quadrant_1024_and_2048_runs(W):
    """Config 3 at its own sizes: 1024^2 in FP64 and FP32-bulk and 2048^2 in
    FP32-bulk, transmissive, to t = 0.3.  Transmissive sides let mass in where the
    corner states move inwards (SW, NW, SE), so the physical mass M = sum(rho) h^2
    grows; checked: FP32-bulk and FP64 give the same M and a close state, M at
    2048^2 agrees with 1024^2, and |M - M0| stays under t x perimeter x max |rho u|."""
    T = O.TRANSMISSIVE
    masses = {}
    for N in (1024, 2048):
        n = (N, N)
        h2 = (1.0 / N) ** 2
        cfg = O.Cfg(dim=2, n=n, bc=((T, T), (T, T)))
        U0 = I.quadrant_riemann(n)
        M0 = O.sums(cfg, U0)[0] * h2
        u32, st32 = gpu_run(W, cfg, U0, 0.3, W.FP32_BULK)
        assert np.isfinite(u32).all() and u32[0].min() > 0
        M32 = O.sums(cfg, u32)[0] * h2
        masses[N] = M32
        line = "quadrant %d^2: %d steps FP32-bulk; M %.6f -> %.6f" % (N, st32, M0, M32)
        if N == 1024:
            u64, st64 = gpu_run(W, cfg, U0, 0.3, W.FP64)
            M64 = O.sums(cfg, u64)[0] * h2
            d = np.abs(u32[0] - u64[0]).mean() / np.abs(u64[0]).mean()
            line += "; FP64 %d steps, M %.9f; FP32-bulk vs FP64 L1(rho)/mean = %.2e" % (st64, M64, d)
            assert d < 1e-4
            assert abs(M32 - M64) <= 1e-6 * M64
        print(line)
        rho_u_max = max(0.5323 * 1.206, 0.138 * 1.206 * 2 ** 0.5)
        assert abs(M32 - M0) <= 0.3 * 4.0 * rho_u_max
    assert abs(masses[2048] - masses[1024]) <= 1e-2 * masses[1024]
