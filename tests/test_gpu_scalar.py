"""The scalar conservation laws on the GPU (linear advection, Sec. 5.1, and
Burgers' equation, Sec. 5.2) through the C ABI, against the FP64 oracle, plus
the paper's Table 1 full-tensor errors reproduced by GPU runs.  GPU only.

Tolerance of the residual: |a - b| <= 1e-12 max(|b|, |b|_inf) + 1e-13 S / h with
S = alpha |u|_inf + |f(u)|_inf, the bound of the split fluxes (the same
derivation as for the Euler residual: equal WENO sums in a different
expression tree differ by a few ulp of S per interface)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2405_12301_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

P, T, R, IN = O.PERIODIC, O.TRANSMISSIVE, O.REFLECTIVE, O.INFLOW


@pytest.fixture(scope="module")
def W():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_12301_gb300 import build, weno
    build.build()
    weno.lib()
    return weno


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def solver(W, cfg):
    return W.Solver(cfg.dim, cfg.n[:cfg.dim], cfg.lo[:cfg.dim], cfg.hi[:cfg.dim], eps_weno=cfg.eps, cfl=0.5,
                    bc=cfg.bc, bc_state=cfg.bc_state, model=cfg.model)


def scalar_state(dim, n, seed):
    """A seeded field of both signs with planar jumps: the x momentum of a random gas state."""
    return np.ascontiguousarray(I.random_state(dim, n, seed=seed, jumps=True)[1:2])


def rhs_tol(cfg, U, Rref, alpha):
    f = np.abs(U) if cfg.model == O.ADVECT else 0.5 * U * U
    S = alpha * np.abs(U).max() + f.max()
    hmin = min(cfg.spacing(d) for d in range(cfg.dim))
    return 1e-12 * np.maximum(np.abs(Rref), np.abs(Rref).max()) + 1e-13 * S / hmin


def rel_err(a, b):
    return float((np.abs(a - b) / np.maximum(np.abs(b), np.abs(b).max())).max())


CASES = [
    (1, (203,), ((P, P),)),
    (1, (130,), ((R, IN),)),
    (2, (67, 41), ((P, T), (R, P))),
    (2, (40, 129), ((IN, T), (P, P))),
    (3, (35, 29, 30), ((P, P), (T, R), (P, IN))),
]


@pytest.mark.parametrize("model", ["advect", "burgers"])
@pytest.mark.parametrize("dim,n,bc", CASES)
def test_scalar_rhs_step_run_match_oracle(W, model, dim, n, bc):
    m = O.ADVECT if model == "advect" else O.BURGERS
    st = [[[0.7], [-0.4]], [[0.3], [0.9]], [[-0.6], [0.5]]]
    cfg = O.Cfg(dim=dim, n=n, bc=bc, model=m, bc_state=st)
    U = scalar_state(dim, n, seed=900 + sum(n) + m)
    Rref, aref = O.residual(cfg, U)
    s = solver(W, cfg)
    assert s.nf == 1
    Rd = torch.empty(U.shape, dtype=torch.float64, device="cuda")
    s.rhs(dev(U), Rd)
    Rg = host(Rd)
    tol = rhs_tol(cfg, U, Rref, aref[0])
    assert (np.abs(Rg - Rref) <= tol).all(), float((np.abs(Rg - Rref) / tol).max())
    # one step with the CFL dt, then a run of several steps (graph-captured chunks)
    Ud = dev(U)
    s.set_time(0.0)
    s.step(Ud)
    dt = O.cfl_dt(cfg, U, 0.5)
    assert rel_err(host(Ud), O.ssprk3_step(cfg, U, dt)) <= 1e-12
    Uref, steps, _ = O.run(cfg, U, 0.05, cfl=0.5)
    Ud = dev(U)
    s.set_time(0.0)
    assert s.run(Ud, 0.05, graph_steps=4) == steps
    assert rel_err(host(Ud), Uref) <= 1e-10
    s.close()


def test_scalar_models_conserve_the_sum_on_periodic_grids(W):
    n = (48, 40, 36)
    for m in (O.ADVECT, O.BURGERS):
        cfg = O.Cfg(dim=3, n=n, model=m)
        U = scalar_state(3, n, seed=77 + m)
        s = solver(W, cfg)
        Ud = dev(U)
        s0 = s.sums(Ud)[0]
        s.set_time(0.0)
        s.run(Ud, 0.1, graph_steps=8)
        s1 = s.sums(Ud)[0]
        assert abs(s1 - s0) <= 1e-12 * np.abs(U).sum(), (m, s0, s1)
        s.close()


def _l2(err, h, dim):
    return math.sqrt(h ** dim * float((err ** 2).sum()))


@pytest.mark.parametrize("N,want", [(10, 1.47e-2), (20, 6.11e-4), (40, 1.88e-5)])
def test_table1_linear_advection_on_the_gpu(W, N, want):
    """Table 1 (Sec. 5.1), full-tensor column, run on the GPU: u0 = sin(2 pi (x+y+z))
    on [0,1]^3, periodic, dt = h^(5/3), T = 0.1, eps = dx^2.  The GPU run equals the
    oracle's and its L2 error matches the printed value to its three digits."""
    h = 1.0 / N
    cfg = O.Cfg(dim=3, n=(N, N, N), model=O.ADVECT, eps=h * h)
    U0 = I.scalar_sine(3, (N, N, N))
    Uref, steps, _ = O.run(cfg, U0, 0.1, cfl=0.0, dt_coef=1.0)
    s = solver(W, cfg)
    Ud = dev(U0)
    s.set_time(0.0)
    assert s.run(Ud, 0.1, dt=h ** (5.0 / 3.0), graph_steps=16) == steps
    assert s.time()[0] == 0.1
    Ug = host(Ud)
    assert rel_err(Ug, Uref) <= 1e-10
    X = [cfg.centres(d) for d in range(3)]
    Z, Y, Xg = np.meshgrid(X[2], X[1], X[0], indexing="ij")
    e = _l2(Ug[0] - np.sin(2 * np.pi * (Xg + Y + Z - 3 * 0.1)), h, 3)
    print("Table 1 on the GPU: N=%d L2 = %.3e (printed %.2e), %d steps" % (N, e, want, steps))
    assert e == pytest.approx(want, rel=0.005), e


def test_burgers_run_matches_oracle_to_the_paper_time(W):
    """Sec. 5.2 set-up at 40^3: u0 = 0.5 + 0.5 sin(2 pi (x+y+z)), T = 1/(12 pi),
    dt = h^(5/3), eps = dx^2, alpha = max |u|: the GPU run equals the oracle's."""
    N = 40
    h = 1.0 / N
    T_end = 1.0 / (12.0 * math.pi)
    cfg = O.Cfg(dim=3, n=(N, N, N), model=O.BURGERS, eps=h * h)
    U0 = I.scalar_sine(3, (N, N, N), offset=0.5, amp=0.5)
    Uref, steps, _ = O.run(cfg, U0, T_end, cfl=0.0, dt_coef=1.0)
    s = solver(W, cfg)
    Ud = dev(U0)
    s.set_time(0.0)
    assert s.run(Ud, T_end, dt=h ** (5.0 / 3.0), graph_steps=16) == steps
    assert rel_err(host(Ud), Uref) <= 1e-10


def test_scalar_models_refuse_fp32_bulk(W):
    with pytest.raises(W.WenoError) as e:
        W.Solver(2, (16, 16), model=W.MODEL_ADVECT, precision=W.FP32_BULK)
    assert e.value.code == W.ERR_UNSUPPORTED
