"""The oracle: plain FP64 CPU implementation of the WENO5-JS / Lax-Friedrichs /
SSP-RK3 scheme for the compressible Euler equations (Danis et al., Sec. 2 and
Sec. 4), plus exact solutions used to pin it.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg may import this package; the CUDA path never does, and the
two share no code.  Inputs come from ``paper_2405_12301_gb300.inputs``, which
holds none of the scheme's arithmetic.

Every array is numpy FP64 in the layout [field][k][j][i] (x fastest).
"""
import ctypes as C
import dataclasses

import numpy as np

from . import build as _build

_lib = None

EULER, ADVECT, BURGERS = 0, 1, 2
PERIODIC, TRANSMISSIVE, REFLECTIVE, INFLOW = 0, 1, 2, 3
ALPHA_GLOBAL_NORM, ALPHA_PER_DIR = 0, 1


class _OCfg(C.Structure):
    _fields_ = [("dim", C.c_int), ("model", C.c_int), ("n", C.c_int * 3),
                ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("gamma", C.c_double), ("eps", C.c_double),
                ("bc", (C.c_int * 2) * 3), ("alpha_mode", C.c_int),
                ("bc_state", ((C.c_double * 5) * 2) * 3)]


@dataclasses.dataclass
class Cfg:
    """Problem description: grid, gas, WENO epsilon, boundary rules."""
    dim: int
    n: tuple
    lo: tuple = (0.0, 0.0, 0.0)
    hi: tuple = (1.0, 1.0, 1.0)
    gamma: float = 1.4
    eps: float = 1e-6
    bc: tuple = ((PERIODIC, PERIODIC),) * 3
    alpha_mode: int = ALPHA_GLOBAL_NORM
    model: int = EULER
    bc_state: object = None   # [3][2][nf] conserved inflow states (INFLOW sides)

    @property
    def nf(self):
        return self.dim + 2 if self.model == EULER else 1

    @property
    def shape(self):
        n = list(self.n) + [1] * (3 - len(self.n))
        return (self.nf, n[2], n[1], n[0])

    def spacing(self, d):
        return (self.hi[d] - self.lo[d]) / self.n[d]

    def centres(self, d):
        return self.lo[d] + (np.arange(self.n[d]) + 0.5) * self.spacing(d)

    def _c(self):
        c = _OCfg()
        c.dim, c.model = self.dim, self.model
        n = list(self.n) + [1] * (3 - len(self.n))
        for d in range(3):
            c.n[d] = int(n[d])
            c.lo[d] = float(self.lo[d]) if d < len(self.lo) else 0.0
            c.hi[d] = float(self.hi[d]) if d < len(self.hi) else 1.0
            c.bc[d][0], c.bc[d][1] = self.bc[d] if d < len(self.bc) else (PERIODIC, PERIODIC)
        c.gamma, c.eps, c.alpha_mode = self.gamma, self.eps, self.alpha_mode
        if self.bc_state is not None:
            for d in range(3):
                for side in range(2):
                    for f, v in enumerate(self.bc_state[d][side]):
                        c.bc_state[d][side][f] = float(v)
        return c


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(_build.build())
        P = C.POINTER
        d = C.c_double
        L.o_pressure.restype = d
        L.o_pressure.argtypes = [P(_OCfg), P(d)]
        L.o_flux.argtypes = [P(_OCfg), P(d), C.c_int, P(d)]
        L.o_wavespeed.restype = d
        L.o_wavespeed.argtypes = [P(_OCfg), P(d), C.c_int]
        L.o_weno5.restype = d
        L.o_weno5.argtypes = [P(d), d]
        L.o_weno5_beta.argtypes = [P(d), P(d)]
        L.o_weno5_weights.argtypes = [P(d), d, P(d)]
        L.o_weno5_candidates.argtypes = [P(d), P(d)]
        L.o_alpha.argtypes = [P(_OCfg), P(d), P(d)]
        L.o_alpha_max.restype = d
        L.o_alpha_max.argtypes = [P(_OCfg), P(d)]
        L.o_residual_dirs.argtypes = [P(_OCfg), P(d), P(d), C.c_int, P(d)]
        L.o_residual.argtypes = [P(_OCfg), P(d), P(d), P(d)]
        L.o_ssprk3_step.argtypes = [P(_OCfg), P(d), d]
        L.o_cfl_dt.restype = d
        L.o_cfl_dt.argtypes = [P(_OCfg), P(d), d]
        L.o_run.restype = C.c_int64
        L.o_run.argtypes = [P(_OCfg), P(d), d, d, d, d, d, C.c_int64, P(d)]
        L.o_sums.argtypes = [P(_OCfg), P(d), P(d)]
        L.o_cross_eval.argtypes = [P(C.c_int), P(C.c_int), P(C.c_void_p), P(d), d, d, d, P(C.c_int),
                                   C.c_int, C.c_int, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p, P(d)]
        L.o_tt_full.argtypes = [P(C.c_int), P(C.c_int), P(C.c_void_p), P(d)]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _state(cfg, U):
    U = np.ascontiguousarray(U, dtype=np.float64)
    assert U.shape == cfg.shape, (U.shape, cfg.shape)
    return U


# ------------------------------------------------------------------ physics
def pressure(cfg, q):
    q = np.ascontiguousarray(q, dtype=np.float64)
    return lib().o_pressure(C.byref(cfg._c()), _dp(q))


def flux(cfg, q, d):
    q = np.ascontiguousarray(q, dtype=np.float64)
    f = np.zeros(cfg.nf)
    lib().o_flux(C.byref(cfg._c()), _dp(q), d, _dp(f))
    return f


def wavespeed(cfg, q, d=-1):
    q = np.ascontiguousarray(q, dtype=np.float64)
    return lib().o_wavespeed(C.byref(cfg._c()), _dp(q), d)


# --------------------------------------------------------------------- WENO
def weno5(v, eps):
    """WENO5-JS value at x_{i+1/2} from v = (v_{i-2}, ..., v_{i+2})."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    return lib().o_weno5(_dp(v), eps)


def weno5_beta(v):
    v = np.ascontiguousarray(v, dtype=np.float64)
    b = np.zeros(3)
    lib().o_weno5_beta(_dp(v), _dp(b))
    return b


def weno5_weights(v, eps):
    v = np.ascontiguousarray(v, dtype=np.float64)
    w = np.zeros(3)
    lib().o_weno5_weights(_dp(v), eps, _dp(w))
    return w


def weno5_candidates(v):
    v = np.ascontiguousarray(v, dtype=np.float64)
    p = np.zeros(3)
    lib().o_weno5_candidates(_dp(v), _dp(p))
    return p


# ----------------------------------------------------------------- residual
def alpha(cfg, U):
    U = _state(cfg, U)
    a = np.zeros(3)
    lib().o_alpha(C.byref(cfg._c()), _dp(U), _dp(a))
    return a


def alpha_max(cfg, U):
    U = _state(cfg, U)
    return lib().o_alpha_max(C.byref(cfg._c()), _dp(U))


def residual(cfg, U):
    """L(U) and the alpha (3 values) used for its splitting."""
    U = _state(cfg, U)
    R = np.zeros_like(U)
    a = np.zeros(3)
    lib().o_residual(C.byref(cfg._c()), _dp(U), _dp(R), _dp(a))
    return R, a


def residual_dirs(cfg, U, alpha3, dirmask=7):
    """Contribution of the directions in dirmask with given alpha per direction."""
    U = _state(cfg, U)
    R = np.zeros_like(U)
    a = np.ascontiguousarray(np.broadcast_to(np.asarray(alpha3, dtype=np.float64), (3,)))
    lib().o_residual_dirs(C.byref(cfg._c()), _dp(U), _dp(a), dirmask, _dp(R))
    return R


def ssprk3_step(cfg, U, dt):
    U = _state(cfg, U).copy()
    lib().o_ssprk3_step(C.byref(cfg._c()), _dp(U), dt)
    return U


def cfl_dt(cfg, U, cfl):
    U = _state(cfg, U)
    return lib().o_cfl_dt(C.byref(cfg._c()), _dp(U), cfl)


def run(cfg, U, t_end, cfl=0.5, dt_coef=0.0, dt_pow=5.0 / 3.0, t0=0.0, max_steps=1 << 62):
    """Advance to t_end; returns (U, steps, t)."""
    U = _state(cfg, U).copy()
    t = C.c_double(0.0)
    steps = lib().o_run(C.byref(cfg._c()), _dp(U), t0, t_end, cfl, dt_coef, dt_pow, max_steps, C.byref(t))
    return U, int(steps), t.value


def sums(cfg, U):
    U = _state(cfg, U)
    s = np.zeros(cfg.nf)
    lib().o_sums(C.byref(cfg._c()), _dp(U), _dp(s))
    return s


# -------------------------------------------------------- TT pointwise path
def _core_ptrs(cores):
    """cores[f][m]: float32 arrays [n_m, r_{m-1}, r_m]; returns 15 pointers."""
    keep = []
    ptrs = (C.c_void_p * (3 * len(cores)))()
    for f, fc in enumerate(cores):
        for m in range(3):
            a = np.ascontiguousarray(fc[m], dtype=np.float32)
            keep.append(a)
            ptrs[f * 3 + m] = a.ctypes.data
    return ptrs, keep


def cross_eval(n, r, cores, h, alpha, gamma, eps, bc, mode, fd, left, right):
    """Direction-fd residual contribution at the samples (left x n[mode] x right)."""
    n_ = (C.c_int * 3)(*n)
    r_ = (C.c_int * 2)(*r)
    ptrs, keep = _core_ptrs(cores)
    h_ = (C.c_double * 3)(*h)
    bc_ = (C.c_int * 6)(*[int(b) for pair in bc for b in pair])
    left = np.ascontiguousarray(left, dtype=np.int32).reshape(-1, mode) if mode > 0 else np.zeros((1, 0), np.int32)
    right = np.ascontiguousarray(right, dtype=np.int32).reshape(-1, 2 - mode) if mode < 2 else np.zeros((1, 0), np.int32)
    nl, nr = left.shape[0], right.shape[0]
    out = np.zeros((5, nl, n[mode], nr))
    lib().o_cross_eval(n_, r_, ptrs, h_, alpha, gamma, eps, bc_, mode, fd, nl, left.ctypes.data, nr,
                       right.ctypes.data, _dp(out))
    del keep
    return out


def tt_full(n, r, cores3):
    """Full FP64 tensor [k][j][i] of one field from its three cores."""
    n_ = (C.c_int * 3)(*n)
    r_ = (C.c_int * 2)(*r)
    ptrs, keep = _core_ptrs([cores3])
    X = np.zeros((n[2], n[1], n[0]))
    lib().o_tt_full(n_, r_, ptrs, _dp(X))
    del keep
    return X
