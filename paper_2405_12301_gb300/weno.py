"""ctypes binding of the GB300 WENO5-JS library (include/weno_gb300.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``_lib/libweno_gb300.so``.  Device arrays are torch tensors (FP64,
contiguous, on the current CUDA device); the binding passes their data
pointers and torch's current stream.  There is no CPU fallback: if the library
is missing or a call fails, an exception is raised.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libweno_gb300.so")

OK, ERR_ARG, ERR_CUDA, ERR_NONPHYSICAL, ERR_TIMEOUT, ERR_UNSUPPORTED = range(6)
BC_PERIODIC, BC_TRANSMISSIVE, BC_REFLECTIVE, BC_INFLOW = 0, 1, 2, 3
FP64, FP32_BULK = 0, 1
ALPHA_GLOBAL_NORM, ALPHA_PER_DIR = 0, 1
MODEL_EULER, MODEL_ADVECT, MODEL_BURGERS = 0, 1, 2
CROSS_FP64_CHECK, CROSS_GRAPH = 1, 2

EXPORTS = ("weno_init", "weno_destroy", "weno_set_stream", "weno_alpha", "weno_rhs", "weno_set_time",
           "weno_get_time", "weno_ssprk3_step", "weno_run", "weno_run_host", "weno_sums", "weno_sync",
           "weno_last_error", "weno_cross_eval", "weno_profile_enable", "weno_profile_read",
           "weno_sums_noalloc", "weno_tt_round", "weno_maxvol", "weno_tt_cross", "weno_cross_autotune",
           "weno_tune_save", "weno_tune_load")
PROFILE_KINDS = 8


class WenoError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("weno status %d: %s" % (code, msg))
        self.code = code


class weno_grid(C.Structure):
    _fields_ = [("dim", C.c_int32), ("reserved", C.c_int32), ("n", C.c_int64 * 3),
                ("lo", C.c_double * 3), ("hi", C.c_double * 3)]


class weno_params(C.Structure):
    _fields_ = [("gamma", C.c_double), ("eps_weno", C.c_double), ("cfl", C.c_double),
                ("bc", (C.c_int32 * 2) * 3), ("precision", C.c_int32), ("alpha_mode", C.c_int32),
                ("bc_state", ((C.c_double * 5) * 2) * 3), ("model", C.c_int32), ("reserved", C.c_int32)]


class weno_tt_instance(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("r", C.c_int32 * 2), ("reserved", C.c_int32),
                ("core", (C.c_void_p * 3) * 5), ("h", C.c_double * 3), ("alpha", C.c_double),
                ("bc", (C.c_int32 * 2) * 3)]


class weno_fiber_set(C.Structure):
    _fields_ = [("instance", C.c_int32), ("mode", C.c_int32), ("flux_dir", C.c_int32), ("reserved", C.c_int32),
                ("n_left", C.c_int64), ("n_right", C.c_int64), ("left", C.c_void_p), ("right", C.c_void_p),
                ("out", C.c_void_p)]


class weno_tt3(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("r", C.c_int32 * 2), ("core", C.c_void_p * 3)]


TT_MAX_TERMS, TT_MAX_RANK = 4, 96


class weno_tt_round_problem(C.Structure):
    _fields_ = [("n_terms", C.c_int32), ("reserved", C.c_int32), ("coef", C.c_double * TT_MAX_TERMS),
                ("term", weno_tt3 * TT_MAX_TERMS), ("out", weno_tt3), ("cap", C.c_int64 * 3), ("norm", C.c_double)]


class weno_maxvol_problem(C.Structure):
    _fields_ = [("n", C.c_int32), ("r", C.c_int32), ("A", C.c_void_p), ("B", C.c_void_p), ("idx", C.c_void_p)]


_lib = None


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libweno_gb300.so is missing; run __graft_entry__.build() (needs nvcc)")
        L = C.CDLL(LIB_PATH)
        P, d, i64, i32, vp = C.POINTER, C.c_double, C.c_int64, C.c_int32, C.c_void_p
        L.weno_init.argtypes = [P(vp), P(weno_grid), P(weno_params), vp]
        L.weno_destroy.argtypes = [vp]
        L.weno_set_stream.argtypes = [vp, vp]
        L.weno_alpha.argtypes = [vp, vp, vp]
        L.weno_rhs.argtypes = [vp, vp, vp, vp]
        L.weno_set_time.argtypes = [vp, d]
        L.weno_get_time.argtypes = [vp, P(d), P(i64)]
        L.weno_ssprk3_step.argtypes = [vp, vp, d, d]
        L.weno_run.argtypes = [vp, vp, d, d, i64, i32, P(i64)]
        L.weno_run_host.argtypes = [vp, vp, d, d, i64, i32, P(i64)]
        L.weno_sums.argtypes = [vp, vp, vp]
        L.weno_sync.argtypes = [vp]
        L.weno_last_error.argtypes = [vp]
        L.weno_last_error.restype = C.c_char_p
        L.weno_cross_eval.argtypes = [vp, P(weno_tt_instance), i32, P(weno_fiber_set), i32, i32]
        L.weno_profile_enable.argtypes = [vp, i32]
        L.weno_profile_read.argtypes = [vp, P(d), P(i64), P(i64)]
        L.weno_sums_noalloc.argtypes = [vp, i32, i64, vp, vp]
        L.weno_tt_round.argtypes = [vp, P(weno_tt_round_problem), i32, d]
        L.weno_maxvol.argtypes = [vp, P(weno_maxvol_problem), i32, d, i32, P(i32)]
        L.weno_tt_cross.argtypes = [vp, P(weno_tt_instance), i32, i32, P(weno_tt_cross_problem), i32, d, i32]
        L.weno_cross_autotune.argtypes = [vp, P(weno_tt_instance), i32, P(weno_fiber_set), i32, i32, i32, P(i32),
                                          P(d)]
        L.weno_tune_save.argtypes = [vp, C.c_char_p]
        L.weno_tune_load.argtypes = [vp, C.c_char_p, P(i32)]
        for name in EXPORTS:
            if name != "weno_last_error":
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _check(h, code):
    if code != OK:
        msg = lib().weno_last_error(h)
        raise WenoError(code, msg.decode() if msg else "")
    return code


def _ptr(t, dtype=None):
    import torch
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError("expected dtype %s, got %s" % (dtype, t.dtype))
    return C.c_void_p(t.data_ptr())


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


# ------------------------------------------------------------ thin wrappers
def weno_init(dim=None, n=None, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), gamma=1.4, eps_weno=1e-6, cfl=0.5,
              bc=((BC_PERIODIC, BC_PERIODIC),) * 3, precision=FP64, alpha_mode=ALPHA_GLOBAL_NORM, stream=None,
              bc_state=None, model=MODEL_EULER):
    """Returns a handle (c_void_p).  dim=None makes a cross-eval-only handle."""
    g = None
    if dim is not None:
        g = weno_grid()
        g.dim = dim
        nn = list(n) + [1] * (3 - len(n))
        for k in range(3):
            g.n[k] = int(nn[k])
            g.lo[k] = float(lo[k]) if k < len(lo) else 0.0
            g.hi[k] = float(hi[k]) if k < len(hi) else 1.0
    p = weno_params()
    p.gamma, p.eps_weno, p.cfl = gamma, eps_weno, cfl
    for k in range(3):
        p.bc[k][0], p.bc[k][1] = bc[k] if k < len(bc) else (BC_PERIODIC, BC_PERIODIC)
    p.precision, p.alpha_mode, p.model = precision, alpha_mode, model
    if bc_state is not None:  # [3][2][nf] conserved states of the inflow sides
        for k in range(3):
            for side in range(2):
                for f, v in enumerate(bc_state[k][side]):
                    p.bc_state[k][side][f] = float(v)
    h = C.c_void_p()
    code = lib().weno_init(C.byref(h), C.byref(g) if g is not None else None, C.byref(p),
                           stream if stream is not None else _stream())
    if code != OK:
        raise WenoError(code, lib().weno_last_error(None).decode())
    return h


def weno_destroy(h):
    return _check(h, lib().weno_destroy(h))


def weno_set_stream(h, stream=None):
    """Binds a torch CUDA stream (default: the current one) to the handle."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    return _check(h, lib().weno_set_stream(h, C.c_void_p(st.cuda_stream)))


def weno_alpha(h, U, alpha_out):
    import torch
    return _check(h, lib().weno_alpha(h, _ptr(U, torch.float64), _ptr(alpha_out, torch.float64)))


def weno_rhs(h, U, R, alpha_out=None):
    import torch
    a = _ptr(alpha_out, torch.float64) if alpha_out is not None else None
    return _check(h, lib().weno_rhs(h, _ptr(U, torch.float64), _ptr(R, torch.float64), a))


def weno_set_time(h, t):
    return _check(h, lib().weno_set_time(h, float(t)))


def weno_get_time(h):
    t, s = C.c_double(), C.c_int64()
    _check(h, lib().weno_get_time(h, C.byref(t), C.byref(s)))
    return t.value, s.value


def weno_ssprk3_step(h, U, t_end, dt=0.0):
    import torch
    return _check(h, lib().weno_ssprk3_step(h, _ptr(U, torch.float64), float(t_end), float(dt)))


def weno_run(h, U, t_end, dt=0.0, max_steps=1 << 62, graph_steps=16):
    import torch
    s = C.c_int64()
    _check(h, lib().weno_run(h, _ptr(U, torch.float64), float(t_end), float(dt), int(max_steps),
                             int(graph_steps), C.byref(s)))
    return s.value


def weno_run_host(h, U_host, t_end, dt=0.0, max_steps=1 << 62, graph_steps=16):
    """U_host: a contiguous FP64 CPU tensor (pinned is fastest), updated in place."""
    import torch
    if U_host.is_cuda or not U_host.is_contiguous() or U_host.dtype != torch.float64:
        raise ValueError("expected a contiguous FP64 CPU tensor")
    s = C.c_int64()
    _check(h, lib().weno_run_host(h, C.c_void_p(U_host.data_ptr()), float(t_end), float(dt), int(max_steps),
                                  int(graph_steps), C.byref(s)))
    return s.value


def weno_sums(h, U, nf):
    import torch
    out = (C.c_double * nf)()
    _check(h, lib().weno_sums(h, _ptr(U, torch.float64), out))
    return list(out)


def weno_sums_noalloc(U, sums_out, stream=None):
    """Conservation sums into the device tensor sums_out (nf doubles) without any
    device allocation; U is [nf, ...] FP64 on the current device."""
    import torch
    nf = U.shape[0]
    code = lib().weno_sums_noalloc(_ptr(U, torch.float64), nf, U.numel() // nf, _ptr(sums_out, torch.float64),
                                   stream if stream is not None else _stream())
    if code != OK:
        raise WenoError(code, lib().weno_last_error(None).decode())
    return code


def weno_sync(h):
    return _check(h, lib().weno_sync(h))


def weno_profile_enable(h, enable=True):
    return _check(h, lib().weno_profile_enable(h, 1 if enable else 0))


def weno_profile_read(h):
    """(ms per kind, launches per kind, total kernel launches) since the last enable."""
    ms = (C.c_double * PROFILE_KINDS)()
    n = (C.c_int64 * PROFILE_KINDS)()
    tot = C.c_int64()
    _check(h, lib().weno_profile_read(h, ms, n, C.byref(tot)))
    return list(ms), list(n), tot.value


def tt_caps(n, R1, R2):
    """Output capacities (doubles per core) that always suffice for a sum of summed ranks R1, R2."""
    k3 = min(n[2], R2)
    k2 = min(n[1] * k3, R1)
    kc = min(n[0], k2)
    ke = min(kc * n[1], k3)
    return (n[0] * kc, n[1] * kc * ke, n[2] * ke)


def weno_tt_round(h, problems, eps_tt):
    """problems: list of term lists [(coef, [core0, core1, core2]), ...], cores FP64 CUDA
    tensors shaped [n_m, r_{m-1}, r_m].  Returns [(cores, norm)] with the rounded cores
    as CUDA tensors of the chosen ranks."""
    import torch
    arr = (weno_tt_round_problem * len(problems))()
    keep = []
    for i, terms in enumerate(problems):
        P = arr[i]
        P.n_terms = len(terms)
        R1 = R2 = 0
        for t, (c, cores) in enumerate(terms):
            P.coef[t] = float(c)
            X = P.term[t]
            for m in range(3):
                X.n[m] = int(cores[m].shape[0])
                X.core[m] = _ptr(cores[m], torch.float64).value
            X.r[0], X.r[1] = int(cores[0].shape[2]), int(cores[1].shape[2])
            R1 += X.r[0]
            R2 += X.r[1]
        n = [int(terms[0][1][m].shape[0]) for m in range(3)]
        caps = tt_caps(n, R1, R2)
        bufs = [torch.empty(max(1, c), dtype=torch.float64, device="cuda") for c in caps]
        keep.append(bufs)
        for m in range(3):
            P.out.core[m] = bufs[m].data_ptr()
            P.cap[m] = caps[m]
    _check(h, lib().weno_tt_round(h, arr, len(problems), float(eps_tt)))
    out = []
    for i, bufs in enumerate(keep):
        o = arr[i].out
        n, r1, r2 = list(o.n), o.r[0], o.r[1]
        cores = [bufs[0][:n[0] * r1].view(n[0], 1, r1), bufs[1][:n[1] * r1 * r2].view(n[1], r1, r2),
                 bufs[2][:n[2] * r2].view(n[2], r2, 1)]
        out.append((cores, arr[i].norm))
    return out


def weno_maxvol(h, mats, delta=1e-2, max_iters=200):
    """mats: FP64 CUDA tensors n x r.  Returns [(idx int32 tensor, B tensor, swaps)]."""
    import torch
    arr = (weno_maxvol_problem * len(mats))()
    outs = []
    for i, A in enumerate(mats):
        n, r = A.shape
        B = torch.empty_like(A)
        idx = torch.empty(r, dtype=torch.int32, device=A.device)
        arr[i].n, arr[i].r = n, r
        arr[i].A = _ptr(A, torch.float64).value
        arr[i].B = B.data_ptr()
        arr[i].idx = idx.data_ptr()
        outs.append((idx, B))
    sw = (C.c_int32 * len(mats))()
    _check(h, lib().weno_maxvol(h, arr, len(mats), float(delta), int(max_iters), sw))
    return [(idx, B, int(sw[i])) for i, (idx, B) in enumerate(outs)]


def _instances(instances):
    import torch
    inst = (weno_tt_instance * len(instances))()
    for k, d in enumerate(instances):
        for m in range(3):
            inst[k].n[m] = int(d["n"][m])
            inst[k].h[m] = float(d["h"][m])
            inst[k].bc[m][0], inst[k].bc[m][1] = d["bc"][m]
        for m in range(2):
            inst[k].r[m] = int(d["r"][m])
        for f in range(5):
            for m in range(3):
                inst[k].core[f][m] = _ptr(d["cores"][f][m], torch.float32).value
        inst[k].alpha = float(d["alpha"])
    return inst


def _fiber_sets(sets, fp64_check):
    import torch
    fs = (weno_fiber_set * len(sets))()
    for k, s in enumerate(sets):
        fs[k].instance, fs[k].mode, fs[k].flux_dir = s["instance"], s["mode"], s["flux_dir"]
        fs[k].n_left = s["left"].shape[0] if s["left"] is not None else 1
        fs[k].n_right = s["right"].shape[0] if s["right"] is not None else 1
        fs[k].left = _ptr(s["left"], torch.int32).value if s["left"] is not None else None
        fs[k].right = _ptr(s["right"], torch.int32).value if s["right"] is not None else None
        fs[k].out = _ptr(s["out"], torch.float64 if fp64_check else torch.float32).value
    return fs


def weno_cross_eval(h, instances, sets, fp64_check=False, graph=False):
    """instances: list of dict(n, r, cores=[5][3] CUDA float32 tensors, h, alpha, bc);
    sets: list of dict(instance, mode, flux_dir, left, right, out) with CUDA tensors."""
    inst = _instances(instances)
    fs = _fiber_sets(sets, fp64_check)
    flags = (CROSS_FP64_CHECK if fp64_check else 0) | (CROSS_GRAPH if graph else 0)
    return _check(h, lib().weno_cross_eval(h, inst, len(instances), fs, len(sets), flags))


def weno_cross_autotune(h, instances, sets, fp64_check=False, reps=3):
    """Times every kernel variant and grid size on this workload; returns
    ((threads per CTA, samples per chunk, CTAs per SM), ms per evaluation)."""
    inst = _instances(instances)
    fs = _fiber_sets(sets, fp64_check)
    choice = (C.c_int32 * 3)()
    ms = C.c_double()
    _check(h, lib().weno_cross_autotune(h, inst, len(instances), fs, len(sets), CROSS_FP64_CHECK if fp64_check else 0,
                                        int(reps), choice, C.byref(ms)))
    return tuple(choice), ms.value


def weno_tune_save(h, path):
    return _check(h, lib().weno_tune_save(h, os.fsencode(path)))


def weno_tune_load(h, path):
    n = C.c_int32()
    _check(h, lib().weno_tune_load(h, os.fsencode(path), C.byref(n)))
    return n.value


class weno_tt_cross_problem(C.Structure):
    _fields_ = [("r", C.c_int32 * 2), ("J1", C.c_void_p), ("J2", C.c_void_p), ("I1", C.c_void_p),
                ("I2", C.c_void_p), ("core", C.c_void_p * 3)]


def weno_tt_cross(h, instances, flux_dir, ranks, J1s, J2s, sweeps=1, delta=1e-2, fp64_check=False):
    """TT-cross of the flux_dir residual of every instance.  ranks: [(r1, r2)];
    J1s / J2s: initial right index sets, int32 CUDA tensors [r1][3] / [r2][2]
    (updated in place).  Returns [dict(cores, I1, I2, J1, J2)] of CUDA tensors."""
    import torch
    inst = _instances(instances)
    arr = (weno_tt_cross_problem * len(instances))()
    outs = []
    for i, d in enumerate(instances):
        r1, r2 = ranks[i]
        n = [int(x) for x in d["n"]]
        o = dict(cores=[torch.empty((n[0], 1, r1), dtype=torch.float64, device="cuda"),
                        torch.empty((n[1], r1, r2), dtype=torch.float64, device="cuda"),
                        torch.empty((n[2], r2, 5), dtype=torch.float64, device="cuda")],
                 I1=torch.empty(r1, dtype=torch.int32, device="cuda"),
                 I2=torch.empty((r2, 2), dtype=torch.int32, device="cuda"), J1=J1s[i], J2=J2s[i])
        P = arr[i]
        P.r[0], P.r[1] = r1, r2
        P.J1 = _ptr(J1s[i], torch.int32).value
        P.J2 = _ptr(J2s[i], torch.int32).value
        P.I1 = o["I1"].data_ptr()
        P.I2 = o["I2"].data_ptr()
        for m in range(3):
            P.core[m] = o["cores"][m].data_ptr()
        outs.append(o)
    _check(h, lib().weno_tt_cross(h, inst, len(instances), int(flux_dir), arr, int(sweeps), float(delta),
                                  CROSS_FP64_CHECK if fp64_check else 0))
    return outs


class Solver:
    """Owns one handle: a grid, its parameters and its scratch."""

    def __init__(self, dim, n, lo=None, hi=None, **kw):
        lo = lo if lo is not None else (0.0,) * dim
        hi = hi if hi is not None else (1.0,) * dim
        self.dim, self.n = dim, tuple(n)
        self.nf = dim + 2 if kw.get("model", MODEL_EULER) == MODEL_EULER else 1
        self.h = weno_init(dim, n, lo, hi, **kw)

    def close(self):
        if self.h is not None:
            weno_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def rhs(self, U, R, alpha_out=None):
        return weno_rhs(self.h, U, R, alpha_out)

    def alpha(self, U, out):
        return weno_alpha(self.h, U, out)

    def set_time(self, t):
        return weno_set_time(self.h, t)

    def time(self):
        return weno_get_time(self.h)

    def step(self, U, t_end=float("inf"), dt=0.0):
        return weno_ssprk3_step(self.h, U, t_end, dt)

    def run(self, U, t_end, dt=0.0, max_steps=1 << 62, graph_steps=16):
        return weno_run(self.h, U, t_end, dt, max_steps, graph_steps)

    def run_host(self, U_host, t_end, dt=0.0, max_steps=1 << 62, graph_steps=16):
        return weno_run_host(self.h, U_host, t_end, dt, max_steps, graph_steps)

    def sums(self, U):
        return weno_sums(self.h, U, self.nf)

    def sync(self):
        return weno_sync(self.h)

    def set_stream(self, stream=None):
        return weno_set_stream(self.h, stream)

    def profile_enable(self, enable=True):
        return weno_profile_enable(self.h, enable)

    def profile_read(self):
        return weno_profile_read(self.h)
