"""Seeded synthetic inputs for the WENO5-JS Euler workloads.

This module is shared by the oracle's tests and the CUDA path's tests and
benchmark.  It holds initial conditions, random smooth/discontinuous states,
TT cores and cross index sets, and none of the scheme's arithmetic (no flux,
splitting, reconstruction or time stepping).  Initial conditions are stated in
primitive variables (rho, u, p) and handed over in conserved form
U = (rho, rho u, ..., rho E), rho E = p / (gamma - 1) + rho |u|^2 / 2.

All arrays are numpy FP64 in the layout [field][k][j][i] (x fastest), interior
cells only, cell-centred: x_i = lo + (i + 1/2) h.
"""
import numpy as np

MASTER_SEED = 12301


def centres(n, lo, hi):
    h = (hi - lo) / n
    return lo + (np.arange(n) + 0.5) * h


def _grid(dim, n, lo, hi):
    """Meshgrid of cell centres as arrays shaped [nz][ny][nx]."""
    n = list(n) + [1] * (3 - len(n))
    lo = list(lo) + [0.0] * (3 - len(lo))
    hi = list(hi) + [1.0] * (3 - len(hi))
    axes = [centres(n[d], lo[d], hi[d]) if d < dim else np.zeros(1) for d in range(3)]
    Z, Y, X = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    return X, Y, Z


def conserved(dim, rho, vel, p, gamma=1.4):
    """Conserved state [nf][nz][ny][nx] from primitive fields."""
    ke = sum(vel[d] * vel[d] for d in range(dim))
    U = [rho] + [rho * vel[d] for d in range(dim)] + [p / (gamma - 1.0) + 0.5 * rho * ke]
    return np.ascontiguousarray(np.stack([np.broadcast_to(u, rho.shape) for u in U]), dtype=np.float64)


# ----------------------------------------------------------- initial states
def density_wave(dim, n, t=0.0, length=2.0, amp=0.2, gamma=1.4):
    """rho = 1 + amp sin(pi (sum_d x_d - dim t)), u_d = 1, p = 1 on [0, length)^dim.

    At t > 0 this is the exact advected solution of the Euler equations."""
    X, Y, Z = _grid(dim, n, [0.0] * 3, [length] * 3)
    s = X + (Y if dim > 1 else 0.0) + (Z if dim > 2 else 0.0)
    rho = 1.0 + amp * np.sin(np.pi * (s - dim * t))
    vel = [np.ones_like(rho) for _ in range(dim)]
    return conserved(dim, rho, vel, np.ones_like(rho), gamma)


def quadrant_riemann(n, split=(0.5, 0.5), gamma=1.4):
    """2D four-quadrant Riemann problem on [0,1]^2, (p, rho, u, v) per quadrant:
    NE (1.5, 1.5, 0, 0), NW (0.3, 0.5323, 1.206, 0), SW (0.029, 0.138, 1.206, 1.206),
    SE (0.3, 0.5323, 0, 1.206)."""
    X, Y, _ = _grid(2, n, [0.0, 0.0], [1.0, 1.0])
    east, north = X > split[0], Y > split[1]
    table = {  # (east, north): (p, rho, u, v)
        (True, True): (1.5, 1.5, 0.0, 0.0),
        (False, True): (0.3, 0.5323, 1.206, 0.0),
        (False, False): (0.029, 0.138, 1.206, 1.206),
        (True, False): (0.3, 0.5323, 0.0, 1.206),
    }
    p = np.zeros_like(X)
    rho = np.zeros_like(X)
    u = np.zeros_like(X)
    v = np.zeros_like(X)
    for (e, nn), (pp, rr, uu, vv) in table.items():
        m = (east == e) & (north == nn)
        p[m], rho[m], u[m], v[m] = pp, rr, uu, vv
    return conserved(2, rho, [u, v], p, gamma)


def sod(dim, n, gamma=1.4, split=0.5):
    """Sod shock tube along x on [0,1]^dim: (rho, u, p) = (1, 0, 1) for x < split,
    (0.125, 0, 0.1) otherwise."""
    X, _, _ = _grid(dim, n, [0.0] * 3, [1.0] * 3)
    left = X < split
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    vel = [np.zeros_like(rho) for _ in range(dim)]
    return conserved(dim, rho, vel, p, gamma)


def scalar_sine(dim, n, offset=0.0, amp=1.0):
    """u0 = offset + amp sin(2 pi (x + y + z)) on [0,1]^dim (one field)."""
    X, Y, Z = _grid(dim, n, [0.0] * 3, [1.0] * 3)
    s = X + (Y if dim > 1 else 0.0) + (Z if dim > 2 else 0.0)
    return np.ascontiguousarray((offset + amp * np.sin(2 * np.pi * s))[None], dtype=np.float64)


def _smooth(rng, shape_axes, modes=3, kmax=3):
    """Random smooth periodic field on the unit cube (sum of sine products)."""
    X, Y, Z = shape_axes
    g = np.zeros_like(X)
    for _ in range(modes):
        k = rng.integers(1, kmax + 1, size=3)
        ph = rng.uniform(0, 2 * np.pi, size=3)
        a = rng.uniform(-1, 1)
        g += a * np.sin(2 * np.pi * k[0] * X + ph[0]) * np.sin(2 * np.pi * k[1] * Y + ph[1]) \
            * np.sin(2 * np.pi * k[2] * Z + ph[2])
    return g / max(1.0, np.abs(g).max())


def random_state(dim, n, seed, jumps=False, gamma=1.4, length=1.0):
    """Seeded random positive state: smooth (rho, u, p) perturbations, plus, when
    jumps is set, a few planar discontinuities (contact and pressure jumps)."""
    rng = np.random.default_rng(seed)
    ax = _grid(dim, n, [0.0] * 3, [length] * 3)
    unit = tuple(a / length for a in ax)
    rho = 1.0 + 0.3 * _smooth(rng, unit)
    p = 1.0 + 0.3 * _smooth(rng, unit)
    vel = [0.5 * _smooth(rng, unit) for _ in range(dim)]
    if jumps:
        for _ in range(2):
            nrm = rng.normal(size=3)
            nrm[dim:] = 0.0
            nrm /= np.linalg.norm(nrm)
            c = rng.uniform(0.3, 0.7)
            side = (nrm[0] * unit[0] + nrm[1] * unit[1] + nrm[2] * unit[2]) > c * nrm.sum()
            rho = np.where(side, rho * rng.uniform(0.3, 0.6), rho)
            p = np.where(side, p * rng.uniform(0.2, 0.5), p)
    return conserved(dim, rho, vel, p, gamma)


# ------------------------------------------------------- TT cores and fibers
def tt_svd3(X, r1, r2):
    """Rank-(r1, r2) TT-SVD of a 3D torch tensor X[k][j][i] (mode 0 = i = x).

    Returns cores [n0, 1, r1], [n1, r1, r2], [n2, r2, 1] (FP64 torch tensors).  Uses
    the leading eigenvectors of the Gram matrices of the first and last unfoldings,
    which is enough for generating inputs (the cores are the input; nothing is
    compared against the full tensor)."""
    import torch
    n2, n1, n0 = X.shape
    dev = X.device
    eigh = lambda G: torch.linalg.eigh(G.cpu())[1].to(dev)  # small Gram matrices: eigh on the host
    A = X.permute(2, 1, 0).reshape(n0, n1 * n2)             # [i, (j,k)]
    V1 = eigh(A @ A.T)[:, -r1:]                              # [n0, r1]
    B = (V1.T @ A).reshape(r1 * n1, n2)                      # [(a,j), k]
    V3 = eigh(B.T @ B)[:, -r2:]                              # [n2, r2]
    C2 = (B @ V3).reshape(r1, n1, r2)                        # [a, j, b]
    return V1.reshape(n0, 1, r1), C2.permute(1, 0, 2).contiguous(), V3.reshape(n2, r2, 1)


def tt_instance(seed, n=None, r=None, gamma=1.4, device=None):
    """One seeded 3D Euler instance in TT form: n per mode from {64,128,256,512}
    and ranks in 2..32 unless given; fields are sums of 1-4 random-phase sine
    products plus a tanh front of width 4 cells, combined into primitives
    rho = 1 + 0.2 g1, p = 1 + 0.2 g2, u_d = 0.5 g_{2+d}, converted to conserved
    form and TT-SVD'd to the drawn ranks; cores are stored FP32.

    Returns dict(n=[3], r=[2], cores=[5][3] float32 numpy arrays)."""
    rng = np.random.default_rng(seed)
    if n is None:
        n = [int(rng.choice([64, 128, 256, 512])) for _ in range(3)]
    if r is None:
        r = [int(rng.integers(2, 33)) for _ in range(2)]
    r = [min(r[0], n[0]), min(r[1], n[2])]
    xs = [centres(n[d], 0.0, 1.0) for d in range(3)]
    hmin = 1.0 / max(n)
    nrm = rng.normal(size=3)
    nrm /= np.linalg.norm(nrm)
    cfront = float(rng.uniform(0.3, 0.7)) * nrm.sum()
    gs = []
    for _ in range(5):
        M = int(rng.integers(1, 5))
        terms = []
        for _m in range(M):
            k = rng.integers(1, 4, size=3)
            ph = rng.uniform(0, 2 * np.pi, size=3)
            terms.append((rng.uniform(-1, 1), k, ph))
        gs.append(terms)
    front_amp = 0.5
    try:
        import torch
        use_torch = True
    except ImportError:  # pragma: no cover
        use_torch = False
    if use_torch:
        dev = device or ("cuda" if torch.cuda.is_available() else "cpu")
        T = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
        Xg = [T(x) for x in xs]
        Z, Y, X = torch.meshgrid(Xg[2], Xg[1], Xg[0], indexing="ij")
        front = front_amp * torch.tanh((nrm[0] * X + nrm[1] * Y + nrm[2] * Z - cfront) / (4 * hmin))
        g = []
        for terms in gs:
            acc = front.clone()
            scale = sum(abs(a) for a, _, _ in terms)
            for a, k, ph in terms:
                acc += (a / max(scale, 1e-12)) * torch.sin(2 * np.pi * k[0] * X + ph[0]) \
                    * torch.sin(2 * np.pi * k[1] * Y + ph[1]) * torch.sin(2 * np.pi * k[2] * Z + ph[2])
            g.append(acc)
        rho = 1.0 + 0.2 * g[0]
        p = 1.0 + 0.2 * g[1]
        vel = [0.5 * g[2 + d] for d in range(3)]
        ke = vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2
        fields = [rho, rho * vel[0], rho * vel[1], rho * vel[2], p / (gamma - 1.0) + 0.5 * rho * ke]
        cores = []
        for F in fields:
            c0, c1, c2 = tt_svd3(F, r[0], r[1])
            cores.append([c.to(torch.float32).cpu().numpy().copy() for c in (c0, c1, c2)])
            del c0, c1, c2
        del fields, rho, p, vel, g, X, Y, Z, front
        if dev == "cuda":
            torch.cuda.empty_cache()
    else:  # pragma: no cover
        raise RuntimeError("tt_instance needs torch for the TT-SVD")
    return dict(n=n, r=r, cores=cores)


def cross_index_sets(seed, n, r, mode):
    """Seeded TT-cross index sets for a sweep over `mode`: r_{mode-1} left
    multi-indices over the modes before it and r_mode right multi-indices over
    the modes after it, drawn without replacement (int32)."""
    rng = np.random.default_rng(seed)
    rl = 1 if mode == 0 else r[mode - 1]
    rr = 1 if mode == 2 else r[mode]

    def draw(count, modes):
        if not modes:
            return np.zeros((1, 0), np.int32)
        total = int(np.prod([n[m] for m in modes]))
        count = min(count, total)
        flat = rng.choice(total, size=count, replace=False)
        idx = []
        for m in modes:
            idx.append(flat % n[m])
            flat = flat // n[m]
        return np.ascontiguousarray(np.stack(idx, axis=1).astype(np.int32))

    left = draw(rl, list(range(mode)))
    right = draw(rr, list(range(mode + 1, 3)))
    return left, right
