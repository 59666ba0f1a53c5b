"""weno_cross_eval (pointwise residual at TT-cross samples) against the
oracle's pointwise evaluation from the same FP32 cores.  GPU only.

Tolerances:
  * FP64 check mode: 1e-12 relative to the field scale max(|b|, |b_f|_inf)
    plus 1e-13 S / h (ulp-level differences of the interface fluxes, S the
    split-flux scale), as for the full-grid FP64 residual.
  * FP32 mode: 64 * 2^-24 * V / h, V = (1 + alpha) times the largest variation
    of the state over the tensor times (1 + max |u|): the FP32 path contracts
    differences of core rows, so its rounding scales with the variation.
"""
import numpy as np
import pytest

import oracle as O
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


def make_instance(seed, n, r, bc, alpha=None):
    inst = I.tt_instance(seed=seed, n=n, r=r, device="cpu")
    n, r, cores = inst["n"], inst["r"], inst["cores"]
    U = np.stack([O.tt_full(n, r, cores[f]) for f in range(5)])
    cfg = O.Cfg(dim=3, n=tuple(n), hi=(1.0, 1.0, 1.0), bc=(bc,) * 3)
    a = alpha if alpha is not None else 1.05 * O.alpha_max(cfg, U)
    return dict(n=n, r=r, cores=cores, h=[1.0 / n[0], 1.0 / n[1], 1.0 / n[2]], bc=(bc,) * 3, alpha=a, U=U)


def dev_instance(inst):
    d = dict(inst)
    d["cores"] = [[torch.from_numpy(c).cuda() for c in fc] for fc in inst["cores"]]
    return d


def make_sets(inst, k, seed, fp64, which=None):
    sets, refs = [], []
    for mode in range(3):
        for fd in range(3):
            if which is not None and (mode, fd) not in which:
                continue
            left, right = I.cross_index_sets(seed + 10 * mode + fd, inst["n"], inst["r"], mode)
            out = torch.zeros((5, left.shape[0], inst["n"][mode], right.shape[0]),
                              dtype=torch.float64 if fp64 else torch.float32, device="cuda")
            sets.append(dict(instance=k, mode=mode, flux_dir=fd,
                             left=torch.from_numpy(left).cuda() if mode > 0 else None,
                             right=torch.from_numpy(right).cuda() if mode < 2 else None, out=out))
            refs.append((mode, fd, left, right))
    return sets, refs


def oracle_out(inst, mode, fd, left, right):
    return O.cross_eval(inst["n"], inst["r"], inst["cores"], inst["h"], inst["alpha"], 1.4, 1e-6, inst["bc"],
                        mode, fd, left, right)


def tol_fp64(ref, inst):
    S = inst["alpha"] * np.abs(inst["U"]).max() + np.abs(inst["U"][4]).max()
    t = np.empty_like(ref)
    for f in range(5):
        t[f] = 1e-12 * np.maximum(np.abs(ref[f]), np.abs(ref[f]).max()) + 1e-13 * S * max(inst["n"])
    return t


def tol_fp32(inst):
    U = inst["U"]
    var = max(float(U[f].max() - U[f].min()) for f in range(5))
    umax = float((np.abs(U[1:4]) / U[0]).max())
    return 64 * 2.0 ** -24 * (1 + inst["alpha"]) * var * (1 + umax) * max(inst["n"])


@pytest.mark.parametrize("bc", [O.PERIODIC, O.TRANSMISSIVE, O.REFLECTIVE])
@pytest.mark.parametrize("fp64", [True, False])
def test_cross_eval_matches_oracle(W, bc, fp64):
    inst = make_instance(3, [12, 16, 10], [3, 5], (bc, bc))
    h = W.weno_init(None, precision=W.FP64)
    sets, refs = make_sets(inst, 0, 40, fp64)
    W.weno_cross_eval(h, [dev_instance(inst)], sets, fp64_check=fp64)
    W.weno_sync(h)
    worst = 0.0
    for s, (mode, fd, left, right) in zip(sets, refs):
        ref = oracle_out(inst, mode, fd, left, right)
        got = s["out"].double().cpu().numpy()
        tol = tol_fp64(ref, inst) if fp64 else tol_fp32(inst)
        worst = max(worst, float((np.abs(got - ref) / tol).max()))
        assert (np.abs(got - ref) <= tol).all(), (mode, fd, float(np.abs(got - ref).max()))
    print("worst error / tolerance:", worst)
    W.weno_destroy(h)


def test_cross_eval_batched_uneven_instances(W):
    """Several instances of different sizes and ranks, all sets in one launch."""
    insts = [make_instance(11, [16, 24, 12], [4, 6], (O.PERIODIC,) * 2),
             make_instance(12, [20, 12, 28], [7, 3], (O.TRANSMISSIVE,) * 2),
             make_instance(13, [10, 10, 10], [2, 2], (O.REFLECTIVE,) * 2)]
    h = W.weno_init(None)
    allsets, allrefs = [], []
    for k, inst in enumerate(insts):
        sets, refs = make_sets(inst, k, 70 + k, True)
        allsets += sets
        allrefs += [(k,) + r for r in refs]
    W.weno_cross_eval(h, [dev_instance(i) for i in insts], allsets, fp64_check=True)
    W.weno_sync(h)
    for s, (k, mode, fd, left, right) in zip(allsets, allrefs):
        ref = oracle_out(insts[k], mode, fd, left, right)
        got = s["out"].cpu().numpy()
        assert (np.abs(got - ref) <= tol_fp64(ref, insts[k])).all(), (k, mode, fd)
    W.weno_destroy(h)


def test_cross_eval_long_fiber_per_sample_path(W):
    """n_mode > 512 with the stencil along the fiber takes the per-sample path."""
    inst = make_instance(21, [520, 6, 5], [2, 2], (O.PERIODIC,) * 2)
    h = W.weno_init(None)
    for fp64 in (True, False):
        sets, refs = make_sets(inst, 0, 90, fp64, which={(0, 0)})
        W.weno_cross_eval(h, [dev_instance(inst)], sets, fp64_check=fp64)
        W.weno_sync(h)
        ref = oracle_out(inst, *refs[0][:2], refs[0][2], refs[0][3])
        got = sets[0]["out"].double().cpu().numpy()
        tol = tol_fp64(ref, inst) if fp64 else tol_fp32(inst)
        assert (np.abs(got - ref) <= tol).all()
    W.weno_destroy(h)


def test_cross_eval_bad_index_is_reported(W):
    """An index set holding an index outside its mode is skipped and reported as
    WENO_ERR_ARG; nothing out of bounds is read."""
    inst = make_instance(5, [8, 9, 10], [2, 3], (O.PERIODIC,) * 2)
    h = W.weno_init(None)
    sets, _ = make_sets(inst, 0, 5, True, which={(1, 0)})
    sets[0]["left"][0, 0] = 1000
    W.weno_cross_eval(h, [dev_instance(inst)], sets, fp64_check=True)
    with pytest.raises(W.WenoError) as e:
        W.weno_sync(h)
    assert e.value.code == W.ERR_ARG
    W.weno_sync(h)
    W.weno_destroy(h)


def test_cross_eval_rejects_inflow_sides(W):
    """Inflow ghosts are a full-grid rule only: the TT path refuses them before
    launching anything."""
    inst = make_instance(6, [8, 9, 10], [2, 3], (O.PERIODIC,) * 2)
    inst["bc"] = ((O.INFLOW, O.TRANSMISSIVE),) + ((O.PERIODIC, O.PERIODIC),) * 2
    h = W.weno_init(None)
    sets, _ = make_sets(inst, 0, 6, True, which={(0, 0)})
    with pytest.raises(W.WenoError) as e:
        W.weno_cross_eval(h, [dev_instance(inst)], sets, fp64_check=True)
    assert e.value.code == W.ERR_UNSUPPORTED
    W.weno_sync(h)
    W.weno_destroy(h)


def test_cross_eval_full_workload_sampled(W):
    """The benchmark's 64-instance workload (n in {64..512}, ranks 2..32), all 9 sets
    per instance in one launch; a few fibers per set are checked against the oracle."""
    rng = np.random.default_rng(5)
    insts = [I.tt_instance(seed=I.MASTER_SEED + k) for k in range(64)]
    dinsts, sets, meta = [], [], []
    for k, inst in enumerate(insts):
        inst["h"] = [1.0 / x for x in inst["n"]]
        inst["bc"] = ((O.PERIODIC, O.PERIODIC),) * 3
        inst["alpha"] = 3.0
        dinsts.append(dev_instance(inst))
        for mode in range(3):
            for fd in range(3):
                left, right = I.cross_index_sets(1000 * k + 10 * mode + fd, inst["n"], inst["r"], mode)
                out = torch.zeros((5, left.shape[0], inst["n"][mode], right.shape[0]), dtype=torch.float32,
                                  device="cuda")
                sets.append(dict(instance=k, mode=mode, flux_dir=fd,
                                 left=torch.from_numpy(left).cuda() if mode > 0 else None,
                                 right=torch.from_numpy(right).cuda() if mode < 2 else None, out=out))
                meta.append((k, mode, fd, left, right))
    h = W.weno_init(None)
    W.weno_cross_eval(h, dinsts, sets)
    W.weno_sync(h)
    for s, (k, mode, fd, left, right) in zip(sets, meta):
        if rng.random() > 0.15:
            continue
        inst = insts[k]
        li = rng.integers(left.shape[0])
        ri = rng.integers(right.shape[0])
        ref = oracle_out(inst, mode, fd, left[li:li + 1], right[ri:ri + 1])
        got = s["out"][:, li:li + 1, :, ri:ri + 1].double().cpu().numpy()
        scale = np.abs(ref).max(axis=(1, 2, 3), keepdims=True)
        assert np.isfinite(got).all()
        assert (np.abs(got - ref) <= 2e-3 * scale + 1e-3).all(), (k, mode, fd, float(np.abs(got - ref).max()))
    W.weno_destroy(h)


def _uneven_workload():
    insts = [make_instance(31, [24, 40, 18], [5, 7], (O.PERIODIC,) * 2),
             make_instance(32, [36, 20, 30], [9, 4], (O.REFLECTIVE,) * 2)]
    allsets, allrefs = [], []
    for k, inst in enumerate(insts):
        for fp64 in (True,):
            sets, refs = make_sets(inst, k, 120 + k, fp64)
            allsets += sets
            allrefs += [(k,) + r for r in refs]
    return insts, allsets, allrefs


def test_cross_graph_replays_with_new_index_contents(W):
    """WENO_CROSS_GRAPH: the first call captures, later calls with the same
    descriptors replay; the index arrays are changed in place between calls and
    every replay equals a direct evaluation of the same inputs (bitwise: same
    kernels, same configuration)."""
    insts, sets, refs = _uneven_workload()
    dinsts = [dev_instance(i) for i in insts]
    h = W.weno_init(None)
    rng = np.random.default_rng(8)
    for rep in range(3):
        if rep:
            for s, (k, mode, fd, left, right) in zip(sets, refs):
                n = insts[k]["n"]
                if s["left"] is not None:
                    s["left"].copy_(torch.from_numpy(np.stack([rng.integers(0, n[m], s["left"].shape[0])
                                                               for m in range(mode)], 1).astype(np.int32)))
                if s["right"] is not None:
                    s["right"].copy_(torch.from_numpy(np.stack([rng.integers(0, n[m], s["right"].shape[0])
                                                                for m in range(mode + 1, 3)], 1).astype(np.int32)))
        W.weno_cross_eval(h, dinsts, sets, fp64_check=True, graph=True)
        W.weno_sync(h)
        got = [s["out"].clone() for s in sets]
        W.weno_cross_eval(h, dinsts, sets, fp64_check=True)
        W.weno_sync(h)
        for g, s in zip(got, sets):
            assert torch.equal(g, s["out"])
        # and the values are the oracle's
        k, mode, fd, _, _ = refs[4]
        left = sets[4]["left"].cpu().numpy() if sets[4]["left"] is not None else np.zeros((1, 0), np.int32)
        right = sets[4]["right"].cpu().numpy() if sets[4]["right"] is not None else np.zeros((1, 0), np.int32)
        ref = oracle_out(insts[k], mode, fd, left, right)
        assert (np.abs(got[4].cpu().numpy() - ref) <= tol_fp64(ref, insts[k])).all()
    W.weno_destroy(h)


def test_autotune_picks_a_compiled_variant_and_keeps_results(W, tmp_path):
    """The tuner times every variant; FP64 evaluation with the tuned variant is
    bitwise the default one's (the per-sample arithmetic does not depend on the
    chunking), and the choice survives a save / load through the cache file."""
    insts, sets, refs = _uneven_workload()
    dinsts = [dev_instance(i) for i in insts]
    h0 = W.weno_init(None)
    W.weno_cross_eval(h0, dinsts, sets, fp64_check=True)
    W.weno_sync(h0)
    base = [s["out"].clone() for s in sets]
    h = W.weno_init(None)
    choice, ms = W.weno_cross_autotune(h, dinsts, sets, fp64_check=True, reps=1)
    print("tuned:", choice, "%.3f ms" % ms)
    assert choice[0] in (128, 256) and choice[1] in (32, 64, 128) and 1 <= choice[2] <= 4 and ms > 0
    W.weno_cross_eval(h, dinsts, sets, fp64_check=True)
    W.weno_sync(h)
    for b, s in zip(base, sets):
        assert torch.equal(b, s["out"])
    path = str(tmp_path / "tune.txt")
    W.weno_tune_save(h, path)
    h2 = W.weno_init(None)
    assert W.weno_tune_load(h2, path) >= 1
    for x in (h0, h, h2):
        W.weno_destroy(x)
