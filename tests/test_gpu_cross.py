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


def _tt_state_subgrid(inst, stride):
    """The five fields of a TT instance at every stride-th point of each mode
    (an FP64 einsum of its FP32 cores), [5][k][j][i]."""
    out = []
    for f in range(5):
        g1, g2, g3 = [np.asarray(c, dtype=np.float64) for c in inst["cores"][f]]
        out.append(np.einsum("ia,jab,kb->kji", g1[::stride, 0, :], g2[::stride], g3[::stride, :, 0]))
    return np.stack(out)


def test_cross_eval_full_workload_fp64_check_and_fp32(W):
    """The benchmark's 64-instance workload (n in {64..512}, ranks 2..32), all 9
    sets per instance in one launch, once in FP64 check mode and once in FP32.
    A seeded subset of sets is compared sample by sample with the oracle: sets
    that sweep mode 0 or 2 in full, sets that sweep mode 1 on 3 x 3 (left, right)
    index pairs (whole fibers).  The subset always holds sets with max rank >= 16
    on modes of n >= 256, with the stencil along and across the fiber.  FP64
    check mode is held to tol_fp64 and FP32 to tol_fp32, with the state scales
    taken from every 4th point of each mode."""
    rng = np.random.default_rng(5)
    insts = [I.tt_instance(seed=I.MASTER_SEED + k) for k in range(64)]
    dinsts, meta = [], []
    for k, inst in enumerate(insts):
        inst["h"] = [1.0 / x for x in inst["n"]]
        inst["bc"] = ((O.PERIODIC, O.PERIODIC),) * 3
        inst["alpha"] = 3.0
        dinsts.append(dev_instance(inst))
        for mode in range(3):
            for fd in range(3):
                left, right = I.cross_index_sets(1000 * k + 10 * mode + fd, inst["n"], inst["r"], mode)
                meta.append((k, mode, fd, left, right))
    big = [i for i, (k, mode, fd, _, _) in enumerate(meta)
           if max(insts[k]["r"]) >= 16 and insts[k]["n"][mode] >= 256]
    along = [i for i in big if meta[i][1] == meta[i][2]]
    across = [i for i in big if meta[i][1] != meta[i][2]]
    assert along and across
    pick = set(rng.choice(along, size=min(3, len(along)), replace=False).tolist())
    pick |= set(rng.choice(across, size=min(3, len(across)), replace=False).tolist())
    pick |= set(rng.choice(len(meta), size=10, replace=False).tolist())
    h = W.weno_init(None)
    worst = {}
    for fp64 in (True, False):
        sets = []
        for k, mode, fd, left, right in meta:
            out = torch.zeros((5, left.shape[0], insts[k]["n"][mode], right.shape[0]),
                              dtype=torch.float64 if fp64 else torch.float32, device="cuda")
            sets.append(dict(instance=k, mode=mode, flux_dir=fd,
                             left=torch.from_numpy(left).cuda() if mode > 0 else None,
                             right=torch.from_numpy(right).cuda() if mode < 2 else None, out=out))
        W.weno_cross_eval(h, dinsts, sets, fp64_check=fp64)
        W.weno_sync(h)
        w = 0.0
        for i in sorted(pick):
            k, mode, fd, left, right = meta[i]
            inst = dict(insts[k])
            inst["U"] = _tt_state_subgrid(inst, 4)
            got_all = sets[i]["out"].double().cpu().numpy()
            if mode == 1:
                li = rng.choice(left.shape[0], size=min(3, left.shape[0]), replace=False)
                ri = rng.choice(right.shape[0], size=min(3, right.shape[0]), replace=False)
                pairs = [(a, b) for a in li for b in ri]
            else:
                pairs = [(None, None)]
            for a, b in pairs:
                if a is None:
                    ref = oracle_out(inst, mode, fd, left, right)
                    got = got_all
                else:
                    ref = oracle_out(inst, mode, fd, left[a:a + 1], right[b:b + 1])
                    got = got_all[:, a:a + 1, :, b:b + 1]
                assert np.isfinite(got).all()
                tol = tol_fp64(ref, inst) if fp64 else tol_fp32(inst)
                w = max(w, float((np.abs(got - ref) / tol).max()))
                assert (np.abs(got - ref) <= tol).all(), (fp64, k, mode, fd, insts[k]["n"], insts[k]["r"],
                                                          float(np.abs(got - ref).max()))
        worst["fp64" if fp64 else "fp32"] = w
        del sets
        torch.cuda.empty_cache()
    print("full workload, %d sets checked: worst error / tolerance %s" % (len(pick), worst))
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
