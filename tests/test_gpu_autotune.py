"""Launch-shape autotuning (dsmc_tune_set, dsmc_autotune_step, dsmc_autotune_chi).

A launch shape (threads per block, blocks per SM) must never change a
result: each tunable kernel hands whole work items to threads through a
grid-stride loop, so the arithmetic and its order do not depend on the grid.
These tests run the whole step of every path under several shapes and
require bit-identical outputs, check the argument rules of dsmc_tune_set, and
check that the autotuner keeps the fastest of the shapes it measured.
"""
import json
import os
import tempfile

import numpy as np
import pytest

from paper_2602_21244_gb300 import workloads as W

from gpu_util import ctx, cuda, torch, w_bits_tensor

pytestmark = pytest.mark.gpu

JP = W.JAGER_SYNTHETIC_AR
_W = {}


def _wl():
    if "w" not in _W:
        _W["w"] = W.hypersonic(scale=0.1, seed=5)
    return _W["w"]


def _table(D):
    if "table" not in _W:
        w = _wl()
        gas = D.make_gas(dict(w["gas"], model=1))
        _W["table"] = ctx().chi_table_build(gas, D.make_potential(JP), nb=96, nE=96)
    return _W["table"]


def _path(D, kind):
    wts = W.mlp_weights()
    bias = (np.random.default_rng(7).standard_normal(len(wts["bias"])) * 0.05).astype(np.float32)
    mlp = D.make_mlp(8, 128, 3, 3, 0, W.sigma_v(), 273.0, 1e-12)
    return D.make_path({"vhs": D.PATH_VHS, "jager": D.PATH_JAGER, "neural": D.PATH_NEURAL,
                        "table": D.PATH_TABLE}[kind],
                       pot=D.make_potential(JP), n_nodes=32, mlp=mlp,
                       w_bits=w_bits_tensor(wts["W_bits"]), bias=cuda(bias),
                       table=_table(D) if kind == "table" else None)


def _run_step(C, D, kind, st, step=2):
    w = _wl()
    T = torch()
    gas = D.make_gas(dict(w["gas"], model=0 if kind == "vhs" else 1))
    st.cell_id.copy_(cuda(w["cell_id"])); st.vx.copy_(cuda(w["vx"]))
    st.vy.copy_(cuda(w["vy"])); st.vz.copy_(cuda(w["vz"]))
    C.sigma_g_max_init(gas, cuda(w["T_cell"]), 5.0, out=st.sigma_g_max)
    path = _path(D, kind)
    C.step(gas, path, st, step)
    T.cuda.synchronize()
    assert C.sync_status() == 0
    out = {k: getattr(st, k).clone() for k in ("perm", "cell_start", "svx", "svy", "svz", "sigma_g_max",
                                                 "mom", "info")}
    inf = st.info_host()
    # the pair buffer and the round offsets are defined up to the step's counts
    # only, and the order of the pairs inside a round is unspecified: compare
    # each round's pairs sorted by (cell, candidate index)
    ro = st.round_offsets[:inf["n_rounds"] + 1].cpu().numpy()
    pr = st.pairs[:inf["n_pairs"]].cpu().numpy()
    rnd = np.repeat(np.arange(len(ro) - 1), np.diff(ro))
    out["pairs"] = T.from_numpy(pr[np.lexsort((pr[:, 3], pr[:, 2], rnd))])
    out["round_offsets"] = T.from_numpy(ro)
    return out


def _reset(C, D):
    for k in range(len(D.TUNE_KERNELS)):
        C.tune_set(k)


# non-default shapes: small blocks, few blocks per SM, large blocks
SHAPES = [
    {0: (128, 2), 1: (256, 1), 2: (256, 2), 3: (64, 1), 4: (32, 1), 6: (64, 1)},
    {0: (512, 4), 1: (256, 3), 2: (256, 5), 3: (128, 2), 4: (64, 2), 6: (128, 2)},
]


@pytest.mark.parametrize("kind", ["vhs", "jager", "neural", "table"])
def test_launch_shape_does_not_change_the_step(kind):
    from paper_2602_21244_gb300 import dsmc as D
    C = ctx()
    w = _wl()
    st = D.StepState(C, len(w["cell_id"]), w["n_cells"], 1 << 21)
    _reset(C, D)
    ref = _run_step(C, D, kind, st)
    try:
        for shapes in SHAPES:
            for k, (t, b) in shapes.items():
                C.tune_set(k, t, b)
                assert C.tune_get(k) == (t, b)
            got = _run_step(C, D, kind, st)
            for k in ref:
                assert torch().equal(ref[k], got[k]), (kind, shapes, k)
    finally:
        _reset(C, D)


def test_tune_set_rejects_bad_shapes_and_resets():
    from paper_2602_21244_gb300 import dsmc as D
    C = ctx()
    default = C.tune_get(D.TUNE_KERNELS.index("collide_jager"))
    assert default == (128, 0)  # full occupancy
    for args in [(7, 128, 1), (-1, 128, 1), (0, 48, 4), (0, 2048, 1), (1, 512, 4), (0, 128, 0),
                 (0, 128, 65), (4, 256, 1), (1, 128, 2), (2, 64, 1)]:
        with pytest.raises(D.DsmcError) as e:
            C.tune_set(*args)
        assert e.value.code == D.DSMC_ERR_ARG
    C.tune_set(4, 64, 3)
    assert C.tune_get(4) == (64, 3)
    C.tune_set(4)
    assert C.tune_get(4) == default
    for k in range(len(D.TUNE_KERNELS)):
        cands = C.tune_candidates(k)
        assert cands and all(t % 32 == 0 and 1 <= b <= 64 for t, b in cands)


@pytest.mark.parametrize("kind", ["jager", "neural", "table"])
def test_autotune_keeps_the_fastest_measured_shape(kind):
    from paper_2602_21244_gb300 import dsmc as D
    C = ctx()
    w = _wl()
    st = D.StepState(C, len(w["cell_id"]), w["n_cells"], 1 << 21)
    _reset(C, D)
    ref = _run_step(C, D, kind, st)
    gas = D.make_gas(dict(w["gas"], model=1))
    try:
        trials = C.autotune_step(gas, _path(D, kind), st, step=2, reps=2)
        assert C.sync_status() == 0
        tuned = {"gather", "moments", "moment_match"} | {"jager": {"collide_jager"}, "table": {"collide_table"},
                                                          "neural": set()}[kind]
        assert {t["kernel"] for t in trials} == tuned
        for name in tuned:
            mine = [t for t in trials if t["kernel"] == name]
            k = D.TUNE_KERNELS.index(name)
            assert len(mine) == len(C.tune_candidates(k))
            best = min(mine, key=lambda t: t["ms"])
            assert C.tune_get(k) == (best["threads"], best["blocks_per_sm"])
            assert all(t["ms"] > 0 for t in mine)
        # the tuned shapes give the same step, bit for bit
        got = _run_step(C, D, kind, st)
        for k in ref:
            assert torch().equal(ref[k], got[k]), (kind, k)
        # the cache stores and re-applies them per device and size bucket
        with tempfile.TemporaryDirectory() as td:
            path = os.path.join(td, "tune.json")
            D.tune_cache_store(path, C, len(w["cell_id"]), trials)
            saved = C.tuned_shapes()
            _reset(C, D)
            applied = D.tune_cache_apply(path, C, len(w["cell_id"]))
            assert set(applied) == tuned
            assert C.tuned_shapes() == saved
            cache = json.load(open(path))
            dev = torch().cuda.get_device_name(0)
            assert D.size_bucket(len(w["cell_id"])) in cache[dev]["gather"]
    finally:
        _reset(C, D)


def test_autotune_chi_batch():
    from paper_2602_21244_gb300 import dsmc as D
    C = ctx()
    b, g = W.chi_pairs(1 << 18, seed=3)
    gas = D.make_gas(dict(mass=W.M_AR, fn_over_vc=1.0, dt=1.0))
    pot = D.make_potential(JP)
    bt, gt = cuda(b), cuda(g)
    _reset(C, D)
    ref = C.jager_chi(gas, pot, bt, gt, n_nodes=32)
    try:
        trials = C.autotune_chi(gas, pot, bt, gt, n_nodes=32, reps=2)
        assert C.sync_status() == 0
        k = D.TUNE_KERNELS.index("jager_chi")
        assert len(trials) == len(C.tune_candidates(k))
        best = min(trials, key=lambda t: t["ms"])
        assert C.tune_get(k) == (best["threads"], best["blocks_per_sm"])
        got = C.jager_chi(gas, pot, bt, gt, n_nodes=32)
        torch().cuda.synchronize()
        assert torch().equal(ref, got)
    finally:
        _reset(C, D)
