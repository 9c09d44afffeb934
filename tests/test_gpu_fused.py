"""The fused collision step (dsmc_step_fused): one kernel per cell group
takes the sorted particles through moments, NTC selection, rounds, pair
updates and moment matching in shared memory.

It runs the unfused kernels' arithmetic through the same device functions,
so it must equal dsmc_step bit for bit (sorted velocities, moments,
(sigma g)_max, pair and candidate counts, rounds) -- on the test gases, on
cells too large for a shared-memory batch (global-memory fallback), on long
runs of empty cells (batches cut at 128 cells) and over several steps.  It
is also held directly against the FP64 oracle: the VHS step within the
whole-step tolerance of the unfused path (1e-12 relative), the look-up step
within the look-up collide's gates.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2602_21244_gb300 import workloads as W

from gpu_util import KB, ctx, cuda, host, torch

pytestmark = pytest.mark.gpu

JP = W.JAGER_SYNTHETIC_AR
LO, HI = math.log(5.0), math.log(6.0e4)
FIELDS = ("perm", "cell_start", "svx", "svy", "svz", "mom", "sigma_g_max")


def _gas_dict(w, path):
    # the look-up path collides with sigma = pi b_max^2 (model 1), VHS with model 0
    return dict(w["gas"], model=1 if path == "table" else 0)


def _path(D, C, gas, path):
    if path == "vhs":
        return D.make_path(D.PATH_VHS)
    tab = C.chi_table_build(gas, D.make_potential(JP), nb=128, nE=128, lnE_min=LO, lnE_max=HI)
    return D.make_path(D.PATH_TABLE, table=tab)


def _states(w, gas, capacity=1 << 22):
    from paper_2602_21244_gb300 import dsmc as D
    C = ctx()
    n, nc = len(w["cell_id"]), w["n_cells"]
    sts = [D.StepState(C, n, nc, capacity) for _ in range(2)]
    for st in sts:
        C.sigma_g_max_init(gas, cuda(w["T_cell"]), 5.0, out=st.sigma_g_max)
        _load(st, w["cell_id"], w["vx"], w["vy"], w["vz"])
    return sts


def _load(st, cid, vx, vy, vz):
    st.cell_id.copy_(cuda(cid)); st.vx.copy_(cuda(vx)); st.vy.copy_(cuda(vy)); st.vz.copy_(cuda(vz))


def _assert_same(a, b, tag):
    T = torch()
    assert a.info_host() == b.info_host(), (tag, a.info_host(), b.info_host())
    for k in FIELDS:
        x, y = getattr(a, k), getattr(b, k)
        if k in ("svx", "svy", "svz", "perm"):   # slots past the last cell are unspecified
            n = int(host(a.cell_start)[-1])
            x, y = x[:n], y[:n]
        assert T.equal(x, y), (tag, k)


def _big_cells(seed=5):
    """Cells of very different sizes: one of 3000 particles (beyond a
    shared-memory batch), one of 1000 (within it, but with more candidates
    than a batch holds), one of 700, 1500 empty cells in a row, and small
    cells of 0..24 particles; Maxwellian argon at 300..3000 K.  F_N/V_c is
    set so that the 3000-particle cell draws about 3e4 NTC candidates with
    sigma = pi b_max^2."""
    rng = np.random.default_rng(seed)
    n_cells = 2400
    counts = rng.integers(0, 25, n_cells)
    counts[300:1800] = 0
    counts[50] = 3000
    counts[120] = 1000
    counts[2000] = 700
    T = 300.0 + 2700.0 * rng.random(n_cells)
    cid = np.repeat(np.arange(n_cells, dtype=np.int32), counts)
    sig = np.sqrt(KB * T[cid] / W.M_AR)
    v = rng.standard_normal((len(cid), 3)) * sig[:, None]
    v[:, 0] += 500.0
    p = rng.permutation(len(cid))
    gas = dict(W.hypersonic(scale=0.05)["gas"], model=1)
    sg = O.sigma_g_max_init(O.make_gas(**gas), T, 5.0)
    gas["fn_over_vc"] = 3e4 / (0.5 * 3000 * 2999 * sg[50] * gas["dt"])
    return dict(n_cells=n_cells, cell_id=cid[p].astype(np.int32), vx=v[p, 0].copy(), vy=v[p, 1].copy(),
                vz=v[p, 2].copy(), T_cell=T, gas=gas)


def _workload(name):
    if name == "couette":
        return W.couette()
    if name == "cavity40":
        return W.cavity(nx=40, ny=40)
    if name == "hyper01":
        return W.hypersonic(scale=0.1)
    return _big_cells()


@pytest.mark.parametrize("path", ["vhs", "table"])
@pytest.mark.parametrize("name", ["couette", "cavity40", "hyper01", "big_cells"])
def test_fused_step_equals_unfused_bitwise(name, path):
    from paper_2602_21244_gb300 import dsmc as D
    C = ctx()
    w = _workload(name)
    gas = D.make_gas(_gas_dict(w, path))
    P = _path(D, C, gas, path)
    a, b = _states(w, gas)
    for step in (0, 1, 2):
        C.step(gas, P, a, step)
        C.step_fused(gas, P, b, step)
        assert C.sync_status() == 0
        _assert_same(a, b, (name, path, step))
        # the next step starts from the new state (sorted order, same cells)
        cid = np.repeat(np.arange(w["n_cells"], dtype=np.int32), np.diff(host(a.cell_start)))
        for st in (a, b):
            n = len(cid)
            _load(st, cid, host(st.svx)[:n], host(st.svy)[:n], host(st.svz)[:n])
    assert a.info_host()["n_pairs"] > 0


def test_fused_vhs_matches_oracle_step():
    from paper_2602_21244_gb300 import dsmc as D
    C = ctx()
    w = W.hypersonic(scale=0.1)
    gd = _gas_dict(w, "vhs")
    gas_o = O.make_gas(**gd)
    sg0 = O.sigma_g_max_init(gas_o, w["T_cell"], 5.0)
    ref = O.step(gas_o, w["cell_id"], w["vx"], w["vy"], w["vz"], w["n_cells"], sg0, 7, path="vhs",
                 capacity=1 << 22)
    st = D.StepState(C, len(w["cell_id"]), w["n_cells"], 1 << 20)
    st.sigma_g_max.copy_(cuda(sg0))
    _load(st, w["cell_id"], w["vx"], w["vy"], w["vz"])
    C.step_fused(D.make_gas(gd), D.make_path(D.PATH_VHS), st, 7)
    assert C.sync_status() == 0
    info = st.info_host()
    assert np.array_equal(host(st.perm), ref["perm"])
    assert np.array_equal(host(st.cell_start), ref["cell_start"])
    assert info["n_pairs"] == ref["pairs"]["n_pairs"] and info["n_rounds"] == ref["pairs"]["n_rounds"]
    assert info["n_candidates"] == ref["pairs"]["n_cand"]
    rel = np.abs(host(st.sigma_g_max) - ref["sgmax"]) / ref["sgmax"]
    assert rel.max() <= 4e-16
    # moments under the gates of the moments parity test
    m, mr = host(st.mom), ref["mom"]
    assert np.array_equal(m[:, 0], mr[:, 0])
    assert np.all(np.abs(m[:, 1:4] - mr[:, 1:4]) <= 1e-13 * np.maximum(mr[:, :1], 1) * 3000.0)
    assert np.all(np.abs(m[:, 4] - mr[:, 4]) <= 1e-12 * np.maximum(mr[:, 4], 1e-300))
    for a, k in ((st.svx, "vx"), (st.svy, "vy"), (st.svz, "vz")):
        got = host(a)
        assert np.all(np.abs(got - ref[k]) <= 1e-12 * np.maximum(np.abs(ref[k]), 3000.0)), np.abs(got - ref[k]).max()


def test_fused_table_matches_oracle():
    """The look-up step against the oracle's sort, moments, selection,
    look-up collide (one table for both sides: the oracle's, uploaded) and
    moment matching."""
    from paper_2602_21244_gb300 import dsmc as D
    C = ctx()
    w = W.hypersonic(scale=0.06)
    gd = _gas_dict(w, "table")
    gas_o = O.make_gas(**gd)
    table = O.chi_table(O.make_pot(JP), gd["b_max"] * 1e10, 65, 49, LO, HI).astype(np.float32)
    sg0 = O.sigma_g_max_init(gas_o, w["T_cell"], 5.0)
    perm, cs, sx, sy, sz = O.sort_cells(w["cell_id"], w["vx"], w["vy"], w["vz"], w["n_cells"])
    mom = O.cell_moments(cs, sx, sy, sz)
    pr = O.select_pairs(gas_o, cs, sx, sy, sz, sg0, 4, capacity=1 << 22)
    rx, ry, rz = O.collide_table(gas_o, table, LO, HI, pr, 4, sx, sy, sz)
    ox, oy, oz = O.moment_match(cs, mom, rx, ry, rz)
    st = D.StepState(C, len(w["cell_id"]), w["n_cells"], 1 << 20)
    st.sigma_g_max.copy_(cuda(sg0))
    _load(st, w["cell_id"], w["vx"], w["vy"], w["vz"])
    tab = D.ChiTable(cuda(table), LO, HI)
    C.step_fused(D.make_gas(gd), D.make_path(D.PATH_TABLE, table=tab), st, 4)
    assert C.sync_status() == 0
    info = st.info_host()
    assert np.array_equal(host(st.perm), perm)
    assert info["n_pairs"] == pr["n_pairs"] and info["n_rounds"] == pr["n_rounds"]
    assert np.array_equal(host(st.sigma_g_max), pr["sgmax"])
    gx, gy, gz = host(st.svx), host(st.svy), host(st.svz)
    dv = np.sqrt((gx - ox) ** 2 + (gy - oy) ** 2 + (gz - oz) ** 2)
    c8000 = math.sqrt(2 * KB * 8000.0 / W.M_AR)
    assert np.mean(dv > 1e-4 * c8000) < 2e-3, (np.mean(dv > 1e-4 * c8000), dv.max())
    # moment matching restores every cell's momentum and energy
    m1 = O.cell_moments(cs, gx, gy, gz)
    n = np.maximum(mom[:, 0], 1)
    assert np.all(np.abs(m1[:, 1:4] - mom[:, 1:4]) <= 1e-12 * n[:, None] * 3000.0)
    assert np.all(np.abs(m1[:, 4] - mom[:, 4]) <= 1e-12 * np.maximum(mom[:, 4], 1e-300))


def test_fused_large_cell_scratch_exhausted_is_reported():
    """The 3000-particle cell needs candidate scratch in the pair buffer; with
    16 slots it must record DSMC_ERR_CAPACITY, leave that cell uncollided and
    still finish the step (no fault)."""
    from paper_2602_21244_gb300 import dsmc as D
    C = ctx()
    w = _big_cells()
    gas = D.make_gas(_gas_dict(w, "vhs"))
    a, = _states(w, gas, capacity=16)[:1]
    C.step_fused(gas, D.make_path(D.PATH_VHS), a, 0)
    assert C.sync_status() == D.DSMC_ERR_CAPACITY
    cs = host(a.cell_start)
    m = host(a.mom)
    assert m[50, 0] == 3000 and m[2000, 0] == 700
    # the skipped cell keeps its particles' velocities up to moment matching
    m1 = O.cell_moments(cs, host(a.svx), host(a.svy), host(a.svz))
    assert np.allclose(m1[50], m[50], rtol=1e-12, atol=1e-9)


def test_fused_rejects_other_paths_and_empty_input():
    from paper_2602_21244_gb300 import dsmc as D
    C = ctx()
    w = W.couette()
    gas = D.make_gas(w["gas"])
    st = D.StepState(C, len(w["cell_id"]), w["n_cells"], 1 << 16)
    with pytest.raises(D.DsmcError) as e:
        C.step_fused(gas, D.make_path(D.PATH_JAGER, pot=D.make_potential(JP)), st, 0)
    assert e.value.code == D.DSMC_ERR_UNSUPPORTED
    # no particles: every cell's moments are zero, nothing is selected
    e0 = D.StepState(C, 0, 7, 16)
    e0.sigma_g_max.fill_(1e-12)
    C.step_fused(gas, D.make_path(D.PATH_VHS), e0, 0)
    assert C.sync_status() == 0
    assert np.all(host(e0.mom) == 0.0) and np.all(host(e0.cell_start) == 0)
    assert e0.info_host()["n_pairs"] == 0 and e0.info_host()["n_rounds"] == 0
