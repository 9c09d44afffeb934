"""The look-up path (Sec. 3.4.5): chi table built on the GPU with the exact
chi, and the pair update with chi by bilinear interpolation in a table,
through the C ABI against the FP64 oracle (oracle/dsmc_oracle.c:
or_chi_table, or_chi_lookup, or_collide_table, pinned in
test_oracle_pins.py).

Gates: table nodes as the chi batch (1e-5 |chi| + 1e-6, a few
ill-conditioned nodes allowed: the kernel takes b and E in FP32), with the
absolute term 1e-6 (1 + depth/E): below the well depth the FP32 integrand
G = G0 - dG cancels terms of size |V|/E, so its absolute rounding error,
and that of chi, grows by that factor (at the table's lowest energy, 5 K,
depth/E = 29); the
collide with one uploaded table: each pair's chi within 2e-5 rad of the
oracle's FP64 interpolation (FP32 coordinates and weights), velocities
within the compounded effect, pair energy and momentum exact.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2602_21244_gb300 import workloads as W

from gpu_util import KB, ctx, cuda, gpu_step_pieces, host, sel_host, torch

pytestmark = pytest.mark.gpu

JP = W.JAGER_SYNTHETIC_AR
LO, HI = math.log(5.0), math.log(6.0e4)


def _gas():
    return dict(mass=W.M_AR, d_ref=4.17e-10, omega=0.81, T_ref=273.0, fn_over_vc=1.0, dt=1.0, model=1,
                b_max=1.2e-9)


def test_chi_table_hard_sphere_closed_form():
    from paper_2602_21244_gb300 import dsmc as D
    C = ctx()
    t = C.chi_table_build(D.make_gas(_gas()), D.make_potential(W.HARD_SPHERE_AR), nb=65, nE=9, lnE_min=LO,
                          lnE_max=HI)
    assert C.sync_status() == 0
    T = host(t.chi)
    b = (np.arange(65) * 12.0 / 64).astype(np.float32).astype(np.float64)
    want = np.where(b < 3.6, 2 * np.arccos(np.minimum(b / 3.6, 1.0)), 0.0)
    assert np.abs(T - want[None, :]).max() <= 1e-5 * np.pi + 1e-6


def test_chi_table_jager_matches_oracle():
    from paper_2602_21244_gb300 import dsmc as D
    C = ctx()
    nb, nE = 33, 17
    t = C.chi_table_build(D.make_gas(_gas()), D.make_potential(JP), nb=nb, nE=nE, lnE_min=LO, lnE_max=HI,
                          n_nodes=128)
    assert C.sync_status() == 0
    T = host(t.chi)
    ref = O.chi_table(O.make_pot(JP), 12.0, nb, nE, LO, HI)
    P = O.make_pot(JP)
    bad, ill = [], 0
    depth = -min(O.pot_V(P, r) for r in np.linspace(3.0, 6.0, 301))
    for j in range(nE):
        E = math.exp(LO + j * (HI - LO) / (nE - 1))
        for i in range(nb):
            err = abs(T[j, i] - ref[j, i])
            if err <= 1e-5 * abs(ref[j, i]) + 1e-6 * (1.0 + depth / E):
                continue
            b = 12.0 * i / (nb - 1)
            h = 1e-4
            sens = (abs(O.chi(P, b * (1 + h), E) - O.chi(P, b * (1 - h), E)) +
                    abs(O.chi(P, b, E * (1 + h)) - O.chi(P, b, E * (1 - h)))) / (2 * h)
            if sens * 2.0 ** -24 > 1e-6:
                ill += 1
            else:
                bad.append((i, j, ref[j, i], T[j, i]))
    assert not bad, bad[:5]
    assert ill <= 3


def test_collide_table_matches_oracle():
    from paper_2602_21244_gb300 import dsmc as D
    w = W.hypersonic(scale=0.06)
    gas = O.make_gas(**w["gas"])
    # one table for both sides: the oracle's, uploaded
    table = O.chi_table(O.make_pot(JP), w["gas"]["b_max"] * 1e10, 65, 49, LO, HI).astype(np.float32)
    sg0 = O.sigma_g_max_init(gas, w["T_cell"], 5.0)
    perm, cs, sx, sy, sz = O.sort_cells(w["cell_id"], w["vx"], w["vy"], w["vz"], w["n_cells"])
    pr = O.select_pairs(gas, cs, sx, sy, sz, sg0, 4, capacity=1 << 22)
    rx, ry, rz, chi_ref = O.collide_table(gas, table, LO, HI, pr, 4, sx, sy, sz, want_chi=True)
    Dg, srt, mom, sg, sel = gpu_step_pieces(w, sg0, step=4)
    C = ctx()
    sh = sel_host(sel)
    assert sh["n_pairs"] == pr["n_pairs"]
    chi_gpu = torch().zeros(max(sh["n_pairs"], 1), dtype=torch().float32, device="cuda")
    tab = D.ChiTable(cuda(table), LO, HI)
    C.collide_table(Dg, tab, 4, sel, srt["svx"], srt["svy"], srt["svz"], chi_out=chi_gpu)
    assert C.sync_status() == 0
    p = sh["pairs"]
    order = np.lexsort((p[:, 3], p[:, 2]))
    cg = host(chi_gpu)[:sh["n_pairs"]][order]
    err = np.abs(cg - chi_ref)
    # later pairs see velocities already moved by earlier chi differences
    assert np.mean(err > 2e-5) < 2e-3 and err.max() < 1e-2, (np.mean(err > 2e-5), err.max())
    dv = np.sqrt((host(srt["svx"]) - rx) ** 2 + (host(srt["svy"]) - ry) ** 2 + (host(srt["svz"]) - rz) ** 2)
    c8000 = math.sqrt(2 * KB * 8000.0 / W.M_AR)
    assert np.mean(dv > 1e-4 * c8000) < 2e-3, (np.mean(dv > 1e-4 * c8000), dv.max())
    e0 = np.sum(sx ** 2 + sy ** 2 + sz ** 2)
    e1 = np.sum(host(srt["svx"]) ** 2 + host(srt["svy"]) ** 2 + host(srt["svz"]) ** 2)
    assert abs(e1 / e0 - 1) < 1e-12
    assert abs(np.sum(host(srt["svx"])) - np.sum(sx)) < 1e-9 * np.abs(sx).sum()


def test_table_path_step_graph_equals_direct_step():
    from paper_2602_21244_gb300 import dsmc as D
    T = torch()
    w = W.hypersonic(scale=0.1)
    C = ctx()
    n, nc = len(w["cell_id"]), w["n_cells"]
    gas = D.make_gas(dict(w["gas"], model=1))
    tab = C.chi_table_build(gas, D.make_potential(JP), nb=128, nE=128, lnE_min=LO, lnE_max=HI)
    path = D.make_path(D.PATH_TABLE, table=tab)
    sts = [D.StepState(C, n, nc, 1 << 21) for _ in range(2)]
    for st in sts:
        C.sigma_g_max_init(gas, cuda(w["T_cell"]), 5.0, out=st.sigma_g_max)
    s = T.cuda.Stream()
    T.cuda.synchronize()
    C.step_graph_capture(gas, path, sts[1], s)
    for step in (0, 1):
        for st in sts:
            st.cell_id.copy_(cuda(w["cell_id"])); st.vx.copy_(cuda(w["vx"]))
            st.vy.copy_(cuda(w["vy"])); st.vz.copy_(cuda(w["vz"]))
        T.cuda.synchronize()
        C.step(gas, path, sts[0], step)
        C.step_graph_launch(step, s)
        T.cuda.synchronize()
        assert C.sync_status() == 0
        a, b = sts
        assert a.info_host() == b.info_host()
        for k in ("perm", "cell_start", "svx", "svy", "svz", "sigma_g_max", "mom"):
            assert T.equal(getattr(a, k), getattr(b, k)), (step, k)
    # conservation after moment matching
    st = sts[0]
    m = host(C.cell_moments(st.cell_start, st.svx, st.svy, st.svz))
    assert np.allclose(m[:, 1:4], host(st.mom)[:, 1:4], rtol=0, atol=1e-9 * 3000 * np.maximum(m[:, :1], 1))
    rel = np.abs(m[:, 4] - host(st.mom)[:, 4]) / np.maximum(host(st.mom)[:, 4], 1e-300)
    assert rel.max() <= 1e-12
