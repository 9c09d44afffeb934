"""The look-up path (Sec. 3.4.4): chi table built on the GPU with the exact
chi, and the pair update with chi by bilinear interpolation in a table,
through the C ABI against the FP64 oracle (oracle/dsmc_oracle.c:
or_chi_table, or_chi_lookup, or_collide_given_chi, pinned in
test_oracle_pins.py).

Gates: table nodes as the chi batch (1e-5 |chi| + 1e-6, a few
ill-conditioned nodes allowed: the kernel takes b and E in FP32), with the
absolute term 1e-6 (1 + depth/E): below the well depth the FP32 integrand
G = G0 - dG cancels terms of size |V|/E, so its absolute rounding error,
and that of chi, grows by that factor (at the table's lowest energy, 5 K,
depth/E = 29).

The collide forms the rotated direction in FP32 and scales it to the
pair's exact |v_r| in FP64.  Its velocities are compared, element by
element, with the oracle's FP64 rotation driven by the kernel's own chi
(or_collide_given_chi), under a bound derived from the FP32 steps: the
direction is within ROT_K = 4e-6 rad of the exact deflection (FP32
rounding of v_r, 2^-24 each component; the frame c, a, a few ulps; sincosf
of chi and eps, 2^-23; the azimuth formed in FP32 from a 2^-23-accurate
uniform, 2 pi (2^-23 + 2^-24 + 2^-25) = 1.3e-6 rad; the three-term sums,
4 ulps; about 2.4e-6 rad in all, doubled), so each particle of a pair moves
by at most ROT_K g / 2.  Later pairs of a particle see its earlier error:
with e_in = B_i + B_j the bound on the pair's input error, v_r -> v_r' is
Lipschitz with L = 3 + 2 g/q (q = |(v_ry, v_rz)|: Bird's frame turns at
rate 1/q), so B_i = B_j = e_in/2 + (L e_in + ROT_K g)/2 after the pair.
Each pair's chi is checked against the oracle's FP64 interpolation at the
pair's pre-collision state within 2e-5 rad (FP32 table coordinates and
weights) where that state is exact (both particles' first collision of the
step; every pair of the disjoint-pair case).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2602_21244_gb300 import workloads as W

from gpu_util import KB, c_ref, ctx, cuda, gpu_step_pieces, host, sel_host, torch

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


ROT_K = 4e-6


def _lookup_chi(table, bA, bmax_A, vr):
    """The oracle's FP64 interpolation at each pair's (b/b_max, ln E_r/k_B)."""
    g = np.sqrt((vr ** 2).sum(1))
    lnE = np.log(O.e_kelvin(W.M_AR, g))
    return np.array([O.chi_lookup(table, LO, HI, float(x), float(y)) for x, y in zip(bA / bmax_A, lnE)])


def _propagated_bound(pr, vr, n):
    """Per-particle bound on |v_gpu - v_oracle| after the pairs in candidate
    order (module docstring)."""
    B = np.zeros(n)
    g = np.sqrt((vr ** 2).sum(1))
    q = np.sqrt(vr[:, 1] ** 2 + vr[:, 2] ** 2)
    for p in range(pr["n_pairs"]):
        i, j = pr["i"][p], pr["j"][p]
        e_in = B[i] + B[j]
        L = 3.0 + 2.0 * g[p] / max(q[p], 1e-300) if e_in > 0 else 0.0
        B[i] = B[j] = 0.5 * e_in + 0.5 * (L * e_in + ROT_K * g[p])
    return B


def _gpu_table(D, table):
    return D.ChiTable(cuda(table), LO, HI)


def test_collide_table_matches_oracle():
    from paper_2602_21244_gb300 import dsmc as D
    w = W.hypersonic(scale=0.06)
    gas = O.make_gas(**w["gas"])
    bmax_A = w["gas"]["b_max"] * 1e10
    # one table for both sides: the oracle's, uploaded
    table = O.chi_table(O.make_pot(JP), bmax_A, 65, 49, LO, HI).astype(np.float32)
    sg0 = O.sigma_g_max_init(gas, w["T_cell"], 5.0)
    perm, cs, sx, sy, sz = O.sort_cells(w["cell_id"], w["vx"], w["vy"], w["vz"], w["n_cells"])
    pr = O.select_pairs(gas, cs, sx, sy, sz, sg0, 4, capacity=1 << 22)
    Dg, srt, mom, sg, sel = gpu_step_pieces(w, sg0, step=4)
    C = ctx()
    sh = sel_host(sel)
    assert sh["n_pairs"] == pr["n_pairs"]
    chi_gpu = torch().zeros(max(sh["n_pairs"], 1), dtype=torch().float32, device="cuda")
    C.collide_table(Dg, _gpu_table(D, table), 4, sel, srt["svx"], srt["svy"], srt["svz"], chi_out=chi_gpu)
    assert C.sync_status() == 0
    p = sh["pairs"]
    order = np.lexsort((p[:, 3], p[:, 2]))
    cg = host(chi_gpu)[:sh["n_pairs"]][order].astype(np.float64)
    rx, ry, rz, vr, bA = O.collide_given_chi(gas, pr, 4, cg, sx, sy, sz, want_vr=True)
    n = len(sx)
    B = _propagated_bound(pr, vr, n)
    got = [host(a) for a in (srt["svx"], srt["svy"], srt["svz"])]
    dv = np.sqrt(sum((g_ - r_) ** 2 for g_, r_ in zip(got, (rx, ry, rz))))
    slack = 1e-12 * np.maximum(np.sqrt(rx ** 2 + ry ** 2 + rz ** 2), c_ref(W.M_AR))
    assert np.all(dv <= B + slack), np.max(dv - B - slack)
    # chi per pair where the pair's pre-collision state is exact on both sides
    seen = np.zeros(n, bool)
    fresh = np.zeros(pr["n_pairs"], bool)
    for q_ in range(pr["n_pairs"]):
        i, j = pr["i"][q_], pr["j"][q_]
        fresh[q_] = not (seen[i] or seen[j])
        seen[i] = seen[j] = True
    ref_chi = _lookup_chi(table, bA[fresh], bmax_A, vr[fresh])
    assert np.abs(cg[fresh] - ref_chi).max() <= 2e-5, np.abs(cg[fresh] - ref_chi).max()
    e0 = np.sum(sx ** 2 + sy ** 2 + sz ** 2)
    e1 = np.sum(got[0] ** 2 + got[1] ** 2 + got[2] ** 2)
    assert abs(e1 / e0 - 1) < 1e-12
    assert abs(np.sum(got[0]) - np.sum(sx)) < 1e-9 * np.abs(sx).sum()
    print(f"{pr['n_pairs']} pairs ({fresh.sum()} first collisions), max |dv|/bound "
          f"{np.max(dv / (B + slack)):.3f}")


def test_collide_table_disjoint_pairs_rotation_bound():
    """Pairs that share no particle (one round, no dependencies; the pair list
    built by hand): every pair's velocities within the single-collision
    bound ROT_K g / 2 of the oracle's rotation by the kernel's chi, and its
    chi within 2e-5 rad of the oracle's interpolation.  Relative velocities
    include the directions where Bird's frame is degenerate or nearly so
    (v_r along x, and q/g = 1e-7, 1e-5, 1e-3)."""
    from paper_2602_21244_gb300 import dsmc as D
    T = torch()
    rng = np.random.default_rng(12)
    npairs = 20000
    bmax_A = 12.0
    table = O.chi_table(O.make_pot(JP), bmax_A, 65, 49, LO, HI).astype(np.float32)
    cm = rng.standard_normal((npairs, 3)) * 300.0 + np.array([2000.0, -100.0, 50.0])
    g = 300.0 * 50.0 ** rng.random(npairs)
    d = rng.standard_normal((npairs, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    for k, qg in enumerate([0.0, 1e-7, 1e-5, 1e-3]):
        for s_ in range(5):
            r = 4 * (5 * k + s_)
            for t in range(4):
                ang = rng.random() * 2 * np.pi
                d[r + t] = [(-1) ** t * math.sqrt(1 - qg * qg), qg * math.cos(ang), qg * math.sin(ang)]
    vi, vj = cm + 0.5 * g[:, None] * d, cm - 0.5 * g[:, None] * d
    v = np.empty((2 * npairs, 3))
    v[0::2], v[1::2] = vi, vj
    pidx = np.arange(npairs, dtype=np.int32)
    pr = dict(i=2 * pidx, j=2 * pidx + 1, cell=pidx // 64, m=pidx % 64, n_pairs=npairs)
    sel = dict(pairs=cuda(np.stack([pr["i"], pr["j"], pr["cell"], pr["m"]], 1).astype(np.int32)),
               deps=cuda(np.zeros(npairs, np.int32)),
               round_offsets=cuda(np.r_[0, npairs, np.zeros(1024, np.int64)].astype(np.int32)),
               info=cuda(np.array([npairs, npairs, 1], np.int64)))
    gas_d = D.make_gas(dict(mass=W.M_AR, d_ref=4.17e-10, omega=0.81, T_ref=273.0, fn_over_vc=1.0, dt=1.0,
                            seed=9, model=1, b_max=1.2e-9))
    gas_o = O.make_gas(W.M_AR, 4.17e-10, 0.81, 273.0, 1.0, 1.0, 9, model=1, b_max=1.2e-9)
    vx, vy, vz = (cuda(np.ascontiguousarray(v[:, c])) for c in range(3))
    chi_gpu = T.zeros(npairs, dtype=T.float32, device="cuda")
    C = ctx()
    C.collide_table(gas_d, _gpu_table(D, table), 6, sel, vx, vy, vz, chi_out=chi_gpu)
    assert C.sync_status() == 0
    cg = host(chi_gpu).astype(np.float64)
    rx, ry, rz, vr, bA = O.collide_given_chi(gas_o, pr, 6, cg, v[:, 0], v[:, 1], v[:, 2], want_vr=True)
    got = np.stack([host(vx), host(vy), host(vz)], 1)
    ref = np.stack([rx, ry, rz], 1)
    dv = np.linalg.norm(got - ref, axis=1)
    gp = np.repeat(g, 2)
    ratio = dv / (0.5 * ROT_K * gp + 1e-12 * np.maximum(np.linalg.norm(ref, axis=1), c_ref(W.M_AR)))
    assert ratio.max() <= 1.0, ratio.max()
    ref_chi = _lookup_chi(table, bA, bmax_A, vr)
    assert np.abs(cg - ref_chi).max() <= 2e-5, np.abs(cg - ref_chi).max()
    print(f"disjoint pairs: max |dv| / (ROT_K g/2) {ratio.max():.3f}")


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
