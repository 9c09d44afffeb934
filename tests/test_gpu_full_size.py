"""The hypersonic gas at its full size (9,144,283 particles, 150,000 cells)
through dsmc_step on the VHS, look-up and Jager paths, as the bench runs
them (the neural path's full-size case sits with the other neural tests).

Every path: perm, cell_start, the step's pair, candidate and round counts
and every pair (cell, candidate, particles, round) bit-exact against the
oracle; every cell's momentum and energy after moment matching within 1e-12
of its pre-collision moments.

VHS (Sec. 2.1; FP64 throughout): every particle's velocity within 1e-12 of
the oracle's collide and moment matching.

Look-up and Jager: the oracle cannot redo millions of exact chi in seconds,
so pairs whose two particles collide only once in the step are sampled.
Their inputs are the sorted pre-collision state, and their final relative
velocity is the pair's post-collision one scaled by moment matching's
alpha > 0, so its direction is the collide's.  Moving chi by d moves that
direction by a chord of at most |d|; the gates are those of the per-kernel
tests:
  look-up -- within 2e-5 rad (FP32 interpolation) plus ROT_K = 4e-6 rad
    (the FP32 rotation) plus S of the oracle's collide with chi by FP64
    interpolation in the same table.  S bounds what the FP32 rounding of the
    pair's table coordinates does to the interpolant: x = sqrt(U1) (nb - 1)
    is within (nb - 1) 2.5 2^-24 of its FP64 value, and y = (ln E_r - ln E_min)
    / d(ln E) within (nE - 1) 2^-22 (logf's ulp and the FP32 E_r at
    ln E_r <= 11, the product's rounding), i.e. both within 2^-22 of the
    normalised coordinate; S is the interpolant's largest change over
    2^-21 (twice that) along each axis, from the oracle's lookup.  On a fine
    table that term matters where chi is steep (orbiting, low E_r): on the
    512 x 512 table it reaches 1e-3 rad there and stays near 1e-7 elsewhere;
  Jager -- within 1e-5 |chi| + 1e-6 (1 + depth/E_r) rad of the oracle's
    FP64 rotation by its chi at the kernel's FP32 inputs (b from tag 4, E_r
    from the FP32 g^2): the gate of the chi table's nodes, which the same
    device code fills.  Below the well depth the FP32 integrand
    G = G0 - dG cancels terms of size |V|/E_r, so its absolute rounding
    error, and chi's, grows by that factor; the full gas has pairs down to
    E_r/k_B of a few K, far below the chi batch's sample (g >= 300 m/s,
    E_r/k_B >= 108 K).  A pair outside the gate that the FP32 rounding of
    its inputs alone moves by more than 1e-6 rad is ill-conditioned (near
    orbiting): counted, at most 1e-3 of the sample.
A slack of 1e-11 vmax / g covers the FP64 rounding of the update and of
moment matching on a pair of relative speed g.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2602_21244_gb300 import workloads as W

from gpu_util import KB, ctx, cuda, host, pairs_round_of, sel_host

pytestmark = pytest.mark.gpu

JP = W.JAGER_SYNTHETIC_AR
LO, HI = math.log(5.0), math.log(6.0e4)
ROT_K = 4e-6
STEP = 3


def _full_size_step(model, kind, path_kw=lambda w: {}):
    """One step of the full hypersonic gas through dsmc_step (path_kw(w):
    the path's arguments for workload w); the oracle's sort, moments and
    selection beside it, checked bit for bit."""
    from paper_2602_21244_gb300 import dsmc as D
    w = W.hypersonic()
    w = dict(w, gas=dict(w["gas"], model=model))
    n, nc = len(w["cell_id"]), w["n_cells"]
    gas_o = O.make_gas(**w["gas"])
    sg0 = O.sigma_g_max_init(gas_o, w["T_cell"], 5.0)
    perm, cs, sx, sy, sz = O.sort_cells(w["cell_id"], w["vx"], w["vy"], w["vz"], nc)
    mom = O.cell_moments(cs, sx, sy, sz)
    pr = O.select_pairs(gas_o, cs, sx, sy, sz, sg0, STEP, capacity=1 << 24)
    C = ctx()
    st = D.StepState(C, n, nc, 1 << 24)
    st.sigma_g_max.copy_(cuda(sg0))
    st.cell_id.copy_(cuda(w["cell_id"])); st.vx.copy_(cuda(w["vx"]))
    st.vy.copy_(cuda(w["vy"])); st.vz.copy_(cuda(w["vz"]))
    C.step(D.make_gas(w["gas"]), D.make_path(kind, **path_kw(w)), st, STEP)
    assert C.sync_status() == 0
    assert np.array_equal(host(st.perm), perm) and np.array_equal(host(st.cell_start), cs)
    inf = st.info_host()
    assert inf["n_pairs"] == pr["n_pairs"] and inf["n_candidates"] == pr["n_cand"]
    assert inf["n_rounds"] == pr["n_rounds"]
    sh = sel_host(st.sel)
    p = sh["pairs"]
    order = np.lexsort((p[:, 3], p[:, 2]))
    assert np.array_equal(p[order, 0], pr["i"]) and np.array_equal(p[order, 1], pr["j"])
    assert np.array_equal(p[order, 3], pr["m"]) and np.array_equal(pairs_round_of(sh)[order], pr["round"])
    got = [host(a) for a in (st.svx, st.svy, st.svz)]
    return dict(gas_o=gas_o, cs=cs, s=(sx, sy, sz), mom=mom, pr=pr, got=got, n=n)


def check_conservation(cs, mom, got, s):
    """Every cell's momentum and energy after moment matching against its
    pre-collision moments."""
    m1 = O.cell_moments(cs, *got)
    nn = np.maximum(mom[:, 0], 1)
    vmax = max(np.abs(a).max() for a in s)
    assert np.all(np.abs(m1[:, 1:4] - mom[:, 1:4]) <= 1e-12 * nn[:, None] * vmax)
    e0 = mom[:, 4] + (mom[:, 1] ** 2 + mom[:, 2] ** 2 + mom[:, 3] ** 2) / nn
    e1 = m1[:, 4] + (m1[:, 1] ** 2 + m1[:, 2] ** 2 + m1[:, 3] ** 2) / nn
    assert np.all(np.abs(e1 - e0) <= 1e-12 * np.maximum(e0, 1e-300))


def once_sample(pr, n, k, seed):
    """Up to k pairs (candidate order) whose two particles collide only once
    in the step, as a pair dict."""
    cnt = np.bincount(np.concatenate([pr["i"], pr["j"]]), minlength=n)
    once = np.flatnonzero((cnt[pr["i"]] == 1) & (cnt[pr["j"]] == 1))
    pick = np.sort(np.random.default_rng(seed).choice(once, size=min(k, len(once)), replace=False))
    return dict(i=pr["i"][pick], j=pr["j"][pick], cell=pr["cell"][pick], m=pr["m"][pick], n_pairs=len(pick))


def directions(v, sub):
    """Unit relative velocity v_i - v_j of each sampled pair, and its norm."""
    d = np.stack([c[sub["i"]] - c[sub["j"]] for c in v], 1)
    g = np.linalg.norm(d, axis=1)
    return d / g[:, None], g


def direction_slack(s, g):
    return 1e-11 * max(np.abs(a).max() for a in s) / g


def lookup_sensitivity(table, gas_o, sub, s, bmax_A, h=2.0 ** -21):
    """S per sampled pair: the largest change of the oracle's interpolant
    when the normalised coordinates b/b_max and (ln E_r - ln E_min) /
    (ln E_max - ln E_min) move by h each (b from tag 4, E_r from the pair's
    pre-collision relative velocity)."""
    *_, vr, bA = O.collide_given_chi(gas_o, sub, STEP, np.zeros(max(sub["n_pairs"], 1)), *s, want_vr=True)
    bt = bA / bmax_A
    lnE = np.log(O.e_kelvin(W.M_AR, np.linalg.norm(vr, axis=1)))
    out = np.zeros(len(bt))
    for q, (a, e) in enumerate(zip(bt, lnE)):
        c = O.chi_lookup(table, LO, HI, a, e)

        def dev(a_, e_):
            return abs(O.chi_lookup(table, LO, HI, a_, e_) - c)
        out[q] = max(dev(a + h, e), dev(a - h, e)) + max(dev(a, e + h * (HI - LO)), dev(a, e - h * (HI - LO)))
    return out


def check_table_directions(got, ref, sub, s, S):
    """Look-up path: the step's directions against the oracle's collide
    (ref: its post-collision velocities of the sampled pairs; S: the
    coordinate-rounding term per pair)."""
    u, g = directions(got, sub)
    u_o, _ = directions(ref, sub)
    err = np.linalg.norm(u - u_o, axis=1)
    base = 2e-5 + ROT_K + direction_slack(s, g)
    gate = base + S
    assert np.all(err <= gate), (err / gate).max()
    return (err / gate).max(), int(np.sum(err > base))


def _sensitivity(P, b, E, h=1e-4):
    s1 = abs(O.chi(P, b * (1 + h), E) - O.chi(P, b * (1 - h), E)) / (2 * h)
    s2 = abs(O.chi(P, b, E * (1 + h) ** 2) - O.chi(P, b, E * (1 - h) ** 2)) / (2 * h)
    return s1 + s2


def kernel_inputs(gas_o, sub, s):
    """Each sampled pair's chi inputs as the Jager collide forms them: b
    (Angstrom, tag 4) rounded to FP32, E_r/k_B = FP32 (m / 4 k_B) times the
    FP32 g^2 of its pre-collision relative velocity."""
    *_, vr, bA = O.collide_given_chi(gas_o, sub, STEP, np.zeros(max(sub["n_pairs"], 1)), *s, want_vr=True)
    g2 = (vr ** 2).sum(1).astype(np.float32)
    E = (np.float32(W.M_AR / (4.0 * KB)) * g2).astype(np.float64)
    return bA.astype(np.float32).astype(np.float64), E


def check_jager_directions(got, gas_o, P, sub, s, max_ill_frac=1e-3):
    """Jager path: the step's directions against the oracle's FP64 rotation
    by its own chi at the kernel's FP32 inputs."""
    b, E = kernel_inputs(gas_o, sub, s)
    chi_ref = O.chi_many(P, b, E)
    ref = O.collide_given_chi(gas_o, sub, STEP, chi_ref, *s)
    u, g = directions(got, sub)
    u_o, _ = directions(ref, sub)
    err = np.linalg.norm(u - u_o, axis=1)
    depth = -min(O.pot_V(P, r) for r in np.linspace(3.0, 6.0, 601))
    gate = 1e-5 * np.abs(chi_ref) + 1e-6 * (1.0 + depth / E) + direction_slack(s, g)
    bad, ill = [], []
    for q in np.flatnonzero(err > gate):
        if _sensitivity(P, float(b[q]), float(E[q])) * 2.0 ** -24 > 1e-6:
            ill.append(q)
        else:
            bad.append((float(b[q]), float(E[q]), float(chi_ref[q]), float(err[q])))
    assert not bad, (len(bad), bad[:5])
    assert len(ill) <= max(3, max_ill_frac * sub["n_pairs"]), len(ill)
    gated = np.setdiff1d(np.arange(sub["n_pairs"]), ill)
    return len(ill), float(np.max(err[gated] / gate[gated])), int(np.sum(E < depth))


def test_full_size_vhs_step():
    from paper_2602_21244_gb300 import dsmc as D
    r = _full_size_step(0, D.PATH_VHS)
    cx, cy, cz = O.collide_vhs(r["gas_o"], r["pr"], STEP, *r["s"])
    ref = O.moment_match(r["cs"], r["mom"], cx, cy, cz)
    vmax = max(np.abs(a).max() for a in r["s"])
    for g_, r_ in zip(r["got"], ref):
        assert np.all(np.abs(g_ - r_) <= 1e-12 * np.maximum(np.abs(r_), vmax)), np.abs(g_ - r_).max()
    check_conservation(r["cs"], r["mom"], r["got"], r["s"])
    print(f"{r['pr']['n_pairs']} pairs")


def test_full_size_table_step():
    """The look-up path with the bench's table shape (512 x 512 nodes over
    b/b_max and ln E_r/k_B in [ln 5, ln 6e4]), the table built by the oracle
    and uploaded."""
    from paper_2602_21244_gb300 import dsmc as D
    tab = {}

    def path_kw(w):
        # b_max of the gas in Angstrom: the table's b axis
        tab["chi"] = O.chi_table(O.make_pot(JP), w["gas"]["b_max"] * 1e10, 512, 512, LO, HI).astype(np.float32)
        return dict(table=D.ChiTable(cuda(tab["chi"]), LO, HI))

    r = _full_size_step(1, D.PATH_TABLE, path_kw)
    table = tab["chi"]
    sub = once_sample(r["pr"], r["n"], 20000, seed=43)
    ref = O.collide_table(r["gas_o"], table, LO, HI, sub, STEP, *r["s"])
    S = lookup_sensitivity(table, r["gas_o"], sub, r["s"], r["gas_o"].b_max * 1e10)
    worst, steep = check_table_directions(r["got"], ref, sub, r["s"], S)
    check_conservation(r["cs"], r["mom"], r["got"], r["s"])
    print(f"{r['pr']['n_pairs']} pairs, {sub['n_pairs']} sampled, max error / gate {worst:.3f}, "
          f"{steep} beyond 2e-5 + ROT_K (steep chi)")


def test_full_size_jager_step():
    from paper_2602_21244_gb300 import dsmc as D
    r = _full_size_step(1, D.PATH_JAGER, lambda w: dict(pot=D.make_potential(JP), n_nodes=32))
    sub = once_sample(r["pr"], r["n"], 10000, seed=47)
    ill, worst, below = check_jager_directions(r["got"], r["gas_o"], O.make_pot(JP), sub, r["s"])
    check_conservation(r["cs"], r["mom"], r["got"], r["s"])
    print(f"{r['pr']['n_pairs']} pairs, {sub['n_pairs']} sampled ({below} below the well depth), "
          f"{ill} ill-conditioned, max error / gate of the others {worst:.3f}")
