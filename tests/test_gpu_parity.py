"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Integer and index work (sort, selection, rounds) must match bit for bit;
floating point within the stated tolerances: FP64 paths 1e-12 relative,
FP32 Jager chi 1e-5 relative (+1e-6 rad) on well-conditioned pairs, bf16
MLP 2e-2 on normalised velocity; conservation after moment matching 1e-12.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2602_21244_gb300 import workloads as W

from gpu_util import (KB, c_ref, ctx, cuda, expected_buckets, expected_deps, gpu_step_pieces, host,
                      pairs_round_of, sel_host, torch, w_bits_tensor)

pytestmark = pytest.mark.gpu


_WORKLOADS = {
    "couette": lambda: W.couette(),
    "cavity40": lambda: W.cavity(nx=40, ny=40),
    "cavity200": lambda: W.cavity(nx=200, ny=200),   # the C2 gas at its stated size
    "hyper01": lambda: W.hypersonic(scale=0.1),
}

WL = {}


def wl(name):
    if name not in WL:
        WL[name] = _WORKLOADS[name]()
    return WL[name]


def oracle_sorted(w):
    return O.sort_cells(w["cell_id"], w["vx"], w["vy"], w["vz"], w["n_cells"])


# ------------------------------------------------------------------ tensor-core layout

@pytest.mark.parametrize("layout", [0, 1, 2, 3, 8, 10])
@pytest.mark.parametrize("N,K", [(16, 16), (128, 16), (16, 128), (128, 128), (256, 64), (32, 128)])
def test_tc_selftest_matches_matmul(N, K, layout):
    T = torch()
    rng = np.random.default_rng(N * 1000 + K)
    A = rng.standard_normal((128, K))
    B = rng.standard_normal((N, K))
    Ab, Bb = W.bf16_bits(A), W.bf16_bits(B)
    D = host(ctx().tc_selftest(w_bits_tensor(Ab), w_bits_tensor(Bb), layout=layout))
    ref = W.bf16_value(Ab) @ W.bf16_value(Bb).T
    assert np.abs(D - ref).max() <= 1e-4 * np.abs(ref).max() + 1e-5
    assert ctx().sync_status() == 0


# ------------------------------------------------------------------ sort / moments

@pytest.mark.parametrize("name", ["couette", "cavity40", "hyper01"])
def test_sort_bit_exact(name):
    w = wl(name)
    perm, cs, sx, sy, sz = oracle_sorted(w)
    C = ctx()
    out = C.sort_cells(cuda(w["cell_id"]), cuda(w["vx"]), cuda(w["vy"]), cuda(w["vz"]), w["n_cells"])
    assert C.sync_status() == 0
    assert np.array_equal(host(out["perm"]), perm)
    assert np.array_equal(host(out["cell_start"]), cs)
    assert np.array_equal(host(out["svx"]), sx) and np.array_equal(host(out["svz"]), sz)


def test_sort_edge_cases():
    C = ctx()
    T = torch()
    rng = np.random.default_rng(5)
    # big cell (> shared-memory capacity of the per-cell sort), empty cells, ragged tail
    cid = np.concatenate([np.full(3000, 2), rng.integers(0, 7, 501), np.full(5, 6)]).astype(np.int32)
    rng.shuffle(cid)
    v = [rng.standard_normal(len(cid)) for _ in range(3)]
    perm, cs, sx, _, _ = O.sort_cells(cid, *v, 9)
    out = C.sort_cells(cuda(cid), *[cuda(x) for x in v], 9)
    assert np.array_equal(host(out["perm"]), perm) and np.array_equal(host(out["cell_start"]), cs)
    assert np.array_equal(host(out["svx"]), sx)
    # no particles at all
    e = T.zeros(0, dtype=T.int32, device="cuda")
    ef = T.zeros(0, dtype=T.float64, device="cuda")
    out = C.sort_cells(e, ef, ef, ef, 4)
    assert host(out["cell_start"]).tolist() == [0, 0, 0, 0, 0]
    assert C.sync_status() == 0
    # a cell id out of range is reported on the device
    bad = cuda(np.array([0, 1, 9], np.int32))
    C.sort_cells(bad, *[cuda(np.zeros(3)) for _ in range(3)], 3)
    assert C.sync_status() == -1
    assert C.sync_status() == 0


@pytest.mark.parametrize("name", ["couette", "hyper01"])
def test_moments(name):
    w = wl(name)
    perm, cs, sx, sy, sz = oracle_sorted(w)
    ref = O.cell_moments(cs, sx, sy, sz)
    C = ctx()
    mom = host(C.cell_moments(cuda(cs), cuda(sx), cuda(sy), cuda(sz)))
    assert np.array_equal(mom[:, 0], ref[:, 0])
    scale = np.maximum(ref[:, 0], 1)[:, None] * 3000.0
    assert np.all(np.abs(mom[:, 1:4] - ref[:, 1:4]) <= 1e-13 * scale)
    assert np.all(np.abs(mom[:, 4] - ref[:, 4]) <= 1e-12 * np.maximum(ref[:, 4], 1e-300))


def _ragged_cells(seed=11):
    """Cells of sizes 0, 1, 2, 7, 33, 1023, 1024 (the coarsened integer unit
    starts there), 4099, and 29 small ones: 37 cells, not a multiple of the
    32-cell batch; mean velocities from 0 to 1e4 m/s over thermal spreads from
    1e-3 to 1e3 m/s, one cell with components of very different magnitude."""
    rng = np.random.default_rng(seed)
    sizes = [0, 1, 2, 7, 33, 1023, 1024, 4099] + list(rng.integers(0, 80, 29))
    vs, cs = [], [0]
    for q, N in enumerate(sizes):
        u = rng.uniform(-1e4, 1e4, 3) * (q % 3 == 0)
        sd = 10.0 ** rng.uniform(-3, 3)
        v = u + sd * rng.standard_normal((N, 3))
        if q == 6 and N:
            v[:, 2] *= 1e-9
        vs.append(v)
        cs.append(cs[-1] + N)
    v = np.concatenate(vs)
    return np.array(cs, np.int32), v[:, 0].copy(), v[:, 1].copy(), v[:, 2].copy()


def test_moments_and_match_ragged_cells():
    cs, vx, vy, vz = _ragged_cells()
    C = ctx()
    ref = O.cell_moments(cs, vx, vy, vz)
    mom = host(C.cell_moments(cuda(cs), cuda(vx), cuda(vy), cuda(vz)))
    assert C.sync_status() == 0
    assert np.array_equal(mom[:, 0], ref[:, 0])
    scale = np.maximum(ref[:, 0], 1)[:, None] * np.abs(np.stack([vx, vy, vz], 1)).max()
    assert np.all(np.abs(mom[:, 1:4] - ref[:, 1:4]) <= 1e-13 * scale)
    # Theta: 1e-12, plus the documented rounding of each component to the
    # cell's integer unit (the ulp of its largest component, 2^c coarser for
    # cells of 2^(10+c-1) or more particles): |dTheta| <= unit sqrt(3 n Theta) + 3 n unit^2 / 4
    n = ref[:, 0]
    vmax = np.array([np.abs(np.stack([vx, vy, vz], 1)[cs[k]:cs[k + 1]]).max() if cs[k + 1] > cs[k] else 0.0
                     for k in range(len(cs) - 1)])
    c = np.array([max(0, int(q).bit_length() - 10) for q in n])
    unit = np.spacing(vmax) * 2.0 ** c
    gate = 1e-12 * ref[:, 4] + unit * np.sqrt(3 * n * ref[:, 4]) + 0.75 * n * unit ** 2
    assert np.all(np.abs(mom[:, 4] - ref[:, 4]) <= gate)
    # match the moments of a perturbed copy back to the originals
    rng = np.random.default_rng(3)
    px, py, pz = (a * (1 + 0.1 * rng.standard_normal(len(a))) + 5.0 for a in (vx, vy, vz))
    rx, ry, rz = O.moment_match(cs, ref, px, py, pz)
    gx, gy, gz = cuda(px), cuda(py), cuda(pz)
    C.moment_match(cuda(cs), cuda(ref), gx, gy, gz)
    assert C.sync_status() == 0
    for g_, r_ in ((gx, rx), (gy, ry), (gz, rz)):
        g_ = host(g_)
        assert np.all(np.abs(g_ - r_) <= 1e-12 * np.maximum(np.abs(r_), np.abs(r_).max() * 1e-3))
    m2 = O.cell_moments(cs, host(gx), host(gy), host(gz))
    assert np.all(np.abs(m2[:, 1:4] - ref[:, 1:4]) <= 1e-12 * scale)
    # energy: 1e-12, plus the FP64 rounding of the stored velocities, which
    # moves Theta by up to 2 |v| 2^-53 sd per particle (n sd^2 in all)
    big = ref[:, 0] >= 2
    sd = np.sqrt(ref[:, 4] / np.maximum(ref[:, 0], 1))
    gate = 1e-12 + 8 * 2.0 ** -53 * vmax[big] / sd[big]
    assert np.all(np.abs(m2[big, 4] - ref[big, 4]) <= gate * ref[big, 4])


# ------------------------------------------------------------------ selection

def _sgmax0(w, gas):
    return O.sigma_g_max_init(gas, w["T_cell"], 5.0)


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("name,model", [("couette", 0), ("cavity40", 0), ("hyper01", 1), ("hyper01", 0)])
def test_select_bit_exact(name, model, order):
    """order 0: buckets are rounds; 1: claim levels (round + the cell's
    slack to the last round)."""
    w = dict(wl(name))
    w["gas"] = dict(w["gas"], model=model)
    gas = O.make_gas(**w["gas"])
    perm, cs, sx, sy, sz = oracle_sorted(w)
    sg0 = _sgmax0(w, gas)
    ref = O.select_pairs(gas, cs, sx, sy, sz, sg0, 3, capacity=1 << 22)
    _, srt, mom, sg, sel = gpu_step_pieces(w, sg0, step=3, order=order)
    assert ctx().sync_status() == 0
    sh = sel_host(sel)
    assert sh["n_pairs"] == ref["n_pairs"] and sh["n_cand"] == ref["n_cand"]
    assert sh["n_rounds"] == ref["n_rounds"]
    p = sh["pairs"]
    rr = pairs_round_of(sh)
    bucket = expected_buckets(ref, w["n_cells"], order)
    if order == 1 and name == "hyper01":
        assert not np.array_equal(bucket, ref["round"])   # there the levels do move pairs
    order_ = np.lexsort((p[:, 3], p[:, 2]))
    assert np.array_equal(p[order_, 0], ref["i"]) and np.array_equal(p[order_, 1], ref["j"])
    assert np.array_equal(p[order_, 2], ref["cell"]) and np.array_equal(p[order_, 3], ref["m"])
    assert np.array_equal(rr[order_], bucket)
    # inside a bucket the list is in cell order, candidate order within a cell
    ro_ = np.lexsort((ref["m"], ref["cell"], bucket))
    assert np.array_equal(p[:, 2], ref["cell"][ro_]) and np.array_equal(p[:, 3], ref["m"][ro_])
    # deps: 1-based buckets of the previous pair of each particle, derived
    # here from the oracle's pairs in candidate order and its rounds
    deps = host(sel["deps"])[:sh["n_pairs"]].view(np.uint32)
    assert np.array_equal(deps[order_], expected_deps(ref, bucket))
    rel = np.abs(host(sg) - ref["sgmax"]) / ref["sgmax"]
    assert rel.max() <= (0.0 if model == 1 else 4e-16)


def _dense_cells(seed=5):
    """Cells of 2, 40, 120, 383, 384, 385 and 600 particles (the FP32 staging
    holds 384) at a number density that gives a few hundred candidates per
    particle in the large cells, hence long chains of pairs sharing
    particles: 73 rounds (VHS) and 622 (hard spheres), seven and ten bits of
    round number."""
    rng = np.random.default_rng(seed)
    sizes = [2, 40, 120, 383, 384, 385, 600]
    cs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    n = int(cs[-1])
    s = math.sqrt(KB * 300.0 / W.M_AR)
    v = rng.standard_normal((n, 3)) * s + np.array([300.0, 0.0, 0.0])
    return cs, v[:, 0].copy(), v[:, 1].copy(), v[:, 2].copy()


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("model", [1, 0])
def test_select_bit_exact_dense_cells(model, order):
    cs, vx, vy, vz = _dense_cells()
    nc = len(cs) - 1
    gas_d = dict(mass=W.M_AR, d_ref=4.17e-10, omega=0.81, T_ref=273.0, fn_over_vc=1e21, dt=1e-7,
                 seed=7, model=model, b_max=1.2e-9)
    gas = O.make_gas(**gas_d)
    sg0 = O.sigma_g_max_init(gas, np.full(nc, 300.0), 3.0)
    ref = O.select_pairs(gas, cs, vx, vy, vz, sg0, 2, capacity=1 << 22)
    assert ref["n_rounds"] > 64, ref["n_rounds"]
    from paper_2602_21244_gb300 import dsmc as D
    C = ctx()
    sg = cuda(sg0).clone()
    sel = C.select_pairs(D.make_gas(gas_d), cuda(cs), cuda(vx), cuda(vy), cuda(vz), sg, 2, 1 << 22,
                         order=order)
    assert C.sync_status() == 0
    sh = sel_host(sel)
    assert sh["n_pairs"] == ref["n_pairs"] and sh["n_cand"] == ref["n_cand"]
    assert sh["n_rounds"] == ref["n_rounds"]
    p = sh["pairs"]
    rr = pairs_round_of(sh)
    bucket = expected_buckets(ref, nc, order)
    order_ = np.lexsort((p[:, 3], p[:, 2]))
    assert np.array_equal(p[order_, 0], ref["i"]) and np.array_equal(p[order_, 1], ref["j"])
    assert np.array_equal(p[order_, 3], ref["m"]) and np.array_equal(rr[order_], bucket)
    ro_ = np.lexsort((ref["m"], ref["cell"], bucket))
    assert np.array_equal(p[:, 2], ref["cell"][ro_]) and np.array_equal(p[:, 3], ref["m"][ro_])
    deps = host(sel["deps"])[:sh["n_pairs"]].view(np.uint32)
    assert np.array_equal(deps[order_], expected_deps(ref, bucket))
    rel = np.abs(host(sg) - ref["sgmax"]) / ref["sgmax"]
    assert rel.max() <= (0.0 if model == 1 else 4e-16)


def test_select_capacity_overflow_reported():
    w = wl("hyper01")
    gas = O.make_gas(**w["gas"])
    _, srt, mom, sg, sel = gpu_step_pieces(w, _sgmax0(w, gas), capacity=100)
    assert ctx().sync_status() == -3
    sh = sel_host(sel)
    assert sh["n_pairs"] > 100 and sh["n_rounds"] == 0


# ------------------------------------------------------------------ VHS + moment matching

def _tol_v(v_ref, scale):
    return 1e-12 * np.maximum(np.abs(v_ref), scale)


@pytest.mark.parametrize("name", ["couette", "hyper01"])
def test_collide_vhs_and_moment_match(name):
    w = dict(wl(name))
    w["gas"] = dict(w["gas"], model=0)
    gas = O.make_gas(**w["gas"])
    sg0 = _sgmax0(w, gas)
    ref = O.step(gas, w["cell_id"], w["vx"], w["vy"], w["vz"], w["n_cells"], sg0, 2, path="vhs",
                 capacity=1 << 22)
    from paper_2602_21244_gb300 import dsmc as D
    Dg, srt, mom, sg, sel = gpu_step_pieces(w, sg0, step=2)
    C = ctx()
    C.collide_vhs(Dg, 2, sel, srt["svx"], srt["svy"], srt["svz"])
    C.moment_match(srt["cell_start"], mom, srt["svx"], srt["svy"], srt["svz"])
    assert C.sync_status() == 0
    scale = 3000.0
    for a, b in zip((srt["svx"], srt["svy"], srt["svz"]), ("vx", "vy", "vz")):
        got = host(a)
        assert np.all(np.abs(got - ref[b]) <= _tol_v(ref[b], scale)), np.abs(got - ref[b]).max()
    # conservation per cell after moment matching
    m2 = O.cell_moments(ref["cell_start"], host(srt["svx"]), host(srt["svy"]), host(srt["svz"]))
    m0 = ref["mom"]
    n = np.maximum(m0[:, 0], 1)
    assert np.all(np.abs(m2[:, 1:4] - m0[:, 1:4]) <= 1e-12 * n[:, None] * scale)
    assert np.all(np.abs(m2[:, 4] - m0[:, 4]) <= 1e-12 * np.maximum(m0[:, 4], 1e-300))


def test_full_step_vhs_multi_step():
    """The C0 Couette gas for its stated 100 steps, each step's perm and pair
    count bit-exact and its velocities within 1e-12 of the oracle's, every
    step continuing from the oracle's state."""
    from paper_2602_21244_gb300 import dsmc as D
    T = torch()
    w = wl("couette")
    gas_o = O.make_gas(**w["gas"])
    sg = _sgmax0(w, gas_o)
    C = ctx()
    st = D.StepState(C, len(w["cell_id"]), w["n_cells"], 1 << 16)
    st.sigma_g_max.copy_(cuda(sg))
    cid, vx, vy, vz = w["cell_id"], w["vx"], w["vy"], w["vz"]
    path = D.make_path(D.PATH_VHS)
    gas = D.make_gas(w["gas"])
    total = 0
    for s in range(100):
        ref = O.step(gas_o, cid, vx, vy, vz, w["n_cells"], sg, s, path="vhs")
        st.cell_id.copy_(cuda(cid)); st.vx.copy_(cuda(vx)); st.vy.copy_(cuda(vy)); st.vz.copy_(cuda(vz))
        C.step(gas, path, st, s)
        assert C.sync_status() == 0
        assert np.array_equal(host(st.perm), ref["perm"])
        assert st.info_host()["n_pairs"] == ref["pairs"]["n_pairs"]
        total += ref["pairs"]["n_pairs"]
        for a, b in ((st.svx, "vx"), (st.svy, "vy"), (st.svz, "vz")):
            assert np.all(np.abs(host(a) - ref[b]) <= _tol_v(ref[b], 3000.0))
        # continue from the oracle's state (sorted order, same cells)
        cid = np.repeat(np.arange(w["n_cells"], dtype=np.int32), np.diff(ref["cell_start"]))
        vx, vy, vz, sg = ref["vx"], ref["vy"], ref["vz"], ref["sgmax"]
        st.sigma_g_max.copy_(cuda(sg))
    assert total > 500


# ------------------------------------------------------------------ Jager chi

JP = W.JAGER_SYNTHETIC_AR


def _gas_ar():
    return dict(mass=W.M_AR, d_ref=4.17e-10, omega=0.81, T_ref=273.0, fn_over_vc=1.0, dt=1.0,
                seed=0, model=1, b_max=1.2e-9)


def test_chi_hard_sphere_closed_form():
    from paper_2602_21244_gb300 import dsmc as D
    b, g = W.chi_pairs(1 << 16, seed=3)
    chi = host(ctx().jager_chi(D.make_gas(_gas_ar()), D.make_potential(W.HARD_SPHERE_AR), cuda(b),
                               cuda(g), n_nodes=32))
    bd = b.astype(np.float64)
    want = np.where(bd < 3.6, 2 * np.arccos(np.minimum(bd / 3.6, 1.0)), 0.0)
    assert np.abs(chi - want).max() <= 1e-5 * np.pi + 1e-6


def _sensitivity(P, b, E, h=1e-4):
    s1 = abs(O.chi(P, b * (1 + h), E) - O.chi(P, b * (1 - h), E)) / (2 * h)
    s2 = abs(O.chi(P, b, E * (1 + h) ** 2) - O.chi(P, b, E * (1 - h) ** 2)) / (2 * h)
    return s1 + s2


def _check_chi(P, b, E, chi_gpu, max_ill_frac=1e-3):
    """J5: |chi_gpu - chi_ref| <= 1e-5 |chi_ref| + 1e-6 rad with the oracle
    evaluated at the kernel's FP32 inputs; a pair whose chi the FP32
    rounding of its inputs alone moves by more than 1e-6 rad
    ((|b dchi/db| + |g dchi/dg|) 2^-24 > 1e-6, near orbiting) is
    ill-conditioned: counted, not gated, at most max_ill_frac of the pairs."""
    ref = O.chi_many(P, b, E)
    err = np.abs(chi_gpu - ref)
    out = np.flatnonzero(err > 1e-5 * np.abs(ref) + 1e-6)
    bad, ill = [], 0
    for q in out:
        if _sensitivity(P, float(b[q]), float(E[q])) * 2.0 ** -24 > 1e-6:
            ill += 1
        else:
            bad.append((float(b[q]), float(E[q]), float(ref[q]), float(chi_gpu[q])))
    assert not bad, (len(bad), bad[:5])
    assert ill <= max(3, max_ill_frac * len(b)), ill
    return ill


def _kernel_energy(g2):
    """E_r/k_B as the kernels form it: FP32 (m/(4 k_B)) times FP32 g^2."""
    return (np.float32(W.M_AR / (4.0 * KB)) * np.asarray(g2, np.float64).astype(np.float32)).astype(np.float64)


@pytest.mark.parametrize("n_nodes", [32, 48])
def test_chi_jager_parity_sampled(n_nodes):
    """C1 batch, a stratified sample of 2 x 10^4 of its 2^22 pairs: half
    below 1.5 well depths (E_r/k_B < 215 K, where orbiting, multiple roots and
    the finer bracket and quadrature act), half above."""
    from paper_2602_21244_gb300 import dsmc as D
    b, g = W.chi_pairs(1 << 22, seed=0)
    chi = host(ctx().jager_chi(D.make_gas(_gas_ar()), D.make_potential(JP), cuda(b), cuda(g),
                               n_nodes=n_nodes))
    assert ctx().sync_status() == 0
    g32 = g.astype(np.float32)
    E = (np.float32(W.M_AR / (4.0 * KB)) * g32 * g32).astype(np.float64)
    P = O.make_pot(JP)
    depth = -min(O.pot_V(P, r) for r in np.linspace(3.0, 6.0, 601))
    rng = np.random.default_rng(1)
    low = np.flatnonzero(E < 1.5 * depth)
    high = np.flatnonzero(E >= 1.5 * depth)
    idx = np.concatenate([rng.choice(low, 10000, replace=False), rng.choice(high, 10000, replace=False)])
    ill = _check_chi(P, b[idx].astype(np.float64), E[idx], chi[idx].astype(np.float64))
    print(f"n_nodes {n_nodes}: {len(idx)} pairs ({len(low)} of 2^22 below 1.5 well depths), "
          f"{ill} ill-conditioned")


# ------------------------------------------------------------------ neural operator

def _mlp_setup(d_in=8, n_hidden=3, act=0):
    from paper_2602_21244_gb300 import dsmc as D
    wts = W.mlp_weights(d_in=d_in, n_hidden=n_hidden)
    bias = np.random.default_rng(7).standard_normal(len(wts["bias"])) * 0.05
    bias = bias.astype(np.float32).astype(np.float64)
    mlp_o = O.make_mlp(d_in, 128, n_hidden, 3, act, W.sigma_v(), 273.0, 1e-12)
    mlp_d = D.make_mlp(d_in, 128, n_hidden, 3, act, W.sigma_v(), 273.0, 1e-12)
    return wts, bias, mlp_o, mlp_d


@pytest.mark.parametrize("n", [1, 127, 128, 1000, 4099])
def test_mlp_forward_parity(n):
    wts, bias, mlp_o, mlp_d = _mlp_setup()
    x = np.random.default_rng(n).standard_normal((n, 8)) * 1.5
    y = host(ctx().mlp_forward(mlp_d, w_bits_tensor(wts["W_bits"]), cuda(bias, torch().float32),
                               cuda(x, torch().float32)))
    assert ctx().sync_status() == 0
    xr = x.astype(np.float32).astype(np.float64)
    yb = O.mlp_forward(mlp_o, wts["W"], bias, xr, bf16=True)
    y64 = O.mlp_forward(mlp_o, wts["W"], bias, xr, bf16=False)
    sc = np.abs(y64).max()
    assert np.abs(y - yb).max() <= 1e-2 * sc
    assert np.abs(y - y64).max() <= 3e-2 * sc


# every shape the tensor-core MLP accepts: input width, hidden layers, activation
MLP_SHAPES = [(6, 1, 0), (8, 2, 1), (6, 4, 0), (8, 4, 1), (8, 3, 1), (6, 3, 0)]


@pytest.mark.parametrize("d_in,n_hidden,act", MLP_SHAPES)
def test_mlp_forward_shapes(d_in, n_hidden, act):
    """The standalone MLP for each accepted shape: within 1e-2 of the output
    scale of the oracle's bf16-storage emulation and 3e-2 of its FP64 forward
    (2 tiles and a ragged tail)."""
    wts, bias, mlp_o, mlp_d = _mlp_setup(d_in, n_hidden, act)
    x = np.random.default_rng(17 + n_hidden).standard_normal((300, d_in)) * 1.5
    y = host(ctx().mlp_forward(mlp_d, w_bits_tensor(wts["W_bits"]), cuda(bias, torch().float32),
                               cuda(x, torch().float32)))
    assert ctx().sync_status() == 0
    xr = x.astype(np.float32).astype(np.float64)
    yb = O.mlp_forward(mlp_o, wts["W"], bias, xr, bf16=True)
    y64 = O.mlp_forward(mlp_o, wts["W"], bias, xr, bf16=False)
    sc = np.abs(y64).max()
    assert np.abs(y - yb).max() <= 1e-2 * sc
    assert np.abs(y - y64).max() <= 3e-2 * sc


@pytest.mark.parametrize("name,shape", [("cavity40", (8, 3, 0)), ("hyper01", (8, 3, 0)), ("cavity200", (8, 3, 0)),
                                        ("hyper01", (6, 2, 1)), ("cavity40", (8, 4, 0)),
                                        ("hyper01", (6, 1, 0))])
def test_collide_neural_parity(name, shape):
    """Gate (2e-2) on the normalised post-collision relative velocity v_r'/|v_r| of
    every pair against the FP64 oracle; a tighter gate against the oracle's
    bf16-storage emulation catches layout and indexing errors.  shape = (input
    width, hidden layers, activation)."""
    w = wl(name)
    gas = O.make_gas(**w["gas"])
    wts, bias, mlp_o, mlp_d = _mlp_setup(*shape)
    sg0 = _sgmax0(w, gas)
    perm, cs, sx, sy, sz = oracle_sorted(w)
    mom = O.cell_moments(cs, sx, sy, sz)
    pr = O.select_pairs(gas, cs, sx, sy, sz, sg0, 1, capacity=1 << 22)
    *refb, ub = O.collide_neural(gas, mlp_o, wts["W"], bias, mom, pr, 1, sx, sy, sz, bf16=True, want_u=True)
    *ref64, u64 = O.collide_neural(gas, mlp_o, wts["W"], bias, mom, pr, 1, sx, sy, sz, want_u=True)
    Dg, srt, momg, sg, sel = gpu_step_pieces(w, sg0, step=1)
    C = ctx()
    sh = sel_host(sel)
    ug = torch().zeros((max(sh["n_pairs"], 1), 3), dtype=torch().float32, device="cuda")
    C.collide_neural(Dg, mlp_d, w_bits_tensor(wts["W_bits"]), cuda(bias, torch().float32), 1, momg,
                     sel, srt["svx"], srt["svy"], srt["svz"], u_out=ug)
    assert C.sync_status() == 0
    p = sh["pairs"]
    order = np.lexsort((p[:, 3], p[:, 2]))
    u = host(ug)[:sh["n_pairs"]][order]
    du64 = np.linalg.norm(u - u64, axis=1)
    dub = np.linalg.norm(u - ub, axis=1)
    assert du64.max() <= 2e-2, du64.max()
    assert dub.max() <= 2e-3, dub.max()
    sv = W.sigma_v()
    got = [host(a) for a in (srt["svx"], srt["svy"], srt["svz"])]
    dvb = max(np.abs(g_ - r_).max() for g_, r_ in zip(got, refb))
    assert dvb / sv <= 5e-3, dvb / sv
    # the projection keeps every pair on its energy shell: cell energies unchanged
    m1 = O.cell_moments(cs, *got)
    e0 = mom[:, 4] + (mom[:, 1] ** 2 + mom[:, 2] ** 2 + mom[:, 3] ** 2) / np.maximum(mom[:, 0], 1)
    e1 = m1[:, 4] + (m1[:, 1] ** 2 + m1[:, 2] ** 2 + m1[:, 3] ** 2) / np.maximum(m1[:, 0], 1)
    assert np.all(np.abs(e1 - e0) <= 1e-12 * np.maximum(e0, 1e-300))


# ------------------------------------------------------------------ C4 at full size

def test_c4_full_size_neural_step():
    """The hypersonic gas at its full size (9,144,283 particles, 150,000
    cells) through dsmc_step on the neural path, as the bench times it.
    Bit-exact: perm, cell_start, the step's pair, candidate and round counts,
    every pair (cell, candidate, particles, claim level).  Sampled: 20,000 pairs
    whose particles collide exactly once in the step -- their inputs are the
    sorted pre-collision state and their final relative velocity is the
    pair's post-collision one scaled by moment matching's alpha > 0, so its
    direction is the collide's u -- within 2e-3 of the oracle's bf16-storage
    emulation and 2e-2 of its FP64 forward.  At every cell: momentum and
    energy after moment matching within 1e-12 of the pre-collision moments."""
    from paper_2602_21244_gb300 import dsmc as D
    T = torch()
    w = W.hypersonic()
    n, nc = len(w["cell_id"]), w["n_cells"]
    gas_o = O.make_gas(**w["gas"])
    sg0 = _sgmax0(w, gas_o)
    step = 3
    perm, cs, sx, sy, sz = oracle_sorted(w)
    mom = O.cell_moments(cs, sx, sy, sz)
    pr = O.select_pairs(gas_o, cs, sx, sy, sz, sg0, step, capacity=1 << 24)
    wts, bias, mlp_o, mlp_d = _mlp_setup()
    C = ctx()
    st = D.StepState(C, n, nc, 1 << 24)
    st.sigma_g_max.copy_(cuda(sg0))
    st.cell_id.copy_(cuda(w["cell_id"])); st.vx.copy_(cuda(w["vx"]))
    st.vy.copy_(cuda(w["vy"])); st.vz.copy_(cuda(w["vz"]))
    path = D.make_path(D.PATH_NEURAL, mlp=mlp_d, w_bits=w_bits_tensor(wts["W_bits"]), bias=cuda(bias, T.float32))
    C.step(D.make_gas(w["gas"]), path, st, step)
    assert C.sync_status() == 0
    assert np.array_equal(host(st.perm), perm) and np.array_equal(host(st.cell_start), cs)
    inf = st.info_host()
    assert inf["n_pairs"] == pr["n_pairs"] and inf["n_candidates"] == pr["n_cand"]
    assert inf["n_rounds"] == pr["n_rounds"]
    sh = sel_host(st.sel)
    p = sh["pairs"]
    order = np.lexsort((p[:, 3], p[:, 2]))
    assert np.array_equal(p[order, 0], pr["i"]) and np.array_equal(p[order, 1], pr["j"])
    # the neural step buckets its pairs by claim level
    assert np.array_equal(p[order, 3], pr["m"])
    assert np.array_equal(pairs_round_of(sh)[order], expected_buckets(pr, nc, 1))
    # pairs whose two particles collide only once in the step
    cnt = np.bincount(np.concatenate([pr["i"], pr["j"]]), minlength=n)
    once = np.flatnonzero((cnt[pr["i"]] == 1) & (cnt[pr["j"]] == 1))
    pick = np.sort(np.random.default_rng(41).choice(once, size=min(20000, len(once)), replace=False))
    sub = dict(i=pr["i"][pick], j=pr["j"][pick], cell=pr["cell"][pick], m=pr["m"][pick], n_pairs=len(pick))
    *_, ub = O.collide_neural(gas_o, mlp_o, wts["W"], bias, mom, sub, step, sx, sy, sz, bf16=True, want_u=True)
    *_, u64 = O.collide_neural(gas_o, mlp_o, wts["W"], bias, mom, sub, step, sx, sy, sz, want_u=True)
    got = [host(a) for a in (st.svx, st.svy, st.svz)]
    d = np.stack([g_[sub["i"]] - g_[sub["j"]] for g_ in got], 1)
    u = d / np.linalg.norm(d, axis=1, keepdims=True)
    assert np.linalg.norm(u - ub, axis=1).max() <= 2e-3
    assert np.linalg.norm(u - u64, axis=1).max() <= 2e-2
    # conservation at every cell after moment matching
    m1 = O.cell_moments(cs, *got)
    nn = np.maximum(mom[:, 0], 1)
    vmax = max(np.abs(sx).max(), np.abs(sy).max(), np.abs(sz).max())
    assert np.all(np.abs(m1[:, 1:4] - mom[:, 1:4]) <= 1e-12 * nn[:, None] * vmax)
    e0 = mom[:, 4] + (mom[:, 1] ** 2 + mom[:, 2] ** 2 + mom[:, 3] ** 2) / nn
    e1 = m1[:, 4] + (m1[:, 1] ** 2 + m1[:, 2] ** 2 + m1[:, 3] ** 2) / nn
    assert np.all(np.abs(e1 - e0) <= 1e-12 * np.maximum(e0, 1e-300))


# ------------------------------------------------------------------ host-buffer step

def test_step_host_matches_device_step():
    from paper_2602_21244_gb300 import dsmc as D
    T = torch()
    w = wl("hyper01")
    C = ctx()
    gas = D.make_gas(w["gas"])
    n, nc = len(w["cell_id"]), w["n_cells"]
    st = D.StepState(C, n, nc, 1 << 20)
    C.sigma_g_max_init(gas, cuda(w["T_cell"]), 5.0, out=st.sigma_g_max)
    st.cell_id.copy_(cuda(w["cell_id"])); st.vx.copy_(cuda(w["vx"]))
    st.vy.copy_(cuda(w["vy"])); st.vz.copy_(cuda(w["vz"]))
    path = D.make_path(D.PATH_VHS)
    C.step(gas, path, st, 0)
    assert C.sync_status() == 0
    C.reserve(n, nc, 1 << 20)
    pin = lambda a: T.from_numpy(np.ascontiguousarray(a)).pin_memory()
    outs = [T.empty(n, dtype=T.float64).pin_memory() for _ in range(3)]
    perm = T.empty(n, dtype=T.int32).pin_memory()
    npairs = C.step_host(gas, path, pin(w["cell_id"]), pin(w["vx"]), pin(w["vy"]), pin(w["vz"]),
                         pin(w["T_cell"]), 0, perm, *outs)
    assert npairs == st.info_host()["n_pairs"]
    assert np.array_equal(perm.numpy(), host(st.perm))
    for o, a in zip(outs, (st.svx, st.svy, st.svz)):
        assert np.array_equal(o.numpy(), host(a))


# ------------------------------------------------------------------ Jager collide

def test_collide_jager_parity():
    """J6: the collide's velocities, element by element, within 1e-12
    (relative to max(|v|, c_ref)) of the oracle's rotation and
    centre-of-mass update driven by the kernel's own chi (FP64 rotation on
    both sides); J5: each pair's chi against the oracle at the kernel's FP32
    inputs (b from tag 4, E from the pair's pre-collision velocities);
    pairs bit-exact; pair energy and momentum exact."""
    from paper_2602_21244_gb300 import dsmc as D
    w = W.hypersonic(scale=0.06)
    gas = O.make_gas(**w["gas"])
    P = O.make_pot(JP)
    sg0 = _sgmax0(w, gas)
    perm, cs, sx, sy, sz = oracle_sorted(w)
    pr = O.select_pairs(gas, cs, sx, sy, sz, sg0, 4, capacity=1 << 22)
    Dg, srt, mom, sg, sel = gpu_step_pieces(w, sg0, step=4)
    C = ctx()
    sh = sel_host(sel)
    assert sh["n_pairs"] == pr["n_pairs"]
    chi_gpu = torch().zeros(max(sh["n_pairs"], 1), dtype=torch().float32, device="cuda")
    C.collide_jager(Dg, D.make_potential(JP), 4, sel, srt["svx"], srt["svy"], srt["svz"],
                    n_nodes=32, chi_out=chi_gpu)
    assert C.sync_status() == 0
    p = sh["pairs"]
    order = np.lexsort((p[:, 3], p[:, 2]))
    for c, k in enumerate(("i", "j", "cell", "m")):
        assert np.array_equal(p[order, c], pr[k])
    cg = host(chi_gpu)[:sh["n_pairs"]][order].astype(np.float64)
    rx, ry, rz, vr, bA = O.collide_given_chi(gas, pr, 4, cg, sx, sy, sz, want_vr=True)
    got = [host(a) for a in (srt["svx"], srt["svy"], srt["svz"])]
    cr = c_ref(W.M_AR)
    worst = 0.0
    for g_, r_ in zip(got, (rx, ry, rz)):
        rel = np.abs(g_ - r_) / np.maximum(np.abs(r_), cr)
        worst = max(worst, rel.max())
    assert worst <= 1e-12, worst
    _check_chi(P, bA.astype(np.float32).astype(np.float64), _kernel_energy((vr ** 2).sum(1)), cg)
    e0 = np.sum(sx ** 2 + sy ** 2 + sz ** 2)
    e1 = np.sum(got[0] ** 2 + got[1] ** 2 + got[2] ** 2)
    assert abs(e1 / e0 - 1) < 1e-12
    assert abs(np.sum(got[0]) - np.sum(sx)) < 1e-9 * np.abs(sx).sum()
    print(f"{sh['n_pairs']} pairs, worst velocity difference {worst:.2e} of max(|v|, c_ref)")


# ------------------------------------------------------------------ failure detection

@pytest.mark.parametrize("which", [0, 1, 2])
def test_bounded_waits_time_out_without_hanging(which):
    C = ctx()
    import time
    t0 = time.time()
    C.selftest_timeout(which, limit_ns=20_000_000)
    assert C.sync_status() == -4
    assert time.time() - t0 < 10
    # the context is still usable afterwards
    w = wl("couette")
    out = C.sort_cells(cuda(w["cell_id"]), cuda(w["vx"]), cuda(w["vy"]), cuda(w["vz"]), w["n_cells"])
    assert C.sync_status() == 0


# ------------------------------------------------------------------ CUDA graph of the step

@pytest.mark.parametrize("kind", ["vhs", "jager", "neural"])
def test_step_graph_replay_equals_direct_step(kind):
    from paper_2602_21244_gb300 import dsmc as D
    T = torch()
    w = wl("hyper01")
    C = ctx()
    n, nc = len(w["cell_id"]), w["n_cells"]
    gas = D.make_gas(dict(w["gas"], model=0 if kind == "vhs" else 1))
    wts, bias, _, mlp_d = _mlp_setup()
    path = D.make_path({"vhs": D.PATH_VHS, "jager": D.PATH_JAGER, "neural": D.PATH_NEURAL}[kind],
                       pot=D.make_potential(JP), n_nodes=32, mlp=mlp_d,
                       w_bits=w_bits_tensor(wts["W_bits"]), bias=cuda(bias, T.float32))
    sts = [D.StepState(C, n, nc, 1 << 21) for _ in range(2)]
    for st in sts:
        C.sigma_g_max_init(gas, cuda(w["T_cell"]), 5.0, out=st.sigma_g_max)
    s = T.cuda.Stream()
    T.cuda.synchronize()
    C.step_graph_capture(gas, path, sts[1], s)
    for step in (0, 1, 2):
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
            assert T.equal(getattr(a, k), getattr(b, k)), (kind, step, k)


# ------------------------------------------------------------------ FP64 helpers of the refinement

def test_refinement_exp_and_reciprocal_match_cuda():
    """The turning-point refinement's own FP64 exponential and reciprocal
    (written from the mathematics) against CUDA's exp and division on 10^6
    arguments each: within 4 ulp (exp over the arguments the potential
    produces and beyond; each side within about 2 ulp of e^x), 1 ulp
    (reciprocal)."""
    rng = np.random.default_rng(17)
    x = np.concatenate([rng.uniform(-60.0, 5.0, 500000), rng.uniform(-700.0, 700.0, 500000)])
    C = ctx()
    xe = cuda(x)
    own, ref = host(C.selftest_math(0, xe)), host(C.selftest_math(1, xe))
    assert np.all(np.abs(own - ref) <= 4 * np.spacing(np.abs(ref))), np.max(np.abs(own - ref) / np.spacing(np.abs(ref)))
    r = np.exp(rng.uniform(np.log(1e-3), np.log(1e6), 1000000))
    xr = cuda(r)
    own, ref = host(C.selftest_math(2, xr)), host(C.selftest_math(3, xr))
    assert np.all(np.abs(own - ref) <= np.spacing(np.abs(ref))), np.max(np.abs(own - ref) / np.spacing(np.abs(ref)))
    assert C.sync_status() == 0
