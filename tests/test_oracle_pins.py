"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: published
known-answer vectors, closed forms, library routines, invariants, brute force
or statistics with a stated confidence.  No GPU is used.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate, special, stats

import oracle as O
from paper_2602_21244_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")
KB = O.KB


# ------------------------------------------------------------------ Philox (reading R1)

def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLD, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = O.philox4x32_10(v[0:4], v[4:6])
        assert list(out) == v[6:10]


def test_philox_stream_uniform_and_u53():
    w = O.philox_stream(seed=12345, cell=7, step=3, tag=O.TAG_CAND, sub=0, n=200000)
    # each 32-bit word: 16 equal bins of the top 4 bits, chi^2 at 1e-6 level
    for c in range(4):
        h = np.bincount((w[:, c] >> 28).astype(np.int64), minlength=16)
        chi2 = ((h - h.mean()) ** 2 / h.mean()).sum()
        assert stats.chi2.sf(chi2, 15) > 1e-6
    assert O.u53(0, 0) == 0.0
    assert O.u53(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    assert O.u53(0x80000000, 0) == 0.5


# ------------------------------------------------------------------ sort (Sec. 2.6 (1))

def test_sort_is_stable_counting_sort():
    rng = np.random.default_rng(3)
    n, nc = 5000, 37
    cid = rng.integers(0, nc, n).astype(np.int32)
    cid[:50] = 5  # long equal run
    v = [rng.standard_normal(n) for _ in range(3)]
    perm, cs, sx, sy, sz = O.sort_cells(cid, *v, nc)
    ref = np.argsort(cid, kind="stable")  # library stable sort
    assert np.array_equal(perm, ref)
    assert np.array_equal(cs, np.concatenate([[0], np.cumsum(np.bincount(cid, minlength=nc))]))
    assert np.array_equal(sx, v[0][ref]) and np.array_equal(sz, v[2][ref])
    with pytest.raises(ValueError):
        O.sort_cells(np.array([0, 3], np.int32), np.zeros(2), np.zeros(2), np.zeros(2), 3)


def test_sort_empty_and_empty_cells():
    perm, cs, *_ = O.sort_cells(np.zeros(0, np.int32), np.zeros(0), np.zeros(0), np.zeros(0), 4)
    assert len(perm) == 0 and list(cs) == [0, 0, 0, 0, 0]


def test_cell_moments_two_pass():
    rng = np.random.default_rng(4)
    cs = np.array([0, 0, 1, 7, 30], np.int32)
    v = [rng.standard_normal(30) * 300 + 1e4 for _ in range(3)]
    mom = O.cell_moments(cs, *v)
    for k in range(4):
        a, b = cs[k], cs[k + 1]
        assert mom[k, 0] == b - a
        if b > a:
            V = np.stack([x[a:b] for x in v], 1)
            np.testing.assert_allclose(mom[k, 1:4], V.sum(0), rtol=1e-14)
            np.testing.assert_allclose(mom[k, 4], (b - a) * V.var(0).sum(), rtol=1e-12, atol=1e-9)


# ------------------------------------------------------------------ NTC selection (Sec. 2.2)

def _equilibrium(n_cells, per_cell, T, seed=0):
    rng = np.random.default_rng(seed)
    s = math.sqrt(KB * T / W.M_AR)
    n = n_cells * per_cell
    cs = np.arange(0, n + 1, per_cell).astype(np.int32)
    return cs, rng.standard_normal(n) * s, rng.standard_normal(n) * s, rng.standard_normal(n) * s


def test_brute_force_pair_frequencies_tiny_cells():
    # N = 5 per cell; (sigma g)_max tiny so every candidate is accepted, and
    # F_N/V_c dt large so that M = 10 per cell: the empirical frequency of each
    # ordered pair (i, j), i != j, must be 1/20.
    per = 5
    cs, vx, vy, vz = _equilibrium(200, per, 273.0, seed=1)
    gas = O.make_gas(W.M_AR, 4.17e-10, 0.81, 273.0, 2.0 ** 100, 1.0, 99, model=1, b_max=1e-10)
    sg = np.full(200, 2.0 ** -100)  # below every sigma g: all accepted
    counts = np.zeros((per, per))
    total = 0
    for step in range(3):
        pr = O.select_pairs(gas, cs, vx, vy, vz, sg, step, capacity=1 << 22)
        li = pr["i"] - cs[pr["cell"]]
        lj = pr["j"] - cs[pr["cell"]]
        assert np.all(li != lj)
        np.add.at(counts, (li, lj), 1)
        total += pr["n_pairs"]
        # M = floor(1/2 N(N-1) F dt sgmax + U) = 10 per cell exactly
        assert pr["n_pairs"] == 200 * 10
    exp_ = total / (per * (per - 1))
    obs = counts[~np.eye(per, dtype=bool)]
    chi2 = ((obs - exp_) ** 2 / exp_).sum()
    assert stats.chi2.sf(chi2, per * (per - 1) - 1) > 1e-4
    assert np.all(np.diag(counts) == 0)


@pytest.mark.parametrize("T,omega", [(273.0, 0.81), (600.0, 0.81), (400.0, 0.5)])
def test_vhs_equilibrium_collision_frequency(T, omega):
    # Closed form (Bird 1994, VHS): nu = 4 d_ref^2 n sqrt(pi k T_ref/m) (T/T_ref)^(1-omega).
    # With N particles in every cell, one step accepts on average
    #   n_cells * 1/2 N(N-1) (F_N/V_c) (nu/n) dt   pairs.
    n_cells, per, d, Tref, n_dens = 400, 50, 4.17e-10, 273.0, 1e20
    cs, vx, vy, vz = _equilibrium(n_cells, per, T, seed=2)
    fn = n_dens / per
    nu = 4.0 * d * d * n_dens * math.sqrt(math.pi * KB * Tref / W.M_AR) * (T / Tref) ** (1 - omega)
    dt = 5e-5
    gas = O.make_gas(W.M_AR, d, omega, Tref, fn, dt, 7, model=0)
    sg = O.sigma_g_max_init(gas, np.full(n_cells, T), 5.0)
    tot = 0
    steps = 4
    for s in range(steps):
        pr = O.select_pairs(gas, cs, vx, vy, vz, sg.copy(), s, capacity=1 << 22)
        tot += pr["n_pairs"]
    expected = steps * n_cells * 0.5 * per * (per - 1) * fn * (nu / n_dens) * dt
    assert expected > 4e4
    assert abs(tot / expected - 1.0) < 4.0 / math.sqrt(expected) + 1e-3


def test_rounds_reproduce_sequential_order():
    # Reading R4: pairs of one round share no particle; applying the pairs
    # round-major gives bit-for-bit the candidate-order result.
    wl = W.hypersonic(scale=0.06)
    gas = O.make_gas(**wl["gas"])
    perm, cs, sx, sy, sz = O.sort_cells(wl["cell_id"], wl["vx"], wl["vy"], wl["vz"], wl["n_cells"])
    sg = O.sigma_g_max_init(gas, wl["T_cell"], 5.0)
    pr = O.select_pairs(gas, cs, sx, sy, sz, sg, 0, capacity=1 << 22)
    assert pr["n_rounds"] > 3
    for r in range(pr["n_rounds"]):
        sel = pr["round"] == r
        parts = np.concatenate([pr["i"][sel], pr["j"][sel]])
        assert len(np.unique(parts)) == len(parts)
    a = O.collide_vhs(gas, pr, 0, sx, sy, sz)
    order = np.lexsort((pr["m"], pr["cell"], pr["round"]))
    pr2 = {k: (v[order] if isinstance(v, np.ndarray) and len(v) == pr["n_pairs"] else v)
           for k, v in pr.items()}
    b = O.collide_vhs(gas, pr2, 0, sx, sy, sz)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    # each pair in round r > 0 shares a particle with an earlier pair of round r-1
    for q in np.nonzero(pr["round"] > 0)[0][:2000]:
        c = pr["cell"][q]
        prev = (pr["cell"] == c) & (pr["round"] == pr["round"][q] - 1) & (pr["m"] < pr["m"][q])
        pts = set(pr["i"][prev]) | set(pr["j"][prev])
        assert pr["i"][q] in pts or pr["j"][q] in pts


def test_claim_levels_reproduce_sequential_order():
    # Reading R4 with the neural step's bucketing: level = round + (R - 1 -
    # the last round of the pair's cell).  Each level's pairs share no
    # particle, each particle's pairs keep their order, and applying the
    # pairs level-major gives bit-for-bit the candidate-order result; the
    # reversed level order (a plausible sign slip) does not.
    wl = W.hypersonic(scale=0.06)
    gas = O.make_gas(**wl["gas"])
    perm, cs, sx, sy, sz = O.sort_cells(wl["cell_id"], wl["vx"], wl["vy"], wl["vz"], wl["n_cells"])
    sg = O.sigma_g_max_init(gas, wl["T_cell"], 5.0)
    pr = O.select_pairs(gas, cs, sx, sy, sz, sg, 0, capacity=1 << 22)
    R = pr["n_rounds"]
    last = np.full(wl["n_cells"], -1)
    np.maximum.at(last, pr["cell"], pr["round"])
    lvl = pr["round"] + (R - 1) - last[pr["cell"]]
    assert lvl.min() >= 0 and lvl.max() == R - 1 and not np.array_equal(lvl, pr["round"])
    for v in range(R):
        sel = lvl == v
        parts = np.concatenate([pr["i"][sel], pr["j"][sel]])
        assert len(np.unique(parts)) == len(parts)
    a = O.collide_vhs(gas, pr, 0, sx, sy, sz)

    def apply(key):
        order = np.lexsort((pr["m"], pr["cell"], key))
        pr2 = {k: (v[order] if isinstance(v, np.ndarray) and len(v) == pr["n_pairs"] else v)
               for k, v in pr.items()}
        return O.collide_vhs(gas, pr2, 0, sx, sy, sz)
    for x, y in zip(a, apply(lvl)):
        assert np.array_equal(x, y)
    assert not all(np.array_equal(x, y) for x, y in zip(a, apply((R - 1) - lvl)))


def test_sigma_g_max_only_grows_and_capacity():
    wl = W.couette()
    gas = O.make_gas(**wl["gas"])
    perm, cs, sx, sy, sz = O.sort_cells(wl["cell_id"], wl["vx"], wl["vy"], wl["vz"], wl["n_cells"])
    sg0 = np.full(wl["n_cells"], 1e-20)
    pr = O.select_pairs(gas, cs, sx, sy, sz, sg0, 0)
    assert np.all(pr["sgmax"] >= sg0)
    with pytest.raises(RuntimeError):
        big = np.full(wl["n_cells"], 1e-13)
        O.select_pairs(gas, cs, sx, sy, sz, big, 0, capacity=4)


# ------------------------------------------------------------------ VHS scatter

def _pair_setup(n=20000, seed=5):
    rng = np.random.default_rng(seed)
    vx, vy, vz = (rng.standard_normal(2 * n) * 300 for _ in range(3))
    pairs = dict(i=np.arange(0, 2 * n, 2, dtype=np.int32), j=np.arange(1, 2 * n, 2, dtype=np.int32),
                 cell=np.zeros(n, np.int32), m=np.arange(n, dtype=np.int32), n_pairs=n)
    return pairs, vx, vy, vz


def test_vhs_isotropic_and_conserving():
    pairs, vx, vy, vz = _pair_setup(100000)
    gas = O.make_gas(W.M_AR, 4.17e-10, 0.81, 273.0, 1.0, 1.0, 11)
    ox, oy, oz = O.collide_vhs(gas, pairs, 4, vx, vy, vz)
    i, j = pairs["i"], pairs["j"]
    vr0 = np.stack([vx[i] - vx[j], vy[i] - vy[j], vz[i] - vz[j]], 1)
    vr1 = np.stack([ox[i] - ox[j], oy[i] - oy[j], oz[i] - oz[j]], 1)
    g0, g1 = np.linalg.norm(vr0, axis=1), np.linalg.norm(vr1, axis=1)
    np.testing.assert_allclose(g1, g0, rtol=1e-13)
    np.testing.assert_allclose(ox[i] + ox[j], vx[i] + vx[j], rtol=0, atol=1e-10)
    u = vr1 / g1[:, None]
    # cos of the lab polar angle uniform on [-1,1] (KS), <u> = 0, <u u^T> = I/3
    assert stats.kstest(u[:, 0], "uniform", args=(-1, 2)).pvalue > 1e-4
    assert np.all(np.abs(u.mean(0)) < 5 / math.sqrt(len(u)))
    np.testing.assert_allclose(u.T @ u / len(u), np.eye(3) / 3, atol=6e-3)


def test_relaxation_to_maxwellian_mean_speed():
    # Paper Sec. 3.1: the equilibrium speed distribution has mean sqrt(8kT/(pi m)).
    # Start from a mono-speed isotropic gas and relax it with VHS collisions.
    rows = [l.split() for l in open(os.path.join(GOLD, "maxwell_mean_speed.txt"))
            if l.strip() and not l.startswith("#")]
    T_p, c_th, c_sim, rel = map(float, rows[0])
    assert abs((c_th - c_sim) / c_th * 100 - rel) < 1e-3  # the paper's numbers agree
    # The paper's printed 380.2270 m/s at 272.78 K implies a mass of about
    # 6.6335e-26 kg (its stated 6.63e-26 kg gives 380.33 m/s): the formula is pinned
    # to 3e-4 relative, the printed mass to 3 digits.
    m_impl = 8 * KB * T_p / (math.pi * c_th ** 2)
    assert abs(m_impl / 6.63e-26 - 1.0) < 1e-3
    rng = np.random.default_rng(8)
    n_cells, per = 40, 1000
    n = n_cells * per
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    c0 = 400.0
    vx, vy, vz = (c0 * d[:, 0]).copy(), (c0 * d[:, 1]).copy(), (c0 * d[:, 2]).copy()
    cid = np.repeat(np.arange(n_cells, dtype=np.int32), per)
    T = W.M_AR * c0 * c0 / (3 * KB)
    gas = O.make_gas(W.M_AR, 4.17e-10, 0.81, 273.0, 1e20 / per, 2e-5, 3)
    sg = O.sigma_g_max_init(gas, np.full(n_cells, T), 5.0)
    for s in range(20):
        res = O.step(gas, cid, vx, vy, vz, n_cells, sg, s, path="vhs", capacity=1 << 22)
        cid = np.repeat(np.arange(n_cells, dtype=np.int32), per)
        vx, vy, vz, sg = res["vx"], res["vy"], res["vz"], res["sgmax"]
    speed = np.sqrt(vx * vx + vy * vy + vz * vz)
    T_now = W.M_AR * np.mean(speed ** 2) / (3 * KB)
    assert abs(T_now / T - 1) < 1e-10  # energy conserved
    c_theory = math.sqrt(8 * KB * T_now / (math.pi * W.M_AR))
    stat = speed.std() / math.sqrt(n) / c_theory  # standard error of the mean
    assert abs(speed.mean() / c_theory - 1) < 4 * stat + 5e-4
    assert abs(speed.mean() / c0 - 1) > 0.05  # it did relax (mono-speed mean would be c0)


# ------------------------------------------------------------------ moment matching (Sec. 2.5)

def test_moment_match_restores_moments_and_reduces_to_paper():
    rng = np.random.default_rng(9)
    cs = np.array([0, 1, 2, 40, 41, 100], np.int32)
    n = cs[-1]
    v0 = [rng.standard_normal(n) * 300 + 500 for _ in range(3)]
    mom = O.cell_moments(cs, *v0)
    v1 = [x * 1.1 + rng.standard_normal(n) * 20 for x in v0]
    o = O.moment_match(cs, mom, *v1)
    m2 = O.cell_moments(cs, *o)
    np.testing.assert_allclose(m2[:, 1:4], mom[:, 1:4], rtol=1e-12, atol=1e-9)
    e0 = [np.sum(sum(x[cs[k]:cs[k + 1]] ** 2 for x in v0)) for k in range(5)]
    e1 = [np.sum(sum(x[cs[k]:cs[k + 1]] ** 2 for x in o)) for k in range(5)]
    np.testing.assert_allclose(e1, e0, rtol=1e-12)
    # zero mean velocity before and after: centred form == alpha v with
    # alpha = sqrt(E_pre/E_post) (Eq. cell_energy_clamp)
    a = rng.standard_normal((30, 3)); a -= a.mean(0)
    b = rng.standard_normal((30, 3)); b -= b.mean(0)
    cs1 = np.array([0, 30], np.int32)
    momA = O.cell_moments(cs1, a[:, 0], a[:, 1], a[:, 2])
    o = O.moment_match(cs1, momA, b[:, 0], b[:, 1], b[:, 2])
    alpha = math.sqrt(np.sum(a * a) / np.sum(b * b))
    np.testing.assert_allclose(np.stack(o, 1), alpha * b, rtol=1e-12, atol=1e-14)
    # unchanged velocities: identity to rounding
    o = O.moment_match(cs, mom, *v0)
    for x, y in zip(o, v0):
        np.testing.assert_allclose(x, y, rtol=1e-13)


# ------------------------------------------------------------------ Jager potential (Sec. 3.4.1)

JP = O.make_pot(W.JAGER_SYNTHETIC_AR)


@pytest.mark.parametrize("n", [6, 8, 10, 12, 14, 16])
def test_tang_toennies_damping_is_incomplete_gamma(n):
    for x in [0.0, 0.3, 2.0, 7.5, 14.4, 40.0]:
        assert abs(O.tt_damp(n, x) - special.gammainc(n + 1, x)) < 1e-14


def test_repulsive_exponent_polynomial_recovered():
    p = dict(W.JAGER_SYNTHETIC_AR, C=[0.0] * 6)
    P = O.make_pot(p)
    rs = np.array([1.7, 2.4, 3.3, 4.6])
    y = np.log([O.pot_V(P, r) / p["A"] for r in rs])
    X = np.stack([rs, rs * rs, 1 / rs, 1 / rs ** 2], 1)
    coef = np.linalg.solve(X, y)
    np.testing.assert_allclose(coef, [p["a1"], p["a2"], p["am1"], p["am2"]], rtol=1e-9, atol=1e-11)


def test_dispersion_asymptote_and_terms():
    # far out the damping is 1 and the repulsion negligible: V = -sum C_2n / r^2n
    for r in [25.0, 40.0]:
        far = -sum(c / r ** (2 * n) for n, c in zip(range(3, 9), W.JAGER_SYNTHETIC_AR["C"]))
        assert abs(O.pot_V(JP, r) / far - 1) < 1e-10
    # each C_2n enters with its own power: perturb one at a time
    for q in range(6):
        p = dict(W.JAGER_SYNTHETIC_AR)
        p["C"] = list(p["C"]); p["C"][q] *= 2.0
        P = O.make_pot(p)
        r = 30.0
        dV = O.pot_V(P, r) - O.pot_V(JP, r)
        assert abs(dV / (-W.JAGER_SYNTHETIC_AR["C"][q] / r ** (6 + 2 * q)) - 1) < 1e-6


def test_potential_derivative_and_core_continuity():
    for r in [0.5, 1.2, 1.6, 2.5, 3.4, 3.757, 5.0, 9.0]:
        if abs(r - 0.4 * 3.757) < 0.02:
            continue
        h = 1e-3 * r  # fourth-order central difference
        V = lambda x: O.pot_V(JP, x)
        fd = (-V(r + 2 * h) + 8 * V(r + h) - 8 * V(r - h) + V(r - 2 * h)) / (12 * h)
        assert abs(O.pot_dV(JP, r) - fd) <= 1e-6 * max(1.0, abs(V(r)) / r), r
    r0 = 0.4 * W.JAGER_SYNTHETIC_AR["R_eps"]
    for f in (O.pot_V, O.pot_dV):
        lo, hi = f(JP, r0 * (1 - 1e-12)), f(JP, r0 * (1 + 1e-12))
        assert abs(lo - hi) <= 1e-7 * abs(hi)
    assert abs(O.pot_dV(JP, 3.757)) < 1e-4 and abs(O.pot_V(JP, 3.757) + 143.2) < 1e-6


# ------------------------------------------------------------------ scattering angle (Sec. 3.4.2, 3.4.4)

def test_hard_sphere_chi_closed_form():
    hs = O.make_pot(W.HARD_SPHERE_AR)
    for b in np.linspace(0, 5, 41):
        want = 2 * math.acos(b / 3.6) if b < 3.6 else 0.0
        assert abs(O.chi(hs, b, 700.0) - want) < 1e-12


@pytest.mark.parametrize("kappa,E", [(500.0, 300.0), (2.0e4, 1.0e4), (50.0, 10.0)])
def test_coulomb_chi_closed_form(kappa, E):
    P = O.make_pot(dict(kind=2, kappa=kappa, p=1.0))
    for b in [0.05, 0.5, 1.0, 3.0, 10.0]:
        assert abs(O.chi(P, b, E) - 2 * math.atan(kappa / (2 * E * b))) < 1e-12


def test_inverse_square_chi_closed_form():
    P = O.make_pot(dict(kind=2, kappa=2000.0, p=2.0))
    for E in [30.0, 300.0, 3e4]:
        for b in [0.05, 0.5, 2.0, 10.0]:
            want = math.pi * (1 - b / math.sqrt(b * b + 2000.0 / E))
            assert abs(O.chi(P, b, E) - want) < 1e-12


def test_hard_sphere_transport_cross_section():
    # Q^(2) = 2 pi int (1 - cos^2 chi) b db = (2/3) pi d^2 for hard spheres
    hs = O.make_pot(W.HARD_SPHERE_AR)
    d = 3.6
    q, _ = integrate.quad(lambda b: (1 - math.cos(O.chi(hs, b, 500.0)) ** 2) * b, 0, d,
                          epsabs=1e-13, epsrel=1e-12)
    assert abs(2 * math.pi * q / (2 / 3 * math.pi * d * d) - 1) < 1e-9


def test_rmin_is_outermost_root():
    for E in [108.0, 500.0, 5e4]:
        for b in [0.5, 3.0, 4.5, 9.0]:
            r = O.rmin(JP, b, E)
            F = lambda x: 1 - b * b / (x * x) - O.pot_V(JP, x) / E
            assert abs(F(r)) < 1e-10
            xs = r * np.exp(np.linspace(1e-9, 2.5, 4000))
            assert all(F(x) > 0 for x in xs)


def test_chi_against_independent_quadrature():
    # scipy's adaptive Gauss-Kronrod on the u-form with the u = 1 - s^2 split,
    # completely independent of the oracle's tanh-sinh rule
    for E, b in [(300.0, 2.5), (1000.0, 4.0), (5e4, 0.7), (150.0, 6.0)]:
        r = O.rmin(JP, b, E)
        bt = b / r

        def f(s):
            u = 1 - s * s
            Gv = 1 - (bt * u) ** 2 - O.pot_V(JP, r / u) / E
            return 2 * s / math.sqrt(Gv) if Gv > 0 else 0.0
        I, _ = integrate.quad(f, 1e-4, 1, epsabs=1e-13, epsrel=1e-12, limit=400)
        # the first [0, 1e-4] piece from the local expansion G ~ c s^2
        c = 2 * bt * bt - r * O.pot_dV(JP, r) / E
        I += 2 * 1e-4 / math.sqrt(c)
        assert abs(O.chi(JP, b, E) - (math.pi - 2 * bt * I)) < 1e-6


def test_chi_limits():
    assert O.chi(JP, 0.0, 500.0) == math.pi
    assert abs(O.chi(JP, 40.0, 500.0)) < 1e-5
    # high energy, small b: nearly head-on repulsion
    assert O.chi(JP, 0.05, 2.7e5) > 3.0


def test_deflect_geometry():
    rng = np.random.default_rng(2)
    for _ in range(200):
        vr = rng.standard_normal(3) * 500
        chi, eps = rng.uniform(-4, 4), rng.uniform(0, 2 * math.pi)
        out = O.deflect(vr, chi, eps)
        g = np.linalg.norm(vr)
        assert abs(np.linalg.norm(out) - g) < 1e-10 * g
        assert abs(np.dot(out, vr) / (g * g) - math.cos(chi)) < 1e-12
        # eps and eps + pi deflect to mirror images about v_r
        o2 = O.deflect(vr, chi, eps + math.pi)
        np.testing.assert_allclose(out + o2, 2 * math.cos(chi) * vr, atol=1e-9 * g)
    out = O.deflect(np.array([300.0, 0, 0]), 0.5, 0.0)
    np.testing.assert_allclose(out, [300 * math.cos(0.5), 300 * math.sin(0.5), 0], atol=1e-12)


def test_chi_batch_energy_is_the_reduced_mass_kinetic_energy():
    """Sec. 3.4.2: the scattering integral depends on the relative kinetic
    energy E_r = (1/2) mu g^2 with the reduced mass mu = m1 m2 / (m1 + m2)
    (m/2 for like particles).  With a repulsive Coulomb potential V = kappa/r
    the deflection angle has the closed form tan(chi/2) = kappa / (2 E_r b),
    so the (b, g) batch pins the g -> E mapping of the oracle."""
    kappa = 3.0e3
    P = O.make_pot(dict(kind=2, kappa=kappa, p=1.0))
    gas = O.make_gas(W.M_AR, 4.17e-10, 0.81, 273.0, 1.0, 1.0, 0, model=1, b_max=1.2e-9)
    b = np.array([0.3, 1.0, 2.5, 4.0, 7.5, 11.0])
    g = np.array([300.0, 1200.0, 4000.0, 800.0, 15000.0, 2500.0])
    mu = W.M_AR * W.M_AR / (W.M_AR + W.M_AR)
    E = 0.5 * mu * g * g / KB
    want = 2.0 * np.arctan(kappa / (2.0 * E * b))
    got = O.chi_batch(gas, P, b, g)
    np.testing.assert_allclose(got, want, rtol=1e-10, atol=1e-13)


def _hs_jager_run(n=100_000, g=1500.0, step=3):
    """n pairs of distinct particles, all with the same relative velocity
    g * d (d a fixed unit vector), through the oracle's Jager collide with
    the hard-sphere potential."""
    d = np.array([0.3, -0.5, 0.81])
    d /= np.linalg.norm(d)
    vi = 0.5 * g * d + np.array([120.0, -40.0, 15.0])
    vj = -0.5 * g * d + np.array([120.0, -40.0, 15.0])
    vx = np.empty(2 * n); vy = np.empty(2 * n); vz = np.empty(2 * n)
    vx[0::2], vy[0::2], vz[0::2] = vi
    vx[1::2], vy[1::2], vz[1::2] = vj
    p = np.arange(n, dtype=np.int32)
    pairs = dict(i=2 * p, j=2 * p + 1, cell=p // 1000, m=p % 1000, n_pairs=n)
    gas = O.make_gas(W.M_AR, 4.17e-10, 0.81, 273.0, 1.0, 1.0, 77, model=1, b_max=1.2e-9)
    ox, oy, oz, chi = O.collide_jager(gas, O.make_pot(W.HARD_SPHERE_AR), pairs, step, vx, vy, vz, want_chi=True)
    vr1 = np.stack([ox[0::2] - ox[1::2], oy[0::2] - oy[1::2], oz[0::2] - oz[1::2]], 1)
    return d, g, chi, vr1


def test_jager_collide_impact_parameter_and_azimuth_draws():
    """The collide draws b with b^2 uniform on [0, b_max^2] and eps uniform on
    [0, 2 pi) (Sec. 3.4.2: b up to b_max; the azimuth of an isotropic
    collision plane).  With hard spheres (d = 3.6 A) these fix: P(chi = 0) =
    P(b > d) = 1 - (d/b_max)^2 = 0.91; given b < d, cos^2(chi/2) = (b/d)^2 is
    uniform on [0, 1]; the azimuth of v_r' about the common v_r is uniform on
    [0, 2 pi) and the angle between v_r and v_r' is |chi|."""
    n = 100_000
    d, g, chi, vr1 = _hs_jager_run(n)
    zero = np.abs(chi) < 1e-9
    p0 = 1.0 - (3.6 / 12.0) ** 2
    assert abs(zero.mean() - p0) < 4.0 * math.sqrt(p0 * (1 - p0) / n), zero.mean()
    c2 = np.cos(0.5 * chi[~zero]) ** 2
    assert stats.kstest(c2, "uniform").pvalue > 1e-3
    # |v_r'| = g and the angle between v_r and v_r' is chi
    np.testing.assert_allclose(np.linalg.norm(vr1, axis=1), g, rtol=1e-12)
    cosang = vr1 @ d / g
    np.testing.assert_allclose(cosang, np.cos(chi), atol=1e-11)
    # azimuth about d in a fixed frame (e1, e2) perpendicular to d
    e1 = np.cross(d, [0.0, 0.0, 1.0]); e1 /= np.linalg.norm(e1)
    e2 = np.cross(d, e1)
    sel = np.abs(np.sin(chi)) > 1e-3
    phi = np.mod(np.arctan2(vr1[sel] @ e2, vr1[sel] @ e1), 2 * math.pi)
    assert stats.kstest(phi / (2 * math.pi), "uniform").pvalue > 1e-3


def test_neural_collide_cell_temperature():
    """Sec. 2.2: the MLP sees the cell's kinetic temperature, (3/2) k T =
    (1/2) m <|v - u|^2>.  A cell of six particles at u + (+-a, 0, 0),
    u + (0, +-a, 0), u + (0, 0, +-a) has <|v - u|^2> = a^2, so it is at
    T = m a^2 / (3 k) by construction; the collide's direction must equal the
    network's output for the features formed with that T (network and noise
    are pinned by their own tests)."""
    wts, mlp = _mlp()
    bias = np.random.default_rng(3).standard_normal(len(wts["bias"])) * 0.05
    T_known = 800.0
    a = math.sqrt(3.0 * KB * T_known / W.M_AR)
    u = np.array([150.0, -320.0, 40.0])
    offs = np.array([[a, 0, 0], [-a, 0, 0], [0, a, 0], [0, -a, 0], [0, 0, a], [0, 0, -a]])
    v = u + offs
    vx, vy, vz = v[:, 0].copy(), v[:, 1].copy(), v[:, 2].copy()
    cs = np.array([0, 6], np.int32)
    mom = O.cell_moments(cs, vx, vy, vz)
    gas = O.make_gas(W.M_AR, 4.17e-10, 0.81, 273.0, 1.0, 1.0, 21, model=1, b_max=1.2e-9)
    for (i, j, m) in [(0, 3, 0), (4, 1, 5), (2, 5, 9)]:
        pairs = dict(i=np.array([i], np.int32), j=np.array([j], np.int32), cell=np.array([0], np.int32),
                     m=np.array([m], np.int32), n_pairs=1)
        *_, ug = O.collide_neural(gas, mlp, wts["W"], bias, mom, pairs, 2, vx, vy, vz, want_u=True)
        vr = v[i] - v[j]
        xi = O.noise4(21, 0, m, 2)
        x = np.concatenate([vr / W.sigma_v(), [T_known / 273.0], xi])[None, :]
        y = O.mlp_forward(mlp, wts["W"], bias, x)[0]
        np.testing.assert_allclose(ug[0], y / np.linalg.norm(y), rtol=0, atol=1e-12)


# ------------------------------------------------------------------ neural operator (Sec. 2.2-2.3)

def _mlp(d_in=8):
    wts = W.mlp_weights(d_in=d_in)
    mlp = O.make_mlp(d_in, 128, 3, 3, 0, W.sigma_v(), 273.0, 1e-12)
    return wts, mlp


def test_mlp_forward_matches_torch_sequential():
    torch = pytest.importorskip("torch")
    wts, mlp = _mlp()
    from oracle.train import split_layers, split_bias
    Ws, bs = split_layers(wts["dims"], wts["W"]), split_bias(wts["dims"], wts["bias"] + 0.01)
    layers = []
    for l in range(4):
        lin = torch.nn.Linear(wts["dims"][l], wts["dims"][l + 1]).double()
        lin.weight.data = torch.tensor(Ws[l]); lin.bias.data = torch.tensor(bs[l])
        layers += [lin] + ([torch.nn.SiLU()] if l < 3 else [])
    net = torch.nn.Sequential(*layers)
    x = np.random.default_rng(0).standard_normal((64, 8))
    y = O.mlp_forward(mlp, wts["W"], wts["bias"] + 0.01, x)
    ref = net(torch.tensor(x)).detach().numpy()
    np.testing.assert_allclose(y, ref, rtol=1e-12, atol=1e-13)
    # bf16 mode: input and hidden activations as two bf16 terms each
    xt = torch.tensor(x)
    hi = xt.to(torch.bfloat16).double()
    h = hi + (xt - hi).to(torch.bfloat16).double()
    for l in range(4):
        h = layers[2 * l](h)
        if l < 3:
            a = torch.nn.functional.silu(h)
            hi = a.to(torch.bfloat16).double()
            h = hi + (a - hi).to(torch.bfloat16).double()
    yb = O.mlp_forward(mlp, wts["W"], wts["bias"] + 0.01, x, bf16=True)
    np.testing.assert_allclose(yb, h.detach().numpy(), rtol=1e-12, atol=1e-13)


def test_bf16_rounding_nearest_even():
    torch = pytest.importorskip("torch")
    xs = np.random.default_rng(1).standard_normal(2000) * 10 ** np.random.default_rng(2).uniform(-3, 3, 2000)
    ref = torch.tensor(xs, dtype=torch.float32).to(torch.bfloat16).double().numpy()
    assert all(O.bf16_round(x) == r for x, r in zip(xs, ref))
    np.testing.assert_array_equal(W.bf16_value(W.bf16_bits(xs)), ref)


def test_latent_noise_is_standard_normal():
    z = np.array([O.noise4(5, 3, m, 2) for m in range(20000)])
    for c in range(4):
        assert stats.kstest(z[:, c], "norm").pvalue > 1e-4
    assert abs(np.corrcoef(z[:, 0], z[:, 1])[0, 1]) < 0.05


def test_neural_collide_conserves_pair_invariants():
    wts, mlp = _mlp()
    pairs, vx, vy, vz = _pair_setup(500)
    gas = O.make_gas(W.M_AR, 4.17e-10, 0.81, 273.0, 1.0, 1.0, 11)
    mom = np.array([[1000.0, 0, 0, 0, 1000 * 3 * KB * 300 / W.M_AR]])
    ox, oy, oz = O.collide_neural(gas, mlp, wts["W"], wts["bias"], mom, pairs, 1, vx, vy, vz)
    i, j = pairs["i"], pairs["j"]
    e0 = vx[i] ** 2 + vx[j] ** 2 + vy[i] ** 2 + vy[j] ** 2 + vz[i] ** 2 + vz[j] ** 2
    e1 = ox[i] ** 2 + ox[j] ** 2 + oy[i] ** 2 + oy[j] ** 2 + oz[i] ** 2 + oz[j] ** 2
    np.testing.assert_allclose(e1, e0, rtol=1e-13)
    np.testing.assert_allclose(ox[i] + ox[j], vx[i] + vx[j], atol=1e-10)
    assert np.mean(np.abs(ox - vx)) > 1.0  # it scattered


# ------------------------------------------------------------------ training oracle (Sec. 2.6)

def _train_case(n=64, seed=0):
    from oracle import train as T
    wts = W.mlp_weights()
    dims = wts["dims"]
    rng = np.random.default_rng(seed)
    Ws = [w + rng.standard_normal(w.shape) * 0.05 for w in T.split_layers(dims, wts["W"])]
    bs = [rng.standard_normal(b.shape) * 0.05 for b in T.split_bias(dims, wts["bias"])]
    hv = W.harvest_inputs(n, seed=seed)
    gas = O.make_gas(W.M_AR, 4.17e-10, 0.81, 273.0, 1.0, 1.0, 3)
    vit, vjt = O.harvest_jager(gas, JP, hv["vi"], hv["vj"], hv["b"], hv["eps"])
    xi = T.train_noise(3, 1, n)
    return T, dims, Ws, bs, hv, vit, vjt, xi


def test_train_gradient_central_differences():
    T, dims, Ws, bs, hv, vit, vjt, xi = _train_case()
    sv = W.sigma_v()
    args = (hv["vi"], hv["vj"], hv["T"], xi, vit, vjt, sv, 273.0)
    loss, cache = T.forward(dims, Ws, bs, *args)
    dW, db = T.backward(dims, Ws, bs, cache, sv)
    rng = np.random.default_rng(1)
    h = 1e-3
    worst = 0.0
    for _ in range(256):
        l = int(rng.integers(0, 4))
        if rng.random() < 0.2:
            q = int(rng.integers(0, bs[l].size))
            arr, g = bs[l], db[l].ravel()[q]
            idx = np.unravel_index(q, bs[l].shape)
        else:
            q = int(rng.integers(0, Ws[l].size))
            arr, g = Ws[l], dW[l].ravel()[q]
            idx = np.unravel_index(q, Ws[l].shape)
        old = arr[idx]

        def cd(step):
            arr[idx] = old + step; lp, _ = T.forward(dims, Ws, bs, *args)
            arr[idx] = old - step; lm, _ = T.forward(dims, Ws, bs, *args)
            arr[idx] = old
            return (lp - lm) / (2 * step)
        # central differences at h = 1e-3, Richardson-extrapolated with h/2
        fd = (4 * cd(h / 2) - cd(h)) / 3
        scale = max(abs(fd), 1e-3 * np.max(np.abs(dW[l])))
        worst = max(worst, abs(fd - g) / scale)
    assert worst < 1e-5, worst


def test_train_gradient_matches_torch_autograd():
    torch = pytest.importorskip("torch")
    T, dims, Ws, bs, hv, vit, vjt, xi = _train_case(n=128, seed=4)
    sv = W.sigma_v()
    loss, cache = T.forward(dims, Ws, bs, hv["vi"], hv["vj"], hv["T"], xi, vit, vjt, sv, 273.0)
    dW, db = T.backward(dims, Ws, bs, cache, sv)
    tW = [torch.tensor(w, requires_grad=True) for w in Ws]
    tb = [torch.tensor(b, requires_grad=True) for b in bs]
    vi, vj = torch.tensor(hv["vi"]), torch.tensor(hv["vj"])
    vr = vi - vj
    x = torch.cat([vr / sv, torch.tensor(hv["T"] / 273.0)[:, None], torch.tensor(xi)], 1)
    h = x
    for l in range(4):
        h = torch.nn.functional.linear(h, tW[l], tb[l])
        if l < 3:
            h = torch.nn.functional.silu(h)
    vrp = vr.norm(dim=1, keepdim=True) * h / h.norm(dim=1, keepdim=True)
    cm = 0.5 * (vi + vj)
    P = torch.cat([(cm + 0.5 * vrp).reshape(-1, 16, 3), (cm - 0.5 * vrp).reshape(-1, 16, 3)], 1)
    Q = torch.cat([vi.reshape(-1, 16, 3), vj.reshape(-1, 16, 3)], 1)
    Tt = torch.cat([torch.tensor(vit).reshape(-1, 16, 3), torch.tensor(vjt).reshape(-1, 16, 3)], 1)
    up, uq = P.mean(1, keepdim=True), Q.mean(1, keepdim=True)
    alpha = torch.sqrt(((Q - uq) ** 2).sum((1, 2)) / ((P - up) ** 2).sum((1, 2)))
    Vn = uq + alpha[:, None, None] * (P - up)
    L = (((Vn - Tt) / sv) ** 2).sum() / (2 * 128)
    L.backward()
    assert abs(L.item() - loss) < 1e-12 * abs(loss)
    for l in range(4):
        np.testing.assert_allclose(dW[l], tW[l].grad.numpy(), rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(db[l], tb[l].grad.numpy(), rtol=1e-9, atol=1e-12)


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    from oracle import train as T
    rng = np.random.default_rng(0)
    th = rng.standard_normal(50)
    p = torch.tensor(th.copy(), requires_grad=True)
    opt = torch.optim.Adam([p], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    m, v = np.zeros(50), np.zeros(50)
    for t in range(1, 6):
        g = rng.standard_normal(50)
        th, m, v = T.adam(th, g, m, v, t)
        p.grad = torch.tensor(g)
        opt.step()
    np.testing.assert_allclose(th, p.detach().numpy(), rtol=1e-12, atol=1e-14)


# ------------------------------------------------------------------ look-up table (Sec. 3.4.4)

def test_chi_table_nodes_hard_sphere_closed_form():
    """Table nodes: b = b_max i/(nb-1) and E = exp(lnE_min + j dE); the hard
    sphere's chi = 2 arccos(b/d) for b < d, independent of E, pins both maps."""
    hs = O.make_pot(W.HARD_SPHERE_AR)
    nb, nE, bmax = 13, 5, 6.0
    T = O.chi_table(hs, bmax, nb, nE, math.log(5.0), math.log(6e4))
    for j in range(nE):
        for i in range(nb):
            b = bmax * i / (nb - 1)
            want = 2 * math.acos(b / 3.6) if b < 3.6 else 0.0
            assert abs(T[j, i] - want) < 1e-12


def test_chi_table_energy_axis_coulomb_closed_form():
    """The energy axis: Coulomb chi = 2 atan(kappa/(2 E b)) at each node."""
    P = O.make_pot(dict(kind=2, kappa=500.0, p=1.0))
    nb, nE, bmax, lo, hi = 5, 7, 8.0, math.log(10.0), math.log(1e4)
    T = O.chi_table(P, bmax, nb, nE, lo, hi)
    for j in range(nE):
        E = math.exp(lo + j * (hi - lo) / (nE - 1))
        for i in range(1, nb):
            b = bmax * i / (nb - 1)
            assert abs(T[j, i] - 2 * math.atan(500.0 / (2 * E * b))) < 1e-12


def test_chi_lookup_is_bilinear():
    """Bilinear interpolation reproduces a bilinear function of the grid
    coordinates exactly, returns node values at nodes, and clamps ln E."""
    nb, nE, lo, hi = 9, 6, 1.0, 4.0
    jj, ii = np.meshgrid(np.arange(nE), np.arange(nb), indexing="ij")
    T = (1.0 + 2.0 * ii + 3.0 * jj + 0.5 * ii * jj).astype(np.float32)   # exact in float
    rng = np.random.default_rng(3)
    for _ in range(200):
        bt, lnE = rng.random(), lo + (hi - lo) * rng.random()
        x, y = bt * (nb - 1), (lnE - lo) / (hi - lo) * (nE - 1)
        assert abs(O.chi_lookup(T, lo, hi, bt, lnE) - (1 + 2 * x + 3 * y + 0.5 * x * y)) < 1e-12
    assert O.chi_lookup(T, lo, hi, 0.5, lo) == T[0, 4]
    assert O.chi_lookup(T, lo, hi, 1.0, hi) == T[-1, -1]
    assert O.chi_lookup(T, lo, hi, 0.25, lo - 5.0) == O.chi_lookup(T, lo, hi, 0.25, lo)
    assert O.chi_lookup(T, lo, hi, 0.25, hi + 5.0) == O.chi_lookup(T, lo, hi, 0.25, hi)


def test_collide_table_with_constant_chi_is_the_rotation():
    """A table holding one angle everywhere: every pair is the Bird rotation
    by that angle (checked against or_deflect), energy and momentum kept."""
    w = W.couette()
    gas = O.make_gas(**dict(w["gas"], model=1))
    perm, cs, sx, sy, sz = O.sort_cells(w["cell_id"], w["vx"], w["vy"], w["vz"], w["n_cells"])
    sg = O.sigma_g_max_init(gas, w["T_cell"], 5.0)
    pr = O.select_pairs(gas, cs, sx, sy, sz, sg, 2, capacity=1 << 16)
    T = np.full((4, 4), 0.7, np.float32)
    vx, vy, vz, chi = O.collide_table(gas, T, 0.0, 10.0, pr, 2, sx, sy, sz, want_chi=True)
    assert np.all(chi == np.float32(0.7))
    e0 = np.sum(sx ** 2 + sy ** 2 + sz ** 2)
    assert abs(np.sum(vx ** 2 + vy ** 2 + vz ** 2) / e0 - 1) < 1e-13
    assert abs(np.sum(vx) - np.sum(sx)) < 1e-9 * np.abs(sx).sum()
    # the first pair of the step sees the input velocities: rotation by 0.7
    p0 = 0
    i, j = pr["i"][p0], pr["j"][p0]
    vr = np.array([sx[i] - sx[j], sy[i] - sy[j], sz[i] - sz[j]])
    g = np.linalg.norm(vr)
    assert g > 0
    vrp_out = np.array([vx[i] - vx[j], vy[i] - vy[j], vz[i] - vz[j]])
    # the rotated vector keeps |v_r| and makes the angle 0.7 with v_r (if i, j
    # take part in no later pair of the step)
    later = np.concatenate([pr["i"][1:], pr["j"][1:]])
    if i not in later and j not in later:
        assert abs(np.linalg.norm(vrp_out) - g) < 1e-10 * g
        assert abs(np.dot(vr, vrp_out) / g ** 2 - math.cos(float(np.float32(0.7)))) < 1e-12


# ------------------------------------------------------------------ transport integrals (reading R8)

def test_transport_hard_sphere_closed_forms():
    """Rigid spheres (b_max = d, so the u-integrand is a polynomial and the rule
    exact): Q2 = (2/3) pi d^2, Omega22 = pi d^2 and Eq. (chapman_enskog) gives the
    textbook first-order viscosity 5/16 sqrt(pi m k T) / (pi d^2)."""
    hs = O.make_pot(W.HARD_SPHERE_AR)
    d = 3.6e-10
    q = O.transport_q2(hs, [10.0, 1e3, 1e5], 3.6, b_panels=4)
    assert np.allclose(q, 2 / 3 * math.pi * d * d, rtol=1e-12, atol=0)
    T = np.array([300.0, 3000.0])
    om, mu = O.transport_viscosity(hs, W.M_AR, T, 3.6, b_panels=4, x_panels=8)
    assert np.allclose(om, math.pi * d * d, rtol=1e-12, atol=0)
    want = 5 / 16 * np.sqrt(math.pi * W.M_AR * KB * T) / (math.pi * d * d)
    assert np.allclose(mu, want, rtol=1e-12, atol=0)


def test_transport_inverse_power_scaling():
    """V = kappa/r^p: chi depends on b (E/kappa)^(1/p) only, so Q2 ~ E^(-2/p),
    and the Maxwellian average gives Omega22(T) = Q2(E = kT) Gamma(4 - 2/p)/4
    exactly; mu ~ T^(1/2 + 2/p).  (b_max = 12 A, where sin^2 chi < 1e-12.)"""
    p = 12.0
    P = O.make_pot(dict(kind=2, kappa=1.3e9, p=p))
    q = O.transport_q2(P, [300.0, 3000.0], 12.0, b_panels=8)
    assert abs(q[1] / q[0] - 10.0 ** (-2 / p)) < 1e-8
    om, mu = O.transport_viscosity(P, W.M_AR, [1000.0], 12.0, b_panels=8, x_panels=8)
    q1000 = O.transport_q2(P, [1000.0], 12.0, b_panels=8)[0]
    # the rule applied to the scaled integrand (implementation: weights, x^3 e^-x, 1/4)
    x, wx = O.composite_gl(8, 0.0, O.X_MAX)
    assert abs(om[0] / (q1000 * np.sum(wx * x ** (3 - 2 / p) * np.exp(-x)) / 4) - 1) < 1e-9
    # and against the closed form (the 8-panel rule's own error on x^(3-2/p) e^-x is 2.9e-8)
    assert abs(om[0] / (q1000 * math.gamma(4 - 2 / p) / 4) - 1) < 1e-7
    want = 5 / 16 * math.sqrt(math.pi * W.M_AR * KB * 1000.0) / om[0]
    assert abs(mu[0] / want - 1) < 1e-14


# ------------------------------------------------------------------ chi-MLP surrogate (reading R9)

def _chi_torch(torch, wts):
    from oracle.train import split_layers, split_bias
    Ws, bs = split_layers(wts["dims"], wts["W"]), split_bias(wts["dims"], wts["bias"])
    layers = []
    for l in range(6):
        lin = torch.nn.Linear(wts["dims"][l], wts["dims"][l + 1]).double()
        lin.weight.data = torch.tensor(Ws[l]); lin.bias.data = torch.tensor(bs[l])
        layers += [lin, torch.nn.SiLU() if l < 5 else torch.nn.Softplus()]
    return layers


def test_chi_mlp_forward_matches_torch_sequential():
    """Fig. nn_architecture: 2 -> 512, 512, 512, 256, 128 (SiLU) -> 1 (Softplus);
    FP64 against torch nn.Sequential, and the bf16-storage emulation against the
    same network with torch's bf16 rounding applied where the kernel stores."""
    torch = pytest.importorskip("torch")
    wts = W.chi_mlp_weights()
    layers = _chi_torch(torch, wts)
    x = np.random.default_rng(4).uniform(0, 1, (40, 2))
    y = O.chi_mlp_forward(wts["W"], wts["bias"], x)
    ref = torch.nn.Sequential(*layers)(torch.tensor(x)).detach().numpy()[:, 0]
    np.testing.assert_allclose(y, ref, rtol=1e-12, atol=1e-14)
    assert np.all(y >= 0)
    xt = torch.tensor(x)
    hi = xt.to(torch.bfloat16).double()
    h = hi + (xt - hi).to(torch.bfloat16).double()
    for l in range(6):
        h = layers[2 * l + 1](layers[2 * l](h))
        if l < 4:
            h = h.to(torch.bfloat16).double()
    yb = O.chi_mlp_forward(wts["W"], wts["bias"], x, bf16=True)
    np.testing.assert_allclose(yb, h.detach().numpy()[:, 0], rtol=1e-12, atol=1e-14)


def test_chi_mlp_table_is_forward_at_the_nodes():
    wts = W.chi_mlp_weights()
    T = O.chi_mlp_table(wts["W"], wts["bias"], 5, 3)
    y = O.chi_mlp_forward(wts["W"], wts["bias"], [[1.0, 0.25], [0.0, 1.0]])
    assert T.shape == (3, 5)
    np.testing.assert_allclose([T[2, 1], T[0, 4]], np.expm1(y), rtol=1e-15)
    assert np.all(T >= 0)


# ------------------------------------------------------------------ threads and the given-chi mode

def test_oracle_results_do_not_depend_on_threads():
    """The oracle's parallel loops (cells, independent pairs, table nodes)
    must reproduce its sequential results bit for bit."""
    w = W.hypersonic(scale=0.05)
    P = O.make_pot(W.JAGER_SYNTHETIC_AR)
    wts = W.mlp_weights()
    mlp = O.make_mlp(8, 128, 3, 3, 0, W.sigma_v(), 273.0, 1e-12)
    table = O.chi_table(P, 12.0, 33, 17, math.log(5.0), math.log(6e4)).astype(np.float32)
    runs = []
    n0 = O.num_threads()
    try:
        for nt in (1, max(2, n0)):
            O.set_num_threads(nt)
            gas = O.make_gas(**dict(w["gas"], model=1))
            sg = O.sigma_g_max_init(gas, w["T_cell"], 5.0)
            perm, cs, sx, sy, sz = O.sort_cells(w["cell_id"], w["vx"], w["vy"], w["vz"], w["n_cells"])
            mom = O.cell_moments(cs, sx, sy, sz)
            pr = O.select_pairs(gas, cs, sx, sy, sz, sg, 2, capacity=1 << 20)
            out = [mom, pr["sgmax"], pr["i"], pr["j"], pr["round"]]
            out += list(O.collide_vhs(gas, pr, 2, sx, sy, sz))
            out += list(O.collide_neural(gas, mlp, wts["W"], wts["bias"], mom, pr, 2, sx, sy, sz))
            out += list(O.collide_table(gas, table, math.log(5.0), math.log(6e4), pr, 2, sx, sy, sz))
            sub = {k: (v[:400] if isinstance(v, np.ndarray) else v) for k, v in pr.items()}
            sub["n_pairs"] = min(400, pr["n_pairs"])
            out += list(O.collide_jager(gas, P, sub, 2, sx, sy, sz))
            out += list(O.moment_match(cs, mom, *O.collide_vhs(gas, pr, 2, sx, sy, sz)))
            out.append(O.chi_batch(gas, P, *W.chi_pairs(300, seed=4)))
            runs.append(out)
    finally:
        O.set_num_threads(n0)
    for a, b in zip(*runs):
        assert np.array_equal(a, b)


def test_given_chi_mode_reproduces_the_jager_collide():
    """Fed the Jager collide's own chi, the given-chi mode must give the same
    velocities bit for bit (same rotation, azimuth and update), and record
    each pair's pre-collision v_r."""
    w = W.hypersonic(scale=0.03)
    gas = O.make_gas(**dict(w["gas"], model=1))
    P = O.make_pot(W.JAGER_SYNTHETIC_AR)
    sg = O.sigma_g_max_init(gas, w["T_cell"], 5.0)
    perm, cs, sx, sy, sz = O.sort_cells(w["cell_id"], w["vx"], w["vy"], w["vz"], w["n_cells"])
    pr = O.select_pairs(gas, cs, sx, sy, sz, sg, 5, capacity=1 << 20)
    *ref, chi = O.collide_jager(gas, P, pr, 5, sx, sy, sz, want_chi=True)
    *got, vr, b_imp = O.collide_given_chi(gas, pr, 5, chi, sx, sy, sz, want_vr=True)
    for x, y in zip(ref, got):
        assert np.array_equal(x, y)
    # the first pair of each cell sees the input velocities
    first = np.r_[0, np.flatnonzero(np.diff(pr["cell"])) + 1]
    i, j = pr["i"][first], pr["j"][first]
    np.testing.assert_array_equal(vr[first], np.stack([sx[i] - sx[j], sy[i] - sy[j], sz[i] - sz[j]], 1))
    # its impact parameters reproduce the collide's chi
    E = O.e_kelvin(W.M_AR, np.linalg.norm(vr, axis=1))
    np.testing.assert_allclose(O.chi_many(P, b_imp[:200], E[:200]), chi[:200], rtol=1e-9, atol=1e-12)
