"""FP64 CPU oracle of the DSMC collision step (arXiv 2602.21244).

TEST INFRASTRUCTURE ONLY: only tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library never calls it, and it shares no code with it.

The heavy parts are plain C in ``dsmc_oracle.c`` (built here with gcc,
``-ffp-contract=off``); the training oracle is numpy in ``train.py``.  Every
function cites the section or equation of the paper it follows; readings of
silent or ambiguous passages are listed in the C file header.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dsmc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

KB = 1.380649e-23

# Philox tags (reading R1 of the oracle header)
TAG_NTC, TAG_CAND, TAG_ISO, TAG_JAGER, TAG_NOISE, TAG_HARVEST = 1, 2, 3, 4, 5, 6


def build(force: bool = False, openmp: bool = True) -> str:
    """Compile the C oracle with gcc (no FMA contraction), with OpenMP where
    the compiler has it (the results do not depend on the thread count)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                    "-o", _LIB + ".tmp", _SRC, "-lm"]
            r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True) if openmp else None
            if r is None or r.returncode != 0:
                subprocess.run(base, check=True)
            os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class Gas(C.Structure):
    _fields_ = [("mass", C.c_double), ("d_ref", C.c_double), ("omega", C.c_double),
                ("T_ref", C.c_double), ("fn_over_vc", C.c_double), ("dt", C.c_double),
                ("seed", C.c_uint64), ("model", C.c_int32), ("pad_", C.c_int32),
                ("b_max", C.c_double)]


class Pot(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pad_", C.c_int32), ("A", C.c_double),
                ("a1", C.c_double), ("a2", C.c_double), ("am1", C.c_double),
                ("am2", C.c_double), ("beta", C.c_double), ("C", C.c_double * 6),
                ("R_eps", C.c_double), ("At", C.c_double), ("at", C.c_double),
                ("d_hs", C.c_double), ("kappa", C.c_double), ("p", C.c_double)]


class Mlp(C.Structure):
    _fields_ = [("d_in", C.c_int32), ("width", C.c_int32), ("n_hidden", C.c_int32),
                ("d_out", C.c_int32), ("act", C.c_int32), ("pad_", C.c_int32),
                ("sigma_v", C.c_double), ("T_ref", C.c_double), ("eps", C.c_double)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P = C.POINTER
        d, i32, i64, u32, u64 = C.c_double, C.c_int32, C.c_int64, C.c_uint32, C.c_uint64
        vp = C.c_void_p
        sig = {
            "or_philox4x32_10": (None, [vp, vp, vp]),
            "or_philox_stream": (None, [u64, u32, u64, u32, u32, i64, vp]),
            "or_u53": (d, [u32, u32]),
            "or_sigma": (d, [P(Gas), d]),
            "or_sigma_g_max_init": (None, [P(Gas), i32, vp, d, vp]),
            "or_sort_cells": (C.c_int, [i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp]),
            "or_cell_moments": (None, [i32, vp, vp, vp, vp, vp]),
            "or_select_pairs": (C.c_int, [P(Gas), i32, vp, vp, vp, vp, vp, u64, i64,
                                          vp, vp, vp, vp, vp, vp, vp, vp]),
            "or_collide_vhs": (None, [P(Gas), i64, vp, vp, vp, vp, u64, vp, vp, vp]),
            "or_moment_match": (None, [i32, vp, vp, vp, vp, vp]),
            "or_tt_damp": (d, [i32, d]),
            "or_pot_V": (d, [P(Pot), d]),
            "or_pot_dV": (d, [P(Pot), d]),
            "or_rmin": (d, [P(Pot), d, d]),
            "or_chi": (d, [P(Pot), d, d]),
            "or_chi_batch": (None, [P(Gas), P(Pot), i64, vp, vp, vp]),
            "or_deflect": (None, [vp, d, d, vp]),
            "or_collide_jager": (None, [P(Gas), P(Pot), i64, vp, vp, vp, vp, u64, vp, vp, vp, vp]),
            "or_collide_given_chi": (None, [P(Gas), i64, vp, vp, vp, vp, u64, vp, vp, vp, vp, vp, vp]),
            "or_chi_many": (None, [P(Pot), i64, vp, vp, vp]),
            "or_num_threads": (C.c_int, []),
            "or_set_num_threads": (None, [C.c_int]),
            "or_bf16_round": (d, [d]),
            "or_mlp_forward": (None, [P(Mlp), vp, vp, i64, vp, C.c_int, vp]),
            "or_noise4": (None, [u64, i32, i32, u64, vp]),
            "or_neural_features": (None, [P(Mlp), vp, d, vp, vp]),
            "or_collide_neural": (None, [P(Gas), P(Mlp), vp, vp, vp, i64, vp, vp, vp, vp, u64,
                                         C.c_int, vp, vp, vp, vp]),
            "or_harvest_jager": (None, [P(Gas), P(Pot), i64, vp, vp, vp, vp, vp, vp]),
            "or_chi_table": (None, [P(Pot), d, i32, i32, d, d, vp]),
            "or_chi_lookup": (d, [vp, i32, i32, d, d, d, d]),
            "or_collide_table": (None, [P(Gas), vp, i32, i32, d, d, i64, vp, vp, vp, vp, u64, vp, vp, vp, vp]),
            "or_transport_q2": (d, [P(Pot), d, d, i32, vp, vp]),
            "or_transport_viscosity": (None, [P(Pot), d, i32, vp, d, i32, vp, vp, i32, vp, vp, vp, vp]),
            "or_chi_mlp_forward": (None, [vp, vp, i64, vp, C.c_int, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


# ----------------------------------------------------------------- struct helpers

def make_gas(mass, d_ref, omega, T_ref, fn_over_vc, dt, seed, model=0, b_max=0.0) -> Gas:
    return Gas(mass, d_ref, omega, T_ref, fn_over_vc, dt, seed, model, 0, b_max)


def make_pot(p: dict) -> Pot:
    P = Pot()
    P.kind = int(p.get("kind", 0))
    for k in ("A", "a1", "a2", "am1", "am2", "beta", "R_eps", "At", "at", "d_hs", "kappa", "p"):
        setattr(P, k, float(p.get(k, 0.0)))
    Cs = p.get("C", [0.0] * 6)
    for q in range(6):
        P.C[q] = float(Cs[q])
    return P


def make_mlp(d_in, width, n_hidden, d_out, act, sigma_v, T_ref, eps) -> Mlp:
    return Mlp(d_in, width, n_hidden, d_out, act, 0, sigma_v, T_ref, eps)


# ----------------------------------------------------------------- Philox (R1)

def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def philox_stream(seed, cell, step, tag, sub, n) -> np.ndarray:
    out = np.zeros((n, 4), np.uint32)
    lib().or_philox_stream(seed, cell, step, tag, sub, n, _p(out))
    return out


def u53(a, b) -> float:
    return lib().or_u53(int(a), int(b))


# ----------------------------------------------------------------- step pieces

def sigma(gas: Gas, g: float) -> float:
    return lib().or_sigma(C.byref(gas), g)


def sigma_g_max_init(gas: Gas, T: np.ndarray, factor: float = 5.0) -> np.ndarray:
    T = _f64(T)
    out = np.zeros_like(T)
    lib().or_sigma_g_max_init(C.byref(gas), len(T), _p(T), factor, _p(out))
    return out


def sort_cells(cell_id, vx, vy, vz, n_cells):
    """Stable counting sort by cell (Sec. 2.6 (1))."""
    cid = _i32(cell_id)
    vx, vy, vz = _f64(vx), _f64(vy), _f64(vz)
    n = len(cid)
    perm = np.zeros(n, np.int32)
    cs = np.zeros(n_cells + 1, np.int32)
    s = [np.zeros(n) for _ in range(3)]
    rc = lib().or_sort_cells(n, n_cells, _p(cid), _p(vx), _p(vy), _p(vz), _p(perm), _p(cs),
                             _p(s[0]), _p(s[1]), _p(s[2]))
    if rc != 0:
        raise ValueError("cell id out of range")
    return perm, cs, s[0], s[1], s[2]


def cell_moments(cell_start, vx, vy, vz) -> np.ndarray:
    cs = _i32(cell_start)
    nc = len(cs) - 1
    mom = np.zeros((nc, 5))
    lib().or_cell_moments(nc, _p(cs), _p(_f64(vx)), _p(_f64(vy)), _p(_f64(vz)), _p(mom))
    return mom


def select_pairs(gas: Gas, cell_start, vx, vy, vz, sgmax, step, capacity=None):
    """NTC selection, readings R2-R4.  Returns a dict of cell-major pair
    arrays (candidate order) and the updated (sigma g)_max."""
    cs = _i32(cell_start)
    nc = len(cs) - 1
    sg = _f64(sgmax).copy()
    if capacity is None:
        capacity = 1 << 20
    arrs = [np.zeros(capacity, np.int32) for _ in range(5)]
    n_pairs = C.c_int64(0)
    n_cand = C.c_int64(0)
    n_rounds = C.c_int32(0)
    rc = lib().or_select_pairs(C.byref(gas), nc, _p(cs), _p(_f64(vx)), _p(_f64(vy)), _p(_f64(vz)),
                               _p(sg), step, capacity, *[_p(a) for a in arrs],
                               C.byref(n_pairs), C.byref(n_cand), C.byref(n_rounds))
    if rc != 0:
        raise RuntimeError(f"oracle select: capacity {capacity} < {n_pairs.value}")
    n = n_pairs.value
    i, j, cell, m, rnd = (a[:n].copy() for a in arrs)
    return dict(i=i, j=j, cell=cell, m=m, round=rnd, n_pairs=n, n_cand=n_cand.value,
                n_rounds=n_rounds.value, sgmax=sg)


def collide_vhs(gas: Gas, pairs: dict, step, vx, vy, vz):
    vx, vy, vz = _f64(vx).copy(), _f64(vy).copy(), _f64(vz).copy()
    lib().or_collide_vhs(C.byref(gas), pairs["n_pairs"], _p(pairs["i"]), _p(pairs["j"]),
                         _p(pairs["cell"]), _p(pairs["m"]), step, _p(vx), _p(vy), _p(vz))
    return vx, vy, vz


def moment_match(cell_start, mom_pre, vx, vy, vz):
    cs = _i32(cell_start)
    vx, vy, vz = _f64(vx).copy(), _f64(vy).copy(), _f64(vz).copy()
    lib().or_moment_match(len(cs) - 1, _p(cs), _p(_f64(mom_pre)), _p(vx), _p(vy), _p(vz))
    return vx, vy, vz


# ----------------------------------------------------------------- potentials / chi

def tt_damp(n: int, x: float) -> float:
    return lib().or_tt_damp(n, x)


def pot_V(pot: Pot, r: float) -> float:
    return lib().or_pot_V(C.byref(pot), r)


def pot_dV(pot: Pot, r: float) -> float:
    return lib().or_pot_dV(C.byref(pot), r)


def rmin(pot: Pot, b: float, E: float) -> float:
    return lib().or_rmin(C.byref(pot), b, E)


def chi(pot: Pot, b: float, E: float) -> float:
    """Signed deflection angle, b in Angstrom, E = E_r/k_B in Kelvin."""
    return lib().or_chi(C.byref(pot), b, E)


def chi_batch(gas: Gas, pot: Pot, b, g) -> np.ndarray:
    b, g = _f64(b), _f64(g)
    out = np.zeros_like(b)
    lib().or_chi_batch(C.byref(gas), C.byref(pot), len(b), _p(b), _p(g), _p(out))
    return out


def e_kelvin(mass: float, g):
    return 0.25 * mass * np.asarray(g, dtype=np.float64) ** 2 / KB


def deflect(vr, chi_v, eps):
    vr = _f64(vr)
    out = np.zeros(3)
    lib().or_deflect(_p(vr), chi_v, eps, _p(out))
    return out


def collide_jager(gas: Gas, pot: Pot, pairs: dict, step, vx, vy, vz, want_chi=False):
    vx, vy, vz = _f64(vx).copy(), _f64(vy).copy(), _f64(vz).copy()
    chi_out = np.zeros(max(pairs["n_pairs"], 1))
    lib().or_collide_jager(C.byref(gas), C.byref(pot), pairs["n_pairs"], _p(pairs["i"]),
                           _p(pairs["j"]), _p(pairs["cell"]), _p(pairs["m"]), step,
                           _p(vx), _p(vy), _p(vz), _p(chi_out))
    if want_chi:
        return vx, vy, vz, chi_out[:pairs["n_pairs"]]
    return vx, vy, vz


def collide_given_chi(gas: Gas, pairs: dict, step, chi, vx, vy, vz, want_vr=False):
    """The rotation and centre-of-mass update of the Jager collide with each
    pair's chi given (pair order, e.g. a GPU kernel's own chi) and the
    azimuth from tag 4.  want_vr: also each pair's pre-collision v_r [n x 3]
    and impact parameter b (Angstrom, tag 4)."""
    vx, vy, vz = _f64(vx).copy(), _f64(vy).copy(), _f64(vz).copy()
    n = pairs["n_pairs"]
    chi = _f64(chi)
    assert len(chi) >= n
    vr = np.zeros((max(n, 1), 3))
    b = np.zeros(max(n, 1))
    lib().or_collide_given_chi(C.byref(gas), n, _p(_i32(pairs["i"])), _p(_i32(pairs["j"])),
                               _p(_i32(pairs["cell"])), _p(_i32(pairs["m"])), step, _p(chi), _p(vx), _p(vy),
                               _p(vz), _p(vr), _p(b))
    if want_vr:
        return vx, vy, vz, vr[:n], b[:n]
    return vx, vy, vz


def chi_many(pot: Pot, b, E) -> np.ndarray:
    """chi at independent points (b in Angstrom, E = E_r/k_B in K)."""
    b, E = _f64(b), _f64(E)
    out = np.zeros_like(b)
    lib().or_chi_many(C.byref(pot), len(b), _p(b), _p(E), _p(out))
    return out


def num_threads() -> int:
    """Threads of the oracle's parallel loops (1 if built without OpenMP)."""
    return int(lib().or_num_threads())


def set_num_threads(n: int) -> None:
    lib().or_set_num_threads(int(n))


def chi_table(pot: Pot, bmax_A: float, nb: int, nE: int, lnE_min: float, lnE_max: float) -> np.ndarray:
    """[nE x nb] table of chi on the uniform (b/b_max, ln E) grid (FP64)."""
    out = np.zeros((nE, nb))
    lib().or_chi_table(C.byref(pot), bmax_A, nb, nE, lnE_min, lnE_max, _p(out))
    return out


def chi_lookup(table, lnE_min: float, lnE_max: float, bt: float, lnE: float) -> float:
    t = np.ascontiguousarray(table, dtype=np.float32)
    nE, nb = t.shape
    return lib().or_chi_lookup(_p(t), nb, nE, lnE_min, lnE_max, bt, lnE)


def collide_table(gas: Gas, table, lnE_min: float, lnE_max: float, pairs: dict, step, vx, vy, vz,
                  want_chi=False):
    t = np.ascontiguousarray(table, dtype=np.float32)
    nE, nb = t.shape
    vx, vy, vz = _f64(vx).copy(), _f64(vy).copy(), _f64(vz).copy()
    chi_out = np.zeros(max(pairs["n_pairs"], 1))
    lib().or_collide_table(C.byref(gas), _p(t), nb, nE, lnE_min, lnE_max, pairs["n_pairs"], _p(pairs["i"]),
                           _p(pairs["j"]), _p(pairs["cell"]), _p(pairs["m"]), step, _p(vx), _p(vy), _p(vz),
                           _p(chi_out))
    if want_chi:
        return vx, vy, vz, chi_out[:pairs["n_pairs"]]
    return vx, vy, vz


def harvest_jager(gas: Gas, pot: Pot, vi, vj, b, eps):
    vi, vj, b, eps = _f64(vi), _f64(vj), _f64(b), _f64(eps)
    n = len(b)
    vio, vjo = np.zeros((n, 3)), np.zeros((n, 3))
    lib().or_harvest_jager(C.byref(gas), C.byref(pot), n, _p(vi), _p(vj), _p(b), _p(eps),
                           _p(vio), _p(vjo))
    return vio, vjo


# ----------------------------------------------------------------- neural path

def bf16_round(x: float) -> float:
    return lib().or_bf16_round(x)


def mlp_forward(mlp: Mlp, W: np.ndarray, bias: np.ndarray, x: np.ndarray, bf16=False):
    x = _f64(x)
    n = x.shape[0]
    y = np.zeros((n, mlp.d_out))
    lib().or_mlp_forward(C.byref(mlp), _p(_f64(W)), _p(_f64(bias)), n, _p(x), int(bf16), _p(y))
    return y


def noise4(seed, cell, m, step) -> np.ndarray:
    z = np.zeros(4)
    lib().or_noise4(seed, cell, m, step, _p(z))
    return z


def collide_neural(gas: Gas, mlp: Mlp, W, bias, mom_pre, pairs: dict, step, vx, vy, vz,
                   bf16=False, want_u=False):
    vx, vy, vz = _f64(vx).copy(), _f64(vy).copy(), _f64(vz).copy()
    u = np.zeros((max(pairs["n_pairs"], 1), 3))
    lib().or_collide_neural(C.byref(gas), C.byref(mlp), _p(_f64(W)), _p(_f64(bias)),
                            _p(_f64(mom_pre)), pairs["n_pairs"], _p(pairs["i"]), _p(pairs["j"]),
                            _p(pairs["cell"]), _p(pairs["m"]), step, int(bf16),
                            _p(vx), _p(vy), _p(vz), _p(u))
    if want_u:
        return vx, vy, vz, u[:pairs["n_pairs"]]
    return vx, vy, vz


# ----------------------------------------------------------------- whole step

def step(gas: Gas, cell_id, vx, vy, vz, n_cells, sgmax, step_idx, path="vhs",
         pot: Pot | None = None, mlp: Mlp | None = None, W=None, bias=None, bf16=False,
         capacity=None):
    """One collision step: sort, pre moments, NTC selection, collisions of
    one path in candidate order, centred moment matching (Sec. 2.1-2.6)."""
    perm, cs, sx, sy, sz = sort_cells(cell_id, vx, vy, vz, n_cells)
    mom = cell_moments(cs, sx, sy, sz)
    pairs = select_pairs(gas, cs, sx, sy, sz, sgmax, step_idx, capacity)
    if path == "vhs":
        cx, cy, cz = collide_vhs(gas, pairs, step_idx, sx, sy, sz)
    elif path == "jager":
        cx, cy, cz = collide_jager(gas, pot, pairs, step_idx, sx, sy, sz)
    elif path == "neural":
        cx, cy, cz = collide_neural(gas, mlp, W, bias, mom, pairs, step_idx, sx, sy, sz, bf16)
    else:
        raise ValueError(path)
    ox, oy, oz = moment_match(cs, mom, cx, cy, cz)
    return dict(perm=perm, cell_start=cs, mom=mom, pairs=pairs, vx=ox, vy=oy, vz=oz,
                sgmax=pairs["sgmax"])


# ------------------------------------------------------------------ transport integrals (reading R8)
X_MAX = 60.0   # x = E/(kT) range of the Omega(2,2) rule; x^3 e^-x beyond it is below 1e-20


def composite_gl(panels: int, lo: float, hi: float, n: int = 16):
    """Composite Gauss-Legendre rule: `panels` equal panels of [lo, hi], n
    nodes each (numpy's leggauss for the nodes on [-1, 1])."""
    t, w = np.polynomial.legendre.leggauss(n)
    h = (hi - lo) / panels
    xs = np.concatenate([lo + h * (p + 0.5 * (t + 1.0)) for p in range(panels)])
    ws = np.concatenate([0.5 * h * w for _ in range(panels)])
    return xs, ws


def transport_q2(pot: Pot, E_kelvin, bmax_A: float, b_panels: int = 32) -> np.ndarray:
    """Q2(E) in m^2 (reading R8), rule in u = (b/b_max)^2 on [0, 1]."""
    u, wu = composite_gl(b_panels, 0.0, 1.0)
    E = np.atleast_1d(np.asarray(E_kelvin, dtype=np.float64))
    return np.array([lib().or_transport_q2(C.byref(pot), float(e), bmax_A, len(u), _p(u), _p(wu)) for e in E])


def transport_viscosity(pot: Pot, mass: float, T_kelvin, bmax_A: float, b_panels: int = 32,
                        x_panels: int = 8):
    """(Omega22 in m^2, mu in Pa s) at the temperatures T (reading R8)."""
    u, wu = composite_gl(b_panels, 0.0, 1.0)
    x, wx = composite_gl(x_panels, 0.0, X_MAX)
    T = _f64(np.atleast_1d(np.asarray(T_kelvin, dtype=np.float64)))
    om = np.zeros(len(T)); mu = np.zeros(len(T))
    lib().or_transport_viscosity(C.byref(pot), mass, len(T), _p(T), bmax_A, len(u), _p(u), _p(wu),
                                 len(x), _p(x), _p(wx), _p(om), _p(mu))
    return om, mu


# ------------------------------------------------------------------ chi-MLP surrogate (reading R9)
CHI_LNE_MIN, CHI_LNE_MAX = math.log(5.0), math.log(6.0e4)


def chi_mlp_forward(W, bias, x, bf16=False) -> np.ndarray:
    """Softplus output y (~ ln(1 + chi)) of the chi-MLP for inputs x [n x 2] =
    [ln(E_r)*, b/b_max]."""
    x = _f64(np.asarray(x, dtype=np.float64).reshape(-1, 2))
    y = np.zeros(len(x))
    lib().or_chi_mlp_forward(_p(_f64(W)), _p(_f64(bias)), len(x), _p(x), int(bf16), _p(y))
    return y


def chi_mlp_table(W, bias, nb: int, nE: int, bf16=False) -> np.ndarray:
    """The look-up table of Sec. 3.4.4 synthesised by the chi-MLP: node (j, i)
    at ln(E_r)* = j/(nE-1), b/b_max = i/(nb-1), chi = e^y - 1; [nE x nb]."""
    xe = np.repeat(np.arange(nE) / (nE - 1), nb)
    xb = np.tile(np.arange(nb) / (nb - 1), nE)
    y = chi_mlp_forward(W, bias, np.stack([xe, xb], 1), bf16)
    return np.expm1(y).reshape(nE, nb)
