"""Seeded synthetic inputs shaped like the paper's flows.

This module holds no arithmetic of the method: it draws particles, cell
indices, pair parameters and network weights with numpy's seeded generator
and returns plain arrays.  Both the CUDA library and the CPU oracle consume
exactly these arrays.

Gases (argon, m = 6.63e-26 kg, Sec. 3.1):

* ``couette``    -- 100 cells x 50 particles, Maxwellian 273 K plus a linear
  x-velocity from -100 to +100 m/s (shape of the Couette runs, Sec. 3.2).
* ``cavity``     -- 200 x 200 cells, Poisson(20) particles per cell, 273 K plus
  a solid-body rotation of peak 100 m/s (shape of the lid-driven cavity,
  Sec. 3.3: Kn 0.1, L = 1 mm gives n = 1.294e22 m^-3).
* ``hypersonic`` -- 500 x 300 cells around a solid disc (radius 60 cells);
  density, temperature and velocity follow a tanh shock profile from the
  Mach 10 free stream (40 per cell, 200 K, 2634.1 m/s, n = 4.247e20 m^-3,
  Sec. 3.5) to 250 per cell at 8000 K next to the disc.

Particles are generated cell by cell and then shuffled, so that the cell
sort has real work to do.
"""
from __future__ import annotations

import math

import numpy as np

KB = 1.380649e-23
M_AR = 6.63e-26

# SYNTHETIC Argon-like parameters of the Jager potential FORM (Eq. jager_potential,
# Eq. damping; r in Angstrom, V/k_B in Kelvin).  The paper prints no coefficients.
# Textbook Ar dispersion magnitudes; A and a1 put the well at 3.757 A, -143.2 K;
# At, at make V and V' continuous at 0.4 R_eps.  Derived by
# oracle/fit_jager_synthetic.py.
JAGER_SYNTHETIC_AR = dict(
    kind=0,
    A=114415969.03,
    a1=-3.4946784034,
    a2=-0.012,
    am1=-0.35,
    am2=0.05,
    beta=3.84,
    C=[445857.0, 3151413.0, 26675750.0, 270414200.0, 3282794000.0, 47726480000.0],
    R_eps=3.757,
    At=45831936.4256,
    at=2.890909017194,
)

HARD_SPHERE_AR = dict(kind=1, d_hs=3.6)  # d = 3.6e-10 m


def _shuffle(rng, cell_id, vx, vy, vz):
    p = rng.permutation(len(cell_id))
    return (np.ascontiguousarray(cell_id[p], np.int32), np.ascontiguousarray(vx[p]),
            np.ascontiguousarray(vy[p]), np.ascontiguousarray(vz[p]))


def _gas(**kw):
    base = dict(mass=M_AR, d_ref=4.17e-10, omega=0.81, T_ref=273.0, fn_over_vc=2e18,
                dt=1e-7, seed=0, model=0, b_max=1.2e-9)
    base.update(kw)
    return base


def _particles(rng, counts, T, ux, uy):
    """Maxwellian velocities per cell: v ~ N(u_k, k T_k / m) per component."""
    counts = np.asarray(counts, np.int64)
    cell_id = np.repeat(np.arange(len(counts), dtype=np.int32), counts)
    s = np.sqrt(KB * np.repeat(np.asarray(T, np.float64), counts) / M_AR)
    n = int(counts.sum())
    vx = rng.standard_normal(n) * s + np.repeat(np.asarray(ux, np.float64), counts)
    vy = rng.standard_normal(n) * s + np.repeat(np.asarray(uy, np.float64), counts)
    vz = rng.standard_normal(n) * s
    return cell_id, vx, vy, vz


def couette(seed=0, n_cells=100, per_cell=50, T=273.0, u_wall=100.0):
    rng = np.random.default_rng(seed)
    k = np.arange(n_cells)
    ux = -u_wall + 2.0 * u_wall * (k + 0.5) / n_cells
    cell_id, vx, vy, vz = _particles(rng, np.full(n_cells, per_cell), np.full(n_cells, T), ux,
                                     np.zeros(n_cells))
    cell_id, vx, vy, vz = _shuffle(rng, cell_id, vx, vy, vz)
    return dict(name=f"couette {n_cells}x{per_cell}", n_cells=n_cells, cell_id=cell_id,
                vx=vx, vy=vy, vz=vz, T_cell=np.full(n_cells, T),
                gas=_gas(fn_over_vc=1e20 / per_cell, dt=1e-7, seed=seed))


def cavity(seed=0, nx=200, ny=200, mean=20.0, T=273.0, u_peak=100.0, dt=5.3e-8):
    rng = np.random.default_rng(seed)
    counts = rng.poisson(mean, nx * ny)
    ix, iy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    x = (ix.ravel() + 0.5) - 0.5 * nx
    y = (iy.ravel() + 0.5) - 0.5 * ny
    rmax = math.hypot(0.5 * nx, 0.5 * ny)
    # solid-body rotation: u = omega x r with |u| = u_peak r / r_max
    ux = -u_peak * y / rmax
    uy = u_peak * x / rmax
    cell_id, vx, vy, vz = _particles(rng, counts, np.full(nx * ny, T), ux, uy)
    cell_id, vx, vy, vz = _shuffle(rng, cell_id, vx, vy, vz)
    return dict(name=f"cavity {nx}x{ny} Poisson({mean:g})", n_cells=nx * ny, cell_id=cell_id,
                vx=vx, vy=vy, vz=vz, T_cell=np.full(nx * ny, T),
                gas=_gas(fn_over_vc=1.294e22 / mean, dt=dt, seed=seed))


def hypersonic(seed=0, nx=500, ny=300, radius=60.0, cx=350.0, cy=150.0, scale=1.0,
               model=1):
    """Mach-10 argon gas around a disc.  ``scale`` < 1 shrinks the box and the
    disc together (same profile in cell units) for small test cases."""
    rng = np.random.default_rng(seed)
    nx_s, ny_s = max(4, int(round(nx * scale))), max(4, int(round(ny * scale)))
    R, X0, Y0 = radius * scale, cx * scale, cy * scale
    width, thick = 35.0 * scale, 6.0 * scale
    ix, iy = np.meshgrid(np.arange(nx_s), np.arange(ny_s), indexing="ij")
    d = np.hypot(ix.ravel() + 0.5 - X0, iy.ravel() + 0.5 - Y0) - R
    s = 0.5 * (1.0 - np.tanh((d - width) / max(thick, 1e-9)))
    solid = d < 0.0
    lam = np.where(solid, 0.0, 40.0 + 210.0 * s)
    counts = rng.poisson(lam)
    T = 200.0 + 7800.0 * s
    ux = 2634.1 * (1.0 - 0.9 * s)
    cell_id, vx, vy, vz = _particles(rng, counts, T, ux, np.zeros_like(ux))
    cell_id, vx, vy, vz = _shuffle(rng, cell_id, vx, vy, vz)
    return dict(name=f"hypersonic {nx_s}x{ny_s} disc r={R:g}", n_cells=nx_s * ny_s,
                cell_id=cell_id, vx=vx, vy=vy, vz=vz, T_cell=T,
                gas=_gas(fn_over_vc=4.247e20 / 40.0, dt=1e-7, seed=seed, model=model,
                         b_max=1.2e-9))


def chi_pairs(n=1 << 22, seed=0, b_max_A=12.0, g_lo=300.0, g_ratio=50.0):
    """Pair batch of the Jager deflection-angle workload: g = 300*50^U m/s,
    b = b_max sqrt(U) (uniform in b^2), both float32; b in Angstrom."""
    rng = np.random.default_rng(seed)
    g = (g_lo * g_ratio ** rng.random(n)).astype(np.float32)
    b = (b_max_A * np.sqrt(rng.random(n))).astype(np.float32)
    return b, g


def harvest_inputs(n=1 << 20, seed=0, b_max_A=12.0):
    """Random pre-collision pairs for training-data harvesting: g log-uniform
    in [300, 15000] m/s, direction of v_r uniform on the sphere, centre of mass
    Maxwellian at T log-uniform in [200, 8000] K, b uniform in b^2, eps uniform."""
    rng = np.random.default_rng(seed)
    g = 300.0 * 50.0 ** rng.random(n)
    mu = 2.0 * rng.random(n) - 1.0
    ph = 2.0 * np.pi * rng.random(n)
    st = np.sqrt(1.0 - mu * mu)
    e = np.stack([mu, st * np.cos(ph), st * np.sin(ph)], 1)
    T = 200.0 * 40.0 ** rng.random(n)
    vcm = rng.standard_normal((n, 3)) * np.sqrt(KB * T / (2.0 * M_AR))[:, None]
    vr = g[:, None] * e
    vi = vcm + 0.5 * vr
    vj = vcm - 0.5 * vr
    b = b_max_A * np.sqrt(rng.random(n))
    eps = 2.0 * np.pi * rng.random(n)
    return dict(vi=np.ascontiguousarray(vi), vj=np.ascontiguousarray(vj), b=b, eps=eps, T=T)


def bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round float64 values to bfloat16 (nearest even); return the raw bits."""
    f = np.ascontiguousarray(x, np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return u.astype(np.uint16)


def bf16_value(bits: np.ndarray) -> np.ndarray:
    return (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def mlp_weights(d_in=8, width=128, n_hidden=3, d_out=3, seed=1):
    """Xavier-uniform weights (a = sqrt(6/(fan_in+fan_out))), zero biases,
    rounded to bf16.  Layers are row-major [out x in], concatenated."""
    rng = np.random.default_rng(seed)
    dims = [d_in] + [width] * n_hidden + [d_out]
    ws, bs = [], []
    for l in range(len(dims) - 1):
        a = math.sqrt(6.0 / (dims[l] + dims[l + 1]))
        ws.append(rng.uniform(-a, a, size=(dims[l + 1], dims[l])).ravel())
        bs.append(np.zeros(dims[l + 1]))
    W = np.concatenate(ws)
    bits = bf16_bits(W)
    return dict(dims=dims, W_bits=bits, W=bf16_value(bits),
                bias=np.concatenate(bs).astype(np.float32).astype(np.float64))


# chi-MLP surrogate (Fig. nn_architecture): inputs [ln(E_r)*, b/b_max], five
# SiLU hidden layers, one Softplus output
CHI_MLP_DIMS = [2, 512, 512, 512, 256, 128, 1]


def chi_mlp_weights(seed=3):
    """Xavier-uniform weights rounded to bf16 and small uniform biases (the
    trained weights are not available), layers row-major [out x in],
    concatenated."""
    rng = np.random.default_rng(seed)
    dims = CHI_MLP_DIMS
    ws, bs = [], []
    for l in range(len(dims) - 1):
        a = math.sqrt(6.0 / (dims[l] + dims[l + 1]))
        ws.append(rng.uniform(-a, a, size=(dims[l + 1], dims[l])).ravel())
        bs.append(rng.uniform(-0.1, 0.1, size=dims[l + 1]))
    W = np.concatenate(ws)
    bits = bf16_bits(W)
    return dict(dims=dims, W_bits=bits, W=bf16_value(bits),
                bias=np.concatenate(bs).astype(np.float32).astype(np.float64))


def sigma_v(T_ref=273.0, mass=M_AR):
    """Scale of one relative-velocity component at T_ref: sqrt(2 k T_ref / m)."""
    return math.sqrt(2.0 * KB * T_ref / mass)
