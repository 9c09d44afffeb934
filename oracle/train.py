"""FP64 numpy oracle of one training step of the neural collision operator.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The loss follows the paper's training statement (Sec. 2.6: MSE against the
harvested post-collision state) with the physics layers of Sec. 2.3 and
Sec. 2.5 in the graph:

  x      = [v_r/sigma_v, T/T_ref, xi]                 Eq. (mlp_input)
  y      = f_theta(x)                                  Eq. (mlp_output), SiLU layers (Sec. 3.4.2 layer form)
  v_r'   = |v_r| y/|y|                                 Eq. (energy_shell_projection), reading R6
  v_i'   = v_cm + v_r'/2,  v_j' = v_cm - v_r'/2        Sec. 2.3 pair update
  v_new  = u_pre + alpha (v' - u_post) per group       Eq. (cell_energy_clamp), reading R5
  L      = mean over particles |v_new - v_target|^2 / sigma_v^2

Groups ("pseudo-cells") are G consecutive pairs (2G particles: the G first
particles then the G second ones).  The gradient is written out by hand
(chain rule, layer by layer); Adam follows Kingma & Ba (2015), Algorithm 1.
"""
from __future__ import annotations

import numpy as np

from . import TAG_NOISE, philox_stream


def split_layers(dims, flat):
    out, o = [], 0
    for l in range(len(dims) - 1):
        n = dims[l + 1] * dims[l]
        out.append(flat[o:o + n].reshape(dims[l + 1], dims[l]))
        o += n
    return out


def split_bias(dims, flat):
    out, o = [], 0
    for l in range(len(dims) - 1):
        out.append(flat[o:o + dims[l + 1]])
        o += dims[l + 1]
    return out


def train_noise(seed: int, t: int, n: int) -> np.ndarray:
    """Latent noise of training pair p at step t: Philox tag 5 with counter
    (idx=p, cell=0, step=t), Box-Muller on two 53-bit uniforms per pair of
    normals (subs 0 and 1)."""
    z = np.zeros((n, 4))
    for sub in (0, 1):
        w = philox_stream(seed, 0, t, TAG_NOISE, sub, n).astype(np.uint64)
        u1 = ((w[:, 0] << 32 | w[:, 1]) >> 11).astype(np.float64) * 2.0 ** -53
        u2 = ((w[:, 2] << 32 | w[:, 3]) >> 11).astype(np.float64) * 2.0 ** -53
        rho = np.sqrt(-2.0 * np.log(1.0 - u1))
        z[:, 2 * sub] = rho * np.cos(2.0 * np.pi * u2)
        z[:, 2 * sub + 1] = rho * np.sin(2.0 * np.pi * u2)
    return z


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(dims, W, b, vi, vj, T, xi, vi_t, vj_t, sigma_v, T_ref, group=16, act="silu"):
    """Returns (loss, cache).  W, b are lists of per-layer arrays."""
    n = vi.shape[0]
    vr = vi - vj
    g = np.sqrt(np.sum(vr * vr, 1))
    if dims[0] == 8:
        x = np.concatenate([vr / sigma_v, (T / T_ref)[:, None], xi[:, :4]], 1)
    else:
        x = np.concatenate([vr / sigma_v, xi[:, :3]], 1)
    hs, zs = [x], []
    h = x
    L = len(W)
    for l in range(L):
        z = h @ W[l].T + b[l]
        zs.append(z)
        if l < L - 1:
            h = silu(z) if act == "silu" else np.maximum(z, 0.0)
            hs.append(h)
    y = zs[-1]
    ny = np.sqrt(np.sum(y * y, 1))
    u = y / ny[:, None]
    vrp = g[:, None] * u
    vcm = 0.5 * (vi + vj)
    pi_ = vcm + 0.5 * vrp
    pj_ = vcm - 0.5 * vrp
    # groups of G pairs: particles [pi of the group..., pj of the group...]
    ng = n // group
    P = np.concatenate([pi_.reshape(ng, group, 3), pj_.reshape(ng, group, 3)], 1)
    Q = np.concatenate([vi.reshape(ng, group, 3), vj.reshape(ng, group, 3)], 1)
    Tt = np.concatenate([vi_t.reshape(ng, group, 3), vj_t.reshape(ng, group, 3)], 1)
    u_pre = Q.mean(1, keepdims=True)
    th_pre = np.sum((Q - u_pre) ** 2, (1, 2))
    u_post = P.mean(1, keepdims=True)
    D = P - u_post
    th_post = np.sum(D * D, (1, 2))
    alpha = np.sqrt(th_pre / th_post)
    Vn = u_pre + alpha[:, None, None] * D
    R = (Vn - Tt) / sigma_v
    loss = np.sum(R * R) / (2 * n)
    cache = dict(hs=hs, zs=zs, y=y, ny=ny, u=u, g=g, D=D, th_post=th_post, alpha=alpha,
                 R=R, Vn=Vn, n=n, ng=ng, group=group, act=act)
    return loss, cache


def backward(dims, W, b, cache, sigma_v):
    """Hand-written gradient of the loss of ``forward`` w.r.t. W and b."""
    n, ng, G = cache["n"], cache["ng"], cache["group"]
    Gv = 2.0 * cache["R"] / (sigma_v * 2 * n)           # dL/dVn
    D, alpha, th = cache["D"], cache["alpha"], cache["th_post"]
    Gbar = Gv.mean(1, keepdims=True)
    S = np.sum(Gv * D, (1, 2))
    dP = alpha[:, None, None] * (Gv - Gbar) - (alpha * S / th)[:, None, None] * D
    dpi = dP[:, :G].reshape(n, 3)
    dpj = dP[:, G:].reshape(n, 3)
    dvrp = 0.5 * (dpi - dpj)
    u, ny, g = cache["u"], cache["ny"], cache["g"]
    dy = (g / ny)[:, None] * (dvrp - u * np.sum(u * dvrp, 1, keepdims=True))
    hs, zs = cache["hs"], cache["zs"]
    dW, db = [None] * len(W), [None] * len(W)
    dz = dy
    for l in range(len(W) - 1, -1, -1):
        dW[l] = dz.T @ hs[l]
        db[l] = dz.sum(0)
        if l > 0:
            dh = dz @ W[l]
            z = zs[l - 1]
            dz = dh * (silu_grad(z) if cache["act"] == "silu" else (z > 0).astype(np.float64))
    return dW, db


def adam(theta, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1); t counts from 1."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
