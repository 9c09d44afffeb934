"""Training of the neural collision operator on the GPU (through the C ABI)
against the FP64 oracle of oracle/train.py (itself pinned by central finite
differences and by torch autograd in test_oracle_pins.py).

Gates: loss within 1e-3 relative; per-tensor gradient ||g_gpu - g_ref|| /
||g_ref|| <= 2e-2 (bf16 tensor-core GEMMs with FP32 accumulation);
forward velocities within 2e-2 sigma_v; the backward from an external
dL/dv equals the fused loss path bit for bit; Adam in FP32 within 1e-5.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import train as OT
from paper_2602_21244_gb300 import workloads as W

from gpu_util import ctx, cuda, host, torch

pytestmark = pytest.mark.gpu
SEED, T_STEP = 11, 3


def _setup(n, seed=0):
    wts = W.mlp_weights()
    dims = wts["dims"]
    rng = np.random.default_rng(seed)
    Wl = [w + rng.standard_normal(w.shape) * 0.05 for w in OT.split_layers(dims, wts["W"])]
    Wflat = W.bf16_value(W.bf16_bits(np.concatenate([w.ravel() for w in Wl])))
    bflat = (rng.standard_normal(len(wts["bias"])) * 0.05).astype(np.float32).astype(np.float64)
    theta = np.concatenate([Wflat, bflat]).astype(np.float32)
    hv = W.harvest_inputs(n, seed=seed)
    gas = O.make_gas(W.M_AR, 4.17e-10, 0.81, 273.0, 1.0, 1.0, 3)
    vit, vjt = O.harvest_jager(gas, O.make_pot(W.JAGER_SYNTHETIC_AR), hv["vi"], hv["vj"], hv["b"], hv["eps"])
    return dims, theta, hv, vit, vjt


def _mlp():
    from paper_2602_21244_gb300 import dsmc as D
    return D.make_mlp(8, 128, 3, 3, 0, W.sigma_v(), 273.0, 1e-12)


def _oracle(dims, theta, hv, vit, vjt):
    nW = sum(dims[l] * dims[l + 1] for l in range(4))
    Ws = OT.split_layers(dims, theta[:nW].astype(np.float64))
    bs = OT.split_bias(dims, theta[nW:].astype(np.float64))
    xi = OT.train_noise(SEED, T_STEP, len(hv["T"]))
    loss, cache = OT.forward(dims, Ws, bs, hv["vi"], hv["vj"], hv["T"], xi, vit, vjt, W.sigma_v(), 273.0)
    dW, db = OT.backward(dims, Ws, bs, cache, W.sigma_v())
    return loss, dW, db, cache


def _split(dims, g):
    out, o = [], 0
    for l in range(4):
        out.append(g[o:o + dims[l] * dims[l + 1]]); o += dims[l] * dims[l + 1]
    for l in range(4):
        out.append(g[o:o + dims[l + 1]]); o += dims[l + 1]
    return out


def _gpu_inputs(hv, vit, vjt):
    return (cuda(hv["vi"]), cuda(hv["vj"]), cuda(hv["T"]), cuda(vit), cuda(vjt))


@pytest.mark.parametrize("n", [128, 1040])
def test_loss_and_gradient_match_oracle(n):
    dims, theta, hv, vit, vjt = _setup(n)
    loss, dW, db, _ = _oracle(dims, theta, hv, vit, vjt)
    C = ctx()
    g, l = C.train_loss_grad(_mlp(), cuda(theta), SEED, T_STEP, *_gpu_inputs(hv, vit, vjt))
    assert C.sync_status() == 0
    assert abs(float(l.item()) / loss - 1) < 1e-3
    parts = _split(dims, host(g).astype(np.float64))
    refs = [d.ravel() for d in dW] + [d.ravel() for d in db]
    for q, (a, b) in enumerate(zip(parts, refs)):
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert rel <= 2e-2, (q, rel)


def test_operator_forward_matches_oracle_and_conserves():
    n = 1040
    dims, theta, hv, vit, vjt = _setup(n, seed=2)
    _, _, _, cache = _oracle(dims, theta, hv, vit, vjt)
    Vn = cache["Vn"]  # [groups, 32, 3]: 16 first particles then 16 second
    ref_i = Vn[:, :16].reshape(n, 3)
    ref_j = Vn[:, 16:].reshape(n, 3)
    C = ctx()
    vi, vj, T, _, _ = _gpu_inputs(hv, vit, vjt)
    oi, oj = C.neural_operator_forward(_mlp(), cuda(theta), SEED, T_STEP, vi, vj, T)
    assert C.sync_status() == 0
    oi, oj = host(oi), host(oj)
    sv = W.sigma_v()
    assert np.abs(oi - ref_i).max() / sv <= 2e-2 and np.abs(oj - ref_j).max() / sv <= 2e-2
    # each pseudo-cell keeps its momentum and energy
    P0 = (hv["vi"] + hv["vj"]).reshape(-1, 16, 3).sum(1)
    P1 = (oi + oj).reshape(-1, 16, 3).sum(1)
    E0 = (hv["vi"] ** 2 + hv["vj"] ** 2).reshape(-1, 16 * 3).sum(1)
    E1 = (oi ** 2 + oj ** 2).reshape(-1, 16 * 3).sum(1)
    assert np.abs(P1 - P0).max() <= 1e-12 * np.abs(hv["vi"]).max() * 32
    assert np.abs(E1 / E0 - 1).max() <= 1e-12


def test_backward_from_external_gradient_equals_fused_loss_path():
    n = 512
    dims, theta, hv, vit, vjt = _setup(n, seed=3)
    C = ctx()
    vi, vj, T, ti, tj = _gpu_inputs(hv, vit, vjt)
    th = cuda(theta)
    g_fused, _ = C.train_loss_grad(_mlp(), th, SEED, T_STEP, vi, vj, T, ti, tj)
    oi, oj = C.neural_operator_forward(_mlp(), th, SEED, T_STEP, vi, vj, T)
    sc = (1.0 / W.sigma_v()) * (1.0 / W.sigma_v()) / n
    gi, gj = (oi - ti) * sc, (oj - tj) * sc
    g_ext = C.neural_operator_backward(_mlp(), th, SEED, T_STEP, vi, vj, T, gi, gj)
    assert C.sync_status() == 0
    assert torch().equal(g_fused, g_ext)


def test_autograd_function_matches_plain_pytorch_fp64():
    T_ = torch()
    from paper_2602_21244_gb300 import dsmc as D
    n = 256
    dims, theta, hv, vit, vjt = _setup(n, seed=4)
    C = ctx()
    vi, vj, T, ti, tj = _gpu_inputs(hv, vit, vjt)
    th = cuda(theta).requires_grad_(True)
    oi, oj = D.NeuralCollisionOperator.apply(th, vi, vj, T, C, _mlp(), SEED, T_STEP)
    loss = (((oi - ti) ** 2).sum() + ((oj - tj) ** 2).sum()) / (W.sigma_v() ** 2 * 2 * n)
    loss.backward()
    g_gpu = th.grad.detach().cpu().double().numpy()
    # plain-PyTorch FP64 reference of the same operator and loss
    nW = sum(dims[l] * dims[l + 1] for l in range(4))
    tt = T_.tensor(theta.astype(np.float64), requires_grad=True)
    Ws, bs, o = [], [], 0
    for l in range(4):
        Ws.append(tt[o:o + dims[l] * dims[l + 1]].reshape(dims[l + 1], dims[l])); o += dims[l] * dims[l + 1]
    for l in range(4):
        bs.append(tt[o:o + dims[l + 1]]); o += dims[l + 1]
    Vi, Vj = T_.tensor(hv["vi"]), T_.tensor(hv["vj"])
    vr = Vi - Vj
    xi = T_.tensor(OT.train_noise(SEED, T_STEP, n))
    x = T_.cat([vr / W.sigma_v(), T_.tensor(hv["T"] / 273.0)[:, None], xi], 1)
    h = x
    for l in range(4):
        h = T_.nn.functional.linear(h, Ws[l], bs[l])
        if l < 3:
            h = T_.nn.functional.silu(h)
    vrp = vr.norm(dim=1, keepdim=True) * h / h.norm(dim=1, keepdim=True)
    cm = 0.5 * (Vi + Vj)
    P = T_.cat([(cm + 0.5 * vrp).reshape(-1, 16, 3), (cm - 0.5 * vrp).reshape(-1, 16, 3)], 1)
    Q = T_.cat([Vi.reshape(-1, 16, 3), Vj.reshape(-1, 16, 3)], 1)
    up, uq = P.mean(1, keepdim=True), Q.mean(1, keepdim=True)
    alpha = T_.sqrt(((Q - uq) ** 2).sum((1, 2)) / ((P - up) ** 2).sum((1, 2)))
    Vn = uq + alpha[:, None, None] * (P - up)
    Tt = T_.cat([T_.tensor(vit).reshape(-1, 16, 3), T_.tensor(vjt).reshape(-1, 16, 3)], 1)
    L = (((Vn - Tt) / W.sigma_v()) ** 2).sum() / (2 * n)
    L.backward()
    g_ref = tt.grad.numpy()
    assert abs(float(loss) / float(L) - 1) < 1e-3
    for a, b in zip(_split(dims, g_gpu), _split(dims, g_ref)):
        assert np.linalg.norm(a - b) / np.linalg.norm(b) <= 2e-2


def test_adam_step_matches_oracle_and_training_reduces_loss():
    n = 1024
    dims, theta, hv, vit, vjt = _setup(n, seed=5)
    C = ctx()
    mlp = _mlp()
    vi, vj, T, ti, tj = _gpu_inputs(hv, vit, vjt)
    th = cuda(theta)
    m = torch().zeros_like(th)
    v = torch().zeros_like(th)
    nW = sum(dims[l] * dims[l + 1] for l in range(4))
    g, _ = C.train_loss_grad(mlp, th, SEED, 1, vi, vj, T, ti, tj)
    gh = host(g).astype(np.float64)
    C.adam_step(nW, g, th, m, v, 1, lr=1e-3)
    ref, _, _ = OT.adam(theta.astype(np.float64), gh, np.zeros_like(gh), np.zeros_like(gh), 1)
    assert np.abs(host(th) - ref).max() <= 1e-5 * np.abs(ref).max() + 1e-7
    # a few full steps on the same batch lower the loss
    ws = C.train_workspace()
    grad = torch().empty_like(th)
    loss = torch().zeros(1, dtype=torch().float64, device="cuda")
    losses = []
    for step in range(2, 30):
        C.train_step(mlp, th, m, v, step, 3e-3, SEED, vi, vj, T, ti, tj, grad, loss, ws)
        losses.append(float(loss.item()))
    assert C.sync_status() == 0
    assert losses[-1] < 0.9 * losses[0], losses[::7]


@pytest.mark.parametrize("n", [1040, 1 << 16])
def test_recomputation_equals_stored_activations(n):
    """The backward recomputes every hidden layer's pre-activation from the
    forward's own MMA operands; the stored-activation variant writes them in
    the forward and reads them back.  Both must give the same loss and the
    same gradient bit for bit (several tiles per CTA at 2^16 pairs)."""
    dims, theta, hv, vit, vjt = _setup(n, seed=4)
    C = ctx()
    args = (_mlp(), cuda(theta), SEED, T_STEP, *_gpu_inputs(hv, vit, vjt))
    g1, l1 = C.train_loss_grad(*args)
    g2, l2 = C.train_loss_grad_stored(*args)
    assert C.sync_status() == 0
    assert torch().equal(g1, g2)
    assert float(l1.item()) == float(l2.item())
