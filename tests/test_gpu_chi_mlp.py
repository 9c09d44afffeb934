"""chi-MLP surrogate (Fig. nn_architecture, reading R9) through the C ABI
(dsmc_chi_mlp_pack / _forward / _table) against the FP64 oracle
(oracle/dsmc_oracle.c: or_chi_mlp_forward, pinned against torch in
test_oracle_pins.py).

Gates, relative to the largest |y|: 1e-3 against the oracle's emulation of
the kernel's storage (input as two bf16 terms, hidden activations 1-4 as
single bf16 terms; what remains is FP32 accumulation and the SiLU
evaluation, plus the rare activation that rounds to the other neighbouring
bf16 value); 2e-2 against plain FP64 (single bf16 storage of the
activations, 2^-9 relative each, as the bf16 gate of the collision MLP).
Measured: 6e-5 and 1.5e-4.
"""
import numpy as np
import pytest

import oracle as O
from paper_2602_21244_gb300 import workloads as W

from gpu_util import ctx, cuda, host, torch

pytestmark = pytest.mark.gpu

_NET = {}


def _net():
    if "p" not in _NET:
        wts = W.chi_mlp_weights()
        C = ctx()
        wb = cuda(wts["W_bits"].view(np.int16))
        bias = cuda(wts["bias"], torch().float32)
        _NET["p"] = (wts, C.chi_mlp_pack(wb), bias)
    return _NET["p"]


@pytest.mark.parametrize("n", [1, 127, 128, 1000, 4099])
def test_chi_mlp_forward_parity(n):
    wts, packed, bias = _net()
    C = ctx()
    x = np.random.default_rng(n).uniform(0, 1, (n, 2)).astype(np.float32)
    y, chi = C.chi_mlp_forward(packed, bias, cuda(x))
    assert C.sync_status() == 0
    y, chi = host(y), host(chi)
    ye = O.chi_mlp_forward(wts["W"], wts["bias"], x.astype(np.float64), bf16=True)
    y64 = O.chi_mlp_forward(wts["W"], wts["bias"], x.astype(np.float64))
    sc = np.abs(y64).max()
    assert np.abs(y - ye).max() <= 1e-3 * sc
    assert np.abs(y - y64).max() <= 2e-2 * sc
    np.testing.assert_allclose(chi, np.expm1(y.astype(np.float64)), rtol=1e-6, atol=1e-7)
    assert np.all(y >= 0)


def test_chi_mlp_table_matches_oracle_and_is_deterministic():
    wts, packed, bias = _net()
    C = ctx()
    T1 = C.chi_mlp_table(packed, bias, 33, 17)
    T2 = C.chi_mlp_table(packed, bias, 33, 17)
    torch().cuda.synchronize()
    assert C.sync_status() == 0
    assert torch().equal(T1, T2)
    Te = O.chi_mlp_table(wts["W"], wts["bias"], 33, 17, bf16=True)
    T = host(T1)
    assert T.shape == (17, 33)
    assert np.abs(T - Te).max() <= 1e-3 * np.abs(Te).max()
    # the full-size table of Sec. 3.4.4 against forward at sampled nodes
    big = host(C.chi_mlp_table(packed, bias, 512, 512))
    rng = np.random.default_rng(9)
    j, i = rng.integers(0, 512, 64), rng.integers(0, 512, 64)
    x = np.stack([j / 511.0, i / 511.0], 1).astype(np.float32)
    _, chi = C.chi_mlp_forward(packed, bias, cuda(x))
    assert C.sync_status() == 0
    np.testing.assert_allclose(big[j, i], host(chi), rtol=0, atol=0)


def test_chi_mlp_rejects_bad_arguments():
    from paper_2602_21244_gb300 import dsmc as D
    wts, packed, bias = _net()
    C = ctx()
    with pytest.raises(D.DsmcError) as e:
        C.chi_mlp_table(packed, bias, 1, 17)
    assert e.value.code == D.DSMC_ERR_ARG
