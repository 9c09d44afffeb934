"""Transport integrals (Eq. chapman_enskog and the two integrals after it,
reading R8) through the C ABI: dsmc_transport_q2 and dsmc_transport_viscosity
against closed forms (rigid spheres, inverse-power scaling) and against the
FP64 oracle (oracle/dsmc_oracle.c: or_transport_q2, or_transport_viscosity,
pinned in test_oracle_pins.py) with the same quadrature rule.

Gates: chi at each node carries the FP32 error of the chi kernel (1e-5 |chi|
+ 1e-6 (1 + depth/E) rad, the last term below the well depth); sin^2 chi moves
by at most |sin 2 chi| times that, so Q2 (a positive average of sin^2 chi) is
gated at 2e-5 relative for energies down to 20 K (depth/E = 7), the
Maxwellian averages Omega22 and mu at 1e-5; rigid spheres (chi = 2 arccos(b/d)
in FP32) at 1e-6.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2602_21244_gb300 import workloads as W

from gpu_util import KB, ctx, cuda, host, torch

pytestmark = pytest.mark.gpu

JP = W.JAGER_SYNTHETIC_AR


def _gas(D):
    return D.make_gas(dict(mass=W.M_AR, fn_over_vc=1.0, dt=1.0))


def test_transport_hard_sphere_closed_forms():
    from paper_2602_21244_gb300 import dsmc as D
    C = ctx()
    hs = D.make_potential(W.HARD_SPHERE_AR)
    d = 3.6e-10
    q = host(C.transport_q2(hs, cuda(np.array([10.0, 1e3, 1e5])), 3.6, b_panels=4))
    assert C.sync_status() == 0
    assert np.allclose(q, 2 / 3 * math.pi * d * d, rtol=1e-6, atol=0)
    T = np.array([300.0, 3000.0, 2e4])
    om, mu = C.transport_viscosity(_gas(D), hs, cuda(T), 3.6, b_panels=4, x_panels=8)
    assert C.sync_status() == 0
    assert np.allclose(host(om), math.pi * d * d, rtol=1e-6, atol=0)
    want = 5 / 16 * np.sqrt(math.pi * W.M_AR * KB * T) / (math.pi * d * d)
    assert np.allclose(host(mu), want, rtol=1e-6, atol=0)


def test_transport_inverse_power_matches_oracle_and_scaling():
    from paper_2602_21244_gb300 import dsmc as D
    C = ctx()
    p = 12.0
    spec = dict(kind=2, kappa=1.3e9, p=p)
    E = np.array([300.0, 3000.0])
    q = host(C.transport_q2(D.make_potential(spec), cuda(E), 12.0, b_panels=8))
    qo = O.transport_q2(O.make_pot(spec), E, 12.0, b_panels=8)
    assert np.allclose(q, qo, rtol=2e-5, atol=0)
    assert abs(q[1] / q[0] / 10.0 ** (-2 / p) - 1) < 2e-5
    om, mu = C.transport_viscosity(_gas(D), D.make_potential(spec), cuda(np.array([1000.0])), 12.0, b_panels=8,
                                   x_panels=8)
    omo, muo = O.transport_viscosity(O.make_pot(spec), W.M_AR, [1000.0], 12.0, b_panels=8, x_panels=8)
    assert C.sync_status() == 0
    assert abs(host(om)[0] / omo[0] - 1) < 1e-5 and abs(host(mu)[0] / muo[0] - 1) < 1e-5


def test_transport_jager_matches_oracle():
    from paper_2602_21244_gb300 import dsmc as D
    C = ctx()
    P, PO = D.make_potential(JP), O.make_pot(JP)
    E = np.array([20.0, 60.0, 150.0, 300.0, 1000.0, 5000.0, 3e4])
    q = host(C.transport_q2(P, cuda(E), 12.0, b_panels=8))
    qo = O.transport_q2(PO, E, 12.0, b_panels=8)
    assert C.sync_status() == 0
    assert np.all(np.abs(q / qo - 1) < 2e-5), q / qo - 1
    T = np.array([1500.0, 6000.0])
    om, mu = C.transport_viscosity(_gas(D), P, cuda(T), 12.0, b_panels=8, x_panels=4)
    omo, muo = O.transport_viscosity(PO, W.M_AR, T, 12.0, b_panels=8, x_panels=4)
    assert C.sync_status() == 0
    assert np.all(np.abs(host(om) / omo - 1) < 1e-5) and np.all(np.abs(host(mu) / muo - 1) < 1e-5)


def test_transport_is_deterministic_and_reports_bad_energies():
    from paper_2602_21244_gb300 import dsmc as D
    C = ctx()
    P = D.make_potential(JP)
    T = cuda(np.geomspace(500.0, 2e4, 16))
    a = C.transport_viscosity(_gas(D), P, T)
    b = C.transport_viscosity(_gas(D), P, T)
    torch().cuda.synchronize()
    assert C.sync_status() == 0
    assert torch().equal(a[0], b[0]) and torch().equal(a[1], b[1])
    # mu rises with T for this gas over the paper's range (1500 K to 6000 K)
    m = host(a[1])
    assert np.all(np.diff(m) > 0)
    C.transport_q2(P, cuda(np.array([300.0, -1.0])), 12.0)
    assert C.sync_status() == D.DSMC_ERR_ARG
    assert C.sync_status() == 0
