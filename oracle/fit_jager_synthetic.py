"""Derive the SYNTHETIC Argon-like parameter set for the Jager potential form.

The paper (Sec. 3.4.1, Eq. jager_potential and Eq. damping) gives only the
functional form and says its coefficients come from Jager et al. (2009); no
number is printed.  This script builds a stand-in with textbook Ar-Ar
magnitudes so that every term of the form is exercised:

* dispersion C6, C8, C10 of Ar in atomic units (64.3, 1623, 49060 Eh a0^n),
  C12..C16 from the Tang-Toennies recursion C_{2n+6} = (C_{2n+4}/C_{2n+2})^3 C_{2n};
* fixed small a2, a_-1, a_-2 and damping beta;
* A and a1 solved so that the well minimum is at R_eps = 3.757 A with depth
  143.2 K;
* the screened-Coulomb core At exp(-at r)/r below 0.4 R_eps chosen so that
  V and V' are continuous at 0.4 R_eps.

Run ``python -m oracle.fit_jager_synthetic`` to print the set.  It calls only
the oracle.  The printed literals are the ones in the workloads module.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import fsolve

import oracle as O

EH_K = 315775.02480407  # Hartree in Kelvin
A0 = 0.529177210903     # Bohr radius in Angstrom
R_EPS = 3.757
DEPTH = 143.2


def dispersion():
    c6, c8, c10 = (64.3 * EH_K * A0 ** 6, 1623.0 * EH_K * A0 ** 8, 49060.0 * EH_K * A0 ** 10)
    cs = [c6, c8, c10]
    for _ in range(3):
        cs.append((cs[-1] / cs[-2]) ** 3 * cs[-3])
    return [float(f"{c:.6e}") for c in cs]


def build():
    base = dict(kind=0, a2=-0.012, am1=-0.35, am2=0.05, beta=3.84, C=dispersion(),
                R_eps=R_EPS, At=0.0, at=0.0)

    def resid(x):
        p = dict(base, A=float(np.exp(x[0])), a1=float(x[1]))
        P = O.make_pot(p)
        return [O.pot_dV(P, R_EPS) * 10.0, O.pot_V(P, R_EPS) + DEPTH]

    sol = fsolve(resid, [np.log(3.8e8), -3.9], xtol=1e-14)
    p = dict(base, A=float(f"{np.exp(sol[0]):.10e}"), a1=float(f"{sol[1]:.10f}"))
    P = O.make_pot(p)
    r0 = 0.4 * R_EPS
    V0, dV0 = O.pot_V(P, r0 + 1e-12), O.pot_dV(P, r0 + 1e-12)
    at = -dV0 / V0 - 1.0 / r0
    At = r0 * V0 * np.exp(at * r0)
    p["at"] = float(f"{at:.12e}")
    p["At"] = float(f"{At:.12e}")
    return p


if __name__ == "__main__":
    p = build()
    print("JAGER_SYNTHETIC_AR = dict(")
    for k, v in p.items():
        print(f"    {k}={v!r},")
    print(")")
    P = O.make_pot(p)
    rs = np.linspace(3.0, 4.5, 3001)
    V = np.array([O.pot_V(P, r) for r in rs])
    print("# minimum", rs[V.argmin()], V.min(), "zero crossing",
          rs[np.argmin(np.abs(V[:1000]))])
