"""Independent mathematics used by the tests to pin the oracle and the tables.

Nothing here is shared with the oracle or the CUDA path: these are textbook
formulas restated for the tests.

* Adams-Neumann product formula for Legendre polynomials (J. C. Adams, Proc.
  R. Soc. 27 (1878)), the Legendre instance of the product-to-sum identity of
  Eq. (3) of arXiv:1703.09619:
      P_m P_n = sum_{r=0}^{min(m,n)} A_{m-r} A_r A_{n-r} / A_{m+n-r}
                * (2m+2n-4r+1)/(2m+2n-2r+1) * P_{m+n-2r},
      A_r = (2r-1)!! / r!.
* Derivative expansion P'_m = sum_{j = m-1, m-3, ... >= 0} (2j+1) P_j.
* Closed forms of the one-dimensional integrals with a unit coupling factor.
"""
from __future__ import annotations

from fractions import Fraction
from functools import lru_cache

import numpy as np
from numpy.polynomial import legendre as L


@lru_cache(maxsize=None)
def _A(r: int) -> Fraction:
    num = 1
    for i in range(1, 2 * r, 2):
        num *= i
    den = 1
    for i in range(1, r + 1):
        den *= i
    return Fraction(num, den)


@lru_cache(maxsize=None)
def adams_neumann(m: int, n: int) -> dict:
    """Exact rational coefficients {k: c_k} with P_m P_n = sum c_k P_k."""
    out = {}
    for r in range(min(m, n) + 1):
        k = m + n - 2 * r
        c = _A(m - r) * _A(r) * _A(n - r) / _A(m + n - r) * Fraction(2 * m + 2 * n - 4 * r + 1,
                                                                      2 * m + 2 * n - 2 * r + 1)
        out[k] = out.get(k, Fraction(0)) + c
    return out


def derivative_expansion(m: int) -> dict:
    """{j: 2j+1} with P'_m = sum_j (2j+1) P_j."""
    return {j: Fraction(2 * j + 1) for j in range(m - 1, -1, -2)}


@lru_cache(maxsize=None)
def product_coeffs(d1: int, d2: int, m1: int, m2: int) -> dict:
    """Exact {k: c_k} with P^{(d1)}_{m1} P^{(d2)}_{m2} = sum_k c_k P_k (d in {0,1})."""
    left = derivative_expansion(m1) if d1 else {m1: Fraction(1)}
    right = derivative_expansion(m2) if d2 else {m2: Fraction(1)}
    out = {}
    for i, ci in left.items():
        for j, cj in right.items():
            for k, ck in adams_neumann(i, j).items():
                out[k] = out.get(k, Fraction(0)) + ci * cj * ck
    return {k: v for k, v in out.items() if v != 0}


def product_dense(d1, d2, m1, m2, K):
    c = np.zeros(K)
    for k, v in product_coeffs(d1, d2, m1, m2).items():
        c[k] = float(v)
    return c


TYPE_D = {"vv": (0, 0), "dv": (1, 0), "vd": (0, 1), "dd": (1, 1)}


def closed_form_1d(t: str, m1: int, m2: int) -> float:
    """int_{-1}^{1} P^{(d1)}_{m1} P^{(d2)}_{m2} dx for a unit coupling factor."""
    if t == "vv":
        return 2.0 / (2 * m1 + 1) if m1 == m2 else 0.0
    if t == "dv":
        return 2.0 if (m2 < m1 and (m1 + m2) % 2 == 1) else 0.0
    if t == "vd":
        return 2.0 if (m1 < m2 and (m1 + m2) % 2 == 1) else 0.0
    mn = min(m1, m2)
    return float(mn * (mn + 1)) if (m1 + m2) % 2 == 0 else 0.0


def legendre_power_coeffs(m: int, deriv: int) -> np.ndarray:
    """Power-series coefficients (ascending) of P_m or P'_m."""
    c = np.zeros(m + 1)
    c[m] = 1.0
    if deriv:
        c = L.legder(c)
    return L.leg2poly(c)


def monomial_integral(j: int) -> float:
    """int_{-1}^{1} x^j dx."""
    return 2.0 / (j + 1) if j % 2 == 0 else 0.0


def dof_list(orders_e):
    """[(g, m, n, p)] in the output's dof order: component-major, then (m Nv + n) Nw + p."""
    out = []
    for g, (Nu, Nv, Nw) in enumerate(orders_e):
        for m in range(Nu):
            for n in range(Nv):
                for p in range(Nw):
                    out.append((g, m, n, p))
    return out
