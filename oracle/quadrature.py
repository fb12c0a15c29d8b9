"""Reference-element basis functions and quadrature rules of the oracle.

Reference prism: the triangle {xi >= 0, eta >= 0, xi + eta <= 1} times zeta in
[-1, 1] (the extruded P1 x P1 element with 6 nodes, Sec. 2.1 / Sec. 2.4).

* horizontal basis  phi_0 = 1 - xi - eta, phi_1 = xi, phi_2 = eta
* vertical basis    psi_0 = (1 + zeta)/2 (top node), psi_1 = (1 - zeta)/2 (bottom node)

Quadrature (all integrands of the scheme are polynomials of degree <= 2 in
(xi, eta) and <= 3 in zeta):

* triangle: the 3 edge-midpoint rule, exact for degree 2 (weights 1/3 of the area)
* interval: 2-point Gauss-Legendre, exact for degree 3
* lateral quadrilateral faces: 2-point Gauss along the edge x 2-point Gauss in zeta.
  Upwind fluxes are evaluated at these 4 points; this rule is part of the scheme's
  definition (a reading: the paper does not state its face quadrature).
"""
from __future__ import annotations

import numpy as np

GAUSS_Z, GAUSS_W = np.polynomial.legendre.leggauss(2)

# (xi, eta, weight) with weights summing to 1; integral over the reference triangle
# of f is 0.5 * sum_g w_g f(g)
TRI_RULE = [(0.5, 0.0, 1.0 / 3.0), (0.5, 0.5, 1.0 / 3.0), (0.0, 0.5, 1.0 / 3.0)]

# reference gradients of phi_a: d/dxi, d/deta
GRAD_REF = np.array([[-1.0, -1.0], [1.0, 0.0], [0.0, 1.0]])


def phi(xi: float, eta: float) -> np.ndarray:
    return np.array([1.0 - xi - eta, xi, eta])


def psi(z: float) -> np.ndarray:
    return np.array([(1.0 + z) * 0.5, (1.0 - z) * 0.5])


def dpsi() -> np.ndarray:
    """d psi_c / d zeta (constant)."""
    return np.array([0.5, -0.5])


def int_psi_psi() -> np.ndarray:
    """G_cd = integral over [-1,1] of psi_c psi_d, by Gauss quadrature."""
    G = np.zeros((2, 2))
    for z, w in zip(GAUSS_Z, GAUSS_W):
        G += w * np.outer(psi(z), psi(z))
    return G
