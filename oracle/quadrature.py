"""Reference-element basis functions and quadrature rules of the oracle.

Reference prism: the triangle {xi >= 0, eta >= 0, xi + eta <= 1} times zeta in
[-1, 1] (the extruded P1 x P1 element with 6 nodes, Sec. 2.1 / Sec. 2.4).

* horizontal basis  phi_0 = 1 - xi - eta, phi_1 = xi, phi_2 = eta
* vertical basis    psi_0 = (1 + zeta)/2 (top node), psi_1 = (1 - zeta)/2 (bottom node)

Quadrature (all integrands of the scheme are polynomials of degree <= 2 in
(xi, eta) and <= 3 in zeta):

* triangle: the 3 edge-midpoint rule, exact for degree 2 (weights 1/3 of the area);
  the 6-point degree-4 rule (Strang and Fix; Dunavant 1985) for the vertical
  diffusion of the coupled column system, whose coefficient 1/z_zeta is not a
  polynomial
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


def _tri_rule4():
    """Symmetric 6-point rule exact for degree 4: the orbits (a, a, 1 - 2a) and
    (b, b, 1 - 2b) with the closed forms of the published rule,
        a, b = (8 - sqrt(10) +- sqrt(38 - 44 sqrt(2/5))) / 18,
        w_a, w_b = (620 +- sqrt(213125 - 53320 sqrt(10))) / 3720."""
    r = np.sqrt(38.0 - 44.0 * np.sqrt(0.4))
    a = (8.0 - np.sqrt(10.0) + r) / 18.0
    b = (8.0 - np.sqrt(10.0) - r) / 18.0
    q = np.sqrt(213125.0 - 53320.0 * np.sqrt(10.0))
    wa, wb = (620.0 + q) / 3720.0, (620.0 - q) / 3720.0
    return [(a, a, wa), (a, 1.0 - 2.0 * a, wa), (1.0 - 2.0 * a, a, wa),
            (b, b, wb), (b, 1.0 - 2.0 * b, wb), (1.0 - 2.0 * b, b, wb)]


# (xi, eta, weight), weights summing to 1, exact for degree 4
TRI_RULE4 = _tri_rule4()

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
