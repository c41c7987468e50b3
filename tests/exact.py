"""Analytic references that pin the oracle.  None of this calls the oracle or the
CUDA library; each routine is written from the mathematics it names.

- ``maxwellian_moment``: moments of the Maxwellian of Eq. (5) (D = 2, I extra
  degrees of freedom) by tensor-product Gauss-Hermite quadrature, exact for the
  polynomial degrees of Eq. (6).
- ``RiemannExact``: the exact solution of the 1-D Euler Riemann problem for an
  ideal gas (two-shock/two-rarefaction pressure function solved by Newton's
  method, then self-similar sampling), as in standard gas-dynamics texts.
- ``rankine_hugoniot``: post-shock state of a normal shock of Mach number Ma.
- ``taylor_green_velocity``: the decaying Taylor-Green vortex, Eqs. (22)-(23).
"""
from __future__ import annotations

import math

import numpy as np


# --------------------------------------------------------------------- Eq. (5)

def _gh(n=10):
    x, w = np.polynomial.hermite_e.hermegauss(n)     # weight exp(-x^2 / 2)
    return x, w / math.sqrt(2.0 * math.pi)           # normalised: sum w = 1


def maxwellian_moment(phi, I, rho, ux, uy, T, central=False, n=10):
    """Integral of f_eq(v, eta) * phi(vx, vy, eta) over v and eta, Eq. (5) with
    D = 2, m = 1.  phi takes numpy arrays.  With central=True the argument is the
    peculiar velocity v - u.  I = 0 is the limit where eta is fixed at 0."""
    x, w = _gh(n)
    s = math.sqrt(T)
    cx = s * x[:, None, None]
    cy = s * x[None, :, None]
    if I > 0:
        eta = math.sqrt(I * T) * x[None, None, :]
        we = w[None, None, :]
    else:
        eta = np.zeros((1, 1, 1))
        we = np.ones((1, 1, 1))
    wt = w[:, None, None] * w[None, :, None] * we
    if central:
        vals = phi(cx + 0 * eta, cy + 0 * eta, eta + 0 * cx)
    else:
        vals = phi(ux + cx + 0 * eta, uy + cy + 0 * eta, eta + 0 * cx)
    return rho * float(np.sum(wt * vals))


def moment_rows():
    """The 16 functions Psi_k(c, eta) of Eq. (6), k = 1..16, as (label, callable)."""
    def w(cx, cy, e):
        return cx * cx + cy * cy + e * e
    return [
        ("1", lambda cx, cy, e: 1.0 + 0 * cx),
        ("x", lambda cx, cy, e: cx),
        ("y", lambda cx, cy, e: cy),
        ("w", lambda cx, cy, e: w(cx, cy, e)),
        ("xx", lambda cx, cy, e: cx * cx),
        ("xy", lambda cx, cy, e: cx * cy),
        ("yy", lambda cx, cy, e: cy * cy),
        ("wx", lambda cx, cy, e: w(cx, cy, e) * cx),
        ("wy", lambda cx, cy, e: w(cx, cy, e) * cy),
        ("xxx", lambda cx, cy, e: cx ** 3),
        ("xxy", lambda cx, cy, e: cx * cx * cy),
        ("xyy", lambda cx, cy, e: cx * cy * cy),
        ("yyy", lambda cx, cy, e: cy ** 3),
        ("wxx", lambda cx, cy, e: w(cx, cy, e) * cx * cx),
        ("wxy", lambda cx, cy, e: w(cx, cy, e) * cx * cy),
        ("wyy", lambda cx, cy, e: w(cx, cy, e) * cy * cy),
    ]


# ------------------------------------------------------------ exact Riemann

class RiemannExact:
    """Exact solution of the Riemann problem for the 1-D Euler equations of an
    ideal gas with ratio gamma.  States are (rho, u, p)."""

    def __init__(self, left, right, gamma):
        self.g = gamma
        self.L = tuple(map(float, left))
        self.R = tuple(map(float, right))
        self.cL = math.sqrt(gamma * self.L[2] / self.L[0])
        self.cR = math.sqrt(gamma * self.R[2] / self.R[0])
        self.p_star, self.u_star = self._solve()

    def _fk(self, p, state, c):
        """Velocity jump across the left or right wave for star pressure p."""
        rho, _, pk = state
        g = self.g
        if p > pk:   # shock
            A = 2.0 / ((g + 1.0) * rho)
            B = (g - 1.0) / (g + 1.0) * pk
            return (p - pk) * math.sqrt(A / (p + B))
        return 2.0 * c / (g - 1.0) * ((p / pk) ** ((g - 1.0) / (2.0 * g)) - 1.0)   # rarefaction

    def _solve(self):
        du = self.R[1] - self.L[1]
        p = max(1e-10, 0.5 * (self.L[2] + self.R[2]))
        for _ in range(200):
            F = self._fk(p, self.L, self.cL) + self._fk(p, self.R, self.cR) + du
            dF = self._dfk(p, self.L, self.cL) + self._dfk(p, self.R, self.cR)
            pn = max(1e-12, p - F / dF)
            if abs(pn - p) <= 1e-15 * (pn + p):
                p = pn
                break
            p = pn
        fL = self._fk(p, self.L, self.cL)
        fR = self._fk(p, self.R, self.cR)
        u = 0.5 * (self.L[1] + self.R[1]) + 0.5 * (fR - fL)
        return p, u

    def _dfk(self, p, state, c):
        rho, _, pk = state
        g = self.g
        if p > pk:
            A = 2.0 / ((g + 1.0) * rho)
            B = (g - 1.0) / (g + 1.0) * pk
            q = math.sqrt(A / (p + B))
            return q * (1.0 - 0.5 * (p - pk) / (B + p))
        return (p / pk) ** (-(g + 1.0) / (2.0 * g)) / (rho * c)

    def sample(self, xi):
        """(rho, u, p) at similarity coordinate xi = (x - x0) / t (array)."""
        xi = np.asarray(xi, dtype=float)
        out = np.zeros((3,) + xi.shape)
        for idx, s in np.ndenumerate(xi):
            out[(slice(None),) + idx] = self._sample1(float(s))
        return out

    def _sample1(self, s):
        g = self.g
        ps, us = self.p_star, self.u_star
        if s <= us:
            rho, u, p = self.L
            c = self.cL
            if ps > p:   # left shock
                SL = u - c * math.sqrt((g + 1) / (2 * g) * ps / p + (g - 1) / (2 * g))
                if s <= SL:
                    return rho, u, p
                r = rho * (ps / p + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / p + 1)
                return r, us, ps
            cs = c * (ps / p) ** ((g - 1) / (2 * g))
            if s <= u - c:
                return rho, u, p
            if s >= us - cs:
                return rho * (ps / p) ** (1 / g), us, ps
            fac = 2 / (g + 1) + (g - 1) / ((g + 1) * c) * (u - s)
            return (rho * fac ** (2 / (g - 1)), 2 / (g + 1) * (c + (g - 1) / 2 * u + s),
                    p * fac ** (2 * g / (g - 1)))
        rho, u, p = self.R
        c = self.cR
        if ps > p:       # right shock
            SR = u + c * math.sqrt((g + 1) / (2 * g) * ps / p + (g - 1) / (2 * g))
            if s >= SR:
                return rho, u, p
            r = rho * (ps / p + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / p + 1)
            return r, us, ps
        cs = c * (ps / p) ** ((g - 1) / (2 * g))
        if s >= u + c:
            return rho, u, p
        if s <= us + cs:
            return rho * (ps / p) ** (1 / g), us, ps
        fac = 2 / (g + 1) - (g - 1) / ((g + 1) * c) * (u - s)
        return (rho * fac ** (2 / (g - 1)), 2 / (g + 1) * (-c + (g - 1) / 2 * u + s),
                p * fac ** (2 * g / (g - 1)))


def rankine_hugoniot(Ma, gamma, rho1=1.0, p1=1.0):
    """Post-shock (rho, u, p) behind a normal shock of Mach Ma running into gas at
    rest (rho1, p1); also the shock speed."""
    g = gamma
    c1 = math.sqrt(g * p1 / rho1)
    M2 = Ma * Ma
    rho2 = rho1 * (g + 1) * M2 / ((g - 1) * M2 + 2)
    p2 = p1 * (1 + 2 * g / (g + 1) * (M2 - 1))
    s = Ma * c1
    u2 = s * (1 - rho1 / rho2)
    return rho2, u2, p2, s


# --------------------------------------------------------------- Taylor-Green

def taylor_green_velocity(X, Y, t, U0, k, nu):
    """Eqs. (22)-(23) in the orientation u = U0 sin(kx) cos(ky) e^{-2 nu k^2 t},
    v = -U0 cos(kx) sin(ky) e^{-2 nu k^2 t}."""
    d = math.exp(-2.0 * nu * k * k * t)
    return U0 * np.sin(k * X) * np.cos(k * Y) * d, -U0 * np.cos(k * X) * np.sin(k * Y) * d
