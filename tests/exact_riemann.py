"""Exact solution of the Riemann problem between two stiffened gases.

Test infrastructure, independent of both the oracle and the CUDA path: the
textbook exact solver for the Euler equations (pressure function, star state
and wave sampling), written with the stiffened-gas shift P = p + p_inf so that
each material obeys p + gamma p_inf = (gamma - 1) rho e. It serves as the
"exact" reference of the shock-tube tests of Sec. 5.4/5.5.
"""
from __future__ import annotations

import math

import numpy as np


class Side:
    def __init__(self, rho, u, p, gamma, pinf):
        self.rho, self.u, self.p, self.g, self.pinf = rho, u, p, gamma, pinf
        self.P = p + pinf
        self.c = math.sqrt(gamma * self.P / rho)

    def f_and_df(self, p):
        P = p + self.pinf
        g = self.g
        if P > self.P:  # shock
            A = 2.0 / ((g + 1.0) * self.rho)
            B = (g - 1.0) / (g + 1.0) * self.P
            s = math.sqrt(A / (P + B))
            return (P - self.P) * s, s * (1.0 - 0.5 * (P - self.P) / (P + B))
        # rarefaction
        r = P / self.P
        e = (g - 1.0) / (2.0 * g)
        f = 2.0 * self.c / (g - 1.0) * (r ** e - 1.0)
        df = 1.0 / (self.rho * self.c) * r ** (-(g + 1.0) / (2.0 * g))
        return f, df


def star_state(L: Side, R: Side, tol=1e-14):
    """Pressure and velocity in the star region (Newton on the pressure function)."""
    p_lo = max(-L.pinf, -R.pinf) + 1e-12 * max(L.P, R.P)
    p = max(0.5 * (L.p + R.p), p_lo + 1e-6 * max(L.P, R.P))
    for _ in range(200):
        fL, dL = L.f_and_df(p)
        fR, dR = R.f_and_df(p)
        F = fL + fR + (R.u - L.u)
        dp = F / (dL + dR)
        pn = p - dp
        if pn <= p_lo:
            pn = 0.5 * (p + p_lo)
        if abs(pn - p) <= tol * max(abs(pn), 1.0):
            p = pn
            break
        p = pn
    fL, _ = L.f_and_df(p)
    fR, _ = R.f_and_df(p)
    u = 0.5 * (L.u + R.u) + 0.5 * (fR - fL)
    return p, u


def sample(L: Side, R: Side, p_s, u_s, xi):
    """(rho, u, p, side) at similarity coordinate xi = x / t; side 0 = left material."""
    if xi <= u_s:
        K, sgn, side = L, 1.0, 0
    else:
        K, sgn, side = R, -1.0, 1
    g = K.g
    P_s = p_s + K.pinf
    # mirror the right side to the left-side formulas with sgn
    u_k = K.u
    if P_s > K.P:  # shock
        gr = (g - 1.0) / (g + 1.0)
        S = u_k - sgn * K.c * math.sqrt((g + 1.0) / (2.0 * g) * P_s / K.P + (g - 1.0) / (2.0 * g))
        behind = (xi >= S) if sgn > 0 else (xi <= S)
        if behind:
            rho = K.rho * (P_s / K.P + gr) / (gr * P_s / K.P + 1.0)
            return rho, u_s, p_s, side
        return K.rho, K.u, K.p, side
    # rarefaction
    c_s = K.c * (P_s / K.P) ** ((g - 1.0) / (2.0 * g))
    head = u_k - sgn * K.c
    tail = u_s - sgn * c_s
    if (sgn > 0 and xi <= head) or (sgn < 0 and xi >= head):
        return K.rho, K.u, K.p, side
    if (sgn > 0 and xi >= tail) or (sgn < 0 and xi <= tail):
        return K.rho * (P_s / K.P) ** (1.0 / g), u_s, p_s, side
    # inside the fan
    c = 2.0 / (g + 1.0) + sgn * (g - 1.0) / ((g + 1.0) * K.c) * (u_k - xi)
    rho = K.rho * c ** (2.0 / (g - 1.0))
    u = 2.0 / (g + 1.0) * (sgn * K.c + (g - 1.0) / 2.0 * u_k + xi)
    P = K.P * c ** (2.0 * g / (g - 1.0))
    return rho, u, P - K.pinf, side


def solve(L: Side, R: Side, x, x0, t):
    """rho, u, p arrays of the exact solution at positions x and time t."""
    p_s, u_s = star_state(L, R)
    out = np.array([sample(L, R, p_s, u_s, (xi - x0) / t) for xi in np.asarray(x)])
    return out[:, 0], out[:, 1], out[:, 2], out[:, 3]
