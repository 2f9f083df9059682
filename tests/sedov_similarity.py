"""Sedov-Taylor point blast in 3D: the self-similar solution, integrated
here from the Euler equations (test infrastructure; independent of the
oracle and of the GPU library).

With the shock radius R(t) = xi0 (E t^2 / rho1)^(1/5), its speed
D = dR/dt = 2R / (5t) and xi = r / R, write u = D U(xi), rho = rho1 G(xi),
p = rho1 D^2 P(xi).  Mass, momentum and entropy conservation in spherical
symmetry (dD/dt = -3 D^2 / (2R)) become, with w = U - xi,

    w G' + G U' = -2 G U / xi
    w U' + P' / G = 3 U / 2
    w (P'/P - gamma G'/G) = 3

with the strong-shock jump conditions at xi = 1: G = (gamma+1)/(gamma-1),
U = P = 2/(gamma+1).  The blast energy fixes xi0:
E = 4 pi rho1 R^3 D^2 I,  I = int_0^1 xi^2 (G U^2 / 2 + P / (gamma-1)) dxi,
so xi0 = (25 / (16 pi I))^(1/5).  The paper's Sedov test (§3.1) compares
with this solution (peak density (gamma+1)/(gamma-1) = 4 at gamma = 5/3).
"""
from __future__ import annotations

import math

import numpy as np


def _rhs(xi, y, gamma):
    G, U, P = y
    w = U - xi
    # eliminate G' and P' (first and third equations) from the second
    Up = (1.5 * U * G * w - 3.0 * P + 2.0 * gamma * P * U / xi) / (G * w * w - gamma * P)
    Gp = -G * (Up + 2.0 * U / xi) / w
    Pp = P * (3.0 / w + gamma * Gp / G)
    return np.array([Gp, Up, Pp])


def profile(gamma=5.0 / 3.0, xi_min=1e-4, n=20000):
    """(xi, G, U, P) from the shock (xi = 1) inwards to xi_min, by classical
    fourth-order Runge-Kutta on a grid uniform in ln xi."""
    s = np.linspace(0.0, math.log(xi_min), n + 1)   # s = ln xi
    y = np.array([(gamma + 1.0) / (gamma - 1.0), 2.0 / (gamma + 1.0), 2.0 / (gamma + 1.0)])
    out = np.empty((n + 1, 4))
    out[0] = (1.0, *y)

    def f(si, yi):
        xi = math.exp(si)
        return xi * _rhs(xi, yi, gamma)   # d/ds = xi d/dxi

    for k in range(n):
        hs = s[k + 1] - s[k]
        k1 = f(s[k], y)
        k2 = f(s[k] + 0.5 * hs, y + 0.5 * hs * k1)
        k3 = f(s[k] + 0.5 * hs, y + 0.5 * hs * k2)
        k4 = f(s[k + 1], y + hs * k3)
        y = y + hs / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
        out[k + 1] = (math.exp(s[k + 1]), *y)
    return out


def xi0(gamma=5.0 / 3.0, n=20000):
    """The dimensionless shock-radius constant of the 3D blast."""
    pr = profile(gamma, n=n)
    xi, G, U, P = pr.T
    f = xi ** 2 * (0.5 * G * U * U + P / (gamma - 1.0))
    # trapezoid in xi (the grid runs from 1 down to xi_min; the part below
    # xi_min adds O(xi_min^3))
    I = float(np.sum(0.5 * (f[1:] + f[:-1]) * (xi[:-1] - xi[1:])))
    return (25.0 / (16.0 * math.pi * I)) ** 0.2


def shock_radius(E, t, rho1=1.0, gamma=5.0 / 3.0):
    return xi0(gamma) * (E * t * t / rho1) ** 0.2
