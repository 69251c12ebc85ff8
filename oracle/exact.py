"""Closed-form steady solutions of the paper's four flows (Sec. 3), in lattice
units (lengths in units of the tangent-vector step Delta x, time in steps).

TEST INFRASTRUCTURE ONLY (part of the oracle): these profiles are the
convergence targets the tests compare the oracle, and through it the CUDA
library, against.

Readings (where the printed formulas are garbled):
  * circular Poiseuille: a force along +theta drives the flow along +theta,
    u = (A/8)(r^2 - R1^2)(R2^2 - r^2)/r with A = alpha g / nu  (the printed
    r^3 coefficient has the opposite sign; the density is unaffected);
  * its lattice-unit b_lat carries the factor M^2 the print dropped;
  * the total mass is rho0 (R2^2 - R1^2)/2 per radian (the print repeats R2).
"""
import math

import numpy as np


def nu_of_tau(tau, T0):
    """Kinematic viscosity of the BGK lattice, nu = T0 (tau - 1/2)."""
    return T0 * (tau - 0.5)


def planar_couette(x, length, u_lo, u_hi):
    """Eqs. 21-22: linear profile between walls at x=0 (speed u_lo) and x=l."""
    x = np.asarray(x, dtype=np.float64)
    return u_lo + (u_hi - u_lo) * x / length


def planar_poiseuille(x, length, g, nu):
    """Eqs. 24-25: parabola of a channel driven by acceleration g along the walls."""
    x = np.asarray(x, dtype=np.float64)
    return g / (2.0 * nu) * x * (length - x)


def planar_poiseuille_mean(length, g, nu):
    """Mean of the parabola, g l^2 / (12 nu)."""
    return g * length ** 2 / (12.0 * nu)


class Annulus:
    """u_theta(r) = a r + b / r + (Ap / 8) r^3 between R1 and R2 (Eqs. 26, 39)
    and its leading-order density (Eqs. 31, 44-46)."""

    def __init__(self, R1, R2, a, b, Ap=0.0):
        self.R1, self.R2, self.a, self.b, self.Ap = float(R1), float(R2), a, b, Ap

    @classmethod
    def couette(cls, R1, R2, Omega1, Omega2=0.0):
        """Eq. 27."""
        d = R2 ** 2 - R1 ** 2
        a = (Omega2 * R2 ** 2 - Omega1 * R1 ** 2) / d
        b = R1 ** 2 * R2 ** 2 * (Omega1 - Omega2) / d
        return cls(R1, R2, a, b, 0.0)

    @classmethod
    def poiseuille(cls, R1, R2, A):
        """No-slip at both radii, azimuthal acceleration alpha g r with
        A = alpha g / nu; the flow follows the force."""
        return cls(R1, R2, A / 8.0 * (R1 ** 2 + R2 ** 2), -A / 8.0 * R1 ** 2 * R2 ** 2, -A)

    def u(self, r):
        r = np.asarray(r, dtype=np.float64)
        return self.a * r + self.b / r + self.Ap / 8.0 * r ** 3

    def mean_u(self):
        """Radial mean of u (Eq. 42)."""
        R1, R2, a, b, Ap = self.R1, self.R2, self.a, self.b, self.Ap
        return (a / 2.0 * (R2 + R1) + b * math.log(R2 / R1) / (R2 - R1)
                + Ap / 32.0 * (R2 + R1) * (R2 ** 2 + R1 ** 2))

    def h(self, r):
        """Integral of u^2 / r from R1 (Eqs. 45 / 31)."""
        r = np.asarray(r, dtype=np.float64)
        a, b, Ap, R1 = self.a, self.b, self.Ap, self.R1
        return (-b ** 2 / (2.0 * r ** 2) + 2.0 * a * b * np.log(r / R1)
                + 0.5 * (a ** 2 + b * Ap / 4.0) * r ** 2 + a * Ap * r ** 4 / 16.0
                + Ap ** 2 * r ** 6 / 384.0)

    def H(self):
        """Integral of r h(r) over [R1, R2] (Eqs. 30, 46)."""
        R1, R2, a, b, Ap = self.R1, self.R2, self.a, self.b, self.Ap
        L = math.log(R2 / R1)
        return (-b ** 2 / 2.0 * L + a * b * (R2 ** 2 * L - (R2 ** 2 - R1 ** 2) / 2.0)
                + (a ** 2 + b * Ap / 4.0) * (R2 ** 4 - R1 ** 4) / 8.0
                + a * Ap / 96.0 * (R2 ** 6 - R1 ** 6) + Ap ** 2 / 3072.0 * (R2 ** 8 - R1 ** 8))

    def rho(self, r, rho0, T0):
        """Leading-order density with the total mass of the uniform state."""
        return rho0 * (1.0 + (self.h(r) - 2.0 * self.H() / (self.R2 ** 2 - self.R1 ** 2)) / T0)


def circular_couette_lattice(Nr, M, omega1, omega2=0.0):
    """(a_lat, b_lat) of Eq. 33 with the inner radius M = R1/Delta_r."""
    den = Nr * (2.0 * M + Nr)
    a = (omega2 * (M + Nr) ** 2 - omega1 * M ** 2) / den
    b = M ** 2 * (Nr + M) ** 2 * (omega1 - omega2) / den
    return a, b
