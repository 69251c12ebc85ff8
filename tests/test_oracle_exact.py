"""Pins of the closed-form solutions (Sec. 3) and of the unit conventions
behind them, by recomputing the parameter tables the paper prints."""
import math

import numpy as np
import pytest
from scipy import integrate

import clbm_inputs as I
from conftest import golden
from oracle import exact as E

T0 = {9: 1.0 / 3.0, 21: 2.0 / 3.0}


def _rows(section):
    out, cur = [], None
    for line in open(golden("parameter_tables.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("["):
            cur = line
            continue
        if cur.startswith("[" + section):
            out.append(line.split())
    assert out
    return out


def _close(x, printed, rel=0.02, ab=0.0):
    return abs(x - printed) <= rel * abs(printed) + ab


def _close_printed(x, text, rel=0.015):
    """x agrees with a value printed as ``text``, to half a unit of its last
    digit plus the rounding carried by the 3-digit inputs."""
    d = len(text.split(".")[1]) if "." in text else 0
    return abs(x - float(text)) <= 0.5 * 10 ** (-d) + rel * abs(x)


def test_planar_couette_table():
    for Q, tau, N, U, nu, _, Ma, Re, _ in _rows("planar Couette"):
        Q, tau, N, U, nu, Ma, Re = int(Q), float(tau), int(N), float(U), float(nu), float(Ma), float(Re)
        assert _close(E.nu_of_tau(tau, T0[Q]), nu, ab=1e-3)
        assert _close(U / math.sqrt(T0[Q]), Ma, ab=2e-3)
        assert _close(U * N / E.nu_of_tau(tau, T0[Q]), Re, rel=0.03)


def test_planar_poiseuille_table():
    """U_lat is the mean of the parabola: g = 12 nu U / N^2; Fr = U / sqrt(g N)."""
    for Q, tau, N, U, nu, g, Ma, Re, Frs in _rows("planar Poiseuille"):
        Q, tau, N = int(Q), float(tau), int(N)
        U, g = float(U), float(g)
        nu_ = E.nu_of_tau(tau, T0[Q])
        g_calc = 12 * nu_ * U / N ** 2
        assert _close(g_calc, g, rel=0.03)
        assert abs(E.planar_poiseuille_mean(N, g_calc, nu_) - U) < 1e-12
        assert _close_printed(U / math.sqrt(g * N), Frs)


def test_circular_couette_table():
    """M = R1/Delta_r = N_r / 10 for R2/R1 = 11; U_lat = Omega1 M; Re = U N_r / nu;
    N_theta is N_r 2 pi R1 / (R2 - R1) to within 1 % (the tables round it
    differently from row to row)."""
    for Q, Nt, Nr, Om, nu, U, Ma, Re in _rows("circular Couette"):
        Q, Nt, Nr = int(Q), int(Nt), int(Nr)
        Om, U, Ma, Re = float(Om), float(U), float(Ma), float(Re)
        M = 1.0 * Nr / 10.0
        assert _close(Om * M, U, rel=0.01)
        assert _close(U * Nr / E.nu_of_tau(1.0, T0[Q]), Re, rel=0.01)
        assert _close(U / math.sqrt(T0[Q]), Ma, ab=2e-3)
        assert abs(I.n_theta(Nr, 1.0, 11.0) - Nt) <= 0.01 * Nt


def test_circular_poiseuille_table_pins_b_lat_and_M():
    """With u = (A/8)(r^2-M^2)((M+N)^2-r^2)/r (lattice units, M = N_r/10), the
    printed g_lat is the azimuthal acceleration at the inner wall, A nu M, when
    A is fixed by the printed mean velocity; this needs b_lat = (A/8) M^2 (M+N)^2."""
    for Nt, Nr, nu, U, g, Ma, Re, Frs in _rows("circular Poiseuille"):
        Nr, nu, U, g, Re = int(Nr), float(nu), float(U), float(g), float(Re)
        M = Nr / 10.0
        unit = E.Annulus.poiseuille(M, M + Nr, 1.0)
        A = U / unit.mean_u()
        assert _close(A * nu * M, g, rel=0.03)
        assert _close(U * Nr / nu, Re, rel=0.01)
        assert _close_printed(U / math.sqrt(g * Nr), Frs)
        assert abs(I.n_theta(Nr, 1.0, 11.0) - int(Nt)) <= 0.01 * int(Nt)


def test_annulus_couette_boundary_values_and_ode():
    R1, R2, O1, O2 = 1.3, 2.9, 0.7, -0.2
    s = E.Annulus.couette(R1, R2, O1, O2)
    assert abs(s.u(R1) - O1 * R1) < 1e-14 and abs(s.u(R2) - O2 * R2) < 1e-14
    r = np.linspace(R1, R2, 7)[1:-1]
    h = 1e-4
    lap = (-s.u(r) / r ** 2 + (s.u(r + h) - 2 * s.u(r) + s.u(r - h)) / h ** 2
           + (s.u(r + h) - s.u(r - h)) / (2 * h) / r)
    assert np.abs(lap).max() < 1e-5


def test_annulus_poiseuille_follows_force():
    """nu (-u/r^2 + (r u')'/r) + alpha g r = 0 with u = 0 at both walls, and u
    has the sign of the force (reading of the Sec. 3.4 sign)."""
    R1, R2, A = 1.0, 3.0, 0.37
    s = E.Annulus.poiseuille(R1, R2, A)
    assert abs(s.u(R1)) < 1e-14 and abs(s.u(R2)) < 1e-13
    r = np.linspace(R1, R2, 9)[1:-1]
    assert (s.u(r) > 0).all()
    h = 1e-4
    L = (-s.u(r) / r ** 2 + (s.u(r + h) - 2 * s.u(r) + s.u(r - h)) / h ** 2
         + (s.u(r + h) - s.u(r - h)) / (2 * h) / r)
    np.testing.assert_allclose(L, -A * r, rtol=1e-5)


@pytest.mark.parametrize("kind", ["couette", "poiseuille"])
def test_annulus_density_mass_and_radial_balance(kind):
    """rho' = rho0 u^2 / (r T0) and int r rho dr = rho0 (R2^2 - R1^2) / 2."""
    R1, R2, rho0, T = 1.0, 2.5, 1.0, 1.0 / 3.0
    s = (E.Annulus.couette(R1, R2, 0.05, 0.0) if kind == "couette"
         else E.Annulus.poiseuille(R1, R2, 0.04))
    mass = integrate.quad(lambda r: r * s.rho(r, rho0, T), R1, R2, epsabs=1e-14)[0]
    assert abs(mass - rho0 * (R2 ** 2 - R1 ** 2) / 2) < 1e-12
    r = np.linspace(R1, R2, 6)[1:-1]
    h = 1e-5
    drho = (s.rho(r + h, rho0, T) - s.rho(r - h, rho0, T)) / (2 * h)
    np.testing.assert_allclose(drho, rho0 * s.u(r) ** 2 / (r * T), rtol=1e-6)
    Hq = integrate.quad(lambda r: r * s.h(r), R1, R2, epsabs=1e-14)[0]
    assert abs(Hq - s.H()) < 1e-12 * max(1.0, abs(Hq))


def test_planar_limits_of_annulus_solutions():
    """Sec. 3.3/3.4: with the gap fixed and R1 -> infinity the circular flows
    become planar Couette and planar Poiseuille."""
    l = 1.0
    R1 = 1e5
    x = np.linspace(0.1, 0.9, 5) * l
    cou = E.Annulus.couette(R1, R1 + l, 0.0, 0.3 / (R1 + l))
    np.testing.assert_allclose(cou.u(R1 + x), E.planar_couette(x, l, 0.0, 0.3), rtol=2e-4)
    G, nu = 2e-3, 0.1
    A = G / nu / R1  # acceleration alpha g R1 = G at the inner wall
    poi = E.Annulus.poiseuille(R1, R1 + l, A)
    np.testing.assert_allclose(poi.u(R1 + x), E.planar_poiseuille(x, l, G, nu), rtol=2e-4)


def test_lattice_unit_couette_coefficients():
    Nr, M, w1 = 64, 6.4, 3.82e-2
    a, b = E.circular_couette_lattice(Nr, M, w1)
    s = E.Annulus.couette(M, M + Nr, w1)
    assert abs(a - s.a) < 1e-15 and abs(b - s.b) < 1e-12
