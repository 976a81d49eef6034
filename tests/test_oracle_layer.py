"""Pins for the single-layer solutions of the oracle.

Two-stream forms (eqs. 8-15): compared with a 50-digit matrix-exponential
solution of the two-stream ODE as a two-point boundary-value problem,
    dF_up/dtau = g1 F_up - g2 F_dn - 2 pi (1 - w0) B(tau)
    dF_dn/dtau = g2 F_up - g1 F_dn + 2 pi (1 - w0) B(tau)
(tau downwards), with g1 + g2 = D (1 - w0 g0) and g1 - g2 = D (1 - w0): the
eigenvalue of this system is eq. (8)'s exponent, its eigenvector ratio is
zeta_-/zeta_+ of eq. (13), and its isothermal pure-absorption solution is
eq. (9).  The readings taken for eq. (15) (Planck values at the interface
they belong to; gradient prefactor eps/(1 - w0 g0)) are exactly what this
comparison fixes.

Exact forms (eqs. 3-6): compared with a numerical angular quadrature of the
formal solution of eq. (1) for B linear in tau.
"""
import math

import mpmath as mp
import pytest
from scipy import integrate

import oracle

PI = math.pi


def ode_layer(F1up, F2dn, B1, B2, dtau, w0, g0, D=2.0):
    mp.mp.dps = 50
    g1 = mp.mpf(D) * (1 - mp.mpf(w0) * (1 + mp.mpf(g0)) / 2)
    g2 = mp.mpf(D) * mp.mpf(w0) * (1 - mp.mpf(g0)) / 2
    s = 2 * mp.pi * (1 - mp.mpf(w0))
    Bp = (mp.mpf(B1) - mp.mpf(B2)) / mp.mpf(dtau)     # dB/dt, t from the top down
    M = mp.matrix([[g1, -g2, -s * B2, -s * Bp],
                   [g2, -g1, s * B2, s * Bp],
                   [0, 0, 0, 0],
                   [0, 0, 1, 0]])
    Phi = mp.expm(M * mp.mpf(dtau))
    U0 = (mp.mpf(F1up) - Phi[0, 1] * F2dn - Phi[0, 2]) / Phi[0, 0]
    F1dn = Phi[1, 0] * U0 + Phi[1, 1] * F2dn + Phi[1, 2]
    return float(U0), float(F1dn)


CASES = [(dt, w0, g0) for dt in (2e-4, 0.01, 0.3, 1.5, 6.0)
         for w0 in (0.0, 0.3, 0.9) for g0 in (-0.5, 0.0, 0.5)]


@pytest.mark.parametrize("dtau,w0,g0", CASES)
def test_twostream_layer_matches_ode(dtau, w0, g0):
    F1up, F2dn, B1, B2 = 3.1e7, 1.2e7, 1.4e7, 0.9e7
    u, d = oracle.layer_twostream(F1up, F2dn, B1, B2, dtau, w0, g0)
    ue, de = ode_layer(F1up, F2dn, B1, B2, dtau, w0, g0)
    scale = max(F1up, F2dn, PI * B1)
    assert abs(u - ue) < 1e-11 * scale and abs(d - de) < 1e-11 * scale


@pytest.mark.parametrize("D", [1.66, 2.0])
def test_twostream_layer_matches_ode_other_D(D):
    p = oracle.params(D=D)
    u, d = oracle.layer_twostream(2e7, 5e6, 1e7, 8e6, 0.7, 0.6, 0.3, p)
    ue, de = ode_layer(2e7, 5e6, 1e7, 8e6, 0.7, 0.6, 0.3, D=D)
    assert u == pytest.approx(ue, rel=1e-12) and d == pytest.approx(de, rel=1e-12)


def test_thin_sublayer_uses_isothermal_mean_planck():
    # below dtau_iso the layer is isothermal at the mean of its two Planck values
    u, d = oracle.layer_twostream(3e7, 1e7, 1.5e7, 1.0e7, 5e-5, 0.4, 0.2)
    ue, de = ode_layer(3e7, 1e7, 1.25e7, 1.25e7, 5e-5, 0.4, 0.2)
    assert u == pytest.approx(ue, rel=1e-13) and d == pytest.approx(de, rel=1e-13)


def test_pure_scattering_form_matches_conservative_ode_and_conserves_net_flux():
    for dtau in (1e-3, 0.5, 20.0):
        for g0 in (-0.5, 0.0, 0.7):
            u, d = oracle.layer_twostream(3e7, 1e7, 1.5e7, 1.0e7, dtau, 1.0 - 1e-8, g0)
            ue, de = ode_layer(3e7, 1e7, 0.0, 0.0, dtau, 1.0, g0)
            assert u == pytest.approx(ue, rel=1e-12) and d == pytest.approx(de, rel=1e-12)
            assert (u - 1e7) == pytest.approx(3e7 - d, rel=1e-14)     # net flux conserved


def test_pure_scattering_limits():
    # transparent: fluxes pass unchanged; opaque: the layer reflects
    u, d = oracle.layer_twostream(3e7, 1e7, 0, 0, 1e-12, 1.0, 0.0)
    assert u == pytest.approx(3e7, rel=1e-10) and d == pytest.approx(1e7, rel=1e-10)
    u, d = oracle.layer_twostream(3e7, 1e7, 0, 0, 1e12, 1.0, 0.0)
    assert u == pytest.approx(1e7, rel=1e-9) and d == pytest.approx(3e7, rel=1e-9)


def test_printed_gradient_prefactor_differs_only_with_forward_scattering():
    base = oracle.layer_twostream(2e7, 5e6, 1e7, 8e6, 0.7, 0.6, 0.3)
    printed = oracle.layer_twostream(2e7, 5e6, 1e7, 8e6, 0.7, 0.6, 0.3, oracle.params(printed_gradient=1))
    assert abs(base[0] - printed[0]) > 1e3
    b0 = oracle.layer_twostream(2e7, 5e6, 1e7, 8e6, 0.7, 0.6, 0.0)
    p0 = oracle.layer_twostream(2e7, 5e6, 1e7, 8e6, 0.7, 0.6, 0.0, oracle.params(printed_gradient=1))
    assert b0 == p0


def _formal_solution(F1up, F2dn, B1, B2, dtau):
    """Angular quadrature of the formal solution of eq. (1), B linear in tau, isotropic incidence."""
    Bt = lambda t: B2 + (B1 - B2) * t / dtau

    def I_up(mu):      # intensity leaving the top at angle mu
        src, _ = integrate.quad(lambda v: Bt(mu * v) * math.exp(-v), 0.0, dtau / mu, epsabs=0, epsrel=1e-13)
        return F1up / PI * math.exp(-dtau / mu) + src

    def I_dn(mu):      # intensity leaving the bottom
        src, _ = integrate.quad(lambda v: Bt(dtau - mu * v) * math.exp(-v), 0.0, dtau / mu, epsabs=0, epsrel=1e-13)
        return F2dn / PI * math.exp(-dtau / mu) + src

    up, _ = integrate.quad(lambda mu: 2 * PI * mu * I_up(mu), 1e-12, 1.0, epsabs=0, epsrel=1e-12, limit=200)
    dn, _ = integrate.quad(lambda mu: 2 * PI * mu * I_dn(mu), 1e-12, 1.0, epsabs=0, epsrel=1e-12, limit=200)
    return up, dn


@pytest.mark.parametrize("dtau", [3e-3, 0.2, 1.0, 4.0, 15.0])
def test_exact_layer_matches_formal_solution(dtau):
    F1up, F2dn, B1, B2 = 3.1e7, 1.2e7, 1.4e7, 0.9e7
    u, d = oracle.layer_exact(F1up, F2dn, B1, B2, dtau)
    ue, de = _formal_solution(F1up, F2dn, B1, B2, dtau)
    assert u == pytest.approx(ue, rel=1e-9) and d == pytest.approx(de, rel=1e-9)


def test_exact_layer_thick_limit_is_eddington_barbier():
    # deep layer: emergent flux -> pi (B_top + 2/3 dB/dtau)
    B1, B2, dtau = 2.0e7, 1.0e7, 400.0
    u, _ = oracle.layer_exact(5e7, 0.0, B1, B2, dtau)
    assert u == pytest.approx(PI * (B2 + (2.0 / 3.0) * (B1 - B2) / dtau), rel=1e-12)
