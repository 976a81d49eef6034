"""Pins for the oracle's special functions, quadrature, Planck function, grid and table lookup.

Each check compares the oracle with something other than itself: scipy/numpy
library routines, numerical quadrature, closed-form properties.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special

import oracle
import synth


@pytest.mark.parametrize("x", [1e-8, 1e-3, 0.3, 0.999, 1.0, 1.001, 2.5, 10.0, 50.0, 300.0])
def test_E1_matches_scipy(x):
    assert oracle.E1(x) == pytest.approx(special.exp1(x), rel=2e-14)


@pytest.mark.parametrize("x", [1e-6, 1e-2, 0.5, 1.0, 3.0, 12.0, 40.0])
def test_exact_transmission_is_2E3_and_angular_integral(x):
    t = oracle.trans_exact(x)
    assert t == pytest.approx(2.0 * special.expn(3, x), rel=1e-11, abs=1e-300)
    q, _ = integrate.quad(lambda mu: 2.0 * mu * math.exp(-x / mu) if mu > 0 else 0.0, 0.0, 1.0,
                          epsabs=0, epsrel=1e-13, limit=200)
    assert t == pytest.approx(q, rel=1e-9)


def test_exact_diffusivity_limits_and_monotone():
    # Fig. 1: D -> 2 for thin layers, -> 1 for thick ones, decreasing in between
    x = np.logspace(-8, math.log10(600.0), 60)   # 2E3 underflows double beyond ~700
    D = np.array([oracle.diffusivity_exact(v) for v in x])
    assert D[0] == pytest.approx(2.0, abs=1e-5)
    assert 1.0 < D[-1] < 1.011
    assert (np.diff(D) < 0).all()


@pytest.mark.parametrize("G", [1, 2, 8, 20])
def test_gauss_legendre_matches_numpy_and_integrates_polynomials(G):
    x, w = oracle.gauss_legendre(G)
    xr, wr = np.polynomial.legendre.leggauss(G)
    assert np.allclose(x, xr, rtol=0, atol=1e-14)
    assert np.allclose(w, wr, rtol=0, atol=1e-14)
    for k in range(2 * G):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert np.dot(w, x ** k) == pytest.approx(exact, abs=1e-13)


def test_planck_bins_sum_to_stefan_boltzmann():
    # pi * sum_l B_l(T) over a fine wavenumber grid -> sigma T^4
    edges = np.linspace(1e-3, 60000.0, 400001)
    for T in (300.0, 1500.0, 3000.0):
        s = sum(oracle.planck_bin(a, b, T) for a, b in zip(edges[:-1:97], edges[97::97]))
        tot = math.pi * s
        assert tot == pytest.approx(oracle.SIGMA_SB * T ** 4, rel=2e-4)


def test_planck_rayleigh_jeans_and_zero_temperature():
    # h c nu << k T: B_nu -> 2 c k T nu^2 (Rayleigh-Jeans); T <= 0 emits nothing
    kB, c = 1.380649e-16, 2.99792458e10
    b = oracle.planck_bin(0.999, 1.001, 5000.0)
    assert b == pytest.approx(2 * c * kB * 5000.0 * 1.0 * 0.002, rel=2e-4)
    assert oracle.planck_bin(10.0, 20.0, 0.0) == 0.0


def _atm(n=7, P_top=1e-5, P_bot=10.0, grav=2000.0):
    w = synth.config1()
    a = w.atms[0]
    a = synth.Atmosphere(n_layers=n, P_top_bar=P_top, P_bot_bar=P_bot, grav=grav, T_irr=a.T_irr, T_int=a.T_int,
                         T_star=a.T_star, nu_edges=a.nu_edges, omega0=a.omega0, g0=a.g0, table_id=0,
                         T_init=np.full(n, 1000.0))
    return oracle.Atm(a, w.tables[0]), w


def test_grid_geometry():
    atm, _ = _atm()
    lp, P, dm, Pl = oracle.grid(atm)
    n = atm.n
    assert Pl[0] == pytest.approx(10.0 * 1e6, rel=1e-14) and Pl[-1] == pytest.approx(1e-5 * 1e6, rel=1e-14)
    r = Pl[1:] / Pl[:-1]
    assert np.allclose(r, r[0], rtol=1e-12)                       # even in log P
    Pi = P[0::2]
    assert np.allclose(Pi[1:-1], np.sqrt(Pl[:-1] * Pl[1:]), rtol=1e-12)   # geometric means
    assert Pi[0] == pytest.approx(Pl[0] / math.sqrt(r[0]), rel=1e-12)
    assert Pi[-1] == pytest.approx(Pl[-1] * math.sqrt(r[0]), rel=1e-12)
    assert dm.sum() == pytest.approx((Pi[0] - Pi[-1]) / 2000.0, rel=1e-12)
    assert (dm > 0).all() and len(dm) == 2 * n


def test_point_temperatures():
    T = np.array([900.0, 1100.0, 1000.0])
    Tp = oracle.point_temperatures(T)
    assert Tp.tolist() == [900.0, 900.0, 1000.0, 1100.0, 1050.0, 1000.0, 1000.0]


def test_table_coord_nodes_and_clamping():
    x0, dx, nx = 200.0, 2800.0 / 19, 20
    for k in range(nx):
        i, w = oracle.table_coord(x0 + k * dx, x0, dx, nx)
        v = x0 + (i + w) * dx
        assert v == pytest.approx(x0 + k * dx, rel=1e-14)
        assert 0 <= i <= nx - 2 and 0.0 <= w <= 1.0
    assert oracle.table_coord(x0 - 50.0, x0, dx, nx) == (0, 0.0)
    assert oracle.table_coord(x0 + 1e6, x0, dx, nx) == (nx - 2, 1.0)
    i, w = oracle.table_coord(x0 + (nx - 1) * dx, x0, dx, nx)
    assert i == nx - 2 and w == pytest.approx(1.0, abs=1e-14)
    # brute force: the bracketing nodes of random points
    rng = np.random.default_rng(1)
    for x in rng.uniform(x0, x0 + (nx - 1) * dx, 200):
        i, w = oracle.table_coord(x, x0, dx, nx)
        assert x0 + i * dx <= x * (1 + 1e-15) and x <= (x0 + (i + 1) * dx) * (1 + 1e-15)


def test_interp_reproduces_bilinear_function():
    # a table built from f = a + b T + c logP + d T logP is interpolated exactly inside the table
    atm_w, w = _atm(n=9, P_top=1e-5, P_bot=10.0)
    t = w.tables[0]
    lP = t.log10P0 + t.dlog10P * np.arange(t.nP)
    Tn = t.T0 + t.dT * np.arange(t.nT)
    coef = np.random.default_rng(3).uniform(0.1, 1.0, (4, t.L, t.G))
    f = lambda T, l: coef[0] + coef[1] * T / 1000 + coef[2] * l + coef[3] * T / 1000 * l
    k = np.empty((t.nP, t.nT, t.L, t.G))
    for a in range(t.nP):
        for b in range(t.nT):
            k[a, b] = f(Tn[b], lP[a])
    atm = oracle.Atm(atm_w.src, t, kappa64=k)
    T = np.linspace(2900.0, 250.0, atm.n)
    kap, idx, wts = oracle.interp_opacity(atm, T)
    lp, _, _, _ = oracle.grid(atm)
    Tp = oracle.point_temperatures(T)
    for p in range(2 * atm.n + 1):
        assert np.allclose(kap[p], f(Tp[p], lp[p]), rtol=1e-12)


def test_interp_clamps_outside_table():
    atm, w = _atm(n=4, P_top=1e-9, P_bot=1e5)   # beyond both pressure ends of the table
    T = np.array([50.0, 100.0, 5000.0, 9000.0])  # beyond both temperature ends
    kap, idx, wts = oracle.interp_opacity(atm, T)
    t = w.tables[0]
    kt = t.kappa_for_oracle()
    assert np.array_equal(kap[0], kt[t.nP - 1, 0])        # bottom: high P, low T corner
    assert np.array_equal(kap[-1], kt[0, t.nT - 1])       # top: low P, high T corner


def test_boundary_spectra_normalisation():
    atm, _ = _atm()
    toa, bint = oracle.boundary_spectra(atm)
    s = atm.src
    assert toa.sum() == pytest.approx(oracle.SIGMA_SB * s.T_irr ** 4, rel=1e-13)
    assert bint.sum() == pytest.approx(oracle.SIGMA_SB * s.T_int ** 4, rel=1e-13)
    bs = np.array([oracle.planck_bin(a, b, s.T_star) for a, b in zip(s.nu_edges[:-1], s.nu_edges[1:])])
    assert np.allclose(toa / toa.sum(), bs / bs.sum(), rtol=1e-12)
