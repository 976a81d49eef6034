"""Pins of the oracle's isothermal-layer grid (Sect. 2.2.1, eqs. 9, 11 and 14): the grid on
which the emission spectra are computed after convergence (Sect. 3, post-processing).

- an isothermal cavity carries pi B at every interface, with and without scattering;
- a semi-infinite isothermal slab emits the closed form pi B (1 - e^{-2 tau}) + e^{-2 tau} F0;
- on a homogeneous isothermal medium the fixed point of the passes coincides with the
  non-isothermal grid's (both solve the same two-stream equations exactly, layer by layer);
- for a non-isothermal profile the isothermal grid approaches the non-isothermal result as the
  layers are refined (Sect. 2.1.3: enough isothermal layers agree with non-isothermal ones).
"""
import math

import numpy as np

import oracle
import synth
from test_oracle_column import _atm, _cavity_atm, _const_table, _planck


def test_isothermal_grid_cavity_pure_absorption():
    atm, B = _cavity_atm(1100.0)
    r = oracle.flux_sweep_iso(atm, np.full(20, 1100.0))
    assert r["rc"] == 0
    tot = math.pi * B.sum()
    assert np.allclose(r["Fup"], tot, rtol=1e-12) and np.allclose(r["Fdn"], tot, rtol=1e-12)
    assert np.allclose(r["toa"], math.pi * B, rtol=1e-12)


def test_isothermal_grid_cavity_with_scattering_converges_to_pi_b():
    L, G = 12, 4
    w0 = np.linspace(0.05, 0.95, L).astype(np.float32)
    g0 = np.linspace(-0.5, 0.6, L).astype(np.float32)
    atm, B = _cavity_atm(900.0, L, G, w0, g0)
    r = oracle.flux_sweep_iso(atm, np.full(20, 900.0), n_passes=600)
    tot = math.pi * B.sum()
    assert np.allclose(r["Fup"], tot, rtol=1e-8) and np.allclose(r["Fdn"], tot, rtol=1e-8)
    assert np.allclose(r["toa"], math.pi * B, rtol=1e-8)


def test_isothermal_grid_semi_infinite_slab_closed_form():
    L, G, n, T = 10, 6, 30, 1300.0
    kap = np.logspace(-6, -2, L * G).reshape(L, G)
    t, k = _const_table(L, G, kap)
    a = _atm(n, L, 0.0, 0.0, 5000.0)
    atm = oracle.Atm(a, t, kappa64=k)
    r = oracle.flux_sweep_iso(atm, np.full(n, T))
    _, P, _, _ = oracle.grid(atm)
    _, w = oracle.gauss_legendre(G)
    B = _planck(a, T)
    tau = kap * (P[0] - P[-1]) / a.grav
    e = np.exp(-2.0 * tau)
    F0 = math.pi * B[:, None] * (1 - e)
    Ftop = math.pi * B[:, None] * (1 - e) + e * F0
    assert np.allclose(r["toa"], (Ftop * (w / 2)).sum(axis=1), rtol=1e-12)


def test_isothermal_grid_matches_sublayered_grid_on_a_homogeneous_medium():
    # constant kappa and T: each isothermal layer is the two sublayers of the non-isothermal grid
    # merged; at the fixed point of the passes both grids hold the exact two-stream solution
    L, G, n, T = 8, 4, 16, 1150.0
    kap = np.logspace(-4, -1, L * G).reshape(L, G)
    t, k = _const_table(L, G, kap)
    a = _atm(n, L, 1400.0, 250.0, 5800.0, omega0=np.linspace(0.0, 0.9, L).astype(np.float32),
             g0=np.linspace(0.0, 0.5, L).astype(np.float32), P_top=1e-4, P_bot=1e-1)
    atm = oracle.Atm(a, t, kappa64=k)
    Tl = np.full(n, T)
    iso = oracle.flux_sweep_iso(atm, Tl, n_passes=4000)
    sub = oracle.flux_sweep(atm, Tl, n_passes=4000)
    assert np.allclose(iso["Fup"], sub["Fup"], rtol=1e-9) and np.allclose(iso["Fdn"], sub["Fdn"], rtol=1e-9)
    assert np.allclose(iso["toa"], sub["toa"], rtol=1e-9)


def _emergent(n, iso):
    wl = synth.config1()
    base = wl.atms[0]
    a = synth.Atmosphere(n_layers=n, P_top_bar=1e-6, P_bot_bar=1e2, grav=1000.0, T_irr=1200.0, T_int=100.0,
                         T_star=5000.0, nu_edges=base.nu_edges, omega0=base.omega0, g0=base.g0, table_id=0,
                         T_init=np.full(n, 1000.0))
    atm = oracle.Atm(a, wl.tables[0])
    x = np.linspace(0.0, 1.0, n)
    T = 1500.0 - 600.0 * x + 100.0 * np.sin(6.0 * x)
    r = oracle.flux_sweep_iso(atm, T) if iso else oracle.flux_sweep(atm, T)
    return r["Fup"][-1]


def test_isothermal_layers_converge_to_non_isothermal_under_refinement():
    err = {n: abs(_emergent(n, True) / _emergent(n, False) - 1.0) for n in (25, 100, 400)}
    assert err[25] > err[100] > err[400]
    assert err[400] < 0.02 * err[25]
