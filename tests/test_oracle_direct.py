"""Pins of the oracle's direct column solve: the exact solution of the coupled two-stream
equations, i.e. the limit of the scattering passes of Sect. 2.2.3.

- the affine layer coefficients reproduce the layer solutions they come from (eqs. 11, 14, 15);
- the direct solve equals many passes of the iteration (both grids), and one pass without
  scattering (where one pass is exact);
- conservative scattering conserves the net flux exactly (no pass truncation);
- an isothermal cavity carries pi B everywhere.
"""
import math

import numpy as np

import oracle
import synth
from test_oracle_column import _atm, _cavity_atm, _const_table


def test_affine_coefficients_reproduce_the_layer_solutions():
    rng = np.random.default_rng(5)
    p = oracle.params()
    for _ in range(300):
        kind = rng.integers(0, 3)
        w0 = [0.0, rng.uniform(0, 0.98), 1.0][kind]
        g0 = rng.uniform(-0.5, 0.7)
        dtau = 10 ** rng.uniform(-7, 2)
        B1, B2 = rng.uniform(1e3, 1e8, 2)
        F1, F2 = rng.uniform(0, 1e8, 2)
        c = oracle.layer_affine(B1, B2, dtau, w0, g0, p)
        up, dn = oracle.layer_twostream(F1, F2, B1, B2, dtau, w0, g0, p)
        scale = max(abs(up), abs(dn), F1, F2, B1, B2)
        assert abs(c[0] * F1 + c[1] * F2 + c[2] - up) < 1e-12 * scale
        assert abs(c[3] * F2 + c[4] * F1 + c[5] - dn) < 1e-12 * scale


def _close(a, b, tol):
    for k in ("Fup", "Fdn", "toa"):
        assert np.max(np.abs(a[k] - b[k]) / np.maximum(np.abs(b[k]), 1e-300)) < tol, k


def test_direct_solve_is_the_limit_of_the_passes():
    wl = synth.small_scattering(L=8, n=20)
    atm = oracle.Atm.from_workload(wl)
    T = synth.perturbed_profile(wl.atms[0], 3)
    d = oracle.flux_direct(atm, T)
    assert d["rc"] == 0
    _close(d, oracle.flux_sweep(atm, T, n_passes=4000), 1e-9)
    di = oracle.flux_direct(atm, T, iso=True)
    assert di["rc"] == 0
    _close(di, oracle.flux_sweep_iso(atm, T, n_passes=4000), 1e-9)
    # a handful of passes is still visibly short of the limit
    five = oracle.flux_sweep(atm, T, n_passes=5)
    assert np.max(np.abs(five["toa"] / d["toa"] - 1)) > 1e-6


def test_direct_solve_without_scattering_equals_one_pass():
    wl = synth.config1()
    atm = oracle.Atm.from_workload(wl)
    T = synth.perturbed_profile(wl.atms[0], 2, amp=500)
    _close(oracle.flux_direct(atm, T), oracle.flux_sweep(atm, T, n_passes=1), 1e-11)


def test_direct_solve_conserves_net_flux_under_conservative_scattering():
    L, G, n = 6, 3, 25
    kap = np.logspace(-5, -1, L * G).reshape(L, G)
    t, k = _const_table(L, G, kap)
    a = _atm(n, L, 1000.0, 300.0, 5000.0, omega0=np.ones(L, np.float32),
             g0=np.linspace(-0.4, 0.6, L).astype(np.float32))
    atm = oracle.Atm(a, t, kappa64=k)
    r = oracle.flux_direct(atm, np.linspace(1500, 800, n))
    net = r["Fup"] - r["Fdn"]
    assert np.max(np.abs(net - net[0])) < 1e-9 * np.max(r["Fup"])
    # pure scattering emits nothing: the net flux is the internal flux at every interface
    assert abs(net[0] - oracle.SIGMA_SB * 300.0 ** 4) < 1e-9 * np.max(r["Fup"])


def test_direct_solve_isothermal_cavity_with_scattering():
    L, G = 12, 4
    w0 = np.linspace(0.05, 0.95, L).astype(np.float32)
    g0 = np.linspace(-0.5, 0.6, L).astype(np.float32)
    atm, B = _cavity_atm(900.0, L, G, w0, g0)
    tot = math.pi * B.sum()
    for iso in (False, True):
        r = oracle.flux_direct(atm, np.full(20, 900.0), iso=iso)
        assert np.allclose(r["Fup"], tot, rtol=1e-11) and np.allclose(r["Fdn"], tot, rtol=1e-11)
        assert np.allclose(r["toa"], math.pi * B, rtol=1e-11)


def test_pass_truncation_error_against_the_exact_solution():
    # reading of the scattering passes (Sect. 2.2.3): from a cold start the error of K passes
    # against the exact column solution falls geometrically with K; a temperature step's
    # 1 + 4 passes start warm, from the previous step's field
    wl = synth.small_scattering(L=8, n=20)
    atm = oracle.Atm.from_workload(wl)
    T = synth.perturbed_profile(wl.atms[0], 3)
    d = oracle.flux_direct(atm, T)
    err = []
    for K in (1, 2, 5, 10, 20):
        r = oracle.flux_sweep(atm, T, n_passes=K)
        err.append(max(np.max(np.abs(r["Fup"] / d["Fup"] - 1)), np.max(np.abs(r["toa"] / d["toa"] - 1))))
    assert all(a > b for a, b in zip(err, err[1:]))
    assert err[-1] < 1e-3 * err[0]
