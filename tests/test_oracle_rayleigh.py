"""Pins of the oracle's H2 Rayleigh scattering (Sect. 2.1.4, eqs. 16-17).

- the opacity agrees with an independent published fit of the H2 Rayleigh cross section
  (Dalgarno & Williams 1962: sigma = 8.14e-13/l^4 + 1.28e-6/l^6 + 1.61/l^8 cm^2, l in Angstrom)
  to a few per cent over 0.3-2 um, and approaches the lambda^-4 law at long wavelengths;
- with an opacity constant along the column, per-sublayer omega0 = kappa_R/(kappa + kappa_R)
  reproduces the per-bin path given that omega0 and the total opacity;
- an atmosphere scattering only (no absorption) conserves its net flux exactly.
"""
import numpy as np

import oracle
import synth
from test_oracle_column import _atm, _const_table

MP = 1.67262192369e-24


def _kappa_dw(lam_um):
    la = lam_um * 1e4
    sigma = 8.14e-13 / la ** 4 + 1.28e-6 / la ** 6 + 1.61 / la ** 8
    return sigma / (2.4 * MP)


def _kappa(lam_um):
    nu = 1e4 / lam_um
    return oracle.rayleigh_kappa(nu * (1 - 1e-9), nu * (1 + 1e-9))


def test_rayleigh_opacity_matches_an_independent_fit():
    for lam in np.geomspace(0.3, 2.0, 12):
        assert abs(_kappa(lam) / _kappa_dw(lam) - 1.0) < 0.05, lam
    # long wavelengths: the refractive index is constant, the cross section goes as lambda^-4
    assert abs(_kappa(100.0) / _kappa(200.0) / 16.0 - 1.0) < 1e-4


def test_per_sublayer_albedo_reproduces_the_per_bin_path_for_constant_opacity():
    L, G, n = 10, 1, 30
    e = synth.nu_edges(L)
    kR = np.array([oracle.rayleigh_kappa(x, y) for x, y in zip(e[:-1], e[1:])])
    kabs = np.logspace(-6, -2, L)
    g0 = np.linspace(0.0, 0.5, L).astype(np.float32)
    # Rayleigh path: the table holds the absorption only
    t1, k1 = _const_table(L, G, kabs[:, None])
    a1 = _atm(n, L, 1300.0, 200.0, 5800.0, g0=g0, P_top=1e-5, P_bot=10.0)
    r1 = oracle.flux_sweep(oracle.Atm(a1, t1, kappa64=k1, rayleigh=True), np.linspace(1600, 900, n), n_passes=5)
    # per-bin path: total opacity in the table, omega0 given per bin (float64 inputs)
    w0 = kR / (kabs + kR)
    t2, k2 = _const_table(L, G, (kabs + kR)[:, None])
    a2 = _atm(n, L, 1300.0, 200.0, 5800.0, g0=g0, P_top=1e-5, P_bot=10.0)
    atm2 = oracle.Atm(a2, t2, kappa64=k2)
    atm2.w0[:] = w0
    r2 = oracle.flux_sweep(atm2, np.linspace(1600, 900, n), n_passes=5)
    for k in ("Fup", "Fdn", "toa"):
        assert np.allclose(r1[k], r2[k], rtol=1e-10), k


def test_scattering_only_atmosphere_conserves_net_flux():
    L, G, n = 6, 3, 25
    t, k = _const_table(L, G, np.full((L, G), 1e-30))
    a = _atm(n, L, 1000.0, 300.0, 5000.0, g0=np.linspace(0.0, 0.4, L).astype(np.float32), P_top=1e-5, P_bot=1e2)
    atm = oracle.Atm(a, t, kappa64=k, rayleigh=True)
    r = oracle.flux_direct(atm, np.linspace(1500, 800, n))
    assert r["rc"] == 0
    net = r["Fup"] - r["Fdn"]
    assert np.max(np.abs(net - net[0])) < 1e-9 * np.max(r["Fup"])
