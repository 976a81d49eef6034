"""Pins of the oracle's tabulated Planck and transmission functions (Sect. 2.6: a 10 K grid in T
and a 0.1 grid in log10 opacity, here in log10 of the layer exponent x = lambda dtau, which is
proportional to the opacity).

- the transmission table reproduces 1 - e^-x at its nodes, lies below it between them (the
  function is concave) within the linear-interpolation bound (dx)^2/8 max|u''|, and is x itself
  below the first node;
- the Planck table reproduces the bin's Planck intensity at the 10 K nodes and is the mean of the
  two neighbouring nodes halfway between them;
- an isothermal cavity at a node temperature stays at pi B with the tabulated transmission
  (Kirchhoff's law holds for any transmission value);
- tabulated fluxes stay within 1% of the exact ones on a scattering column, and differ from them;
- the tabulated radiative equilibrium lies within 0.2 K of the exact one.
"""
import math

import numpy as np

import oracle
import synth
from test_oracle_column import _cavity_atm


def test_transmission_table_nodes_and_interpolation_bound():
    x_nodes = 10.0 ** (oracle.TAB_X0 + 0.1 * np.arange(oracle.TAB_NX))
    for x in x_nodes[:-1]:
        assert abs(oracle.tab_one_minus_trans(x) / -math.expm1(-x) - 1.0) < 1e-14
    rng = np.random.default_rng(3)
    for i in rng.integers(0, oracle.TAB_NX - 1, 400):
        x0, x1 = x_nodes[i], x_nodes[i + 1]
        x = x0 + rng.uniform(0.0, 1.0) * (x1 - x0)
        u, ex = oracle.tab_one_minus_trans(x), -math.expm1(-x)
        assert u <= ex * (1 + 1e-14)
        assert ex - u <= (x1 - x0) ** 2 / 8.0 * math.exp(-x0) * (1 + 1e-9) + 1e-300
    x = 1e-9
    assert oracle.tab_one_minus_trans(x) == x
    assert oracle.tab_one_minus_trans(1e3) == 1.0


def test_planck_table_nodes_and_midpoints():
    e = synth.nu_edges(30)
    for lo, hi in zip(e[:-1:3], e[1::3]):
        for T in (200.0, 870.0, 1500.0, 2990.0):
            assert oracle.tab_planck_bin(lo, hi, T) == oracle.planck_bin(lo, hi, T) or \
                abs(oracle.tab_planck_bin(lo, hi, T) / oracle.planck_bin(lo, hi, T) - 1) < 1e-13
            m = oracle.tab_planck_bin(lo, hi, T + 5.0)
            avg = 0.5 * (oracle.planck_bin(lo, hi, T) + oracle.planck_bin(lo, hi, T + 10.0))
            assert abs(m - avg) <= 1e-13 * avg + 1e-300


def test_isothermal_cavity_at_a_node_temperature_with_tabulated_transmission():
    L, G = 12, 4
    w0 = np.linspace(0.0, 0.9, L).astype(np.float32)
    g0 = np.linspace(-0.3, 0.5, L).astype(np.float32)
    atm, B = _cavity_atm(900.0, L, G, w0, g0)
    r = oracle.flux_sweep(atm, np.full(20, 900.0), n_passes=400, p=oracle.params(tabulate=1), spectra=True)
    ref = math.pi * B[:, None]
    assert np.allclose(r["up_spec"], ref, rtol=1e-9) and np.allclose(r["dn_spec"], ref, rtol=1e-9)


def test_tabulated_fluxes_close_to_exact():
    wl = synth.small_scattering(L=10, n=30)
    atm = oracle.Atm.from_workload(wl)
    T = synth.perturbed_profile(wl.atms[0], 2)
    ex = oracle.flux_sweep(atm, T, n_passes=5)
    tb = oracle.flux_sweep(atm, T, n_passes=5, p=oracle.params(tabulate=1))
    # the tables move the fluxes by ~1e-4 (measured 9.6e-5 upward, 1.9e-4 downward here)
    for k in ("Fup", "Fdn"):
        d = np.max(np.abs(tb[k] / ex[k] - 1))
        assert 1e-6 < d < 5e-4, (k, d)


def test_tabulated_equilibrium_close_to_the_exact_one():
    # Sect. 2.6: the grid resolutions suffice for a converged model; here the tabulated
    # equilibrium of a 40-layer scattering column lies within 0.2 K of the exact one (0.06 K seen)
    wl = synth.small_scattering(L=30, n=40)
    atm = oracle.Atm.from_workload(wl)
    Ts = []
    for tab in (0, 1):
        st = oracle.State(atm, wl.atms[0].T_init)
        rc, _, _ = oracle.solve_re(atm, st, oracle.params(tabulate=tab, tol=1e-10, max_iter=200000))
        assert rc == oracle.CONVERGED
        Ts.append(st.T.copy())
    d = np.abs(Ts[1] - Ts[0])
    assert 1e-4 < d.max() < 0.2, d.max()


def test_temperatures_above_the_planck_table_stop_the_iteration():
    # the Planck table of Sect. 2.6 ends at 6000 K: a profile that reaches above it ends the
    # iteration with its own status instead of continuing on the last node's values; below the
    # table's top, and without tables, the step is an ordinary one
    wl = synth.small_scattering(L=6, n=20)
    atm = oracle.Atm.from_workload(wl)
    for T0, tab, want in ((6100.0, 1, oracle.OUT_OF_RANGE), (5000.0, 1, oracle.UPDATED), (6100.0, 0, oracle.UPDATED)):
        T = np.full(20, T0)
        p = oracle.params(tabulate=tab)
        r = oracle.flux_sweep(atm, T, n_passes=5, p=p)
        st = oracle.State(atm, T)
        rc, _, _ = oracle.temp_update(atm, st, r["Fup"], r["Fdn"], p)
        assert rc == want, (T0, tab, rc)
