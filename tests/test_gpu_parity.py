"""GPU parity: the CUDA path through the C ABI vs the FP64 CPU oracle on the same seeded inputs.

Tolerances: table indices and weights bit-exact; opacities 2e-6
relative (float32 bilinear of the float32 table); bolometric fluxes 1e-5 relative; net flux 1e-5
of the local flux; emergent spectrum 1e-5 of the bin's larger TOA stream; one temperature step
1e-12 relative with bit-exact multipliers and sign histories; converged temperatures 0.1 K.
"""
import numpy as np
import pytest

import oracle
import synth
import paper_1606_05474_b300 as hp
from helpers import make_plan, pack, rel_err

pytestmark = pytest.mark.gpu

FLUX_TOL = 1e-5


def _oracle_sweep(wl, a, T, **kw):
    return oracle.flux_sweep(oracle.Atm.from_workload(wl, a), T, **kw)


@pytest.mark.parametrize("case", ["config1", "scat", "clamp"])
def test_interp_opacity_indices_bit_exact(case):
    if case == "config1":
        wl = synth.config1(); T = synth.perturbed_profile(wl.atms[0], 1, amp=900)
    elif case == "scat":
        wl = synth.small_scattering(L=9, n=45); T = synth.perturbed_profile(wl.atms[0], 2)
    else:
        wl = synth.small_scattering(L=5, n=30)
        T = np.linspace(80.0, 4000.0, 30)         # below and above the table's temperature range
    plan = make_plan(wl)
    kap, idx, w = plan.interp_opacity(pack([T]))
    okap, oidx, ow = oracle.interp_opacity(oracle.Atm.from_workload(wl), T)
    assert np.array_equal(idx.cpu().numpy(), oidx)
    assert np.array_equal(w.cpu().numpy(), ow)                      # bit-exact weights
    assert rel_err(kap.cpu().numpy(), okap.reshape(-1)) < 2e-6


def _check_toa(toa, r, atm, tol=FLUX_TOL):
    # emergent spectrum: per bin, relative to the bin's larger TOA stream (the emergent flux or
    # the incident one); a reflected flux that is a small fraction of the incident stream
    # inherits float32 rounding of that stream
    inc, _ = oracle.boundary_spectra(atm)
    g = toa.cpu().numpy().astype(np.float64)
    scale = np.maximum(np.abs(r["toa"]), inc)
    assert np.max(np.abs(g - r["toa"]) / scale) < tol


def _check_fluxes(Fu, Fd, r, tol=FLUX_TOL):
    Fu = Fu.cpu().numpy(); Fd = Fd.cpu().numpy()
    assert rel_err(Fu, r["Fup"]) < tol
    assert rel_err(Fd, r["Fdn"]) < tol
    scale = np.maximum(r["Fup"], r["Fdn"])
    assert np.max(np.abs((Fu - Fd) - (r["Fup"] - r["Fdn"])) / scale) < tol


def test_flux_sweep_pure_absorption_config1():
    wl = synth.config1()
    T = synth.perturbed_profile(wl.atms[0], 4)
    plan = make_plan(wl)
    Fu, Fd, toa = plan.flux_sweep(pack([T]))
    r = _oracle_sweep(wl, 0, T)
    _check_fluxes(Fu, Fd, r)
    _check_toa(toa, r, oracle.Atm.from_workload(wl))


@pytest.mark.parametrize("n,L", [(40, 12), (111, 7), (200, 5), (239, 3), (2, 4), (40, 1)])
def test_flux_sweep_scattering_cold_then_warm(n, L):
    # several lane tiles and a ragged tail (2n+1 not a multiple of 32), five passes,
    # then a second evaluation at new temperatures warm-started from the first
    wl = synth.small_scattering(L=L, n=n)
    atm = oracle.Atm.from_workload(wl)
    T1 = synth.perturbed_profile(wl.atms[0], 5)
    T2 = T1 + 7.0 * np.sin(np.arange(n))
    plan = make_plan(wl)
    Fu, Fd, toa = plan.flux_sweep(pack([T1]), n_passes=5)
    warm = np.zeros(atm.L * atm.G * (2 * n + 1))
    r1 = oracle.flux_sweep(atm, T1, n_passes=5, warm=warm, warm_valid=False)
    _check_fluxes(Fu, Fd, r1)
    _check_toa(toa, r1, atm)
    Fu2, Fd2, _ = plan.flux_sweep(pack([T2]), n_passes=5, warm=True)
    r2 = oracle.flux_sweep(atm, T2, n_passes=5, warm=warm, warm_valid=True)
    _check_fluxes(Fu2, Fd2, r2)


def test_flux_sweep_full_size_single_atmosphere():
    # 100 layers x 3000 bins x 20 g with scattering, the launch configuration the benchmark times
    wl = synth.config2()
    T = synth.perturbed_profile(wl.atms[0], 6)
    plan = make_plan(wl)
    Fu, Fd, toa = plan.flux_sweep(pack([T]))
    r = _oracle_sweep(wl, 0, T)
    _check_fluxes(Fu, Fd, r)
    _check_toa(toa, r, oracle.Atm.from_workload(wl))


def test_pure_scattering_bins_conserve_net_flux():
    wl = synth.small_scattering(L=4, n=20)
    wl.atms[0].omega0[:] = 1.0
    T = synth.perturbed_profile(wl.atms[0], 8)
    plan = make_plan(wl)
    Fu, Fd, _ = plan.flux_sweep(pack([T]), n_passes=5)
    r = _oracle_sweep(wl, 0, T, n_passes=5)
    _check_fluxes(Fu, Fd, r)


def test_temperature_step_matches_oracle():
    import torch
    wl = synth.config1()
    atm = oracle.Atm.from_workload(wl)
    T = synth.perturbed_profile(wl.atms[0], 9)
    plan = make_plan(wl)
    st = oracle.State(atm, T)
    Tg = pack([T])
    state = plan.new_state()
    for step in range(12):                                   # enough steps to exercise the 6-step rule
        r = oracle.flux_sweep(atm, st.T)
        Fu = torch.from_numpy(r["Fup"]).cuda(); Fd = torch.from_numpy(r["Fdn"]).cuda()
        Tg.copy_(torch.from_numpy(st.T))
        plan.temp_update(Fu, Fd, Tg, state)
        rc, metric, dT = oracle.temp_update(atm, st, r["Fup"], r["Fdn"])
        assert rel_err(Tg.cpu().numpy(), st.T) < 1e-12
        assert np.array_equal(state["hist"].cpu().numpy(), st.hist.astype(np.uint8))
        assert np.array_equal(state["nhist"].cpu().numpy(), st.nhist.astype(np.uint8))
        assert rel_err(state["mult"].cpu().numpy(), st.mult) < 1e-15
        assert state["metric"].item() == pytest.approx(metric, rel=1e-12)


def test_deterministic_repeat():
    wl = synth.small_scattering(L=16, n=60)
    T = pack([synth.perturbed_profile(wl.atms[0], 10)])
    plan = make_plan(wl)
    a = [x.clone() for x in plan.flux_sweep(T, n_passes=5)]
    b = plan.flux_sweep(T, n_passes=5)
    for x, y in zip(a, b):
        assert bool((x == y).all())


def test_single_gauss_point_and_two_bins():
    # G = 1 (weight 1) with scattering, the smallest grid the method allows
    wl = synth.small_scattering(L=2, n=3, G=1)
    T = synth.perturbed_profile(wl.atms[0], 12)
    plan = make_plan(wl)
    Fu, Fd, toa = plan.flux_sweep(pack([T]), n_passes=5)
    r = _oracle_sweep(wl, 0, T, n_passes=5)
    _check_fluxes(Fu, Fd, r)


def test_species_mixing_matches_mixed_table():
    # eq. (34): the opacity of a mixed atmosphere is the weighted sum of its species' tables;
    # bilinear interpolation is linear, so the oracle interpolates the element-wise mixed table
    wl = synth.learned_dataset(3, L=40, n=60)
    plan = make_plan(wl)
    Ts = [synth.perturbed_profile(a, 30 + i) for i, a in enumerate(wl.atms)]
    Fu, Fd, toa = plan.flux_sweep(pack(Ts), n_passes=5)
    Fus, Fds = plan.split_interfaces(Fu.cpu().numpy()), plan.split_interfaces(Fd.cpu().numpy())
    for i, a in enumerate(wl.atms):
        atm = oracle.Atm.from_workload(wl, i)
        r = oracle.flux_sweep(atm, Ts[i], n_passes=5)
        assert rel_err(Fus[i], r["Fup"]) < FLUX_TOL and rel_err(Fds[i], r["Fdn"]) < FLUX_TOL


@pytest.mark.parametrize("G", [6, 20])
def test_species_mixing_three_tables(G):
    # eq. (34) with three species on the per-thread gather (G not a multiple of 4) and on the
    # four-Gauss-point one, several lane tiles and a ragged tail; the emergent spectrum too
    import dataclasses
    L, n = 11, 45
    tabs = [synth.make_ktable(synth.SEED_BASE + 31, j, L, G, -6.0, 3.0) for j in range(3)]
    a0 = synth.small_scattering(L=L, n=n, G=G).atms[0]
    wl = synth.Workload(name=f"mix3-{G}", atms=[dataclasses.replace(a0, species=[(0, 0.5), (1, 0.3), (2, 0.2)])],
                        tables=tabs, n_scat=4)
    T = synth.perturbed_profile(wl.atms[0], 41)
    plan = make_plan(wl)
    Fu, Fd, toa = plan.flux_sweep(pack([T]), n_passes=5)
    r = _oracle_sweep(wl, 0, T, n_passes=5)
    _check_fluxes(Fu, Fd, r)
    _check_toa(toa, r, oracle.Atm.from_workload(wl, 0))


@pytest.mark.parametrize("n,L,passes", [(40, 12, 1), (40, 12, 81), (101, 9, 81), (239, 3, 5)])
def test_isothermal_layer_grid_emission_spectrum(n, L, passes):
    # the grid of the post-processing spectra (isothermal layers, Sect. 2.2.1 and Sect. 3),
    # cold start, up to 1 + 80 scattering passes (Sect. 2.2.3)
    wl = synth.small_scattering(L=L, n=n)
    atm = oracle.Atm.from_workload(wl)
    T = synth.perturbed_profile(wl.atms[0], 9)
    plan = make_plan(wl, iso_layers=1)
    toa, Fu, Fd = plan.emission_spectrum(pack([T]), n_passes=passes)
    r = oracle.flux_sweep_iso(atm, T, n_passes=passes)
    assert r["rc"] == 0
    _check_fluxes(Fu, Fd, r)
    _check_toa(toa, r, atm)


def test_isothermal_layer_grid_temperature_step():
    # the radiative-equilibrium step runs unchanged on the isothermal grid: one step from the
    # oracle's fluxes on that grid
    wl = synth.small_scattering(L=10, n=30)
    atm = oracle.Atm.from_workload(wl)
    T = synth.perturbed_profile(wl.atms[0], 3)
    plan = make_plan(wl, iso_layers=1)
    Tg = pack([T])
    Fu, Fd, _ = plan.flux_sweep(Tg, n_passes=5, want_toa=False)
    r = oracle.flux_sweep_iso(atm, T, n_passes=5)
    _check_fluxes(Fu, Fd, r)
    st = oracle.State(atm, T)
    oracle.temp_update(atm, st, Fu.cpu().numpy(), Fd.cpu().numpy())
    state = plan.new_state()
    plan.temp_update(Fu, Fd, Tg, state)
    assert rel_err(Tg.cpu().numpy(), st.T) < 1e-12


@pytest.mark.parametrize("n,L,iso", [(40, 12, 0), (111, 7, 0), (239, 3, 0), (2, 4, 0), (40, 9, 1), (101, 5, 1)])
def test_direct_column_solve_matches_oracle(n, L, iso):
    # the exact solution of the coupled column equations (the limit of the passes of Sect. 2.2.3):
    # warp-parallel adding method vs the oracle's banded elimination
    import paper_1606_05474_b300 as hp
    wl = synth.small_scattering(L=L, n=n)
    atm = oracle.Atm.from_workload(wl)
    T = synth.perturbed_profile(wl.atms[0], 6)
    plan = make_plan(wl, iso_layers=iso)
    Fu, Fd, toa = plan.flux_sweep(pack([T]), n_passes=hp.DIRECT)
    r = oracle.flux_direct(atm, T, iso=bool(iso))
    assert r["rc"] == 0
    _check_fluxes(Fu, Fd, r)
    _check_toa(toa, r, atm)


def test_direct_column_solve_conservative_scattering():
    # pure-scattering bins over the reflecting lower boundary: the regime where the reflectance
    # stays 1 and a naive formulation cancels
    import paper_1606_05474_b300 as hp
    wl = synth.small_scattering(L=6, n=60)
    a = wl.atms[0]
    a.omega0 = np.ones(a.n_bins, np.float32)
    atm = oracle.Atm.from_workload(wl)
    T = synth.perturbed_profile(a, 8)
    plan = make_plan(wl)
    Fu, Fd, toa = plan.flux_sweep(pack([T]), n_passes=hp.DIRECT)
    r = oracle.flux_direct(atm, T)
    _check_fluxes(Fu, Fd, r)
    _check_toa(toa, r, atm)


@pytest.mark.parametrize("n,L,direct", [(40, 12, 0), (111, 7, 0), (40, 9, 1)])
def test_rayleigh_scattering_matches_oracle(n, L, direct):
    # H2 Rayleigh opacity joins every sublayer (Sect. 2.1.4): omega0 and the two-stream constants
    # per sublayer and g, formed in the sweep
    import paper_1606_05474_b300 as hp
    wl = synth.small_scattering(L=L, n=n)
    atm = oracle.Atm.from_workload(wl, rayleigh=True)
    T = synth.perturbed_profile(wl.atms[0], 12)
    plan = make_plan(wl, rayleigh=1)
    if direct:
        Fu, Fd, toa = plan.flux_sweep(pack([T]), n_passes=hp.DIRECT)
        r = oracle.flux_direct(atm, T)
    else:
        Fu, Fd, toa = plan.flux_sweep(pack([T]), n_passes=5)
        r = oracle.flux_sweep(atm, T, n_passes=5)
    assert r["rc"] == 0
    _check_fluxes(Fu, Fd, r)
    _check_toa(toa, r, atm)


def test_rayleigh_scattering_only_conserves_net_flux():
    # no absorption: every sublayer is pure scattering (per sublayer, in emitting bins)
    import paper_1606_05474_b300 as hp
    wl = synth.small_scattering(L=6, n=40)
    wl.tables[0].kappa32[...] = 1e-30
    atm = oracle.Atm.from_workload(wl, rayleigh=True)
    T = synth.perturbed_profile(wl.atms[0], 13)
    plan = make_plan(wl, rayleigh=1)
    Fu, Fd, toa = plan.flux_sweep(pack([T]), n_passes=hp.DIRECT)
    r = oracle.flux_direct(atm, T)
    _check_fluxes(Fu, Fd, r)
    net = (Fu - Fd).cpu().numpy()
    assert np.max(np.abs(net - net[0])) < 1e-5 * np.max(r["Fup"])


@pytest.mark.parametrize("n,L,G", [(40, 12, 7), (150, 5, 3), (200, 3, 9)])
def test_thirty_two_lane_columns_odd_gauss_points(n, L, G):
    # a warp per Gauss point taking the points in two rounds: an odd G leaves the last warp idle
    # in the second round; cold then warm-started passes, and the exact column solve
    wl = synth.small_scattering(L=L, n=n, G=G)
    atm = oracle.Atm.from_workload(wl)
    T1 = synth.perturbed_profile(wl.atms[0], 14)
    T2 = T1 + 4.0 * np.sin(np.arange(n))
    plan = make_plan(wl, col_lanes=32)
    Fu, Fd, toa = plan.flux_sweep(pack([T1]), n_passes=5)
    warm = np.zeros(atm.L * atm.G * (2 * n + 1))
    r1 = oracle.flux_sweep(atm, T1, n_passes=5, warm=warm, warm_valid=False)
    _check_fluxes(Fu, Fd, r1)
    _check_toa(toa, r1, atm)
    Fu2, Fd2, toa2 = plan.flux_sweep(pack([T2]), n_passes=5, warm=True)
    r2 = oracle.flux_sweep(atm, T2, n_passes=5, warm=warm, warm_valid=True)
    _check_fluxes(Fu2, Fd2, r2)
    _check_toa(toa2, r2, atm)
    Fu3, Fd3, toa3 = plan.flux_sweep(pack([T1]), n_passes=hp.DIRECT)
    r3 = oracle.flux_direct(atm, T1)
    _check_fluxes(Fu3, Fd3, r3)


@pytest.mark.parametrize("n,L,G", [(36, 9, 20), (40, 12, 7), (111, 7, 20), (119, 4, 3)])
def test_sixteen_lane_columns_match_oracle(n, L, G):
    # two Gauss points per warp (16 lanes per column; odd G leaves half a warp idle), cold
    # then warm-started passes
    wl = synth.small_scattering(L=L, n=n, G=G)
    atm = oracle.Atm.from_workload(wl)
    T1 = synth.perturbed_profile(wl.atms[0], 8)
    T2 = T1 + 5.0 * np.cos(np.arange(n))
    plan = make_plan(wl, col_lanes=16)
    Fu, Fd, toa = plan.flux_sweep(pack([T1]), n_passes=5)
    warm = np.zeros(atm.L * atm.G * (2 * n + 1))
    r1 = oracle.flux_sweep(atm, T1, n_passes=5, warm=warm, warm_valid=False)
    _check_fluxes(Fu, Fd, r1)
    _check_toa(toa, r1, atm)
    Fu2, Fd2, toa2 = plan.flux_sweep(pack([T2]), n_passes=5, warm=True)
    r2 = oracle.flux_sweep(atm, T2, n_passes=5, warm=warm, warm_valid=True)
    _check_fluxes(Fu2, Fd2, r2)
    _check_toa(toa2, r2, atm)


def test_sixteen_lane_columns_full_size():
    wl = synth.config2()
    T = synth.perturbed_profile(wl.atms[0], 6)
    Fu, Fd, toa = make_plan(wl, col_lanes=16).flux_sweep(pack([T]))
    r = _oracle_sweep(wl, 0, T)
    _check_fluxes(Fu, Fd, r)
    _check_toa(toa, r, oracle.Atm.from_workload(wl))


def test_sixteen_lane_columns_reject_what_they_do_not_cover():
    for n in (23, 120):
        with pytest.raises(hp.HeliosError, match="16-lane"):
            make_plan(synth.small_scattering(L=3, n=n), col_lanes=16)
    with pytest.raises(hp.HeliosError):
        make_plan(synth.small_scattering(L=3, n=40), col_lanes=8)


@pytest.mark.parametrize("n,lanes", [(40, 16), (40, 32), (111, 0), (119, 0)])
def test_exact_solve_leaves_the_warm_start_of_the_passes(n, lanes):
    # the exact solve stores its upward deviations in the iterated sweep's layout (16 or 32
    # lanes per column): passes warm-started from it at the same temperatures stay at the limit,
    # while passes from a misplaced start would be visibly short of it
    wl = synth.small_scattering(L=6, n=n)
    atm = oracle.Atm.from_workload(wl)
    T = synth.perturbed_profile(wl.atms[0], 9)
    plan = make_plan(wl, col_lanes=lanes)
    plan.flux_sweep(pack([T]), n_passes=hp.DIRECT)
    Fu, Fd, toa = plan.flux_sweep(pack([T]), n_passes=5, warm=True)
    d = oracle.flux_direct(atm, T)
    _check_fluxes(Fu, Fd, d)
    _check_toa(toa, d, atm)
    cold = oracle.flux_sweep(atm, T, n_passes=5)
    assert np.max(np.abs(cold["toa"] / d["toa"] - 1)) > 1e-4
