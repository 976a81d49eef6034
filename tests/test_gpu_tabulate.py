"""GPU parity of the tabulated Planck and transmission functions (Sect. 2.6; params.tabulate)
with the oracle's tabulated path: fluxes and spectrum within the sweep tolerance (1e-5), cold and
warm, at 16 and 32 lanes per column and at full size; the RE solve converges to the oracle's
tabulated equilibrium within 0.1 K; and the tables are in use (the result differs from the
functions themselves by their interpolation error).  Combinations without a tabulated form are
rejected."""
import numpy as np
import pytest

import oracle
import synth
import paper_1606_05474_b300 as hp
from helpers import make_plan, pack
from test_gpu_parity import _check_fluxes, _check_toa

pytestmark = pytest.mark.gpu

TAB = oracle.params(tabulate=1)


@pytest.mark.parametrize("n,L,lanes", [(40, 12, 0), (111, 7, 0), (200, 5, 0), (40, 9, 32), (2, 4, 0)])
def test_tabulated_sweep_matches_the_tabulated_oracle(n, L, lanes):
    wl = synth.small_scattering(L=L, n=n)
    atm = oracle.Atm.from_workload(wl)
    T1 = synth.perturbed_profile(wl.atms[0], 5)
    T2 = T1 + 7.0 * np.sin(np.arange(n))
    plan = make_plan(wl, tabulate=1, col_lanes=lanes)
    warm = np.zeros(atm.L * atm.G * (2 * n + 1))
    Fu, Fd, toa = plan.flux_sweep(pack([T1]), n_passes=5)
    r1 = oracle.flux_sweep(atm, T1, n_passes=5, p=TAB, warm=warm, warm_valid=False)
    _check_fluxes(Fu, Fd, r1)
    _check_toa(toa, r1, atm)
    Fu2, Fd2, toa2 = plan.flux_sweep(pack([T2]), n_passes=5, warm=True)
    r2 = oracle.flux_sweep(atm, T2, n_passes=5, p=TAB, warm=warm, warm_valid=True)
    _check_fluxes(Fu2, Fd2, r2)
    _check_toa(toa2, r2, atm)


def test_tabulated_full_size_and_in_use():
    wl = synth.config2()
    atm = oracle.Atm.from_workload(wl)
    T = synth.perturbed_profile(wl.atms[0], 6)
    Fu, Fd, toa = make_plan(wl, tabulate=1).flux_sweep(pack([T]))
    r = oracle.flux_sweep(atm, T, p=TAB)
    _check_fluxes(Fu, Fd, r)
    _check_toa(toa, r, atm)
    ex = oracle.flux_sweep(atm, T)
    assert np.max(np.abs(Fu.cpu().numpy() / ex["Fup"] - 1)) > 1e-6


def test_tabulated_re_solve_reaches_the_tabulated_equilibrium():
    wl = synth.small_scattering(L=30, n=40)
    atm = oracle.Atm.from_workload(wl)
    st = oracle.State(atm, wl.atms[0].T_init)
    rc, _, _ = oracle.solve_re(atm, st, oracle.params(tabulate=1, tol=1e-10, max_iter=200000))
    assert rc == oracle.CONVERGED
    plan = make_plan(wl, tabulate=1, max_iter=100000)
    T = pack([wl.atms[0].T_init])
    iters, status = plan.solve_re(T)
    assert status.item() == 1
    assert np.abs(T.cpu().numpy() - st.T).max() < 0.1


def test_tabulate_rejects_what_has_no_tabulated_form():
    wl = synth.small_scattering(L=3, n=20)
    for kw in ({"iso_layers": 1}, {"direct": 1}, {"rayleigh": 1}, {"tabulate": 2}):
        with pytest.raises(hp.HeliosError):
            make_plan(wl, **({"tabulate": 1} | kw))
    plan = make_plan(wl, tabulate=1)
    with pytest.raises(hp.HeliosError):
        plan.flux_sweep(pack([synth.perturbed_profile(wl.atms[0], 1)]), n_passes=hp.DIRECT)


def test_temperatures_above_the_planck_table_stop_the_atmosphere():
    # as in the oracle: with tables, an atmosphere whose profile is above the Planck table's 6000 K
    # stops as OUT_OF_RANGE; the other atmospheres of the batch step on
    import paper_1606_05474_b300 as hp
    wls = [synth.small_scattering(L=6, n=20, seed_offset=k) for k in (1, 2)]
    atms = [w.atms[0] for w in wls]
    atms[1].table_id = 1
    wl = synth.Workload(name="two", atms=atms, tables=[w.tables[0] for w in wls])
    plan = make_plan(wl, tabulate=1)
    T = pack([np.full(20, 6100.0), np.full(20, 5000.0)])
    state = plan.new_state()
    plan.re_step(T, state, warm=False)
    st = state["status"].cpu().numpy()
    assert st[0] == hp.ATM_OUT_OF_RANGE and st[1] == hp.ATM_ACTIVE
