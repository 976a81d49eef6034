"""GPU radiative-equilibrium iteration vs the FP64 oracle: converged profiles within 0.1 K,
the converged net flux equal to sigma T_int^4, the grey two-band profile, and ragged batches."""
import numpy as np
import pytest

import oracle
import synth
from helpers import make_plan, pack

pytestmark = pytest.mark.gpu


def _oracle_solve(wl, a, tol=1e-10):
    atm = oracle.Atm.from_workload(wl, a)
    st = oracle.State(atm, wl.atms[a].T_init)
    rc, it, m = oracle.solve_re(atm, st, oracle.params(tol=tol, max_iter=200000))
    assert rc == oracle.CONVERGED
    return st.T, it


@pytest.mark.parametrize("which", ["config1", "scat"])
def test_converged_profile_within_0p1K(which):
    wl = synth.config1() if which == "config1" else synth.small_scattering(L=30, n=40)
    Tref, it_ref = _oracle_solve(wl, 0)
    plan = make_plan(wl, max_iter=100000)
    T = pack([wl.atms[0].T_init])
    iters, status = plan.solve_re(T)
    assert status.item() == 1
    dT = np.abs(T.cpu().numpy() - Tref)
    assert dT.max() < 0.1, (dT.max(), np.argmax(dT))


def test_converged_net_flux_is_internal_flux():
    # at convergence every layer has |dF_i| < tol sigma T_i^4, so the net flux departs from its
    # BOA value sigma T_int^4 by at most sum_i tol sigma T_i^4; the TOA emits what enters
    wl = synth.config1()
    tol = 1e-7
    plan = make_plan(wl, max_iter=100000, tol=tol)
    T = pack([wl.atms[0].T_init])
    iters, status = plan.solve_re(T)
    assert status.item() == 1
    Fu, Fd, _ = plan.flux_sweep(T, warm=True)
    net = (Fu - Fd).cpu().numpy()
    Tn = T.cpu().numpy()
    bound = tol * oracle.SIGMA_SB * np.sum(Tn ** 4)
    assert np.abs(net - oracle.SIGMA_SB * 100.0 ** 4).max() <= bound
    assert abs(net[0] - oracle.SIGMA_SB * 100.0 ** 4) < 1e-6 * Fu[0].item()
    assert abs(Fu[-1].item() - oracle.SIGMA_SB * (1200.0 ** 4 + 100.0 ** 4)) <= bound


def test_grey_two_band_profile():
    wl = synth.grey_two_band(n=50)
    plan = make_plan(wl, max_iter=200000, tol=1e-7)   # the float32 noise floor of the metric is near 1e-8
    T = pack([wl.atms[0].T_init])
    iters, status = plan.solve_re(T)
    assert status.item() == 1
    atm = oracle.Atm.from_workload(wl)
    _, P, _, Pl = oracle.grid(atm)
    gam, kth, D = wl.meta["gamma"], wl.meta["kappa_th"], 2.0
    tau = kth * (Pl - P[-1]) / wl.atms[0].grav
    T4 = (D / 4) * (100.0 ** 4 * (1 + D * tau) + 1200.0 ** 4 * (1 + 1 / gam + (gam - 1 / gam) * np.exp(-D * gam * tau)))
    assert np.abs(T.cpu().numpy() / T4 ** 0.25 - 1).max() < 1e-3


def test_batched_ragged_equals_one_by_one():
    wl = synth.config3(A=5, n_tables=2, atm_ids=[3, 17, 42, 64, 100])
    for a in wl.atms:                      # keep the test short: fewer bins, same raggedness
        L = max(3, a.n_bins // 100)
        a.nu_edges = a.nu_edges[:L + 1]; a.omega0 = a.omega0[:L]; a.g0 = a.g0[:L]
    plan = make_plan(wl, bins_per_item=4)
    Ts = [synth.perturbed_profile(a, i) for i, a in enumerate(wl.atms)]
    Fu, Fd, toa = plan.flux_sweep(pack(Ts), n_passes=5)
    Fus = plan.split_interfaces(Fu.cpu().numpy())
    for i, a in enumerate(wl.atms):
        one = synth.Workload(name="one", atms=[a], tables=wl.tables, n_scat=4)
        p1 = make_plan(one, bins_per_item=4)
        fu1, fd1, _ = p1.flux_sweep(pack([Ts[i]]), n_passes=5)
        assert np.array_equal(fu1.cpu().numpy(), Fus[i])
        r = oracle.flux_sweep(oracle.Atm(a, wl.tables[a.table_id]), Ts[i], n_passes=5)
        assert np.max(np.abs(Fus[i] / r["Fup"] - 1)) < 1e-5


def test_invalid_batches_are_rejected():
    from paper_1606_05474_b300 import HeliosError
    wl = synth.small_scattering(L=4, n=10)
    wl.atms[0].n_layers = 1
    with pytest.raises(HeliosError):
        make_plan(wl)
    wl = synth.small_scattering(L=4, n=300)            # beyond the supported 239 layers
    with pytest.raises(HeliosError):
        make_plan(wl)


def test_full_size_converged_profile_matches_stored_oracle_profile():
    # 100 layers x 3000 bins x 20 g with scattering, isothermal start; the stored profile was
    # converged by the FP64 oracle to tol 1e-9 (tests/golden/make_golden.py)
    import os
    golden = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "config2_converged_T.txt"))
    wl = synth.config2()
    plan = make_plan(wl, max_iter=100000)
    T = pack([wl.atms[0].T_init])
    iters, status = plan.solve_re(T)
    assert status.item() == 1
    dT = np.abs(T.cpu().numpy() - golden)
    assert dT.max() < 0.1, (dT.max(), int(np.argmax(dT)))
