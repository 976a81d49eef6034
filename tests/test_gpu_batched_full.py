"""Parity at the batched workload's full size, in the launch configuration the bench times:
4096 ragged atmospheres (layers U{50..200}, bins U{300..3000} x 20 g, scattering, 64-table
pool) in one plan with autotuned bins per item and launch mode, one cold flux evaluation of
the whole batch and one warm RE step, checked against the FP64 oracle on sampled atmospheres
(the shortest, the longest, and a few in between), one by one.  Tolerances as the small
parity cases: 1e-5 relative on bolometric fluxes, net flux and the emergent spectrum."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_full_batched_workload_matches_oracle_on_sampled_atmospheres(tmp_path):
    import torch
    import paper_1606_05474_b300 as hp
    from helpers import ctx
    wl = synth.config3(A=4096)
    kap = [torch.from_numpy(t.kappa32).cuda() for t in wl.tables]
    tuned = hp.autotune(ctx(), wl.atms, wl.tables, kap, cache_path=str(tmp_path / "tune.json"))
    plan = hp.Plan(ctx(), wl.atms, wl.tables, kap, tuned)
    T0 = [synth.perturbed_profile(a, i) for i, a in enumerate(wl.atms)]
    T = torch.from_numpy(np.concatenate(T0)).cuda()
    Fu, Fd, toa = plan.flux_sweep(T, n_passes=5, warm=False)
    Fus, Fds = plan.split_interfaces(Fu.cpu().numpy()), plan.split_interfaces(Fd.cpu().numpy())
    toas = plan.split_bins(toa.cpu().numpy().astype(np.float64))
    cost = np.array([a.n_layers * a.n_bins for a in wl.atms])
    sample = sorted({int(np.argmin(cost)), int(np.argmax(cost)), 7, 1234, 2047, 4095})
    for a in sample:
        atm = oracle.Atm(wl.atms[a], wl.tables[wl.atms[a].table_id])
        r = oracle.flux_sweep(atm, T0[a], n_passes=5)
        assert r["rc"] == 0
        assert np.max(np.abs(Fus[a] / r["Fup"] - 1)) < 1e-5, a
        assert np.max(np.abs(Fds[a] / r["Fdn"] - 1)) < 1e-5, a
        scale = np.maximum(r["Fup"], r["Fdn"])
        assert np.max(np.abs((Fus[a] - Fds[a]) - (r["Fup"] - r["Fdn"])) / scale) < 1e-5, a
        inc, _ = oracle.boundary_spectra(atm)
        assert np.max(np.abs(toas[a] - r["toa"]) / np.maximum(np.abs(r["toa"]), inc)) < 1e-5, a
    # one temperature step of the whole batch against the oracle's step on the sampled ones
    state = plan.new_state()
    plan.temp_update(Fu, Fd, T, state)
    Ts = plan.split_layers(T.cpu().numpy())
    for a in sample:
        atm = oracle.Atm(wl.atms[a], wl.tables[wl.atms[a].table_id])
        st = oracle.State(atm, T0[a])
        oracle.temp_update(atm, st, Fus[a], Fds[a])
        assert np.max(np.abs(Ts[a] / st.T - 1)) < 1e-12, a
