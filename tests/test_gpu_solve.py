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
    # 0.5 % (the discrete scheme differs from the continuous solution by the layer
    # discretisation; the top layers, of tiny optical depth, are also where eq. (29) constrains T
    # least); most layers agree to 0.1 %
    err = np.abs(T.cpu().numpy() / T4 ** 0.25 - 1)
    assert err.max() < 5e-3 and np.median(err) < 1e-3, (err.max(), np.median(err))


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


def _small_ragged(ids, max_bins=40):
    # the batched workload's ragged atmospheres, re-gridded to fewer bins over the same 0.3-200 um range
    wl = synth.config3(A=len(ids), n_tables=2, atm_ids=ids)
    for i, a in enumerate(wl.atms):
        L = min(a.n_bins, max_bins - 3 * i)
        a.nu_edges = synth.nu_edges(L); a.omega0 = synth.rayleigh_like_omega0(a.nu_edges); a.g0 = a.g0[:L]
    return wl


def test_persistent_and_per_item_launches_agree_bitwise():
    # ragged layer counts give several lane-chunk groups, which run concurrently on their own streams
    wl = _small_ragged([1, 5, 9, 33, 70, 111])
    assert len({(2 * a.n_layers + 1 + 31) // 32 | 1 for a in wl.atms}) >= 2
    Ts = pack([synth.perturbed_profile(a, i) for i, a in enumerate(wl.atms)])
    outs = []
    for pers in (0, 1):
        p = make_plan(wl, bins_per_item=3, persistent=pers)
        outs.append([x.clone() for x in p.flux_sweep(Ts, n_passes=5)])
    for x, y in zip(*outs):
        assert bool((x == y).all())


def test_batched_solve_matches_oracle_per_atmosphere():
    wl = _small_ragged([2, 40, 77], max_bins=24)
    plan = make_plan(wl, max_iter=100000)
    T = pack([a.T_init for a in wl.atms])
    iters, status = plan.solve_re(T)
    assert (status.cpu().numpy() == 1).all()
    got = plan.split_layers(T.cpu().numpy())
    for a, Tg in zip(wl.atms, got):
        atm = oracle.Atm(a, wl.tables[a.table_id])
        st = oracle.State(atm, a.T_init)
        rc, it, m = oracle.solve_re(atm, st, oracle.params(tol=1e-10, max_iter=200000))
        assert rc == oracle.CONVERGED
        assert np.abs(Tg - st.T).max() < 0.1


def test_autotune_picks_a_candidate_and_caches_it(tmp_path):
    import paper_1606_05474_b300 as hp
    from helpers import ctx
    import torch
    wl = _small_ragged([3, 8, 13, 21], max_bins=64)
    kap = [torch.from_numpy(t.kappa32).cuda() for t in wl.tables]
    cache = str(tmp_path / "tune.json")
    p = hp.autotune(ctx(), wl.atms, wl.tables, kap, cache_path=cache)
    assert p.bins_per_item in (1, 2, 4, 8, 16, 32) and p.persistent in (0, 1)
    import json
    d = json.load(open(cache))
    assert len(d) == 1 and list(d.values())[0]["bins_per_item"] == p.bins_per_item
    p2 = hp.autotune(ctx(), wl.atms, wl.tables, kap, cache_path=cache)       # cache hit
    assert (p2.bins_per_item, p2.persistent) == (p.bins_per_item, p.persistent)


def test_device_while_loop_and_host_loop_agree_bitwise():
    # the conditional-WHILE graph runs the same kernels in the same order as the host-checked
    # chunks, so temperatures, iteration counts and statuses agree bit for bit; a small chunk
    # makes both loops go round many times, and a low cap retires one atmosphere at max_iter
    wl = _small_ragged([3, 20, 41], max_bins=16)
    outs = []
    for dl in (1, 0):
        p = make_plan(wl, device_loop=dl, check_every=3, max_iter=400)
        T = pack([a.T_init for a in wl.atms])
        iters, status = p.solve_re(T)
        outs.append((T.clone(), iters.clone(), status.clone()))
    for x, y in zip(*outs):
        assert bool((x == y).all())
    st = outs[0][2].cpu().numpy()
    assert set(st.tolist()) <= {1, 2}
    # a second solve on the same plan relaunches the cached graph with a fresh budget
    p = make_plan(wl, device_loop=1, check_every=3, max_iter=400)
    for _ in range(2):
        T = pack([a.T_init for a in wl.atms])
        iters, status = p.solve_re(T)
        assert bool((T == outs[0][0]).all()) and bool((iters == outs[0][1]).all())


def test_direct_column_solve_reaches_the_same_equilibrium():
    # every temperature step with the exact column solution instead of 1 + 4 passes: the same
    # fixed point (at convergence the warm-started passes reach the exact solution too)
    wl = synth.small_scattering(L=30, n=40)
    Tref, _ = _oracle_solve(wl, 0)
    plan = make_plan(wl, max_iter=100000, direct=1)
    assert plan.info.passes == -1
    T = pack([wl.atms[0].T_init])
    iters, status = plan.solve_re(T)
    assert status.item() == 1
    assert np.abs(T.cpu().numpy() - Tref).max() < 0.1


def test_re_step_equals_sweep_plus_temperature_update_bitwise():
    import torch
    wl = _small_ragged([3, 20, 41], max_bins=16)
    T0 = [synth.perturbed_profile(a, i) for i, a in enumerate(wl.atms)]
    pa, pb = make_plan(wl), make_plan(wl)
    Ta, Tb = pack(T0), pack(T0)
    sa, sb = pa.new_state(), pb.new_state()
    Fub = torch.empty(pb.info.interfaces, dtype=torch.float64, device="cuda"); Fdb = torch.empty_like(Fub)
    for k in range(4):
        Fua, Fda, _ = pa.flux_sweep(Ta, warm=k > 0, want_toa=False)
        pa.temp_update(Fua, Fda, Ta, sa)
        pb.re_step(Tb, sb, warm=k > 0, out=(Fub, Fdb))
        assert bool((Fua == Fub).all()) and bool((Fda == Fdb).all())
        assert bool((Ta == Tb).all())
        for key in ("mult", "hist", "nhist", "status", "iters", "metric"):
            assert bool((sa[key] == sb[key]).all()), key


def test_re_step_with_host_temperatures_equals_re_step_bitwise():
    # helios_re_step_host: host temperatures in, new temperatures and statuses out, the same step
    import torch
    wl = _small_ragged([3, 20, 41], max_bins=16)
    T0 = [synth.perturbed_profile(a, i) for i, a in enumerate(wl.atms)]
    pa, pb = make_plan(wl), make_plan(wl)
    Ta = pack(T0)
    Th = torch.from_numpy(np.concatenate(T0)).pin_memory()
    Td = torch.empty_like(Ta)
    Sh = torch.zeros(pb.A, dtype=torch.int32).pin_memory()
    sa, sb = pa.new_state(), pb.new_state()
    for k in range(4):
        pa.re_step(Ta, sa, warm=k > 0)
        pb.re_step_host(Th, Td, sb, Sh, warm=k > 0)
        torch.cuda.synchronize()
        assert np.array_equal(Th.numpy(), Ta.cpu().numpy())
        assert np.array_equal(Sh.numpy(), sa["status"].cpu().numpy())


def test_solve_equals_a_loop_of_re_steps():
    # helios_solve_re (graph loop; the next step's point quantities prepared by the post kernel)
    # and a host loop of helios_re_step reach the same temperatures in the same number of steps
    wl = synth.small_scattering(L=12, n=30)
    p1 = make_plan(wl, max_iter=20000)
    T1 = pack([wl.atms[0].T_init])
    iters, status = p1.solve_re(T1)
    assert status.item() == 1
    p2 = make_plan(wl)
    T2 = pack([wl.atms[0].T_init])
    s2 = p2.new_state()
    for k in range(20000):
        p2.re_step(T2, s2, warm=k > 0)
        if s2["status"].item() == 1:          # stop at the first converged step, as the solve does
            break
    assert s2["status"].item() == 1
    assert int(s2["iters"].item()) == int(iters.item())
    assert bool((T1 == T2).all())


def test_rayleigh_atmosphere_converges_to_the_oracle_profile():
    wl = synth.small_scattering(L=16, n=30)
    atm = oracle.Atm.from_workload(wl, rayleigh=True)
    st = oracle.State(atm, wl.atms[0].T_init)
    rc, it, m = oracle.solve_re(atm, st, oracle.params(tol=1e-10, max_iter=200000))
    assert rc == oracle.CONVERGED
    plan = make_plan(wl, max_iter=100000, rayleigh=1)
    T = pack([wl.atms[0].T_init])
    iters, status = plan.solve_re(T)
    assert status.item() == 1
    assert np.abs(T.cpu().numpy() - st.T).max() < 0.1


def test_measured_peaks_are_plausible():
    # FP32 FMA and MUFU ex2 rates of the device: B300 has 148 SMs of 128 FP32 lanes and 16 MUFU
    # lanes at up to ~2 GHz (nominal 77 TFLOP/s and 4.8 T op/s)
    import paper_1606_05474_b300 as hp
    from helpers import ctx
    f, u = hp.measure_peaks(ctx())
    assert 20.0 < f < 100.0, f
    assert 1.0 < u < 12.0, u


def test_dependent_launches_give_the_same_step_bitwise():
    # the kernels of an evaluation launch as programmatic dependents of one another unless the
    # sweep-timing events are on; both ways the step must be the same, bit for bit
    import torch
    wl = synth.small_scattering(L=24, n=60)
    T0 = synth.perturbed_profile(wl.atms[0], 4)
    res = []
    for timing in (0, 4):
        plan = make_plan(wl)
        plan.set_timing(timing)
        T = pack([T0])
        st = plan.new_state()
        Fu = torch.empty(plan.info.interfaces, dtype=torch.float64, device="cuda"); Fd = torch.empty_like(Fu)
        for k in range(3):
            plan.re_step(T, st, warm=k > 0, out=(Fu, Fd))
        Fs, Gs, toa = plan.flux_sweep(T, warm=True)
        torch.cuda.synchronize()
        res.append([x.cpu().numpy().copy() for x in (T, Fu, Fd, Fs, Gs, toa, st["mult"], st["metric"])])
    for a, b in zip(*res):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("where", ["device", "host"])
def test_checkpoint_resume_continues_bit_for_bit(where):
    # an iteration checkpointed after 7 steps (the caller's arrays plus the plan's exported
    # state) and resumed in a fresh plan of the same inputs continues exactly as the uninterrupted
    # iteration: temperatures, multipliers, sign histories, statuses and step counts bit for bit
    import torch
    import paper_1606_05474_b300 as hp
    wls = [synth.small_scattering(L=9, n=40), synth.small_scattering(L=7, n=130, seed_offset=8)]
    wl = synth.Workload(name="ragged", atms=[w.atms[0] for w in wls], tables=[wls[0].tables[0], wls[1].tables[0]],
                        n_scat=4)
    wl.atms[1].table_id = 1
    T0 = [synth.perturbed_profile(a, 17 + i) for i, a in enumerate(wl.atms)]
    plan = make_plan(wl)
    T = pack(T0)
    st = plan.new_state()
    for k in range(7):
        plan.re_step(T, st, warm=k > 0)
    out = None if where == "device" else torch.empty(0)
    if out is not None:
        n = plan.export_state().numel()
        out = torch.empty(n, dtype=torch.uint8).pin_memory()
    ck = plan.export_state(out=out)
    torch.cuda.synchronize()
    ck_T, ck_st = T.clone(), {k: v.clone() for k, v in st.items()}
    for _ in range(5):
        plan.re_step(T, st, warm=True)
    torch.cuda.synchronize()
    plan2 = make_plan(wl)
    with pytest.raises(hp.HeliosError):
        plan2.export_state()                    # nothing to checkpoint before a first evaluation
    plan2.import_state(ck)
    for _ in range(5):
        plan2.re_step(ck_T, ck_st, warm=True)
    torch.cuda.synchronize()
    assert torch.equal(ck_T, T)
    for k in ("mult", "hist", "nhist", "status", "iters", "metric"):
        assert torch.equal(ck_st[k], st[k]), k
    # a checkpoint of a plan of another shape is refused
    other = make_plan(synth.small_scattering(L=9, n=41))
    with pytest.raises(hp.HeliosError):
        other.import_state(ck)
