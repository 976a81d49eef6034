"""The allocation-free flux evaluation, helios_flux_sweep_noalloc, through the C ABI.

Some callers cannot allocate device memory: a framework that owns the whole memory pool of
the device, or code running where cudaMalloc is not allowed.  This entry point serves them:
its working memory is a fixed array inside the library, so the call allocates nothing; the
caller passes the inputs and the output buffers.  The tests check it against the plan-based
helios_flux_sweep (cold start) on the same atmosphere, on two calls in a row with different
temperatures, because every call reuses the same array and must not see what the previous
call left there; against the FP64 oracle; that a call after the first leaves the device's free
memory unchanged; that its stated size limits are reachable together; and that it refuses a
stream that is capturing a graph.  This file is collected last so that a run stopping at the first failure has
run every other test before it.
"""
import numpy as np
import pytest

import synth
from helpers import make_plan, pack

pytestmark = pytest.mark.gpu

TOL = 1e-5      # the flux tolerance of the parity tests


def _out(plan):
    import torch
    n1 = int(plan.info.interfaces)
    return (torch.empty(n1, dtype=torch.float64, device="cuda"), torch.empty(n1, dtype=torch.float64, device="cuda"),
            torch.empty(int(plan.info.bins), dtype=torch.float32, device="cuda"))


def test_noalloc_matches_plan_sweep_on_two_calls_in_a_row():
    import paper_1606_05474_b300 as hp
    import torch
    wl = synth.config2()
    atm, tab = wl.atms[0], wl.tables[0]
    plan = make_plan(wl)
    kappa = plan.kappa[0]
    profiles = [synth.perturbed_profile(atm, 21), synth.perturbed_profile(atm, 22, amp=500.0)]
    for T in profiles:
        Tg = pack([T])
        ref = [x.clone() for x in plan.flux_sweep(Tg, warm=False)]
        got = hp.flux_sweep_noalloc(atm, tab, kappa, Tg, _out(plan))
        torch.cuda.synchronize()
        for r, g in zip(ref, got):
            r = r.cpu().numpy().astype(np.float64); g = g.cpu().numpy().astype(np.float64)
            assert np.max(np.abs(g - r) / np.maximum(np.abs(r), 1e-30)) < TOL


def test_noalloc_rejects_atmospheres_beyond_its_fixed_size():
    import paper_1606_05474_b300 as hp
    wl = synth.small_scattering(L=4, n=300)
    plan_free = wl.atms[0]
    import torch
    kappa = torch.from_numpy(wl.tables[0].kappa32).cuda()
    T = torch.full((300,), 1000.0, dtype=torch.float64, device="cuda")
    out = (torch.empty(301, dtype=torch.float64, device="cuda"), torch.empty(301, dtype=torch.float64, device="cuda"),
           None)
    with pytest.raises(hp.HeliosError) as e:
        hp.flux_sweep_noalloc(plan_free, wl.tables[0], kappa, T, out)
    assert e.value.code == -1 and b"n_layers" in hp._lib.load().helios_last_error()


def test_no_alloc_rejects_the_direct_solve():
    import paper_1606_05474_b300 as hp
    from paper_1606_05474_b300 import HeliosError
    import synth
    import torch
    wl = synth.small_scattering(L=4, n=10)
    kap = torch.from_numpy(wl.tables[0].kappa32).cuda()
    T = torch.from_numpy(np.asarray(wl.atms[0].T_init, np.float64)).cuda()
    Fu = torch.empty(11, dtype=torch.float64, device="cuda"); Fd = torch.empty_like(Fu)
    with pytest.raises(HeliosError):
        hp.flux_sweep_noalloc(wl.atms[0], wl.tables[0], kap, T, (Fu, Fd, None), n_passes=hp.DIRECT)


def test_noalloc_matches_the_oracle_and_allocates_nothing():
    # against the FP64 oracle directly (cold start, 1 + 4 passes), and the property the entry point
    # exists for: after a first call on the device, further calls leave the device's free memory
    # unchanged
    import paper_1606_05474_b300 as hp
    import oracle
    import torch
    wl = synth.small_scattering(L=24, n=111)
    atm, tab = wl.atms[0], wl.tables[0]
    kappa = torch.from_numpy(tab.kappa32).cuda()
    n = atm.n_layers
    out = (torch.empty(n + 1, dtype=torch.float64, device="cuda"), torch.empty(n + 1, dtype=torch.float64, device="cuda"),
           torch.empty(atm.n_bins, dtype=torch.float32, device="cuda"))
    T = synth.perturbed_profile(atm, 31)
    Tg = pack([T])
    hp.flux_sweep_noalloc(atm, tab, kappa, Tg, out)          # first call on this device: set-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    Fu, Fd, toa = hp.flux_sweep_noalloc(atm, tab, kappa, Tg, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    r = oracle.flux_sweep(oracle.Atm.from_workload(wl), T, n_passes=5)
    for g, o in ((Fu, r["Fup"]), (Fd, r["Fdn"])):
        assert np.max(np.abs(g.cpu().numpy() / o - 1)) < TOL
    inc, _ = oracle.boundary_spectra(oracle.Atm.from_workload(wl))
    scale = np.maximum(np.abs(r["toa"]), inc)
    assert np.max(np.abs(toa.cpu().numpy() - r["toa"]) / scale) < TOL


def test_noalloc_takes_its_stated_limits_together():
    # 239 layers x 8192 bins x 20 Gauss points: the largest atmosphere the header states, accepted
    # (no warm start is kept, so the limits are reachable together)
    import paper_1606_05474_b300 as hp
    import torch
    wl = synth.small_scattering(L=8192, n=239, G=20)
    atm, tab = wl.atms[0], wl.tables[0]
    kappa = torch.from_numpy(tab.kappa32).cuda()
    out = (torch.empty(240, dtype=torch.float64, device="cuda"), torch.empty(240, dtype=torch.float64, device="cuda"),
           None)
    Fu, Fd, _ = hp.flux_sweep_noalloc(atm, tab, kappa, pack([atm.T_init]), out)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(Fu).all()) and bool(torch.isfinite(Fd).all())


@pytest.mark.filterwarnings("ignore:The CUDA Graph is empty")
def test_noalloc_refuses_a_capturing_stream():
    # the refused call records nothing, so the captured graph is empty by design
    import paper_1606_05474_b300 as hp
    import torch
    wl = synth.small_scattering(L=4, n=10)
    atm, tab = wl.atms[0], wl.tables[0]
    kappa = torch.from_numpy(tab.kappa32).cuda()
    T = pack([atm.T_init])
    out = (torch.empty(11, dtype=torch.float64, device="cuda"), torch.empty(11, dtype=torch.float64, device="cuda"), None)
    hp.flux_sweep_noalloc(atm, tab, kappa, T, out)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        g.capture_begin()
        try:
            with pytest.raises(hp.HeliosError):
                hp.flux_sweep_noalloc(atm, tab, kappa, T, out, stream=s)
        finally:
            g.capture_end()
    assert b"capturing" in hp._lib.load().helios_last_error()
