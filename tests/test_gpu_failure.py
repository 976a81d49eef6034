"""Failure handling of the RE iteration (host-visible, no GPU fault): a non-finite atmosphere is
frozen with status NONFINITE while the others in the batch end exactly as they would alone,
and degenerate batches are rejected before any GPU work.  A NaN temperature is safe on the
device by construction: the table coordinate of a NaN is index 0 with weight 0 (every
table access stays in bounds) and the NaN propagates only through the Planck values, the
fluxes and the metric of eq. (29)."""
import numpy as np
import pytest

import synth
from helpers import make_plan, pack
from test_gpu_solve import _small_ragged

pytestmark = pytest.mark.gpu


def test_nonfinite_atmosphere_is_frozen_and_the_rest_are_unaffected():
    wl = _small_ragged([3, 20, 41], max_bins=16)
    starts = [np.array(a.T_init, dtype=np.float64) for a in wl.atms]
    starts[1][5] = np.nan
    plan = make_plan(wl, max_iter=100000)
    T = pack(starts)
    iters, status = plan.solve_re(T)
    st = status.cpu().numpy()
    assert st[1] == 3 and st[0] != 3 and st[2] != 3
    assert int(iters[1].item()) == 1                      # caught at the first metric
    Ts = plan.split_layers(T.cpu().numpy())
    assert np.isnan(Ts[1][5]) and np.array_equal(np.isnan(Ts[1]), np.isnan(starts[1]))
    # the other atmospheres end exactly as they do alone (converged or at the iteration cap)
    for i in (0, 2):
        one = synth.Workload(name="one", atms=[wl.atms[i]], tables=wl.tables, n_scat=4)
        p1 = make_plan(one, max_iter=100000)
        T1 = pack([starts[i]])
        it1, st1 = p1.solve_re(T1)
        assert st1.item() == st[i] and it1.item() == iters[i].item()
        assert np.array_equal(T1.cpu().numpy(), Ts[i])


def test_degenerate_batches_are_rejected():
    from paper_1606_05474_b300 import HeliosError
    wl = synth.small_scattering(L=4, n=10)
    with pytest.raises(HeliosError):                      # no atmospheres
        make_plan(synth.Workload(name="empty", atms=[], tables=wl.tables, n_scat=4))
    wl0 = synth.small_scattering(L=4, n=10)
    a = wl0.atms[0]
    a.nu_edges = a.nu_edges[:1]; a.omega0 = a.omega0[:0]; a.g0 = a.g0[:0]
    with pytest.raises(HeliosError):                      # no bins
        make_plan(wl0)
    wl1 = synth.small_scattering(L=4, n=10)
    wl1.atms[0].P_top_bar = wl1.atms[0].P_bot_bar         # empty pressure range
    with pytest.raises(HeliosError):
        make_plan(wl1)
    with pytest.raises(HeliosError):                      # invalid parameters
        make_plan(wl, n_scat=-1)
    with pytest.raises(HeliosError):
        make_plan(wl, iso_layers=2)
