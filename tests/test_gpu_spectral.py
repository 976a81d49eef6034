"""GPU parity of the per-bin fluxes at every point (helios_flux_sweep's F_spec output) against the
FP64 oracle's per-bin fluxes, element by element, and of the emergent spectrum relative to each
bin's own emergent flux.

Tolerances:
- per-bin flux at a point: 1e-5 of the larger of the bin's two streams at that point (the same
  convention as the net flux; a stream that is a small fraction of the other carries the
  float32 rounding of the larger one).  Elements whose larger stream is below 1e-20 of the bin's
  largest flux anywhere in the column are not compared (their float32 values lie in the
  subnormal range or at zero once the Wien factor underflows);
- emergent spectrum relative to the bin's own emergent flux: 1e-5 wherever the emergent flux is
  at least 1 % of the incident one, 1e-3 everywhere (reflected fractions far below 1 % of the
  incident stream inherit its float32 rounding).

Thin-sublayer switch (Sect. 2.2.1, reading R9): the isothermal form is chosen where
dtau < 1e-4, the GPU deciding on its float32 optical depth and the oracle on its double one.
The two can differ only for a sublayer whose double optical depth lies within float32 rounding
of the threshold; such flips are counted, and the bins that hold one are left out of the
element-wise comparison (their fluxes differ by the jump between the two forms, O(dtau dB)).
"""
import numpy as np
import pytest

import oracle
import synth
import paper_1606_05474_b300 as hp
from helpers import make_plan, pack

FLUX_TOL = 1e-5
FLIP_BAND = 3e-7          # relative distance from the threshold within which float32 may decide otherwise


def flip_bins(atm, T, dtau_iso=1e-4):
    """Bins in which some (sublayer, g) has a double optical depth within float32 rounding of the
    thin-sublayer threshold (where the two sides may take different forms)."""
    kap, _, _ = oracle.interp_opacity(atm, T)             # [2n+1][L][G]
    _, _, dm, _ = oracle.grid(atm)                        # [2n]
    ks = 0.5 * (kap[:-1] + kap[1:])                       # sublayer means
    dtau = ks * dm[:, None, None]
    near = np.abs(dtau / dtau_iso - 1.0) < FLIP_BAND
    return np.unique(np.nonzero(near)[1])


def check_spec(plan, spec, r, skip_bins=(), a=0, tol=FLUX_TOL):
    """Element-wise comparison of the GPU's per-bin point fluxes with the oracle's up_spec/dn_spec;
    returns the largest relative error."""
    up, dn = plan.split_spec(spec)[a]
    ou, od = r["up_spec"], r["dn_spec"]                  # [L][2n+1]
    keep = np.ones(ou.shape[0], bool)
    keep[list(skip_bins)] = False
    scale = np.maximum(np.abs(ou), np.abs(od))
    colmax = scale.max(axis=1, keepdims=True)
    mask = (scale >= 1e-20 * colmax) & keep[:, None]
    e_up = np.abs(up.astype(np.float64) - ou) / np.where(mask, scale, 1.0)
    e_dn = np.abs(dn.astype(np.float64) - od) / np.where(mask, scale, 1.0)
    worst = float(max(e_up[mask].max(), e_dn[mask].max()))
    assert worst < tol, f"per-bin flux error {worst:.3e}"
    return worst


def check_toa_own(toa, r, atm):
    """Emergent spectrum relative to each bin's own emergent flux; returns (max where the emergent
    flux is >= 1 % of the incident one, max overall)."""
    inc, _ = oracle.boundary_spectra(atm)
    g = toa.cpu().numpy().astype(np.float64)
    own = np.abs(g - r["toa"]) / np.abs(r["toa"])
    big = np.abs(r["toa"]) >= 1e-2 * inc
    e_big = float(own[big].max()) if big.any() else 0.0
    e_all = float(own.max())
    assert e_big < 1e-5, f"own-relative emergent error {e_big:.3e} in bins with >= 1 % of the incident flux"
    assert e_all < 1e-3, f"own-relative emergent error {e_all:.3e}"
    return e_big, e_all


def _spec_buf(plan):
    import torch
    return torch.empty(int(plan.info.spec_floats), dtype=torch.float32, device="cuda")


@pytest.mark.gpu
@pytest.mark.parametrize("n,L,lanes", [(111, 12, 0), (40, 12, 16), (40, 12, 32), (200, 5, 0), (2, 4, 0)])
def test_per_bin_fluxes_cold_then_warm(n, L, lanes):
    # several lane tiles and a ragged tail, five passes cold, then a warm-started evaluation at new
    # temperatures; every bin at every point
    wl = synth.small_scattering(L=L, n=n)
    atm = oracle.Atm.from_workload(wl)
    T1 = synth.perturbed_profile(wl.atms[0], 5)
    T2 = T1 + 7.0 * np.sin(np.arange(n))
    plan = make_plan(wl, col_lanes=lanes)
    spec = _spec_buf(plan)
    warm = np.zeros(atm.L * atm.G * (2 * n + 1))
    _, _, toa = plan.flux_sweep(pack([T1]), n_passes=5, spec=spec)
    r1 = oracle.flux_sweep(atm, T1, n_passes=5, warm=warm, warm_valid=False, spectra=True)
    check_spec(plan, spec, r1, flip_bins(atm, T1))
    check_toa_own(toa, r1, atm)
    _, _, toa2 = plan.flux_sweep(pack([T2]), n_passes=5, warm=True, spec=spec)
    r2 = oracle.flux_sweep(atm, T2, n_passes=5, warm=warm, warm_valid=True, spectra=True)
    check_spec(plan, spec, r2, flip_bins(atm, T2))
    check_toa_own(toa2, r2, atm)


@pytest.mark.gpu
def test_per_bin_fluxes_rayleigh():
    wl = synth.small_scattering(L=9, n=60)
    atm = oracle.Atm.from_workload(wl, rayleigh=True)
    T = synth.perturbed_profile(wl.atms[0], 12)
    plan = make_plan(wl, rayleigh=1)
    spec = _spec_buf(plan)
    plan.flux_sweep(pack([T]), n_passes=5, spec=spec)
    r = oracle.flux_sweep(atm, T, n_passes=5, spectra=True)
    check_spec(plan, spec, r)


@pytest.mark.gpu
def test_per_bin_fluxes_full_size_single_atmosphere():
    # 100 layers x 3000 bins x 20 g with scattering, the benchmark's launch configuration: all
    # 3000 x 201 x 2 per-bin point fluxes
    wl = synth.config2()
    atm = oracle.Atm.from_workload(wl)
    T = synth.perturbed_profile(wl.atms[0], 6)
    plan = make_plan(wl)
    spec = _spec_buf(plan)
    _, _, toa = plan.flux_sweep(pack([T]), spec=spec)
    r = oracle.flux_sweep(atm, T, spectra=True)
    flips = flip_bins(atm, T)
    assert len(flips) <= 3
    check_spec(plan, spec, r, flips)
    check_toa_own(toa, r, atm)


@pytest.mark.gpu
def test_per_bin_fluxes_ragged_batch():
    # three atmospheres of different depths and bin counts in one plan: each block of the packed
    # output against its own oracle evaluation
    wls = [synth.small_scattering(L=L, n=n, seed_offset=k) for k, (n, L) in enumerate([(30, 7), (120, 4), (57, 9)])]
    atms = [w.atms[0] for w in wls]
    for i, a in enumerate(atms):
        a.table_id = i
    wl = synth.Workload(name="ragged-3", atms=atms, tables=[w.tables[0] for w in wls])
    plan = make_plan(wl)
    Ts = [synth.perturbed_profile(a, 40 + i) for i, a in enumerate(atms)]
    spec = _spec_buf(plan)
    plan.flux_sweep(pack(Ts), n_passes=5, spec=spec)
    for i in range(3):
        atm = oracle.Atm.from_workload(wl, i)
        r = oracle.flux_sweep(atm, Ts[i], n_passes=5, spectra=True)
        check_spec(plan, spec, r, flip_bins(atm, Ts[i]), a=i)


@pytest.mark.gpu
def test_caller_owned_warm_start_buffer():
    # a caller-owned warm-start buffer gives the same evaluations, bit for bit, as the plan's own
    import torch
    wl = synth.small_scattering(L=10, n=50)
    T1 = synth.perturbed_profile(wl.atms[0], 3)
    T2 = T1 + 4.0 * np.cos(np.arange(50))
    p1, p2 = make_plan(wl), make_plan(wl)
    buf = torch.zeros(int(p2.info.warm_floats), dtype=torch.float32, device="cuda")
    a1 = [x.clone() for x in p1.flux_sweep(pack([T1]), n_passes=5)]
    b1 = p2.flux_sweep(pack([T1]), n_passes=5, warm_buf=buf)
    a2 = [x.clone() for x in p1.flux_sweep(pack([T2]), n_passes=5, warm=True)]
    b2 = p2.flux_sweep(pack([T2]), n_passes=5, warm=True, warm_buf=buf)
    for x, y in zip(a1 + a2, list(b1) + list(b2)):
        assert bool((x == y).all())
    with pytest.raises(ValueError):
        p2.flux_sweep(pack([T1]), warm_buf=buf[1:])


def test_flip_detector_finds_a_planted_threshold_crossing():
    # the detector itself: scale one table row so that a sublayer's double optical depth sits
    # exactly on the threshold, and it must be reported in that bin
    wl = synth.small_scattering(L=4, n=20)
    atm = oracle.Atm.from_workload(wl)
    T = np.full(20, 1000.0)
    kap, _, _ = oracle.interp_opacity(atm, T)
    _, _, dm, _ = oracle.grid(atm)
    s, l, g = 7, 2, 3
    dtau = 0.5 * (kap[s, l, g] + kap[s + 1, l, g]) * dm[s]
    atm.kappa.reshape(atm.s.nP, atm.s.nT, atm.s.L_table, atm.s.G)[:, :, l, g] *= 1e-4 / dtau
    assert l in flip_bins(atm, T)
