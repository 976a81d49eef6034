"""Pins of the op-counting build of the oracle (the source of the roofline's algorithmic FP32 and
SFU counts): the counts of one layer solution written out by hand from its formulas (Sect. 2.1.3,
eqs. 12-15, and eq. 14 for pure scattering), and the split of an evaluation into work done once
(coefficients) and work repeated per pass (recurrences)."""
import ctypes

import numpy as np
import pytest

import synth
from oracle import opcount as oc


def _layer_counts(dtau, w0, g0=0.2):
    lib = oc._load()
    P = ctypes.POINTER
    lib.ref_layer_twostream.argtypes = [oc._CNum] * 7 + [P(oc._ParamsC), P(oc._CNum), P(oc._CNum)]
    p = oc._params()
    u, d = oc._CNum(), oc._CNum()
    lib.ref_opcount_reset()
    lib.ref_layer_twostream(oc._cn(10.0, 1), oc._cn(5.0, 1), oc._cn(3.0), oc._cn(2.0), oc._cn(dtau), oc._cn(w0),
                            oc._cn(g0), ctypes.byref(p), ctypes.byref(u), ctypes.byref(d))
    return oc._counts()


def test_one_layer_flux_work_by_hand():
    # eq. (15): F2up = (xi F1up - beta F2dn + S2) / alpha and F1dn alike: per stream two products
    # with a flux, the difference, the source added, and the quotient by alpha (a multiply by a
    # coefficient's reciprocal): 3 multiplies and 2 additions each, nothing else on the fluxes
    for dtau in (0.5, 1e-5):                      # linear-B and thin (eq. 11) forms
        c = _layer_counts(dtau, 0.3)
        assert c["flux"] == {"add": 4, "mul": 6, "div": 0, "exp": 0, "sqrt": 0, "log": 0, "pow": 0}
        assert c["coef"]["exp"] == 1 and c["coef"]["sqrt"] == 2      # eq. (8) transmission; eq. (13) ratio
    # eq. (14), pure scattering: x = a (F1up - F2dn) / (2 + a), F2up = F1up - x, F1dn = F2dn + x
    c = _layer_counts(0.5, 1.0)
    assert c["flux"] == {"add": 3, "mul": 2, "div": 0, "exp": 0, "sqrt": 0, "log": 0, "pow": 0}
    assert c["coef"]["exp"] == 0


def test_evaluation_split_into_once_and_per_pass():
    wl = synth.small_scattering(L=6, n=20)
    T = synth.perturbed_profile(wl.atms[0], 3)
    r1 = oc.flux_evaluation(wl.atms[0], wl.tables[0], T, 1)
    r5 = oc.flux_evaluation(wl.atms[0], wl.tables[0], T, 5)
    assert r1["coef"] == r5["coef"]                                  # coefficients once per evaluation
    per_pass = {k: (r5["flux"][k] - r1["flux"][k]) / 4 for k in oc.CATS}
    # one pass: one call's worth of flux work per sublayer and Gauss point (no pure-scattering
    # sublayers here: 6 multiplies, 4 additions each)
    subs = 2 * 20 * 6 * wl.G
    assert per_pass["mul"] == pytest.approx(6 * subs)
    # plus the BOA condition of eq. (22), one addition per column and pass (halved with the rest of
    # the per-pass work, which the oracle does twice): 0.3 % here
    assert per_pass["add"] == pytest.approx(4 * subs + 6 * wl.G / 2)
    # per sublayer and g the coefficients cost one exponential (eq. 8) and two square roots
    assert r1["coef"]["exp"] >= subs and r1["coef"]["sqrt"] == pytest.approx(2 * subs)
    assert r5["fp32"] > r1["fp32"] and r5["per_cell"]["fp32"] > 100
