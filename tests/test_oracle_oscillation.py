"""Pin of the oracle's timestep oscillation control (Sect. 2.2.4, reading R6 and cap R7).

The rule, restated from the section: each layer keeps the signs of its last six temperature
changes.  Once six are recorded, six equal signs (a monotonic run) raise the layer's timestep
multiplier by 10 %, and a sign change anywhere among them (an oscillation; the section treats
the two cases as complementary) lowers it by 33 %.  Nothing changes before six signs exist, and
the multiplier is capped (10).

The oracle's temperature step is driven here by hand-made bolometric fluxes whose net-flux
divergence has a chosen sign in every layer (a positive divergence cools the layer, eq. 24 with
the sign of reading R5), so the sequence of step signs is known in advance; the expected
multipliers below are written out from the rule's text, not computed by the oracle.
"""
import numpy as np
import pytest

import oracle
import synth


def _atm(n=4):
    wl = synth.config1()
    a = wl.atms[0]
    a = synth.Atmosphere(n_layers=n, P_top_bar=a.P_top_bar, P_bot_bar=a.P_bot_bar, grav=a.grav, T_irr=a.T_irr,
                         T_int=a.T_int, T_star=a.T_star, nu_edges=a.nu_edges, omega0=a.omega0, g0=a.g0,
                         table_id=0, T_init=np.full(n, 1000.0))
    return oracle.Atm(a, wl.tables[0])


def _fluxes(signs, scale=1e3):
    """Bolometric fluxes whose divergence dF_i = F_net(i+1) - F_net(i) has the sign opposite to
    signs[i] (so the temperature change of layer i has sign signs[i]); F_dn = 0."""
    n = len(signs)
    fu = np.zeros(n + 1)
    for i, s in enumerate(signs):
        fu[i + 1] = fu[i] - s * scale          # dF_i = -s * scale
    return fu, np.zeros(n + 1)


def _run(atm, seq, mult_max=10.0):
    """Apply temperature steps whose per-layer signs follow seq (a list of per-step sign tuples);
    returns the multipliers after every step and the final state."""
    p = oracle.params(mult_max=mult_max, tol=1e-30)
    st = oracle.State(atm, np.full(atm.n, 1000.0))
    out = []
    for signs in seq:
        signs = tuple(signs) + (signs[-1],) * (atm.n - len(signs))     # extra layers follow the last
        st.T[:] = 1000.0                       # keep every step far from the floor and the metric high
        fu, fd = _fluxes(signs)
        rc, metric, dT = oracle.temp_update(atm, st, fu, fd, p)
        assert rc == oracle.UPDATED
        assert np.all(np.sign(dT) == np.array(signs))
        out.append(st.mult.copy())
    return np.array(out), st


def test_no_change_before_six_signs_then_monotonic_growth():
    atm = _atm(2)
    m, st = _run(atm, [(+1,)] * 8)
    np.testing.assert_array_equal(m[:5, 0], [1.0] * 5)           # fewer than six signs recorded
    assert m[5, 0] == pytest.approx(1.1, rel=1e-15)              # six equal signs: +10 %
    assert m[6, 0] == pytest.approx(1.21, rel=1e-15)
    assert m[7, 0] == pytest.approx(1.331, rel=1e-15)
    assert st.nhist[0] == 6 and st.hist[0] == 0b111111


def test_monotonic_cooling_counts_like_heating():
    atm = _atm(2)
    m, st = _run(atm, [(-1,)] * 6)
    assert m[5, 0] == pytest.approx(1.1, rel=1e-15)
    assert st.hist[0] == 0


def test_strict_alternation_damps():
    atm = _atm(2)
    m, st = _run(atm, [(+1,), (-1,)] * 4)
    np.testing.assert_array_equal(m[:5, 0], [1.0] * 5)
    assert m[5, 0] == pytest.approx(0.67, rel=1e-15)
    assert m[6, 0] == pytest.approx(0.67 ** 2, rel=1e-15)
    assert m[7, 0] == pytest.approx(0.67 ** 3, rel=1e-15)
    assert st.hist[0] == 0b101010                               # newest sign in bit 0 (a negative step last)


def test_period_four_cycle_counts_as_oscillation():
    # ++--++ has sign changes but is not a strict alternation: under reading R6 it damps
    atm = _atm(2)
    m, _ = _run(atm, [(+1,), (+1,), (-1,), (-1,), (+1,), (+1,), (-1,)])
    assert m[5, 0] == pytest.approx(0.67, rel=1e-15)
    assert m[6, 0] == pytest.approx(0.67 ** 2, rel=1e-15)


def test_single_change_after_monotonic_run():
    # six + raise the multiplier; one - makes the window mixed, so it falls by 33 % while a + is
    # still among the last six signs, and a run of six equal signs (the first - and the five after
    # it) raises it again
    atm = _atm(2)
    seq = [(+1,)] * 6 + [(-1,)] + [(-1,)] * 6
    m, _ = _run(atm, seq)
    assert m[5, 0] == pytest.approx(1.1, rel=1e-15)
    assert m[6, 0] == pytest.approx(1.1 * 0.67, rel=1e-15)
    # steps 7..10: the window still holds a + -> damped each time; step 11: six - -> raised
    expect = 1.1 * 0.67
    for k in range(7, 11):
        expect *= 0.67
        assert m[k, 0] == pytest.approx(expect, rel=1e-14)
    assert m[11, 0] == pytest.approx(expect * 1.1, rel=1e-14)
    assert m[12, 0] == pytest.approx(expect * 1.21, rel=1e-14)


def test_cap_on_the_multiplier():
    atm = _atm(2)
    m, _ = _run(atm, [(+1,)] * 40, mult_max=10.0)
    # 1.1^k first exceeds 10 at k = 25 (1.1^24 = 9.85, 1.1^25 = 10.83): steps 6..29 grow, then capped
    assert m[28, 0] == pytest.approx(1.1 ** 24, rel=1e-13)
    assert m[29, 0] == 10.0
    assert np.all(m[29:, 0] == 10.0)
    # a lower cap binds exactly at the cap
    m2, _ = _run(atm, [(+1,)] * 10, mult_max=1.2)
    assert m2[5, 0] == pytest.approx(1.1, rel=1e-15)
    assert m2[6, 0] == 1.2 and m2[9, 0] == 1.2


def test_layers_are_independent():
    atm = _atm(3)
    seq = [(+1, +1, +1), (+1, -1, +1), (+1, +1, -1), (+1, -1, -1), (+1, +1, +1), (+1, -1, -1)]
    m, _ = _run(atm, seq)
    assert m[5, 0] == pytest.approx(1.1, rel=1e-15)          # layer 0: six +
    assert m[5, 1] == pytest.approx(0.67, rel=1e-15)         # layer 1: alternating
    assert m[5, 2] == pytest.approx(0.67, rel=1e-15)         # layer 2: mixed
