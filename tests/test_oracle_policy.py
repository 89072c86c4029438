"""Pins for the step metrics and conditions (Sec. III-D, Eqs. 3-6, Conditions 1-3),
computed by hand or in closed form."""
import math

import numpy as np
import pytest

import oracle

P = oracle.Policy(l=0, t=10, m=1, rsd_limit=0.5, ndec_limit=0, reldec_limit=0.45, max_iter=100)


def test_constant_history():
    rsd, ndec, reldec = oracle.step_metrics([0.25] * 11, 10)   # dyadic: the mean is exact
    assert rsd == 0.0 and ndec == 0 and reldec == 0.0
    assert oracle.step_decide(rsd, ndec, reldec, 10, P) == 4          # Condition 3 only


@pytest.mark.parametrize("t", [5, 25, 250])
def test_geometric_decay_closed_form(t):
    q = 0.9
    seq = [q ** i for i in range(t + 1)]          # resid[j-t .. j]
    rsd, ndec, reldec = oracle.step_metrics(seq, t)
    assert ndec == t                              # every step decreases
    assert reldec == pytest.approx(1 - q ** (t - 1), rel=1e-14)
    mu = (1 - q ** t) / (t * (1 - q))
    m2 = (1 - q ** (2 * t)) / (t * (1 - q * q))
    assert rsd == pytest.approx(math.sqrt(m2 - mu * mu) / mu, rel=1e-9)


def test_window_uses_last_t_plus_one_entries():
    seq = [5.0, 4.0, 100.0, 1.0, 2.0, 1.0, 3.0]   # t = 3 -> window 1.0 2.0 1.0 | 3.0
    rsd, ndec, reldec = oracle.step_metrics(seq, 3)
    avg = 4.0 / 3
    assert rsd == pytest.approx(math.sqrt(((1 - avg) ** 2 * 2 + (2 - avg) ** 2) / 3) / avg)
    assert ndec == 1                               # only 2.0 > 1.0; 1.0 < 3.0
    assert reldec == 0.0                           # (resid[j-t] - resid[j-1]) / resid[j-t]
    with pytest.raises(ValueError):
        oracle.step_metrics([1.0, 2.0], 3)


def test_conditions_by_hand():
    t = 10
    # C1: large RSD and few decreases
    assert oracle.step_decide(0.6, 3, 0.9, t, P) & 1
    assert not oracle.step_decide(0.4, 3, 0.9, t, P) & 1
    assert not oracle.step_decide(0.6, 5, 0.9, t, P) & 1              # nDec = t/2 is not < t/2
    # C2: many decreases but slow relative decrease
    assert oracle.step_decide(0.1, 5, 0.2, t, P) == 2
    assert oracle.step_decide(0.1, 9, 0.5, t, P) == 0
    # C3: no decrease at all; a single decrease is not "no decrease"
    assert oracle.step_decide(0.0, 0, 0.9, t, P) == 4
    assert oracle.step_decide(0.4, 1, 0.9, t, P) == 0
    # nDec limit replaces t/2 when set
    P2 = oracle.Policy(l=0, t=10, m=1, rsd_limit=0.5, ndec_limit=8, reldec_limit=0.45, max_iter=1)
    assert oracle.step_decide(0.6, 6, 0.9, t, P2) & 1
    assert oracle.step_decide(0.1, 8, 0.2, t, P2) == 2
