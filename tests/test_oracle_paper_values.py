"""Pins against values the paper prints (Eq. 6 parameters, Table I)."""
import json
import math
import os

import numpy as np

from oracle import debye

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_debye_parameters_match_paper():
    p = _load("paper_debye_skin.json")
    assert debye.SKIN == {"eps_inf": p["eps_inf"], "eps_s": p["eps_s"], "eps_2": p["eps_2"],
                          "tau1": p["tau1_s"], "tau2": p["tau2_s"]}


def test_debye_limits_and_loss_sign():
    p = _load("paper_debye_skin.json")
    # static limit -> eps_s, optical limit -> eps_inf, intermediate plateau -> eps_2
    assert abs(debye.eps_r(0.0) - p["eps_s"]) < 1e-12
    assert abs(debye.eps_r(1e20) - p["eps_inf"]) < 1e-6
    # first relaxation: loss peak of height (eps_s - eps_2)/2 at w tau1 = 1 (the second
    # term adds (eps_2 - eps_inf) w tau2 / (1 + (w tau2)^2) = 0.012 there)
    f1 = 1.0 / (2 * math.pi * p["tau1_s"])
    assert abs(-debye.eps_r(f1).imag - (p["eps_s"] - p["eps_2"]) / 2) < 0.02
    # the real part of a sum of Debye terms falls monotonically with frequency
    re = [debye.eps_r(f).real for f in np.logspace(8, 15, 50)]
    assert np.all(np.diff(re) < 0)
    # e^{+j w t}: a lossy medium has Im eps_r < 0 at every frequency
    for f in np.logspace(9, 14, 21):
        assert debye.eps_r(f).imag < 0
    e = debye.eps_r(p["exposure_frequency_hz"])
    assert 3.0 < e.real < 3.6 and -1.5 < e.imag < -1.0


def test_table1_rates_and_sampling_density():
    rows = _load("paper_table1_compression.json")["rows"]
    for prev, cur in zip(rows, rows[1:]):
        eri = math.log(cur["time_s"] / prev["time_s"]) / math.log(cur["N"] / prev["N"])
        assert abs(eri - cur["eri"]) < 0.005
    for r in rows:
        assert abs(r["N"] / r["k0"] - 18.0) < 0.01
