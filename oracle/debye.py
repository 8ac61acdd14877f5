"""Double-Debye skin permittivity, Eq. 6 (oracle, test infrastructure).

eps_r(w) = eps_inf + (eps_s - eps_2)/(1 + j w tau1) + (eps_2 - eps_inf)/(1 + j w tau2)

with the skin parameters given right after Eq. 6: eps_inf = 3, eps_s = 60,
eps_2 = 3.6, tau1 = 10 ps, tau2 = 0.2 ps.
"""
from __future__ import annotations

import math

SKIN = {"eps_inf": 3.0, "eps_s": 60.0, "eps_2": 3.6, "tau1": 10e-12, "tau2": 0.2e-12}


def eps_r(freq_hz: float, eps_inf=SKIN["eps_inf"], eps_s=SKIN["eps_s"], eps_2=SKIN["eps_2"],
          tau1=SKIN["tau1"], tau2=SKIN["tau2"]) -> complex:
    w = 2.0 * math.pi * freq_hz
    return eps_inf + (eps_s - eps_2) / (1.0 + 1j * w * tau1) + (eps_2 - eps_inf) / (1.0 + 1j * w * tau2)
