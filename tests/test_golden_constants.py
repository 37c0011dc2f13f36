"""The reduced application's constants against the values the paper prints
(tests/golden/reduced_app_constants.txt, each line with its citation): the
oracle's and the binding's defaults and the initial box state must carry
them."""
import inspect
import os

import numpy as np

import oracle
from paper_1802_05839_gb300 import inputs, wx

HERE = os.path.dirname(os.path.abspath(__file__))


def golden():
    vals = {}
    for line in open(os.path.join(HERE, "golden", "reduced_app_constants.txt")):
        if line.strip() and not line.startswith("#"):
            name, value = line.split()[:2]
            vals[name] = float(value)
    return vals


def test_oracle_defaults_are_the_papers():
    g = golden()
    p = oracle.pf_params(8, 8, 4)
    assert p.radiation == g["radiation_per_step"]
    assert p.transfer == g["transfer"]
    assert p.T_surf == g["T_surface_well"] and p.T_pbl == g["T_top_well"]


def test_binding_defaults_are_the_papers():
    g = golden()
    d = inspect.signature(wx.ReducedApp.set_params).parameters
    assert d["radiation"].default == g["radiation_per_step"]
    assert d["transfer"].default == g["transfer"]
    assert d["T_surf"].default == g["T_surface_well"] and d["T_pbl"].default == g["T_top_well"]


def test_box_state_is_the_papers():
    g = golden()
    n = 16
    E = inputs.paper_box_state(n, n, n)
    inner = E[n // 4:3 * n // 4, 1 + n // 4:1 + 3 * n // 4, 1 + n // 4:1 + 3 * n // 4]
    assert np.all(inner == g["box_temperature"])
    assert E.sum() == g["box_temperature"] * (n // 2) ** 3        # nothing else is warm
    assert np.all(E[0] == g["background_temperature"])


def test_time_step_is_the_papers():
    assert inputs.small_case().dt == golden()["dt"]
    assert inputs.paper_grid_case(8, 8, 4).dt == golden()["dt"]
