"""Values the paper prints, kept as cited text fixtures under tests/golden/,
against the workloads built from them and against the oracle.

slab_table3.txt     Sec. 3.2, Table 3: the two-slab conduction benchmark
gearbox_table6.txt  Sec. 4.1, Table 6: lubricant and gear properties
"""
import math
import os

import numpy as np
import pytest
from scipy.special import erf, erfc

from paper_2512_09904_b300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                out[k] = float(v)
    return out


def test_slab_table_diffusivities():
    # the table's diffusivity column is alpha = k / (c_p rho) of its other columns
    g = load("slab_table3.txt")
    for s in ("l", "r"):
        assert g[f"alpha_{s}"] == pytest.approx(g[f"k_{s}"] / (g[f"cp_{s}"] * g[f"rho_{s}"]), rel=1e-12)


def test_slab_workload_follows_table():
    g = load("slab_table3.txt")
    case = W.slab(dx=g["dx"], h_over_dx=g["h_over_dx"])
    m = case.materials
    assert (m[0]["rho0"], m[0]["k"], m[0]["cp"]) == (g["rho_l"], g["k_l"], g["cp_l"])
    assert (m[1]["rho0"], m[1]["k"], m[1]["cp"]) == (g["rho_r"], g["k_r"], g["cp_r"])
    f = W.flatten(case)
    x, T = f["pos"][:, 0], f["T"]
    assert x.min() > 0.0 and x.max() < g["length"]
    left = x < g["interface_x"]
    assert np.all(T[left] == g["T_left"]) and np.all(T[~left] == g["T_right"])
    assert np.all(f["mat"][left] == 0) and np.all(f["mat"][~left] == 1)


def test_slab_at_the_papers_resolution_matches_the_contact_solution(oracle):
    # the paper's run: dx = 0.0125, h = 1.0 dx, profile at t = 2.0.  Two
    # semi-infinite media in contact: the interface sits at
    # T_i = (e_r T_r + e_l T_l) / (e_l + e_r), e = sqrt(k rho c_p), and each side
    # follows the error-function solution with its own diffusivity.
    g = load("slab_table3.txt")
    case = W.slab(dx=g["dx"], h_over_dx=g["h_over_dx"], dt_ad=0.02)
    sim = oracle.OracleSim(case)
    sim.step(int(round(g["t_compare"] / 0.02)))
    t = sim.time()["t"]
    assert t == pytest.approx(g["t_compare"], rel=1e-12)
    x, T = sim.field("pos")[:, 0], sim.field("T")
    el = math.sqrt(g["k_l"] * g["rho_l"] * g["cp_l"])
    er = math.sqrt(g["k_r"] * g["rho_r"] * g["cp_r"])
    Ti = (er * g["T_right"] + el * g["T_left"]) / (el + er)
    xi = g["interface_x"]
    ana = np.where(x < xi,
                   g["T_left"] + (Ti - g["T_left"]) * erfc((xi - x) / (2 * np.sqrt(g["alpha_l"] * t))),
                   Ti + (g["T_right"] - Ti) * erf((x - xi) / (2 * np.sqrt(g["alpha_r"] * t))))
    assert np.abs(T - ana).max() < 1e-2


def test_gear_bath_follows_table6():
    g = load("gearbox_table6.txt")
    case = W.gear_bath(dx=5e-3)
    m = case.materials
    oil, gear = m[0], m[1]
    assert (oil["rho0"], oil["k"], oil["cp"], oil["T_init"]) == (g["rho_oil"], g["k_oil"], g["cp_oil"], g["T_oil"])
    assert (gear["rho0"], gear["k"], gear["T_init"]) == (g["rho_gear"], g["k_gear"], g["T_gear"])
    assert gear["fixed_T"] == 1  # the gears are held at their temperature
