"""Pins of the oracle's coupled trajectory to Table 2 (section 3.1 of the paper:
one particle settling in a 0.001 x 0.001 x 0.005 m cavity, Table 1's properties,
Stokes' law Eq. 17). CPU only.

With the readings the oracle takes (force density g = 2 (rho_l U - j_l) from the
moving bounce-back, Eqs. 6-7; A_p = pi d^2 / 4 in Eq. 12; Eq. 13 for the
particle), the terminal velocity at the paper's relaxation times does not
reproduce Table 2's numerical column: the steady slip alone is
m (1 - rho_f/rho_p) g / (2 A_p rho_l) = (6 nu / d) V_Stokes, which at h/d = 4 and
tau = 0.65 is already 1.20 V_Stokes, and the fluid dragged down with the particle
adds to it. The paper states that it calibrated its parameters against Stokes'
law in this test. So the pins are:
  - at the paper's tau, every row within 25 % of Table 2, the slip equal to its
    closed form, the fluid moving with the particle, the speed growing with the
    diameter (as section 3.1 reports), and the deviations equal to the ones
    recorded in tests/golden/table2_oracle.txt;
  - at the tau recorded there for each row, the oracle reproduces Table 2's
    numerical column within 0.5 %.
"""
import multiprocessing as mp
import os
import sys

import numpy as np
import pytest

from conftest import ROOT, read_golden

sys.path.insert(0, os.path.join(ROOT, "tests", "golden"))
import make_table2_oracle as t2  # noqa: E402


def _run(args):
    hd, tau = args
    return t2.terminal_velocity(hd, tau, t2.properties())


@pytest.fixture(scope="module")
def runs():
    table = read_golden("table2_settling.txt")
    rec = read_golden("table2_oracle.txt")
    jobs = [(r[0], float(r[3])) for r in table] + [(r[0], float(r[4])) for r in rec]
    with mp.get_context("spawn").Pool(min(len(jobs), os.cpu_count() or 1)) as pool:
        res = pool.map(_run, jobs)
    n = len(table)
    return table, rec, res[:n], res[n:]


def test_terminal_velocity_at_paper_tau(runs):
    table, rec, at_paper, _ = runs
    props = t2.properties()
    rr = props["rho_p"] / props["rho_f"]
    speeds = []
    for (hd, v_stokes, v_num, tau, _dt), (_, _, v_rec, dev_rec, _), (v, U, u_fl, glu) in zip(
            table, rec, at_paper):
        v_num, v_stokes, tau = float(v_num), float(v_stokes), float(tau)
        d = 1.0 / float(hd)
        # the band: 25 % of Table 2 (the closed-form slip bound below is 20 % at h/d = 4)
        assert abs(v / v_num - 1.0) <= 0.25, (hd, v, v_num)
        # steady slip: U - u_l = -m (1 - 1/rho_r) g / (2 A_p rho_l), rho_l = 1 to 1e-4
        m = rr * np.pi * d ** 3 / 6.0
        slip = -m * (1.0 - 1.0 / rr) * glu / (2.0 * np.pi * d * d / 4.0)
        assert (U - u_fl) == pytest.approx(slip, rel=2e-3)
        # the fluid at the particle moves down with it, so |U| exceeds the slip
        assert u_fl < 0.0 and U < slip < 0.0
        # the deviation recorded in the golden file (same run)
        assert v / v_num - 1.0 == pytest.approx(float(dev_rec), abs=5e-4)
        speeds.append(abs(v))
    # section 3.1: the settling speed grows with the particle size (h/d 4 -> 1)
    assert all(a < b for a, b in zip(speeds, speeds[1:]))


def test_slip_bound_rules_out_a_tighter_band_at_h_over_d_4():
    """(6 nu / d) V_Stokes, the slip alone, against Table 2's numerical value at
    h/d = 4, tau = 0.65: at least 19 % above it."""
    hd, v_stokes, v_num, tau, _dt = read_golden("table2_settling.txt")[0]
    nu = (float(tau) - 0.5) / 3.0
    d = 1.0 / float(hd)
    assert 6.0 * nu / d * abs(float(v_stokes)) / abs(float(v_num)) - 1.0 > 0.19


def test_calibrated_tau_reproduces_table2(runs):
    table, rec, _, at_cal = runs
    for (hd, _vs, v_num, tau, _dt), (_, _, _, _, tau_c), (v, *_rest) in zip(table, rec, at_cal):
        assert v / float(v_num) - 1.0 == pytest.approx(0.0, abs=5e-3), (hd, tau_c, v)
        # the calibrated tau stays within 0.1 of the paper's
        assert abs(float(tau_c) - float(tau)) < 0.1
