"""Write ``table2_oracle.txt``: the oracle's single-particle terminal velocities on
the setup of Table 2 (section 3.1 of the paper), and the relaxation time at which
the oracle reproduces each row of Table 2's numerical column.

Only the oracle runs here (test infrastructure). The setup: D3Q15, a
10 x 10 x 50 lattice with walls on every face (the 0.001 x 0.001 x 0.005 m
cavity at h = 1e-4 m), the 4-point cosine delta, Table 1's properties converted
to lattice units with the time step that tau fixes (Table 2's last column).
The particle starts at rest at (5, 5, 25) lu, mid-height, so that the terminal
velocity is that of the free fall between the top and bottom walls (the paper
starts it 1 lu below the top wall; a full fall at h/d = 4 takes about 10^6
steps). After STEPS steps the velocity is steady (the drag relaxes in well
under a step and the fluid within about (10 lu)^2 / nu steps).

    python tests/golden/make_table2_oracle.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import units  # noqa: E402
from oracle.oracle import Oracle  # noqa: E402

STEPS = 3000
START = (5.0, 5.0, 25.0)


def read_rows(name):
    rows = []
    with open(os.path.join(HERE, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def properties():
    return {k: float(v) for k, v in read_rows("table1_properties.txt")}


def terminal_velocity(hd, tau, props, steps=STEPS):
    """Physical terminal velocity (m/s, negative = downward) of the oracle's
    particle of diameter h / hd at relaxation time tau, and its lattice-unit
    velocity, position and interpolated fluid velocity after `steps` steps."""
    h = props["h"]
    d = 1.0 / float(hd)
    dt = units.time_step(tau, h, props["mu"], props["rho_f"])
    glu = units.accel_to_lattice(props["g"], dt, h)
    o = Oracle(15, (10, 10, 50), (0, 0, 0), tau, delta_width=4, gravity=(0, 0, -glu),
               x0=[list(START)], diameter=[d], density_ratio=[props["rho_p"] / props["rho_f"]])
    o.step(steps)
    fl = o.interp_pops(o.X[0])
    u_fluid = float((o.e[:, 2] * fl).sum() / fl.sum())
    return units.velocity_to_physical(o.U[0, 2], dt, h), float(o.U[0, 2]), u_fluid, glu


def calibrate(hd, v_target, tau0, props, tol=2e-4):
    """Secant search for the tau at which the oracle's terminal velocity equals
    v_target."""
    a, b = tau0 - 0.05, tau0 + 0.05
    fa = terminal_velocity(hd, a, props)[0] / v_target - 1.0
    fb = terminal_velocity(hd, b, props)[0] / v_target - 1.0
    for _ in range(12):
        c = b - fb * (b - a) / (fb - fa)
        fc = terminal_velocity(hd, c, props)[0] / v_target - 1.0
        a, fa, b, fb = b, fb, c, fc
        if abs(fc) < tol:
            break
    return b


def main():
    props = properties()
    out = ["# Oracle terminal velocities on the Table 2 setup (written by make_table2_oracle.py;",
           "# only the oracle ran). Particle at rest at (5, 5, 25) lu, D3Q15 10x10x50 walls,",
           f"# 4-point delta, {STEPS} steps. Columns: h/d_p, tau of Table 2, oracle terminal",
           "# velocity at that tau (m/s), its deviation from Table 2's numerical column,",
           "# tau at which the oracle reproduces the numerical column."]
    for hd, _vs, v_num, tau, _dt in read_rows("table2_settling.txt"):
        v, *_ = terminal_velocity(hd, float(tau), props)
        tau_c = calibrate(hd, float(v_num), float(tau), props)
        out.append(f"{hd} {tau} {v:.6e} {v / float(v_num) - 1.0:+.5f} {tau_c:.5f}")
        print(out[-1], flush=True)
    with open(os.path.join(HERE, "table2_oracle.txt"), "w") as fh:
        fh.write("\n".join(out) + "\n")


if __name__ == "__main__":
    main()
