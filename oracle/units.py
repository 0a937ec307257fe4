"""Physical <-> lattice unit conversion and Stokes' settling law (test infrastructure).

The relaxation time fixes the lattice viscosity nu_lu = (tau - 1/2) / 3; with the
physical viscosity nu = mu / rho_f and spacing h this fixes the time step
dt = nu_lu h^2 / nu (Table 2, last column). Accelerations scale by dt^2 / h,
velocities by dt / h.
"""


def nu_lattice(tau):
    return (tau - 0.5) / 3.0


def time_step(tau, h, mu, rho_f):
    """Physical time step (s) of a lattice with spacing h (m) at relaxation time tau."""
    return nu_lattice(tau) * h * h / (mu / rho_f)


def accel_to_lattice(a, dt, h):
    return a * dt * dt / h


def velocity_to_physical(v_lu, dt, h):
    return v_lu * h / dt


def stokes_velocity(rho_p, rho_f, d, g, mu):
    """Stokes settling speed, Eq. (17): (rho_p - rho_f) d^2 g / (18 mu)."""
    return (rho_p - rho_f) * d * d * g / (18.0 * mu)
