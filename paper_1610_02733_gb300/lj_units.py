"""Lennard-Jones units of the Kremer-Grest test system (Sec. 4) in the
library's lattice units.

The paper states its test in LJ units: bead mass mu, LJ length sigma and
energy epsilon, time tau = (mu sigma^2 / epsilon)^(1/2); lattice spacing
a = sigma, fluid density rho = 1 mu / sigma^3, k_B T = 1 epsilon, shear
viscosity eta = 3 epsilon tau / sigma^3; MD time step dt (in tau) and
m = tau_LB / dt MD steps per LB step.  The library works in lattice units
(a = 1, tau_LB = 1, bead mass 1).  With tau_LB = m dt tau, one lattice
energy unit mu a^2 / tau_LB^2 is epsilon / (m dt)^2, so

    energies and k_B T      x (m dt)^2
    forces (epsilon/sigma)  x (m dt)^2
    velocities (sigma/tau)  x  m dt
    friction (mu/tau)       x  m dt
    kinematic viscosity     eta / rho = 3 sigma^2/tau  ->  3 m dt
    MD time step            1 / m.

The Kremer-Grest interactions (Sec. 4): LJ between all beads, cut off at
2^(7/6) sigma, and FENE springs with the parameters of the standard model
(k = 30 epsilon / sigma^2, R0 = 1.5 sigma)."""

R_CUT_KG = 2.0 ** (7.0 / 6.0)  # Sec. 4: LJ cut off at 2^(7/6) sigma
K_FENE = 30.0                  # epsilon / sigma^2, standard Kremer-Grest springs
R0_FENE = 1.5                  # sigma


def lattice_params(m: int, dt: float, zeta: float, *, kT: float = 1.0, eta: float = 3.0, rho: float = 1.0,
                   eps: float = 1.0) -> dict:
    """Lattice-unit parameters of one point of the paper's grid: m MD steps
    per LB step, MD time step dt (in tau), friction zeta (in mu/tau),
    temperature kT and LJ energy eps (in epsilon), shear viscosity eta (in
    epsilon tau / sigma^3), fluid density rho (in mu / sigma^3)."""
    if m < 1 or not dt > 0 or not zeta >= 0:
        raise ValueError("need m >= 1, dt > 0, zeta >= 0")
    t = m * dt  # tau_LB in units of tau
    e = t * t   # epsilon in lattice energy units (for eps = 1)
    return {
        "n_sub": int(m),
        "tau_lb": t,
        "rho0": float(rho),
        "nu": eta / rho * t,
        "kT": kT * e,
        "zeta": zeta * t,
        "lj_eps": eps * e,
        "lj_sigma": 1.0,
        "lj_rc": R_CUT_KG,
        "fene_k": K_FENE * eps * e,
        "fene_R0": R0_FENE,
        "velocity_scale": t,   # lattice velocity per sigma/tau
        "energy_scale": e,     # lattice energy per epsilon
    }


def temperature_in_lj(kT_lattice: float, params: dict) -> float:
    """k_B T in units of epsilon from a lattice-unit kinetic temperature."""
    return kT_lattice / params["energy_scale"]
