"""Physical units of the graphene runs (Part II, "Model and Methods" and "Results").

The Dirac fluid of charge-neutral graphene is modelled with the massless relativistic
lattice Boltzmann method, the Fermi velocity v_F playing the part of the speed of light:
lattice velocities are in units of v_F.  Lengths and times use "modified natural units"
with hbar = k_B = 1 and v_F = 1, energies in eV:

    length  [hbar v_F / eV],  time [hbar / eV],  kinematic viscosity [hbar v_F^2 / eV].

The kinematic viscosity is the classical nu = eta / rho with the mass density built from
the quasi-particle number density and an effective mass, rho = n m*, quoted in natural
units (c = 1) and rescaled by (c / v_F)^2.  The Reynolds number is Re = L U / nu with the
impurity diameter as L and the inflow speed as U.

v_F: the text quotes v_F ~ 1.1e6 m/s in passing, but the flow speed 1e5 m/s = 0.1 v_F and
the viscosity 11.8 hbar v_F^2 / eV (from 0.000132 hbar c^2 / eV) both fix v_F = 1.0e6 m/s,
and with it Re reproduces the printed 6.37 (one impurity, L = D = 0.5 um) and 12.74 (two
impurities, taken as L = 2 D).
"""
import math

HBAR_EV_S = 6.582119569e-16       # hbar in eV s (CODATA 2018, exact SI definition)
C_M_S = 299792458.0               # speed of light, m/s
V_F_M_S = 1.0e6                   # Fermi velocity of the graphene runs (see module docstring)
M_E_EV = 5.11e5                   # electron mass in eV / c^2 (the value the paper uses)

# transport inputs quoted in the paper (natural units, c = hbar = 1)
ETA_GRAPHENE = 2.633e3            # dynamic viscosity, eV^2 / (c^2 hbar)
N_GRAPHENE = 38.93                # number density, eV^2 / (hbar^2 c^2)


def length_unit_m(v_f=V_F_M_S):
    """One hbar v_F / eV in metres."""
    return HBAR_EV_S * v_f


def to_natural_length(metres, v_f=V_F_M_S):
    """A length in metres in units of hbar v_F / eV."""
    return metres / length_unit_m(v_f)


def kinematic_viscosity_natural(eta=ETA_GRAPHENE, n=N_GRAPHENE, m_eff=1.0):
    """nu = eta / (n m*) in hbar c^2 / eV (natural units, c = 1); m* in electron masses."""
    return eta / (n * m_eff * M_E_EV)


def kinematic_viscosity_vf(eta=ETA_GRAPHENE, n=N_GRAPHENE, m_eff=1.0, v_f=V_F_M_S):
    """The same viscosity in hbar v_F^2 / eV: hbar c^2 / eV = (c / v_F)^2 hbar v_F^2 / eV."""
    return kinematic_viscosity_natural(eta, n, m_eff) * (C_M_S / v_f) ** 2


def reynolds(length_m, speed_vf, nu_vf=None, v_f=V_F_M_S):
    """Re = L U / nu with L in metres, U in units of v_F and nu in hbar v_F^2 / eV
    (default: the graphene value from the paper's eta, n and m* = m_e)."""
    nu = kinematic_viscosity_vf(v_f=v_f) if nu_vf is None else nu_vf
    return to_natural_length(length_m, v_f) * speed_vf / nu


class LatticeUnits:
    """Lattice <-> physical conversion of a run: `spacing_m` metres between nodes, streaming
    displacement C = dt / a nodes per step at the particle speed v_F.

    - lattice velocity u (in units of the particle speed) = u_phys / v_F;
    - one step = C * spacing_m / v_F seconds;
    - node index x = position / spacing_m.
    """

    def __init__(self, spacing_m, courant=0.5, v_f=V_F_M_S):
        self.spacing_m = float(spacing_m)
        self.courant = float(courant)
        self.v_f = float(v_f)

    def step_seconds(self):
        return self.courant * self.spacing_m / self.v_f

    def velocity_lattice(self, metres_per_second):
        return metres_per_second / self.v_f

    def velocity_m_s(self, lattice_velocity):
        return lattice_velocity * self.v_f

    def nodes(self, metres):
        return metres / self.spacing_m

    def diameter_nodes(self, metres):
        """Odd integer node diameter closest to a physical diameter (discs are centred on a node)."""
        d = self.nodes(metres)
        k = int(math.floor((d - 1.0) / 2.0 + 0.5))
        return 2 * k + 1


def temperature_lattice(eps=1.0):
    """T(eps) of the paper's momentum set in lattice units: eps = 3 T^4 / pi^2."""
    return (math.pi * math.pi * eps / 3.0) ** 0.25


def eta_over_s_for_reynolds(reynolds_number, length_nodes, speed, a=0.1, eps0=1.0):
    """eta/s that gives a lattice run the Reynolds number Re = L U / nu, with the relativistic
    kinematic viscosity nu = eta / (eps + P) = (eta/s) / T (eps + P = T s at zero chemical
    potential), L = length_nodes * a in lattice length units and U in units of the particle
    speed."""
    return length_nodes * a * speed * temperature_lattice(eps0) / reynolds_number
