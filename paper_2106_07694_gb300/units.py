"""Physical parameters of the paper's tank experiments mapped to lattice units (host-side
scalars, no device work), for building the parameters of a sweep.

  Stokes settling velocity   V_s = D_p^2 g (rho_p - rho(S)) / (18 mu)      (Sec. 2.2.1, Eq. stokes_vel)
  particle volume fraction   phi_0 = C / rho_p, C in g/l = kg/m^3          (Sec. 2.2, Table 1)
  relaxation time            tau = nu / c_s^2 + 1/2, lattice units,
                             c_s^2 = 1/3                                   (Sec. 2.3.1, Eq. tau)
  lattice scale              a cell of dx metres and a step of dt seconds: velocity v dt/dx,
                             kinematic viscosity nu dt/dx^2, acceleration g dt^2/dx

The simulation's force is F = -A c along the vertical with c = phi/phi_0 and
A = gravity * density_contrast, so the particle term g (rho_p - rho_0)/rho_0 phi of
Eq. forceterm becomes gravity = g dt^2/dx and density_contrast = (rho_p/rho_0 - 1) phi_0;
with the sugar scalar (S = rho_S/S_0), sugar_contrast = rho_f/rho_0 - 1 and
vs_sugar = sugar_contrast / (rho_p/rho_0 - 1) (Eq. stokes_vel with rho(S) = rho_0 (1 + S* S)).
"""
from dataclasses import dataclass

CS2 = 1.0 / 3.0  # lattice speed of sound squared (D2Q9, D3Q19)
G_EARTH = 9.81   # m/s^2


def stokes_velocity(diameter, rho_p, rho_f, mu, g=G_EARTH):
    """Terminal velocity of a small sphere in a viscous fluid (Eq. stokes_vel), m/s."""
    return diameter ** 2 * g * (rho_p - rho_f) / (18.0 * mu)


def volume_fraction(concentration, rho_p):
    """Particle volume fraction of a suspension of `concentration` g/l (= kg/m^3) of
    particles of density rho_p kg/m^3 (Table 1)."""
    return concentration / rho_p


def tau_from_viscosity(nu_lattice):
    """BGK relaxation time of a lattice kinematic viscosity (Eq. tau, dt = 1)."""
    return nu_lattice / CS2 + 0.5


def viscosity_from_tau(tau):
    """Lattice kinematic viscosity of a BGK relaxation time (Eq. tau, dt = 1)."""
    return CS2 * (tau - 0.5)


@dataclass(frozen=True)
class LatticeScale:
    """A lattice cell of dx metres and a time step of dt seconds."""
    dx: float
    dt: float

    @classmethod
    def from_tau(cls, dx, nu, tau):
        """The time step that gives relaxation time tau for kinematic viscosity nu (m^2/s)."""
        return cls(dx, viscosity_from_tau(tau) * dx * dx / nu)

    def velocity(self, v):
        return v * self.dt / self.dx

    def viscosity(self, nu):
        return nu * self.dt / (self.dx * self.dx)

    def acceleration(self, a):
        return a * self.dt * self.dt / self.dx

    def steps(self, seconds):
        return seconds / self.dt


def lattice_params(scale, diameter, concentration, rho_p, rho_f, mu, rho_0=1000.0, g=G_EARTH, sugar=False):
    """Simulation keyword parameters (tau, gravity, density_contrast, settling_velocity and,
    with sugar, the sugar parameters) of particles of `diameter` m and density rho_p at
    `concentration` g/l above a lower layer of density rho_f (sugar solution, or the same
    fluid when rho_f = rho_0), in a fluid of dynamic viscosity mu and reference density
    rho_0, on the lattice `scale`.  The settling velocity is the Stokes velocity in the
    particle-laden fluid of density rho_0 (Eq. stokes_vel with S = 0)."""
    phi0 = volume_fraction(concentration, rho_p)
    R = rho_p / rho_0 - 1.0
    out = dict(tau=tau_from_viscosity(scale.viscosity(mu / rho_0)),
               gravity=scale.acceleration(g),
               density_contrast=R * phi0,
               settling_velocity=scale.velocity(stokes_velocity(diameter, rho_p, rho_0, mu, g)))
    if sugar:
        s_star = rho_f / rho_0 - 1.0
        out.update(sugar=True, sugar_contrast=s_star, phi0=phi0, vs_sugar=s_star / R)
    return out
