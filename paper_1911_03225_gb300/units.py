"""Dimensionless variables of the layer problem (Sec. 3.2.1).

x~ = x/b, t~ = V_s t / b, sigma~ = sigma/mu, eta~ = V_s eta / mu, alpha~ = b alpha,
with V_s = sqrt(mu/rho) the elastic shear-wave speed.  The library itself works in these
dimensionless units; this module converts to and from SI.
"""
import math
from dataclasses import dataclass


@dataclass(frozen=True)
class Material:
    b: float      # Burgers vector norm [m]
    mu: float     # shear modulus [Pa]
    rho: float    # density [kg/m^3]
    eta: float    # viscous drag [Pa s / m]

    @property
    def shear_wave_speed(self) -> float:
        return math.sqrt(self.mu / self.rho)

    def stress_scale(self) -> float:
        """Stress that gives a unit celerity: V_s eta [Pa]."""
        return self.shear_wave_speed * self.eta

    def eta_dimensionless(self) -> float:
        return self.shear_wave_speed * self.eta / self.mu

    def time_seconds(self, t_dimless: float) -> float:
        return t_dimless * self.b / self.shear_wave_speed

    def length_dimensionless(self, x_m: float) -> float:
        return x_m / self.b

    def alpha_dimensionless(self, alpha_per_m: float) -> float:
        return self.b * alpha_per_m


def cfl_time_step(cfl: float, dx: float, v0: float) -> float:
    """Time step from the CFL rule |v0| dt / dx = CFL (Sec. 4.3, Sec. 5.2)."""
    return cfl * dx / abs(v0)
