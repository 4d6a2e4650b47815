"""Friedmann background and linear growth for a LambdaCDM run (Sec. IV-A.2).

Test infrastructure only (see ``oracle/__init__``).

The paper's run models a LambdaCDM universe (Omega_c = 0.214, Omega_b =
0.044, so Omega_m = 0.258, flat, from z = 99 to z = 0) and gives no
integrator; the readings of ``dynamics`` carry over with the background
generalised (H0 = 1, lengths in fine cells, time variable a):

* E(a) = H(a) / H0 = sqrt(Omega_m a^-3 + Omega_k a^-2 + Omega_L), with
  Omega_k = 1 - Omega_m - Omega_L.
* With p = a^2 dx/dt the equations of motion are dp/dt = -grad(phi) and
  dx/dt = p / a^2, with lap(phi) = (3/2) Omega_m delta / a.  In terms of a
  (dt = da / (a E)): dp/da = (3 Omega_m / (8 pi rho_bar)) g / (a^2 E) and
  dx/da = p / (a^3 E), g the unit-G field.  So the kick factor from a_lo to
  a_hi is (3 Omega_m / (8 pi rho_bar)) int da / (a^2 E) and the drift factor
  from a_n to a_n+1 is int da / (a^3 E).  Omega_m = 1, Omega_L = 0 gives the
  Einstein-de Sitter factors of ``dynamics`` (2 (sqrt(a_hi) - sqrt(a_lo)) and
  2 (a_n^-1/2 - a_n+1^-1/2)).
* Growing mode (matter, curvature and Lambda; Heath 1977):
  D(a) = (5/2) Omega_m E(a) int_0^a da' / (a' E(a'))^3, normalised so that
  D(a) -> a at early times, and f = dln D / dln a
  = dln E / dln a + 1 / (a^2 E^3 I(a)) with I the integral and
  dln E / dln a = -((3/2) Omega_m a^-3 + Omega_k a^-2) / E^2.
  The Zel'dovich ICs put x = q + D Psi and p = a^2 dx/dt = a^2 E f D Psi.

The integrals use scipy.integrate.quad (the library evaluates them its own
way).
"""

import math

from scipy import integrate

_QUAD = dict(epsabs=0.0, epsrel=1e-13, limit=200)


class Cosmology:
    """Background (Omega_m, Omega_L); EdS is Cosmology(1.0, 0.0)."""

    def __init__(self, omega_m=1.0, omega_l=0.0):
        if not omega_m > 0.0:
            raise ValueError("omega_m must be positive")
        self.om = float(omega_m)
        self.ol = float(omega_l)
        self.ok = 1.0 - self.om - self.ol

    def E(self, a):
        e2 = self.om / a ** 3 + self.ok / a ** 2 + self.ol
        if not e2 > 0.0:
            raise ValueError("no expanding background at a = %g" % a)
        return math.sqrt(e2)

    def kick_integral(self, a_lo, a_hi):
        """int_{a_lo}^{a_hi} da / (a^2 E(a))."""
        return integrate.quad(lambda a: 1.0 / (a * a * self.E(a)), a_lo, a_hi, **_QUAD)[0]

    def drift_integral(self, a_lo, a_hi):
        """int_{a_lo}^{a_hi} da / (a^3 E(a))."""
        return integrate.quad(lambda a: 1.0 / (a ** 3 * self.E(a)), a_lo, a_hi, **_QUAD)[0]

    def _growth_integral(self, a):
        # int_0^a da' / (a' E)^3; near 0 the integrand is a'^(3/2) / Omega_m^(3/2)
        return integrate.quad(lambda x: 1.0 / (x * self.E(x)) ** 3, 0.0, a, **_QUAD)[0]

    def growth(self, a):
        """D(a), with D -> a as a -> 0."""
        return 2.5 * self.om * self.E(a) * self._growth_integral(a)

    def growth_rate(self, a):
        """f = dln D / dln a."""
        E = self.E(a)
        dlnE = (-1.5 * self.om / a ** 3 - self.ok / a ** 2) / (E * E)
        return dlnE + 1.0 / (a * a * E ** 3 * self._growth_integral(a))

    def ic_momentum_factor(self, a):
        """p / (D Psi) of the growing mode at a: a^2 E(a) f(a)."""
        return a * a * self.E(a) * self.growth_rate(a)
