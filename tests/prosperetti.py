"""Prosperetti's initial-value solution for the amplitude of a small capillary
wave between two fluids of equal kinematic viscosity (eq:decay_wave_amplitude
and eq:algebraic_equation of the paper, Sec. 5.1), with the garbled terms
restored by dimensional analysis:
  * the first term's denominator is 8(1 - 4 gamma) nu^2 k^4 + omega_0^2;
  * the complementary error function's argument is z_i sqrt(t);
  * the quartic's constant term is (1 - 4 gamma) nu^2 k^4 + omega_0^2.
With these, eta(0) / eta_0 = 1, which the printed form does not give."""
import numpy as np


def amplitude(t, k, nu, sigma, rho_H, rho_L):
    from scipy.special import erfc
    gam = rho_H * rho_L / (rho_H + rho_L) ** 2
    om0sq = sigma * k ** 3 / (rho_H + rho_L)
    a = np.sqrt(nu * k * k)
    z = np.roots([1.0, -4 * gam * a, 2 * (1 - 6 * gam) * a * a, 4 * (1 - 3 * gam) * a ** 3,
                  (1 - 4 * gam) * a ** 4 + om0sq]).astype(complex)
    t = np.asarray(t, float)
    res = (4 * (1 - 4 * gam) * nu ** 2 * k ** 4 / (8 * (1 - 4 * gam) * nu ** 2 * k ** 4 + om0sq)
           * erfc(np.sqrt(nu * k * k * t))).astype(complex)
    for i in range(4):
        Zi = np.prod([z[j] - z[i] for j in range(4) if j != i])
        res = res + z[i] / Zi * om0sq / (z[i] ** 2 - nu * k * k) * np.exp((z[i] ** 2 - nu * k * k) * t) \
            * erfc(z[i] * np.sqrt(t))
    return res.real
