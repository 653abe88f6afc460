// FP64 host numerics of the PM library: background, growth, leapfrog integrals
// and the Eisenstein-Hu no-wiggle linear power spectrum (Sec. 3 setup).
#pragma once

namespace pmhost {

constexpr double kCLight = 2997.92458;  // c in units of 100 km/s (H0 = 1 units)

struct Cosmo {
    double omega_m, omega_b, h, n_s, sigma8;
    double t_cmb = 2.7255;
    double amp = 0.0;  // sigma_8 normalisation of A k^n_s T^2
};

double E(const Cosmo& c, double a);                     // H/H0 = sqrt(Om a^-3 + 1 - Om)
double omega_m_a(const Cosmo& c, double a);             // Om a^-3 / E^2
double conformal_hubble(const Cosmo& c, double a);      // a E / c, h/Mpc
double growth_D(const Cosmo& c, double a);              // D(1) = 1
double growth_f(const Cosmo& c, double a);              // dlnD/dlna
double kick_integral(const Cosmo& c, double a0, double a1);   // int da / (a^2 E)
double drift_integral(const Cosmo& c, double a0, double a1);  // int da / (a^3 E)
// Growth-matched leapfrog factors, exact for the linear growing mode x = q + D Psi,
// p = growth_p Psi, whose force is g = (3/2) Om D Psi (FastPM, Feng et al. 2016).
double growth_p(const Cosmo& c, double a);                                 // a^2 E f D
double kick_growth(const Cosmo& c, double a0, double a1, double a_force);  // force taken at a_force
double drift_growth(const Cosmo& c, double a0, double a1, double a_mom);   // momenta held at a_mom
double transfer_eh_nowiggle(const Cosmo& c, double k);        // k in h/Mpc
void normalise_sigma8(Cosmo& c);                        // sets c.amp
double power_linear(const Cosmo& c, double k);          // z = 0, (Mpc/h)^3

}  // namespace pmhost
