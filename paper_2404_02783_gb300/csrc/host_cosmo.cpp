// FP64 host numerics: adaptive composite Gauss-Legendre quadrature and the
// LambdaCDM quantities the PM step needs once per step or once per run.
#include "host_cosmo.h"

#include <cmath>
#include <mutex>

namespace pmhost {

namespace {

constexpr int kGL = 20;

struct GaussLegendre {
    double x[kGL], w[kGL];
    GaussLegendre() {
        // Roots of P_20 by Newton iteration on the three-term recurrence
        // (j+1) P_{j+1} = (2j+1) z P_j - j P_{j-1}; weights 2 / ((1 - z^2) P_20'(z)^2).
        const int n = kGL;
        for (int i = 0; i < (n + 1) / 2; ++i) {
            double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
            double dp = 1.0;
            for (int it = 0; it < 100; ++it) {
                double p0 = 1.0, p1 = 0.0;
                for (int j = 1; j <= n; ++j) {
                    const double p2 = p1;
                    p1 = p0;
                    p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
                }
                dp = n * (z * p0 - p1) / (z * z - 1.0);
                const double dz = p0 / dp;
                z -= dz;
                if (std::fabs(dz) < 1e-16) break;
            }
            x[i] = -z;
            x[n - 1 - i] = z;
            w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
        }
    }
};

const GaussLegendre& gl() {
    static const GaussLegendre g;
    return g;
}

template <class F>
double panel(const F& f, double a, double b) {
    const GaussLegendre& g = gl();
    const double m = 0.5 * (a + b), h = 0.5 * (b - a);
    double s = 0.0;
    for (int i = 0; i < kGL; ++i) s += g.w[i] * f(m + h * g.x[i]);
    return s * h;
}

// Bisect until the panel pair agrees with the parent within an error density
// tol_per_unit * width (so the total error stays below tol_per_unit * (b - a)), at
// roundoff level, or at depth 40.
template <class F>
double adapt(const F& f, double a, double b, double whole, double tol_per_unit, int depth) {
    const double m = 0.5 * (a + b);
    const double l = panel(f, a, m), r = panel(f, m, b);
    const double err = std::fabs(l + r - whole);
    if (depth >= 40 || err <= tol_per_unit * (b - a) || err <= 4e-16 * (std::fabs(l) + std::fabs(r)))
        return l + r;
    return adapt(f, a, m, l, tol_per_unit, depth + 1) + adapt(f, m, b, r, tol_per_unit, depth + 1);
}

// Integral of f over [a, b] to an absolute error of about rel * |integral|.
template <class F>
double integrate(const F& f, double a, double b, double rel = 1e-14) {
    if (a == b) return 0.0;
    double est = 0.0;
    for (int i = 0; i < 8; ++i) est += panel(f, a + (b - a) * i / 8.0, a + (b - a) * (i + 1) / 8.0);
    const double tol = std::fmax(std::fabs(est) * rel, 1e-300);
    return adapt(f, a, b, panel(f, a, b), tol / std::fabs(b - a), 0);
}

// I(a) = int_0^a da' / (a' E)^3.  With a' = s^2: (a'E)^3 = s^-3 (Om + OL s^6)^{3/2},
// so I(a) = int_0^{sqrt a} 2 s^4 / (Om + OL s^6)^{3/2} ds, a smooth integrand.
double growth_integral(const Cosmo& c, double a) {
    const double om = c.omega_m, ol = 1.0 - c.omega_m;
    auto f = [om, ol](double s) {
        const double s2 = s * s;
        const double q = om + ol * s2 * s2 * s2;
        return 2.0 * s2 * s2 / (q * std::sqrt(q));
    };
    return integrate(f, 0.0, std::sqrt(a));
}

double tophat(double x) {
    if (std::fabs(x) < 1e-3) return 1.0 - x * x / 10.0;
    return 3.0 * (std::sin(x) - x * std::cos(x)) / (x * x * x);
}

}  // namespace

double E(const Cosmo& c, double a) { return std::sqrt(c.omega_m / (a * a * a) + 1.0 - c.omega_m); }

double omega_m_a(const Cosmo& c, double a) {
    const double e = E(c, a);
    return c.omega_m / (a * a * a) / (e * e);
}

double conformal_hubble(const Cosmo& c, double a) { return a * E(c, a) / kCLight; }

double growth_D(const Cosmo& c, double a) {
    const double d = 2.5 * c.omega_m * E(c, a) * growth_integral(c, a);
    const double d1 = 2.5 * c.omega_m * E(c, 1.0) * growth_integral(c, 1.0);
    return d / d1;
}

double growth_f(const Cosmo& c, double a) {
    const double e = E(c, a);
    const double dlne = -1.5 * c.omega_m / (a * a * a) / (e * e);
    return dlne + 1.0 / (a * a * e * e * e * growth_integral(c, a));
}

double kick_integral(const Cosmo& c, double a0, double a1) {
    return integrate([&c](double a) { return 1.0 / (a * a * E(c, a)); }, a0, a1);
}

double drift_integral(const Cosmo& c, double a0, double a1) {
    return integrate([&c](double a) { return 1.0 / (a * a * a * E(c, a)); }, a0, a1);
}

double growth_p(const Cosmo& c, double a) { return a * a * E(c, a) * growth_f(c, a) * growth_D(c, a); }

// p goes from growth_p(a0) Psi to growth_p(a1) Psi under the kick K g with g = (3/2) Om D(a_force) Psi.
double kick_growth(const Cosmo& c, double a0, double a1, double a_force) {
    return (growth_p(c, a1) - growth_p(c, a0)) / (1.5 * c.omega_m * growth_D(c, a_force));
}

// x goes from D(a0) Psi to D(a1) Psi under the drift F p with p = growth_p(a_mom) Psi.
double drift_growth(const Cosmo& c, double a0, double a1, double a_mom) {
    return (growth_D(c, a1) - growth_D(c, a0)) / growth_p(c, a_mom);
}

double transfer_eh_nowiggle(const Cosmo& c, double k) {
    // Eisenstein & Hu (1998), Eqs. 26 and 28-31.
    const double omh2 = c.omega_m * c.h * c.h, obh2 = c.omega_b * c.h * c.h;
    const double theta = c.t_cmb / 2.7;
    const double fb = c.omega_b / c.omega_m;
    const double s = 44.5 * std::log(9.83 / omh2) / std::sqrt(1.0 + 10.0 * std::pow(obh2, 0.75));
    const double alpha = 1.0 - 0.328 * std::log(431.0 * omh2) * fb + 0.38 * std::log(22.3 * omh2) * fb * fb;
    const double ks = 0.43 * k * c.h * s;
    const double gam = c.omega_m * c.h * (alpha + (1.0 - alpha) / (1.0 + ks * ks * ks * ks));
    const double q = k * theta * theta / gam;
    const double L0 = std::log(2.0 * M_E + 1.8 * q);
    const double C0 = 14.2 + 731.0 / (1.0 + 62.5 * q);
    return L0 / (L0 + C0 * q * q);
}

void normalise_sigma8(Cosmo& c) {
    const double R = 8.0;
    auto f = [&c, R](double lnk) {
        const double k = std::exp(lnk);
        const double t = transfer_eh_nowiggle(c, k);
        const double w = tophat(k * R);
        return k * k * k * std::pow(k, c.n_s) * t * t * w * w / (2.0 * M_PI * M_PI);
    };
    const double s2 = integrate(f, std::log(1e-7), std::log(1e3), 1e-13);
    c.amp = c.sigma8 * c.sigma8 / s2;
}

double power_linear(const Cosmo& c, double k) {
    const double t = transfer_eh_nowiggle(c, k);
    return c.amp * std::pow(k, c.n_s) * t * t;
}

}  // namespace pmhost
