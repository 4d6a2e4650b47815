// cosmo.h -- the Friedmann background on the host, in float64 (Sec. IV-A.2:
// the paper's run is LambdaCDM).  With H0 = 1, lengths in fine cells and
// p = a^2 dx/dt, the equations of motion in terms of a are
//   dp/da = (3 Omega_m / (8 pi rho_bar)) g / (a^2 E(a)),  dx/da = p / (a^3 E(a)),
// E(a) = sqrt(Omega_m a^-3 + Omega_k a^-2 + Omega_L), so a step's kick and
// drift factors are integrals of 1 / (a^2 E) and 1 / (a^3 E) over a.  The
// growing mode of the Zel'dovich initial conditions has D(a) proportional to
// E(a) int_0^a da' / (a' E)^3 (Heath 1977) and p = a^2 E f (x - q), f the
// logarithmic growth rate.  Einstein-de Sitter (Omega_m = 1) keeps its closed
// forms.  Integrals use composite Gauss-Legendre quadrature; the nodes come
// from Newton's iteration on the three-term Legendre recurrence.
#pragma once

#include <math.h>

namespace pmpm {

struct Background {
    bool eds = true;                 // Omega_m = 1, Omega_L = 0: closed forms
    double om = 1.0, ol = 0.0, ok = 0.0;
};

inline Background background_of(double omega_m, double omega_l) {
    Background b;
    if (omega_m > 0.0 && !(omega_m == 1.0 && omega_l == 0.0)) {
        b.eds = false;
        b.om = omega_m;
        b.ol = omega_l;
        b.ok = 1.0 - omega_m - omega_l;
    }
    return b;
}

inline double bg_E2(const Background& b, double a) {
    return b.om / (a * a * a) + b.ok / (a * a) + b.ol;
}

// 32-point Gauss-Legendre rule on [-1, 1]
struct GaussRule {
    static constexpr int kN = 32;
    double x[kN], w[kN];
    GaussRule() {
        const double pi = 3.141592653589793238462643383279502884;
        for (int i = 0; i < (kN + 1) / 2; ++i) {
            double z = cos(pi * (i + 0.75) / (kN + 0.5)), dp = 1.0;
            for (int it = 0; it < 100; ++it) {
                double p0 = 1.0, p1 = 0.0;            // P_j(z), P_{j-1}(z)
                for (int j = 1; j <= kN; ++j) {
                    const double p2 = p1;
                    p1 = p0;
                    p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
                }
                dp = kN * (z * p0 - p1) / (z * z - 1.0);
                const double dz = p0 / dp;
                z -= dz;
                if (fabs(dz) < 1e-16) break;
            }
            x[i] = -z;
            x[kN - 1 - i] = z;
            w[i] = w[kN - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
        }
    }
};

// int_lo^hi f over `panels` equal panels
template <class F>
double gauss_integrate(F f, double lo, double hi, int panels = 8) {
    static const GaussRule g;
    double sum = 0.0;
    const double h = (hi - lo) / panels;
    for (int p = 0; p < panels; ++p) {
        const double c = lo + (p + 0.5) * h, r = 0.5 * h;
        for (int i = 0; i < GaussRule::kN; ++i) sum += g.w[i] * r * f(c + r * g.x[i]);
    }
    return sum;
}

// int_lo^hi da / (a^2 E)
inline double bg_kick_integral(const Background& b, double lo, double hi) {
    if (b.eds) return 2.0 * (sqrt(hi) - sqrt(lo));
    return gauss_integrate([&](double a) { return 1.0 / (a * a * sqrt(bg_E2(b, a))); }, lo, hi);
}

// int_lo^hi da / (a^3 E)
inline double bg_drift_integral(const Background& b, double lo, double hi) {
    if (b.eds) return 2.0 * (1.0 / sqrt(lo) - 1.0 / sqrt(hi));
    return gauss_integrate([&](double a) { return 1.0 / (a * a * a * sqrt(bg_E2(b, a))); }, lo, hi);
}

// p / (x - q) of the growing mode at a: a^2 E f (sqrt(a) for EdS)
inline double bg_ic_momentum_factor(const Background& b, double a) {
    if (b.eds) return sqrt(a);
    const double E = sqrt(bg_E2(b, a));
    // I = int_0^a da' / (a' E)^3 with a' = a s^2: smooth in s at s = 0
    const double I = gauss_integrate(
        [&](double s) {
            const double ap = a * s * s;
            if (ap <= 0.0) return 0.0;
            const double ae = ap * sqrt(bg_E2(b, ap));
            return 2.0 * a * s / (ae * ae * ae);
        },
        0.0, 1.0);
    const double dlnE = (-1.5 * b.om / (a * a * a) - b.ok / (a * a)) / (E * E);
    const double f = dlnE + 1.0 / (a * a * E * E * E * I);
    return a * a * E * f;
}

}  // namespace pmpm
