/*
 * quadrature.cpp -- Gauss-Hermite velocity sets for the library (Sec. 2.1).
 *
 * 1-D abscissae are the roots of the probabilists' Hermite polynomial He_n
 * (chi^(n) of Eq. (hermipol) in one dimension) in closed form:
 *   n = 3: He_3 = x^3 - 3x                  -> 0, +/- sqrt(3)
 *   n = 4: He_4 = x^4 - 6x^2 + 3            -> x^2 = 3 -/+ sqrt(6)
 *   n = 6: He_6 = x^6 - 15x^4 + 45x^2 - 15  -> x^2 = z, z^3 - 15 z^2 + 45 z - 15 = 0,
 *          solved with z = t + 5, t^3 - 30 t - 40 = 0 by the trigonometric
 *          (three real roots) formula.
 * Weights use the Christoffel-number form of a Gauss rule,
 *   w = 1 / sum_{k<n} He_k(x)^2 / k!,
 * which equals the n! / [n He_{n-1}(x)]^2 of Eq. (weight) at the roots. 2-D sets follow
 * the product rule: alpha = iy * n + ix.
 */
#include <cmath>

namespace lbq {

static double he(int n, double x)
{
    double a = 1.0, b = x;
    if (n == 0) return a;
    for (int k = 1; k < n; ++k) {
        double c = x * b - k * a;
        a = b;
        b = c;
    }
    return b;
}

/* Ascending abscissae and weights of the n-point rule, n in {3, 4, 6}; returns n or -1. */
int gauss_hermite_1d(int n, double *x, double *w)
{
    if (n == 3) {
        const double r = std::sqrt(3.0);
        x[0] = -r; x[1] = 0.0; x[2] = r;
    } else if (n == 4) {
        const double s6 = std::sqrt(6.0);
        const double a = std::sqrt(3.0 - s6), b = std::sqrt(3.0 + s6);
        x[0] = -b; x[1] = -a; x[2] = a; x[3] = b;
    } else if (n == 6) {
        const double pi = std::acos(-1.0);
        const double m = 2.0 * std::sqrt(10.0);
        const double phi = std::acos(2.0 / std::sqrt(10.0)) / 3.0;
        double z[3];
        for (int k = 0; k < 3; ++k) z[k] = 5.0 + m * std::cos(phi - 2.0 * pi * k / 3.0);
        /* ascending z */
        for (int i = 0; i < 3; ++i)
            for (int j = i + 1; j < 3; ++j)
                if (z[j] < z[i]) { double t = z[i]; z[i] = z[j]; z[j] = t; }
        for (int k = 0; k < 3; ++k) {
            x[2 - k] = -std::sqrt(z[k]);
            x[3 + k] = std::sqrt(z[k]);
        }
    } else {
        return -1;
    }
    for (int i = 0; i < n; ++i) {
        double s = 0.0, fact = 1.0;
        for (int k = 0; k < n; ++k) {
            if (k > 0) fact *= k;
            const double h = he(k, x[i]);
            s += h * h / fact;
        }
        w[i] = 1.0 / s;
    }
    return n;
}

/* Product set of q = n * n populations; returns q or -1. */
int velocity_set(int q, double *cx, double *cy, double *w)
{
    int n = q == 9 ? 3 : q == 16 ? 4 : q == 36 ? 6 : 0;
    double x[6], w1[6];
    if (n == 0 || gauss_hermite_1d(n, x, w1) != n) return -1;
    for (int iy = 0; iy < n; ++iy)
        for (int ix = 0; ix < n; ++ix) {
            const int a = iy * n + ix;
            cx[a] = x[ix];
            cy[a] = x[iy];
            w[a] = w1[ix] * w1[iy];
        }
    return q;
}

}  // namespace lbq
