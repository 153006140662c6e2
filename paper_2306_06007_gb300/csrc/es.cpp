// "Exponential of semicircle" (ES) spreading kernel: parameters and Fourier transform.
//
// The paper uses the ES pulse of Barnett, Magland and af Klinteberg (2019) through
// its type-3 engine (footnote on spreading kernels, Sect. 2.1); the kernel is
//   phi(z) = exp(beta (sqrt(1 - (2 z / w)^2) - 1)),  |z| <= w/2 grid cells,
// with width w ~ number of digits of accuracy per dimension.
#include <cmath>
#include <stdexcept>

#include "hvox_internal.h"

namespace hvox {

int es_width(double eps, double sigma) {
    const double wd = std::ceil(std::log(1.0 / eps) / (M_PI * std::sqrt(1.0 - 1.0 / sigma)));
    return (int)std::min(1e6, std::max(2.0, wd));
}

ESKernel es_params(double eps, double sigma) {
    if (!(eps > 0.0) || !(sigma > 1.0)) fail(HVOX_EINVAL, "es_params: need eps > 0 and sigma > 1");
    ESKernel k;
    k.w = es_width(eps, sigma);
    if (k.w > 16) fail(HVOX_EUNSUPPORTED, "es_params: tolerance needs a kernel wider than 16 cells");
    k.beta = 0.97 * M_PI * k.w * (1.0 - 1.0 / (2.0 * sigma));
    return k;
}

ESKernel es_with_width(int w, double sigma) {
    if (w < 2 || w > 16 || !(sigma > 1.0)) fail(HVOX_EINVAL, "es_with_width: need 2 <= w <= 16 and sigma > 1");
    ESKernel k;
    k.w = w;
    k.beta = 0.97 * M_PI * k.w * (1.0 - 1.0 / (2.0 * sigma));
    return k;
}

ESKernel es_params_within(double eps_tight, double eps, double sigma) {
    if (es_width(eps_tight, sigma) <= 16) return es_params(eps_tight, sigma);
    ESKernel k = es_params(eps, sigma);  // refuses tolerances beyond a 16-cell kernel
    k.w = 16;
    k.beta = 0.97 * M_PI * k.w * (1.0 - 1.0 / (2.0 * sigma));
    return k;
}

void gauss_legendre(int q, std::vector<double> &x, std::vector<double> &wt) {
    x.assign(q, 0.0);
    wt.assign(q, 0.0);
    for (int i = 0; i < q; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (q + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            // Legendre recurrence: (m+1) P_{m+1} = (2m+1) z P_m - m P_{m-1}
            double p0 = 1.0, p1 = z;
            for (int m = 1; m < q; ++m) {
                double p2 = ((2.0 * m + 1.0) * z * p1 - m * p0) / (m + 1.0);
                p0 = p1;
                p1 = p2;
            }
            dp = q * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int m = 1; m < q; ++m) {
            double p2 = ((2.0 * m + 1.0) * z * p1 - m * p0) / (m + 1.0);
            p0 = p1;
            p1 = p2;
        }
        dp = q * (z * p1 - p0) / (z * z - 1.0);
        x[i] = z;
        wt[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

int es_quad_nodes(const ESKernel &k) { return 3 * k.w + 32; }

// Nodes and weights of Phi(xi) = sum_m f_m cos(xi z_m). With z = (w/2) sin(theta) the
// integrand exp(beta (cos(theta) - 1)) cos(xi z) (w/2) cos(theta) is smooth on
// [-pi/2, pi/2], so Gauss-Legendre in theta converges geometrically.
void es_ft_nodes(const ESKernel &k, std::vector<double> &z, std::vector<double> &f) {
    std::vector<double> x, wt;
    int q = es_quad_nodes(k);
    gauss_legendre(q, x, wt);
    const double half = 0.5 * k.w;
    z.resize(q);
    f.resize(q);
    for (int m = 0; m < q; ++m) {
        double th = 0.5 * M_PI * x[m];
        z[m] = half * std::sin(th);
        f[m] = 0.5 * M_PI * wt[m] * half * std::cos(th) * std::exp(k.beta * (std::cos(th) - 1.0));
    }
}

void es_ft(const ESKernel &k, const double *xi, int64_t n, double *out) {
    std::vector<double> z, f;
    es_ft_nodes(k, z, f);
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (size_t m = 0; m < z.size(); ++m) s += f[m] * std::cos(xi[i] * z[m]);
        out[i] = s;
    }
}

// Chebyshev interpolant of 1/Phi(tau) on [0, tau_max] in u = 2 (tau/tau_max)^2 - 1, of the
// smallest even degree (8 .. 32) whose relative error on a fine check grid is <= tol.
void fit_inv_phi(const ESKernel &k, double tau_max, double tol, std::vector<double> &coef) {
    const int n_check = 2001;
    std::vector<double> tc(n_check), fc(n_check);
    for (int i = 0; i < n_check; ++i) tc[i] = tau_max * (double)i / (n_check - 1);
    es_ft(k, tc.data(), n_check, fc.data());
    std::vector<double> best;
    double best_err = INFINITY;
    for (int deg = 8; deg <= 32; deg += 2) {
        const int n = deg + 1;
        std::vector<double> tau(n), f(n), c(n, 0.0);
        for (int j = 0; j < n; ++j) {
            double u = std::cos(M_PI * (j + 0.5) / n);
            tau[j] = tau_max * std::sqrt(0.5 * (u + 1.0));
        }
        es_ft(k, tau.data(), n, f.data());
        for (int m = 0; m < n; ++m) {
            double sum = 0.0;
            for (int j = 0; j < n; ++j) sum += (1.0 / f[j]) * std::cos(m * M_PI * (j + 0.5) / n);
            c[m] = 2.0 * sum / n;
        }
        c[0] *= 0.5;
        double err = 0.0;
        for (int i = 0; i < n_check; ++i) {
            double u = 2.0 * (tc[i] / tau_max) * (tc[i] / tau_max) - 1.0;
            double b1 = 0, b2 = 0;
            for (int m = deg; m >= 1; --m) {
                double b0 = c[m] + 2.0 * u * b1 - b2;
                b2 = b1;
                b1 = b0;
            }
            double v = c[0] + u * b1 - b2;
            err = std::max(err, std::fabs(v * fc[i] - 1.0));
        }
        if (err < best_err) {
            best_err = err;
            best = c;
        }
        if (err <= tol) break;
    }
    coef = best;
}

}  // namespace hvox
