/*
 * Oracle: plain CPU FP64 direct evaluation of the HVOX measurement sums.
 *
 * TEST INFRASTRUCTURE ONLY. Only tests, the smoke check and the benchmark's CPU
 * baseline may load this file's library. It shares no code with the GPU path.
 *
 * Definitions (Sect. 2, Eq. 2 and Eq. 3, with the 2*pi of a wavelength-unit
 * baseline written out and the direction named by its effect):
 *
 *   sky -> vis:  V_k = sum_n  a_n I_n exp(+isign * j * 2 pi <p_k, r_n>)
 *   vis -> sky:  I_n = a_n Re sum_k V_k exp(-isign * j * 2 pi <p_k, r_n>)
 *
 * r_n are pixel positions (unit vectors), p_k baselines in wavelengths, a_n the
 * tessellation weights (NULL means 1), isign = -1 reproduces Eq. 2. The second
 * sum is the exact adjoint of the first under the real inner product, with the
 * real part taken because the sky is real (Listing 1 forces a real adjoint).
 *
 * Accuracy measures (they are not part of the method):
 *  - the phase t = <p, r> (in turns, up to ~1e5) is formed as an unevaluated sum
 *    hi + lo with error-free products and sums (TwoProduct by fma, TwoSum), so the
 *    fraction t - rint(t) keeps ~1e-16 absolute accuracy;
 *  - cos/sin are taken of 2*pi*fraction, never of a large argument;
 *  - each output is a Neumaier-compensated sum.
 * Outputs are independent, so the loop over outputs runs under OpenMP.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static const double TWO_PI = 6.283185307179586476925286766559;

/* Error-free sum: a + b = s + e exactly (Knuth TwoSum). */
static inline void two_sum(double a, double b, double *s, double *e) {
    double x = a + b;
    double bv = x - a;
    double av = x - bv;
    *e = (a - av) + (b - bv);
    *s = x;
}

/* Fraction of the turn count <p, r> in [-0.5, 0.5], accurate to ~1e-16. */
static inline double phase_turns(const double *p, const double *r) {
    double hi = 0.0, lo = 0.0;
    for (int d = 0; d < 3; ++d) {
        double prod = p[d] * r[d];
        double perr = fma(p[d], r[d], -prod); /* exact: prod + perr = p*r */
        double s, e;
        two_sum(hi, prod, &s, &e);
        hi = s;
        lo += e + perr;
    }
    double whole = rint(hi);
    double f = (hi - whole) + lo; /* hi - whole is exact */
    return f - rint(f);
}

/* Neumaier compensated accumulator. */
typedef struct { double sum, comp; } acc_t;

static inline void acc_add(acc_t *a, double x) {
    double t = a->sum + x;
    if (fabs(a->sum) >= fabs(x))
        a->comp += (a->sum - t) + x;
    else
        a->comp += (x - t) + a->sum;
    a->sum = t;
}

static inline double acc_value(const acc_t *a) { return a->sum + a->comp; }

/* V_k for one k. */
static void sky2vis_one(int64_t k, const double *pix, const double *weight, const double *sky,
                        int64_t n_pix, const double *uvw, int isign, double *out2) {
    acc_t re = {0.0, 0.0}, im = {0.0, 0.0};
    const double *p = uvw + 3 * k;
    for (int64_t n = 0; n < n_pix; ++n) {
        double c = sky[n] * (weight ? weight[n] : 1.0);
        double ang = TWO_PI * phase_turns(p, pix + 3 * n);
        acc_add(&re, c * cos(ang));
        acc_add(&im, c * (isign > 0 ? sin(ang) : -sin(ang)));
    }
    out2[0] = acc_value(&re);
    out2[1] = acc_value(&im);
}

/* I_n for one n. */
static double vis2sky_one(int64_t n, const double *pix, const double *weight, const double *vis2,
                          int64_t n_vis, const double *uvw, int isign) {
    acc_t re = {0.0, 0.0};
    const double *r = pix + 3 * n;
    for (int64_t k = 0; k < n_vis; ++k) {
        double ang = TWO_PI * phase_turns(uvw + 3 * k, r);
        /* Re(V e^{-isign j ang}) = Vr cos(ang) + isign * Vi sin(ang) */
        double s = sin(ang);
        acc_add(&re, vis2[2 * k] * cos(ang));
        acc_add(&re, vis2[2 * k + 1] * (isign > 0 ? s : -s));
    }
    return (weight ? weight[n] : 1.0) * acc_value(&re);
}

/* Full sky -> vis: vis2 is (n_vis, 2) interleaved re/im. */
void oracle_sky2vis(const double *pix, const double *weight, const double *sky, int64_t n_pix,
                    const double *uvw, int64_t n_vis, int isign, double *vis2) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < n_vis; ++k)
        sky2vis_one(k, pix, weight, sky, n_pix, uvw, isign, vis2 + 2 * k);
}

/* Selected outputs only: vis2[2*s] for k = idx[s]. */
void oracle_sky2vis_sample(const double *pix, const double *weight, const double *sky, int64_t n_pix,
                           const double *uvw, const int64_t *idx, int64_t n_idx, int isign, double *vis2) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t s = 0; s < n_idx; ++s)
        sky2vis_one(idx[s], pix, weight, sky, n_pix, uvw, isign, vis2 + 2 * s);
}

void oracle_vis2sky(const double *pix, const double *weight, int64_t n_pix, const double *uvw,
                    const double *vis2, int64_t n_vis, int isign, double *sky) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t n = 0; n < n_pix; ++n)
        sky[n] = vis2sky_one(n, pix, weight, vis2, n_vis, uvw, isign);
}

void oracle_vis2sky_sample(const double *pix, const double *weight, const double *uvw, const double *vis2,
                           int64_t n_vis, const int64_t *idx, int64_t n_idx, int isign, double *sky) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t s = 0; s < n_idx; ++s)
        sky[s] = vis2sky_one(idx[s], pix, weight, vis2, n_vis, uvw, isign);
}

/* Phase fraction of single (p, r) pairs, exposed so that tests can pin the
 * large-argument reduction against exact rational arithmetic. */
void oracle_phase_turns(const double *uvw, const double *pix, int64_t n, double *out) {
    for (int64_t i = 0; i < n; ++i) out[i] = phase_turns(uvw + 3 * i, pix + 3 * i);
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
