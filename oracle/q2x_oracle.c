/*
 * q2x_oracle.c -- FP64 CPU oracle for the Q2X moments.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is built and loaded by tests/,
 * by __graft_entry__.smoke() and by bench.py's CPU-baseline leg; the product
 * path (the CUDA library) never links, loads or calls it, and it shares no
 * code, header, table or constant with the CUDA kernels.
 *
 * What it computes is the plain definition, not the paper's recursions:
 * each coefficient of Eq. (bas4) is an integral of density x R_n^{-m}(y - c)
 * (or density x n.grad R_n^{-m} for the double layer) over the element,
 * done by collapsed Gauss-Legendre product quadrature (the paper's comparison
 * method of Sec. 4.2.1), which is exact for these polynomial integrands.
 * R_n^m is evaluated from its definition Eq. (bas1)-(bas2) in Cartesian form
 * (harmonics_body.h), never from Eq. (int2) or Lemmas 1-5.
 * Leaf sums (Eq. (st4)) use Neumaier-compensated FP64 summation over the
 * leaf's elements in index order.
 *
 * Every function here has pins in tests/test_oracle_*.py (closed forms,
 * symmetry, harmonicity, Gauss exactness, centroid relations, far-field
 * convergence, exact rational integration); none is "parity unpinned".
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PMAX 40
#define ORACLE_NQMAX 64
#define ORACLE_NORM_COEFF 0
#define ORACLE_NORM_MOMENT 1

static double oracle_fact(int n)
{
    double f = 1.0;
    for (int k = 2; k <= n; ++k) f *= (double)k;
    return f;
}

/* Gauss-Legendre rule with k nodes, mapped to [0,1]: Newton iteration on
 * P_k from the three-term recurrence (j P_j = (2j-1) t P_{j-1} - (j-1) P_{j-2}),
 * weights 2 / ((1 - t^2) P_k'(t)^2), halved by the map t -> (1+t)/2. */
int oracle_gauss_legendre(int k, double* x, double* w)
{
    if (k < 1 || k > ORACLE_NQMAX) return -1;
    for (int i = 0; i < k; ++i) {
        double t = cos(M_PI * ((double)i + 0.75) / ((double)k + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 200; ++it) {
            double p0 = 1.0, p1 = t;
            for (int j = 2; j <= k; ++j) {
                double p2 = ((2.0 * j - 1.0) * t * p1 - (j - 1.0) * p0) / (double)j;
                p0 = p1;
                p1 = p2;
            }
            if (k == 1) {
                p0 = 1.0;
                p1 = t;
            }
            dp = (double)k * (t * p1 - p0) / (t * t - 1.0);
            double dt = p1 / dp;
            t -= dt;
            if (fabs(dt) < 1e-17) break;
        }
        {
            double p0 = 1.0, p1 = t;
            for (int j = 2; j <= k; ++j) {
                double p2 = ((2.0 * j - 1.0) * t * p1 - (j - 1.0) * p0) / (double)j;
                p0 = p1;
                p1 = p2;
            }
            dp = (double)k * (t * p1 - p0) / (t * t - 1.0);
        }
        x[i] = 0.5 * (1.0 + t);
        w[i] = 1.0 / ((1.0 - t * t) * dp * dp);
    }
    return 0;
}

/* complex-step variant (S = double complex), must precede the real one */
#define S double complex
#define FN(x) x##_c
#define SQRT(x) csqrt(x)
#define IS_REAL 0
#define ORACLE_REAL_PART(x) creal(x)
#include "harmonics_body.h"
#undef S
#undef FN
#undef SQRT
#undef IS_REAL
#undef ORACLE_REAL_PART

/* real variant */
#define S double
#define FN(x) x##_r
#define SQRT(x) sqrt(x)
#define IS_REAL 1
#define ORACLE_REAL_PART(x) (x)
#include "harmonics_body.h"
#undef S
#undef FN
#undef SQRT
#undef IS_REAL
#undef ORACLE_REAL_PART

static int nvert_of(int kind) { return kind + 2; }

static void set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------- exports */

int oracle_rnm(double x, double y, double z, int p, double* re, double* im)
{
    if (p < 0 || p > ORACLE_PMAX) return -1;
    rnm_r(x, y, z, p, re, im);
    return 0;
}

int oracle_snm(double x, double y, double z, int p, double* re, double* im)
{
    if (p < 0 || p > ORACLE_PMAX) return -1;
    snm_r(x, y, z, p, re, im);
    return 0;
}

/* Element moments.
 *   kind     0 segment (2 vertices), 1 triangle (3), 2 tetrahedron (4)
 *   layer    0 single, 1 double (triangle only)
 *   density  0 constant: sigma[n_elem]; 1 linear: sigma[n_vert] (triangle only)
 *   vxyz     SoA 3 x n_vert (x block, y block, z block)
 *   idx      SoA nv x n_elem (vertex k of element e at idx[k*n_elem + e])
 *   leaf_off CSR int64[n_leaves+1] over the element order, or NULL: one
 *            "leaf" per element (then n_leaves == n_elem)
 *   leaf_c   SoA 3 x n_leaves expansion centres
 *   leaf_p   int32[n_leaves] per-leaf degree (<= p), or NULL (= p)
 *   out      n_leaves x (p+1)^2, zero above each leaf's degree
 *   nq       Gauss nodes per direction (<= 0: ceil((p+4)/2))
 * Returns 0, or a negative code for a bad argument or element. */
int oracle_moments(int kind, int layer, int density, int norm, int p, int nq, int64_t n_vert,
                   const double* vxyz, int64_t n_elem, const int32_t* idx, const double* sigma,
                   int64_t n_leaves, const int64_t* leaf_off, const double* leaf_c,
                   const int32_t* leaf_p, double* out, int nthreads)
{
    if (p < 0 || p > ORACLE_PMAX || kind < 0 || kind > 2) return -1;
    if (nq <= 0) nq = (p + 5) / 2;
    if (!leaf_off && n_leaves != n_elem) return -1;
    int np = (p + 1) * (p + 1);
    int nv = nvert_of(kind);
    int status = 0;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t L = 0; L < n_leaves; ++L) {
        double* o = out + L * np;
        double comp[(ORACLE_PMAX + 1) * (ORACLE_PMAX + 1)];
        double one[(ORACLE_PMAX + 1) * (ORACLE_PMAX + 1)];
        for (int k = 0; k < np; ++k) o[k] = comp[k] = 0.0;
        int64_t e0 = leaf_off ? leaf_off[L] : L;
        int64_t e1 = leaf_off ? leaf_off[L + 1] : L + 1;
        int pl = leaf_p ? leaf_p[L] : p;
        if (pl > p) pl = p;
        if (pl < 0) continue;
        double c[3] = {leaf_c[L], leaf_c[n_leaves + L], leaf_c[2 * n_leaves + L]};
        for (int64_t e = e0; e < e1; ++e) {
            double X[12];
            double sg[3];
            for (int k = 0; k < nv; ++k) {
                int64_t vk = idx[(int64_t)k * n_elem + e];
                for (int d = 0; d < 3; ++d) X[3 * k + d] = vxyz[(int64_t)d * n_vert + vk];
                if (density == 1 && k < 3) sg[k] = sigma[vk];
            }
            if (density == 0) sg[0] = sigma[e];
            int rc = element_moments_r(kind, layer, density, norm, pl, nq, X, sg, c, one);
            if (rc) {
                status = rc;
                continue;
            }
            int npl = (pl + 1) * (pl + 1);
            for (int k = 0; k < npl; ++k) {
                /* Neumaier summation */
                double t = o[k] + one[k];
                if (fabs(o[k]) >= fabs(one[k]))
                    comp[k] += (o[k] - t) + one[k];
                else
                    comp[k] += (one[k] - t) + o[k];
                o[k] = t;
            }
        }
        for (int k = 0; k < np; ++k) o[k] += comp[k];
    }
    return status;
}

/* Complex-step variant for derivative checks: per-element single-layer
 * moments with complex vertex coordinates (re + i*im), real densities and
 * real per-element centres elem_c (SoA 3 x n_elem). */
int oracle_moments_cs(int kind, int density, int norm, int p, int nq, int64_t n_vert,
                      const double* vre, const double* vim, int64_t n_elem, const int32_t* idx,
                      const double* sigma, const double* elem_c, double* out_re, double* out_im,
                      int nthreads)
{
    if (p < 0 || p > ORACLE_PMAX || kind < 0 || kind > 2) return -1;
    if (nq <= 0) nq = (p + 5) / 2;
    int np = (p + 1) * (p + 1);
    int nv = nvert_of(kind);
    int status = 0;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t e = 0; e < n_elem; ++e) {
        double complex X[12];
        double complex one[(ORACLE_PMAX + 1) * (ORACLE_PMAX + 1)];
        double sg[3];
        for (int k = 0; k < nv; ++k) {
            int64_t vk = idx[(int64_t)k * n_elem + e];
            for (int d = 0; d < 3; ++d)
                X[3 * k + d] = vre[(int64_t)d * n_vert + vk] + I * vim[(int64_t)d * n_vert + vk];
            if (density == 1 && k < 3) sg[k] = sigma[vk];
        }
        if (density == 0) sg[0] = sigma[e];
        double c[3] = {elem_c[e], elem_c[n_elem + e], elem_c[2 * n_elem + e]};
        int rc = element_moments_c(kind, 0, density, norm, p, nq, X, sg, c, one);
        if (rc) {
            status = rc;
            continue;
        }
        for (int k = 0; k < np; ++k) {
            out_re[e * np + k] = creal(one[k]);
            out_im[e * np + k] = cimag(one[k]);
        }
    }
    return status;
}

/* Single-layer potential of the elements [e0, e1) at targets r (AoS 3 x n_tgt):
 *   out[i] = (1/4pi) sum_e int_e sigma(y) / |r_i - y| dmu(y)
 * (the potential that the coefficients of Eq. (st4) expand, Eq. (bas3)), by
 * the collapsed Gauss-Legendre product rules of element_moments with nq
 * nodes per direction: accurate to rounding for targets well separated from
 * the elements, where the integrand is analytic on the element (near targets
 * need the graded rules of nearfield.py).  Density as in oracle_moments
 * (constant per element, or linear per vertex for triangles). */
int oracle_potential(int kind, int density, int nq, int64_t n_vert, const double* vxyz, int64_t n_elem,
                     const int32_t* idx, const double* sigma, int64_t e0, int64_t e1, int64_t n_tgt,
                     const double* tgt, double* out, int nthreads)
{
    if (kind < 0 || kind > 2 || nq < 1 || nq > ORACLE_NQMAX || e0 < 0 || e1 > n_elem || e0 > e1) return -1;
    if (density == 1 && kind != 1) return -3;
    double gx[ORACLE_NQMAX], gw[ORACLE_NQMAX];
    oracle_gauss_legendre(nq, gx, gw);
    int nv = nvert_of(kind);
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < n_tgt; ++i) {
        const double* r = tgt + 3 * i;
        double acc = 0.0, comp = 0.0;
        for (int64_t e = e0; e < e1; ++e) {
            double X[12], sg[3] = {0.0, 0.0, 0.0};
            for (int k = 0; k < nv; ++k) {
                int64_t vk = idx[(int64_t)k * n_elem + e];
                for (int d = 0; d < 3; ++d) X[3 * k + d] = vxyz[(int64_t)d * n_vert + vk];
                if (density == 1) sg[k] = sigma[vk];
            }
            if (density == 0) sg[0] = sigma[e];
            double Ru[3], Rv[3], Rw[3];
            for (int d = 0; d < 3; ++d) {
                Ru[d] = X[3 + d] - X[d];
                Rv[d] = (kind >= 1) ? X[6 + d] - X[d] : 0.0;
                Rw[d] = (kind >= 2) ? X[9 + d] - X[d] : 0.0;
            }
            double J;
            double cr[3] = {Ru[1] * Rv[2] - Ru[2] * Rv[1], Ru[2] * Rv[0] - Ru[0] * Rv[2],
                            Ru[0] * Rv[1] - Ru[1] * Rv[0]};
            if (kind == 0)
                J = sqrt(Ru[0] * Ru[0] + Ru[1] * Ru[1] + Ru[2] * Ru[2]);
            else if (kind == 1)
                J = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
            else
                J = fabs(cr[0] * Rw[0] + cr[1] * Rw[1] + cr[2] * Rw[2]);
            int ns = nq, nt = (kind >= 1) ? nq : 1, nr = (kind >= 2) ? nq : 1;
            double s = 0.0;
            for (int is = 0; is < ns; ++is)
                for (int it = 0; it < nt; ++it)
                    for (int ir = 0; ir < nr; ++ir) {
                        double u = gx[is], v = 0.0, w = 0.0, wt = gw[is];
                        if (kind == 1) {
                            v = (1.0 - u) * gx[it];
                            wt *= gw[it] * (1.0 - u);
                        } else if (kind == 2) {
                            v = (1.0 - u) * gx[it];
                            w = (1.0 - u) * (1.0 - gx[it]) * gx[ir];
                            wt *= gw[it] * gw[ir] * (1.0 - u) * (1.0 - u) * (1.0 - gx[it]);
                        }
                        double dens = (density == 1) ? sg[0] * (1.0 - u - v) + sg[1] * u + sg[2] * v : sg[0];
                        double dx = X[0] + Ru[0] * u + Rv[0] * v + Rw[0] * w - r[0];
                        double dy = X[1] + Ru[1] * u + Rv[1] * v + Rw[1] * w - r[1];
                        double dz = X[2] + Ru[2] * u + Rv[2] * v + Rw[2] * w - r[2];
                        s += wt * dens / sqrt(dx * dx + dy * dy + dz * dz);
                    }
            double term = s * J / (4.0 * M_PI);
            /* Neumaier summation over the elements */
            double t = acc + term;
            if (fabs(acc) >= fabs(term))
                comp += (acc - t) + term;
            else
                comp += (term - t) + acc;
            acc = t;
        }
        out[i] = acc + comp;
    }
    return 0;
}

/* Far-field series of Eq. (st4)/(bas3): phi(r) = sum_{n<=p} sum_m F_n^m
 * S_n^m(r - c) for packed COEFF-normalised coefficients F (the imaginary parts
 * of negative orders follow from F_n^{-m} = (-1)^m conj(F_n^m), Eq. (bas2.1)).
 * Returns Re phi in out[i] and Im phi (should vanish) in out_im[i]. */
int oracle_farfield(int p, const double* coef, const double* c, int64_t n_pts,
                    const double* pts, double* out, double* out_im)
{
    if (p < 0 || p > ORACLE_PMAX) return -1;
    double re[(ORACLE_PMAX + 1) * (ORACLE_PMAX + 1)], im[(ORACLE_PMAX + 1) * (ORACLE_PMAX + 1)];
    for (int64_t i = 0; i < n_pts; ++i) {
        snm_r(pts[3 * i] - c[0], pts[3 * i + 1] - c[1], pts[3 * i + 2] - c[2], p, re, im);
        double complex acc = 0.0;
        for (int n = 0; n <= p; ++n) {
            int k0 = n * n + n;
            for (int m = -n; m <= n; ++m) {
                int am = m < 0 ? -m : m;
                double complex F = coef[k0 + am] + (am ? I * coef[k0 - am] : 0.0);
                if (m < 0) F = ((am & 1) ? -1.0 : 1.0) * conj(F);
                acc += F * (re[k0 + m] + I * im[k0 + m]);
            }
        }
        out[i] = creal(acc);
        if (out_im) out_im[i] = cimag(acc);
    }
    return 0;
}
