/*
 * Scalar-generic body of the oracle's harmonic evaluator and quadrature
 * moments.  TEST INFRASTRUCTURE ONLY: this file is included twice by
 * q2x_oracle.c, once with S = double and once with S = double complex (the
 * complex-step variant).  Nothing here is shared with the CUDA path.
 *
 * The including file defines:
 *   S        scalar type
 *   FN(x)    name mangling (x##_r or x##_c)
 *   SQRT(x)  square root for S
 *   IS_REAL  1 for the real variant
 */

/* Regular solid harmonics R_n^m(x,y,z) of Eq. (bas1), evaluated for all
 * 0 <= n <= p, -n <= m <= n, WITHOUT the paper's recursions: the Cartesian form
 *   r^n P_n^|m|(cos t) e^{+-i|m|phi} = Pi_n^|m|(z, r^2) * (x +- i y)^|m|
 * with the Condon-Shortley sign of Eq. (bas2) in Pi_m^m = (-1)^m (2m-1)!!, and
 * the textbook three-term recurrence in n for the associated Legendre part:
 *   (n-m) Pi_n^m = (2n-1) z Pi_{n-1}^m - (n+m-1) r^2 Pi_{n-2}^m.
 * (x + i y)^m = C_m + i S_m is carried as two real polynomials, so Re R and
 * Im R are real polynomials in (x, y, z) and the complex-step variant
 * differentiates them exactly.
 * Output: re[k], im[k] with k = n*n + n + m. */
static void FN(rnm)(S x, S y, S z, int p, S* re, S* im)
{
    S C[ORACLE_PMAX + 2], Sm[ORACLE_PMAX + 2];
    C[0] = 1.0;
    Sm[0] = 0.0;
    for (int m = 1; m <= p; ++m) {
        C[m] = x * C[m - 1] - y * Sm[m - 1];
        Sm[m] = x * Sm[m - 1] + y * C[m - 1];
    }
    S r2 = x * x + y * y + z * z;
    for (int m = 0; m <= p; ++m) {
        double dfact = 1.0; /* (2m-1)!! */
        for (int k = 2 * m - 1; k > 1; k -= 2) dfact *= (double)k;
        if (m & 1) dfact = -dfact;
        S pim1 = 0.0, pim2 = 0.0;
        for (int n = m; n <= p; ++n) {
            S pi;
            if (n == m)
                pi = dfact;
            else if (n == m + 1)
                pi = (double)(2 * m + 1) * z * pim1;
            else
                pi = ((double)(2 * n - 1) * z * pim1 - (double)(n + m - 1) * r2 * pim2) /
                     (double)(n - m);
            pim2 = pim1;
            pim1 = pi;
            /* R_n^{+-m} = (-1)^n i^m / (n+m)! * pi * (C_m +- i S_m) */
            double f = ((n & 1) ? -1.0 : 1.0) / oracle_fact(n + m);
            S a = f * pi * C[m];
            S b = f * pi * Sm[m];
            S pr, pim, nr, nim; /* R^{+m} = pr + i pim ; R^{-m} = nr + i nim */
            switch (m & 3) {
            case 0: pr = a;  pim = b;  nr = a;  nim = -b; break;
            case 1: pr = -b; pim = a;  nr = b;  nim = a;  break;
            case 2: pr = -a; pim = -b; nr = -a; nim = b;  break;
            default: pr = b; pim = -a; nr = -b; nim = -a; break;
            }
            int k0 = n * n + n;
            re[k0 + m] = pr;
            im[k0 + m] = pim;
            if (m > 0) {
                re[k0 - m] = nr;
                im[k0 - m] = nim;
            }
        }
    }
}

/* Singular solid harmonics S_n^m of Eq. (bas1):
 *   S_n^m = i^{-|m|} (n-|m|)! r^{-n-1} P_n^|m|(cos t) e^{i m phi},
 * built from the same Cartesian Legendre part divided by r^{2n+1}. */
static void __attribute__((unused)) FN(snm)(S x, S y, S z, int p, S* re, S* im)
{
    S C[ORACLE_PMAX + 2], Sm[ORACLE_PMAX + 2];
    C[0] = 1.0;
    Sm[0] = 0.0;
    for (int m = 1; m <= p; ++m) {
        C[m] = x * C[m - 1] - y * Sm[m - 1];
        Sm[m] = x * Sm[m - 1] + y * C[m - 1];
    }
    S r2 = x * x + y * y + z * z;
    S rinv = 1.0 / SQRT(r2);
    for (int m = 0; m <= p; ++m) {
        double dfact = 1.0;
        for (int k = 2 * m - 1; k > 1; k -= 2) dfact *= (double)k;
        if (m & 1) dfact = -dfact;
        S pim1 = 0.0, pim2 = 0.0;
        for (int n = m; n <= p; ++n) {
            S pi;
            if (n == m)
                pi = dfact;
            else if (n == m + 1)
                pi = (double)(2 * m + 1) * z * pim1;
            else
                pi = ((double)(2 * n - 1) * z * pim1 - (double)(n + m - 1) * r2 * pim2) /
                     (double)(n - m);
            pim2 = pim1;
            pim1 = pi;
            S rp = rinv; /* r^{-(2n+1)} */
            for (int k = 0; k < 2 * n; ++k) rp *= rinv;
            S f = oracle_fact(n - m) * pi * rp;
            S a = f * C[m];
            S b = f * Sm[m];
            /* i^{-m} (a +- i b) */
            S pr, pim, nr, nim;
            switch (m & 3) {
            case 0: pr = a;  pim = b;  nr = a;  nim = -b; break;
            case 1: pr = b;  pim = -a; nr = -b; nim = -a; break;
            case 2: pr = -a; pim = -b; nr = -a; nim = b;  break;
            default: pr = -b; pim = a; nr = b;  nim = a;  break;
            }
            int k0 = n * n + n;
            re[k0 + m] = pr;
            im[k0 + m] = pim;
            if (m > 0) {
                re[k0 - m] = nr;
                im[k0 - m] = nim;
            }
        }
    }
}

/* Moments of ONE element about centre c by collapsed Gauss-Legendre product
 * quadrature (the paper's own comparison method, Sec. 4.2.1), exact for the
 * polynomial integrands when nq >= (p+3)/2.
 *
 * Element parametrisation of Eqs. (map1)-(map3): r = x1 + Ru u (+ Rv v (+ Rw w)),
 * Jacobian of Eq. (map4): |Ru| (segment), |Ru x Rv| (triangle),
 * |(Ru x Rv).Rw| (tetrahedron).
 * Collapsed coordinates: triangle u = s, v = (1-s) t, dudv = (1-s) ds dt;
 * tetrahedron u = s, v = (1-s) t, w = (1-s)(1-t) r, dudvdw = (1-s)^2 (1-t).
 *
 * Density: constant sig[0], or linear sig[0]*(1-u-v) + sig[1]*u + sig[2]*v
 * (triangle only; vertex k carries sig[k-1]).
 *
 * Output (packed, k = n*n+n+m), per norm:
 *   ORACLE_NORM_COEFF : F_n^m = (1/4pi)(-1)^n int sig R_n^{-m}(y-c)       Eq. (bas4)
 *                       double layer: (1/4pi)(-1)^n int sig n.grad R_n^{-m}
 *   ORACLE_NORM_MOMENT: int sig R_n^m(y-c)   (double layer: int sig n.grad R_n^m)
 *   packed value: Re F_n^m at m >= 0, Im F_n^|m| at m < 0.
 * The double layer (real variant only) takes n.grad of each real polynomial by a
 * complex step of size h along the unit normal n = (Ru x Rv)/J. */
static int FN(element_moments)(int kind, int layer, int density, int norm, int p, int nq,
                               const S* X, const double* sig, const double* c, S* out)
{
    int np = (p + 1) * (p + 1);
    double gx[ORACLE_NQMAX], gw[ORACLE_NQMAX];
    if (nq < 1 || nq > ORACLE_NQMAX || p < 0 || p > ORACLE_PMAX) return -1;
    oracle_gauss_legendre(nq, gx, gw);

    S Ru[3], Rv[3], Rw[3];
    for (int d = 0; d < 3; ++d) {
        Ru[d] = X[3 + d] - X[d];
        Rv[d] = (kind >= 1) ? X[6 + d] - X[d] : 0.0;
        Rw[d] = (kind >= 2) ? X[9 + d] - X[d] : 0.0;
    }
    S J, nrm[3] = {0.0, 0.0, 0.0};
    (void)nrm;
    if (kind == 0) {
        J = SQRT(Ru[0] * Ru[0] + Ru[1] * Ru[1] + Ru[2] * Ru[2]);
    } else {
        S cr[3] = {Ru[1] * Rv[2] - Ru[2] * Rv[1], Ru[2] * Rv[0] - Ru[0] * Rv[2],
                   Ru[0] * Rv[1] - Ru[1] * Rv[0]};
        if (kind == 1) {
            J = SQRT(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
            for (int d = 0; d < 3; ++d) nrm[d] = cr[d] / J;
        } else {
            S det = cr[0] * Rw[0] + cr[1] * Rw[1] + cr[2] * Rw[2];
            J = (ORACLE_REAL_PART(det) < 0.0) ? -det : det;
        }
    }
    if (layer == 1 && kind != 1) return -2;
    if (density == 1 && kind != 1) return -3;

    S* acc = out;
    for (int k = 0; k < np; ++k) acc[k] = 0.0;
    S re[(ORACLE_PMAX + 1) * (ORACLE_PMAX + 1)], im[(ORACLE_PMAX + 1) * (ORACLE_PMAX + 1)];

    int ns = nq, nt = (kind >= 1) ? nq : 1, nr = (kind >= 2) ? nq : 1;
    for (int is = 0; is < ns; ++is)
        for (int it = 0; it < nt; ++it)
            for (int ir = 0; ir < nr; ++ir) {
                double u, v = 0.0, w = 0.0, wt;
                if (kind == 0) {
                    u = gx[is];
                    wt = gw[is];
                } else if (kind == 1) {
                    u = gx[is];
                    v = (1.0 - gx[is]) * gx[it];
                    wt = gw[is] * gw[it] * (1.0 - gx[is]);
                } else {
                    u = gx[is];
                    v = (1.0 - gx[is]) * gx[it];
                    w = (1.0 - gx[is]) * (1.0 - gx[it]) * gx[ir];
                    wt = gw[is] * gw[it] * gw[ir] * (1.0 - gx[is]) * (1.0 - gx[is]) *
                         (1.0 - gx[it]);
                }
                double dens = (density == 1)
                                  ? sig[0] * (1.0 - u - v) + sig[1] * u + sig[2] * v
                                  : sig[0];
                S y[3];
                for (int d = 0; d < 3; ++d)
                    y[d] = X[d] + Ru[d] * u + Rv[d] * v + Rw[d] * w - c[d];
                if (layer == 0) {
                    FN(rnm)(y[0], y[1], y[2], p, re, im);
                } else {
#if IS_REAL
                    /* n.grad of each real polynomial by complex step */
                    double complex yc[3], rc[(ORACLE_PMAX + 1) * (ORACLE_PMAX + 1)],
                        ic[(ORACLE_PMAX + 1) * (ORACLE_PMAX + 1)];
                    const double h = 1e-30;
                    for (int d = 0; d < 3; ++d) yc[d] = y[d] + I * h * nrm[d];
                    rnm_c(yc[0], yc[1], yc[2], p, rc, ic);
                    for (int k = 0; k < np; ++k) {
                        re[k] = cimag(rc[k]) / h;
                        im[k] = cimag(ic[k]) / h;
                    }
#else
                    return -4;
#endif
                }
                double f = wt * dens;
                for (int n = 0; n <= p; ++n) {
                    int k0 = n * n + n;
                    if (norm == ORACLE_NORM_COEFF) {
                        /* F_n^m = (1/4pi)(-1)^n int R_n^{-m}: read R at -m */
                        double sgn = ((n & 1) ? -1.0 : 1.0) / (4.0 * M_PI);
                        acc[k0] += sgn * f * re[k0];
                        for (int m = 1; m <= n; ++m) {
                            acc[k0 + m] += sgn * f * re[k0 - m]; /* Re F_n^m */
                            acc[k0 - m] += sgn * f * im[k0 - m]; /* Im F_n^m */
                        }
                    } else {
                        acc[k0] += f * re[k0];
                        for (int m = 1; m <= n; ++m) {
                            acc[k0 + m] += f * re[k0 + m];
                            acc[k0 - m] += f * im[k0 + m];
                        }
                    }
                }
            }
    for (int k = 0; k < np; ++k) acc[k] *= J;
    return 0;
}
