// q2x_vjp.cuh -- adjoint of the triangle single-layer Q2X (constant density):
// given G = d loss / d coef (one row per leaf), accumulate d loss / d vertex
// coordinates and d loss / d density.
//
// With F_c = sigma J U_c(x1, x2, x3) the packed coefficients of one triangle
// (Eq. (bas10)), loss = sum_c G_c F_c, lambda_k the barycentric coordinate of
// vertex k and y = sum_k lambda_k x_k:
//   d loss / d x_k     = sigma [ (dJ/dx_k) sum_c G_c U_c + J sum_c G_c dU_c/dx_k ]
//   dU_c / dx_k        = (1/4pi)(-1)^n int_T lambda_k grad R_n^{-m}(y - r*) du dv
//   d loss / d sigma   = J sum_c G_c U_c
// The e_d component of int lambda_k grad R is a double-layer moment with unit
// "normal" e_d and linear density lambda_k (Eq. (bas8), Eq. (rec15)), so it is
// the stencil A_{e_d} applied to the lambda_k-weighted face row Iw^(k) of the
// linear-density chain one degree lower:
//   e_x: (b - a)/2 (m > 0), Re b (m = 0);  e_y: -(i/2)(a + b) (m > 0), Im b (m = 0);
//   e_z: -c  (a = x^{m-1}, b = x^{m+1}, c = x^m of that row).
// The chain carries q, j, i and, for k = 2, 3, E^(k) and Iw^(k) (sources
// (n+1) q and j); Iw^(1) = (n+3) i - Iw^(2) - Iw^(3) because sum_k lambda_k = 1.
// In the scaled frame y' = (y - r*)/rho, rho = 2^s: U_c = rho^n U'_c,
// dU_c/dx = rho^{n-1} dU'_c/dy', J = rho^2 J', so with G'_c = G_c rho^{n+1}
//   d loss / d x_k = sigma [ (dJ'/dy'_k) S_U + J' S_V,k ],  d loss / d sigma = rho J' S_U,
// S_U = sum_c G'_c U'_c, S_V,k = sum_c G'_c dU'_c/dy'_k.  q2x_vjp_weights folds
// rho^{n+1}, 1/(n+2)!, 1/4pi and the packing sign of each column into one
// weight per leaf and column.
#pragma once

#include "q2x_kernels.cuh"

namespace q2x {

struct VjpArgs {
    int64_t n_elem, n_vert;
    const double* vx;
    const double* vy;
    const double* vz;
    const int32_t* idx;
    const double* sigma;
    int64_t n_leaves;
    const int64_t* leaf_off;  // NULL: per-element
    const double* leaf_c;
    const double* leaf_rho;
    const int32_t* leaf_p;
    int p_max, np_max, norm;
    const void* w;            // [n_leaves][np_max] weights (T)
    double* grad_v;           // SoA 3 x n_vert, accumulated
    double* grad_sigma;       // n_elem or NULL, overwritten
    unsigned* err;
};

// weight of column c of leaf L: G_c * rho^{n+1} * sign(c) / (n+2)! (/ 4pi for COEFF)
template <typename T>
__global__ void q2x_vjp_weights(const double* __restrict__ G, const double* __restrict__ leaf_rho,
                                const int32_t* __restrict__ leaf_p, int64_t n_leaves, int np, int p_max,
                                int norm, T* __restrict__ w)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_leaves * np) return;
    const int64_t L = i / np;
    const int c = (int)(i - L * np);
    int n, m;
    col_nm(c, n, m);
    const int pL = leaf_p ? leaf_p[L] : p_max;
    const int s = leaf_rho ? scale_exponent(leaf_rho[L]) : 0;
    double v = 0.0;
    if (n <= pL && pL <= p_max) {
        v = G[i] * c_inv_fact_d[n + 2] * pow2d(s * (n + 1));
        if (norm == 0) v *= INV_4PI;
        if (column_negative(norm, n, m)) v = -v;
    }
    w[i] = (T)v;
}

template <typename T, int P>
__global__ void __launch_bounds__(128, 2) q2x_tri_vjp_kernel(const VjpArgs a)
{
    constexpr int NL = 7;  // q, j, i, E2, Iw2, E3, Iw3
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= a.n_elem) return;
    int64_t L = e;
    if (a.leaf_off) L = leaf_search(a.leaf_off, 0, a.n_leaves - 1, e);
    int pL = a.leaf_p ? __ldg(a.leaf_p + L) : a.p_max;
    unsigned errbits = 0;
    if (pL < 0 || pL > a.p_max) {
        errbits |= 4u;
        pL = -1;
    }
    const double cx = __ldg(a.leaf_c + L), cy = __ldg(a.leaf_c + a.n_leaves + L),
                 cz = __ldg(a.leaf_c + 2 * a.n_leaves + L);
    const int sexp = a.leaf_rho ? scale_exponent(__ldg(a.leaf_rho + L)) : 0;
    Frame<T, 3> F;
    load_frame<T, KIND_TRI, DENS_CONST>(a.vx, a.vy, a.vz, a.idx, a.sigma, a.n_elem, a.n_vert, e, true, cx, cy, cz,
                                        sexp, errbits, pL, F);
    if (errbits) atomicOr(a.err, errbits);
    if (pL < 0) {
        if (a.grad_sigma) a.grad_sigma[e] = 0.0;
        return;
    }
    const T sig = F.s1;
    // local vertex coordinates back from the stencil coefficients (x1: level i,
    // x2: level q, x3: level j); edges and the Jacobian from the frame (formed
    // from the exact splits of the FP64 inputs)
    const T x1[3] = {T(2) * F.LX[2], T(2) * F.LY[2], F.LZ[2]};
    const T x2[3] = {T(2) * F.LX[0], T(2) * F.LY[0], F.LZ[0]};
    const T x3[3] = {T(2) * F.LX[1], T(2) * F.LY[1], F.LZ[1]};
    const T eu[3] = {F.eu[0], F.eu[1], F.eu[2]};
    const T ev[3] = {F.ev[0], F.ev[1], F.ev[2]};
    const T J = F.J;
    const T nh[3] = {T(2) * F.XN, T(2) * F.YN, F.ZN};
    // dJ/dx2 = ev x n, dJ/dx3 = n x eu, dJ/dx1 = -(both)
    T dJ[3][3];
    dJ[1][0] = ev[1] * nh[2] - ev[2] * nh[1];
    dJ[1][1] = ev[2] * nh[0] - ev[0] * nh[2];
    dJ[1][2] = ev[0] * nh[1] - ev[1] * nh[0];
    dJ[2][0] = nh[1] * eu[2] - nh[2] * eu[1];
    dJ[2][1] = nh[2] * eu[0] - nh[0] * eu[2];
    dJ[2][2] = nh[0] * eu[1] - nh[1] * eu[0];
#pragma unroll
    for (int d = 0; d < 3; ++d) dJ[0][d] = -(dJ[1][d] + dJ[2][d]);

    const T* w = reinterpret_cast<const T*>(a.w) + L * (int64_t)a.np_max;
    // stencil vertex of each level
    const int vtx[NL] = {1, 2, 0, 2, 0, 2, 0};
    T LX[NL], LY[NL], LZ[NL];
    const T* xs[3] = {x1, x2, x3};
#pragma unroll
    for (int k = 0; k < NL; ++k) {
        LX[k] = T(0.5) * xs[vtx[k]][0];
        LY[k] = T(0.5) * xs[vtx[k]][1];
        LZ[k] = xs[vtx[k]][2];
    }
    T Rr[NL][P + 2], Ri[NL][P + 2];
#pragma unroll
    for (int k = 0; k < NL; ++k)
#pragma unroll
        for (int m = 0; m <= P + 1; ++m) Rr[k][m] = Ri[k][m] = T(0);
    T SU = T(0), SV[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) SV[k][0] = SV[k][1] = SV[k][2] = T(0);

#pragma unroll 1
    for (int n = 0; n <= pL; ++n) {
        const T c2 = T(n + 1);
        const T c3 = T(n + 3);
        const T* wn = w + n * n + n;        // weights of degree n, column (n, 0)
        const T* wn1 = w + (n + 1) * (n + 1) + (n + 1);  // degree n + 1
        const bool grad_next = (n + 1 <= pL);
        T pr[NL], pi[NL];
#pragma unroll
        for (int k = 0; k < NL; ++k) pr[k] = pi[k] = T(0);
#pragma unroll
        for (int m = 0; m <= P; ++m) {
            if (m <= n) {
                T nr[NL], ni[NL];
#pragma unroll
                for (int k = 0; k < NL; ++k) {
                    const T cr = Rr[k][m], ci = Ri[k][m];
                    const T br = Rr[k][m + 1], bi = Ri[k][m + 1];
                    T sr, si;
                    if (k == 0) {
                        sr = (n == 0 && m == 0) ? T(1) : T(0);
                        si = T(0);
                    } else if (k == 1 || k == 2) {
                        sr = nr[k - 1];  // j <- q, i <- j
                        si = ni[k - 1];
                    } else if (k == 3) {
                        sr = c2 * nr[0];  // E2 <- (n+1) q
                        si = c2 * ni[0];
                    } else if (k == 5) {
                        sr = nr[1];  // E3 <- j
                        si = ni[1];
                    } else {
                        sr = nr[k - 1];  // Iw2 <- E2, Iw3 <- E3
                        si = ni[k - 1];
                    }
                    T vr, vi;
                    if (m == 0) {
                        vr = fma(T(2) * LX[k], br, sr);
                        vr = fma(T(2) * LY[k], bi, vr);
                        vr = fma(-LZ[k], cr, vr);
                        vi = T(0);
                    } else {
                        vr = fma(LX[k], br - pr[k], sr);
                        vr = fma(LY[k], bi + pi[k], vr);
                        vr = fma(-LZ[k], cr, vr);
                        vi = fma(LX[k], bi - pi[k], si);
                        vi = fma(-LY[k], br + pr[k], vi);
                        vi = fma(-LZ[k], ci, vi);
                    }
                    nr[k] = vr;
                    ni[k] = vi;
                    pr[k] = cr;
                    pi[k] = ci;
                    Rr[k][m] = vr;
                    Ri[k][m] = vi;
                }
                // S_U: forward moment i^ of (n, m)
                {
                    const T re_c = (m & 1) ? ni[2] : nr[2];
                    const T im_c = (m & 1) ? nr[2] : ni[2];
                    SU = fma(__ldg(wn + m), re_c, SU);
                    if (m > 0) SU = fma(__ldg(wn - m), im_c, SU);
                }
            }
        }
        // S_V: degree n + 1 from the rows Iw^(k)_n (now in Rr/Ri), m = 0..n+1
        if (grad_next) {
#pragma unroll
            for (int m = 0; m <= P + 1; ++m) {
                if (m <= n + 1) {
                    const T wre = __ldg(wn1 + m);
                    const T wim = (m > 0) ? __ldg(wn1 - m) : T(0);
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        // row of Iw^(k): k = 1 derived, k = 2 level 4, k = 3 level 6
                        auto row = [&](int mm, T& r, T& i_) {
                            if (mm < 0 || mm > n) {
                                r = i_ = T(0);
                                return;
                            }
                            if (k == 0) {
                                r = c3 * Rr[2][mm] - Rr[4][mm] - Rr[6][mm];
                                i_ = c3 * Ri[2][mm] - Ri[4][mm] - Ri[6][mm];
                            } else {
                                const int lv = (k == 1) ? 4 : 6;
                                r = Rr[lv][mm];
                                i_ = Ri[lv][mm];
                            }
                        };
                        T ar, ai, br, bi, cr, ci;
                        row(m - 1, ar, ai);
                        row(m + 1, br, bi);
                        row(m, cr, ci);
                        T gx_r, gx_i, gy_r, gy_i, gz_r, gz_i;
                        if (m == 0) {
                            gx_r = br;
                            gy_r = bi;
                            gz_r = -cr;
                            gx_i = gy_i = gz_i = T(0);
                        } else {
                            gx_r = T(0.5) * (br - ar);
                            gx_i = T(0.5) * (bi - ai);
                            gy_r = T(0.5) * (bi + ai);
                            gy_i = T(-0.5) * (br + ar);
                            gz_r = -cr;
                            gz_i = -ci;
                        }
                        const T gr[3] = {gx_r, gy_r, gz_r};
                        const T gi[3] = {gx_i, gy_i, gz_i};
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            const T re_c = (m & 1) ? gi[d] : gr[d];
                            const T im_c = (m & 1) ? gr[d] : gi[d];
                            SV[k][d] = fma(wre, re_c, SV[k][d]);
                            if (m > 0) SV[k][d] = fma(wim, im_c, SV[k][d]);
                        }
                    }
                }
            }
        }
    }
    // scatter d loss / d x_k (FP64 accumulation)
    double* gv[3] = {a.grad_v, a.grad_v + a.n_vert, a.grad_v + 2 * a.n_vert};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int64_t v = __ldg(a.idx + (int64_t)k * a.n_elem + e);
        if (v < 0 || v >= a.n_vert) continue;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double g = (double)sig * ((double)dJ[k][d] * (double)SU + (double)J * (double)SV[k][d]);
            atomicAdd(gv[d] + v, g);
        }
    }
    if (a.grad_sigma) a.grad_sigma[e] = pow2d(sexp) * (double)J * (double)SU;
}

}  // namespace q2x
