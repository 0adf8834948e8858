// q2x_evaluate.cu -- far-field evaluation of expansions at target points
// (the M2P step that consumes the Q2X / M2M coefficients).
//
// Eq. (bas3) expands the Green's function in S_n^m about r*, so a box whose
// coefficients are F_n^m (Eq. (bas4), COEFF norm) has the potential
//   phi(x) = sum_{n<=p} sum_{|m|<=n} F_n^m S_n^m(x - r*)
//          = sum_n [F_n^0 S_n^0 + 2 Re sum_{m>0} F_n^m S_n^m]   (Eq. (bas2.1)),
// and raw moments M_n^m (MOMENT norm) give phi = (1/4pi) sum (-1)^n M_n^{-m} S_n^m.
// S_n^m = i^{-m} (n-m)! r^{-2n-1} T_n^m for m >= 0 (Eq. (bas1)) with
// T_n^m = r^n P_n^m(cos theta) e^{i m phi}, the solid harmonic polynomial built
// by the associated-Legendre recurrences in Cartesian form:
//   T_m^m = (-1)^m (2m-1)!! (x + iy)^m,  T_{m+1}^m = (2m+1) z T_m^m,
//   (n - m) T_n^m = (2n-1) z T_{n-1}^m - (n+m-1) r^2 T_{n-2}^m.
// One thread per (target, list entry); the order loop is outer, so a thread
// holds two T values and needs no table.  FP64.
#include <cuda_runtime.h>

#include <cstdint>

#include "q2x.h"
#include "q2x_plan.h"

namespace q2x {

struct EvalArgs {
    int p, np, norm, accumulate;
    int64_t n_exp, n_tgt;
    const double* coef;    // [n_exp][np]
    const double* exp_c;   // SoA 3 x n_exp
    const double* tgt;     // SoA 3 x n_tgt
    const int64_t* tgt_off;  // [n_tgt + 1] CSR into exp_idx
    const int64_t* exp_idx;
    double* out;           // [n_tgt]
    unsigned* err;
};

// k! (exact as doubles for k <= 20) and 1/k, k = 0..20
struct FactTab {
    double v[Q2X_P_MAX + 1];
    double inv[Q2X_P_MAX + 1];
};
constexpr FactTab make_fact_tab()
{
    FactTab t{};
    double f = 1.0;
    for (int k = 0; k <= Q2X_P_MAX; ++k) {
        if (k > 0) f *= k;
        t.v[k] = f;
        t.inv[k] = k > 0 ? 1.0 / k : 0.0;
    }
    return t;
}
static __constant__ FactTab c_fact = make_fact_tab();

// Far-field value of one expansion at offset (x, y, z) from its centre.
__device__ double eval_one(const double* __restrict__ F, int p, int norm, double x, double y, double z)
{
    const double r2 = x * x + y * y + z * z;
    if (!(r2 > 0.0)) return 0.0;  // at the centre the series does not apply
    const double ir2 = 1.0 / r2;
    const double ir = sqrt(ir2);
    double total = 0.0;
    // (x + iy)^m (-1)^m (2m-1)!! = T_m^m, updated per order
    double tmr = 1.0, tmi = 0.0;
#pragma unroll 1
    for (int m = 0; m <= p; ++m) {
        if (m > 0) {  // T_m^m = -(2m-1) (x + iy) T_{m-1}^{m-1}
            const double f = -(double)(2 * m - 1);
            const double nr = f * (x * tmr - y * tmi);
            const double ni = f * (x * tmi + y * tmr);
            tmr = nr;
            tmi = ni;
        }
        // i^{-m} rotation of the order-m column
        double rot_r, rot_i;
        switch (m & 3) {
            case 0: rot_r = 1.0; rot_i = 0.0; break;
            case 1: rot_r = 0.0; rot_i = -1.0; break;
            case 2: rot_r = -1.0; rot_i = 0.0; break;
            default: rot_r = 0.0; rot_i = 1.0; break;
        }
        double t2r = 0.0, t2i = 0.0;  // T_{n-2}^m
        double t1r = tmr, t1i = tmi;  // T_{n-1}^m, starting at n = m
        // r^{-2n-1} at n = m
        double irp = ir;
        for (int j = 0; j < m; ++j) irp *= ir2;
        double col = 0.0;
#pragma unroll 1
        for (int n = m; n <= p; ++n) {
            double tr, ti;
            if (n == m) {
                tr = t1r;
                ti = t1i;
            } else {
                const double a = (double)(2 * n - 1), b = (double)(n + m - 1), inv = c_fact.inv[n - m];
                tr = (a * z * t1r - b * r2 * t2r) * inv;
                ti = (a * z * t1i - b * r2 * t2i) * inv;
                t2r = t1r;
                t2i = t1i;
                t1r = tr;
                t1i = ti;
                irp *= ir2;
            }
            // S_n^m = i^{-m} (n-m)! r^{-2n-1} T_n^m
            const double sc = c_fact.v[n - m] * irp;
            const double sr = sc * (rot_r * tr - rot_i * ti);
            const double si = sc * (rot_r * ti + rot_i * tr);
            // coefficient of (n, m): COEFF F_n^m; MOMENT (1/4pi)(-1)^n M_n^{-m} = ... (-1)^{n+m} conj(M_n^m)
            const int k0 = n * n + n;
            double cr = __ldg(F + k0 + m);
            double ci = m ? __ldg(F + k0 - m) : 0.0;
            if (norm != 0) {
                const double sg = (((n + m) & 1) ? -1.0 : 1.0) * 0.079577471545947667884;
                cr = sg * cr;
                ci = -sg * ci;
            }
            const double v = cr * sr - ci * si;  // Re(coef * S)
            col += (m == 0) ? v : 2.0 * v;
        }
        total += col;
    }
    return total;
}

__global__ void q2x_evaluate_kernel(const EvalArgs a)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.n_tgt) return;
    int64_t j0 = __ldg(a.tgt_off + t), j1 = __ldg(a.tgt_off + t + 1);
    if (j0 < 0 || j1 < j0) {
        atomicOr(a.err, 8u);
        j0 = j1 = 0;
    }
    const double x = __ldg(a.tgt + t), y = __ldg(a.tgt + a.n_tgt + t), z = __ldg(a.tgt + 2 * a.n_tgt + t);
    double acc = 0.0;
#pragma unroll 1
    for (int64_t j = j0; j < j1; ++j) {
        const int64_t e = __ldg(a.exp_idx + j);
        if (e < 0 || e >= a.n_exp) {
            atomicOr(a.err, 1u);
            continue;
        }
        acc += eval_one(a.coef + e * (int64_t)a.np, a.p, a.norm, x - __ldg(a.exp_c + e),
                        y - __ldg(a.exp_c + a.n_exp + e), z - __ldg(a.exp_c + 2 * a.n_exp + e));
    }
    a.out[t] = a.accumulate ? a.out[t] + acc : acc;
}

// ---------------------------------------------------------------- curl
// A value and its gradient (forward-mode derivative in x, y, z): the far-field
// recurrences above are rational in (x, y, z), so carrying gradients through
// them gives grad S_n^m exactly (to rounding), with no separate formulas.
struct D4 {
    double v, x, y, z;
};
__device__ __forceinline__ D4 d4(double v) { return D4{v, 0.0, 0.0, 0.0}; }
__device__ __forceinline__ D4 operator+(D4 a, D4 b) { return D4{a.v + b.v, a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ D4 operator-(D4 a, D4 b) { return D4{a.v - b.v, a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ D4 operator*(double s, D4 a) { return D4{s * a.v, s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ D4 operator*(D4 a, D4 b)
{
    return D4{a.v * b.v, fma(a.v, b.x, a.x * b.v), fma(a.v, b.y, a.y * b.v), fma(a.v, b.z, a.z * b.v)};
}

// Gradients of the three component series A_k(x) = sum F^(k)_n^m S_n^m(x - c)
// at offset (x, y, z): g[k] += grad A_k.  F3 holds the three packed rows of
// one expansion, `stride` apart (COEFF norm).
__device__ void grad_one(const double* __restrict__ F3, int64_t stride, int p, double x, double y, double z,
                         double g[3][3])
{
    const double r2v = x * x + y * y + z * z;
    if (!(r2v > 0.0)) return;
    const D4 X{x, 1.0, 0.0, 0.0}, Y{y, 0.0, 1.0, 0.0}, Z{z, 0.0, 0.0, 1.0};
    const D4 r2 = X * X + Y * Y + Z * Z;
    // 1/r^2 and 1/r with their gradients: d(1/r2) = -dr2 / r2^2, d(r^-1) = -(1/2) r^-3 dr2
    const double ir2v = 1.0 / r2v, irv = sqrt(ir2v);
    const D4 ir2{ir2v, -r2.x * ir2v * ir2v, -r2.y * ir2v * ir2v, -r2.z * ir2v * ir2v};
    const double c = -0.5 * irv * ir2v;
    const D4 ir{irv, c * r2.x, c * r2.y, c * r2.z};
    D4 tmr = d4(1.0), tmi = d4(0.0);
#pragma unroll 1
    for (int m = 0; m <= p; ++m) {
        if (m > 0) {
            const double f = -(double)(2 * m - 1);
            const D4 nr = f * (X * tmr - Y * tmi);
            const D4 ni = f * (X * tmi + Y * tmr);
            tmr = nr;
            tmi = ni;
        }
        double rot_r, rot_i;
        switch (m & 3) {
            case 0: rot_r = 1.0; rot_i = 0.0; break;
            case 1: rot_r = 0.0; rot_i = -1.0; break;
            case 2: rot_r = -1.0; rot_i = 0.0; break;
            default: rot_r = 0.0; rot_i = 1.0; break;
        }
        D4 t2r = d4(0.0), t2i = d4(0.0);
        D4 t1r = tmr, t1i = tmi;
        D4 irp = ir;
        for (int j = 0; j < m; ++j) irp = irp * ir2;
        const double w = m ? 2.0 : 1.0;
#pragma unroll 1
        for (int n = m; n <= p; ++n) {
            D4 tr, ti;
            if (n == m) {
                tr = t1r;
                ti = t1i;
            } else {
                const double a = (double)(2 * n - 1), b = (double)(n + m - 1), inv = c_fact.inv[n - m];
                tr = inv * (a * (Z * t1r) - b * (r2 * t2r));
                ti = inv * (a * (Z * t1i) - b * (r2 * t2i));
                t2r = t1r;
                t2i = t1i;
                t1r = tr;
                t1i = ti;
                irp = irp * ir2;
            }
            const D4 sc = c_fact.v[n - m] * irp;
            const D4 sr = sc * (rot_r * tr - rot_i * ti);
            const D4 si = sc * (rot_r * ti + rot_i * tr);
            const int k0 = n * n + n;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const double cr = __ldg(F3 + k * stride + k0 + m);
                const double ci = m ? __ldg(F3 + k * stride + k0 - m) : 0.0;
                g[k][0] += w * (cr * sr.x - ci * si.x);
                g[k][1] += w * (cr * sr.y - ci * si.y);
                g[k][2] += w * (cr * sr.z - ci * si.z);
            }
        }
    }
}

// H = curl A at each target (Eq. (st3)): expansions with three component rows.
__global__ void q2x_evaluate_curl_kernel(const EvalArgs a)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.n_tgt) return;
    int64_t j0 = __ldg(a.tgt_off + t), j1 = __ldg(a.tgt_off + t + 1);
    if (j0 < 0 || j1 < j0) {
        atomicOr(a.err, 8u);
        j0 = j1 = 0;
    }
    const double x = __ldg(a.tgt + t), y = __ldg(a.tgt + a.n_tgt + t), z = __ldg(a.tgt + 2 * a.n_tgt + t);
    double g[3][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};  // g[k][j] = d A_k / d x_j
#pragma unroll 1
    for (int64_t j = j0; j < j1; ++j) {
        const int64_t e = __ldg(a.exp_idx + j);
        if (e < 0 || e >= a.n_exp) {
            atomicOr(a.err, 1u);
            continue;
        }
        grad_one(a.coef + e * (int64_t)a.np, a.n_exp * (int64_t)a.np, a.p, x - __ldg(a.exp_c + e),
                 y - __ldg(a.exp_c + a.n_exp + e), z - __ldg(a.exp_c + 2 * a.n_exp + e), g);
    }
    const double h[3] = {g[2][1] - g[1][2], g[0][2] - g[2][0], g[1][0] - g[0][1]};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double* o = a.out + d * a.n_tgt + t;
        *o = a.accumulate ? *o + h[d] : h[d];
    }
}

}  // namespace q2x

extern "C" q2x_status q2x_evaluate_curl(q2x_plan_t plan, int p, int64_t n_exp, const double* coef3,
                                        const double* exp_c, int64_t n_tgt, const double* tgt,
                                        const int64_t* tgt_off, const int64_t* exp_idx, double* out3,
                                        int accumulate)
{
    if (!plan) return q2x_fail(nullptr, Q2X_ERR_ARG, "plan is NULL");
    if (plan->norm != 0) return q2x_fail(plan, Q2X_ERR_UNSUPPORTED, "curl evaluation needs the COEFF norm");
    if (p < 0 || p > plan->p_max) return q2x_fail(plan, Q2X_ERR_RANGE, "p = %d outside 0..%d", p, plan->p_max);
    if (n_exp < 0 || n_tgt < 0) return q2x_fail(plan, Q2X_ERR_ARG, "negative size");
    if (accumulate != 0 && accumulate != 1) return q2x_fail(plan, Q2X_ERR_ARG, "accumulate must be 0 or 1");
    if (n_tgt == 0) return Q2X_OK;
    if (!tgt || !tgt_off || !exp_idx || !out3) return q2x_fail(plan, Q2X_ERR_ARG, "NULL target array");
    if (n_exp > 0 && (!coef3 || !exp_c)) return q2x_fail(plan, Q2X_ERR_ARG, "NULL expansion array");
    cudaError_t e = cudaSetDevice(plan->device);
    if (e != cudaSuccess) return q2x_cuda_fail(plan, e, "cudaSetDevice");
    q2x::EvalArgs a;
    a.p = p;
    a.np = (p + 1) * (p + 1);
    a.norm = 0;
    a.accumulate = accumulate;
    a.n_exp = n_exp;
    a.n_tgt = n_tgt;
    a.coef = coef3;
    a.exp_c = exp_c;
    a.tgt = tgt;
    a.tgt_off = tgt_off;
    a.exp_idx = exp_idx;
    a.out = out3;
    a.err = plan->d_err;
    q2x::q2x_evaluate_curl_kernel<<<(unsigned)((n_tgt + 127) / 128), 128, 0, plan->stream>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return q2x_cuda_fail(plan, e, "q2x_evaluate_curl_kernel launch");
    plan->launches += 1;
    return Q2X_OK;
}

extern "C" q2x_status q2x_evaluate(q2x_plan_t plan, int p, int64_t n_exp, const double* coef, const double* exp_c,
                                   int64_t n_tgt, const double* tgt, const int64_t* tgt_off,
                                   const int64_t* exp_idx, double* out, int accumulate)
{
    if (!plan) return q2x_fail(nullptr, Q2X_ERR_ARG, "plan is NULL");
    if (p < 0 || p > plan->p_max) return q2x_fail(plan, Q2X_ERR_RANGE, "p = %d outside 0..%d", p, plan->p_max);
    if (n_exp < 0 || n_tgt < 0) return q2x_fail(plan, Q2X_ERR_ARG, "negative size");
    if (accumulate != 0 && accumulate != 1) return q2x_fail(plan, Q2X_ERR_ARG, "accumulate must be 0 or 1");
    if (n_tgt == 0) return Q2X_OK;
    if (!tgt || !tgt_off || !exp_idx || !out) return q2x_fail(plan, Q2X_ERR_ARG, "NULL target array");
    if (n_exp > 0 && (!coef || !exp_c)) return q2x_fail(plan, Q2X_ERR_ARG, "NULL expansion array");
    cudaError_t e = cudaSetDevice(plan->device);
    if (e != cudaSuccess) return q2x_cuda_fail(plan, e, "cudaSetDevice");
    q2x::EvalArgs a;
    a.p = p;
    a.np = (p + 1) * (p + 1);
    a.norm = plan->norm;
    a.accumulate = accumulate;
    a.n_exp = n_exp;
    a.n_tgt = n_tgt;
    a.coef = coef;
    a.exp_c = exp_c;
    a.tgt = tgt;
    a.tgt_off = tgt_off;
    a.exp_idx = exp_idx;
    a.out = out;
    a.err = plan->d_err;
    const int64_t grid = (n_tgt + 127) / 128;
    q2x::q2x_evaluate_kernel<<<(unsigned)grid, 128, 0, plan->stream>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return q2x_cuda_fail(plan, e, "q2x_evaluate_kernel launch");
    plan->launches += 1;
    return Q2X_OK;
}
