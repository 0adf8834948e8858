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
// Since T_n^m = P_n T_m^m with a real sequence P_n, each order's column is
// summed as Re(i^{-m} T_m^m sum_n F_n^m U_n) with U_n = (n-m)! r^{-2n-1} P_n
// from a division-free real recurrence (see eval_one).  One thread per
// target, looping over the target's expansion list (CSR).  FP64.
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

// Recurrence constants of the scaled column sequence below: a_n = 2n - 1
// and c_{n,m} = (n + m - 1)(n - m - 1), read warp-uniformly.
struct EvalTab {
    double a[Q2X_P_MAX + 1];
    double c[Q2X_P_MAX + 1][Q2X_P_MAX + 1];  // [n][m]
};
constexpr EvalTab make_eval_tab()
{
    EvalTab t{};
    for (int n = 0; n <= Q2X_P_MAX; ++n) {
        t.a[n] = 2.0 * n - 1.0;
        for (int m = 0; m <= Q2X_P_MAX; ++m) t.c[n][m] = (double)((n + m - 1) * (n - m - 1));
    }
    return t;
}
static __constant__ EvalTab c_eval = make_eval_tab();

// Far-field value of one expansion at offset (x, y, z) from its centre.
// With T_n^m the Cartesian associated-Legendre polynomials (Eqs. (bas1)-
// (bas2)), T_n^m = P_n T_m^m for a real sequence P_n (P_m = 1, P_{m-1} = 0)
// that obeys the same three-term recurrence in n, so that
//   S_n^m = i^{-m} (n-m)! r^{-2n-1} T_n^m = i^{-m} T_m^m U_n,
//   U_n = (n-m)! r^{-2n-1} P_n,
//   U_n = a_n (z / r^2) U_{n-1} - c_{n,m} U_{n-2} / r^2,  U_m = r^{-2m-1},
// and the order-m column sums to Re(i^{-m} T_m^m sum_n F_n^m U_n): per term
// a real three-term step and two FMAs, no division.  For MOMENT
// coefficients, F_n^m = (1/4pi)(-1)^{n+m} conj(M_n^m); the sign (-1)^{n-m}
// is absorbed by running the recurrence with -z.
__device__ double eval_one(const double* __restrict__ F, int p, int norm, double x, double y, double z)
{
    const double r2 = x * x + y * y + z * z;
    if (!(r2 > 0.0)) return 0.0;  // at the centre the series does not apply
    const double rho2 = 1.0 / r2;
    const double zr = (norm != 0 ? -z : z) * rho2;
    double rp = sqrt(rho2);       // r^{-2m-1}
    double tmr = 1.0, tmi = 0.0;  // T_m^m = (-1)^m (2m-1)!! (x + iy)^m
    double total = 0.0;
#pragma unroll 1
    for (int m = 0; m <= p; ++m) {
        if (m > 0) {  // T_m^m = -(2m-1) (x + iy) T_{m-1}^{m-1}
            const double f = -c_eval.a[m];
            const double nr = f * (x * tmr - y * tmi);
            const double ni = f * (x * tmi + y * tmr);
            tmr = nr;
            tmi = ni;
            rp *= rho2;
        }
        const int km = m * m + m;
        double u1 = rp, u2 = 0.0;  // U_n, U_{n-1}
        double ar = __ldg(F + km + m) * u1;
        double ai = m ? __ldg(F + km - m) * u1 : 0.0;
#pragma unroll 1
        for (int n = m + 1; n <= p; ++n) {
            const double u = fma(c_eval.a[n] * zr, u1, -(c_eval.c[n][m] * rho2) * u2);
            u2 = u1;
            u1 = u;
            const int k0 = n * n + n;
            ar = fma(__ldg(F + k0 + m), u, ar);
            if (m) ai = fma(__ldg(F + k0 - m), u, ai);
        }
        if (norm != 0) {  // conj, 1/4pi
            ar *= 0.079577471545947667884;
            ai *= -0.079577471545947667884;
        }
        const double wr = tmr * ar - tmi * ai, wi = tmr * ai + tmi * ar;
        // Re(i^{-m} w)
        const double col = ((m & 3) == 0) ? wr : ((m & 3) == 1) ? wi : ((m & 3) == 2) ? -wr : -wi;
        total += m ? 2.0 * col : col;
    }
    return total;
}

__global__ void q2x_evaluate_kernel(const EvalArgs a)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.n_tgt) return;
    int64_t j0 = __ldg(a.tgt_off + t), j1 = __ldg(a.tgt_off + t + 1);
    if (j0 < 0 || j1 < j0 || (j1 > j0 && a.exp_idx == nullptr)) {  // an empty list set may pass NULL
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

__device__ __forceinline__ D4 fma4(double s, D4 a, D4 acc)
{
    return D4{fma(s, a.v, acc.v), fma(s, a.x, acc.x), fma(s, a.y, acc.y), fma(s, a.z, acc.z)};
}

// Gradients of the three component series A_k(x) = sum F^(k)_n^m S_n^m(x - c)
// at offset (x, y, z): g[k] += grad A_k.  F3 holds the three packed rows of
// one expansion, `stride` apart (COEFF norm).  The same column form as
// eval_one, S_n^m = i^{-m} T_m^m U_n, carried in value-and-gradient numbers.
__device__ void grad_one(const double* __restrict__ F3, int64_t stride, int p, double x, double y, double z,
                         double g[3][3])
{
    const double r2v = x * x + y * y + z * z;
    if (!(r2v > 0.0)) return;
    const D4 X{x, 1.0, 0.0, 0.0}, Y{y, 0.0, 1.0, 0.0}, Z{z, 0.0, 0.0, 1.0};
    // 1/r^2 and 1/r with their gradients: d(1/r^2) = -2 x / r^4, d(1/r) = -x / r^3
    const double ir2v = 1.0 / r2v, irv = sqrt(ir2v);
    const double c2 = -2.0 * ir2v * ir2v, c1 = -irv * ir2v;
    const D4 rho2{ir2v, c2 * x, c2 * y, c2 * z};
    const D4 zr = Z * rho2;
    D4 rp{irv, c1 * x, c1 * y, c1 * z};  // r^{-2m-1}
    D4 tmr = d4(1.0), tmi = d4(0.0);    // T_m^m
#pragma unroll 1
    for (int m = 0; m <= p; ++m) {
        if (m > 0) {
            const double f = -c_eval.a[m];
            const D4 nr = f * (X * tmr - Y * tmi);
            const D4 ni = f * (X * tmi + Y * tmr);
            tmr = nr;
            tmi = ni;
            rp = rp * rho2;
        }
        const int km = m * m + m;
        D4 u1 = rp, u2 = d4(0.0);
        D4 ar[3], ai[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            ar[k] = __ldg(F3 + k * stride + km + m) * u1;
            ai[k] = m ? __ldg(F3 + k * stride + km - m) * u1 : d4(0.0);
        }
#pragma unroll 1
        for (int n = m + 1; n <= p; ++n) {
            const D4 u = c_eval.a[n] * (zr * u1) - c_eval.c[n][m] * (rho2 * u2);
            u2 = u1;
            u1 = u;
            const int k0 = n * n + n;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                ar[k] = fma4(__ldg(F3 + k * stride + k0 + m), u, ar[k]);
                if (m) ai[k] = fma4(__ldg(F3 + k * stride + k0 - m), u, ai[k]);
            }
        }
        const double w = m ? 2.0 : 1.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            // Re(i^{-m} T_m^m A): only the part the order's rotation selects
            D4 col;
            if ((m & 1) == 0)
                col = tmr * ar[k] - tmi * ai[k];  // Re(T A)
            else
                col = tmr * ai[k] + tmi * ar[k];  // Im(T A)
            const double sg = ((m & 3) >= 2) ? -w : w;
            g[k][0] = fma(sg, col.x, g[k][0]);
            g[k][1] = fma(sg, col.y, g[k][1]);
            g[k][2] = fma(sg, col.z, g[k][2]);
        }
    }
}

// H = curl A at each target (Eq. (st3)): expansions with three component rows.
__global__ void q2x_evaluate_curl_kernel(const EvalArgs a)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.n_tgt) return;
    int64_t j0 = __ldg(a.tgt_off + t), j1 = __ldg(a.tgt_off + t + 1);
    if (j0 < 0 || j1 < j0 || (j1 > j0 && a.exp_idx == nullptr)) {  // an empty list set may pass NULL
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
    if (!tgt || !tgt_off || !out3) return q2x_fail(plan, Q2X_ERR_ARG, "NULL target array");
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
    if (!tgt || !tgt_off || !out) return q2x_fail(plan, Q2X_ERR_ARG, "NULL target array");
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
