// q2x_translate.cu -- translation of expansions to new centres (the
// multipole-to-multipole step fed by the Q2X leaf coefficients).
//
// With x = y - c_src and t = c_src - c_dst, the Taylor series of R_n^m in
// (xi, eta, z) and the derivative rules of Eq. (bas5) give the finite sum
//   R_n^m(x + t) = sum_{k=0..n} sum_{l=-k..k} R_k^l(t) R_{n-k}^{m-l}(x),
// so, term by term in Eq. (bas4), for every degree n <= p exactly:
//   MOMENT: M_n^m(dst) = sum_{k,l} R_k^l(t) M_{n-k}^{m-l}(src)
//   COEFF : F_n^m(dst) = sum_{k,l} (-1)^k R_k^l(t) F_{n-k}^{m+l}(src).
// R_k^l(t) comes from the point recursion of Eq. (rec2),
//   R_n^m = [i xi R_{n-1}^{m-1} + i eta R_{n-1}^{m+1} - z R_{n-1}^m] / n,
// xi = (x + iy)/2, eta = (x - iy)/2, R_0^0 = 1.
//
// Two kernels: one warp per source unpacks the source row to complex values
// in shared memory, builds R(t) there and writes the translated row (outputs
// n, m >= 0); one warp per destination then adds its sources' rows in source
// order (deterministic) and packs them.  FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "q2x.h"
#include "q2x_kernels.cuh"
#include "q2x_plan.h"

namespace q2x {

constexpr int TR_WARPS = 4;
constexpr int TR_MAX_OUT_PER_LANE = ((Q2X_P_MAX + 1) * (Q2X_P_MAX + 2) / 2 + 31) / 32;  // 8

struct TransArgs {
    int p, np, n_out, norm, accumulate;
    int wps, wps_log2;  // warps per source (a power of two; splits one translation's outputs)
    int64_t n_src, n_dst;
    const double* src_coef;
    const double* src_c;
    const int64_t* dst_off;
    const double* dst_c;
    double* dst_coef;
    double2* rows;  // [n_src][n_out] translated rows, complex (n, m >= 0)
    unsigned* err;
};

// degree and order of output o = n(n+1)/2 + m, 0 <= m <= n
__device__ __forceinline__ void out_nm(int o, int& n, int& m)
{
    n = (int)((sqrtf(8.0f * (float)o + 1.0f) - 1.0f) * 0.5f);
    if ((n + 1) * (n + 2) / 2 <= o) ++n;
    if (n * (n + 1) / 2 > o) --n;
    m = o - n * (n + 1) / 2;
}

// 1/n for the point recursion (n = 1..Q2X_P_MAX), no division in the kernel
struct InvN {
    double v[Q2X_P_MAX + 1];
};
constexpr InvN make_inv_n()
{
    InvN t{};
    for (int n = 1; n <= Q2X_P_MAX; ++n) t.v[n] = 1.0 / n;
    return t;
}
static __constant__ InvN c_inv_n = make_inv_n();

// wps warps per source: each builds the source's complex row and R(t) and
// writes the translated outputs o = sub*32 + lane + 32*wps*i of its share.
__global__ void __launch_bounds__(TR_WARPS * 32) q2x_translate_rows(const TransArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int64_t gw = (int64_t)blockIdx.x * TR_WARPS + wib;
    const int64_t s = gw >> a.wps_log2;
    const int sub = (int)(gw & (a.wps - 1));
    if (s >= a.n_src) return;
    const int p = a.p, np = a.np, n_out = a.n_out;
    double2* Fc = reinterpret_cast<double2*>(smem_raw) + (size_t)wib * 2 * np;
    double2* Rc = Fc + np;
    // destination of s: the range of dst_off holding it (clamped; ranges are
    // validated by the combine kernel)
    int64_t lo = 0, hi = a.n_dst - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (__ldg(a.dst_off + mid) <= s)
            lo = mid;
        else
            hi = mid - 1;
    }
    const int64_t d = lo;

    // ---- complex source row F[n][m], m = -n..n (Eq. (bas2.1) for m < 0)
    const double* src = a.src_coef + s * (int64_t)np;
    for (int k = lane; k < np; k += 32) {
        int n, m;
        col_nm(k, n, m);
        const int am = m < 0 ? -m : m;
        const int k0 = n * n + n;
        const double re = __ldg(src + k0 + am);
        const double im = am ? __ldg(src + k0 - am) : 0.0;
        if (m >= 0)
            Fc[k] = make_double2(re, im);
        else
            Fc[k] = (am & 1) ? make_double2(-re, im) : make_double2(re, -im);
    }
    // ---- R_k^l(t), t = c_src - c_dst, row by row
    const double tx = __ldg(a.src_c + s) - __ldg(a.dst_c + d);
    const double ty = __ldg(a.src_c + a.n_src + s) - __ldg(a.dst_c + a.n_dst + d);
    const double tz = __ldg(a.src_c + 2 * a.n_src + s) - __ldg(a.dst_c + 2 * a.n_dst + d);
    if (lane == 0) Rc[0] = make_double2(1.0, 0.0);
    __syncwarp();
    // i xi = (-y + i x)/2, i eta = (y + i x)/2
    const double ixr = -0.5 * ty, ixi = 0.5 * tx;
    const double ier = 0.5 * ty, iei = 0.5 * tx;
#pragma unroll 1
    for (int n = 1; n <= p; ++n) {
        const double inv = c_inv_n.v[n];
        const int kp = (n - 1) * (n - 1) + (n - 1);  // centre of row n-1
        for (int m = -n + lane; m <= n; m += 32) {
            double2 v = make_double2(0.0, 0.0);
            if (m - 1 >= -(n - 1) && m - 1 <= n - 1) {  // i xi R_{n-1}^{m-1}
                const double2 r = Rc[kp + m - 1];
                v.x += ixr * r.x - ixi * r.y;
                v.y += ixr * r.y + ixi * r.x;
            }
            if (m + 1 >= -(n - 1) && m + 1 <= n - 1) {  // i eta R_{n-1}^{m+1}
                const double2 r = Rc[kp + m + 1];
                v.x += ier * r.x - iei * r.y;
                v.y += ier * r.y + iei * r.x;
            }
            if (m >= -(n - 1) && m <= n - 1) {  // - z R_{n-1}^m
                const double2 r = Rc[kp + m];
                v.x -= tz * r.x;
                v.y -= tz * r.y;
            }
            Rc[n * n + n + m] = make_double2(v.x * inv, v.y * inv);
        }
        __syncwarp();
    }
    // ---- contraction: lane takes outputs lane, lane + 32, ... (mixed degrees)
    double2* row = a.rows + s * (int64_t)n_out;
    // F index step along l: +1 for COEFF (F_{n-k}^{m+l}), -1 for MOMENT (M_{n-k}^{m-l})
    const int fs = (a.norm == 0) ? 1 : -1;
    // outputs are visited in "snake" order over the lanes (lane L of a block
    // of 64 takes L and 63 - L), pairing costly high degrees with cheap low
    // ones; the warps of a source take interleaved blocks
    const int stride = 32 * a.wps;
#pragma unroll 1
    for (int q = sub * 32 + lane; q < n_out + stride; q += stride) {
        const int blk = q / 64, pos = q % 64;
        const int o = blk * 64 + ((pos < 32) ? pos : 95 - pos);  // pos 32..63 -> 63..32
        if (o >= n_out) continue;
        int n, m;
        out_nm(o, n, m);
        double ar = 0.0, ai = 0.0;
#pragma unroll 1
        for (int k = 0; k <= n; ++k) {
            const int nn = n - k;
            const int kr = k * k + k, kf = nn * nn + nn;
            // |m + fs l| <= n - k and |l| <= k
            const int l0 = (fs > 0) ? max(-k, -nn - m) : max(-k, m - nn);
            const int l1 = (fs > 0) ? min(k, nn - m) : min(k, m + nn);
            // two independent accumulator pairs (even / odd l)
            double sr0 = 0.0, si0 = 0.0, sr1 = 0.0, si1 = 0.0;
            int l = l0;
            for (; l + 1 <= l1; l += 2) {
                const double2 r0 = Rc[kr + l], f0 = Fc[kf + m + fs * l];
                const double2 r1 = Rc[kr + l + 1], f1 = Fc[kf + m + fs * (l + 1)];
                sr0 = fma(r0.x, f0.x, fma(-r0.y, f0.y, sr0));
                si0 = fma(r0.x, f0.y, fma(r0.y, f0.x, si0));
                sr1 = fma(r1.x, f1.x, fma(-r1.y, f1.y, sr1));
                si1 = fma(r1.x, f1.y, fma(r1.y, f1.x, si1));
            }
            if (l <= l1) {
                const double2 r0 = Rc[kr + l], f0 = Fc[kf + m + fs * l];
                sr0 = fma(r0.x, f0.x, fma(-r0.y, f0.y, sr0));
                si0 = fma(r0.x, f0.y, fma(r0.y, f0.x, si0));
            }
            double sr = sr0 + sr1, si = si0 + si1;
            if (fs > 0 && (k & 1)) {  // (-1)^k of the COEFF formula
                sr = -sr;
                si = -si;
            }
            ar += sr;
            ai += si;
        }
        row[o] = make_double2(ar, ai);
    }
}

// One warp per destination: its sources' rows added in source order, packed.
__global__ void q2x_translate_combine(const TransArgs a)
{
    const int lane = threadIdx.x & 31;
    const int64_t d = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (d >= a.n_dst) return;
    int64_t s0 = __ldg(a.dst_off + d), s1 = __ldg(a.dst_off + d + 1);
    if (s0 < 0 || s1 < s0 || s1 > a.n_src || (d == 0 && s0 != 0) || (d == a.n_dst - 1 && s1 != a.n_src)) {
        if (lane == 0) atomicOr(a.err, 8u);  // bad offsets: this destination gets zeros
        s0 = s1 = 0;
    }
    double* out = a.dst_coef + d * (int64_t)a.np;
    for (int o = lane; o < a.n_out; o += 32) {
        double2 v = make_double2(0.0, 0.0);
        for (int64_t s = s0; s < s1; ++s) {
            const double2 r = a.rows[s * (int64_t)a.n_out + o];
            v.x += r.x;
            v.y += r.y;
        }
        int n, m;
        out_nm(o, n, m);
        const int k0 = n * n + n;
        if (a.accumulate) {
            out[k0 + m] += v.x;
            if (m > 0) out[k0 - m] += v.y;
        } else {
            out[k0 + m] = v.x;
            if (m > 0) out[k0 - m] = v.y;
        }
    }
}

}  // namespace q2x

extern "C" q2x_status q2x_translate(q2x_plan_t plan, int p, int64_t n_src, const double* src_coef,
                                    const double* src_c, int64_t n_dst, const int64_t* dst_off,
                                    const double* dst_c, double* dst_coef, int accumulate)
{
    if (!plan) return q2x_fail(nullptr, Q2X_ERR_ARG, "plan is NULL");
    if (p < 0 || p > plan->p_max) return q2x_fail(plan, Q2X_ERR_RANGE, "p = %d outside 0..%d", p, plan->p_max);
    if (n_src < 0 || n_dst < 0) return q2x_fail(plan, Q2X_ERR_ARG, "negative size");
    if (accumulate != 0 && accumulate != 1) return q2x_fail(plan, Q2X_ERR_ARG, "accumulate must be 0 or 1");
    if (n_dst == 0) return Q2X_OK;
    if (n_dst > 0x7fffffffLL || n_src > ((int64_t)1 << 36)) return q2x_fail(plan, Q2X_ERR_ARG, "size too large");
    if (!dst_off || !dst_c || !dst_coef) return q2x_fail(plan, Q2X_ERR_ARG, "NULL destination array");
    if (n_src > 0 && (!src_coef || !src_c)) return q2x_fail(plan, Q2X_ERR_ARG, "NULL source array");
    cudaError_t e = cudaSetDevice(plan->device);
    if (e != cudaSuccess) return q2x_cuda_fail(plan, e, "cudaSetDevice");
    q2x::TransArgs a;
    a.p = p;
    a.np = (p + 1) * (p + 1);
    a.n_out = (p + 1) * (p + 2) / 2;
    a.norm = plan->norm;
    a.accumulate = accumulate;
    a.n_src = n_src;
    a.n_dst = n_dst;
    a.src_coef = src_coef;
    a.src_c = src_c;
    a.dst_off = dst_off;
    a.dst_c = dst_c;
    a.dst_coef = dst_coef;
    a.err = plan->d_err;
    q2x_status st = q2x_plan_workspace(plan, sizeof(double2) * (size_t)(n_src > 0 ? n_src : 1) * a.n_out);
    if (st != Q2X_OK) return st;
    a.rows = static_cast<double2*>(plan->ws);
    if (n_src > 0) {
        const size_t smem = (size_t)q2x::TR_WARPS * 2 * a.np * sizeof(double2);
        e = cudaFuncSetAttribute(q2x::q2x_translate_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return q2x_cuda_fail(plan, e, "cudaFuncSetAttribute");
        // few sources (the top of a tree): split each translation over up to
        // 8 warps so the level is not one warp's latency
        const int64_t target = (int64_t)plan->num_sms * 8;
        const int64_t want = std::max<int64_t>(1, std::min<int64_t>({8, target / n_src, (a.n_out + 31) / 32}));
        a.wps_log2 = 0;
        while ((2LL << a.wps_log2) <= want) ++a.wps_log2;
        a.wps = 1 << a.wps_log2;
        const int64_t warps = n_src * a.wps;
        const int64_t grid = (warps + q2x::TR_WARPS - 1) / q2x::TR_WARPS;
        q2x::q2x_translate_rows<<<(unsigned)grid, q2x::TR_WARPS * 32, smem, plan->stream>>>(a);
        e = cudaGetLastError();
        if (e != cudaSuccess) return q2x_cuda_fail(plan, e, "q2x_translate_rows launch");
        plan->launches += 1;
    }
    q2x::q2x_translate_combine<<<(unsigned)((n_dst + 3) / 4), 128, 0, plan->stream>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return q2x_cuda_fail(plan, e, "q2x_translate_combine launch");
    plan->launches += 1;
    return Q2X_OK;
}
