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
// n, m >= 0) from a flattened term schedule that gives every lane the same
// work; one warp per destination then adds its sources' rows in source order
// (deterministic) and packs them.  FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "q2x.h"
#include "q2x_kernels.cuh"
#include "q2x_plan.h"

namespace q2x {

constexpr int TR_WARPS = 4;

struct TransArgs {
    int p, np, n_out, norm, accumulate;
    int cta_per_source;  // 1: the four warps of a CTA share one source's terms
    int cta_per_dst;     // 1: the combine gives each destination a CTA of four warps
    int64_t n_src, n_dst;
    const double* src_coef;
    const double* src_c;
    const int64_t* dst_off;
    const double* dst_c;
    double* dst_coef;
    double2* rows;  // [n_src][n_out] translated rows, complex (n, m >= 0)
    unsigned* err;
    const double* rt = nullptr;     // precomputed packed R(t) rows (NULL: built per source)
    const int32_t* t_idx = nullptr;  // row of rt for each source
    int64_t n_t = 0;
};

// R_k^l(t) for |l| <= k <= p into Rc (complex, index k^2 + k + l) and -R
// into Rc + TR_NP_MAX, by the point recursion of Eq. (rec2); one warp.
__device__ void build_r(double2* Rc, int p, double tx, double ty, double tz, int lane);

// Packed real row of R(t) (Re at n^2+n+m, Im at n^2+n-m, m > 0) unpacked
// into Rc and -Rc (R_n^{-m} = (-1)^m conj R_n^m); one warp.
// (threads tid, tid + nthr, ... of the warp or CTA that shares Rc)
__device__ void unpack_r(double2* Rc, const double* __restrict__ row, int np, int tid, int nthr);

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

// Term schedule of the contraction: every (output o = n(n+1)/2 + m, k, l)
// term in output order, for p up to Q2X_P_MAX (the terms of degrees <= p
// are a prefix).  Code: bits 0-9 the R row index k^2 + k + l, plus
// Q2X_P_MAX's (p+1)^2 when the term carries the COEFF sign (-1)^k (the warp
// keeps -R there); bits 10-18 the F row index; bits 19-26 the output o.
constexpr int TR_NP_MAX = (Q2X_P_MAX + 1) * (Q2X_P_MAX + 1);
constexpr int tr_term_count(int p)
{
    int t = 0;
    for (int n = 0; n <= p; ++n)
        for (int m = 0; m <= n; ++m)
            for (int k = 0; k <= n; ++k) {
                const int nn = n - k;
                const int l0 = (-k > -nn - m) ? -k : -nn - m, l1 = (k < nn - m) ? k : nn - m;
                if (l1 >= l0) t += l1 - l0 + 1;
            }
    return t;
}
constexpr int TR_TERMS = tr_term_count(Q2X_P_MAX);
struct TermTab {
    uint32_t code[2][TR_TERMS];  // [norm]
    int end[Q2X_P_MAX + 1];      // terms of degrees <= p: [0, end[p])
};
constexpr TermTab make_terms()
{
    TermTab tt{};
    for (int norm = 0; norm < 2; ++norm) {
        int t = 0;
        for (int n = 0; n <= Q2X_P_MAX; ++n) {
            for (int m = 0; m <= n; ++m) {
                const int o = n * (n + 1) / 2 + m;
                for (int k = 0; k <= n; ++k) {
                    const int nn = n - k;
                    int l0 = 0, l1 = -1;
                    if (norm == 0) {  // F_{n-k}^{m+l}
                        l0 = (-k > -nn - m) ? -k : -nn - m;
                        l1 = (k < nn - m) ? k : nn - m;
                    } else {  // M_{n-k}^{m-l}
                        l0 = (-k > m - nn) ? -k : m - nn;
                        l1 = (k < m + nn) ? k : m + nn;
                    }
                    for (int l = l0; l <= l1; ++l) {
                        const int ri = k * k + k + l + ((norm == 0 && (k & 1)) ? TR_NP_MAX : 0);
                        const int fi = nn * nn + nn + (norm == 0 ? m + l : m - l);
                        tt.code[norm][t++] = (uint32_t)ri | ((uint32_t)fi << 10) | ((uint32_t)o << 19);
                    }
                }
            }
            if (norm == 0) tt.end[n] = t;
        }
    }
    return tt;
}
static __device__ const TermTab g_terms = make_terms();

__device__ void build_r(double2* Rc, int p, double tx, double ty, double tz, int lane)
{
    if (lane == 0) {
        Rc[0] = make_double2(1.0, 0.0);
        Rc[TR_NP_MAX] = make_double2(-1.0, 0.0);
    }
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
            const double2 rv = make_double2(v.x * inv, v.y * inv);
            Rc[n * n + n + m] = rv;
            Rc[TR_NP_MAX + n * n + n + m] = make_double2(-rv.x, -rv.y);
        }
        __syncwarp();
    }
}

__device__ void unpack_r(double2* Rc, const double* __restrict__ row, int np, int tid, int nthr)
{
    for (int k = tid; k < np; k += nthr) {
        int n, m;
        col_nm(k, n, m);
        const int am = m < 0 ? -m : m;
        const int k0 = n * n + n;
        const double re = __ldg(row + k0 + am);
        const double im = am ? __ldg(row + k0 - am) : 0.0;
        const double2 v = (m >= 0) ? make_double2(re, im)
                                   : ((am & 1) ? make_double2(-re, im) : make_double2(re, -im));
        Rc[k] = v;
        Rc[TR_NP_MAX + k] = make_double2(-v.x, -v.y);
    }
}

// One warp per translation vector: R(t) built in shared memory, then packed.
__global__ void __launch_bounds__(TR_WARPS * 32) q2x_translation_rows_kernel(int p, int64_t n_t,
                                                                            const double* __restrict__ t,
                                                                            double* rt)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * TR_WARPS + wib;
    if (i >= n_t) return;
    double2* Rc = reinterpret_cast<double2*>(smem_raw) + (size_t)wib * 2 * TR_NP_MAX;
    build_r(Rc, p, __ldg(t + i), __ldg(t + n_t + i), __ldg(t + 2 * n_t + i), lane);
    const int np = (p + 1) * (p + 1);
    double* out = rt + i * (int64_t)np;
    for (int k = lane; k < np; k += 32) {
        int n, m;
        col_nm(k, n, m);
        const double2 v = Rc[n * n + n + (m < 0 ? -m : m)];
        out[k] = (m >= 0) ? v.x : v.y;
    }
}

// One warp per source (or, for the few sources at the top of a tree, one
// CTA of four warps per source): the source's complex row and R(t) (and
// -R(t)) in shared memory -- the warp's own copy, or one copy per CTA built
// by its first warp -- then the contraction over the
// flattened term list, each lane a contiguous run of terms (equal work per
// lane).  Outputs wholly inside a lane's run are written by that lane; the
// partial sums of an output split across runs are added in run order by the
// lane whose run holds its first part.
__global__ void __launch_bounds__(TR_WARPS * 32) q2x_translate_rows(const TransArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int64_t s = a.cta_per_source ? (int64_t)blockIdx.x : (int64_t)blockIdx.x * TR_WARPS + wib;
    const int nsub = a.cta_per_source ? TR_WARPS : 1;  // runs of 32 lanes sharing the source
    const int sub = a.cta_per_source ? wib : 0;
    if (s >= a.n_src) return;
    const int p = a.p, np = a.np;
    // one copy of the source row and R(t) per source: per warp, or shared by
    // the CTA's warps (built by its first warp)
    const bool cta = a.cta_per_source != 0;
    double2* Fc = reinterpret_cast<double2*>(smem_raw) + (size_t)(cta ? 0 : wib) * 3 * TR_NP_MAX;
    double2* Rc = Fc + TR_NP_MAX;  // R at [0, TR_NP_MAX), -R at [TR_NP_MAX, 2 TR_NP_MAX)
    __shared__ int s_head_o[TR_WARPS][32], s_tail_o[TR_WARPS][32];
    __shared__ double2 s_head_v[TR_WARPS][32], s_tail_v[TR_WARPS][32];
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

    // with precomputed R(t) rows every warp of a CTA takes part in filling
    // the shared copy; the recursion for R(t) is one warp's
    const bool rt_mode = a.rt != nullptr;
    const int tid = (cta && rt_mode) ? (int)threadIdx.x : lane;
    const int nthr = (cta && rt_mode) ? TR_WARPS * 32 : 32;
    if (!cta || rt_mode || wib == 0) {
        // ---- complex source row F[n][m], m = -n..n (Eq. (bas2.1) for m < 0)
        const double* src = a.src_coef + s * (int64_t)np;
        for (int k = tid; k < np; k += nthr) {
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
        // ---- R_k^l(t), t = c_src - c_dst: a precomputed row, or the recursion
        if (a.rt) {
            int ti = __ldg(a.t_idx + s);
            if (ti < 0 || ti >= a.n_t) {
                if (tid == 0) atomicOr(a.err, 1u);
                ti = -1;
            }
            if (ti >= 0) {
                unpack_r(Rc, a.rt + (int64_t)ti * np, np, tid, nthr);
            } else {
                for (int k = tid; k < np; k += nthr) Rc[k] = Rc[TR_NP_MAX + k] = make_double2(0.0, 0.0);
            }
            __syncwarp();
        } else {
            const double tx = __ldg(a.src_c + s) - __ldg(a.dst_c + d);
            const double ty = __ldg(a.src_c + a.n_src + s) - __ldg(a.dst_c + a.n_dst + d);
            const double tz = __ldg(a.src_c + 2 * a.n_src + s) - __ldg(a.dst_c + 2 * a.n_dst + d);
            build_r(Rc, p, tx, ty, tz, lane);
        }
    }
    if (cta) __syncthreads();  // the shared row and R(t) are complete
    // ---- contraction over this lane's run of terms
    double2* row = a.rows + s * (int64_t)a.n_out;
    const uint32_t* code = g_terms.code[a.norm ? 1 : 0];
    const int T = g_terms.end[p];
    const int C = (T + 32 * nsub - 1) / (32 * nsub);
    const int t0 = min((sub * 32 + lane) * C, T), t1 = min(t0 + C, T);
    int cur = -1, head = -1;
    double cr = 0.0, ci = 0.0;
    double2 head_v = make_double2(0.0, 0.0);
    // unrolled so that the term codes of several iterations are in flight
    // at once (the small levels at the top of a tree are latency-bound)
#pragma unroll 4
    for (int t = t0; t < t1; ++t) {
        const uint32_t cd = __ldg(code + t);
        const int o = (int)(cd >> 19);
        if (o != cur) {
            if (cur >= 0) {
                if (head < 0) {
                    head = cur;
                    head_v = make_double2(cr, ci);
                } else {
                    row[cur] = make_double2(cr, ci);  // wholly inside this run
                }
            }
            cur = o;
            cr = ci = 0.0;
        }
        const double2 r = Rc[cd & 1023u], f = Fc[(cd >> 10) & 511u];
        cr = fma(r.x, f.x, fma(-r.y, f.y, cr));
        ci = fma(r.x, f.y, fma(r.y, f.x, ci));
    }
    if (head < 0) {
        s_head_o[wib][lane] = cur;
        s_head_v[wib][lane] = make_double2(cr, ci);
        s_tail_o[wib][lane] = -1;
    } else {
        s_head_o[wib][lane] = head;
        s_head_v[wib][lane] = head_v;
        s_tail_o[wib][lane] = cur;
        s_tail_v[wib][lane] = make_double2(cr, ci);
    }
    if (a.cta_per_source)
        __syncthreads();
    else
        __syncwarp();
    // boundary partials, summed in run order by the run that holds each
    // output's first partial (all runs at once; the same order of addition
    // as one sequential pass over the runs)
    const int nr = 32 * nsub;
    const int j = sub * 32 + lane;
    auto slot = [&](int R) { return a.cta_per_source ? (R >> 5) : wib; };
    auto HO = [&](int R) { return s_head_o[slot(R)][R & 31]; };
    auto TO = [&](int R) { return s_tail_o[slot(R)][R & 31]; };
    auto HV = [&](int R) { return s_head_v[slot(R)][R & 31]; };
    const int ho = HO(j);
    if (ho >= 0) {
        const int prev = (j == 0) ? -1 : (TO(j - 1) >= 0 ? TO(j - 1) : HO(j - 1));
        if (ho != prev) {
            double2 v = HV(j);
            int r = j;
            while (TO(r) < 0 && r + 1 < nr && HO(r + 1) == ho) {
                ++r;
                const double2 w = HV(r);
                v.x += w.x;
                v.y += w.y;
            }
            row[ho] = v;
        }
    }
    const int to = TO(j);
    if (to >= 0) {
        double2 v = s_tail_v[slot(j)][lane];
        int r = j;
        while (r + 1 < nr && HO(r + 1) == to) {
            ++r;
            const double2 w = HV(r);
            v.x += w.x;
            v.y += w.y;
            if (TO(r) >= 0) break;
        }
        row[to] = v;
    }
}

// One warp per destination (few destinations, the top of a tree: a CTA of
// four warps per destination, its outputs split over 128 threads): its
// sources' rows added in source order, packed.
__global__ void q2x_translate_combine(const TransArgs a)
{
    const int lane = a.cta_per_dst ? (int)threadIdx.x : (int)(threadIdx.x & 31);
    const int nthr = a.cta_per_dst ? (int)blockDim.x : 32;
    const int64_t d = a.cta_per_dst ? (int64_t)blockIdx.x
                                    : (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (d >= a.n_dst) return;
    int64_t s0 = __ldg(a.dst_off + d), s1 = __ldg(a.dst_off + d + 1);
    if (s0 < 0 || s1 < s0 || s1 > a.n_src || (d == 0 && s0 != 0) || (d == a.n_dst - 1 && s1 != a.n_src)) {
        if (lane == 0) atomicOr(a.err, 8u);  // bad offsets: this destination gets zeros
        s0 = s1 = 0;
    }
    double* out = a.dst_coef + d * (int64_t)a.np;
    for (int o = lane; o < a.n_out; o += nthr) {
        double2 v = make_double2(0.0, 0.0);
#pragma unroll 4
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

static q2x_status translate_impl(q2x_plan_t plan, int p, int64_t n_src, const double* src_coef,
                                 const double* src_c, int64_t n_dst, const int64_t* dst_off, const double* dst_c,
                                 double* dst_coef, int accumulate, const double* rt, const int32_t* t_idx,
                                 int64_t n_t)
{
    if (!plan) return q2x_fail(nullptr, Q2X_ERR_ARG, "plan is NULL");
    if (p < 0 || p > plan->p_max) return q2x_fail(plan, Q2X_ERR_RANGE, "p = %d outside 0..%d", p, plan->p_max);
    if (n_src < 0 || n_dst < 0) return q2x_fail(plan, Q2X_ERR_ARG, "negative size");
    if (accumulate != 0 && accumulate != 1) return q2x_fail(plan, Q2X_ERR_ARG, "accumulate must be 0 or 1");
    if (n_dst == 0) return Q2X_OK;
    if (n_dst > 0x7fffffffLL || n_src > ((int64_t)1 << 36)) return q2x_fail(plan, Q2X_ERR_ARG, "size too large");
    if (!dst_off || !dst_coef || (!rt && !dst_c)) return q2x_fail(plan, Q2X_ERR_ARG, "NULL destination array");
    if (n_src > 0 && (!src_coef || (!rt && !src_c) || (rt && (!t_idx || n_t <= 0))))
        return q2x_fail(plan, Q2X_ERR_ARG, "NULL source array or translation rows");
    cudaError_t e = cudaSetDevice(plan->device);
    if (e != cudaSuccess) return q2x_cuda_fail(plan, e, "cudaSetDevice");
    q2x::TransArgs a;
    a.cta_per_source = 0;
    a.cta_per_dst = (n_dst <= (int64_t)plan->num_sms) ? 1 : 0;
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
    a.rt = rt;
    a.t_idx = t_idx;
    a.n_t = n_t;
    q2x_status st = q2x_plan_workspace(plan, sizeof(double2) * (size_t)(n_src > 0 ? n_src : 1) * a.n_out);
    if (st != Q2X_OK) return st;
    a.rows = static_cast<double2*>(plan->ws);
    if (n_src > 0) {
        const size_t smem = (size_t)q2x::TR_WARPS * 3 * q2x::TR_NP_MAX * sizeof(double2);
        e = cudaFuncSetAttribute(q2x::q2x_translate_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return q2x_cuda_fail(plan, e, "cudaFuncSetAttribute");
        // few sources (the top of a tree): a CTA per source, so a level is
        // not the latency of one warp's FP64 stream
        a.cta_per_source = (n_src * 4 <= (int64_t)plan->num_sms * 8) ? 1 : 0;
        const int64_t grid = a.cta_per_source ? n_src : (n_src + q2x::TR_WARPS - 1) / q2x::TR_WARPS;
        const size_t smem_launch = a.cta_per_source ? smem / q2x::TR_WARPS : smem;  // one shared copy
        q2x::q2x_translate_rows<<<(unsigned)grid, q2x::TR_WARPS * 32, smem_launch, plan->stream>>>(a);
        e = cudaGetLastError();
        if (e != cudaSuccess) return q2x_cuda_fail(plan, e, "q2x_translate_rows launch");
        plan->launches += 1;
    }
    q2x::q2x_translate_combine<<<(unsigned)(a.cta_per_dst ? n_dst : (n_dst + 3) / 4), 128, 0, plan->stream>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return q2x_cuda_fail(plan, e, "q2x_translate_combine launch");
    plan->launches += 1;
    return Q2X_OK;
}

extern "C" q2x_status q2x_translate(q2x_plan_t plan, int p, int64_t n_src, const double* src_coef,
                                    const double* src_c, int64_t n_dst, const int64_t* dst_off,
                                    const double* dst_c, double* dst_coef, int accumulate)
{
    return translate_impl(plan, p, n_src, src_coef, src_c, n_dst, dst_off, dst_c, dst_coef, accumulate, nullptr,
                          nullptr, 0);
}

extern "C" q2x_status q2x_translate_rt(q2x_plan_t plan, int p, int64_t n_src, const double* src_coef, int64_t n_t,
                                       const double* rt, const int32_t* t_idx, int64_t n_dst,
                                       const int64_t* dst_off, double* dst_coef, int accumulate)
{
    if (!plan) return q2x_fail(nullptr, Q2X_ERR_ARG, "plan is NULL");
    if (n_src > 0 && (!rt || !t_idx)) return q2x_fail(plan, Q2X_ERR_ARG, "NULL translation rows");
    return translate_impl(plan, p, n_src, src_coef, nullptr, n_dst, dst_off, nullptr, dst_coef, accumulate,
                          n_src > 0 ? rt : nullptr, t_idx, n_t);
}

extern "C" q2x_status q2x_translation_rows(q2x_plan_t plan, int p, int64_t n_t, const double* t, double* rt)
{
    if (!plan) return q2x_fail(nullptr, Q2X_ERR_ARG, "plan is NULL");
    if (p < 0 || p > plan->p_max) return q2x_fail(plan, Q2X_ERR_RANGE, "p = %d outside 0..%d", p, plan->p_max);
    if (n_t < 0) return q2x_fail(plan, Q2X_ERR_ARG, "negative size");
    if (n_t == 0) return Q2X_OK;
    if (!t || !rt) return q2x_fail(plan, Q2X_ERR_ARG, "NULL array");
    if (n_t > ((int64_t)1 << 36)) return q2x_fail(plan, Q2X_ERR_ARG, "size too large");
    cudaError_t e = cudaSetDevice(plan->device);
    if (e != cudaSuccess) return q2x_cuda_fail(plan, e, "cudaSetDevice");
    const size_t smem = (size_t)q2x::TR_WARPS * 2 * q2x::TR_NP_MAX * sizeof(double2);
    e = cudaFuncSetAttribute(q2x::q2x_translation_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return q2x_cuda_fail(plan, e, "cudaFuncSetAttribute");
    q2x::q2x_translation_rows_kernel<<<(unsigned)((n_t + q2x::TR_WARPS - 1) / q2x::TR_WARPS), q2x::TR_WARPS * 32,
                                       smem, plan->stream>>>(p, n_t, t, rt);
    e = cudaGetLastError();
    if (e != cudaSuccess) return q2x_cuda_fail(plan, e, "q2x_translation_rows launch");
    plan->launches += 1;
    return Q2X_OK;
}
