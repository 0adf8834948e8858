// q2x_kernels.cuh -- Q2X recursion kernels for sm_103a.
//
// One warp owns a contiguous range of T = 32*R elements (elements are sorted
// by leaf).  Each lane runs one element through the paper's recursions in the
// "tilde" basis (Eqs. (rec10)-(rec15)), degree by degree, with the row of every
// level held in registers.  All levels of the chain advance together at each
// order m (level k's source at (n, m) is level k-1's new value at (n, m)), so
// no source rows are stored.  After each chunk of degrees the 32 lanes stage
// their coefficients in shared memory and the warp switches to a
// lane-per-column layout to form per-leaf (segmented) sums over its rows.
// Leaves that lie wholly inside the warp's range are written directly; the two
// boundary leaves of a range go to slot partials that q2x_fixup_kernel
// combines in a fixed order (deterministic, no atomics on the data path).
//
// Division-free ("hat") form of the recursions.  Writing every level with a
// factorial weight, x^_n = (n + d)! x_n (d = depth of the level in its chain),
// turns each of the paper's level recursions
//     (n + d) x_n = A_v x_{n-1} + s_n                              (Lemmas 1-5)
// into x^_n = A_v x^_{n-1} + s^_n, where A_v is the tilde stencil of
// Eq. (rec10): (A_v a)^m = -xi_v a^{m-1} + eta_v a^{m+1} - z_v a^m for m > 0 and
// 2 Re(eta_v a^1) - z_v a^0 for m = 0, with (xi_v, eta_v, z_v) the local
// coordinates of one vertex: x2 for q (Eq. (rec2)), x3 for j (Eq. (rec12)), x4
// for b (Eq. (rec14.1)) and x1 for p, i, a (Eqs. (rec10), (rec12), (rec14.1)).
// The 1/(n+d)! goes into the per-column output constant.  All levels start
// from q^_0 = seed and zero rows at n = -1, which reproduces the starting
// values of Eq. (rec3) (p_0 = j_0 = 1, i_0 = b_0 = 1/2, a_0 = 1/6).
// The FP64 kernels compute the point level q^ by an equivalent recursion
// over the order at fixed degree (see g_qtab below) and run the degree's
// orders from n down to 0; the FP32 kernels run the stencil on every level,
// orders 0 up to n.
//
// Linear density on triangles (not in the paper; derived by the same
// integration by parts as Lemma 2 with the weight w = s1(1-u-v) + s2 u + s3 v):
//     (n+2) E_n  = A_x3 E_{n-1}  + s2 q_n + s3 j_n      E = int_edge w h
//     (n+3) Iw_n = A_x1 Iw_{n-1} + E_n + s1 i_n        Iw = int_T w g
// so the chain is q, j, E, i, Iw (5 levels), hat weights n!, (n+1)!, (n+2)!,
// (n+2)!, (n+3)!; in hat form E^_n = A E^_{n-1} + (n+1) s2 q^_n + s3 j^_n and
// Iw^_n = A Iw^_{n-1} + E^_n + s1 i^_n.
//
// Double layer (Eq. (rec15)): l~_n = A_nrm i~_{n-1} with the unit normal in
// place of the vertex (xi = (n_x + i n_y)/2, eta = conj xi, z = n_z); it uses
// the row of degree n-1 before that row is advanced.
//
// Output map (Eq. (bas10) with x_n^m = i^{-m} x~_n^m of Eq. (rec7) and the
// symmetry of Eq. (bas2.1)): with x~ = a + i b, the packed real outputs are
//   COEFF : F_n^m = (J/4pi)(-1)^{n+m} i^m conj(x~)   -> Re/Im = +-a or +-b
//   MOMENT: int R_n^m = J i^{-m} x~
// Re takes a for even m and b for odd m; Im the other; the sign is folded
// into the per-column constant.
//
// Scaled local frame: y' = (x - r*) / 2^s with 2^s >= rho_leaf, so |y'| <~ 1;
// homogeneity of R_n^m (degree n) and the Jacobian (degree dim) give the factor
// 2^{s (n + dim)} (double layer 2^{s (n + 1)}), applied exactly as an exponent
// shift when the FP64 coefficient is formed.  In the FP32 path the inputs are
// split exactly into FP32 pairs with integer operations, the Jacobian and the
// seed are formed in FP64 from the FP64 vertices (once per element), each
// round's 32-row column sums are added into compensated FP32 leaf sums, and a
// leaf's coefficients are re-biased exactly into FP64: no FP64 arithmetic runs
// per moment or per round.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "q2x.h"

#include <type_traits>
#include <utility>

namespace q2x {

enum : int { KIND_SEG = 0, KIND_TRI = 1, KIND_TET = 2 };
enum : int { DENS_CONST = 0, DENS_LINEAR = 1 };

constexpr int WARPS_PER_CTA = 4;  // CTAs of the FP64 element kernel and of the Galerkin kernel

// Warps per CTA of the element kernel.  Warps never cooperate (each owns its
// range and its shared-memory region), so FP32 CTAs are single warps: the
// number of resident warps is then set by the registers alone, which are
// allotted per SM sub-partition (16 K each: 4 warps at <= 128 registers, 3 at
// <= 168, 2 at <= 256).  The FP64 kernel keeps CTAs of four warps (measured
// 2 % faster than single warps at the same occupancy).
template <typename T>
__host__ __device__ constexpr int elem_warps_per_cta()
{
    return sizeof(T) == 4 ? 1 : WARPS_PER_CTA;
}

// Stage tile geometry per precision: CHUNK columns per layer, LD = padded
// row stride (36 floats keeps 16-byte aligned columns for 128-bit loads and
// conflict-free row writes; 33 doubles for the FP64 tile).
template <typename T>
struct KCfg;
template <>
struct KCfg<float> {
    static constexpr int CHUNK = 48;
    static constexpr int LD = 36;
};
template <>
struct KCfg<double> {
    static constexpr int CHUNK = 44;
    static constexpr int LD = 33;
};

struct ElemArgs {
    int64_t n_elem, n_vert;
    const double* vx;
    const double* vy;
    const double* vz;
    const int32_t* idx;       // SoA nv x n_elem
    const double* sigma;      // n_elem (const) or n_vert (linear)
    int64_t n_leaves;
    const int64_t* leaf_off;  // NULL: per-element expansions
    const double* leaf_c;     // SoA 3 x n_leaves
    const double* leaf_rho;   // NULL: unit scale (s = 0)
    const int32_t* leaf_p;    // NULL: p_max
    int p_max;
    int np_max;               // (p_max + 1)^2
    double* coef[3];          // outputs: layers (single, double), or the three components of a
                              // vector density; NULL = skip
    const double* wvec;       // vector density: SoA 3 x n_elem components per element
    int nacc;                 // output slots per leaf: 2 (layers) or 3 (vector components)
    int accumulate;
    int norm;                 // 0 COEFF, 1 MOMENT
    int64_t T;                // elements per warp range, multiple of 32
    int64_t n_ranges;
    double* slots;            // [n_ranges][2 slots][nacc outputs][np_max] FP64 partial sums
    unsigned* err;
};

// ------------------------------------------------------------- constants

// 1/k! for k = 0..24 (compile-time values, no upload).
#define Q2X_INV_FACT_LIST                                                                          \
    1.0, 1.0, 0.5, 0.16666666666666666667, 0.041666666666666666667, 0.0083333333333333333333,   \
        0.0013888888888888888889, 0.00019841269841269841270, 2.4801587301587301587e-05,         \
        2.7557319223985890653e-06, 2.7557319223985890653e-07, 2.5052108385441718775e-08,        \
        2.0876756987868098979e-09, 1.6059043836821614599e-10, 1.1470745597729724714e-11,        \
        7.6471637318198164759e-13, 4.7794773323873852974e-14, 2.8114572543455207632e-15,        \
        1.5619206968586226462e-16, 8.2206352466243297170e-18, 4.1103176233121648585e-19,        \
        1.9572941063391261231e-20, 8.8967913924505732867e-22, 3.8681701706306840377e-23,        \
        1.6117375710961183490e-24
static __constant__ double c_inv_fact_d[25] = {Q2X_INV_FACT_LIST};
constexpr double INV_4PI = 0.079577471545947667884;

// chunk of degrees starting at nb for a kernel of capacity P: the longest run
// of degrees whose column count (2n+1 each) fits C; a degree with more
// columns than that forms a chunk of its own.
__host__ __device__ constexpr int chunk_end(int nb, int P, int C)
{
    int ne = nb + 1;
    while (ne <= P && (ne + 1) * (ne + 1) - nb * nb <= C) ++ne;
    return ne;
}

// ------------------------------------------------------------- bit helpers

// exponent s with 2^s >= rho for finite rho > 0 (0 otherwise), from the bits
__device__ __forceinline__ int scale_exponent(double rho)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(rho);
    const int e = (int)((b >> 52) & 0x7FF);
    if ((b >> 63) || e == 0x7FF || e == 0) return 0;  // negative, non-finite, zero or denormal
    int s = e - 1023;
    if (b & 0xFFFFFFFFFFFFFull) s += 1;
    return max(-100, min(100, s));
}

__device__ __forceinline__ bool finite_bits(double x)
{
    return (((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FF) != 0x7FF;
}

// 2^k as a double, by construction
__device__ __forceinline__ double pow2d(int k)
{
    k = max(-1022, min(1023, k));
    return __longlong_as_double((long long)(k + 1023) << 52);
}

// 2^k as a float
__device__ __forceinline__ float pow2f(int k)
{
    k = max(-126, min(127, k));
    return __int_as_float((k + 127) << 23);
}

// FP32 value v times 2^k, returned exactly as a double, using integer
// operations only (re-biases the exponent field; FP32 denormals flush to 0).
__device__ __forceinline__ double f32_scaled_to_f64(float v, int k)
{
    const unsigned int b = __float_as_uint(v);
    const unsigned int e = (b >> 23) & 0xFF;
    if (e == 0) return 0.0;
    const unsigned long long sign = (unsigned long long)(b >> 31) << 63;
    long long de = (long long)e - 127 + 1023 + k;
    if (de <= 0) return 0.0;
    if (de >= 2047) de = 2046;
    const unsigned long long mant = (unsigned long long)(b & 0x7FFFFF) << 29;
    return __longlong_as_double((long long)(sign | ((unsigned long long)de << 52) | mant));
}

// Split of a double into hi + lo floats with integer operations only: hi keeps
// the leading 24 significand bits (truncated), lo the rest rounded to 24 bits,
// so |x - hi - lo| <= 2^-47 |x|.  |x| < 2^-103 gives lo = 0, |x| < 2^-126 gives
// hi = lo = 0; a non-finite or too large x sets bad.
__device__ __forceinline__ void split_f64(double x, float& hi, float& lo, bool& bad)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FF);
    const unsigned int sign = (unsigned int)(b >> 63) << 31;
    const int ex = e - 1023;
    if (e == 0x7FF || ex > 127) {
        bad = true;
        hi = lo = 0.f;
        return;
    }
    if (ex < -126) {
        hi = lo = 0.f;
        return;
    }
    hi = __uint_as_float(sign | ((unsigned int)(ex + 127) << 23) |
                         (unsigned int)((b >> 29) & 0x7FFFFF));
    const unsigned int ml = (unsigned int)(b & 0x1FFFFFFFull);
    if (ex < -103 || ml == 0) {
        lo = 0.f;
        return;
    }
    // ml * 2^(ex - 52) = (ml * 2^-29) * 2^(ex - 23)
    const float l = __uint2float_rn(ml) * 1.862645149230957e-09f * pow2f(ex - 23);
    lo = sign ? -l : l;
}

// ------------------------------------------------- packed FP32 complex pairs
// A complex FP32 value (re, im) lives in one 64-bit register pair and is
// operated on with Blackwell's paired FP32 instructions (add/sub/mul/fma
// .rn.f32x2), so one tilde-stencil update costs about half the instructions
// of the scalar form.
struct cf {
    unsigned long long v;
};
__device__ __forceinline__ cf cf_make(float re, float im)
{
    cf r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(re), "f"(im));
    return r;
}
__device__ __forceinline__ void cf_parts(cf a, float& re, float& im)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(re), "=f"(im) : "l"(a.v));
}
__device__ __forceinline__ cf cf_add(cf a, cf b)
{
    cf r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ cf cf_sub(cf a, cf b)
{
    cf r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ cf cf_mul(cf a, cf b)
{
    cf r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ cf cf_fma(cf a, cf b, cf c)
{
    cf r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}
__device__ __forceinline__ cf cf_zero()
{
    cf r;
    r.v = 0ull;
    return r;
}

// One tilde-stencil update in packed form: with a = x^{m-1}, b = x^{m+1},
// c = x^m of degree n-1 and xi = X + iY,
//   -xi a + eta b - z c + src = X (b - a) + (Y, -Y) * swap(a + b) - z c + src.
// (At m = 0, Eq. (rec11) gives the real value 2 Re(eta b) - z c + src, which
// the degree loop computes in scalar form.)  The two neighbour combinations
// are formed once per row entry and shared by every stencil applied to it
// (the output level and its double layer).
struct cf_nb {
    cf d, s;  // b - a and a + b (both packed)
};
__device__ __forceinline__ cf_nb cf_neighbours(cf a, cf b) { return cf_nb{cf_sub(b, a), cf_add(a, b)}; }
__device__ __forceinline__ cf cf_stencil_nb(const cf_nb& nb, cf c, cf src, cf X2, cf YmY, cf nZ2)
{
    cf t = cf_fma(nZ2, c, src);
    t = cf_fma(X2, nb.d, t);
    // the Y term as two scalar FMAs that read the halves of a + b crosswise
    // (the swap costs no instruction); forming swap(a + b) into a register
    // pair for a paired FMA costs more than the extra FMA (measured)
    float tr, ti, sr, si, yy, ny;
    cf_parts(t, tr, ti);
    cf_parts(nb.s, sr, si);
    cf_parts(YmY, yy, ny);
    return cf_make(fmaf(yy, si, tr), fmaf(ny, sr, ti));
}

// column c -> (n, m), exact for c < 2^20
__device__ __forceinline__ void col_nm(int c, int& n, int& m)
{
    const float f = (float)c + 0.5f;
    n = (int)(f * rsqrtf(f));
    if (n * n > c) --n;
    if ((n + 1) * (n + 1) <= c) ++n;
    m = c - n * n - n;
}

// Sign of the packed output of column (n, m) (m < 0: the Im part of order
// |m|), relative to the staged component (a = Re x~ for even |m|, b = Im x~
// for odd |m| in the Re column, the other one in the Im column):
//   COEFF : (-1)^{n+m} i^m conj(a + ib): Re = {a, b, -a, -b}, Im = {-b, a, b, -a}
//   MOMENT: i^{-m}(a + ib):              Re = {a, b, -a, -b}, Im = {b, -a, -b, a}
__device__ __forceinline__ bool column_negative(int norm, int n, int m_signed)
{
    const int m = m_signed < 0 ? -m_signed : m_signed;
    const int r = m & 3;
    bool neg;
    if (m_signed >= 0)
        neg = r >= 2;
    else if (norm == 0)
        neg = !(r == 1 || r == 2);
    else
        neg = !(r == 0 || r == 3);
    if (norm == 0 && ((n + m) & 1)) neg = !neg;
    return neg;
}

// 1/k! (/4pi for COEFF) as an FP32 significand in [1, 2) and a power of two,
// for the FP32 finish (compile-time table)
struct FinishTab {
    float mant[2][25];
    int expo[2][25];
};
constexpr FinishTab make_finish_tab()
{
    FinishTab t{};
    double f = 1.0;
    for (int k = 0; k < 25; ++k) {
        if (k > 0) f /= k;
        for (int nm = 0; nm < 2; ++nm) {
            double v = nm == 0 ? f * INV_4PI : f;
            int e = 0;
            while (v >= 2.0) {
                v *= 0.5;
                ++e;
            }
            while (v < 1.0) {
                v *= 2.0;
                --e;
            }
            float m = (float)v;
            if (m >= 2.0f) {
                m = 1.0f;
                ++e;
            }
            t.mant[nm][k] = m;
            t.expo[nm][k] = e;
        }
    }
    return t;
}
static __constant__ FinishTab c_finish = make_finish_tab();

// Per-column descriptor of the real packing k = n^2 + n + m (k < 441):
// bits 0-4 the degree n, bit 5 / bit 6 the output sign (column_negative) for
// COEFF / MOMENT.  A compile-time table read through the read-only cache, so
// the flush of a leaf column needs no square root or sign logic.
struct ColTab {
    unsigned short v[(Q2X_P_MAX + 1) * (Q2X_P_MAX + 1)];
};
constexpr ColTab make_col_tab()
{
    ColTab t{};
    for (int n = 0; n <= Q2X_P_MAX; ++n)
        for (int m = -n; m <= n; ++m) {
            const int am = m < 0 ? -m : m;
            const int r = am & 3;
            bool neg[2] = {false, false};
            for (int nm = 0; nm < 2; ++nm) {
                bool g = false;
                if (m >= 0)
                    g = r >= 2;
                else if (nm == 0)
                    g = !(r == 1 || r == 2);
                else
                    g = !(r == 0 || r == 3);
                if (nm == 0 && ((n + am) & 1)) g = !g;
                neg[nm] = g;
            }
            t.v[n * n + n + m] = (unsigned short)(n | (neg[0] ? 32 : 0) | (neg[1] ? 64 : 0));
        }
    return t;
}
static __device__ const ColTab g_coltab = make_col_tab();

__device__ __forceinline__ int col_desc(int c)
{
    return (int)__ldg(&g_coltab.v[c]);
}

// Point level in the FP64 path: recursion over the order at a fixed degree.
// Reading the point stencil of Eqs. (rec2), (rec10), (rec11) as multiplication
// by the Laurent polynomial f(w) = -xi w - z + eta / w (xi = (x + iy)/2,
// eta = conj xi, z of the level's vertex) gives T_n^m = seed [w^m] f(w)^n.
// The coefficients of g = f^n satisfy f g' = n f' g; comparing the powers w^m
// gives, with T_n^m = (-xi)^m Q_n^m and 4 |xi|^2 = x^2 + y^2,
//   (n - m) Q_n^m = -(m + 1) z Q_n^{m+1} - (n + m + 2) |xi|^2 Q_n^{m+2},
// Q_n^n = 1, Q_n^{n-1} = -n z: a real recursion downwards in m that needs no
// row of the previous degree.  Q_n^m is a polynomial in z and |xi|^2, so the
// recursion has no division by |xi| and stays accurate near the axis (checked
// against exact rational arithmetic to p = 20).  Per entry it costs six FP64
// operations against ten for the stencil.  A(n, m) = -(m + 1)/(n - m) and
// B(n, m) = -(n + m + 2)/(n - m) for m <= n - 2.
struct QTab {
    double a[(Q2X_P_MAX + 1) * (Q2X_P_MAX + 1)];
    double b[(Q2X_P_MAX + 1) * (Q2X_P_MAX + 1)];
};
constexpr QTab make_q_tab()
{
    QTab t{};
    for (int n = 0; n <= Q2X_P_MAX; ++n)
        for (int m = 0; m + 2 <= n; ++m) {
            t.a[n * (Q2X_P_MAX + 1) + m] = -(double)(m + 1) / (double)(n - m);
            t.b[n * (Q2X_P_MAX + 1) + m] = -(double)(n + m + 2) / (double)(n - m);
        }
    return t;
}
static __constant__ QTab g_qtab = make_q_tab();  // warp-uniform reads: the constant cache

// final coefficient of column (n, m) (its descriptor from col_desc) from a
// sum acc: acc * sign / (n+d)! (/ 4pi for COEFF) * 2^(s (n + shift_n0)), the
// power of two being the leaf scale of the frame (exact).
// FP32 sums: one FP32 multiply by the table significand (relative rounding
// 2^-24), then the power of two is applied while re-biasing into FP64, so
// tiny coefficients cannot underflow and no FP64 arithmetic is needed.
__device__ __forceinline__ double finish_desc(float acc, int norm, int desc, int d, int shift_n0, int s)
{
    const int n = desc & 31;
    float v = acc * c_finish.mant[norm][n + d];
    if ((desc >> (5 + norm)) & 1) v = -v;
    return f32_scaled_to_f64(v, s * (n + shift_n0) + c_finish.expo[norm][n + d]);
}
__device__ __forceinline__ double finish_desc(double acc, int norm, int desc, int d, int shift_n0, int s)
{
    const int n = desc & 31;
    double cst = c_inv_fact_d[n + d];
    if (norm == 0) cst *= INV_4PI;
    if ((desc >> (5 + norm)) & 1) cst = -cst;
    return acc * cst * pow2d(s * (n + shift_n0));
}

// compile-time loop: f(std::integral_constant<int, I>) for I in [B, E)
template <int B, int E, typename F>
__device__ __forceinline__ void static_for(F&& f)
{
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

// ---------------------------------------------------------- leaf lookup

// leaf containing element e: largest L in [lo, hi] with off[L] <= e
__device__ __forceinline__ int64_t leaf_search(const int64_t* __restrict__ off, int64_t lo,
                                               int64_t hi, int64_t e)
{
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= e)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// first L in [lo, hi] with off[L] >= e (hi if none)
__device__ __forceinline__ int64_t leaf_lower(const int64_t* __restrict__ off, int64_t lo,
                                              int64_t hi, int64_t e)
{
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (__ldg(off + mid) < e)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// ------------------------------------------------------------ reduction

// Run bookkeeping of one warp range.  A "run" is a maximal set of consecutive
// rows of the same leaf.  A leaf's info word = 128 * (scale exponent s) +
// 2 * (p_leaf + 1) + complete, where complete means the leaf lies wholly in
// [e_lo, e_hi) and p_leaf = -1 marks an invalid leaf degree (all zero).
// Moments above p_leaf are computed like the others and dropped here, when
// the leaf's sums are finished.
struct RangeCtx {
    int64_t w, e_lo, e_hi, L_first;
    int d_out0, d_out1, d_out2;           // hat depth of each output's level
    int shift_n00, shift_n01, shift_n02;  // shift = s * (n + shift_n0 of the output)
    int nacc;                             // outputs per leaf
    // (scalars with selects: an array indexed at run time would live in local memory)
    __device__ __forceinline__ int d_out(int ly) const { return ly == 0 ? d_out0 : ly == 1 ? d_out1 : d_out2; }
    __device__ __forceinline__ int shift_n0(int ly) const
    {
        return ly == 0 ? shift_n00 : ly == 1 ? shift_n01 : shift_n02;
    }
};

// The range walk's warp-uniform state.  FP32 keeps it in registers; FP64 keeps
// it in shared memory (WarpWalk, written by lane 0, read through a volatile
// pointer), since values live across the degree loop would otherwise hold
// registers beside its rows for the loop's whole length (the FP64 level-9
// kernel: 140 bytes of spill stores with them in registers, 8 without; 0.8 %
// of its time).  In FP32 the extra shared-memory reads cost 6 %.
struct WarpWalk {
    int64_t w, e_lo, e_hi, L_first, L_last;
    int64_t e_cur;      // first element of the current round
    int64_t open_leaf;  // leaf of the run open at the start of the round
    int open_info;
    unsigned gstart;    // groups of the round that start a new leaf (bit 4g)
    int n_taken;        // elements of the round
    int last;           // last active lane of the round
};
#define Q2X_WALK_FIELDS(X)                                                                         \
    X(int64_t, w) X(int64_t, e_lo) X(int64_t, e_hi) X(int64_t, L_first) X(int64_t, L_last)     \
        X(int64_t, e_cur) X(int64_t, open_leaf) X(int, open_info) X(unsigned, gstart) X(int, n_taken) X(int, last)
template <bool SMEM>
struct Walk;
template <>
struct Walk<false> {
    WarpWalk v;
    __device__ __forceinline__ Walk(WarpWalk*, int) {}
#define Q2X_WALK_REG(T, f)                                                                         \
    __device__ __forceinline__ T f() const { return v.f; }                                         \
    __device__ __forceinline__ void set_##f(T x) { v.f = x; }
    Q2X_WALK_FIELDS(Q2X_WALK_REG)
#undef Q2X_WALK_REG
    __device__ __forceinline__ void sync() const {}
};
template <>
struct Walk<true> {
    volatile WarpWalk* p;
    int lane;
    __device__ __forceinline__ Walk(WarpWalk* q, int l) : p(q), lane(l) {}
#define Q2X_WALK_SMEM(T, f)                                                                        \
    __device__ __forceinline__ T f() const { return p->f; }                                        \
    __device__ __forceinline__ void set_##f(T x) const                                             \
    {                                                                                              \
        if (lane == 0) p->f = x;                                                                   \
    }
    Q2X_WALK_FIELDS(Q2X_WALK_SMEM)
#undef Q2X_WALK_SMEM
    __device__ __forceinline__ void sync() const { __syncwarp(); }
};
#undef Q2X_WALK_FIELDS

// Running sum of one column over a leaf's rounds.  FP32: compensated (each
// round's 32-row partial is added by TwoSum and the rounding errors are
// accumulated beside the sum), so the leaf sum keeps FP32 accuracy relative
// to its own size however many rounds a leaf spans; all on the FP32 pipe.
// FP64: a plain sum.  8 bytes either way.
template <typename T>
struct LeafSum;
template <>
struct LeafSum<float> {
    float s, c;
    __device__ __forceinline__ void zero() { s = c = 0.f; }
    __device__ __forceinline__ void add(float x)
    {
        const float t = s + x;  // TwoSum: t + e = s + x exactly
        const float bp = t - s;
        c += (s - (t - bp)) + (x - bp);
        s = t;
    }
    __device__ __forceinline__ float rounded() const { return s + c; }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }  // exact
};
template <>
struct LeafSum<double> {
    double s;
    __device__ __forceinline__ void zero() { s = 0.0; }
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double rounded() const { return s; }
    __device__ __forceinline__ double value() const { return s; }
};
static_assert(sizeof(LeafSum<float>) == 8 && sizeof(LeafSum<double>) == 8, "shared-memory layout assumes 8 bytes");

// Flush a column's leaf sum: a complete leaf is finished and written; a leaf
// that straddles the range goes to its FP64 slot partial.
template <typename T>
__device__ __forceinline__ void flush_value(const ElemArgs& a, const RangeCtx& rc, int ly, int c,
                                            const LeafSum<T>& acc, long long L, int info)
{
    if (info & 1) {
        const int desc = col_desc(c);
        double v = 0.0;
        if ((desc & 31) < ((info >> 1) & 63))  // n <= p_leaf
            v = finish_desc(acc.rounded(), a.norm, desc, rc.d_out(ly), rc.shift_n0(ly), info >> 7);
        double* dst = a.coef[ly] + (int64_t)L * a.np_max + c;
        if (a.accumulate)
            *dst += v;
        else
            *dst = v;
    } else {
        const int slot = (L == rc.L_first) ? 0 : 1;
        a.slots[((rc.w * 2 + slot) * rc.nacc + ly) * (int64_t)a.np_max + c] = acc.value();
    }
}

// Sums of the eight groups of four rows of a staged column (rows 4g..4g+3 to
// s[g], each as (r0 + r1) + (r2 + r3)); all loads independent.
__device__ __forceinline__ void group_sums(const float* col, float (&s)[8])
{
    float4 v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = *reinterpret_cast<const float4*>(col + 4 * i);
#pragma unroll
    for (int i = 0; i < 8; ++i) s[i] = (v[i].x + v[i].y) + (v[i].z + v[i].w);
}
__device__ __forceinline__ void group_sums(const double* col, double (&s)[8])
{
#pragma unroll
    for (int i = 0; i < 8; ++i) s[i] = (col[4 * i] + col[4 * i + 1]) + (col[4 * i + 2] + col[4 * i + 3]);
}

// Sum of s[g] over groups g0 <= g < g1 as a fixed pairwise tree (groups
// outside the interval contribute exact zeros).
template <typename T>
__device__ __forceinline__ T tree8(const T (&s)[8], int g0, int g1)
{
    T t[8];
#pragma unroll
    for (int g = 0; g < 8; ++g) t[g] = (g >= g0 && g < g1) ? s[g] : T(0);
    return ((t[0] + t[1]) + (t[2] + t[3])) + ((t[4] + t[5]) + (t[6] + t[7]));
}

// Sum of all 32 rows of a column (the single-leaf tiles of the batch kernel)
// as a fixed pairwise tree.  FP32: with paired adds, rows r and r + 2 of each
// group of four first, then the groups pairwise, both halves at once (15
// paired adds and one scalar add instead of 31 adds).
template <typename T>
__device__ __forceinline__ T sum_rows32(const T* col)
{
    T s[8];
    group_sums(col, s);
    return ((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7]));
}
template <>
__device__ __forceinline__ float sum_rows32<float>(const float* col)
{
    float4 v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = *reinterpret_cast<const float4*>(col + 4 * i);
    cf a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = cf_add(cf_make(v[i].x, v[i].y), cf_make(v[i].z, v[i].w));
    const cf d = cf_add(cf_add(cf_add(a[0], a[1]), cf_add(a[2], a[3])), cf_add(cf_add(a[4], a[5]), cf_add(a[6], a[7])));
    float x, y;
    cf_parts(d, x, y);
    return x + y;
}

// Per-element expansions (no leaves): row r of a staged chunk is the complete
// expansion of element rowleaf[r], finished and written directly.  Out of
// line, a call made in that mode only, so that the leaf-mode degree loop does
// not carry this code: the element kernel is sensitive to instruction fetch
// (compiled out, the path's inlined copy cost 3 % of the level-9 FP32 step).
template <typename T, int CH>
__device__ __noinline__ void flush_rows_per_elem(const T* tile, const long long* rowleaf, const int* rowinfo,
                                                 int nrows, int c0, int ncols, bool want0, bool want1,
                                                 double* coef0, double* coef1, int np, int norm, int accumulate,
                                                 int d0, int d1, int sh0, int sh1)
{
    constexpr int LD = KCfg<T>::LD;
    const int lane = threadIdx.x & 31;
    const int total = ((want0 ? 1 : 0) + (want1 ? 1 : 0)) * ncols;
    for (int i = lane; i < nrows * total; i += 32) {
        const int r = i / total, tc = i - r * total;
        const int second = (tc >= ncols) ? 1 : 0;
        const int ly = want0 ? second : 1;
        const int j = tc - second * ncols, c = c0 + j;
        const int info = rowinfo[r];
        const int desc = col_desc(c);
        double v = 0.0;
        if ((desc & 31) < ((info >> 1) & 63))  // n <= p of the element
            v = finish_desc(tile[(ly * CH + j) * LD + r], norm, desc, ly == 0 ? d0 : d1, ly == 0 ? sh0 : sh1,
                            info >> 7);
        double* dst = (ly == 0 ? coef0 : coef1) + (int64_t)rowleaf[r] * np + c;
        if (accumulate)
            *dst += v;
        else
            *dst = v;
    }
}

// Segmented column sums of one staged chunk: columns [c0, c0 + ncols) of each
// wanted layer.  Rows come in eight groups of four lanes; a leaf always starts
// at a group boundary (the round assigns elements to lanes that way; padding
// and idle lanes hold exact zeros), so a column is reduced by its eight group
// sums: one pairwise tree when the whole round belongs to the open run
// (gstart == 0), else the runs between the set bits of gstart (bit 4g: group
// g starts a new leaf, whose id and info are rowleaf[4g], rowinfo[4g]) are
// summed and flushed in order.  The wanted layers' columns form one index
// space; lane j owns indices j, j+32, ...; the open run's sum lives in accb
// between chunks and rounds (a LeafSum: compensated in FP32).  Per-element
// expansions (no leaves): flush_rows_per_elem, out of line.
// All control flow is warp-uniform.
template <typename T, int CH = KCfg<T>::CHUNK>
__device__ __forceinline__ void reduce_chunk(const ElemArgs& a, const RangeCtx& rc, const T* tile,
                                             LeafSum<T>* accb, const long long* rowleaf, const int* rowinfo,
                                             long long open_leaf, int open_info, unsigned gstart,
                                             int nrows, int c0, int ncols, bool want0, bool want1,
                                             bool per_elem)
{
    constexpr int LD = KCfg<T>::LD;
    const int lane = threadIdx.x & 31;
    const int nlay = (want0 ? 1 : 0) + (want1 ? 1 : 0);
    const int total = nlay * ncols;
    if (per_elem) {
        flush_rows_per_elem<T, CH>(tile, rowleaf, rowinfo, nrows, c0, ncols, want0, want1, a.coef[0], a.coef[1],
                                   a.np_max, a.norm, a.accumulate, rc.d_out(0), rc.d_out(1), rc.shift_n0(0),
                                   rc.shift_n0(1));
        return;
    }
#pragma unroll 1
    for (int tc = lane; tc < total; tc += 32) {
        const int second = (tc >= ncols) ? 1 : 0;
        const int ly = want0 ? second : 1;
        const int j = tc - second * ncols;
        const int c = c0 + j;
        T s[8];
        group_sums(tile + (ly * CH + j) * LD, s);
        LeafSum<T> acc = accb[ly * a.np_max + c];
        if (gstart == 0) {
            acc.add(((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7])));
        } else {
            long long L = open_leaf;
            int info = open_info;
            unsigned mask = gstart;
            int g0 = 0;
            while (mask) {
                const int r = __ffs(mask) - 1;
                const int g1 = r >> 2;
                acc.add(tree8(s, g0, g1));
                flush_value<T>(a, rc, ly, c, acc, L, info);
                acc.zero();
                L = rowleaf[r];
                info = rowinfo[r];
                g0 = g1;
                mask &= mask - 1;
            }
            acc.add(tree8(s, g0, 8));
        }
        accb[ly * a.np_max + c] = acc;
    }
}

// four consecutive values of a staged column (FP32 columns are 16-byte
// aligned; FP64 columns only 8-byte aligned, LD = 33), and of a 16-byte
// aligned shared array
__device__ __forceinline__ void load4_col(const float* p, float (&v)[4])
{
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
}
__device__ __forceinline__ void load4_col(const double* p, double (&v)[4])
{
    v[0] = p[0], v[1] = p[1], v[2] = p[2], v[3] = p[3];
}
__device__ __forceinline__ void load4_aligned(const float* p, float (&v)[4]) { load4_col(p, v); }
__device__ __forceinline__ void load4_aligned(const double* p, double (&v)[4])
{
    const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
    v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
}

// Vector density (segments carrying a 3-component current): the staged rows
// are the elements' unit-density moments, and component j of a leaf's sum is
// the sum over its rows of w_j(row) * row, w_j the element's j-th component
// (rowwt[j][32] in shared memory): the three components of Eq. (st3) from one
// recursion pass.  Per column and component, each group of four rows gives a
// weighted group sum (one multiply-add per row); the group sums are reduced
// and flushed per leaf like reduce_chunk's, each component into its own
// output (the column is re-read from shared memory per component, so the
// group sums stay in registers).  Leaf mode only.
template <typename T>
__device__ __forceinline__ void reduce_chunk_vec(const ElemArgs& a, const RangeCtx& rc, const T* tile,
                                                 LeafSum<T>* accb, const T* rowwt, const long long* rowleaf,
                                                 const int* rowinfo, long long open_leaf, int open_info,
                                                 unsigned gstart, int c0, int ncols)
{
    constexpr int LD = KCfg<T>::LD;
    const int lane = threadIdx.x & 31;
#pragma unroll 1
    for (int j = lane; j < ncols; j += 32) {
        const int c = c0 + j;
        const T* col = tile + j * LD;
#pragma unroll 1
        for (int q = 0; q < 3; ++q) {
            if (a.coef[q] == nullptr) continue;
            T s[8];
#pragma unroll
            for (int g = 0; g < 8; ++g) {
                T v[4], wq[4];
                load4_col(col + 4 * g, v);
                load4_aligned(rowwt + q * 32 + 4 * g, wq);  // the same address in every lane (broadcast)
                s[g] = fma(wq[3], v[3], fma(wq[2], v[2], fma(wq[1], v[1], wq[0] * v[0])));
            }
            LeafSum<T> acc = accb[q * a.np_max + c];
            if (gstart == 0) {
                acc.add(((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7])));
            } else {
                long long L = open_leaf;
                int info = open_info;
                unsigned mask = gstart;
                int g0 = 0;
                while (mask) {
                    const int r = __ffs(mask) - 1;
                    const int g1 = r >> 2;
                    acc.add(tree8(s, g0, g1));
                    flush_value<T>(a, rc, q, c, acc, L, info);
                    acc.zero();
                    L = rowleaf[r];
                    info = rowinfo[r];
                    g0 = g1;
                    mask &= mask - 1;
                }
                acc.add(tree8(s, g0, 8));
            }
            accb[q * a.np_max + c] = acc;
        }
    }
}

// ---------------------------------------------------------- chain layout

// Levels of the chain per element kind: the vertex of each level's stencil
// (0 = x1, 1 = x2, 2 = x3, 3 = x4).  Level k's source is level k-1's new value
// except for the linear-density chain (see the kernel).
template <int KIND, int DENS>
struct Chain;
template <>
struct Chain<KIND_SEG, DENS_CONST> {  // q (x2), p (x1)
    static constexpr int NL = 2, D_OUT = 1;
    __host__ __device__ static constexpr int vert(int k) { return k == 0 ? 1 : 0; }
};
template <>
struct Chain<KIND_TRI, DENS_CONST> {  // q (x2), j (x3), i (x1)
    static constexpr int NL = 3, D_OUT = 2;
    __host__ __device__ static constexpr int vert(int k) { return k == 0 ? 1 : k == 1 ? 2 : 0; }
};
template <>
struct Chain<KIND_TRI, DENS_LINEAR> {  // q (x2), j (x3), E (x3), i (x1), Iw (x1)
    static constexpr int NL = 5, D_OUT = 3;
    __host__ __device__ static constexpr int vert(int k) { return k == 0 ? 1 : (k == 1 || k == 2) ? 2 : 0; }
};
template <>
struct Chain<KIND_TET, DENS_CONST> {  // q (x2), j (x3), b (x4), a (x1)
    static constexpr int NL = 4, D_OUT = 3;
    __host__ __device__ static constexpr int vert(int k) { return k == 0 ? 1 : k == 1 ? 2 : k == 2 ? 3 : 0; }
};

// ------------------------------------------------------------------ kernel

// Per-lane element setup: gather the vertices of element e, translate them to
// the leaf centre (cx, cy, cz) and scale by 2^-sexp (FP32: from exact hi/lo
// splits of the FP64 inputs), read the densities, and form the stencil
// coefficients of every level of the chain, the unit normal (triangles) and
// the seed J * density (linear density: J).  In the FP32 path the seed is
// formed in FP64 (Jacobian of Eq. (map4) from the FP64 vertices, times the
// FP64 density) and rounded once to FP32; the densities the linear chain
// reads are rounded to FP32.  An inactive lane, a bad vertex index or a
// non-finite input gives an all-zero frame and pL = -1; errbits collects the
// device error bits.
template <typename T, int NL>
struct Frame {
    T LX[NL], LY[NL], LZ[NL];  // stencil vertex of each level: X = x/2, Y = y/2, z
    T XN, YN, ZN;              // the same for the unit normal (double layer)
    T s1, s2, s3;              // densities (vertex values for linear density)
    T seed;
    T J;                       // Jacobian in the scaled frame
    T eu[3], ev[3];            // edges x2 - x1, x3 - x1 (triangles; eu only for segments)
};

template <typename T, int KIND, int DENS, bool UNIT = false>
__device__ __forceinline__ void load_frame(const double* __restrict__ vx, const double* __restrict__ vy,
                                           const double* __restrict__ vz, const int32_t* __restrict__ idx,
                                           const double* __restrict__ sigma, int64_t n_elem, int64_t n_vert,
                                           int64_t e, bool active, double cx, double cy, double cz, int sexp,
                                           unsigned& errbits, int& pL,
                                           Frame<T, Chain<KIND, DENS>::NL>& F)
{
    using C = Chain<KIND, DENS>;
    constexpr int NL = C::NL;
    constexpr int NV = KIND + 2;
    constexpr bool FP32 = sizeof(T) == 4;
    constexpr bool LIN = (KIND == KIND_TRI && DENS == DENS_LINEAR);
    // ---- gather vertices into the scaled local frame
    T vxl[NV], vyl[NV], vzl[NV];
    T edge[NV - 1][3];  // x_k - x1 in the scaled frame, k = 2..NV
    T s1 = T(0), s2 = T(0), s3 = T(0);
    double xd[NV][3];   // FP32 path: the FP64 vertices, for the FP64 seed
    double dens0 = 0.0;
    bool bad = !active;
    {
        int64_t vid[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            int64_t v = active ? (int64_t)__ldg(idx + (int64_t)k * n_elem + e) : 0;
            if (v < 0 || v >= n_vert) {
                if (active) errbits |= 1u;
                bad = true;
                v = 0;
            }
            vid[k] = v;
        }
        double dens[3] = {UNIT ? 1.0 : 0.0, 0.0, 0.0};
        if (active && !UNIT) {
            if (DENS == DENS_LINEAR) {
#pragma unroll
                for (int k = 0; k < 3; ++k) dens[k] = __ldg(sigma + vid[k]);
            } else {
                dens[0] = __ldg(sigma + e);
            }
        }
        if constexpr (FP32) {
            bool nf = !(finite_bits(dens[0]) && finite_bits(dens[1]) && finite_bits(dens[2]));
            s1 = __double2float_rn(dens[0]);
            s2 = __double2float_rn(dens[1]);
            s3 = __double2float_rn(dens[2]);
            dens0 = dens[0];
            float sh[NV][3], sl[NV][3];
            float chx, clx, chy, cly, chz, clz;
            split_f64(cx, chx, clx, nf);
            split_f64(cy, chy, cly, nf);
            split_f64(cz, chz, clz, nf);
            const float inv = pow2f(-sexp);
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                float hx, lx, hy, ly, hz, lz;
                xd[k][0] = active ? __ldg(vx + vid[k]) : 0.0;
                xd[k][1] = active ? __ldg(vy + vid[k]) : 0.0;
                xd[k][2] = active ? __ldg(vz + vid[k]) : 0.0;
                split_f64(xd[k][0], hx, lx, nf);
                split_f64(xd[k][1], hy, ly, nf);
                split_f64(xd[k][2], hz, lz, nf);
                vxl[k] = ((hx - chx) + (lx - clx)) * inv;
                vyl[k] = ((hy - chy) + (ly - cly)) * inv;
                vzl[k] = ((hz - chz) + (lz - clz)) * inv;
                sh[k][0] = hx;
                sh[k][1] = hy;
                sh[k][2] = hz;
                sl[k][0] = lx;
                sl[k][1] = ly;
                sl[k][2] = lz;
            }
            // edge vectors x_k - x1 from the exact splits: the hi parts of nearby
            // vertices subtract exactly, so the edges (hence J and the normal)
            // keep FP32 accuracy relative to the edge length itself
#pragma unroll
            for (int k = 1; k < NV; ++k)
#pragma unroll
                for (int d = 0; d < 3; ++d) edge[k - 1][d] = ((sh[k][d] - sh[0][d]) + (sl[k][d] - sl[0][d])) * inv;
            if (nf && active) {
                errbits |= 2u;
                bad = true;
            }
        } else {
            if (!(finite_bits(dens[0]) && finite_bits(dens[1]) && finite_bits(dens[2]))) {
                errbits |= 2u;
                bad = true;
            }
            s1 = dens[0];
            s2 = dens[1];
            s3 = dens[2];
            const double inv = pow2d(-sexp);
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                const double x = active ? __ldg(vx + vid[k]) : 0.0;
                const double y = active ? __ldg(vy + vid[k]) : 0.0;
                const double zz = active ? __ldg(vz + vid[k]) : 0.0;
                if (!(finite_bits(x) && finite_bits(y) && finite_bits(zz))) {
                    if (active) errbits |= 2u;
                    bad = true;
                }
                vxl[k] = (x - cx) * inv;
                vyl[k] = (y - cy) * inv;
                vzl[k] = (zz - cz) * inv;
            }
#pragma unroll
            for (int k = 1; k < NV; ++k) {
                edge[k - 1][0] = vxl[k] - vxl[0];
                edge[k - 1][1] = vyl[k] - vyl[0];
                edge[k - 1][2] = vzl[k] - vzl[0];
            }
        }
    }
    if (bad) {  // contributes exact zeros (no NaN can leak into the sums)
        pL = -1;
#pragma unroll
        for (int k = 0; k < NV; ++k) vxl[k] = vyl[k] = vzl[k] = T(0);
#pragma unroll
        for (int k = 0; k < NV - 1; ++k) edge[k][0] = edge[k][1] = edge[k][2] = T(0);
        s1 = s2 = s3 = T(0);
    }

    // ---- Jacobian in the scaled frame, unit normal, seed
    T J, nx = T(0), ny = T(0), nz = T(0);
    {
        const T ux = edge[0][0], uy = edge[0][1], uz = edge[0][2];
        if constexpr (KIND == KIND_SEG) {
            J = sqrt(ux * ux + uy * uy + uz * uz);
        } else {
            const T wx = edge[NV >= 3 ? 1 : 0][0], wy = edge[NV >= 3 ? 1 : 0][1], wz = edge[NV >= 3 ? 1 : 0][2];
            const T cxp = uy * wz - uz * wy, cyp = uz * wx - ux * wz, czp = ux * wy - uy * wx;
            if constexpr (KIND == KIND_TRI) {
                J = sqrt(cxp * cxp + cyp * cyp + czp * czp);
                const T inv = (J > T(0)) ? T(1) / J : T(0);
                nx = cxp * inv;
                ny = cyp * inv;
                nz = czp * inv;
            } else {
                const T tx = edge[NV - 2][0], ty = edge[NV - 2][1], tz = edge[NV - 2][2];
                J = fabs(cxp * tx + cyp * ty + czp * tz);
            }
        }
    }
    T seed;
    if constexpr (FP32) {
        // Jacobian (Eq. (map4)) and seed in FP64, once per element; the frame
        // scale 2^-sexp enters as an exact power of two per dimension
        double ed[NV - 1][3];
#pragma unroll
        for (int k = 1; k < NV; ++k)
#pragma unroll
            for (int d = 0; d < 3; ++d) ed[k - 1][d] = xd[k][d] - xd[0][d];
        double J64;
        if constexpr (KIND == KIND_SEG) {
            J64 = sqrt(ed[0][0] * ed[0][0] + ed[0][1] * ed[0][1] + ed[0][2] * ed[0][2]);
        } else {
            const int kv = NV >= 3 ? 1 : 0;
            const double qx = ed[0][1] * ed[kv][2] - ed[0][2] * ed[kv][1];
            const double qy = ed[0][2] * ed[kv][0] - ed[0][0] * ed[kv][2];
            const double qz = ed[0][0] * ed[kv][1] - ed[0][1] * ed[kv][0];
            if constexpr (KIND == KIND_TRI)
                J64 = sqrt(qx * qx + qy * qy + qz * qz);
            else
                J64 = fabs(qx * ed[NV - 2][0] + qy * ed[NV - 2][1] + qz * ed[NV - 2][2]);
        }
        J64 *= pow2d(-(KIND + 1) * sexp);
        const double seed64 = LIN ? J64 : J64 * dens0;
        seed = (bad || pL < 0) ? 0.f : __double2float_rn(seed64);
    } else {
        seed = LIN ? J : J * s1;
        if (pL < 0) seed = T(0);
    }

    // stencil coefficients of each level: X = x/2, Y = y/2, z
#pragma unroll
    for (int k = 0; k < NL; ++k) {
        const int v = C::vert(k);
        F.LX[k] = T(0.5) * vxl[v];
        F.LY[k] = T(0.5) * vyl[v];
        F.LZ[k] = vzl[v];
    }
    F.XN = T(0.5) * nx;
    F.YN = T(0.5) * ny;
    F.ZN = nz;
    F.s1 = s1;
    F.s2 = s2;
    F.s3 = s3;
    F.seed = seed;
    F.J = J;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        F.eu[d] = edge[0][d];
        F.ev[d] = edge[NV >= 3 ? 1 : 0][d];
    }

}

// The degree loop of one round: advance every level of the chain from degree
// 0 to pw (rows in registers; the order loop is unrolled to the capacity P),
// stage each degree's single- and double-layer values of this lane's element
// in column order of the stage tile (layer 1 at tile + CHUNK*LD), and call
// reduce(c0, ncols) whenever a chunk of columns [c0, c0 + ncols) is complete.
//
// FP64: the rows of levels k < NS live in shared memory (srows, [NS][P + 1][32]
// complex entries, one 16-byte entry per lane and order) instead of registers;
// ElemCfg chooses NS and the stage-tile width CH.
template <typename T, int P, int KIND, int DENS, int OUTS, bool WIDE = false, int NS = 0,
          int CH = KCfg<T>::CHUNK, typename Reduce>
__device__ __forceinline__ void run_chain(const Frame<T, Chain<KIND, DENS>::NL>& F, int pw, T* tile,
                                          int lane, Reduce&& reduce, double2* srows = nullptr)
{
    using C = Chain<KIND, DENS>;
    constexpr int NL = C::NL;
    constexpr int OUT = NL - 1;
    constexpr int LD = KCfg<T>::LD;
    constexpr bool FP32 = sizeof(T) == 4;
    constexpr bool LIN = (KIND == KIND_TRI && DENS == DENS_LINEAR);
    constexpr bool want0 = (OUTS & 1) != 0;
    constexpr bool want1 = (KIND == KIND_TRI) && (OUTS & 2) != 0;
    // columns staged per chunk: a single-layer pass may use both halves of a
    // two-layer tile (WIDE), which halves the reductions per round
    constexpr int CAP = (WIDE && !want1) ? 2 * CH : CH;
    static_assert(NS == 0 || (sizeof(T) == 8 && NS < NL), "shared-memory rows: FP64 levels below the output");
    static_assert(CAP >= 2 * P + 1, "a chunk must hold one degree's columns");
    const T s1 = F.s1, s2 = F.s2, s3 = F.s3, seed = F.seed;
    const T XN = F.XN, YN = F.YN, ZN = F.ZN;
    const T* LX = F.LX;
    const T* LY = F.LY;
    const T* LZ = F.LZ;
    // Degree loop at run time (compact code).  The order loop is unrolled to
    // the capacity P so every row entry stays in a register; orders above n
    // are skipped by warp-uniform branches.
    int nb = 0;  // first degree of the chunk being staged
    if constexpr (FP32) {
        // ---- FP32: packed complex arithmetic, orders 0..n of each degree
        // (the unrolled order loop leaves at the first order above n, one
        // uniform branch per order; separate tests of every order cost 19 %)
        cf X2[NL], YmY[NL], nZ2[NL];
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            X2[k] = cf_make(LX[k], LX[k]);
            YmY[k] = cf_make(LY[k], -LY[k]);
            nZ2[k] = cf_make(-LZ[k], -LZ[k]);
        }
        const cf XN2 = cf_make(XN, XN), YNm = cf_make(YN, -YN), nZN2 = cf_make(-ZN, -ZN);
        const cf s1p = cf_make(s1, s1), s3p = cf_make(s3, s3);
        cf R[NL][P + 1];
#pragma unroll
        for (int k = 0; k < NL; ++k)
#pragma unroll
            for (int m = 0; m <= P; ++m) R[k][m] = cf_zero();
#pragma unroll 1
        for (int n = 0; n <= pw; ++n) {
            float* trow0 = reinterpret_cast<float*>(tile) + (n * n - nb * nb + n) * LD + lane;
            float* trow1 = trow0 + CH * LD;
            const float c2f = (float)(n + 1) * (float)s2;
            const cf c2p = cf_make(c2f, c2f);
            const cf sd = cf_make((n == 0) ? (float)seed : 0.f, 0.f);
            // The neighbours (b - a, a + b) of order m + 1 are formed at order
            // m, before x^m is replaced: the new entry then takes the old
            // one's register (formed at order m + 1, the old x^m would stay
            // live beside the new one and cost a register copy per entry).
            cf_nb nbn[NL];
#pragma unroll
            for (int m = 0; m <= P; ++m) {
                if (m > n) break;
                cf nw[NL];
#pragma unroll
                for (int k = 0; k < NL; ++k) {
                    const cf c = R[k][m];
                    // m = 0 (Eq. (rec11)): 2 Re(eta b) - z c + src, real; scalar
                    float br0 = 0.f, bi0 = 0.f, cr0 = 0.f, ci0 = 0.f;
                    if (m == 0) {
                        const cf b = (P > 0) ? R[k][P > 0 ? 1 : 0] : cf_zero();
                        cf_parts(b, br0, bi0);
                        cf_parts(c, cr0, ci0);
                    }
                    const cf_nb nbk = (m == 0) ? cf_nb{cf_zero(), cf_zero()} : nbn[k];
                    if (m < P) nbn[k] = cf_neighbours(c, (m + 2 <= P) ? R[k][m + 2 <= P ? m + 2 : P] : cf_zero());
                    if (KIND == KIND_TRI && k == OUT && want1) {
                        // double layer from the output level's row n-1
                        float dr, di;
                        if (m == 0) {
                            dr = fmaf(2.f * XN, br0, fmaf(2.f * YN, bi0, -ZN * cr0));
                            di = 0.f;
                        } else {
                            cf dl = cf_stencil_nb(nbk, c, cf_zero(), XN2, YNm, nZN2);
                            cf_parts(dl, dr, di);
                        }
                        trow1[m * LD] = (m & 1) ? di : dr;
                        if (m > 0) trow1[-m * LD] = (m & 1) ? dr : di;
                    }
                    cf src;
                    if (k == 0)
                        src = (m == 0) ? sd : cf_zero();
                    else if (LIN && k == 2)
                        src = cf_fma(c2p, nw[0], cf_mul(s3p, nw[1]));  // (n+1) s2 q^ + s3 j^
                    else if (LIN && k == 3)
                        src = nw[1];  // i^ <- j^
                    else if (LIN && k == 4)
                        src = cf_fma(s1p, nw[3], nw[2]);  // E^ + s1 i^
                    else
                        src = nw[k > 0 ? k - 1 : 0];
                    if (m == 0) {
                        float sr0, si0;
                        cf_parts(src, sr0, si0);
                        nw[k] = cf_make(fmaf(2.f * LX[k], br0, fmaf(2.f * LY[k], bi0, fmaf(-LZ[k], cr0, sr0))), 0.f);
                    } else {
                        nw[k] = cf_stencil_nb(nbk, c, src, X2[k], YmY[k], nZ2[k]);
                    }
                    R[k][m] = nw[k];
                }
                if (want0) {
                    float vr, vi;
                    cf_parts(nw[OUT], vr, vi);
                    trow0[m * LD] = (m & 1) ? vi : vr;
                    if (m > 0) trow0[-m * LD] = (m & 1) ? vr : vi;
                }
            }
            if (n == pw || (n + 2) * (n + 2) - nb * nb > CAP) {
                __syncwarp();
                reduce(nb * nb, (n + 1) * (n + 1) - nb * nb);
                __syncwarp();
                nb = n + 1;
            }
        }
    } else {
        // ---- FP64: scalar arithmetic, exact order bounds, orders from n down
        // to 0.  Level 0 (the point level) is T_n^m = w_m Q_n^m with the
        // element's w_m = seed (-xi)^m (its row: computed once, read-only)
        // and Q_n^m from the order recursion of g_qtab, carried in two
        // scalars.  Levels k >= 1 use the stencil: the old entry m - 1 is
        // still in the row, the old entry m + 1 is carried down from the
        // previous order.  The first two orders of each degree (m = n, n - 1)
        // use specialised bodies without the neighbours known to vanish, so no
        // DFMA is spent on zero operands.
        T Rr[NL][P + 1], Ri[NL][P + 1];
#pragma unroll
        for (int k = 0; k < NL; ++k)
#pragma unroll
            for (int m = 0; m <= P; ++m) Rr[k][m] = Ri[k][m] = T(0);
        {
            T wr = seed, wi = T(0);
            const T mx = -LX[0], my = -LY[0];
            static_for<0, P + 1>([&](auto m_c) {
                constexpr int m = decltype(m_c)::value;
                if (m <= pw) {
                    if (m > 0) {
                        const T tr = fma(wr, mx, -wi * my);
                        wi = fma(wr, my, wi * mx);
                        wr = tr;
                    }
                    if (NS > 0)
                        srows[m * 32 + lane] = make_double2(wr, wi);
                    else
                        Rr[0][m] = wr, Ri[0][m] = wi;
                }
            });
        }
        const T zq = LZ[0], x2q = fma(LX[0], LX[0], LY[0] * LY[0]);  // z and |xi|^2 of the point level
#pragma unroll 1
        for (int n = 0; n <= pw; ++n) {
            T* trow0 = tile + (n * n - nb * nb + n) * LD + lane;
            T* trow1 = trow0 + CH * LD;
            const T c2 = T(n + 1) * s2;
            const T nz = -T(n) * zq;  // Q_n^{n-1}
            const double* qa = g_qtab.a + n * (Q2X_P_MAX + 1);
            const double* qb = g_qtab.b + n * (Q2X_P_MAX + 1);
            T Q1 = T(0), Q2 = T(0);   // Q_n^{m+1}, Q_n^{m+2}
            T br[NL], bi[NL];         // old entry m + 1 of each level
#pragma unroll
            for (int k = 0; k < NL; ++k) br[k] = bi[k] = T(0);
            // body of order m; HB: old entry m + 1 present, HC: old entry m present
            auto body = [&](auto m_c, auto hb_c, auto hc_c) {
                constexpr int m = decltype(m_c)::value;
                constexpr bool HB = decltype(hb_c)::value && (m < P);
                constexpr bool HC = decltype(hc_c)::value;
                T nr[NL], ni[NL];
                {
                    T Q;
                    if (!HC)
                        Q = T(1);  // m = n
                    else if (!HB)
                        Q = nz;  // m = n - 1
                    else
                        Q = fma(qa[m] * zq, Q1, (qb[m] * x2q) * Q2);
                    Q2 = Q1;
                    Q1 = Q;
                    T wr, wi;
                    if (NS > 0) {
                        const double2 v = srows[m * 32 + lane];
                        wr = v.x, wi = v.y;
                    } else {
                        wr = Rr[0][m], wi = Ri[0][m];
                    }
                    if (HC) {
                        nr[0] = wr * Q;
                        ni[0] = (m == 0) ? T(0) : wi * Q;
                    } else {
                        nr[0] = wr;
                        ni[0] = (m == 0) ? T(0) : wi;
                    }
                }
#pragma unroll
                for (int k = 1; k < NL; ++k) {
                    // degree n-1 entries m - 1 (a) and m (c) from the row; m + 1 (b) carried
                    T ar = T(0), ai = T(0), cr = T(0), ci = T(0);
                    const T bR = HB ? br[k] : T(0), bI = HB ? bi[k] : T(0);
                    if (k < NS) {
                        if (m > 0) {
                            const double2 v = srows[(k * (P + 1) + (m > 0 ? m - 1 : 0)) * 32 + lane];
                            ar = v.x, ai = v.y;
                        }
                        if (HC) {
                            const double2 v = srows[(k * (P + 1) + m) * 32 + lane];
                            cr = v.x, ci = v.y;
                        }
                    } else {
                        if (m > 0) ar = Rr[k][m > 0 ? m - 1 : 0], ai = Ri[k][m > 0 ? m - 1 : 0];
                        if (HC) cr = Rr[k][m], ci = Ri[k][m];
                    }
                    if (KIND == KIND_TRI && k == OUT && want1) {
                        T dr = T(0), di = T(0);
                        if (m == 0) {
                            if (HB) dr = fma(T(2) * XN, bR, fma(T(2) * YN, bI, dr));
                            if (HC) dr = fma(-ZN, cr, dr);
                        } else {
                            if (HB) {
                                dr = fma(XN, bR - ar, fma(YN, bI + ai, dr));
                                di = fma(XN, bI - ai, fma(-YN, bR + ar, di));
                            } else {
                                dr = fma(-XN, ar, fma(YN, ai, dr));
                                di = fma(-XN, ai, fma(-YN, ar, di));
                            }
                            if (HC) {
                                dr = fma(-ZN, cr, dr);
                                di = fma(-ZN, ci, di);
                            }
                        }
                        trow1[m * LD] = (m & 1) ? di : dr;
                        if (m > 0) trow1[-m * LD] = (m & 1) ? dr : di;
                    }
                    T sr, si;
                    if (LIN && k == 2) {
                        sr = fma(c2, nr[0], s3 * nr[1]);
                        si = fma(c2, ni[0], s3 * ni[1]);
                    } else if (LIN && k == 3) {
                        sr = nr[1];
                        si = ni[1];
                    } else if (LIN && k == 4) {
                        sr = fma(s1, nr[3], nr[2]);
                        si = fma(s1, ni[3], ni[2]);
                    } else {
                        sr = nr[k - 1];
                        si = ni[k - 1];
                    }
                    T vr = sr, vi = (m == 0) ? T(0) : si;
                    if (m == 0) {
                        if (HB) vr = fma(T(2) * LY[k], bI, fma(T(2) * LX[k], bR, vr));
                        if (HC) vr = fma(-LZ[k], cr, vr);
                    } else {
                        if (HB) {
                            vr = fma(LY[k], bI + ai, fma(LX[k], bR - ar, vr));
                            vi = fma(-LY[k], bR + ar, fma(LX[k], bI - ai, vi));
                        } else {
                            vr = fma(LY[k], ai, fma(-LX[k], ar, vr));
                            vi = fma(-LY[k], ar, fma(-LX[k], ai, vi));
                        }
                        if (HC) {
                            vr = fma(-LZ[k], cr, vr);
                            vi = fma(-LZ[k], ci, vi);
                        }
                    }
                    nr[k] = vr;
                    ni[k] = vi;
                    br[k] = cr;
                    bi[k] = ci;
                    if (k < NS) {
                        srows[(k * (P + 1) + m) * 32 + lane] = make_double2(vr, vi);
                    } else {
                        Rr[k][m] = vr;
                        Ri[k][m] = vi;
                    }
                }
                if (want0) {
                    T vr = nr[OUT], vi = ni[OUT];
                    trow0[m * LD] = (m & 1) ? vi : vr;
                    if (m > 0) trow0[-m * LD] = (m & 1) ? vr : vi;
                }
            };
            using TT = std::integral_constant<bool, true>;
            using FF = std::integral_constant<bool, false>;
            static_for<0, P + 1>([&](auto i_c) {
                constexpr int m = P - decltype(i_c)::value;
                using MC = std::integral_constant<int, m>;
                if (m + 1 < n)
                    body(MC{}, TT{}, TT{});
                else if (m + 1 == n)
                    body(MC{}, FF{}, TT{});
                else if (m == n)
                    body(MC{}, FF{}, FF{});
            });
            if (n == pw || (n + 2) * (n + 2) - nb * nb > CAP) {
                __syncwarp();
                reduce(nb * nb, (n + 1) * (n + 1) - nb * nb);
                __syncwarp();
                nb = n + 1;
            }
        }
    }
}

// Output slots per leaf of an element-kernel instantiation: the three
// components of a vector density, the two layers when the double layer is
// requested (slot 1; slot 0 is the single layer), else the single layer only.
__host__ __device__ constexpr int elem_outputs(int kind, int outs)
{
    return (outs & 4) ? 3 : (kind == KIND_TRI && (outs & 2)) ? 2 : 1;
}

// Shared memory per warp: stage tile [2 layers][CHUNK][LD] of T, open-run sums
// [nacc outputs][np_max] (LeafSum, 8 bytes), row leaves [32], row infos [32],
// the walk state (FP64), with a vector density the row weights [3][32] of T between the tile and the
// sums (the tile's size keeps them 16-byte aligned).
// (rounded up to 128 bytes so every warp's tile keeps the 16-byte alignment of
// the 128-bit column loads)
template <typename T>
__host__ __device__ constexpr size_t warp_smem_bytes(int np_max, int nacc = 2, int ch = KCfg<T>::CHUNK)
{
    return (sizeof(T) * (size_t)(2 * ch * KCfg<T>::LD + (nacc == 3 ? 96 : 0)) +
            sizeof(LeafSum<T>) * (size_t)(nacc * np_max) + sizeof(long long) * 32 + sizeof(int) * 32 +
            sizeof(WarpWalk) + 127) / 128 * 128;
}

// Stage-tile width and shared-memory rows of one element-kernel
// instantiation.  FP64 runs two CTAs of four warps per SM (two warps per
// sub-partition, 255 registers each); rows of NL (P + 1) complex FP64 entries
// beyond about 140 registers spill, so the lowest levels move to shared
// memory (run_chain's NS), as many as that needs and the SM's 228 KB leave
// room for: 28,928 bytes per warp ((228 KB - 2 x 1 KB reserved) / 8), with a
// stage tile narrowed to 32 columns per layer, which is done only where a
// chunk still holds one degree's 2P + 1 columns.  The FP64 pipe retires one
// warp FMA in about 64 cycles, so a stencil's two 16-byte shared loads and one
// store per lane cost nothing measurable; they replace local-memory spills.
// FP32 keeps every row in registers and 48 columns per layer.
template <typename T, int P, int KIND, int DENS, int OUTS>
struct ElemCfg {
    static constexpr int NL = Chain<KIND, DENS>::NL;
    static constexpr int NACC = elem_outputs(KIND, OUTS);
    static constexpr bool TWO_LAYERS = KIND == KIND_TRI && (OUTS & 2) != 0;
    static constexpr int CH_NARROW = 32;
    static constexpr int ns_narrow()
    {
        if (sizeof(T) == 4) return 0;
        if ((TWO_LAYERS ? CH_NARROW : 2 * CH_NARROW) < 2 * P + 1) return 0;
        const size_t per_warp = (228 * 1024 - 2 * 1024) / 8;
        const size_t base = warp_smem_bytes<double>((P + 1) * (P + 1), NACC, CH_NARROW);
        const size_t level = (size_t)(P + 1) * 32 * 16;
        int ns = 0;
        while (ns < NL - 1 && (NL - ns) * (P + 1) * 4 > 140 && base + (size_t)(ns + 1) * level <= per_warp) ++ns;
        return ns;
    }
    static constexpr int NS = ns_narrow();
    static constexpr int CH = NS > 0 ? CH_NARROW : KCfg<T>::CHUNK;
    static constexpr size_t ROW_BYTES = (size_t)NS * (P + 1) * 32 * 16;  // [NS][P + 1][32] double2
    __host__ __device__ static constexpr size_t warp_bytes(int np_max)
    {
        return warp_smem_bytes<T>(np_max, NACC, CH) + ROW_BYTES;  // the first term is a multiple of 128
    }
};

// Resident CTAs per SM the element kernel is compiled for, which caps its
// registers: FP32 chains whose rows leave room run 4 warps per sub-partition
// (segments up to P = 16, constant-density single-layer triangles up to
// P = 8) or 3 (segments at P = 20, those triangles up to P = 20; at most 4
// bytes of spill stores), the rest, and FP64, 2 warps per sub-partition (no
// cap below 255 registers).
template <typename T, int P, int KIND, int DENS, int OUTS>
__host__ __device__ constexpr int min_ctas()
{
    if constexpr (sizeof(T) == 4) {
        if (KIND == KIND_SEG && OUTS == 1 && P <= 16) return 16;
        if (KIND == KIND_SEG && OUTS == 1) return 12;
        if (KIND == KIND_TRI && DENS == DENS_CONST && OUTS == 1 && P <= 8) return 16;
        if (KIND == KIND_TRI && DENS == DENS_CONST && OUTS == 1) return 12;
        return 8;
    } else {
        return 2;
    }
}

// OUTS: bit 0 = single layer, bit 1 = double layer (triangles), bit 2 = vector
// density (segments: three current components weighting one unit-density
// pass); a compile-time choice so each kernel holds exactly one copy of the
// degree loop.
template <typename T, int P, int KIND, int DENS, int OUTS>
__global__ void __launch_bounds__(elem_warps_per_cta<T>() * 32, (min_ctas<T, P, KIND, DENS, OUTS>()))
    q2x_elem_kernel(const ElemArgs a)
{
    using C = Chain<KIND, DENS>;
    constexpr int NL = C::NL;
    using Cfg = ElemCfg<T, P, KIND, DENS, OUTS>;
    constexpr int CH = Cfg::CH, LD = KCfg<T>::LD, NS = Cfg::NS;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int64_t w = (int64_t)blockIdx.x * elem_warps_per_cta<T>() + wib;
    if (w >= a.n_ranges) return;

    constexpr bool VEC = (OUTS & 4) != 0;  // vector density: three weighted outputs of one pass
    constexpr int NACC = elem_outputs(KIND, OUTS);
    unsigned char* wsm = smem_raw + (size_t)wib * Cfg::warp_bytes(a.np_max);
    double2* srows = reinterpret_cast<double2*>(wsm + warp_smem_bytes<T>(a.np_max, NACC, CH));  // NS > 0 only
    T* tile = reinterpret_cast<T*>(wsm);
    T* rowwt = tile + 2 * CH * LD;  // vector density only: [3][32]
    // 2 CH LD sizeof(T) and 96 sizeof(T) are multiples of 16
    LeafSum<T>* accb = reinterpret_cast<LeafSum<T>*>(tile + 2 * CH * LD + (VEC ? 96 : 0));
    long long* rowleaf = reinterpret_cast<long long*>(accb + NACC * a.np_max);
    int* rowinfo = reinterpret_cast<int*>(rowleaf + 32);
    Walk<sizeof(T) == 8> wk(reinterpret_cast<WarpWalk*>(rowinfo + 32), lane);  // 8-byte aligned

    constexpr bool want0 = (OUTS & 1) != 0 || VEC;
    constexpr bool want1 = (KIND == KIND_TRI) && (OUTS & 2) != 0;
    static_assert(NACC == (VEC ? 3 : want1 ? 2 : 1), "output slots");
    const bool per_elem = a.leaf_off == nullptr;
    const int np = a.np_max;
    const int pw = a.p_max;

    // the range and its constants
    auto range_ctx = [&]() {
        RangeCtx rc;
        rc.w = wk.w();
        rc.e_lo = wk.e_lo();
        rc.e_hi = wk.e_hi();
        rc.L_first = wk.L_first();
        // output 1 is the double layer (one hat degree less, scale exponent
        // n + 1), or a vector component (the single layer's constants)
        rc.d_out0 = rc.d_out2 = C::D_OUT;
        rc.d_out1 = VEC ? C::D_OUT : C::D_OUT - 1;
        rc.shift_n00 = rc.shift_n02 = KIND + 1;
        rc.shift_n01 = VEC ? KIND + 1 : 1;
        rc.nacc = NACC;
        return rc;
    };
    {
        const int64_t e_lo = w * a.T, e_hi = min(e_lo + a.T, a.n_elem);
        int64_t L_first, L_last;
        if (per_elem) {
            L_first = e_lo;
            L_last = e_hi - 1;
        } else {
            L_first = leaf_search(a.leaf_off, 0, a.n_leaves - 1, e_lo);
            L_last = leaf_search(a.leaf_off, L_first, a.n_leaves - 1, e_hi - 1);
        }
        wk.set_w(w);
        wk.set_e_lo(e_lo);
        wk.set_e_hi(e_hi);
        wk.set_L_first(L_first);
        wk.set_L_last(L_last);
        wk.set_e_cur(e_lo);
        wk.set_open_leaf(L_first);
        wk.sync();
    }

    for (int k = lane; k < NACC * np; k += 32) accb[k].zero();

    // zero the coefficients of empty leaves [La, Lb) (overwrite mode)
    auto zero_leaves = [&](int64_t La, int64_t Lb) {
        if (a.accumulate) return;
#pragma unroll 1
        for (int64_t L = La; L < Lb; ++L)
#pragma unroll 1
            for (int c = lane; c < np; c += 32) {
                if (VEC) {
#pragma unroll
                    for (int q = 0; q < 3; ++q)
                        if (a.coef[q]) a.coef[q][L * np + c] = 0.0;
                } else {
                    if (want0) a.coef[0][L * np + c] = 0.0;
                    if (want1) a.coef[1][L * np + c] = 0.0;
                }
            }
    };
    if (!per_elem) {
        zero_leaves(leaf_lower(a.leaf_off, 0, a.n_leaves, wk.e_lo()), wk.L_first());
        if (wk.e_hi() == a.n_elem) zero_leaves(wk.L_last() + 1, a.n_leaves);
    }

    auto leaf_info = [&](int64_t L) -> int {
        bool complete = true;
        if (!per_elem) complete = __ldg(a.leaf_off + L) >= wk.e_lo() && __ldg(a.leaf_off + L + 1) <= wk.e_hi();
        const int s = a.leaf_rho ? scale_exponent(__ldg(a.leaf_rho + L)) : 0;
        int pl = pw;
        if (a.leaf_p) {
            pl = __ldg(a.leaf_p + L);
            if (pl < 0 || pl > pw) pl = -1;
        }
        return s * 128 + (pl + 1) * 2 + (complete ? 1 : 0);
    };
    {
        const int oi = leaf_info(wk.L_first());
        wk.set_open_info(oi);
        __syncwarp();
    }

    // Rounds of at most 32 elements.  The next 32 elements of the range are
    // the candidates; candidate b that starts a new leaf is moved to the next
    // multiple of four lanes (the lanes skipped are padding), candidates that
    // no longer fit wait for the next round.  Per-element expansions take 32
    // consecutive elements without padding.
#pragma unroll 1
    while (true) {
        const int64_t e_cur = wk.e_cur(), e_hi = wk.e_hi();
        if (e_cur >= e_hi) break;
        const long long open_leaf = wk.open_leaf();
        const int64_t ec = e_cur + lane;
        const bool cand = ec < e_hi;
        int64_t Lc = open_leaf;
        if (cand) Lc = per_elem ? ec : leaf_search(a.leaf_off, open_leaf, wk.L_last(), ec);
        const long long Lcprev = __shfl_up_sync(0xffffffffu, (long long)Lc, 1);
        const bool cstart = cand && ((lane == 0) ? (Lc != open_leaf) : (Lc != Lcprev));
        const unsigned B = __ballot_sync(0xffffffffu, cstart);
        int my_off = 0;    // padding before this lane's candidate
        int src_off = 0;   // padding before this lane's position
        bool is_pad = false;
        if (!per_elem) {
            unsigned mk = B & ~1u;
            int O = 0;
            while (mk) {
                const int bb = __ffs(mk) - 1;
                mk &= mk - 1;
                const int pp = bb + O;  // position of candidate bb before its own padding
                if (pp >= 32) break;
                const int pad = (-pp) & 3;
                if (lane >= bb) my_off = O + pad;
                if (lane >= pp) {
                    is_pad = lane < pp + pad;
                    src_off = O + pad;
                }
                O += pad;
            }
        }
        const bool taken = cand && (lane + my_off) < 32;
        const int n_taken = __popc(__ballot_sync(0xffffffffu, taken));
        // this lane's element (position space)
        const int ci = lane - src_off;
        const bool active = !is_pad && ci < n_taken;
        const int64_t e = e_cur + ci;
        const long long Lsh = __shfl_sync(0xffffffffu, (long long)Lc, ci & 31);
        const int64_t L = active ? (int64_t)Lsh : (int64_t)open_leaf;
        // empty leaves between consecutive runs (overwrite mode)
        if (!per_elem && !a.accumulate) {
            unsigned mk = B & ((n_taken >= 32) ? 0xffffffffu : ((1u << n_taken) - 1u));
            while (mk) {
                const int bb = __ffs(mk) - 1;
                mk &= mk - 1;
                const long long cur = __shfl_sync(0xffffffffu, (long long)Lc, bb);
                const long long prv = __shfl_sync(0xffffffffu, Lcprev, bb);
                const long long prev = (bb == 0) ? open_leaf : prv;
                if (cur > prev + 1) zero_leaves(prev + 1, cur);
            }
        }

        // ---- this lane's leaf centre, scale, degree
        unsigned errbits = 0;
        int pL = pw, sexp = 0, info = 0;
        double cx = 0.0, cy = 0.0, cz = 0.0;
        if (active) {
            cx = __ldg(a.leaf_c + L);
            cy = __ldg(a.leaf_c + a.n_leaves + L);
            cz = __ldg(a.leaf_c + 2 * a.n_leaves + L);
            info = leaf_info(L);
            sexp = info >> 7;
            pL = ((info >> 1) & 63) - 1;
            if (pL < 0) errbits |= 4u;  // leaf degree out of range
            if (!(finite_bits(cx) && finite_bits(cy) && finite_bits(cz))) errbits |= 2u;
        }
        // group g (lanes 4g..4g+3) starts a new leaf: bit 4g
        const unsigned gstart =
            __ballot_sync(0xffffffffu, active && (lane & 3) == 0 && ((B >> (ci & 31)) & 1u));
        const int last = 31 - __clz(__ballot_sync(0xffffffffu, active));
        rowleaf[lane] = (long long)L;
        rowinfo[lane] = info;
        wk.set_gstart(gstart);
        wk.set_n_taken(n_taken);
        wk.set_last(last);
        if constexpr (VEC) {
            // this lane's element's current components: the row weights (a
            // non-finite component zeroes the whole segment)
            double wq[3];
            bool fin = true;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                wq[q] = active ? __ldg(a.wvec + (int64_t)q * a.n_elem + e) : 0.0;
                fin = fin && finite_bits(wq[q]);
            }
            if (!fin) errbits |= 2u;
#pragma unroll
            for (int q = 0; q < 3; ++q) rowwt[q * 32 + lane] = fin ? (T)wq[q] : T(0);
        }
        __syncwarp();

        Frame<T, NL> F;
        load_frame<T, KIND, DENS, VEC>(a.vx, a.vy, a.vz, a.idx, a.sigma, a.n_elem, a.n_vert, e, active, cx, cy, cz,
                                       sexp, errbits, pL, F);
        if (errbits) atomicOr(a.err, errbits);
        run_chain<T, P, KIND, DENS, VEC ? 1 : OUTS, true, NS, CH>(F, pw, tile, lane, [&](int c0, int ncols) {
            const RangeCtx rc = range_ctx();
            if constexpr (VEC)
                reduce_chunk_vec<T>(a, rc, tile, accb, rowwt, rowleaf, rowinfo, wk.open_leaf(), wk.open_info(),
                                    wk.gstart(), c0, ncols);
            else
                reduce_chunk<T, CH>(a, rc, tile, accb, rowleaf, rowinfo, wk.open_leaf(), wk.open_info(), wk.gstart(),
                                    wk.n_taken(), c0, ncols, want0, want1, per_elem);
        }, srows);
        // the run open at the end of this round (every lane reads the walk
        // state before it is updated)
        {
            const int lst = wk.last();
            const long long ol = rowleaf[lst];
            const int oi = rowinfo[lst];
            const int64_t en = wk.e_cur() + wk.n_taken();
            wk.sync();
            wk.set_open_leaf(ol);
            wk.set_open_info(oi);
            wk.set_e_cur(en);
        }
        __syncwarp();
    }

    // ---- flush the run left open at the end of the range
#pragma unroll 1
    for (int ly = 0; ly < NACC && !per_elem; ++ly) {
        if (VEC ? a.coef[ly] == nullptr : ((ly == 0 && !want0) || (ly == 1 && !want1) || ly == 2)) continue;
#pragma unroll 1
        for (int c = lane; c < np; c += 32)
            flush_value<T>(a, range_ctx(), ly, c, accb[ly * np + c], wk.open_leaf(), wk.open_info());
    }
}

// Combine the slot partials of leaves that span several warp ranges.  One warp
// per range boundary w (1 <= w < n_ranges) and block row (blockIdx.y, blocks
// of 32 columns strided by gridDim.y): the leaf L containing element w*T is
// handled there iff w is the last range L touches.  A lane sums its column's
// FP64 partials of the ranges wf..w as compensated (Neumaier) sums in a fixed
// order, so that the result does not depend on scheduling: one chain for a
// leaf over at most 8 ranges, else partial i into accumulator i mod 4 and the
// four combined in order.  Then it scales the total like a complete run.  The
// four chains and, for few ranges, one block row per 32 columns keep the
// dependent FP64 adds short when a small problem's leaf spans tens of ranges
// (each FP64 add holds the sub-partition's FP64 pipe for about 64 cycles).
static __global__ void q2x_fixup_kernel(const ElemArgs a, int d0, int d1, int d2, int s0, int s1, int s2)
{
    const int lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5) + 1;
    if (w >= a.n_ranges || a.leaf_off == nullptr) return;
    const int64_t e = w * a.T;
    const int64_t L = leaf_search(a.leaf_off, 0, a.n_leaves - 1, e);
    const int64_t o0 = __ldg(a.leaf_off + L), o1 = __ldg(a.leaf_off + L + 1);
    if (o0 < 0 || o1 > a.n_elem || o1 <= o0) return;  // bad offsets (reported elsewhere)
    if (o0 >= e) return;                 // starts in this range: not spanning here
    if ((o1 - 1) / a.T != w) return;     // not the last range of L
    const int np = a.np_max;
    const int64_t wf = o0 / a.T;
    const int slot_first = (o0 == wf * a.T) ? 0 : 1;
    const int s = a.leaf_rho ? scale_exponent(__ldg(a.leaf_rho + L)) : 0;
    int pl = a.p_max;
    if (a.leaf_p) {
        pl = __ldg(a.leaf_p + L);
        if (pl < 0 || pl > a.p_max) pl = -1;
    }
    const double* slots = a.slots;
    for (int c = (int)blockIdx.y * 32 + lane; c < np; c += (int)gridDim.y * 32) {
        const int desc = col_desc(c);
        for (int ly = 0; ly < a.nacc; ++ly) {
            if (a.coef[ly] == nullptr) continue;
            // partial i: range wf + i (slot slot_first for i = 0, else slot 0)
            auto partial = [&](int64_t i) {
                const int64_t row = (i == 0) ? wf * 2 + slot_first : (wf + i) * 2;
                return __ldg(slots + (row * a.nacc + ly) * (int64_t)np + c);
            };
            auto step = [](double& sm, double& cp, double x) {  // Neumaier
                const double t = sm + x;
                if (fabs(sm) >= fabs(x))
                    cp += (sm - t) + x;
                else
                    cp += (x - t) + sm;
                sm = t;
            };
            const int64_t K = w - wf + 1;  // partials of the leaf
            double tot, tc = 0.0;
            if (K <= 8) {
                // a leaf over a few ranges (large problems): one chain
                tot = partial(0);
                for (int64_t i = 1; i < K; ++i) step(tot, tc, partial(i));
            } else {
                double sum[4] = {0.0, 0.0, 0.0, 0.0}, comp[4] = {0.0, 0.0, 0.0, 0.0};
                int64_t i = 0;
                for (; i + 4 <= K; i += 4) {
                    double x[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) x[u] = partial(i + u);
#pragma unroll
                    for (int u = 0; u < 4; ++u) step(sum[u], comp[u], x[u]);
                }
                for (int u = 0; i < K; ++i, ++u) step(sum[u], comp[u], partial(i));
                tot = sum[0];
                tc = comp[0] + comp[1] + comp[2] + comp[3];
                for (int u = 1; u < 4; ++u) step(tot, tc, sum[u]);
            }
            tot += tc;
            const double v = ((desc & 31) <= pl)
                                 ? finish_desc(tot, a.norm, desc, ly == 0 ? d0 : ly == 1 ? d1 : d2,
                                               ly == 0 ? s0 : ly == 1 ? s1 : s2, s)
                                 : 0.0;
            double* dst = a.coef[ly] + L * np + c;
            if (a.accumulate)
                *dst += v;
            else
                *dst = v;
        }
    }
}

// The fix-up launch for a range split (n_ranges > 1): 4 warps per block over
// the boundaries; with few boundaries (a small problem, whose leaves can span
// many ranges) one block row per 32 columns, else one row looping over them
// (each warp's leaf search is then done once).
inline cudaError_t launch_fixup(const ElemArgs& a, cudaStream_t st, int d0, int d1, int d2, int s0, int s1, int s2)
{
    if (a.n_ranges <= 1) return cudaSuccess;
    const unsigned rows = (a.n_ranges <= 257) ? (unsigned)((a.np_max + 31) / 32) : 1u;
    const dim3 grid((unsigned)((a.n_ranges - 1 + 3) / 4), rows);
    q2x_fixup_kernel<<<grid, 128, 0, st>>>(a, d0, d1, d2, s0, s1, s2);
    return cudaGetLastError();
}

}  // namespace q2x

namespace q2x {

// Launch helpers (explicitly instantiated in q2x_inst_*.cu).
//
// The dynamic shared-memory limit of an instantiation is raised once per
// device, to what its largest degree (P) needs, and not on every launch: a
// plan's p_max <= P needs no more (warp_smem_bytes grows with the column count).
constexpr int kMaxDevices = 64;

// dynamic shared memory of one launch: every warp's region
template <typename T, int P, int KIND, int DENS, int OUTS>
size_t elem_launch_smem(int np_max)
{
    return elem_warps_per_cta<T>() * ElemCfg<T, P, KIND, DENS, OUTS>::warp_bytes(np_max);
}

template <typename T, int P, int KIND, int DENS, int OUTS>
cudaError_t elem_smem_attribute()
{
    static int done[kMaxDevices] = {};  // 0 not yet, 1 set (benign race: the set is idempotent)
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < kMaxDevices && done[dev]) return cudaSuccess;
    const size_t smem_max = elem_launch_smem<T, P, KIND, DENS, OUTS>((P + 1) * (P + 1));
    e = cudaFuncSetAttribute(q2x_elem_kernel<T, P, KIND, DENS, OUTS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_max);
    if (e == cudaSuccess && dev >= 0 && dev < kMaxDevices) done[dev] = 1;
    return e;
}

template <typename T, int P, int KIND, int DENS, int OUTS>
cudaError_t launch_elem(const ElemArgs& a, int grid, cudaStream_t st)
{
    cudaError_t e = elem_smem_attribute<T, P, KIND, DENS, OUTS>();
    if (e != cudaSuccess) return e;
    const size_t smem = elem_launch_smem<T, P, KIND, DENS, OUTS>(a.np_max);
    q2x_elem_kernel<T, P, KIND, DENS, OUTS><<<grid, elem_warps_per_cta<T>() * 32, smem, st>>>(a);
    return cudaGetLastError();
}

template <typename T, int P, int KIND, int DENS, int OUTS>
cudaError_t occupancy_elem(int* blocks_per_sm, int np_max)
{
    cudaError_t e = elem_smem_attribute<T, P, KIND, DENS, OUTS>();
    if (e != cudaSuccess) return e;
    const size_t smem = elem_launch_smem<T, P, KIND, DENS, OUTS>(np_max);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, q2x_elem_kernel<T, P, KIND, DENS, OUTS>,
                                                         elem_warps_per_cta<T>() * 32, smem);
}

}  // namespace q2x

#define Q2X_INSTANTIATE(T, P, KIND, DENS, OUTS)                                                  \
    template cudaError_t q2x::launch_elem<T, P, KIND, DENS, OUTS>(const q2x::ElemArgs&, int, cudaStream_t); \
    template cudaError_t q2x::occupancy_elem<T, P, KIND, DENS, OUTS>(int*, int);                    \
    template size_t q2x::elem_launch_smem<T, P, KIND, DENS, OUTS>(int);

#define Q2X_DECLARE(T, P, KIND, DENS, OUTS)                                                      \
    extern template cudaError_t q2x::launch_elem<T, P, KIND, DENS, OUTS>(const q2x::ElemArgs&, int, \
                                                                         cudaStream_t);            \
    extern template cudaError_t q2x::occupancy_elem<T, P, KIND, DENS, OUTS>(int*, int);             \
    extern template size_t q2x::elem_launch_smem<T, P, KIND, DENS, OUTS>(int);

// capacity bins of the kernels
#define Q2X_FOR_BINS(X, T, KIND, DENS, OUTS)                                                     \
    X(T, 4, KIND, DENS, OUTS) X(T, 8, KIND, DENS, OUTS) X(T, 12, KIND, DENS, OUTS)               \
        X(T, 16, KIND, DENS, OUTS) X(T, 20, KIND, DENS, OUTS)
