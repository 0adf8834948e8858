// q2x_kernels.cuh -- Q2X recursion kernels for sm_103a.
//
// One warp owns a contiguous range of T = 32*R elements (elements are sorted
// by leaf).  Each lane runs one element through the paper's recursions in the
// "tilde" basis (Eqs. (rec10)-(rec15)), row by row in the degree n, with the
// row of every level held in registers.  After each chunk of degrees the 32
// lanes stage their coefficients in shared memory and the warp switches to a
// lane-per-column layout to form segmented (per-leaf) sums over its rows.
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
//
// Linear density on triangles (not in the paper; derived by the same
// integration by parts as Lemma 2 with the weight w = s1(1-u-v) + s2 u + s3 v):
//     (n+2) E_n  = A_x3 E_{n-1}  + s2 q_n + s3 j_n      E = int_edge w h
//     (n+3) Iw_n = A_x1 Iw_{n-1} + E_n + s1 i_n        Iw = int_T w g
// so the chain is q, j, E, i, Iw (5 levels), hat weights n!, (n+1)!, (n+2)!,
// (n+2)!, (n+3)!.
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
// shift when the FP64 coefficient is formed.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace q2x {

enum : int { KIND_SEG = 0, KIND_TRI = 1, KIND_TET = 2 };
enum : int { DENS_CONST = 0, DENS_LINEAR = 1 };

constexpr int WARPS_PER_CTA = 4;
constexpr int CHUNK_COLS = 64;  // columns per layer staged per reduction chunk
constexpr int TILE_LD = 33;     // padded leading dimension of the stage tile

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
    double* coef[2];          // output layers (single, double); NULL = skip
    int accumulate;
    int norm;                 // 0 COEFF, 1 MOMENT
    int64_t T;                // elements per warp range, multiple of 32
    int64_t n_ranges;
    void* slots;              // [n_ranges][2 slots][2 layers][np_max] accumulators
    unsigned* err;
};

// ------------------------------------------------------------- small helpers

__host__ __device__ constexpr double inv_fact(int n)
{
    double f = 1.0;
    for (int k = 2; k <= n; ++k) f *= (double)k;
    return 1.0 / f;
}

// chunk of degrees starting at nb for a kernel of capacity P: the longest run
// of degrees whose column count (2n+1 each) fits CHUNK_COLS; a degree with
// more columns than that forms a chunk of its own.
__host__ __device__ constexpr int chunk_end(int nb, int P)
{
    int ne = nb + 1;
    while (ne <= P && (ne + 1) * (ne + 1) - nb * nb <= CHUNK_COLS) ++ne;
    return ne;
}

// exponent s with 2^s >= rho (rho > 0, finite); 0 for rho <= 0 or non-finite
__device__ __forceinline__ int scale_exponent(double rho)
{
    if (!(rho > 0.0) || !(rho < 1e300)) return 0;
    unsigned long long b = (unsigned long long)__double_as_longlong(rho);
    int e = (int)((b >> 52) & 0x7FF);
    unsigned long long mant = b & 0xFFFFFFFFFFFFFull;
    if (e == 0) return -1022;
    int s = e - 1023;
    if (mant != 0) s += 1;
    return max(-120, min(120, s));
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
    unsigned int b = __float_as_uint(v);
    unsigned int e = (b >> 23) & 0xFF;
    if (e == 0) return 0.0;
    unsigned long long sign = (unsigned long long)(b >> 31) << 63;
    long long de = (long long)e - 127 + 1023 + k;
    if (de <= 0) return 0.0;
    if (de >= 2047) de = 2046;
    unsigned long long mant = (unsigned long long)(b & 0x7FFFFF) << 29;
    return __longlong_as_double((long long)(sign | ((unsigned long long)de << 52) | mant));
}

// Split of a double into hi + lo floats with integer operations only: hi keeps
// the leading 24 significand bits (truncated), lo the rest rounded to 24 bits,
// so |x - hi - lo| <= 2^-47 |x|.  |x| < 2^-103 gives lo = 0, |x| < 2^-126 gives
// hi = lo = 0; a non-finite or too large x sets bad.
__device__ __forceinline__ void split_f64(double x, float& hi, float& lo, bool& bad)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    int e = (int)((b >> 52) & 0x7FF);
    unsigned int sign = (unsigned int)(b >> 63) << 31;
    int ex = e - 1023;
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
    unsigned int ml = (unsigned int)(b & 0x1FFFFFFFull);
    if (ex < -103 || ml == 0) {
        lo = 0.f;
        return;
    }
    // ml * 2^(ex - 52) = (ml * 2^-29) * 2^(ex - 23)
    float l = __uint2float_rn(ml) * 1.862645149230957e-09f * pow2f(ex - 23);
    lo = sign ? -l : l;
}

// per-column output constant: sign * 1/(n+d)! * (1/4pi for COEFF)
__device__ __forceinline__ double column_const(int norm, int n, int m_signed, int d)
{
    const int m = m_signed < 0 ? -m_signed : m_signed;
    const bool is_im = m_signed < 0;
    const int r = m & 3;
    double s;
    if (norm == 0) {
        // (-1)^{n+m} i^m conj(a + ib): Re = {a, b, -a, -b}, Im = {-b, a, b, -a}
        s = is_im ? ((r == 1 || r == 2) ? 1.0 : -1.0) : ((r <= 1) ? 1.0 : -1.0);
        if ((n + m) & 1) s = -s;
        s *= 0.079577471545947667884;  // 1/(4 pi)
    } else {
        // i^{-m}(a + ib): Re = {a, b, -a, -b}, Im = {b, -a, -b, a}
        s = is_im ? ((r == 0 || r == 3) ? 1.0 : -1.0) : ((r <= 1) ? 1.0 : -1.0);
    }
    return s * inv_fact(n + d);
}

// final coefficient from an accumulated sum: acc * cst * 2^shift
__device__ __forceinline__ double finish_value(float acc, double cst, int shift)
{
    return f32_scaled_to_f64(acc * (float)cst, shift);
}
__device__ __forceinline__ double finish_value(double acc, double cst, int shift)
{
    return acc * cst * pow2d(shift);
}

// column index -> (n, m)
__device__ __forceinline__ void col_nm(int c, int& n, int& m)
{
    n = (int)sqrtf((float)c);
    while (n * n > c) --n;
    while ((n + 1) * (n + 1) <= c) ++n;
    m = c - n * n - n;
}

// --------------------------------------------------------------- recursion

// One row of the tilde stencil, in place: on entry re/im hold degree n-1
// (entries >= n are zero), on exit degree n:
//   x^m <- -xi x^{m-1} + eta x^{m+1} - z x^m + src^m       (m > 0)
//   x^0 <- 2 Re(eta x^1) - z x^0 + src^0
// with xi = X + iY, eta = X - iY.
template <typename T, int P>
__device__ __forceinline__ void stencil_row(T (&re)[P + 1], T (&im)[P + 1], const int n, const T X,
                                            const T Y, const T z, const T (&sre)[P + 1],
                                            const T (&sim)[P + 1])
{
    T pr = T(0), pi = T(0);
#pragma unroll
    for (int m = 0; m <= P; ++m) {
        if (m <= n) {
            const T cr = re[m], ci = im[m];
            const T br = (m < P) ? re[(m < P) ? m + 1 : P] : T(0);
            const T bi = (m < P) ? im[(m < P) ? m + 1 : P] : T(0);
            T nr, ni;
            if (m == 0) {
                nr = fma(T(2) * X, br, sre[0]);
                nr = fma(T(2) * Y, bi, nr);
                nr = fma(-z, cr, nr);
                ni = T(0);
            } else {
                const T dr = br - pr, di = bi - pi;
                const T sr = br + pr, si = bi + pi;
                nr = fma(X, dr, sre[m]);
                nr = fma(Y, si, nr);
                nr = fma(-z, cr, nr);
                ni = fma(X, di, sim[m]);
                ni = fma(-Y, sr, ni);
                ni = fma(-z, ci, ni);
            }
            re[m] = nr;
            im[m] = ni;
            pr = cr;
            pi = ci;
        }
    }
}

// Stencil of a row WITHOUT updating it (double layer): value m of degree n
// goes to f(m, re, im).
template <typename T, int P, typename F>
__device__ __forceinline__ void stencil_apply(const T (&re)[P + 1], const T (&im)[P + 1],
                                              const int n, const T X, const T Y, const T z, F&& f)
{
#pragma unroll
    for (int m = 0; m <= P; ++m) {
        if (m <= n) {
            const T cr = re[m], ci = im[m];
            const T br = (m < P) ? re[(m < P) ? m + 1 : P] : T(0);
            const T bi = (m < P) ? im[(m < P) ? m + 1 : P] : T(0);
            const T ar = (m >= 1) ? re[(m >= 1) ? m - 1 : 0] : T(0);
            const T ai = (m >= 1) ? im[(m >= 1) ? m - 1 : 0] : T(0);
            T nr, ni;
            if (m == 0) {
                nr = T(2) * X * br;
                nr = fma(T(2) * Y, bi, nr);
                nr = fma(-z, cr, nr);
                ni = T(0);
            } else {
                const T dr = br - ar, di = bi - ai;
                const T sr = br + ar, si = bi + ai;
                nr = X * dr;
                nr = fma(Y, si, nr);
                nr = fma(-z, cr, nr);
                ni = X * di;
                ni = fma(-Y, sr, ni);
                ni = fma(-z, ci, ni);
            }
            f(m, nr, ni);
        }
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
// rows of the same leaf.  info = (shift exponent << 1) | complete, where
// complete means the leaf lies wholly in [e_lo, e_hi).
struct RangeCtx {
    int64_t w, e_lo, e_hi, L_first;
    int dim;         // 1, 2, 3: power of the scale in the Jacobian
    int d_out[2];    // hat depth of each layer's output level
    int shift_n0[2]; // shift = s * (n + shift_n0[layer])
};

template <typename T>
__device__ __forceinline__ void flush_value(const ElemArgs& a, const RangeCtx& rc, int ly, int c,
                                            T acc, long long L, int info)
{
    if (info & 1) {
        int n, m;
        col_nm(c, n, m);
        const double cst = column_const(a.norm, n, m, rc.d_out[ly]);
        const int shift = (info >> 1) * (n + rc.shift_n0[ly]);
        const double v = finish_value(acc, cst, shift);
        double* dst = a.coef[ly] + (int64_t)L * a.np_max + c;
        if (a.accumulate)
            *dst += v;
        else
            *dst = v;
    } else {
        const int slot = (L == rc.L_first) ? 0 : 1;
        T* sl = reinterpret_cast<T*>(a.slots) + (((rc.w * 2 + slot) * 2 + ly) * (int64_t)a.np_max + c);
        *sl = acc;
    }
}

// Segmented column sums of one staged chunk: columns [c0, c0 + ncols) of each
// wanted layer, rows 0..nrows-1.  Lane j owns columns j, j+32, ...; its running
// sum (the open run) lives in accb between chunks and rounds.
template <typename T>
__device__ __noinline__ void reduce_chunk(const ElemArgs& a, const RangeCtx& rc, const T* tile,
                                          T* accb, const long long* rowleaf, const int* rowinfo,
                                          long long open_leaf, int open_info, int nrows, int c0,
                                          int ncols, bool want0, bool want1)
{
    const int lane = threadIdx.x & 31;
#pragma unroll 1
    for (int ly = 0; ly < 2; ++ly) {
        if ((ly == 0 && !want0) || (ly == 1 && !want1)) continue;
        const T* tl = tile + ly * CHUNK_COLS * TILE_LD;
        for (int j = lane; j < ncols; j += 32) {
            const int c = c0 + j;
            T acc = accb[ly * a.np_max + c];
            long long L = open_leaf;
            int info = open_info;
            for (int r = 0; r < nrows; ++r) {
                const long long Lr = rowleaf[r];
                if (Lr != L) {
                    flush_value<T>(a, rc, ly, c, acc, L, info);
                    acc = T(0);
                    L = Lr;
                    info = rowinfo[r];
                }
                acc += tl[j * TILE_LD + r];
            }
            accb[ly * a.np_max + c] = acc;
        }
    }
}

// ------------------------------------------------------------------ kernel

// Shared memory per warp: stage tile [2 layers][CHUNK_COLS][TILE_LD] of T,
// open-run sums [2 layers][np_max] of T, row leaves [32], row infos [32].
template <typename T>
__host__ __device__ constexpr size_t warp_smem_bytes(int np_max)
{
    return sizeof(T) * (size_t)(2 * CHUNK_COLS * TILE_LD + 2 * np_max) + sizeof(long long) * 32 +
           sizeof(int) * 32;
}

template <typename T, int P, int KIND, int DENS>
__global__ void __launch_bounds__(WARPS_PER_CTA * 32, (sizeof(T) == 8) ? 1 : 2)
    q2x_elem_kernel(const ElemArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int64_t w = (int64_t)blockIdx.x * WARPS_PER_CTA + wib;
    if (w >= a.n_ranges) return;

    constexpr bool FP32 = sizeof(T) == 4;
    constexpr int NV = KIND + 2;
    // hat depth of the single-layer output level; the double layer is formed
    // from row n-1 of that level, one factorial lower
    constexpr int D_OUT =
        (KIND == KIND_SEG) ? 1 : (KIND == KIND_TET) ? 3 : (DENS == DENS_LINEAR ? 3 : 2);

    unsigned char* wsm = smem_raw + (size_t)wib * warp_smem_bytes<T>(a.np_max);
    T* tile = reinterpret_cast<T*>(wsm);
    T* accb = tile + 2 * CHUNK_COLS * TILE_LD;
    long long* rowleaf = reinterpret_cast<long long*>(accb + 2 * a.np_max);
    int* rowinfo = reinterpret_cast<int*>(rowleaf + 32);

    const bool want0 = a.coef[0] != nullptr;
    const bool want1 = (KIND == KIND_TRI) && a.coef[1] != nullptr;
    const bool per_elem = a.leaf_off == nullptr;
    const int np = a.np_max;
    const int pw = a.p_max;

    RangeCtx rc;
    rc.w = w;
    rc.e_lo = w * a.T;
    rc.e_hi = min(rc.e_lo + a.T, a.n_elem);
    rc.dim = KIND + 1;
    rc.d_out[0] = D_OUT;
    rc.d_out[1] = D_OUT - 1;
    rc.shift_n0[0] = KIND + 1;
    rc.shift_n0[1] = 1;

    int64_t L_last;
    if (per_elem) {
        rc.L_first = rc.e_lo;
        L_last = rc.e_hi - 1;
    } else {
        rc.L_first = leaf_search(a.leaf_off, 0, a.n_leaves - 1, rc.e_lo);
        L_last = leaf_search(a.leaf_off, rc.L_first, a.n_leaves - 1, rc.e_hi - 1);
    }

    for (int k = lane; k < 2 * np; k += 32) accb[k] = T(0);

    // zero the coefficients of empty leaves [La, Lb) (overwrite mode)
    auto zero_leaves = [&](int64_t La, int64_t Lb) {
        if (a.accumulate) return;
        for (int64_t L = La; L < Lb; ++L)
            for (int c = lane; c < np; c += 32) {
                if (want0) a.coef[0][L * np + c] = 0.0;
                if (want1) a.coef[1][L * np + c] = 0.0;
            }
    };
    if (!per_elem) {
        zero_leaves(leaf_lower(a.leaf_off, 0, a.n_leaves, rc.e_lo), rc.L_first);
        if (rc.e_hi == a.n_elem) zero_leaves(L_last + 1, a.n_leaves);
    }

    auto leaf_info = [&](int64_t L) -> int {
        bool complete = true;
        if (!per_elem) complete = __ldg(a.leaf_off + L) >= rc.e_lo && __ldg(a.leaf_off + L + 1) <= rc.e_hi;
        const int s = a.leaf_rho ? scale_exponent(__ldg(a.leaf_rho + L)) : 0;
        return (s << 1) | (complete ? 1 : 0);
    };
    long long open_leaf = rc.L_first;
    int open_info = leaf_info(rc.L_first);

    for (int64_t e0 = rc.e_lo; e0 < rc.e_hi; e0 += 32) {
        const int64_t e = e0 + lane;
        const bool active = e < rc.e_hi;
        const int nrows = (int)min((int64_t)32, rc.e_hi - e0);

        // ---- this lane's leaf, centre, scale, degree
        int64_t L = open_leaf;
        if (active) L = per_elem ? e : leaf_search(a.leaf_off, open_leaf, L_last, e);
        unsigned errbits = 0;
        int pL = pw, sexp = 0;
        double cx = 0.0, cy = 0.0, cz = 0.0;
        int info = 0;
        if (active) {
            cx = __ldg(a.leaf_c + L);
            cy = __ldg(a.leaf_c + a.n_leaves + L);
            cz = __ldg(a.leaf_c + 2 * a.n_leaves + L);
            if (a.leaf_p) {
                pL = __ldg(a.leaf_p + L);
                if (pL < 0 || pL > pw) {
                    errbits |= 4u;
                    pL = -1;
                }
            }
            info = leaf_info(L);
            sexp = info >> 1;
            if (!(isfinite(cx) && isfinite(cy) && isfinite(cz))) errbits |= 2u;
        }
        __syncwarp();
        rowleaf[lane] = (long long)L;
        rowinfo[lane] = info;
        __syncwarp();
        // empty leaves between consecutive rows
        if (!per_elem && !a.accumulate) {
            long long prev = open_leaf;
            for (int r = 0; r < nrows; ++r) {
                const long long Lr = rowleaf[r];
                if (Lr > prev + 1) zero_leaves(prev + 1, Lr);
                prev = Lr;
            }
        }

        // ---- gather vertices into the scaled local frame
        T vxl[NV], vyl[NV], vzl[NV];
        T s1 = T(0), s2 = T(0), s3 = T(0);
        bool bad = !active;
        {
            int64_t vid[NV];
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                int64_t v = active ? (int64_t)__ldg(a.idx + (int64_t)k * a.n_elem + e) : 0;
                if (v < 0 || v >= a.n_vert) {
                    if (active) errbits |= 1u;
                    bad = true;
                    v = 0;
                }
                vid[k] = v;
            }
            double dens[3] = {0.0, 0.0, 0.0};
            if (active) {
                if (DENS == DENS_LINEAR) {
#pragma unroll
                    for (int k = 0; k < 3; ++k) dens[k] = __ldg(a.sigma + vid[k]);
                } else {
                    dens[0] = __ldg(a.sigma + e);
                }
            }
            if (!(isfinite(dens[0]) && isfinite(dens[1]) && isfinite(dens[2]))) {
                errbits |= 2u;
                bad = true;
            }
            s1 = (T)dens[0];
            s2 = (T)dens[1];
            s3 = (T)dens[2];
            if constexpr (FP32) {
                bool nf = false;
                float chx, clx, chy, cly, chz, clz;
                split_f64(cx, chx, clx, nf);
                split_f64(cy, chy, cly, nf);
                split_f64(cz, chz, clz, nf);
                const float inv = pow2f(-sexp);
#pragma unroll
                for (int k = 0; k < NV; ++k) {
                    float hx, lx, hy, ly, hz, lz;
                    split_f64(active ? __ldg(a.vx + vid[k]) : 0.0, hx, lx, nf);
                    split_f64(active ? __ldg(a.vy + vid[k]) : 0.0, hy, ly, nf);
                    split_f64(active ? __ldg(a.vz + vid[k]) : 0.0, hz, lz, nf);
                    vxl[k] = ((hx - chx) + (lx - clx)) * inv;
                    vyl[k] = ((hy - chy) + (ly - cly)) * inv;
                    vzl[k] = ((hz - chz) + (lz - clz)) * inv;
                }
                if (nf && active) {
                    errbits |= 2u;
                    bad = true;
                }
            } else {
                const double inv = pow2d(-sexp);
#pragma unroll
                for (int k = 0; k < NV; ++k) {
                    const double x = active ? __ldg(a.vx + vid[k]) : 0.0;
                    const double y = active ? __ldg(a.vy + vid[k]) : 0.0;
                    const double zz = active ? __ldg(a.vz + vid[k]) : 0.0;
                    if (!(isfinite(x) && isfinite(y) && isfinite(zz))) {
                        if (active) errbits |= 2u;
                        bad = true;
                    }
                    vxl[k] = (x - cx) * inv;
                    vyl[k] = (y - cy) * inv;
                    vzl[k] = (zz - cz) * inv;
                }
            }
        }
        if (errbits) atomicOr(a.err, errbits);
        if (bad) pL = -1;

        // ---- Jacobian in the scaled frame, unit normal, seed
        T J, nx = T(0), ny = T(0), nz = T(0);
        {
            const T ux = vxl[1] - vxl[0], uy = vyl[1] - vyl[0], uz = vzl[1] - vzl[0];
            if constexpr (KIND == KIND_SEG) {
                J = sqrt(ux * ux + uy * uy + uz * uz);
            } else {
                const T wx = vxl[2] - vxl[0], wy = vyl[2] - vyl[0], wz = vzl[2] - vzl[0];
                const T cxp = uy * wz - uz * wy, cyp = uz * wx - ux * wz, czp = ux * wy - uy * wx;
                if constexpr (KIND == KIND_TRI) {
                    J = sqrt(cxp * cxp + cyp * cyp + czp * czp);
                    const T inv = (J > T(0)) ? T(1) / J : T(0);
                    nx = cxp * inv;
                    ny = cyp * inv;
                    nz = czp * inv;
                } else {
                    const T tx = vxl[NV - 1] - vxl[0], ty = vyl[NV - 1] - vyl[0],
                            tz = vzl[NV - 1] - vzl[0];
                    J = fabs(cxp * tx + cyp * ty + czp * tz);
                }
            }
        }
        T seed = (DENS == DENS_LINEAR) ? J : J * s1;
        if (pL < 0) seed = T(0);

        // chain vertices (half coordinates for xi/eta)
        const T X1 = T(0.5) * vxl[0], Y1 = T(0.5) * vyl[0], Z1 = vzl[0];
        const T X2 = T(0.5) * vxl[1], Y2 = T(0.5) * vyl[1], Z2 = vzl[1];
        const T X3 = T(0.5) * vxl[NV >= 3 ? 2 : 0], Y3 = T(0.5) * vyl[NV >= 3 ? 2 : 0],
                Z3 = vzl[NV >= 3 ? 2 : 0];
        const T X4 = T(0.5) * vxl[NV - 1], Y4 = T(0.5) * vyl[NV - 1], Z4 = vzl[NV - 1];
        const T XN = T(0.5) * nx, YN = T(0.5) * ny, ZN = nz;

        // ---- level rows; degree n-1 on entry of step n
        // q: q^ (x2) | l1: p^ (segment, x1) or j^ (x3)
        // l2: i^ (tri const, x1) | E^ (tri linear, x3) | b^ (tet, x4)
        // l3: i^ (tri linear, x1) | a^ (tet, x1) | l4: Iw^ (tri linear, x1)
        T q_r[P + 1], q_i[P + 1], l1_r[P + 1], l1_i[P + 1], l2_r[P + 1], l2_i[P + 1];
        T l3_r[P + 1], l3_i[P + 1], l4_r[P + 1], l4_i[P + 1], s_r[P + 1], s_i[P + 1];
#pragma unroll
        for (int m = 0; m <= P; ++m) {
            q_r[m] = q_i[m] = l1_r[m] = l1_i[m] = l2_r[m] = l2_i[m] = T(0);
            l3_r[m] = l3_i[m] = l4_r[m] = l4_i[m] = s_r[m] = s_i[m] = T(0);
        }

        int nb = 0;  // first degree of the chunk being staged
#pragma unroll
        for (int n = 0; n <= P; ++n) {
            if (n > pw) break;
            const bool keep = (n <= pL);
            const int cb = n * n - nb * nb + n;  // tile column of (n, m = 0)
            // -- double layer from the row of degree n-1 (before advancing it)
            if constexpr (KIND == KIND_TRI) {
                if (want1) {
                    T* t1 = tile + CHUNK_COLS * TILE_LD;
                    auto put = [&](int m, T vr, T vi) {
                        if (!keep) vr = vi = T(0);
                        t1[(cb + m) * TILE_LD + lane] = (m & 1) ? vi : vr;
                        if (m > 0) t1[(cb - m) * TILE_LD + lane] = (m & 1) ? vr : vi;
                    };
                    if constexpr (DENS == DENS_LINEAR)
                        stencil_apply<T, P>(l4_r, l4_i, n, XN, YN, ZN, put);
                    else
                        stencil_apply<T, P>(l2_r, l2_i, n, XN, YN, ZN, put);
                }
            }
            // -- advance the chain to degree n
            s_r[0] = (n == 0) ? seed : T(0);
            stencil_row<T, P>(q_r, q_i, n, X2, Y2, Z2, s_r, s_i);  // q^_n = A_x2 q^_{n-1}
            s_r[0] = T(0);
            if constexpr (KIND == KIND_SEG) {
                stencil_row<T, P>(l1_r, l1_i, n, X1, Y1, Z1, q_r, q_i);  // p^
            } else {
                stencil_row<T, P>(l1_r, l1_i, n, X3, Y3, Z3, q_r, q_i);  // j^
                if constexpr (KIND == KIND_TRI && DENS == DENS_CONST) {
                    stencil_row<T, P>(l2_r, l2_i, n, X1, Y1, Z1, l1_r, l1_i);  // i^
                } else if constexpr (KIND == KIND_TRI) {
                    // E^_n = A_x3 E^_{n-1} + (n+1) s2 q^_n + s3 j^_n
                    const T c2 = T(n + 1) * s2;
#pragma unroll
                    for (int m = 0; m <= P; ++m)
                        if (m <= n) {
                            s_r[m] = fma(c2, q_r[m], s3 * l1_r[m]);
                            s_i[m] = fma(c2, q_i[m], s3 * l1_i[m]);
                        }
                    stencil_row<T, P>(l2_r, l2_i, n, X3, Y3, Z3, s_r, s_i);
                    stencil_row<T, P>(l3_r, l3_i, n, X1, Y1, Z1, l1_r, l1_i);  // i^
                    // Iw^_n = A_x1 Iw^_{n-1} + E^_n + s1 i^_n
#pragma unroll
                    for (int m = 0; m <= P; ++m)
                        if (m <= n) {
                            s_r[m] = fma(s1, l3_r[m], l2_r[m]);
                            s_i[m] = fma(s1, l3_i[m], l2_i[m]);
                        }
                    stencil_row<T, P>(l4_r, l4_i, n, X1, Y1, Z1, s_r, s_i);
#pragma unroll
                    for (int m = 0; m <= P; ++m) s_r[m] = s_i[m] = T(0);
                } else {
                    stencil_row<T, P>(l2_r, l2_i, n, X4, Y4, Z4, l1_r, l1_i);  // b^
                    stencil_row<T, P>(l3_r, l3_i, n, X1, Y1, Z1, l2_r, l2_i);  // a^
                }
            }
            // -- stage the single-layer row of degree n
            if (want0) {
#pragma unroll
                for (int m = 0; m <= P; ++m) {
                    if (m <= n) {
                        T vr, vi;
                        if constexpr (KIND == KIND_SEG) {
                            vr = l1_r[m];
                            vi = l1_i[m];
                        } else if constexpr (KIND == KIND_TRI && DENS == DENS_CONST) {
                            vr = l2_r[m];
                            vi = l2_i[m];
                        } else if constexpr (KIND == KIND_TRI) {
                            vr = l4_r[m];
                            vi = l4_i[m];
                        } else {
                            vr = l3_r[m];
                            vi = l3_i[m];
                        }
                        if (!keep) vr = vi = T(0);
                        tile[(cb + m) * TILE_LD + lane] = (m & 1) ? vi : vr;
                        if (m > 0) tile[(cb - m) * TILE_LD + lane] = (m & 1) ? vr : vi;
                    }
                }
            }
            // -- reduce the chunk when it is complete (chunk ends are compile-time;
            //    a run-time p_max below P ends the last chunk early)
            const int ne = chunk_end(nb, P);
            if (n + 1 == ne) {
                __syncwarp();
                reduce_chunk<T>(a, rc, tile, accb, rowleaf, rowinfo, open_leaf, open_info, nrows,
                                nb * nb, (n + 1) * (n + 1) - nb * nb, want0, want1);
                __syncwarp();
                nb = n + 1;
            } else if (n == pw) {
                __syncwarp();
                reduce_chunk<T>(a, rc, tile, accb, rowleaf, rowinfo, open_leaf, open_info, nrows,
                                nb * nb, (n + 1) * (n + 1) - nb * nb, want0, want1);
                __syncwarp();
            }
        }
        // the run open at the end of this round
        open_leaf = rowleaf[nrows - 1];
        open_info = rowinfo[nrows - 1];
    }

    // ---- flush the run left open at the end of the range
    __syncwarp();
    for (int ly = 0; ly < 2; ++ly) {
        if ((ly == 0 && !want0) || (ly == 1 && !want1)) continue;
        for (int c = lane; c < np; c += 32)
            flush_value<T>(a, rc, ly, c, accb[ly * np + c], open_leaf, open_info);
    }
}

// Combine the slot partials of leaves that span several warp ranges.  One warp
// per range boundary w (1 <= w < n_ranges): the leaf L containing element w*T,
// handled here iff w is the last range L touches.  Partials are summed in range
// order (compensated in FP32), then scaled like a complete run.
template <typename T>
__global__ void q2x_fixup_kernel(const ElemArgs a, int dim, int d0, int d1)
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
    const int64_t wf = o0 / a.T;
    const int slot_first = (o0 == wf * a.T) ? 0 : 1;
    const int s = a.leaf_rho ? scale_exponent(__ldg(a.leaf_rho + L)) : 0;
    const int np = a.np_max;
    const T* slots = reinterpret_cast<const T*>(a.slots);
    for (int ly = 0; ly < 2; ++ly) {
        if (a.coef[ly] == nullptr) continue;
        for (int c = lane; c < np; c += 32) {
            T sum = slots[((wf * 2 + slot_first) * 2 + ly) * (int64_t)np + c];
            T comp = T(0);
            for (int64_t ww = wf + 1; ww <= w; ++ww) {
                const T x = slots[((ww * 2 + 0) * 2 + ly) * (int64_t)np + c];
                // Kahan-Babuska (Neumaier) step
                const T t = sum + x;
                if (fabs(sum) >= fabs(x))
                    comp += (sum - t) + x;
                else
                    comp += (x - t) + sum;
                sum = t;
            }
            sum += comp;
            int n, m;
            col_nm(c, n, m);
            const double cst = column_const(a.norm, n, m, ly == 0 ? d0 : d1);
            const int shift = s * (n + (ly == 0 ? dim : 1));
            const double v = finish_value(sum, cst, shift);
            double* dst = a.coef[ly] + L * np + c;
            if (a.accumulate)
                *dst += v;
            else
                *dst = v;
        }
    }
}

}  // namespace q2x

namespace q2x {

// Launch helpers (explicitly instantiated in q2x_inst_*.cu).
template <typename T, int P, int KIND, int DENS>
cudaError_t launch_elem(const ElemArgs& a, int grid, size_t smem, cudaStream_t st)
{
    auto k = q2x_elem_kernel<T, P, KIND, DENS>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, WARPS_PER_CTA * 32, smem, st>>>(a);
    return cudaGetLastError();
}

template <typename T, int P, int KIND, int DENS>
cudaError_t occupancy_elem(int* blocks_per_sm, size_t smem)
{
    auto k = q2x_elem_kernel<T, P, KIND, DENS>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, WARPS_PER_CTA * 32, smem);
}

}  // namespace q2x

#define Q2X_INSTANTIATE(T, P, KIND, DENS)                                                        \
    template cudaError_t q2x::launch_elem<T, P, KIND, DENS>(const q2x::ElemArgs&, int, size_t,  \
                                                            cudaStream_t);                       \
    template cudaError_t q2x::occupancy_elem<T, P, KIND, DENS>(int*, size_t);

#define Q2X_DECLARE(T, P, KIND, DENS)                                                            \
    extern template cudaError_t q2x::launch_elem<T, P, KIND, DENS>(const q2x::ElemArgs&, int,   \
                                                                   size_t, cudaStream_t);        \
    extern template cudaError_t q2x::occupancy_elem<T, P, KIND, DENS>(int*, size_t);

// capacity bins of the unrolled kernels
#define Q2X_FOR_BINS(X, T, KIND, DENS) X(T, 4, KIND, DENS) X(T, 8, KIND, DENS) X(T, 12, KIND, DENS) X(T, 16, KIND, DENS) X(T, 20, KIND, DENS)
