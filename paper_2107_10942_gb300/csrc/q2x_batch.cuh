// q2x_batch.cuh -- ragged mixed-kind Q2X batch: one persistent kernel over a
// tile list, then a deterministic per-leaf combine.
//
// A tile is a run of at most T elements of ONE kind inside ONE leaf, so every
// round of 32 elements a warp processes shares the leaf centre, scale and
// degree p_leaf: the degree loop runs exactly to p_leaf (no work above it),
// every staged chunk is summed by the pairwise fast path, and each tile ends
// with one finished FP64 row of partial coefficients.  Warps of a persistent
// grid pull tiles through an atomic counter in the host-chosen order (grouped
// by kind and degree bin, most expensive first).  The combine kernel adds the
// partial rows of each leaf in slot order (slots are numbered leaf by leaf),
// so the result does not depend on which warp ran which tile.
#pragma once

#include "q2x_kernels.cuh"

namespace q2x {

struct BatchKind {
    int64_t n_elem, n_vert;
    const double* vx;
    const double* vy;
    const double* vz;
    const int32_t* idx;
    const double* sigma;
};

// combo: 0 segments, 1 triangles constant density, 2 triangles linear
// density, 3 tetrahedra; bin: index of the capacity P in {4, 8, 12, 16, 20}
struct BatchTile {
    int32_t combo;
    int32_t bin;
    int32_t leaf;
    int32_t pad;
    int64_t slot;
    int64_t e_lo, e_hi;
};

struct BatchArgs {
    BatchKind kind[3];  // segments, triangles, tetrahedra
    int64_t n_leaves;
    const double* leaf_c;
    const double* leaf_rho;
    const int32_t* leaf_p;
    int p_max, np_max, norm;
    const BatchTile* tiles;
    int64_t n_tiles;
    unsigned long long* counter;
    double* partial;  // [n_slots][np_max]
    unsigned* err;
};

constexpr int BATCH_WARPS = 4;

// stage tile [2 CHUNK][LD] of T (single-layer passes stage twice CHUNK
// columns per reduction), then the tile's column sums [np_max] (LeafSum)
template <typename T>
__host__ __device__ constexpr size_t batch_warp_smem_bytes(int np_max)
{
    return (sizeof(T) * (size_t)(2 * KCfg<T>::CHUNK * KCfg<T>::LD) + sizeof(LeafSum<T>) * (size_t)np_max + 127) /
           128 * 128;
}

template <typename T, int P, int KIND, int DENS>
__device__ __forceinline__ void batch_tile(const BatchArgs& b, const BatchTile& t, T* tile, LeafSum<T>* accb,
                                           int lane)
{
    using C = Chain<KIND, DENS>;
    constexpr int LD = KCfg<T>::LD;
    const BatchKind& K = b.kind[KIND];
    const int64_t L = t.leaf;
    const int np = b.np_max;
    int pL = b.leaf_p ? __ldg(b.leaf_p + L) : b.p_max;
    unsigned errbits = 0;
    if (pL < 0 || pL > b.p_max || pL > P) {
        errbits |= 4u;  // leaf degree out of range
        pL = -1;
    }
    const double cx = __ldg(b.leaf_c + L), cy = __ldg(b.leaf_c + b.n_leaves + L),
                 cz = __ldg(b.leaf_c + 2 * b.n_leaves + L);
    if (!(finite_bits(cx) && finite_bits(cy) && finite_bits(cz))) errbits |= 2u;
    const int sexp = b.leaf_rho ? scale_exponent(__ldg(b.leaf_rho + L)) : 0;
    for (int c = lane; c < np; c += 32) accb[c].zero();
    __syncwarp();
    if (pL >= 0) {
#pragma unroll 1
        for (int64_t e0 = t.e_lo; e0 < t.e_hi; e0 += 32) {
            const int64_t e = e0 + lane;
            const bool active = e < t.e_hi;
            int pl = pL;
            Frame<T, C::NL> F;
            load_frame<T, KIND, DENS>(K.vx, K.vy, K.vz, K.idx, K.sigma, K.n_elem, K.n_vert, e, active, cx, cy,
                                      cz, sexp, errbits, pl, F);
            run_chain<T, P, KIND, DENS, 1, true>(F, pL, tile, lane, [&](int c0, int ncols) {
                // each round's 32 rows summed pairwise, the rounds accumulated
                // in a LeafSum (compensated in FP32)
                for (int j = lane; j < ncols; j += 32) accb[c0 + j].add(sum_rows32(tile + j * LD));
            });
        }
    }
    if (errbits) atomicOr(b.err, errbits);
    __syncwarp();
    double* out = b.partial + t.slot * (int64_t)np;
    const int npl = (pL + 1) * (pL + 1);
#pragma unroll 1
    for (int c = lane; c < np; c += 32) {
        double v = 0.0;
        if (c < npl) v = finish_desc(accb[c].rounded(), b.norm, col_desc(c), C::D_OUT, KIND + 1, sexp);
        out[c] = v;
    }
    __syncwarp();
}

#define Q2X_BATCH_CASE(T, COMBO, KIND, DENS, BIN, P)                                              \
    case (COMBO)*5 + (BIN):                                                                       \
        batch_tile<T, P, KIND, DENS>(b, t, tile, accb, lane);                                     \
        break;
#define Q2X_BATCH_COMBO(T, COMBO, KIND, DENS)                                                     \
    Q2X_BATCH_CASE(T, COMBO, KIND, DENS, 0, 4)                                                    \
    Q2X_BATCH_CASE(T, COMBO, KIND, DENS, 1, 8)                                                    \
    Q2X_BATCH_CASE(T, COMBO, KIND, DENS, 2, 12)                                                   \
    Q2X_BATCH_CASE(T, COMBO, KIND, DENS, 3, 16)                                                   \
    Q2X_BATCH_CASE(T, COMBO, KIND, DENS, 4, 20)

template <typename T>
__global__ void __launch_bounds__(BATCH_WARPS * 32, 2) q2x_batch_kernel(const BatchArgs b)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    unsigned char* wsm = smem_raw + (size_t)wib * batch_warp_smem_bytes<T>(b.np_max);
    T* tile = reinterpret_cast<T*>(wsm);
    LeafSum<T>* accb = reinterpret_cast<LeafSum<T>*>(tile + 2 * KCfg<T>::CHUNK * KCfg<T>::LD);  // 2 CHUNK LD sizeof(T) % 8 == 0
#pragma unroll 1
    while (true) {
        unsigned long long ti = 0;
        if (lane == 0) ti = atomicAdd(b.counter, 1ull);
        ti = __shfl_sync(0xffffffffu, ti, 0);
        if (ti >= (unsigned long long)b.n_tiles) break;
        const BatchTile t = b.tiles[ti];
        switch (t.combo * 5 + t.bin) {
            Q2X_BATCH_COMBO(T, 0, KIND_SEG, DENS_CONST)
            Q2X_BATCH_COMBO(T, 1, KIND_TRI, DENS_CONST)
            Q2X_BATCH_COMBO(T, 2, KIND_TRI, DENS_LINEAR)
            Q2X_BATCH_COMBO(T, 3, KIND_TET, DENS_CONST)
            default:
                break;
        }
    }
}

// coef[L] (+)= sum of the partial rows slot_off[L] .. slot_off[L+1]-1, in order
__global__ void q2x_batch_combine(const double* __restrict__ partial, const int64_t* __restrict__ slot_off,
                                  int np, int64_t n_leaves, double* coef, int accumulate);

}  // namespace q2x
