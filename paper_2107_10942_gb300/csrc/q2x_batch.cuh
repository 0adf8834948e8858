// q2x_batch.cuh -- ragged mixed-kind Q2X batch: persistent kernels over a
// tile list, then a deterministic per-leaf combine.
//
// A tile is a run of at most T elements of ONE kind inside ONE leaf, so every
// round of 32 elements a warp processes shares the leaf centre, scale and
// degree p_leaf: the degree loop runs exactly to p_leaf (no work above it),
// every staged chunk is summed by the pairwise fast path, and each tile ends
// with one finished FP64 row of partial coefficients.  The host orders the
// tiles by degree bin (highest first), kind and cost, and cuts the list into
// groups of one (kind, bin); each group has its own persistent kernel,
// compiled for its chain alone (registers, and so resident warps, follow that
// chain, not the most expensive one), whose warps pull the group's tiles
// through the group's atomic counter.  The groups' kernels run on parallel
// graph branches, so one group's tail overlaps the next.  The combine kernel
// adds the partial rows of each leaf in slot order (slots are numbered leaf by
// leaf), so the result does not depend on which warp ran which tile.
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
// density, 3 tetrahedra; bin: index of the capacity P in {4, 8, 12, 16, 20};
// flags bit 0: the tile is its leaf's only one, and its finished row goes
// straight to coef[leaf] (else to partial row slot, for the combine)
struct BatchTile {
    int32_t combo;
    int32_t bin;
    int32_t leaf;
    int32_t flags;
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
    unsigned long long* counter;  // one per group
    double* partial;  // [n_slots][np_max]
    unsigned* err;
    double* coef;                 // rows of single-tile leaves (flags bit 0)
    int accumulate;               // those rows are added to coef
    const int64_t* n_tiles_dev;   // tile count on the device (a kernel launched with t1 < 0)
};

constexpr int BATCH_WARPS = 4;

// stage tile [2 CH][LD] of T (single-layer passes stage 2 CH columns per
// reduction), then the tile's column sums [np] (LeafSum)
template <typename T>
__host__ __device__ constexpr size_t batch_warp_smem_bytes(int np, int ch = KCfg<T>::CHUNK)
{
    return (sizeof(T) * (size_t)(2 * ch * KCfg<T>::LD) + sizeof(LeafSum<T>) * (size_t)np + 127) / 128 * 128;
}

// One group's kernel: the chain's capacity P, its stage-tile width and the
// CTAs per SM it is compiled for.  FP32 uses the element kernel's register
// targets (CTAs of four warps here: 4, 3 or 2 per SM) and 40-column chunks, so
// that 16 warps of the small chains fit in shared memory.
template <typename T, int P, int KIND, int DENS>
struct BatchCfg {
    static constexpr int CH = sizeof(T) == 4 ? 40 : KCfg<T>::CHUNK;
    static constexpr int NP = (P + 1) * (P + 1);
    static constexpr int MIN_CTAS = sizeof(T) == 4 ? min_ctas<T, P, KIND, DENS, 1>() / 4 : 2;
    static constexpr size_t WARP_BYTES = batch_warp_smem_bytes<T>(NP, CH);
};

template <typename T, int P, int KIND, int DENS, int CH>
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
    constexpr int NPC = (P + 1) * (P + 1);  // accb holds the columns up to the capacity
    for (int c = lane; c < NPC; c += 32) accb[c].zero();
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
            run_chain<T, P, KIND, DENS, 1, true, 0, CH>(F, pL, tile, lane, [&](int c0, int ncols) {
                // each round's 32 rows summed pairwise, the rounds accumulated
                // in a LeafSum (compensated in FP32)
                for (int j = lane; j < ncols; j += 32) accb[c0 + j].add(sum_rows32(tile + j * LD));
            });
        }
    }
    if (errbits) atomicOr(b.err, errbits);
    __syncwarp();
    const bool direct = (t.flags & 1) != 0;
    double* out = direct ? b.coef + L * (int64_t)np : b.partial + t.slot * (int64_t)np;
    const bool add = direct && b.accumulate;
    const int npl = (pL + 1) * (pL + 1);
#pragma unroll 1
    for (int c = lane; c < np; c += 32) {
        double v = 0.0;
        if (c < npl) v = finish_desc(accb[c].rounded(), b.norm, col_desc(c), C::D_OUT, KIND + 1, sexp);
        if (add)
            out[c] += v;
        else
            out[c] = v;
    }
    __syncwarp();
}

// The persistent kernel of one group: tiles t0 .. t1-1 of the sorted list
// (t1 < 0: t0 .. t0 + *n_tiles_dev - 1), pulled through the group's counter g.
template <typename T, int P, int KIND, int DENS>
__global__ void __launch_bounds__(BATCH_WARPS * 32, (BatchCfg<T, P, KIND, DENS>::MIN_CTAS))
    q2x_batch_group_kernel(const BatchArgs b, int64_t t0, int64_t t1, int g)
{
    using BC = BatchCfg<T, P, KIND, DENS>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    unsigned char* wsm = smem_raw + (size_t)wib * BC::WARP_BYTES;
    T* tile = reinterpret_cast<T*>(wsm);
    LeafSum<T>* accb = reinterpret_cast<LeafSum<T>*>(tile + 2 * BC::CH * KCfg<T>::LD);  // 2 CH LD sizeof(T) % 8 == 0
    const int64_t nt = (t1 < 0) ? __ldg(b.n_tiles_dev) : t1 - t0;
#pragma unroll 1
    while (true) {
        unsigned long long ti = 0;
        if (lane == 0) ti = atomicAdd(b.counter + g, 1ull);
        ti = __shfl_sync(0xffffffffu, ti, 0);
        if (ti >= (unsigned long long)nt) break;
        const BatchTile t = b.tiles[t0 + (int64_t)ti];
        batch_tile<T, P, KIND, DENS, BC::CH>(b, t, tile, accb, lane);
    }
}

// Host entry points of one group's kernel (explicitly instantiated in
// q2x_batch_f32.cu / q2x_batch_f64.cu).
struct BatchGroupFns {
    cudaError_t (*launch)(const BatchArgs&, int64_t t0, int64_t t1, int g, int grid, cudaStream_t);
    cudaError_t (*occupancy)(int* blocks_per_sm);
    size_t smem;
};

template <typename T, int P, int KIND, int DENS>
cudaError_t batch_group_occupancy(int* blocks_per_sm)
{
    const size_t smem = BATCH_WARPS * BatchCfg<T, P, KIND, DENS>::WARP_BYTES;
    cudaError_t e = cudaFuncSetAttribute(q2x_batch_group_kernel<T, P, KIND, DENS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, q2x_batch_group_kernel<T, P, KIND, DENS>,
                                                         BATCH_WARPS * 32, smem);
}

template <typename T, int P, int KIND, int DENS>
cudaError_t batch_group_launch(const BatchArgs& b, int64_t t0, int64_t t1, int g, int grid, cudaStream_t st)
{
    const size_t smem = BATCH_WARPS * BatchCfg<T, P, KIND, DENS>::WARP_BYTES;
    cudaError_t e = cudaFuncSetAttribute(q2x_batch_group_kernel<T, P, KIND, DENS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    q2x_batch_group_kernel<T, P, KIND, DENS><<<grid, BATCH_WARPS * 32, smem, st>>>(b, t0, t1, g);
    return cudaGetLastError();
}

#define Q2X_BATCH_FNS(T, KIND, DENS, P)                                                            \
    BatchGroupFns{&batch_group_launch<T, P, KIND, DENS>, &batch_group_occupancy<T, P, KIND, DENS>,    \
                  BATCH_WARPS * BatchCfg<T, P, KIND, DENS>::WARP_BYTES}
#define Q2X_BATCH_FNS_ROW(T, KIND, DENS)                                                           \
    {Q2X_BATCH_FNS(T, KIND, DENS, 4), Q2X_BATCH_FNS(T, KIND, DENS, 8), Q2X_BATCH_FNS(T, KIND, DENS, 12), \
     Q2X_BATCH_FNS(T, KIND, DENS, 16), Q2X_BATCH_FNS(T, KIND, DENS, 20)}

// [combo][bin] of a precision: combo 0 segments, 1 triangles constant
// density, 2 triangles linear density, 3 tetrahedra; bins P = 4, 8, 12, 16, 20
const BatchGroupFns* batch_group_table_f32();
const BatchGroupFns* batch_group_table_f64();

// coef[L] (+)= sum of the partial rows slot_off[L] .. slot_off[L+1]-1, in order
__global__ void q2x_batch_combine(const double* __restrict__ partial, const int64_t* __restrict__ slot_off,
                                  int np, int64_t n_leaves, double* coef, int accumulate);

// ---- Leaf tiles of one element set (q2x_tiles.cu): the single-layer FP32
// path of the element calls.  Every leaf of n_L > 0 elements becomes
// ceil(n_L / T) tiles of one kind and degree bin (balanced sizes); a leaf of
// one tile writes its row straight to coef, a leaf of several sums its tiles'
// rows in the combine.  All on the device, in stream order: no host
// synchronisation, so the call stays capturable in a CUDA graph.
struct LeafTileWork {
    BatchTile* tiles;       // [max_tiles]
    int64_t* tile_pre;      // [n_leaves]: a leaf's first tile within its block of leaves
    int64_t* slot_pre;      // [n_leaves]: its first partial row within the block
    int64_t* block_tiles;   // [n_blocks] (then their exclusive prefix)
    int64_t* block_slots;   // [n_blocks]
    int64_t* slot_off;      // [n_leaves + 1]: partial rows of each multi-tile leaf
    int64_t* n_tiles;       // [1]
    unsigned long long* counter;  // [1]
    int64_t max_tiles, max_slots; // buffer sizes: tiles and partial rows past them are dropped
    int64_t n_elem;               // element ranges are clamped to [0, n_elem)
};
constexpr int kLeafTileBlock = 1024;  // leaves per block of the tile count
inline int64_t leaf_tile_blocks(int64_t n_leaves) { return (n_leaves + kLeafTileBlock - 1) / kLeafTileBlock; }
inline int64_t leaf_tile_max_tiles(int64_t n_leaves, int64_t n_elem, int64_t T) { return n_leaves + (n_elem + T - 1) / T; }
inline int64_t leaf_tile_max_slots(int64_t n_elem, int64_t T) { return 2 * ((n_elem + T - 1) / T); }
// tile list of leaf_off with at most T elements per tile
cudaError_t leaf_tiles_build(const int64_t* leaf_off, int64_t n_leaves, int64_t T, int combo, int bin,
                             const LeafTileWork& w, cudaStream_t st);
// coef rows of the multi-tile leaves (sum of their partial rows in order) and,
// unless accumulating, zero rows for empty leaves
cudaError_t leaf_tiles_combine(const double* partial, const int64_t* slot_off, const int64_t* leaf_off,
                               int np, int64_t n_leaves, double* coef, int accumulate, cudaStream_t st);

}  // namespace q2x
