// q2x_tiles.cu -- leaf tiles of one element set, built on the device: the
// tile list the single-layer FP32 path runs through the batch's persistent
// tile kernel (see q2x_batch.cuh), and its combine.
#include <cuda_runtime.h>

#include <cstdint>

#include "q2x_batch.cuh"

namespace q2x {

namespace {

// inclusive warp scan of v
__device__ __forceinline__ int64_t warp_scan(int64_t v, int lane)
{
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int64_t u = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += u;
    }
    return v;
}

// exclusive block scan of two counts (blockDim.x == kLeafTileBlock); the
// block totals go to *tot_a, *tot_b
__device__ __forceinline__ void block_scan2(int64_t a, int64_t b, int64_t& ea, int64_t& eb, int64_t* tot_a,
                                            int64_t* tot_b)
{
    __shared__ int64_t wa[32], wb[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t ia = warp_scan(a, lane), ib = warp_scan(b, lane);
    if (lane == 31) {
        wa[wid] = ia;
        wb[wid] = ib;
    }
    __syncthreads();
    if (wid == 0) {
        const int64_t xa = warp_scan(wa[lane], lane), xb = warp_scan(wb[lane], lane);
        wa[lane] = xa - wa[lane];
        wb[lane] = xb - wb[lane];
        if (lane == 31) {
            *tot_a = xa;
            *tot_b = xb;
        }
    }
    __syncthreads();
    ea = wa[wid] + ia - a;
    eb = wb[wid] + ib - b;
}

// element range of leaf L clamped to [0, n_elem) (offsets that decrease or
// leave the range are reported by the offset check; here they only must not
// lead outside the buffers)
__device__ __forceinline__ void leaf_range(const int64_t* leaf_off, int64_t L, int64_t n_elem, int64_t& e0,
                                           int64_t& e1)
{
    e0 = __ldg(leaf_off + L);
    e1 = __ldg(leaf_off + L + 1);
    e0 = e0 < 0 ? 0 : e0 > n_elem ? n_elem : e0;
    e1 = e1 < e0 ? e0 : e1 > n_elem ? n_elem : e1;
}

// tiles of leaf L (0 if empty) and its partial rows (its tiles if it has
// several, else 0)
__device__ __forceinline__ void leaf_counts(const int64_t* leaf_off, int64_t L, int64_t T, int64_t n_elem,
                                            int64_t& nt, int64_t& ns)
{
    int64_t e0, e1;
    leaf_range(leaf_off, L, n_elem, e0, e1);
    const int64_t n = e1 - e0;
    nt = n > 0 ? (n + T - 1) / T : 0;
    ns = nt >= 2 ? nt : 0;
}

__global__ void __launch_bounds__(kLeafTileBlock) leaf_tile_count_kernel(const int64_t* leaf_off, int64_t n_leaves,
                                                                       int64_t T, LeafTileWork w)
{
    const int64_t L = (int64_t)blockIdx.x * kLeafTileBlock + threadIdx.x;
    int64_t nt = 0, ns = 0;
    if (L < n_leaves) leaf_counts(leaf_off, L, T, w.n_elem, nt, ns);
    int64_t et, es;
    block_scan2(nt, ns, et, es, w.block_tiles + blockIdx.x, w.block_slots + blockIdx.x);
    if (L < n_leaves) {
        w.tile_pre[L] = et;
        w.slot_pre[L] = es;
    }
}

// exclusive prefix of the block totals, in place (one block, chunks of
// kLeafTileBlock); the grand total of tiles to *n_tiles
__global__ void __launch_bounds__(kLeafTileBlock) leaf_tile_scan_kernel(int64_t n_blocks, LeafTileWork w)
{
    __shared__ int64_t carry[2];
    if (threadIdx.x == 0) carry[0] = carry[1] = 0;
    __syncthreads();
    for (int64_t b0 = 0; b0 < n_blocks; b0 += kLeafTileBlock) {
        const int64_t b = b0 + threadIdx.x;
        const int64_t vt = b < n_blocks ? w.block_tiles[b] : 0, vs = b < n_blocks ? w.block_slots[b] : 0;
        __shared__ int64_t tot_t, tot_s;
        int64_t et, es;
        block_scan2(vt, vs, et, es, &tot_t, &tot_s);
        if (b < n_blocks) {
            w.block_tiles[b] = carry[0] + et;
            w.block_slots[b] = carry[1] + es;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            carry[0] += tot_t;
            carry[1] += tot_s;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *w.n_tiles = carry[0] < w.max_tiles ? carry[0] : w.max_tiles;
}

// one thread per leaf: its tiles (balanced sizes, at most T elements) and
// its partial-row offset
__global__ void leaf_tile_fill_kernel(const int64_t* leaf_off, int64_t n_leaves, int64_t T, int combo, int bin,
                                      LeafTileWork w)
{
    const int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (L >= n_leaves) return;
    const int64_t blk = L / kLeafTileBlock;
    const int64_t t0 = w.block_tiles[blk] + w.tile_pre[L];
    const int64_t s0 = w.block_slots[blk] + w.slot_pre[L];
    int64_t nt, ns;
    leaf_counts(leaf_off, L, T, w.n_elem, nt, ns);
    const int64_t smax = w.max_slots;
    w.slot_off[L] = s0 < smax ? s0 : smax;
    if (L == n_leaves - 1) w.slot_off[n_leaves] = s0 + ns < smax ? s0 + ns : smax;
    if (nt == 0) return;
    int64_t e0, e1;
    leaf_range(leaf_off, L, w.n_elem, e0, e1);
    const int64_t chunk = (e1 - e0 + nt - 1) / nt;
    for (int64_t i = 0; i < nt; ++i) {
        if (t0 + i >= w.max_tiles) break;  // past the counted tiles (bad offsets only)
        BatchTile t;
        t.combo = combo;
        t.bin = bin;
        t.leaf = (int32_t)L;
        t.flags = (nt == 1) ? 1 : 0;
        t.slot = (nt == 1) ? 0 : s0 + i;
        t.e_lo = e0 + i * chunk;
        t.e_hi = (t.e_lo + chunk < e1) ? t.e_lo + chunk : e1;
        if (nt > 1 && s0 + i >= smax) {  // no partial row left (bad offsets only): an empty tile
            t.flags = 1;
            t.slot = 0;
            t.e_hi = t.e_lo;
        }
        w.tiles[t0 + i] = t;
    }
}

// one warp per 32 leaves: each lane reads one leaf's slot and element
// ranges; the warp then handles, one after the other, the leaves that have
// work (several tiles: their partial rows summed in slot order; empty and
// not accumulating: a zero row), columns over the lanes
__global__ void leaf_tile_combine_kernel(const double* __restrict__ partial, const int64_t* __restrict__ slot_off,
                                         const int64_t* __restrict__ leaf_off, int np, int64_t n_leaves, double* coef,
                                         int accumulate)
{
    const int lane = threadIdx.x & 31;
    const int64_t L0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32;
    if (L0 >= n_leaves) return;  // warp-uniform
    const int64_t L = L0 + lane;
    long long s0 = 0, s1 = 0;
    bool work = false;
    if (L < n_leaves) {
        s0 = slot_off[L];
        s1 = slot_off[L + 1];
        const bool empty = __ldg(leaf_off + L + 1) == __ldg(leaf_off + L);
        // a single-tile leaf wrote its own row
        work = s1 > s0 || (empty && !accumulate);
    }
    unsigned mask = __ballot_sync(0xffffffffu, work);
    while (mask) {
        const int r = __ffs(mask) - 1;
        mask &= mask - 1;
        const long long a0 = __shfl_sync(0xffffffffu, s0, r), a1 = __shfl_sync(0xffffffffu, s1, r);
        double* row = coef + (L0 + r) * np;
        if (a1 == a0) {  // an empty leaf is zero
            for (int c = lane; c < np; c += 32) row[c] = 0.0;
        } else {
            for (int c = lane; c < np; c += 32) {
                double acc = 0.0;
                for (long long sl = a0; sl < a1; ++sl) acc += partial[sl * np + c];
                row[c] = accumulate ? row[c] + acc : acc;
            }
        }
    }
}

}  // namespace

cudaError_t leaf_tiles_build(const int64_t* leaf_off, int64_t n_leaves, int64_t T, int combo, int bin,
                             const LeafTileWork& w, cudaStream_t st)
{
    const int64_t nb = leaf_tile_blocks(n_leaves);
    leaf_tile_count_kernel<<<(unsigned)nb, kLeafTileBlock, 0, st>>>(leaf_off, n_leaves, T, w);
    leaf_tile_scan_kernel<<<1, kLeafTileBlock, 0, st>>>(nb, w);
    leaf_tile_fill_kernel<<<(unsigned)((n_leaves + 255) / 256), 256, 0, st>>>(leaf_off, n_leaves, T, combo, bin, w);
    return cudaGetLastError();
}

cudaError_t leaf_tiles_combine(const double* partial, const int64_t* slot_off, const int64_t* leaf_off, int np,
                               int64_t n_leaves, double* coef, int accumulate, cudaStream_t st)
{
    const int warps = 8;
    const int64_t n_warps = (n_leaves + 31) / 32;
    leaf_tile_combine_kernel<<<(unsigned)((n_warps + warps - 1) / warps), warps * 32, 0, st>>>(
        partial, slot_off, leaf_off, np, n_leaves, coef, accumulate);
    return cudaGetLastError();
}

}  // namespace q2x
