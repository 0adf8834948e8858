// q2x_api.cu -- C ABI of the Q2X library (declared in include/q2x.h):
// argument checks, plan and workspace management, kernel dispatch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "q2x.h"
#include "q2x_batch.cuh"
#include "q2x_kernels.cuh"
#include "q2x_plan.h"

// explicit instantiations live in q2x_inst_*.cu
#define Q2X_DECLARE_ALL(T)                                                                         \
    Q2X_FOR_BINS(Q2X_DECLARE, T, q2x::KIND_SEG, q2x::DENS_CONST, 1)                                \
    Q2X_FOR_BINS(Q2X_DECLARE, T, q2x::KIND_TRI, q2x::DENS_CONST, 1)                                \
    Q2X_FOR_BINS(Q2X_DECLARE, T, q2x::KIND_TRI, q2x::DENS_CONST, 2)                                \
    Q2X_FOR_BINS(Q2X_DECLARE, T, q2x::KIND_TRI, q2x::DENS_CONST, 3)                                \
    Q2X_FOR_BINS(Q2X_DECLARE, T, q2x::KIND_TRI, q2x::DENS_LINEAR, 1)                               \
    Q2X_FOR_BINS(Q2X_DECLARE, T, q2x::KIND_TRI, q2x::DENS_LINEAR, 2)                               \
    Q2X_FOR_BINS(Q2X_DECLARE, T, q2x::KIND_TRI, q2x::DENS_LINEAR, 3)                               \
    Q2X_FOR_BINS(Q2X_DECLARE, T, q2x::KIND_TET, q2x::DENS_CONST, 1)                                \
    Q2X_FOR_BINS(Q2X_DECLARE, T, q2x::KIND_SEG, q2x::DENS_CONST, 4)
Q2X_DECLARE_ALL(float)
Q2X_DECLARE_ALL(double)

namespace {

struct KernelEntry {
    cudaError_t (*launch)(const q2x::ElemArgs&, int, cudaStream_t);
    cudaError_t (*occupancy)(int*, int);
    size_t (*smem)(int);  // dynamic shared memory of a launch at np_max columns
};

constexpr int kNumBins = 5;
constexpr int kBins[kNumBins] = {4, 8, 12, 16, 20};
constexpr int kNumCombos = 9;

#define Q2X_ENTRY(T, P, KIND, DENS, OUTS) \
    {&q2x::launch_elem<T, P, KIND, DENS, OUTS>, &q2x::occupancy_elem<T, P, KIND, DENS, OUTS>, \
     &q2x::elem_launch_smem<T, P, KIND, DENS, OUTS>},
#define Q2X_ROW(T, KIND, DENS, OUTS) {Q2X_FOR_BINS(Q2X_ENTRY, T, KIND, DENS, OUTS)},
#define Q2X_ROWS(T)                                                                                          \
    {Q2X_ROW(T, q2x::KIND_SEG, q2x::DENS_CONST, 1) Q2X_ROW(T, q2x::KIND_TRI, q2x::DENS_CONST, 1)              \
         Q2X_ROW(T, q2x::KIND_TRI, q2x::DENS_CONST, 2) Q2X_ROW(T, q2x::KIND_TRI, q2x::DENS_CONST, 3)          \
             Q2X_ROW(T, q2x::KIND_TRI, q2x::DENS_LINEAR, 1) Q2X_ROW(T, q2x::KIND_TRI, q2x::DENS_LINEAR, 2)   \
                 Q2X_ROW(T, q2x::KIND_TRI, q2x::DENS_LINEAR, 3) Q2X_ROW(T, q2x::KIND_TET, q2x::DENS_CONST, 1)    \
                     Q2X_ROW(T, q2x::KIND_SEG, q2x::DENS_CONST, 4)}
// [precision: 0 FP64, 1 FP32][combo][bin]; combos: 0 segments, 1-3 triangles
// constant density (single, double, both), 4-6 linear density, 7 tetrahedra,
// 8 segments carrying a vector density
const KernelEntry kTable[2][kNumCombos][kNumBins] = {Q2X_ROWS(double), Q2X_ROWS(float)};

int combo_index(int kind, int dens, bool single, bool dbl, bool vec = false)
{
    if (vec) return 8;
    if (kind == q2x::KIND_SEG) return 0;
    if (kind == q2x::KIND_TET) return 7;
    const int outs = (single ? 1 : 0) | (dbl ? 2 : 0);
    return (dens == Q2X_DENSITY_LINEAR ? 4 : 1) + outs - 1;
}

thread_local std::string g_create_error;

}  // namespace

q2x_status q2x_fail(q2x_plan_t plan, q2x_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (plan)
        plan->last_error = buf;
    else
        g_create_error = buf;
    return st;
}

q2x_status q2x_cuda_fail(q2x_plan_t plan, cudaError_t e, const char* what)
{
    return q2x_fail(plan, Q2X_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

namespace {

#define fail q2x_fail
#define cuda_fail q2x_cuda_fail

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// grow the workspace to at least `bytes` (synchronises the plan's stream
// before releasing the old buffer)
q2x_status ensure_ws(q2x_plan_t plan, size_t bytes)
{
    if (bytes <= plan->ws_bytes) return Q2X_OK;
    cudaError_t e;
    if (plan->ws) {
        e = cudaStreamSynchronize(plan->stream);
        if (e != cudaSuccess) return cuda_fail(plan, e, "cudaStreamSynchronize");
        cudaFree(plan->ws);
        plan->ws = nullptr;
        plan->ws_bytes = 0;
    }
    bytes = align_up(std::max<size_t>(bytes, 1 << 20), 1 << 20);
    e = cudaMalloc(&plan->ws, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(plan, Q2X_ERR_OOM, "workspace allocation of %zu bytes failed", bytes);
    }
    plan->ws_bytes = bytes;
    return Q2X_OK;
}

q2x_status take_event(q2x_plan_t plan, cudaEvent_t* ev)
{
    if (!plan->ev_pool.empty()) {
        *ev = plan->ev_pool.back();
        plan->ev_pool.pop_back();
        return Q2X_OK;
    }
    cudaError_t e = cudaEventCreate(ev);
    if (e != cudaSuccess) return cuda_fail(plan, e, "cudaEventCreate");
    return Q2X_OK;
}

int bin_index(int p)
{
    for (int b = 0; b < kNumBins; ++b)
        if (p <= kBins[b]) return b;
    return -1;
}

// ------------------------------------------------------------ small kernels

// leaf_off must be non-decreasing with leaf_off[0] = 0, leaf_off[n_leaves] = n_elem
__global__ void check_leaf_off_kernel(const int64_t* off, int64_t n_leaves, int64_t n_elem,
                                      unsigned* err)
{
    const int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (L > n_leaves) return;
    const int64_t o = off[L];
    bool bad = (o < 0 || o > n_elem);
    if (L == 0 && o != 0) bad = true;
    if (L == n_leaves && o != n_elem) bad = true;
    if (L < n_leaves && off[L + 1] < o) bad = true;
    if (bad) atomicOr(err, Q2X_DEVERR_LEAF_OFF);
}

// per-leaf scale: largest distance from the centre to a vertex of its
// elements, as the bit pattern of a non-negative float (atomicMax on ints
// orders non-negative floats correctly)
__global__ void leaf_rho_kernel(int64_t n_elem, int64_t n_vert, int nv, const double* vx,
                                const double* vy, const double* vz, const int32_t* idx,
                                int64_t n_leaves, const int64_t* off, const double* leaf_c,
                                int* rho_bits)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_elem) return;
    int64_t L = e;
    if (off) L = q2x::leaf_search(off, 0, n_leaves - 1, e);
    const double cx = leaf_c[L], cy = leaf_c[n_leaves + L], cz = leaf_c[2 * n_leaves + L];
    float dmax = 0.f;
    for (int k = 0; k < nv; ++k) {
        int64_t v = idx[(int64_t)k * n_elem + e];
        if (v < 0 || v >= n_vert) continue;
        const float dx = (float)(vx[v] - cx), dy = (float)(vy[v] - cy), dz = (float)(vz[v] - cz);
        const float d = sqrtf(dx * dx + dy * dy + dz * dz);
        if (d == d) dmax = fmaxf(dmax, d);
    }
    atomicMax(rho_bits + L, __float_as_int(dmax));
}

__global__ void rho_bits_to_double(const int* bits, double* rho, int64_t n)
{
    const int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (L < n) rho[L] = (double)__int_as_float(bits[L]);
}

// segmented sum of per-element rows: one thread per (leaf, column), eight
// rows in flight per step; every column is summed in element order
// (deterministic, the same order as a plain loop)
__global__ void leaf_reduce_kernel(const double* __restrict__ elem, int np, int64_t n_elem,
                                   int64_t n_leaves, const int64_t* __restrict__ off, double* coef,
                                   int accumulate)
{
    constexpr int U = 8;
    // the leaves' columns back to back, so that a warp is full even where a
    // leaf's last columns do not fill one
    const int64_t unit = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t L = unit / np;
    if (L >= n_leaves) return;
    const int c = (int)(unit - L * np);
    // clamped: a bad leaf_off is reported by check_leaf_off_kernel, never read past
    const int64_t e0 = min(max(off[L], (int64_t)0), n_elem);
    const int64_t e1 = min(max(off[L + 1], e0), n_elem);
    const double* col = elem + c;
    double acc = 0.0;
    int64_t e = e0;
    for (; e + U <= e1; e += U) {
        double v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = __ldg(col + (e + u) * np);
#pragma unroll
        for (int u = 0; u < U; ++u) acc += v[u];
    }
    for (; e < e1; ++e) acc += __ldg(col + e * np);
    double* d = coef + L * np + c;
    *d = accumulate ? *d + acc : acc;
}

// The same walk with NW weighted sums per column: acc_j = fma(w_j[e], v, acc_j)
// in element order.
template <int NW>
__global__ void leaf_reduce_weighted_kernel(const double* __restrict__ elem, int np, int64_t n_elem,
                                            const double* __restrict__ w, int64_t w_stride, int64_t n_leaves,
                                            const int64_t* __restrict__ off, double* coef, int64_t coef_stride,
                                            int accumulate)
{
    constexpr int U = 8;
    // one warp per (leaf, 32 columns): the leaf's weights are read once per warp
    const int lane = threadIdx.x & 31;
    const int groups = (np + 31) >> 5;
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t L = gw / groups;
    if (L >= n_leaves) return;
    const int c = (int)(gw - L * groups) * 32 + lane;
    if (c >= np) return;
    const int64_t e0 = min(max(off[L], (int64_t)0), n_elem);
    const int64_t e1 = min(max(off[L + 1], e0), n_elem);
    const double* col = elem + c;
    double acc[NW];
#pragma unroll
    for (int j = 0; j < NW; ++j) acc[j] = 0.0;
    int64_t e = e0;
    for (; e + U <= e1; e += U) {
        double v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = __ldg(col + (e + u) * np);
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int j = 0; j < NW; ++j) acc[j] = fma(__ldg(w + j * w_stride + e + u), v[u], acc[j]);
    }
    for (; e < e1; ++e) {
        const double v = __ldg(col + e * np);
#pragma unroll
        for (int j = 0; j < NW; ++j) acc[j] = fma(__ldg(w + j * w_stride + e), v, acc[j]);
    }
#pragma unroll
    for (int j = 0; j < NW; ++j) {
        double* d = coef + j * coef_stride + L * np + c;
        *d = accumulate ? *d + acc[j] : acc[j];
    }
}

// --------------------------------------------------------------- dispatch

// Elements per leaf tile of the FP32-mixed single-layer path.
constexpr int64_t kLeafTileElems = 256;

// workspace of the leaf-tile path (after the per-leaf scales): the tile list,
// the scans, and the partial rows of leaves of several tiles
size_t leaf_tile_ws_bytes(int64_t n_elem, int64_t n_leaves, int np)
{
    const int64_t nb = q2x::leaf_tile_blocks(n_leaves);
    const int64_t mt = q2x::leaf_tile_max_tiles(n_leaves, n_elem, kLeafTileElems);
    const int64_t ms = q2x::leaf_tile_max_slots(n_elem, kLeafTileElems);
    return align_up(sizeof(q2x::BatchTile) * (size_t)mt, 256) + 2 * align_up(sizeof(int64_t) * (size_t)n_leaves, 256) +
           2 * align_up(sizeof(int64_t) * (size_t)nb, 256) + align_up(sizeof(int64_t) * (size_t)(n_leaves + 1), 256) +
           256 + 256 + align_up(sizeof(double) * (size_t)ms * np, 256);
}

q2x_status run_elements(q2x_plan_t plan, int kind, int dens, int64_t n_elem, int64_t n_vert,
                        const double* vxyz, const int32_t* idx, const double* sigma,
                        int64_t n_leaves, const int64_t* leaf_off, const double* leaf_c,
                        const double* leaf_rho, const int32_t* leaf_p, double* coef0,
                        double* coef1, int accumulate, const double* wvec = nullptr, double* coef2 = nullptr)
{
    // wvec: a vector density (segments): the three components weight one
    // unit-density pass, into coef0, coef1, coef2
    const bool vec = wvec != nullptr;
    if (!plan) return fail(nullptr, Q2X_ERR_ARG, "plan is NULL");
    if (n_elem < 0 || n_vert < 0 || n_leaves < 0)
        return fail(plan, Q2X_ERR_ARG, "negative size (n_elem=%lld n_vert=%lld n_leaves=%lld)",
                    (long long)n_elem, (long long)n_vert, (long long)n_leaves);
    if (!coef0 && !coef1 && !coef2) return fail(plan, Q2X_ERR_ARG, "no output requested");
    if (vec && (kind != q2x::KIND_SEG || !leaf_off))
        return fail(plan, Q2X_ERR_ARG, "a vector density needs segments in leaf mode");
    if (accumulate != 0 && accumulate != 1) return fail(plan, Q2X_ERR_ARG, "accumulate must be 0 or 1");
    if (!leaf_off && n_leaves != n_elem)
        return fail(plan, Q2X_ERR_ARG, "per-element mode (leaf_off NULL) needs n_leaves == n_elem");
    if (n_elem > 0) {
        if (!vxyz || !idx || (!sigma && !vec))
            return fail(plan, Q2X_ERR_ARG, "vxyz, idx and sigma must be non-NULL");
        if (n_vert <= 0) return fail(plan, Q2X_ERR_ARG, "n_vert must be positive");
        if (n_leaves <= 0) return fail(plan, Q2X_ERR_ARG, "n_leaves must be positive");
        if (n_elem > ((int64_t)1 << 40)) return fail(plan, Q2X_ERR_ARG, "n_elem too large");
    }
    if (n_leaves > 0 && !leaf_c) return fail(plan, Q2X_ERR_ARG, "leaf_c must be non-NULL");
    if (dens != Q2X_DENSITY_CONST && dens != Q2X_DENSITY_LINEAR)
        return fail(plan, Q2X_ERR_ARG, "bad density mode %d", dens);

    cudaError_t e = cudaSetDevice(plan->device);
    if (e != cudaSuccess) return cuda_fail(plan, e, "cudaSetDevice");
    const int np = (plan->p_max + 1) * (plan->p_max + 1);

    if (n_elem == 0) {
        if (!accumulate && n_leaves > 0) {
            for (double* c : {coef0, coef1, coef2})
                if (c) {
                    e = cudaMemsetAsync(c, 0, sizeof(double) * (size_t)n_leaves * np, plan->stream);
                    if (e != cudaSuccess) return cuda_fail(plan, e, "cudaMemsetAsync");
                }
        }
        return Q2X_OK;
    }

    const int prec = plan->prec;  // 0 FP64, 1 FP32-mixed
    const int combo = combo_index(kind, dens, coef0 != nullptr, kind == q2x::KIND_TRI && coef1 != nullptr, vec);
    const bool dbl = kind == q2x::KIND_TRI && coef1 != nullptr;
    const int nacc = q2x::elem_outputs(kind, vec ? 4 : dbl ? 2 : 1);
    const int nv = kind + 2;
    const int bin = bin_index(plan->p_max);
    if (bin < 0) return fail(plan, Q2X_ERR_RANGE, "p_max %d above %d", plan->p_max, Q2X_P_MAX);
    const KernelEntry& ke = kTable[prec][combo][bin];
    const int wpc = prec ? q2x::elem_warps_per_cta<float>() : q2x::elem_warps_per_cta<double>();

    int& occ = plan->occ_cache[prec][combo][bin];
    if (occ == 0) {
        e = ke.occupancy(&occ, np);
        if (e != cudaSuccess) return cuda_fail(plan, e, "occupancy query");
        if (occ <= 0) return fail(plan, Q2X_ERR_CUDA, "kernel does not fit on the device (smem %zu)", ke.smem(np));
    }
    // FP32-mixed single layer in leaf mode: leaf tiles through the batch's
    // persistent tile kernel (q2x_tiles.cu): a round holds one leaf's elements,
    // so every staged chunk is summed pairwise, with no leaf-boundary work in
    // the degree loop, and warps pull tiles from a counter
    // (its workspace bound assumes every tile needs a partial row: beyond
    // 8 GiB the element kernel, whose workspace is per warp range, runs)
    const bool tiles = prec == 1 && leaf_off && !vec && coef0 && !(kind == q2x::KIND_TRI && coef1) &&
                       n_leaves < ((int64_t)1 << 31) && leaf_tile_ws_bytes(n_elem, n_leaves, np) <= ((size_t)8 << 30);
    const int64_t resident_warps = (int64_t)occ * wpc * plan->num_sms;
    // one range per resident warp (ranges need not be multiples of 32: rounds
    // are formed per leaf inside the kernel), at least one full round each
    int64_t T = (n_elem + resident_warps - 1) / resident_warps;
    T = std::max<int64_t>(32, T);
    const int64_t n_ranges = (n_elem + T - 1) / T;

    // workspace: slots, then per-leaf scale (FP32 without leaf_rho)
    const bool need_rho = prec == 1 && leaf_rho == nullptr;
    const size_t slot_bytes = tiles ? 0 : align_up(sizeof(double) * (size_t)n_ranges * 2 * nacc * np, 256);  // FP64 partials
    const size_t rho_bytes = need_rho ? align_up(sizeof(double) * (size_t)n_leaves, 256) : 0;
    const size_t bits_bytes = need_rho ? align_up(sizeof(int) * (size_t)n_leaves, 256) : 0;
    const size_t tile_bytes = tiles ? leaf_tile_ws_bytes(n_elem, n_leaves, np) : 0;
    q2x_status st = ensure_ws(plan, slot_bytes + rho_bytes + bits_bytes + tile_bytes);
    if (st != Q2X_OK) return st;
    unsigned char* ws = static_cast<unsigned char*>(plan->ws);

    if (leaf_off) {
        const int64_t nb = (n_leaves + 1 + 255) / 256;
        check_leaf_off_kernel<<<(unsigned)nb, 256, 0, plan->stream>>>(leaf_off, n_leaves, n_elem, plan->d_err);
        plan->launches += 1;
    }
    if (need_rho) {
        int* bits = reinterpret_cast<int*>(ws + slot_bytes + rho_bytes);
        double* rho = reinterpret_cast<double*>(ws + slot_bytes);
        e = cudaMemsetAsync(bits, 0, sizeof(int) * (size_t)n_leaves, plan->stream);
        if (e != cudaSuccess) return cuda_fail(plan, e, "cudaMemsetAsync");
        leaf_rho_kernel<<<(unsigned)((n_elem + 255) / 256), 256, 0, plan->stream>>>(
            n_elem, n_vert, nv, vxyz, vxyz + n_vert, vxyz + 2 * n_vert, idx, n_leaves, leaf_off, leaf_c, bits);
        rho_bits_to_double<<<(unsigned)((n_leaves + 255) / 256), 256, 0, plan->stream>>>(bits, rho, n_leaves);
        plan->launches += 2;
        leaf_rho = rho;
    }

    if (tiles) {
        unsigned char* p = ws + slot_bytes + rho_bytes + bits_bytes;
        auto take = [&](size_t bytes) {
            unsigned char* q = p;
            p += align_up(bytes, 256);
            return q;
        };
        const int64_t nb = q2x::leaf_tile_blocks(n_leaves);
        const int64_t mt = q2x::leaf_tile_max_tiles(n_leaves, n_elem, kLeafTileElems);
        const int64_t ms = q2x::leaf_tile_max_slots(n_elem, kLeafTileElems);
        q2x::LeafTileWork w;
        w.tiles = reinterpret_cast<q2x::BatchTile*>(take(sizeof(q2x::BatchTile) * (size_t)mt));
        w.tile_pre = reinterpret_cast<int64_t*>(take(sizeof(int64_t) * (size_t)n_leaves));
        w.slot_pre = reinterpret_cast<int64_t*>(take(sizeof(int64_t) * (size_t)n_leaves));
        w.block_tiles = reinterpret_cast<int64_t*>(take(sizeof(int64_t) * (size_t)nb));
        w.block_slots = reinterpret_cast<int64_t*>(take(sizeof(int64_t) * (size_t)nb));
        w.slot_off = reinterpret_cast<int64_t*>(take(sizeof(int64_t) * (size_t)(n_leaves + 1)));
        w.n_tiles = reinterpret_cast<int64_t*>(take(sizeof(int64_t)));
        w.counter = reinterpret_cast<unsigned long long*>(take(sizeof(unsigned long long)));
        double* partial = reinterpret_cast<double*>(take(sizeof(double) * (size_t)ms * np));
        w.max_tiles = mt;
        w.max_slots = ms;
        w.n_elem = n_elem;
        const int tcombo = (kind == q2x::KIND_SEG) ? 0 : (kind == q2x::KIND_TET) ? 3 : (dens == Q2X_DENSITY_LINEAR ? 2 : 1);
        const q2x::BatchGroupFns& f = q2x::batch_group_table_f32()[tcombo * 5 + bin];
        int& tocc = plan->tile_occ[tcombo][bin];
        if (tocc == 0) {
            e = f.occupancy(&tocc);
            if (e != cudaSuccess) return cuda_fail(plan, e, "tile kernel occupancy query");
            if (tocc <= 0) return fail(plan, Q2X_ERR_CUDA, "tile kernel does not fit on the device (smem %zu)", f.smem);
        }
        e = q2x::leaf_tiles_build(leaf_off, n_leaves, kLeafTileElems, tcombo, bin, w, plan->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(w.counter, 0, sizeof(unsigned long long), plan->stream);
        if (e != cudaSuccess) return cuda_fail(plan, e, "leaf tile list");
        q2x::BatchArgs b{};
        b.kind[kind].n_elem = n_elem;
        b.kind[kind].n_vert = n_vert;
        b.kind[kind].vx = vxyz;
        b.kind[kind].vy = vxyz + n_vert;
        b.kind[kind].vz = vxyz + 2 * n_vert;
        b.kind[kind].idx = idx;
        b.kind[kind].sigma = sigma;
        b.n_leaves = n_leaves;
        b.leaf_c = leaf_c;
        b.leaf_rho = leaf_rho;
        b.leaf_p = leaf_p;
        b.p_max = plan->p_max;
        b.np_max = np;
        b.norm = plan->norm;
        b.tiles = w.tiles;
        b.n_tiles = 0;
        b.counter = w.counter;
        b.partial = partial;
        b.err = plan->d_err;
        b.coef = coef0;
        b.accumulate = accumulate;
        b.n_tiles_dev = w.n_tiles;
        cudaEvent_t ev0 = nullptr, ev1 = nullptr;
        if (plan->timing) {
            st = take_event(plan, &ev0);
            if (st == Q2X_OK) st = take_event(plan, &ev1);
            if (st != Q2X_OK) return st;
            cudaEventRecord(ev0, plan->stream);
        }
        e = f.launch(b, 0, -1, 0, tocc * plan->num_sms, plan->stream);
        if (e != cudaSuccess) return cuda_fail(plan, e, "tile kernel launch");
        if (plan->timing) {
            cudaEventRecord(ev1, plan->stream);
            plan->ev_pending.emplace_back(ev0, ev1);
        }
        e = q2x::leaf_tiles_combine(partial, w.slot_off, leaf_off, np, n_leaves, coef0, accumulate, plan->stream);
        if (e != cudaSuccess) return cuda_fail(plan, e, "leaf tile combine");
        plan->launches += 5;
        return Q2X_OK;
    }

    q2x::ElemArgs a;
    a.n_elem = n_elem;
    a.n_vert = n_vert;
    a.vx = vxyz;
    a.vy = vxyz + n_vert;
    a.vz = vxyz + 2 * n_vert;
    a.idx = idx;
    a.sigma = sigma;
    a.n_leaves = n_leaves;
    a.leaf_off = leaf_off;
    a.leaf_c = leaf_c;
    a.leaf_rho = leaf_rho;
    a.leaf_p = leaf_p;
    a.p_max = plan->p_max;
    a.np_max = np;
    a.coef[0] = coef0;
    a.coef[1] = (kind == q2x::KIND_TRI || vec) ? coef1 : nullptr;
    a.coef[2] = vec ? coef2 : nullptr;
    a.wvec = wvec;
    a.nacc = nacc;
    a.accumulate = accumulate;
    a.norm = plan->norm;
    a.T = T;
    a.n_ranges = n_ranges;
    a.slots = reinterpret_cast<double*>(ws);
    a.err = plan->d_err;

    const int grid = (int)((n_ranges + wpc - 1) / wpc);
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (plan->timing) {
        st = take_event(plan, &ev0);
        if (st == Q2X_OK) st = take_event(plan, &ev1);
        if (st != Q2X_OK) return st;
        cudaEventRecord(ev0, plan->stream);
    }
    e = ke.launch(a, grid, plan->stream);
    if (e != cudaSuccess) return cuda_fail(plan, e, "element kernel launch");
    if (plan->timing) {
        cudaEventRecord(ev1, plan->stream);
        plan->ev_pending.emplace_back(ev0, ev1);
    }
    plan->launches += 1;
    if (leaf_off && n_ranges > 1) {
        const int d_out = (kind == q2x::KIND_SEG) ? 1 : (kind == q2x::KIND_TET) ? 3 : (dens == Q2X_DENSITY_LINEAR ? 3 : 2);
        if (vec)
            e = q2x::launch_fixup(a, plan->stream, d_out, d_out, d_out, kind + 1, kind + 1, kind + 1);
        else
            e = q2x::launch_fixup(a, plan->stream, d_out, d_out - 1, d_out, kind + 1, 1, kind + 1);
        if (e != cudaSuccess) return cuda_fail(plan, e, "fixup kernel launch");
        plan->launches += 1;
    }
    return Q2X_OK;
}

}  // namespace

// ===================================================================== ABI

q2x_status q2x_plan_workspace(q2x_plan_t plan, size_t bytes)
{
    return ensure_ws(plan, bytes);
}

extern "C" {

q2x_status q2x_plan(q2x_plan_t* out, int p_max, q2x_norm norm, q2x_precision precision,
                    void* cuda_stream)
{
    if (!out) return fail(nullptr, Q2X_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (p_max < 0 || p_max > Q2X_P_MAX)
        return fail(nullptr, Q2X_ERR_RANGE, "p_max %d outside 0..%d", p_max, Q2X_P_MAX);
    if (norm != Q2X_NORM_COEFF && norm != Q2X_NORM_MOMENT) return fail(nullptr, Q2X_ERR_ARG, "bad norm %d", (int)norm);
    if (precision != Q2X_FP64 && precision != Q2X_FP32_MIXED)
        return fail(nullptr, Q2X_ERR_ARG, "bad precision %d", (int)precision);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, Q2X_ERR_CUDA, "no CUDA device: %s", cudaGetErrorString(e));
    }
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail(nullptr, Q2X_ERR_CUDA, "device query: %s", cudaGetErrorString(e));
    q2x_plan_s* p = new q2x_plan_s();
    p->p_max = p_max;
    p->norm = (int)norm;
    p->prec = (precision == Q2X_FP32_MIXED) ? 1 : 0;
    p->stream = static_cast<cudaStream_t>(cuda_stream);
    p->device = dev;
    p->num_sms = sms;
    e = cudaMalloc(&p->d_err, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(p->d_err, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMallocHost(&p->h_err, sizeof(unsigned));
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (p->d_err) cudaFree(p->d_err);
        delete p;
        return fail(nullptr, Q2X_ERR_CUDA, "plan allocation: %s", cudaGetErrorString(e));
    }
    *out = p;
    return Q2X_OK;
}

q2x_status q2x_plan_destroy(q2x_plan_t plan)
{
    if (!plan) return Q2X_ERR_ARG;
    cudaSetDevice(plan->device);
    cudaStreamSynchronize(plan->stream);
    if (plan->ws) cudaFree(plan->ws);
    if (plan->d_err) cudaFree(plan->d_err);
    for (cudaEvent_t ev : plan->ev_pool) cudaEventDestroy(ev);
    for (auto& pr : plan->ev_pending) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    if (plan->h_err) cudaFreeHost(plan->h_err);
    delete plan;
    return Q2X_OK;
}

q2x_status q2x_plan_set_stream(q2x_plan_t plan, void* cuda_stream)
{
    if (!plan) return Q2X_ERR_ARG;
    plan->stream = static_cast<cudaStream_t>(cuda_stream);
    return Q2X_OK;
}

q2x_status q2x_plan_set_kernel_timing(q2x_plan_t plan, int enable)
{
    if (!plan) return Q2X_ERR_ARG;
    plan->timing = enable ? 1 : 0;
    return Q2X_OK;
}

q2x_status q2x_plan_kernel_timing(q2x_plan_t plan, double* total_ms, int64_t* n_launches)
{
    if (!plan || !total_ms || !n_launches) return fail(plan, Q2X_ERR_ARG, "NULL argument");
    cudaSetDevice(plan->device);
    cudaError_t e = cudaStreamSynchronize(plan->stream);
    if (e != cudaSuccess) return cuda_fail(plan, e, "cudaStreamSynchronize");
    double tot = 0.0;
    for (auto& pr : plan->ev_pending) {
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, pr.first, pr.second);
        if (e != cudaSuccess) return cuda_fail(plan, e, "cudaEventElapsedTime");
        tot += ms;
        plan->ev_pool.push_back(pr.first);
        plan->ev_pool.push_back(pr.second);
    }
    *total_ms = tot;
    *n_launches = (int64_t)plan->ev_pending.size();
    plan->ev_pending.clear();
    return Q2X_OK;
}

int64_t q2x_launch_count(q2x_plan_t plan) { return plan ? plan->launches : -1; }

const char* q2x_last_error(q2x_plan_t plan) { return plan ? plan->last_error.c_str() : g_create_error.c_str(); }

q2x_status q2x_device_errors(q2x_plan_t plan, uint32_t* bits)
{
    if (!plan || !bits) return Q2X_ERR_ARG;
    cudaSetDevice(plan->device);
    cudaError_t e = cudaMemcpyAsync(plan->h_err, plan->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, plan->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(plan->stream);
    if (e != cudaSuccess) return cuda_fail(plan, e, "reading the device error word");
    *bits = *plan->h_err;
    if (*bits) {
        e = cudaMemsetAsync(plan->d_err, 0, sizeof(unsigned), plan->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(plan->stream);
        if (e != cudaSuccess) return cuda_fail(plan, e, "clearing the device error word");
    }
    return Q2X_OK;
}

q2x_status q2x_sync(q2x_plan_t plan)
{
    uint32_t bits = 0;
    q2x_status st = q2x_device_errors(plan, &bits);
    if (st != Q2X_OK) return st;
    if (bits)
        return fail(plan, Q2X_ERR_DEVICE_INPUT, "device-side input check failed (bits 0x%x:%s%s%s%s)", bits,
                    (bits & Q2X_DEVERR_INDEX) ? " vertex index out of range" : "",
                    (bits & Q2X_DEVERR_NONFINITE) ? " non-finite input" : "",
                    (bits & Q2X_DEVERR_LEAF_P) ? " leaf_p out of range" : "",
                    (bits & Q2X_DEVERR_LEAF_OFF) ? " bad leaf_off" : "");
    return Q2X_OK;
}

q2x_status q2x_reserve(q2x_plan_t plan, int64_t n_elem, int64_t n_leaves)
{
    if (!plan || n_elem < 0 || n_leaves < 0) return fail(plan, Q2X_ERR_ARG, "bad reserve arguments");
    cudaSetDevice(plan->device);
    const int np = (plan->p_max + 1) * (plan->p_max + 1);
    // worst case: one range per 32 elements; FP64 partials in both precisions
    const int64_t n_ranges = (n_elem + 31) / 32;
    const size_t elem = align_up(sizeof(double) * (size_t)n_ranges * 2 * 3 * np, 256);
    size_t tile = plan->prec == 1 ? leaf_tile_ws_bytes(n_elem, n_leaves, np) : 0;
    if (tile > ((size_t)8 << 30)) tile = 0;  // such calls run the element kernel
    const size_t bytes = std::max(elem, tile) + align_up(sizeof(double) * (size_t)n_leaves, 256) +
                         align_up(sizeof(int) * (size_t)n_leaves, 256);
    return ensure_ws(plan, bytes);
}

int64_t q2x_workspace_bytes(q2x_plan_t plan) { return plan ? (int64_t)plan->ws_bytes : -1; }

q2x_status q2x_segments(q2x_plan_t plan, int64_t n_elem, int64_t n_vert, const double* vxyz,
                        const int32_t* idx, const double* sigma, int64_t n_leaves,
                        const int64_t* leaf_off, const double* leaf_c, const double* leaf_rho,
                        const int32_t* leaf_p, double* coef, int accumulate)
{
    if (!coef) return fail(plan, Q2X_ERR_ARG, "coef is NULL");
    return run_elements(plan, q2x::KIND_SEG, Q2X_DENSITY_CONST, n_elem, n_vert, vxyz, idx, sigma,
                        n_leaves, leaf_off, leaf_c, leaf_rho, leaf_p, coef, nullptr, accumulate);
}

q2x_status q2x_triangles(q2x_plan_t plan, int64_t n_elem, int64_t n_vert, const double* vxyz,
                         const int32_t* idx, q2x_density density, const double* sigma,
                         int64_t n_leaves, const int64_t* leaf_off, const double* leaf_c,
                         const double* leaf_rho, const int32_t* leaf_p, double* coef_single,
                         double* coef_double, int accumulate)
{
    return run_elements(plan, q2x::KIND_TRI, (int)density, n_elem, n_vert, vxyz, idx, sigma, n_leaves,
                        leaf_off, leaf_c, leaf_rho, leaf_p, coef_single, coef_double, accumulate);
}

q2x_status q2x_triangles_single(q2x_plan_t plan, int64_t n_elem, int64_t n_vert,
                                const double* vxyz, const int32_t* idx, q2x_density density,
                                const double* sigma, int64_t n_leaves, const int64_t* leaf_off,
                                const double* leaf_c, const double* leaf_rho,
                                const int32_t* leaf_p, double* coef, int accumulate)
{
    if (!coef) return fail(plan, Q2X_ERR_ARG, "coef is NULL");
    return run_elements(plan, q2x::KIND_TRI, (int)density, n_elem, n_vert, vxyz, idx, sigma, n_leaves,
                        leaf_off, leaf_c, leaf_rho, leaf_p, coef, nullptr, accumulate);
}

q2x_status q2x_triangles_double(q2x_plan_t plan, int64_t n_elem, int64_t n_vert,
                                const double* vxyz, const int32_t* idx, q2x_density density,
                                const double* sigma, int64_t n_leaves, const int64_t* leaf_off,
                                const double* leaf_c, const double* leaf_rho,
                                const int32_t* leaf_p, double* coef, int accumulate)
{
    if (!coef) return fail(plan, Q2X_ERR_ARG, "coef is NULL");
    return run_elements(plan, q2x::KIND_TRI, (int)density, n_elem, n_vert, vxyz, idx, sigma, n_leaves,
                        leaf_off, leaf_c, leaf_rho, leaf_p, nullptr, coef, accumulate);
}

q2x_status q2x_tetra(q2x_plan_t plan, int64_t n_elem, int64_t n_vert, const double* vxyz,
                     const int32_t* idx, const double* sigma, int64_t n_leaves,
                     const int64_t* leaf_off, const double* leaf_c, const double* leaf_rho,
                     const int32_t* leaf_p, double* coef, int accumulate)
{
    if (!coef) return fail(plan, Q2X_ERR_ARG, "coef is NULL");
    return run_elements(plan, q2x::KIND_TET, Q2X_DENSITY_CONST, n_elem, n_vert, vxyz, idx, sigma,
                        n_leaves, leaf_off, leaf_c, leaf_rho, leaf_p, coef, nullptr, accumulate);
}

q2x_status q2x_leaf_reduce(q2x_plan_t plan, int64_t n_elem, int p, const double* elem,
                           int64_t n_leaves, const int64_t* leaf_off, double* coef, int accumulate)
{
    if (!plan) return fail(nullptr, Q2X_ERR_ARG, "plan is NULL");
    if (p < 0 || p > plan->p_max) return fail(plan, Q2X_ERR_RANGE, "p %d outside 0..%d", p, plan->p_max);
    if (n_elem < 0 || n_leaves < 0) return fail(plan, Q2X_ERR_ARG, "negative size");
    if (!leaf_off || !coef || (n_elem > 0 && !elem)) return fail(plan, Q2X_ERR_ARG, "NULL pointer");
    if (accumulate != 0 && accumulate != 1) return fail(plan, Q2X_ERR_ARG, "accumulate must be 0 or 1");
    if (n_leaves == 0) return Q2X_OK;
    cudaError_t e = cudaSetDevice(plan->device);
    if (e != cudaSuccess) return cuda_fail(plan, e, "cudaSetDevice");
    const int np = (p + 1) * (p + 1);
    check_leaf_off_kernel<<<(unsigned)((n_leaves + 1 + 255) / 256), 256, 0, plan->stream>>>(leaf_off, n_leaves, n_elem,
                                                                                           plan->d_err);
    const int warps = 8;
    const int64_t units = n_leaves * (int64_t)np;  // (leaf, column) threads
    leaf_reduce_kernel<<<(unsigned)((units + warps * 32 - 1) / (warps * 32)), warps * 32, 0, plan->stream>>>(
        elem, np, n_elem, n_leaves, leaf_off, coef, accumulate);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(plan, e, "leaf_reduce launch");
    plan->launches += 2;
    return Q2X_OK;
}

q2x_status q2x_segments_vector(q2x_plan_t plan, int64_t n_elem, int64_t n_vert, const double* vxyz,
                               const int32_t* idx, const double* current, int64_t n_leaves,
                               const int64_t* leaf_off, const double* leaf_c, const double* leaf_rho,
                               const int32_t* leaf_p, double* coef3, int accumulate)
{
    if (!plan) return fail(nullptr, Q2X_ERR_ARG, "plan is NULL");
    if (n_elem < 0 || n_vert < 0 || n_leaves < 0) return fail(plan, Q2X_ERR_ARG, "negative size");
    if (accumulate != 0 && accumulate != 1) return fail(plan, Q2X_ERR_ARG, "accumulate must be 0 or 1");
    if (!leaf_off || !coef3) return fail(plan, Q2X_ERR_ARG, "leaf_off and coef3 must be non-NULL");
    if (n_elem > 0 && (!vxyz || !idx || !current || !leaf_c || n_vert <= 0 || n_leaves <= 0))
        return fail(plan, Q2X_ERR_ARG, "NULL array or empty mesh");
    if (n_elem > ((int64_t)1 << 40)) return fail(plan, Q2X_ERR_ARG, "n_elem too large");
    if (n_leaves == 0) return Q2X_OK;
    cudaError_t e = cudaSetDevice(plan->device);
    if (e != cudaSuccess) return cuda_fail(plan, e, "cudaSetDevice");
    const int np = (plan->p_max + 1) * (plan->p_max + 1);
    if (n_elem == 0) {
        if (!accumulate) {
            e = cudaMemsetAsync(coef3, 0, sizeof(double) * 3 * (size_t)n_leaves * np, plan->stream);
            if (e != cudaSuccess) return cuda_fail(plan, e, "cudaMemsetAsync");
        }
        return Q2X_OK;
    }
    // one pass over the segments: unit-density moments staged per round and
    // reduced three times, weighted by the components (element kernel, vector mode)
    const int64_t nl_np = n_leaves * (int64_t)np;
    return run_elements(plan, q2x::KIND_SEG, Q2X_DENSITY_CONST, n_elem, n_vert, vxyz, idx, nullptr, n_leaves, leaf_off,
                        leaf_c, leaf_rho, leaf_p, coef3, coef3 + nl_np, accumulate, current, coef3 + 2 * nl_np);
}

q2x_status q2x_leaf_reduce_weighted(q2x_plan_t plan, int64_t n_elem, int p, const double* elem, int n_w,
                                    const double* w, int64_t w_stride, int64_t n_leaves,
                                    const int64_t* leaf_off, double* coef, int64_t coef_stride,
                                    int accumulate)
{
    if (!plan) return fail(nullptr, Q2X_ERR_ARG, "plan is NULL");
    if (p < 0 || p > plan->p_max) return fail(plan, Q2X_ERR_RANGE, "p %d outside 0..%d", p, plan->p_max);
    if (n_w < 1 || n_w > 4) return fail(plan, Q2X_ERR_ARG, "n_w %d outside 1..4", n_w);
    if (n_elem < 0 || n_leaves < 0 || w_stride < 0 || coef_stride < 0) return fail(plan, Q2X_ERR_ARG, "negative size");
    if (!leaf_off || !coef || (n_elem > 0 && (!elem || !w))) return fail(plan, Q2X_ERR_ARG, "NULL pointer");
    if (accumulate != 0 && accumulate != 1) return fail(plan, Q2X_ERR_ARG, "accumulate must be 0 or 1");
    const int np = (p + 1) * (p + 1);
    if (n_w > 1 && (w_stride < n_elem || coef_stride < n_leaves * (int64_t)np))
        return fail(plan, Q2X_ERR_ARG, "component strides overlap");
    if (n_leaves == 0) return Q2X_OK;
    cudaError_t e = cudaSetDevice(plan->device);
    if (e != cudaSuccess) return cuda_fail(plan, e, "cudaSetDevice");
    check_leaf_off_kernel<<<(unsigned)((n_leaves + 1 + 255) / 256), 256, 0, plan->stream>>>(leaf_off, n_leaves, n_elem,
                                                                                           plan->d_err);
    const int warps = 8;
    const int64_t units = n_leaves * (int64_t)((np + 31) / 32);  // (leaf, 32-column group) warps
    const unsigned grid = (unsigned)((units + warps - 1) / warps);
    switch (n_w) {
        case 1:
            leaf_reduce_weighted_kernel<1><<<grid, warps * 32, 0, plan->stream>>>(
                elem, np, n_elem, w, w_stride, n_leaves, leaf_off, coef, coef_stride, accumulate);
            break;
        case 2:
            leaf_reduce_weighted_kernel<2><<<grid, warps * 32, 0, plan->stream>>>(
                elem, np, n_elem, w, w_stride, n_leaves, leaf_off, coef, coef_stride, accumulate);
            break;
        case 3:
            leaf_reduce_weighted_kernel<3><<<grid, warps * 32, 0, plan->stream>>>(
                elem, np, n_elem, w, w_stride, n_leaves, leaf_off, coef, coef_stride, accumulate);
            break;
        default:
            leaf_reduce_weighted_kernel<4><<<grid, warps * 32, 0, plan->stream>>>(
                elem, np, n_elem, w, w_stride, n_leaves, leaf_off, coef, coef_stride, accumulate);
            break;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(plan, e, "leaf_reduce_weighted launch");
    plan->launches += 2;
    return Q2X_OK;
}

}  // extern "C"
