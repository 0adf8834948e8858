// q2x_batch_api.cu -- ragged mixed batch (include/q2x.h): tile list and its
// groups, graph capture of the groups' persistent kernels and the per-leaf
// combine, autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "q2x.h"
#include "q2x_batch.cuh"
#include "q2x_plan.h"

namespace q2x {

__global__ void q2x_batch_combine(const double* __restrict__ partial, const int64_t* __restrict__ slot_off,
                                  int np, int64_t n_leaves, double* coef, int accumulate)
{
    const int lane = threadIdx.x & 31;
    const int64_t L = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (L >= n_leaves) return;
    const int64_t s0 = slot_off[L], s1 = slot_off[L + 1];
    for (int c = lane; c < np; c += 32) {
        double acc = 0.0;
        for (int64_t s = s0; s < s1; ++s) acc += partial[s * np + c];
        double* d = coef + L * np + c;
        *d = accumulate ? *d + acc : acc;
    }
}
}  // namespace q2x

struct q2x_batch_s {
    q2x_plan_t plan = nullptr;
    int prec = 0;
    int tile_elems = 0;
    q2x::BatchArgs args{};
    q2x::BatchTile* d_tiles = nullptr;
    int64_t* d_slot_off = nullptr;
    double* d_partial = nullptr;
    unsigned long long* d_counter = nullptr;  // one per group
    int64_t n_tiles = 0, n_slots = 0, n_leaves = 0;
    double* coef = nullptr;
    int accumulate = 0;
    int n_groups = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

constexpr int kBins[5] = {4, 8, 12, 16, 20};

void free_batch(q2x_batch_s* b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->d_tiles) cudaFree(b->d_tiles);
    if (b->d_slot_off) cudaFree(b->d_slot_off);
    if (b->d_partial) cudaFree(b->d_partial);
    if (b->d_counter) cudaFree(b->d_counter);
    delete b;
}

q2x_status check_kind(q2x_plan_t plan, const q2x_batch_elements& k, int kind, int64_t n_leaves,
                      std::vector<int64_t>& off)
{
    if (k.n_elem < 0 || k.n_vert < 0) return q2x_fail(plan, Q2X_ERR_ARG, "batch: negative size (kind %d)", kind);
    if (k.n_elem == 0) return Q2X_OK;
    if (!k.vxyz || !k.idx || !k.sigma || !k.leaf_off || k.n_vert <= 0)
        return q2x_fail(plan, Q2X_ERR_ARG, "batch: kind %d has NULL arrays or no vertices", kind);
    if (kind == 1 && k.density != Q2X_DENSITY_CONST && k.density != Q2X_DENSITY_LINEAR)
        return q2x_fail(plan, Q2X_ERR_ARG, "batch: bad triangle density");
    off.resize(n_leaves + 1);
    cudaError_t e = cudaMemcpy(off.data(), k.leaf_off, sizeof(int64_t) * (n_leaves + 1), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return q2x_cuda_fail(plan, e, "batch: reading leaf_off");
    if (off[0] != 0 || off[n_leaves] != k.n_elem)
        return q2x_fail(plan, Q2X_ERR_ARG, "batch: leaf_off of kind %d must run from 0 to n_elem", kind);
    for (int64_t L = 0; L < n_leaves; ++L)
        if (off[L + 1] < off[L]) return q2x_fail(plan, Q2X_ERR_ARG, "batch: leaf_off of kind %d decreases", kind);
    return Q2X_OK;
}

q2x_status build_batch(q2x_plan_t plan, const q2x_batch_desc* d, int tile_elems, q2x_batch_s** out)
{
    *out = nullptr;
    if (!plan || !d) return q2x_fail(plan, Q2X_ERR_ARG, "batch: NULL plan or descriptor");
    if (d->n_leaves <= 0 || d->n_leaves >= ((int64_t)1 << 31) || !d->leaf_c || !d->coef)
        return q2x_fail(plan, Q2X_ERR_ARG, "batch: need 0 < n_leaves < 2^31, leaf_c and coef");
    if (plan->prec == 1 && !d->leaf_rho) return q2x_fail(plan, Q2X_ERR_ARG, "batch: FP32-mixed needs leaf_rho");
    if (d->accumulate != 0 && d->accumulate != 1) return q2x_fail(plan, Q2X_ERR_ARG, "batch: accumulate must be 0 or 1");
    if (tile_elems <= 0) tile_elems = 256;
    cudaError_t e = cudaSetDevice(plan->device);
    if (e != cudaSuccess) return q2x_cuda_fail(plan, e, "cudaSetDevice");
    const int64_t nl = d->n_leaves;
    const q2x_batch_elements* kinds[3] = {&d->segments, &d->triangles, &d->tetra};
    std::vector<int64_t> off[3];
    for (int k = 0; k < 3; ++k) {
        q2x_status st = check_kind(plan, *kinds[k], k, nl, off[k]);
        if (st != Q2X_OK) return st;
    }
    std::vector<int32_t> lp(nl, plan->p_max);
    if (d->leaf_p) {
        e = cudaMemcpy(lp.data(), d->leaf_p, sizeof(int32_t) * nl, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return q2x_cuda_fail(plan, e, "batch: reading leaf_p");
    }
    // ---- tiles, slots numbered leaf by leaf
    std::vector<q2x::BatchTile> tiles;
    std::vector<int64_t> slot_off(nl + 1, 0);
    std::vector<double> cost;
    int64_t slot = 0;
    for (int64_t L = 0; L < nl; ++L) {
        slot_off[L] = slot;
        const int p = lp[L];
        if (p < 0 || p > plan->p_max) return q2x_fail(plan, Q2X_ERR_RANGE, "batch: leaf_p[%lld] = %d", (long long)L, p);
        int bin = 0;
        while (kBins[bin] < p) ++bin;
        for (int k = 0; k < 3; ++k) {
            if (kinds[k]->n_elem == 0) continue;
            const int64_t e0 = off[k][L], e1 = off[k][L + 1];
            if (e1 <= e0) continue;
            const int64_t n = e1 - e0;
            const int64_t nt = (n + tile_elems - 1) / tile_elems;
            const int64_t chunk = (n + nt - 1) / nt;
            const int combo = (k == 0) ? 0 : (k == 2) ? 3 : (kinds[1]->density == Q2X_DENSITY_LINEAR ? 2 : 1);
            const int levels = (combo == 0) ? 2 : (combo == 1) ? 3 : (combo == 2) ? 5 : 4;
            for (int64_t a = e0; a < e1; a += chunk) {
                q2x::BatchTile t{};
                t.combo = combo;
                t.bin = bin;
                t.leaf = (int32_t)L;
                t.slot = slot++;
                t.e_lo = a;
                t.e_hi = std::min(e1, a + chunk);
                tiles.push_back(t);
                cost.push_back((double)(t.e_hi - t.e_lo) * levels * (p + 1) * (p + 2) / 2.0);
            }
        }
    }
    slot_off[nl] = slot;
    // execution order: degree bin (high first), kind, then cost (high first)
    std::vector<int64_t> ord(tiles.size());
    for (size_t i = 0; i < ord.size(); ++i) ord[i] = (int64_t)i;
    std::stable_sort(ord.begin(), ord.end(), [&](int64_t x, int64_t y) {
        if (tiles[x].bin != tiles[y].bin) return tiles[x].bin > tiles[y].bin;
        if (tiles[x].combo != tiles[y].combo) return tiles[x].combo < tiles[y].combo;
        return cost[x] > cost[y];
    });
    std::vector<q2x::BatchTile> sorted(tiles.size());
    for (size_t i = 0; i < ord.size(); ++i) sorted[i] = tiles[ord[i]];
    // groups: runs of one (kind, bin) in that order, one persistent kernel each
    struct Group {
        int combo, bin;
        int64_t t0, t1;
        int grid;
    };
    std::vector<Group> groups;
    for (int64_t i = 0; i < (int64_t)sorted.size(); ++i) {
        if (groups.empty() || groups.back().combo != sorted[i].combo || groups.back().bin != sorted[i].bin)
            groups.push_back(Group{sorted[i].combo, sorted[i].bin, i, i + 1, 0});
        else
            groups.back().t1 = i + 1;
    }

    q2x_batch_s* b = new q2x_batch_s();
    b->plan = plan;
    b->prec = plan->prec;
    b->tile_elems = tile_elems;
    b->n_tiles = (int64_t)sorted.size();
    b->n_slots = slot;
    b->n_leaves = nl;
    b->coef = d->coef;
    b->accumulate = d->accumulate;
    const int np = (plan->p_max + 1) * (plan->p_max + 1);
    bool ok = true;
    ok = ok && cudaMalloc(&b->d_tiles, sizeof(q2x::BatchTile) * std::max<int64_t>(1, b->n_tiles)) == cudaSuccess;
    ok = ok && cudaMalloc(&b->d_slot_off, sizeof(int64_t) * (nl + 1)) == cudaSuccess;
    ok = ok && cudaMalloc(&b->d_partial, sizeof(double) * std::max<int64_t>(1, slot) * np) == cudaSuccess;
    ok = ok && cudaMalloc(&b->d_counter, sizeof(unsigned long long) * std::max<size_t>(1, groups.size())) ==
                   cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_batch(b);
        return q2x_fail(plan, Q2X_ERR_OOM, "batch: device allocation failed");
    }
    if (b->n_tiles)
        e = cudaMemcpy(b->d_tiles, sorted.data(), sizeof(q2x::BatchTile) * b->n_tiles, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_slot_off, slot_off.data(), sizeof(int64_t) * (nl + 1), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_batch(b);
        return q2x_cuda_fail(plan, e, "batch: uploading the tile list");
    }
    q2x::BatchArgs& a = b->args;
    for (int k = 0; k < 3; ++k) {
        const q2x_batch_elements& K = *kinds[k];
        a.kind[k].n_elem = K.n_elem;
        a.kind[k].n_vert = K.n_vert;
        a.kind[k].vx = K.vxyz;
        a.kind[k].vy = K.vxyz ? K.vxyz + K.n_vert : nullptr;
        a.kind[k].vz = K.vxyz ? K.vxyz + 2 * K.n_vert : nullptr;
        a.kind[k].idx = K.idx;
        a.kind[k].sigma = K.sigma;
    }
    a.n_leaves = nl;
    a.leaf_c = d->leaf_c;
    a.leaf_rho = d->leaf_rho;
    a.leaf_p = d->leaf_p;
    a.p_max = plan->p_max;
    a.np_max = np;
    a.norm = plan->norm;
    a.tiles = b->d_tiles;
    a.n_tiles = b->n_tiles;
    a.counter = b->d_counter;
    a.partial = b->d_partial;
    a.err = plan->d_err;
    a.coef = b->coef;  // unused here: every tile has a partial row (flags 0)
    a.accumulate = b->accumulate;
    a.n_tiles_dev = nullptr;
    const q2x::BatchGroupFns* fns = b->prec ? q2x::batch_group_table_f32() : q2x::batch_group_table_f64();
    for (Group& gr : groups) {
        const q2x::BatchGroupFns& f = fns[gr.combo * 5 + gr.bin];
        int occ = 0;
        e = f.occupancy(&occ);
        if (e != cudaSuccess || occ <= 0) {
            free_batch(b);
            return q2x_fail(plan, Q2X_ERR_CUDA, "batch: group kernel does not fit (smem %zu, %s)", f.smem,
                            cudaGetErrorString(e));
        }
        const int64_t want = (gr.t1 - gr.t0 + q2x::BATCH_WARPS - 1) / q2x::BATCH_WARPS;
        gr.grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)occ * plan->num_sms, want));
    }
    b->n_groups = (int)groups.size();

    // ---- capture [reset, the groups' persistent kernels on parallel
    // branches (groups dealt round-robin in execution order), combine]
    constexpr int kBranches = 4;
    const int nbr = std::min<int>(kBranches, (int)groups.size());
    cudaStream_t cs = nullptr, br[kBranches] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[kBranches] = {};
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    for (int i = 0; i < nbr && e == cudaSuccess; ++i) e = cudaStreamCreateWithFlags(&br[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming);
    for (int i = 0; i < nbr && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ev_join[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned long long) * std::max<size_t>(1, groups.size()), cs);
    if (e == cudaSuccess && nbr > 0) {
        e = cudaEventRecord(ev_fork, cs);
        for (int i = 0; i < nbr && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(br[i], ev_fork, 0);
        for (size_t g = 0; g < groups.size() && e == cudaSuccess; ++g) {
            const Group& gr = groups[g];
            e = fns[gr.combo * 5 + gr.bin].launch(a, gr.t0, gr.t1, (int)g, gr.grid, br[g % nbr]);
        }
        for (int i = 0; i < nbr && e == cudaSuccess; ++i) e = cudaEventRecord(ev_join[i], br[i]);
        for (int i = 0; i < nbr && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(cs, ev_join[i], 0);
    }
    if (e == cudaSuccess) {
        const int warps = 8;
        q2x::q2x_batch_combine<<<(unsigned)((nl + warps - 1) / warps), warps * 32, 0, cs>>>(
            b->d_partial, b->d_slot_off, np, nl, b->coef, b->accumulate);
        e = cudaGetLastError();
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cs ? cudaStreamEndCapture(cs, &g) : cudaSuccess;
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) {
        b->graph = g;
        e = cudaGraphInstantiate(&b->exec, g, 0);
    } else if (g) {
        cudaGraphDestroy(g);
    }
    if (cs) cudaStreamDestroy(cs);
    for (int i = 0; i < nbr; ++i) {
        if (br[i]) cudaStreamDestroy(br[i]);
        if (ev_join[i]) cudaEventDestroy(ev_join[i]);
    }
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_batch(b);
        return q2x_cuda_fail(plan, e, "batch: graph capture");
    }
    *out = b;
    return Q2X_OK;
}

}  // namespace

extern "C" {

q2x_status q2x_batch_build(q2x_plan_t plan, const q2x_batch_desc* desc, int tile_elems, q2x_batch_t* out)
{
    if (!out) return q2x_fail(plan, Q2X_ERR_ARG, "batch: out is NULL");
    return build_batch(plan, desc, tile_elems, out);
}

q2x_status q2x_batch_run(q2x_batch_t b)
{
    if (!b) return Q2X_ERR_ARG;
    cudaSetDevice(b->plan->device);
    cudaError_t e = cudaGraphLaunch(b->exec, b->plan->stream);
    if (e != cudaSuccess) return q2x_cuda_fail(b->plan, e, "batch: cudaGraphLaunch");
    b->plan->launches += b->n_groups + 1;
    return Q2X_OK;
}

q2x_status q2x_batch_destroy(q2x_batch_t b)
{
    if (!b) return Q2X_ERR_ARG;
    cudaSetDevice(b->plan->device);
    cudaStreamSynchronize(b->plan->stream);
    free_batch(b);
    return Q2X_OK;
}

q2x_status q2x_batch_info(q2x_batch_t b, int64_t* n_tiles, int64_t* n_slots, int* tile_elems)
{
    if (!b) return Q2X_ERR_ARG;
    if (n_tiles) *n_tiles = b->n_tiles;
    if (n_slots) *n_slots = b->n_slots;
    if (tile_elems) *tile_elems = b->tile_elems;
    return Q2X_OK;
}

q2x_status q2x_batch_tune(q2x_plan_t plan, const q2x_batch_desc* desc, const int* candidates, int n_candidates,
                          int reps, int* best, float* ms)
{
    if (!plan || !desc || !candidates || n_candidates <= 0 || !best || reps <= 0)
        return q2x_fail(plan, Q2X_ERR_ARG, "batch_tune: bad arguments");
    cudaSetDevice(plan->device);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return q2x_fail(plan, Q2X_ERR_CUDA, "batch_tune: cudaEventCreate");
    float best_ms = 1e30f;
    *best = candidates[0];
    q2x_status st = Q2X_OK;
    for (int i = 0; i < n_candidates && st == Q2X_OK; ++i) {
        q2x_batch_s* b = nullptr;
        st = build_batch(plan, desc, candidates[i], &b);
        if (st != Q2X_OK) break;
        cudaGraphLaunch(b->exec, plan->stream);  // warm-up
        cudaEventRecord(e0, plan->stream);
        for (int r = 0; r < reps; ++r) cudaGraphLaunch(b->exec, plan->stream);
        cudaEventRecord(e1, plan->stream);
        cudaError_t e = cudaEventSynchronize(e1);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        free_batch(b);
        if (e != cudaSuccess) {
            st = q2x_cuda_fail(plan, e, "batch_tune: timing");
            break;
        }
        t /= (float)reps;
        if (ms) ms[i] = t;
        if (t < best_ms) {
            best_ms = t;
            *best = candidates[i];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

}  // extern "C"
