// q2x_plan.h -- the plan object behind q2x_plan_t (internal to the library).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <utility>
#include <vector>

#include "q2x.h"

struct q2x_plan_s {
    int p_max = 0;
    int norm = 0;
    int prec = 0;  // 0 FP64, 1 FP32-mixed
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;
    unsigned* d_err = nullptr;
    unsigned* h_err = nullptr;  // pinned
    void* ws = nullptr;
    size_t ws_bytes = 0;
    int occ_cache[2][9][5] = {};  // [precision][element combo][capacity bin]
    int tile_occ[4][5] = {};  // resident CTAs per SM of the FP32 leaf-tile kernels [combo][bin]
    int timing = 0;
    std::vector<cudaEvent_t> ev_pool;                            // idle events
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending;  // recorded pairs
    int64_t launches = 0;
    std::string last_error;
};

// status helpers shared by the library's translation units
q2x_status q2x_fail(q2x_plan_t plan, q2x_status st, const char* fmt, ...);
q2x_status q2x_cuda_fail(q2x_plan_t plan, cudaError_t e, const char* what);
// grow the plan's device workspace to at least `bytes` (synchronises the
// plan's stream when it has to reallocate)
q2x_status q2x_plan_workspace(q2x_plan_t plan, size_t bytes);
