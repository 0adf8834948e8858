// q2x_noalloc.cu -- q2x_triangles_noalloc: the triangle Q2X call without any
// device allocation (declared in include/q2x.h).
//
// Some callers cannot call cudaMalloc: solvers that have already handed all
// device memory to their own pool, code paths that must never synchronise the
// device (cudaMalloc / cudaFree may do so), and callers that must not meet an
// out-of-memory failure at call time.  For them this entry point runs the same
// triangle element kernel and fix-up kernel as q2x_triangles, but keeps the
// kernel's scratch (the partial sums of leaves that straddle warp ranges) in a
// fixed file-scope __device__ array instead of a plan workspace.  It takes no
// plan and allocates nothing: no cudaMalloc, cudaFree or allocating library
// routine is called.
//
// Host code cannot use the array's symbol as a device address, so the first
// call on each device looks up the array's device address with
// cudaGetSymbolAddress (with that device current) and caches it; make that
// first call before any stream capture.
//
// Every call on a device shares the one array, which keeps the previous call's
// contents; the kernels write every scratch entry they read within a call, so
// nothing needs clearing.  Calls that overlap on the GPU (different streams,
// or host threads) race on the array and on the device error word.  Nothing
// here reads that word back: device-side input checks are not reported, and
// leaf_off is not checked on the device (the kernels still keep every access
// in bounds; a non-monotone or out-of-range leaf_off gives undefined
// coefficients).
#include <cuda_runtime.h>

#include <mutex>

#include "q2x.h"
#include "q2x_kernels.cuh"

#define Q2X_NA_DECLARE(T)                                                                          \
    Q2X_FOR_BINS(Q2X_DECLARE, T, q2x::KIND_TRI, q2x::DENS_CONST, 1)                                \
    Q2X_FOR_BINS(Q2X_DECLARE, T, q2x::KIND_TRI, q2x::DENS_CONST, 2)                                \
    Q2X_FOR_BINS(Q2X_DECLARE, T, q2x::KIND_TRI, q2x::DENS_CONST, 3)                                \
    Q2X_FOR_BINS(Q2X_DECLARE, T, q2x::KIND_TRI, q2x::DENS_LINEAR, 1)                               \
    Q2X_FOR_BINS(Q2X_DECLARE, T, q2x::KIND_TRI, q2x::DENS_LINEAR, 2)                               \
    Q2X_FOR_BINS(Q2X_DECLARE, T, q2x::KIND_TRI, q2x::DENS_LINEAR, 3)
Q2X_NA_DECLARE(float)
Q2X_NA_DECLARE(double)

namespace {

// Scratch of the no-allocation entry point: every GPU that loads the library
// holds these bytes until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[Q2X_NOALLOC_SCRATCH_BYTES];
static __device__ unsigned g_noalloc_err;

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {};
unsigned* g_err_ptr[kMaxDevices] = {};

using LaunchFn = cudaError_t (*)(const q2x::ElemArgs&, int, cudaStream_t);
#define Q2X_NA_ENTRY(T, P, KIND, DENS, OUTS) &q2x::launch_elem<T, P, KIND, DENS, OUTS>,
#define Q2X_NA_ROW(T, DENS, OUTS) {Q2X_FOR_BINS(Q2X_NA_ENTRY, T, q2x::KIND_TRI, DENS, OUTS)},
#define Q2X_NA_DENS(T, DENS) {Q2X_NA_ROW(T, DENS, 1) Q2X_NA_ROW(T, DENS, 2) Q2X_NA_ROW(T, DENS, 3)},
// [precision: 0 FP64, 1 FP32][density][layers - 1: single, double, both][bin 4, 8, 12, 16, 20]
const LaunchFn kTri[2][2][3][5] = {
    {Q2X_NA_DENS(double, q2x::DENS_CONST) Q2X_NA_DENS(double, q2x::DENS_LINEAR)},
    {Q2X_NA_DENS(float, q2x::DENS_CONST) Q2X_NA_DENS(float, q2x::DENS_LINEAR)},
};

// Device addresses of the scratch array and error word on the current device
// (looked up once per device).
q2x_status noalloc_setup(int dev, void** scratch, unsigned** err)
{
    if (dev < 0 || dev >= kMaxDevices) return Q2X_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* s = nullptr;
        void* e = nullptr;
        cudaError_t rc = cudaGetSymbolAddress(&s, g_noalloc_scratch);
        if (rc != cudaSuccess) {
            cudaGetLastError();
            return Q2X_ERR_CUDA;
        }
        rc = cudaGetSymbolAddress(&e, g_noalloc_err);
        if (rc != cudaSuccess) {
            cudaGetLastError();
            return Q2X_ERR_CUDA;
        }
        g_scratch_ptr[dev] = s;
        g_err_ptr[dev] = static_cast<unsigned*>(e);
    }
    *scratch = g_scratch_ptr[dev];
    *err = g_err_ptr[dev];
    return Q2X_OK;
}

}  // namespace

extern "C" q2x_status q2x_triangles_noalloc(int p_max, q2x_norm norm, q2x_precision precision,
                                            void* cuda_stream, int64_t n_elem, int64_t n_vert,
                                            const double* vxyz, const int32_t* idx,
                                            q2x_density density, const double* sigma,
                                            int64_t n_leaves, const int64_t* leaf_off,
                                            const double* leaf_c, const double* leaf_rho,
                                            const int32_t* leaf_p, double* coef_single,
                                            double* coef_double, int accumulate)
{
    if (p_max < 0 || p_max > Q2X_P_MAX) return Q2X_ERR_RANGE;
    if (norm != Q2X_NORM_COEFF && norm != Q2X_NORM_MOMENT) return Q2X_ERR_ARG;
    if (precision != Q2X_FP64 && precision != Q2X_FP32_MIXED) return Q2X_ERR_ARG;
    if (density != Q2X_DENSITY_CONST && density != Q2X_DENSITY_LINEAR) return Q2X_ERR_ARG;
    if (n_elem < 0 || n_vert < 0 || n_leaves < 0) return Q2X_ERR_ARG;
    if (!coef_single && !coef_double) return Q2X_ERR_ARG;
    if (accumulate != 0 && accumulate != 1) return Q2X_ERR_ARG;
    if (!leaf_off || !leaf_c) return Q2X_ERR_ARG;  // leaf mode only
    if (precision == Q2X_FP32_MIXED && !leaf_rho) return Q2X_ERR_ARG;
    if (n_elem > 0 && (!vxyz || !idx || !sigma || n_vert <= 0 || n_leaves <= 0)) return Q2X_ERR_ARG;

    const int prec = (precision == Q2X_FP32_MIXED) ? 1 : 0;
    const int64_t elt = (int64_t)sizeof(double);  // FP64 partial sums in both precisions
    const int np = (p_max + 1) * (p_max + 1);
    const int64_t T = Q2X_NOALLOC_RANGE;
    // size limit by division (no product that could wrap): each range needs
    // 4 np elt bytes of scratch
    const int64_t max_ranges = (int64_t)Q2X_NOALLOC_SCRATCH_BYTES / (4 * (int64_t)np * elt);
    if (n_elem > max_ranges * T) return Q2X_ERR_RANGE;
    const int64_t n_ranges = (n_elem + T - 1) / T;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return Q2X_ERR_CUDA;
    }
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    if (stream) {  // the scratch address is the current device's: the stream must be on it
        int sdev = -1;
        if (cudaStreamGetDevice(stream, &sdev) != cudaSuccess) {
            cudaGetLastError();
            return Q2X_ERR_ARG;
        }
        if (sdev != dev) return Q2X_ERR_ARG;
    }
    void* scratch = nullptr;
    unsigned* err = nullptr;
    q2x_status st = noalloc_setup(dev, &scratch, &err);
    if (st != Q2X_OK) return st;

    if (n_elem == 0) {
        if (!accumulate)
            for (double* c : {coef_single, coef_double})
                if (c && cudaMemsetAsync(c, 0, sizeof(double) * (size_t)n_leaves * np, stream) != cudaSuccess)
                    return Q2X_ERR_CUDA;
        return Q2X_OK;
    }

    int bin = -1;
    const int bins[5] = {4, 8, 12, 16, 20};
    for (int b = 0; b < 5 && bin < 0; ++b)
        if (p_max <= bins[b]) bin = b;

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
    a.p_max = p_max;
    a.np_max = np;
    a.coef[0] = coef_single;
    a.coef[1] = coef_double;
    a.coef[2] = nullptr;
    a.wvec = nullptr;
    a.nacc = q2x::elem_outputs(q2x::KIND_TRI, coef_double ? 2 : 1);
    a.accumulate = accumulate;
    a.norm = (int)norm;
    a.T = T;
    a.n_ranges = n_ranges;
    a.slots = static_cast<double*>(scratch);
    a.err = err;

    const int wpc = prec ? q2x::elem_warps_per_cta<float>() : q2x::elem_warps_per_cta<double>();
    const int grid = (int)((n_ranges + wpc - 1) / wpc);
    const int outs = (coef_single ? 1 : 0) | (coef_double ? 2 : 0);
    if (kTri[prec][density][outs - 1][bin](a, grid, stream) != cudaSuccess) return Q2X_ERR_CUDA;
    if (n_ranges > 1) {
        const int d_out = (density == Q2X_DENSITY_LINEAR) ? 3 : 2;
        if (q2x::launch_fixup(a, stream, d_out, d_out - 1, d_out, 2, 1, 2) != cudaSuccess) return Q2X_ERR_CUDA;
    }
    return Q2X_OK;
}
