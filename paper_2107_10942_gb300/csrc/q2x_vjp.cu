// q2x_vjp.cu -- q2x_triangles_single_vjp (include/q2x.h): the adjoint kernels
// of q2x_vjp.cuh and their dispatch.
#include <cuda_runtime.h>

#include <algorithm>

#include "q2x.h"
#include "q2x_plan.h"
#include "q2x_vjp.cuh"

namespace {

template <typename T, int P>
cudaError_t launch_vjp(const q2x::VjpArgs& a, cudaStream_t st)
{
    const int threads = 128;
    const unsigned grid = (unsigned)((a.n_elem + threads - 1) / threads);
    q2x::q2x_tri_vjp_kernel<T, P><<<grid, threads, 0, st>>>(a);
    return cudaGetLastError();
}

using VjpFn = cudaError_t (*)(const q2x::VjpArgs&, cudaStream_t);
// [precision: 0 FP64, 1 FP32][bin 4, 8, 12, 16, 20]
const VjpFn kVjp[2][5] = {
    {&launch_vjp<double, 4>, &launch_vjp<double, 8>, &launch_vjp<double, 12>, &launch_vjp<double, 16>,
     &launch_vjp<double, 20>},
    {&launch_vjp<float, 4>, &launch_vjp<float, 8>, &launch_vjp<float, 12>, &launch_vjp<float, 16>,
     &launch_vjp<float, 20>},
};

}  // namespace

extern "C" q2x_status q2x_triangles_single_vjp(q2x_plan_t plan, int64_t n_elem, int64_t n_vert,
                                               const double* vxyz, const int32_t* idx, const double* sigma,
                                               int64_t n_leaves, const int64_t* leaf_off, const double* leaf_c,
                                               const double* leaf_rho, const int32_t* leaf_p,
                                               const double* grad_coef, double* grad_vxyz, double* grad_sigma)
{
    if (!plan) return q2x_fail(nullptr, Q2X_ERR_ARG, "plan is NULL");
    if (n_elem < 0 || n_vert < 0 || n_leaves < 0) return q2x_fail(plan, Q2X_ERR_ARG, "vjp: negative size");
    if (!leaf_off && n_leaves != n_elem)
        return q2x_fail(plan, Q2X_ERR_ARG, "vjp: per-element mode needs n_leaves == n_elem");
    if (n_elem == 0) return Q2X_OK;
    if (!vxyz || !idx || !sigma || !leaf_c || !grad_coef || !grad_vxyz || n_vert <= 0 || n_leaves <= 0)
        return q2x_fail(plan, Q2X_ERR_ARG, "vjp: NULL array or empty mesh");
    cudaError_t e = cudaSetDevice(plan->device);
    if (e != cudaSuccess) return q2x_cuda_fail(plan, e, "cudaSetDevice");
    const int prec = plan->prec;
    const int np = (plan->p_max + 1) * (plan->p_max + 1);
    const int bins[5] = {4, 8, 12, 16, 20};
    int bin = 0;
    while (bins[bin] < plan->p_max) ++bin;
    // workspace: the per-leaf weights (grows the plan's buffer if needed)
    const size_t bytes = (prec ? sizeof(float) : sizeof(double)) * (size_t)n_leaves * np;
    q2x_status st = q2x_plan_workspace(plan, bytes);
    if (st != Q2X_OK) return st;
    const int64_t nw = n_leaves * np;
    const unsigned wgrid = (unsigned)((nw + 255) / 256);
    if (prec)
        q2x::q2x_vjp_weights<float><<<wgrid, 256, 0, plan->stream>>>(grad_coef, leaf_rho, leaf_p, n_leaves, np,
                                                                    plan->p_max, plan->norm,
                                                                    static_cast<float*>(plan->ws));
    else
        q2x::q2x_vjp_weights<double><<<wgrid, 256, 0, plan->stream>>>(grad_coef, leaf_rho, leaf_p, n_leaves, np,
                                                                     plan->p_max, plan->norm,
                                                                     static_cast<double*>(plan->ws));
    e = cudaGetLastError();
    if (e != cudaSuccess) return q2x_cuda_fail(plan, e, "vjp: weights launch");
    q2x::VjpArgs a;
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
    a.norm = plan->norm;
    a.w = plan->ws;
    a.grad_v = grad_vxyz;
    a.grad_sigma = grad_sigma;
    a.err = plan->d_err;
    e = kVjp[prec][bin](a, plan->stream);
    if (e != cudaSuccess) return q2x_cuda_fail(plan, e, "vjp: kernel launch");
    plan->launches += 2;
    return Q2X_OK;
}
