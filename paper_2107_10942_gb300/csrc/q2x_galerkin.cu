// q2x_galerkin.cu -- receiver-side (Galerkin) integration of local
// expansions over triangles: for every triangle e in leaf L,
//   out[e] = sum_c w[L][c] P_c(e),
// P(e) the packed coefficients of triangle e alone (single or double layer,
// density sigma_e, the plan's norm; Eq. (bas4)/(bas10)) and w a packed weight
// row per leaf.  With the MOMENT norm and w built from a local expansion
// phi(y) = sum L_n^m R_n^m(y - c) (w = L_n^0 at (n,0); 2 Re L_n^m at (n,m);
// -2 Im L_n^m at (n,-m)), out[e] is the integral of sigma_e phi over the
// triangle (single layer) or of sigma_e n.grad phi (double layer) -- the
// receiving side of a Galerkin boundary-element FMM.
//
// The per-element moments come from the same recursion chain as the Q2X
// element kernel (Lemmas 2-3, Eqs. (rec10)-(rec15)); instead of the leaf sum,
// each lane contracts its own element's staged row with the leaf's weights,
// which a first kernel folds together with the per-column finish constants
// (1/(n+d)!, the packing sign, 1/4pi, the leaf's power-of-two scale).  FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "q2x.h"
#include "q2x_kernels.cuh"
#include "q2x_plan.h"

namespace q2x {

struct GalArgs {
    int64_t n_elem, n_vert;
    const double* vx;
    const double* vy;
    const double* vz;
    const int32_t* idx;
    const double* sigma;      // n_elem weights of the elements' test functions
    int64_t n_leaves;
    const int64_t* leaf_off;  // CSR over the elements
    const double* leaf_c;
    const double* leaf_rho;
    int p, np;
    const double* wf;         // [n_leaves][np] folded weights
    double* out;
    unsigned* err;
};

// wf[L][c] = w[L][c] * finish constant of column c for leaf L
__global__ void q2x_galerkin_weights(const double* __restrict__ w, const double* __restrict__ leaf_rho,
                                     int64_t n_leaves, int np, int norm, int d, int shift_n0, double* wf)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_leaves * np) return;
    const int64_t L = i / np;
    const int c = (int)(i - L * np);
    const int s = leaf_rho ? scale_exponent(__ldg(leaf_rho + L)) : 0;
    wf[i] = __ldg(w + i) * finish_desc(1.0, norm, col_desc(c), d, shift_n0, s);
}

template <int P, int OUTS>
__global__ void __launch_bounds__(WARPS_PER_CTA * 32, 2) q2x_galerkin_kernel(const GalArgs a)
{
    constexpr int CH = KCfg<double>::CHUNK, LD = KCfg<double>::LD;
    constexpr int LY = (OUTS == 2) ? 1 : 0;  // staged layer read back
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    double* tile = reinterpret_cast<double*>(smem_raw + (size_t)wib * warp_smem_bytes<double>(a.np));
    const int64_t gw = (int64_t)blockIdx.x * WARPS_PER_CTA + wib;
    const int64_t nw = (int64_t)gridDim.x * WARPS_PER_CTA;
#pragma unroll 1
    for (int64_t e0 = gw * 32; e0 < a.n_elem; e0 += nw * 32) {
        const int64_t e = e0 + lane;
        const bool active = e < a.n_elem;
        int64_t L = 0;
        unsigned errbits = 0;
        double cx = 0.0, cy = 0.0, cz = 0.0;
        int sexp = 0;
        if (active) {
            L = leaf_search(a.leaf_off, 0, a.n_leaves - 1, e);
            cx = __ldg(a.leaf_c + L);
            cy = __ldg(a.leaf_c + a.n_leaves + L);
            cz = __ldg(a.leaf_c + 2 * a.n_leaves + L);
            if (!(finite_bits(cx) && finite_bits(cy) && finite_bits(cz))) errbits |= 2u;
            sexp = a.leaf_rho ? scale_exponent(__ldg(a.leaf_rho + L)) : 0;
        }
        int pl = a.p;
        Frame<double, 3> F;
        // sigma (the test function's weight) rides in the frame's seed
        load_frame<double, KIND_TRI, DENS_CONST>(a.vx, a.vy, a.vz, a.idx, a.sigma, a.n_elem, a.n_vert, e, active,
                                                 cx, cy, cz, sexp, errbits, pl, F);
        if (errbits) atomicOr(a.err, errbits);
        const double* wrow = a.wf + L * (int64_t)a.np;
        double acc = 0.0;
        run_chain<double, P, KIND_TRI, DENS_CONST, OUTS>(F, a.p, tile, lane, [&](int c0, int ncols) {
            if (active)
                for (int j = 0; j < ncols; ++j) acc = fma(tile[(LY * CH + j) * LD + lane], __ldg(wrow + c0 + j), acc);
        });
        if (active) a.out[e] = acc;
    }
}

template <int P, int OUTS>
cudaError_t launch_galerkin(const GalArgs& a, int num_sms, cudaStream_t st)
{
    auto k = q2x_galerkin_kernel<P, OUTS>;
    const size_t smem = WARPS_PER_CTA * warp_smem_bytes<double>(a.np);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, WARPS_PER_CTA * 32, smem);
    if (e != cudaSuccess) return e;
    const int64_t need = (a.n_elem + 32 * WARPS_PER_CTA - 1) / (32 * WARPS_PER_CTA);
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)std::max(per_sm, 1) * num_sms));
    k<<<(unsigned)grid, WARPS_PER_CTA * 32, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace q2x

extern "C" q2x_status q2x_galerkin_triangles(q2x_plan_t plan, int64_t n_elem, int64_t n_vert, const double* vxyz,
                                             const int32_t* idx, const double* sigma, int64_t n_leaves,
                                             const int64_t* leaf_off, const double* leaf_c,
                                             const double* leaf_rho, int layer, const double* w, double* out)
{
    if (!plan) return q2x_fail(nullptr, Q2X_ERR_ARG, "plan is NULL");
    if (n_elem < 0 || n_vert < 0 || n_leaves < 0) return q2x_fail(plan, Q2X_ERR_ARG, "negative size");
    if (layer != 0 && layer != 1) return q2x_fail(plan, Q2X_ERR_ARG, "layer must be 0 (single) or 1 (double)");
    if (n_elem == 0) return Q2X_OK;
    if (!vxyz || !idx || !sigma || !leaf_off || !leaf_c || !w || !out || n_vert <= 0 || n_leaves <= 0)
        return q2x_fail(plan, Q2X_ERR_ARG, "NULL array or empty mesh");
    if (n_elem > ((int64_t)1 << 40)) return q2x_fail(plan, Q2X_ERR_ARG, "n_elem too large");
    cudaError_t e = cudaSetDevice(plan->device);
    if (e != cudaSuccess) return q2x_cuda_fail(plan, e, "cudaSetDevice");
    const int p = plan->p_max;
    const int np = (p + 1) * (p + 1);
    q2x_status st = q2x_plan_workspace(plan, sizeof(double) * (size_t)n_leaves * np);
    if (st != Q2X_OK) return st;
    double* wf = static_cast<double*>(plan->ws);
    using C = q2x::Chain<q2x::KIND_TRI, q2x::DENS_CONST>;
    const int d = layer ? C::D_OUT - 1 : C::D_OUT;
    const int shift_n0 = layer ? 1 : q2x::KIND_TRI + 1;
    const int64_t nw = n_leaves * np;
    q2x::q2x_galerkin_weights<<<(unsigned)((nw + 255) / 256), 256, 0, plan->stream>>>(w, leaf_rho, n_leaves, np,
                                                                                     plan->norm, d, shift_n0, wf);
    e = cudaGetLastError();
    if (e != cudaSuccess) return q2x_cuda_fail(plan, e, "galerkin weights launch");
    q2x::GalArgs a;
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
    a.p = p;
    a.np = np;
    a.wf = wf;
    a.out = out;
    a.err = plan->d_err;
    const int bins[5] = {4, 8, 12, 16, 20};
    int bin = 0;
    while (bins[bin] < p) ++bin;
#define Q2X_GAL_CASE(B, PP)                                                                           \
    case B:                                                                                           \
        e = layer ? q2x::launch_galerkin<PP, 2>(a, plan->num_sms, plan->stream)                       \
                  : q2x::launch_galerkin<PP, 1>(a, plan->num_sms, plan->stream);                      \
        break;
    switch (bin) {
        Q2X_GAL_CASE(0, 4)
        Q2X_GAL_CASE(1, 8)
        Q2X_GAL_CASE(2, 12)
        Q2X_GAL_CASE(3, 16)
        Q2X_GAL_CASE(4, 20)
    }
#undef Q2X_GAL_CASE
    if (e != cudaSuccess) return q2x_cuda_fail(plan, e, "galerkin kernel launch");
    plan->launches += 2;
    return Q2X_OK;
}
