// q2x_nearfield.cu -- exact potentials of constant-density elements at
// target points (the near field next to the expansions; Sec. 4.1's closed
// forms as a kernel):
//   segment:      int 1/|r - y| dl = log((R_b + s_b) / (R_a + s_a))     (Eqs. (num1)-(num3))
//   triangle:     int 1/|r - y| dS = sum_edges t_i log((R+ + s+)/(R- + s-)) - |h| Omega'
//   triangle, double layer: int n.(r - y)/|r - y|^3 dS = sign(h) Omega'  (signed solid angle)
//   tetrahedron:  int 1/|r - y| dV = -1/2 sum_faces h_j int_face 1/|r - y| dS  (Eqs. (num7)-(num8))
// with, per triangle edge i (vertices in order, n = (x2-x1)x(x3-x1)/J, m_i
// the outward in-plane edge normal, r0 the projection of r on the plane,
// h = n.(r - x1)): s-/s+ the edge coordinates of the edge's ends seen from
// r0, t_i = (a_i - r0).m_i, R-/R+ the distances from r to the ends and
//   Omega' = sum_i [atan(t_i s+ / (t_i^2 + h^2 + |h| R+)) - atan(t_i s- / (t_i^2 + h^2 + |h| R-))].
// Each contribution is multiplied by sigma_e / (4 pi) (the Green's function
// of Eq. (bas3)).  The logarithms form each factor R + s as d0^2 / (R - s)
// where s < 0, away from cancellation; heights and in-plane distances at the
// rounding level of their own computation count as zero.  One thread per
// target, looping over the target's element list.  FP64.
#include <cuda_runtime.h>

#include <cstdint>

#include "q2x.h"
#include "q2x_plan.h"

namespace q2x {

constexpr double NF_INV_4PI = 0.079577471545947667884;
constexpr double NF_SNAP = 16.0 * 2.220446049250313e-16;  // 16 units of FP64 rounding

struct NearArgs {
    int kind, layer, accumulate;
    int64_t n_elem, n_vert, n_tgt;
    const double* vx;
    const double* vy;
    const double* vz;
    const int32_t* idx;
    const double* sigma;
    const double* tgt;
    const int64_t* tgt_off;
    const int64_t* elem_idx;
    double* out;
    unsigned* err;
};

struct V3 {
    double x, y, z;
};
__device__ __forceinline__ V3 sub(V3 a, V3 b) { return V3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross(V3 a, V3 b)
{
    return V3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ V3 scale(V3 a, double s) { return V3{a.x * s, a.y * s, a.z * s}; }

// log((R+ + s+) / (R- + s-)) for a line piece whose ends sit at edge
// coordinates s- < s+ from the foot of the perpendicular, at distances R-,
// R+ from the target, d02 the squared distance to the line.  Since
// (R + s)(R - s) = d02 at both ends, the same value is log((R- - s-) /
// (R+ - s+)); each factor is formed without cancellation: R + s directly for
// s >= 0, as d02 / (R - s) for s < 0 (and mirrored for the second form,
// used when the piece lies mostly behind the foot).
__device__ __forceinline__ double line_log(double sm, double sp, double Rm, double Rp, double d02)
{
    if (sm + sp >= 0.0) {
        const double den = (sm >= 0.0) ? Rm + sm : d02 / (Rm - sm);
        return log((Rp + sp) / den);
    }
    const double den = (sp <= 0.0) ? Rp - sp : d02 / (Rp + sp);
    return log((Rm - sm) / den);
}

// int 1/|r - y| dS over the triangle (x1, x2, x3) and the signed solid angle
__device__ void tri_potential(V3 x1, V3 x2, V3 x3, V3 r, double& single, double& solid)
{
    const V3 nr = cross(sub(x2, x1), sub(x3, x1));
    const double J = sqrt(dot(nr, nr));
    single = solid = 0.0;
    if (!(J > 0.0)) return;
    const V3 n = scale(nr, 1.0 / J);
    const V3 dr = sub(r, x1);
    double h = dot(n, dr);
    // a height at the rounding level of its own computation is taken as zero:
    // the target is in the plane, where the double layer has the direct value 0
    if (fabs(h) <= NF_SNAP * sqrt(dot(dr, dr))) h = 0.0;
    const double ah = fabs(h);
    const V3 r0 = sub(r, scale(n, h));
    double S = 0.0, Om = 0.0;
    const V3 ends[4] = {x1, x2, x3, x1};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const V3 a = ends[i], b = ends[i + 1];
        const V3 e = sub(b, a);
        const double L = sqrt(dot(e, e));
        if (!(L > 0.0)) continue;
        const V3 l = scale(e, 1.0 / L);
        const V3 m = cross(l, n);
        const V3 ar = sub(a, r0);
        const double sm = dot(ar, l), sp = dot(sub(b, r0), l);
        double t = dot(ar, m);
        if (fabs(t) <= NF_SNAP * sqrt(dot(ar, ar))) t = 0.0;  // target on the edge's line
        const double d02 = t * t + h * h;
        const double Rm = sqrt(d02 + sm * sm), Rp = sqrt(d02 + sp * sp);
        if (t != 0.0) S += t * line_log(sm, sp, Rm, Rp, d02);
        Om += atan2(t * sp, d02 + ah * Rp) - atan2(t * sm, d02 + ah * Rm);
    }
    single = S - ah * Om;
    solid = (h > 0.0) ? Om : ((h < 0.0) ? -Om : 0.0);
}

__global__ void q2x_nearfield_kernel(const NearArgs a)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.n_tgt) return;
    int64_t j0 = __ldg(a.tgt_off + t), j1 = __ldg(a.tgt_off + t + 1);
    if (j0 < 0 || j1 < j0) {
        atomicOr(a.err, 8u);
        j0 = j1 = 0;
    }
    const V3 r{__ldg(a.tgt + t), __ldg(a.tgt + a.n_tgt + t), __ldg(a.tgt + 2 * a.n_tgt + t)};
    const int nv = a.kind + 2;
    double acc = 0.0;
#pragma unroll 1
    for (int64_t j = j0; j < j1; ++j) {
        const int64_t e = __ldg(a.elem_idx + j);
        if (e < 0 || e >= a.n_elem) {
            atomicOr(a.err, 1u);
            continue;
        }
        V3 X[4];
        bool bad = false;
        for (int k = 0; k < nv; ++k) {
            const int64_t v = __ldg(a.idx + (int64_t)k * a.n_elem + e);
            if (v < 0 || v >= a.n_vert) {
                bad = true;
                X[k] = V3{0.0, 0.0, 0.0};
            } else {
                X[k] = V3{__ldg(a.vx + v), __ldg(a.vy + v), __ldg(a.vz + v)};
            }
        }
        if (bad) {
            atomicOr(a.err, 1u);
            continue;
        }
        double val = 0.0;
        if (a.kind == 0) {  // segment
            const V3 ev = sub(X[1], X[0]);
            const double L = sqrt(dot(ev, ev));
            if (L > 0.0) {
                const V3 l = scale(ev, 1.0 / L);
                const V3 pa = sub(X[0], r), pb = sub(X[1], r);
                const double sm = dot(pa, l), sp = dot(pb, l);
                const V3 c = cross(pa, l);
                val = line_log(sm, sp, sqrt(dot(pa, pa)), sqrt(dot(pb, pb)), dot(c, c));
            }
        } else if (a.kind == 1) {  // triangle
            double single, solid;
            tri_potential(X[0], X[1], X[2], r, single, solid);
            val = a.layer ? solid : single;
        } else {  // tetrahedron: faces with outward normals
            const V3 c = scale(V3{X[0].x + X[1].x + X[2].x + X[3].x, X[0].y + X[1].y + X[2].y + X[3].y,
                                  X[0].z + X[1].z + X[2].z + X[3].z},
                               0.25);
            const int F[4][3] = {{1, 2, 3}, {0, 3, 2}, {0, 1, 3}, {0, 2, 1}};
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                V3 p0 = X[F[f][0]], p1 = X[F[f][1]], p2 = X[F[f][2]];
                V3 nr = cross(sub(p1, p0), sub(p2, p0));
                if (dot(nr, sub(p0, c)) < 0.0) {  // orient outward
                    const V3 tmp = p1;
                    p1 = p2;
                    p2 = tmp;
                    nr = scale(nr, -1.0);
                }
                const double Jf = sqrt(dot(nr, nr));
                if (!(Jf > 0.0)) continue;
                const double hf = dot(scale(nr, 1.0 / Jf), sub(r, p0));
                double single, solid;
                tri_potential(p0, p1, p2, r, single, solid);
                val += -0.5 * hf * single;
            }
        }
        acc += __ldg(a.sigma + e) * val;
    }
    acc *= NF_INV_4PI;
    a.out[t] = a.accumulate ? a.out[t] + acc : acc;
}

}  // namespace q2x

extern "C" q2x_status q2x_nearfield(q2x_plan_t plan, int kind, int layer, int64_t n_elem, int64_t n_vert,
                                    const double* vxyz, const int32_t* idx, const double* sigma, int64_t n_tgt,
                                    const double* tgt, const int64_t* tgt_off, const int64_t* elem_idx,
                                    double* out, int accumulate)
{
    if (!plan) return q2x_fail(nullptr, Q2X_ERR_ARG, "plan is NULL");
    if (kind < 0 || kind > 2) return q2x_fail(plan, Q2X_ERR_ARG, "kind must be 0 (segment), 1 (triangle), 2 (tetra)");
    if (layer != 0 && !(layer == 1 && kind == 1))
        return q2x_fail(plan, Q2X_ERR_UNSUPPORTED, "the double layer is defined for triangles only");
    if (n_elem < 0 || n_vert < 0 || n_tgt < 0) return q2x_fail(plan, Q2X_ERR_ARG, "negative size");
    if (accumulate != 0 && accumulate != 1) return q2x_fail(plan, Q2X_ERR_ARG, "accumulate must be 0 or 1");
    if (n_tgt == 0) return Q2X_OK;
    if (!tgt || !tgt_off || !elem_idx || !out) return q2x_fail(plan, Q2X_ERR_ARG, "NULL target array");
    if (n_elem > 0 && (!vxyz || !idx || !sigma || n_vert <= 0))
        return q2x_fail(plan, Q2X_ERR_ARG, "NULL element array or no vertices");
    cudaError_t e = cudaSetDevice(plan->device);
    if (e != cudaSuccess) return q2x_cuda_fail(plan, e, "cudaSetDevice");
    q2x::NearArgs a;
    a.kind = kind;
    a.layer = layer;
    a.accumulate = accumulate;
    a.n_elem = n_elem;
    a.n_vert = n_vert;
    a.n_tgt = n_tgt;
    a.vx = vxyz;
    a.vy = vxyz ? vxyz + n_vert : nullptr;
    a.vz = vxyz ? vxyz + 2 * n_vert : nullptr;
    a.idx = idx;
    a.sigma = sigma;
    a.tgt = tgt;
    a.tgt_off = tgt_off;
    a.elem_idx = elem_idx;
    a.out = out;
    a.err = plan->d_err;
    q2x::q2x_nearfield_kernel<<<(unsigned)((n_tgt + 127) / 128), 128, 0, plan->stream>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return q2x_cuda_fail(plan, e, "q2x_nearfield_kernel launch");
    plan->launches += 1;
    return Q2X_OK;
}
