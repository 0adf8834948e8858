// q2x_nearfield.cu -- exact potentials of constant-density elements at
// target points (the near field next to the expansions; Sec. 4.1's closed
// forms as kernels):
//   segment:      int 1/|r - y| dl = log((R_b + s_b) / (R_a + s_a))     (Eqs. (num1)-(num3))
//   triangle:     int 1/|r - y| dS = sum_edges t_i log((R+ + s+)/(R- + s-)) - h Omega  (Eq. (num5))
//   triangle, double layer: int n.(r - y)/|r - y|^3 dS = Omega, the signed solid angle
//   tetrahedron:  int 1/|r - y| dV = -1/2 sum_faces h_j int_face 1/|r - y| dS  (Eqs. (num7)-(num8))
// with, per triangle edge i (n the unit normal, m_i the outward in-plane edge
// normal, h = n.(r - x1) the target's height): s-/s+ the coordinates of the
// edge's ends along it from the foot of the perpendicular, t_i the signed
// distance of the target's projection from the edge's line, R-/R+ the
// distances from r to the ends.  The paper writes Omega as a sum of atan
// pairs over the edges; here it is one atan2 of the triangle's solid angle.
// Each contribution is multiplied by sigma_e / (4 pi) (the Green's function
// of Eq. (bas3)).
//
// A first kernel writes one frame per face (triangle: 1, tetrahedron: 4,
// outward): origin, in-plane axes, normal and the 2D vertex positions and
// edge directions, so that the per-pair work is the target's three frame
// coordinates, three vertex distances, three log1p, one atan2 and one
// division per edge.  The second runs one thread per target over the
// target's element list (CSR).  Logarithms form each factor R + s as
// d0^2 / (R - s) where s < 0, away from cancellation; heights and in-plane
// distances below the rounding of the coordinates count as zero.  FP64.
#include <cuda_runtime.h>

#include <cstdint>

#include "q2x.h"
#include "q2x_plan.h"

namespace q2x {

constexpr double NF_INV_4PI = 0.079577471545947667884;
constexpr double NF_SNAP = 16.0 * 2.220446049250313e-16;  // 16 ulps of the coordinates' magnitude

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

// log((R+ + s+) / (R- + s-)) for a line piece of length L whose ends sit at
// coordinates s- < s+ along it from the foot of the perpendicular, at
// distances R-, R+ from the target, d02 the squared distance to the line.
// As (R + s)(R - s) = d02 at both ends, the value is also log((R- - s-) /
// (R+ - s+)), the form taken when the piece lies mostly behind the foot.
// With N/D the ratio, N - D = L (1 +- (s- + s+) / (R- + R+)) exactly (from
// R+^2 - R-^2 = s+^2 - s-^2), a sum of non-negative terms, so log1p((N - D)
// / D) keeps full relative accuracy when the target is far from a short
// piece; D is formed as d02 / (R - s) where R + s would cancel.  One
// division.
__device__ __forceinline__ double line_log(double sm, double sp, double Rm, double Rp, double d02, double L)
{
    const double Sg = Rm + Rp, sg = sm + sp;
    const double num = L * (Sg + fabs(sg));
    const double a = (sg >= 0.0) ? Rm : Rp;
    const double s = (sg >= 0.0) ? sm : -sp;
    // selects, not branches: lanes see an edge from either side
    const bool ahead = s >= 0.0;
    const double numer = ahead ? num : num * (a - s);
    const double denom = Sg * (ahead ? a + s : d02);
    return log1p(numer / denom);
}

// A flat face in its own frame: origin x1, in-plane axes u (along the first
// edge) and w = n x u, unit normal n; vertices at (0, 0), (L0, 0), (v3x,
// v3y) (counter-clockwise about n); edge i runs from vertex i to i + 1 with
// unit direction l_i (l_0 = (1, 0)) and length L_i; J = twice the area.
// J = 0 marks a degenerate face.
struct Face {
    double x1[3], u[3], w[3], n[3];
    double J, L0, v3x, v3y, l1x, l1y, l2x, l2y, L1, L2;
};
constexpr int FACE_DOUBLES = sizeof(Face) / sizeof(double);
static_assert(FACE_DOUBLES == 22, "face record is 22 doubles");

__device__ void make_face(V3 x1, V3 x2, V3 x3, Face& F)
{
    const V3 e0 = sub(x2, x1), e2 = sub(x3, x1);
    const V3 nr = cross(e0, e2);
    const double J = sqrt(dot(nr, nr)), L0 = sqrt(dot(e0, e0));
    F.J = (J > 0.0 && L0 > 0.0) ? J : 0.0;
    const double iJ = F.J > 0.0 ? 1.0 / J : 0.0, iL0 = F.J > 0.0 ? 1.0 / L0 : 0.0;
    const V3 n = scale(nr, iJ), u = scale(e0, iL0), w = cross(n, u);
    F.x1[0] = x1.x, F.x1[1] = x1.y, F.x1[2] = x1.z;
    F.u[0] = u.x, F.u[1] = u.y, F.u[2] = u.z;
    F.w[0] = w.x, F.w[1] = w.y, F.w[2] = w.z;
    F.n[0] = n.x, F.n[1] = n.y, F.n[2] = n.z;
    F.L0 = L0;
    F.v3x = dot(e2, u);
    F.v3y = dot(e2, w);
    const double d1x = F.v3x - L0, d1y = F.v3y;
    F.L1 = sqrt(d1x * d1x + d1y * d1y);
    F.L2 = sqrt(F.v3x * F.v3x + F.v3y * F.v3y);
    const double i1 = F.L1 > 0.0 ? 1.0 / F.L1 : 0.0, i2 = F.L2 > 0.0 ? 1.0 / F.L2 : 0.0;
    F.l1x = d1x * i1, F.l1y = d1y * i1;
    F.l2x = -F.v3x * i2, F.l2y = -F.v3y * i2;
}

// One thread per face: kind 1 one face per triangle (its own vertex order),
// kind 2 four faces per tetrahedron (opposite vertex 0..3, each ordered so
// that its normal points out of the tetrahedron).
__global__ void q2x_nearfield_faces(const NearArgs a, Face* faces)
{
    const int fpe = a.kind == 2 ? 4 : 1;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n_elem * fpe) return;
    const int64_t e = i / fpe;
    const int f = (int)(i - e * fpe);
    const int nv = a.kind + 2;
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
    Face F;
    if (bad) {
        atomicOr(a.err, 1u);
        F = Face{};  // J = 0: contributes nothing
    } else if (a.kind == 1) {
        make_face(X[0], X[1], X[2], F);
    } else {
        // faces opposite vertex 0..3, outward when det[x1-x0, x2-x0, x3-x0] > 0
        const int T[4][3] = {{1, 2, 3}, {0, 3, 2}, {0, 1, 3}, {0, 2, 1}};
        V3 p0 = X[T[f][0]], p1 = X[T[f][1]], p2 = X[T[f][2]];
        const V3 e1 = sub(X[1], X[0]), e2 = sub(X[2], X[0]), e3 = sub(X[3], X[0]);
        const double det = dot(e1, cross(e2, e3));
        const double scale3 = sqrt(dot(e1, e1) * dot(e2, e2) * dot(e3, e3));
        if (!(fabs(det) > NF_SNAP * 4.0 * scale3)) {
            F = Face{};  // zero volume (to rounding): no potential, and no outward side to orient
        } else {
            if (det < 0.0) {  // negatively ordered vertices: every face flips
                const V3 tmp = p1;
                p1 = p2;
                p2 = tmp;
            }
            make_face(p0, p1, p2, F);
        }
    }
    faces[i] = F;
}

// int 1/|r - y| dS over a face (single) and the double-layer kernel's
// integral int n.(r - y)/|r - y|^3 dS (solid) at the target r, h its height:
//   single = sum_i t_i log((R_{i+1} + s+)/(R_i + s-)) - h * solid,
//   solid  = 2 atan2(J h, R1R2R3 + (R1.R2)R3 + (R1.R3)R2 + (R2.R3)R1),
// R_i = x_i - r (the solid angle of the face as Van Oosterom and Strackee
// write it, its determinant being -J h); the edge sum of the paper's form is
// the same quantity as three atan pairs.  A target in the plane (h = 0 after
// the snap) gets solid = 0, its direct value.
__device__ __forceinline__ void face_potential(const Face* __restrict__ Fp, V3 r, double& single, double& solid,
                                               double& h_out)
{
    const double J = __ldg(&Fp->J);
    single = solid = h_out = 0.0;
    if (!(J > 0.0)) return;
    const V3 x1{__ldg(&Fp->x1[0]), __ldg(&Fp->x1[1]), __ldg(&Fp->x1[2])};
    const V3 d = sub(r, x1);
    const double rx = d.x * __ldg(&Fp->u[0]) + d.y * __ldg(&Fp->u[1]) + d.z * __ldg(&Fp->u[2]);
    const double ry = d.x * __ldg(&Fp->w[0]) + d.y * __ldg(&Fp->w[1]) + d.z * __ldg(&Fp->w[2]);
    double h = d.x * __ldg(&Fp->n[0]) + d.y * __ldg(&Fp->n[1]) + d.z * __ldg(&Fp->n[2]);
    // heights and in-plane distances below the rounding of the coordinates
    // are taken as zero: a target within that of the plane is in it
    const double tol = NF_SNAP * (fabs(r.x) + fabs(r.y) + fabs(r.z) + fabs(x1.x) + fabs(x1.y) + fabs(x1.z));
    if (fabs(h) <= tol) h = 0.0;
    const double h2 = h * h;
    const double L0 = __ldg(&Fp->L0), v3x = __ldg(&Fp->v3x), v3y = __ldg(&Fp->v3y);
    // vertex offsets from the target's projection, and distances
    const double ax = -rx, ay = -ry, bx = L0 - rx, by = -ry, cx = v3x - rx, cy = v3y - ry;
    const double R1 = sqrt(ax * ax + ay * ay + h2), R2 = sqrt(bx * bx + by * by + h2),
                 R3 = sqrt(cx * cx + cy * cy + h2);
    const double lx[3] = {1.0, __ldg(&Fp->l1x), __ldg(&Fp->l2x)};
    const double ly[3] = {0.0, __ldg(&Fp->l1y), __ldg(&Fp->l2y)};
    const double Ls[3] = {L0, __ldg(&Fp->L1), __ldg(&Fp->L2)};
    const double px[4] = {ax, bx, cx, ax}, py[4] = {ay, by, cy, ay};
    const double Rv[4] = {R1, R2, R3, R1};
    double S = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const double sm = px[i] * lx[i] + py[i] * ly[i];
        const double sp = px[i + 1] * lx[i] + py[i + 1] * ly[i];
        double t = px[i] * ly[i] - py[i] * lx[i];  // offset . m_i, m_i = (l_y, -l_x) the outward normal
        if (fabs(t) <= tol) t = 0.0;                // target on the edge's line
        if (t != 0.0 && Ls[i] > 0.0) S += t * line_log(sm, sp, Rv[i], Rv[i + 1], t * t + h2, Ls[i]);
    }
    if (h != 0.0) {
        const double den = R1 * R2 * R3 + (ax * bx + ay * by + h2) * R3 + (ax * cx + ay * cy + h2) * R2 +
                           (bx * cx + by * cy + h2) * R1;
        solid = 2.0 * atan2(J * h, den);
    }
    single = S - h * solid;
    h_out = h;
}

__global__ void q2x_nearfield_kernel(const NearArgs a, const Face* __restrict__ faces)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.n_tgt) return;
    int64_t j0 = __ldg(a.tgt_off + t), j1 = __ldg(a.tgt_off + t + 1);
    if (j0 < 0 || j1 < j0 || (j1 > j0 && a.elem_idx == nullptr)) {  // an empty list set may pass NULL
        atomicOr(a.err, 8u);
        j0 = j1 = 0;
    }
    const V3 r{__ldg(a.tgt + t), __ldg(a.tgt + a.n_tgt + t), __ldg(a.tgt + 2 * a.n_tgt + t)};
    double acc = 0.0;
#pragma unroll 1
    for (int64_t j = j0; j < j1; ++j) {
        const int64_t e = __ldg(a.elem_idx + j);
        if (e < 0 || e >= a.n_elem) {
            atomicOr(a.err, 1u);
            continue;
        }
        double val = 0.0;
        if (a.kind == 0) {  // segment
            const int64_t v0 = __ldg(a.idx + e), v1 = __ldg(a.idx + a.n_elem + e);
            if (v0 < 0 || v0 >= a.n_vert || v1 < 0 || v1 >= a.n_vert) {
                atomicOr(a.err, 1u);
                continue;
            }
            const V3 X0{__ldg(a.vx + v0), __ldg(a.vy + v0), __ldg(a.vz + v0)};
            const V3 X1{__ldg(a.vx + v1), __ldg(a.vy + v1), __ldg(a.vz + v1)};
            const V3 ev = sub(X1, X0);
            const double L = sqrt(dot(ev, ev));
            if (L > 0.0) {
                const V3 l = scale(ev, 1.0 / L);
                const V3 pa = sub(X0, r), pb = sub(X1, r);
                const V3 c = cross(pa, l);
                val = line_log(dot(pa, l), dot(pb, l), sqrt(dot(pa, pa)), sqrt(dot(pb, pb)), dot(c, c), L);
            }
        } else if (a.kind == 1) {  // triangle
            double single, solid, h;
            face_potential(faces + e, r, single, solid, h);
            val = a.layer ? solid : single;
        } else {  // tetrahedron: -1/2 sum over the outward faces of h_f int_f 1/|r - y| dS
#pragma unroll 1
            for (int f = 0; f < 4; ++f) {
                double single, solid, h;
                face_potential(faces + 4 * e + f, r, single, solid, h);
                val -= 0.5 * h * single;
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
    if (n_elem > ((int64_t)1 << 36) || n_tgt > ((int64_t)1 << 36))
        return q2x_fail(plan, Q2X_ERR_ARG, "n_elem or n_tgt too large");
    if (!tgt || !tgt_off || !out) return q2x_fail(plan, Q2X_ERR_ARG, "NULL target array");
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
    q2x::Face* faces = nullptr;
    if (kind > 0 && n_elem > 0) {
        const int64_t nf = n_elem * (kind == 2 ? 4 : 1);
        q2x_status st = q2x_plan_workspace(plan, sizeof(q2x::Face) * (size_t)nf);
        if (st != Q2X_OK) return st;
        faces = static_cast<q2x::Face*>(plan->ws);
        q2x::q2x_nearfield_faces<<<(unsigned)((nf + 127) / 128), 128, 0, plan->stream>>>(a, faces);
        e = cudaGetLastError();
        if (e != cudaSuccess) return q2x_cuda_fail(plan, e, "q2x_nearfield_faces launch");
        plan->launches += 1;
    }
    q2x::q2x_nearfield_kernel<<<(unsigned)((n_tgt + 127) / 128), 128, 0, plan->stream>>>(a, faces);
    e = cudaGetLastError();
    if (e != cudaSuccess) return q2x_cuda_fail(plan, e, "q2x_nearfield_kernel launch");
    plan->launches += 1;
    return Q2X_OK;
}
