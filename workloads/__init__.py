"""Seeded synthetic inputs for Q2X (geometry, densities, octree leaves).

This module is the ONE piece shared by the oracle side (tests, CPU baseline)
and the CUDA side (binding, bench).  It draws random numbers and builds
meshes, element orderings and leaf lists; it holds none of the method's
arithmetic (no harmonics, no moments, no recursions).

Every array is numpy.  Layouts follow the C-ABI:
  vxyz     float64 (3, n_vert)   SoA vertex coordinates
  idx      int32   (k, n_elem)   SoA element connectivity, k = 2 / 3 / 4
  sigma    float64 (n_elem,) constant density or (n_vert,) linear density
  leaf_off int64   (n_leaves+1,) CSR over the (leaf-sorted) element order
  leaf_c   float64 (3, n_leaves) expansion centres (leaf box centres)
  leaf_rho float64 (n_leaves,)   max distance from the centre to a vertex
                                 of the leaf's elements (scale of the leaf)
  leaf_p   int32   (n_leaves,)   per-leaf degree
"""
from __future__ import annotations

import math

import numpy as np

# ------------------------------------------------------------------ meshes


def icosphere(level: int):
    """Unit icosphere: the 12 icosahedron vertices, `level` rounds of
    midpoint subdivision with projection to the sphere.  Faces are outward,
    counter-clockwise.  Child faces of face f are 4f..4f+3 (generation order).
    Returns vxyz (3, nv) float64, tri (3, nf) int32."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
                  [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
                  [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                  [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                  [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                  [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    for _ in range(level):
        nv = v.shape[0]
        a, b, c = f[:, 0], f[:, 1], f[:, 2]
        e = np.stack([np.minimum(a, b), np.maximum(a, b),
                      np.minimum(b, c), np.maximum(b, c),
                      np.minimum(c, a), np.maximum(c, a)], axis=1).reshape(-1, 2)
        key = e[:, 0] * nv + e[:, 1]
        ukey, inv = np.unique(key, return_inverse=True)
        mid = v[ukey // nv] + v[ukey % nv]
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        v = np.concatenate([v, mid], axis=0)
        m = (inv + nv).reshape(-1, 3)
        ab, bc, ca = m[:, 0], m[:, 1], m[:, 2]
        f = np.stack([np.stack([a, ab, ca], 1), np.stack([b, bc, ab], 1),
                      np.stack([c, ca, bc], 1), np.stack([ab, bc, ca], 1)], axis=1).reshape(-1, 3)
    return np.ascontiguousarray(v.T), np.ascontiguousarray(f.T.astype(np.int32))


def _real_sh_basis(dirs: np.ndarray, lmax: int) -> np.ndarray:
    """Real orthonormal spherical harmonics Y_lm, 1 <= l <= lmax, at unit
    directions dirs (3, n); rows ordered (l, m = -l..l).  Used only to draw
    a smooth random radial bump."""
    x, y, z = dirs
    ct = np.clip(z, -1.0, 1.0)
    st = np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
    phi = np.arctan2(y, x)
    # unnormalised P_l^m (no Condon-Shortley sign; it cancels in |Y|^2 anyway)
    P = {}
    P[(0, 0)] = np.ones_like(ct)
    for m in range(1, lmax + 1):
        P[(m, m)] = (2 * m - 1) * st * P[(m - 1, m - 1)]
    for m in range(0, lmax + 1):
        if m + 1 <= lmax:
            P[(m + 1, m)] = (2 * m + 1) * ct * P[(m, m)]
        for l in range(m + 2, lmax + 1):
            P[(l, m)] = ((2 * l - 1) * ct * P[(l - 1, m)] - (l + m - 1) * P[(l - 2, m)]) / (l - m)
    rows = []
    for l in range(1, lmax + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            nrm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
            if m == 0:
                rows.append(nrm * P[(l, 0)])
            elif m > 0:
                rows.append(math.sqrt(2.0) * nrm * P[(l, am)] * np.cos(am * phi))
            else:
                rows.append(math.sqrt(2.0) * nrm * P[(l, am)] * np.sin(am * phi))
    return np.stack(rows)


def sh_perturb(vxyz: np.ndarray, seed: int, lmax: int = 6, amp: float = 0.1) -> np.ndarray:
    """Radial bump r(y) = 1 + amp * f(y) / max_vertices |f|, f = sum_{l=1..lmax,m}
    c_lm Y_lm with c_lm ~ N(0,1) from `seed`, applied to unit-sphere vertices."""
    rng = np.random.default_rng(seed)
    dirs = vxyz / np.linalg.norm(vxyz, axis=0, keepdims=True)
    B = _real_sh_basis(dirs, lmax)
    c = rng.standard_normal(B.shape[0])
    f = c @ B
    r = 1.0 + amp * f / np.max(np.abs(f))
    return np.ascontiguousarray(dirs * r[None, :])


def filaments(n_fil: int, n_steps: int, step: float, seed: int, r0: float = 0.9):
    """Random-walk vortex filaments in the unit ball: start ~ U(ball r <= r0),
    isotropic steps of length `step`, reflected radially at r = 1.
    Returns vxyz (3, n_fil*(n_steps+1)), seg (2, n_fil*n_steps) int32."""
    rng = np.random.default_rng(seed)
    starts = np.empty((n_fil, 3))
    got = 0
    while got < n_fil:
        cand = rng.uniform(-r0, r0, size=(2 * n_fil, 3))
        cand = cand[np.linalg.norm(cand, axis=1) <= r0]
        k = min(n_fil - got, cand.shape[0])
        starts[got:got + k] = cand[:k]
        got += k
    d = rng.standard_normal(size=(n_steps, n_fil, 3))
    d /= np.linalg.norm(d, axis=2, keepdims=True)
    pts = np.empty((n_steps + 1, n_fil, 3))
    pts[0] = starts
    for s in range(n_steps):
        q = pts[s] + step * d[s]
        r = np.linalg.norm(q, axis=1)
        out = r > 1.0
        if np.any(out):
            q[out] *= ((2.0 - r[out]) / r[out])[:, None]
        pts[s + 1] = q
    v = pts.transpose(1, 0, 2).reshape(-1, 3)  # filament-major
    base = (np.arange(n_fil) * (n_steps + 1))[:, None] + np.arange(n_steps)[None, :]
    seg = np.stack([base.reshape(-1), base.reshape(-1) + 1]).astype(np.int32)
    return np.ascontiguousarray(v.T), seg


def kuhn_tets(spacing: float, seed: int, radius: float = 1.0, jitter: float = 0.15,
              max_tets: int | None = None):
    """Kuhn 6-tetrahedron split of the grid cubes (edge `spacing`) whose centres
    lie in the ball of `radius`; vertices not on the boundary of the cube set
    jittered U[-jitter*h, jitter*h]^3; every tetrahedron positively oriented.
    Returns vxyz (3, nv), tet (4, nt) int32 (truncated to max_tets)."""
    rng = np.random.default_rng(seed)
    h = spacing
    n = int(math.ceil(radius / h)) + 1
    ax = np.arange(-n, n)
    I, J, K = np.meshgrid(ax, ax, ax, indexing="ij")
    cen = (np.stack([I, J, K], -1).reshape(-1, 3) + 0.5) * h
    keep = np.linalg.norm(cen, axis=1) <= radius
    cubes = np.stack([I, J, K], -1).reshape(-1, 3)[keep]
    # unique grid vertices
    corners = np.array([[i, j, k] for i in (0, 1) for j in (0, 1) for k in (0, 1)])
    allv = (cubes[:, None, :] + corners[None, :, :]).reshape(-1, 3)
    side = 2 * n + 2
    key = (allv[:, 0] + n) * side * side + (allv[:, 1] + n) * side + (allv[:, 2] + n)
    ukey, inv = np.unique(key, return_inverse=True)
    cnt = np.bincount(inv)  # corners sharing a vertex: 8 => interior
    gi = np.stack([ukey // (side * side), (ukey // side) % side, ukey % side], 1) - n
    verts = gi.astype(np.float64) * h
    interior = cnt == 8
    verts[interior] += rng.uniform(-jitter * h, jitter * h, size=(int(interior.sum()), 3))
    cv = inv.reshape(-1, 8)  # local corner index (i*4 + j*2 + k)
    tets = []
    for perm in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
        path = [np.zeros(3, dtype=int)]
        for ax_ in perm:
            nxt = path[-1].copy()
            nxt[ax_] = 1
            path.append(nxt)
        loc = [p[0] * 4 + p[1] * 2 + p[2] for p in path]
        tets.append(np.stack([cv[:, l] for l in loc], 0))
    T = np.stack(tets, 1).reshape(4, -1)  # cube-major, 6 tets per cube
    # orientation: det((x2-x1) x (x3-x1) . (x4-x1)) > 0, else swap x3 <-> x4
    X = verts[T]  # (4, nt, 3)
    det = np.einsum("ij,ij->i", np.cross(X[1] - X[0], X[2] - X[0]), X[3] - X[0])
    neg = det < 0
    T[2, neg], T[3, neg] = T[3, neg].copy(), T[2, neg].copy()
    if max_tets is not None:
        T = T[:, :max_tets]
    used, remap = np.unique(T.reshape(-1), return_inverse=True)
    T = remap.reshape(4, -1).astype(np.int32)
    return np.ascontiguousarray(verts[used].T), np.ascontiguousarray(T)


# ------------------------------------------------------------------ leaves


def _morton3(ix, iy, iz, depth):
    code = np.zeros(ix.shape, dtype=np.int64)
    for b in range(depth):
        code |= ((ix >> b) & 1) << (3 * b + 2)
        code |= ((iy >> b) & 1) << (3 * b + 1)
        code |= ((iz >> b) & 1) << (3 * b)
    return code


def element_centres(vxyz: np.ndarray, idx: np.ndarray) -> np.ndarray:
    """Vertex mean of each element, (3, n_elem)."""
    return np.mean(vxyz[:, idx], axis=1)


def uniform_leaves(centres: np.ndarray, lo: float, size: float, depth: int):
    """Finest-level cell of each element centre in the cube [lo, lo+size]^3 at
    `depth` (half-open cells, clamped), non-empty cells only, sorted by Morton
    code (ties keep element order).  Returns (order, leaf_of_sorted, leaf_c,
    cell_h) where `order` permutes elements into leaf order."""
    h = size / (1 << depth)
    ijk = np.floor((centres - lo) / h).astype(np.int64)
    ijk = np.clip(ijk, 0, (1 << depth) - 1)
    code = _morton3(ijk[0], ijk[1], ijk[2], depth)
    order = np.argsort(code, kind="stable")
    sc = code[order]
    ucode, first = np.unique(sc, return_index=True)
    leaf_of = np.searchsorted(ucode, sc)
    cell = ijk[:, order][:, first]
    leaf_c = lo + (cell.astype(np.float64) + 0.5) * h
    return order, leaf_of, leaf_c, h


def adaptive_leaves(centres: np.ndarray, lo: float, size: float, max_per_leaf: int,
                    max_depth: int):
    """Adaptive octree over the element centres: split a box while it holds more
    than `max_per_leaf` elements, up to `max_depth`.  Returns (order, leaf_of,
    leaf_c, leaf_h) with leaves in depth-first Morton order (non-empty only)."""
    n = centres.shape[1]
    full = _morton3(*np.clip(np.floor((centres - lo) / (size / (1 << max_depth))).astype(np.int64),
                             0, (1 << max_depth) - 1), max_depth)
    order = np.argsort(full, kind="stable")
    sc = full[order]
    leaves = []  # (start, end, depth, prefix)

    def rec(s, e, d, prefix):
        if e - s <= max_per_leaf or d == max_depth:
            leaves.append((s, e, d, prefix))
            return
        shift = 3 * (max_depth - d - 1)
        child = (sc[s:e] >> shift) & 7
        bounds = np.searchsorted(child, np.arange(9))
        for ch in range(8):
            cs, ce = s + bounds[ch], s + bounds[ch + 1]
            if ce > cs:
                rec(cs, ce, d + 1, (prefix << 3) | ch)

    rec(0, n, 0, 0)
    nl = len(leaves)
    leaf_of = np.empty(n, dtype=np.int64)
    leaf_c = np.empty((3, nl))
    leaf_h = np.empty(nl)
    for li, (s, e, d, prefix) in enumerate(leaves):
        leaf_of[s:e] = li
        ix = iy = iz = 0
        for b in range(d):
            t = (prefix >> (3 * (d - 1 - b))) & 7
            ix = (ix << 1) | ((t >> 2) & 1)
            iy = (iy << 1) | ((t >> 1) & 1)
            iz = (iz << 1) | (t & 1)
        h = size / (1 << d)
        leaf_c[:, li] = lo + (np.array([ix, iy, iz]) + 0.5) * h
        leaf_h[li] = h
    return order, leaf_of, leaf_c, leaf_h


def csr_from_leaf_of(leaf_of_sorted: np.ndarray, n_leaves: int) -> np.ndarray:
    cnt = np.bincount(leaf_of_sorted, minlength=n_leaves)
    off = np.zeros(n_leaves + 1, dtype=np.int64)
    np.cumsum(cnt, out=off[1:])
    return off


def leaf_rho(vxyz, idx_sorted, leaf_off, leaf_c) -> np.ndarray:
    """Max distance from each leaf centre to a vertex of the leaf's elements."""
    n_leaves = leaf_off.shape[0] - 1
    leaf_of = np.repeat(np.arange(n_leaves), np.diff(leaf_off))
    d = np.zeros(idx_sorted.shape[1])
    for k in range(idx_sorted.shape[0]):
        dv = vxyz[:, idx_sorted[k]] - leaf_c[:, leaf_of]
        d = np.maximum(d, np.sqrt(np.sum(dv * dv, axis=0)))
    rho = np.zeros(n_leaves)
    np.maximum.at(rho, leaf_of, d)
    return rho


# ------------------------------------------------------------------ problems


def make_problem(vxyz, idx, sigma, sigma_per_vertex, order, leaf_of, leaf_c, p, leaf_p=None):
    """Reorder elements into leaf order and assemble the argument dict."""
    idx_s = np.ascontiguousarray(idx[:, order])
    sig = sigma if sigma_per_vertex else np.ascontiguousarray(sigma[order])
    n_leaves = leaf_c.shape[1]
    off = csr_from_leaf_of(leaf_of, n_leaves)
    rho = leaf_rho(vxyz, idx_s, off, leaf_c)
    if leaf_p is None:
        leaf_p = np.full(n_leaves, p, dtype=np.int32)
    return dict(vxyz=np.ascontiguousarray(vxyz, dtype=np.float64), idx=idx_s,
                sigma=np.ascontiguousarray(sig, dtype=np.float64), leaf_off=off,
                leaf_c=np.ascontiguousarray(leaf_c), leaf_rho=rho,
                leaf_p=np.ascontiguousarray(leaf_p, dtype=np.int32), p=int(p))


def perturbed_sphere(level: int, seed: int):
    v, t = icosphere(level)
    return sh_perturb(v, seed), t


def cfg_icosphere_l3(p: int = 10, seed: int = 0):
    """1280-triangle unit icosphere, constant density U[-1,1], one expansion
    about the origin."""
    v, t = icosphere(3)
    rng = np.random.default_rng(seed)
    sig = rng.uniform(-1.0, 1.0, size=t.shape[1])
    order = np.arange(t.shape[1])
    leaf_of = np.zeros(t.shape[1], dtype=np.int64)
    prob = make_problem(v, t, sig, False, order, leaf_of, np.zeros((3, 1)), p)
    prob.update(kind="triangle", density="const", layers=("single",), name="icosphere-L3")
    return prob


def cfg_sphere_linear(level: int = 7, depth: int = 5, p: int = 12, seed_shape: int = 1,
                      seed_sigma: int = 2):
    """SH-perturbed icosphere, linear per-vertex density U[-1,1], uniform octree
    of `depth` over the cube [-1.125, 1.125]^3, single + double layer."""
    v, t = perturbed_sphere(level, seed_shape)
    rng = np.random.default_rng(seed_sigma)
    sig = rng.uniform(-1.0, 1.0, size=v.shape[1])
    order, leaf_of, leaf_c, _ = uniform_leaves(element_centres(v, t), -1.125, 2.25, depth)
    prob = make_problem(v, t, sig, True, order, leaf_of, leaf_c, p)
    prob.update(kind="triangle", density="linear", layers=("single", "double"),
                name="sphere-L%d-linear-depth%d" % (level, depth))
    return prob


def cfg_sphere_const(level: int = 9, depth: int = 7, p: int = 16, seed_shape: int = 3,
                     seed_sigma: int = 33):
    """SH-perturbed icosphere, constant density U[-1,1], uniform octree."""
    v, t = perturbed_sphere(level, seed_shape)
    rng = np.random.default_rng(seed_sigma)
    sig = rng.uniform(-1.0, 1.0, size=t.shape[1])
    order, leaf_of, leaf_c, _ = uniform_leaves(element_centres(v, t), -1.125, 2.25, depth)
    prob = make_problem(v, t, sig, False, order, leaf_of, leaf_c, p)
    prob.update(kind="triangle", density="const", layers=("single",),
                name="sphere-L%d-const-depth%d" % (level, depth))
    return prob


def random_triangles(n: int, seed: int, spread: float = 1.0, size: float = 0.05):
    """n independent random triangles (3n vertices) around random points."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(-spread, spread, size=(3, n))
    v = np.concatenate([c + size * rng.standard_normal((3, n)) for _ in range(3)], axis=1)
    t = np.stack([np.arange(n), np.arange(n) + n, np.arange(n) + 2 * n]).astype(np.int32)
    return v, t


def cfg_mixed_ball(n_fil=2000, n_steps=1000, step=1e-3, tri_level=9, n_tri=4_000_000, tet_spacing=0.0293,
                   n_tet=1_000_000, max_per_leaf=2000, max_depth=12, p_lo=8, p_hi=20, seed=4):
    """Mixed elements in the unit ball sharing one adaptive octree:
    random-walk filament segments (density U[-1,1]), the first n_tri triangles
    of the perturbed level-`tri_level` sphere scaled by 0.9 (constant density
    U[-1,1]), and Kuhn tetrahedra of a jittered grid (density U[0,1]).  A box is
    split while it holds more than max_per_leaf elements of any kind, up to
    max_depth; per-leaf degree p_leaf ~ U{p_lo..p_hi}.
    Returns dict(kinds={segment, triangle, tetra: dict(vxyz, idx, sigma,
    leaf_off)}, leaf_c, leaf_rho, leaf_p, leaf_depth, p); the octree cube is
    [-1, 1]^3."""
    rng = np.random.default_rng(seed)
    kinds = {}
    vs, es = filaments(n_fil, n_steps, step, seed=seed + 1)
    kinds["segment"] = dict(vxyz=vs, idx=es, sigma=rng.uniform(-1, 1, es.shape[1]))
    vt, tt = perturbed_sphere(tri_level, seed=seed + 2)
    tt = np.ascontiguousarray(tt[:, :n_tri])
    used, remap = np.unique(tt.reshape(-1), return_inverse=True)
    tt = remap.reshape(3, -1).astype(np.int32)
    vt = np.ascontiguousarray(0.9 * vt[:, used])
    kinds["triangle"] = dict(vxyz=vt, idx=tt, sigma=rng.uniform(-1, 1, tt.shape[1]))
    vq, tq = kuhn_tets(tet_spacing, seed=seed + 3, radius=1.0, max_tets=n_tet)
    kinds["tetra"] = dict(vxyz=vq, idx=tq, sigma=rng.uniform(0, 1, tq.shape[1]))
    names = ["segment", "triangle", "tetra"]
    cents = [element_centres(kinds[k]["vxyz"], kinds[k]["idx"]) for k in names]
    allc = np.concatenate(cents, axis=1)
    order, leaf_of, leaf_c, leaf_h = adaptive_leaves(allc, -1.0, 2.0, max_per_leaf, max_depth)
    n_leaves = leaf_c.shape[1]
    leaf_all = np.empty(allc.shape[1], dtype=np.int64)
    leaf_all[order] = leaf_of
    base = 0
    rho = np.zeros(n_leaves)
    for k, c in zip(names, cents):
        n = c.shape[1]
        lk = leaf_all[base:base + n]
        base += n
        o = np.argsort(lk, kind="stable")
        d = kinds[k]
        d["idx"] = np.ascontiguousarray(d["idx"][:, o])
        d["sigma"] = np.ascontiguousarray(d["sigma"][o])
        d["leaf_off"] = csr_from_leaf_of(lk[o], n_leaves)
        rho = np.maximum(rho, leaf_rho(d["vxyz"], d["idx"], d["leaf_off"], leaf_c))
        d["vxyz"] = np.ascontiguousarray(d["vxyz"], dtype=np.float64)
    rho = np.where(rho > 0, rho, 0.5 * np.sqrt(3.0) * leaf_h)
    leaf_p = rng.integers(p_lo, p_hi + 1, size=n_leaves).astype(np.int32)
    leaf_depth = np.rint(np.log2(2.0 / leaf_h)).astype(np.int64)
    return dict(kinds=kinds, leaf_c=np.ascontiguousarray(leaf_c), leaf_rho=rho, leaf_p=leaf_p, p=int(p_hi),
                leaf_depth=leaf_depth, name="mixed-ball")


def cfg_sphere_adjoint(level: int = 8, n_tri: int = 1_000_000, depth: int = 6, p: int = 12, seed_shape: int = 5,
                       seed_sigma: int = 6, seed_g: int = 7):
    """Perturbed level-`level` sphere truncated to its first n_tri triangles,
    constant density U[-1,1], uniform octree of `depth`, and a seeded N(0,1)
    adjoint G (one row of (p+1)^2 per leaf)."""
    v, t = perturbed_sphere(level, seed_shape)
    t = np.ascontiguousarray(t[:, :n_tri])
    used, remap = np.unique(t.reshape(-1), return_inverse=True)
    t = remap.reshape(3, -1).astype(np.int32)
    v = np.ascontiguousarray(v[:, used])
    rng = np.random.default_rng(seed_sigma)
    sig = rng.uniform(-1.0, 1.0, size=t.shape[1])
    order, leaf_of, leaf_c, _ = uniform_leaves(element_centres(v, t), -1.125, 2.25, depth)
    prob = make_problem(v, t, sig, False, order, leaf_of, leaf_c, p)
    prob.update(kind="triangle", density="const", layers=("single",), name="sphere-L%d-adjoint" % level)
    prob["G"] = np.random.default_rng(seed_g).standard_normal((leaf_c.shape[1], (p + 1) ** 2))
    return prob
