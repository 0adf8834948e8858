"""Shared test helpers: small seeded problems and the normalised coefficient
error used for parity (scaled coefficients M^_n^m = M_n^m sqrt((n+|m|)!(n-|m|)!)
/ rho^n, double layer / (n rho^{n-1}); per leaf, max |dM^| / max |M^_ref|)."""
import math

import numpy as np

import workloads as W

NV = {"segment": 2, "triangle": 3, "tetra": 4}


def scale_vector(p, rho, layer=0):
    s = np.zeros((p + 1) ** 2)
    for n in range(p + 1):
        for m in range(-n, n + 1):
            f = math.sqrt(math.factorial(n + abs(m)) * math.factorial(n - abs(m)))
            if layer == 0:
                s[n * n + n + m] = f / rho ** n
            else:
                s[n * n + n + m] = f / (max(n, 1) * rho ** max(n - 1, 0))
    return s


def norm_err(test, ref, p, rho, layer=0):
    """max over leaves of the normalised error; rho per leaf."""
    test = np.asarray(test)
    ref = np.asarray(ref)
    worst = 0.0
    for L in range(ref.shape[0]):
        s = scale_vector(p, max(rho[L], 1e-300), layer)
        a = test[L] * s
        b = ref[L] * s
        den = np.max(np.abs(b))
        num = np.max(np.abs(a - b))
        if den == 0:
            e = num
        else:
            e = num / den
        worst = max(worst, e)
    return worst


def random_problem(kind, sizes, seed, p, size=0.04, spread=0.6, density="const", centre_jitter=0.02,
                   leaf_p=None):
    """Leaves with the given element counts (0 allowed), random centres, small
    random simplices near each centre; elements already sorted by leaf."""
    rng = np.random.default_rng(seed)
    nl = len(sizes)
    nv = NV[kind]
    centres = rng.uniform(-spread, spread, size=(3, nl))
    n = int(sum(sizes))
    leaf_of = np.repeat(np.arange(nl), sizes)
    base = centres[:, leaf_of] + centre_jitter * rng.standard_normal((3, n))
    verts = [base + size * rng.standard_normal((3, n)) for _ in range(nv)]
    vxyz = np.concatenate(verts, axis=1) if n else np.zeros((3, 1))
    idx = np.stack([np.arange(n) + k * n for k in range(nv)]).astype(np.int32) if n else \
        np.zeros((nv, 0), dtype=np.int32)
    if kind == "tetra" and n:
        X = [vxyz[:, idx[k]] for k in range(4)]
        det = np.einsum("ij,ij->j", np.cross((X[1] - X[0]).T, (X[2] - X[0]).T).T, X[3] - X[0])
        neg = det < 0
        idx[2, neg], idx[3, neg] = idx[3, neg].copy(), idx[2, neg].copy()
    if density == "linear":
        sigma = rng.uniform(-1, 1, size=vxyz.shape[1])
    else:
        sigma = rng.uniform(-1, 1, size=max(n, 0))
    off = W.csr_from_leaf_of(leaf_of, nl)
    rho = W.leaf_rho(vxyz, idx, off, centres) if n else np.ones(nl)
    rho = np.where(rho > 0, rho, 1.0)
    if leaf_p is None:
        leaf_p = np.full(nl, p, dtype=np.int32)
    return dict(vxyz=np.ascontiguousarray(vxyz), idx=np.ascontiguousarray(idx), sigma=sigma, leaf_off=off,
                leaf_c=np.ascontiguousarray(centres), leaf_rho=rho, leaf_p=np.asarray(leaf_p, dtype=np.int32),
                p=p, kind=kind, density=density)


def oracle_coef(orc, prob, layer=0, norm=0, per_element=False):
    dens = 1 if prob.get("density") == "linear" else 0
    if per_element:
        n = prob["idx"].shape[1]
        leaf_of = np.repeat(np.arange(prob["leaf_c"].shape[1]), np.diff(prob["leaf_off"]))
        return orc.moments(prob["kind"], prob["vxyz"], prob["idx"], prob["sigma"], prob["p"], leaf_off=None,
                           leaf_c=prob["leaf_c"][:, leaf_of], layer=layer, density=dens, norm=norm)
    return orc.moments(prob["kind"], prob["vxyz"], prob["idx"], prob["sigma"], prob["p"],
                       leaf_off=prob["leaf_off"], leaf_c=prob["leaf_c"], leaf_p=prob["leaf_p"], layer=layer,
                       density=dens, norm=norm)
