"""Python binding of the Q2X C ABI: argument marshalling from torch CUDA
tensors to the library's pointers and sizes.  Every computation happens in
the CUDA library; nothing here computes a moment."""
from __future__ import annotations

import ctypes

import torch

from ._lib import check, lib

NORM_COEFF, NORM_MOMENT = 0, 1
FP64, FP32_MIXED = 0, 1
DENSITY_CONST, DENSITY_LINEAR = 0, 1
_NORMS = {"coeff": 0, "moment": 1, 0: 0, 1: 1}
_PRECS = {"fp64": 0, "fp32": 1, "fp32_mixed": 1, 0: 0, 1: 1}
_DENS = {"const": 0, "constant": 0, "linear": 1, 0: 0, 1: 1}


def n_coef(p: int) -> int:
    return (p + 1) * (p + 1)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _need(t, dtype, name, shape=None):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch tensor" % name)
    if t.device.type != "cuda":
        raise ValueError("%s must be a CUDA tensor (the library takes device pointers)" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("%s has shape %s, expected %s" % (name, tuple(t.shape), tuple(shape)))
    return t


class PlanGraph:
    """A captured sequence of q2x calls (Plan.capture)."""

    def __init__(self, graph, kernels):
        self.graph = graph
        self.kernels = kernels  # kernels launched per replay

    def replay(self):
        self.graph.replay()


class Plan:
    """A q2x_plan: degree bound, normalisation, precision, stream and the
    library-owned workspace.  Calls are asynchronous on the plan's stream;
    `sync()` waits and raises on device-side input errors."""

    def __init__(self, p_max: int, norm="coeff", precision="fp64", stream=None):
        self.p_max = int(p_max)
        self.norm = _NORMS[norm]
        self.precision = _PRECS[precision]
        if stream is None and torch.cuda.is_available():
            stream = torch.cuda.current_stream()
        self._stream = stream
        h = ctypes.c_void_p()
        # without a CUDA device the library itself reports Q2X_ERR_CUDA
        check(lib().q2x_plan(ctypes.byref(h), self.p_max, self.norm, self.precision,
                             ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().q2x_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        self._stream = stream
        check(lib().q2x_plan_set_stream(self._h, ctypes.c_void_p(stream.cuda_stream)), self._h)

    def capture(self, fn):
        """Record the q2x calls that fn() makes on this plan as one CUDA graph
        and return a PlanGraph whose replay() re-runs them on the current
        stream with one host launch (same buffers; their contents may
        change between replays).  fn runs once eagerly first, so that the
        plan's workspace and kernel attributes are set before the capture."""
        fn()
        torch.cuda.synchronize()
        side = torch.cuda.Stream()
        old = self._stream
        n0 = self.launch_count()
        self.set_stream(side)
        graph = torch.cuda.CUDAGraph()
        try:
            with torch.cuda.graph(graph, stream=side):
                fn()
        finally:
            self.set_stream(old)
        return PlanGraph(graph, self.launch_count() - n0)

    def sync(self):
        check(lib().q2x_sync(self._h), self._h)

    def device_errors(self) -> int:
        bits = ctypes.c_uint32(0)
        check(lib().q2x_device_errors(self._h, ctypes.byref(bits)), self._h)
        return int(bits.value)

    def reserve(self, n_elem: int, n_leaves: int):
        check(lib().q2x_reserve(self._h, int(n_elem), int(n_leaves)), self._h)

    def workspace_bytes(self) -> int:
        return int(lib().q2x_workspace_bytes(self._h))

    def launch_count(self) -> int:
        """Kernels this plan has launched so far."""
        return int(lib().q2x_launch_count(self._h))

    def set_kernel_timing(self, enable: bool = True):
        """Time every element-kernel launch with the library's own CUDA events."""
        check(lib().q2x_plan_set_kernel_timing(self._h, int(bool(enable))), self._h)

    def kernel_timing(self):
        """(total ms, launches) of the element kernels timed since the last query."""
        ms = ctypes.c_double(0.0)
        n = ctypes.c_int64(0)
        check(lib().q2x_plan_kernel_timing(self._h, ctypes.byref(ms), ctypes.byref(n)), self._h)
        return float(ms.value), int(n.value)

    # ------------------------------------------------------------ helpers
    def _leaf_args(self, n_elem, leaf_off, leaf_c, leaf_rho, leaf_p):
        if leaf_off is None:
            n_leaves = n_elem
        else:
            _need(leaf_off, torch.int64, "leaf_off")
            n_leaves = leaf_off.shape[0] - 1
        _need(leaf_c, torch.float64, "leaf_c", (3, n_leaves))
        _need(leaf_rho, torch.float64, "leaf_rho", (n_leaves,))
        _need(leaf_p, torch.int32, "leaf_p", (n_leaves,))
        return n_leaves

    def _out(self, coef, n_leaves, device, accumulate):
        nc = n_coef(self.p_max)
        if coef is None:
            if accumulate:
                raise ValueError("accumulate=True needs an output tensor")
            return torch.empty((n_leaves, nc), dtype=torch.float64, device=device)
        return _need(coef, torch.float64, "coef", (n_leaves, nc))

    def _geom(self, vxyz, idx, nv):
        _need(vxyz, torch.float64, "vxyz")
        _need(idx, torch.int32, "idx")
        if vxyz.dim() != 2 or vxyz.shape[0] != 3:
            raise ValueError("vxyz must be (3, n_vert)")
        if idx.dim() != 2 or idx.shape[0] != nv:
            raise ValueError("idx must be (%d, n_elem)" % nv)
        return vxyz.shape[1], idx.shape[1]

    # ---------------------------------------------------------- elements
    def segments(self, vxyz, idx, sigma, leaf_off, leaf_c, leaf_rho=None, leaf_p=None, coef=None,
                 accumulate=False):
        n_vert, n_elem = self._geom(vxyz, idx, 2)
        _need(sigma, torch.float64, "sigma", (n_elem,))
        n_leaves = self._leaf_args(n_elem, leaf_off, leaf_c, leaf_rho, leaf_p)
        coef = self._out(coef, n_leaves, vxyz.device, accumulate)
        check(lib().q2x_segments(self._h, n_elem, n_vert, _ptr(vxyz), _ptr(idx), _ptr(sigma), n_leaves,
                                 _ptr(leaf_off), _ptr(leaf_c), _ptr(leaf_rho), _ptr(leaf_p), _ptr(coef),
                                 int(bool(accumulate))), self._h)
        return coef

    def tetra(self, vxyz, idx, sigma, leaf_off, leaf_c, leaf_rho=None, leaf_p=None, coef=None,
              accumulate=False):
        n_vert, n_elem = self._geom(vxyz, idx, 4)
        _need(sigma, torch.float64, "sigma", (n_elem,))
        n_leaves = self._leaf_args(n_elem, leaf_off, leaf_c, leaf_rho, leaf_p)
        coef = self._out(coef, n_leaves, vxyz.device, accumulate)
        check(lib().q2x_tetra(self._h, n_elem, n_vert, _ptr(vxyz), _ptr(idx), _ptr(sigma), n_leaves,
                              _ptr(leaf_off), _ptr(leaf_c), _ptr(leaf_rho), _ptr(leaf_p), _ptr(coef),
                              int(bool(accumulate))), self._h)
        return coef

    def triangles(self, vxyz, idx, sigma, leaf_off, leaf_c, leaf_rho=None, leaf_p=None, density="const",
                  single=True, double=False, coef_single=None, coef_double=None, accumulate=False):
        """Single and/or double layer in one pass; returns (coef_single, coef_double)
        with None for a layer not requested."""
        n_vert, n_elem = self._geom(vxyz, idx, 3)
        dens = _DENS[density]
        _need(sigma, torch.float64, "sigma", (n_vert if dens == 1 else n_elem,))
        n_leaves = self._leaf_args(n_elem, leaf_off, leaf_c, leaf_rho, leaf_p)
        cs = self._out(coef_single, n_leaves, vxyz.device, accumulate) if single else None
        cd = self._out(coef_double, n_leaves, vxyz.device, accumulate) if double else None
        if cs is None and cd is None:
            raise ValueError("request at least one layer")
        check(lib().q2x_triangles(self._h, n_elem, n_vert, _ptr(vxyz), _ptr(idx), dens, _ptr(sigma), n_leaves,
                                  _ptr(leaf_off), _ptr(leaf_c), _ptr(leaf_rho), _ptr(leaf_p), _ptr(cs), _ptr(cd),
                                  int(bool(accumulate))), self._h)
        return cs, cd

    def triangles_single_vjp(self, vxyz, idx, sigma, leaf_off, leaf_c, grad_coef, leaf_rho=None, leaf_p=None,
                             grad_vxyz=None, grad_sigma=True):
        """Adjoint of triangles(single layer, constant density): returns
        (d loss/d vxyz, d loss/d sigma or None) for loss = sum(grad_coef * coef).
        grad_vxyz, if given, is accumulated into (+=)."""
        n_vert, n_elem = self._geom(vxyz, idx, 3)
        _need(sigma, torch.float64, "sigma", (n_elem,))
        n_leaves = self._leaf_args(n_elem, leaf_off, leaf_c, leaf_rho, leaf_p)
        _need(grad_coef, torch.float64, "grad_coef", (n_leaves, n_coef(self.p_max)))
        if grad_vxyz is None:
            grad_vxyz = torch.zeros_like(vxyz)
        _need(grad_vxyz, torch.float64, "grad_vxyz", tuple(vxyz.shape))
        gs = torch.empty_like(sigma) if grad_sigma is True else grad_sigma
        check(lib().q2x_triangles_single_vjp(self._h, n_elem, n_vert, _ptr(vxyz), _ptr(idx), _ptr(sigma), n_leaves,
                                             _ptr(leaf_off), _ptr(leaf_c), _ptr(leaf_rho), _ptr(leaf_p),
                                             _ptr(grad_coef), _ptr(grad_vxyz), _ptr(gs)), self._h)
        return grad_vxyz, gs

    def leaf_reduce(self, elem, p, leaf_off, coef=None, accumulate=False):
        _need(elem, torch.float64, "elem")
        _need(leaf_off, torch.int64, "leaf_off")
        nc = n_coef(p)
        if elem.dim() != 2 or elem.shape[1] != nc:
            raise ValueError("elem must be (n_elem, (p+1)^2)")
        n_leaves = leaf_off.shape[0] - 1
        if coef is None:
            if accumulate:
                raise ValueError("accumulate=True needs an output tensor")
            coef = torch.empty((n_leaves, nc), dtype=torch.float64, device=elem.device)
        _need(coef, torch.float64, "coef", (n_leaves, nc))
        check(lib().q2x_leaf_reduce(self._h, elem.shape[0], int(p), _ptr(elem), n_leaves, _ptr(leaf_off),
                                    _ptr(coef), int(bool(accumulate))), self._h)
        return coef


    def translate(self, src_coef, src_c, dst_off, dst_c, dst_coef=None, accumulate=False, p=None):
        """Expansions about src_c (rows of src_coef) translated to the
        destination centres dst_c and summed per destination over the CSR
        ranges dst_off (q2x_translate).  Returns dst_coef (n_dst, (p+1)^2)."""
        p = self.p_max if p is None else int(p)
        nc = n_coef(p)
        _need(src_coef, torch.float64, "src_coef")
        if src_coef.dim() != 2 or src_coef.shape[1] != nc:
            raise ValueError("src_coef must be (n_src, (p+1)^2)")
        n_src = src_coef.shape[0]
        _need(src_c, torch.float64, "src_c", (3, n_src))
        _need(dst_off, torch.int64, "dst_off")
        n_dst = dst_off.shape[0] - 1
        _need(dst_c, torch.float64, "dst_c", (3, n_dst))
        if dst_coef is None:
            if accumulate:
                raise ValueError("accumulate=True needs an output tensor")
            dst_coef = torch.empty((n_dst, nc), dtype=torch.float64, device=src_coef.device)
        _need(dst_coef, torch.float64, "dst_coef", (n_dst, nc))
        check(lib().q2x_translate(self._h, p, n_src, _ptr(src_coef), _ptr(src_c), n_dst, _ptr(dst_off),
                                  _ptr(dst_c), _ptr(dst_coef), int(bool(accumulate))), self._h)
        return dst_coef

    def translation_rows(self, t, p=None, out=None):
        """R_n^m(t) for the translation vectors t (3, n_t), packed like the
        coefficients, as (n_t, (p+1)^2) (q2x_translation_rows)."""
        p = self.p_max if p is None else int(p)
        _need(t, torch.float64, "t")
        if t.dim() != 2 or t.shape[0] != 3:
            raise ValueError("t must be (3, n_t)")
        n_t = t.shape[1]
        if out is None:
            out = torch.empty((n_t, n_coef(p)), dtype=torch.float64, device=t.device)
        _need(out, torch.float64, "out", (n_t, n_coef(p)))
        check(lib().q2x_translation_rows(self._h, p, n_t, _ptr(t), _ptr(out)), self._h)
        return out

    def translate_rt(self, src_coef, rt, t_idx, dst_off, dst_coef=None, accumulate=False, p=None):
        """translate() with R(t) from precomputed rows: source s uses row
        t_idx[s] of rt (q2x_translate_rt)."""
        p = self.p_max if p is None else int(p)
        nc = n_coef(p)
        _need(src_coef, torch.float64, "src_coef")
        if src_coef.dim() != 2 or src_coef.shape[1] != nc:
            raise ValueError("src_coef must be (n_src, (p+1)^2)")
        n_src = src_coef.shape[0]
        _need(rt, torch.float64, "rt")
        if rt.dim() != 2 or rt.shape[1] != nc:
            raise ValueError("rt must be (n_t, (p+1)^2)")
        _need(t_idx, torch.int32, "t_idx", (n_src,))
        _need(dst_off, torch.int64, "dst_off")
        n_dst = dst_off.shape[0] - 1
        if dst_coef is None:
            if accumulate:
                raise ValueError("accumulate=True needs an output tensor")
            dst_coef = torch.empty((n_dst, nc), dtype=torch.float64, device=src_coef.device)
        _need(dst_coef, torch.float64, "dst_coef", (n_dst, nc))
        check(lib().q2x_translate_rt(self._h, p, n_src, _ptr(src_coef), rt.shape[0], _ptr(rt), _ptr(t_idx), n_dst,
                                     _ptr(dst_off), _ptr(dst_coef), int(bool(accumulate))), self._h)
        return dst_coef


    def evaluate(self, coef, exp_c, tgt, tgt_off=None, exp_idx=None, out=None, accumulate=False, p=None):
        """Far-field potential at the targets tgt (3, n_tgt) of the expansions
        (coef rows about exp_c) listed per target by the CSR tgt_off/exp_idx
        (default: every target evaluates every expansion).  q2x_evaluate."""
        p = self.p_max if p is None else int(p)
        nc = n_coef(p)
        _need(coef, torch.float64, "coef")
        if coef.dim() != 2 or coef.shape[1] != nc:
            raise ValueError("coef must be (n_exp, (p+1)^2)")
        n_exp = coef.shape[0]
        _need(exp_c, torch.float64, "exp_c", (3, n_exp))
        _need(tgt, torch.float64, "tgt")
        if tgt.dim() != 2 or tgt.shape[0] != 3:
            raise ValueError("tgt must be (3, n_tgt)")
        n_tgt = tgt.shape[1]
        if tgt_off is None:
            tgt_off = torch.arange(n_tgt + 1, dtype=torch.int64, device=tgt.device) * n_exp
            exp_idx = torch.arange(n_exp, dtype=torch.int64, device=tgt.device).repeat(n_tgt)
        _need(tgt_off, torch.int64, "tgt_off", (n_tgt + 1,))
        _need(exp_idx, torch.int64, "exp_idx")
        if out is None:
            if accumulate:
                raise ValueError("accumulate=True needs an output tensor")
            out = torch.empty(n_tgt, dtype=torch.float64, device=tgt.device)
        _need(out, torch.float64, "out", (n_tgt,))
        check(lib().q2x_evaluate(self._h, p, n_exp, _ptr(coef), _ptr(exp_c), n_tgt, _ptr(tgt), _ptr(tgt_off),
                                 _ptr(exp_idx), _ptr(out), int(bool(accumulate))), self._h)
        return out


    def leaf_reduce_weighted(self, elem, p, leaf_off, weights, coef=None, accumulate=False):
        """coef[j][L] (+)= sum_{e in leaf L} weights[j][e] elem[e] for the n_w
        rows of weights (n_w <= 4), in element order (q2x_leaf_reduce_weighted).
        weights (n_w, n_elem) and coef (n_w, n_leaves, (p+1)^2) may be views
        whose rows are strided (e.g. a column range of a larger array)."""
        _need(elem, torch.float64, "elem")
        _need(leaf_off, torch.int64, "leaf_off")
        nc = n_coef(p)
        if elem.dim() != 2 or elem.shape[1] != nc:
            raise ValueError("elem must be (n_elem, (p+1)^2)")
        n_elem, n_leaves = elem.shape[0], leaf_off.shape[0] - 1
        if not (isinstance(weights, torch.Tensor) and weights.is_cuda and weights.dtype == torch.float64
                and weights.dim() == 2 and weights.shape[1] == n_elem and 1 <= weights.shape[0] <= 4
                and (weights.stride(1) == 1 or n_elem <= 1)):
            raise ValueError("weights must be a CUDA float64 (n_w <= 4, n_elem) array with unit column stride")
        n_w = weights.shape[0]
        if coef is None:
            if accumulate:
                raise ValueError("accumulate=True needs an output tensor")
            coef = torch.empty((n_w, n_leaves, nc), dtype=torch.float64, device=elem.device)
        if not (isinstance(coef, torch.Tensor) and coef.is_cuda and coef.dtype == torch.float64
                and tuple(coef.shape) == (n_w, n_leaves, nc) and coef.stride(2) == 1 and coef.stride(1) == nc):
            raise ValueError("coef must be a CUDA float64 (n_w, n_leaves, (p+1)^2) array with dense rows")
        check(lib().q2x_leaf_reduce_weighted(self._h, n_elem, int(p), _ptr(elem), n_w, _ptr(weights),
                                             weights.stride(0), n_leaves, _ptr(leaf_off), _ptr(coef),
                                             coef.stride(0), int(bool(accumulate))), self._h)
        return coef

    def segments_vector(self, vxyz, idx, current, leaf_off, leaf_c, leaf_rho=None, leaf_p=None, coef3=None,
                        accumulate=False):
        """Coefficients of the three components of a vector line density
        (current (3, n_elem), constant per segment), as (3, n_leaves,
        (p+1)^2) (q2x_segments_vector: one recursion pass for all three
        components, Eq. (st3))."""
        n_vert, n_elem = self._geom(vxyz, idx, 2)
        _need(current, torch.float64, "current", (3, n_elem))
        if leaf_off is None:
            raise ValueError("segments_vector needs leaf_off")
        n_leaves = self._leaf_args(n_elem, leaf_off, leaf_c, leaf_rho, leaf_p)
        nc = n_coef(self.p_max)
        if coef3 is None:
            if accumulate:
                raise ValueError("accumulate=True needs an output tensor")
            coef3 = torch.empty((3, n_leaves, nc), dtype=torch.float64, device=vxyz.device)
        _need(coef3, torch.float64, "coef3", (3, n_leaves, nc))
        check(lib().q2x_segments_vector(self._h, n_elem, n_vert, _ptr(vxyz), _ptr(idx), _ptr(current), n_leaves,
                                        _ptr(leaf_off), _ptr(leaf_c), _ptr(leaf_rho), _ptr(leaf_p), _ptr(coef3),
                                        int(bool(accumulate))), self._h)
        return coef3

    def evaluate_curl(self, coef3, exp_c, tgt, tgt_off=None, exp_idx=None, out=None, accumulate=False, p=None):
        """curl of the far field of vector expansions coef3 (3, n_exp,
        (p+1)^2) about exp_c at the targets (3, n_tgt): the Biot-Savart field
        H of Eq. (st3) for line currents (q2x_evaluate_curl).  Returns (3, n_tgt)."""
        p = self.p_max if p is None else int(p)
        nc = n_coef(p)
        _need(coef3, torch.float64, "coef3")
        if coef3.dim() != 3 or coef3.shape[0] != 3 or coef3.shape[2] != nc:
            raise ValueError("coef3 must be (3, n_exp, (p+1)^2)")
        n_exp = coef3.shape[1]
        _need(exp_c, torch.float64, "exp_c", (3, n_exp))
        _need(tgt, torch.float64, "tgt")
        if tgt.dim() != 2 or tgt.shape[0] != 3:
            raise ValueError("tgt must be (3, n_tgt)")
        n_tgt = tgt.shape[1]
        if tgt_off is None:
            tgt_off = torch.arange(n_tgt + 1, dtype=torch.int64, device=tgt.device) * n_exp
            exp_idx = torch.arange(n_exp, dtype=torch.int64, device=tgt.device).repeat(n_tgt)
        _need(tgt_off, torch.int64, "tgt_off", (n_tgt + 1,))
        _need(exp_idx, torch.int64, "exp_idx")
        if out is None:
            if accumulate:
                raise ValueError("accumulate=True needs an output tensor")
            out = torch.empty((3, n_tgt), dtype=torch.float64, device=tgt.device)
        _need(out, torch.float64, "out", (3, n_tgt))
        check(lib().q2x_evaluate_curl(self._h, p, n_exp, _ptr(coef3), _ptr(exp_c), n_tgt, _ptr(tgt),
                                      _ptr(tgt_off), _ptr(exp_idx), _ptr(out), int(bool(accumulate))), self._h)
        return out

    def nearfield(self, kind, vxyz, idx, sigma, tgt, tgt_off=None, elem_idx=None, layer=0, out=None,
                  accumulate=False):
        """Exact potentials (1/4pi) sigma_e int_e G of the listed elements at
        the targets (3, n_tgt); default: every target, every element
        (q2x_nearfield).  kind: "segment" | "triangle" | "tetra"."""
        k = {"segment": 0, "triangle": 1, "tetra": 2}[kind]
        n_vert, n_elem = self._geom(vxyz, idx, k + 2)
        _need(sigma, torch.float64, "sigma", (n_elem,))
        _need(tgt, torch.float64, "tgt")
        if tgt.dim() != 2 or tgt.shape[0] != 3:
            raise ValueError("tgt must be (3, n_tgt)")
        n_tgt = tgt.shape[1]
        if tgt_off is None:
            tgt_off = torch.arange(n_tgt + 1, dtype=torch.int64, device=tgt.device) * n_elem
            elem_idx = torch.arange(n_elem, dtype=torch.int64, device=tgt.device).repeat(n_tgt)
        _need(tgt_off, torch.int64, "tgt_off", (n_tgt + 1,))
        _need(elem_idx, torch.int64, "elem_idx")
        if out is None:
            if accumulate:
                raise ValueError("accumulate=True needs an output tensor")
            out = torch.empty(n_tgt, dtype=torch.float64, device=tgt.device)
        _need(out, torch.float64, "out", (n_tgt,))
        check(lib().q2x_nearfield(self._h, k, int(layer), n_elem, n_vert, _ptr(vxyz), _ptr(idx), _ptr(sigma), n_tgt,
                                  _ptr(tgt), _ptr(tgt_off), _ptr(elem_idx), _ptr(out), int(bool(accumulate))),
              self._h)
        return out

    def galerkin_triangles(self, vxyz, idx, weights, leaf_off, leaf_c, leaf_rho=None, sigma=None, layer=0,
                           out=None):
        """Per-triangle contraction sum_c weights[L][c] P_c(e) of each
        triangle's own packed coefficients (q2x_galerkin_triangles); with a
        MOMENT plan and local_expansion_weights(L) it integrates the local
        expansion over each triangle (layer 0) or its normal derivative
        (layer 1).  sigma: per-triangle weights (default 1)."""
        n_vert, n_elem = self._geom(vxyz, idx, 3)
        n_leaves = self._leaf_args(n_elem, leaf_off, leaf_c, leaf_rho, None)
        _need(weights, torch.float64, "weights", (n_leaves, n_coef(self.p_max)))
        if sigma is None:
            sigma = torch.ones(n_elem, dtype=torch.float64, device=vxyz.device)
        _need(sigma, torch.float64, "sigma", (n_elem,))
        if out is None:
            out = torch.empty(n_elem, dtype=torch.float64, device=vxyz.device)
        _need(out, torch.float64, "out", (n_elem,))
        check(lib().q2x_galerkin_triangles(self._h, n_elem, n_vert, _ptr(vxyz), _ptr(idx), _ptr(sigma), n_leaves,
                                           _ptr(leaf_off), _ptr(leaf_c), _ptr(leaf_rho), int(layer), _ptr(weights),
                                           _ptr(out)), self._h)
        return out


def local_expansion_weights(L_re, L_im, p):
    """Packed Galerkin weights of local expansions phi(y) = sum L_n^m R_n^m(y-c)
    given by the real and imaginary parts of L_n^m for m >= 0 (tensors
    (..., (p+1)^2) indexed k = n*n+n+m with m >= 0 used): L_n^0 at (n, 0),
    2 Re L_n^m at (n, m), -2 Im L_n^m at (n, -m)."""
    w = torch.zeros_like(L_re)
    for n in range(p + 1):
        k0 = n * n + n
        w[..., k0] = L_re[..., k0]
        for m in range(1, n + 1):
            w[..., k0 + m] = 2.0 * L_re[..., k0 + m]
            w[..., k0 - m] = -2.0 * L_im[..., k0 + m]
    return w


PEAK_KINDS = {"dfma": 0, "ffma": 1, "ffma2": 2}


def alu_peak_probe(kind: str, iters: int, sink, stream=None) -> float:
    """Launch the library's FMA-chain probe (q2x_alu_peak_probe) on `stream`
    (default: the current stream); returns the flops the launch performs.
    `sink` is a one-element float64 CUDA tensor."""
    _need(sink, torch.float64, "sink")
    if stream is None:
        stream = torch.cuda.current_stream()
    flops = ctypes.c_double(0.0)
    check(lib().q2x_alu_peak_probe(PEAK_KINDS[kind], int(iters), _ptr(sink), ctypes.c_void_p(stream.cuda_stream),
                                   ctypes.byref(flops)))
    return float(flops.value)


def problem_to_device(prob: dict, device="cuda") -> dict:
    """Copy a workloads-style problem dict (numpy arrays) to device tensors."""
    out = {}
    for k, v in prob.items():
        if hasattr(v, "dtype") and hasattr(v, "shape"):
            out[k] = torch.from_numpy(v).to(device)
        else:
            out[k] = v
    return out


class Batch:
    """A ragged mixed-kind batch (q2x_batch_*): per-leaf degrees, several
    element kinds summed into the same leaves, run as one CUDA-graph replay.

    kinds: segments / triangles / tetra, each a dict with torch CUDA tensors
    vxyz (3, n_vert) f64, idx (k, n_elem) i32, sigma f64, leaf_off (n_leaves+1)
    i64 and, for triangles, density ("const" | "linear"); None to omit.
    The tensors are referenced, not copied: keep them alive and unchanged in
    shape while the batch exists."""

    def __init__(self, plan: Plan, leaf_c, leaf_rho=None, leaf_p=None, coef=None, segments=None, triangles=None,
                 tetra=None, accumulate=False, tile_elems=0):
        from ._lib import BatchDesc
        n_leaves = leaf_c.shape[1]
        _need(leaf_c, torch.float64, "leaf_c", (3, n_leaves))
        _need(leaf_rho, torch.float64, "leaf_rho", (n_leaves,))
        _need(leaf_p, torch.int32, "leaf_p", (n_leaves,))
        self.plan = plan
        self.coef = plan._out(coef, n_leaves, leaf_c.device, accumulate)
        self._keep = [leaf_c, leaf_rho, leaf_p, self.coef]
        d = BatchDesc()
        d.n_leaves = n_leaves
        d.leaf_c = leaf_c.data_ptr()
        d.leaf_rho = leaf_rho.data_ptr() if leaf_rho is not None else None
        d.leaf_p = leaf_p.data_ptr() if leaf_p is not None else None
        d.coef = self.coef.data_ptr()
        d.accumulate = int(bool(accumulate))
        for name, nv, kd in (("segments", 2, segments), ("triangles", 3, triangles), ("tetra", 4, tetra)):
            el = getattr(d, name)
            if kd is None:
                el.n_elem = 0
                continue
            n_vert, n_elem = plan._geom(kd["vxyz"], kd["idx"], nv)
            dens = _DENS[kd.get("density", "const")] if name == "triangles" else 0
            _need(kd["sigma"], torch.float64, name + ".sigma", (n_vert if dens == 1 else n_elem,))
            _need(kd["leaf_off"], torch.int64, name + ".leaf_off", (n_leaves + 1,))
            el.n_elem, el.n_vert = n_elem, n_vert
            el.vxyz, el.idx, el.sigma = kd["vxyz"].data_ptr(), kd["idx"].data_ptr(), kd["sigma"].data_ptr()
            el.leaf_off, el.density = kd["leaf_off"].data_ptr(), dens
            self._keep += [kd["vxyz"], kd["idx"], kd["sigma"], kd["leaf_off"]]
        self._desc = d
        h = ctypes.c_void_p()
        check(lib().q2x_batch_build(plan.handle, ctypes.byref(d), int(tile_elems), ctypes.byref(h)), plan.handle)
        self._h = h

    def run(self):
        """Replay the batch's CUDA graph on the plan's stream (asynchronous)."""
        check(lib().q2x_batch_run(self._h), self.plan.handle)
        return self.coef

    def info(self):
        nt, ns, te = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
        check(lib().q2x_batch_info(self._h, ctypes.byref(nt), ctypes.byref(ns), ctypes.byref(te)))
        return dict(tiles=nt.value, slots=ns.value, tile_elems=te.value)

    def close(self):
        if getattr(self, "_h", None):
            lib().q2x_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def tune(plan: Plan, candidates=(64, 128, 256, 512, 1024, 2048), reps=5, **kwargs):
        """Time every candidate tile size; returns (best, {candidate: ms})."""
        probe = Batch(plan, tile_elems=candidates[0], **kwargs)  # validates and holds the descriptor
        cand = (ctypes.c_int * len(candidates))(*candidates)
        ms = (ctypes.c_float * len(candidates))()
        best = ctypes.c_int()
        check(lib().q2x_batch_tune(plan.handle, ctypes.byref(probe._desc), cand, len(candidates), int(reps),
                                   ctypes.byref(best), ms), plan.handle)
        probe.close()
        return int(best.value), {c: float(t) for c, t in zip(candidates, ms)}


def autotuned_tile(plan: Plan, key: str, cache_path: str, **batch_kwargs) -> int:
    """Tile size for a batch from the JSON autotune table at cache_path, keyed
    by device name, precision, p_max and `key` (the caller's description of the
    workload shape); tunes and records it when missing."""
    import json
    import os
    dev = torch.cuda.get_device_name()
    full = "%s|prec=%d|p=%d|%s" % (dev, plan.precision, plan.p_max, key)
    table = {}
    if os.path.exists(cache_path):
        with open(cache_path) as f:
            table = json.load(f)
    if full in table:
        return int(table[full]["tile_elems"])
    best, times = Batch.tune(plan, **batch_kwargs)
    table[full] = {"tile_elems": best, "ms": {str(k): v for k, v in times.items()}}
    os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
    tmp = cache_path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, cache_path)
    return best


class TrianglesSingle(torch.autograd.Function):
    """coef = Q2X single layer of constant-density triangles, differentiable in
    the vertex coordinates and the densities (backward: the library's adjoint
    kernel, q2x_triangles_single_vjp)."""

    @staticmethod
    def forward(ctx, vxyz, sigma, plan, idx, leaf_off, leaf_c, leaf_rho, leaf_p):
        coef, _ = plan.triangles(vxyz.detach(), idx, sigma.detach(), leaf_off, leaf_c, leaf_rho, leaf_p,
                                 density="const", single=True)
        ctx.save_for_backward(vxyz, sigma)
        ctx.plan = plan
        ctx.rest = (idx, leaf_off, leaf_c, leaf_rho, leaf_p)
        return coef

    @staticmethod
    def backward(ctx, grad_coef):
        vxyz, sigma = ctx.saved_tensors
        idx, leaf_off, leaf_c, leaf_rho, leaf_p = ctx.rest
        gv, gs = ctx.plan.triangles_single_vjp(vxyz.detach(), idx, sigma.detach(), leaf_off, leaf_c,
                                               grad_coef.contiguous(), leaf_rho, leaf_p)
        return gv, gs, None, None, None, None, None, None


def triangles_single(vxyz, sigma, plan, idx, leaf_off, leaf_c, leaf_rho=None, leaf_p=None):
    """Differentiable single-layer Q2X of constant-density triangles."""
    return TrianglesSingle.apply(vxyz, sigma, plan, idx, leaf_off, leaf_c, leaf_rho, leaf_p)
