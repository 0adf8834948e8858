"""Algorithmic operation counts and peaks for the roofline of the Q2X kernels.

The count follows the kernels' formulation of the tilde recursion (Eq. (rec10)
and its relatives): one level update of (n, m) from the row of degree n-1 is

  m > 0:  re = X (b_r - a_r) + Y (b_i + a_i) - z c_r + s_r
          im = X (b_i - a_i) - Y (b_r + a_r) - z c_i + s_i
  m = 0:  re = 2 X b_r + 2 Y b_i - z c_r + s_r

with a = x^{m-1}, b = x^{m+1}, c = x^m of degree n-1.  Only terms whose operand
exists (|order| <= n-1) are counted: 4 adds + 4 FMAs for the xi/eta pair when
both a and b exist, 4 FMAs when only a does, 2 FMAs for the z term, 2 FMAs
for m = 0's eta term; the source rides in the FMA addend.  FMA = 2 flops.
The leaf reduction adds one flop per element and output column.

The FP64 kernels compute the point level (level 0) by a recursion over the
order at fixed degree instead of the stencil (`point="order"`, counted by
`point_level_order_flops`); the FP32 kernels use the stencil for every level."""
from __future__ import annotations

# GB300 (recipe figures): 152 SMs, 2070 MHz maximum SM clock; FP32: 128 lanes
# per SM; FP64 nominal 1.25 TFLOP/s, i.e. 2 FP64 FMA lanes per SM per clock.
N_SM = 152
CLOCK_HZ = 2.070e9
PEAK_FP32_FLOPS = N_SM * 128 * 2 * CLOCK_HZ   # 80.5 TFLOP/s
PEAK_FP64_FLOPS = N_SM * 2 * 2 * CLOCK_HZ     # 1.26 TFLOP/s


def stencil_flops(n: int, m: int) -> int:
    if n == 0:
        return 0
    if m == 0:
        return (4 if n - 1 >= 1 else 0) + 2
    has_b = m + 1 <= n - 1
    has_c = m <= n - 1
    return (12 if has_b else 8) + (4 if has_c else 0)


def level_flops(p: int) -> int:
    return sum(stencil_flops(n, m) for n in range(p + 1) for m in range(n + 1))


def point_level_order_flops(p: int) -> int:
    """Flops per element of the FP64 kernels' point level: the element's row
    w_m = seed (-xi)^m (a complex multiply, 6 flops, per m >= 1) and |xi|^2
    (3 flops); per degree n >= 1, Q_n^{n-1} = -n z (1 flop); per entry, none at
    m = n (T_n^n = w_n), the order recursion at m <= n - 2 (three multiplies
    and one FMA, 5 flops) and the product w_m Q_n^m at m <= n - 1 (2 flops,
    1 at m = 0 where w_0 is real)."""
    f = 6 * p + 3
    for n in range(1, p + 1):
        f += 1
        for m in range(n):
            f += (1 if m == 0 else 2) + (5 if m <= n - 2 else 0)
    return f


def element_flops(kind: str, density: str = "const", layers=("single",), p: int = 12,
                  point: str = "stencil") -> int:
    """Flops per element of one Q2X pass (recursion + double layer + reduction).
    point: "stencil" (FP32 kernels) or "order" (FP64 kernels) for level 0."""
    L = level_flops(p)
    L0 = L if point == "stencil" else point_level_order_flops(p)
    entries = sum(n + 1 for n in range(p + 1))
    if kind == "segment":
        f = L0 + L
    elif kind == "tetra":
        f = L0 + 3 * L
    elif density == "const":
        f = L0 + 2 * L
    else:
        # 5 levels; E source c2 q + s3 j (1 mul + 1 fma per part) and Iw source
        # s1 i + E (1 fma per part); m = 0 entries are real
        f = L0 + 4 * L + 6 * entries - 3 * (p + 1) + 4 * entries - 2 * (p + 1) + (p + 1)
    if "double" in layers:
        f += L
    f += len(layers) * (p + 1) ** 2
    return f


def vjp_flops(p: int = 12) -> int:
    """Flops per triangle of the single-layer adjoint (q2x_tri_vjp_kernel):
    seven chain levels (q, j, i and E, Iw for the barycentric weights of
    vertices 2 and 3), and per (n, m >= 0) ten contractions with the folded
    weights (S_U and the three directions of the three vertices; 4 flops
    each) plus the e_x / e_y neighbour combinations of the three weighted
    rows (8 adds each)."""
    entries = sum(n + 1 for n in range(p + 1))
    return 7 * level_flops(p) + 10 * 4 * entries + 3 * 8 * entries
