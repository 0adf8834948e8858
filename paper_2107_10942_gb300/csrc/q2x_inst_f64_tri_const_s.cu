// Explicit instantiations of the element kernel: f64, triangles-constant-density-single-layer.
#include "q2x_kernels.cuh"
Q2X_FOR_BINS(Q2X_INSTANTIATE, double, q2x::KIND_TRI, q2x::DENS_CONST, 1)
