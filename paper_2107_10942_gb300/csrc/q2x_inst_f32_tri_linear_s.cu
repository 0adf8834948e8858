// Explicit instantiations of the element kernel: f32, triangles-linear-density-single-layer.
#include "q2x_kernels.cuh"
Q2X_FOR_BINS(Q2X_INSTANTIATE, float, q2x::KIND_TRI, q2x::DENS_LINEAR, 1)
