// Explicit instantiations of the element kernel: f32, segments carrying a vector density.
#include "q2x_kernels.cuh"
Q2X_FOR_BINS(Q2X_INSTANTIATE, float, q2x::KIND_SEG, q2x::DENS_CONST, 4)
