// Explicit instantiations of the element kernel: f32, tetrahedra.
#include "q2x_kernels.cuh"
Q2X_FOR_BINS(Q2X_INSTANTIATE, float, q2x::KIND_TET, q2x::DENS_CONST, 1)
