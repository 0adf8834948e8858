// Explicit instantiations of the element kernel: f64, tetrahedra.
#include "q2x_kernels.cuh"
Q2X_FOR_BINS(Q2X_INSTANTIATE, double, q2x::KIND_TET, q2x::DENS_CONST, 1)
