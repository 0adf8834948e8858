// The per-group persistent batch kernels, FP32-mixed instances (see q2x_batch.cuh).
#include "q2x_batch.cuh"

namespace q2x {

const BatchGroupFns* batch_group_table_f32()
{
    static const BatchGroupFns t[4][5] = {Q2X_BATCH_FNS_ROW(float, KIND_SEG, DENS_CONST),
                                          Q2X_BATCH_FNS_ROW(float, KIND_TRI, DENS_CONST),
                                          Q2X_BATCH_FNS_ROW(float, KIND_TRI, DENS_LINEAR),
                                          Q2X_BATCH_FNS_ROW(float, KIND_TET, DENS_CONST)};
    return &t[0][0];
}

}  // namespace q2x
