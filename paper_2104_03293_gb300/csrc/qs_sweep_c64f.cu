// Sweep kernel instantiations: complex64 forward (hot path), every variant.
#include "qs_sweep.cuh"

namespace qs {

#define QS_C64F(KIND, V)                                                                      \
    if (kind == KIND && variant == V) {                                                       \
        if (grid_only) return grid_cfg<float, 13, 6, 1, KIND, V>();                           \
        *status = launch_sweep_cfg<float, 13, 6, 1, KIND, V>(*L, grid, st);                   \
        return 0;                                                                             \
    }

int sweep_c64f(int kind, int variant, bool grid_only, const SweepLaunch* L, int grid, cudaStream_t st,
               cudaError_t* status) {
    QS_C64F(0, V_FULL) QS_C64F(0, V_PHASE) QS_C64F(0, V_LEAN)
    QS_C64F(1, V_FULL) QS_C64F(1, V_PHASE) QS_C64F(1, V_LEAN)
    QS_C64F(2, V_FULL) QS_C64F(2, V_PHASE) QS_C64F(2, V_LEAN)
    if (status) *status = cudaErrorInvalidValue;
    return 0;
}

}  // namespace qs
