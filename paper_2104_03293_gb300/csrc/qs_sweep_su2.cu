// Sweep kernel instantiations whose layers apply general single-spin
// unitaries (variant V_SU2, the x + z exponentials of Eq. AQA4):
// complex64 and complex128 forward.
#include "qs_sweep.cuh"

namespace qs {

#define QS_SU(DT, Real, K_, R_, KIND)                                                         \
    if (dtype == DT && kind == KIND) {                                                        \
        if (grid_only) return grid_cfg<Real, K_, R_, 1, KIND, V_SU2>();                       \
        *status = launch_sweep_cfg<Real, K_, R_, 1, KIND, V_SU2>(*L, grid, st);               \
        return 0;                                                                             \
    }

int sweep_su2(int dtype, int kind, bool grid_only, const SweepLaunch* L, int grid, cudaStream_t st,
              cudaError_t* status) {
    QS_SU(0, float, 13, 6, 0)
    QS_SU(0, float, 13, 6, 1)
    QS_SU(0, float, 13, 6, 2)
    QS_SU(1, double, 12, 5, 0)
    QS_SU(1, double, 12, 5, 1)
    if (status) *status = cudaErrorInvalidValue;
    return 0;
}

}  // namespace qs
