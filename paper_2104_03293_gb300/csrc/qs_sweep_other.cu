// Sweep kernel instantiations: complex64 adjoint and complex128 (all FULL).
#include "qs_sweep.cuh"

namespace qs {

#define QS_OTH(DT, AD, Real, K_, R_, NA_, KIND)                                               \
    if (dtype == DT && adjoint == AD && kind == KIND) {                                       \
        if (grid_only) return grid_cfg<Real, K_, R_, NA_, KIND, V_FULL>();                    \
        *status = launch_sweep_cfg<Real, K_, R_, NA_, KIND, V_FULL>(*L, grid, st);            \
        return 0;                                                                             \
    }

int sweep_other(int dtype, int adjoint, int kind, bool grid_only, const SweepLaunch* L, int grid, cudaStream_t st,
                cudaError_t* status) {
    QS_OTH(0, 1, float, 13, 5, 2, 0)
    QS_OTH(0, 1, float, 13, 5, 2, 1)
    QS_OTH(0, 1, float, 13, 5, 2, 2)
    QS_OTH(1, 0, double, 12, 5, 1, 0)
    QS_OTH(1, 0, double, 12, 5, 1, 1)
    QS_OTH(1, 1, double, 12, 4, 2, 0)
    QS_OTH(1, 1, double, 12, 4, 2, 1)
    if (status) *status = cudaErrorInvalidValue;
    return 0;
}

}  // namespace qs
