// Sweep kernel instantiations that record the per-layer spin expectations
// <Z_q> (T_ZEXP sweeps, variant V_ZFULL): complex64 and complex128 forward.
#include "qs_sweep.cuh"

namespace qs {

#define QS_ZX(DT, Real, K_, R_, KIND)                                                         \
    if (dtype == DT && kind == KIND) {                                                        \
        if (grid_only) return grid_cfg<Real, K_, R_, 1, KIND, V_ZFULL>();                     \
        *status = launch_sweep_cfg<Real, K_, R_, 1, KIND, V_ZFULL>(*L, grid, st);             \
        return 0;                                                                             \
    }

int sweep_zexp(int dtype, int kind, bool grid_only, const SweepLaunch* L, int grid, cudaStream_t st,
               cudaError_t* status) {
    QS_ZX(0, float, 13, 6, 0)
    QS_ZX(0, float, 13, 6, 1)
    QS_ZX(0, float, 13, 6, 2)
    QS_ZX(1, double, 12, 5, 0)
    QS_ZX(1, double, 12, 5, 1)
    if (status) *status = cudaErrorInvalidValue;
    return 0;
}

}  // namespace qs
