// Dispatch of the sweep kernel (templates in qs_sweep.cuh; instantiations in
// qs_sweep_c64f.cu, qs_sweep_other.cu and qs_sweep_zexp.cu, compiled in parallel).
#include "qs_internal.h"
#include "qs_pair.h"

namespace qs {

int sweep_c64f(int kind, int variant, bool grid_only, const SweepLaunch* L, int grid, cudaStream_t st,
               cudaError_t* status);
int sweep_other(int dtype, int adjoint, int kind, bool grid_only, const SweepLaunch* L, int grid, cudaStream_t st,
                cudaError_t* status);
int sweep_zexp(int dtype, int kind, bool grid_only, const SweepLaunch* L, int grid, cudaStream_t st,
               cudaError_t* status);
int sweep_su2(int dtype, int kind, bool grid_only, const SweepLaunch* L, int grid, cudaStream_t st,
              cudaError_t* status);

cudaError_t launch_sweep(const SweepLaunch& L, int grid, cudaStream_t st) {
    if (L.total_tiles <= 0) return cudaSuccess;
    const int64_t groups = L.total_tiles / (L.group > 0 ? L.group : 1);
    if (grid > groups) grid = (int)groups;
    if (grid < 1) grid = 1;
    if (L.pairc == 1 && !L.adjoint) return launch_sweep_runs(L, grid, st);
    if (L.pairc) return L.adjoint ? launch_sweep_pair_adj(L, grid, st) : launch_sweep_pair(L, grid, st);
    cudaError_t s = cudaErrorInvalidValue;
    if (!L.adjoint && L.variant == V_SU2) sweep_su2(L.dtype, L.kind, false, &L, grid, st, &s);
    else if (!L.adjoint && (L.variant == V_ZFULL || L.variant == V_ZPHASE)) sweep_zexp(L.dtype, L.kind, false, &L, grid, st, &s);
    else if (L.dtype == 0 && !L.adjoint) sweep_c64f(L.kind, L.variant, false, &L, grid, st, &s);
    else sweep_other(L.dtype, L.adjoint, L.kind, false, &L, grid, st, &s);
    return s;
}

int sweep_grid(int dtype, int adjoint, int kind) {
    if (dtype == 0 && !adjoint) return sweep_c64f(kind, 0, true, nullptr, 0, nullptr, nullptr);
    return sweep_other(dtype, adjoint, kind, true, nullptr, 0, nullptr, nullptr);
}

int pair_choice(int dtype, int adjoint, int kind, int c, int variant) {
    if (dtype != 0) return 0;
    if (kind == 0)  // run-structured shape A
        return (c == kRunBits && (adjoint || variant == V_PHASE || variant == V_LEAN)) ? 1 : 0;
    if (kind != 1 || !(c == 2 || c == 3)) return 0;
    return (adjoint || variant == V_PHASE || variant == V_LEAN || variant == V_ZPHASE) ? c : 0;
}

int sweep_variant(int flags, int nrounds, const SweepRound* rounds) {
    if (flags & T_SU2) return V_SU2;
    if (flags & T_ZEXP)  // spin expectations: with or without the other fused work
        return (flags & (T_GEN | T_READOUT | T_WRITE_LAM | T_ADJOINT)) ? V_ZFULL : V_ZPHASE;
    if (flags & (T_GEN | T_READOUT | T_WRITE_LAM | T_ADJOINT)) return 0;  // full
    for (int r = 0; r < nrounds; ++r)
        if (rounds[r].phase_pre || rounds[r].phase_post) return 1;       // phase
    return 2;                                                             // rotations only
}

}  // namespace qs
