// Host-side planning declarations (no CUDA dependencies).
#pragma once

#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include "qs_internal.h"

namespace qs {

struct IsingInt {
    int n = 0, shift = 0;
    std::vector<int32_t> h, ei, ej, J;  // weights scaled by 2^shift
    int64_t bound = 0;                   // sum |h| + sum |J| (scaled)
};

// 0 = ok, 1 = QS_EINVAL, 5 = QS_ENOTINT; err receives the reason.
int validate_ising(int n, const double* hfield, int n_edges, const int32_t* edges, const double* J, IsingInt& out,
                   std::string& err);

struct Shape {
    int K, c, g0, nt;
    int64_t ntiles;
};

struct PlanSweep {
    int shape = 0;
    int nr = 0;
    int flags = 0;
    SweepRound r[kMaxRounds];
};

std::vector<Shape> make_shapes(int nphys, const KernelCfg& cfg);
void shape_regq(const Shape& s, int R, int g, int* regq);
int num_layouts(int K, int R);
std::vector<PlanSweep> plan_forward(int S, int p, bool gen);
std::vector<PlanSweep> plan_reverse(const std::vector<PlanSweep>& fwd, const std::vector<Shape>& shapes, int p);
int count_sweeps(int nphys, int dtype, int p);

}  // namespace qs
