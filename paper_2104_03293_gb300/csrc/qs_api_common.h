// Host-side helpers shared by the single-state and batched C ABI.
#pragma once

#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "qs_internal.h"
#include "qs_plan.h"

namespace qs {

int set_error(int code, const char* fmt, ...);
int cuda_error(cudaError_t e, const char* where);

// Owned device allocation that only grows.
struct DevBuf {
    void* ptr = nullptr;
    size_t cap = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    DevBuf(DevBuf&& o) noexcept : ptr(o.ptr), cap(o.cap) { o.ptr = nullptr; o.cap = 0; }
    DevBuf& operator=(DevBuf&& o) noexcept {
        if (this != &o) { release(); ptr = o.ptr; cap = o.cap; o.ptr = nullptr; o.cap = 0; }
        return *this;
    }
    ~DevBuf() { release(); }
    int reserve(size_t bytes);
    void release();
};

// Pinned staging buffer + device copy; waits for the previous upload to have
// been consumed before the staging buffer is rewritten.
struct Uploader {
    void* host = nullptr;
    size_t host_cap = 0;
    cudaEvent_t ev = nullptr;
    DevBuf dev;
    Uploader() = default;
    Uploader(const Uploader&) = delete;
    Uploader& operator=(const Uploader&) = delete;
    ~Uploader();
    int upload(const void* src, size_t bytes, cudaStream_t st);
};

// One Ising instance on the device: cost programs per tile shape and layout
// for the forward and the adjoint kernel configurations, the enumeration
// program, the flat term list of the plain path, and the ground-state data.
struct Instance {
    bool valid = false;
    int n = 0, nphys = 0, dtype = 0, shift = 0;
    int64_t cmin = 0, cmax = 0, argmin = 0, count = 0;
    int cost_lo = 0, range = 1;
    std::vector<Shape> shapes[2];                      // [forward, adjoint]
    size_t prog_off[2][kMaxShapes][kMaxLayouts] = {};  // layout programs (sweep_kernel layouts), int32 offsets
    size_t tprog_off[2][kMaxShapes] = {};              // tile programs of the shapes
    size_t prog_pair[kMaxShapes][2] = {};              // packed-pair layouts (forward shapes)
    size_t prog_pair_adj[kMaxShapes][3] = {};          // packed-pair adjoint layouts (adjoint shapes)
    PairQ pair_q[kMaxShapes] = {};                     // host copies of the packed-pair forward Q tables
    PairAdjQ pair_adj_q[kMaxShapes] = {};              // and of the adjoint ones
    size_t enum_off = 0, plain_off = 0;
    int plain_nf = 0, plain_ne = 0, plain_const0 = 0;
    DevBuf progs;
    const int32_t* prog(size_t off) const { return reinterpret_cast<const int32_t*>(progs.ptr) + off; }
    int set(int n, int nphys, int dtype, const double* hfield, int n_edges, const int32_t* edges, const double* J,
            cudaStream_t st, DevBuf& enum_scratch, ShapeRule rule = ShapeRule{});
};

}  // namespace qs
