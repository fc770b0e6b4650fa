// The plan object behind the opaque pppm_plan handle (shared by the C ABI
// implementation and the correction-network code).
#pragma once

#include <cuda.h>

#include <vector>

#include "internal.cuh"

struct pppm_plan {
    int precision = PPPM_FP32;
    int device = 0;
    double box[3] = {0, 0, 0};
    int mesh[3] = {0, 0, 0};
    int order = 5;
    double beta = 0.0;
    pppm_options opt{};
    pppm::Geo g{};
    pppm::Radix rad[3]{};
    pppm::LineBlocks lb[4]{};  // strided-line FFT passes (LB_*)
    size_t esz = 4;  // sizeof(real)
    // mesh workspace
    double* G64 = nullptr;
    void* G = nullptr;
    void* tw[3] = {nullptr, nullptr, nullptr};
    void* rho = nullptr;
    void* cx[3] = {nullptr, nullptr, nullptr};
    void* fields = nullptr;  // padded (ghosted) field meshes, see FieldLayout
    pppm::FieldLayout flayout{};
    bool potential = false;  // also produce the mesh potential (padded, planar: phi)
    void* phi = nullptr;     // padded potential mesh, Xp x Yp x Zp (allocated on demand)
    bool pdl = true;         // programmatic dependent launch between the kernels of a solve
    long long wait_limit = 1ll << 26;  // polls of the gather's bounded wait for its tile copy
    CUtensorMap fmap;        // 4D TMA descriptor of the padded fields
    bool fmap_ok = false;
    void* partial = nullptr;
    unsigned int* counter = nullptr;
    int* status = nullptr;
    // tiles
    int tileT = 0;
    void* patch = nullptr;
    int* cov_off = nullptr;
    int2* cov_ent = nullptr;
    int4* cov2 = nullptr;  // two-slot cover table (null when some index has more covers)
    int* tile_count = nullptr;
    int2* tiles = nullptr;     // per tile (first slot, end slot) of the tile-ordered site data
    int region_cap = 0;        // slots of a tile's fixed region (0: compact layout only)
    int* region_flag = nullptr;  // device: [0] a region overflowed, [1] blocks of the sort done
    int* spread_ticket = nullptr;  // device: the spread's tile ticket (zero between launches)
    // sites
    int64_t cap = 0;       // per-site arrays in the caller's order
    int64_t slot_cap = 0;  // tile-ordered arrays (srec, scell, sorig) and tile_of/slot_of
    int* tile_of = nullptr;
    int* slot_of = nullptr;
    void* rec = nullptr;
    int* cell = nullptr;
    void* srec = nullptr;
    int* scell = nullptr;
    int* sorig = nullptr;
    // host-API staging
    cudaStream_t own = nullptr;
    void* h_stage = nullptr;  // device buffers of the host-pointer calls
    size_t h_stage_bytes = 0;
    double* h_tail = nullptr;  // pinned read-back: energy, virial[6], status word
    // bumped whenever a workspace buffer is reallocated or an option changes:
    // a captured graph older than this no longer matches the plan
    uint64_t gen = 1;
    // graph of the device part of the host-pointer call (its buffers are fixed)
    pppm_graph* host_g = nullptr;
    int64_t host_graph_n = -1;
    int host_graph_in = 0;
    uint64_t host_graph_gen = 0;
    cudaStream_t last = nullptr;
    // optional per-kernel timing with CUDA events (pppm_profile_enable)
    bool prof_on = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<int> pend_slot;
    std::vector<cudaEvent_t> pend_a, pend_b;
    double prof_ms[16] = {};
    int64_t prof_calls[16] = {};
};

