// Fast charge spread: tile edge and order are compile-time constants, each
// site's B-spline weights are evaluated on chip from its 16-byte record, and
// every axis holds at least one full tile.
#include <atomic>
#include <climits>

#include <cuda.h>

#include "bspline.cuh"
#include "internal.cuh"

namespace pppm {

void upload_bspline_spread() { bsp_upload_this_unit(); }

constexpr int kSpreadWarps = 4;
constexpr int kResidentCacheDevices = 64;
//
// The kernels below are the ones the workloads run: tile edge and order are
// compile-time constants (so every index is constant arithmetic) and every
// axis has at least one full tile (N >= T).  The kernels above stay as the
// general path for meshes smaller than a tile.

constexpr int kFastCap = 256;  // sites per tile ordered by index in the fast spread
constexpr int kStage = 32;     // sites staged per batch (one per lane)

// Spread: as k_spread, with the tile's sites staged through shared memory in
// batches of 32 (the next batch's records are loaded into registers while the
// current one is spread; at staging each lane writes its site's weight row,
// evaluated from the record) and a padded patch pitch
// (PZ odd) that keeps the p^2 stencil rows of a site in distinct banks.  The
// canonical order (by original index) comes from ranking the tile's sites by
// counting: one pass of broadcast compares, no sorting network.
template <typename T>
struct Vec16T;
template <>
struct Vec16T<float> {
    typedef float4 t;
};
template <>
struct Vec16T<double> {
    typedef double2 t;
};

// A site record by 16-byte loads, and 16-byte vector a of a row of weights.
__device__ __forceinline__ Rec<float> load_rec(const Rec<float>* p) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    Rec<float> r;
    r.x0[0] = v.x;
    r.x0[1] = v.y;
    r.x0[2] = v.z;
    r.q = v.w;
    return r;
}
__device__ __forceinline__ Rec<double> load_rec(const Rec<double>* p) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p));
    const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
    Rec<double> r;
    r.x0[0] = a.x;
    r.x0[1] = a.y;
    r.x0[2] = b.x;
    r.q = b.y;
    return r;
}
template <typename T>
__device__ __forceinline__ typename Vec16T<T>::t vec16(const T* w, int a);
template <>
__device__ __forceinline__ float4 vec16<float>(const float* w, int a) {
    return make_float4(w[4 * a], w[4 * a + 1], w[4 * a + 2], w[4 * a + 3]);
}
template <>
__device__ __forceinline__ double2 vec16<double>(const double* w, int a) {
    return make_double2(w[2 * a], w[2 * a + 1]);
}

template <typename T, int P, int TILE>
struct __align__(16) SpreadWarpSmem {  // 16-byte aligned: staged rows take vector stores
    static constexpr int E = TILE + P - 1, PZ = E | 1, PLANE = E * PZ, PSIZE = E * PLANE;
    static constexpr int WSP = wstride(P) + 4;  // staging row pitch (conflict-free 16-byte stores)
    union {
        int keys[kFastCap];  // original indices, while ranking
        T st_w[kStage][WSP];  // staged weights, while spreading
    } u;
    T pt[PSIZE];
    int st_cell[kStage];
    short perm[kFastCap];  // canonical position -> slot in the tile
};

// One tile by one warp: rank its sites, spread them in canonical order into
// the warp's shared patch, write the patch out.  Ends with __syncwarp, after
// which the warp may start on its next tile.
template <typename T, int P, int TILE>
__device__ __forceinline__ void spread_tile(int tile, SpreadWarpSmem<T, P, TILE>& W,
                                            const int2* __restrict__ tiles, const int* __restrict__ scell,
                                            const int* __restrict__ sorig, const Rec<T>* __restrict__ srec,
                                            T* __restrict__ patch, int* order, int* tmp) {
    typedef SpreadWarpSmem<T, P, TILE> WarpSmem;
    typedef typename Vec16T<T>::t V;
    constexpr int PZ = WarpSmem::PZ, PLANE = WarpSmem::PLANE, PSIZE = WarpSmem::PSIZE;
    constexpr int WS = wstride(P), NV = WS * (int)sizeof(T) / 16;  // 16-byte vectors per weight row
    const int lane = threadIdx.x & 31;
    const int2 tr = tiles[tile];
    const int s0 = tr.x;
    const int c = tr.y - s0;
    const bool ranked = c > 1 && c <= kFastCap;
    if (ranked) {
        for (int i = lane; i < c; i += 32) W.u.keys[i] = __ldg(&sorig[s0 + i]);
        // pad to a multiple of 4 with keys larger than every site index
        if (lane < ((c + 3) & ~3) - c) W.u.keys[c + lane] = INT_MAX;
    }
    // patch rows as 16-byte vectors where the patch size allows
    constexpr bool kVec = (PSIZE * sizeof(T)) % 16 == 0;
    constexpr int NV16 = PSIZE * (int)sizeof(T) / 16;
    if constexpr (kVec) {
        for (int i = lane; i < NV16; i += 32) reinterpret_cast<float4*>(W.pt)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
        for (int i = lane; i < PSIZE; i += 32) W.pt[i] = T(0);
    }
    __syncwarp();
    if (ranked) {
        // rank of item i = number of items with a smaller original index
        // (keys compared four at a time, from 16-byte broadcast loads)
        const int c4 = (c + 3) >> 2;
        const int4* k4 = reinterpret_cast<const int4*>(W.u.keys);
        for (int i = lane; i < c; i += 32) {
            const int ki = W.u.keys[i];
            int r = 0;
            for (int j = 0; j < c4; ++j) {
                const int4 kk = k4[j];
                r += (kk.x < ki) + (kk.y < ki) + (kk.z < ki) + (kk.w < ki);
            }
            W.perm[r] = (short)i;
        }
    }
    __syncwarp();
    const bool dense = c > kFastCap;  // ranked from global memory instead
    if (dense) rank_dense_tile(sorig + s0, c, order + s0, tmp + s0, W.u.keys);
    // lane -> stencil rows (iy, iz); orders above 5 have more rows than lanes
    constexpr int NR = (P * P + 31) / 32;
    int roff[NR], riy[NR], riz[NR];
    bool ract[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) {
        const int row = lane + 32 * j;
        ract[j] = row < P * P;
        riy[j] = ract[j] ? row / P : 0;
        riz[j] = ract[j] ? row % P : 0;
        roff[j] = riy[j] * PZ + riz[j];
    }
    // registers holding the next batch's records and cells (one site a
    // lane); a lane turns its site's record into the weight row when the
    // batch is staged
    Rec<T> nr;
    int ncell = 0;
    auto fetch = [&](int t0) {
        if (lane < kStage && t0 + lane < c) {
            const int s = s0 + (ranked ? (int)W.perm[t0 + lane] : (dense ? __ldcg(&order[s0 + t0 + lane]) : t0 + lane));
            nr = load_rec(srec + s);
            ncell = __ldg(&scell[s]);
        }
    };
    BspCoef<T, P> co;
    co.load();
    fetch(0);
    for (int t0 = 0; t0 < c; t0 += kStage) {
        const int nb = min(kStage, c - t0);
        if (lane < nb) {
            T w[WS];
            site_weights<T, P>(co, nr, w);
            V* dst = reinterpret_cast<V*>(&W.u.st_w[lane][0]);
#pragma unroll
            for (int a = 0; a < NV; ++a) dst[a] = vec16<T>(w, a);
            W.st_cell[lane] = ncell;
        }
        __syncwarp();
        fetch(t0 + kStage);  // in flight while this batch is spread
        for (int j = 0; j < nb; ++j) {
            const int cl = W.st_cell[j];
            const int lx = cl & 255, ly = (cl >> 8) & 255, lz = (cl >> 16) & 255;
            T wxq[P];
            if constexpr (sizeof(T) == 4 && P >= 4) {  // staged rows are 16-byte aligned
                const float4 q4 = *reinterpret_cast<const float4*>(&W.u.st_w[j][0]);
                wxq[0] = q4.x;
                wxq[1] = q4.y;
                wxq[2] = q4.z;
                wxq[3] = q4.w;
#pragma unroll
                for (int a = 4; a < P; ++a) wxq[a] = W.u.st_w[j][a];
            } else {
#pragma unroll
                for (int a = 0; a < P; ++a) wxq[a] = W.u.st_w[j][a];
            }
            T* base0 = W.pt + lx * PLANE + ly * PZ + lz;
#pragma unroll
            for (int jr = 0; jr < NR; ++jr) {
                if (ract[jr]) {
                    const T wyz = W.u.st_w[j][P + riy[jr]] * W.u.st_w[j][2 * P + riz[jr]];
                    T* b = base0 + roff[jr];
#pragma unroll
                    for (int a = 0; a < P; ++a) b[a * PLANE] += wxq[a] * wyz;
                }
            }
            __syncwarp();
        }
        __syncwarp();
    }
    T* dst = patch + (size_t)tile * PSIZE;  // same padded layout as the shared patch
    if constexpr (kVec) {
        for (int i = lane; i < NV16; i += 32)
            reinterpret_cast<float4*>(dst)[i] = reinterpret_cast<const float4*>(W.pt)[i];
    } else {
        for (int i = lane; i < PSIZE; i += 32) dst[i] = W.pt[i];
    }
    __syncwarp();
}

// Tiles are handed to warps dynamically: warp w of the (resident-sized) grid
// first takes tile w, then draws further tiles from a ticket counter until
// the tiles run out, so that SMs whose warps finish early take more tiles.
// Every warp draws exactly one ticket past the last tile; the warp drawing the
// very last ticket (no warp touches the counter after it) sets the counter
// back to zero for the next launch.  The counter must be zero before the
// first launch.
template <typename T, int P, int TILE>
__global__ void __launch_bounds__(kSpreadWarps * 32)
k_spread_fast(Geo g, const int2* __restrict__ tiles, const int* __restrict__ scell,
              const int* __restrict__ sorig, const Rec<T>* __restrict__ srec, T* __restrict__ patch, int* order,
              int* tmp, int* ticket) {
    pdl_enter();
    typedef SpreadWarpSmem<T, P, TILE> WarpSmem;
    extern __shared__ __align__(32) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSmem& W = reinterpret_cast<WarpSmem*>(smem_raw)[warp];
    const int nwarps = (int)gridDim.x * kSpreadWarps;
    const int dyn = g.ntiles > nwarps ? g.ntiles - nwarps : 0;  // tiles handed out by ticket
    int tile = (int)blockIdx.x * kSpreadWarps + warp;
    if (tile >= g.ntiles) tile = -1;
    for (;;) {
        if (tile >= 0) spread_tile<T, P, TILE>(tile, W, tiles, scell, sorig, srec, patch, order, tmp);
        int t = 0;
        if (lane == 0) t = atomicAdd(ticket, 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= dyn) {
            if (lane == 0 && t == dyn + nwarps - 1) atomicExch(ticket, 0);
            return;  // whole warp; no block-level barrier in this kernel
        }
        tile = nwarps + t;
    }
}

template <typename T, int P, int TILE>
static cudaError_t spread_fast(cudaStream_t s, const Geo& g, const int2* tiles, const int* scell,
                               const int* sorig, const Rec<T>* srec, T* patch, int* order, int* tmp, int* ticket) {
    auto kern = k_spread_fast<T, P, TILE>;
    const size_t smem = kSpreadWarps * sizeof(SpreadWarpSmem<T, P, TILE>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // as many blocks as are resident at once (the tiles beyond them go by
    // ticket): resident blocks an SM x SMs, queried once per device
    static std::atomic<int> resident[kResidentCacheDevices];  // 0: not queried yet
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    const bool cached = dev >= 0 && dev < kResidentCacheDevices;
    int cap = cached ? resident[dev].load(std::memory_order_relaxed) : 0;
    if (cap <= 0) {
        int nsm = 0, per = 0;
        if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kSpreadWarps * 32, smem)) != cudaSuccess)
            return e;
        cap = per >= 1 && nsm >= 1 ? per * nsm : 0;
        if (cached && cap > 0) resident[dev].store(cap, std::memory_order_relaxed);
    }
    int blocks = (g.ntiles + kSpreadWarps - 1) / kSpreadWarps;
    if (cap > 0 && blocks > cap) blocks = cap;
    return launch_k(kern, dim3(blocks), dim3(kSpreadWarps * 32), smem, s, g, tiles, scell, sorig, srec, patch, order,
                    tmp, ticket);
}


#define PPPM_FAST_SWITCH(FN, T_, ...)                                                             \
    switch (g.order * 16 + g.T) {                                                                 \
        case 2 * 16 + 4: return FN<T_, 2, 4>(__VA_ARGS__);                                        \
        case 2 * 16 + 8: return FN<T_, 2, 8>(__VA_ARGS__);                                        \
        case 3 * 16 + 4: return FN<T_, 3, 4>(__VA_ARGS__);                                        \
        case 3 * 16 + 8: return FN<T_, 3, 8>(__VA_ARGS__);                                        \
        case 4 * 16 + 4: return FN<T_, 4, 4>(__VA_ARGS__);                                        \
        case 4 * 16 + 8: return FN<T_, 4, 8>(__VA_ARGS__);                                        \
        case 5 * 16 + 4: return FN<T_, 5, 4>(__VA_ARGS__);                                        \
        case 5 * 16 + 8: return FN<T_, 5, 8>(__VA_ARGS__);                                        \
        case 6 * 16 + 4: return FN<T_, 6, 4>(__VA_ARGS__);                                        \
        case 6 * 16 + 8: return FN<T_, 6, 8>(__VA_ARGS__);                                        \
        case 7 * 16 + 4: return FN<T_, 7, 4>(__VA_ARGS__);                                        \
        case 7 * 16 + 8: return FN<T_, 7, 8>(__VA_ARGS__);                                        \
    }


template <typename T>
cudaError_t launch_spread_fast(cudaStream_t s, const Geo& g, const int2* tiles, const int* scell,
                               const int* sorig, const Rec<T>* srec, T* patch, int* order, int* tmp, int* ticket) {
    PPPM_FAST_SWITCH(spread_fast, T, s, g, tiles, scell, sorig, srec, patch, order, tmp, ticket)
    return cudaErrorNotSupported;
}

template cudaError_t launch_spread_fast<float>(cudaStream_t, const Geo&, const int2*, const int*, const int*,
                                               const Rec<float>*, float*, int*, int*, int*);
template cudaError_t launch_spread_fast<double>(cudaStream_t, const Geo&, const int2*, const int*, const int*,
                                                const Rec<double>*, double*, int*, int*, int*);

}  // namespace pppm
