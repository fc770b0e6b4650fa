// Binning and sort of the sites by mesh tile: location of every site on the
// mesh (its cell, tile and B-spline arguments, see bspline.cuh), written in
// tile order as a 16-byte record, a cell and an original index.
//
// Two layouts of the tile-ordered site data:
//   compact   per-tile counts (k_bin), their scan (k_scan), a scatter to tile
//             order (k_scatter); a tile's sites are consecutive, tiles in order;
//   regions   every tile owns a fixed region of `cap` slots: one kernel
//             (k_bin_direct) locates each site, takes a slot in its tile's
//             region with an atomic and writes its data there (no scan, no
//             second pass over the sites).  A tile that receives more than
//             `cap` sites sets a flag, and the kernel's last block then
//             rebuilds the compact layout in the same arrays.
// Either way tiles[t] = (first slot, end slot) of tile t, and the order of the
// sites inside a tile is their arrival order: the spread puts them into a
// canonical order itself and the gather does not depend on it.
#include <climits>
#include <vector>

#include <cuda.h>

#include "internal.cuh"

namespace pppm {

void upload_bspline_generic();
void upload_bspline_spread();
void upload_bspline_gather();

// Fills the B-spline piece tables of every translation unit that uses them.
void upload_bspline_coefficients() {
    upload_bspline_generic();
    upload_bspline_spread();
    upload_bspline_gather();
}

// ------------------------------------------------------------------ binning

// Locate one coordinate in FP32 from a float position: u = x N / L with N/L held
// as a double-float pair (the product is then accurate to ~1e-12 cells, where a
// plain FP32 product would be off by ~1e-5 cells at 129 A), base point g and
// B-spline argument x0 (see bspline.cuh).  Returns false for a non-finite or
// absurdly distant coordinate, which is then placed at the origin.
__device__ __forceinline__ bool locate(float x, float s_hi, float s_lo, double /*s*/, int N, bool odd, int& g,
                                       float& x0) {
    float u = x * s_hi;
    float e = fmaf(x, s_hi, -u);
    float ul = fmaf(x, s_lo, e);
    bool ok = fabsf(u) < 4.0e6f;
    if (!ok) { u = 0.f; ul = 0.f; }
    float gf = odd ? floorf(u + 0.5f) : floorf(u);
    float d = (u - gf) + ul;
    if (odd) {
        if (d >= 0.5f) { gf += 1.f; d -= 1.f; } else if (d < -0.5f) { gf -= 1.f; d += 1.f; }
        x0 = 0.5f - d;
    } else {
        if (d >= 1.f) { gf += 1.f; d -= 1.f; } else if (d < 0.f) { gf -= 1.f; d += 1.f; }
        x0 = 1.f - d;
    }
    int gi = (int)gf % N;
    g = gi < 0 ? gi + N : gi;
    return ok;
}

// FP64 location (FP64 plans, and FP32 plans fed double positions).
template <typename T>
__device__ __forceinline__ bool locate(double x, float, float, double s, int N, bool odd, int& g, T& x0) {
    double u = x * s;
    bool ok = fabs(u) < 1.0e12;
    if (!ok) u = 0.0;
    double gd = odd ? floor(u + 0.5) : floor(u);
    double d = u - gd;
    x0 = (T)(odd ? 0.5 - d : 1.0 - d);
    long long gi = (long long)gd % N;
    g = (int)(gi < 0 ? gi + N : gi);
    return ok;
}

// Site i: its record (B-spline arguments and charge), tile and packed local
// cell; false for a non-finite or far-away position or a non-finite charge
// (the site is then placed at the origin with charge 0).
template <typename T, typename In>
__device__ __forceinline__ bool site_locate(const Geo& g, const In* __restrict__ pos, const In* __restrict__ q, int i,
                                            Rec<T>& r, int& t, int& cell) {
    const bool odd = (g.order & 1) != 0;
    int gc[3];
    bool ok = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        T x0;
        if constexpr (sizeof(T) == 4 && sizeof(In) == 4) {
            float xf;
            ok &= locate((float)pos[3 * i + d], g.s_hi[d], g.s_lo[d], g.s[d], g.N[d], odd, gc[d], xf);
            x0 = xf;
        } else {
            ok &= locate<T>((double)pos[3 * i + d], 0.f, 0.f, g.s[d], g.N[d], odd, gc[d], x0);
        }
        r.x0[d] = x0;
    }
    T qi = (T)q[i];
    if (!isfinite((double)qi)) { ok = false; qi = (T)0; }
    r.q = qi;
    const int tx = gc[0] / g.T, ty = gc[1] / g.T, tz = gc[2] / g.T;
    t = (tx * g.nt[1] + ty) * g.nt[2] + tz;
    cell = (gc[0] - tx * g.T) | ((gc[1] - ty * g.T) << 8) | ((gc[2] - tz * g.T) << 16);
    return ok;
}

template <typename T, typename In>
__global__ void k_bin(Geo g, const In* __restrict__ pos, const In* __restrict__ q, int n,
                      int* __restrict__ tile_count, int* __restrict__ tile_of, int* __restrict__ slot_of,
                      Rec<T>* __restrict__ rec, int* __restrict__ cell, int* __restrict__ status) {
    pdl_enter();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < n;
    const int lane = threadIdx.x & 31;
    int t = -1 - lane, cl = 0;
    Rec<T> r;
    if (valid && !site_locate<T, In>(g, pos, q, i, r, t, cl)) atomicOr(status, 1);
    // one atomic per distinct tile in the warp; lanes of a tile get consecutive slots
    const unsigned peers = __match_any_sync(0xffffffffu, t);
    const int leader = __ffs(peers) - 1;
    const int rank = __popc(peers & ((1u << lane) - 1u));
    int base = 0;
    if (valid && lane == leader) base = atomicAdd(&tile_count[t], __popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (valid) {
        tile_of[i] = t;
        slot_of[i] = base + rank;
        rec[i] = r;
        cell[i] = cl;
    }
}

template <typename T, typename In>
cudaError_t launch_bin(cudaStream_t s, const Geo& g, const In* pos, const In* q, int n, int* tile_count,
                       int* tile_of, int* slot_of, Rec<T>* rec, int* cell, int* status) {
    if (n == 0) return cudaSuccess;
    k_bin<T, In><<<(n + 255) / 256, 256, 0, s>>>(g, pos, q, n, tile_count, tile_of, slot_of, rec, cell, status);
    return cudaGetLastError();
}

// Exclusive scan of the per-tile counts by one block into tiles[t] = (start,
// start + count).  Each thread sums a contiguous chunk; warps scan their chunk
// sums with shuffles; one warp scans the 32 warp totals; two barriers in all.
// count(i) gives the count of tile i (read twice, before tiles[i] is written).
template <typename F>
__device__ __forceinline__ void scan_tiles(F count, int ntiles, int2* __restrict__ tiles) {
    __shared__ int wsum[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nthr = blockDim.x;
    const int chunk = (ntiles + nthr - 1) / nthr;
    const int b = tid * chunk, e = min(b + chunk, ntiles);
    int sum = 0;
    for (int i = b; i < e; ++i) sum += count(i);
    int incl = sum;  // inclusive scan within the warp
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += v;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = lane < (nthr >> 5) ? wsum[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += v;
        }
        wsum[lane] = w;  // inclusive totals of warps 0..lane
    }
    __syncthreads();
    int run = (warp > 0 ? wsum[warp - 1] : 0) + incl - sum;
    for (int i = b; i < e; ++i) {
        const int c = count(i);
        tiles[i] = make_int2(run, run + c);
        run += c;
    }
}

__global__ void __launch_bounds__(1024) k_scan(const int* __restrict__ count, int ntiles, int2* __restrict__ tiles) {
    pdl_enter();
    scan_tiles([&](int i) { return count[i]; }, ntiles, tiles);
}

cudaError_t launch_scan(cudaStream_t s, const int* count, int ntiles, int2* tiles) {
    return launch_k(k_scan, dim3(1), dim3(1024), 0, s, count, ntiles, tiles);
}

// Site i's data at slot dst of the tile order: its record (B-spline
// arguments and charge; the spread and the gather evaluate the weights from
// it on chip), cell and original index.
template <typename T>
__device__ __forceinline__ void write_site(const Rec<T>& r, int cl, int i, int dst, Rec<T>* __restrict__ srec,
                                           int* __restrict__ scell, int* __restrict__ sorig) {
    srec[dst] = r;
    scell[dst] = cl;
    sorig[dst] = i;
}

template <typename T>
__global__ void k_scatter(int n, const int* __restrict__ tile_of, const int* __restrict__ slot_of,
                          const int2* __restrict__ tiles, const Rec<T>* __restrict__ rec,
                          const int* __restrict__ cell, Rec<T>* __restrict__ srec, int* __restrict__ scell,
                          int* __restrict__ sorig) {
    pdl_enter();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    write_site<T>(rec[i], cell[i], i, tiles[tile_of[i]].x + slot_of[i], srec, scell, sorig);
}

template <typename T>
cudaError_t launch_scatter(cudaStream_t s, const Geo& g, int n, const int* tile_of, const int* slot_of,
                           const int2* tiles, const Rec<T>* rec, const int* cell, Rec<T>* srec, int* scell,
                           int* sorig) {
    if (n == 0) return cudaSuccess;
    const int blocks = (n + 255) / 256;
    return launch_k(k_scatter<T>, dim3(blocks), dim3(256), 0, s, n, tile_of, slot_of, tiles, rec, cell, srec, scell,
                    sorig);
}

// ------------------------------------------------------------------ fixed regions
__global__ void k_tiles_init(int2* __restrict__ tiles, int ntiles, int cap, int* __restrict__ flag) {
    pdl_enter();
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += gridDim.x * blockDim.x)
        tiles[t] = make_int2(t * cap, t * cap);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        flag[0] = 0;  // overflow
        flag[1] = 0;  // blocks of the sort done
    }
}

// One pass: locate, take a slot of the tile's region, write the site there.
// The last block to finish checks the overflow flag; if a region overflowed
// it rebuilds the compact layout alone (a scan of the counts, then every site
// again to start + its arrival rank): slow, but only for such inputs, and no
// extra launch on the normal path.
template <typename T, typename In>
__global__ void __launch_bounds__(256)
k_bin_direct(Geo g, const In* __restrict__ pos, const In* __restrict__ q, int n, DirectArgs<T> a) {
    pdl_enter();
    __shared__ bool last;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < n;
    const int lane = threadIdx.x & 31;
    int t = -1 - lane, cl = 0;
    Rec<T> r;
    if (valid && !site_locate<T, In>(g, pos, q, i, r, t, cl)) atomicOr(a.status, 1);
    // one atomic per distinct tile in the warp; lanes of a tile get consecutive slots
    const unsigned peers = __match_any_sync(0xffffffffu, t);
    const int leader = __ffs(peers) - 1;
    const int rank = __popc(peers & ((1u << lane) - 1u));
    int base = 0;
    if (valid && lane == leader) base = atomicAdd(&a.tiles[t].y, __popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (valid) {
        const int slot = base + rank, r0 = t * a.cap;
        a.tile_of[i] = t;
        a.slot_of[i] = slot - r0;  // arrival rank in the tile
        if (slot < r0 + a.cap) write_site<T>(r, cl, i, slot, a.srec, a.scell, a.sorig);
        else atomicExch(a.flag, 1);  // the region overflowed
    }
    // the block's writes, ordered before its count by the barrier and one
    // (cumulative) fence
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(a.flag + 1, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!last || __ldcg(a.flag) == 0) return;  // uniform across the block
    __threadfence();
    scan_tiles([&](int k) { return __ldcg(&a.tiles[k].y) - k * a.cap; }, g.ntiles, a.tiles);
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        Rec<T> rk;
        int tk = 0, ck = 0;
        site_locate<T, In>(g, pos, q, k, rk, tk, ck);  // the same record, tile and cell as above
        write_site<T>(rk, ck, k, a.tiles[tk].x + __ldcg(&a.slot_of[k]), a.srec, a.scell, a.sorig);
    }
}

cudaError_t launch_tiles_init(cudaStream_t s, int2* tiles, int ntiles, int cap, int* flag) {
    return launch_k(k_tiles_init, dim3((ntiles + 255) / 256), dim3(256), 0, s, tiles, ntiles, cap, flag);
}

template <typename T, typename In>
cudaError_t launch_bin_direct(cudaStream_t s, const Geo& g, const In* pos, const In* q, int n,
                              const DirectArgs<T>& a) {
    if (n == 0) return cudaSuccess;
    const int blocks = (n + 255) / 256;
    return launch_k(k_bin_direct<T, In>, dim3(blocks), dim3(256), 0, s, g, pos, q, n, a);
}

// The kernels that read the sites (the nodes of a captured step whose
// position and charge pointers are patched on replay): the compact layout's
// binning kernel, with arguments (Geo, pos, q, n, six pointers), and the
// region sort, with (Geo, pos, q, n, DirectArgs).
bool is_bin_kernel(const void* func) {
    return func == (const void*)k_bin<float, float> || func == (const void*)k_bin<float, double> ||
           func == (const void*)k_bin<double, float> || func == (const void*)k_bin<double, double>;
}

bool is_site_kernel(const void* func) {
    return func == (const void*)k_bin_direct<float, float> || func == (const void*)k_bin_direct<float, double> ||
           func == (const void*)k_bin_direct<double, float> || func == (const void*)k_bin_direct<double, double>;
}

#define PPPM_INST_T(T)                                                                                          \
    template cudaError_t launch_scatter<T>(cudaStream_t, const Geo&, int, const int*, const int*, const int2*,    \
                                           const Rec<T>*, const int*, Rec<T>*, int*, int*);
PPPM_INST_T(float)
PPPM_INST_T(double)
#define PPPM_INST_TI(T, I)                                                                                       \
    template cudaError_t launch_bin<T, I>(cudaStream_t, const Geo&, const I*, const I*, int, int*, int*, int*,   \
                                          Rec<T>*, int*, int*);
PPPM_INST_TI(float, float)
PPPM_INST_TI(float, double)
PPPM_INST_TI(double, float)
PPPM_INST_TI(double, double)
#define PPPM_INST_DIRECT(T, I)                                                                                   \
    template cudaError_t launch_bin_direct<T, I>(cudaStream_t, const Geo&, const I*, const I*, int,              \
                                                 const DirectArgs<T>&);
PPPM_INST_DIRECT(float, float)
PPPM_INST_DIRECT(float, double)
PPPM_INST_DIRECT(double, float)
PPPM_INST_DIRECT(double, double)

}  // namespace pppm
