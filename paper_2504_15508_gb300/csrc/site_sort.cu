// Binning and sort of the sites by mesh tile: location of every site on the
// mesh, per-tile counts, their scan, and the scatter to tile order with each
// site's B-spline weights evaluated once (order-p stencil, bspline.cuh).
#include <climits>

#include <cuda.h>

#include "bspline.cuh"
#include "internal.cuh"

namespace pppm {

void upload_bspline_generic();

// Fills the B-spline piece tables of every translation unit that uses them.
void upload_bspline_coefficients() {
    bsp_upload_this_unit();
    upload_bspline_generic();
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

template <typename T, typename In>
__global__ void k_bin(Geo g, const In* __restrict__ pos, const In* __restrict__ q, int n,
                      int* __restrict__ tile_count, int* __restrict__ tile_of, int* __restrict__ slot_of,
                      Rec<T>* __restrict__ rec, int* __restrict__ cell, int* __restrict__ status) {
    pdl_enter();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < n;
    const int lane = threadIdx.x & 31;
    int t = -1 - lane, lx = 0, ly = 0, lz = 0;
    Rec<T> r;
    if (valid) {
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
        if (!ok) atomicOr(status, 1);
        const int tx = gc[0] / g.T, ty = gc[1] / g.T, tz = gc[2] / g.T;
        t = (tx * g.nt[1] + ty) * g.nt[2] + tz;
        lx = gc[0] - tx * g.T;
        ly = gc[1] - ty * g.T;
        lz = gc[2] - tz * g.T;
    }
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
        cell[i] = lx | (ly << 8) | (lz << 16);
    }
}

template <typename T, typename In>
cudaError_t launch_bin(cudaStream_t s, const Geo& g, const In* pos, const In* q, int n, int* tile_count,
                       int* tile_of, int* slot_of, Rec<T>* rec, int* cell, int* status) {
    if (n == 0) return cudaSuccess;
    k_bin<T, In><<<(n + 255) / 256, 256, 0, s>>>(g, pos, q, n, tile_count, tile_of, slot_of, rec, cell, status);
    return cudaGetLastError();
}

// Exclusive scan of the per-tile counts by one block: start[0..ntiles].
// Each thread sums a contiguous chunk; warps scan their chunk sums with
// shuffles; one warp scans the 32 warp totals; two barriers in all.
__global__ void __launch_bounds__(1024) k_scan(const int* __restrict__ count, int ntiles, int* __restrict__ start) {
    pdl_enter();
    __shared__ int wsum[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int chunk = (ntiles + 1023) / 1024;
    const int b = tid * chunk, e = min(b + chunk, ntiles);
    int sum = 0;
    for (int i = b; i < e; ++i) sum += count[i];
    int incl = sum;  // inclusive scan within the warp
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += v;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = wsum[lane];
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
        start[i] = run;
        run += count[i];
    }
    if (tid == 1023) start[ntiles] = wsum[31];
}

cudaError_t launch_scan(cudaStream_t s, const int* count, int ntiles, int* start) {
    return launch_k(k_scan, dim3(1), dim3(1024), 0, s, count, ntiles, start);
}

// Scatter to tile order.  Each site's B-spline weights are evaluated here,
// once, one thread per site: swt holds per site {q W_x[0..p-1], W_y[0..p-1],
// W_z[0..p-1]} padded to wstride(p) values; the fast spread and gather read
// them instead of re-evaluating the splines in every lane.
template <typename T, int P>
__global__ void k_scatter(int n, const int* __restrict__ tile_of, const int* __restrict__ slot_of,
                          const int* __restrict__ tile_start, const Rec<T>* __restrict__ rec,
                          const int* __restrict__ cell, Rec<T>* __restrict__ srec, int* __restrict__ scell,
                          int* __restrict__ sorig, T* __restrict__ swt) {
    pdl_enter();
    constexpr int WS = wstride(P);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int dst = tile_start[tile_of[i]] + slot_of[i];
    const Rec<T> r = rec[i];
    if (srec) srec[dst] = r;  // only the generic spread and gather read the records
    scell[dst] = cell[i];
    sorig[dst] = i;
    BspCoef<T, P> co;
    co.load();
    T w[WS];
    T t[P];
    co.all(r.x0[0], t);
#pragma unroll
    for (int a = 0; a < P; ++a) w[a] = t[a] * r.q;
    co.all(r.x0[1], t);
#pragma unroll
    for (int a = 0; a < P; ++a) w[P + a] = t[a];
    co.all(r.x0[2], t);
#pragma unroll
    for (int a = 0; a < P; ++a) w[2 * P + a] = t[a];
#pragma unroll
    for (int a = 3 * P; a < WS; ++a) w[a] = T(0);
    T* o = swt + (size_t)dst * WS;
#pragma unroll
    for (int a = 0; a < WS; a += 4) {
        if constexpr (sizeof(T) == 4) {
            *reinterpret_cast<float4*>(o + a) = make_float4(w[a], w[a + 1], w[a + 2], w[a + 3]);
        } else {
            *reinterpret_cast<double2*>(o + a) = make_double2(w[a], w[a + 1]);
            *reinterpret_cast<double2*>(o + a + 2) = make_double2(w[a + 2], w[a + 3]);
        }
    }
}

template <typename T>
cudaError_t launch_scatter(cudaStream_t s, const Geo& g, int n, const int* tile_of, const int* slot_of,
                           const int* tile_start, const Rec<T>* rec, const int* cell, Rec<T>* srec, int* scell,
                           int* sorig, T* swt) {
    if (n == 0) return cudaSuccess;
    const int blocks = (n + 255) / 256;
#define PPPM_SCATTER_P(PP)                                                                                  \
    case PP:                                                                                                \
        return launch_k(k_scatter<T, PP>, dim3(blocks), dim3(256), 0, s, n, tile_of, slot_of, tile_start, rec,   \
                        cell, srec, scell, sorig, swt);
    switch (g.order) {
        PPPM_SCATTER_P(2)
        PPPM_SCATTER_P(3)
        PPPM_SCATTER_P(4)
        PPPM_SCATTER_P(5)
        PPPM_SCATTER_P(6)
        PPPM_SCATTER_P(7)
        default: return cudaErrorInvalidValue;
    }
#undef PPPM_SCATTER_P
    return cudaGetLastError();
}


#define PPPM_INST_T(T)                                                                                          \
    template cudaError_t launch_scatter<T>(cudaStream_t, const Geo&, int, const int*, const int*, const int*,     \
                                           const Rec<T>*, const int*, Rec<T>*, int*, int*, T*);
PPPM_INST_T(float)
PPPM_INST_T(double)
#define PPPM_INST_TI(T, I)                                                                                       \
    template cudaError_t launch_bin<T, I>(cudaStream_t, const Geo&, const I*, const I*, int, int*, int*, int*,   \
                                          Rec<T>*, int*, int*);
PPPM_INST_TI(float, float)
PPPM_INST_TI(float, double)
PPPM_INST_TI(double, float)
PPPM_INST_TI(double, double)

// the bin kernel's entry (the one node of a captured step that reads the sites)
bool is_bin_kernel(const void* func) {
    return func == (const void*)k_bin<float, float> || func == (const void*)k_bin<float, double> ||
           func == (const void*)k_bin<double, float> || func == (const void*)k_bin<double, double>;
}

}  // namespace pppm
