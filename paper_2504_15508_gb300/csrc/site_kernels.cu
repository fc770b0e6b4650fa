// Per-site kernels of the PPPM path: binning and sort of the sites by mesh
// tile, the atomics-free charge spread, the fold of the tile patches into the
// mesh, and the force interpolation (gather).
//
// Charge assignment and force interpolation use the same order-p B-spline
// stencil (bspline.cuh); the spread is the transpose of the gather.
#include <climits>

#include <cuda.h>

#include "bspline.cuh"
#include "internal.cuh"

namespace pppm {

// Piece coefficients of N_p on [0, 1] for p = 1..7, from the Cox-de Boor
// recursion carried out on polynomials in x0 (FP64 on the host).
void upload_bspline_coefficients() {
    static bool done = false;
    if (done) return;
    double cd[kMaxOrder + 1][kMaxOrder][kMaxOrder] = {};
    float cf[kMaxOrder + 1][kMaxOrder][kMaxOrder] = {};
    // piece j of N_m as a polynomial in x0: poly[j][k] = coefficient of x0^k, for t = x0 + j.
    double poly[kMaxOrder][kMaxOrder] = {};
    poly[0][0] = 1.0;  // N_1(x0) = 1 on [0, 1]
    for (int p = 1; p <= kMaxOrder; ++p) {
        if (p > 1) {
            double nxt[kMaxOrder][kMaxOrder] = {};
            for (int j = 0; j < p; ++j) {
                // N_p(x0 + j) = ((x0 + j) N_{p-1}(x0 + j) + (p - x0 - j) N_{p-1}(x0 + j - 1)) / (p - 1)
                for (int k = 0; k < p - 1; ++k) {
                    double a = (j < p - 1) ? poly[j][k] : 0.0;      // N_{p-1}(x0 + j)
                    double b = (j >= 1) ? poly[j - 1][k] : 0.0;     // N_{p-1}(x0 + j - 1)
                    nxt[j][k + 1] += a - b;                          // x0 * (a - b)
                    nxt[j][k] += j * a + (p - j) * b;
                }
                for (int k = 0; k < p; ++k) nxt[j][k] /= (p - 1);
            }
            for (int j = 0; j < kMaxOrder; ++j)
                for (int k = 0; k < kMaxOrder; ++k) poly[j][k] = nxt[j][k];
        }
        for (int j = 0; j < p; ++j)
            for (int k = 0; k < p; ++k) {
                cd[p][j][k] = poly[j][k];
                cf[p][j][k] = (float)poly[j][k];
            }
    }
    cudaMemcpyToSymbol(c_bsp_d, cd, sizeof(cd));
    cudaMemcpyToSymbol(c_bsp_f, cf, sizeof(cf));
    done = true;
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
__global__ void __launch_bounds__(1024) k_scan(const int* __restrict__ count, int ntiles, int* __restrict__ start) {
    __shared__ int part[1024];
    const int tid = threadIdx.x;
    const int chunk = (ntiles + 1023) / 1024;
    const int b = tid * chunk, e = min(b + chunk, ntiles);
    int sum = 0;
    for (int i = b; i < e; ++i) sum += count[i];
    part[tid] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        int v = tid >= off ? part[tid - off] : 0;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    int run = part[tid] - sum;
    for (int i = b; i < e; ++i) {
        start[i] = run;
        run += count[i];
    }
    if (tid == 1023) start[ntiles] = part[1023];
}

cudaError_t launch_scan(cudaStream_t s, const int* count, int ntiles, int* start) {
    k_scan<<<1, 1024, 0, s>>>(count, ntiles, start);
    return cudaGetLastError();
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
    constexpr int WS = wstride(P);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int dst = tile_start[tile_of[i]] + slot_of[i];
    const Rec<T> r = rec[i];
    srec[dst] = r;
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
        k_scatter<T, PP><<<blocks, 256, 0, s>>>(n, tile_of, slot_of, tile_start, rec, cell, srec, scell, sorig, \
                                                swt);                                                       \
        break;
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

// ------------------------------------------------------------------ spread
//
// One warp per tile of T^3 cells.  The warp accumulates the p^3 contributions
// of every site whose base point lies in the tile into a private shared-memory
// patch covering the tile plus the stencil halo, one site after another, in
// the order of the sites' original indices (so the result does not depend on
// the order the binning produced).  Lane (iy, iz) adds the p values along x of
// its stencil row (orders 6 and 7 give a lane two rows); no two lanes touch
// the same point, and consecutive sites are separated by __syncwarp, so no
// atomics are needed.  The patch is then
// written to global scratch; k_fold sums overlapping patches.
constexpr int kSpreadWarps = 4;
constexpr int kSpreadCap = 512;

template <typename T, int P>
__global__ void __launch_bounds__(kSpreadWarps * 32)
k_spread(Geo g, const int* __restrict__ tile_start, const Rec<T>* __restrict__ srec,
         const int* __restrict__ scell, const int* __restrict__ sorig, T* __restrict__ patch) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tile = blockIdx.x * kSpreadWarps + warp;
    const int Ex = g.E[0], Ey = g.E[1], Ez = g.E[2], Pz = g.Pz;
    const int plane = Ey * Pz;
    const int psize = Ex * plane;
    T* pt = reinterpret_cast<T*>(smem_raw) + warp * psize;
    int2* keys = reinterpret_cast<int2*>(reinterpret_cast<T*>(smem_raw) + kSpreadWarps * psize) + warp * kSpreadCap;
    if (tile >= g.ntiles) return;  // whole warp; no block-level barrier below

    for (int i = lane; i < psize; i += 32) pt[i] = T(0);
    const int s0 = tile_start[tile];
    const int c = tile_start[tile + 1] - s0;
    const bool sorted = c > 1 && c <= kSpreadCap;
    if (sorted) {
        int cp = 2;
        while (cp < c) cp <<= 1;
        for (int i = lane; i < cp; i += 32) keys[i] = i < c ? make_int2(sorig[s0 + i], s0 + i) : make_int2(INT_MAX, -1);
        __syncwarp();
        for (int k = 2; k <= cp; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = lane; i < cp; i += 32) {
                    int ixj = i ^ j;
                    if (ixj > i) {
                        int2 a = keys[i], b = keys[ixj];
                        bool up = (i & k) == 0;
                        if ((a.x > b.x) == up) { keys[i] = b; keys[ixj] = a; }
                    }
                }
                __syncwarp();
            }
    }
    __syncwarp();

    // lane -> stencil rows (iy, iz); orders above 5 have more rows than lanes
    constexpr int NR = (P * P + 31) / 32;
    BspCoef<T, P> cx;
    cx.load();
    BspPiece<T, P> py[NR], pz[NR];
    int roff[NR];
    bool ract[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) {
        const int row = lane + 32 * j;
        ract[j] = row < P * P;
        const int iy = ract[j] ? row / P : 0, iz = ract[j] ? row % P : 0;
        py[j].load(iy);
        pz[j].load(iz);
        roff[j] = iy * Pz + iz;
    }
    for (int t = 0; t < c; ++t) {
        const int s = sorted ? keys[t].y : s0 + t;
        const Rec<T> r = srec[s];
        const int cl = scell[s];
        const int lx = cl & 255, ly = (cl >> 8) & 255, lz = (cl >> 16) & 255;
        T wx[P];
        cx.all(r.x0[0], wx);
        T* base0 = pt + lx * plane + ly * Pz + lz;
#pragma unroll
        for (int j = 0; j < NR; ++j) {
            const T wyz = py[j].eval(r.x0[1]) * pz[j].eval(r.x0[2]) * r.q;
            if (ract[j]) {
                T* base = base0 + roff[j];
#pragma unroll
                for (int a = 0; a < P; ++a) base[a * plane] += wx[a] * wyz;
            }
        }
        __syncwarp();
    }
    T* dst = patch + (size_t)tile * psize;  // same padded layout as the shared patch
    for (int i = lane; i < psize; i += 32) dst[i] = pt[i];
}

template <typename T, int P>
static cudaError_t spread_p(cudaStream_t s, const Geo& g, const int* tile_start, const Rec<T>* srec,
                            const int* scell, const int* sorig, T* patch) {
    const int psize = g.E[0] * g.E[1] * g.Pz;
    size_t smem = (size_t)kSpreadWarps * psize * sizeof(T) + (size_t)kSpreadWarps * kSpreadCap * sizeof(int2);
    cudaError_t e = cudaFuncSetAttribute(k_spread<T, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int blocks = (g.ntiles + kSpreadWarps - 1) / kSpreadWarps;
    k_spread<T, P><<<blocks, kSpreadWarps * 32, smem, s>>>(g, tile_start, srec, scell, sorig, patch);
    return cudaGetLastError();
}

template <typename T, int P, int TILE>
static cudaError_t spread_fast(cudaStream_t, const Geo&, const int*, const int*, const int*, const T*, T*);
template <typename T, int P, int TILE, typename Out>
static cudaError_t gather_fast(cudaStream_t, const Geo&, const int*, const int*, const int*, const T*, const T*,
                               double, Out*);
template <typename T, int P, int TILE, typename Out>
static cudaError_t gather_tma(cudaStream_t, const Geo&, const int*, const int*, const int*, const T*, const void*,
                              double, Out*, int*);

// The fast kernels need full tiles on every axis and a tile edge of 4 or 8.
static bool fast_tiles(const Geo& g) {
    return (g.T == 4 || g.T == 8) && g.Tt[0] == g.T && g.Tt[1] == g.T && g.Tt[2] == g.T;
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
cudaError_t launch_spread(cudaStream_t s, const Geo& g, const int* tile_start, const Rec<T>* srec,
                          const int* scell, const int* sorig, const T* swt, T* patch) {
    if (fast_tiles(g)) {
        PPPM_FAST_SWITCH(spread_fast, T, s, g, tile_start, scell, sorig, swt, patch)
    }
    switch (g.order) {
        case 2: return spread_p<T, 2>(s, g, tile_start, srec, scell, sorig, patch);
        case 3: return spread_p<T, 3>(s, g, tile_start, srec, scell, sorig, patch);
        case 4: return spread_p<T, 4>(s, g, tile_start, srec, scell, sorig, patch);
        case 5: return spread_p<T, 5>(s, g, tile_start, srec, scell, sorig, patch);
        case 6: return spread_p<T, 6>(s, g, tile_start, srec, scell, sorig, patch);
        case 7: return spread_p<T, 7>(s, g, tile_start, srec, scell, sorig, patch);
    }
    return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------ fold
//
// Each mesh point sums, in a fixed order, the patch entries that cover it.
// cov_off/cov_ent hold per axis the list of (tile index, patch coordinate)
// pairs covering each mesh index (CSR, built on the host with the periodic
// wrap); the three axes' lists are concatenated, axis d starting at
// cov_off[d * (Nmax + 1)] with Nmax = max N.
template <typename T>
__global__ void k_fold(Geo g, const T* __restrict__ patch, const int* __restrict__ cov_off,
                       const int2* __restrict__ cov_ent, int nmax1, T scale, T* __restrict__ rho) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)g.N[0] * g.N[1] * g.N[2];
    if (idx >= total) return;
    const int z = (int)(idx % g.N[2]);
    const int y = (int)((idx / g.N[2]) % g.N[1]);
    const int x = (int)(idx / ((int64_t)g.N[1] * g.N[2]));
    const int* ox = cov_off;
    const int* oy = cov_off + nmax1;
    const int* oz = cov_off + 2 * nmax1;
    const int psz = g.E[0] * g.E[1] * g.Pz;
    T sum = T(0);
    for (int a = ox[x]; a < ox[x + 1]; ++a) {
        const int2 ex = cov_ent[a];
        for (int b = oy[y]; b < oy[y + 1]; ++b) {
            const int2 ey = cov_ent[b];
            for (int c = oz[z]; c < oz[z + 1]; ++c) {
                const int2 ez = cov_ent[c];
                const int tile = (ex.x * g.nt[1] + ey.x) * g.nt[2] + ez.x;
                sum += patch[(size_t)tile * psz + (ex.y * g.E[1] + ey.y) * g.Pz + ez.y];
            }
        }
    }
    rho[idx] = sum * scale;
}

// ------------------------------------------------------------------ gather
//
// One block per tile.  The three field meshes over the tile plus its stencil
// halo are staged in shared memory (periodic wrap applied while loading);
// then each thread interpolates one site: F = prefactor * q * sum W W W E.
constexpr int kGatherThreads = 64;

template <typename T, int P, typename Out>
__global__ void __launch_bounds__(kGatherThreads)
k_gather(Geo g, const int* __restrict__ tile_start, const Rec<T>* __restrict__ srec,
         const int* __restrict__ scell, const int* __restrict__ sorig, const T* __restrict__ fields, FieldLayout fl,
         double prefactor, Out* __restrict__ forces) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tile = blockIdx.x;
    const int s0 = tile_start[tile], s1 = tile_start[tile + 1];
    if (s0 == s1) return;  // uniform across the block
    const int Ex = g.E[0], Ey = g.E[1], Ez = g.E[2];
    const int psz = Ex * Ey * Ez;
    T* fx = reinterpret_cast<T*>(smem_raw);
    T* fy = fx + psz;
    T* fz = fy + psz;
    const int tx = tile / (g.nt[1] * g.nt[2]);
    const int ty = (tile / g.nt[2]) % g.nt[1];
    const int tz = tile % g.nt[2];
    const int ox = tx * g.T + g.kmin, oy = ty * g.T + g.kmin, oz = tz * g.T + g.kmin;
    const int eyz = Ey * Ez;
    for (int i = threadIdx.x; i < psz; i += blockDim.x) {
        int cx = i / eyz, rem = i - cx * eyz, cy = rem / Ez, cz = rem - cy * Ez;
        int mx = (ox + cx) % g.N[0]; mx += mx < 0 ? g.N[0] : 0;
        int my = (oy + cy) % g.N[1]; my += my < 0 ? g.N[1] : 0;
        int mz = (oz + cz) % g.N[2]; mz += mz < 0 ? g.N[2] : 0;
        const int64_t f = fl.padded ? ((int64_t)(mx - g.kmin) * fl.Yp + (my - g.kmin)) * fl.Zp + (mz - g.kmin)
                                    : ((int64_t)mx * g.N[1] + my) * g.N[2] + mz;
        fx[i] = fields[f];
        fy[i] = fields[fl.fstride + f];
        fz[i] = fields[2 * fl.fstride + f];
    }
    __syncthreads();
    BspCoef<T, P> co;
    co.load();
    for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
        const Rec<T> r = srec[s];
        const int cl = scell[s];
        const int lx = cl & 255, ly = (cl >> 8) & 255, lz = (cl >> 16) & 255;
        T wx[P], wy[P], wz[P];
        co.all(r.x0[0], wx);
        co.all(r.x0[1], wy);
        co.all(r.x0[2], wz);
        T ax = T(0), ay = T(0), az = T(0);
#pragma unroll
        for (int a = 0; a < P; ++a) {
#pragma unroll
            for (int b = 0; b < P; ++b) {
                const T wab = wx[a] * wy[b];
                const int base = ((lx + a) * Ey + (ly + b)) * Ez + lz;
#pragma unroll
                for (int c = 0; c < P; ++c) {
                    const T w = wab * wz[c];
                    ax += w * fx[base + c];
                    ay += w * fy[base + c];
                    az += w * fz[base + c];
                }
            }
        }
        const T sc = (T)prefactor * r.q;
        const int o = sorig[s];
        forces[3 * (int64_t)o] = (Out)(sc * ax);
        forces[3 * (int64_t)o + 1] = (Out)(sc * ay);
        forces[3 * (int64_t)o + 2] = (Out)(sc * az);
    }
}

template <typename T, int P, typename Out>
static cudaError_t gather_p(cudaStream_t s, const Geo& g, const int* tile_start, const Rec<T>* srec,
                            const int* scell, const int* sorig, const T* fields, const FieldLayout& fl,
                            double prefactor, Out* forces) {
    size_t smem = 3ull * g.E[0] * g.E[1] * g.E[2] * sizeof(T);
    cudaError_t e = cudaFuncSetAttribute(k_gather<T, P, Out>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_gather<T, P, Out><<<g.ntiles, kGatherThreads, smem, s>>>(g, tile_start, srec, scell, sorig, fields, fl,
                                                               prefactor, forces);
    return cudaGetLastError();
}

#define PPPM_FAST_SWITCH_G(FN, T_, O_, ...)                                                       \
    switch (g.order * 16 + g.T) {                                                                 \
        case 2 * 16 + 4: return FN<T_, 2, 4, O_>(__VA_ARGS__);                                    \
        case 2 * 16 + 8: return FN<T_, 2, 8, O_>(__VA_ARGS__);                                    \
        case 3 * 16 + 4: return FN<T_, 3, 4, O_>(__VA_ARGS__);                                    \
        case 3 * 16 + 8: return FN<T_, 3, 8, O_>(__VA_ARGS__);                                    \
        case 4 * 16 + 4: return FN<T_, 4, 4, O_>(__VA_ARGS__);                                    \
        case 4 * 16 + 8: return FN<T_, 4, 8, O_>(__VA_ARGS__);                                    \
        case 5 * 16 + 4: return FN<T_, 5, 4, O_>(__VA_ARGS__);                                    \
        case 5 * 16 + 8: return FN<T_, 5, 8, O_>(__VA_ARGS__);                                    \
        case 6 * 16 + 4: return FN<T_, 6, 4, O_>(__VA_ARGS__);                                    \
        case 6 * 16 + 8: return FN<T_, 6, 8, O_>(__VA_ARGS__);                                    \
        case 7 * 16 + 4: return FN<T_, 7, 4, O_>(__VA_ARGS__);                                    \
        case 7 * 16 + 8: return FN<T_, 7, 8, O_>(__VA_ARGS__);                                    \
    }

template <typename T, typename Out>
cudaError_t launch_gather(cudaStream_t s, const Geo& g, const int* tile_start, const Rec<T>* srec,
                          const int* scell, const int* sorig, const T* swt, const T* fields, const FieldLayout& fl,
                          const void* tmap, double prefactor, Out* forces, int* status) {
    if (fast_tiles(g)) {
        if (fl.padded && tmap) {
            PPPM_FAST_SWITCH_G(gather_tma, T, Out, s, g, tile_start, scell, sorig, swt, tmap, prefactor, forces,
                               status)
        }
        if (!fl.padded) {
            PPPM_FAST_SWITCH_G(gather_fast, T, Out, s, g, tile_start, scell, sorig, swt, fields, prefactor, forces)
        }
    }
    switch (g.order) {
        case 2: return gather_p<T, 2, Out>(s, g, tile_start, srec, scell, sorig, fields, fl, prefactor, forces);
        case 3: return gather_p<T, 3, Out>(s, g, tile_start, srec, scell, sorig, fields, fl, prefactor, forces);
        case 4: return gather_p<T, 4, Out>(s, g, tile_start, srec, scell, sorig, fields, fl, prefactor, forces);
        case 5: return gather_p<T, 5, Out>(s, g, tile_start, srec, scell, sorig, fields, fl, prefactor, forces);
        case 6: return gather_p<T, 6, Out>(s, g, tile_start, srec, scell, sorig, fields, fl, prefactor, forces);
        case 7: return gather_p<T, 7, Out>(s, g, tile_start, srec, scell, sorig, fields, fl, prefactor, forces);
    }
    return cudaErrorInvalidValue;
}


// ------------------------------------------------------------------ fast paths
//
// The kernels below are the ones the workloads run: tile edge and order are
// compile-time constants (so every index is constant arithmetic) and every
// axis has at least one full tile (N >= T).  The kernels above stay as the
// general path for meshes smaller than a tile.

constexpr int kFastCap = 256;  // sites per tile ordered by index in the fast spread

// Spread: as k_spread, with the tile's records staged through shared memory in
// batches of 32 (one coalesced load per lane instead of one dependent load per
// site) and a padded patch pitch (PZ odd) that keeps the p^2 stencil rows of a
// site in distinct banks.
template <typename T, int P, int TILE>
struct SpreadWarpSmem {
    static constexpr int E = TILE + P - 1, PZ = E | 1, PLANE = E * PZ, PSIZE = E * PLANE;
    static constexpr int WSP = wstride(P) + 4;  // staging row pitch (keeps vector stores conflict-light)
    T st_w[32][WSP];
    T pt[PSIZE];
    int st_cell[32];
    int2 keys[kFastCap];
};

template <typename T, int P, int TILE>
__global__ void __launch_bounds__(kSpreadWarps * 32)
k_spread_fast(Geo g, const int* __restrict__ tile_start, const int* __restrict__ scell,
              const int* __restrict__ sorig, const T* __restrict__ swt, T* __restrict__ patch) {
    typedef SpreadWarpSmem<T, P, TILE> WarpSmem;
    constexpr int E = WarpSmem::E, PZ = WarpSmem::PZ, PLANE = WarpSmem::PLANE, PSIZE = WarpSmem::PSIZE;
    constexpr int WS = wstride(P);
    extern __shared__ __align__(32) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tile = blockIdx.x * kSpreadWarps + warp;
    WarpSmem& W = reinterpret_cast<WarpSmem*>(smem_raw)[warp];
    if (tile >= g.ntiles) return;  // whole warp; no block-level barrier below
    for (int i = lane; i < PSIZE; i += 32) W.pt[i] = T(0);
    const int s0 = tile_start[tile];
    const int c = tile_start[tile + 1] - s0;
    const bool sorted = c > 1 && c <= kFastCap;
    if (sorted) {
        int cp = 2;
        while (cp < c) cp <<= 1;
        for (int i = lane; i < cp; i += 32)
            W.keys[i] = i < c ? make_int2(sorig[s0 + i], s0 + i) : make_int2(INT_MAX, -1);
        __syncwarp();
        for (int k = 2; k <= cp; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = lane; i < cp; i += 32) {
                    const int ixj = i ^ j;
                    if (ixj > i) {
                        const int2 a = W.keys[i], b = W.keys[ixj];
                        if ((a.x > b.x) == ((i & k) == 0)) { W.keys[i] = b; W.keys[ixj] = a; }
                    }
                }
                __syncwarp();
            }
    }
    __syncwarp();
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
    for (int t0 = 0; t0 < c; t0 += 32) {
        const int nb = min(32, c - t0);
        if (lane < nb) {
            const int s = sorted ? W.keys[t0 + lane].y : s0 + t0 + lane;
            const T* src = swt + (size_t)s * WS;
#pragma unroll
            for (int a = 0; a < WS; ++a) W.st_w[lane][a] = src[a];
            W.st_cell[lane] = scell[s];
        }
        __syncwarp();
        for (int j = 0; j < nb; ++j) {
            const int cl = W.st_cell[j];
            const int lx = cl & 255, ly = (cl >> 8) & 255, lz = (cl >> 16) & 255;
            T wxq[P];
#pragma unroll
            for (int a = 0; a < P; ++a) wxq[a] = W.st_w[j][a];
            T* base0 = W.pt + lx * PLANE + ly * PZ + lz;
#pragma unroll
            for (int jr = 0; jr < NR; ++jr) {
                if (ract[jr]) {
                    const T wyz = W.st_w[j][P + riy[jr]] * W.st_w[j][2 * P + riz[jr]];
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
    for (int i = lane; i < PSIZE; i += 32) dst[i] = W.pt[i];
}

template <typename T, int P, int TILE>
static cudaError_t spread_fast(cudaStream_t s, const Geo& g, const int* tile_start, const int* scell,
                               const int* sorig, const T* swt, T* patch) {
    const size_t smem = kSpreadWarps * sizeof(SpreadWarpSmem<T, P, TILE>);
    cudaError_t e = cudaFuncSetAttribute(k_spread_fast<T, P, TILE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const int blocks = (g.ntiles + kSpreadWarps - 1) / kSpreadWarps;
    k_spread_fast<T, P, TILE><<<blocks, kSpreadWarps * 32, smem, s>>>(g, tile_start, scell, sorig, swt, patch);
    return cudaGetLastError();
}

// Gather: one block (4 warps) per tile; the three field meshes over the tile
// and its halo are staged in shared memory with the padded pitch.  A warp
// takes the tile's sites eight at a time: lane (iy, iz) forms its row's share
// W_y W_z sum_x W_x E of each of the eight forces, then a transposing butterfly
// (31 shuffles for 8 sites x 4 components) leaves lane L holding the total of
// site L/4, component L%4, which it scales and stores.
constexpr int kGatherWarps = 4;

template <typename T, int P, int TILE, typename Out>
__global__ void __launch_bounds__(kGatherWarps * 32)
k_gather_fast(Geo g, const int* __restrict__ tile_start, const int* __restrict__ scell,
              const int* __restrict__ sorig, const T* __restrict__ swt, const T* __restrict__ fields,
              double prefactor, Out* __restrict__ forces) {
    constexpr int E = TILE + P - 1, PZ = E | 1, PLANE = E * PZ, PSIZE = E * PLANE;
    constexpr int WS = wstride(P), WSP = WS + 4;
    constexpr size_t STAGE_BYTES = (kGatherWarps * 8 * WSP * sizeof(T) + 31) / 32 * 32;
    constexpr size_t FIELD_BYTES = (3 * PSIZE * sizeof(T) + 31) / 32 * 32;
    extern __shared__ __align__(32) unsigned char smem_raw[];
    T* st_w = reinterpret_cast<T*>(smem_raw);  // [warps][8][WSP]
    T* fx = reinterpret_cast<T*>(smem_raw + STAGE_BYTES);
    T* fy = fx + PSIZE;
    T* fz = fy + PSIZE;
    int* st_cell = reinterpret_cast<int*>(smem_raw + STAGE_BYTES + FIELD_BYTES);
    int* st_orig = st_cell + kGatherWarps * 8;
    int* map = st_orig + kGatherWarps * 8;  // 3 * E mesh indices of the patch coordinates
    const int tile = blockIdx.x;
    const int s0 = tile_start[tile], s1 = tile_start[tile + 1];
    if (s0 == s1) return;  // uniform across the block
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tx = tile / (g.nt[1] * g.nt[2]);
    const int ty = (tile / g.nt[2]) % g.nt[1];
    const int tz = tile % g.nt[2];
    if (threadIdx.x < 3 * E) {
        const int d = threadIdx.x / E, c = threadIdx.x - d * E;
        const int t = d == 0 ? tx : (d == 1 ? ty : tz);
        int m = (t * TILE + g.kmin + c) % g.N[d];
        map[threadIdx.x] = m < 0 ? m + g.N[d] : m;
    }
    __syncthreads();
    const int64_t N3 = (int64_t)g.N[0] * g.N[1] * g.N[2];
    for (int i = threadIdx.x; i < E * E * E; i += blockDim.x) {
        const int x = i / (E * E), y = (i / E) % E, z = i % E;
        const int64_t f = ((int64_t)map[x] * g.N[1] + map[E + y]) * g.N[2] + map[2 * E + z];
        const int o = x * PLANE + y * PZ + z;
        fx[o] = fields[f];
        fy[o] = fields[N3 + f];
        fz[o] = fields[2 * N3 + f];
    }
    __syncthreads();
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
    T* ww = st_w + warp * 8 * WSP;
    int* wcell = st_cell + warp * 8;
    int* worig = st_orig + warp * 8;
    const int nsites = s1 - s0;
    for (int b = warp * 8; b < nsites; b += kGatherWarps * 8) {
        const int nb = min(8, nsites - b);
        for (int k = lane; k < nb * WS; k += 32) {
            const int j = k / WS, a = k - j * WS;
            ww[j * WSP + a] = swt[(size_t)(s0 + b + j) * WS + a];
        }
        if (lane < nb) {
            wcell[lane] = scell[s0 + b + lane];
            worig[lane] = sorig[s0 + b + lane];
        }
        __syncwarp();
        T v[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = T(0);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (j < nb) {
                const int cl = wcell[j];
                const int lx = cl & 255, ly = (cl >> 8) & 255, lz = (cl >> 16) & 255;
                const T* wj = ww + j * WSP;
                const int base0 = lx * PLANE + ly * PZ + lz;
#pragma unroll
                for (int jr = 0; jr < NR; ++jr) {
                    if (ract[jr]) {
                        const T wyz = wj[P + riy[jr]] * wj[2 * P + riz[jr]];
                        const int o0 = base0 + roff[jr];
#pragma unroll
                        for (int a = 0; a < P; ++a) {
                            const T w = wj[a] * wyz;
                            const int o = o0 + a * PLANE;
                            v[4 * j] += w * fx[o];
                            v[4 * j + 1] += w * fy[o];
                            v[4 * j + 2] += w * fz[o];
                        }
                    }
                }
            }
        }
        // transposing butterfly: after step h, lane keeps the half of its values
        // selected by its bit h and adds the partner's copy of the same half
#pragma unroll
        for (int h = 16; h >= 1; h >>= 1) {
            const bool up = (lane & h) != 0;
#pragma unroll
            for (int i = 0; i < h; ++i) {
                const T send = up ? v[i] : v[i + h];
                const T keep = up ? v[i + h] : v[i];
                v[i] = keep + __shfl_xor_sync(0xffffffffu, send, h);
            }
        }
        const int site = lane >> 2, comp = lane & 3;
        if (site < nb && comp < 3) forces[3 * (int64_t)worig[site] + comp] = (Out)((T)prefactor * v[0]);
        __syncwarp();
    }
}

template <typename T, int P, int TILE, typename Out>
static cudaError_t gather_fast(cudaStream_t s, const Geo& g, const int* tile_start, const int* scell,
                               const int* sorig, const T* swt, const T* fields, double prefactor, Out* forces) {
    constexpr int E = TILE + P - 1, PZ = E | 1, WSP = wstride(P) + 4;
    const size_t smem = (kGatherWarps * 8 * WSP * sizeof(T) + 31) / 32 * 32 +
                        (3 * (size_t)E * E * PZ * sizeof(T) + 31) / 32 * 32 + kGatherWarps * 8 * 2 * sizeof(int) +
                        3 * E * sizeof(int);
    cudaError_t e = cudaFuncSetAttribute(k_gather_fast<T, P, TILE, Out>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_gather_fast<T, P, TILE, Out><<<g.ntiles, kGatherWarps * 32, smem, s>>>(g, tile_start, scell, sorig, swt,
                                                                             fields, prefactor, forces);
    return cudaGetLastError();
}

// Gather with TMA staging: the three padded field meshes form one 4D tensor
// (z, y, x, field); the tile's stencil patch is the box starting at padded
// coordinates (tz T, ty T, tx T, 0), fetched by a single cp.async.bulk.tensor
// issued by one thread and waited on through an mbarrier.  The wait is
// bounded: if it runs out the block records PPPM_ERR_TIMEOUT in the status
// word (bit 2) and returns without touching the patch.
constexpr long long kTmaSpinLimit = 1ll << 26;

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t phase) {
    for (long long it = 0; it < kTmaSpinLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(mbar), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}

template <typename T, int P, int TILE, typename Out>
__global__ void __launch_bounds__(kGatherWarps * 32)
k_gather_tma(Geo g, const int* __restrict__ tile_start, const int* __restrict__ scell,
             const int* __restrict__ sorig, const T* __restrict__ swt, const __grid_constant__ CUtensorMap tmap,
             double prefactor, Out* __restrict__ forces, int* __restrict__ status) {
    constexpr int E = TILE + P - 1, EZ = (E + 3) & ~3, PLANE = E * EZ, PSIZE = E * PLANE;
    constexpr int WS = wstride(P), WSP = WS + 4;
    constexpr uint32_t TX_BYTES = 3u * PSIZE * sizeof(T);
    constexpr size_t FIELD_BYTES = (3 * PSIZE * sizeof(T) + 127) / 128 * 128;
    constexpr size_t STAGE_BYTES = (kGatherWarps * 8 * WSP * sizeof(T) + 31) / 32 * 32;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* fx = reinterpret_cast<T*>(smem_raw);  // TMA box: [field][x][y][z]
    T* fy = fx + PSIZE;
    T* fz = fy + PSIZE;
    T* st_w = reinterpret_cast<T*>(smem_raw + FIELD_BYTES);  // [warps][8][WSP]
    int* st_cell = reinterpret_cast<int*>(smem_raw + FIELD_BYTES + STAGE_BYTES);
    int* st_orig = st_cell + kGatherWarps * 8;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(st_orig + kGatherWarps * 8);
    const int tile = blockIdx.x;
    const int s0 = tile_start[tile], s1 = tile_start[tile + 1];
    if (s0 == s1) return;  // uniform across the block
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t mbar_s = (uint32_t)__cvta_generic_to_shared(mbar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar_s) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int tx = tile / (g.nt[1] * g.nt[2]);
        const int ty = (tile / g.nt[2]) % g.nt[1];
        const int tz = tile % g.nt[2];
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(fx);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar_s), "r"(TX_BYTES)
                     : "memory");
        asm volatile(
            "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
            "[%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
            "l"(reinterpret_cast<uint64_t>(&tmap)), "r"(tz * TILE), "r"(ty * TILE), "r"(tx * TILE), "r"(0),
            "r"(mbar_s)
            : "memory");
    }
    constexpr int NR = (P * P + 31) / 32;
    int roff[NR], riy[NR], riz[NR];
    bool ract[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) {
        const int row = lane + 32 * j;
        ract[j] = row < P * P;
        riy[j] = ract[j] ? row / P : 0;
        riz[j] = ract[j] ? row % P : 0;
        roff[j] = riy[j] * EZ + riz[j];
    }
    if (!mbar_wait_bounded(mbar_s, 0)) {
        if (threadIdx.x == 0) atomicOr(status, 2);
        mbar_wait_bounded(mbar_s, 0);  // give the copy in flight a second bounded chance to land
        return;
    }
    T* ww = st_w + warp * 8 * WSP;
    int* wcell = st_cell + warp * 8;
    int* worig = st_orig + warp * 8;
    const int nsites = s1 - s0;
    for (int b = warp * 8; b < nsites; b += kGatherWarps * 8) {
        const int nb = min(8, nsites - b);
        for (int k = lane; k < nb * WS; k += 32) {
            const int j = k / WS, a = k - j * WS;
            ww[j * WSP + a] = swt[(size_t)(s0 + b + j) * WS + a];
        }
        if (lane < nb) {
            wcell[lane] = scell[s0 + b + lane];
            worig[lane] = sorig[s0 + b + lane];
        }
        __syncwarp();
        T v[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = T(0);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (j < nb) {
                const int cl = wcell[j];
                const int lx = cl & 255, ly = (cl >> 8) & 255, lz = (cl >> 16) & 255;
                const T* wj = ww + j * WSP;
                const int base0 = lx * PLANE + ly * EZ + lz;
#pragma unroll
                for (int jr = 0; jr < NR; ++jr) {
                    if (ract[jr]) {
                        const T wyz = wj[P + riy[jr]] * wj[2 * P + riz[jr]];
                        const int o0 = base0 + roff[jr];
#pragma unroll
                        for (int a = 0; a < P; ++a) {
                            const T w = wj[a] * wyz;
                            const int o = o0 + a * PLANE;
                            v[4 * j] += w * fx[o];
                            v[4 * j + 1] += w * fy[o];
                            v[4 * j + 2] += w * fz[o];
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int h = 16; h >= 1; h >>= 1) {
            const bool up = (lane & h) != 0;
#pragma unroll
            for (int i = 0; i < h; ++i) {
                const T send = up ? v[i] : v[i + h];
                const T keep = up ? v[i + h] : v[i];
                v[i] = keep + __shfl_xor_sync(0xffffffffu, send, h);
            }
        }
        const int site = lane >> 2, comp = lane & 3;
        if (site < nb && comp < 3) forces[3 * (int64_t)worig[site] + comp] = (Out)((T)prefactor * v[0]);
        __syncwarp();
    }
}

template <typename T, int P, int TILE, typename Out>
static cudaError_t gather_tma(cudaStream_t s, const Geo& g, const int* tile_start, const int* scell,
                              const int* sorig, const T* swt, const void* tmap, double prefactor, Out* forces,
                              int* status) {
    constexpr int E = TILE + P - 1, EZ = (E + 3) & ~3, WSP = wstride(P) + 4;
    const size_t smem = (3 * (size_t)E * E * EZ * sizeof(T) + 127) / 128 * 128 +
                        (kGatherWarps * 8 * WSP * sizeof(T) + 31) / 32 * 32 + kGatherWarps * 8 * 2 * sizeof(int) +
                        16;
    cudaError_t e = cudaFuncSetAttribute(k_gather_tma<T, P, TILE, Out>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_gather_tma<T, P, TILE, Out><<<g.ntiles, kGatherWarps * 32, smem, s>>>(
        g, tile_start, scell, sorig, swt, *reinterpret_cast<const CUtensorMap*>(tmap), prefactor, forces, status);
    return cudaGetLastError();
}

// Fold with one block per mesh row (x, y): the x and y cover lists are the
// same for the whole block, the z list is read per point.
template <typename T>
__global__ void k_fold_rows(Geo g, const T* __restrict__ patch, const int* __restrict__ cov_off,
                            const int2* __restrict__ cov_ent, int nmax1, T scale, T* __restrict__ rho) {
    const int row = blockIdx.x;
    const int x = row / g.N[1], y = row - x * g.N[1];
    const int* ox = cov_off;
    const int* oy = cov_off + nmax1;
    const int* oz = cov_off + 2 * nmax1;
    const int psz = g.E[0] * g.E[1] * g.Pz;
    const int ax0 = __ldg(&ox[x]), ax1 = __ldg(&ox[x + 1]);
    const int ay0 = __ldg(&oy[y]), ay1 = __ldg(&oy[y + 1]);
    T* out = rho + (int64_t)row * g.N[2];
    for (int z = threadIdx.x; z < g.N[2]; z += blockDim.x) {
        const int az0 = __ldg(&oz[z]), az1 = __ldg(&oz[z + 1]);
        T sum = T(0);
        for (int a = ax0; a < ax1; ++a) {
            const int2 ex = __ldg(&cov_ent[a]);
            for (int b = ay0; b < ay1; ++b) {
                const int2 ey = __ldg(&cov_ent[b]);
                const int tb = (ex.x * g.nt[1] + ey.x) * g.nt[2];
                const int ob = (ex.y * g.E[1] + ey.y) * g.Pz;
                for (int c = az0; c < az1; ++c) {
                    const int2 ez = __ldg(&cov_ent[c]);
                    sum += patch[(size_t)(tb + ez.x) * psz + ob + ez.y];
                }
            }
        }
        out[z] = sum * scale;
    }
}

template <typename T>
cudaError_t launch_fold(cudaStream_t s, const Geo& g, const T* patch, const int* cov_off, const int2* cov_ent,
                        T scale, T* rho) {
    int64_t total = (int64_t)g.N[0] * g.N[1] * g.N[2];
    int nmax1 = 1 + (g.N[0] > g.N[1] ? (g.N[0] > g.N[2] ? g.N[0] : g.N[2]) : (g.N[1] > g.N[2] ? g.N[1] : g.N[2]));
    if (g.N[2] >= 32) {
        const int threads = g.N[2] >= 128 ? 128 : (g.N[2] >= 64 ? 64 : 32);
        k_fold_rows<T><<<g.N[0] * g.N[1], threads, 0, s>>>(g, patch, cov_off, cov_ent, nmax1, scale, rho);
        return cudaGetLastError();
    }
    k_fold<T><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(g, patch, cov_off, cov_ent, nmax1, scale, rho);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ instantiations
#define PPPM_INST_T(T)                                                                                          \
    template cudaError_t launch_scatter<T>(cudaStream_t, const Geo&, int, const int*, const int*, const int*,     \
                                           const Rec<T>*, const int*, Rec<T>*, int*, int*, T*);                  \
    template cudaError_t launch_spread<T>(cudaStream_t, const Geo&, const int*, const Rec<T>*, const int*,       \
                                          const int*, const T*, T*);                                             \
    template cudaError_t launch_fold<T>(cudaStream_t, const Geo&, const T*, const int*, const int2*, T, T*);
PPPM_INST_T(float)
PPPM_INST_T(double)
#define PPPM_INST_TI(T, I)                                                                                       \
    template cudaError_t launch_bin<T, I>(cudaStream_t, const Geo&, const I*, const I*, int, int*, int*, int*,   \
                                          Rec<T>*, int*, int*);                                                   \
    template cudaError_t launch_gather<T, I>(cudaStream_t, const Geo&, const int*, const Rec<T>*, const int*,     \
                                             const int*, const T*, const T*, const FieldLayout&, const void*,    \
                                             double, I*, int*);
PPPM_INST_TI(float, float)
PPPM_INST_TI(float, double)
PPPM_INST_TI(double, float)
PPPM_INST_TI(double, double)

}  // namespace pppm
