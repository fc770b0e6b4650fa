// General-path spread and gather (any mesh, tiles possibly larger than the
// mesh), the fold of tile patches into a mesh, and the dispatchers that send
// full-tile cases to the fast kernels.  Charge assignment and force
// interpolation use the same order-p B-spline stencil (bspline.cuh); the
// spread is the transpose of the gather.
#include <climits>

#include <cuda.h>

#include "bspline.cuh"
#include "internal.cuh"

namespace pppm {

// this translation unit's copy of the B-spline piece table
void upload_bspline_generic() { bsp_upload_this_unit(); }

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
k_spread(Geo g, const int2* __restrict__ tiles, const Rec<T>* __restrict__ srec,
         const int* __restrict__ scell, const int* __restrict__ sorig, T* __restrict__ patch, int* order,
         int* tmp) {
    pdl_enter();
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
    const int2 tr = tiles[tile];
    const int s0 = tr.x;
    const int c = tr.y - s0;
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
    const bool dense = c > kSpreadCap;  // ranked from global memory instead
    if (dense) rank_dense_tile(sorig + s0, c, order + s0, tmp + s0, reinterpret_cast<int*>(keys));

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
        const int s = sorted ? keys[t].y : s0 + (dense ? __ldcg(&order[s0 + t]) : t);
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
static cudaError_t spread_p(cudaStream_t s, const Geo& g, const int2* tiles, const Rec<T>* srec,
                            const int* scell, const int* sorig, T* patch, int* order, int* tmp) {
    const int psize = g.E[0] * g.E[1] * g.Pz;
    size_t smem = (size_t)kSpreadWarps * psize * sizeof(T) + (size_t)kSpreadWarps * kSpreadCap * sizeof(int2);
    cudaError_t e = cudaFuncSetAttribute(k_spread<T, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int blocks = (g.ntiles + kSpreadWarps - 1) / kSpreadWarps;
    return launch_k(k_spread<T, P>, dim3(blocks), dim3(kSpreadWarps * 32), smem, s, g, tiles, srec, scell, sorig,
                    patch, order, tmp);
}


template <typename T>
cudaError_t launch_spread(cudaStream_t s, const Geo& g, const int2* tiles, const Rec<T>* srec,
                          const int* scell, const int* sorig, T* patch, int* order, int* tmp, int* ticket) {
    if (fast_tiles(g)) {
        cudaError_t e = launch_spread_fast<T>(s, g, tiles, scell, sorig, srec, patch, order, tmp, ticket);
        if (e != cudaErrorNotSupported) return e;
    }
    switch (g.order) {
        case 2: return spread_p<T, 2>(s, g, tiles, srec, scell, sorig, patch, order, tmp);
        case 3: return spread_p<T, 3>(s, g, tiles, srec, scell, sorig, patch, order, tmp);
        case 4: return spread_p<T, 4>(s, g, tiles, srec, scell, sorig, patch, order, tmp);
        case 5: return spread_p<T, 5>(s, g, tiles, srec, scell, sorig, patch, order, tmp);
        case 6: return spread_p<T, 6>(s, g, tiles, srec, scell, sorig, patch, order, tmp);
        case 7: return spread_p<T, 7>(s, g, tiles, srec, scell, sorig, patch, order, tmp);
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
    pdl_enter();
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

// Fold with one block per mesh row (x, y): the x and y cover lists are the
// same for the whole block, the z list is read per point.
template <typename T>
__global__ void k_fold_rows(Geo g, const T* __restrict__ patch, const int* __restrict__ cov_off,
                            const int2* __restrict__ cov_ent, int nmax1, T scale, T* __restrict__ rho) {
    pdl_enter();
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
        return launch_k(k_fold_rows<T>, dim3(g.N[0] * g.N[1]), dim3(threads), 0, s, g, patch, cov_off, cov_ent, nmax1,
                        scale, rho);
    }
    return launch_k(k_fold<T>, dim3((unsigned)((total + 255) / 256)), dim3(256), 0, s, g, patch, cov_off, cov_ent, nmax1,
                    scale, rho);
}

// ------------------------------------------------------------------ gather
//
// One block per tile.  The three field meshes over the tile plus its stencil
// halo are staged in shared memory (periodic wrap applied while loading);
// then each thread interpolates one site: F = prefactor * q * sum W W W E.
constexpr int kGatherThreads = 64;

template <typename T, int P, typename Out>
__global__ void __launch_bounds__(kGatherThreads)
k_gather(Geo g, const int2* __restrict__ tiles, const Rec<T>* __restrict__ srec,
         const int* __restrict__ scell, const int* __restrict__ sorig, const T* __restrict__ fields, FieldLayout fl,
         double prefactor, Out* __restrict__ forces) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tile = blockIdx.x;
    const int2 tr = tiles[tile];
    const int s0 = tr.x, s1 = tr.y;
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
        const int64_t f = fl.pstride * (fl.padded ? ((int64_t)(mx - g.kmin) * fl.Yp + (my - g.kmin)) * fl.Zp +
                                                        (mz - g.kmin)
                                                  : ((int64_t)mx * g.N[1] + my) * g.N[2] + mz);
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
static cudaError_t gather_p(cudaStream_t s, const Geo& g, const int2* tiles, const Rec<T>* srec,
                            const int* scell, const int* sorig, const T* fields, const FieldLayout& fl,
                            double prefactor, Out* forces) {
    size_t smem = 3ull * g.E[0] * g.E[1] * g.E[2] * sizeof(T);
    cudaError_t e = cudaFuncSetAttribute(k_gather<T, P, Out>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return launch_k(k_gather<T, P, Out>, dim3(g.ntiles), dim3(kGatherThreads), smem, s, g, tiles, srec, scell,
                    sorig, fields, fl, prefactor, forces);
}

template <typename T, typename Out>
cudaError_t launch_gather(cudaStream_t s, const Geo& g, const int2* tiles, const Rec<T>* srec,
                          const int* scell, const int* sorig, const T* fields, const FieldLayout& fl,
                          const void* tmap, double prefactor, Out* forces, int* status, long long wait_limit) {
    if (fast_tiles(g) && fl.padded && tmap) {
        cudaError_t e = launch_gather_tma<T, Out>(s, g, tiles, scell, sorig, srec, tmap, prefactor, forces, status,
                                                  wait_limit);
        if (e != cudaErrorNotSupported) return e;
    }
    switch (g.order) {
        case 2: return gather_p<T, 2, Out>(s, g, tiles, srec, scell, sorig, fields, fl, prefactor, forces);
        case 3: return gather_p<T, 3, Out>(s, g, tiles, srec, scell, sorig, fields, fl, prefactor, forces);
        case 4: return gather_p<T, 4, Out>(s, g, tiles, srec, scell, sorig, fields, fl, prefactor, forces);
        case 5: return gather_p<T, 5, Out>(s, g, tiles, srec, scell, sorig, fields, fl, prefactor, forces);
        case 6: return gather_p<T, 6, Out>(s, g, tiles, srec, scell, sorig, fields, fl, prefactor, forces);
        case 7: return gather_p<T, 7, Out>(s, g, tiles, srec, scell, sorig, fields, fl, prefactor, forces);
    }
    return cudaErrorInvalidValue;
}

#define PPPM_INST_T(T)                                                                                          \
    template cudaError_t launch_spread<T>(cudaStream_t, const Geo&, const int2*, const Rec<T>*, const int*,      \
                                          const int*, T*, int*, int*, int*);                                     \
    template cudaError_t launch_fold<T>(cudaStream_t, const Geo&, const T*, const int*, const int2*, T, T*);
PPPM_INST_T(float)
PPPM_INST_T(double)
#define PPPM_INST_TI(T, I)                                                                                       \
    template cudaError_t launch_gather<T, I>(cudaStream_t, const Geo&, const int2*, const Rec<T>*, const int*,    \
                                             const int*, const T*, const FieldLayout&, const void*,              \
                                             double, I*, int*, long long);
PPPM_INST_TI(float, float)
PPPM_INST_TI(float, double)
PPPM_INST_TI(double, float)
PPPM_INST_TI(double, double)

}  // namespace pppm
