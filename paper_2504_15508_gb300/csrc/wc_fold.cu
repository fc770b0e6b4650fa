// Fold of the Wannier-centroid forces onto atoms, Eq. DPLR:F_final.
//
// W_n = R_host(n) + Delta_n(R) (Eq. DPLR:Wn), so the long-range force on atom j
// is its own site force, plus the force on every WC it hosts, plus
// J^T F_W(n) for every Jacobian block J = dDelta_n/dR_j listed in its row.
// One warp per four consecutive atoms: their rows are one contiguous run of
// blocks, which the lanes stride over (each block component is one coalesced
// load across the warp) with several blocks in flight per lane; each block is
// added to its row's accumulator, a fixed xor butterfly sums the lanes, and
// lane r adds atom r's site and host terms in row order.  Every atom's sum
// has a fixed order: the result is bitwise reproducible.  The kernel streams
// the Jacobian once (40 B per block in FP32) and is HBM-bound for realistic
// neighbour counts.
#include <cstdint>

#include "internal.cuh"

namespace pppm {

constexpr int kFoldWarps = 8;
constexpr int kFoldAtoms = 4;  // atoms per warp: their rows are one contiguous run of blocks

template <typename T>
__global__ void __launch_bounds__(kFoldWarps * 32)
k_wc_fold(int64_t n_atoms, int64_t n_wc, const T* __restrict__ f_sites, const int* __restrict__ host_ptr,
          const int* __restrict__ host_wc, const int64_t* __restrict__ jac_ptr, const int* __restrict__ jac_wc,
          const T* __restrict__ jac, T* __restrict__ f_atoms, int* __restrict__ status) {
    const int lane = threadIdx.x & 31;
    const int64_t groups = (n_atoms + kFoldAtoms - 1) / kFoldAtoms;
    const int64_t warps = (int64_t)gridDim.x * kFoldWarps;
    const T* fw = f_sites + 3 * n_atoms;
    bool bad = false;
    for (int64_t grp = (int64_t)blockIdx.x * kFoldWarps + (threadIdx.x >> 5); grp < groups; grp += warps) {
        const int64_t j0 = grp * kFoldAtoms;
        const int na = (int)min((int64_t)kFoldAtoms, n_atoms - j0);
        // lane r's own terms of atom j0 + r (its site force, its hosted-WC
        // range), loaded first so that they arrive while the Jacobian runs
        T f0 = T(0), f1 = T(0), f2 = T(0);
        int h0 = 0, h1 = 0;
        if (lane < na) {
            const int64_t j = j0 + lane;
            f0 = f_sites[3 * j];
            f1 = f_sites[3 * j + 1];
            f2 = f_sites[3 * j + 2];
            if (host_ptr) {
                h0 = host_ptr[j];
                h1 = host_ptr[j + 1];
            }
        }
        T acc[kFoldAtoms][3];
#pragma unroll
        for (int r = 0; r < kFoldAtoms; ++r) acc[r][0] = acc[r][1] = acc[r][2] = T(0);
        if (jac_ptr) {
            int64_t bnd[kFoldAtoms + 1];
#pragma unroll
            for (int r = 0; r <= kFoldAtoms; ++r) bnd[r] = jac_ptr[j0 + min(r, na)];
            // lanes stride over the group's blocks; each block belongs to one row r
#pragma unroll 4
            for (int64_t k = bnd[0] + lane; k < bnd[kFoldAtoms]; k += 32) {
                const int n = __ldg(&jac_wc[k]);
                if (n < 0 || n >= n_wc) {
                    bad = true;
                    continue;
                }
                const T* J = jac + 9 * k;
                const T g0 = fw[3 * (int64_t)n], g1 = fw[3 * (int64_t)n + 1], g2 = fw[3 * (int64_t)n + 2];
                // (J^T g)_b = sum_a J[a][b] g_a
                const T c0 = __ldg(&J[0]) * g0 + __ldg(&J[3]) * g1 + __ldg(&J[6]) * g2;
                const T c1 = __ldg(&J[1]) * g0 + __ldg(&J[4]) * g1 + __ldg(&J[7]) * g2;
                const T c2 = __ldg(&J[2]) * g0 + __ldg(&J[5]) * g1 + __ldg(&J[8]) * g2;
#pragma unroll
                for (int r = 0; r < kFoldAtoms; ++r) {
                    if (k >= bnd[r] && k < bnd[r + 1]) {
                        acc[r][0] += c0;
                        acc[r][1] += c1;
                        acc[r][2] += c2;
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < kFoldAtoms; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int h = 16; h >= 1; h >>= 1) acc[r][c] += __shfl_xor_sync(0xffffffffu, acc[r][c], h);
        }
        // lane r finishes atom j0 + r: its own force, the WCs it hosts, the Jacobian sum
        T s0 = T(0), s1 = T(0), s2 = T(0);
#pragma unroll
        for (int r = 0; r < kFoldAtoms; ++r)
            if (lane == r) { s0 = acc[r][0]; s1 = acc[r][1]; s2 = acc[r][2]; }
        if (lane < na) {
            const int64_t j = j0 + lane;
            if (host_ptr) {
                for (int h = h0; h < h1; ++h) {
                    const int n = host_wc[h];
                    if (n < 0 || n >= n_wc) {
                        bad = true;
                        continue;
                    }
                    f0 += fw[3 * (int64_t)n];
                    f1 += fw[3 * (int64_t)n + 1];
                    f2 += fw[3 * (int64_t)n + 2];
                }
            }
            f_atoms[3 * j] = f0 + s0;
            f_atoms[3 * j + 1] = f1 + s1;
            f_atoms[3 * j + 2] = f2 + s2;
        }
    }
    if (bad && status) atomicOr(status, 1);
}

template <typename T>
int wc_fold(void* stream, int64_t n_atoms, int64_t n_wc, const T* f_sites, const int* host_ptr, const int* host_wc,
            const int64_t* jac_ptr, const int* jac_wc, const T* jac, T* f_atoms, int* status) {
    if (n_atoms < 0 || n_wc < 0 || (n_atoms > 0 && (!f_sites || !f_atoms))) return PPPM_ERR_INVALID_ARG;
    if ((host_ptr && !host_wc) || (jac_ptr && (!jac_wc || !jac))) return PPPM_ERR_INVALID_ARG;
    if (n_atoms == 0) return PPPM_OK;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return PPPM_ERR_CUDA;
    int64_t blocks = ((n_atoms + kFoldAtoms - 1) / kFoldAtoms + kFoldWarps - 1) / kFoldWarps;
    const int64_t cap = (int64_t)nsm * 8;  // 8 resident blocks of 8 warps per SM
    if (blocks > cap) blocks = cap;
    k_wc_fold<T><<<(unsigned)blocks, kFoldWarps * 32, 0, (cudaStream_t)stream>>>(
        n_atoms, n_wc, f_sites, host_ptr, host_wc, jac_ptr, jac_wc, jac, f_atoms, status);
    return cudaGetLastError() == cudaSuccess ? PPPM_OK : PPPM_ERR_CUDA;
}

}  // namespace pppm

extern "C" {

int pppm_wc_fold(void* stream, int64_t n_atoms, int64_t n_wc, const double* f_sites, const int* host_ptr,
                 const int* host_wc, const int64_t* jac_ptr, const int* jac_wc, const double* jac, double* f_atoms,
                 int* status) {
    return pppm::wc_fold<double>(stream, n_atoms, n_wc, f_sites, host_ptr, host_wc, jac_ptr, jac_wc, jac, f_atoms,
                                 status);
}

int pppm_wc_fold_f32(void* stream, int64_t n_atoms, int64_t n_wc, const float* f_sites, const int* host_ptr,
                     const int* host_wc, const int64_t* jac_ptr, const int* jac_wc, const float* jac,
                     float* f_atoms, int* status) {
    return pppm::wc_fold<float>(stream, n_atoms, n_wc, f_sites, host_ptr, host_wc, jac_ptr, jac_wc, jac, f_atoms,
                                status);
}

}  // extern "C"
