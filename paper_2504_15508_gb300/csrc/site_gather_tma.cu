// Force interpolation with TMA-staged field patches (padded field meshes with
// the three fields of a point interleaved in 16 bytes, compile-time tile edge
// and order, per-site weights evaluated on chip from the sites' records).
#include <climits>

#include <cuda.h>

#include "bspline.cuh"
#include "internal.cuh"

namespace pppm {

void upload_bspline_gather() { bsp_upload_this_unit(); }

constexpr int kGatherWarps = 4;

// Gather with TMA staging: the interleaved padded fields form one 3D tensor
// (4 z + component, y, x), the components of a z row being contiguous; the
// tile's stencil patch is the box starting at padded coordinates
// (4 tz T, ty T, tx T), fetched by a single cp.async.bulk.tensor
// issued by one thread and waited on through an mbarrier.  The wait is
// bounded (the plan's wait limit, 2^26 polls by default): if it runs out the
// block records PPPM_ERR_TIMEOUT in the status word (bit 2), waits once more,
// bounded by kTmaSpinLimit, so that a copy still in flight lands before the
// block exits, and returns without touching the patch.
constexpr long long kTmaSpinLimit = 1ll << 26;

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t phase, long long limit) {
    for (long long it = 0; it < limit; ++it) {
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

// One mesh point of the interleaved padded fields (E_x, E_y, E_z, phi) in
// shared memory, read with 16-byte loads.
template <typename T>
struct Point4;
template <>
struct Point4<float> {
    static __device__ __forceinline__ void load(const float* p, float& x, float& y, float& z) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        x = v.x;
        y = v.y;
        z = v.z;
    }
};
template <>
struct Point4<double> {
    static __device__ __forceinline__ void load(const double* p, double& x, double& y, double& z) {
        const double2 a = *reinterpret_cast<const double2*>(p);
        x = a.x;
        y = a.y;
        z = p[2];
    }
};

// The first P entries of a 16-byte-aligned shared row (the x weights of a
// site): 16-byte loads where the type allows.
template <typename T, int P>
__device__ __forceinline__ void load_row(const T* w, T (&out)[P]) {
    int a = 0;
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (; a + 4 <= P; a += 4) {
            const float4 q = *reinterpret_cast<const float4*>(w + a);
            out[a] = q.x;
            out[a + 1] = q.y;
            out[a + 2] = q.z;
            out[a + 3] = q.w;
        }
    }
#pragma unroll
    for (; a < P; ++a) out[a] = w[a];
}

// Lane order of the p^2 stencil rows (iy, iz) of a site.  A warp's 16-byte
// shared loads are served a quarter-warp (8 lanes) at a time, one 16-byte
// bank group per lane; row (iy, iz) starts in group (iy EZ + iz) mod 8 (plus
// the same site offset for every row).  Rows are ordered by (k, group), k
// counting the earlier rows of the same group, so that consecutive lanes walk
// the groups round-robin: with EZ = 13 and p = 5 each quarter-warp touches 8
// distinct groups.  Computed on the host, passed as a kernel parameter.
struct LaneRows {
    unsigned char row[64];  // slot (lane + 32 j) -> row iy p + iz
};

static LaneRows order_rows(int p, int ez) {
    auto grp = [&](int r) { return ((r / p) * ez + r % p) & 7; };
    int key[64];
    int seen[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = 0; i < p * p; ++i) key[i] = (seen[grp(i)]++) * 8 + grp(i);
    LaneRows lr{};
    for (int i = 0; i < p * p; ++i) {
        int pos = 0;
        for (int j = 0; j < p * p; ++j) pos += key[j] < key[i] || (key[j] == key[i] && j < i);
        lr.row[pos] = (unsigned char)i;
    }
    return lr;
}

template <typename T, int P, int TILE, typename Out>
__global__ void __launch_bounds__(kGatherWarps * 32, 6)  // shared memory holds six blocks an SM
k_gather_tma(Geo g, const int2* __restrict__ tiles, const int* __restrict__ scell,
             const int* __restrict__ sorig, const Rec<T>* __restrict__ srec, const __grid_constant__ CUtensorMap tmap,
             const __grid_constant__ LaneRows lanes, double prefactor, Out* __restrict__ forces,
             int* __restrict__ status, long long wait_limit) {
    pdl_enter();
    // TMA box: [x][y][z][component], z extent EZ points, 4 components a point
    constexpr int E = TILE + P - 1, EZ = gather_box_z(P, TILE), PLANE = E * EZ, PSIZE = E * PLANE;
    constexpr int WS = wstride(P), WSP = WS + 4;
    constexpr uint32_t TX_BYTES = 4u * PSIZE * sizeof(T);
    constexpr size_t FIELD_BYTES = (4 * PSIZE * sizeof(T) + 127) / 128 * 128;
    constexpr size_t STAGE_BYTES = (kGatherWarps * 8 * WSP * sizeof(T) + 31) / 32 * 32;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const T* fbox = reinterpret_cast<const T*>(smem_raw);
    T* st_w = reinterpret_cast<T*>(smem_raw + FIELD_BYTES);  // [warps][8][WSP]
    int* st_cell = reinterpret_cast<int*>(smem_raw + FIELD_BYTES + STAGE_BYTES);
    int* st_orig = st_cell + kGatherWarps * 8;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(st_orig + kGatherWarps * 8);
    const int tile = blockIdx.x;
    const int2 tr = tiles[tile];
    const int s0 = tr.x, s1 = tr.y;
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
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(smem_raw);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar_s), "r"(TX_BYTES)
                     : "memory");
        // innermost coordinate 4 tz T elements: a whole number of 16-byte points
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
            "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
            "l"(reinterpret_cast<uint64_t>(&tmap)), "r"(4 * tz * TILE), "r"(ty * TILE), "r"(tx * TILE), "r"(mbar_s)
            : "memory");
    }
    constexpr int NR = (P * P + 31) / 32;
    int roff[NR], riy[NR], riz[NR];
    bool ract[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) {
        const int slot = lane + 32 * j;
        ract[j] = slot < P * P;
        const int row = ract[j] ? (int)lanes.row[slot] : 0;
        riy[j] = row / P;
        riz[j] = row % P;
        roff[j] = 4 * (riy[j] * EZ + riz[j]);
    }
    T* ww = st_w + warp * 8 * WSP;
    int* wcell = st_cell + warp * 8;
    int* worig = st_orig + warp * 8;
    const int nsites = s1 - s0;
    // registers holding the next batch of 8 sites (one record entry a lane:
    // lane 4 j + d holds x0 of axis d of site j, lane 4 j + 3 its charge; the
    // cell and original index of site j in lane j): the first batch is
    // fetched while the TMA copy is in flight, each later one while the
    // previous batch is being interpolated.  At staging, lanes 4 j + d
    // (d < 3) evaluate the p weights of their axis into the batch's rows.
    const int sj = lane >> 2, sd = lane & 3;
    T nrv = T(0);
    int ncell = 0, norig = 0;
    auto fetch = [&](int b) {
        const int nb = min(8, nsites - b);
        if (nb <= 0) return;
        if (sj < nb) nrv = __ldg(reinterpret_cast<const T*>(srec + s0 + b + sj) + sd);
        if (lane < nb) {
            ncell = __ldg(&scell[s0 + b + lane]);
            norig = __ldg(&sorig[s0 + b + lane]);
        }
    };
    BspCoef<T, P> co;
    co.load();
    fetch(warp * 8);
    if (!mbar_wait_bounded(mbar_s, 0, wait_limit)) {
        if (threadIdx.x == 0) atomicOr(status, 2);
        mbar_wait_bounded(mbar_s, 0, kTmaSpinLimit);  // give the copy in flight a second bounded chance to land
        return;
    }
    for (int b = warp * 8; b < nsites; b += kGatherWarps * 8) {
        const int nb = min(8, nsites - b);
        {
            const T qj = __shfl_sync(0xffffffffu, nrv, lane | 3);  // the charge of this lane's site
            if (sj < nb && sd < 3) {
                T t[P];
                co.all(nrv, t);
                if (sd == 0) {
#pragma unroll
                    for (int a = 0; a < P; ++a) t[a] = t[a] * qj;
                }
#pragma unroll
                for (int a = 0; a < P; ++a) ww[sj * WSP + sd * P + a] = t[a];
            }
        }
        if (lane < nb) {
            wcell[lane] = ncell;
            worig[lane] = norig;
        }
        __syncwarp();
        fetch(b + kGatherWarps * 8);
        T v[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = T(0);
        auto interp = [&](int j) {  // site j of the batch into v[4 j .. 4 j + 2]
            const int cl = wcell[j];
            const int lx = cl & 255, ly = (cl >> 8) & 255, lz = (cl >> 16) & 255;
            const T* wj = ww + j * WSP;
            T wx[P];
            load_row<T, P>(wj, wx);
            const T* base0 = fbox + 4 * (lx * PLANE + ly * EZ + lz);
#pragma unroll
            for (int jr = 0; jr < NR; ++jr) {
                if (ract[jr]) {
                    const T wyz = wj[P + riy[jr]] * wj[2 * P + riz[jr]];
                    const T* o0 = base0 + roff[jr];
#pragma unroll
                    for (int a = 0; a < P; ++a) {
                        const T w = wx[a] * wyz;
                        T ex, ey, ez;
                        Point4<T>::load(o0 + 4 * a * PLANE, ex, ey, ez);
                        v[4 * j] += w * ex;
                        v[4 * j + 1] += w * ey;
                        v[4 * j + 2] += w * ez;
                    }
                }
            }
        };
        if (nb == 8) {  // no per-site branch: the loads of a site can overlap the previous one's arithmetic
#pragma unroll
            for (int j = 0; j < 8; ++j) interp(j);
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (j < nb) interp(j);
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
static cudaError_t gather_tma(cudaStream_t s, const Geo& g, const int2* tiles, const int* scell,
                              const int* sorig, const Rec<T>* srec, const void* tmap, double prefactor, Out* forces,
                              int* status, long long wait_limit) {
    constexpr int E = TILE + P - 1, EZ = gather_box_z(P, TILE), WSP = wstride(P) + 4;
    const size_t smem = (4 * (size_t)E * E * EZ * sizeof(T) + 127) / 128 * 128 +
                        (kGatherWarps * 8 * WSP * sizeof(T) + 31) / 32 * 32 + kGatherWarps * 8 * 2 * sizeof(int) +
                        8;
    cudaError_t e = cudaFuncSetAttribute(k_gather_tma<T, P, TILE, Out>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    static const LaneRows lanes = order_rows(P, EZ);
    return launch_k(k_gather_tma<T, P, TILE, Out>, dim3(g.ntiles), dim3(kGatherWarps * 32), smem, s, g, tiles,
                    scell, sorig, srec, *reinterpret_cast<const CUtensorMap*>(tmap), lanes, prefactor, forces, status,
                    wait_limit);
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
cudaError_t launch_gather_tma(cudaStream_t s, const Geo& g, const int2* tiles, const int* scell, const int* sorig,
                              const Rec<T>* srec, const void* tmap, double prefactor, Out* forces, int* status,
                              long long wait_limit) {
    PPPM_FAST_SWITCH_G(gather_tma, T, Out, s, g, tiles, scell, sorig, srec, tmap, prefactor, forces, status,
                       wait_limit)
    return cudaErrorNotSupported;
}

#define PPPM_INST_G(T, O)                                                                                       \
    template cudaError_t launch_gather_tma<T, O>(cudaStream_t, const Geo&, const int2*, const int*, const int*,  \
                                                 const Rec<T>*, const void*, double, O*, int*, long long);
PPPM_INST_G(float, float)
PPPM_INST_G(float, double)
PPPM_INST_G(double, float)
PPPM_INST_G(double, double)

}  // namespace pppm
