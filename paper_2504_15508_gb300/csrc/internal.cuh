// Internal declarations shared by the CUDA translation units of the PPPM
// library: element types, the geometry block passed to kernels by value, the
// FFT radix plan, and the host-side launchers each .cu file provides.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pppm.h"

namespace pppm {

template <typename T> struct Cx;
template <> struct Cx<float> { typedef float2 t; };
template <> struct Cx<double> { typedef double2 t; };

// Sorted per-site record: x0 of the three axes (the B-spline argument, see
// bspline.cuh) and the charge.
template <typename T> struct __align__(4 * sizeof(T)) Rec { T x0[3]; T q; };

constexpr int kMaxOrder = 7;
constexpr int kMaxRadixStages = 16;
constexpr int kSortCap = 1024;       // sites per tile sorted by index in the spread
constexpr int kMaxMesh = 2048;

// Values in a site's row of B-spline weights of order p (the spread and the
// gather stage one row a site in shared memory): 3p weights padded to a
// multiple of 4.
__host__ __device__ constexpr int wstride(int p) { return (3 * p + 3) & ~3; }

// Radix plan of one FFT length: L = prod(r[0..n-1]), each r in {2, 3, 4, 5, 8}.
struct Radix {
    int L;
    int n;
    int r[kMaxRadixStages];
};

// Geometry of one box, passed to every kernel by value.
struct Geo {
    int N[3];        // mesh points per axis
    int Hz;          // Nz/2 + 1, complex points along z of the half spectrum
    float s_hi[3];   // N/L as a double-float pair (FP32 site location)
    float s_lo[3];
    double s[3];     // N/L in double
    double L[3];     // box edges
    float kfac_f[3]; // 2 pi / L, wavevector per index step
    double kfac_d[3];
    int order;       // B-spline order p
    int kmin;        // offset of the first stencil point from the base point
    int T;           // tile edge in cells (same on every axis, clamped to N per axis)
    int Tt[3];       // tile edge per axis after clamping
    int nt[3];       // tiles per axis
    int ntiles;
    int E[3];        // patch extent per axis = Tt + p - 1
    int Pz;          // z pitch of a spread patch, in shared memory and in the patch scratch
};

// Where the forward z FFT reads its real input: a mesh, or the spread's tile
// patches summed on the fly (the fold), through the per-axis cover lists.
// Each mesh index is covered by at most two tile patches per axis when every
// axis holds at least T + p - 1 points; cov2[d * nmax + m] lists them as
// {tile, coordinate, tile, coordinate}, tile -1 for an empty slot.
template <typename R>
struct PatchSrc {
    const R* patch;       // nullptr: read the mesh
    const int4* cov2;     // two-slot cover table, 3 axes of nmax entries each
    int nmax;
    int psz;              // elements per tile patch = E0 * E1 * Pz
};

template <typename R> __host__ __device__ __forceinline__ R kfac(const Geo& g, int d);
template <> __host__ __device__ __forceinline__ float kfac<float>(const Geo& g, int d) { return g.kfac_f[d]; }
template <> __host__ __device__ __forceinline__ double kfac<double>(const Geo& g, int d) { return g.kfac_d[d]; }

// Layout of the field meshes E_x, E_y, E_z (and the potential phi).
// Unpadded: consecutive Nx x Ny x Nz meshes, one per field (fstride = N,
// pstride = 1).  Padded ("ghosted"): the mesh extended by p - 1 periodic ghost
// points per axis, so that a tile's stencil patch is one contiguous box
// (padded index = mesh index - kmin, extents Xp = Nx + p - 1, Yp = Ny + p - 1,
// Zp = Nz + p - 1), with the values of a point interleaved as
// (E_x, E_y, E_z, 0) in 4 consecutive elements (fstride = 1, pstride = 4):
// the force interpolation reads a point's three fields with one 16-byte load.
// The potential, when produced, has a padded mesh of its own (one value a
// point).
struct FieldLayout {
    int padded;
    int Xp, Yp, Zp;
    int64_t fstride;  // elements between the same point of consecutive fields
    int64_t pstride;  // elements between consecutive mesh points
};

// Programmatic dependent launch.  Within a plan's solve sequence each kernel
// is launched with programmatic stream serialization: its blocks may be
// scheduled while the previous kernel's last blocks still run, and it waits
// (griddepcontrol.wait, the first statement of every such kernel) until that
// kernel has completed and its writes are visible before touching memory.
// Each kernel also allows its successor to be scheduled as soon as all of its
// own blocks have started.  Outside the sequence (or with per-kernel event
// timing on) launches are plain; the wait is then a no-op.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Canonical order of a tile that holds more sites than a spread kernel ranks
// in shared memory: order[r] = the slot i (0 <= i < c) whose key (original site
// index, keys[i] >= 0, all distinct) is the r-th smallest.  A stable LSD radix
// sort of the slots by key, 8-bit digits, as many passes as the largest key
// has bytes, by one warp: O(c) work per pass whatever the tile's size (a bad
// frame can put every site into one tile).  tmp holds c more ints of scratch;
// hist is 256 ints of the warp's own shared memory.  Global buffers are
// written and re-read by the same warp, with L2 loads and __syncwarp between
// the phases.  Every lane of the warp must call it; it ends with __syncwarp,
// after which every lane may read order[] (with L2 loads).
__device__ __forceinline__ void rank_dense_tile(const int* keys, int c, int* order, int* tmp, int* hist) {
    const int lane = (int)(threadIdx.x & 31);
    int kmax = 0;
    for (int i = lane; i < c; i += 32) kmax = max(kmax, __ldcg(&keys[i]));
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
    int npass = 1;
    while (npass < 4 && (kmax >> (8 * npass)) != 0) ++npass;
    // the last pass must land in order[]: the first writes order[] for an odd
    // number of passes, tmp[] for an even one
    int* src = nullptr;
    int* dst = (npass & 1) ? order : tmp;
    for (int pass = 0; pass < npass; ++pass) {
        const int shift = 8 * pass;
        for (int b = lane; b < 256; b += 32) hist[b] = 0;
        __syncwarp();
        for (int i = lane; i < c; i += 32) {
            const int slot = src ? __ldcg(&src[i]) : i;
            atomicAdd(&hist[(__ldcg(&keys[slot]) >> shift) & 255], 1);
        }
        __syncwarp();
        {  // exclusive scan of the 256 counts, eight consecutive bins a lane
            int v[8], sum = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                v[k] = hist[8 * lane + k];
                sum += v[k];
            }
            int incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            int run = incl - sum;
            __syncwarp();
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                hist[8 * lane + k] = run;
                run += v[k];
            }
        }
        __syncwarp();
        // stable scatter: chunks of 32 in order, lanes of a chunk in order
        for (int base = 0; base < c; base += 32) {
            const int i = base + lane;
            const bool act = i < c;
            const int slot = act ? (src ? __ldcg(&src[i]) : i) : 0;
            const int d = act ? ((__ldcg(&keys[slot]) >> shift) & 255) : 256 + lane;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            const int rank = __popc(peers & ((1u << lane) - 1u));
            const int leader = __ffs(peers) - 1;
            int b0 = 0;
            if (act) b0 = hist[d];
            __syncwarp();
            if (act) {
                __stcg(&dst[b0 + rank], slot);
                if (lane == leader) hist[d] = b0 + __popc(peers);
            }
            __syncwarp();
        }
        src = dst;
        dst = (dst == order) ? tmp : order;
    }
    __syncwarp();
}

// Integer (64-bit fixed-point) accumulation of the spread patches of the
// batched form.
//
// Slot (lane + 32 j) -> stencil row iy p + iz, so that the 64-bit accesses of
// each half-warp (served 16 lanes, 128 bytes, at a time) fall on distinct
// bank pairs: row (iy, iz) starts at element iy PZ + iz (plus the same site
// offset for every row), bank pair (iy PZ + iz) mod 16; rows are ordered by
// (occurrence, bank pair) so that consecutive slots walk the bank pairs
// round-robin.  Computed on the host, passed to the kernels by value.
struct RedRows {
    unsigned char row[64];
};

inline RedRows red_rows(int p, int pz) {
    auto grp = [&](int r) { return ((r / p) * pz + r % p) & 15; };
    int key[64];
    int seen[16] = {};
    for (int i = 0; i < p * p; ++i) key[i] = (seen[grp(i)]++) * 16 + grp(i);
    RedRows rr{};
    for (int i = 0; i < p * p; ++i) {
        int pos = 0;
        for (int j = 0; j < p * p; ++j) pos += key[j] < key[i] || (key[j] == key[i] && j < i);
        rr.row[pos] = (unsigned char)i;
    }
    return rr;
}

// Exact accumulation of a tile patch in two 32-bit integer words a value.
// Each stencil term x (an FP32 product) is scaled to f = x 2^k and split as
// f = h + l 2^-K, h = rint(f) and l = rint((f - h) 2^K); the patch keeps
// sum h and sum l in separate int32 arrays (added with 32-bit shared-memory
// atomics, so the order of the additions does not matter), and the value is
// (sum h 2^K + sum l) 2^-(k+K).  For a tile of c sites whose largest |q Wx|
// is m (Wy, Wz <= 1, so |x| <= m):
//   k = min(22 - e1, 30 - e), m < 2^e1, m c < 2^e: |f| < 2^22 (h is exact
//       by the 1.5 2^23 offset) and sum |h| <= c m 2^k + c/2 < 2^31;
//   K = min(22, 31 - bits(c)): |l| <= 2^(K-1) and sum |l| < 2^30.
// f itself is the FP32 product scaled by a power of two, and for |f| >= 2 the
// split is exact, so the patch is the exact sum of the FP32 terms up to
// 2^-(k+K+1) <= m 2^-45 a term.
struct SplitScale {
    int k, K;
    bool finite;
};

__device__ __forceinline__ SplitScale split_scale(unsigned m_bits, int c) {
    const float mq = __uint_as_float(m_bits);
    SplitScale r{0, 22, true};
    if (!(mq > 0.f)) return r;  // no charge: any scale
    const float m = mq * (float)max(c, 1);
    if (!isfinite(m)) {
        r.finite = false;
        return r;
    }
    const int e1 = (int)((m_bits >> 23) & 255u) - 126;                  // mq < 2^e1
    const int e = (int)((__float_as_uint(m) >> 23) & 255u) - 126;       // m < 2^e
    r.k = min(100, min(22 - e1, 30 - e));
    r.K = min(22, 31 - (32 - __clz(max(c, 1))));
    return r;
}

// the split of f = x 2^k (|f| < 2^22) into h = rint(f) and l = rint((f - h) 2^K)
__device__ __forceinline__ void split_term(float f, float twoK, int& h, int& l) {
    constexpr float kMagic = 12582912.f;  // 1.5 2^23: adding it rounds |v| < 2^22 to an integer
    const float t = f + kMagic;
    h = __float_as_int(t) - __float_as_int(kMagic);
    const float r = f - (t - kMagic);
    l = __float_as_int(fmaf(r, twoK, kMagic)) - __float_as_int(kMagic);
}

// 2^k from its exponent bits (-126 <= k <= 127)
__device__ __forceinline__ float pow2f(int k) { return __uint_as_float((unsigned)(k + 127) << 23); }

extern thread_local bool g_pdl;  // launches of this host thread use PDL

struct PdlScope {
    bool old;
    explicit PdlScope(bool on) : old(g_pdl) { g_pdl = on; }
    ~PdlScope() { g_pdl = old; }
};

template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
    if (!g_pdl) {
        kern<<<grid, block, smem, s>>>(args...);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// z extent (in points) of the TMA box of field patches: at least the patch
// edge T + p - 1, and odd, so that the 16-byte points of the stencil rows of a
// site fall on distinct bank groups (see k_gather_tma)
__host__ __device__ constexpr int gather_box_z(int p, int t) { return (t + p - 1) | 1; }

// Bundle shape of a strided-line FFT pass in the batched kernel (lines along
// y or x, B adjacent kz columns per block).
struct Bundle {
    int B;           // lines per block
    int nb;          // bundles per outer index = ceil(Hz / B)
};

// Blocks of a strided-line FFT pass of a plan: the lines (along y or x) are
// numbered f = outer Hz + kz over the other two indices, and a block takes B
// consecutive f (it may span two outer rows), so B can be chosen per pass to
// fill whole waves of resident blocks (choose_line_blocks).
struct LineBlocks {
    int B;     // lines per block, at most 16
    int nblk;  // blocks = ceil(outer Hz / B)
};
// the passes of a plan
enum { LB_Y = 0, LB_X_INFLUENCE = 1, LB_Y_INVERSE3 = 2, LB_X = 3 };

// The fast spread and gather need full tiles on every axis and a tile edge of 4 or 8.
inline bool fast_tiles(const Geo& g) {
    return (g.T == 4 || g.T == 8) && g.Tt[0] == g.T && g.Tt[1] == g.T && g.Tt[2] == g.T;
}

// Arguments of the one-pass site sort into fixed tile regions (site_sort.cu):
// the kernels that read the sites take (Geo, pos, q, n, DirectArgs), so that a
// captured step can patch the site pointers of each such node alike.
template <typename T>
struct DirectArgs {
    int2* tiles;    // per tile: (first slot, end slot)
    int cap;        // slots of a tile's region
    int* flag;      // [0] set when a region overflowed (the compact layout is then rebuilt),
                    // [1] blocks of the sort done
    int* tile_of;   // per site: its tile
    int* slot_of;   // per site: its arrival rank in the tile
    Rec<T>* srec;   // tile order: records (B-spline arguments, charge)
    int* scell;
    int* sorig;
    int* status;
};

// ------------------------------------------------------------------ launchers
// site_sort.cu.  Tile-ordered site data are described by tiles[t] = (first
// slot, end slot) of tile t.
template <typename T, typename In>
cudaError_t launch_bin(cudaStream_t s, const Geo& g, const In* pos, const In* q, int n, int* tile_count,
                       int* tile_of, int* slot_of, Rec<T>* rec, int* cell, int* status);
cudaError_t launch_scan(cudaStream_t s, const int* count, int ntiles, int2* tiles);
template <typename T>
cudaError_t launch_scatter(cudaStream_t s, const Geo& g, int n, const int* tile_of, const int* slot_of,
                           const int2* tiles, const Rec<T>* rec, const int* cell, Rec<T>* srec, int* scell,
                           int* sorig);
// fixed regions of a.cap slots per tile: init (also zeroes the two flag words),
// then the one-pass sort
cudaError_t launch_tiles_init(cudaStream_t s, int2* tiles, int ntiles, int cap, int* flag);
template <typename T, typename In>
cudaError_t launch_bin_direct(cudaStream_t s, const Geo& g, const In* pos, const In* q, int n,
                              const DirectArgs<T>& a);
bool is_bin_kernel(const void* func);   // (Geo, pos, q, n, six pointers)
bool is_site_kernel(const void* func);  // (Geo, pos, q, n, DirectArgs)
// order, tmp: n ints of scratch each in tile order (the binning's slot and
// tile arrays, dead once the scatter has run), used to rank tiles denser than
// the shared-memory ranking.  ticket: one device int, zero before the first
// launch, which the full-tile spread uses to hand tiles to warps and leaves
// at zero when it completes (one per plan: two spreads that may run at the
// same time need two)
template <typename T>
cudaError_t launch_spread(cudaStream_t s, const Geo& g, const int2* tiles, const Rec<T>* srec,
                          const int* scell, const int* sorig, T* patch, int* order, int* tmp, int* ticket);
template <typename T>
cudaError_t launch_fold(cudaStream_t s, const Geo& g, const T* patch, const int* cov_off, const int2* cov_ent,
                        T scale, T* rho);
template <typename T, typename Out>
cudaError_t launch_gather(cudaStream_t s, const Geo& g, const int2* tiles, const Rec<T>* srec,
                          const int* scell, const int* sorig, const T* fields, const FieldLayout& fl,
                          const void* tmap, double prefactor, Out* forces, int* status, long long wait_limit);
void upload_bspline_coefficients();
// full-tile fast paths (cudaErrorNotSupported when the order/tile has none)
template <typename T>
cudaError_t launch_spread_fast(cudaStream_t s, const Geo& g, const int2* tiles, const int* scell,
                               const int* sorig, const Rec<T>* srec, T* patch, int* order, int* tmp, int* ticket);
// wait_limit: spins of the first bounded wait for a tile's field copy (0: it
// runs out at once, the copy is then waited for once more before the block
// returns; a test of the timeout path)
template <typename T, typename Out>
cudaError_t launch_gather_tma(cudaStream_t s, const Geo& g, const int2* tiles, const int* scell, const int* sorig,
                              const Rec<T>* srec, const void* tmap, double prefactor, Out* forces, int* status,
                              long long wait_limit);

// fft_kernels.cu
template <typename T>
cudaError_t launch_fft_z_r2c(cudaStream_t s, const Geo& g, const Radix& rz, const typename Cx<T>::t* tw,
                             const T* in, typename Cx<T>::t* out, const PatchSrc<T>& ps);
template <typename T>
cudaError_t launch_fft_bundle(cudaStream_t s, const Geo& g, int axis, int sign, const Radix& r, const LineBlocks& lb,
                              const typename Cx<T>::t* tw, typename Cx<T>::t* data);
template <typename T>
cudaError_t launch_fft_x_influence(cudaStream_t s, const Geo& g, const Radix& rx, const LineBlocks& lb,
                                   const typename Cx<T>::t* tw, const T* G, double beta, double e_scale,
                                   double c_field, typename Cx<T>::t* S, typename Cx<T>::t* Bx, T* partial,
                                   unsigned int* counter, double prefactor, double* energy, double* virial);
template <typename T>
cudaError_t launch_fft_y_inverse3(cudaStream_t s, const Geo& g, const Radix& ry, const LineBlocks& lb,
                                  const typename Cx<T>::t* tw, typename Cx<T>::t* A, typename Cx<T>::t* Bx,
                                  typename Cx<T>::t* D);
// nf fields: out[f] = C2R_z(src[f] * (mulkz[f] ? -i kz' : 1)); src/out arrays of nf pointers
template <typename T>
cudaError_t launch_fft_z_c2r(cudaStream_t s, const Geo& g, const Radix& rz, const typename Cx<T>::t* tw, int nf,
                             const typename Cx<T>::t* const* src, const int* mulkz, T* const* out,
                             const FieldLayout& fl);
int x_influence_blocks(const LineBlocks& lb);
// B of each pass (LB_*), from the resident blocks per SM of its kernel
template <typename T>
cudaError_t choose_line_blocks(const Geo& g, const Radix rad[3], int nsm, LineBlocks lb[4]);

// influence.cu
cudaError_t launch_influence(cudaStream_t s, const Geo& g, double beta, int alias, double* G);
template <typename T>
cudaError_t launch_convert(cudaStream_t s, const double* in, T* out, int64_t n);
template <typename T>
cudaError_t launch_twiddles(cudaStream_t s, int L, typename Cx<T>::t* tw);

}  // namespace pppm
