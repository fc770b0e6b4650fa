// pppm_spread_noalloc: the charge spread of pppm_spread for callers that
// cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is off limits -- inside a
// host callback or a custom allocator hook, in a process whose device memory
// is carved up by another framework's pool, or in a plugin that must not grow
// the footprint at run time.  Such a caller still owns its inputs and its
// output, but it cannot create a plan (plans allocate their workspace).
//
// Instead of a plan's workspace, this entry point uses one file-scope device
// array of kNoAllocScratchBytes (32 MiB).  Every GPU that loads the library
// holds that array until the process exits.  All calls share it and it keeps
// the previous call's contents; what must start at zero (the per-tile
// counters) is cleared on the stream at the start of every call.  Two calls
// whose kernels overlap on the GPU (different streams, or different host
// threads) race on the array and give wrong results: serialize them.
//
// The device address of the array is looked up with cudaGetSymbolAddress the
// first time the entry point runs on a device (with that device current);
// in host code the array's name is only a host-side stand-in and must never
// be passed to a kernel.  That first call also uploads the B-spline
// coefficient table, so it should come before any stream capture.  Each call
// puts only memsets and kernel launches on the caller's stream: the fold's
// cover lists are built by a kernel inside the scratch array, so nothing is
// copied from host memory.
#include <cmath>
#include <mutex>

#include "internal.cuh"

using namespace pppm;

namespace {

constexpr size_t kNoAllocScratchBytes = 32ull << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_setup_lock;
void* g_scratch_addr[kMaxDevices] = {};

size_t round256(size_t x) { return (x + 255) & ~size_t(255); }

bool smooth235_na(int n) {
    if (n < 1) return false;
    for (int r : {2, 3, 5})
        while (n % r == 0) n /= r;
    return n == 1;
}

// Device address of the scratch array on the current device (set up once).
int scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PPPM_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return PPPM_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_setup_lock);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return PPPM_ERR_CUDA;
        upload_bspline_coefficients();
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return PPPM_OK;
}

// The fold's cover lists, the same lists a plan builds on the host: for axis d
// and mesh index m, the pairs (tile t, patch coordinate c) with
// (t T + kmin + c) mod N_d = m, ordered by t and then c; off[d nmax1 + m] is
// where list m starts in ent (one running index over the three axes) and
// off[d nmax1 + N_d] where axis d ends.  One block: each thread counts the
// lists of its indices, a block-wide exclusive scan turns the counts into
// offsets, then each thread writes its lists.
constexpr int kCoverThreads = 1024;

__device__ int cover_entries(const Geo& g, int d, int m, int2* out) {
    const int N = g.N[d], T = g.T;
    int k = 0;
    for (int t = 0; t < g.nt[d]; ++t) {
        int cells = N - t * T;
        if (cells > g.Tt[d]) cells = g.Tt[d];
        const int e = cells + g.order - 1;
        int c = (m - t * T - g.kmin) % N;
        if (c < 0) c += N;
        for (; c < e; c += N) {
            if (out) out[k] = make_int2(t, c);
            ++k;
        }
    }
    return k;
}

__global__ void __launch_bounds__(kCoverThreads) k_cover_lists(Geo g, int nmax1, int* off, int2* ent) {
    __shared__ int wsum[kCoverThreads / 32];
    const int total = 3 * nmax1;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int chunk = (total + kCoverThreads - 1) / kCoverThreads;
    const int b = tid * chunk, e = min(b + chunk, total);
    int sum = 0;
    for (int i = b; i < e; ++i) {
        const int d = i / nmax1, m = i - d * nmax1;
        const int c = m < g.N[d] ? cover_entries(g, d, m, nullptr) : 0;
        off[i] = c;
        sum += c;
    }
    int incl = sum;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = wsum[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += v;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    int run = (warp > 0 ? wsum[warp - 1] : 0) + incl - sum;
    for (int i = b; i < e; ++i) {
        const int c = off[i];
        off[i] = run;
        const int d = i / nmax1, m = i - d * nmax1;
        if (m < g.N[d]) cover_entries(g, d, m, ent + run);
        run += c;
    }
}

}  // namespace

extern "C" int pppm_spread_noalloc(const double box[3], const int mesh[3], int order, void* stream,
                                   const double* pos, const double* q, int64_t n, float* rho) {
    if (!box || !mesh || !rho || n < 0 || (n > 0 && (!pos || !q))) return PPPM_ERR_INVALID_ARG;
    if (order < 2 || order > kMaxOrder) return PPPM_ERR_BAD_ORDER;
    for (int d = 0; d < 3; ++d) {
        if (!(box[d] > 0.0) || !std::isfinite(box[d])) return PPPM_ERR_BAD_BOX;
        if (!smooth235_na(mesh[d]) || mesh[d] < order || mesh[d] > kMaxMesh) return PPPM_ERR_BAD_MESH;
    }
    if (n > ((int64_t)1 << 30)) return PPPM_ERR_TOO_LARGE;
    void* base = nullptr;
    int rc = scratch_address(&base);
    if (rc != PPPM_OK) return rc;

    // geometry and tiles, chosen exactly as a plan chooses them
    Geo g{};
    for (int d = 0; d < 3; ++d) {
        g.N[d] = mesh[d];
        g.L[d] = box[d];
        g.s[d] = (double)mesh[d] / box[d];
        g.s_hi[d] = (float)g.s[d];
        g.s_lo[d] = (float)(g.s[d] - (double)g.s_hi[d]);
        g.kfac_d[d] = 6.283185307179586476925 / box[d];
        g.kfac_f[d] = (float)g.kfac_d[d];
    }
    g.Hz = mesh[2] / 2 + 1;
    g.order = order;
    g.kmin = (order % 2) ? -(order - 1) / 2 : -order / 2 + 1;
    const int64_t N3 = (int64_t)mesh[0] * mesh[1] * mesh[2];
    const int T = ((double)n / (double)N3) * 512.0 <= 160.0 ? 8 : 4;
    g.T = T;
    g.ntiles = 1;
    for (int d = 0; d < 3; ++d) {
        g.Tt[d] = T < g.N[d] ? T : g.N[d];
        g.nt[d] = (g.N[d] + T - 1) / T;
        g.E[d] = g.Tt[d] + order - 1;
        g.ntiles *= g.nt[d];
    }
    g.Pz = g.E[2] | 1;

    // fold cover lists: built on the device, into the scratch array, by k_cover_lists
    int nmax = mesh[0];
    if (mesh[1] > nmax) nmax = mesh[1];
    if (mesh[2] > nmax) nmax = mesh[2];
    const int nmax1 = nmax + 1;
    // entries per axis: every tile contributes (its cells + p - 1) pairs
    size_t nent = 0;
    for (int d = 0; d < 3; ++d)
        for (int t = 0; t < g.nt[d]; ++t) {
            int cells = g.N[d] - t * T;
            if (cells > g.Tt[d]) cells = g.Tt[d];
            nent += (size_t)(cells + order - 1);
        }

    // carve the scratch array
    const size_t nn = (size_t)n;
    const size_t psz = (size_t)g.E[0] * g.E[1] * g.Pz;
    size_t at = 0;
    auto take = [&](size_t bytes) {
        size_t o = at;
        at += round256(bytes ? bytes : 1);
        return o;
    };
    const size_t o_count = take(sizeof(int) * g.ntiles);
    const size_t o_tiles = take(sizeof(int2) * g.ntiles);
    const size_t o_tile = take(sizeof(int) * nn);
    const size_t o_slot = take(sizeof(int) * nn);
    const size_t o_rec = take(sizeof(Rec<float>) * nn);
    const size_t o_cell = take(sizeof(int) * nn);
    const size_t o_srec = take(sizeof(Rec<float>) * nn);
    const size_t o_scell = take(sizeof(int) * nn);
    const size_t o_sorig = take(sizeof(int) * nn);
    const size_t o_patch = take(sizeof(float) * psz * g.ntiles);
    const size_t o_off = take(sizeof(int) * 3 * (size_t)nmax1);
    const size_t o_ent = take(sizeof(int2) * nent);
    const size_t o_status = take(sizeof(int));
    const size_t o_ticket = take(sizeof(int));
    if (at > kNoAllocScratchBytes) return PPPM_ERR_TOO_LARGE;
    unsigned char* b = static_cast<unsigned char*>(base);
    int* tile_count = reinterpret_cast<int*>(b + o_count);
    int2* tiles = reinterpret_cast<int2*>(b + o_tiles);
    int* tile_of = reinterpret_cast<int*>(b + o_tile);
    int* slot_of = reinterpret_cast<int*>(b + o_slot);
    Rec<float>* rec = reinterpret_cast<Rec<float>*>(b + o_rec);
    int* cell = reinterpret_cast<int*>(b + o_cell);
    Rec<float>* srec = reinterpret_cast<Rec<float>*>(b + o_srec);
    int* scell = reinterpret_cast<int*>(b + o_scell);
    int* sorig = reinterpret_cast<int*>(b + o_sorig);
    float* patch = reinterpret_cast<float*>(b + o_patch);
    int* cov_off = reinterpret_cast<int*>(b + o_off);
    int2* cov_ent = reinterpret_cast<int2*>(b + o_ent);
    int* status = reinterpret_cast<int*>(b + o_status);
    int* ticket = reinterpret_cast<int*>(b + o_ticket);

    cudaStream_t s = (cudaStream_t)stream;
    const double h3 = (box[0] / mesh[0]) * (box[1] / mesh[1]) * (box[2] / mesh[2]);
#define NA_CK(x)                                        \
    do {                                                \
        if ((x) != cudaSuccess) return PPPM_ERR_CUDA;   \
    } while (0)
    k_cover_lists<<<1, kCoverThreads, 0, s>>>(g, nmax1, cov_off, cov_ent);
    NA_CK(cudaGetLastError());
    NA_CK(cudaMemsetAsync(tile_count, 0, sizeof(int) * g.ntiles, s));
    NA_CK(cudaMemsetAsync(status, 0, sizeof(int), s));
    NA_CK(cudaMemsetAsync(ticket, 0, sizeof(int), s));
    NA_CK((launch_bin<float, double>(s, g, pos, q, (int)n, tile_count, tile_of, slot_of, rec, cell, status)));
    NA_CK(launch_scan(s, tile_count, g.ntiles, tiles));
    NA_CK(launch_scatter<float>(s, g, (int)n, tile_of, slot_of, tiles, rec, cell, srec, scell, sorig));
    NA_CK(launch_spread<float>(s, g, tiles, srec, scell, sorig, patch, slot_of, tile_of, ticket));
    NA_CK(launch_fold<float>(s, g, patch, cov_off, cov_ent, (float)(1.0 / h3), rho));
#undef NA_CK
    return PPPM_OK;
}
