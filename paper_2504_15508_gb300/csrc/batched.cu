// Many independent boxes in one persistent launch.
//
// Every box goes through the same stages as a single-box evaluation (bin,
// scan, scatter, spread, fold + z FFT, y FFT, x FFT + influence + energy,
// y inverse, z inverse, gather).  The host lists the work as items
// (box, stage, chunk), stage-major: all boxes' stage-0 items first, then all
// stage-1 items, and so on.  A grid of persistent blocks pulls items from a
// device counter in that order; an item of stage s of box b first waits until
// all stage s-1 items of box b are done.  Because every item waits only on
// items queued before it, and those have all been pulled by running blocks,
// the waits always end; each one is still bounded by a spin limit, after
// which the block records PPPM_ERR_TIMEOUT (bit 4 of the status word), skips
// the item's work and goes on, so that no launch can hang.
//
// Data produced inside the launch is read with L2-only loads (__ldcg): L1 is
// not coherent across SMs and a block may meet data another SM rewrote.
//
// FP32 only; the tile edge T (4 or 8) is a template parameter picked by the
// batch plan's autotuner.
#include <cuda.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "fft_common.cuh"
#include "internal.cuh"

namespace pppm {
namespace batch {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
enum Stage { S_BIN, S_SCAN, S_SCATTER, S_SPREAD, S_ZR2C, S_YFWD, S_XINF, S_YINV, S_ZC2R, S_GATHER, NSTAGE };
constexpr int kSiteChunk = 1024;  // sites per bin / scatter item
constexpr int kZPairs = 8;        // row pairs per z-pass item, at least
constexpr int kZRows = 512;       // and up to about this many points (pairs x Nz) an item
constexpr int kSpreadTiles = kWarps;
constexpr int kGatherTiles = 2;   // four warps per tile

struct BoxDesc {
    Geo g;
    Radix rad[3];
    Bundle bd;
    FieldLayout fl;
    long long site0;
    int nsite;
    int tile0;   // into tile_count
    int ts0;     // into tile_start (ntiles + 1 entries per box)
    long long patch0;
    long long c0;  // complex half-spectrum offset
    long long f0;  // padded field offset (3 fields)
    long long G0;
    int tw0[3];
    int cov0;
    int nmax;
    int part0;
    float e_scale, c_field, beta;
    int zp;  // row pairs per z-pass item
    int nitems[NSTAGE];
};

struct Bufs {
    const float* pos;
    const float* q;
    float* forces;
    double* energy;
    double* virial;
    int* tile_count;
    int* tile_start;
    int* tile_of;
    int* slot_of;
    Rec<float>* rec;
    int* cell;
    int* scell;
    int* sorig;
    Rec<float>* srec;  // tile order: the sites' records (B-spline arguments, charge)
    float* patch;
    float2* cx0;
    float2* cx1;
    float2* cx2;
    float* fields;
    const float* G;
    const float2* tw;
    const int4* cov2;
    float* partial;
    unsigned int* box_counter;
    int* box_fail;  // set when a wait of the box ran out: its later stages skip their work
    int* status;
    double prefactor;
    int dft_max;  // lines up to this length take the tensor-core DFT (0: all take the FFT)
    int qgroup;     // node size of the int32-quantised DFT (0: off)
    double qscale;  // its scale
    int wait_probe;  // 1: box 0's scan waits for one binning item more than exist (its wait runs out)
    RedRows red_rows;  // lane -> stencil row of the spread's shared-memory atomics
};

// ------------------------------------------------------------------ helpers
// All p B-spline weights N_p(x0 + j), j = 0..p-1, by the Cox-de Boor recursion
// (the same weights the single-box path takes from its piece table).
template <int P>
__device__ __forceinline__ void bspline_all(float x0, float w[P]) {
    w[0] = 1.f;
#pragma unroll
    for (int m = 2; m <= P; ++m) {
        const float inv = 1.f / (m - 1);
        w[m - 1] = (1.f - x0) * w[m - 2] * inv;  // (m - x0 - (m - 1)) N_{m-1}(x0 + m - 2)
#pragma unroll
        for (int j = m - 2; j >= 1; --j) w[j] = ((x0 + j) * w[j] + (m - x0 - j) * w[j - 1]) * inv;
        w[0] = x0 * w[0] * inv;
    }
}

__device__ __forceinline__ bool locate_f(float x, float s_hi, float s_lo, int N, bool odd, int& g, float& x0) {
    float u = x * s_hi;
    const float e = fmaf(x, s_hi, -u);
    float ul = fmaf(x, s_lo, e);
    const bool ok = fabsf(u) < 4.0e6f;
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
    const int gi = (int)gf % N;
    g = gi < 0 ? gi + N : gi;
    return ok;
}

template <typename X>
__device__ __forceinline__ X ldcg(const X* p) { return __ldcg(p); }

// ------------------------------------------------------------------ stages
template <int P>
__device__ void st_bin(const BoxDesc& D, int idx, const Bufs& B) {
    const Geo& g = D.g;
    const bool odd = (g.order & 1) != 0;
    const int lane = threadIdx.x & 31;
    for (int k = 0; k < kSiteChunk / kThreads; ++k) {
        const int i = idx * kSiteChunk + k * kThreads + threadIdx.x;
        const bool valid = i < D.nsite;
        const long long gi = D.site0 + i;
        int t = -1 - lane, lx = 0, ly = 0, lz = 0;
        Rec<float> r;
        if (valid) {
            int gc[3];
            bool ok = true;
#pragma unroll
            for (int d = 0; d < 3; ++d) ok &= locate_f(B.pos[3 * gi + d], g.s_hi[d], g.s_lo[d], g.N[d], odd, gc[d], r.x0[d]);
            float qi = B.q[gi];
            if (!isfinite(qi)) { ok = false; qi = 0.f; }
            r.q = qi;
            if (!ok) atomicOr(B.status, 1);
            const int tx = gc[0] / g.T, ty = gc[1] / g.T, tz = gc[2] / g.T;
            t = (tx * g.nt[1] + ty) * g.nt[2] + tz;
            lx = gc[0] - tx * g.T;
            ly = gc[1] - ty * g.T;
            lz = gc[2] - tz * g.T;
        }
        const unsigned peers = __match_any_sync(0xffffffffu, t);
        const int leader = __ffs(peers) - 1;
        const int rank = __popc(peers & ((1u << lane) - 1u));
        int base = 0;
        if (valid && lane == leader) base = atomicAdd(&B.tile_count[D.tile0 + t], __popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (valid) {
            B.tile_of[gi] = t;
            B.slot_of[gi] = base + rank;
            B.rec[gi] = r;
            B.cell[gi] = lx | (ly << 8) | (lz << 16);
        }
    }
}

__device__ void st_scan(const BoxDesc& D, const Bufs& B, int* sh) {
    const int nt = D.g.ntiles;
    const int tid = threadIdx.x;
    const int chunk = (nt + kThreads - 1) / kThreads;
    const int b = tid * chunk, e = min(b + chunk, nt);
    int sum = 0;
    for (int i = b; i < e; ++i) sum += ldcg(&B.tile_count[D.tile0 + i]);
    sh[tid] = sum;
    __syncthreads();
    for (int off = 1; off < kThreads; off <<= 1) {
        const int v = tid >= off ? sh[tid - off] : 0;
        __syncthreads();
        sh[tid] += v;
        __syncthreads();
    }
    int run = sh[tid] - sum;
    for (int i = b; i < e; ++i) {
        B.tile_start[D.ts0 + i] = run;
        run += ldcg(&B.tile_count[D.tile0 + i]);
    }
    if (tid == kThreads - 1) B.tile_start[D.ts0 + nt] = sh[kThreads - 1];
}

// Scatter: a thread's kSiteChunk / kThreads sites, their independent loads
// (tile, slot, record, cell) issued together before any store, then each
// site's cell, index and 16-byte record written at its slot of the tile
// order (the spread and the gather evaluate the weights from the record).
template <int P>
__device__ void st_scatter(const BoxDesc& D, int idx, const Bufs& B) {
    constexpr int KS = kSiteChunk / kThreads;
    int tt[KS], sl[KS], cl[KS];
    float4 rr[KS];
#pragma unroll
    for (int k = 0; k < KS; ++k) {
        const int i = idx * kSiteChunk + k * kThreads + threadIdx.x;
        if (i < D.nsite) {
            const long long gi = D.site0 + i;
            tt[k] = ldcg(&B.tile_of[gi]);
            sl[k] = ldcg(&B.slot_of[gi]);
            cl[k] = ldcg(&B.cell[gi]);
            rr[k] = __ldcg(reinterpret_cast<const float4*>(&B.rec[gi]));
        }
    }
    int st[KS];
#pragma unroll
    for (int k = 0; k < KS; ++k) {
        const int i = idx * kSiteChunk + k * kThreads + threadIdx.x;
        if (i < D.nsite) st[k] = ldcg(&B.tile_start[D.ts0 + tt[k]]);
    }
#pragma unroll
    for (int k = 0; k < KS; ++k) {
        const int i = idx * kSiteChunk + k * kThreads + threadIdx.x;
        if (i >= D.nsite) continue;
        const long long dst = D.site0 + st[k] + sl[k];
        B.scell[dst] = cl[k];
        B.sorig[dst] = i;
        reinterpret_cast<float4*>(B.srec)[dst] = rr[k];
    }
}

// Spread: the item's kSpreadTiles tiles one after another, each by the whole
// block.  A tile's patch is accumulated in shared memory exactly, as two
// int32 words a value (split_scale / split_term: sum of rint(x 2^k) and sum
// of the remainders at 2^-K) with 32-bit shared-memory atomics: integer sums
// do not depend on the order in which the warps add their sites, so the
// result is bitwise reproducible with no ordering of the tile's sites.  The
// patch keeps the padded pitch and is written out as FP32.  The sites' weight
// rows are evaluated from their records into shared memory, kThreads sites
// at a time (one thread a site), before the warps spread them.
template <int P, int TILE>
struct SpreadRed {
    static constexpr int E = TILE + P - 1, PZ = E | 1, PLANE = E * PZ, PSIZE = E * PLANE;
    static constexpr int WSR = wstride(P) + 4;  // row pitch: conflict-free 16-byte row stores
    // accumulators, per-warp maxima, then the rows (16-byte aligned)
    static constexpr size_t rows_off() { return (2 * sizeof(int) * PSIZE + sizeof(unsigned) * kWarps + 15) / 16 * 16; }
    static constexpr size_t bytes() { return rows_off() + sizeof(float) * kThreads * WSR; }
};

// Site t's weight row from its record: q W_x, W_y, W_z (p each), padded.
template <int P>
__device__ __forceinline__ void weight_row(const float4& r, float (&w)[wstride(P)]) {
    float t[P];
    bspline_all<P>(r.x, t);
#pragma unroll
    for (int a = 0; a < P; ++a) w[a] = t[a] * r.w;
    bspline_all<P>(r.y, t);
#pragma unroll
    for (int a = 0; a < P; ++a) w[P + a] = t[a];
    bspline_all<P>(r.z, t);
#pragma unroll
    for (int a = 0; a < P; ++a) w[2 * P + a] = t[a];
#pragma unroll
    for (int a = 3 * P; a < wstride(P); ++a) w[a] = 0.f;
}

template <int P, int TILE>
__device__ void st_spread(const BoxDesc& D, int idx, const Bufs& B, unsigned char* smem) {
    typedef SpreadRed<P, TILE> L;
    constexpr int PZ = L::PZ, PLANE = L::PLANE, PSIZE = L::PSIZE, WSR = L::WSR;
    constexpr int WS = wstride(P);
    int* acc_h = reinterpret_cast<int*>(smem);
    int* acc_l = acc_h + PSIZE;
    unsigned* wmax = reinterpret_cast<unsigned*>(acc_l + PSIZE);
    float* rows = reinterpret_cast<float*>(smem + L::rows_off());
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int NR = (P * P + 31) / 32;
    int roff[NR], riy[NR], riz[NR];
    bool ract[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) {
        const int slot = lane + 32 * j;
        ract[j] = slot < P * P;
        const int row = ract[j] ? (int)B.red_rows.row[slot] : 0;
        riy[j] = row / P;
        riz[j] = row % P;
        roff[j] = riy[j] * PZ + riz[j];
    }
    for (int k = 0; k < kSpreadTiles; ++k) {
        const int tile = idx * kSpreadTiles + k;
        if (tile >= D.g.ntiles) break;  // uniform across the block
        const int s0 = ldcg(&B.tile_start[D.ts0 + tile]);
        const int c = ldcg(&B.tile_start[D.ts0 + tile + 1]) - s0;
        const long long sb = D.site0 + s0;
        for (int i = threadIdx.x; i < 2 * PSIZE; i += kThreads) acc_h[i] = 0;
        unsigned mb = 0;  // largest |q Wx| of the tile
        for (int t = threadIdx.x; t < c; t += kThreads) {
            const float4 r = __ldcg(reinterpret_cast<const float4*>(B.srec + sb + t));
            float wx[P];
            bspline_all<P>(r.x, wx);
#pragma unroll
            for (int a = 0; a < P; ++a) mb = max(mb, __float_as_uint(fabsf(wx[a] * r.w)));
        }
        mb = __reduce_max_sync(0xffffffffu, mb);
        if (lane == 0) wmax[warp] = mb;
        __syncthreads();
#pragma unroll
        for (int w = 0; w < kWarps; ++w) mb = max(mb, wmax[w]);
        const SplitScale sc = split_scale(mb, c);
        const float S = pow2f(sc.k), twoK = pow2f(sc.K);
        for (int c0 = 0; c0 < c; c0 += kThreads) {  // chunks of kThreads sites (uniform)
            const int cn = min(kThreads, c - c0);
            if (c0 > 0) __syncthreads();  // the previous chunk's rows are read no more
            if ((int)threadIdx.x < cn) {
                const float4 r = __ldcg(reinterpret_cast<const float4*>(B.srec + sb + c0 + threadIdx.x));
                float w[WS];
                weight_row<P>(r, w);
                float4* o = reinterpret_cast<float4*>(rows + threadIdx.x * WSR);
#pragma unroll
                for (int a = 0; a < WS / 4; ++a) o[a] = make_float4(w[4 * a], w[4 * a + 1], w[4 * a + 2], w[4 * a + 3]);
            }
            __syncthreads();
            for (int t = warp; t < cn; t += kWarps) {
                const float* w = rows + t * WSR;
                float wxq[P];
#pragma unroll
                for (int a = 0; a < P; ++a) wxq[a] = w[a];
                const int cl = ldcg(&B.scell[sb + c0 + t]);
                const int lx = cl & 255, ly = (cl >> 8) & 255, lz = (cl >> 16) & 255;
                const int base0 = lx * PLANE + ly * PZ + lz;
#pragma unroll
                for (int jr = 0; jr < NR; ++jr) {
                    if (ract[jr]) {
                        const float wyzS = w[P + riy[jr]] * w[2 * P + riz[jr]] * S;
                        const int b = base0 + roff[jr];
#pragma unroll
                        for (int a = 0; a < P; ++a) {
                            int h, l;
                            split_term(wxq[a] * wyzS, twoK, h, l);
                            atomicAdd(&acc_h[b + a * PLANE], h);
                            atomicAdd(&acc_l[b + a * PLANE], l);
                        }
                    }
                }
            }
        }
        __syncthreads();
        float* dst = B.patch + D.patch0 + (long long)tile * PSIZE;
        const float i1 = pow2f(-sc.k), i2 = pow2f(-sc.K);
        for (int i = threadIdx.x; i < PSIZE; i += kThreads) {
            const long long v = (long long)acc_h[i] * (1ll << sc.K) + acc_l[i];
            dst[i] = sc.finite ? __ll2float_rn(v) * i2 * i1 : __int_as_float(0x7fffffff);
        }
        __syncthreads();
    }
}

// fold of the patches covering (x, y, z): up to four cover slots per axis
// (ragged last tiles near the periodic seam can add a third or fourth), in a
// fixed order, empty slots (tile -1) skipped
struct Cover4 {
    int t[4], c[4];
};

__device__ __forceinline__ Cover4 load_cover(const Bufs& B, const BoxDesc& D, int d, int m) {
    const int4 a = __ldg(&B.cov2[D.cov0 + 2 * (d * D.nmax + m)]);
    const int4 b = __ldg(&B.cov2[D.cov0 + 2 * (d * D.nmax + m) + 1]);
    Cover4 r;
    r.t[0] = a.x; r.c[0] = a.y; r.t[1] = a.z; r.c[1] = a.w;
    r.t[2] = b.x; r.c[2] = b.y; r.t[3] = b.z; r.c[3] = b.w;
    return r;
}

__device__ __forceinline__ float fold_point_b(const BoxDesc& D, const Bufs& B, const Cover4& cx, const Cover4& cy,
                                              int z) {
    const Geo& g = D.g;
    const Cover4 cz = load_cover(B, D, 2, z);
    const int psz = g.E[0] * g.E[1] * g.Pz;
    float sum = 0.f;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        if (cx.t[a] < 0) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            if (cy.t[b] < 0) continue;
            const int tb = (cx.t[a] * g.nt[1] + cy.t[b]) * g.nt[2];
            const int ob = (cx.c[a] * g.E[1] + cy.c[b]) * g.Pz;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if (cz.t[c] < 0) continue;
                sum += ldcg(&B.patch[D.patch0 + (long long)(tb + cz.t[c]) * psz + ob + cz.c[c]]);
            }
        }
    }
    return sum;
}

// With the quantised DFT every transform follows the paper's chain literally:
// each real z line is its own complex line (no two-for-one packing, whose
// quantised partial sums would mix two lines), and each of the three ik
// spectra -i k_d phi_hat is formed before the first inverse pass (the default
// chain multiplies by k_y and k_z after the x pass, which is the same only
// in exact arithmetic).
// node size of the quantised DFT along axis d of this box: lines of at most
// 18 points that the node size divides; 0 = not quantised
__device__ __forceinline__ int qg(const BoxDesc& D, const Bufs& B, int d) {
    const int L = D.rad[d].L, g = B.qgroup;
    return (g > 0 && L <= kDftTcMax && L % g == 0) ? g : 0;
}

__device__ __forceinline__ bool quant_chain(const BoxDesc& D, const Bufs& B) {
    return (qg(D, B, 0) | qg(D, B, 1) | qg(D, B, 2)) != 0;
}

__device__ void st_zr2c_quant(const BoxDesc& D, int idx, const Bufs& B, unsigned char* smem) {
    const Geo& g = D.g;
    const int Nz = g.N[2], Hz = g.Hz, rows = g.N[0] * g.N[1];
    float2* a = reinterpret_cast<float2*>(smem);
    float2* b = a + D.zp * Nz;
    const int pair0 = idx * D.zp;
    const int np = min(D.zp, (rows + 1) / 2 - pair0);
    float2* out = B.cx0 + D.c0;
    for (int half = 0; half < 2; ++half) {
        for (int p = threadIdx.x >> 5; p < np; p += kWarps) {
            const int r = 2 * (pair0 + p) + half;
            if (r < rows) {
                const int x = r / g.N[1], y = r - x * g.N[1];
                const Cover4 cx = load_cover(B, D, 0, x), cy = load_cover(B, D, 1, y);
                for (int t = threadIdx.x & 31; t < Nz; t += 32)
                    a[p * Nz + t] = make_float2(fold_point_b(D, B, cx, cy, t), 0.f);
            } else {
                for (int t = threadIdx.x & 31; t < Nz; t += 32) a[p * Nz + t] = make_float2(0.f, 0.f);
            }
        }
        __syncthreads();
        const float2* res = dft_quant(a, b, np, Nz, 1, Nz, qg(D, B, 2), B.qscale, B.tw + D.tw0[2], -1.f, B.status);
        for (int p = threadIdx.x >> 5; p < np; p += kWarps) {
            const int r = 2 * (pair0 + p) + half;
            if (r < rows)
                for (int k = threadIdx.x & 31; k < Hz; k += 32) out[(long long)r * Hz + k] = res[p * Nz + k];
        }
        __syncthreads();
    }
}

template <bool Q, bool CT>
__device__ void st_zr2c(const BoxDesc& D, int idx, const Bufs& B, unsigned char* smem) {
    if constexpr (Q)
        if (qg(D, B, 2) > 0) return st_zr2c_quant(D, idx, B, smem);
    const Geo& g = D.g;
    const int Nz = g.N[2], Hz = g.Hz, rows = g.N[0] * g.N[1];
    float2* a = reinterpret_cast<float2*>(smem);
    float2* b = a + D.zp * Nz;
    const int pair0 = idx * D.zp;
    const int np = min(D.zp, (rows + 1) / 2 - pair0);
    for (int p = threadIdx.x >> 5; p < np; p += kWarps) {
        const int r0 = 2 * (pair0 + p), r1 = r0 + 1;
        const int x0 = r0 / g.N[1], y0 = r0 - x0 * g.N[1];
        const Cover4 cx0 = load_cover(B, D, 0, x0), cy0 = load_cover(B, D, 1, y0);
        Cover4 cx1, cy1;
        for (int k = 0; k < 4; ++k) { cx1.t[k] = -1; cx1.c[k] = 0; cy1.t[k] = -1; cy1.c[k] = 0; }
        if (r1 < rows) {
            const int x1 = r1 / g.N[1], y1 = r1 - x1 * g.N[1];
            cx1 = load_cover(B, D, 0, x1);
            cy1 = load_cover(B, D, 1, y1);
        }        for (int t = threadIdx.x & 31; t < Nz; t += 32)
            a[p * Nz + t] = make_float2(fold_point_b(D, B, cx0, cy0, t), fold_point_b(D, B, cx1, cy1, t));
    }
    __syncthreads();
    float2* res = line_transform_t<Q, CT, -1, false>(a, b, np, Nz, 1, D.rad[2], B.tw + D.tw0[2], B.dft_max, qg(D, B, 2), B.qscale, B.status);
    float2* out = B.cx0 + D.c0;
    for (int p = threadIdx.x >> 5; p < np; p += kWarps) {
        const int r0 = 2 * (pair0 + p), r1 = r0 + 1;
        for (int k = threadIdx.x & 31; k < Hz; k += 32) {
            const float2 z = res[p * Nz + k];
            const float2 zc = cconj(res[p * Nz + (k == 0 ? 0 : Nz - k)]);
            out[(long long)r0 * Hz + k] = cscale(cadd(z, zc), 0.5f);
            const float2 d = csub(z, zc);
            if (r1 < rows) out[(long long)r1 * Hz + k] = make_float2(0.5f * d.y, -0.5f * d.x);
        }
    }
}

// lines along y of the complex spectrum (outer index x), in place
template <bool Q, bool CT>
__device__ void st_yfwd(const BoxDesc& D, int idx, const Bufs& B, unsigned char* smem) {
    const Geo& g = D.g;
    const int Hz = g.Hz, L = g.N[1], Bw = D.bd.B;
    const int outer = idx / D.bd.nb, bi = idx - outer * D.bd.nb;
    const int kz0 = bi * Bw, nl = min(Bw, Hz - kz0);
    float2* a = reinterpret_cast<float2*>(smem);
    float2* b = a + L * Bw;
    float2* base = B.cx0 + D.c0 + (long long)outer * L * Hz + kz0;
    for (int i = threadIdx.x; i < L * nl; i += kThreads) {
        const int t = i / nl, l = i - t * nl;
        a[t * Bw + l] = ldcg(&base[(long long)t * Hz + l]);
    }
    __syncthreads();
    float2* res = line_transform_t<Q, CT, -1, true>(a, b, nl, 1, Bw, D.rad[1], B.tw + D.tw0[1], B.dft_max, qg(D, B, 1), B.qscale, B.status);
    for (int i = threadIdx.x; i < L * nl; i += kThreads) {
        const int t = i / nl, l = i - t * nl;
        base[(long long)t * Hz + l] = res[t * Bw + l];
    }
}

__device__ __forceinline__ void tsum_pair(float& h, float& l, float h2, float l2) {
    const float s = h + h2, bp = s - h;
    const float err = (h - (s - bp)) + (h2 - bp);
    h = s;
    l = l + l2 + err;
}

// x FFT, influence multiply with energy/virial, inverse x FFTs; the last item
// of a box sums that box's partials (compensated FP32, FP64 final)
template <bool Q, bool CT>
__device__ void st_xinf(const BoxDesc& D, int box, int idx, const Bufs& B, unsigned char* smem) {
    const Geo& g = D.g;
    const int Nx = g.N[0], Ny = g.N[1], Nz = g.N[2], Hz = g.Hz, Bw = D.bd.B;
    const int y = idx / D.bd.nb, bi = idx - y * D.bd.nb;
    const int kz0 = bi * Bw, nl = min(Bw, Hz - kz0);
    const long long es = (long long)Ny * Hz;
    float2* a0 = reinterpret_cast<float2*>(smem);
    float2* a1 = a0 + Nx * Bw;
    float2* b0 = a1 + Nx * Bw;
    float2* b1 = b0 + Nx * Bw;
    float* red = reinterpret_cast<float*>(b1 + Nx * Bw);  // [kWarps][14]
    float2* base = B.cx0 + D.c0 + (long long)y * Hz + kz0;
    for (int i = threadIdx.x; i < Nx * nl; i += kThreads) {
        const int t = i / nl, l = i - t * nl;
        a0[t * Bw + l] = ldcg(&base[t * es + l]);
    }
    __syncthreads();
    float2* rh = line_transform_t<Q, CT, -1, true>(a0, a1, nl, 1, Bw, D.rad[0], B.tw + D.tw0[0], B.dft_max, qg(D, B, 0), B.qscale, B.status);
    float2* pbuf = (rh == a0) ? a1 : a0;
    const int my = y <= Ny / 2 ? y : y - Ny;
    const float ky = g.kfac_f[1] * my;
    const bool nyq_y = (Ny % 2 == 0) && (y == Ny / 2);
    const float inv4b2 = 1.f / (4.f * D.beta * D.beta);
    float hi[7], lo[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) { hi[q] = 0.f; lo[q] = 0.f; }
    const float* G = B.G + D.G0;
    for (int i = threadIdx.x; i < Nx * nl; i += kThreads) {
        const int t = i / nl, l = i - t * nl;
        const int kz = kz0 + l;
        const int mx = t <= Nx / 2 ? t : t - Nx;
        const float kx = g.kfac_f[0] * mx, kzv = g.kfac_f[2] * kz;
        const bool nyq_x = (Nx % 2 == 0) && (t == Nx / 2);
        const float gk = __ldg(&G[((long long)t * Ny + y) * Hz + kz]);
        const float2 v = rh[t * Bw + l];
        const bool plane1 = (kz == 0) || ((Nz % 2 == 0) && (kz == Nz / 2));
        const float k2 = kx * kx + ky * ky + kzv * kzv;
        if (k2 > 0.f) {
            const float e = (plane1 ? 1.f : 2.f) * D.e_scale * gk * (v.x * v.x + v.y * v.y);
            const float c = 2.f * (1.f + k2 * inv4b2) / k2;
            const float fxy = (plane1 || (nyq_x == nyq_y)) ? 1.f : 0.f;
            const float fxz = (plane1 || !nyq_x) ? 1.f : 0.f;
            const float fyz = (plane1 || !nyq_y) ? 1.f : 0.f;
            const float vals[7] = {e, e * (1.f - c * kx * kx), e * (1.f - c * ky * ky), e * (1.f - c * kzv * kzv),
                                   -e * c * kx * ky * fxy, -e * c * kx * kzv * fxz, -e * c * ky * kzv * fyz};
#pragma unroll
            for (int q = 0; q < 7; ++q) tsum_pair(hi[q], lo[q], vals[q], 0.f);
        }
        const float2 Pv = cscale(v, gk * D.c_field);
        const float kxd = nyq_x ? 0.f : kx;
        pbuf[t * Bw + l] = Pv;
        b0[t * Bw + l] = make_float2(kxd * Pv.y, -kxd * Pv.x);
    }
    __syncthreads();
    bool chain = false;
    if constexpr (Q) chain = quant_chain(D, B);
    if (chain) {
        float2* obx = B.cx1 + D.c0 + (long long)y * Hz + kz0;
        // x inverses of -i k_x P (-> cx1), -i k_y P (-> cx2) and -i k_z P (-> cx0)
        float2* oby = B.cx2 + D.c0 + (long long)y * Hz + kz0;
        const float kyd = nyq_y ? 0.f : ky;
        for (int d = 0; d < 3; ++d) {
            if (d > 0) {
                for (int i = threadIdx.x; i < Nx * nl; i += kThreads) {
                    const int t = i / nl, l = i - t * nl, kz = kz0 + l;
                    const float kd = d == 1 ? kyd : (((Nz % 2 == 0) && (kz == Nz / 2)) ? 0.f : g.kfac_f[2] * kz);
                    const float2 Pv = pbuf[t * Bw + l];
                    b0[t * Bw + l] = make_float2(kd * Pv.y, -kd * Pv.x);
                }
                __syncthreads();
            }
            const float2* r = line_transform_t<Q, CT, 1, true>(b0, b1, nl, 1, Bw, D.rad[0], B.tw + D.tw0[0], B.dft_max,
                                                qg(D, B, 0), B.qscale, B.status);
            float2* o = d == 0 ? obx : (d == 1 ? oby : base);
            for (int i = threadIdx.x; i < Nx * nl; i += kThreads) {
                const int t = i / nl, l = i - t * nl;
                o[t * es + l] = r[t * Bw + l];
            }
            __syncthreads();
        }
    } else {
        float2* rA = line_transform_t<Q, CT, 1, true>(pbuf, rh, nl, 1, Bw, D.rad[0], B.tw + D.tw0[0], B.dft_max, qg(D, B, 0), B.qscale, B.status);
        float2* rB = line_transform_t<Q, CT, 1, true>(b0, b1, nl, 1, Bw, D.rad[0], B.tw + D.tw0[0], B.dft_max, qg(D, B, 0), B.qscale, B.status);
        float2* obx = B.cx1 + D.c0 + (long long)y * Hz + kz0;
        for (int i = threadIdx.x; i < Nx * nl; i += kThreads) {
            const int t = i / nl, l = i - t * nl;
            base[t * es + l] = rA[t * Bw + l];
            obx[t * es + l] = rB[t * Bw + l];
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        float h = hi[q], l2 = lo[q];
        for (int off = 16; off > 0; off >>= 1)
            tsum_pair(h, l2, __shfl_down_sync(0xffffffffu, h, off), __shfl_down_sync(0xffffffffu, l2, off));
        if (lane == 0) { red[warp * 14 + 2 * q] = h; red[warp * 14 + 2 * q + 1] = l2; }
    }
    __syncthreads();
    __shared__ bool last;
    if (threadIdx.x < 7) {
        const int q = threadIdx.x;
        float h = red[2 * q], l2 = red[2 * q + 1];
        for (int w = 1; w < kWarps; ++w) tsum_pair(h, l2, red[w * 14 + 2 * q], red[w * 14 + 2 * q + 1]);
        B.partial[(long long)(D.part0 + idx) * 14 + 2 * q] = h;
        B.partial[(long long)(D.part0 + idx) * 14 + 2 * q + 1] = l2;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&B.box_counter[box], 1u) == (unsigned)D.nitems[S_XINF] - 1;
    __syncthreads();
    if (last) {
        __threadfence();
        if (warp < 7) {
            const int q = warp;
            float h = 0.f, l2 = 0.f;
            for (int it = lane; it < D.nitems[S_XINF]; it += 32)
                tsum_pair(h, l2, ldcg(&B.partial[(long long)(D.part0 + it) * 14 + 2 * q]),
                          ldcg(&B.partial[(long long)(D.part0 + it) * 14 + 2 * q + 1]));
            for (int off = 16; off > 0; off >>= 1)
                tsum_pair(h, l2, __shfl_down_sync(0xffffffffu, h, off), __shfl_down_sync(0xffffffffu, l2, off));
            if (lane == 0) {
                const double s = ((double)h + (double)l2) * B.prefactor;
                if (q == 0) B.energy[box] = s;
                else B.virial[6 * box + q - 1] = s;
            }
        }
    }
}

template <bool Q, bool CT>
__device__ void st_yinv(const BoxDesc& D, int idx, const Bufs& B, unsigned char* smem) {
    const Geo& g = D.g;
    const int Ny = g.N[1], Hz = g.Hz, Bw = D.bd.B;
    const int x = idx / D.bd.nb, bi = idx - x * D.bd.nb;
    const int kz0 = bi * Bw, nl = min(Bw, Hz - kz0);
    const long long off = D.c0 + (long long)x * Ny * Hz + kz0;
    float2* buf = reinterpret_cast<float2*>(smem);
    const int sz = Ny * Bw;
    for (int i = threadIdx.x; i < Ny * nl; i += kThreads) {
        const int t = i / nl, l = i - t * nl;
        const float2 va = ldcg(&B.cx0[off + (long long)t * Hz + l]);
        const int my = t <= Ny / 2 ? t : t - Ny;
        const float kyd = ((Ny % 2 == 0) && (t == Ny / 2)) ? 0.f : g.kfac_f[1] * my;
        buf[t * Bw + l] = va;
        bool chain = false;
        if constexpr (Q) chain = quant_chain(D, B);
        // the chain mode formed -i k_y P before the x pass, in cx2
        buf[2 * sz + t * Bw + l] = chain ? ldcg(&B.cx2[off + (long long)t * Hz + l]) : make_float2(kyd * va.y, -kyd * va.x);
        buf[4 * sz + t * Bw + l] = ldcg(&B.cx1[off + (long long)t * Hz + l]);
    }
    __syncthreads();
    float2* rC = line_transform_t<Q, CT, 1, true>(buf, buf + sz, nl, 1, Bw, D.rad[1], B.tw + D.tw0[1], B.dft_max, qg(D, B, 1), B.qscale, B.status);
    float2* rD = line_transform_t<Q, CT, 1, true>(buf + 2 * sz, buf + 3 * sz, nl, 1, Bw, D.rad[1], B.tw + D.tw0[1], B.dft_max, qg(D, B, 1), B.qscale, B.status);
    float2* rE = line_transform_t<Q, CT, 1, true>(buf + 4 * sz, buf + 5 * sz, nl, 1, Bw, D.rad[1], B.tw + D.tw0[1], B.dft_max, qg(D, B, 1), B.qscale, B.status);
    for (int i = threadIdx.x; i < Ny * nl; i += kThreads) {
        const int t = i / nl, l = i - t * nl;
        B.cx0[off + (long long)t * Hz + l] = rC[t * Bw + l];
        B.cx2[off + (long long)t * Hz + l] = rD[t * Bw + l];
        B.cx1[off + (long long)t * Hz + l] = rE[t * Bw + l];
    }
}

// z inverse of (Ex', D, -i kz' C) -> E_x, E_y, E_z into the padded field layout
// one z line of a field, written into the padded layout with its ghost images
__device__ __forceinline__ void store_field_row(const BoxDesc& D, const Bufs& B, int f, int r, const float2* line,
                                                bool imag) {
    const Geo& g = D.g;
    const FieldLayout& fl = D.fl;
    const int Nz = g.N[2], Ny = g.N[1], Nx = g.N[0];
    const int kmin = g.kmin, zlen = Nz + g.order - 1;
    float* out = B.fields + D.f0 + f * fl.fstride;
    const int x = r / Ny, y = r - x * Ny;
    const int px0 = x - kmin, py0 = y - kmin;
    const int pxg = px0 + Nx < fl.Xp ? px0 + Nx : (px0 - Nx >= 0 ? px0 - Nx : -1);
    const int pyg = py0 + Ny < fl.Yp ? py0 + Ny : (py0 - Ny >= 0 ? py0 - Ny : -1);
    float* o00 = out + ((long long)px0 * fl.Yp + py0) * fl.Zp;
    float* o10 = pxg >= 0 ? out + ((long long)pxg * fl.Yp + py0) * fl.Zp : nullptr;
    float* o01 = pyg >= 0 ? out + ((long long)px0 * fl.Yp + pyg) * fl.Zp : nullptr;
    float* o11 = (pxg >= 0 && pyg >= 0) ? out + ((long long)pxg * fl.Yp + pyg) * fl.Zp : nullptr;
    for (int pz = threadIdx.x & 31; pz < zlen; pz += 32) {
        int zz = pz + kmin;
        zz += zz < 0 ? Nz : 0;
        zz -= zz >= Nz ? Nz : 0;
        const float2 zv = line[zz];
        const float v = imag ? zv.y : zv.x;
        o00[pz] = v;
        if (o10) o10[pz] = v;
        if (o01) o01[pz] = v;
        if (o11) o11[pz] = v;
    }
}

// quantised z inverse: each row's Hermitian line transformed on its own
// (fields already multiplied by -i k_d), real part kept
__device__ void st_zc2r_quant(const BoxDesc& D, int idx, const Bufs& B, unsigned char* smem) {
    const Geo& g = D.g;
    const int Nz = g.N[2], Hz = g.Hz, rows = g.N[0] * g.N[1];
    const int pair0 = idx * D.zp;
    const int np = min(D.zp, (rows + 1) / 2 - pair0);
    const int nlines = 3 * np;
    float2* a = reinterpret_cast<float2*>(smem);
    float2* b = a + 3 * D.zp * Nz;
    const float2* srcs[3] = {B.cx1 + D.c0, B.cx2 + D.c0, B.cx0 + D.c0};
    for (int half = 0; half < 2; ++half) {
        for (int line = threadIdx.x >> 5; line < nlines; line += kWarps) {
            const int f = line / np, p = line - f * np;
            const int r = 2 * (pair0 + p) + half;
            for (int t = threadIdx.x & 31; t < Nz; t += 32) {
                const int kk = t < Hz ? t : Nz - t;
                float2 h = r < rows ? ldcg(&srcs[f][(long long)r * Hz + kk]) : make_float2(0.f, 0.f);
                if (t >= Hz) h.y = -h.y;
                a[line * Nz + t] = h;
            }
        }
        __syncthreads();
        const float2* res = dft_quant(a, b, nlines, Nz, 1, Nz, qg(D, B, 2), B.qscale, B.tw + D.tw0[2], 1.f, B.status);
        for (int line = threadIdx.x >> 5; line < nlines; line += kWarps) {
            const int f = line / np, p = line - f * np;
            const int r = 2 * (pair0 + p) + half;
            if (r < rows) store_field_row(D, B, f, r, res + line * Nz, false);
        }
        __syncthreads();
    }
}

template <bool Q, bool CT>
__device__ void st_zc2r(const BoxDesc& D, int idx, const Bufs& B, unsigned char* smem) {
    if constexpr (Q)
        if (qg(D, B, 2) > 0) return st_zc2r_quant(D, idx, B, smem);
    bool chain = false;
    if constexpr (Q) chain = quant_chain(D, B);
    const Geo& g = D.g;
    const int Nz = g.N[2], Hz = g.Hz, rows = g.N[0] * g.N[1], Ny = g.N[1], Nx = g.N[0];
    const int pair0 = idx * D.zp;
    const int np = min(D.zp, (rows + 1) / 2 - pair0);
    const int nlines = 3 * np;
    float2* a = reinterpret_cast<float2*>(smem);
    float2* b = a + 3 * D.zp * Nz;
    const float2* srcs[3] = {B.cx1 + D.c0, B.cx2 + D.c0, B.cx0 + D.c0};
    const bool even = (Nz % 2) == 0;
    for (int line = threadIdx.x >> 5; line < nlines; line += kWarps) {
        const int f = line / np, p = line - f * np;
        const int r0 = 2 * (pair0 + p), r1 = r0 + 1;
        const float2* src = srcs[f];
        for (int t = threadIdx.x & 31; t < Nz; t += 32) {
            const int kk = t < Hz ? t : Nz - t;
            float2 h0 = ldcg(&src[(long long)r0 * Hz + kk]);
            float2 h1 = r1 < rows ? ldcg(&src[(long long)r1 * Hz + kk]) : make_float2(0.f, 0.f);
            if (f == 2 && !chain) {
                const float kzd = (even && kk == Nz / 2) ? 0.f : g.kfac_f[2] * kk;
                h0 = make_float2(kzd * h0.y, -kzd * h0.x);
                h1 = make_float2(kzd * h1.y, -kzd * h1.x);
            }
            if (kk == 0 || (even && kk == Nz / 2)) { h0.y = 0.f; h1.y = 0.f; }
            if (t >= Hz) { h0.y = -h0.y; h1.y = -h1.y; }
            a[line * Nz + t] = make_float2(h0.x - h1.y, h0.y + h1.x);
        }
    }
    __syncthreads();
    float2* res = line_transform_t<Q, CT, 1, false>(a, b, nlines, Nz, 1, D.rad[2], B.tw + D.tw0[2], B.dft_max, qg(D, B, 2), B.qscale, B.status);
    const FieldLayout& fl = D.fl;
    const int kmin = g.kmin, zlen = Nz + g.order - 1;
    for (int line = threadIdx.x >> 5; line < nlines; line += kWarps) {
        const int f = line / np, p = line - f * np;
        float* out = B.fields + D.f0 + f * fl.fstride;
        for (int half = 0; half < 2; ++half) {
            const int r = 2 * (pair0 + p) + half;
            if (r >= rows) break;
            const int x = r / Ny, y = r - x * Ny;
            const int px0 = x - kmin, py0 = y - kmin;
            const int pxg = px0 + Nx < fl.Xp ? px0 + Nx : (px0 - Nx >= 0 ? px0 - Nx : -1);
            const int pyg = py0 + Ny < fl.Yp ? py0 + Ny : (py0 - Ny >= 0 ? py0 - Ny : -1);
            float* o00 = out + ((long long)px0 * fl.Yp + py0) * fl.Zp;
            float* o10 = pxg >= 0 ? out + ((long long)pxg * fl.Yp + py0) * fl.Zp : nullptr;
            float* o01 = pyg >= 0 ? out + ((long long)px0 * fl.Yp + pyg) * fl.Zp : nullptr;
            float* o11 = (pxg >= 0 && pyg >= 0) ? out + ((long long)pxg * fl.Yp + pyg) * fl.Zp : nullptr;
            for (int pz = threadIdx.x & 31; pz < zlen; pz += 32) {
                int zz = pz + kmin;
                zz += zz < 0 ? Nz : 0;
                zz -= zz >= Nz ? Nz : 0;
                const float2 zv = res[line * Nz + zz];
                const float v = half ? zv.y : zv.x;
                o00[pz] = v;
                if (o10) o10[pz] = v;
                if (o01) o01[pz] = v;
                if (o11) o11[pz] = v;
            }
        }
    }
}

// Gather: two tiles per item, four warps per tile; the tile's stencil patch is
// read from the padded fields (no wrap needed) into shared memory.
template <int P, int TILE>
__device__ void st_gather(const BoxDesc& D, int idx, const Bufs& B, unsigned char* smem) {
    constexpr int E = TILE + P - 1, PZ = E | 1, PLANE = E * PZ, PSIZE = E * PLANE;
    constexpr int WS = wstride(P), WSP = WS + 4;
    const Geo& g = D.g;
    const FieldLayout& fl = D.fl;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = warp >> 2, wg = warp & 3;  // tile group, warp within it
    const int tile = idx * kGatherTiles + grp;
    float* fx = reinterpret_cast<float*>(smem) + grp * 3 * PSIZE;
    float* fy = fx + PSIZE;
    float* fz = fy + PSIZE;
    float* st_w = reinterpret_cast<float*>(smem) + kGatherTiles * 3 * PSIZE;
    int* st_cell = reinterpret_cast<int*>(st_w + kWarps * 8 * WSP);
    int* st_orig = st_cell + kWarps * 8;
    int s0 = 0, s1 = 0;
    if (tile < g.ntiles) {
        s0 = ldcg(&B.tile_start[D.ts0 + tile]);
        s1 = ldcg(&B.tile_start[D.ts0 + tile + 1]);
        const int tx = tile / (g.nt[1] * g.nt[2]);
        const int ty = (tile / g.nt[2]) % g.nt[1];
        const int tz = tile % g.nt[2];
        const float* f0 = B.fields + D.f0;
        for (int i = (threadIdx.x & 127); i < E * E * E; i += 128) {
            const int x = i / (E * E), y = (i / E) % E, z = i % E;
            const int px = tx * TILE + x, py = ty * TILE + y, pz = tz * TILE + z;
            float vx = 0.f, vy = 0.f, vz = 0.f;
            if (px < fl.Xp && py < fl.Yp && pz < fl.Zp) {
                const long long o = ((long long)px * fl.Yp + py) * fl.Zp + pz;
                vx = ldcg(&f0[o]);
                vy = ldcg(&f0[fl.fstride + o]);
                vz = ldcg(&f0[2 * fl.fstride + o]);
            }
            const int so = x * PLANE + y * PZ + z;
            fx[so] = vx;
            fy[so] = vy;
            fz[so] = vz;
        }
    }
    __syncthreads();
    if (tile >= g.ntiles) return;
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
    float* ww = st_w + warp * 8 * WSP;
    int* wcell = st_cell + warp * 8;
    int* worig = st_orig + warp * 8;
    const int nsites = s1 - s0;
    const long long sb = D.site0 + s0;
    const int sj = lane >> 2, sd = lane & 3;  // record entry sd of site sj of a batch
    for (int b = wg * 8; b < nsites; b += 4 * 8) {
        const int nb = min(8, nsites - b);
        {  // lanes 4 j + d (d < 3) evaluate the p weights of axis d of site j (x times q)
            const float rv = sj < nb ? ldcg(reinterpret_cast<const float*>(B.srec + sb + b + sj) + sd) : 0.f;
            const float qj = __shfl_sync(0xffffffffu, rv, lane | 3);
            if (sj < nb && sd < 3) {
                float t[P];
                bspline_all<P>(rv, t);
                if (sd == 0) {
#pragma unroll
                    for (int a = 0; a < P; ++a) t[a] = t[a] * qj;
                }
#pragma unroll
                for (int a = 0; a < P; ++a) ww[sj * WSP + sd * P + a] = t[a];
            }
        }
        if (lane < nb) {
            wcell[lane] = ldcg(&B.scell[sb + b + lane]);
            worig[lane] = ldcg(&B.sorig[sb + b + lane]);
        }
        __syncwarp();
        float v[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = 0.f;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (j < nb) {
                const int cl = wcell[j];
                const int lx = cl & 255, ly = (cl >> 8) & 255, lz = (cl >> 16) & 255;
                const float* wj = ww + j * WSP;
                const int base0 = lx * PLANE + ly * PZ + lz;
#pragma unroll
                for (int jr = 0; jr < NR; ++jr) {
                    if (ract[jr]) {
                        const float wyz = wj[P + riy[jr]] * wj[2 * P + riz[jr]];
                        const int o0 = base0 + roff[jr];
#pragma unroll
                        for (int a = 0; a < P; ++a) {
                            const float w = wj[a] * wyz;
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
                const float send = up ? v[i] : v[i + h];
                const float keep = up ? v[i + h] : v[i];
                v[i] = keep + __shfl_xor_sync(0xffffffffu, send, h);
            }
        }
        const int site = lane >> 2, comp = lane & 3;
        if (site < nb && comp < 3)
            B.forces[3 * (D.site0 + worig[site]) + comp] = (float)B.prefactor * v[0];
        __syncwarp();
    }
}

// ------------------------------------------------------------------ the persistent kernel
template <int P, int TILE, bool Q>
__global__ void __launch_bounds__(kThreads, 2)  // two resident blocks per SM: 16 warps to hide latency
k_batched(const BoxDesc* __restrict__ boxes, const int2* __restrict__ items, int nitems, unsigned int* head,
          int* done, Bufs B, long long spin_limit) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_item;
    __shared__ int s_ok;
    __shared__ __align__(16) BoxDesc sbox;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(head, 1u);
        __syncthreads();
        const int it = s_item;
        if (it >= nitems) return;
        const int2 I = items[it];
        const int box = I.x & 0xffff, stage = I.x >> 16, idx = I.y;
        {
            const int* src = reinterpret_cast<const int*>(boxes + box);
            int* dst = reinterpret_cast<int*>(&sbox);
            for (int w = threadIdx.x; w < (int)(sizeof(BoxDesc) / sizeof(int)); w += kThreads) dst[w] = src[w];
        }
        if (threadIdx.x == 0) {
            int ok = 1;
            if (stage > 0) {
                // the probe makes one wait unsatisfiable, so that it must run out
                const int need = boxes[box].nitems[stage - 1] + ((B.wait_probe && box == 0 && stage == S_SCAN) ? 1 : 0);
                const volatile int* cnt = done + box * NSTAGE + stage - 1;
                long long spins = 0;
                while (*cnt < need) {
                    if (++spins > spin_limit) {
                        ok = 0;
                        atomicOr(B.status, 4);
                        *(volatile int*)(B.box_fail + box) = 1;
                        break;
                    }
                    __nanosleep(64);
                }
            }
            __threadfence();
            if (ok && *(volatile int*)(B.box_fail + box)) ok = 0;
            s_ok = ok;
        }
        __syncthreads();
        if (s_ok) {
            switch (stage) {
                case S_BIN: st_bin<P>(sbox, idx, B); break;
                case S_SCAN: st_scan(sbox, B, reinterpret_cast<int*>(smem)); break;
                case S_SCATTER: st_scatter<P>(sbox, idx, B); break;
                case S_SPREAD: st_spread<P, TILE>(sbox, idx, B, smem); break;
                case S_ZR2C: st_zr2c<Q, false>(sbox, idx, B, smem); break;
                case S_YFWD: st_yfwd<Q, false>(sbox, idx, B, smem); break;
                case S_XINF: st_xinf<Q, false>(sbox, box, idx, B, smem); break;
                case S_YINV: st_yinv<Q, false>(sbox, idx, B, smem); break;
                case S_ZC2R: st_zc2r<Q, false>(sbox, idx, B, smem); break;
                case S_GATHER: st_gather<P, TILE>(sbox, idx, B, smem); break;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(done + box * NSTAGE + stage, 1);
        }
    }
}

template <int P, int TILE>
size_t stage_smem(int maxN, int maxB, int maxZ) {
    size_t m = SpreadRed<P, TILE>::bytes();
    m = std::max(m, (size_t)kThreads * sizeof(int));
    m = std::max(m, (size_t)(2 * maxZ) * sizeof(float2));
    m = std::max(m, (size_t)(2 * maxN * maxB) * sizeof(float2));
    m = std::max(m, (size_t)(4 * maxN * maxB) * sizeof(float2) + kWarps * 14 * sizeof(float));
    m = std::max(m, (size_t)(6 * maxN * maxB) * sizeof(float2));
    m = std::max(m, (size_t)(6 * maxZ) * sizeof(float2));
    constexpr int E = TILE + P - 1, PZ = E | 1;
    m = std::max(m, (size_t)kGatherTiles * 3 * E * E * PZ * sizeof(float) +
                        (size_t)kWarps * 8 * (wstride(P) + 4) * sizeof(float) + 2 * kWarps * 8 * sizeof(int));
    return (m + 127) / 128 * 128;
}

template <int P, int TILE, bool Q>
cudaError_t launch(cudaStream_t s, const BoxDesc* boxes, const int2* items, int nitems, unsigned int* head, int* done,
                   const Bufs& B, long long spin_limit, int maxN, int maxB, int maxZ, int* grid_out) {
    const size_t smem = stage_smem<P, TILE>(maxN, maxB, maxZ);
    cudaError_t e = cudaFuncSetAttribute(k_batched<P, TILE, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batched<P, TILE, Q>, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int grid = std::min(nsm * per_sm, nitems);
    if (grid_out) *grid_out = grid;
    k_batched<P, TILE, Q><<<grid, kThreads, smem, s>>>(boxes, items, nitems, head, done, B, spin_limit);
    return cudaGetLastError();
}

// Shared memory of one stage alone (the persistent kernel takes the largest).
template <int P, int TILE>
size_t stage_smem_of(int stage, int maxN, int maxB, int maxZ) {
    constexpr int E = TILE + P - 1, PZ = E | 1;
    size_t m = 0;
    switch (stage) {
        case S_BIN: case S_SCATTER: m = 16; break;
        case S_SCAN: m = (size_t)kThreads * sizeof(int); break;
        case S_SPREAD: m = SpreadRed<P, TILE>::bytes(); break;
        case S_ZR2C: m = (size_t)(2 * maxZ) * sizeof(float2); break;
        case S_YFWD: m = (size_t)(2 * maxN * maxB) * sizeof(float2); break;
        case S_XINF: m = (size_t)(4 * maxN * maxB) * sizeof(float2) + kWarps * 14 * sizeof(float); break;
        case S_YINV: m = (size_t)(6 * maxN * maxB) * sizeof(float2); break;
        case S_ZC2R: m = (size_t)(6 * maxZ) * sizeof(float2); break;
        case S_GATHER:
            m = (size_t)kGatherTiles * 3 * E * E * PZ * sizeof(float) +
                (size_t)kWarps * 8 * (wstride(P) + 4) * sizeof(float) + 2 * kWarps * 8 * sizeof(int);
            break;
    }
    return (m + 127) / 128 * 128;
}

// Staged launch: one kernel per stage over that stage's items of every box
// (block b takes item b of the stage's contiguous range of the stage-major
// list); stream order replaces the persistent kernel's waits, and each stage
// gets its own register and shared-memory budget.
template <int P, int TILE, bool Q, int STAGE>
__global__ void __launch_bounds__(kThreads, 4)  // four resident blocks an SM: 64 registers
k_stage(const BoxDesc* __restrict__ boxes, const int2* __restrict__ items, Bufs B) {
    pdl_enter();
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(16) BoxDesc sbox;
    const int2 I = items[blockIdx.x];
    const int box = I.x & 0xffff, idx = I.y;
    {
        const int* src = reinterpret_cast<const int*>(boxes + box);
        int* dst = reinterpret_cast<int*>(&sbox);
        for (int w = threadIdx.x; w < (int)(sizeof(BoxDesc) / sizeof(int)); w += kThreads) dst[w] = src[w];
    }
    __syncthreads();
    if constexpr (STAGE == S_BIN) st_bin<P>(sbox, idx, B);
    if constexpr (STAGE == S_SCAN) st_scan(sbox, B, reinterpret_cast<int*>(smem));
    if constexpr (STAGE == S_SCATTER) st_scatter<P>(sbox, idx, B);
    if constexpr (STAGE == S_SPREAD) st_spread<P, TILE>(sbox, idx, B, smem);
    if constexpr (STAGE == S_ZR2C) st_zr2c<Q, !Q>(sbox, idx, B, smem);
    if constexpr (STAGE == S_YFWD) st_yfwd<Q, !Q>(sbox, idx, B, smem);
    if constexpr (STAGE == S_XINF) st_xinf<Q, !Q>(sbox, box, idx, B, smem);
    if constexpr (STAGE == S_YINV) st_yinv<Q, !Q>(sbox, idx, B, smem);
    if constexpr (STAGE == S_ZC2R) st_zc2r<Q, !Q>(sbox, idx, B, smem);
    if constexpr (STAGE == S_GATHER) st_gather<P, TILE>(sbox, idx, B, smem);
}

template <int P, int TILE, bool Q, int STAGE>
cudaError_t launch_one_stage(cudaStream_t s, const BoxDesc* boxes, const int2* items, int start, int count,
                             const Bufs& B, int maxN, int maxB, int maxZ) {
    if (count == 0) return cudaSuccess;
    const size_t smem = stage_smem_of<P, TILE>(STAGE, maxN, maxB, maxZ);
    auto kern = k_stage<P, TILE, Q, STAGE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return launch_k(kern, dim3(count), dim3(kThreads), smem, s, boxes, items + start, B);
}

template <int P, int TILE, bool Q>
cudaError_t launch_staged(cudaStream_t s, const BoxDesc* boxes, const int2* items, const int* stage_start,
                          const Bufs& B, int maxN, int maxB, int maxZ) {
    PdlScope pdl(true);
    cudaError_t e = cudaSuccess;
#define PPPM_STAGE(ST)                                                                                      \
    e = launch_one_stage<P, TILE, Q, ST>(s, boxes, items, stage_start[ST], stage_start[ST + 1] - stage_start[ST], \
                                         B, maxN, maxB, maxZ);                                              \
    if (e != cudaSuccess) return e;
    // the FFT stages do not depend on the order or the tile edge: one
    // instantiation of each serves every batch
#define PPPM_FFT_STAGE(ST)                                                                                  \
    e = launch_one_stage<5, 8, Q, ST>(s, boxes, items, stage_start[ST], stage_start[ST + 1] - stage_start[ST], \
                                      B, maxN, maxB, maxZ);                                                 \
    if (e != cudaSuccess) return e;
    PPPM_STAGE(S_BIN) PPPM_STAGE(S_SCAN) PPPM_STAGE(S_SCATTER) PPPM_STAGE(S_SPREAD) PPPM_FFT_STAGE(S_ZR2C)
    PPPM_FFT_STAGE(S_YFWD) PPPM_FFT_STAGE(S_XINF) PPPM_FFT_STAGE(S_YINV) PPPM_FFT_STAGE(S_ZC2R) PPPM_STAGE(S_GATHER)
#undef PPPM_FFT_STAGE
#undef PPPM_STAGE
    return e;
}

}  // namespace batch
}  // namespace pppm

// ====================================================================== host side
using namespace pppm;
using namespace pppm::batch;

struct pppm_batch {
    int nbox = 0;
    int order = 5;
    double beta = 0.4;
    double prefactor = 1.0;
    long long spin_limit = 1ll << 24;
    int dft_max = 0;            // short lines on the tensor cores (off: measured 2 % slower on the batch)
    int quant_group = 0;        // int32-quantised DFT of short lines (an accuracy ablation; off)
    double quant_scale = 1e7;
    int wait_probe = 0;
    int launch_mode = PPPM_BATCH_AUTO;  // requested launch form
    bool staged = false;        // in use: one kernel per stage instead of the persistent launch
    bool mode_tuned = false;    // the launch form has been chosen for the current layout
    std::vector<double> boxes;  // nbox * 3
    std::vector<int> meshes;    // nbox * 3
    int tile = 0;               // chosen tile edge (0 = not tuned yet)
    int forced_tile = 0;
    // device tables
    float* G = nullptr;
    float2* tw = nullptr;
    size_t G_elems = 0, tw_elems = 0;
    std::vector<long long> G0;
    std::vector<int> tw0;  // 3 per box
    // per-tile-edge layout
    struct Layout {
        int T = 0;
        std::vector<BoxDesc> desc;
        std::vector<int2> items;
        int stage_start[NSTAGE + 1] = {};  // each stage's range in the stage-major list
        BoxDesc* d_desc = nullptr;
        int2* d_items = nullptr;
        int4* d_cov2 = nullptr;
        int ntile_total = 0, ntile_start_total = 0;
        long long patch_total = 0;
        int part_total = 0;
        int maxN = 0, maxB = 0, maxZ = 0;
    };
    Layout lay[2];  // T = 4, 8
    std::vector<long long> offsets;  // the offsets the layouts were built for
    // work buffers
    long long cap_sites = 0;
    int* tile_count = nullptr;
    int* tile_start = nullptr;
    int* tile_of = nullptr;
    int* slot_of = nullptr;
    Rec<float>* rec = nullptr;
    int* cell = nullptr;
    int* scell = nullptr;
    int* sorig = nullptr;
    Rec<float>* srec = nullptr;
    float* patch = nullptr;
    long long patch_cap = 0;
    float2* cx[3] = {nullptr, nullptr, nullptr};
    float* fields = nullptr;
    float* partial = nullptr;
    int partial_cap = 0;
    int tile_cap = 0;
    long long c_total = 0, f_total = 0;
    unsigned int* head = nullptr;
    int* done = nullptr;
    unsigned int* box_counter = nullptr;
    int* box_fail = nullptr;
    int* status = nullptr;
    // graph cache
    cudaGraphExec_t exec = nullptr;
    const void* key[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    int key_tile = 0;
    cudaStream_t last = nullptr;
    int last_grid = 0;
};

namespace {

bool smooth235_b(int n) {
    if (n < 1) return false;
    for (int r : {2, 3, 5})
        while (n % r == 0) n /= r;
    return n == 1;
}

int smooth_at_least_b(double x) {
    int n = std::max(1, (int)std::ceil(x - 1e-12));
    while (!smooth235_b(n)) ++n;
    return n;
}

Radix make_radix_b(int L) {
    Radix r{};
    r.L = L;
    int m = L;
    for (int f : {4, 2, 3, 5})
        while (m % f == 0) {
            r.r[r.n++] = f;
            m /= f;
        }
    return r;
}

#define BK(x)                                         \
    do {                                              \
        if ((x) != cudaSuccess) return PPPM_ERR_CUDA; \
    } while (0)

template <typename X>
int balloc(X** p, size_t bytes) {
    *p = nullptr;
    return cudaMalloc((void**)p, bytes ? bytes : 16) == cudaSuccess ? PPPM_OK : PPPM_ERR_CUDA;
}
template <typename X>
void bfree(X*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

// geometry of one box (same conventions as a single-box plan)
Geo box_geo(const double* L, const int* N, int order, int T) {
    Geo g{};
    for (int d = 0; d < 3; ++d) {
        g.N[d] = N[d];
        g.L[d] = L[d];
        g.s[d] = (double)N[d] / L[d];
        g.s_hi[d] = (float)g.s[d];
        g.s_lo[d] = (float)(g.s[d] - (double)g.s_hi[d]);
        g.kfac_d[d] = 6.283185307179586476925 / L[d];
        g.kfac_f[d] = (float)g.kfac_d[d];
    }
    g.Hz = N[2] / 2 + 1;
    g.order = order;
    g.kmin = (order % 2) ? -(order - 1) / 2 : -order / 2 + 1;
    g.T = T;
    g.ntiles = 1;
    for (int d = 0; d < 3; ++d) {
        g.Tt[d] = T < N[d] ? T : N[d];
        g.nt[d] = (N[d] + T - 1) / T;
        g.E[d] = g.Tt[d] + order - 1;
        g.ntiles *= g.nt[d];
    }
    g.Pz = g.E[2] | 1;
    return g;
}

// Build descriptors, the two-slot cover tables and the stage-major item list
// for tile edge T and the given site offsets.
int build_layout(pppm_batch* P, int li, int T) {
    auto& Y = P->lay[li];
    bfree(Y.d_desc);
    bfree(Y.d_items);
    bfree(Y.d_cov2);
    Y = pppm_batch::Layout();
    Y.T = T;
    const int p = P->order;
    std::vector<int4> cov;
    long long patch0 = 0, c0 = 0, f0 = 0;
    int tile0 = 0, ts0 = 0, part0 = 0;
    Y.desc.resize(P->nbox);
    for (int b = 0; b < P->nbox; ++b) {
        BoxDesc& D = Y.desc[b];
        D = BoxDesc();
        const double* L = &P->boxes[3 * b];
        const int* N = &P->meshes[3 * b];
        D.g = box_geo(L, N, p, T);
        for (int d = 0; d < 3; ++d) {
            if (D.g.Tt[d] != T || N[d] < T + p - 1) return PPPM_ERR_BAD_MESH;  // every axis needs full tiles
            D.rad[d] = make_radix_b(N[d]);
            D.tw0[d] = P->tw0[3 * b + d];
        }
        const int maxN = std::max(N[0], std::max(N[1], N[2]));
        Y.maxN = std::max(Y.maxN, maxN);
        int nb = (D.g.Hz + 15) / 16;
        D.bd.B = (D.g.Hz + nb - 1) / nb;
        D.bd.nb = (D.g.Hz + D.bd.B - 1) / D.bd.B;
        Y.maxB = std::max(Y.maxB, D.bd.B);
        D.fl.padded = 1;
        D.fl.Xp = N[0] + p - 1;
        D.fl.Yp = N[1] + p - 1;
        D.fl.Zp = (N[2] + p - 1 + 3) & ~3;
        D.fl.fstride = (long long)D.fl.Xp * D.fl.Yp * D.fl.Zp;
        D.fl.pstride = 1;
        D.site0 = P->offsets[b];
        D.nsite = (int)(P->offsets[b + 1] - P->offsets[b]);
        D.tile0 = tile0;
        D.ts0 = ts0;
        tile0 += D.g.ntiles;
        ts0 += D.g.ntiles + 1;
        D.patch0 = patch0;
        patch0 += (long long)D.g.ntiles * D.g.E[0] * D.g.E[1] * D.g.Pz;
        const long long NH = (long long)N[0] * N[1] * D.g.Hz;
        D.c0 = c0;
        c0 += NH;
        D.f0 = f0;
        f0 += 3 * D.fl.fstride;
        D.G0 = P->G0[b];
        const double h3 = (L[0] / N[0]) * (L[1] / N[1]) * (L[2] / N[2]);
        const double Ntot = (double)N[0] * N[1] * N[2];
        D.e_scale = (float)(1.0 / (2.0 * Ntot * h3));
        D.c_field = (float)(1.0 / (Ntot * h3));
        D.beta = (float)P->beta;
        // cover table (two slots per mesh index)
        D.nmax = maxN;
        D.cov0 = (int)cov.size();
        cov.resize(cov.size() + 2 * 3 * (size_t)maxN, make_int4(-1, 0, -1, 0));
        for (int d = 0; d < 3; ++d)
            for (int t = 0; t < D.g.nt[d]; ++t) {
                int cells = N[d] - t * T;
                if (cells > T) cells = T;
                for (int c = 0; c < cells + p - 1; ++c) {
                    int m = (t * T + D.g.kmin + c) % N[d];
                    if (m < 0) m += N[d];
                    int4& v0 = cov[D.cov0 + 2 * ((size_t)d * maxN + m)];
                    int4& v1 = cov[D.cov0 + 2 * ((size_t)d * maxN + m) + 1];
                    if (v0.x < 0) { v0.x = t; v0.y = c; }
                    else if (v0.z < 0) { v0.z = t; v0.w = c; }
                    else if (v1.x < 0) { v1.x = t; v1.y = c; }
                    else if (v1.z < 0) { v1.z = t; v1.w = c; }
                    else return PPPM_ERR_BAD_MESH;
                }
            }
        // every stage waits only on the one before it, so no stage may be
        // empty: a box without sites still gets one (idle) binning and one
        // scatter item, or its spread would not wait for its scan
        D.nitems[S_BIN] = std::max(1, (D.nsite + kSiteChunk - 1) / kSiteChunk);
        D.nitems[S_SCAN] = 1;
        D.nitems[S_SCATTER] = D.nitems[S_BIN];
        D.nitems[S_SPREAD] = (D.g.ntiles + kSpreadTiles - 1) / kSpreadTiles;
        const int npairs = (N[0] * N[1] + 1) / 2;
        // short z lines: more row pairs an item, so that an item holds ~kZRows points
        D.zp = std::max(kZPairs, kZRows / N[2]);
        Y.maxZ = std::max(Y.maxZ, D.zp * N[2]);
        D.nitems[S_ZR2C] = (npairs + D.zp - 1) / D.zp;
        D.nitems[S_YFWD] = N[0] * D.bd.nb;
        D.nitems[S_XINF] = N[1] * D.bd.nb;
        D.nitems[S_YINV] = N[0] * D.bd.nb;
        D.nitems[S_ZC2R] = D.nitems[S_ZR2C];
        D.nitems[S_GATHER] = (D.g.ntiles + kGatherTiles - 1) / kGatherTiles;
        D.part0 = part0;
        part0 += D.nitems[S_XINF];
    }
    // stage-major work list; bigger boxes first within a stage
    std::vector<int> order(P->nbox);
    for (int b = 0; b < P->nbox; ++b) order[b] = b;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return Y.desc[a].g.ntiles > Y.desc[b].g.ntiles; });
    for (int s = 0; s < NSTAGE; ++s) {
        Y.stage_start[s] = (int)Y.items.size();
        for (int b : order)
            for (int i = 0; i < Y.desc[b].nitems[s]; ++i) Y.items.push_back(make_int2(b | (s << 16), i));
    }
    Y.stage_start[NSTAGE] = (int)Y.items.size();
    Y.ntile_total = tile0;
    Y.ntile_start_total = ts0;
    Y.patch_total = patch0;
    Y.part_total = part0;
    P->c_total = c0;
    P->f_total = f0;
    int rc;
    if ((rc = balloc(&Y.d_desc, sizeof(BoxDesc) * Y.desc.size())) != PPPM_OK) return rc;
    if ((rc = balloc(&Y.d_items, sizeof(int2) * Y.items.size())) != PPPM_OK) return rc;
    if ((rc = balloc(&Y.d_cov2, sizeof(int4) * cov.size())) != PPPM_OK) return rc;
    BK(cudaMemcpy(Y.d_desc, Y.desc.data(), sizeof(BoxDesc) * Y.desc.size(), cudaMemcpyHostToDevice));
    BK(cudaMemcpy(Y.d_items, Y.items.data(), sizeof(int2) * Y.items.size(), cudaMemcpyHostToDevice));
    BK(cudaMemcpy(Y.d_cov2, cov.data(), sizeof(int4) * cov.size(), cudaMemcpyHostToDevice));
    // grow the shared work buffers
    if (Y.patch_total > P->patch_cap) {
        bfree(P->patch);
        if ((rc = balloc(&P->patch, sizeof(float) * Y.patch_total)) != PPPM_OK) return rc;
        P->patch_cap = Y.patch_total;
    }
    if (std::max(Y.ntile_start_total, Y.part_total * 14) > P->tile_cap) {
        bfree(P->tile_count);
        bfree(P->tile_start);
        bfree(P->partial);
        const int cap = std::max(Y.ntile_start_total, Y.part_total * 14);
        if ((rc = balloc(&P->tile_count, sizeof(int) * cap)) != PPPM_OK) return rc;
        if ((rc = balloc(&P->tile_start, sizeof(int) * cap)) != PPPM_OK) return rc;
        if ((rc = balloc(&P->partial, sizeof(float) * cap)) != PPPM_OK) return rc;
        P->tile_cap = cap;
    }
    return PPPM_OK;
}

int ensure_sites(pppm_batch* P, long long n) {
    if (n <= P->cap_sites) return PPPM_OK;
    bfree(P->tile_of);
    bfree(P->slot_of);
    bfree(P->rec);
    bfree(P->cell);
    bfree(P->scell);
    bfree(P->sorig);
    bfree(P->srec);
    P->cap_sites = 0;
    int rc;
    if ((rc = balloc(&P->tile_of, sizeof(int) * n)) != PPPM_OK) return rc;
    if ((rc = balloc(&P->slot_of, sizeof(int) * n)) != PPPM_OK) return rc;
    if ((rc = balloc(&P->rec, sizeof(Rec<float>) * n)) != PPPM_OK) return rc;
    if ((rc = balloc(&P->cell, sizeof(int) * n)) != PPPM_OK) return rc;
    if ((rc = balloc(&P->scell, sizeof(int) * n)) != PPPM_OK) return rc;
    if ((rc = balloc(&P->sorig, sizeof(int) * n)) != PPPM_OK) return rc;
    if ((rc = balloc(&P->srec, sizeof(Rec<float>) * n)) != PPPM_OK) return rc;
    P->cap_sites = n;
    return PPPM_OK;
}

// Launch one batched evaluation (memsets + persistent kernel) on stream s.
int enqueue(pppm_batch* P, cudaStream_t s, int li, const float* pos, const float* q, double* energies, float* forces,
            double* virials) {
    auto& Y = P->lay[li];
    BK(cudaMemsetAsync(P->tile_count, 0, sizeof(int) * Y.ntile_total, s));
    BK(cudaMemsetAsync(P->head, 0, sizeof(unsigned int), s));
    BK(cudaMemsetAsync(P->done, 0, sizeof(int) * NSTAGE * P->nbox, s));
    BK(cudaMemsetAsync(P->box_counter, 0, sizeof(unsigned int) * P->nbox, s));
    BK(cudaMemsetAsync(P->box_fail, 0, sizeof(int) * P->nbox, s));
    Bufs B{};
    B.pos = pos;
    B.q = q;
    B.forces = forces;
    B.energy = energies;
    B.virial = virials;
    B.tile_count = P->tile_count;
    B.tile_start = P->tile_start;
    B.tile_of = P->tile_of;
    B.slot_of = P->slot_of;
    B.rec = P->rec;
    B.cell = P->cell;
    B.scell = P->scell;
    B.sorig = P->sorig;
    B.srec = P->srec;
    B.patch = P->patch;
    B.cx0 = P->cx[0];
    B.cx1 = P->cx[1];
    B.cx2 = P->cx[2];
    B.fields = P->fields;
    B.G = P->G;
    B.tw = P->tw;
    B.cov2 = Y.d_cov2;
    B.partial = P->partial;
    B.box_counter = P->box_counter;
    B.box_fail = P->box_fail;
    B.status = P->status;
    B.prefactor = P->prefactor;
    B.dft_max = P->dft_max;
    B.qgroup = P->quant_group;
    B.qscale = P->quant_scale;
    B.wait_probe = P->wait_probe;
    B.red_rows = red_rows(P->order, (Y.T + P->order - 1) | 1);
    cudaError_t e = cudaErrorInvalidValue;
    const int n = (int)Y.items.size();
    const bool quant = P->quant_group > 0;
#define BATCH_CASE(PP, TT, QQ)                                                                                   \
    if (P->order == PP && Y.T == TT && quant == QQ)                                                              \
        e = P->staged ? launch_staged<PP, TT, QQ>(s, Y.d_desc, Y.d_items, Y.stage_start, B, Y.maxN, Y.maxB,      \
                                                  Y.maxZ)                                                          \
                      : launch<PP, TT, QQ>(s, Y.d_desc, Y.d_items, n, P->head, P->done, B, P->spin_limit, Y.maxN, \
                                           Y.maxB, Y.maxZ, &P->last_grid);
    BATCH_CASE(3, 4, false) BATCH_CASE(3, 8, false) BATCH_CASE(5, 4, false) BATCH_CASE(5, 8, false)
    BATCH_CASE(7, 4, false) BATCH_CASE(7, 8, false)
    BATCH_CASE(5, 4, true) BATCH_CASE(5, 8, true)  // the quantised ablation: order 5 only
#undef BATCH_CASE
    BK(e);
    return PPPM_OK;
}

int prepare(pppm_batch* P, const int64_t* offsets) {
    std::vector<long long> off(P->nbox + 1);
    BK(cudaMemcpy(off.data(), offsets, sizeof(long long) * (P->nbox + 1), cudaMemcpyDeviceToHost));
    for (int b = 0; b < P->nbox; ++b)
        if (off[b + 1] < off[b] || off[b] < 0) return PPPM_ERR_INVALID_ARG;
    if (off != P->offsets) {
        P->offsets = off;
        int rc;
        if ((rc = ensure_sites(P, off[P->nbox])) != PPPM_OK) return rc;
        if ((rc = build_layout(P, 0, 4)) != PPPM_OK) return rc;
        // tile edge 8 needs every axis of every box to hold 8 + p - 1 points;
        // if one does not, only tile edge 4 is available
        rc = build_layout(P, 1, 8);
        if (rc == PPPM_ERR_BAD_MESH) P->lay[1].T = 0;
        else if (rc != PPPM_OK) return rc;
        if (P->exec) cudaGraphExecDestroy(P->exec);
        P->exec = nullptr;
        P->tile = P->forced_tile;
    }
    return PPPM_OK;
}

// Autotuner: time warm evaluations of every candidate tile edge (4 and 8,
// or the forced one) and launch form (persistent and staged, or the
// requested one), keep the fastest.
int autotune(pppm_batch* P, const float* pos, const float* q, double* energies, float* forces, double* virials) {
    cudaStream_t s = nullptr;
    BK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = 1e30f;
    int best_T = P->forced_tile ? P->forced_tile : 8;
    bool best_staged = P->launch_mode == PPPM_BATCH_STAGED;
    for (int li = 0; li < 2; ++li) {
        if (P->lay[li].T == 0) continue;  // not available for these meshes
        if (P->forced_tile && P->lay[li].T != P->forced_tile) continue;
        for (int m = 0; m < 2; ++m) {
            const bool staged = m == 1;
            if (P->launch_mode != PPPM_BATCH_AUTO && staged != (P->launch_mode == PPPM_BATCH_STAGED)) continue;
            P->staged = staged;
            float ms_sum = 0.f;
            for (int rep = 0; rep < 3; ++rep) {
                if (enqueue(P, s, li, pos, q, energies, forces, virials) != PPPM_OK) { ms_sum = 1e30f; break; }
                cudaEventRecord(a, s);
                if (enqueue(P, s, li, pos, q, energies, forces, virials) != PPPM_OK) { ms_sum = 1e30f; break; }
                cudaEventRecord(b, s);
                cudaEventSynchronize(b);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, a, b);
                if (rep > 0) ms_sum += ms;
            }
            if (ms_sum < best) { best = ms_sum; best_T = P->lay[li].T; best_staged = staged; }
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaStreamDestroy(s);
    P->tile = best_T;
    P->staged = best_staged;
    P->mode_tuned = true;
    return PPPM_OK;
}

}  // namespace

extern "C" {

int pppm_batch_create(int nbox, const double* boxes, const int* meshes, int order, double beta,
                      pppm_batch** out) {
    if (!out) return PPPM_ERR_INVALID_ARG;
    *out = nullptr;
    if (nbox < 1 || nbox > 65535 || !boxes || !(beta > 0.0) || !std::isfinite(beta)) return PPPM_ERR_INVALID_ARG;
    if (order != 3 && order != 5 && order != 7) return PPPM_ERR_BAD_ORDER;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return PPPM_ERR_CUDA;
    pppm_batch* P = new (std::nothrow) pppm_batch();
    if (!P) return PPPM_ERR_CUDA;
    P->nbox = nbox;
    P->order = order;
    P->beta = beta;
    P->boxes.assign(boxes, boxes + 3 * nbox);
    P->meshes.resize(3 * nbox);
    auto fail = [&](int code) {
        pppm_batch_destroy(P);
        return code;
    };
    for (int b = 0; b < nbox; ++b)
        for (int d = 0; d < 3; ++d) {
            const double L = boxes[3 * b + d];
            if (!(L > 0.0) || !std::isfinite(L)) return fail(PPPM_ERR_BAD_BOX);
            int m = meshes ? meshes[3 * b + d] : smooth_at_least_b(L / 1.2);
            if (!smooth235_b(m) || m < 4 + order - 1 || m > 512) return fail(PPPM_ERR_BAD_MESH);
            P->meshes[3 * b + d] = m;
        }
    // influence functions (FP64 on the device, FP32 copies) and twiddles, per box
    long long G_total = 0;
    int tw_total = 0;
    P->G0.resize(nbox);
    P->tw0.resize(3 * nbox);
    for (int b = 0; b < nbox; ++b) {
        const int* N = &P->meshes[3 * b];
        P->G0[b] = G_total;
        G_total += (long long)N[0] * N[1] * (N[2] / 2 + 1);
        for (int d = 0; d < 3; ++d) {
            P->tw0[3 * b + d] = tw_total;
            tw_total += N[d];
        }
    }
    if (balloc(&P->G, sizeof(float) * G_total) != PPPM_OK) return fail(PPPM_ERR_CUDA);
    if (balloc(&P->tw, sizeof(float2) * tw_total) != PPPM_OK) return fail(PPPM_ERR_CUDA);
    double* G64 = nullptr;
    long long maxNH = 0;
    for (int b = 0; b < nbox; ++b) {
        const int* N = &P->meshes[3 * b];
        maxNH = std::max(maxNH, (long long)N[0] * N[1] * (N[2] / 2 + 1));
    }
    if (balloc(&G64, sizeof(double) * maxNH) != PPPM_OK) return fail(PPPM_ERR_CUDA);
    for (int b = 0; b < nbox; ++b) {
        const int* N = &P->meshes[3 * b];
        const Geo g = box_geo(&P->boxes[3 * b], N, order, 8);
        if (launch_influence(nullptr, g, beta, 2, G64) != cudaSuccess ||
            launch_convert<float>(nullptr, G64, P->G + P->G0[b], (long long)N[0] * N[1] * (N[2] / 2 + 1)) !=
                cudaSuccess) {
            bfree(G64);
            return fail(PPPM_ERR_CUDA);
        }
        for (int d = 0; d < 3; ++d)
            if (launch_twiddles<float>(nullptr, N[d], P->tw + P->tw0[3 * b + d]) != cudaSuccess) {
                bfree(G64);
                return fail(PPPM_ERR_CUDA);
            }
        if (cudaDeviceSynchronize() != cudaSuccess) {
            bfree(G64);
            return fail(PPPM_ERR_CUDA);
        }
    }
    bfree(G64);
    // mesh work buffers (sized by the meshes alone)
    long long c_total = 0, f_total = 0;
    for (int b = 0; b < nbox; ++b) {
        const int* N = &P->meshes[3 * b];
        c_total += (long long)N[0] * N[1] * (N[2] / 2 + 1);
        f_total += 3ll * (N[0] + order - 1) * (N[1] + order - 1) * ((N[2] + order - 1 + 3) & ~3);
    }
    for (int c = 0; c < 3; ++c)
        if (balloc(&P->cx[c], sizeof(float2) * c_total) != PPPM_OK) return fail(PPPM_ERR_CUDA);
    if (balloc(&P->fields, sizeof(float) * f_total) != PPPM_OK) return fail(PPPM_ERR_CUDA);
    if (balloc(&P->head, sizeof(unsigned int)) != PPPM_OK) return fail(PPPM_ERR_CUDA);
    if (balloc(&P->done, sizeof(int) * NSTAGE * nbox) != PPPM_OK) return fail(PPPM_ERR_CUDA);
    if (balloc(&P->box_counter, sizeof(unsigned int) * nbox) != PPPM_OK) return fail(PPPM_ERR_CUDA);
    if (balloc(&P->box_fail, sizeof(int) * nbox) != PPPM_OK) return fail(PPPM_ERR_CUDA);
    if (balloc(&P->status, sizeof(int)) != PPPM_OK) return fail(PPPM_ERR_CUDA);
    if (cudaMemset(P->status, 0, sizeof(int)) != cudaSuccess) return fail(PPPM_ERR_CUDA);
    const char* env = getenv("PPPM_BATCH_TILE");
    if (env && (atoi(env) == 4 || atoi(env) == 8)) P->forced_tile = atoi(env);
    *out = P;
    return PPPM_OK;
}

int pppm_batch_set(pppm_batch* P, double prefactor, int tile, long long spin_limit) {
    if (!P || !std::isfinite(prefactor) || (tile != 0 && tile != 4 && tile != 8) || spin_limit < 1)
        return PPPM_ERR_INVALID_ARG;
    P->prefactor = prefactor;
    P->forced_tile = tile;
    P->tile = tile;
    P->spin_limit = spin_limit;
    if (P->exec) cudaGraphExecDestroy(P->exec);
    P->exec = nullptr;
    return PPPM_OK;
}

int pppm_batch_set_launch(pppm_batch* P, int mode) {
    if (!P || (mode != PPPM_BATCH_PERSISTENT && mode != PPPM_BATCH_STAGED && mode != PPPM_BATCH_AUTO))
        return PPPM_ERR_INVALID_ARG;
    P->launch_mode = mode;
    P->mode_tuned = false;  // re-tune the launch form (and the tile edge unless forced)
    P->tile = P->forced_tile;
    if (P->exec) cudaGraphExecDestroy(P->exec);
    P->exec = nullptr;
    return PPPM_OK;
}

int pppm_batch_set_wait_probe(pppm_batch* P, int on) {
    if (!P) return PPPM_ERR_INVALID_ARG;
    P->wait_probe = on != 0;
    if (P->exec) cudaGraphExecDestroy(P->exec);
    P->exec = nullptr;
    return PPPM_OK;
}

int pppm_batch_set_dft(pppm_batch* P, int max_len) {
    if (!P || max_len < 0 || max_len > kDftTcMax) return PPPM_ERR_INVALID_ARG;
    P->dft_max = max_len;
    P->tile = P->forced_tile;  // re-tune the tile edge with the new transforms
    if (P->exec) cudaGraphExecDestroy(P->exec);
    P->exec = nullptr;
    return PPPM_OK;
}

int pppm_batch_set_quantized(pppm_batch* P, int group, double scale) {
    if (!P || group < 0 || group > kDftTcMax || (group > 0 && P->order != 5)) return PPPM_ERR_INVALID_ARG;
    if (!(scale >= 1.0 && scale <= 1e15)) return PPPM_ERR_INVALID_ARG;
    P->quant_group = group;
    P->quant_scale = scale;
    P->tile = P->forced_tile;
    if (P->exec) cudaGraphExecDestroy(P->exec);
    P->exec = nullptr;
    return PPPM_OK;
}

int pppm_batch_meshes(const pppm_batch* P, int* meshes) {
    if (!P || !meshes) return PPPM_ERR_INVALID_ARG;
    std::memcpy(meshes, P->meshes.data(), sizeof(int) * 3 * P->nbox);
    return PPPM_OK;
}

int pppm_batch_tile(const pppm_batch* P) { return P ? P->tile : PPPM_ERR_INVALID_ARG; }

int pppm_batch_launch(const pppm_batch* P) {
    if (!P) return PPPM_ERR_INVALID_ARG;
    if (!P->mode_tuned) return P->launch_mode;
    return P->staged ? PPPM_BATCH_STAGED : PPPM_BATCH_PERSISTENT;
}

int pppm_compute_batched(pppm_batch* P, void* stream, const float* pos, const float* q, const int64_t* offsets,
                         double* energies, float* forces, double* virials) {
    if (!P || !offsets || !energies || !virials) return PPPM_ERR_INVALID_ARG;
    int rc;
    if ((rc = prepare(P, offsets)) != PPPM_OK) return rc;
    const long long n = P->offsets[P->nbox];
    if (n > 0 && (!pos || !q || !forces)) return PPPM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    P->last = s;
    if (!P->tile || !P->mode_tuned) {
        if ((rc = autotune(P, pos, q, energies, forces, virials)) != PPPM_OK) return rc;
    }
    const int li = P->tile == 4 ? 0 : 1;
    if (P->lay[li].T == 0) return PPPM_ERR_BAD_MESH;  // tile edge 8 forced on a mesh too small for it
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    BK(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone || s == nullptr) return enqueue(P, s, li, pos, q, energies, forces, virials);
    // one graph (memsets + the persistent launch), re-captured when the pointers change
    const void* key[6] = {pos, q, energies, forces, virials, offsets};
    bool same = P->exec && P->key_tile == P->tile;
    for (int i = 0; i < 6 && same; ++i) same = key[i] == P->key[i];
    if (!same) {
        cudaGraph_t graph = nullptr;
        BK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        rc = enqueue(P, s, li, pos, q, energies, forces, virials);
        cudaError_t e = cudaStreamEndCapture(s, &graph);
        if (rc != PPPM_OK) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        BK(e);
        if (P->exec) cudaGraphExecDestroy(P->exec);
        P->exec = nullptr;
        e = cudaGraphInstantiate(&P->exec, graph, 0);
        cudaGraphDestroy(graph);
        BK(e);
        for (int i = 0; i < 6; ++i) P->key[i] = key[i];
        P->key_tile = P->tile;
    }
    BK(cudaGraphLaunch(P->exec, s));
    return PPPM_OK;
}

int pppm_batch_status(pppm_batch* P) {
    if (!P) return PPPM_ERR_INVALID_ARG;
    if (P->last) BK(cudaStreamSynchronize(P->last));
    else BK(cudaDeviceSynchronize());
    int st = 0;
    BK(cudaMemcpy(&st, P->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st) BK(cudaMemset(P->status, 0, sizeof(int)));
    if (st & 4) return PPPM_ERR_TIMEOUT;
    if (st & 1) return PPPM_ERR_NONFINITE;
    if (st & 8) return PPPM_ERR_TOO_LARGE;  // a quantised partial sum was clamped to int32
    return PPPM_OK;
}

void pppm_batch_destroy(pppm_batch* P) {
    if (!P) return;
    cudaDeviceSynchronize();
    if (P->exec) cudaGraphExecDestroy(P->exec);
    for (auto& Y : P->lay) {
        bfree(Y.d_desc);
        bfree(Y.d_items);
        bfree(Y.d_cov2);
    }
    bfree(P->G);
    bfree(P->tw);
    bfree(P->tile_count);
    bfree(P->tile_start);
    bfree(P->tile_of);
    bfree(P->slot_of);
    bfree(P->rec);
    bfree(P->cell);
    bfree(P->scell);
    bfree(P->sorig);
    bfree(P->srec);
    bfree(P->patch);
    for (int c = 0; c < 3; ++c) bfree(P->cx[c]);
    bfree(P->fields);
    bfree(P->partial);
    bfree(P->head);
    bfree(P->done);
    bfree(P->box_counter);
    bfree(P->box_fail);
    bfree(P->status);
    delete P;
}

}  // extern "C"
