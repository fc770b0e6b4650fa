// Learned correction of a coarse-mesh PPPM: a small per-site network maps
// local features of the coarse mesh potential to a correction of the field,
// trained on forces of a fine-mesh PPPM of the same positions.
//
//   features  x_i = [27 samples of the coarse mesh potential phi, interpolated
//             with the site's order-p B-spline weights at r_i + h (dx, dy, dz),
//             d in {-1, 0, 1}^3, times s_in; one-hot site type (3); then
//             either 2 zeros (the stated set, 32 per site) or sin, cos of
//             2 pi u_d per axis, u = position in mesh units (6), and 12 zeros
//             (the cell set, 48 per site)] (BF16)
//   network   h1 = tanh(W1 x + b1) (n_in -> 64), h2 = tanh(W2 h1 + b2) (64 -> 64),
//             y = W3 h2 + b3 (64 -> 3); BF16 weights, FP32 accumulation
//   forces    F_i = F_coarse,i + q_i s_out y_i
//   training  target t_i = (F_fine,i - F_coarse,i) / (q_i s_out); loss mean |y - t|^2;
//             Adam on FP32 master weights, BF16 copies for inference
//
// Inference runs on the tensor cores (mma.sync m16n8k16 BF16 -> FP32; the
// accumulator fragments of one layer are exactly the A fragments of the next,
// so a warp chains all three layers in registers).  Training is FP32 on the
// CUDA cores, one block of 128 threads per 128 sites, with the per-block weight
// gradients reduced in a fixed order before the Adam step.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "internal.cuh"
#include "plan.cuh"

namespace pppm {
namespace corr {

constexpr int NH = 64, NOUT = 3, NOUT_PAD = 8;
constexpr int K2P = NH + 8;
// Sizes and offsets of a network with NIN inputs (48: cell set, 32: stated set).
template <int NIN>
struct Net {
    static_assert(NIN == 32 || NIN == 48, "input widths of the two feature sets");
    static constexpr int KC1 = NIN / 16;  // k-chunks of the first layer
    static constexpr int O_W1 = 0, O_B1 = O_W1 + NH * NIN, O_W2 = O_B1 + NH, O_B2 = O_W2 + NH * NH,
                         O_W3 = O_B2 + NH, O_B3 = O_W3 + NOUT * NH, NPARAM = O_B3 + NOUT;
    // BF16 weight layout for the tensor-core forward: rows padded so that the
    // per-lane B-fragment loads hit distinct banks (row pitches of 28 and 20
    // words put the eight row groups of a fragment load on distinct banks)
    static constexpr int K1P = NIN + 8;
    static constexpr int BW1 = 0, BW2 = BW1 + NH * K1P, BW3 = BW2 + NH * K2P, NBF = BW3 + NOUT_PAD * K2P;
    static constexpr int XP = NIN + 1;  // training: padded row of the feature tile
};
constexpr int kNinCell = 48, kNinStated = 32;

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

// ------------------------------------------------------------------ features
__device__ __forceinline__ void locate_site(float x, float s_hi, float s_lo, int N, bool odd, int& g, float& x0) {
    float u = x * s_hi;
    const float e = fmaf(x, s_hi, -u);
    float ul = fmaf(x, s_lo, e);
    if (!(fabsf(u) < 4.0e6f)) { u = 0.f; ul = 0.f; }
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
}

// all p weights N_p(x0 + j) by the Cox-de Boor recursion
template <int P>
__device__ __forceinline__ void bspline_all(float x0, float w[P]) {
    w[0] = 1.f;
#pragma unroll
    for (int m = 2; m <= P; ++m) {
        const float inv = 1.f / (m - 1);
        w[m - 1] = (1.f - x0) * w[m - 2] * inv;
#pragma unroll
        for (int j = m - 2; j >= 1; --j) w[j] = ((x0 + j) * w[j] + (m - x0 - j) * w[j - 1]) * inv;
        w[0] = x0 * w[0] * inv;
    }
}

// One thread per site.  The 27 samples share the site's weights; with the
// (p+2)^3 mesh values around the site they are three separable contractions.
// With the solve's tile order given (tiles, sorig), block b takes the sites of
// tile b, so the sites of a warp lie in one tile and their mesh rows overlap
// (a warp's loads touch a few rows instead of 32 scattered ones); without it
// thread t takes site t.
template <int P, int NIN>
__device__ __forceinline__ void site_features(const Geo& g, const FieldLayout& fl, const float* __restrict__ phi,
                                              const float* __restrict__ pos, const signed char* __restrict__ types,
                                              int i, float s_in, __nv_bfloat16* __restrict__ feat) {
    constexpr int W = P + 2;
    const bool odd = (g.order & 1) != 0;
    int gc[3];
    float w[3][P];
    float dfrac[3];  // u - g, the offset of the site from its base mesh point
    int idx[3][W];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float x0;
        locate_site(pos[3 * i + d], g.s_hi[d], g.s_lo[d], g.N[d], odd, gc[d], x0);
        dfrac[d] = odd ? 0.5f - x0 : 1.f - x0;
        bspline_all<P>(x0, w[d]);
#pragma unroll
        for (int a = 0; a < W; ++a) {
            int m = (gc[d] + g.kmin - 1 + a) % g.N[d];
            m += m < 0 ? g.N[d] : 0;
            idx[d][a] = m - g.kmin;  // padded coordinate
        }
    }
    float F[27];
#pragma unroll
    for (int k = 0; k < 27; ++k) F[k] = 0.f;
#pragma unroll
    for (int a = 0; a < W; ++a) {  // x offset of the mesh row
        float Sy[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) Sy[k] = 0.f;
#pragma unroll
        for (int b = 0; b < W; ++b) {  // y offset
            const float* row = phi + ((int64_t)idx[0][a] * fl.Yp + idx[1][b]) * fl.Zp * fl.pstride;
            float v[W];
#pragma unroll
            for (int c = 0; c < W; ++c) v[c] = __ldg(&row[idx[2][c] * fl.pstride]);
            float Sz[3];
#pragma unroll
            for (int dz = 0; dz < 3; ++dz) {
                float s = 0.f;
#pragma unroll
                for (int kz = 0; kz < P; ++kz) s += w[2][kz] * v[dz + kz];
                Sz[dz] = s;
            }
#pragma unroll
            for (int dy = 0; dy < 3; ++dy) {
                const int ky = b - dy;
                if (ky >= 0 && ky < P) {
#pragma unroll
                    for (int dz = 0; dz < 3; ++dz) Sy[dy * 3 + dz] += w[1][ky] * Sz[dz];
                }
            }
        }
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
            const int kx = a - dx;
            if (kx >= 0 && kx < P) {
#pragma unroll
                for (int k = 0; k < 9; ++k) F[dx * 9 + k] += w[0][kx] * Sy[k];
            }
        }
    }
    // the row as NIN / 2 packed pairs, written with 16-byte stores
    float v[NIN];
#pragma unroll
    for (int k = 0; k < 27; ++k) v[k] = F[k] * s_in;
    const int ty = types[i];
#pragma unroll
    for (int k = 0; k < 3; ++k) v[27 + k] = ty == k ? 1.f : 0.f;
    if constexpr (NIN == kNinCell) {
#pragma unroll
        for (int d = 0; d < 3; ++d) sincospif(2.f * dfrac[d], &v[30 + 2 * d], &v[31 + 2 * d]);
#pragma unroll
        for (int k = 36; k < NIN; ++k) v[k] = 0.f;
    } else {
        (void)dfrac;
#pragma unroll
        for (int k = 30; k < NIN; ++k) v[k] = 0.f;
    }
    uint4* o = reinterpret_cast<uint4*>(feat + (int64_t)i * NIN);
#pragma unroll
    for (int k = 0; k < NIN / 8; ++k) {
        uint4 w;
        w.x = pack_bf16(v[8 * k + 0], v[8 * k + 1]);
        w.y = pack_bf16(v[8 * k + 2], v[8 * k + 3]);
        w.z = pack_bf16(v[8 * k + 4], v[8 * k + 5]);
        w.w = pack_bf16(v[8 * k + 6], v[8 * k + 7]);
        o[k] = w;
    }
}

template <int P, int NIN>
__global__ void k_features(Geo g, FieldLayout fl, const float* __restrict__ phi, const float* __restrict__ pos,
                           const signed char* __restrict__ types, const int2* __restrict__ tiles,
                           const int* __restrict__ sorig, int n, float s_in, __nv_bfloat16* __restrict__ feat) {
    if (tiles) {
        const int2 tr = tiles[blockIdx.x];
        for (int s = tr.x + threadIdx.x; s < tr.y; s += blockDim.x)
            site_features<P, NIN>(g, fl, phi, pos, types, __ldg(&sorig[s]), s_in, feat);
    } else {
        const int t = blockIdx.x * blockDim.x + threadIdx.x;
        if (t < n) site_features<P, NIN>(g, fl, phi, pos, types, t, s_in, feat);
    }
}

// ------------------------------------------------------------------ tensor-core forward
__device__ __forceinline__ void mma_bf16(float d[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}


// accumulators of eight n-tiles (64 columns) -> tanh -> A fragments of four k-chunks
__device__ __forceinline__ void act_to_a(const float acc[8][4], const float* __restrict__ bias, int tig,
                                         uint32_t a[4][4]) {
#pragma unroll
    for (int kc = 0; kc < 4; ++kc)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int nt = 2 * kc + h;
            const int col = nt * 8 + 2 * tig;
            const float b0 = bias[col], b1 = bias[col + 1];
            a[kc][2 * h] = pack_bf16(tanhf(acc[nt][0] + b0), tanhf(acc[nt][1] + b1));
            a[kc][2 * h + 1] = pack_bf16(tanhf(acc[nt][2] + b0), tanhf(acc[nt][3] + b1));
        }
}

// One warp per 16 sites (grid-stride).  With forces/q given, adds
// q_i s_out y_i to forces (the corrected PPPM); else writes y to out.
template <int NIN>
__global__ void __launch_bounds__(128)
k_mlp_forward(const __nv_bfloat16* __restrict__ feat, int n, const __nv_bfloat16* __restrict__ wbf,
              const float* __restrict__ master, float s_out, const float* __restrict__ q, float* __restrict__ forces,
              float* __restrict__ out) {
    typedef Net<NIN> L;
    constexpr int NBF = L::NBF, KC1 = L::KC1, K1P = L::K1P, BW1 = L::BW1, BW2 = L::BW2, BW3 = L::BW3;
    constexpr int O_B1 = L::O_B1, O_B2 = L::O_B2, O_B3 = L::O_B3;
    __shared__ __align__(16) __nv_bfloat16 sw[NBF];
    __shared__ float sb[NH + NH + NOUT_PAD];
    for (int k = threadIdx.x; k < NBF; k += blockDim.x) sw[k] = wbf[k];
    for (int k = threadIdx.x; k < NH; k += blockDim.x) {  // biases are BF16 parameters too
        sb[k] = __bfloat162float(__float2bfloat16_rn(master[O_B1 + k]));
        sb[NH + k] = __bfloat162float(__float2bfloat16_rn(master[O_B2 + k]));
    }
    if (threadIdx.x < NOUT_PAD)
        sb[2 * NH + threadIdx.x] =
            threadIdx.x < NOUT ? __bfloat162float(__float2bfloat16_rn(master[O_B3 + threadIdx.x])) : 0.f;
    __syncthreads();
    const int lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
    const int warps = gridDim.x * (blockDim.x >> 5);
    const uint32_t* w32 = reinterpret_cast<const uint32_t*>(sw);
    for (int tile = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); tile * 16 < n; tile += warps) {
        const int r0 = tile * 16 + gid, r1 = r0 + 8;
        // layer 1: A from the features (16 x NIN), NIN / 16 k-chunks
        uint32_t a1[KC1][4];
        const uint32_t* f0 = reinterpret_cast<const uint32_t*>(feat + (int64_t)min(r0, n - 1) * NIN);
        const uint32_t* f1 = reinterpret_cast<const uint32_t*>(feat + (int64_t)min(r1, n - 1) * NIN);
#pragma unroll
        for (int kc = 0; kc < KC1; ++kc) {
            a1[kc][0] = f0[kc * 8 + tig];
            a1[kc][1] = f1[kc * 8 + tig];
            a1[kc][2] = f0[kc * 8 + 4 + tig];
            a1[kc][3] = f1[kc * 8 + 4 + tig];
        }
        float acc[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
            const int nrow = nt * 8 + gid;  // output unit handled by this lane's B fragment
#pragma unroll
            for (int kc = 0; kc < KC1; ++kc) {
                const uint32_t b0 = w32[(BW1 + nrow * K1P + kc * 16) / 2 + tig];
                const uint32_t b1 = w32[(BW1 + nrow * K1P + kc * 16 + 8) / 2 + tig];
                mma_bf16(acc[nt], a1[kc], b0, b1);
            }
        }
        uint32_t a2[4][4];
        act_to_a(acc, sb, tig, a2);
        // layer 2
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
            const int nrow = nt * 8 + gid;
#pragma unroll
            for (int kc = 0; kc < 4; ++kc) {
                const uint32_t b0 = w32[(BW2 + nrow * K2P + kc * 16) / 2 + tig];
                const uint32_t b1 = w32[(BW2 + nrow * K2P + kc * 16 + 8) / 2 + tig];
                mma_bf16(acc[nt], a2[kc], b0, b1);
            }
        }
        uint32_t a3[4][4];
        act_to_a(acc, sb + NH, tig, a3);
        // layer 3 (three outputs padded to an n-tile of 8)
        float y[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kc = 0; kc < 4; ++kc) {
            const uint32_t b0 = w32[(BW3 + gid * K2P + kc * 16) / 2 + tig];
            const uint32_t b1 = w32[(BW3 + gid * K2P + kc * 16 + 8) / 2 + tig];
            mma_bf16(y, a3[kc], b0, b1);
        }
        // lane holds rows r0 (y[0], y[1]) and r1 (y[2], y[3]) at columns 2 tig, 2 tig + 1
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int r = h ? r1 : r0;
            if (r >= n) continue;
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int c = 2 * tig + e;
                if (c >= NOUT) continue;
                const float v = y[2 * h + e] + sb[2 * NH + c];
                if (forces) forces[3 * (int64_t)r + c] += q[r] * s_out * v;
                else out[3 * (int64_t)r + c] = v;
            }
        }
    }
}

// ------------------------------------------------------------------ tcgen05 forward
// The same network on the fifth-generation tensor cores: one CTA takes 128
// sites at a time (M = 128), each layer one chain of tcgen05.mma kind::f16
// instructions (BF16 operands from shared memory, FP32 accumulators in
// tensor memory) issued by one thread, N = 64 for the hidden layers and 16
// (three outputs, zero rows above) for the last, K = 16 per instruction.
// The accumulators are read back with tcgen05.ld (eight warps: lane t of
// warp w holds row 32 (w mod 4) + t, warps 0-3 its columns 0-31 and warps 4-7
// its columns 32-63), biased, passed through tanh, rounded to BF16 and stored
// as the next layer's A operand; the MMA's completion is signalled through an
// mbarrier (tcgen05.commit) and waited on with a bounded spin.  Each thread
// fetches its half of the next tile's feature row while the current tile's
// layers run.
//
// Operands use the no-swizzle K-major canonical layout: 8-row x 16-byte core
// matrices (8 rows of 8 BF16 values, 128 contiguous bytes), the K-chunks of
// an 8-row group 128 bytes apart (leading byte offset) and the 8-row groups
// K/8 * 128 bytes apart (stride byte offset).  One MMA with K = 16 reads two
// K-chunks, so the k-th MMA of a layer starts 256 k bytes in.
namespace tc {

constexpr int kRows = 128;             // sites per tile (MMA M)
constexpr int kThreads = 256;          // warps w and w + 4 share TMEM lanes 32 (w mod 4) + 0..31
constexpr uint32_t kTmemCols = 64;     // each layer's accumulators in columns 0..63 (outputs: 0..15)
constexpr int kOutCol = 0, kOutN = 16;
constexpr long long kSpin = 1ll << 26; // polls of the second wait, after a first one ran out

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (r, k) of a K-major operand with K columns
__host__ __device__ constexpr uint32_t canon(int r, int k, int K) {
    return (uint32_t)((r >> 3) * (K / 8) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor: start, leading and stride byte offsets
// (16-byte units), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major
__host__ __device__ constexpr uint32_t idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t id, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(id), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ bool wait_bounded(uint32_t mbar, uint32_t parity, long long limit) {
    for (long long it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive FP32 columns of this warp's 32 rows: thread t gets row t.
// The registers are valid only after wait_ld, which takes them as operands so
// that no use of them can be scheduled ahead of the wait.
__device__ __forceinline__ void ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void wait_ld(uint32_t (&r)[16]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
}

template <int NIN>
struct Smem {
    // the second hidden layer's activations replace the first's (A3 = A2):
    // the layer-2 MMA has completed before they are written
    static constexpr uint32_t W1 = 0, W2 = W1 + 64 * NIN * 2, W3 = W2 + 64 * 64 * 2, A1 = W3 + kOutN * 64 * 2,
                              A2 = A1 + kRows * NIN * 2, A3 = A2, BIAS = A2 + kRows * 64 * 2,
                              MBAR = BIAS + (64 + 64 + kOutN) * 4, TSLOT = MBAR + 8, BYTES = TSLOT + 8;
};

// hidden activations of this thread's row, columns 32 hf .. 32 hf + 31:
// tanh(acc + b) -> BF16 -> the next layer's A operand
__device__ __forceinline__ void hidden_out(uint32_t tmem_row, const float* __restrict__ b, unsigned char* a_op,
                                           int row, int hf) {
    uint32_t v[2][16];
    ld16(tmem_row + 32 * hf, v[0]);  // both loads in flight before the waits
    ld16(tmem_row + 32 * hf + 16, v[1]);
    wait_ld(v[0]);
    wait_ld(v[1]);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int c0 = 32 * hf + 16 * q;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint4 pk;
            uint32_t* w = reinterpret_cast<uint32_t*>(&pk);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int c = c0 + 8 * h + 2 * e;
                w[e] = pack_bf16(tanhf(__uint_as_float(v[q][8 * h + 2 * e]) + b[c]),
                                 tanhf(__uint_as_float(v[q][8 * h + 2 * e + 1]) + b[c + 1]));
            }
            *reinterpret_cast<uint4*>(a_op + canon(row, c0 + 8 * h, 64)) = pk;
        }
    }
}

template <int NIN>
__global__ void __launch_bounds__(kThreads)
k_mlp_forward_tc(const __nv_bfloat16* __restrict__ feat, int n, const __nv_bfloat16* __restrict__ wbf,
                 const float* __restrict__ master, float s_out, const float* __restrict__ q,
                 float* __restrict__ forces, float* __restrict__ out, int* __restrict__ status,
                 long long wait_limit) {
    typedef Net<NIN> L;
    typedef Smem<NIN> S;
    constexpr int K1P = L::K1P, BW1 = L::BW1, BW2 = L::BW2, BW3 = L::BW3;
    extern __shared__ __align__(1024) unsigned char sm[];
    const int t = threadIdx.x, warp = t >> 5;
    const int row = 32 * (warp & 3) + (t & 31), hf = warp >> 2;  // tile row and column half of this thread
    const uint32_t base = smem_u32(sm);
    const uint32_t mbar = base + S::MBAR;
    float* bias = reinterpret_cast<float*>(sm + S::BIAS);
    // weights into the canonical K-major layout (rows are output units)
    for (int i = t; i < 64 * NIN; i += kThreads) {
        const int r = i / NIN, k = i - r * NIN;
        *reinterpret_cast<__nv_bfloat16*>(sm + S::W1 + canon(r, k, NIN)) = wbf[BW1 + r * K1P + k];
    }
    for (int i = t; i < 64 * 64; i += kThreads) {
        const int r = i >> 6, k = i & 63;
        *reinterpret_cast<__nv_bfloat16*>(sm + S::W2 + canon(r, k, 64)) = wbf[BW2 + r * K2P + k];
    }
    for (int i = t; i < kOutN * 64; i += kThreads) {
        const int r = i >> 6, k = i & 63;
        *reinterpret_cast<__nv_bfloat16*>(sm + S::W3 + canon(r, k, 64)) =
            r < NOUT ? wbf[BW3 + r * K2P + k] : __float2bfloat16_rn(0.f);
    }
    for (int k = t; k < 64; k += kThreads) {  // biases are BF16 parameters too
        bias[k] = __bfloat162float(__float2bfloat16_rn(master[L::O_B1 + k]));
        bias[64 + k] = __bfloat162float(__float2bfloat16_rn(master[L::O_B2 + k]));
    }
    if (t < kOutN) bias[128 + t] = t < NOUT ? __bfloat162float(__float2bfloat16_rn(master[L::O_B3 + t])) : 0.f;
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(base + S::TSLOT),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(sm + S::TSLOT);
    const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16);  // this warp's 32 lanes
    uint32_t phase = 0;
    bool failed = false;  // the same in every thread (decided at a barrier)
    // one layer: D[col ..] = A (128 x K) W^T (K x N); false if its completion
    // was not seen within the spin limit
    auto layer = [&](uint32_t a_off, uint32_t b_off, int K, int N, uint32_t col) {
        // every thread's operand stores are done: hand the tile to the tensor cores
        fence_async_smem();
        fence_before();
        __syncthreads();
        if (t == 0) {
            fence_after();
            const uint32_t id = idesc(kRows, N);
            for (int k = 0; k < K / 16; ++k)
                mma(tmem + col, desc(base + a_off + 256 * k, 128, K / 8 * 128),
                    desc(base + b_off + 256 * k, 128, K / 8 * 128), id, k > 0);
            commit(mbar);
        }
        const bool ok = wait_bounded(mbar, phase, wait_limit);
        failed = __syncthreads_or(!ok) != 0;
        if (!failed) phase ^= 1;
        fence_after();
        return !failed;
    };
    const int ntile = (n + kRows - 1) / kRows;
    // this thread's half of a feature row (zeros past the end), fetched one
    // tile ahead so that the loads overlap the current tile's layers
    constexpr int NCH = NIN / 16;  // 16-byte chunks a thread
    uint4 nf[NCH];
    auto fetch = [&](int tile) {
        const int r = tile * kRows + row;
        const uint4* src = reinterpret_cast<const uint4*>(feat + (int64_t)min(r, n - 1) * NIN) + hf * NCH;
#pragma unroll
        for (int c = 0; c < NCH; ++c) nf[c] = r < n ? __ldg(&src[c]) : make_uint4(0, 0, 0, 0);
    };
    if (blockIdx.x < ntile) fetch(blockIdx.x);
    for (int tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        const int r = tile * kRows + row;
#pragma unroll
        for (int c = 0; c < NCH; ++c)
            *reinterpret_cast<uint4*>(sm + S::A1 + canon(row, 8 * (hf * NCH + c), NIN)) = nf[c];
        if (tile + (int)gridDim.x < ntile) fetch(tile + gridDim.x);
        if (!layer(S::A1, S::W1, NIN, 64, 0)) break;
        hidden_out(trow, bias, sm + S::A2, row, hf);
        if (!layer(S::A2, S::W2, 64, 64, 0)) break;
        hidden_out(trow, bias + 64, sm + S::A3, row, hf);
        if (!layer(S::A3, S::W3, 64, kOutN, kOutCol)) break;
        uint32_t y[16];
        ld16(trow + kOutCol, y);  // warp-wide; the second half of the warps drops it
        wait_ld(y);
        if (hf == 0 && r < n) {
#pragma unroll
            for (int c = 0; c < NOUT; ++c) {
                const float v = __uint_as_float(y[c]) + bias[128 + c];
                if (forces) forces[3 * (int64_t)r + c] += q[r] * s_out * v;
                else out[3 * (int64_t)r + c] = v;
            }
        }
    }
    fence_before();
    __syncthreads();
    if (failed) {
        if (t == 0) atomicOr(status, 2);
        wait_bounded(mbar, phase, kSpin);  // an MMA still in flight lands before the memory is released
    }
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

}  // namespace tc

// FP32 master -> padded BF16 copy for the forward
template <int NIN>
__global__ void k_to_bf16(const float* __restrict__ master, __nv_bfloat16* __restrict__ wbf) {
    typedef Net<NIN> L;
    constexpr int NBF = L::NBF, K1P = L::K1P, BW2 = L::BW2, BW3 = L::BW3, O_W1 = L::O_W1, O_W2 = L::O_W2,
                  O_W3 = L::O_W3;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < NBF; k += gridDim.x * blockDim.x) {
        float v = 0.f;
        if (k < BW2) {
            const int r = k / K1P, c = k - r * K1P;
            if (c < NIN) v = master[O_W1 + r * NIN + c];
        } else if (k < BW3) {
            const int r = (k - BW2) / K2P, c = (k - BW2) - r * K2P;
            if (c < NH) v = master[O_W2 + r * NH + c];
        } else {
            const int r = (k - BW3) / K2P, c = (k - BW3) - r * K2P;
            if (r < NOUT && c < NH) v = master[O_W3 + r * NH + c];
        }
        wbf[k] = __float2bfloat16_rn(v);
    }
}

// ------------------------------------------------------------------ training
constexpr int TB = 128;  // sites per training block
constexpr int HP = NH + 1;

__device__ __forceinline__ float bfr(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// Per block: forward and backward of 128 sites (FP32, weights rounded to BF16
// as used by inference), per-block gradient sums to partial[block][NPARAM],
// and the block's share of the loss to lossp[block].
template <int NIN>
__global__ void __launch_bounds__(TB)
k_mlp_grad(const __nv_bfloat16* __restrict__ feat, const float* __restrict__ target, int64_t nrows,
           const int* __restrict__ idx, int nb, float inv_total, const float* __restrict__ master, float* __restrict__ partial,
           float* __restrict__ lossp) {
    typedef Net<NIN> L;
    constexpr int XP = L::XP, NPARAM = L::NPARAM, O_W1 = L::O_W1, O_B1 = L::O_B1, O_W2 = L::O_W2, O_B2 = L::O_B2,
                  O_W3 = L::O_W3, O_B3 = L::O_B3;
    extern __shared__ __align__(16) float sm[];
    float* W1 = sm;                  // 64 x NIN
    float* W2 = W1 + NH * NIN;       // 64 x 64
    float* W3 = W2 + NH * NH;        // 3 x 64
    float* bb = W3 + NOUT * NH;      // b1 64, b2 64, b3 3 (+1)
    float* X = bb + 2 * NH + 4;      // TB x XP
    float* H1 = X + TB * XP;         // TB x HP
    float* H2 = H1 + TB * HP;        // TB x HP
    float* DY = H2 + TB * HP;        // TB x 4
    float* red = DY + TB * 4;        // 32
    const int t = threadIdx.x;
    for (int k = t; k < NH * NIN; k += TB) W1[k] = bfr(master[O_W1 + k]);
    for (int k = t; k < NH * NH; k += TB) W2[k] = bfr(master[O_W2 + k]);
    for (int k = t; k < NOUT * NH; k += TB) W3[k] = bfr(master[O_W3 + k]);
    for (int k = t; k < NH; k += TB) {
        bb[k] = bfr(master[O_B1 + k]);
        bb[NH + k] = bfr(master[O_B2 + k]);
    }
    if (t < NOUT) bb[2 * NH + t] = bfr(master[O_B3 + t]);
    const int s = blockIdx.x * TB + t;
    int site = s < nb ? (idx ? idx[s] : s) : -1;
    const bool valid = site >= 0 && site < nrows;  // rows outside the table contribute nothing
    if (!valid) site = 0;
    for (int k = 0; k < NIN; ++k) X[t * XP + k] = valid ? __bfloat162float(feat[(int64_t)site * NIN + k]) : 0.f;
    __syncthreads();
    // forward of this thread's site
    for (int j = 0; j < NH; ++j) {
        float z = bb[j];
        for (int k = 0; k < NIN; ++k) z += W1[j * NIN + k] * X[t * XP + k];
        H1[t * HP + j] = tanhf(z);
    }
    for (int j = 0; j < NH; ++j) {
        float z = bb[NH + j];
        for (int k = 0; k < NH; ++k) z += W2[j * NH + k] * H1[t * HP + k];
        H2[t * HP + j] = tanhf(z);
    }
    float l = 0.f;
    for (int c = 0; c < NOUT; ++c) {
        float y = bb[2 * NH + c];
        for (int k = 0; k < NH; ++k) y += W3[c * NH + k] * H2[t * HP + k];
        const float r = valid ? y - target[3 * (int64_t)site + c] : 0.f;
        l += r * r;
        DY[t * 4 + c] = 2.f * r * inv_total;
    }
    // block loss (fixed-order tree)
    for (int off = 16; off > 0; off >>= 1) l += __shfl_down_sync(0xffffffffu, l, off);
    if ((t & 31) == 0) red[t >> 5] = l;
    __syncthreads();
    float* g = partial + (size_t)blockIdx.x * NPARAM;
    if (t == 0) lossp[blockIdx.x] = (red[0] + red[1] + red[2] + red[3]) * inv_total;
    // dW3, db3
    for (int o = t; o < NOUT * NH + NOUT; o += TB) {
        float acc = 0.f;
        if (o < NOUT * NH) {
            const int c = o / NH, j = o - c * NH;
            for (int r = 0; r < TB; ++r) acc += DY[r * 4 + c] * H2[r * HP + j];
            g[O_W3 + o] = acc;
        } else {
            const int c = o - NOUT * NH;
            for (int r = 0; r < TB; ++r) acc += DY[r * 4 + c];
            g[O_B3 + c] = acc;
        }
    }
    __syncthreads();
    // dZ2 over H2 (own row)
    for (int j = 0; j < NH; ++j) {
        float dh = 0.f;
        for (int c = 0; c < NOUT; ++c) dh += DY[t * 4 + c] * W3[c * NH + j];
        const float h = H2[t * HP + j];
        H2[t * HP + j] = dh * (1.f - h * h);
    }
    __syncthreads();
    // dW2 (thread: column k, rows j = t/64 + 2m), db2
    {
        const int k = t & (NH - 1), j0 = t >> 6;
        float acc[NH / 2];
        for (int m = 0; m < NH / 2; ++m) acc[m] = 0.f;
        for (int r = 0; r < TB; ++r) {
            const float hk = H1[r * HP + k];
#pragma unroll
            for (int m = 0; m < NH / 2; ++m) acc[m] += H2[r * HP + j0 + 2 * m] * hk;
        }
        for (int m = 0; m < NH / 2; ++m) g[O_W2 + (j0 + 2 * m) * NH + k] = acc[m];
    }
    if (t < NH) {
        float acc = 0.f;
        for (int r = 0; r < TB; ++r) acc += H2[r * HP + t];
        g[O_B2 + t] = acc;
    }
    __syncthreads();
    // dZ1 over H1 (own row)
    for (int k = 0; k < NH; ++k) {
        float dh = 0.f;
        for (int j = 0; j < NH; ++j) dh += H2[t * HP + j] * W2[j * NH + k];
        const float h = H1[t * HP + k];
        H1[t * HP + k] = dh * (1.f - h * h);
    }
    __syncthreads();
    // dW1 (thread: columns k0 + 16 c, c < NIN / 16, k0 = t % 16; rows j0 + 8 m,
    // m < 8, j0 = t / 16), db1
    {
        static_assert(NIN % 16 == 0 && NH == 64 && TB == 128, "dW1 thread map");
        constexpr int KC = NIN / 16;
        const int k0 = t & 15, j0 = t >> 4;
        float acc[KC][8];
#pragma unroll
        for (int c = 0; c < KC; ++c)
#pragma unroll
            for (int m = 0; m < 8; ++m) acc[c][m] = 0.f;
        for (int r = 0; r < TB; ++r) {
            float xk[KC], hj[8];
#pragma unroll
            for (int c = 0; c < KC; ++c) xk[c] = X[r * XP + k0 + 16 * c];
#pragma unroll
            for (int m = 0; m < 8; ++m) hj[m] = H1[r * HP + j0 + 8 * m];
#pragma unroll
            for (int c = 0; c < KC; ++c)
#pragma unroll
                for (int m = 0; m < 8; ++m) acc[c][m] += hj[m] * xk[c];
        }
#pragma unroll
        for (int c = 0; c < KC; ++c)
#pragma unroll
            for (int m = 0; m < 8; ++m) g[O_W1 + (j0 + 8 * m) * NIN + k0 + 16 * c] = acc[c][m];
    }
    if (t < NH) {
        float acc = 0.f;
        for (int r = 0; r < TB; ++r) acc += H1[r * HP + t];
        g[O_B1 + t] = acc;
    }
}

// Sum the per-block gradients in block order; then either return them or take
// one Adam step (FP32 master, moments m, v) and refresh nothing else (the BF16
// copy is rebuilt by k_to_bf16).
template <int NIN>
__global__ void k_reduce_adam(const float* __restrict__ partial, const float* __restrict__ lossp, int nblk,
                              float* __restrict__ grad_out, float* __restrict__ loss_out, float* __restrict__ master,
                              float* __restrict__ m1, float* __restrict__ m2, float lr, float b1, float b2, float eps,
                              float bc1, float bc2) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0 && loss_out) {
        float l = 0.f;
        for (int b = 0; b < nblk; ++b) l += lossp[b];
        *loss_out = l;
    }
    constexpr int NPARAM = Net<NIN>::NPARAM;
    if (p >= NPARAM) return;
    float gsum = 0.f;
    for (int b = 0; b < nblk; ++b) gsum += partial[(size_t)b * NPARAM + p];
    if (grad_out) grad_out[p] = gsum;
    if (master) {
        const float mm = b1 * m1[p] + (1.f - b1) * gsum;
        const float vv = b2 * m2[p] + (1.f - b2) * gsum * gsum;
        m1[p] = mm;
        m2[p] = vv;
        master[p] -= lr * (mm / bc1) / (sqrtf(vv / bc2) + eps);
    }
}

// training targets t_i = (F_fine,i - F_coarse,i) / (q_i s_out); 0 where q_i = 0
__global__ void k_targets(const float* __restrict__ ff, const float* __restrict__ fc, const float* __restrict__ q,
                          int64_t n, float s_out, float* __restrict__ t) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= 3 * n) return;
    const float qi = q[k / 3];
    t[k] = qi != 0.f ? (ff[k] - fc[k]) / (qi * s_out) : 0.f;
}

// Calibration sums, one partial per block (summed on the host in block order):
// [0] sum of squares of the 27 potential samples, [1] sum over sites with
// q != 0 of |F_fine - F_coarse|^2 / q^2, [2] number of such sites.
constexpr int kCalBlocks = 256;
template <int NIN>
__global__ void __launch_bounds__(256)
k_calibrate(const __nv_bfloat16* __restrict__ feat, const float* __restrict__ ff, const float* __restrict__ fc,
            const float* __restrict__ q, int n, double* __restrict__ part) {
    __shared__ double red[3][8];
    double a = 0.0, b = 0.0, c = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        for (int k = 0; k < 27; ++k) {
            const double v = __bfloat162float(feat[(int64_t)i * NIN + k]);
            a += v * v;
        }
        const float qi = q[i];
        if (qi != 0.f) {
            for (int d = 0; d < 3; ++d) {
                const double e = ((double)ff[3 * (int64_t)i + d] - (double)fc[3 * (int64_t)i + d]) / qi;
                b += e * e;
            }
            c += 1.0;
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, off);
        b += __shfl_down_sync(0xffffffffu, b, off);
        c += __shfl_down_sync(0xffffffffu, c, off);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { red[0][w] = a; red[1][w] = b; red[2][w] = c; }
    __syncthreads();
    if (threadIdx.x < 3) {
        double s = 0.0;
        for (int k = 0; k < 8; ++k) s += red[threadIdx.x][k];
        part[3 * blockIdx.x + threadIdx.x] = s;
    }
}

}  // namespace corr
}  // namespace pppm

// ====================================================================== host side
using namespace pppm;
using namespace pppm::corr;

struct pppm_corr {
    pppm_plan* plan = nullptr;  // coarse plan (borrowed)
    int nin = kNinCell;         // input width: 48 (cell set) or 32 (stated set)
    float* master = nullptr;
    float* m1 = nullptr;
    float* m2 = nullptr;
    __nv_bfloat16* wbf = nullptr;
    float* partial = nullptr;
    float* lossp = nullptr;
    int partial_blocks = 0;
    __nv_bfloat16* feat = nullptr;
    int64_t feat_cap = 0;
    float s_in = 1.f, s_out = 1.f;
    long long step = 0;
    double* ev = nullptr;  // scratch energy/virial of internal coarse evaluations
    int forward = PPPM_FORWARD_MMA_SYNC;  // network forward: mma.sync (faster at these widths) or tcgen05
    long long wait_limit = 1ll << 26;     // polls of a tcgen05 MMA completion before giving up
};

namespace {

#define CC(x)                                          \
    do {                                               \
        if ((x) != cudaSuccess) return PPPM_ERR_CUDA;  \
    } while (0)

// Runs f(std::integral_constant<int, NIN>) for the corrector's input width.
template <typename F>
auto with_nin(int nin, F&& f) {
    if (nin == kNinStated) return f(std::integral_constant<int, kNinStated>{});
    return f(std::integral_constant<int, kNinCell>{});
}

int nparam_of(int nin) { return nin == kNinStated ? Net<kNinStated>::NPARAM : Net<kNinCell>::NPARAM; }
int nbf_of(int nin) { return nin == kNinStated ? Net<kNinStated>::NBF : Net<kNinCell>::NBF; }

int ensure_feat(pppm_corr* C, int64_t n) {
    if (n <= C->feat_cap) return PPPM_OK;
    if (C->feat) cudaFree(C->feat);
    C->feat = nullptr;
    C->feat_cap = 0;
    CC(cudaMalloc((void**)&C->feat, sizeof(__nv_bfloat16) * C->nin * (n > 0 ? n : 1)));
    C->feat_cap = n;
    return PPPM_OK;
}

int ensure_partial(pppm_corr* C, int nblk) {
    if (nblk <= C->partial_blocks) return PPPM_OK;
    if (C->partial) cudaFree(C->partial);
    if (C->lossp) cudaFree(C->lossp);
    C->partial = nullptr;
    C->lossp = nullptr;
    C->partial_blocks = 0;
    CC(cudaMalloc((void**)&C->partial, sizeof(float) * nparam_of(C->nin) * (size_t)nblk));
    CC(cudaMalloc((void**)&C->lossp, sizeof(float) * nblk));
    C->partial_blocks = nblk;
    return PPPM_OK;
}

int refresh_bf16(pppm_corr* C, cudaStream_t s) {
    const int nbf = nbf_of(C->nin);
    with_nin(C->nin, [&](auto N) {
        k_to_bf16<decltype(N)::value><<<(nbf + 255) / 256, 256, 0, s>>>(C->master, C->wbf);
        return 0;
    });
    CC(cudaGetLastError());
    return PPPM_OK;
}

cudaError_t launch_features(pppm_corr* C, cudaStream_t s, const float* pos, const signed char* types, int64_t n,
                            __nv_bfloat16* feat) {
    pppm_plan* P = C->plan;
    const float* phi = (const float*)P->phi;  // padded, one value a point
    FieldLayout pl = P->flayout;
    pl.fstride = 0;
    pl.pstride = 1;
    // every caller runs this right after a solve of the same n sites on the
    // same stream, which left their tile order in the plan
    const bool by_tile = n <= P->slot_cap && P->tiles;
    const int2* tiles = by_tile ? P->tiles : nullptr;
    const int blocks = by_tile ? P->g.ntiles : (int)((n + 127) / 128);
    return with_nin(C->nin, [&](auto N) -> cudaError_t {
        constexpr int NIN = decltype(N)::value;
#define PPPM_FEAT(PP)                                                                                           \
    case PP:                                                                                                    \
        k_features<PP, NIN><<<blocks, 128, 0, s>>>(P->g, pl, phi, pos, types, tiles, P->sorig, (int)n, C->s_in,  \
                                                   feat);                                                         \
        break;
        switch (P->order) {
            PPPM_FEAT(3)
            PPPM_FEAT(4)
            PPPM_FEAT(5)
            PPPM_FEAT(6)
            PPPM_FEAT(7)
            default: return cudaErrorInvalidValue;
        }
#undef PPPM_FEAT
        return cudaGetLastError();
    });
}

int mlp_forward(pppm_corr* C, cudaStream_t s, const __nv_bfloat16* feat, int64_t n, const float* q, float* forces,
                float* out) {
    if (n == 0) return PPPM_OK;
    // both kernels read BF16 pairs as 4-byte words: a feature pointer off the
    // 4-byte grid is rejected before any launch
    if (n > (int64_t(1) << 30) || (reinterpret_cast<uintptr_t>(feat) & 3) != 0) return PPPM_ERR_INVALID_ARG;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    // the tcgen05 kernel reads a feature row as 16-byte vectors
    if (C->forward == PPPM_FORWARD_TCGEN05 && (reinterpret_cast<uintptr_t>(feat) & 15) == 0) {
        cudaError_t e = with_nin(C->nin, [&](auto N) {
            constexpr int NIN = decltype(N)::value;
            const size_t smem = tc::Smem<NIN>::BYTES;
            auto kern = tc::k_mlp_forward_tc<NIN>;
            cudaError_t e2 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e2 != cudaSuccess) return e2;
            // all of the SM's on-chip memory as shared memory, so that as many
            // CTAs are resident as registers and shared memory allow
            e2 = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared);
            if (e2 != cudaSuccess) return e2;
            // resident CTAs an SM from its registers, shared memory, threads
            // and tensor memory (512 columns)
            cudaFuncAttributes fa{};
            e2 = cudaFuncGetAttributes(&fa, kern);
            if (e2 != cudaSuccess) return e2;
            int smem_sm = 0, smem_rsv = 0, regs_sm = 0;
            cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
            cudaDeviceGetAttribute(&smem_rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
            cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
            int per_sm = std::min<int>(512 / (int)tc::kTmemCols, 2048 / tc::kThreads);
            per_sm = std::min<int>(per_sm, smem_sm / (int)(smem + fa.sharedSizeBytes + smem_rsv));
            if (fa.numRegs > 0) per_sm = std::min<int>(per_sm, regs_sm / (fa.numRegs * tc::kThreads));
            const int64_t ntile = (n + tc::kRows - 1) / tc::kRows;
            const int blocks = (int)std::min<int64_t>(ntile, (int64_t)std::max(per_sm, 1) * nsm);
            kern<<<blocks, tc::kThreads, smem, s>>>(feat, (int)n, C->wbf, C->master, C->s_out, q, forces, out,
                                                     C->plan->status, C->wait_limit);
            return cudaGetLastError();
        });
        CC(e);
        return PPPM_OK;
    }
    const int tiles = (int)((n + 15) / 16);
    int blocks = (tiles + 3) / 4;
    if (blocks > 8 * nsm) blocks = 8 * nsm;
    with_nin(C->nin, [&](auto N) {
        k_mlp_forward<decltype(N)::value><<<blocks, 128, 0, s>>>(feat, (int)n, C->wbf, C->master, C->s_out, q,
                                                                  forces, out);
        return 0;
    });
    CC(cudaGetLastError());
    return PPPM_OK;
}

template <int NIN>
constexpr size_t grad_smem() {
    return sizeof(float) * (NH * NIN + NH * NH + NOUT * NH + 2 * NH + 4 + TB * Net<NIN>::XP + 2 * TB * HP + TB * 4 +
                            32);
}

int grad_step(pppm_corr* C, cudaStream_t s, const __nv_bfloat16* feat, const float* target, int64_t nrows,
              const int* idx, int64_t nb, float* grad_out, float* loss_out, bool adam, float lr) {
    if (nb <= 0 || nrows <= 0 || nb > (int64_t(1) << 30) || (!idx && nb > nrows)) return PPPM_ERR_INVALID_ARG;
    const int nblk = (int)((nb + TB - 1) / TB);
    int rc = ensure_partial(C, nblk);
    if (rc != PPPM_OK) return rc;
    const cudaError_t ge = with_nin(C->nin, [&](auto N) -> cudaError_t {
        constexpr int NIN = decltype(N)::value;
        constexpr size_t smem = grad_smem<NIN>();
        const cudaError_t e = cudaFuncSetAttribute(k_mlp_grad<NIN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)smem);
        if (e != cudaSuccess) return e;
        k_mlp_grad<NIN><<<nblk, TB, smem, s>>>(feat, target, nrows, idx, (int)nb, 1.f / (float)nb, C->master,
                                               C->partial, C->lossp);
        return cudaGetLastError();
    });
    CC(ge);
    float bc1 = 1.f, bc2 = 1.f;
    if (adam) {
        C->step += 1;
        bc1 = 1.f - powf(0.9f, (float)C->step);
        bc2 = 1.f - powf(0.999f, (float)C->step);
    }
    const int npar = nparam_of(C->nin);
    with_nin(C->nin, [&](auto N) {
        k_reduce_adam<decltype(N)::value><<<(npar + 255) / 256, 256, 0, s>>>(
            C->partial, C->lossp, nblk, grad_out, loss_out, adam ? C->master : nullptr, C->m1, C->m2, lr, 0.9f,
            0.999f, 1e-8f, bc1, bc2);
        return 0;
    });
    CC(cudaGetLastError());
    if (adam) return refresh_bf16(C, s);
    return PPPM_OK;
}

}  // namespace

extern "C" {

int pppm_corr_create_features(pppm_plan* coarse, int features, pppm_corr** out) {
    if (!out) return PPPM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!coarse || coarse->precision != PPPM_FP32) return PPPM_ERR_INVALID_ARG;
    if (features != PPPM_CORR_CELL && features != PPPM_CORR_STATED) return PPPM_ERR_INVALID_ARG;
    pppm_corr* C = new (std::nothrow) pppm_corr();
    if (!C) return PPPM_ERR_CUDA;
    C->plan = coarse;
    C->nin = features == PPPM_CORR_STATED ? kNinStated : kNinCell;
    const int NPARAM = nparam_of(C->nin), NBF = nbf_of(C->nin);
    auto fail = [&](int code) {
        pppm_corr_destroy(C);
        return code;
    };
    const int prc = pppm_set_potential(coarse, 1);
    if (prc != PPPM_OK) return fail(prc);
    if (cudaMalloc((void**)&C->master, sizeof(float) * NPARAM) != cudaSuccess) return fail(PPPM_ERR_CUDA);
    if (cudaMalloc((void**)&C->m1, sizeof(float) * NPARAM) != cudaSuccess) return fail(PPPM_ERR_CUDA);
    if (cudaMalloc((void**)&C->m2, sizeof(float) * NPARAM) != cudaSuccess) return fail(PPPM_ERR_CUDA);
    if (cudaMalloc((void**)&C->wbf, sizeof(__nv_bfloat16) * NBF) != cudaSuccess) return fail(PPPM_ERR_CUDA);
    if (cudaMalloc((void**)&C->ev, sizeof(double) * 8) != cudaSuccess) return fail(PPPM_ERR_CUDA);
    if (cudaMemset(C->master, 0, sizeof(float) * NPARAM) != cudaSuccess) return fail(PPPM_ERR_CUDA);
    if (cudaMemset(C->m1, 0, sizeof(float) * NPARAM) != cudaSuccess) return fail(PPPM_ERR_CUDA);
    if (cudaMemset(C->m2, 0, sizeof(float) * NPARAM) != cudaSuccess) return fail(PPPM_ERR_CUDA);
    if (refresh_bf16(C, nullptr) != PPPM_OK || cudaDeviceSynchronize() != cudaSuccess) return fail(PPPM_ERR_CUDA);
    *out = C;
    return PPPM_OK;
}

int pppm_corr_create(pppm_plan* coarse, pppm_corr** out) {
    return pppm_corr_create_features(coarse, PPPM_CORR_CELL, out);
}

int pppm_corr_param_count(const pppm_corr* C) { return C ? nparam_of(C->nin) : PPPM_ERR_INVALID_ARG; }

int pppm_corr_feature_width(const pppm_corr* C) { return C ? C->nin : PPPM_ERR_INVALID_ARG; }

void pppm_corr_destroy(pppm_corr* C) {
    if (!C) return;
    cudaDeviceSynchronize();
    for (void* p : {(void*)C->master, (void*)C->m1, (void*)C->m2, (void*)C->wbf, (void*)C->partial, (void*)C->lossp,
                    (void*)C->feat, (void*)C->ev})
        if (p) cudaFree(p);
    delete C;
}

int pppm_corr_nparams(void) { return Net<kNinCell>::NPARAM; }

int pppm_corr_set_weights(pppm_corr* C, const float* params, double s_in, double s_out) {
    if (!C || !params || !(s_in > 0.0) || !(s_out > 0.0)) return PPPM_ERR_INVALID_ARG;
    const int NPARAM = nparam_of(C->nin);
    CC(cudaMemcpy(C->master, params, sizeof(float) * NPARAM, cudaMemcpyHostToDevice));
    CC(cudaMemset(C->m1, 0, sizeof(float) * NPARAM));
    CC(cudaMemset(C->m2, 0, sizeof(float) * NPARAM));
    C->step = 0;
    C->s_in = (float)s_in;
    C->s_out = (float)s_out;
    int rc = refresh_bf16(C, nullptr);
    if (rc != PPPM_OK) return rc;
    CC(cudaDeviceSynchronize());
    return PPPM_OK;
}

int pppm_corr_get_weights(const pppm_corr* C, float* params, double* s_in, double* s_out) {
    if (!C || !params) return PPPM_ERR_INVALID_ARG;
    CC(cudaDeviceSynchronize());
    CC(cudaMemcpy(params, C->master, sizeof(float) * nparam_of(C->nin), cudaMemcpyDeviceToHost));
    if (s_in) *s_in = C->s_in;
    if (s_out) *s_out = C->s_out;
    return PPPM_OK;
}

int pppm_corr_features(pppm_corr* C, void* stream, const float* pos, const float* q, const signed char* types,
                       int64_t n, void* feat, float* forces) {
    if (!C || n < 0 || !feat || (n > 0 && (!pos || !q || !types || !forces))) return PPPM_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(feat) & 15) return PPPM_ERR_INVALID_ARG;  // rows are written as 16-byte vectors
    cudaStream_t s = (cudaStream_t)stream;
    int rc = pppm_compute_f32(C->plan, stream, pos, q, n, C->ev, forces, C->ev + 1);
    if (rc != PPPM_OK) return rc;
    if (n == 0) return PPPM_OK;
    CC(launch_features(C, s, pos, types, n, (__nv_bfloat16*)feat));
    return PPPM_OK;
}

int pppm_corr_targets(pppm_corr* C, void* stream, const float* f_fine, const float* f_coarse, const float* q,
                      int64_t n, float* target) {
    if (!C || n < 0 || (n > 0 && (!f_fine || !f_coarse || !q || !target))) return PPPM_ERR_INVALID_ARG;
    if (n == 0) return PPPM_OK;
    const int64_t m = 3 * n;
    k_targets<<<(unsigned)((m + 255) / 256), 256, 0, (cudaStream_t)stream>>>(f_fine, f_coarse, q, n, C->s_out,
                                                                             target);
    CC(cudaGetLastError());
    return PPPM_OK;
}

int pppm_corr_calibrate(pppm_corr* C, void* stream, const float* pos, const float* q, const signed char* types,
                        int64_t n, const float* f_fine) {
    if (!C || n <= 0 || !pos || !q || !types || !f_fine) return PPPM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = ensure_feat(C, n);
    if (rc != PPPM_OK) return rc;
    float* fc = nullptr;
    double* part = nullptr;
    auto done = [&](int code) {
        if (fc) cudaFree(fc);
        if (part) cudaFree(part);
        return code;
    };
    if (cudaMalloc((void**)&fc, sizeof(float) * 3 * (size_t)n) != cudaSuccess) return done(PPPM_ERR_CUDA);
    if (cudaMalloc((void**)&part, sizeof(double) * 3 * kCalBlocks) != cudaSuccess) return done(PPPM_ERR_CUDA);
    const float keep_in = C->s_in;
    C->s_in = 1.f;
    rc = pppm_corr_features(C, stream, pos, q, types, n, C->feat, fc);
    C->s_in = keep_in;
    if (rc != PPPM_OK) return done(rc);
    with_nin(C->nin, [&](auto N) {
        k_calibrate<decltype(N)::value><<<kCalBlocks, 256, 0, s>>>(C->feat, f_fine, fc, q, (int)n, part);
        return 0;
    });
    if (cudaGetLastError() != cudaSuccess) return done(PPPM_ERR_CUDA);
    std::vector<double> h(3 * kCalBlocks);
    if (cudaMemcpyAsync(h.data(), part, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return done(PPPM_ERR_CUDA);
    double a = 0.0, b = 0.0, c = 0.0;
    for (int k = 0; k < kCalBlocks; ++k) {
        a += h[3 * k];
        b += h[3 * k + 1];
        c += h[3 * k + 2];
    }
    const double rms_in = std::sqrt(a / (27.0 * (double)n));
    const double rms_out = c > 0 ? std::sqrt(b / (3.0 * c)) : 0.0;
    if (!(rms_in > 0.0) || !(rms_out > 0.0) || !std::isfinite(rms_in) || !std::isfinite(rms_out))
        return done(PPPM_ERR_NONFINITE);
    C->s_in = (float)(1.0 / rms_in);
    C->s_out = (float)rms_out;
    return done(PPPM_OK);
}

int pppm_corr_get_scales(const pppm_corr* C, double* s_in, double* s_out) {
    if (!C || !s_in || !s_out) return PPPM_ERR_INVALID_ARG;
    *s_in = C->s_in;
    *s_out = C->s_out;
    return PPPM_OK;
}

int pppm_corr_set_wait_limit(pppm_corr* C, long long spins) {
    if (!C || spins < 0) return PPPM_ERR_INVALID_ARG;
    C->wait_limit = spins;
    return PPPM_OK;
}

int pppm_corr_set_forward(pppm_corr* C, int kind) {
    if (!C || (kind != PPPM_FORWARD_TCGEN05 && kind != PPPM_FORWARD_MMA_SYNC)) return PPPM_ERR_INVALID_ARG;
    C->forward = kind;
    return PPPM_OK;
}

int pppm_corr_forward(pppm_corr* C, void* stream, const void* feat, int64_t n, float* out) {
    if (!C || n < 0 || (n > 0 && (!feat || !out))) return PPPM_ERR_INVALID_ARG;
    return mlp_forward(C, (cudaStream_t)stream, (const __nv_bfloat16*)feat, n, nullptr, nullptr, out);
}

int pppm_corr_apply(pppm_corr* C, void* stream, const float* pos, const float* q, const signed char* types,
                    int64_t n, double* energy, float* forces, double* virial) {
    if (!C || n < 0 || !energy || !virial || (n > 0 && (!pos || !q || !types || !forces)))
        return PPPM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = pppm_compute_f32(C->plan, stream, pos, q, n, energy, forces, virial);
    if (rc != PPPM_OK) return rc;
    if (n == 0) return PPPM_OK;
    if ((rc = ensure_feat(C, n)) != PPPM_OK) return rc;
    CC(launch_features(C, s, pos, types, n, C->feat));
    return mlp_forward(C, s, C->feat, n, q, forces, nullptr);
}

int pppm_corr_grad(pppm_corr* C, void* stream, const void* feat, const float* target, int64_t nrows,
                   const int* idx, int64_t nb, float* grad, float* loss) {
    if (!C || !feat || !target || !grad) return PPPM_ERR_INVALID_ARG;
    return grad_step(C, (cudaStream_t)stream, (const __nv_bfloat16*)feat, target, nrows, idx, nb, grad, loss, false,
                     0.f);
}

int pppm_corr_train_step(pppm_corr* C, void* stream, const void* feat, const float* target, int64_t nrows,
                         const int* idx, int64_t nb, float lr, float* loss) {
    if (!C || !feat || !target || !(lr > 0.f)) return PPPM_ERR_INVALID_ARG;
    return grad_step(C, (cudaStream_t)stream, (const __nv_bfloat16*)feat, target, nrows, idx, nb, nullptr, loss, true,
                     lr);
}

// file: magic "PPPMCORR", version 1, nparams, s_in, s_out, step, master, m1, m2
int pppm_corr_save(const pppm_corr* C, const char* path) {
    if (!C || !path) return PPPM_ERR_INVALID_ARG;
    const int NPARAM = nparam_of(C->nin);
    std::vector<float> buf(3 * (size_t)NPARAM);
    CC(cudaDeviceSynchronize());
    CC(cudaMemcpy(buf.data(), C->master, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost));
    CC(cudaMemcpy(buf.data() + NPARAM, C->m1, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost));
    CC(cudaMemcpy(buf.data() + 2 * NPARAM, C->m2, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost));
    FILE* f = fopen(path, "wb");
    if (!f) return PPPM_ERR_INVALID_ARG;
    const int32_t hdr[2] = {1, NPARAM};
    const double sc[2] = {C->s_in, C->s_out};
    const int64_t st = C->step;
    bool ok = fwrite("PPPMCORR", 1, 8, f) == 8 && fwrite(hdr, sizeof(hdr), 1, f) == 1 &&
              fwrite(sc, sizeof(sc), 1, f) == 1 && fwrite(&st, sizeof(st), 1, f) == 1 &&
              fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    ok = (fclose(f) == 0) && ok;
    return ok ? PPPM_OK : PPPM_ERR_INVALID_ARG;
}

int pppm_corr_load(pppm_corr* C, const char* path) {
    if (!C || !path) return PPPM_ERR_INVALID_ARG;
    const int NPARAM = nparam_of(C->nin);
    FILE* f = fopen(path, "rb");
    if (!f) return PPPM_ERR_INVALID_ARG;
    char magic[8];
    int32_t hdr[2];
    double sc[2];
    int64_t st;
    std::vector<float> buf(3 * (size_t)NPARAM);
    bool ok = fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "PPPMCORR", 8) == 0 &&
              fread(hdr, sizeof(hdr), 1, f) == 1 && hdr[0] == 1 && hdr[1] == NPARAM &&
              fread(sc, sizeof(sc), 1, f) == 1 && fread(&st, sizeof(st), 1, f) == 1 &&
              fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    fclose(f);
    if (!ok) return PPPM_ERR_INVALID_ARG;
    CC(cudaMemcpy(C->master, buf.data(), sizeof(float) * NPARAM, cudaMemcpyHostToDevice));
    CC(cudaMemcpy(C->m1, buf.data() + NPARAM, sizeof(float) * NPARAM, cudaMemcpyHostToDevice));
    CC(cudaMemcpy(C->m2, buf.data() + 2 * NPARAM, sizeof(float) * NPARAM, cudaMemcpyHostToDevice));
    C->s_in = (float)sc[0];
    C->s_out = (float)sc[1];
    C->step = st;
    int rc = refresh_bf16(C, nullptr);
    if (rc != PPPM_OK) return rc;
    CC(cudaDeviceSynchronize());
    return PPPM_OK;
}

}  // extern "C"
