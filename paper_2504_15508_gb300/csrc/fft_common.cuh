// Device helpers shared by the FFT passes and the batched persistent kernel:
// complex arithmetic, the radix-2/3/4/5 butterflies and the run-time radix
// Stockham FFT over lines held in shared memory.
#pragma once

#include "internal.cuh"

namespace pppm {

// ------------------------------------------------------------------ complex helpers
template <typename R> struct CT;
// four reals of one mesh point, stored with one vector store
struct __align__(32) Real4d {
    double x, y, z, w;
};
template <> struct CT<float> {
    typedef float2 C;
    typedef float4 C4;
    static __device__ __forceinline__ C mk(float a, float b) { return make_float2(a, b); }
    static __device__ __forceinline__ C4 mk4(float a, float b, float c, float d) { return make_float4(a, b, c, d); }
};
template <> struct CT<double> {
    typedef double2 C;
    typedef Real4d C4;
    static __device__ __forceinline__ C mk(double a, double b) { return make_double2(a, b); }
    static __device__ __forceinline__ C4 mk4(double a, double b, double c, double d) { return Real4d{a, b, c, d}; }
};

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <typename C, typename R> __device__ __forceinline__ C cscale(C a, R s) { C r; r.x = a.x * s; r.y = a.y * s; return r; }
// multiply by i * s (s = +-1)
template <typename C, typename R> __device__ __forceinline__ C cmul_is(C a, R s) { C r; r.x = -s * a.y; r.y = s * a.x; return r; }
template <typename C> __device__ __forceinline__ C cconj(C a) { C r; r.x = a.x; r.y = -a.y; return r; }

// Small DFT of size Rdx in registers; s = -1 forward, +1 inverse.
template <typename C, typename R>
__device__ __forceinline__ void butterfly(C* v, int Rdx, R s) {
    if (Rdx == 2) {
        C a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if (Rdx == 4) {
        C a02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
        C a13 = cadd(v[1], v[3]), t = cmul_is(csub(v[1], v[3]), s);
        v[0] = cadd(a02, a13);
        v[2] = csub(a02, a13);
        v[1] = cadd(d02, t);
        v[3] = csub(d02, t);
    } else if (Rdx == 3) {
        const R c1 = R(-0.5), s1 = R(0.86602540378443864676);  // cos, sin of 2 pi / 3
        C t1 = cadd(v[1], v[2]);
        C t2 = cmul_is(csub(v[1], v[2]), s * s1);
        C m = cadd(v[0], cscale(t1, c1));
        v[0] = cadd(v[0], t1);
        v[1] = cadd(m, t2);
        v[2] = csub(m, t2);
    } else {  // 5
        const R c1 = R(0.30901699437494742410), c2 = R(-0.80901699437494742410);  // cos 2pi/5, cos 4pi/5
        const R s1 = R(0.95105651629515357212), s2 = R(0.58778525229247312917);   // sin 2pi/5, sin 4pi/5
        C a1 = cadd(v[1], v[4]), b1 = csub(v[1], v[4]);
        C a2 = cadd(v[2], v[3]), b2 = csub(v[2], v[3]);
        C m1 = cadd(v[0], cadd(cscale(a1, c1), cscale(a2, c2)));
        C m2 = cadd(v[0], cadd(cscale(a1, c2), cscale(a2, c1)));
        C n1 = cmul_is(cadd(cscale(b1, s1), cscale(b2, s2)), s);
        C n2 = cmul_is(csub(cscale(b1, s2), cscale(b2, s1)), s);
        v[0] = cadd(v[0], cadd(a1, a2));
        v[1] = cadd(m1, n1);
        v[4] = csub(m1, n1);
        v[2] = cadd(m2, n2);
        v[3] = csub(m2, n2);
    }
}

// Stockham FFT of `nl` lines of length rp.L held in shared buffer `a`
// (element t of line l at a[l * ls + t * ps]); `b` is the scratch partner.
// Returns the buffer holding the result.  line_fast picks which index the
// consecutive threads walk (the one with unit stride).
template <typename R>
__device__ typename CT<R>::C* stockham(typename CT<R>::C* a, typename CT<R>::C* b, int nl, int ls, int ps,
                                       const Radix& rp, const typename CT<R>::C* __restrict__ tw, R s,
                                       bool line_fast) {
    typedef typename CT<R>::C C;
    C* src = a;
    C* dst = b;
    const int L = rp.L;
    int Ns = 1;
    for (int st = 0; st < rp.n; ++st) {
        const int Rdx = rp.r[st];
        const int nbf = L / Rdx;
        const int total = nbf * nl;
        const int tstep = L / (Ns * Rdx);
        for (int it = threadIdx.x; it < total; it += blockDim.x) {
            int line, j;
            if (line_fast) { line = it % nl; j = it / nl; } else { j = it % nbf; line = it / nbf; }
            const int k = j % Ns;
            C v[5];
            const C* sp = src + line * ls;
#pragma unroll
            for (int r = 0; r < 5; ++r)
                if (r < Rdx) v[r] = sp[(j + r * nbf) * ps];
            if (k != 0) {
#pragma unroll
                for (int r = 1; r < 5; ++r)
                    if (r < Rdx) {
                        C w = __ldg(&tw[k * r * tstep]);
                        if (s > R(0)) w.y = -w.y;
                        v[r] = cmul(v[r], w);
                    }
            }
            butterfly<C, R>(v, Rdx, s);
            const int d0 = (j / Ns) * Ns * Rdx + k;
            C* dp = dst + line * ls;
#pragma unroll
            for (int r = 0; r < 5; ++r)
                if (r < Rdx) dp[(d0 + r * Ns) * ps] = v[r];
        }
        __syncthreads();
        C* t = src; src = dst; dst = t;
        Ns *= Rdx;
    }
    return src;
}




// ------------------------------------------------------------------ compile-time engine core
// (used by the single-box passes in fft_kernels.cu and by the batched form's
// staged FFT kernels)
constexpr int kFftThreads = 256;

// ------------------------------------------------------------------ compile-time radix plan
// Radices 16, 10 and 8 are DFTs in registers (below), so the workload lengths
// take two Stockham stages: 128 = 16 x 8, 160 = 16 x 10, 64 = 16 x 4, 32 = 16 x 2.
constexpr int fft_radix(int L, int s) {
    int m = L, i = 0;
    const int fs[7] = {16, 10, 8, 4, 2, 3, 5};
    for (int q = 0; q < 7; ++q)
        while (m % fs[q] == 0) {
            if (i == s) return fs[q];
            m /= fs[q];
            ++i;
        }
    return 1;
}
constexpr int fft_nstages(int L) {
    int n = 0;
    while (fft_radix(L, n) != 1) ++n;
    return n;
}
constexpr int fft_ns(int L, int s) {
    int ns = 1;
    for (int i = 0; i < s; ++i) ns *= fft_radix(L, i);
    return ns;
}

// cos and sin of 2 pi m / N for the twiddles inside the register DFTs
// (N = 8, 10, 16; closed forms of the regular 8-, 10- and 16-gon)
template <int N>
__device__ __forceinline__ constexpr double unit_cos(int m) {
    constexpr double r = 0.70710678118654752440, c8 = 0.92387953251128675613, s8 = 0.38268343236508977173;
    constexpr double c5 = 0.80901699437494742410, c25 = 0.30901699437494742410;
    if (N == 16) {
        const double t[16] = {1, c8, r, s8, 0, -s8, -r, -c8, -1, -c8, -r, -s8, 0, s8, r, c8};
        return t[m & 15];
    } else if (N == 8) {
        const double t[8] = {1, r, 0, -r, -1, -r, 0, r};
        return t[m & 7];
    } else {
        const double t[10] = {1, c5, c25, -c25, -c5, -1, -c5, -c25, c25, c5};
        return t[m % 10];
    }
}
template <int N>
__device__ __forceinline__ constexpr double unit_sin(int m) {
    constexpr double r = 0.70710678118654752440, c8 = 0.92387953251128675613, s8 = 0.38268343236508977173;
    constexpr double s5 = 0.58778525229247312917, s25 = 0.95105651629515357212;
    if (N == 16) {
        const double t[16] = {0, s8, r, c8, 1, c8, r, s8, 0, -s8, -r, -c8, -1, -c8, -r, -s8};
        return t[m & 15];
    } else if (N == 8) {
        const double t[8] = {0, r, 1, r, 0, -r, -1, -r};
        return t[m & 7];
    } else {
        const double t[10] = {0, s5, s25, s25, s5, 0, -s5, -s25, -s25, -s5};
        return t[m % 10];
    }
}

// DFT of N = A B points in registers, X[k] = sum_n x[n] e^{SIGN 2 pi i n k / N}:
// with n = B n1 + n2 and k = k1 + A k2, a size-A DFT over n1 for each n2, the
// twiddle e^{SIGN 2 pi i n2 k1 / N}, then a size-B DFT over n2 for each k1.
template <typename C, typename R, int A, int B, int SIGN>
__device__ __forceinline__ void dft_ab(C* v) {
    constexpr int N = A * B;
    C t[B][A];
#pragma unroll
    for (int n2 = 0; n2 < B; ++n2) {
#pragma unroll
        for (int n1 = 0; n1 < A; ++n1) t[n2][n1] = v[B * n1 + n2];
        butterfly<C, R>(t[n2], A, R(SIGN));
#pragma unroll
        for (int k1 = 1; k1 < A; ++k1)
            if (n2 > 0) {
                const C w = CT<R>::mk(R(unit_cos<N>(n2 * k1)), R(SIGN) * R(unit_sin<N>(n2 * k1)));
                t[n2][k1] = cmul(t[n2][k1], w);
            }
    }
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) {
        C u[B];
#pragma unroll
        for (int n2 = 0; n2 < B; ++n2) u[n2] = t[n2][k1];
        butterfly<C, R>(u, B, R(SIGN));
#pragma unroll
        for (int k2 = 0; k2 < B; ++k2) v[k1 + A * k2] = u[k2];
    }
}

template <typename C, typename R, int RDX, int SIGN>
__device__ __forceinline__ void bfly(C* v) {
    if constexpr (RDX == 16) dft_ab<C, R, 4, 4, SIGN>(v);
    else if constexpr (RDX == 10) dft_ab<C, R, 5, 2, SIGN>(v);
    else if constexpr (RDX == 8) dft_ab<C, R, 4, 2, SIGN>(v);
    else butterfly<C, R>(v, RDX, R(SIGN));
}

// One Stockham stage with every size a constant.  Thread mapping: line-fast
// (bundles, lines adjacent in shared memory) uses 16 lanes per line index and
// the other threads along the butterflies; otherwise consecutive threads walk
// the butterflies of a line and then the lines.
template <typename R, int L, int S, int SIGN, bool LF>
__device__ __forceinline__ void ct_stage(const typename CT<R>::C* __restrict__ src, typename CT<R>::C* __restrict__ dst,
                                         int nl, int ls, int ps, const typename CT<R>::C* __restrict__ tw) {
    typedef typename CT<R>::C C;
    constexpr int RDX = fft_radix(L, S);
    constexpr int NS = fft_ns(L, S);
    constexpr int NBF = L / RDX;
    constexpr int TSTEP = L / (NS * RDX);
    auto one = [&](int line, int j) {
        const int k = j % NS;
        const C* sp = src + line * ls;
        C* dp = dst + line * ls;
        C v[RDX];
#pragma unroll
        for (int r = 0; r < RDX; ++r) v[r] = sp[(j + r * NBF) * ps];
        if (NS > 1) {
#pragma unroll
            for (int r = 1; r < RDX; ++r) {
                C w = __ldg(&tw[k * r * TSTEP]);
                if (SIGN > 0) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        bfly<C, R, RDX, SIGN>(v);
        const int d0 = (j / NS) * NS * RDX + k;
#pragma unroll
        for (int r = 0; r < RDX; ++r) dp[(d0 + r * NS) * ps] = v[r];
    };
    if (LF) {
        const int tl = threadIdx.x & 15, tj = threadIdx.x >> 4;
        for (int line = tl; line < nl; line += 16)
            for (int j = tj; j < NBF; j += kFftThreads >> 4) one(line, j);
    } else {
        for (int it = threadIdx.x; it < nl * NBF; it += kFftThreads) one(it / NBF, it % NBF);
    }
}

template <typename R, int L, int SIGN, bool LF, int S>
__device__ __forceinline__ typename CT<R>::C* ct_fft(typename CT<R>::C* a, typename CT<R>::C* b, int nl, int ls,
                                                     int ps, const typename CT<R>::C* __restrict__ tw) {
    if constexpr (S == fft_nstages(L)) {
        return a;
    } else {
        ct_stage<R, L, S, SIGN, LF>(a, b, nl, ls, ps, tw);
        __syncthreads();
        return ct_fft<R, L, SIGN, LF, S + 1>(b, a, nl, ls, ps, tw);
    }
}

}  // namespace pppm

namespace pppm {

// ------------------------------------------------------------------ short lines on the tensor cores
// The DFT of nl lines of length L <= kDftTcMax as one real matrix product
// (X = F_N x per axis):
//   [Re Y; Im Y] = [[C, -s S], [s S, C]] [Re x; Im x],  C = cos, S = sin of 2 pi k t / L,
// s = -1 forward, +1 inverse, on mma.sync m16n8k8 TF32 tensor-core
// instructions.  Each FP32 operand is split into a TF32 high part and a TF32
// remainder and three products are summed (hi hi + hi lo + lo hi), each
// k-step's in the tensor core and the k-steps in FP32, which keeps the result
// at FP32 accuracy.  Element t of line l is at
// a[l * ls + t * ps]; the result is written to b in the same layout and b is
// returned.  Every thread of the block must call it (it ends with a barrier).
constexpr int kDftTcMax = 18;

__device__ __forceinline__ uint32_t tf32_hi(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void mma_tf32_16x8x8(float d[4], const uint32_t a[4], const uint32_t b[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// element (m, j) of the real-block DFT matrix, 0 outside [0, 2L)^2;
// tw[m] = e^{-2 pi i m / L}
__device__ __forceinline__ float dft_block_elem(int m, int j, int L, const float2* __restrict__ tw, float s) {
    if (m >= 2 * L || j >= 2 * L) return 0.f;
    const int k = m < L ? m : m - L, t = j < L ? j : j - L;
    const float2 w = __ldg(&tw[(k * t) % L]);
    const float c = w.x, sn = -w.y;  // cos, sin of 2 pi k t / L
    if (m < L) return j < L ? c : -s * sn;
    return j < L ? s * sn : c;
}

__device__ inline float2* dft_tc(float2* a, float2* b, int nl, int ls, int ps, int L, const float2* __restrict__ tw,
                          float s) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int gid = lane >> 2, tig = lane & 3;
    const int MT = (2 * L + 15) / 16, KT = (2 * L + 7) / 8, NT = (nl + 7) / 8;
    for (int tile = warp; tile < MT * NT; tile += nwarps) {
        const int mt = tile / NT, nt = tile - mt * NT;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        const int line = nt * 8 + gid;  // this lane's column of B
        for (int kk = 0; kk < KT; ++kk) {
            const int j0 = kk * 8 + tig, j1 = j0 + 4;
            const float av[4] = {dft_block_elem(mt * 16 + gid, j0, L, tw, s),
                                 dft_block_elem(mt * 16 + gid + 8, j0, L, tw, s),
                                 dft_block_elem(mt * 16 + gid, j1, L, tw, s),
                                 dft_block_elem(mt * 16 + gid + 8, j1, L, tw, s)};
            float bv[2] = {0.f, 0.f};
            if (line < nl) {
                if (j0 < 2 * L) {
                    const float2 x = a[line * ls + (j0 < L ? j0 : j0 - L) * ps];
                    bv[0] = j0 < L ? x.x : x.y;
                }
                if (j1 < 2 * L) {
                    const float2 x = a[line * ls + (j1 < L ? j1 : j1 - L) * ps];
                    bv[1] = j1 < L ? x.x : x.y;
                }
            }
            uint32_t ah[4], al[4], bh[2], bl[2];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                ah[q] = tf32_hi(av[q]);
                al[q] = tf32_hi(av[q] - __uint_as_float(ah[q]));
            }
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                bh[q] = tf32_hi(bv[q]);
                bl[q] = tf32_hi(bv[q] - __uint_as_float(bh[q]));
            }
            // each k-step's products start from zero in the tensor core and are
            // added to the running sums in round-to-nearest FP32, so that the
            // tensor core's own accumulation spans only 8 terms
            float pc[4] = {0.f, 0.f, 0.f, 0.f}, ph[4] = {0.f, 0.f, 0.f, 0.f};
            mma_tf32_16x8x8(pc, al, bh);
            mma_tf32_16x8x8(pc, ah, bl);
            mma_tf32_16x8x8(ph, ah, bh);
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] += ph[q] + pc[q];
        }
        // c0, c1: row gid, columns 2 tig, 2 tig + 1; c2, c3: row gid + 8
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int m = mt * 16 + gid + (q >= 2 ? 8 : 0);
            const int n = nt * 8 + 2 * tig + (q & 1);
            if (m < 2 * L && n < nl) {
                float2* dst = &b[n * ls + (m < L ? m : m - L) * ps];
                if (m < L) dst->x = acc[q];
                else dst->y = acc[q];
            }
        }
    }
    __syncthreads();
    return b;
}

// ------------------------------------------------------------------ int32-quantised DFT (ablation)
// The DFT of nl lines of length L as in the paper's hardware-offloaded FFT
// (Section "Hardware-offloaded 3D FFT", its data-quantisation panel): the line
// is split into nodes of `group` consecutive points; each node's partial sum
// of x_t e^{s 2 pi i k t / L} over its points (FP32) is multiplied by `scale`
// (the paper's 10^7), rounded to the nearest integer and clamped to int32 (a
// clamped value sets bit 8 of *status), and the nodes' integers are added
// exactly; the sum is scaled back.  One thread per output; layout and return
// as dft_tc.
__device__ __forceinline__ long long quant_int32(float v, double scale, bool& saturated) {
    double y = rint((double)v * scale);
    if (!(fabs(y) <= 2147483647.0)) {  // also catches a non-finite value
        saturated = true;
        y = y > 0.0 ? 2147483647.0 : -2147483648.0;
    }
    return (long long)y;
}

__device__ inline float2* dft_quant(const float2* a, float2* b, int nl, int ls, int ps, int L, int group,
                                    double scale, const float2* __restrict__ tw, float s,
                                    int* __restrict__ status) {
    bool saturated = false;
    for (int idx = threadIdx.x; idx < nl * L; idx += blockDim.x) {
        const int line = idx / L, k = idx - line * L;
        const float2* x = a + line * ls;
        long long ar = 0, ai = 0;
        for (int t0 = 0; t0 < L; t0 += group) {
            float pr = 0.f, pi = 0.f;
            for (int t = t0; t < t0 + group; ++t) {
                const float2 w = __ldg(&tw[(k * t) % L]);  // e^{-2 pi i k t / L}
                const float wr = w.x, wi = -s * w.y;      // e^{s 2 pi i k t / L}
                const float2 v = x[t * ps];
                pr += v.x * wr - v.y * wi;
                pi += v.x * wi + v.y * wr;
            }
            ar += quant_int32(pr, scale, saturated);
            ai += quant_int32(pi, scale, saturated);
        }
        b[line * ls + k * ps] = make_float2((float)((double)ar / scale), (float)((double)ai / scale));
    }
    if (saturated) atomicOr(status, 8);
    __syncthreads();
    return b;
}

// Stockham FFT of nl lines with the compile-time engine where the length has
// one (2^a 3^b 5^c lengths 8 to 64, the batched form's meshes), the run-time
// one otherwise.
template <int SIGN, bool LF>
__device__ __forceinline__ float2* stockham_ct(float2* a, float2* b, int nl, int ls, int ps, const Radix& rp,
                                               const float2* __restrict__ tw) {
    switch (rp.L) {
#define PPPM_CT_LEN(LL) \
    case LL: return ct_fft<float, LL, SIGN, LF, 0>(a, b, nl, ls, ps, tw);
        PPPM_CT_LEN(8) PPPM_CT_LEN(9) PPPM_CT_LEN(10) PPPM_CT_LEN(12) PPPM_CT_LEN(15) PPPM_CT_LEN(16)
        PPPM_CT_LEN(18) PPPM_CT_LEN(20) PPPM_CT_LEN(24) PPPM_CT_LEN(25) PPPM_CT_LEN(27) PPPM_CT_LEN(30)
        PPPM_CT_LEN(32) PPPM_CT_LEN(36) PPPM_CT_LEN(40) PPPM_CT_LEN(45) PPPM_CT_LEN(48) PPPM_CT_LEN(50)
        PPPM_CT_LEN(54) PPPM_CT_LEN(60) PPPM_CT_LEN(64)
#undef PPPM_CT_LEN
        default: return stockham<float>(a, b, nl, ls, ps, rp, tw, (float)SIGN, LF);
    }
}

// The batched form's line transform, its sign and thread mapping fixed at
// compile time: the int32-quantised DFT with nodes of qg points (qg > 0: that
// ablation is on for this axis; Q compiles the branch in, a separate kernel
// instantiation, so that the default kernels carry none of its registers),
// the tensor-core DFT for short lines (when enabled), else the Stockham FFT,
// from the compile-time engines when CT.
template <bool Q, bool CT, int SIGN, bool LF>
__device__ __forceinline__ float2* line_transform_t(float2* a, float2* b, int nl, int ls, int ps, const Radix& rp,
                                                    const float2* __restrict__ tw, int dft_max, int qg,
                                                    double qscale, int* status) {
    if constexpr (Q)
        if (qg > 0) return dft_quant(a, b, nl, ls, ps, rp.L, qg, qscale, tw, (float)SIGN, status);
    if (rp.L <= dft_max) return dft_tc(a, b, nl, ls, ps, rp.L, tw, (float)SIGN);
    if constexpr (CT) return stockham_ct<SIGN, LF>(a, b, nl, ls, ps, rp, tw);
    return stockham<float>(a, b, nl, ls, ps, rp, tw, (float)SIGN, LF);
}

}  // namespace pppm
