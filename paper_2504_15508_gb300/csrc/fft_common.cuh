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

// line transform for the batched kernel: the int32-quantised DFT with nodes
// of qg points (qg > 0: that ablation is on for this axis), the tensor-core
// DFT for short lines (when enabled), the Stockham FFT otherwise.  Q compiles
// the quantised branch in (a separate kernel instantiation, so that the
// default kernel carries none of its registers).
template <bool Q>
__device__ __forceinline__ float2* line_transform(float2* a, float2* b, int nl, int ls, int ps, const Radix& rp,
                                                  const float2* __restrict__ tw, float s, bool line_fast,
                                                  int dft_max, int qg, double qscale, int* status) {
    if constexpr (Q)
        if (qg > 0) return dft_quant(a, b, nl, ls, ps, rp.L, qg, qscale, tw, s, status);
    if (rp.L <= dft_max) return dft_tc(a, b, nl, ls, ps, rp.L, tw, s);
    return stockham<float>(a, b, nl, ls, ps, rp, tw, s, line_fast);
}

}  // namespace pppm
