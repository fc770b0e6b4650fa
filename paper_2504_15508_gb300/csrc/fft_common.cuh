// Device helpers shared by the FFT passes and the batched persistent kernel:
// complex arithmetic, the radix-2/3/4/5 butterflies and the run-time radix
// Stockham FFT over lines held in shared memory.
#pragma once

#include "internal.cuh"

namespace pppm {

// ------------------------------------------------------------------ complex helpers
template <typename R> struct CT;
template <> struct CT<float> {
    typedef float2 C;
    static __device__ __forceinline__ C mk(float a, float b) { return make_float2(a, b); }
};
template <> struct CT<double> {
    typedef double2 C;
    static __device__ __forceinline__ C mk(double a, double b) { return make_double2(a, b); }
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
