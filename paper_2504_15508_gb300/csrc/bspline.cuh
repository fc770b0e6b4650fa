// Order-p cardinal B-spline charge-assignment weights.
//
// For a site at mesh coordinate u (position / h) the p stencil points are the
// mesh points nearest to u: base g = floor(u + 1/2) for odd p, g = floor(u) for
// even p, points g + kmin + j for j = 0..p-1 (kmin = -(p-1)/2 for odd p,
// -p/2 + 1 for even p).  Point j gets M_p(g + kmin + j - u) with M_p the centred
// cardinal B-spline of order p.  Writing x0 = g + kmin - u + p/2, which lies in
// (0, 1], that weight is N_p(x0 + j), where N_p is the uniform B-spline on
// [0, p).  On x0 in [0, 1] each N_p(x0 + j) is one polynomial piece of degree
// p-1; the pieces' coefficients are built on the host by the recursion
// N_m(t) = (t N_{m-1}(t) + (m - t) N_{m-1}(t - 1)) / (m - 1) applied to
// polynomials, and evaluated here with Horner's rule.
#pragma once

#include "internal.cuh"

namespace pppm {

// c_bsp[p][j][m]: coefficient of x0^m in piece j of the order-p B-spline.
// Each translation unit that includes this header has its own copy, filled by
// bsp_upload_this_unit() (called at plan creation, never during capture).
static __constant__ double c_bsp_d[kMaxOrder + 1][kMaxOrder][kMaxOrder];
static __constant__ float c_bsp_f[kMaxOrder + 1][kMaxOrder][kMaxOrder];

// Piece coefficients of N_p on [0, 1] for p = 1..7, from the Cox-de Boor
// recursion carried out on polynomials in x0 (FP64 on the host).
static void bsp_upload_this_unit() {
    static bool done = false;
    if (done) return;
    double cd[kMaxOrder + 1][kMaxOrder][kMaxOrder] = {};
    float cf[kMaxOrder + 1][kMaxOrder][kMaxOrder] = {};
    // piece j of N_m as a polynomial in x0: poly[j][k] = coefficient of x0^k, for t = x0 + j.
    double poly[kMaxOrder][kMaxOrder] = {};
    poly[0][0] = 1.0;  // N_1(x0) = 1 on [0, 1]
    for (int p = 1; p <= kMaxOrder; ++p) {
        if (p > 1) {
            double nxt[kMaxOrder][kMaxOrder] = {};
            for (int j = 0; j < p; ++j) {
                // N_p(x0 + j) = ((x0 + j) N_{p-1}(x0 + j) + (p - x0 - j) N_{p-1}(x0 + j - 1)) / (p - 1)
                for (int k = 0; k < p - 1; ++k) {
                    const double a = (j < p - 1) ? poly[j][k] : 0.0;  // N_{p-1}(x0 + j)
                    const double b = (j >= 1) ? poly[j - 1][k] : 0.0; // N_{p-1}(x0 + j - 1)
                    nxt[j][k + 1] += a - b;                            // x0 * (a - b)
                    nxt[j][k] += j * a + (p - j) * b;
                }
                for (int k = 0; k < p; ++k) nxt[j][k] /= (p - 1);
            }
            for (int j = 0; j < kMaxOrder; ++j)
                for (int k = 0; k < kMaxOrder; ++k) poly[j][k] = nxt[j][k];
        }
        for (int j = 0; j < p; ++j)
            for (int k = 0; k < p; ++k) {
                cd[p][j][k] = poly[j][k];
                cf[p][j][k] = (float)poly[j][k];
            }
    }
    cudaMemcpyToSymbol(c_bsp_d, cd, sizeof(cd));
    cudaMemcpyToSymbol(c_bsp_f, cf, sizeof(cf));
    done = true;
}

template <typename T> __device__ __forceinline__ T bsp_coef(int p, int j, int m);
template <> __device__ __forceinline__ float bsp_coef<float>(int p, int j, int m) { return c_bsp_f[p][j][m]; }
template <> __device__ __forceinline__ double bsp_coef<double>(int p, int j, int m) { return c_bsp_d[p][j][m]; }

// Coefficients of all P pieces in registers (uniform across the warp).
template <typename T, int P>
struct BspCoef {
    T c[P][P];
    __device__ __forceinline__ void load() {
#pragma unroll
        for (int j = 0; j < P; ++j)
#pragma unroll
            for (int m = 0; m < P; ++m) c[j][m] = bsp_coef<T>(P, j, m);
    }
    __device__ __forceinline__ T piece(int j, T x) const {
        T r = c[j][P - 1];
#pragma unroll
        for (int m = P - 2; m >= 0; --m) r = r * x + c[j][m];
        return r;
    }
    __device__ __forceinline__ void all(T x, T w[P]) const {
#pragma unroll
        for (int j = 0; j < P; ++j) w[j] = piece(j, x);
    }
};

// The per-site weights the spread and the gather use, from a site's record:
// w[0..p-1] = q W_x, w[p..2p-1] = W_y, w[2p..3p-1] = W_z, zeros up to
// wstride(p).  The fast spread evaluates them with this function; the TMA
// gather evaluates the same expressions one axis a lane (BspCoef::all, then
// the x weights times q), so that a site's weights are the same values in
// both.
template <typename T, int P>
__device__ __forceinline__ void site_weights(const BspCoef<T, P>& co, const Rec<T>& r, T (&w)[wstride(P)]) {
    T t[P];
    co.all(r.x0[0], t);
#pragma unroll
    for (int a = 0; a < P; ++a) w[a] = t[a] * r.q;
    co.all(r.x0[1], t);
#pragma unroll
    for (int a = 0; a < P; ++a) w[P + a] = t[a];
    co.all(r.x0[2], t);
#pragma unroll
    for (int a = 0; a < P; ++a) w[2 * P + a] = t[a];
#pragma unroll
    for (int a = 3 * P; a < wstride(P); ++a) w[a] = T(0);
}

// One piece with its coefficients in registers (piece index fixed per thread).
template <typename T, int P>
struct BspPiece {
    T c[P];
    __device__ __forceinline__ void load(int j) {
#pragma unroll
        for (int m = 0; m < P; ++m) c[m] = bsp_coef<T>(P, j, m);
    }
    __device__ __forceinline__ T eval(T x) const {
        T r = c[P - 1];
#pragma unroll
        for (int m = P - 2; m >= 0; --m) r = r * x + c[m];
        return r;
    }
};

}  // namespace pppm
