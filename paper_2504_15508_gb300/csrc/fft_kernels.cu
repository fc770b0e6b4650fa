// Mixed-radix (2, 3, 4, 5) 3D FFT passes of the PPPM path, and the fused
// influence-function pass.
//
// Layout: real meshes are Nx x Ny x Nz (z fastest); spectra are half spectra
// Nx x Ny x Hz complex, Hz = Nz/2 + 1, in the same order.
//
// Every pass moves a batch of 1D lines into shared memory, transforms them
// with a self-sorting (Stockham) mixed-radix FFT between two shared buffers,
// and writes them back:
//   z forward   real rows, two per complex FFT (a + i b), unpacked to two half rows;
//   y, x        strided lines, B consecutive (outer, kz) lines per block;
//   x + G       forward x FFT, multiply by the influence function with the
//               energy/virial reduction, and the inverse x FFTs of G rho and
//               -i kx G rho in one block (Poisson-ik, Section 3.1 of the paper);
//   y inverse   of G rho and -i ky G rho (after x) and of -i kx G rho;
//   z inverse   Hermitian half rows of two rows (or two fields) packed as a + i b.
// Twiddles come from a table of e^{-2 pi i t / L} built on the device in FP64
// with sincospi and rounded to the mesh precision.
//
// Two FFT engines drive the same kernels: CtEngine<L> for the common FP32 mesh
// lengths (32 to 256: every index and radix is a compile-time constant), and
// GenEngine for any other 2^a 3^b 5^c length and for FP64 (radix plan read at
// run time).
#include <type_traits>

#include "fft_common.cuh"
#include "internal.cuh"

namespace pppm {

template <typename R, int L>
struct CtEngine {
    typedef typename CT<R>::C C;
    static constexpr int kLen = L;  // compile-time length (0: known at run time)
    const C* tw;
    __device__ __forceinline__ static constexpr int len() { return L; }
    template <int SIGN, bool LF>
    __device__ __forceinline__ C* run(C* a, C* b, int nl, int ls, int ps) const {
        return ct_fft<R, L, SIGN, LF, 0>(a, b, nl, ls, ps, tw);
    }
};

template <typename R>
struct GenEngine {
    typedef typename CT<R>::C C;
    static constexpr int kLen = 0;
    Radix rp;
    const C* tw;
    __device__ __forceinline__ int len() const { return rp.L; }
    template <int SIGN, bool LF>
    __device__ __forceinline__ C* run(C* a, C* b, int nl, int ls, int ps) const {
        return stockham<R>(a, b, nl, ls, ps, rp, tw, R(SIGN), LF);
    }
};

// Runs f(engine) with the compile-time engine when one exists for (T, L).
template <typename T, typename F>
cudaError_t with_engine(const Radix& r, const typename Cx<T>::t* tw, F&& f) {
    if constexpr (std::is_same<T, float>::value) {
        switch (r.L) {
            case 32: return f(CtEngine<float, 32>{tw});
            case 48: return f(CtEngine<float, 48>{tw});
            case 64: return f(CtEngine<float, 64>{tw});
            case 72: return f(CtEngine<float, 72>{tw});
            case 80: return f(CtEngine<float, 80>{tw});
            case 90: return f(CtEngine<float, 90>{tw});
            case 96: return f(CtEngine<float, 96>{tw});
            case 100: return f(CtEngine<float, 100>{tw});
            case 108: return f(CtEngine<float, 108>{tw});
            case 120: return f(CtEngine<float, 120>{tw});
            case 128: return f(CtEngine<float, 128>{tw});
            case 144: return f(CtEngine<float, 144>{tw});
            case 160: return f(CtEngine<float, 160>{tw});
            case 192: return f(CtEngine<float, 192>{tw});
            case 256: return f(CtEngine<float, 256>{tw});
            default: break;
        }
    }
    return f(GenEngine<T>{r, tw});
}

template <typename K>
cudaError_t set_smem(K kernel, size_t smem) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// 2D loop helpers for the bundle kernels: rows of the line (t) by 16-lane groups,
// lines (l) by lane within the group.
#define BUNDLE_LOOP(t, l, L_, nl_)                                              \
    _Pragma("unroll") for (int t = threadIdx.x >> 4; t < (L_); t += kFftThreads >> 4) \
        for (int l = threadIdx.x & 15; l < (nl_); l += 16)
// the same without unrolling, for loop bodies too heavy to replicate
#define BUNDLE_LOOP_ROLLED(t, l, L_, nl_)                                       \
    _Pragma("unroll 1") for (int t = threadIdx.x >> 4; t < (L_); t += kFftThreads >> 4) \
        for (int l = threadIdx.x & 15; l < (nl_); l += 16)
// line-major loops for the z passes: lines by warp, points by lane
#define LINE_LOOP(line, t, nlines_, len_)                                       \
    for (int line = threadIdx.x >> 5; line < (nlines_); line += kFftThreads >> 5) \
        _Pragma("unroll") for (int t = threadIdx.x & 31; t < (len_); t += 32)

// ------------------------------------------------------------------ z forward (R2C)
// Sum of the tile patches covering mesh point (x, y, z) (the fold of the
// atomics-free spread) in a fixed order: the two x slots, two y slots and two
// z slots give at most eight independent loads, empty slots contributing 0.
template <typename R>
__device__ __forceinline__ R fold_point(const Geo& g, const PatchSrc<R>& ps, int4 cx, int4 cy, int z) {
    const int4 cz = __ldg(&ps.cov2[2 * ps.nmax + z]);
    const int tx[2] = {cx.x, cx.z}, ox[2] = {cx.y, cx.w};
    const int ty[2] = {cy.x, cy.z}, oy[2] = {cy.y, cy.w};
    const int tz[2] = {cz.x, cz.z}, oz[2] = {cz.y, cz.w};
    R sum = R(0);
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                if (tx[a] >= 0 && ty[b] >= 0 && tz[c] >= 0) {
                    const int tile = (tx[a] * g.nt[1] + ty[b]) * g.nt[2] + tz[c];
                    sum += ps.patch[(size_t)tile * ps.psz + (ox[a] * g.E[1] + oy[b]) * g.Pz + oz[c]];
                }
            }
    return sum;
}

template <typename R, typename Eng>
__global__ void __launch_bounds__(kFftThreads)
k_fft_z_r2c(Geo g, Eng eng, const R* __restrict__ in, typename CT<R>::C* __restrict__ out, int rows, int pairs,
            PatchSrc<R> ps) {
    pdl_enter();
    typedef typename CT<R>::C C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // lines interleaved in shared memory: point t of line p at a[t * pairs + p]
    // (pairs odd, so that a run of t is conflict-free; lanes walk the lines
    // in the FFT stages)
    const int Nz = eng.len(), Hz = g.Hz, PL = pairs;
    C* a = reinterpret_cast<C*>(smem_raw);
    C* b = a + pairs * Nz;
    const int pair0 = blockIdx.x * pairs;
    const int npairs_total = (rows + 1) / 2;
    const int np = min(pairs, npairs_total - pair0);
    if (ps.patch) {
        const int4 empty = make_int4(-1, 0, -1, 0);
        for (int p = threadIdx.x >> 5; p < np; p += kFftThreads >> 5) {
            const int r0 = 2 * (pair0 + p), r1 = r0 + 1;
            const int x0 = r0 / g.N[1], y0 = r0 - x0 * g.N[1];
            const int4 cx0 = __ldg(&ps.cov2[x0]), cy0 = __ldg(&ps.cov2[ps.nmax + y0]);
            int4 cx1 = empty, cy1 = empty;
            if (r1 < rows) {
                const int x1 = r1 / g.N[1], y1 = r1 - x1 * g.N[1];
                cx1 = __ldg(&ps.cov2[x1]);
                cy1 = __ldg(&ps.cov2[ps.nmax + y1]);
            }
#pragma unroll 2
            for (int t = threadIdx.x & 31; t < Nz; t += 32) {
                const R va = fold_point(g, ps, cx0, cy0, t);
                const R vb = fold_point(g, ps, cx1, cy1, t);  // empty slots give 0
                a[t * PL + p] = CT<R>::mk(va, vb);
            }
        }
    } else {
        LINE_LOOP(p, t, np, Nz) {
            const int r0 = 2 * (pair0 + p), r1 = r0 + 1;
            const R va = in[(int64_t)r0 * Nz + t];
            const R vb = r1 < rows ? in[(int64_t)r1 * Nz + t] : R(0);
            a[t * PL + p] = CT<R>::mk(va, vb);
        }
    }
    __syncthreads();
    C* res = eng.template run<-1, true>(a, b, np, 1, PL);
    LINE_LOOP(p, k, np, Hz) {
        const int r0 = 2 * (pair0 + p), r1 = r0 + 1;
        const C z = res[k * PL + p];
        const C zc = cconj(res[(k == 0 ? 0 : Nz - k) * PL + p]);
        const C x0 = cscale(cadd(z, zc), R(0.5));
        const C d = csub(z, zc);  // = 2 i X1
        out[(int64_t)r0 * Hz + k] = x0;
        if (r1 < rows) out[(int64_t)r1 * Hz + k] = CT<R>::mk(R(0.5) * d.y, R(-0.5) * d.x);
    }
}

template <typename T>
cudaError_t launch_fft_z_r2c(cudaStream_t s, const Geo& g, const Radix& rz, const typename Cx<T>::t* tw,
                             const T* in, typename Cx<T>::t* out, const PatchSrc<T>& ps) {
    const int rows = g.N[0] * g.N[1];
    // up to 15 row pairs (an odd count) per block, within 32 KB of shared memory
    int pairs = (int)((32 * 1024) / (2 * g.N[2] * sizeof(typename Cx<T>::t)));
    pairs = pairs < 1 ? 1 : (pairs > 15 ? 15 : pairs);
    pairs |= 1;
    const int npairs = (rows + 1) / 2;
    const size_t smem = 2ull * pairs * g.N[2] * sizeof(typename Cx<T>::t);
    return with_engine<T>(rz, tw, [&](auto eng) {
        auto kern = k_fft_z_r2c<T, decltype(eng)>;
        cudaError_t e = set_smem(kern, smem);
        if (e != cudaSuccess) return e;
        return launch_k(kern, dim3((npairs + pairs - 1) / pairs), dim3(kFftThreads), smem, s, g, eng, in, out, rows,
                        pairs, ps);
    });
}

// ------------------------------------------------------------------ strided-line C2C
// axis 1: lines along y (outer index x); axis 0: lines along x (outer index y).
// Four resident blocks (64 registers): with the lines per block chosen for it,
// the strided passes run in one round of blocks at the workload sizes.
template <typename R, typename Eng, int SIGN>
__global__ void __launch_bounds__(kFftThreads, 4)
k_fft_bundle(Geo g, int axis, LineBlocks lb, Eng eng, typename CT<R>::C* __restrict__ data) {
    pdl_enter();
    typedef typename CT<R>::C C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Hz = g.Hz, L = eng.len(), B = lb.B;
    const int64_t es = axis == 1 ? (int64_t)Hz : (int64_t)g.N[1] * Hz;  // along the line
    const int64_t os = axis == 1 ? (int64_t)g.N[1] * Hz : (int64_t)Hz;  // between outer rows
    const int64_t nlines = (int64_t)(axis == 1 ? g.N[0] : g.N[1]) * Hz;
    const int64_t f0 = (int64_t)blockIdx.x * B;
    const int nl = (int)min((int64_t)B, nlines - f0);
    const int l = threadIdx.x & 15;  // this thread's line (B <= 16)
    const int64_t fl = f0 + l;
    const int64_t loff = (fl / Hz) * os + fl % Hz;
    C* a = reinterpret_cast<C*>(smem_raw);
    C* b = a + L * B;
    if (l < nl) {
#pragma unroll
        for (int t = threadIdx.x >> 4; t < L; t += kFftThreads >> 4) a[t * B + l] = data[loff + t * es];
    }
    __syncthreads();
    C* res = eng.template run<SIGN, true>(a, b, nl, 1, B);
    if (l < nl) {
#pragma unroll
        for (int t = threadIdx.x >> 4; t < L; t += kFftThreads >> 4) data[loff + t * es] = res[t * B + l];
    }
}

template <typename T>
cudaError_t launch_fft_bundle(cudaStream_t s, const Geo& g, int axis, int sign, const Radix& r, const LineBlocks& lb,
                              const typename Cx<T>::t* tw, typename Cx<T>::t* data) {
    const size_t smem = 2ull * r.L * lb.B * sizeof(typename Cx<T>::t);
    return with_engine<T>(r, tw, [&](auto eng) {
        auto kern = sign < 0 ? k_fft_bundle<T, decltype(eng), -1> : k_fft_bundle<T, decltype(eng), 1>;
        cudaError_t e = set_smem(kern, smem);
        if (e != cudaSuccess) return e;
        return launch_k(kern, dim3(lb.nblk), dim3(kFftThreads), smem, s, g, axis, lb, eng, data);
    });
}

// a / b for the virial coefficient: in FP32 the 2-ulp hardware quotient (the
// coefficient enters sums that are accurate to ~1e-7 anyway), in FP64 exact
__device__ __forceinline__ float div_approx(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double div_approx(double a, double b) { return a / b; }

// ------------------------------------------------------------------ x + influence
//
// Per block: B consecutive lines along x, numbered y Hz + kz.
//   1. forward FFT along x  -> rho_hat(k) up to the 1/h^3 factor;
//   2. per mode: G, the energy term e = w G |rho_hat|^2 V/(2 N^2) and the virial
//      terms e (delta_ab - 2 (1 + k^2/(4 beta^2)) k_a k_b / k^2), summed plainly
//      over a thread's Nx/16 modes (a relative error of at most Nx/16 roundings
//      of that short sum), then reduced across threads and blocks with
//      compensated (TwoSum) pairs;
//   3. P = G rho_hat / (N h^3) and -i kx' P (kx' = 0 on the Nyquist index);
//   4. inverse FFT along x of both; P -> S (in place), -i kx' P -> Bx.
// The last block to finish sums the per-block partials (TwoSum in the mesh
// precision, hi + lo in FP64 at the end) in a fixed order.
//
// Half-spectrum weights: w = 1 on the kz = 0 plane (and kz = Nz/2 for even Nz),
// 2 elsewhere, standing for the mirror mode -k.  For the off-diagonal virial a
// mirrored mode whose x (or y) index is the Nyquist index keeps that component's
// sign (the index maps to itself, m = +N/2), so a product k_a k_b survives the
// pairing only when both or neither of its components flip sign.
// (h, l) += (h2, l2) with the rounding error of h + h2 carried into l
template <typename R>
__device__ __forceinline__ void two_sum_pair(R& h, R& l, R h2, R l2) {
    R s = h + h2;
    R bp = s - h;
    R err = (h - (s - bp)) + (h2 - bp);
    h = s;
    l = l + l2 + err;
}

template <typename R, typename Eng>
__global__ void __launch_bounds__(kFftThreads, 4)
k_fft_x_influence(Geo g, LineBlocks lb, Eng eng, const R* __restrict__ G, R beta, R e_scale, R c_field,
                  typename CT<R>::C* __restrict__ S, typename CT<R>::C* __restrict__ Bx, R* __restrict__ partial,
                  unsigned int* __restrict__ counter, double prefactor, double* __restrict__ energy,
                  double* __restrict__ virial) {
    pdl_enter();
    typedef typename CT<R>::C C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ R red[kFftThreads / 32][14];
    __shared__ bool is_last;
    const int Nx = eng.len(), Ny = g.N[1], Nz = g.N[2], Hz = g.Hz, B = lb.B;
    // lines along x, numbered f = y Hz + kz: a block's B lines are consecutive in memory
    const int64_t es = (int64_t)Ny * Hz;
    const int64_t f0 = (int64_t)blockIdx.x * B;
    const int nl = (int)min((int64_t)B, es - f0);
    const int lt = threadIdx.x & 15;  // this thread's line (B <= 16)
    const int yl = (int)((f0 + lt) / Hz), kzl = (int)((f0 + lt) - (int64_t)yl * Hz);
    // three line buffers; each transform returns the one holding its result
    // and the others are reused as they free up
    C* a0 = reinterpret_cast<C*>(smem_raw);
    C* a1 = a0 + Nx * B;
    C* b0 = a1 + Nx * B;
    C* base = S + f0;
    BUNDLE_LOOP(t, l, Nx, nl) a0[t * B + l] = base[t * es + l];
    // with a compile-time length of whole 16-row passes, each thread's G values
    // are fetched now so that their latency hides behind the forward FFT
    constexpr bool kPre = Eng::kLen > 0 && Eng::kLen % (kFftThreads / 16) == 0;
    constexpr int NG = kPre ? Eng::kLen / (kFftThreads / 16) : 1;
    R gpre[NG];
    if constexpr (kPre) {
#pragma unroll
        for (int i = 0; i < NG; ++i) {
            const int t = (threadIdx.x >> 4) + i * (kFftThreads / 16);
            gpre[i] = lt < nl ? __ldg(&G[(int64_t)t * es + f0 + lt]) : R(0);
        }
    }
    __syncthreads();
    C* rh = eng.template run<-1, true>(a0, a1, nl, 1, B);
    C* pbuf = (rh == a0) ? a1 : a0;  // free partner of the result buffer

    const int my = yl <= Ny / 2 ? yl : yl - Ny;
    const R ky = kfac<R>(g, 1) * my;
    const bool nyq_y = (Ny % 2 == 0) && (yl == Ny / 2);
    const R inv4b2 = R(1) / (R(4) * beta * beta);
    R acc[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) acc[q] = R(0);
    const int kz = kzl;
    const R kzv = kfac<R>(g, 2) * kz;
    const bool plane1 = (kz == 0) || ((Nz % 2 == 0) && (kz == Nz / 2));
    const R w = plane1 ? R(1) : R(2);
    auto mode = [&](int t, R gk) {  // mode (t, line lt): energy and virial terms, P and -i kx' P
        const int mx = t <= Nx / 2 ? t : t - Nx;
        const R kx = kfac<R>(g, 0) * mx;
        const bool nyq_x = (Nx % 2 == 0) && (t == Nx / 2);
        const C v = rh[t * B + lt];
        const R k2 = kx * kx + ky * ky + kzv * kzv;
        if (k2 > R(0)) {
            const R e = w * e_scale * gk * (v.x * v.x + v.y * v.y);
            const R c = div_approx(R(2) * (R(1) + k2 * inv4b2), k2);
            const R fxy = (plane1 || (nyq_x == nyq_y)) ? R(1) : R(0);
            const R fxz = (plane1 || !nyq_x) ? R(1) : R(0);
            const R fyz = (plane1 || !nyq_y) ? R(1) : R(0);
            acc[0] += e;
            acc[1] += e * (R(1) - c * kx * kx);
            acc[2] += e * (R(1) - c * ky * ky);
            acc[3] += e * (R(1) - c * kzv * kzv);
            acc[4] -= e * c * kx * ky * fxy;
            acc[5] -= e * c * kx * kzv * fxz;
            acc[6] -= e * c * ky * kzv * fyz;
        }
        const C P = cscale(v, gk * c_field);
        const R kxd = nyq_x ? R(0) : kx;
        pbuf[t * B + lt] = P;
        b0[t * B + lt] = CT<R>::mk(kxd * P.y, -kxd * P.x);  // -i kx' P
    };
    if (lt < nl) {
        if constexpr (kPre) {
#pragma unroll
            for (int i = 0; i < NG; ++i) mode((threadIdx.x >> 4) + i * (kFftThreads / 16), gpre[i]);
        } else {
#pragma unroll 1
            for (int t = threadIdx.x >> 4; t < Nx; t += kFftThreads >> 4) mode(t, G[(int64_t)t * es + f0 + lt]);
        }
    }
    __syncthreads();
    C* rA = eng.template run<1, true>(pbuf, rh, nl, 1, B);  // rho_hat is no longer needed: scratch
    C* fr = (rA == pbuf) ? rh : pbuf;
    C* rB = eng.template run<1, true>(b0, fr, nl, 1, B);
    C* obx = Bx + f0;
    BUNDLE_LOOP(t, l, Nx, nl) {
        base[t * es + l] = rA[t * B + l];
        obx[t * es + l] = rB[t * B + l];
    }

    // block reduction of the 7 compensated sums: (hi, lo) pairs combined with TwoSum
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        R h = acc[q], lo = R(0);
        for (int off = 16; off > 0; off >>= 1) {
            const R h2 = __shfl_down_sync(0xffffffffu, h, off);
            const R l2 = __shfl_down_sync(0xffffffffu, lo, off);
            two_sum_pair(h, lo, h2, l2);
        }
        if (lane == 0) { red[warp][2 * q] = h; red[warp][2 * q + 1] = lo; }
    }
    __syncthreads();
    if (threadIdx.x < 7) {
        const int q = threadIdx.x;
        R h = red[0][2 * q], lo = red[0][2 * q + 1];
        for (int w = 1; w < kFftThreads / 32; ++w) two_sum_pair(h, lo, red[w][2 * q], red[w][2 * q + 1]);
        partial[(int64_t)blockIdx.x * 14 + 2 * q] = h;
        partial[(int64_t)blockIdx.x * 14 + 2 * q + 1] = lo;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int done = atomicAdd(counter, 1u);
        is_last = (done == gridDim.x - 1);
    }
    __syncthreads();
    if (is_last) {
        __threadfence();
        if (warp < 7) {  // warp q sums quantity q over all blocks, then the FP64 final sum
            const int q = warp;
            R h = R(0), lo = R(0);
            for (unsigned int b = lane; b < gridDim.x; b += 32) {
                two_sum_pair(h, lo, __ldcg(&partial[(int64_t)b * 14 + 2 * q]),
                             __ldcg(&partial[(int64_t)b * 14 + 2 * q + 1]));
            }
            for (int off = 16; off > 0; off >>= 1) {
                const R h2 = __shfl_down_sync(0xffffffffu, h, off);
                const R l2 = __shfl_down_sync(0xffffffffu, lo, off);
                two_sum_pair(h, lo, h2, l2);
            }
            if (lane == 0) {
                const double sum = ((double)h + (double)lo) * prefactor;
                if (q == 0) energy[0] = sum;
                else virial[q - 1] = sum;
            }
        }
        if (threadIdx.x == 0) *counter = 0u;
    }
}

int x_influence_blocks(const LineBlocks& lb) { return lb.nblk; }

template <typename T>
cudaError_t launch_fft_x_influence(cudaStream_t s, const Geo& g, const Radix& rx, const LineBlocks& lb,
                                   const typename Cx<T>::t* tw, const T* G, double beta, double e_scale,
                                   double c_field, typename Cx<T>::t* S, typename Cx<T>::t* Bx, T* partial,
                                   unsigned int* counter, double prefactor, double* energy, double* virial) {
    const size_t smem = 3ull * g.N[0] * lb.B * sizeof(typename Cx<T>::t);
    return with_engine<T>(rx, tw, [&](auto eng) {
        auto kern = k_fft_x_influence<T, decltype(eng)>;
        cudaError_t e = set_smem(kern, smem);
        if (e != cudaSuccess) return e;
        return launch_k(kern, dim3(x_influence_blocks(lb)), dim3(kFftThreads), smem, s, g, lb, eng, G, (T)beta,
                        (T)e_scale, (T)c_field, S, Bx, partial, counter, prefactor, energy, virial);
    });
}

// ------------------------------------------------------------------ y inverse, three outputs
// C = IFFT_y(A), D = IFFT_y(-i ky' A), Ex' = IFFT_y(Bx); C overwrites A, Ex' overwrites Bx.
template <typename R, typename Eng>
__global__ void __launch_bounds__(kFftThreads, 4)
k_fft_y_inverse3(Geo g, LineBlocks lb, Eng eng, typename CT<R>::C* __restrict__ A, typename CT<R>::C* __restrict__ Bx,
                 typename CT<R>::C* __restrict__ D) {
    pdl_enter();
    typedef typename CT<R>::C C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Ny = eng.len(), Hz = g.Hz, B = lb.B;
    // lines along y, numbered f = x Hz + kz; line f starts at x Ny Hz + kz
    const int64_t f0 = (int64_t)blockIdx.x * B;
    const int nl = (int)min((int64_t)B, (int64_t)g.N[0] * Hz - f0);
    const int64_t fl = f0 + (threadIdx.x & 15);  // this thread's line (B <= 16)
    const int64_t loff = (fl / Hz) * ((int64_t)Ny * Hz) + fl % Hz;
    // four line buffers: the three inputs and a scratch that rotates, each
    // transform leaving its result in one of the two it used
    const int sz = Ny * B;
    C* p0 = reinterpret_cast<C*>(smem_raw);
    C* p1 = p0 + sz;
    C* p2 = p1 + sz;
    C* scr = p2 + sz;
    BUNDLE_LOOP(t, l, Ny, nl) {
        const C va = A[loff + (int64_t)t * Hz];
        const int my = t <= Ny / 2 ? t : t - Ny;
        const R kyd = ((Ny % 2 == 0) && (t == Ny / 2)) ? R(0) : kfac<R>(g, 1) * my;
        p0[t * B + l] = va;
        p1[t * B + l] = CT<R>::mk(kyd * va.y, -kyd * va.x);
        p2[t * B + l] = Bx[loff + (int64_t)t * Hz];
    }
    __syncthreads();
    C* rC = eng.template run<1, true>(p0, scr, nl, 1, B);
    if (rC == scr) scr = p0;
    C* rD = eng.template run<1, true>(p1, scr, nl, 1, B);
    if (rD == scr) scr = p1;
    C* rE = eng.template run<1, true>(p2, scr, nl, 1, B);
    BUNDLE_LOOP(t, l, Ny, nl) {
        A[loff + (int64_t)t * Hz] = rC[t * B + l];
        D[loff + (int64_t)t * Hz] = rD[t * B + l];
        Bx[loff + (int64_t)t * Hz] = rE[t * B + l];
    }
}

template <typename T>
cudaError_t launch_fft_y_inverse3(cudaStream_t s, const Geo& g, const Radix& ry, const LineBlocks& lb,
                                  const typename Cx<T>::t* tw, typename Cx<T>::t* A, typename Cx<T>::t* Bx,
                                  typename Cx<T>::t* D) {
    const size_t smem = 4ull * g.N[1] * lb.B * sizeof(typename Cx<T>::t);
    return with_engine<T>(ry, tw, [&](auto eng) {
        auto kern = k_fft_y_inverse3<T, decltype(eng)>;
        cudaError_t e = set_smem(kern, smem);
        if (e != cudaSuccess) return e;
        return launch_k(kern, dim3(lb.nblk), dim3(kFftThreads), smem, s, g, lb, eng, A, Bx, D);
    });
}

// ------------------------------------------------------------------ z inverse (C2R)
struct ZOut {
    const void* src[4];
    void* out[4];
    int mulkz[4];
    int nf;
    FieldLayout fl;
};

// element f of a 4-entry kernel-parameter array, by selects (a dynamic index
// would copy the whole parameter struct to local memory)
template <typename X>
__device__ __forceinline__ X pick4(const X (&a)[4], int f) {
    return f == 0 ? a[0] : f == 1 ? a[1] : f == 2 ? a[2] : a[3];
}

template <typename R, typename Eng>
__global__ void __launch_bounds__(kFftThreads, 6)  // six resident blocks: two rounds instead of three
k_fft_z_c2r(Geo g, Eng eng, ZOut zo, int rows, int pairs) {
    pdl_enter();
    typedef typename CT<R>::C C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // lines interleaved in shared memory: point t of line L at a[t * PL + L],
    // PL odd (a run of t is conflict-free); lanes walk the lines in the stages
    const int Nz = eng.len(), Hz = g.Hz;
    const int nf = zo.nf;
    const int PL = (nf * pairs) | 1;
    C* a = reinterpret_cast<C*>(smem_raw);
    C* b = a + PL * Nz;
    const int pair0 = blockIdx.x * pairs;
    const int npairs_total = (rows + 1) / 2;
    const int np = min(pairs, npairs_total - pair0);
    const int nlines = nf * np;
    const bool even = (Nz % 2) == 0;
    LINE_LOOP(line, t, nlines, Nz) {
        const int f = line / np, p = line - f * np;
        const int r0 = 2 * (pair0 + p), r1 = r0 + 1;
        const C* src = reinterpret_cast<const C*>(pick4(zo.src, f));
        const int mulkz = pick4(zo.mulkz, f);
        // Hermitian extension: t < Hz reads the half row, t >= Hz the conjugate of Nz - t
        const int kk = t < Hz ? t : Nz - t;
        const bool cj = t >= Hz;
        const bool realonly = (kk == 0) || (even && kk == Nz / 2);
        R kzd = R(0);
        if (mulkz && !(even && kk == Nz / 2)) kzd = kfac<R>(g, 2) * kk;
        C h0 = src[(int64_t)r0 * Hz + kk];
        C h1 = r1 < rows ? src[(int64_t)r1 * Hz + kk] : CT<R>::mk(R(0), R(0));
        if (mulkz) {  // -i kz' h
            h0 = CT<R>::mk(kzd * h0.y, -kzd * h0.x);
            h1 = CT<R>::mk(kzd * h1.y, -kzd * h1.x);
        }
        if (realonly) { h0.y = R(0); h1.y = R(0); }
        if (cj) { h0.y = -h0.y; h1.y = -h1.y; }
        a[t * PL + line] = CT<R>::mk(h0.x - h1.y, h0.y + h1.x);  // h0 + i h1
    }
    __syncthreads();
    C* res = eng.template run<1, true>(a, b, nlines, 1, PL);
    if (!zo.fl.padded) {
        LINE_LOOP(line, t, nlines, Nz) {
            const int f = line / np, p = line - f * np;
            const int r0 = 2 * (pair0 + p), r1 = r0 + 1;
            R* out = reinterpret_cast<R*>(pick4(zo.out, f));
            const C z = res[t * PL + line];
            out[(int64_t)r0 * Nz + t] = z.x;
            if (r1 < rows) out[(int64_t)r1 * Nz + t] = z.y;
        }
        return;
    }
    // padded: the fields of a point are interleaved (E_x, E_y, E_z, 0) and
    // stored with one vector store, the potential (a fourth output) goes to
    // its own padded mesh; every output row also lands on its
    // periodic ghost images, and each row is extended by p - 1 ghost points
    // along z.  One warp per output row, lanes along z.
    const FieldLayout& fl = zo.fl;
    const int Ny = g.N[1], kmin = g.kmin;
    const int zlen = Nz + g.order - 1;
    typedef typename CT<R>::C4 V4;
    V4* out = reinterpret_cast<V4*>(zo.out[0]);
    R* phi = nf == 4 ? reinterpret_cast<R*>(zo.out[3]) : nullptr;  // padded potential, one value a point
    for (int pr = threadIdx.x >> 5; pr < 2 * np; pr += kFftThreads >> 5) {
        const int p = pr >> 1, half = pr & 1;
        const int r = 2 * (pair0 + p) + half;
        if (r >= rows) continue;
        const int x = r / Ny, y = r - x * Ny;
        const int px0 = x - kmin, py0 = y - kmin;
        // at most one ghost image per axis (Xp < 2 Nx)
        const int Nx = g.N[0];
        const int pxg = px0 + Nx < fl.Xp ? px0 + Nx : (px0 - Nx >= 0 ? px0 - Nx : -1);
        const int pyg = py0 + Ny < fl.Yp ? py0 + Ny : (py0 - Ny >= 0 ? py0 - Ny : -1);
        const int64_t r00 = ((int64_t)px0 * fl.Yp + py0) * fl.Zp;  // first point of each image row
        const int64_t r10 = pxg >= 0 ? ((int64_t)pxg * fl.Yp + py0) * fl.Zp : -1;
        const int64_t r01 = pyg >= 0 ? ((int64_t)px0 * fl.Yp + pyg) * fl.Zp : -1;
        const int64_t r11 = (pxg >= 0 && pyg >= 0) ? ((int64_t)pxg * fl.Yp + pyg) * fl.Zp : -1;
        for (int pz = threadIdx.x & 31; pz < zlen; pz += 32) {
            int zz = pz + kmin;
            zz += zz < 0 ? Nz : 0;
            zz -= zz >= Nz ? Nz : 0;
            const C* rz = res + zz * PL + p;  // field f of this pair at rz[f * np]
            R v[4];
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                const C zv = f < nf ? rz[f * np] : CT<R>::mk(R(0), R(0));
                v[f] = half ? zv.y : zv.x;
            }
            const V4 w = CT<R>::mk4(v[0], v[1], v[2], R(0));
            out[r00 + pz] = w;
            if (r10 >= 0) out[r10 + pz] = w;
            if (r01 >= 0) out[r01 + pz] = w;
            if (r11 >= 0) out[r11 + pz] = w;
            if (phi) {
                phi[r00 + pz] = v[3];
                if (r10 >= 0) phi[r10 + pz] = v[3];
                if (r01 >= 0) phi[r01 + pz] = v[3];
                if (r11 >= 0) phi[r11 + pz] = v[3];
            }
        }
    }
}

template <typename T>
cudaError_t launch_fft_z_c2r(cudaStream_t s, const Geo& g, const Radix& rz, const typename Cx<T>::t* tw, int nf,
                             const typename Cx<T>::t* const* src, const int* mulkz, T* const* out,
                             const FieldLayout& fl) {
    ZOut zo;
    zo.nf = nf;
    zo.fl = fl;
    for (int f = 0; f < 4; ++f) {
        zo.src[f] = f < nf ? src[f] : nullptr;
        zo.out[f] = f < nf ? out[f] : nullptr;
        zo.mulkz[f] = f < nf ? mulkz[f] : 0;
    }
    const int rows = g.N[0] * g.N[1];
    // at most 16 lines (nf fields x pairs) per block, the 16 lanes of a group
    // each taking one line in the FFT stages
    int pairs = 16 / nf;
    if (pairs < 1) pairs = 1;
    const int npairs = (rows + 1) / 2;
    const size_t smem = 2ull * ((nf * pairs) | 1) * g.N[2] * sizeof(typename Cx<T>::t);
    return with_engine<T>(rz, tw, [&](auto eng) {
        auto kern = k_fft_z_c2r<T, decltype(eng)>;
        cudaError_t e = set_smem(kern, smem);
        if (e != cudaSuccess) return e;
        return launch_k(kern, dim3((npairs + pairs - 1) / pairs), dim3(kFftThreads), smem, s, g, eng, zo, rows, pairs);
    });
}

// B for one pass: the fewest rounds of resident blocks, then the fewest
// blocks on the busiest SM (a block costs about the same for any B <= 16:
// its lanes are laid out for 16 lines), then the larger B.
template <typename K>
static LineBlocks pick_line_blocks(K kern, size_t bytes_per_line, int64_t lines, int nsm) {
    int maxB = 16;
    while (maxB > 1 && bytes_per_line * maxB > 227 * 1024) --maxB;
    LineBlocks best{1, (int)lines};
    int64_t best_rounds = -1, best_busy = 0;
    if (set_smem(kern, bytes_per_line * maxB) != cudaSuccess) {
        cudaGetLastError();
        return best;
    }
    for (int B = 1; B <= maxB; ++B) {
        int per = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kFftThreads, bytes_per_line * B) !=
                cudaSuccess ||
            per < 1) {
            cudaGetLastError();
            continue;
        }
        const int64_t blocks = (lines + B - 1) / B;
        const int64_t rounds = (blocks + (int64_t)per * nsm - 1) / ((int64_t)per * nsm);
        const int64_t busy = (blocks + nsm - 1) / nsm;
        if (best_rounds < 0 || rounds < best_rounds || (rounds == best_rounds && busy <= best_busy)) {
            best_rounds = rounds;
            best_busy = busy;
            best = LineBlocks{B, (int)blocks};
        }
    }
    return best;
}

template <typename T>
cudaError_t choose_line_blocks(const Geo& g, const Radix rad[3], int nsm, LineBlocks lb[4]) {
    typedef typename Cx<T>::t C;
    const int64_t Hz = g.Hz;
    cudaError_t e = with_engine<T>(rad[1], nullptr, [&](auto eng) {
        lb[LB_Y] = pick_line_blocks(k_fft_bundle<T, decltype(eng), -1>, 2 * sizeof(C) * rad[1].L, g.N[0] * Hz, nsm);
        lb[LB_Y_INVERSE3] =
            pick_line_blocks(k_fft_y_inverse3<T, decltype(eng)>, 4 * sizeof(C) * rad[1].L, g.N[0] * Hz, nsm);
        return cudaSuccess;
    });
    if (e != cudaSuccess) return e;
    return with_engine<T>(rad[0], nullptr, [&](auto eng) {
        lb[LB_X_INFLUENCE] =
            pick_line_blocks(k_fft_x_influence<T, decltype(eng)>, 3 * sizeof(C) * rad[0].L, g.N[1] * Hz, nsm);
        lb[LB_X] = pick_line_blocks(k_fft_bundle<T, decltype(eng), 1>, 2 * sizeof(C) * rad[0].L, g.N[1] * Hz, nsm);
        return cudaSuccess;
    });
}

#define PPPM_INST_FFT(T)                                                                                           \
    template cudaError_t launch_fft_z_r2c<T>(cudaStream_t, const Geo&, const Radix&, const Cx<T>::t*, const T*,    \
                                             Cx<T>::t*, const PatchSrc<T>&);                                       \
    template cudaError_t choose_line_blocks<T>(const Geo&, const Radix*, int, LineBlocks*);                      \
    template cudaError_t launch_fft_bundle<T>(cudaStream_t, const Geo&, int, int, const Radix&, const LineBlocks&, \
                                              const Cx<T>::t*, Cx<T>::t*);                                         \
    template cudaError_t launch_fft_x_influence<T>(cudaStream_t, const Geo&, const Radix&, const LineBlocks&,      \
                                                   const Cx<T>::t*, const T*, double, double, double, Cx<T>::t*,   \
                                                   Cx<T>::t*, T*, unsigned int*, double, double*, double*);        \
    template cudaError_t launch_fft_y_inverse3<T>(cudaStream_t, const Geo&, const Radix&, const LineBlocks&,       \
                                                  const Cx<T>::t*, Cx<T>::t*, Cx<T>::t*, Cx<T>::t*);               \
    template cudaError_t launch_fft_z_c2r<T>(cudaStream_t, const Geo&, const Radix&, const Cx<T>::t*, int,         \
                                             const Cx<T>::t* const*, const int*, T* const*, const FieldLayout&);
PPPM_INST_FFT(float)
PPPM_INST_FFT(double)

}  // namespace pppm
