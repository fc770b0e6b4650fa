/*
 * Direct-sum oracle for the Gaussian-charge long-range energy of DPLR.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file;
 * only the tests, the smoke check and the CPU-baseline leg of the benchmark do.
 * It shares no code with the CUDA implementation.
 *
 * Everything is plain FP64 with loops written straight from the formulas.
 *
 *   egt_direct      E_Gt of Eq. DPLR:EGt with S(m) of Eq. DPLR:Sm (Section 2.1),
 *                   its forces -dE/dr_j (the E_Gt terms of Eq. DPLR:F_inter) and
 *                   its virial Pi_ab = -dE/d(eps_ab) under affine strain.
 *   ewald_real      the real-space (erfc) half of the classical point-charge
 *                   Ewald sum; with egt_direct and the self term it gives the
 *                   full Ewald energy used by the Madelung pin.
 *   erf_shell_sum   1/2 sum_{cells |n|<=R} sum_{i,j}' q_i q_j erf(beta r)/r, the
 *                   brute-force real-space form of E_Gt (up to the self and the
 *                   surface-dipole terms), summed over whole image cells.
 *
 * Conventions: orthorhombic box L[3]; m = (n1/Lx, n2/Ly, n3/Lz); beta is an
 * inverse length (each site is a Gaussian whose pair interaction is
 * erf(beta r)/r); the cut keeps m with pi^2 m^2 / beta^2 <= cut (the
 * "m <= L" of Eq. DPLR:EGt).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* Half space of m vectors: n1 > 0, or n1 == 0 && n2 > 0, or n1 == n2 == 0 && n3 > 0. */
static int in_half_space(int n1, int n2, int n3) {
    if (n1 != 0) return n1 > 0;
    if (n2 != 0) return n2 > 0;
    return n3 > 0;
}

/*
 * E   = 1/(2 pi V) sum_{m != 0} A(m) |S(m)|^2,  A(m) = exp(-pi^2 m^2/beta^2)/m^2
 * F_j = -(2 q_j / V) sum_{m != 0} A(m) m Im(conj(S(m)) e^{-2 pi i m.r_j})
 * Pi_ab = sum_{m != 0} e(m) (delta_ab - 2 (1 + pi^2 m^2/beta^2) m_a m_b / m^2)
 * The sum runs over the half space and doubles each term (the summands are
 * even in m).  Virial order: xx yy zz xy xz yz.
 * Returns the number of m vectors in the half space that were kept.
 */
long egt_direct(int n, const double *pos, const double *q, const double *box,
                double beta, double cut, double *energy, double *forces, double *virial) {
    const double V = box[0] * box[1] * box[2];
    int nmax[3];
    for (int d = 0; d < 3; ++d) nmax[d] = (int)floor(sqrt(cut) * beta * box[d] / M_PI) + 1;

    /* enumerate the kept half-space vectors */
    long cap = (long)(2 * nmax[0] + 1) * (2 * nmax[1] + 1) * (2 * nmax[2] + 1) / 2 + 1;
    int *mv = (int *)malloc(sizeof(int) * 3 * cap);
    long nm = 0;
    for (int n1 = -nmax[0]; n1 <= nmax[0]; ++n1)
        for (int n2 = -nmax[1]; n2 <= nmax[1]; ++n2)
            for (int n3 = -nmax[2]; n3 <= nmax[2]; ++n3) {
                if (!in_half_space(n1, n2, n3)) continue;
                double mx = n1 / box[0], my = n2 / box[1], mz = n3 / box[2];
                double m2 = mx * mx + my * my + mz * mz;
                if (M_PI * M_PI * m2 / (beta * beta) > cut) continue;
                mv[3 * nm] = n1; mv[3 * nm + 1] = n2; mv[3 * nm + 2] = n3;
                ++nm;
            }

    /* per-site, per-axis phase tables e^{-2 pi i n_d r_d / L_d}, n_d in [-nmax, nmax];
       e^{-2 pi i m.r} is their product over the three axes. */
    double *cre[3], *cim[3];
    for (int d = 0; d < 3; ++d) {
        int w = 2 * nmax[d] + 1;
        cre[d] = (double *)malloc(sizeof(double) * (size_t)n * w);
        cim[d] = (double *)malloc(sizeof(double) * (size_t)n * w);
#pragma omp parallel for schedule(static)
        for (int j = 0; j < n; ++j)
            for (int k = -nmax[d]; k <= nmax[d]; ++k) {
                double ph = -2.0 * M_PI * k * pos[3 * j + d] / box[d];
                cre[d][(size_t)j * w + k + nmax[d]] = cos(ph);
                cim[d][(size_t)j * w + k + nmax[d]] = sin(ph);
            }
    }
#define PHASE(j, n1, n2, n3, re, im)                                                     \
    do {                                                                                 \
        size_t i0 = (size_t)(j) * (2 * nmax[0] + 1) + (n1) + nmax[0];                    \
        size_t i1 = (size_t)(j) * (2 * nmax[1] + 1) + (n2) + nmax[1];                    \
        size_t i2 = (size_t)(j) * (2 * nmax[2] + 1) + (n3) + nmax[2];                    \
        double ar = cre[0][i0], ai = cim[0][i0], br = cre[1][i1], bi = cim[1][i1];       \
        double cr = cre[2][i2], ci = cim[2][i2];                                         \
        double abr = ar * br - ai * bi, abi = ar * bi + ai * br;                         \
        re = abr * cr - abi * ci;                                                        \
        im = abr * ci + abi * cr;                                                        \
    } while (0)

    double *Sre = (double *)malloc(sizeof(double) * (nm ? nm : 1));
    double *Sim = (double *)malloc(sizeof(double) * (nm ? nm : 1));
    double *Am = (double *)malloc(sizeof(double) * (nm ? nm : 1));
    /* structure factor S(m) = sum_j q_j e^{-2 pi i m.r_j}  (Eq. DPLR:Sm) */
#pragma omp parallel for schedule(dynamic, 64)
    for (long t = 0; t < nm; ++t) {
        int n1 = mv[3 * t], n2 = mv[3 * t + 1], n3 = mv[3 * t + 2];
        double sr = 0.0, si = 0.0;
        for (int j = 0; j < n; ++j) {
            double er, ei;
            PHASE(j, n1, n2, n3, er, ei);
            sr += q[j] * er;
            si += q[j] * ei;
        }
        Sre[t] = sr;
        Sim[t] = si;
        double mx = n1 / box[0], my = n2 / box[1], mz = n3 / box[2];
        double m2 = mx * mx + my * my + mz * mz;
        Am[t] = exp(-M_PI * M_PI * m2 / (beta * beta)) / m2;
    }

    /* energy and virial: serial sums in a fixed order */
    double E = 0.0, P[6] = {0, 0, 0, 0, 0, 0};
    for (long t = 0; t < nm; ++t) {
        double mx = mv[3 * t] / box[0], my = mv[3 * t + 1] / box[1], mz = mv[3 * t + 2] / box[2];
        double m2 = mx * mx + my * my + mz * mz;
        double e = 2.0 * Am[t] * (Sre[t] * Sre[t] + Sim[t] * Sim[t]) / (2.0 * M_PI * V);
        double c = 2.0 * (1.0 + M_PI * M_PI * m2 / (beta * beta)) / m2;
        E += e;
        P[0] += e * (1.0 - c * mx * mx);
        P[1] += e * (1.0 - c * my * my);
        P[2] += e * (1.0 - c * mz * mz);
        P[3] += e * (-c * mx * my);
        P[4] += e * (-c * mx * mz);
        P[5] += e * (-c * my * mz);
    }
    *energy = E;
    for (int a = 0; a < 6; ++a) virial[a] = P[a];

    /* forces */
    if (forces) {
#pragma omp parallel for schedule(static)
        for (int j = 0; j < n; ++j) {
            double fx = 0.0, fy = 0.0, fz = 0.0;
            for (long t = 0; t < nm; ++t) {
                int n1 = mv[3 * t], n2 = mv[3 * t + 1], n3 = mv[3 * t + 2];
                double er, ei;
                PHASE(j, n1, n2, n3, er, ei);
                /* Im(conj(S) e) = Sre*ei - Sim*er */
                double im = Sre[t] * ei - Sim[t] * er;
                double w = 2.0 * Am[t] * im; /* x2: both half spaces */
                fx += w * (n1 / box[0]);
                fy += w * (n2 / box[1]);
                fz += w * (n3 / box[2]);
            }
            double pre = -2.0 * q[j] / V;
            forces[3 * j] = pre * fx;
            forces[3 * j + 1] = pre * fy;
            forces[3 * j + 2] = pre * fz;
        }
    }
#undef PHASE
    for (int d = 0; d < 3; ++d) { free(cre[d]); free(cim[d]); }
    free(Sre); free(Sim); free(Am); free(mv);
    return nm;
}

/*
 * Real-space part of the point-charge Ewald sum:
 *   1/2 sum_{i,j} sum_{images n} ' q_i q_j erfc(alpha |r_ij + n L|) / |r_ij + n L|
 * over all image vectors with |r| < rcut (the prime drops i == j at n = 0).
 */
double ewald_real(int n, const double *pos, const double *q, const double *box,
                  double alpha, double rcut) {
    int nimg[3];
    for (int d = 0; d < 3; ++d) nimg[d] = (int)ceil(rcut / box[d]) + 1;
    double *per_i = (double *)calloc(n, sizeof(double));
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int j = 0; j < n; ++j)
            for (int a = -nimg[0]; a <= nimg[0]; ++a)
                for (int b = -nimg[1]; b <= nimg[1]; ++b)
                    for (int c = -nimg[2]; c <= nimg[2]; ++c) {
                        if (i == j && a == 0 && b == 0 && c == 0) continue;
                        double dx = pos[3 * j] - pos[3 * i] + a * box[0];
                        double dy = pos[3 * j + 1] - pos[3 * i + 1] + b * box[1];
                        double dz = pos[3 * j + 2] - pos[3 * i + 2] + c * box[2];
                        double r = sqrt(dx * dx + dy * dy + dz * dz);
                        if (r >= rcut) continue;
                        s += q[i] * q[j] * erfc(alpha * r) / r;
                    }
        per_i[i] = s;
    }
    double E = 0.0;
    for (int i = 0; i < n; ++i) E += per_i[i];
    free(per_i);
    return 0.5 * E;
}

/*
 * Brute-force real-space sum of Gaussian-Gaussian interactions over whole image
 * cells, shifted by s = (a Lx, b Ly, c Lz) for integers a, b, c with |s| <= R
 * (a Cartesian sphere), counted once per cell:
 *   out = 1/2 sum_{|s|<=R} sum_{i,j} ' q_i q_j erf(beta |r_j - r_i + s|) / |...|
 * The cell loop is a spherical summation order, so for a neutral cell the limit
 * R -> infinity equals the tin-foil result plus 2 pi |M|^2 / (3V).
 */
double erf_shell_sum(int n, const double *pos, const double *q, const double *box,
                     double beta, double R) {
    int nr[3];
    for (int d = 0; d < 3; ++d) nr[d] = (int)floor(R / box[d]);
    long w0 = 2 * nr[0] + 1, w1 = 2 * nr[1] + 1, w2 = 2 * nr[2] + 1;
    long ncell = w0 * w1 * w2;
    double *per_cell = (double *)calloc(ncell, sizeof(double));
#pragma omp parallel for schedule(dynamic, 16)
    for (long t = 0; t < ncell; ++t) {
        int a = (int)(t / (w1 * w2)) - nr[0], b = (int)((t / w2) % w1) - nr[1], c = (int)(t % w2) - nr[2];
        double sx = a * box[0], sy = b * box[1], sz = c * box[2];
        if (sx * sx + sy * sy + sz * sz > R * R) continue;
        double s = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                if (i == j && a == 0 && b == 0 && c == 0) continue;
                double dx = pos[3 * j] - pos[3 * i] + sx;
                double dy = pos[3 * j + 1] - pos[3 * i + 1] + sy;
                double dz = pos[3 * j + 2] - pos[3 * i + 2] + sz;
                double r = sqrt(dx * dx + dy * dy + dz * dz);
                s += q[i] * q[j] * erf(beta * r) / r;
            }
        per_cell[t] = s;
    }
    double E = 0.0;
    for (long t = 0; t < ncell; ++t) E += per_cell[t];
    free(per_cell);
    return 0.5 * E;
}
