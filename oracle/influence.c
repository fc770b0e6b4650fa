/*
 * Optimal influence function of PPPM with ik differentiation (Hockney and
 * Eastwood), FP64, for the Gaussian reference interaction of Eq. DPLR:EGt.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  This is the same formula
 * as oracle/pppm.py:influence written as plain loops so that large meshes
 * finish in seconds; a test checks that the two agree.
 *
 *   G(k) = sum_{n in [-a,a]^3} (k . k_n / |k_n|^2) 4 pi exp(-|k_n|^2 / (4 beta^2)) U^2(k_n)
 *          / ( |k|^2 [ prod_d sum_{|n_d| <= nd} sinc^{2p}(k_{n,d} h_d / 2) ]^2 )
 *   k_d = 2 pi m_d / L_d, m_d = i_d if i_d <= N_d/2 else i_d - N_d,
 *   k_{n,d} = k_d + 2 pi n_d / h_d,  U(k) = prod_d sinc(k_d h_d / 2)^p,  G(0) = 0.
 * Output layout: G[(ix * Ny + iy) * Nz + iz], full spectrum.
 */
#include <math.h>
#include <stdlib.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

static double sinc(double x) { return x == 0.0 ? 1.0 : sin(x) / x; }

static double kvec(int i, int N, double L) {
    int m = (i <= N / 2) ? i : i - N;
    return 2.0 * M_PI * m / L;
}

void influence_ik(const double *box, const int *mesh, int p, double beta, int alias,
                  int denom_range, double *G) {
    const int Nx = mesh[0], Ny = mesh[1], Nz = mesh[2];
    const double h[3] = {box[0] / Nx, box[1] / Ny, box[2] / Nz};
    long total = (long)Nx * Ny * Nz;
#pragma omp parallel for schedule(static)
    for (long t = 0; t < total; ++t) {
        int ix = (int)(t / ((long)Ny * Nz)), iy = (int)((t / Nz) % Ny), iz = (int)(t % Nz);
        double k[3] = {kvec(ix, Nx, box[0]), kvec(iy, Ny, box[1]), kvec(iz, Nz, box[2])};
        double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        if (k2 == 0.0) { G[t] = 0.0; continue; }
        double den = 1.0;
        for (int d = 0; d < 3; ++d) {
            double s = 0.0;
            for (int nd = -denom_range; nd <= denom_range; ++nd)
                s += pow(sinc((k[d] + 2.0 * M_PI * nd / h[d]) * h[d] / 2.0), 2 * p);
            den *= s;
        }
        double num = 0.0;
        for (int nx = -alias; nx <= alias; ++nx)
            for (int ny = -alias; ny <= alias; ++ny)
                for (int nz = -alias; nz <= alias; ++nz) {
                    double kn[3] = {k[0] + 2.0 * M_PI * nx / h[0], k[1] + 2.0 * M_PI * ny / h[1],
                                    k[2] + 2.0 * M_PI * nz / h[2]};
                    double kn2 = kn[0] * kn[0] + kn[1] * kn[1] + kn[2] * kn[2];
                    double u = sinc(kn[0] * h[0] / 2.0) * sinc(kn[1] * h[1] / 2.0) * sinc(kn[2] * h[2] / 2.0);
                    double dot = k[0] * kn[0] + k[1] * kn[1] + k[2] * kn[2];
                    num += dot / kn2 * 4.0 * M_PI * exp(-kn2 / (4.0 * beta * beta)) * pow(u, 2 * p);
                }
        G[t] = num / (k2 * den * den);
    }
}
