/* A plain C99 caller of the library: one SPH step of a small rotating patch
 * on host arrays through sph_step_host. Compiled and linked by the CPU test
 * suite (which does not run it); on a machine with a GPU it runs as is:
 *   cc -std=c99 -I include tests/c_abi_example.c -L<dir of libsph.so> -lsph -o example
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "sph.h"

int main(void)
{
    const int side = 16;
    const int64_t n = (int64_t)side * side * side;
    const double dx = 1.0 / side, omega = 5.0;
    double *buf = (double *)calloc((size_t)(16 * n + 2), sizeof(double));
    if (!buf) return 1;
    sph_particles P = {0};
    double **f[16] = {&P.x, &P.y, &P.z, &P.vx, &P.vy, &P.vz, &P.m, &P.h,
                      &P.u, &P.rho, &P.p, &P.c, &P.ax, &P.ay, &P.az, &P.du};
    for (int k = 0; k < 16; ++k) *f[k] = buf + (size_t)k * n;
    P.n = n;
    P.time = buf + 16 * n;
    P.dt = buf + 16 * n + 1;
    for (int64_t q = 0; q < n; ++q) {  /* a jitter-free lattice in [-0.5, 0.5]^3 */
        P.x[q] = -0.5 + (q % side + 0.5) * dx;
        P.y[q] = -0.5 + ((q / side) % side + 0.5) * dx;
        P.z[q] = -0.5 + (q / (side * side) + 0.5) * dx;
        P.vx[q] = omega * P.y[q];
        P.vy[q] = -omega * P.x[q];
        P.m[q] = 1000.0 * dx * dx * dx;
        P.h[q] = 1.4395 * dx;
    }
    sph_params prm = {0};
    prm.eos = 0;
    prm.n_target = 100;
    prm.n_tol = 5;
    prm.max_h_iter = 64;
    prm.periodic_z = 1;
    prm.rho0 = 1000.0;
    prm.c0 = 50.0;
    prm.gamma = 5.0 / 3.0;
    prm.alpha = 1.0;
    prm.beta = 2.0;
    prm.eta2 = 0.01;
    prm.cfl = 0.3;
    prm.lz = 1.0;
    prm.sinc_n = 5;
    sph_ctx *ctx = NULL;
    sph_status st = sph_ctx_create(&ctx, n, 120 * n, 0);
    if (st == SPH_OK) st = sph_step_host(ctx, &prm, &P, 1, NULL);
    if (st == SPH_OK) st = sph_sync(ctx, NULL);
    if (st != SPH_OK && st != SPH_E_HNOCONV) {
        fprintf(stderr, "status %d: %s\n", (int)st, ctx ? sph_last_error(ctx) : "no context");
        sph_ctx_destroy(ctx);
        free(buf);
        return 2;
    }
    printf("%s: n=%lld dt=%.6e rho[0]=%.6f\n", sph_version(), (long long)n, *P.dt, P.rho[0]);
    sph_ctx_destroy(ctx);
    free(buf);
    return 0;
}
