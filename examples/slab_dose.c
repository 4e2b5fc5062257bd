/*
 * A dose calculation through the C ABI alone (no Python, no PyTorch):
 * a 6 MV-like point source (SSD 100 cm, 10 x 10 cm field) on a 32 cm water
 * phantom with a 2 cm bone slab at 10-12 cm depth, 64^3 voxels of 0.5 cm.
 * Prints the depth dose on the central axis, sigma/Dmax (Sec. 3.1) and the
 * energy ledger.
 *
 * Build (from the repository root, after the library is built):
 *   gcc -O2 -I include examples/slab_dose.c -L paper_1107_3355_gb300 -lgdpm \
 *       -Wl,-rpath,$PWD/paper_1107_3355_gb300 -o slab_dose
 * Run:
 *   ./slab_dose [histories]            (default 1e7)
 */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "gdpm.h"

#define CHECK(call)                                                                   \
    do {                                                                              \
        int rc_ = (call);                                                             \
        if (rc_ != GDPM_OK) {                                                         \
            fprintf(stderr, "%s failed: %s (%d)\n", #call, gdpm_strerror(rc_), rc_);  \
            return 1;                                                                 \
        }                                                                             \
    } while (0)

static void element(gdpm_material_desc* m, int z, double a, double w) {
    m->Z[m->n_elements] = z;
    m->A[m->n_elements] = a;
    m->mass_fraction[m->n_elements] = w;
    m->n_elements++;
}

int main(int argc, char** argv) {
    const unsigned long long n_hist = argc > 1 ? strtoull(argv[1], NULL, 10) : 10000000ull;
    const int nx = 64, ny = 64, nz = 64;
    const float d = 0.5f;
    const size_t V = (size_t)nx * ny * nz;

    /* materials: water and ICRU-44-like cortical bone, by mass fraction */
    gdpm_material_desc mats[2];
    memset(mats, 0, sizeof(mats));
    element(&mats[0], 1, 1.008, 0.111894);
    element(&mats[0], 8, 15.999, 0.888106);
    mats[0].mean_excitation_MeV = 75.0e-6;
    const int bz[9] = {1, 6, 7, 8, 11, 12, 15, 16, 20};
    const double ba[9] = {1.008, 12.011, 14.007, 15.999, 22.990, 24.305, 30.974, 32.06, 40.078};
    const double bw[9] = {0.034, 0.155, 0.042, 0.435, 0.001, 0.002, 0.103, 0.003, 0.225};
    for (int i = 0; i < 9; ++i) element(&mats[1], bz[i], ba[i], bw[i]);
    mats[1].mean_excitation_MeV = 106.4e-6;

    /* phantom: water, bone between 10 and 12 cm depth */
    unsigned char* mat = malloc(V);
    float* rho = malloc(V * sizeof(float));
    if (!mat || !rho) return 1;
    for (int iz = 0; iz < nz; ++iz) {
        const float zc = (iz + 0.5f) * d;
        const int bone = zc >= 10.f && zc < 12.f;
        for (size_t k = 0; k < (size_t)nx * ny; ++k) {
            mat[(size_t)iz * nx * ny + k] = (unsigned char)bone;
            rho[(size_t)iz * nx * ny + k] = bone ? 1.85f : 1.0f;
        }
    }

    /* a 6 MV-like spectrum: (E0 - k)/k in 24 intervals of 0.25 MeV above 0.25 MeV */
    double edges[25], weights[24];
    for (int b = 0; b <= 24; ++b) edges[b] = 0.25 * b;
    for (int b = 0; b < 24; ++b) {
        const double k = 0.5 * (edges[b] + edges[b + 1]);
        weights[b] = b == 0 ? 0.0 : (6.0 - k) / k;
    }
    gdpm_source_desc src;
    memset(&src, 0, sizeof(src));
    src.particle = GDPM_PHOTON;
    src.geometry = GDPM_GEO_POINT_FIELD;
    const double X = nx * d, Y = ny * d;
    src.origin[0] = X / 2; src.origin[1] = Y / 2; src.origin[2] = -100.0;
    src.direction[2] = 1.0;
    src.center[0] = X / 2; src.center[1] = Y / 2; src.center[2] = 0.0;
    src.axis_u[0] = 1.0; src.axis_v[1] = 1.0;
    src.half_u = 5.0; src.half_v = 5.0;
    src.n_bins = 24;
    src.bin_edges = edges;
    src.bin_weights = weights;
    src.annihilation = 1;

    gdpm_ctx* ctx = NULL;
    gdpm_phantom* ph = NULL;
    gdpm_tables* tb = NULL;
    CHECK(gdpm_context_create(&ctx, 0, NULL, 12345));
    CHECK(gdpm_tables_build(ctx, mats, 2, 0.005, 6.5, 512, 0.05, 0.2, 0.2, 0, &tb));
    CHECK(gdpm_phantom_create(ctx, nx, ny, nz, d, d, d, mat, rho, &ph));
    CHECK(gdpm_source_set(ctx, &src));

    double* dose = malloc(V * sizeof(double));
    double* sigma = malloc(V * sizeof(double));
    if (!dose || !sigma) return 1;
    gdpm_stats st;
    CHECK(gdpm_simulate(ctx, ph, tb, n_hist, 10, dose, sigma, &st));

    printf("histories %lld  transport %.1f ms  sigma/Dmax %.3f %%\n", (long long)st.n_primary,
           st.transport_ms, 100.0 * st.sigma_over_dmax);
    printf("energy: source %.6g  deposited %.6g  escaped %.6g  discarded %.6g  (MeV)\n",
           st.source_energy, st.deposited, st.escaped, st.discarded);
    printf("depth (cm)  dose (MeV/g per history)  sigma\n");
    const int cx = nx / 2, cy = ny / 2;
    for (int iz = 1; iz < nz; iz += 4) {
        const size_t v = (size_t)iz * nx * ny + (size_t)cy * nx + cx;
        printf("%6.2f      %.6e            %.2e\n", (iz + 0.5) * d, dose[v], sigma[v]);
    }
    const double bal = st.deposited + st.escaped + st.discarded - st.source_energy;
    printf("energy balance (relative) %.2e\n", bal / st.source_energy);

    gdpm_phantom_destroy(ph);
    gdpm_tables_destroy(tb);
    gdpm_context_destroy(ctx);
    free(mat); free(rho); free(dose); free(sigma);
    return 0;
}
