/*
 * Serving through the C ABI alone: several dose requests on one resident
 * phantom and table set, submitted together with gdpm_request_submit and
 * collected with gdpm_request_poll as each finishes.  The phantom is the
 * 64^3 water phantom with a 2 cm bone slab of slab_dose.c; the requests are
 * 6 MV-like point-source fields of different sizes and history counts, the
 * small ones (narrow fields, 2e5 histories) beside the large ones (wide
 * fields, 2e6).  Prints, per request, its field, histories, sigma/Dmax, the
 * energy balance and the time from submission to completion.
 *
 * Build (from the repository root, after the library is built):
 *   gcc -O2 -I include examples/serve_requests.c -L paper_1107_3355_gb300 -lgdpm \
 *       -Wl,-rpath,$PWD/paper_1107_3355_gb300 -o serve_requests
 * Run:
 *   ./serve_requests [requests]        (default 8)
 */
#define _POSIX_C_SOURCE 199309L
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#include "gdpm.h"

#define CHECK(call)                                                                   \
    do {                                                                              \
        int rc_ = (call);                                                             \
        if (rc_ != GDPM_OK) {                                                         \
            fprintf(stderr, "%s failed: %s (%d)\n", #call, gdpm_strerror(rc_), rc_);  \
            return 1;                                                                 \
        }                                                                             \
    } while (0)

static double now_ms(void) {
    struct timespec t;
    clock_gettime(CLOCK_MONOTONIC, &t);
    return 1e3 * (double)t.tv_sec + 1e-6 * (double)t.tv_nsec;
}

static void element(gdpm_material_desc* m, int z, double a, double w) {
    m->Z[m->n_elements] = z;
    m->A[m->n_elements] = a;
    m->mass_fraction[m->n_elements] = w;
    m->n_elements++;
}

int main(int argc, char** argv) {
    const int n_req = argc > 1 ? atoi(argv[1]) : 8;
    if (n_req < 1 || n_req > 64) return 1;
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
    double* dose = malloc(V * sizeof(double));
    double* sigma = malloc(V * sizeof(double));
    if (!mat || !rho || !dose || !sigma) return 1;
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

    gdpm_ctx* ctx = NULL;
    gdpm_phantom* ph = NULL;
    gdpm_tables* tb = NULL;
    CHECK(gdpm_context_create(&ctx, 0, NULL, 12345));
    CHECK(gdpm_tables_build(ctx, mats, 2, 0.005, 6.5, 512, 0.05, 0.2, 0.2, 0, &tb));
    CHECK(gdpm_phantom_create(ctx, nx, ny, nz, d, d, d, mat, rho, &ph));

    /* the requests: point source at SSD 100 cm, square fields of 2 to 10 cm */
    uint64_t* id = calloc((size_t)n_req, sizeof(uint64_t));
    double* t_sub = calloc((size_t)n_req, sizeof(double));
    int* done = calloc((size_t)n_req, sizeof(int));
    if (!id || !t_sub || !done) return 1;
    const double X = nx * d, Y = ny * d;
    for (int r = 0; r < n_req; ++r) {
        const int small = r % 2 == 0;
        gdpm_request_desc q;
        memset(&q, 0, sizeof(q));
        q.phantom = ph;
        q.tables = tb;
        q.source.particle = GDPM_PHOTON;
        q.source.geometry = GDPM_GEO_POINT_FIELD;
        q.source.origin[0] = X / 2; q.source.origin[1] = Y / 2; q.source.origin[2] = -100.0;
        q.source.direction[2] = 1.0;
        q.source.center[0] = X / 2; q.source.center[1] = Y / 2;
        q.source.axis_u[0] = 1.0; q.source.axis_v[1] = 1.0;
        q.source.half_u = q.source.half_v = small ? 1.0 : 1.0 + (double)(r % 5);
        q.source.n_bins = 24;
        q.source.bin_edges = edges;
        q.source.bin_weights = weights;
        q.source.annihilation = 1;
        q.n_histories = small ? 200000 : 2000000;
        q.n_batches = 10;
        t_sub[r] = now_ms();
        CHECK(gdpm_request_submit(ctx, &q, &id[r]));
    }

    /* collect each request as it finishes */
    printf("request  field (cm)  histories  sigma/Dmax  energy balance  latency (ms)\n");
    int left = n_req, failed = 0;
    const struct timespec pause = {0, 200000};   /* 0.2 ms between polling rounds */
    while (left > 0) {
        for (int r = 0; r < n_req; ++r) {
            if (done[r]) continue;
            gdpm_stats st;
            int fin = 0;
            const int rc = gdpm_request_poll(ctx, id[r], &fin, dose, sigma, &st);
            if (!fin) continue;
            done[r] = 1;
            --left;
            if (rc != GDPM_OK) {
                fprintf(stderr, "request %d failed: %s (%d)\n", r, gdpm_strerror(rc), rc);
                failed = 1;
                continue;
            }
            const double bal = (st.deposited + st.escaped + st.discarded - st.source_energy) / st.source_energy;
            const double field = r % 2 == 0 ? 2.0 : 2.0 * (1.0 + (double)(r % 5));
            printf("%7d  %10.1f  %9lld  %8.3f %%  %14.2e  %12.1f\n", r, field, (long long)st.n_primary,
                   100.0 * st.sigma_over_dmax, bal, now_ms() - t_sub[r]);
            if (!(fabs(bal) < 1e-5)) failed = 1;
        }
        if (left > 0) nanosleep(&pause, NULL);
    }

    gdpm_phantom_destroy(ph);
    gdpm_tables_destroy(tb);
    gdpm_context_destroy(ctx);
    free(mat); free(rho); free(dose); free(sigma); free(id); free(t_sub); free(done);
    return failed;
}
