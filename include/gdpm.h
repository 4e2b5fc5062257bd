/*
 * gdpm.h -- C ABI of the GB300 (sm_103a) gDPM dose engine.
 *
 * The engine computes radiotherapy dose by coupled photon/electron Monte
 * Carlo transport through a voxel phantom, following gDPM v2.0 (Jia et al.,
 * arXiv:1107.3355): Woodcock-tracked photons with Compton, photoelectric
 * and pair events; condensed-history electrons with CSDA energy loss,
 * discrete (hard) Moller and bremsstrahlung events and hinge multiple
 * scattering (Sec. 2.1); histories split into N_b batches whose spread
 * gives the per-voxel uncertainty (Sec. 2.2.1); cross sections tabulated
 * and linearly interpolated (Sec. 2.2.2); spectrum stratified into equal
 * energy intervals (Sec. 2.3.2); fluence-map beamlets (Sec. 2.3.1).
 *
 * Conventions for every entry point:
 *   - Return value: GDPM_OK (0) or a negative GDPM_E_* code.  No entry point
 *     aborts the process; a device-side fault condition (queue overflow,
 *     iteration cap) is reported as a status code, never by a trap.
 *   - Handles are opaque.  The library owns the device memory it allocates
 *     and frees it in the matching *_destroy call.
 *   - Caller buffers are owned by the caller and are only read or written
 *     during the call.  Unless stated otherwise an input array may live in
 *     host or device memory (the library asks the CUDA runtime which).
 *   - A context binds one CUDA device and one stream.  Calls on a context
 *     are not thread-safe, except gdpm_request_submit/gdpm_request_poll.
 *   - Units: MeV, cm, g/cm3.  Voxel (ix,iy,iz) has flat index
 *     ix + nx*(iy + ny*iz); the phantom spans [0,nx*dx]x[0,ny*dy]x[0,nz*dz].
 */
#ifndef GDPM_H
#define GDPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
#define GDPM_OK 0
#define GDPM_E_ARG (-1)            /* invalid argument or size */
#define GDPM_E_NOMEM (-2)          /* device allocation failed or refused */
#define GDPM_E_QUEUE_OVERFLOW (-3) /* a secondary-particle queue overflowed */
#define GDPM_E_TIMEOUT (-4)        /* a phase or iteration cap was reached */
#define GDPM_E_CUDA (-5)           /* a CUDA runtime call failed */
#define GDPM_E_STATE (-6)          /* call not valid in the current state */
#define GDPM_E_BUSY (-7)           /* request not admitted (memory or slots) */
#define GDPM_E_BOUNDS (-8)         /* checked build only: an index was out of range */

typedef struct gdpm_ctx gdpm_ctx;
typedef struct gdpm_phantom gdpm_phantom;
typedef struct gdpm_tables gdpm_tables;

#define GDPM_MAX_ELEMENTS 16
#define GDPM_MAX_MATERIALS 8
#define GDPM_MAX_BINS 256

/* Material by composition.  Cross sections are built per unit density and
 * scaled by each voxel's density (Sec. 2.1 materials "by mass"). */
typedef struct {
    int n_elements;
    int Z[GDPM_MAX_ELEMENTS];
    double A[GDPM_MAX_ELEMENTS];               /* g/mol */
    double mass_fraction[GDPM_MAX_ELEMENTS];   /* need not sum to 1; normalised */
    double mean_excitation_MeV;                /* Bethe I value */
} gdpm_material_desc;

enum { GDPM_PHOTON = 0, GDPM_ELECTRON = 1 };
enum { GDPM_GEO_PENCIL = 0, GDPM_GEO_POINT_FIELD = 1, GDPM_GEO_BEAMLETS = 2 };
/* Beamlet samplers of a fluence map (Sec. 2.3.1), all drawing beamlet I with
 * probability f_I / sum f over the beamlets of positive weight:
 *   GDPM_SAMPLE_CDF: the I with P(I) <= r < P(I+1) on the cumulative
 *     fluence (binary search; r is the primary's own uniform);
 *   GDPM_SAMPLE_ALIAS: Walker's alias method (table by Vose's procedure);
 *   GDPM_SAMPLE_METROPOLIS: the Metropolis chain of Algorithm A1 -- propose
 *     a uniform J, move there with probability min(1, f_J / f_Iprev).
 *     metropolis_chains C independent chains; history h is step h div C of
 *     chain h mod C, so results depend on the seed, not on scheduling.
 * Alias and Metropolis take their proposal and acceptance words from the
 * Philox block at counter (h, 0, 0, 0); chain c starts at a uniform index
 * from the block at (c, 0, 1, 0). */
enum { GDPM_SAMPLE_CDF = 0, GDPM_SAMPLE_ALIAS = 1, GDPM_SAMPLE_METROPOLIS = 2 };

/* Table/transport flags (gdpm_tables_build). */
#define GDPM_FLAG_COMPTON_ONLY 2   /* zero photoelectric and pair cross sections */
#define GDPM_FLAG_NO_HARD 4        /* no hard Moller/bremsstrahlung events */
#define GDPM_FLAG_SAUTER 8         /* photoelectrons leave at an angle from Sauter's K-shell
                                      distribution (physics variant; default: along the photon) */

/* Source description (Sec. 2.3): particle, energy spectrum, geometry.
 *   GDPM_GEO_PENCIL: all primaries start at `origin` along `direction`.
 *   GDPM_GEO_POINT_FIELD: point source at `origin`; each primary aims at a
 *     point uniform in the rectangle centre `center`, unit axes `axis_u`,
 *     `axis_v`, half widths `half_u`, `half_v`.
 *   GDPM_GEO_BEAMLETS: fluence map (Sec. 2.3.1); `beamlets` holds
 *     n_beamlets rows of 17 doubles: source(3) centre(3) axis_u(3) axis_v(3)
 *     u0 u1 v0 v1 (beamlet rectangle in the axis frame, cm) weight f_I.
 *     `beamlet_sampler` picks the sampler (GDPM_SAMPLE_*, default 0) and
 *     `metropolis_chains` the chain count C of the Metropolis sampler
 *     (0 means 4096; at most 1<<24).
 * Energy: n_bins intervals with edges bin_edges[0..n_bins] and relative
 * weights bin_weights[0..n_bins-1]; a monoenergetic source is one interval
 * with equal edges.  Histories of each batch are allotted to intervals by
 * weight (floor plus largest remainder) and their energies are uniform
 * within the interval (Sec. 2.3.2).  Host arrays; copied by the call. */
typedef struct {
    int particle;
    int geometry;
    double origin[3], direction[3];
    double center[3], axis_u[3], axis_v[3];
    double half_u, half_v;
    int n_bins;
    const double *bin_edges;
    const double *bin_weights;
    int n_beamlets;
    const double *beamlets;
    int annihilation;              /* 1: positrons end in two 0.511 MeV photons (Sec. 2.1) */
    int beamlet_sampler;           /* GDPM_SAMPLE_* (fluence maps only) */
    int metropolis_chains;         /* chains C of GDPM_SAMPLE_METROPOLIS; 0 = 4096 */
} gdpm_source_desc;

/* Run statistics: energy ledger (FP64, MeV) and exact integer counts. */
typedef struct {
    double source_energy, deposited, escaped, discarded;
    int64_t n_primary;
    int64_t ph_created, ph_terminated, ph_flights, ph_real, compton, photoelectric, pair;
    int64_t el_created, el_terminated, el_steps, moller, brems, annihilations;
    int64_t local_deposits;
    int64_t pushes[2], pops[2];    /* queue traffic: [0] photons, [1] electrons */
    int64_t phases, launches;
    double dmax, sigma_over_dmax;  /* Sec. 3.1 precision metric over D > 0.5 Dmax, among
                                      voxels denser than GDPM_PARAM_METRIC_MIN_DENSITY */
    double transport_ms;           /* device time of the transport + fold loop */
    int64_t crossings;             /* voxel boundaries crossed by electrons */
    /* with GDPM_PARAM_PROFILE: summed device time and launch count per kernel
     * kind: [0] photon phase, [1] electron phase, [2] batch fold,
     * [3] primaries (source kernel and Metropolis picks) */
    double kernel_ms[4];
    int64_t kernel_launches[4];
} gdpm_stats;

/* ------------------------------------------------------------------ context */

/* Create a context on CUDA device `device` issuing work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  `seed` keys the
 * Philox4x32-10 generator that stands in for the per-thread generator
 * states of Sec. 2.2.2: key = (seed lo 32 bits, seed hi 32 bits ^ request
 * id).  The context owns the device memory it allocates.
 * Errors: GDPM_E_ARG (bad device, NULL out), GDPM_E_CUDA. */
int gdpm_context_create(gdpm_ctx **out, int device, void *cuda_stream, uint64_t seed);
/* Destroy a context: stops its serving workers and frees its device memory.
 * Phantoms and tables made on it must be destroyed first.
 * Errors: GDPM_E_ARG (NULL). */
int gdpm_context_destroy(gdpm_ctx *ctx);

/* Tuning and run parameters of the transport loop of Sec. 2.2.1 (see
 * GDPM_PARAM_*; each states its range).  They change how the work is
 * launched, not what is computed.
 * Errors: GDPM_E_ARG (unknown parameter or value out of range). */
int gdpm_set_param(gdpm_ctx *ctx, int param, double value);
enum {
    GDPM_PARAM_QUEUE_CAPACITY = 1,   /* particles per queue buffer (0 = automatic), <= 2^31 */
    GDPM_PARAM_BLOCK_THREADS = 2,    /* threads per block of every transport phase kernel:
                                        64..256, multiple of 32; 0 (default): each kernel's
                                        own shape (256; 448 for resumable electron steps) */
    GDPM_PARAM_BLOCKS_PER_SM = 3,    /* persistent CTAs per SM (0 = occupancy) */
    GDPM_PARAM_TALLY_MODE = 4,       /* 0: FP64 atomics; 1: FP32 compensated hi/lo pair */
    GDPM_PARAM_SOURCE_CHUNK = 5,     /* max primaries per transport phase (0 = auto), <= 2^28 */
    GDPM_PARAM_MAX_PHASES = 6,       /* phase cap per batch -> GDPM_E_TIMEOUT */
    GDPM_PARAM_REQUEST_ID = 7,       /* xored into the Philox key high word */
    GDPM_PARAM_SPECULATIVE = 8,      /* phase pairs issued per host check (>=1) */
    GDPM_PARAM_PROFILE = 10,         /* 1: time every launch with CUDA events (stats kernel_ms) */
    GDPM_PARAM_OVERLAP_FOLD = 11,    /* 1 (default): fold batch b while batch b+1 runs */
    GDPM_PARAM_SERVE_SLOTS = 12,     /* requests run side by side by the serving loop (1..16) */
    GDPM_PARAM_SERVE_RESERVE_MB = 13,/* device memory left free when admitting a request */
    GDPM_PARAM_METRIC_MIN_DENSITY = 14,/* sigma/Dmax only over voxels at least this dense
                                          (g/cm3, default 0.05: excludes air) */
    GDPM_PARAM_BATCH_MODE = 15,      /* 0 auto, 1 batches one after another, 2 all batches side
                                        by side (one tally grid per batch, n_batches <= 128,
                                        phases shared by all batches: up to 32M primaries
                                        where their queues fit in a quarter of the device's
                                        memory, else 16M, 8M ...; at most 8M for requests
                                        served by gdpm_request_submit) */
    GDPM_PARAM_CONCURRENT_MAX_HIST = 16, /* auto: side by side when histories per batch <= this
                                            (default 4e9, no limit) ... */
    GDPM_PARAM_CONCURRENT_MAX_MB = 17,   /* ... and the per-batch grids fit in this (default 16384) */
    GDPM_PARAM_GRAPH = 18,           /* 1: batches side by side run their phases as one
                                        CUDA graph launch, a conditional WHILE node that repeats
                                        photon phase, electron phase and a control kernel on the
                                        device until nothing is left (no host checks); 0: the host
                                        loop (default).  Profiling (GDPM_PARAM_PROFILE) uses the
                                        host loop. */
    GDPM_PARAM_MAX_ITERS = 19,       /* loop trips a warp may take in one transport phase
                                        (1..2^31, default 2^22, far above real use).  A warp
                                        that reaches it abandons its particles and the call
                                        returns GDPM_E_TIMEOUT; the next call starts clean. */
    GDPM_PARAM_ELECTRON_WALK = 20,   /* electron phase form, same results either way: 1
                                        resumable steps, whose voxel walk takes at most 3 trips
                                        per loop iteration and resumes in the next, so a track
                                        with many voxel crossings does not hold its warp; 0 a
                                        whole condensed-history step per iteration; 2 (default)
                                        resumable where the phantom holds voxels below 0.05
                                        g/cm3 (air: electrons there take steps hundreds of
                                        voxels long), whole steps otherwise */
    GDPM_PARAM_SERVE_BIG_SLOTS = 21, /* serving slots for large requests, in arrival order
                                        (1..15, fewer than GDPM_PARAM_SERVE_SLOTS; default 1);
                                        the other slots serve small requests.  Set before the
                                        first gdpm_request_submit. */
    GDPM_PARAM_SERVE_SMALL_HIST = 22,/* requests of at most this many histories are small
                                        (default 1e6): they run on high-priority streams */
    GDPM_PARAM_SERVE_PHASE_CAP = 23, /* primaries per transport phase of a served request
                                        (0 = as gdpm_simulate, the default).  A persistent
                                        phase holds its SMs until it drains: shorter phases let
                                        small requests that arrive meanwhile start sooner, at
                                        some throughput of the large ones. */
    GDPM_PARAM_SERVE_SHARE = 24      /* eighths of the SMs (1..8, default 7) a large request's
                                        phases launch on while small requests run */
};

/* ------------------------------------------------------------------ inputs */

/* Upload a voxel phantom (Sec. 2.2.1 initialisation): `material` is nx*ny*nz
 * uint8 material indices into the table set, `density` nx*ny*nz float
 * densities in g/cm3 (> 0), both x fastest.  Host or device arrays; copied.
 * Errors: GDPM_E_ARG (non-positive sizes, nx|ny|nz > 1024, a density that is
 * zero, negative, NaN or infinite), GDPM_E_NOMEM. */
int gdpm_phantom_create(gdpm_ctx *ctx, int nx, int ny, int nz, float dx, float dy, float dz,
                        const uint8_t *material, const float *density, gdpm_phantom **out);
/* Release a phantom (Sec. 2.2.1) and its device memory; waits for work on
 * its context's stream.  Errors: GDPM_E_ARG (NULL). */
int gdpm_phantom_destroy(gdpm_phantom *ph);

/* Build the interpolation tables (Sec. 2.2.2) for n_mats materials on a
 * log-uniform energy grid of n_energy points in [e_min, e_max], on the
 * device in FP64 and stored as FP32: photon attenuation (Klein-Nishina,
 * Z^4/E^3 photoelectric, Bethe-Heitler-shaped pair), electron restricted
 * stopping power and CSDA range (Bethe + Moller + Kramers bremsstrahlung),
 * hard-event cross sections, the range inverse, and the screened-Rutherford
 * screening parameter.  The absorption energies are also the hard-event
 * thresholds (W_cc = eabs_electron, W_cb = eabs_photon).  `ms_loss` is the
 * CSDA energy fraction that limits one multiple-scattering step; `flags`
 * takes GDPM_FLAG_COMPTON_ONLY / GDPM_FLAG_NO_HARD / GDPM_FLAG_SAUTER.
 * Errors: GDPM_E_ARG (n_mats outside 1..8, n_energy < 16, bad energies). */
int gdpm_tables_build(gdpm_ctx *ctx, const gdpm_material_desc *mats, int n_mats,
                      double e_min, double e_max, int n_energy, double eabs_photon,
                      double eabs_electron, double ms_loss, int flags, gdpm_tables **out);
/* Release a table set (Sec. 2.2.2) and its device memory; waits for work on
 * its context's stream.  Errors: GDPM_E_ARG (NULL). */
int gdpm_tables_destroy(gdpm_tables *t);

/* Set the primary source (Sec. 2.3.1-2.3.3).  Copies everything it needs.
 * Errors: GDPM_E_ARG (n_bins outside 1..256, weights not positive in sum,
 * unknown geometry, empty beamlet list). */
int gdpm_source_set(gdpm_ctx *ctx, const gdpm_source_desc *src);

/* ------------------------------------------------------------------ compute */

/* Simulate n_histories primaries in n_batches equal batches (Sec. 2.2.1)
 * and return, per voxel, the mean dose and its standard error in MeV/g per
 * source history (Gy per history = value * 1.602176634e-10).  dose_out and
 * sigma_out hold nx*ny*nz doubles in host or device memory (either may be
 * NULL).  stats_out (host, may be NULL) receives the ledger and counts.
 * The call returns when the results are in place.
 * Errors: GDPM_E_ARG (n_batches < 2, n_histories < n_batches or >= 2^32,
 * material index beyond the table set, source energy outside the table
 * grid), GDPM_E_QUEUE_OVERFLOW, GDPM_E_TIMEOUT, GDPM_E_NOMEM, GDPM_E_CUDA. */
int gdpm_simulate(gdpm_ctx *ctx, gdpm_phantom *ph, gdpm_tables *tb, uint64_t n_histories,
                  int n_batches, double *dose_out, double *sigma_out, gdpm_stats *stats_out);

/* Run until the dose reaches a target precision (Sec. 3.1's metric:
 * sigma/Dmax averaged over the voxels with D > 0.5 Dmax, which Sec. 3.1 and
 * Sec. 3.2 bring below 1 %).  A pilot run of n_pilot histories measures
 * sigma/Dmax; since it falls as N^(-1/2), the next run takes
 * n (sigma/Dmax / target)^2 x 1.4 histories (x 1.05 after that first step:
 * a small pilot reads sigma/Dmax low, since noise inflates Dmax), and so on
 * (at most 8 runs, at most n_max histories in one run) until a run meets
 * the target.  A pilot of a few percent of the histories the target needs
 * usually reaches it in one more run.  Each
 * run is a complete gdpm_simulate in n_batches batches; the outputs and
 * stats_out are those of the last run, *n_total_out (may be NULL) the
 * histories of all runs together.  A run capped at n_max that misses the
 * target still returns GDPM_OK: compare stats_out->sigma_over_dmax with
 * the target.  dose_out / sigma_out as for gdpm_simulate (may be NULL).
 * Errors: GDPM_E_ARG (target <= 0, n_pilot < n_batches, n_max < n_pilot or
 * >= 2^32), GDPM_E_STATE (per-history records are set), and those of
 * gdpm_simulate. */
int gdpm_simulate_to_precision(gdpm_ctx *ctx, gdpm_phantom *ph, gdpm_tables *tb, double target,
                               uint64_t n_pilot, uint64_t n_max, int n_batches, double *dose_out,
                               double *sigma_out, gdpm_stats *stats_out, uint64_t *n_total_out);

/* Checkpoint / resume.  The state of a run is the per-voxel sums over its
 * finished batches, sum1 = sum_b x_b and sum2 = sum_b x_b^2 with x_b the
 * energy per history of batch b (Sec. 2.2.1), plus the index of the next
 * batch.  gdpm_simulate_part runs batches [first_batch, first_batch +
 * n_part) of the n_histories / n_batches calculation (at most 128 at a time)
 * and ADDS their x_b and x_b^2 into sum1, sum2 (nx*ny*nz doubles each, host
 * or device, caller-owned; zero them before the first part).  Histories
 * keep their ids in the whole calculation, so the parts can run in any
 * grouping, in separate processes, and the sums equal those of one
 * uninterrupted run up to the order of FP64 additions.  gdpm_finalize turns
 * the sums of all n_batches batches into dose and sigma (as gdpm_simulate,
 * MeV/g per history; host or device outputs, either may be NULL) and
 * reports Dmax and sigma/Dmax in stats_out.
 * Errors: as gdpm_simulate; GDPM_E_ARG for a batch range outside
 * [0, n_batches) or n_part > 128. */
int gdpm_simulate_part(gdpm_ctx *ctx, gdpm_phantom *ph, gdpm_tables *tb, uint64_t n_histories,
                       int n_batches, int first_batch, int n_part, double *sum1, double *sum2,
                       gdpm_stats *stats_out);
/* gdpm_finalize: the batch statistics of Sec. 2.2.1 Step 4 and the Sec. 3.1
 * metric from the sums above.  Errors: GDPM_E_ARG (NULL context, phantom or
 * sums, n_batches < 2), GDPM_E_NOMEM, GDPM_E_CUDA. */
int gdpm_finalize(gdpm_ctx *ctx, gdpm_phantom *ph, int n_batches, const double *sum1,
                  const double *sum2, double *dose_out, double *sigma_out, gdpm_stats *stats_out);

/* Beamlet dose matrix: every row k of the current source's fluence map
 * (GDPM_GEO_BEAMLETS; its weight is ignored) is a calculation of its own --
 * the beamlet's rectangle as the field of a point source, n_histories[k]
 * primaries in n_batches batches (Sec. 2.2.1, 2.3.1) -- and all of them run
 * through one sequence of transport phases, each with its own tally grids.
 * Beamlet k's histories have ids sum_{j<k} n_histories[j] + 0, 1, ..., so
 * its result equals gdpm_simulate of that beamlet alone with those history
 * ids.  dose_out (and sigma_out, which may be NULL) hold K x nx*ny*nz
 * doubles, beamlet-major, in MeV/g per history of that beamlet; host or
 * device memory.  n_batches >= 2 when sigma_out is given, else >= 1.  The
 * tally grids take K * n_batches * nx*ny*nz * 8 bytes of device memory.
 * stats_out sums the counts and ledger over all beamlets (no sigma/Dmax).
 * Errors: GDPM_E_ARG (source not a fluence map, K * n_batches > 32767, a
 * beamlet with fewer histories than batches, sum >= 2^32, energies outside
 * the tables), GDPM_E_STATE (no source), GDPM_E_NOMEM, GDPM_E_QUEUE_OVERFLOW,
 * GDPM_E_TIMEOUT, GDPM_E_CUDA. */
int gdpm_simulate_beamlets(gdpm_ctx *ctx, gdpm_phantom *ph, gdpm_tables *tb,
                           const uint64_t *n_histories, int n_batches, double *dose_out,
                           double *sigma_out, gdpm_stats *stats_out);

/* Launch configuration chosen by gdpm_autotune. */
typedef struct {
    int batch_mode;            /* GDPM_PARAM_BATCH_MODE value: 1 one after another, 2 side by side */
    uint32_t source_chunk;     /* GDPM_PARAM_SOURCE_CHUNK: primaries per transport phase */
    int speculative;           /* GDPM_PARAM_SPECULATIVE: phase pairs per host check */
    int candidates_tried;
    double histories_per_s;    /* of the best candidate (wall clock, whole call) */
    int electron_walk;         /* GDPM_PARAM_ELECTRON_WALK: 1 resumable steps, 0 whole steps */
    int block_threads;         /* GDPM_PARAM_BLOCK_THREADS of the transport kernels
                                  (0: each kernel's own shape) */
    uint32_t queue_capacity;   /* GDPM_PARAM_QUEUE_CAPACITY (0: 8 per primary of a phase + 65536) */
    int graph;                 /* GDPM_PARAM_GRAPH: 1 device-driven phase loop */
} gdpm_tune_result;

/* Autotuner for the launch configuration of the Sec. 2.2.1 transport loop:
 * run the calculation gdpm_simulate(ph, tb, n_histories, n_batches) with the
 * current source under candidate launch configurations until the wall-clock
 * budget is spent, keep the fastest, and set it on the context.  After one
 * untimed run (allocations), stage 1 tries every combination of batches side
 * by side (when their grids fit) or one after another, 1M / 4M primaries per
 * phase or the side-by-side default (8M or more), and 1 / 2 / 4 phase pairs
 * per host check.  Then, one dimension at a time from the best so far
 * (kept only when more than 1 % faster): the other electron phase form
 * (GDPM_PARAM_ELECTRON_WALK), blocks of 128 / 192 / 256 threads for every
 * phase kernel instead of each kernel's own shape, half the
 * default queue capacity (4 slots per primary of a phase + 65536; a
 * candidate whose queues overflow is skipped), and for batches side by side
 * the device-driven phase loop (GDPM_PARAM_GRAPH).  The primaries per phase
 * also set the default queue capacity (8 per primary + 65536).  Energy-bin
 * sorting of the queues is not a candidate: measured, it made the electron
 * phase 10 % slower, so the engine does not offer it.
 * Results do not depend on the configuration (per-history random streams),
 * only the time does.  `out` is a host struct.
 * Errors: those of gdpm_simulate; GDPM_E_ARG (budget_ms <= 0, NULL out). */
int gdpm_autotune(gdpm_ctx *ctx, gdpm_phantom *ph, gdpm_tables *tb, uint64_t n_histories,
                  int n_batches, double budget_ms, gdpm_tune_result *out);

/* Optional per-history records of the Sec. 2.2.1 transport, for the next
 * gdpm_simulate on this context:
 * rec (device, n*4 int32: real photon interactions, electron steps, hard
 * electron events, banked secondaries) and recd (device, n*2 doubles:
 * escaped energy, electron mass path in g/cm2), indexed by history id.
 * Pass NULL to switch off.  Errors: GDPM_E_ARG. */
int gdpm_set_history_records(gdpm_ctx *ctx, int32_t *rec, double *recd, uint64_t n);

/* ------------------------------------------------------------------ serving */

/* A dose request: one Sec. 2.2.1 calculation (source, history count and
 * batch count) on a phantom/table pair that stays resident.  Serving is not
 * in the paper: requests share the GPU and keep their own random streams.
 * Results are kept on the device until polled. */
typedef struct {
    gdpm_phantom *phantom;
    gdpm_tables *tables;
    gdpm_source_desc source;
    uint64_t n_histories;
    int n_batches;
    uint32_t stream_id;            /* Philox stream (xored into the key high word);
                                      0 = use the request id */
} gdpm_request_desc;

/* Queue a request (one Sec. 2.2.1 calculation); returns at once with its
 * id.  Requests arriving while
 * others run are admitted as slots and device memory free up and share the
 * device with them (continuous batching); each request keeps its own Philox
 * key (request id), so its result does not depend on what else runs.
 * Thread-safe.  Errors: GDPM_E_ARG, GDPM_E_BUSY (queue full). */
int gdpm_request_submit(gdpm_ctx *ctx, const gdpm_request_desc *req, uint64_t *req_id);

/* Poll a request: *done = 1 when finished, then copies its dose/sigma
 * (the batch statistics of Sec. 2.2.1 Step 4)
 * (host or device arrays, nx*ny*nz doubles, may be NULL) and stats, and
 * releases it.  *done = 0 while queued or running.  Thread-safe.
 * Errors: GDPM_E_ARG (unknown id), or the request's own failure code. */
int gdpm_request_poll(gdpm_ctx *ctx, uint64_t req_id, int *done, double *dose_out,
                      double *sigma_out, gdpm_stats *stats_out);

/* ------------------------------------------------------------------ checks */

/* Human-readable text for a status code (static storage). */
const char *gdpm_strerror(int code);

/* Philox4x32-10 (the generator that replaces Sec. 2.2.2's) on the device for
 * n counters (device arrays of 4*n uint32 each, in and out), key (k0, k1).
 * For bitwise comparison with other implementations.
 * Errors: GDPM_E_ARG (NULL or host arrays), GDPM_E_CUDA. */
int gdpm_debug_philox(gdpm_ctx *ctx, const uint32_t *ctr, uint32_t k0, uint32_t k1,
                      uint32_t *out, uint64_t n);

/* Draw n samples from one device-side interaction sampler with the same
 * random-number protocol as the transport (sample s uses history id s,
 * particle id 1, key (seed lo, seed hi)):
 *   kind 0 Klein-Nishina at energy a: out1 = E'/E, out2 = cos(theta)
 *   kind 1 Moller at T = a, W_cc = b: out1 = W/T, out2 = cos(theta_delta)
 *   kind 2 bremsstrahlung at T = a, W_cb = b: out1 = k
 *   kind 3 screened Rutherford with screening a: out1 = mu
 *   kind 4 isotropic: out1 = cos(theta), out2 = phi
 *   kind 5 Sauter photoelectron of kinetic energy a: out1 = cos(theta), out2 = phi
 * These are the interactions of Sec. 2.1 (photons: Compton; electrons: hard
 * Moller and bremsstrahlung events, multiple-scattering deflection; the
 * Sec. 4 photoelectron variant).
 * out1/out2: device arrays of n doubles (out2 may be NULL).
 * Errors: GDPM_E_ARG (unknown kind, host or NULL out1, parameters outside the
 * sampler's domain: a > 0; Moller a > 2b > 0; bremsstrahlung a > b > 0),
 * GDPM_E_CUDA. */
int gdpm_debug_sample(gdpm_ctx *ctx, int kind, double a, double b, uint64_t n,
                      uint64_t seed, double *out1, double *out2);

/* Rate of one hardware resource that the transport kernels use, measured by
 * a persistent grid (SM count x resident blocks of 256 threads) that does
 * nothing else.  The dose tally of Sec. 2.2.2 is a scattered atomic add into
 * the batch grid; the flights and deflections spend FP32, MUFU and (ledger,
 * fold) FP64 issue slots.
 *   GDPM_MB_RED_F64   FP64 atomic add of 1.0 into n_slots doubles of buf,
 *                     uniform random slots, old value unused
 *   GDPM_MB_RED_F32   the same with FP32 (n_slots floats)
 *   GDPM_MB_ATOM_F32  FP32 atomic add whose returned old value is used, as
 *                     in the compensated FP32 pair tally
 *   GDPM_MB_FFMA      FP32 fused multiply-adds, 8 chains per thread
 *   GDPM_MB_DFMA      FP64 fused multiply-adds
 *   GDPM_MB_MUFU_LG2  MUFU base-2 logarithms
 * buf: caller-owned device array (n_slots doubles or floats for the atomic
 * kinds; at least one float for the others, used as a sink).  One untimed
 * launch warms up, then the array is cleared and one launch of about n_ops
 * operations is timed with events on the context's stream, so after an
 * atomic kind the array's elements sum to *ops_done.
 * Out: *ops_done = operations the timed launch did (n_ops rounded up to whole
 * threads), *ms = its device time.  Errors: GDPM_E_ARG (bad kind, NULL or
 * host buf, n_slots outside [1, 2^32), n_ops 0), GDPM_E_CUDA. */
#define GDPM_MB_RED_F64 0
#define GDPM_MB_RED_F32 1
#define GDPM_MB_ATOM_F32 2
#define GDPM_MB_FFMA 3
#define GDPM_MB_DFMA 4
#define GDPM_MB_MUFU_LG2 5
int gdpm_microbench(gdpm_ctx *ctx, int kind, void *buf, uint64_t n_slots, uint64_t n_ops,
                    double *ops_done, double *ms);

/* Copy one FP32 table to a device buffer of doubles:
 *   0 mu_compton [m][i], 1 mu_compton + mu_photo, 2 total mu (cm2/g; the
 *   cumulative forms the transport stores and samples from), 3 CSDA range
 *   (g/cm2), 4 hard Moller, 5 hard bremsstrahlung (cm2/g), 6 energy grid (i),
 *   7 per-material X0 (g/cm2), 8 per-material hard-event majorant (cm2/g),
 *   9 ln A of the screened-Rutherford distribution at 1024 points
 *   ln G1 = ln 1e-10 + k (ln 0.999 - ln 1e-10) / 1023 (the same for every
 *   material set; a context computes it once).
 * These are the tables of Sec. 2.2.2 as the transport reads them.
 * *count receives the number of values written (out may be NULL to query).
 * Errors: GDPM_E_ARG (NULL table set or count, unknown kind), GDPM_E_CUDA. */
int gdpm_tables_export(gdpm_tables *t, int which, double *out, int64_t *count);

/* Generate the primaries of histories [first, first+n) of batch 0 of an
 * n_histories/n_batches run with the current source, as the transport does
 * (Sec. 2.3), without transporting them.  out (device, n*8 doubles per
 * primary: x y z u v w E entered) -- position is on the phantom surface
 * after entry; entered = 0 if the primary misses the phantom.
 * Errors: those of gdpm_simulate's argument checks; GDPM_E_ARG (host or NULL
 * out, first + n beyond the histories of batch 0). */
int gdpm_debug_sources(gdpm_ctx *ctx, gdpm_phantom *ph, gdpm_tables *tb, uint64_t n_histories,
                       int n_batches, uint64_t first, uint64_t n, double *out);

/* Beamlet picked for each history of [first, first+n) by the current
 * source's sampler (Sec. 2.3.1; the source must be a fluence map), written
 * as the beamlet's row in the map to the device array `out` (n int32).  The
 * Metropolis chains are run from their start up to history first+n-1.
 * Errors: GDPM_E_ARG (not a fluence map, host `out`, first+n > 2^32),
 * GDPM_E_STATE (no source set). */
int gdpm_debug_beamlets(gdpm_ctx *ctx, uint64_t first, uint64_t n, int32_t *out);

/* ------------------------------------------------------------------ no allocation */

/* gdpm_simulate_noalloc -- the same dose calculation as gdpm_simulate, for
 * small problems, without allocating any memory.  The paper has no
 * counterpart.  It exists for callers that cannot call cudaMalloc: host
 * applications that hand all device memory to their own allocator (a pool
 * sized at start-up, a planning system with a fixed memory budget) and
 * forbid libraries from allocating behind it.  The call synchronizes its
 * stream and stages small arrays through host memory before it returns, so
 * it is an ordinary blocking call.
 *
 * All work buffers (batch tally, batch sums, particle queues, counters,
 * source arrays, Woodcock majorant) come from one file-scope device array of
 * GDPM_NOALLOC_SCRATCH_BYTES (about 4.1 MB).  Every GPU that loads this
 * library holds that array until the process exits.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) for that
 * device.
 *
 * Limits (GDPM_E_ARG beyond them): nx*ny*nz <= GDPM_NOALLOC_MAX_VOXELS, at
 * most GDPM_NOALLOC_QUEUE_CAPACITY banked particles per queue fill (more is
 * reported as GDPM_E_QUEUE_OVERFLOW), n_batches*(n_bins+1) <=
 * GDPM_NOALLOC_MAX_PREFIX, n_beamlets <= GDPM_NOALLOC_MAX_BEAMLETS,
 * Metropolis chains <= GDPM_NOALLOC_MAX_CHAINS, table
 * grid <= 8192 energies.  dose_out and sigma_out must be device arrays (or
 * NULL); stats_out is a host struct (or NULL).  The phantom, tables and
 * source are the caller's existing handles on this context; the context's
 * per-history records and profiling are not used.  Results equal those of
 * gdpm_simulate with the same seed up to the summation order of the FP64
 * tallies.
 *
 * Every call on a device shares the one array, and it keeps the last call's
 * contents (the call clears what must start at zero).  Calls whose work
 * overlaps on the same GPU -- from two streams, two contexts or two threads
 * -- race on that array and corrupt each other's results: run them one after
 * another.
 * Errors: those of gdpm_simulate, and GDPM_E_ARG beyond the limits above. */
#define GDPM_NOALLOC_MAX_VOXELS 32768
#define GDPM_NOALLOC_QUEUE_CAPACITY 16384
#define GDPM_NOALLOC_MAX_PREFIX 65536
#define GDPM_NOALLOC_MAX_BEAMLETS 1024
#define GDPM_NOALLOC_MAX_CHAINS 65536
#define GDPM_NOALLOC_SCRATCH_BYTES 4098048
int gdpm_simulate_noalloc(gdpm_ctx *ctx, gdpm_phantom *ph, gdpm_tables *tb, uint64_t n_histories,
                          int n_batches, double *dose_out, double *sigma_out,
                          gdpm_stats *stats_out);

#ifdef __cplusplus
}
#endif
#endif /* GDPM_H */
