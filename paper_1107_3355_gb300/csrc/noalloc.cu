// gdpm_simulate_noalloc: the dose calculation of gdpm_simulate for small
// problems, for callers that must not allocate device memory -- a host
// application that hands the GPU's memory to its own allocator (a memory
// pool sized at start-up, an embedded planning system with a fixed budget)
// and forbids libraries from calling cudaMalloc behind its back.  The call
// synchronizes its stream and copies through host memory, so it is an
// ordinary blocking call.  Every work buffer (batch tally, batch sums,
// particle queues, counters, source arrays, majorant) is carved from one
// fixed-size array in device memory that exists for as long as the library
// is loaded; the caller passes the phantom, tables and output arrays.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.h"

namespace gdpm {
namespace {

constexpr size_t kNaMaxVoxels = GDPM_NOALLOC_MAX_VOXELS;
constexpr uint32_t kNaQueueCap = GDPM_NOALLOC_QUEUE_CAPACITY;
constexpr size_t kNaMaxPrefix = GDPM_NOALLOC_MAX_PREFIX;
constexpr int kNaMaxBeamlets = GDPM_NOALLOC_MAX_BEAMLETS;
constexpr uint32_t kNaMaxChains = GDPM_NOALLOC_MAX_CHAINS;
constexpr uint32_t kNaChunk = kNaQueueCap / 8;      // primaries per photon phase
constexpr int kNaMaxEnergy = 8192;
constexpr int kNaCtlRows = 1024;

// Byte offsets of the regions inside the static array (all 256-aligned).
constexpr size_t al(size_t b) { return (b + 255) & ~size_t(255); }
constexpr size_t kOffEdep = 0;
constexpr size_t kOffS1 = kOffEdep + al(kNaMaxVoxels * 8);
constexpr size_t kOffS2 = kOffS1 + al(kNaMaxVoxels * 8);
constexpr size_t kOffQ = kOffS2 + al(kNaMaxVoxels * 8);
constexpr size_t kQBytes = al(size_t(kNaQueueCap) * kQueueWords * 4);
constexpr size_t kOffCtl = kOffQ + 3 * kQBytes;
constexpr size_t kOffPrefix = kOffCtl + al(size_t(kNaCtlRows) * 16);
constexpr size_t kOffCounters = kOffPrefix + al(kNaMaxPrefix * 4);
constexpr size_t kOffLedger = kOffCounters + al(C_NCOUNT * 8);
constexpr size_t kOffStatus = kOffLedger + al(L_NLEDGER * 8);
constexpr size_t kOffMaj = kOffStatus + al(16);
constexpr size_t kOffEdges = kOffMaj + al(size_t(kNaMaxEnergy) * 4);
constexpr size_t kOffBeamlets = kOffEdges + al((GDPM_MAX_BINS + 1) * 4);
constexpr size_t kOffCdf = kOffBeamlets + al(size_t(kNaMaxBeamlets) * 16 * 4);
constexpr size_t kOffRow = kOffCdf + al(size_t(kNaMaxBeamlets) * 8);
constexpr size_t kOffF = kOffRow + al(size_t(kNaMaxBeamlets) * 4);
constexpr size_t kOffCut = kOffF + al(size_t(kNaMaxBeamlets) * 8);
constexpr size_t kOffAlias = kOffCut + al(size_t(kNaMaxBeamlets) * 8);
constexpr size_t kOffChains = kOffAlias + al(size_t(kNaMaxBeamlets) * 4);
constexpr size_t kOffPick = kOffChains + al(size_t(kNaMaxChains) * 4);
constexpr size_t kOffSrc = kOffPick + al(size_t(kNaChunk) * 4);
constexpr size_t kScratchBytes = kOffSrc + al(size_t(kNaChunk) * kSourceWords * 4);
static_assert(kScratchBytes == GDPM_NOALLOC_SCRATCH_BYTES, "header and layout disagree");

// The scratch.  In host code `g_scratch` only names a host-side stand-in; its
// device address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
unsigned char* g_addr[64] = {};

// Device address of the scratch on the current device (set up on the first
// call for that device).
int scratch_address(int device, unsigned char** out) {
    if (device < 0 || device >= 64) return GDPM_E_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) {
            last_cuda_error() = e;
            return GDPM_E_CUDA;
        }
        g_addr[device] = static_cast<unsigned char*>(p);
    }
    *out = g_addr[device];
    return GDPM_OK;
}

}  // namespace
}  // namespace gdpm

using namespace gdpm;

extern "C" int gdpm_simulate_noalloc(gdpm_ctx* ctx, gdpm_phantom* ph, gdpm_tables* tb,
                                     uint64_t n_hist, int n_batches, double* dose_out,
                                     double* sigma_out, gdpm_stats* st) {
    if (!ctx || !ph || !tb) return GDPM_E_ARG;
    const gdpm_source_state& src = ctx->src;
    if (!src.set) return GDPM_E_STATE;
    const size_t V = size_t(ph->nx) * ph->ny * ph->nz;
    const int n_bins = int(src.weights.size());
    BeamletHost bh;
    if (src.desc.geometry == GDPM_GEO_BEAMLETS) beamlet_tables_host(src.beamlets, bh);
    const int n_bl = int(bh.f.size());
    const bool metro = n_bl > 0 && src.desc.beamlet_sampler == GDPM_SAMPLE_METROPOLIS;
    // limits of the fixed scratch
    if (V > kNaMaxVoxels || tb->n_e > kNaMaxEnergy || n_bl > kNaMaxBeamlets ||
        (metro && uint32_t(src.desc.metropolis_chains) > kNaMaxChains) ||
        size_t(n_batches) * (n_bins + 1) > kNaMaxPrefix)
        return GDPM_E_ARG;
    if (n_batches < 2 || n_hist < uint64_t(n_batches) || n_hist >= (1ull << 32)) return GDPM_E_ARG;
    if ((dose_out && !is_device_ptr(dose_out)) || (sigma_out && !is_device_ptr(sigma_out))) return GDPM_E_ARG;
    for (int m = tb->n_mat; m < 256; ++m)
        if (ph->rhomax_host[m] > 0.f) return GDPM_E_ARG;
    double emin = 1e300, emax = 0.0;
    for (int j = 0; j < n_bins; ++j) {
        if (!(src.weights[j] > 0)) continue;
        emin = std::min(emin, src.edges[j]);
        emax = std::max(emax, src.edges[j + 1]);
    }
    if (emax > tb->e_max * (1 + 1e-12) || emin < tb->e_min * (1 - 1e-12)) return GDPM_E_ARG;
    GDPM_CUDA_TRY(cudaSetDevice(ctx->device));
    unsigned char* base = nullptr;
    int rc = scratch_address(ctx->device, &base);
    if (rc) return rc;
    cudaStream_t s = ctx->stream;

    // carve the scratch
    double* edep = reinterpret_cast<double*>(base + kOffEdep);
    double* s1 = reinterpret_cast<double*>(base + kOffS1);
    double* s2 = reinterpret_cast<double*>(base + kOffS2);
    const Queue qph = queue_view(base + kOffQ, kNaQueueCap);
    const Queue qe[2] = {queue_view(base + kOffQ + kQBytes, kNaQueueCap),
                         queue_view(base + kOffQ + 2 * kQBytes, kNaQueueCap)};
    uint32_t* ctl = reinterpret_cast<uint32_t*>(base + kOffCtl);
    uint32_t* prefix_d = reinterpret_cast<uint32_t*>(base + kOffPrefix);
    unsigned long long* counters = reinterpret_cast<unsigned long long*>(base + kOffCounters);
    double* ledger = reinterpret_cast<double*>(base + kOffLedger);
    uint32_t* status = reinterpret_cast<uint32_t*>(base + kOffStatus);
    float* maj = reinterpret_cast<float*>(base + kOffMaj);
    float* edges = reinterpret_cast<float*>(base + kOffEdges);
    float* bl = reinterpret_cast<float*>(base + kOffBeamlets);
    float* cdf = reinterpret_cast<float*>(base + kOffCdf);
    int* bl_row = reinterpret_cast<int*>(base + kOffRow);
    double* bl_f = reinterpret_cast<double*>(base + kOffF);
    uint64_t* al_cut = reinterpret_cast<uint64_t*>(base + kOffCut);
    int* al_alias = reinterpret_cast<int*>(base + kOffAlias);
    uint32_t* chains = reinterpret_cast<uint32_t*>(base + kOffChains);
    uint32_t* pick = reinterpret_cast<uint32_t*>(base + kOffPick);
    const Queue qsrc = source_queue_view(base + kOffSrc, kNaChunk);

    // source arrays and majorant into the scratch
    std::vector<float> ef(src.edges.begin(), src.edges.end());
    GDPM_CUDA_TRY(cudaMemcpyAsync(edges, ef.data(), ef.size() * 4, cudaMemcpyHostToDevice, s));
    if (n_bl > 0) {
        GDPM_CUDA_TRY(cudaMemcpyAsync(bl, bh.rows.data(), size_t(n_bl) * 64, cudaMemcpyHostToDevice, s));
        GDPM_CUDA_TRY(cudaMemcpyAsync(cdf, bh.cdf_up.data(), size_t(n_bl) * 4, cudaMemcpyHostToDevice, s));
        GDPM_CUDA_TRY(cudaMemcpyAsync(bl_row, bh.row.data(), size_t(n_bl) * 4, cudaMemcpyHostToDevice, s));
        GDPM_CUDA_TRY(cudaMemcpyAsync(bl_f, bh.f.data(), size_t(n_bl) * 8, cudaMemcpyHostToDevice, s));
        GDPM_CUDA_TRY(cudaMemcpyAsync(al_cut, bh.cut_t.data(), size_t(n_bl) * 8, cudaMemcpyHostToDevice, s));
        GDPM_CUDA_TRY(cudaMemcpyAsync(al_alias, bh.alias.data(), size_t(n_bl) * 4, cudaMemcpyHostToDevice, s));
    }
    if ((rc = launch_majorant_into(s, ph, tb, maj))) return rc;
    std::vector<uint32_t> prefix(size_t(n_batches) * (n_bins + 1));
    for (int b = 0; b < n_batches; ++b) {
        const uint64_t nb = n_hist / n_batches + (uint64_t(b) < n_hist % n_batches ? 1 : 0);
        allot_prefix(src.weights, nb, &prefix[size_t(b) * (n_bins + 1)]);
    }
    GDPM_CUDA_TRY(cudaMemcpyAsync(prefix_d, prefix.data(), prefix.size() * 4, cudaMemcpyHostToDevice, s));

    // the array keeps the previous call's contents: clear what accumulates
    // FP32 pair mode keeps hi in the first V floats and lo from the next
    // 256-byte boundary: the batch fold reads both halves as float2, so lo
    // must stay 8-byte aligned when V is odd.  al(4V) + 4V <= 8 * kNaMaxVoxels
    // for every V <= kNaMaxVoxels, so both halves fit the edep region.
    const size_t lo_off = al(V * 4);
    const size_t tally_bytes = ctx->tally_mode == 0 ? V * 8 : lo_off + V * 4;
    if (tally_bytes > al(kNaMaxVoxels * 8)) return GDPM_E_ARG;
    GDPM_CUDA_TRY(cudaMemsetAsync(edep, 0, tally_bytes, s));
    GDPM_CUDA_TRY(cudaMemsetAsync(s1, 0, V * 8, s));
    GDPM_CUDA_TRY(cudaMemsetAsync(s2, 0, V * 8, s));
    GDPM_CUDA_TRY(cudaMemsetAsync(counters, 0, C_NCOUNT * 8, s));
    GDPM_CUDA_TRY(cudaMemsetAsync(ledger, 0, L_NLEDGER * 8, s));
    GDPM_CUDA_TRY(cudaMemsetAsync(status, 0, 16, s));

    SimParams P = base_params(ctx, ph, tb, ctx->request_id);
    P.maj = maj;
    P.edep = edep;
    P.edep_hi = reinterpret_cast<float*>(edep);            // FP32 pair mode: hi, then lo
    P.edep_lo = reinterpret_cast<float*>(base + kOffEdep + lo_off);
    if (reinterpret_cast<uintptr_t>(P.edep_lo) % 8 != 0) return GDPM_E_ARG;
    P.counters = counters;
    P.ledger = ledger;
    P.status = status;
    DevSource& S = P.S;
    const gdpm_source_desc& g = src.desc;
    source_fields(src, S);
    S.n_beamlets = n_bl;
    S.edges = edges;
    S.beamlets = n_bl ? bl : nullptr;
    S.bl_cdf = n_bl ? cdf : nullptr;
    S.bl_row = n_bl ? bl_row : nullptr;
    S.bl_f = n_bl ? bl_f : nullptr;
    S.al_cut = n_bl ? al_cut : nullptr;
    S.al_alias = n_bl ? al_alias : nullptr;
    int64_t aux = 0;
    if (metro) {
        if ((rc = launch_metropolis_init(s, P, chains))) return rc;
        ++aux;
    }

    const uint64_t nb_max = (n_hist + n_batches - 1) / n_batches;
    const uint32_t chunk = uint32_t(std::min<uint64_t>(kNaChunk, nb_max));
    const int max_phases = std::min(ctx->max_phases, kNaCtlRows - 4);
    const bool photon_src = g.particle == GDPM_PHOTON;
    GDPM_CUDA_TRY(cudaEventRecord(ctx->ev0, s));
    int64_t phases = 0;
    uint64_t first = 0;
    int run_rc = GDPM_OK;
    uint32_t host[2];
    for (int b = 0; b < n_batches && run_rc == GDPM_OK; ++b) {
        const uint64_t nb = n_hist / n_batches + (uint64_t(b) < n_hist % n_batches ? 1 : 0);
        GDPM_CUDA_TRY(cudaMemsetAsync(ctl, 0, size_t(kNaCtlRows) * 16, s));
        uint64_t left = nb, next = 0;
        int k = photon_src ? 0 : 1, since = 0;
        // photon phase k: P[k] -> E[k+1]; electron phase k: E[k] -> P[k+1], E[k+2]
        for (;;) {
            if (k + 3 >= max_phases) { run_rc = GDPM_E_TIMEOUT; break; }
            const bool ph_phase = (k % 2) == 0;
            PhaseArgs A{};
            A.nb_small = uint32_t(n_hist / n_batches);
            A.nb_rem = uint32_t(n_hist % n_batches);
            A.bin_prefix = prefix_d;
            A.prefix_n = uint32_t(prefix.size());
            if (ph_phase == photon_src && left > 0) {
                A.n_src = uint32_t(std::min<uint64_t>(left, chunk));
                A.src_first = uint32_t(first + next);
                next += A.n_src;
                left -= A.n_src;
                if (metro) {
                    if ((run_rc = launch_metropolis(s, P, A.src_first, A.n_src, chains, pick))) break;
                    A.bl_pick = pick;
                    ++aux;
                }
                A.src = qsrc;
                if ((run_rc = launch_sources(ctx, s, P, A))) break;
                ++aux;
            }
            A.head = ctl + size_t(k) * 4;
            if (ph_phase) {
                A.in = qph;
                A.in_count = k >= 1 ? ctl + size_t(k) * 4 + 1 : nullptr;
                A.out_el = qe[((k + 1) / 2) % 2];
                A.out_el_count = ctl + size_t(k + 1) * 4 + 2;
                A.out_ph = qph;
                A.out_ph_count = ctl + size_t(k + 2) * 4 + 1;
            } else {
                A.in = qe[(k / 2) % 2];
                A.in_count = ctl + size_t(k) * 4 + 2;
                A.out_ph = qph;
                A.out_ph_count = ctl + size_t(k + 1) * 4 + 1;
                A.out_el = qe[((k + 2) / 2) % 2];
                A.out_el_count = ctl + size_t(k + 2) * 4 + 2;
            }
            if ((run_rc = launch_phase(ctx, s, ph_phase ? GDPM_PHOTON : GDPM_ELECTRON, P, A,
                                       A.in_count ? 0u : A.n_src)))
                break;
            ++phases;
            ++k;
            ++since;
            if (!ph_phase && left == 0 && since >= 2 * ctx->speculative) {
                GDPM_CUDA_TRY(cudaMemcpyAsync(&host[0], ctl + size_t(k) * 4 + 1, 4, cudaMemcpyDeviceToHost, s));
                GDPM_CUDA_TRY(cudaMemcpyAsync(&host[1], ctl + size_t(k + 1) * 4 + 2, 4, cudaMemcpyDeviceToHost, s));
                GDPM_CUDA_TRY(cudaStreamSynchronize(s));
                if (host[0] == 0 && host[1] == 0) break;
                since = 0;
            }
        }
        if (run_rc == GDPM_OK) run_rc = launch_fold_into(ctx, s, P, V, uint32_t(nb), s1, s2);
        first += nb;
    }
    GDPM_CUDA_TRY(cudaEventRecord(ctx->ev1, s));
    if (run_rc != GDPM_OK) {
        cudaStreamSynchronize(s);
        return run_rc;
    }
    if ((rc = launch_finalize_into(ctx, s, P, V, n_batches, s1, s2, dose_out, sigma_out))) return rc;
    unsigned long long hc[C_NCOUNT];
    double hl[L_NLEDGER];
    uint32_t hs = 0;
    GDPM_CUDA_TRY(cudaMemcpyAsync(hc, counters, sizeof hc, cudaMemcpyDeviceToHost, s));
    GDPM_CUDA_TRY(cudaMemcpyAsync(hl, ledger, sizeof hl, cudaMemcpyDeviceToHost, s));
    GDPM_CUDA_TRY(cudaMemcpyAsync(&hs, status, 4, cudaMemcpyDeviceToHost, s));
    GDPM_CUDA_TRY(cudaStreamSynchronize(s));
    if (st) {
        std::memset(st, 0, sizeof(*st));
        st->source_energy = hl[L_SOURCE];
        st->deposited = hl[L_DEPOSITED];
        st->escaped = hl[L_ESCAPED];
        st->discarded = hl[L_DISCARDED];
        st->n_primary = int64_t(hc[C_PRIMARY]);
        st->ph_created = int64_t(hc[C_PH_CREATED]);
        st->ph_terminated = int64_t(hc[C_PH_TERMINATED]);
        st->ph_flights = int64_t(hc[C_PH_FLIGHTS]);
        st->ph_real = int64_t(hc[C_PH_REAL]);
        st->compton = int64_t(hc[C_COMPTON]);
        st->photoelectric = int64_t(hc[C_PHOTO]);
        st->pair = int64_t(hc[C_PAIR]);
        st->el_created = int64_t(hc[C_EL_CREATED]);
        st->el_terminated = int64_t(hc[C_EL_TERMINATED]);
        st->el_steps = int64_t(hc[C_EL_STEPS]);
        st->moller = int64_t(hc[C_MOLLER]);
        st->brems = int64_t(hc[C_BREMS]);
        st->annihilations = int64_t(hc[C_ANNIHIL]);
        st->local_deposits = int64_t(hc[C_LOCAL_DEP]);
        st->pushes[0] = int64_t(hc[C_PUSH_PH]);
        st->pushes[1] = int64_t(hc[C_PUSH_EL]);
        st->pops[0] = int64_t(hc[C_POP_PH]);
        st->pops[1] = int64_t(hc[C_POP_EL]);
        st->crossings = int64_t(hc[C_CROSS]);
        st->phases = phases;
        st->launches = phases + aux + n_batches + 3;   // + majorant, folds, finalize, metric
        double dmax;
        std::memcpy(&dmax, &hl[L_DMAX], 8);
        st->dmax = dmax;
        st->sigma_over_dmax = (hl[L_SIGCNT] > 0 && dmax > 0) ? hl[L_SIGSUM] / hl[L_SIGCNT] / dmax : 0.0;
        float ms = 0;
        cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
        st->transport_ms = ms;
    }
    if (hs & ST_BOUNDS) return GDPM_E_BOUNDS;
    if (hs & ST_QUEUE_OVERFLOW) return GDPM_E_QUEUE_OVERFLOW;
    if (hs & ST_ITER_CAP) return GDPM_E_TIMEOUT;
    return GDPM_OK;
}
