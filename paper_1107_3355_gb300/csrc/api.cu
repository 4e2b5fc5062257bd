// C ABI of the engine and the host-side scheduler of one dose calculation.
//
// A calculation runs N_b batches (Sec. 2.2.1).  Within a batch the device
// alternates photon and electron phases (Sec. 2.2.1 Step 3: one particle
// type at a time) until no primaries are left and both queues are empty.
// Queue bookkeeping lives entirely on the device: every phase k owns a pop
// counter, and every queue fill owns its own count, all zeroed once per
// batch, so phases chain without host round trips.  The host checks for an
// empty batch only after the primaries are used up, once per
// `speculative` phase pairs (phases launched on an empty input exit at once).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"

namespace gdpm {

cudaError_t& last_cuda_error() {
    static thread_local cudaError_t e = cudaSuccess;
    return e;
}

int ensure(Buffer& b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.p && b.bytes >= bytes) return GDPM_OK;
    release(b);
    void* p = nullptr;
    const cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return GDPM_E_NOMEM;
    }
    b.p = p;
    b.bytes = bytes;
    return GDPM_OK;
}

void release(Buffer& b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

// Histories of one batch allotted to the spectrum intervals by weight:
// floor, then the remainder one by one to the largest fractional parts
// (ties to the lower interval) (Sec. 2.3.2).  Writes n_bins+1 prefix counts.
void allot_prefix(const std::vector<double>& w, uint64_t nb, uint32_t* prefix) {
    const int K = int(w.size());
    double ws = 0;
    for (double x : w) ws += x;
    std::vector<uint64_t> c(K);
    std::vector<double> frac(K);
    uint64_t given = 0;
    for (int j = 0; j < K; ++j) {
        const double q = double(nb) * (w[j] / ws);
        c[j] = uint64_t(std::floor(q));
        frac[j] = q - std::floor(q);
        given += c[j];
    }
    while (given < nb) {
        int best = -1;
        for (int j = 0; j < K; ++j)
            if (w[j] > 0 && (best < 0 || frac[j] > frac[best])) best = j;
        ++c[best];
        frac[best] = -1.0;
        ++given;
    }
    prefix[0] = 0;
    for (int j = 0; j < K; ++j) prefix[j + 1] = prefix[j] + uint32_t(c[j]);
}

int runner_init(Runner& r, cudaStream_t stream, bool own_stream) {
    r.owns_stream = own_stream;
    if (own_stream) {
        int least = 0, greatest = 0;
        GDPM_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        GDPM_CUDA_TRY(cudaStreamCreateWithPriority(&r.prio_hi, cudaStreamNonBlocking, greatest));
        GDPM_CUDA_TRY(cudaStreamCreateWithPriority(&r.prio_lo, cudaStreamNonBlocking, least));
        r.stream = r.prio_lo;
    } else {
        r.stream = stream;
    }
    GDPM_CUDA_TRY(cudaStreamCreateWithFlags(&r.side, cudaStreamNonBlocking));
    GDPM_CUDA_TRY(cudaEventCreate(&r.ev0));
    GDPM_CUDA_TRY(cudaEventCreate(&r.ev1));
    for (int k = 0; k < 2; ++k) {
        GDPM_CUDA_TRY(cudaEventCreateWithFlags(&r.batch_done[k], cudaEventDisableTiming));
        GDPM_CUDA_TRY(cudaEventCreateWithFlags(&r.fold_done[k], cudaEventDisableTiming));
    }
    return GDPM_OK;
}

void runner_free(Runner& r) {
    if (r.stream) cudaStreamSynchronize(r.stream);
    if (r.side) cudaStreamSynchronize(r.side);
    Workspace& w = r.ws;
    Buffer* bs[] = {&w.edep, &w.edep2, &w.hi2, &w.lo2, &w.s1, &w.s2, &w.hi, &w.lo, &w.qph,
                    &w.qel0, &w.qel1, &w.qsrc, &w.ctl, &w.prefix, &w.counters, &w.ledger, &w.status,
                    &w.edges, &w.beamlets, &w.bl_cdf, &w.bl_row, &w.bl_f, &w.al_cut,
                    &w.al_alias, &w.chains, &w.pick, &w.sub_first, &w.sub_inv, &w.sub_nbig,
                    &w.loop_k, &w.stage};
    for (Buffer* b : bs) release(*b);
    if (r.loop_exec) cudaGraphExecDestroy(r.loop_exec);
    if (r.loop_graph) cudaGraphDestroy(r.loop_graph);
    r.loop_exec = nullptr;
    r.loop_graph = nullptr;
    r.loop_key.clear();
    if (w.pinned_host.p) cudaFreeHost(w.pinned_host.p);
    w.pinned_host.p = nullptr;
    for (cudaEvent_t e : r.prof_events) cudaEventDestroy(e);
    r.prof_events.clear();
    cudaEvent_t evs[] = {r.ev0, r.ev1, r.batch_done[0], r.batch_done[1], r.fold_done[0], r.fold_done[1]};
    for (cudaEvent_t e : evs)
        if (e) cudaEventDestroy(e);
    if (r.side) cudaStreamDestroy(r.side);
    if (r.owns_stream) {
        if (r.prio_hi) cudaStreamSynchronize(r.prio_hi), cudaStreamDestroy(r.prio_hi);
        if (r.prio_lo) cudaStreamSynchronize(r.prio_lo), cudaStreamDestroy(r.prio_lo);
    }
    r.side = r.stream = r.prio_hi = r.prio_lo = nullptr;
}

// Optional per-launch device timing (GDPM_PARAM_PROFILE): an event pair on
// the launching stream around each launch, summed per kernel kind at the end.
static size_t prof_begin(gdpm_ctx* ctx, Runner& r, cudaStream_t st, int kind) {
    if (!ctx->profile) return 0;
    const size_t idx = r.prof_kind.size();
    while (r.prof_events.size() < 2 * (idx + 1)) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        r.prof_events.push_back(e);
    }
    cudaEventRecord(r.prof_events[2 * idx], st);
    r.prof_kind.push_back(kind);
    return idx;
}
static void prof_end(gdpm_ctx* ctx, Runner& r, cudaStream_t st, size_t idx) {
    if (ctx->profile && 2 * idx + 1 < r.prof_events.size()) cudaEventRecord(r.prof_events[2 * idx + 1], st);
}
static void prof_collect(Runner& r, gdpm_stats* st) {
    for (size_t i = 0; i < r.prof_kind.size(); ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.prof_events[2 * i], r.prof_events[2 * i + 1]) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        const int k = r.prof_kind[i];
        if (st && k >= 0 && k < 4) {
            st->kernel_ms[k] += ms;
            st->kernel_launches[k] += 1;
        }
    }
    r.prof_kind.clear();
}

// A particle queue of `cap` slots laid out from `base`: 13 arrays (Queue).
Queue queue_view(void* base, uint32_t cap) {
    Queue q{};
    uint32_t* w = static_cast<uint32_t*>(base);
    float** fs[7] = {&q.x, &q.y, &q.z, &q.u, &q.v, &q.w, &q.E};
    for (int k = 0; k < 7; ++k) *fs[k] = reinterpret_cast<float*>(w + size_t(k) * cap);
    uint32_t** us[6] = {&q.vox, &q.hist, &q.pidlo, &q.pidhi, &q.ctr, &q.flags};
    for (int k = 0; k < 6; ++k) *us[k] = w + size_t(7 + k) * cap;
    q.capacity = cap;
    return q;
}
// A phase's source queue from `base`: x y z u v w E, ctr, flags (kSourceWords arrays).
Queue source_queue_view(void* base, uint32_t cap) {
    Queue q{};
    uint32_t* w = static_cast<uint32_t*>(base);
    float** fs[7] = {&q.x, &q.y, &q.z, &q.u, &q.v, &q.w, &q.E};
    for (int k = 0; k < 7; ++k) *fs[k] = reinterpret_cast<float*>(w + size_t(k) * cap);
    q.ctr = w + size_t(7) * cap;
    q.flags = w + size_t(8) * cap;
    q.capacity = cap;
    return q;
}
static Queue make_queue(const Buffer& b, uint32_t cap) { return queue_view(b.p, cap); }
static Queue make_source_queue(const Buffer& b, uint32_t cap) { return source_queue_view(b.p, cap); }

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Validate a source description and copy what it points to.
static int source_copy(const gdpm_source_desc* s, gdpm_source_state& st) {
    if (!s) return GDPM_E_ARG;
    if (s->particle != GDPM_PHOTON && s->particle != GDPM_ELECTRON) return GDPM_E_ARG;
    if (s->geometry < GDPM_GEO_PENCIL || s->geometry > GDPM_GEO_BEAMLETS) return GDPM_E_ARG;
    if (s->n_bins < 1 || s->n_bins > GDPM_MAX_BINS || !s->bin_edges || !s->bin_weights) return GDPM_E_ARG;
    double ws = 0;
    for (int j = 0; j < s->n_bins; ++j) {
        if (s->bin_weights[j] < 0 || s->bin_edges[j + 1] < s->bin_edges[j]) return GDPM_E_ARG;
        ws += s->bin_weights[j];
    }
    if (!(ws > 0) || !(s->bin_edges[0] >= 0)) return GDPM_E_ARG;
    if (s->geometry == GDPM_GEO_BEAMLETS) {
        if (s->n_beamlets < 1 || !s->beamlets) return GDPM_E_ARG;
        double bw = 0;
        for (int b = 0; b < s->n_beamlets; ++b) {
            if (s->beamlets[size_t(b) * 17 + 16] < 0) return GDPM_E_ARG;
            bw += s->beamlets[size_t(b) * 17 + 16];
        }
        if (!(bw > 0)) return GDPM_E_ARG;
        if (s->beamlet_sampler < GDPM_SAMPLE_CDF || s->beamlet_sampler > GDPM_SAMPLE_METROPOLIS ||
            s->metropolis_chains < 0 || s->metropolis_chains > (1 << 24))
            return GDPM_E_ARG;
    }
    const double dn = s->direction[0] * s->direction[0] + s->direction[1] * s->direction[1] +
                      s->direction[2] * s->direction[2];
    if (s->geometry == GDPM_GEO_PENCIL && !(dn > 0)) return GDPM_E_ARG;
    st.desc = *s;
    st.edges.assign(s->bin_edges, s->bin_edges + s->n_bins + 1);
    st.weights.assign(s->bin_weights, s->bin_weights + s->n_bins);
    if (s->geometry == GDPM_GEO_BEAMLETS)
        st.beamlets.assign(s->beamlets, s->beamlets + size_t(s->n_beamlets) * 17);
    else
        st.beamlets.clear();
    st.desc.bin_edges = nullptr;
    st.desc.bin_weights = nullptr;
    st.desc.beamlets = nullptr;
    if (st.desc.metropolis_chains == 0) st.desc.metropolis_chains = 4096;
    st.set = true;
    return GDPM_OK;
}

// Beamlets of positive weight, their cumulative weights and Walker's alias
// table (Vose's procedure: scaled weights q = f nf / sum f; the last "small"
// entry (q < 1) takes its cut-off q and the last "large" entry as alias,
// which gives up 1 - q of its own mass).  Pure additions and single
// products, so the table is the same on every host.
void beamlet_tables_host(const std::vector<double>& rows17, BeamletHost& out, bool all_rows) {
    const int nb = int(rows17.size() / 17);
    out = BeamletHost{};
    double tot = 0;
    for (int b = 0; b < nb; ++b) tot += rows17[size_t(b) * 17 + 16];
    double acc = 0;
    for (int b = 0; b < nb; ++b) {
        const double w = rows17[size_t(b) * 17 + 16];
        acc += w;
        if (!(w > 0) && !all_rows) continue;
        for (int k = 0; k < 16; ++k) out.rows.push_back(float(rows17[size_t(b) * 17 + k]));
        out.row.push_back(b);
        out.f.push_back(w);
        out.cdf.push_back(tot > 0 ? acc / tot : 0.0);
    }
    const int n = int(out.f.size());
    if (n == 0) return;
    if (all_rows) {            // rows are sub-problems, not sampled: neutral tables
        out.cut.assign(n, 1.0);
        out.alias.resize(n);
        for (int k = 0; k < n; ++k) out.alias[k] = k;
        out.cdf_up.assign(n, 1.0f);
        out.cut_t.assign(n, uint64_t(1) << 32);
        return;
    }
    out.cdf[n - 1] = 1.0;
    double sum = 0;
    for (double w : out.f) sum += w;
    const double scale = double(n) / sum;
    std::vector<double> q(n);
    std::vector<int> small, large;
    for (int k = 0; k < n; ++k) {
        q[k] = out.f[k] * scale;
        (q[k] < 1.0 ? small : large).push_back(k);
    }
    out.cut.assign(n, 1.0);
    out.alias.resize(n);
    for (int k = 0; k < n; ++k) out.alias[k] = k;
    while (!small.empty() && !large.empty()) {
        const int l = small.back(), g = large.back();
        small.pop_back();
        large.pop_back();
        out.cut[l] = q[l];
        out.alias[l] = g;
        q[g] = (q[g] + q[l]) - 1.0;
        (q[g] < 1.0 ? small : large).push_back(g);
    }
    out.cdf_up.resize(n);
    out.cut_t.resize(n);
    for (int k = 0; k < n; ++k) {
        float c = float(out.cdf[k]);
        if (double(c) < out.cdf[k]) c = std::nextafter(c, 2.0f);
        out.cdf_up[k] = c;
        // (x + 1/2) 2^-32 < cut  <=>  x < ceil(cut 2^32 - 1/2); all exact in FP64
        out.cut_t[k] = uint64_t(std::ceil(std::ldexp(out.cut[k], 32) - 0.5));
    }
}


// The source's scalar fields (geometry, spectrum size, sampler); its device
// arrays are left unset.
void source_fields(const gdpm_source_state& s, DevSource& d) {
    const gdpm_source_desc& g = s.desc;
    d.particle = g.particle;
    d.geometry = g.geometry;
    d.annihilation = g.annihilation ? 1 : 0;
    d.n_bins = int(s.weights.size());
    d.n_beamlets = 0;
    d.sampler = g.beamlet_sampler;
    d.n_chains = uint32_t(g.metropolis_chains);
    for (int a = 0; a < 3; ++a) {
        d.origin[a] = float(g.origin[a]);
        d.center[a] = float(g.center[a]);
        d.axis_u[a] = float(g.axis_u[a]);
        d.axis_v[a] = float(g.axis_v[a]);
    }
    const double dn = std::sqrt(g.direction[0] * g.direction[0] + g.direction[1] * g.direction[1] +
                                g.direction[2] * g.direction[2]);
    for (int a = 0; a < 3; ++a) d.direction[a] = dn > 0 ? float(g.direction[a] / dn) : 0.f;
    d.half_u = float(g.half_u);
    d.half_v = float(g.half_v);
    d.edges = nullptr;
    d.beamlets = nullptr;
    d.bl_cdf = nullptr;
    d.bl_row = nullptr;
    d.bl_f = nullptr;
    d.al_cut = nullptr;
    d.al_alias = nullptr;
}

static int source_upload(Runner& r, const gdpm_source_state& s, DevSource& d, bool all_rows = false) {
    const gdpm_source_desc& g = s.desc;
    source_fields(s, d);
    std::vector<float> e(s.edges.begin(), s.edges.end());
    int rc = ensure(r.ws.edges, e.size() * 4);
    if (rc) return rc;
    GDPM_CUDA_TRY(cudaMemcpyAsync(r.ws.edges.p, e.data(), e.size() * 4, cudaMemcpyHostToDevice, r.stream));
    d.edges = static_cast<const float*>(r.ws.edges.p);
    BeamletHost bh;
    if (g.geometry == GDPM_GEO_BEAMLETS) beamlet_tables_host(s.beamlets, bh, all_rows);
    if (!bh.f.empty()) {
        const size_t nbl = bh.f.size();
        Workspace& w = r.ws;
        if ((rc = ensure(w.beamlets, nbl * 64)) || (rc = ensure(w.bl_cdf, nbl * 4)) ||
            (rc = ensure(w.bl_row, nbl * 4)) || (rc = ensure(w.bl_f, nbl * 8)) ||
            (rc = ensure(w.al_cut, nbl * 8)) || (rc = ensure(w.al_alias, nbl * 4)))
            return rc;
        GDPM_CUDA_TRY(cudaMemcpyAsync(w.beamlets.p, bh.rows.data(), nbl * 64, cudaMemcpyHostToDevice, r.stream));
        GDPM_CUDA_TRY(cudaMemcpyAsync(w.bl_cdf.p, bh.cdf_up.data(), nbl * 4, cudaMemcpyHostToDevice, r.stream));
        GDPM_CUDA_TRY(cudaMemcpyAsync(w.bl_row.p, bh.row.data(), nbl * 4, cudaMemcpyHostToDevice, r.stream));
        GDPM_CUDA_TRY(cudaMemcpyAsync(w.bl_f.p, bh.f.data(), nbl * 8, cudaMemcpyHostToDevice, r.stream));
        GDPM_CUDA_TRY(cudaMemcpyAsync(w.al_cut.p, bh.cut_t.data(), nbl * 8, cudaMemcpyHostToDevice, r.stream));
        GDPM_CUDA_TRY(cudaMemcpyAsync(w.al_alias.p, bh.alias.data(), nbl * 4, cudaMemcpyHostToDevice, r.stream));
        d.n_beamlets = int(nbl);
        d.beamlets = static_cast<const float*>(w.beamlets.p);
        d.bl_cdf = static_cast<const float*>(w.bl_cdf.p);
        d.bl_row = static_cast<const int*>(w.bl_row.p);
        d.bl_f = static_cast<const double*>(w.bl_f.p);
        d.al_cut = static_cast<const uint64_t*>(w.al_cut.p);
        d.al_alias = static_cast<const int*>(w.al_alias.p);
    }
    // the host vectors above are staged by the copies; make the copies
    // complete before they go out of scope
    GDPM_CUDA_TRY(cudaStreamSynchronize(r.stream));
    return GDPM_OK;
}

// Woodcock majorant of a (phantom, tables) pair, built once and shared by
// every calculation on that pair.
static int get_majorant(gdpm_ctx* ctx, cudaStream_t st, gdpm_phantom* ph, gdpm_tables* tb, const float** out) {
    std::lock_guard<std::mutex> lk(ctx->maj_mu);
    Buffer& b = ph->maj[tb->id];
    if (!b.p) {
        int rc = ensure(b, sizeof(float) * tb->n_e);
        if (rc) return rc;
        if ((rc = launch_majorant_into(st, ph, tb, static_cast<float*>(b.p)))) return rc;
        GDPM_CUDA_TRY(cudaStreamSynchronize(st));
    }
    *out = static_cast<const float*>(b.p);
    return GDPM_OK;
}

// The electron phase form of a run (GDPM_PARAM_ELECTRON_WALK): automatic
// (2) takes resumable steps where the phantom holds air-like voxels.  An
// electron that reaches air takes a step hundreds of voxels long, and in
// whole steps that one lane holds its warp for the whole walk; without air
// the walks are short and the whole-step form, with less state to carry
// across the loop top, is faster.
int walk_form(const gdpm_ctx* ctx, const gdpm_phantom* ph) {
    if (ctx->electron_walk != 2) return ctx->electron_walk;
    return ph->rhomin_host < kAirDensity ? 1 : 0;
}

SimParams base_params(gdpm_ctx* ctx, gdpm_phantom* ph, gdpm_tables* tb, uint32_t request_id) {
    SimParams P{};
    P.nx = ph->nx; P.ny = ph->ny; P.nz = ph->nz;
    P.dx = ph->dx; P.dy = ph->dy; P.dz = ph->dz;
    P.inv_dx = 1.f / ph->dx; P.inv_dy = 1.f / ph->dy; P.inv_dz = 1.f / ph->dz;
    P.Lx = float(double(ph->nx) * ph->dx);
    P.Ly = float(double(ph->ny) * ph->dy);
    P.Lz = float(double(ph->nz) * ph->dz);
    P.mat = static_cast<const uint8_t*>(ph->mat.p);
    P.rho = static_cast<const float*>(ph->rho.p);
    P.T = tb->dev;
    P.key0 = uint32_t(ctx->seed);
    P.key1 = uint32_t(ctx->seed >> 32) ^ request_id;
    P.tally_mode = ctx->tally_mode;
    P.walk_resumable = walk_form(ctx, ph);
    P.max_iters = ctx->max_iters;   // loop trips per warp and phase (GDPM_PARAM_MAX_ITERS)
    P.tally_lo = 0;
    P.tally_hi = uint64_t(ph->nx) * ph->ny * ph->nz;   // one grid; widened by batched runs
    P.n_records = 0;
    return P;
}

static int validate_run(gdpm_ctx* ctx, gdpm_phantom* ph, gdpm_tables* tb, const gdpm_source_state& src,
                        uint64_t n_hist, int n_batches) {
    if (!ctx || !ph || !tb) return GDPM_E_ARG;
    if (!src.set) return GDPM_E_STATE;
    if (n_batches < 2 || n_hist < uint64_t(n_batches) || n_hist >= (1ull << 32)) return GDPM_E_ARG;
    for (int m = tb->n_mat; m < 256; ++m)
        if (ph->rhomax_host[m] > 0.f) return GDPM_E_ARG;
    // energies that can be drawn: the intervals with positive weight
    double emin = 1e300, emax = 0.0;
    for (size_t j = 0; j < src.weights.size(); ++j) {
        if (!(src.weights[j] > 0)) continue;
        emin = std::min(emin, src.edges[j]);
        emax = std::max(emax, src.edges[j + 1]);
    }
    if (emax > tb->e_max * (1 + 1e-12) || emin < tb->e_min * (1 - 1e-12)) return GDPM_E_ARG;
    return GDPM_OK;
}

// Primaries per transport phase, and no more than one batch (or run) holds.
// Batches side by side share their phases, so those phases can be long (up
// to ctx->auto_chunk primaries, sized from the device's memory): a phase
// ends with a tail in which lanes run out of particles, and longer phases
// make the tail a smaller share.  Batches one after another have one batch
// per phase, up to 2^20 primaries.  A served request may keep shorter phases
// (GDPM_PARAM_SERVE_PHASE_CAP): a persistent phase holds its SMs until it
// drains, and shorter phases let the small requests that arrive meanwhile
// get SMs sooner.
static uint32_t chunk_of(gdpm_ctx* ctx, uint64_t n_per_run, int parts, bool concurrent,
                         bool serving = false) {
    const uint64_t per = (n_per_run + parts - 1) / parts;
    uint32_t chunk = ctx->source_chunk ? ctx->source_chunk : concurrent ? ctx->auto_chunk : (1u << 20);
    if (serving && !ctx->source_chunk && ctx->serve_phase_cap) chunk = std::min(chunk, ctx->serve_phase_cap);
    return uint32_t(std::min<uint64_t>(chunk, per));
}
static uint32_t capacity_of(gdpm_ctx* ctx, uint32_t chunk) {
    return ctx->queue_capacity ? ctx->queue_capacity : 8u * chunk + 65536u;
}

// Run all batches side by side (one tally grid each) or one after another?
static bool side_by_side(gdpm_ctx* ctx, size_t V, uint64_t n_hist, int n_batches) {
    if (ctx->batch_mode == 1 || n_batches > kMaxConcurrentBatches) return false;
    const size_t bytes = V * size_t(n_batches) * 8;
    if (ctx->batch_mode == 2) return true;
    return n_hist / uint64_t(n_batches) <= ctx->concurrent_max_hist && bytes <= ctx->concurrent_max_bytes;
}

// Work buffers for a phantom of V voxels and queues of `cap` particles.
static int prepare_workspace(gdpm_ctx* ctx, Runner& r, size_t V, uint32_t cap, uint32_t chunk,
                             int n_batches, int n_bins, bool concurrent) {
    Workspace& ws = r.ws;
    int rc;
    const size_t clean = ws.edep_clean;
    ws.edep_clean = 0;
    ws.edep_zero = 0;
    if ((rc = ensure(ws.s1, V * 8)) || (rc = ensure(ws.s2, V * 8))) return rc;
    if (concurrent) {
        // one grid per batch: V*n_batches doubles, or hi and lo halves of floats
        const size_t want = V * size_t(n_batches) * 8;
        const bool kept = ws.edep.p && ws.edep.bytes >= want;   // ensure keeps it and its contents
        if ((rc = ensure(ws.edep, want))) return rc;
        ws.edep_zero = kept ? clean : 0;
    } else if (ctx->tally_mode == 0) {
        if ((rc = ensure(ws.edep, V * 8)) || (rc = ensure(ws.edep2, V * 8))) return rc;
    } else {
        if ((rc = ensure(ws.hi, V * 4)) || (rc = ensure(ws.lo, V * 4)) || (rc = ensure(ws.hi2, V * 4)) ||
            (rc = ensure(ws.lo2, V * 4)))
            return rc;
    }
    const size_t qb = size_t(cap) * kQueueWords * 4;
    if ((rc = ensure(ws.qph, qb)) || (rc = ensure(ws.qel0, qb)) || (rc = ensure(ws.qel1, qb))) return rc;
    ws.cap_ph = ws.cap_el = cap;
    // primaries of one phase: at most a chunk
    if ((rc = ensure(ws.qsrc, size_t(chunk) * kSourceWords * 4))) return rc;
    ws.cap_src = chunk;
    if ((rc = ensure(ws.ctl, size_t(ctx->max_phases + 4) * 16)) ||
        (rc = ensure(ws.prefix, size_t(n_batches) * (n_bins + 1) * 4)) ||
        (rc = ensure(ws.counters, C_NCOUNT * 8)) || (rc = ensure(ws.ledger, L_NLEDGER * 8)) ||
        (rc = ensure(ws.status, 16)))
        return rc;
    if (!ws.pinned_host.p) {
        void* h = nullptr;
        GDPM_CUDA_TRY(cudaMallocHost(&h, 4096));
        ws.pinned_host.p = h;
        ws.pinned_host.bytes = 4096;
    }
    return GDPM_OK;
}

// Device bytes a calculation still has to allocate in runner r.
static size_t bytes_needed(gdpm_ctx* ctx, const Runner& r, size_t V, uint64_t n_hist, int n_batches,
                           bool with_result) {
    const bool conc = side_by_side(ctx, V, n_hist, n_batches);
    const uint32_t chunk = chunk_of(ctx, conc ? n_hist : n_hist / n_batches + 1, 1, conc, r.serving);
    const uint32_t cap = capacity_of(ctx, chunk);
    auto grow = [](const Buffer& b, size_t want) { return b.bytes >= want ? size_t(0) : want; };
    const Workspace& w = r.ws;
    size_t n = grow(w.s1, V * 8) + grow(w.s2, V * 8);
    n += conc ? grow(w.edep, V * size_t(n_batches) * 8) : grow(w.edep, V * 8) + grow(w.edep2, V * 8);
    const size_t qb = size_t(cap) * kQueueWords * 4;
    n += grow(w.qph, qb) + grow(w.qel0, qb) + grow(w.qel1, qb);
    n += grow(w.qsrc, size_t(chunk) * kSourceWords * 4);
    if (with_result) n += V * 16;
    return n;
}

// The histories [first, first+n) (one batch, or all batches side by side):
// alternate photon (even k) and electron (odd k) phases.
//   photon phase k consumes fill P[k] (+ photon primaries), banks electrons into E[k+1];
//   electron phase k consumes E[k] (+ electron primaries), banks photons into
//   P[k+1] and electrons into E[k+2].
// ctl row k: [0] pop counter of phase k, [1] count of P[k], [2] count of E[k].
// The phase schedule of one run: queues, counter rows, sources (primaries
// [first, first+n) in chunks of `chunk`), batch layout.  Both the host loop
// and the device-driven loop hand it to the one phase kernel, which derives
// phase k's arguments from it.
static LoopArgs loop_args(gdpm_ctx* ctx, Runner& r, const SimParams& P, const gdpm_source_state& src,
                          uint64_t first, uint64_t n, uint32_t nb_small, uint32_t nb_rem, uint32_t chunk,
                          uint32_t n_sub, uint32_t sub_batches, const uint32_t* sub_first) {
    Workspace& ws = r.ws;
    LoopArgs L{};
    L.qph = make_queue(ws.qph, ws.cap_ph);
    L.qe0 = make_queue(ws.qel0, ws.cap_el);
    L.qe1 = make_queue(ws.qel1, ws.cap_el);
    L.qsrc = make_source_queue(ws.qsrc, ws.cap_src);
    L.ctl = static_cast<uint32_t*>(ws.ctl.p);
    L.status = P.status;
    L.bin_prefix = static_cast<const uint32_t*>(ws.prefix.p);
    L.prefix_n = ws.prefix_n;
    L.sub_first = sub_first;
    const bool metro = P.S.sampler == GDPM_SAMPLE_METROPOLIS && P.S.n_beamlets > 0 && n_sub == 0;
    L.chains = metro ? static_cast<uint32_t*>(ws.chains.p) : nullptr;
    L.pick = metro ? static_cast<uint32_t*>(ws.pick.p) : nullptr;
    L.n_src = uint32_t(n);
    L.first = uint32_t(first);
    L.chunk = chunk;
    L.nb_small = nb_small;
    L.nb_rem = nb_rem;
    L.n_sub = n_sub;
    L.sub_batches = sub_batches;
    L.src_particle = src.desc.particle;
    L.max_phases = ctx->max_phases;
    return L;
}

static int run_phases(gdpm_ctx* ctx, Runner& r, const SimParams& P, const gdpm_source_state& src,
                      uint64_t first, uint64_t n, uint32_t nb_small, uint32_t nb_rem, uint32_t chunk,
                      int64_t& phases, int64_t& aux, uint32_t n_sub = 0, uint32_t sub_batches = 0,
                      const uint32_t* sub_first = nullptr) {
    Range range("transport phases");
    Workspace& ws = r.ws;
    cudaStream_t s = r.stream;
    uint32_t* ctl = static_cast<uint32_t*>(ws.ctl.p);
    GDPM_CUDA_TRY(cudaMemsetAsync(ctl, 0, size_t(ctx->max_phases + 4) * 16, s));
    const Queue qph = make_queue(ws.qph, ws.cap_ph);
    const Queue qe[2] = {make_queue(ws.qel0, ws.cap_el), make_queue(ws.qel1, ws.cap_el)};
    const bool photon_src = src.desc.particle == GDPM_PHOTON;
    uint64_t left = n, next = first;
    int k = photon_src ? 0 : 1;
    int since = 0;
    uint32_t* host = static_cast<uint32_t*>(ws.pinned_host.p);
    for (;;) {
        if (k + 3 >= ctx->max_phases) return GDPM_E_TIMEOUT;
        const bool ph = (k % 2) == 0;
        PhaseArgs A{};
        A.nb_small = nb_small;
        A.nb_rem = nb_rem;
        A.n_sub = n_sub;
        A.sub_batches = sub_batches;
        A.sub_first = sub_first;
        A.bin_prefix = static_cast<const uint32_t*>(ws.prefix.p);
        A.prefix_n = ws.prefix_n;
        if (ph == photon_src && left > 0) {
            A.n_src = uint32_t(std::min<uint64_t>(left, chunk));
            A.src_first = uint32_t(next);
            next += A.n_src;
            left -= A.n_src;
            const size_t ps = prof_begin(ctx, r, s, 3);
            if (P.S.sampler == GDPM_SAMPLE_METROPOLIS && P.S.n_beamlets > 0 && n_sub == 0) {
                // this phase's beamlets: advance the chains (Algorithm A1)
                uint32_t* pick = static_cast<uint32_t*>(ws.pick.p);
                const int rc = launch_metropolis(s, P, A.src_first, A.n_src,
                                                 static_cast<uint32_t*>(ws.chains.p), pick);
                if (rc) return rc;
                A.bl_pick = pick;
                ++aux;
            }
            // this phase's primaries, made before it runs
            A.src = make_source_queue(ws.qsrc, ws.cap_src);
            if (int rc = launch_sources(ctx, s, P, A)) return rc;
            prof_end(ctx, r, s, ps);
            ++aux;
        }
        A.head = ctl + size_t(k) * 4 + 0;
        if (ph) {
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
        const uint32_t hint = A.in_count ? 0u : A.n_src;
        const size_t pi = prof_begin(ctx, r, s, ph ? 0 : 1);
        const uint32_t share = (r.serving && !r.small && ctx->small_running.load() > 0)
                                   ? uint32_t(ctx->serve_share8) : 8u;
        int rc = launch_phase(ctx, s, ph ? GDPM_PHOTON : GDPM_ELECTRON, P, A, hint, share);
        prof_end(ctx, r, s, pi);
        if (rc) return rc;
        ++phases;
        ++k;
        ++since;
        if (!ph && left == 0 && since >= 2 * ctx->speculative) {
            // pending after electron phase k-1: photons P[k], electrons E[k+1]
            GDPM_CUDA_TRY(cudaMemcpyAsync(host, ctl + size_t(k) * 4 + 1, 4, cudaMemcpyDeviceToHost, s));
            GDPM_CUDA_TRY(cudaMemcpyAsync(host + 1, ctl + size_t(k + 1) * 4 + 2, 4, cudaMemcpyDeviceToHost, s));
            GDPM_CUDA_TRY(cudaStreamSynchronize(s));
            if (host[0] == 0 && host[1] == 0) break;
            since = 0;
        }
    }
    return GDPM_OK;
}

// The same phases as run_phases, driven on the device: one launch of a
// CUDA graph whose WHILE node repeats (photon phase, electron phase,
// control) until no primaries or particles are left -- no host checks, no
// per-phase launches.  The instantiated graph is kept on the runner and
// rebuilt when anything it was built for changes.  The phase count is
// read back into *k_host (pinned) when the stream reaches that point.
static int run_phases_graph(gdpm_ctx* ctx, Runner& r, const SimParams& P, const gdpm_source_state& src,
                            uint64_t first, uint64_t n, uint32_t nb_small, uint32_t nb_rem,
                            uint32_t chunk, uint32_t* k_host, uint32_t n_sub = 0,
                            uint32_t sub_batches = 0, const uint32_t* sub_first = nullptr) {
    Workspace& ws = r.ws;
    cudaStream_t s = r.stream;
    int rc;
    if ((rc = ensure(ws.loop_k, 16))) return rc;
    GDPM_CUDA_TRY(cudaMemsetAsync(ws.ctl.p, 0, size_t(ctx->max_phases + 4) * 16, s));
    GDPM_CUDA_TRY(cudaMemsetAsync(ws.loop_k.p, 0, 16, s));
    LoopArgs L = loop_args(ctx, r, P, src, first, n, nb_small, nb_rem, chunk, n_sub, sub_batches, sub_first);
    L.k = static_cast<uint32_t*>(ws.loop_k.p);
    const bool metro = L.pick != nullptr;
    // the graph holds copies of P and L: rebuild when they differ
    std::vector<unsigned char> key(sizeof(SimParams) + sizeof(LoopArgs) + 3 * sizeof(int));
    std::memcpy(key.data(), &P, sizeof(SimParams));
    std::memcpy(key.data() + sizeof(SimParams), &L, sizeof(LoopArgs));
    const int extra[3] = {ctx->block_threads, ctx->blocks_per_sm, ctx->electron_walk};
    std::memcpy(key.data() + sizeof(SimParams) + sizeof(LoopArgs), extra, sizeof(extra));
    if (!r.loop_exec || key != r.loop_key) {
        if (r.loop_exec) cudaGraphExecDestroy(r.loop_exec);
        if (r.loop_graph) cudaGraphDestroy(r.loop_graph);
        r.loop_exec = nullptr;
        r.loop_graph = nullptr;
        r.loop_key.clear();
        if ((rc = build_loop_graph(ctx, P, L, metro, &r.loop_graph, &r.loop_exec))) return rc;
        r.loop_key = key;
    }
    GDPM_CUDA_TRY(cudaGraphLaunch(r.loop_exec, s));
    GDPM_CUDA_TRY(cudaMemcpyAsync(k_host, ws.loop_k.p, 4, cudaMemcpyDeviceToHost, s));
    return GDPM_OK;
}

// Point P's batch tally at buffer `which` (0 or 1).
static void select_tally(Runner& r, SimParams& P, int which) {
    Workspace& ws = r.ws;
    P.edep = static_cast<double*>(which ? ws.edep2.p : ws.edep.p);
    P.edep_hi = static_cast<float*>(which ? ws.hi2.p : ws.hi.p);
    P.edep_lo = static_cast<float*>(which ? ws.lo2.p : ws.lo.p);
}

static void fill_stats(const unsigned long long* c, const double* l, gdpm_stats* st) {
    st->source_energy = l[L_SOURCE];
    st->deposited = l[L_DEPOSITED];
    st->escaped = l[L_ESCAPED];
    st->discarded = l[L_DISCARDED];
    st->n_primary = int64_t(c[C_PRIMARY]);
    st->ph_created = int64_t(c[C_PH_CREATED]);
    st->ph_terminated = int64_t(c[C_PH_TERMINATED]);
    st->ph_flights = int64_t(c[C_PH_FLIGHTS]);
    st->ph_real = int64_t(c[C_PH_REAL]);
    st->compton = int64_t(c[C_COMPTON]);
    st->photoelectric = int64_t(c[C_PHOTO]);
    st->pair = int64_t(c[C_PAIR]);
    st->el_created = int64_t(c[C_EL_CREATED]);
    st->el_terminated = int64_t(c[C_EL_TERMINATED]);
    st->el_steps = int64_t(c[C_EL_STEPS]);
    st->moller = int64_t(c[C_MOLLER]);
    st->brems = int64_t(c[C_BREMS]);
    st->annihilations = int64_t(c[C_ANNIHIL]);
    st->local_deposits = int64_t(c[C_LOCAL_DEP]);
    st->pushes[0] = int64_t(c[C_PUSH_PH]);
    st->pushes[1] = int64_t(c[C_PUSH_EL]);
    st->pops[0] = int64_t(c[C_POP_PH]);
    st->pops[1] = int64_t(c[C_POP_EL]);
    st->crossings = int64_t(c[C_CROSS]);
    double dmax;
    std::memcpy(&dmax, &l[L_DMAX], 8);
    st->dmax = dmax;
    st->sigma_over_dmax = (l[L_SIGCNT] > 0 && dmax > 0) ? l[L_SIGSUM] / l[L_SIGCNT] / dmax : 0.0;
}

// One dose calculation on runner r.
int simulate_impl(gdpm_ctx* ctx, Runner& r, gdpm_phantom* ph, gdpm_tables* tb,
                  const gdpm_source_state& src, uint32_t request_id, uint64_t n_hist, int n_batches,
                  double* dose_out, double* sigma_out, gdpm_stats* st, int32_t* hrec, double* hrecd) {
    Range range("gdpm_simulate");
    int rc = validate_run(ctx, ph, tb, src, n_hist, n_batches);
    if (rc) return rc;
    cudaStream_t s = r.stream;
    const size_t V = size_t(ph->nx) * ph->ny * ph->nz;
    const bool conc = side_by_side(ctx, V, n_hist, n_batches);
    const uint32_t nb_small = uint32_t(n_hist / n_batches), nb_rem = uint32_t(n_hist % n_batches);
    uint32_t chunk = conc ? chunk_of(ctx, n_hist, 1, true, r.serving)
                          : chunk_of(ctx, n_hist, n_batches, false, r.serving);
    const uint32_t cap = capacity_of(ctx, chunk);
    const int n_bins = int(src.weights.size());
    if ((rc = prepare_workspace(ctx, r, V, cap, chunk, n_batches, n_bins, conc))) return rc;
    Workspace& ws = r.ws;
    SimParams P = base_params(ctx, ph, tb, request_id);
    if ((rc = get_majorant(ctx, s, ph, tb, &P.maj))) return rc;
    // spectrum allotment of every batch
    std::vector<uint32_t> prefix(size_t(n_batches) * (n_bins + 1));
    for (int b = 0; b < n_batches; ++b) {
        const uint64_t nb = n_hist / n_batches + (uint64_t(b) < n_hist % n_batches ? 1 : 0);
        allot_prefix(src.weights, nb, &prefix[size_t(b) * (n_bins + 1)]);
    }
    GDPM_CUDA_TRY(cudaMemcpyAsync(ws.prefix.p, prefix.data(), prefix.size() * 4, cudaMemcpyHostToDevice, s));
    ws.prefix_n = uint32_t(prefix.size());
    if ((rc = source_upload(r, src, P.S))) return rc;
    int64_t aux = 0;          // launches besides the transport phases
    if (P.S.sampler == GDPM_SAMPLE_METROPOLIS && P.S.n_beamlets > 0) {
        if ((rc = ensure(ws.chains, size_t(P.S.n_chains) * 4)) || (rc = ensure(ws.pick, size_t(chunk) * 4)))
            return rc;
        if ((rc = launch_metropolis_init(s, P, static_cast<uint32_t*>(ws.chains.p)))) return rc;
        ++aux;
    }
    P.counters = static_cast<unsigned long long*>(ws.counters.p);
    P.ledger = static_cast<double*>(ws.ledger.p);
    P.status = static_cast<uint32_t*>(ws.status.p);
    P.hrec = hrec;
    P.hrecd = hrecd;
    P.n_records = hrec ? ctx->hrec_n : 0;
    GDPM_CUDA_TRY(cudaMemsetAsync(ws.s1.p, 0, V * 8, s));
    GDPM_CUDA_TRY(cudaMemsetAsync(ws.s2.p, 0, V * 8, s));
    const size_t grids = V * size_t(n_batches) * 8;
    if (conc) {
        // the previous calculation's fold cleared the grids it read
        if (ws.edep_zero < grids) GDPM_CUDA_TRY(cudaMemsetAsync(ws.edep.p, 0, grids, s));
    } else if (ctx->tally_mode == 0) {
        GDPM_CUDA_TRY(cudaMemsetAsync(ws.edep.p, 0, V * 8, s));
        GDPM_CUDA_TRY(cudaMemsetAsync(ws.edep2.p, 0, V * 8, s));
    } else {
        GDPM_CUDA_TRY(cudaMemsetAsync(ws.hi.p, 0, V * 4, s));
        GDPM_CUDA_TRY(cudaMemsetAsync(ws.lo.p, 0, V * 4, s));
        GDPM_CUDA_TRY(cudaMemsetAsync(ws.hi2.p, 0, V * 4, s));
        GDPM_CUDA_TRY(cudaMemsetAsync(ws.lo2.p, 0, V * 4, s));
    }
    GDPM_CUDA_TRY(cudaMemsetAsync(ws.counters.p, 0, C_NCOUNT * 8, s));
    GDPM_CUDA_TRY(cudaMemsetAsync(ws.ledger.p, 0, L_NLEDGER * 8, s));
    GDPM_CUDA_TRY(cudaMemsetAsync(ws.status.p, 0, 16, s));
    if (hrec) {
        GDPM_CUDA_TRY(cudaMemsetAsync(hrec, 0, n_hist * 16, s));
        GDPM_CUDA_TRY(cudaMemsetAsync(hrecd, 0, n_hist * 16, s));
    }
    r.prof_kind.clear();
    GDPM_CUDA_TRY(cudaEventRecord(r.ev0, s));
    int64_t phases = 0;
    const uint32_t* graph_k = nullptr;   // device-driven loop: its phase count lands here
    int run_rc = GDPM_OK;
    if (conc) {
        // all batches side by side: particles carry their batch, each batch
        // has its own grid; one fold at the end
        P.batch_stride = V;
        P.tally_hi = V * uint64_t(n_batches);
        P.edep = static_cast<double*>(ws.edep.p);
        P.edep_hi = static_cast<float*>(ws.edep.p);
        P.edep_lo = static_cast<float*>(ws.edep.p) + V * size_t(n_batches);
        if (ctx->use_graph && !ctx->profile) {
            uint32_t* kh = reinterpret_cast<uint32_t*>(static_cast<unsigned char*>(ws.pinned_host.p) + 32);
            run_rc = run_phases_graph(ctx, r, P, src, 0, n_hist, nb_small, nb_rem, chunk, kh);
            graph_k = kh;
            ++aux;                                  // the graph launch
        } else {
            run_rc = run_phases(ctx, r, P, src, 0, n_hist, nb_small, nb_rem, chunk, phases, aux);
        }
        ++aux;
        if (run_rc == GDPM_OK) {
            const size_t pi = prof_begin(ctx, r, s, 2);
            run_rc = launch_fold_batches(ctx, s, P, V, n_batches, nb_small, nb_rem,
                                         static_cast<double*>(ws.s1.p), static_cast<double*>(ws.s2.p));
            prof_end(ctx, r, s, pi);
        }
    } else {
        // Batch b tallies into buffer b%2.  Its fold runs on the side stream
        // while batch b+1 transports into the other buffer; batch b+2 waits
        // for that fold before reusing the buffer.
        cudaStream_t side = ctx->overlap_fold ? r.side : s;
        GDPM_CUDA_TRY(cudaEventRecord(r.fold_done[0], s));
        GDPM_CUDA_TRY(cudaEventRecord(r.fold_done[1], s));
        uint64_t first = 0;
        for (int b = 0; b < n_batches && run_rc == GDPM_OK; ++b) {
            const uint64_t nb = n_hist / n_batches + (uint64_t(b) < n_hist % n_batches ? 1 : 0);
            const int buf = ctx->overlap_fold ? (b & 1) : 0;
            select_tally(r, P, buf);
            GDPM_CUDA_TRY(cudaStreamWaitEvent(s, r.fold_done[buf], 0));
            run_rc = run_phases(ctx, r, P, src, first, nb, nb_small, nb_rem, chunk, phases, aux);
            ++aux;
            if (run_rc == GDPM_OK) {
                GDPM_CUDA_TRY(cudaEventRecord(r.batch_done[buf], s));
                GDPM_CUDA_TRY(cudaStreamWaitEvent(side, r.batch_done[buf], 0));
                const size_t pi = prof_begin(ctx, r, side, 2);
                run_rc = launch_fold_into(ctx, side, P, V, uint32_t(nb), static_cast<double*>(ws.s1.p),
                                          static_cast<double*>(ws.s2.p));
                prof_end(ctx, r, side, pi);
                GDPM_CUDA_TRY(cudaEventRecord(r.fold_done[buf], side));
            }
            first += nb;
        }
        GDPM_CUDA_TRY(cudaStreamWaitEvent(s, r.fold_done[0], 0));
        GDPM_CUDA_TRY(cudaStreamWaitEvent(s, r.fold_done[1], 0));
    }
    GDPM_CUDA_TRY(cudaEventRecord(r.ev1, s));
    if (run_rc != GDPM_OK) {
        cudaStreamSynchronize(s);
        cudaStreamSynchronize(r.side);
        r.prof_kind.clear();
        return run_rc;
    }
    // results: straight into device outputs, or via staging for host outputs
    const bool dev_out = dose_out && sigma_out && is_device_ptr(dose_out) && is_device_ptr(sigma_out);
    double *dd = dose_out, *ds = sigma_out;
    if (!dev_out) {
        if ((rc = ensure(ws.stage, V * 16))) {
            cudaStreamSynchronize(s);       // the fold may still be clearing the grids
            return rc;
        }
        dd = static_cast<double*>(ws.stage.p);
        ds = dd + V;
    }
    if ((rc = launch_finalize_into(ctx, s, P, V, n_batches, static_cast<const double*>(ws.s1.p),
                                   static_cast<const double*>(ws.s2.p), dd, ds))) {
        cudaStreamSynchronize(s);
        return rc;
    }
    if (!dev_out) {
        if (dose_out) GDPM_CUDA_TRY(cudaMemcpyAsync(dose_out, dd, V * 8, cudaMemcpyDefault, s));
        if (sigma_out) GDPM_CUDA_TRY(cudaMemcpyAsync(sigma_out, ds, V * 8, cudaMemcpyDefault, s));
    }
    unsigned char* h = static_cast<unsigned char*>(ws.pinned_host.p);
    unsigned long long* hc = reinterpret_cast<unsigned long long*>(h + 64);
    double* hl = reinterpret_cast<double*>(h + 64 + C_NCOUNT * 8);
    uint32_t* hs = reinterpret_cast<uint32_t*>(h + 64 + C_NCOUNT * 8 + L_NLEDGER * 8);
    GDPM_CUDA_TRY(cudaMemcpyAsync(hc, ws.counters.p, C_NCOUNT * 8, cudaMemcpyDeviceToHost, s));
    GDPM_CUDA_TRY(cudaMemcpyAsync(hl, ws.ledger.p, L_NLEDGER * 8, cudaMemcpyDeviceToHost, s));
    GDPM_CUDA_TRY(cudaMemcpyAsync(hs, ws.status.p, 4, cudaMemcpyDeviceToHost, s));
    GDPM_CUDA_TRY(cudaStreamSynchronize(s));
    if (conc) ws.edep_clean = grids;        // the fold has cleared every grid of this calculation
    if (st) {
        std::memset(st, 0, sizeof(*st));
        fill_stats(hc, hl, st);
        if (graph_k) phases = int64_t(*graph_k);
        st->phases = phases;
        st->launches = phases + aux + 2;    // + finalize and metric
        float ms = 0;
        cudaEventElapsedTime(&ms, r.ev0, r.ev1);
        st->transport_ms = ms;
    }
    prof_collect(r, st);
    if (*hs & ST_BOUNDS) return GDPM_E_BOUNDS;
    if (*hs & ST_QUEUE_OVERFLOW) return GDPM_E_QUEUE_OVERFLOW;
    if (*hs & (ST_ITER_CAP | ST_PHASE_CAP)) return GDPM_E_TIMEOUT;
    return GDPM_OK;
}

// ------------------------------------------------------------------ serving
// Each slot is a host thread with its own runner (streams, buffers).  Slots
// have a class: the first serve_big_slots take large requests (more than
// serve_small_hist histories) in arrival order and run them on the whole
// GPU, one at a time per slot; the other slots take small requests, which
// therefore never wait behind a large one.  While a small request runs,
// large requests launch their phases on serve_share8 eighths of the SMs (7
// by default) and the small one runs on a high-priority stream, so it gets
// the SMs left free.  A request is
// admitted when its slot is free and device memory allows (continuous
// batching: requests join as they arrive, their work overlaps on the GPU).
// Result buffers of served requests come from a pool: cudaFree synchronizes
// the whole device, which would make every poll wait for the other requests.
static int result_acquire(gdpm_ctx* ctx, size_t bytes, Buffer& out) {
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        for (size_t k = 0; k < ctx->result_pool.size(); ++k) {
            if (ctx->result_pool[k].bytes >= bytes) {
                out = ctx->result_pool[k];
                ctx->result_pool.erase(ctx->result_pool.begin() + k);
                return GDPM_OK;
            }
        }
    }
    return ensure(out, bytes);
}
static void result_release(gdpm_ctx* ctx, Buffer& b) {
    if (!b.p) return;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->result_pool.push_back(b);
    b.p = nullptr;
    b.bytes = 0;
}

// slot_class: 0 any request, 1 large requests, 2 small requests
static void serve_worker(gdpm_ctx* ctx, int slot_class) {
    cudaSetDevice(ctx->device);
    Runner r;
    const int init_rc = runner_init(r, nullptr, true);
    r.serving = true;
    for (;;) {
        gdpm_request* q = nullptr;
        bool refused = false;
        {
            std::unique_lock<std::mutex> lk(ctx->mu);
            for (;;) {
                // the oldest pending request of this slot's class
                auto mine = [&]() {
                    for (auto it = ctx->pending.begin(); it != ctx->pending.end(); ++it)
                        if (slot_class == 0 ||
                            ((*it)->desc.n_histories > ctx->serve_small_hist) == (slot_class == 1))
                            return it;
                    return ctx->pending.end();
                };
                ctx->cv.wait(lk, [&] { return ctx->stop || mine() != ctx->pending.end(); });
                if (ctx->stop) break;
                auto it = mine();
                gdpm_request* front = *it;
                const gdpm_phantom* ph = front->desc.phantom;
                const size_t V = size_t(ph->nx) * ph->ny * ph->nz;
                const size_t need = bytes_needed(ctx, r, V, front->desc.n_histories, front->desc.n_batches, true);
                size_t free_b = 0, total_b = 0;
                if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) cudaGetLastError();
                if (total_b > 0 && need + ctx->serve_reserve > total_b) {
                    // larger than the device can ever hold with the reserve: refuse
                    ctx->pending.erase(it);
                    q = front;
                    refused = true;
                    ++ctx->running;
                    break;
                }
                if (ctx->running > 0 && free_b < need + ctx->serve_reserve) {
                    // not admitted yet: wait for a running request to finish
                    ctx->cv.wait_for(lk, std::chrono::milliseconds(2));
                    continue;
                }
                ctx->pending.erase(it);
                q = front;
                ++ctx->running;
                break;
            }
            if (ctx->stop) break;
        }
        int rc = refused ? GDPM_E_NOMEM : init_rc;
        if (rc == GDPM_OK) {
            const gdpm_phantom* ph = q->desc.phantom;
            const size_t V = size_t(ph->nx) * ph->ny * ph->nz;
            rc = result_acquire(ctx, V * 16, q->result);
            if (rc == GDPM_OK) {
                double* d = static_cast<double*>(q->result.p);
                const uint32_t sid = q->desc.stream_id ? q->desc.stream_id : uint32_t(q->id);
                // small requests on the high-priority stream: their CTAs get
                // SMs first whenever a large request's CTAs finish
                r.small = q->desc.n_histories <= ctx->serve_small_hist;
                r.stream = r.small ? r.prio_hi : r.prio_lo;
                if (r.small) ++ctx->small_running;
                rc = simulate_impl(ctx, r, q->desc.phantom, q->desc.tables, q->src, sid,
                                   q->desc.n_histories, q->desc.n_batches, d, d + V, &q->stats,
                                   nullptr, nullptr);
                if (r.small) --ctx->small_running;
                r.small = false;
            }
        }
        {
            std::lock_guard<std::mutex> lk(ctx->mu);
            q->status = rc;
            --ctx->running;
        }
        ctx->cv.notify_all();
    }
    runner_free(r);
}

}  // namespace gdpm

using namespace gdpm;

extern "C" {

const char* gdpm_strerror(int code) {
    switch (code) {
    case GDPM_OK: return "ok";
    case GDPM_E_ARG: return "invalid argument";
    case GDPM_E_NOMEM: return "device memory allocation failed";
    case GDPM_E_QUEUE_OVERFLOW: return "secondary particle queue overflow";
    case GDPM_E_TIMEOUT: return "phase or iteration cap reached";
    case GDPM_E_CUDA: return cudaGetErrorString(last_cuda_error());
    case GDPM_E_STATE: return "call not valid in the current state";
    case GDPM_E_BUSY: return "request not admitted";
    case GDPM_E_BOUNDS: return "checked build: an index was out of range";
    }
    return "unknown status";
}

int gdpm_context_create(gdpm_ctx** out, int device, void* cuda_stream, uint64_t seed) {
    if (!out) return GDPM_E_ARG;
    *out = nullptr;
    int n = 0;
    GDPM_CUDA_TRY(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return GDPM_E_ARG;
    GDPM_CUDA_TRY(cudaSetDevice(device));
    gdpm_ctx* c = new gdpm_ctx();
    c->device = device;
    c->seed = seed;
    cudaDeviceProp prop{};
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        last_cuda_error() = cudaGetLastError();
        delete c;
        return GDPM_E_CUDA;
    }
    c->sm_count = prop.multiProcessorCount;
    // default phase length of side-by-side runs: the largest power of two up
    // to 2^25 primaries whose queues (three of capacity_of(chunk) slots and
    // the source queue) take at most a quarter of the device's memory
    {
        const double per_primary = (3.0 * 8.0 * kQueueWords + kSourceWords) * 4;
        uint32_t ch = 1u << 25;
        while (ch > (1u << 20) && per_primary * ch > 0.25 * double(prop.totalGlobalMem)) ch >>= 1;
        c->auto_chunk = ch;
    }
    const int rc = runner_init(c->run, static_cast<cudaStream_t>(cuda_stream), false);
    if (rc) {
        runner_free(c->run);
        delete c;
        return rc;
    }
    c->stream = c->run.stream;
    c->ev0 = c->run.ev0;
    c->ev1 = c->run.ev1;
    *out = c;
    return GDPM_OK;
}

int gdpm_context_destroy(gdpm_ctx* ctx) {
    if (!ctx) return GDPM_E_ARG;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->stop = true;
    }
    ctx->cv.notify_all();
    for (std::thread& t : ctx->workers)
        if (t.joinable()) t.join();
    cudaSetDevice(ctx->device);
    for (auto& kv : ctx->requests) release(kv.second->result);
    for (Buffer& b : ctx->result_pool) release(b);
    release(ctx->atab_cache);
    runner_free(ctx->run);
    delete ctx;
    return GDPM_OK;
}

int gdpm_set_param(gdpm_ctx* ctx, int param, double v) {
    if (!ctx) return GDPM_E_ARG;
    switch (param) {
    case GDPM_PARAM_QUEUE_CAPACITY:
        // a phase's work indices (primaries + queued particles) are 32-bit
        if (v < 0 || v > 2147483648.0) return GDPM_E_ARG;
        ctx->queue_capacity = uint32_t(v);
        return GDPM_OK;
    case GDPM_PARAM_BLOCK_THREADS:
        if (v != 0 && (v < 64 || v > 256 || int(v) % 32)) return GDPM_E_ARG;
        ctx->block_threads = int(v);
        return GDPM_OK;
    case GDPM_PARAM_BLOCKS_PER_SM:
        if (v < 0 || v > 32) return GDPM_E_ARG;
        ctx->blocks_per_sm = int(v);
        return GDPM_OK;
    case GDPM_PARAM_TALLY_MODE:
        if (v != 0 && v != 1) return GDPM_E_ARG;
        ctx->tally_mode = int(v);
        return GDPM_OK;
    case GDPM_PARAM_SOURCE_CHUNK:
        // the automatic queue capacity, 8 x chunk + 65536, must stay 32-bit
        if (v < 0 || v > 268435456.0) return GDPM_E_ARG;
        ctx->source_chunk = uint32_t(v);
        return GDPM_OK;
    case GDPM_PARAM_MAX_PHASES:
        if (v < 8 || v > 1e6) return GDPM_E_ARG;
        ctx->max_phases = int(v);
        return GDPM_OK;
    case GDPM_PARAM_REQUEST_ID:
        if (v < 0 || v > 4294967295.0) return GDPM_E_ARG;
        ctx->request_id = uint32_t(v);
        return GDPM_OK;
    case GDPM_PARAM_GRAPH:
        if (v != 0 && v != 1) return GDPM_E_ARG;
        ctx->use_graph = int(v);
        return GDPM_OK;
    case GDPM_PARAM_ELECTRON_WALK:
        if (v != 0 && v != 1 && v != 2) return GDPM_E_ARG;
        ctx->electron_walk = int(v);
        return GDPM_OK;
    case GDPM_PARAM_MAX_ITERS:
        if (v < 1 || v > 2147483648.0) return GDPM_E_ARG;
        ctx->max_iters = uint32_t(v);
        return GDPM_OK;
    case GDPM_PARAM_SPECULATIVE:
        if (v < 1 || v > 64) return GDPM_E_ARG;
        ctx->speculative = int(v);
        return GDPM_OK;
    case GDPM_PARAM_PROFILE:
        if (v != 0 && v != 1) return GDPM_E_ARG;
        ctx->profile = int(v);
        return GDPM_OK;
    case GDPM_PARAM_OVERLAP_FOLD:
        if (v != 0 && v != 1) return GDPM_E_ARG;
        ctx->overlap_fold = int(v);
        return GDPM_OK;
    case GDPM_PARAM_SERVE_SLOTS: {
        if (v < 1 || v > 16) return GDPM_E_ARG;
        std::lock_guard<std::mutex> lk(ctx->mu);
        if (!ctx->workers.empty()) return GDPM_E_STATE;
        ctx->serve_slots = int(v);
        return GDPM_OK;
    }
    case GDPM_PARAM_SERVE_BIG_SLOTS: {
        if (v < 1 || v > 15) return GDPM_E_ARG;
        std::lock_guard<std::mutex> lk(ctx->mu);
        if (!ctx->workers.empty()) return GDPM_E_STATE;
        ctx->serve_big_slots = int(v);
        return GDPM_OK;
    }
    case GDPM_PARAM_SERVE_SMALL_HIST:
        if (v < 0 || v > 4.0e9) return GDPM_E_ARG;
        ctx->serve_small_hist = uint64_t(v);
        return GDPM_OK;
    case GDPM_PARAM_SERVE_PHASE_CAP:
        if (v < 0 || v > double(1u << 28)) return GDPM_E_ARG;
        ctx->serve_phase_cap = uint32_t(v);
        return GDPM_OK;
    case GDPM_PARAM_SERVE_SHARE:
        if (v < 1 || v > 8 || v != double(int(v))) return GDPM_E_ARG;
        ctx->serve_share8 = int(v);
        return GDPM_OK;
    case GDPM_PARAM_METRIC_MIN_DENSITY:
        if (v < 0 || v > 100) return GDPM_E_ARG;
        ctx->metric_min_rho = float(v);
        return GDPM_OK;
    case GDPM_PARAM_BATCH_MODE:
        if (v != 0 && v != 1 && v != 2) return GDPM_E_ARG;
        ctx->batch_mode = int(v);
        return GDPM_OK;
    case GDPM_PARAM_CONCURRENT_MAX_HIST:
        if (v < 0 || v > 4.0e9) return GDPM_E_ARG;
        ctx->concurrent_max_hist = uint64_t(v);
        return GDPM_OK;
    case GDPM_PARAM_CONCURRENT_MAX_MB:
        if (v < 0 || v > 1e7) return GDPM_E_ARG;
        ctx->concurrent_max_bytes = size_t(v) << 20;
        return GDPM_OK;
    case GDPM_PARAM_SERVE_RESERVE_MB:
        if (v < 0 || v > 1e7) return GDPM_E_ARG;
        ctx->serve_reserve = size_t(v) << 20;
        return GDPM_OK;
    }
    return GDPM_E_ARG;
}

int gdpm_phantom_create(gdpm_ctx* ctx, int nx, int ny, int nz, float dx, float dy, float dz,
                        const uint8_t* material, const float* density, gdpm_phantom** out) {
    if (!ctx || !out || !material || !density) return GDPM_E_ARG;
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1 || nx > 1024 || ny > 1024 || nz > 1024) return GDPM_E_ARG;
    if (!(dx > 0) || !(dy > 0) || !(dz > 0)) return GDPM_E_ARG;
    GDPM_CUDA_TRY(cudaSetDevice(ctx->device));
    gdpm_phantom* ph = new gdpm_phantom();
    ph->ctx = ctx;
    ph->nx = nx; ph->ny = ny; ph->nz = nz;
    ph->dx = dx; ph->dy = dy; ph->dz = dz;
    const size_t V = size_t(nx) * ny * nz;
    int rc;
    if ((rc = ensure(ph->mat, V)) || (rc = ensure(ph->rho, V * 4))) {
        gdpm_phantom_destroy(ph);
        return rc;
    }
    if (cudaMemcpyAsync(ph->mat.p, material, V, cudaMemcpyDefault, ctx->stream) != cudaSuccess ||
        cudaMemcpyAsync(ph->rho.p, density, V * 4, cudaMemcpyDefault, ctx->stream) != cudaSuccess) {
        last_cuda_error() = cudaGetLastError();
        gdpm_phantom_destroy(ph);
        return GDPM_E_CUDA;
    }
    if ((rc = phantom_density_max(ctx, ph))) {
        gdpm_phantom_destroy(ph);
        return rc;
    }
    *out = ph;
    return GDPM_OK;
}

int gdpm_phantom_destroy(gdpm_phantom* ph) {
    if (!ph) return GDPM_E_ARG;
    if (ph->ctx) cudaStreamSynchronize(ph->ctx->stream);
    release(ph->mat);
    release(ph->rho);
    release(ph->rhomax);
    for (auto& kv : ph->maj) release(kv.second);
    delete ph;
    return GDPM_OK;
}

int gdpm_tables_build(gdpm_ctx* ctx, const gdpm_material_desc* mats, int n_mats, double e_min,
                      double e_max, int n_energy, double eabs_photon, double eabs_electron,
                      double ms_loss, int flags, gdpm_tables** out) {
    if (!ctx || !mats || !out) return GDPM_E_ARG;
    *out = nullptr;
    if (n_mats < 1 || n_mats > GDPM_MAX_MATERIALS || n_energy < 16 || n_energy > 8192) return GDPM_E_ARG;
    if (!(e_min > 0) || !(e_max > e_min * 1.01)) return GDPM_E_ARG;
    if (!(eabs_photon >= e_min) || !(eabs_electron >= e_min / 0.5) || eabs_electron >= e_max ||
        eabs_photon >= e_max || !(ms_loss > 0 && ms_loss < 0.9))
        return GDPM_E_ARG;
    if (flags & ~(GDPM_FLAG_COMPTON_ONLY | GDPM_FLAG_NO_HARD | GDPM_FLAG_SAUTER)) return GDPM_E_ARG;
    for (int m = 0; m < n_mats; ++m) {
        const gdpm_material_desc& d = mats[m];
        if (d.n_elements < 1 || d.n_elements > GDPM_MAX_ELEMENTS || !(d.mean_excitation_MeV > 0))
            return GDPM_E_ARG;
        double ws = 0;
        for (int i = 0; i < d.n_elements; ++i) {
            if (d.Z[i] < 1 || d.Z[i] > 100 || !(d.A[i] > 0) || d.mass_fraction[i] < 0) return GDPM_E_ARG;
            ws += d.mass_fraction[i];
        }
        if (!(ws > 0)) return GDPM_E_ARG;
    }
    GDPM_CUDA_TRY(cudaSetDevice(ctx->device));
    gdpm_tables* t = new gdpm_tables();
    t->ctx = ctx;
    t->id = ctx->next_tables_id++;
    t->n_mat = n_mats;
    t->n_e = n_energy;
    t->e_min = e_min; t->e_max = e_max;
    t->eabs_ph = eabs_photon; t->eabs_el = eabs_electron;
    t->ms_loss = ms_loss;
    t->flags = flags;
    const int rc = build_tables_device(ctx, t, mats);
    if (rc) {
        gdpm_tables_destroy(t);
        return rc;
    }
    if (transport_smem(t, GDPM_ELECTRON) > 200 * 1024 || transport_smem(t, GDPM_PHOTON) > 200 * 1024) {
        gdpm_tables_destroy(t);
        return GDPM_E_ARG;
    }
    *out = t;
    return GDPM_OK;
}

int gdpm_tables_destroy(gdpm_tables* t) {
    if (!t) return GDPM_E_ARG;
    if (t->ctx) cudaStreamSynchronize(t->ctx->stream);
    release(t->ph_tot); release(t->ph_cum); release(t->el); release(t->rinv); release(t->atab);
    delete t;
    return GDPM_OK;
}

int gdpm_source_set(gdpm_ctx* ctx, const gdpm_source_desc* s) {
    if (!ctx || !s) return GDPM_E_ARG;
    gdpm_source_state st;
    const int rc = source_copy(s, st);
    if (rc) return rc;
    ctx->src = std::move(st);
    return GDPM_OK;
}

int gdpm_set_history_records(gdpm_ctx* ctx, int32_t* rec, double* recd, uint64_t n) {
    if (!ctx) return GDPM_E_ARG;
    if ((rec == nullptr) != (recd == nullptr)) return GDPM_E_ARG;
    if (rec && (!is_device_ptr(rec) || !is_device_ptr(recd) || n == 0)) return GDPM_E_ARG;
    ctx->hrec = rec;
    ctx->hrecd = recd;
    ctx->hrec_n = rec ? n : 0;
    return GDPM_OK;
}

int gdpm_simulate(gdpm_ctx* ctx, gdpm_phantom* ph, gdpm_tables* tb, uint64_t n_histories,
                  int n_batches, double* dose_out, double* sigma_out, gdpm_stats* stats_out) {
    if (!ctx) return GDPM_E_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return GDPM_E_CUDA;
    if (ctx->hrec && ctx->hrec_n < n_histories) return GDPM_E_ARG;
    return simulate_impl(ctx, ctx->run, ph, tb, ctx->src, ctx->request_id, n_histories, n_batches,
                         dose_out, sigma_out, stats_out, ctx->hrec, ctx->hrecd);
}

int gdpm_simulate_to_precision(gdpm_ctx* ctx, gdpm_phantom* ph, gdpm_tables* tb, double target,
                               uint64_t n_pilot, uint64_t n_max, int n_batches, double* dose_out,
                               double* sigma_out, gdpm_stats* stats_out, uint64_t* n_total_out) {
    if (!ctx || !(target > 0.0) || n_batches < 2 || n_pilot < uint64_t(n_batches) || n_max < n_pilot ||
        n_max >= (1ull << 32))
        return GDPM_E_ARG;
    if (ctx->hrec) return GDPM_E_STATE;          // per-history records describe a single run
    if (cudaSetDevice(ctx->device) != cudaSuccess) return GDPM_E_CUDA;
    Range range("gdpm_simulate_to_precision");
    gdpm_stats st{};
    uint64_t n = n_pilot, total = 0;
    for (int round = 0; round < 8; ++round) {
        const int rc = simulate_impl(ctx, ctx->run, ph, tb, ctx->src, ctx->request_id, n, n_batches,
                                     dose_out, sigma_out, &st, nullptr, nullptr);
        if (rc) return rc;
        total += n;
        const double sg = st.sigma_over_dmax;
        if (!(sg > 0.0) || sg <= target || n >= n_max) break;
        // sigma/Dmax falls as N^(-1/2): the histories that reach the target.
        // A small pilot reads sigma/Dmax low (noise inflates Dmax and shrinks
        // the D > 0.5 Dmax region): 5e7-history pilots predicted 13 % (6 MV
        // slab) and 24 % (CT plan) too few histories, so the first step takes
        // 40 % to spare; later steps, from large runs, take 5 %.
        const double margin = round == 0 ? 1.4 : 1.05;
        const double want = std::ceil(double(n) * (sg / target) * (sg / target) * margin);
        n = want >= double(n_max) ? n_max : std::max<uint64_t>(uint64_t(want), n + 1);
    }
    if (stats_out) *stats_out = st;
    if (n_total_out) *n_total_out = total;
    return GDPM_OK;
}

int gdpm_simulate_part(gdpm_ctx* ctx, gdpm_phantom* ph, gdpm_tables* tb, uint64_t n_histories,
                       int n_batches, int first_batch, int n_part, double* sum1, double* sum2,
                       gdpm_stats* st) {
    if (!ctx || !sum1 || !sum2) return GDPM_E_ARG;
    Range range("gdpm_simulate_part");
    const gdpm_source_state& src = ctx->src;
    int rc = validate_run(ctx, ph, tb, src, n_histories, n_batches);
    if (rc) return rc;
    if (first_batch < 0 || n_part < 1 || first_batch + n_part > n_batches || n_part > kMaxConcurrentBatches)
        return GDPM_E_ARG;
    GDPM_CUDA_TRY(cudaSetDevice(ctx->device));
    Runner& r = ctx->run;
    cudaStream_t s = r.stream;
    const size_t V = size_t(ph->nx) * ph->ny * ph->nz;
    const uint32_t nb_small = uint32_t(n_histories / n_batches), nb_rem = uint32_t(n_histories % n_batches);
    // batch b holds histories [h(b), h(b+1)), h(b) = b nb_small + min(b, nb_rem)
    auto hb = [&](uint64_t b) { return b * nb_small + std::min<uint64_t>(b, nb_rem); };
    const uint64_t h0 = hb(uint64_t(first_batch)), h1 = hb(uint64_t(first_batch + n_part));
    const uint32_t chunk = chunk_of(ctx, h1 - h0, 1, true);
    const uint32_t cap = capacity_of(ctx, chunk);
    const int n_bins = int(src.weights.size());
    if ((rc = prepare_workspace(ctx, r, V, cap, chunk, n_part, n_bins, true))) return rc;
    Workspace& ws = r.ws;
    SimParams P = base_params(ctx, ph, tb, ctx->request_id);
    if ((rc = get_majorant(ctx, s, ph, tb, &P.maj))) return rc;
    // spectrum allotment of every batch of the whole calculation (the
    // primaries find theirs by their global history id)
    std::vector<uint32_t> prefix(size_t(n_batches) * (n_bins + 1));
    for (int b = 0; b < n_batches; ++b)
        allot_prefix(src.weights, hb(b + 1) - hb(b), &prefix[size_t(b) * (n_bins + 1)]);
    if ((rc = ensure(ws.prefix, prefix.size() * 4))) return rc;
    GDPM_CUDA_TRY(cudaMemcpyAsync(ws.prefix.p, prefix.data(), prefix.size() * 4, cudaMemcpyHostToDevice, s));
    ws.prefix_n = uint32_t(prefix.size());
    if ((rc = source_upload(r, src, P.S))) return rc;
    int64_t aux = 0;
    if (P.S.sampler == GDPM_SAMPLE_METROPOLIS && P.S.n_beamlets > 0) {
        // the chains run from their start through the histories before h0
        if ((rc = ensure(ws.chains, size_t(P.S.n_chains) * 4)) ||
            (rc = ensure(ws.pick, std::max<size_t>(size_t(chunk), h0) * 4)))
            return rc;
        uint32_t* chains = static_cast<uint32_t*>(ws.chains.p);
        if ((rc = launch_metropolis_init(s, P, chains))) return rc;
        if (h0 > 0 && (rc = launch_metropolis(s, P, 0, uint32_t(h0), chains, static_cast<uint32_t*>(ws.pick.p))))
            return rc;
        aux += 2;
    }
    P.counters = static_cast<unsigned long long*>(ws.counters.p);
    P.ledger = static_cast<double*>(ws.ledger.p);
    P.status = static_cast<uint32_t*>(ws.status.p);
    // the part's grids hold batches first_batch.. as slots 0..n_part-1
    const uintptr_t shift = uintptr_t(first_batch) * V;
    P.batch_stride = V;
    P.tally_lo = uint64_t(first_batch) * V;
    P.tally_hi = uint64_t(first_batch + n_part) * V;
    P.edep = reinterpret_cast<double*>(reinterpret_cast<uintptr_t>(ws.edep.p) - shift * 8);
    P.edep_hi = reinterpret_cast<float*>(reinterpret_cast<uintptr_t>(ws.edep.p) - shift * 4);
    P.edep_lo = reinterpret_cast<float*>(reinterpret_cast<uintptr_t>(ws.edep.p) + (V * size_t(n_part) - shift) * 4);
    GDPM_CUDA_TRY(cudaMemsetAsync(ws.edep.p, 0, V * size_t(n_part) * 8, s));
    GDPM_CUDA_TRY(cudaMemsetAsync(ws.counters.p, 0, C_NCOUNT * 8, s));
    GDPM_CUDA_TRY(cudaMemsetAsync(ws.ledger.p, 0, L_NLEDGER * 8, s));
    GDPM_CUDA_TRY(cudaMemsetAsync(ws.status.p, 0, 16, s));
    // the caller's sums, on the device for the fold
    const bool dev = is_device_ptr(sum1) && is_device_ptr(sum2);
    double *d1 = sum1, *d2 = sum2;
    if (!dev) {
        if ((rc = ensure(ws.stage, V * 16))) return rc;
        d1 = static_cast<double*>(ws.stage.p);
        d2 = d1 + V;
        GDPM_CUDA_TRY(cudaMemcpyAsync(d1, sum1, V * 8, cudaMemcpyDefault, s));
        GDPM_CUDA_TRY(cudaMemcpyAsync(d2, sum2, V * 8, cudaMemcpyDefault, s));
    }
    r.prof_kind.clear();
    GDPM_CUDA_TRY(cudaEventRecord(r.ev0, s));
    int64_t phases = 0;
    int run_rc = run_phases(ctx, r, P, src, h0, h1 - h0, nb_small, nb_rem, chunk, phases, aux);
    if (run_rc == GDPM_OK) {
        SimParams Pf = P;
        Pf.edep = static_cast<double*>(ws.edep.p);
        Pf.edep_hi = static_cast<float*>(ws.edep.p);
        Pf.edep_lo = static_cast<float*>(ws.edep.p) + V * size_t(n_part);
        const int n_big = int(std::min<int64_t>(std::max<int64_t>(int64_t(nb_rem) - first_batch, 0), n_part));
        run_rc = launch_fold_batches(ctx, s, Pf, V, n_part, nb_small, uint32_t(n_big), d1, d2);
        ++aux;
    }
    GDPM_CUDA_TRY(cudaEventRecord(r.ev1, s));
    if (run_rc != GDPM_OK) {
        cudaStreamSynchronize(s);
        r.prof_kind.clear();
        return run_rc;
    }
    if (!dev) {
        GDPM_CUDA_TRY(cudaMemcpyAsync(sum1, d1, V * 8, cudaMemcpyDefault, s));
        GDPM_CUDA_TRY(cudaMemcpyAsync(sum2, d2, V * 8, cudaMemcpyDefault, s));
    }
    unsigned char* hp = static_cast<unsigned char*>(ws.pinned_host.p);
    unsigned long long* hc = reinterpret_cast<unsigned long long*>(hp + 64);
    double* hl = reinterpret_cast<double*>(hp + 64 + C_NCOUNT * 8);
    uint32_t* hs = reinterpret_cast<uint32_t*>(hp + 64 + C_NCOUNT * 8 + L_NLEDGER * 8);
    GDPM_CUDA_TRY(cudaMemcpyAsync(hc, ws.counters.p, C_NCOUNT * 8, cudaMemcpyDeviceToHost, s));
    GDPM_CUDA_TRY(cudaMemcpyAsync(hl, ws.ledger.p, L_NLEDGER * 8, cudaMemcpyDeviceToHost, s));
    GDPM_CUDA_TRY(cudaMemcpyAsync(hs, ws.status.p, 4, cudaMemcpyDeviceToHost, s));
    GDPM_CUDA_TRY(cudaStreamSynchronize(s));
    if (st) {
        std::memset(st, 0, sizeof(*st));
        fill_stats(hc, hl, st);
        st->phases = phases;
        st->launches = phases + aux;
        float ms = 0;
        cudaEventElapsedTime(&ms, r.ev0, r.ev1);
        st->transport_ms = ms;
    }
    prof_collect(r, st);
    if (*hs & ST_BOUNDS) return GDPM_E_BOUNDS;
    if (*hs & ST_QUEUE_OVERFLOW) return GDPM_E_QUEUE_OVERFLOW;
    if (*hs & (ST_ITER_CAP | ST_PHASE_CAP)) return GDPM_E_TIMEOUT;
    return GDPM_OK;
}

int gdpm_finalize(gdpm_ctx* ctx, gdpm_phantom* ph, int n_batches, const double* sum1, const double* sum2,
                  double* dose_out, double* sigma_out, gdpm_stats* st) {
    if (!ctx || !ph || !sum1 || !sum2 || n_batches < 2) return GDPM_E_ARG;
    GDPM_CUDA_TRY(cudaSetDevice(ctx->device));
    Runner& r = ctx->run;
    cudaStream_t s = r.stream;
    const size_t V = size_t(ph->nx) * ph->ny * ph->nz;
    Workspace& ws = r.ws;
    int rc;
    if ((rc = ensure(ws.s1, V * 8)) || (rc = ensure(ws.s2, V * 8)) || (rc = ensure(ws.stage, V * 16)) ||
        (rc = ensure(ws.ledger, L_NLEDGER * 8)))
        return rc;
    if (!ws.pinned_host.p) {
        void* h = nullptr;
        GDPM_CUDA_TRY(cudaMallocHost(&h, 4096));
        ws.pinned_host.p = h;
        ws.pinned_host.bytes = 4096;
    }
    GDPM_CUDA_TRY(cudaMemcpyAsync(ws.s1.p, sum1, V * 8, cudaMemcpyDefault, s));
    GDPM_CUDA_TRY(cudaMemcpyAsync(ws.s2.p, sum2, V * 8, cudaMemcpyDefault, s));
    GDPM_CUDA_TRY(cudaMemsetAsync(ws.ledger.p, 0, L_NLEDGER * 8, s));
    SimParams P{};
    P.dx = ph->dx; P.dy = ph->dy; P.dz = ph->dz;
    P.rho = static_cast<const float*>(ph->rho.p);
    P.ledger = static_cast<double*>(ws.ledger.p);
    double* dd = static_cast<double*>(ws.stage.p);
    double* ds = dd + V;
    if ((rc = launch_finalize_into(ctx, s, P, V, n_batches, static_cast<const double*>(ws.s1.p),
                                   static_cast<const double*>(ws.s2.p), dd, ds)))
        return rc;
    if (dose_out) GDPM_CUDA_TRY(cudaMemcpyAsync(dose_out, dd, V * 8, cudaMemcpyDefault, s));
    if (sigma_out) GDPM_CUDA_TRY(cudaMemcpyAsync(sigma_out, ds, V * 8, cudaMemcpyDefault, s));
    double* hl = reinterpret_cast<double*>(static_cast<unsigned char*>(ws.pinned_host.p) + 64 + C_NCOUNT * 8);
    GDPM_CUDA_TRY(cudaMemcpyAsync(hl, ws.ledger.p, L_NLEDGER * 8, cudaMemcpyDeviceToHost, s));
    GDPM_CUDA_TRY(cudaStreamSynchronize(s));
    if (st) {
        std::memset(st, 0, sizeof(*st));
        double dmax;
        std::memcpy(&dmax, &hl[L_DMAX], 8);
        st->dmax = dmax;
        st->sigma_over_dmax = (hl[L_SIGCNT] > 0 && dmax > 0) ? hl[L_SIGSUM] / hl[L_SIGCNT] / dmax : 0.0;
        st->launches = 2;
    }
    return GDPM_OK;
}

int gdpm_autotune(gdpm_ctx* ctx, gdpm_phantom* ph, gdpm_tables* tb, uint64_t n_histories,
                  int n_batches, double budget_ms, gdpm_tune_result* out) {
    if (!ctx || !out || !(budget_ms > 0)) return GDPM_E_ARG;
    int rc = validate_run(ctx, ph, tb, ctx->src, n_histories, n_batches);
    if (rc) return rc;
    GDPM_CUDA_TRY(cudaSetDevice(ctx->device));
    const size_t V = size_t(ph->nx) * ph->ny * ph->nz;
    struct Cfg {
        int mode;          // GDPM_PARAM_BATCH_MODE
        uint32_t chunk;    // GDPM_PARAM_SOURCE_CHUNK
        int spec;          // GDPM_PARAM_SPECULATIVE
        int walk;          // GDPM_PARAM_ELECTRON_WALK
        int threads;       // GDPM_PARAM_BLOCK_THREADS
        uint32_t cap;      // GDPM_PARAM_QUEUE_CAPACITY (0: 8 per primary of a phase + 65536)
        int graph;         // GDPM_PARAM_GRAPH
    };
    const Cfg saved{ctx->batch_mode, ctx->source_chunk, ctx->speculative, ctx->electron_walk,
                    ctx->block_threads, ctx->queue_capacity, ctx->use_graph};
    const int saved_prof = ctx->profile;
    auto apply = [&](const Cfg& c) {
        ctx->batch_mode = c.mode;
        ctx->source_chunk = c.chunk;
        ctx->speculative = c.spec;
        ctx->electron_walk = c.walk;
        ctx->block_threads = c.threads;
        ctx->queue_capacity = c.cap;
        ctx->use_graph = c.graph;
    };
    double spent = 0.0;
    int tried = 0;
    // one calculation under configuration c: its wall time, or a failure code
    auto time_cfg = [&](const Cfg& c, double& ms) -> int {
        apply(c);
        gdpm_stats st{};
        const auto t0 = std::chrono::steady_clock::now();
        const int e = simulate_impl(ctx, ctx->run, ph, tb, ctx->src, ctx->request_id, n_histories,
                                    n_batches, nullptr, nullptr, &st, nullptr, nullptr);
        ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        spent += ms;
        if (e == GDPM_OK) ++tried;
        return e;
    };
    ctx->profile = 0;
    // stage 1: batch mode x primaries per phase x phase pairs per host check
    std::vector<Cfg> cands;
    const bool can_conc = n_batches <= kMaxConcurrentBatches &&
                          V * size_t(n_batches) * 8 <= ctx->concurrent_max_bytes;
    const uint32_t chunks[3] = {1u << 20, 1u << 22, std::max(1u << 23, ctx->auto_chunk)};
    for (int mode = 2; mode >= 1; --mode) {
        if (mode == 2 && !can_conc) continue;
        const uint64_t per = mode == 2 ? n_histories : (n_histories + n_batches - 1) / n_batches;
        uint32_t last = 0;
        for (uint32_t c : chunks) {
            const uint32_t cc = uint32_t(std::min<uint64_t>(c, per));
            if (cc == last) continue;               // the same phases as the previous candidate
            last = cc;
            for (int spec : {1, 2, 4})
                cands.push_back({mode, cc, spec, walk_form(ctx, ph), saved.threads, 0u, 0});
        }
    }
    // an untimed first run: allocations and module loading stay out of the comparison
    double ms = 0.0;
    if ((rc = time_cfg(cands.front(), ms))) {
        apply(saved);
        ctx->profile = saved_prof;
        return rc;
    }
    spent = 0.0;
    tried = 0;
    double best_ms = 1e300;
    Cfg best = cands.front();
    for (const Cfg& c : cands) {
        if ((rc = time_cfg(c, ms))) break;
        if (ms < best_ms) { best_ms = ms; best = c; }
        if (spent >= budget_ms) break;
    }
    // stages 2-5, one dimension at a time from the best so far: the electron
    // phase form, the block shape, half the queue capacity, the device-driven
    // phase loop.  A candidate replaces the best only when more than 1 %
    // faster (single timings are noisy).  A queue capacity too small for this
    // calculation fails with GDPM_E_QUEUE_OVERFLOW and is skipped.
    enum { D_WALK, D_THREADS, D_CAP, D_GRAPH };
    struct Move { int dim, value; };
    const Move moves[] = {{D_WALK, -1}, {D_THREADS, 128}, {D_THREADS, 192}, {D_THREADS, 256},
                          {D_CAP, 0}, {D_GRAPH, 1}};
    for (const Move& mv : moves) {
        if (rc != GDPM_OK || spent >= budget_ms) break;
        Cfg cand = best;
        switch (mv.dim) {
        case D_WALK: cand.walk = 1 - best.walk; break;
        case D_THREADS:
            if (mv.value == best.threads) continue;
            cand.threads = mv.value;
            break;
        case D_CAP:
            cand.cap = uint32_t(std::min<uint64_t>(4ull * best.chunk + 65536u, 0x7FFFFFFFull));
            break;
        default:
            if (best.mode != 2 || best.graph == 1) continue;
            cand.graph = 1;
        }
        const int e = time_cfg(cand, ms);
        if (e == GDPM_E_QUEUE_OVERFLOW) continue;
        if (e) { rc = e; break; }
        if (ms < 0.99 * best_ms) { best_ms = ms; best = cand; }
    }
    ctx->profile = saved_prof;
    if (rc) {
        apply(saved);
        return rc;
    }
    apply(best);
    out->batch_mode = best.mode;
    out->source_chunk = best.chunk;
    out->speculative = best.spec;
    out->candidates_tried = tried;
    out->histories_per_s = double(n_histories) / (best_ms / 1e3);
    out->electron_walk = best.walk;
    out->block_threads = best.threads;
    out->queue_capacity = best.cap;
    out->graph = best.graph;
    return GDPM_OK;
}

int gdpm_simulate_beamlets(gdpm_ctx* ctx, gdpm_phantom* ph, gdpm_tables* tb,
                           const uint64_t* n_histories, int n_batches, double* dose_out,
                           double* sigma_out, gdpm_stats* st) {
    if (!ctx || !n_histories || !dose_out) return GDPM_E_ARG;
    const gdpm_source_state& src = ctx->src;
    if (!src.set) return GDPM_E_STATE;
    if (src.desc.geometry != GDPM_GEO_BEAMLETS) return GDPM_E_ARG;
    Range range("gdpm_simulate_beamlets");
    const uint32_t K = uint32_t(src.beamlets.size() / 17);
    const int nb = n_batches;
    if (nb < 1 || (nb < 2 && sigma_out) || size_t(K) * nb > size_t(kMaxSlots)) return GDPM_E_ARG;
    uint64_t total = 0;
    std::vector<uint32_t> first(K + 1, 0u);
    for (uint32_t k = 0; k < K; ++k) {
        if (n_histories[k] < uint64_t(nb)) return GDPM_E_ARG;
        first[k] = uint32_t(total);
        total += n_histories[k];
        if (total >= (1ull << 32)) return GDPM_E_ARG;
    }
    first[K] = uint32_t(total);
    // the checks of a single calculation (tables cover the spectrum, ...)
    int rc = validate_run(ctx, ph, tb, src, std::max<uint64_t>(total, 2), 2);
    if (rc) return rc;
    GDPM_CUDA_TRY(cudaSetDevice(ctx->device));
    Runner& r = ctx->run;
    cudaStream_t s = r.stream;
    const size_t V = size_t(ph->nx) * ph->ny * ph->nz;
    const uint32_t slots = K * uint32_t(nb);
    const uint32_t chunk = chunk_of(ctx, total, 1, true);
    const uint32_t cap = capacity_of(ctx, chunk);
    const int n_bins = int(src.weights.size());
    if ((rc = prepare_workspace(ctx, r, V, cap, chunk, int(slots), n_bins, true))) return rc;
    Workspace& ws = r.ws;
    SimParams P = base_params(ctx, ph, tb, ctx->request_id);
    if ((rc = get_majorant(ctx, s, ph, tb, &P.maj))) return rc;
    // spectrum allotment of every (sub-problem, batch) slot; batch sizes
    std::vector<uint32_t> prefix(size_t(slots) * (n_bins + 1));
    std::vector<double> inv(2 * size_t(K));
    std::vector<uint32_t> nbig(K);
    for (uint32_t k = 0; k < K; ++k) {
        const uint64_t nk = n_histories[k];
        for (int b = 0; b < nb; ++b) {
            const uint64_t n = nk / nb + (uint64_t(b) < nk % nb ? 1 : 0);
            allot_prefix(src.weights, n, &prefix[(size_t(k) * nb + b) * (n_bins + 1)]);
        }
        inv[2 * k] = 1.0 / double(nk / nb + 1);
        inv[2 * k + 1] = 1.0 / double(nk / nb);
        nbig[k] = uint32_t(nk % nb);
    }
    if ((rc = ensure(ws.sub_first, first.size() * 4)) || (rc = ensure(ws.sub_inv, inv.size() * 8)) ||
        (rc = ensure(ws.sub_nbig, nbig.size() * 4)))
        return rc;
    GDPM_CUDA_TRY(cudaMemcpyAsync(ws.prefix.p, prefix.data(), prefix.size() * 4, cudaMemcpyHostToDevice, s));
    ws.prefix_n = uint32_t(prefix.size());
    GDPM_CUDA_TRY(cudaMemcpyAsync(ws.sub_first.p, first.data(), first.size() * 4, cudaMemcpyHostToDevice, s));
    GDPM_CUDA_TRY(cudaMemcpyAsync(ws.sub_inv.p, inv.data(), inv.size() * 8, cudaMemcpyHostToDevice, s));
    GDPM_CUDA_TRY(cudaMemcpyAsync(ws.sub_nbig.p, nbig.data(), nbig.size() * 4, cudaMemcpyHostToDevice, s));
    if ((rc = source_upload(r, src, P.S, true))) return rc;    // syncs: host vectors may go
    P.counters = static_cast<unsigned long long*>(ws.counters.p);
    P.ledger = static_cast<double*>(ws.ledger.p);
    P.status = static_cast<uint32_t*>(ws.status.p);
    P.batch_stride = V;
    P.tally_hi = V * uint64_t(slots);
    P.edep = static_cast<double*>(ws.edep.p);
    P.edep_hi = static_cast<float*>(ws.edep.p);
    P.edep_lo = static_cast<float*>(ws.edep.p) + V * size_t(slots);
    if (ctx->hrec) {
        if (ctx->hrec_n < total) return GDPM_E_ARG;
        P.hrec = ctx->hrec;
        P.n_records = ctx->hrec_n;
        P.hrecd = ctx->hrecd;
        GDPM_CUDA_TRY(cudaMemsetAsync(ctx->hrec, 0, total * 16, s));
        GDPM_CUDA_TRY(cudaMemsetAsync(ctx->hrecd, 0, total * 16, s));
    }
    GDPM_CUDA_TRY(cudaMemsetAsync(ws.edep.p, 0, V * size_t(slots) * 8, s));
    GDPM_CUDA_TRY(cudaMemsetAsync(ws.counters.p, 0, C_NCOUNT * 8, s));
    GDPM_CUDA_TRY(cudaMemsetAsync(ws.ledger.p, 0, L_NLEDGER * 8, s));
    GDPM_CUDA_TRY(cudaMemsetAsync(ws.status.p, 0, 16, s));
    r.prof_kind.clear();
    GDPM_CUDA_TRY(cudaEventRecord(r.ev0, s));
    int64_t phases = 0, aux = 0;
    const uint32_t* graph_k = nullptr;
    int run_rc;
    if (ctx->use_graph && !ctx->profile) {
        uint32_t* kh = reinterpret_cast<uint32_t*>(static_cast<unsigned char*>(ws.pinned_host.p) + 32);
        run_rc = run_phases_graph(ctx, r, P, src, 0, total, 0, 0, chunk, kh, K, uint32_t(nb),
                                  static_cast<const uint32_t*>(ws.sub_first.p));
        graph_k = kh;
        ++aux;
    } else {
        run_rc = run_phases(ctx, r, P, src, 0, total, 0, 0, chunk, phases, aux, K, uint32_t(nb),
                            static_cast<const uint32_t*>(ws.sub_first.p));
    }
    GDPM_CUDA_TRY(cudaEventRecord(r.ev1, s));
    if (run_rc != GDPM_OK) {
        cudaStreamSynchronize(s);
        r.prof_kind.clear();
        return run_rc;
    }
    // per sub-problem dose (and sigma): straight into device outputs, or in
    // groups of sub-problems through a staging buffer for host outputs
    const bool dev_out = is_device_ptr(dose_out) && (!sigma_out || is_device_ptr(sigma_out));
    const double* sinv = static_cast<const double*>(ws.sub_inv.p);
    const uint32_t* snb = static_cast<const uint32_t*>(ws.sub_nbig.p);
    if (dev_out) {
        for (uint32_t k0 = 0; k0 < K; k0 += 65535u) {
            const uint32_t nk = std::min(K - k0, 65535u);
            if ((rc = launch_fold_sub(ctx, s, P, V, k0, nk, nb, sinv, snb, dose_out + size_t(k0) * V,
                                      sigma_out ? sigma_out + size_t(k0) * V : nullptr)))
                return rc;
            ++aux;
        }
    } else {
        const uint32_t group = uint32_t(std::max<size_t>(1, std::min<size_t>(K, (size_t(256) << 20) / (V * 16))));
        if ((rc = ensure(ws.stage, size_t(group) * V * 16))) return rc;
        double* sd = static_cast<double*>(ws.stage.p);
        double* ss = sd + size_t(group) * V;
        for (uint32_t k0 = 0; k0 < K; k0 += group) {
            const uint32_t nk = std::min(K - k0, group);
            if ((rc = launch_fold_sub(ctx, s, P, V, k0, nk, nb, sinv, snb, sd, sigma_out ? ss : nullptr)))
                return rc;
            ++aux;
            GDPM_CUDA_TRY(cudaMemcpyAsync(dose_out + size_t(k0) * V, sd, size_t(nk) * V * 8, cudaMemcpyDefault, s));
            if (sigma_out)
                GDPM_CUDA_TRY(cudaMemcpyAsync(sigma_out + size_t(k0) * V, ss, size_t(nk) * V * 8, cudaMemcpyDefault, s));
        }
    }
    unsigned char* h = static_cast<unsigned char*>(ws.pinned_host.p);
    unsigned long long* hc = reinterpret_cast<unsigned long long*>(h + 64);
    double* hl = reinterpret_cast<double*>(h + 64 + C_NCOUNT * 8);
    uint32_t* hs = reinterpret_cast<uint32_t*>(h + 64 + C_NCOUNT * 8 + L_NLEDGER * 8);
    GDPM_CUDA_TRY(cudaMemcpyAsync(hc, ws.counters.p, C_NCOUNT * 8, cudaMemcpyDeviceToHost, s));
    GDPM_CUDA_TRY(cudaMemcpyAsync(hl, ws.ledger.p, L_NLEDGER * 8, cudaMemcpyDeviceToHost, s));
    GDPM_CUDA_TRY(cudaMemcpyAsync(hs, ws.status.p, 4, cudaMemcpyDeviceToHost, s));
    GDPM_CUDA_TRY(cudaStreamSynchronize(s));
    if (st) {
        std::memset(st, 0, sizeof(*st));
        fill_stats(hc, hl, st);
        if (graph_k) phases = int64_t(*graph_k);
        st->phases = phases;
        st->launches = phases + aux;
        float ms = 0;
        cudaEventElapsedTime(&ms, r.ev0, r.ev1);
        st->transport_ms = ms;
    }
    prof_collect(r, st);
    if (*hs & ST_BOUNDS) return GDPM_E_BOUNDS;
    if (*hs & ST_QUEUE_OVERFLOW) return GDPM_E_QUEUE_OVERFLOW;
    if (*hs & (ST_ITER_CAP | ST_PHASE_CAP)) return GDPM_E_TIMEOUT;
    return GDPM_OK;
}

int gdpm_debug_philox(gdpm_ctx* ctx, const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* out,
                      uint64_t n) {
    if (!ctx || !ctr || !out || !is_device_ptr(ctr) || !is_device_ptr(out)) return GDPM_E_ARG;
    int rc = launch_debug_philox(ctx, ctr, k0, k1, out, n);
    if (rc) return rc;
    GDPM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return GDPM_OK;
}

int gdpm_debug_sample(gdpm_ctx* ctx, int kind, double a, double b, uint64_t n, uint64_t seed,
                      double* out1, double* out2) {
    if (!ctx || !out1 || kind < 0 || kind > 5 || !is_device_ptr(out1) || (out2 && !is_device_ptr(out2)))
        return GDPM_E_ARG;
    if (kind == 5 && !(a > 0)) return GDPM_E_ARG;
    if (kind == 1 && !(a > 2 * b && b > 0)) return GDPM_E_ARG;
    if (kind == 2 && !(a > b && b > 0)) return GDPM_E_ARG;
    if (kind == 0 && !(a > 0)) return GDPM_E_ARG;
    int rc = launch_debug_sample(ctx, kind, a, b, n, seed, out1, out2);
    if (rc) return rc;
    GDPM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return GDPM_OK;
}

int gdpm_tables_export(gdpm_tables* t, int which, double* out, int64_t* count) {
    if (!t || !count) return GDPM_E_ARG;
    const int M = t->n_mat, n = t->n_e;
    std::vector<double> v;
    cudaStream_t s = t->ctx->stream;
    if (which >= 0 && which <= 2) {
        std::vector<float> tot(size_t(M) * n);
        std::vector<float2> cum(size_t(M) * n);
        GDPM_CUDA_TRY(cudaMemcpyAsync(tot.data(), t->ph_tot.p, tot.size() * 4, cudaMemcpyDeviceToHost, s));
        GDPM_CUDA_TRY(cudaMemcpyAsync(cum.data(), t->ph_cum.p, cum.size() * 8, cudaMemcpyDeviceToHost, s));
        GDPM_CUDA_TRY(cudaStreamSynchronize(s));
        for (size_t k = 0; k < tot.size(); ++k)
            v.push_back(which == 0 ? cum[k].x : (which == 1 ? cum[k].y : tot[k]));
    } else if (which >= 3 && which <= 5) {
        std::vector<float4> el(size_t(M) * n);
        GDPM_CUDA_TRY(cudaMemcpyAsync(el.data(), t->el.p, el.size() * 16, cudaMemcpyDeviceToHost, s));
        GDPM_CUDA_TRY(cudaStreamSynchronize(s));
        for (size_t k = 0; k < el.size(); ++k) v.push_back(which == 3 ? el[k].x : (which == 4 ? el[k].z : el[k].w));
    } else if (which == 6) {
        for (int i = 0; i < n; ++i)
            v.push_back(std::exp(std::log(t->e_min) + i * (std::log(t->e_max) - std::log(t->e_min)) / (n - 1)));
    } else if (which == 7) {
        for (int m = 0; m < M; ++m) v.push_back(t->dev.x0[m]);
    } else if (which == 8) {
        for (int m = 0; m < M; ++m) v.push_back(t->dev.sigmax[m]);
    } else if (which == 9) {
        std::vector<float> a(size_t(t->n_a));
        GDPM_CUDA_TRY(cudaMemcpyAsync(a.data(), t->atab.p, a.size() * 4, cudaMemcpyDeviceToHost, s));
        GDPM_CUDA_TRY(cudaStreamSynchronize(s));
        for (float x : a) v.push_back(x);
    } else {
        return GDPM_E_ARG;
    }
    *count = int64_t(v.size());
    if (out) GDPM_CUDA_TRY(cudaMemcpy(out, v.data(), v.size() * 8, cudaMemcpyDefault));
    return GDPM_OK;
}

// Checks: run the Metropolis chains from their start through history
// n_hist - 1 into the pick buffer (nothing to do for the other samplers).
static int run_chains(Runner& r, const SimParams& P, uint64_t n_hist) {
    if (P.S.sampler != GDPM_SAMPLE_METROPOLIS || P.S.n_beamlets == 0) return GDPM_OK;
    int rc;
    if ((rc = ensure(r.ws.chains, size_t(P.S.n_chains) * 4)) || (rc = ensure(r.ws.pick, n_hist * 4)))
        return rc;
    uint32_t* chains = static_cast<uint32_t*>(r.ws.chains.p);
    if ((rc = launch_metropolis_init(r.stream, P, chains))) return rc;
    return launch_metropolis(r.stream, P, 0, uint32_t(n_hist), chains, static_cast<uint32_t*>(r.ws.pick.p));
}

int gdpm_debug_beamlets(gdpm_ctx* ctx, uint64_t first, uint64_t n, int32_t* out) {
    if (!ctx) return GDPM_E_ARG;
    if (!ctx->src.set) return GDPM_E_STATE;
    if (ctx->src.desc.geometry != GDPM_GEO_BEAMLETS || !out || !is_device_ptr(out) ||
        first + n > (1ull << 32) || n == 0)
        return GDPM_E_ARG;
    GDPM_CUDA_TRY(cudaSetDevice(ctx->device));
    Runner& r = ctx->run;
    SimParams P{};
    P.key0 = uint32_t(ctx->seed);
    P.key1 = uint32_t(ctx->seed >> 32) ^ ctx->request_id;
    int rc;
    if ((rc = source_upload(r, ctx->src, P.S))) return rc;
    if ((rc = run_chains(r, P, first + n))) return rc;
    const uint32_t* pick = P.S.sampler == GDPM_SAMPLE_METROPOLIS ? static_cast<const uint32_t*>(r.ws.pick.p) + first
                                                                  : nullptr;
    if ((rc = launch_debug_beamlets(r.stream, P, uint32_t(first), uint32_t(n), pick, out))) return rc;
    GDPM_CUDA_TRY(cudaStreamSynchronize(r.stream));
    return GDPM_OK;
}

int gdpm_debug_sources(gdpm_ctx* ctx, gdpm_phantom* ph, gdpm_tables* tb, uint64_t n_histories,
                       int n_batches, uint64_t first, uint64_t n, double* out) {
    if (!ctx) return GDPM_E_ARG;
    int rc = validate_run(ctx, ph, tb, ctx->src, n_histories, n_batches);
    if (rc) return rc;
    const uint64_t nb0 = n_histories / n_batches + (n_histories % n_batches ? 1 : 0);
    if (!out || !is_device_ptr(out) || first + n > nb0) return GDPM_E_ARG;
    Runner& r = ctx->run;
    const int n_bins = int(ctx->src.weights.size());
    std::vector<uint32_t> prefix(n_bins + 1);
    allot_prefix(ctx->src.weights, nb0, prefix.data());
    if ((rc = ensure(r.ws.prefix, prefix.size() * 4))) return rc;
    GDPM_CUDA_TRY(cudaMemcpyAsync(r.ws.prefix.p, prefix.data(), prefix.size() * 4, cudaMemcpyHostToDevice, r.stream));
    SimParams P = base_params(ctx, ph, tb, ctx->request_id);
    if ((rc = get_majorant(ctx, r.stream, ph, tb, &P.maj))) return rc;
    if ((rc = source_upload(r, ctx->src, P.S))) return rc;
    PhaseArgs A{};
    A.src_first = uint32_t(first);
    A.nb_small = uint32_t(n_histories / n_batches);
    A.nb_rem = uint32_t(n_histories % n_batches);
    A.bin_prefix = static_cast<const uint32_t*>(r.ws.prefix.p);
    if ((rc = run_chains(r, P, first + n))) return rc;
    if (P.S.sampler == GDPM_SAMPLE_METROPOLIS && P.S.n_beamlets > 0)
        A.bl_pick = static_cast<const uint32_t*>(r.ws.pick.p) + first;
    if ((rc = launch_debug_sources(ctx, P, A, n, out))) return rc;
    GDPM_CUDA_TRY(cudaStreamSynchronize(r.stream));
    return GDPM_OK;
}

int gdpm_request_submit(gdpm_ctx* ctx, const gdpm_request_desc* req, uint64_t* req_id) {
    if (!ctx || !req || !req_id || !req->phantom || !req->tables) return GDPM_E_ARG;
    if (req->n_batches < 2 || req->n_histories < uint64_t(req->n_batches) || req->n_histories >= (1ull << 32))
        return GDPM_E_ARG;
    std::unique_ptr<gdpm_request> q(new gdpm_request());
    int rc = source_copy(&req->source, q->src);
    if (rc) return rc;
    if ((rc = validate_run(ctx, req->phantom, req->tables, q->src, req->n_histories, req->n_batches))) return rc;
    q->desc = *req;
    q->desc.source = q->src.desc;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (ctx->stop) return GDPM_E_STATE;
    if (ctx->pending.size() >= 100000) return GDPM_E_BUSY;
    if (ctx->workers.empty()) {
        const int big = std::min(ctx->serve_big_slots, ctx->serve_slots - 1);
        for (int k = 0; k < ctx->serve_slots; ++k)
            ctx->workers.emplace_back(serve_worker, ctx, ctx->serve_slots == 1 ? 0 : (k < big ? 1 : 2));
    }
    q->id = ctx->next_request++;
    *req_id = q->id;
    ctx->pending.push_back(q.get());
    ctx->requests[q->id] = std::move(q);
    ctx->cv.notify_all();
    return GDPM_OK;
}

int gdpm_request_poll(gdpm_ctx* ctx, uint64_t req_id, int* done, double* dose_out, double* sigma_out,
                      gdpm_stats* stats_out) {
    if (!ctx || !done) return GDPM_E_ARG;
    std::unique_ptr<gdpm_request> q;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        auto it = ctx->requests.find(req_id);
        if (it == ctx->requests.end()) return GDPM_E_ARG;
        if (it->second->status == 1) {
            *done = 0;
            return GDPM_OK;
        }
        q = std::move(it->second);
        ctx->requests.erase(it);
    }
    *done = 1;
    int rc = q->status;
    if (rc == GDPM_OK) {
        const gdpm_phantom* ph = q->desc.phantom;
        const size_t V = size_t(ph->nx) * ph->ny * ph->nz;
        const double* d = static_cast<const double*>(q->result.p);
        if (cudaSetDevice(ctx->device) != cudaSuccess ||
            (dose_out && cudaMemcpy(dose_out, d, V * 8, cudaMemcpyDefault) != cudaSuccess) ||
            (sigma_out && cudaMemcpy(sigma_out, d + V, V * 8, cudaMemcpyDefault) != cudaSuccess)) {
            last_cuda_error() = cudaGetLastError();
            rc = GDPM_E_CUDA;
        }
        if (stats_out) *stats_out = q->stats;
    }
    result_release(ctx, q->result);
    return rc;
}

}  // extern "C"
