// C ABI of the transport library: context, fields, dose and influence matrices.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <mutex>
#include <vector>

#include "../../include/vpmc.h"
#include "context.h"
#include "tables.h"
#include "vpmc_internal.cuh"

using namespace vpmc;

namespace {

thread_local std::string g_error;

vpmc_status fail(vpmc_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_error = buf;
    return st;
}

}  // namespace

vpmc_status vpmc::report_error(vpmc_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_error = buf;
    return st;
}

void vpmc::clear_error() { g_error.clear(); }

namespace {

#define CUDA_TRY(expr)                                                                             \
    do {                                                                                           \
        cudaError_t e_ = (expr);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail(e_ == cudaErrorMemoryAllocation ? VPMC_ERR_OOM : VPMC_ERR_CUDA, "%s: %s (%s:%d)", \
                        #expr, cudaGetErrorString(e_), __FILE__, __LINE__);                        \
    } while (0)

template <class T>
cudaError_t dev_alloc(T** p, size_t n)
{
    *p = nullptr;
    if (n == 0) n = 1;
    return cudaMalloc(reinterpret_cast<void**>(p), n * sizeof(T));
}

// n elements of T from a context's grow-only buffer (reallocated, contents
// lost, only when it is too small).
template <class T>
cudaError_t ensure(DevBuf& b, size_t n, T** out)
{
    const size_t need = (n == 0 ? 1 : n) * sizeof(T);
    if (need > b.bytes) {
        cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
        cudaError_t e = cudaMalloc(&b.p, need);
        if (e != cudaSuccess) {
            *out = nullptr;
            return e;
        }
        b.bytes = need;
    }
    *out = static_cast<T*>(b.p);
    return cudaSuccess;
}

void free_buf(DevBuf& b)
{
    cudaFree(b.p);
    b = DevBuf{};
}

}  // namespace


namespace {

Grid3 to_grid3(const vpmc_grid& g)
{
    Grid3 r;
    r.n[0] = g.nx; r.n[1] = g.ny; r.n[2] = g.nz;
    r.d[0] = (float)g.dx; r.d[1] = (float)g.dy; r.d[2] = (float)g.dz;
    for (int k = 0; k < 3; ++k) r.lo[k] = (float)g.origin[k];
    return r;
}

vpmc_status grow(vpmc_ctx* c, DevItem** p, size_t* cap, size_t n)
{
    if (n <= *cap) return VPMC_OK;
    cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    CUDA_TRY(dev_alloc(p, n));
    *cap = n;
    (void)c;
    return VPMC_OK;
}

vpmc_status grow_boxes(vpmc_ctx* c, size_t n)
{
    if (n <= c->boxes_cap) return VPMC_OK;
    cudaFree(c->d_boxes);
    c->d_boxes = nullptr;
    c->boxes_cap = 0;
    CUDA_TRY(dev_alloc(&c->d_boxes, n));
    c->boxes_cap = n;
    return VPMC_OK;
}

vpmc_status grow_ovf(vpmc_ctx* c, long long n)
{
    if (n <= c->ovf_cap) return VPMC_OK;
    cudaFree(c->d_ovf);
    c->d_ovf = nullptr;
    c->ovf_cap = 0;
    CUDA_TRY(dev_alloc(&c->d_ovf, (size_t)n));
    c->ovf_cap = n;
    return VPMC_OK;
}

vpmc_status grow_phase(vpmc_ctx* c, long long n)
{
    if (n <= c->phase_cap) return VPMC_OK;
    cudaFree(c->d_phase);
    cudaFree(c->d_mid);
    c->d_phase = nullptr;
    c->d_mid = nullptr;
    c->phase_cap = 0;
    CUDA_TRY(dev_alloc(&c->d_phase, (size_t)n));
    CUDA_TRY(dev_alloc(&c->d_mid, (size_t)n));
    c->phase_cap = n;
    return VPMC_OK;
}

vpmc_status grow_scratch(vpmc_ctx* c, size_t n)
{
    if (n <= c->scratch_cap) return VPMC_OK;
    cudaFree(c->d_scratch);
    c->d_scratch = nullptr;
    c->scratch_cap = 0;
    CUDA_TRY(dev_alloc(&c->d_scratch, n));
    c->scratch_cap = n;
    return VPMC_OK;
}

vpmc_status upload_beams(vpmc_ctx* c)
{
    std::vector<float2> poly;
    std::vector<float> kappa;
    std::vector<unsigned char> ras;
    std::vector<float> ras_lb;
    DevBeam tmp[kMaxBeams];
    for (int b = 0; b < kMaxBeams; ++b) {
        tmp[b] = c->beams[b];
        if (!c->beam_set[b] || !c->beams[b].ap) continue;
        tmp[b].poly_off = (int)poly.size();
        for (size_t i = 0; i + 1 < c->poly[b].size(); i += 2)
            poly.push_back(make_float2((float)c->poly[b][i], (float)c->poly[b][i + 1]));
        const int nv = (int)(c->poly[b].size() / 2);
        kappa.resize(poly.size());
        polygon_curvature(c->poly[b].data(), nv, kappa.data() + (poly.size() - nv));
        tmp[b].ras_off = (int)ras.size();
        ras.insert(ras.end(), c->raster[b].begin(), c->raster[b].end());
        ras_lb.insert(ras_lb.end(), c->raster_lb[b].begin(), c->raster_lb[b].end());
    }
    if (poly.size() > (size_t)kMaxPolyVerts)
        return fail(VPMC_ERR_ARG, "aperture polygons have %zu vertices in total (max %d)", poly.size(), kMaxPolyVerts);
    cudaFree(c->d_poly);
    cudaFree(c->d_poly_kappa);
    cudaFree(c->d_raster);
    cudaFree(c->d_raster_lb);
    c->d_poly = nullptr;
    c->d_poly_kappa = nullptr;
    c->d_raster = nullptr;
    c->d_raster_lb = nullptr;
    CUDA_TRY(dev_alloc(&c->d_poly, std::max<size_t>(poly.size(), 1)));
    CUDA_TRY(dev_alloc(&c->d_poly_kappa, std::max<size_t>(kappa.size(), 1)));
    if (!kappa.empty())
        CUDA_TRY(cudaMemcpy(c->d_poly_kappa, kappa.data(), kappa.size() * sizeof(float), cudaMemcpyHostToDevice));
    CUDA_TRY(dev_alloc(&c->d_raster, std::max<size_t>(ras.size(), 1)));
    CUDA_TRY(dev_alloc(&c->d_raster_lb, std::max<size_t>(ras_lb.size(), 1)));
    if (!poly.empty()) CUDA_TRY(cudaMemcpy(c->d_poly, poly.data(), poly.size() * sizeof(float2), cudaMemcpyHostToDevice));
    if (!ras.empty()) CUDA_TRY(cudaMemcpy(c->d_raster, ras.data(), ras.size(), cudaMemcpyHostToDevice));
    if (!ras_lb.empty())
        CUDA_TRY(cudaMemcpy(c->d_raster_lb, ras_lb.data(), ras_lb.size() * sizeof(float), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(c->d_beams, tmp, sizeof(tmp), cudaMemcpyHostToDevice));
    c->n_poly = (int)poly.size();
    return VPMC_OK;
}

// A polygon (n >= 3 vertices, xy pairs) is simple when no two edges meet
// except neighbours at their shared vertex, and neighbours do not fold back
// onto each other.  Closed-segment tests with orientation signs in FP64;
// O(n^2) edge pairs (a 4096-gon takes a few tens of ms, once per beam).
bool polygon_is_simple(const double* xy, int n, int* e1, int* e2)
{
    auto orient = [&](int a, int b, int c) {
        const double v = (xy[2 * b] - xy[2 * a]) * (xy[2 * c + 1] - xy[2 * a + 1]) -
                         (xy[2 * b + 1] - xy[2 * a + 1]) * (xy[2 * c] - xy[2 * a]);
        return (v > 0.0) - (v < 0.0);
    };
    auto within = [&](int a, int b, int p) {         // p collinear with a-b: inside its bounding box
        return std::min(xy[2 * a], xy[2 * b]) <= xy[2 * p] && xy[2 * p] <= std::max(xy[2 * a], xy[2 * b]) &&
               std::min(xy[2 * a + 1], xy[2 * b + 1]) <= xy[2 * p + 1] &&
               xy[2 * p + 1] <= std::max(xy[2 * a + 1], xy[2 * b + 1]);
    };
    for (int i = 0; i < n; ++i) {
        const int a = i, b = (i + 1) % n, c = (i + 2) % n;
        *e1 = i;
        *e2 = (i + 1) % n;
        if (xy[2 * a] == xy[2 * b] && xy[2 * a + 1] == xy[2 * b + 1]) return false;    // repeated vertex
        // neighbours a-b and b-c fold back: collinear with c on the side of a
        if (orient(a, b, c) == 0 && (xy[2 * c] - xy[2 * b]) * (xy[2 * a] - xy[2 * b]) +
                                            (xy[2 * c + 1] - xy[2 * b + 1]) * (xy[2 * a + 1] - xy[2 * b + 1]) > 0.0)
            return false;
    }
    for (int i = 0; i < n; ++i) {
        const int p1 = i, p2 = (i + 1) % n;
        for (int j = i + 2; j < n; ++j) {
            if (i == 0 && j == n - 1) continue;      // neighbours through the closing edge
            const int q1 = j, q2 = (j + 1) % n;
            const int d1 = orient(q1, q2, p1), d2 = orient(q1, q2, p2);
            const int d3 = orient(p1, p2, q1), d4 = orient(p1, p2, q2);
            const bool meet = (d1 * d2 < 0 && d3 * d4 < 0) || (d1 == 0 && within(q1, q2, p1)) ||
                              (d2 == 0 && within(q1, q2, p2)) || (d3 == 0 && within(p1, p2, q1)) ||
                              (d4 == 0 && within(p1, p2, q2));
            if (meet) {
                *e1 = i;
                *e2 = j;
                return false;
            }
        }
    }
    return true;
}

// Checks shared by the dose and influence-matrix paths.
vpmc_status check_spots(vpmc_ctx* c, const vpmc_spot* spots, int n_spots)
{
    if (n_spots < 0 || (n_spots > 0 && !spots)) return fail(VPMC_ERR_ARG, "spots: null pointer or negative count");
    for (int i = 0; i < n_spots; ++i) {
        const vpmc_spot& s = spots[i];
        if (s.beam < 0 || s.beam >= kMaxBeams || !c->beam_set[s.beam])
            return fail(VPMC_ERR_STATE, "spot %d: beam %d was not set with vpmc_set_aperture", i, s.beam);
        if (!(s.energy_mev > 0.5 && s.energy_mev <= 250.0))
            return fail(VPMC_ERR_ARG, "spot %d: energy %g MeV outside (0.5, 250]", i, s.energy_mev);
        if (s.n_hist < 0 || s.n_hist >= (1ll << 32))
            return fail(VPMC_ERR_ARG, "spot %d: n_hist %lld outside [0, 2^32)", i, (long long)s.n_hist);
        if (!(s.sigma_mm >= 0.0) || !(s.div_mrad >= 0.0) || !std::isfinite(s.x_mm) || !std::isfinite(s.y_mm))
            return fail(VPMC_ERR_ARG, "spot %d: invalid position, sigma or divergence", i);
    }
    return VPMC_OK;
}

// The learned aperture surrogate is trained on parallel walls: refuse it for
// spots of a beam with a divergent block.
vpmc_status check_surrogate_walls(const vpmc_ctx* c, const vpmc_spot* spots, int n_spots, int surrogate)
{
    if (!surrogate) return VPMC_OK;
    for (int i = 0; i < n_spots; ++i) {
        const DevBeam& b = c->beams[spots[i].beam];
        if (b.ap && b.ap_sad > 0.0f)
            return fail(VPMC_ERR_ARG, "beam %d: the surrogate models parallel aperture walls only", spots[i].beam);
    }
    return VPMC_OK;
}

vpmc_status check_opts(const vpmc_opts* o)
{
    if (!o) return VPMC_OK;
    if (o->frac_bits < 0 || o->frac_bits > 40) return fail(VPMC_ERR_ARG, "frac_bits %d outside [0, 40]", o->frac_bits);
    if (o->block_size != 0 && (o->block_size < 32 || o->block_size > patient_max_block() || o->block_size % 32))
        return fail(VPMC_ERR_ARG, "block_size %d: must be 0 or a multiple of 32 in [32, %d]", o->block_size,
                    patient_max_block());
    if (o->blocks_per_sm < 0 || o->blocks_per_sm > 1)
        return fail(VPMC_ERR_ARG, "blocks_per_sm %d: the kernel's shared memory allows one block per SM", o->blocks_per_sm);
    if (o->chunk < 0 || o->chunk > 4096) return fail(VPMC_ERR_ARG, "chunk %d outside [0, 4096]", o->chunk);
    if (o->history_cap < 0 || (o->history_cap > 0 && !o->history_out))
        return fail(VPMC_ERR_ARG, "history_cap > 0 needs history_out");
    if (o->surrogate != 0 && o->surrogate != 1) return fail(VPMC_ERR_ARG, "surrogate must be 0 or 1");
    if (o->timeout_iters < 0 || o->timeout_iters > 0x7fffffffll)
        return fail(VPMC_ERR_ARG, "timeout_iters %lld outside [0, 2^31 - 1]", (long long)o->timeout_iters);
    return VPMC_OK;
}

// The status word that an earlier asynchronous dose call left unread: waits
// for that call's work, then reports what its kernels latched.
vpmc_status pending_status(vpmc_ctx* c)
{
    if (!c->status_pending) return VPMC_OK;
    const bool sur = c->status_pending == 2;
    c->status_pending = 0;
    int status = 0, ss = 0;
    CUDA_TRY(cudaMemcpyAsync(&status, c->d_status, sizeof status, cudaMemcpyDeviceToHost, c->stream));
    if (sur && c->sur.status) CUDA_TRY(cudaMemcpyAsync(&ss, c->sur.status, sizeof ss, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (status & 1) return fail(VPMC_ERR_TIMEOUT, "an earlier asynchronous call: histories reached the iteration cap");
    if (status & 6)
        return fail(VPMC_ERR_DEVICE_FLAG, "an earlier asynchronous call: hand-off or query buffer overflow (status %d)",
                    status);
    if (ss) return fail(VPMC_ERR_TIMEOUT, "an earlier asynchronous call: a surrogate tensor-core wait timed out");
    return VPMC_OK;
}

TransportParams base_params(vpmc_ctx* c, const vpmc_opts& o)
{
    TransportParams p{};
    p.tables = c->d_tables;
    p.water = c->water_mat;
    p.ct_lut = reinterpret_cast<const uint16_t*>(c->d_ct);
    p.ctg = c->ctg;
    p.sg = c->sg;
    for (int k = 0; k < 3; ++k) p.nest_shift[k] = c->nest_shift[k];
    p.beams = c->d_beams;
    p.n_beams = kMaxBeams;
    p.scens = c->d_scens;
    p.poly = c->d_poly;
    p.n_poly = c->n_poly;
    p.raster = c->d_raster;
    p.raster_lb = c->d_raster_lb;
    p.range_rejection = o.range_rejection;
    p.items = c->d_items;
    p.boxes = c->d_boxes;
    p.counter = c->d_counter;
    p.stats = c->d_stats;
    p.status = c->d_status;
    p.key0 = (uint32_t)o.seed;
    p.key1_hi = (uint32_t)(o.seed >> 32);
    p.mcs = o.mcs;
    p.straggling = o.straggling;
    p.nuclear = o.nuclear;
    p.fscale = std::ldexp(1.0f, o.frac_bits);
    p.fx32 = o.frac_bits <= 24 ? 1 : 0;
    p.max_iter = o.timeout_iters > 0 ? (int)o.timeout_iters : kMaxIter;
    p.records = reinterpret_cast<HistRecord*>(o.history_out);
    p.rec_cap = o.history_out ? o.history_cap : 0;
    p.phase = c->d_phase;
    p.phase_cap = c->phase_cap;
    p.phase_count = c->d_phase_count;
    p.mid = c->d_mid;
    p.mid_cap = c->phase_cap;
    p.mid_count = c->d_mid_count;
    p.poly_kappa = c->d_poly_kappa;
    p.surrogate = o.surrogate && c->sur_ready ? 1 : 0;
    p.n_rep = 1;                    // set by the influence-matrix path when scenarios share the beam line
    p.rep_cap = c->phase_cap;
    return p;
}

vpmc_status reset_counters(vpmc_ctx* c)
{
    CUDA_TRY(cudaMemsetAsync(c->d_counter, 0, sizeof(unsigned long long), c->stream));
    CUDA_TRY(cudaMemsetAsync(c->d_stats, 0, sizeof(unsigned long long) * kNStats, c->stream));
    CUDA_TRY(cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
    return VPMC_OK;
}

constexpr long long kMaxBatch = 1ll << 26;    // histories per devices -> patient hand-off batch

vpmc_status grow_queries(vpmc_ctx* c, long long n)
{
    if (!c->d_sq_count) CUDA_TRY(dev_alloc(&c->d_sq_count, 1));
    if (n <= c->sq_cap) return VPMC_OK;
    cudaFree(c->d_sq);
    c->d_sq = nullptr;
    c->sq_cap = 0;
    CUDA_TRY(dev_alloc(&c->d_sq, (size_t)n));
    c->sq_cap = n;
    return VPMC_OK;
}

// Hand-off buffer (and, with the surrogate, the query buffer) for one batch.
vpmc_status ensure_phase(vpmc_ctx* c, long long total, bool surrogate = false)
{
    const long long n = std::max<long long>(std::min(total, kMaxBatch), 1);
    vpmc_status st = grow_phase(c, n);
    if (st == VPMC_OK && surrogate) st = grow_queries(c, std::min<long long>(n, c->phase_cap));
    return st;
}

// Enqueues the transport of histories [0, total) of p's items: batches of at
// most phase_cap / n_rep histories, each the devices kernel then the patient
// kernel (which takes n_rep copies of every survivor, one per scenario).
vpmc_status enqueue_transport(vpmc_ctx* c, TransportParams p, long long total, const TuneResult& t)
{
    if (p.n_rep < 1) p.n_rep = 1;
    const long long batch = c->phase_cap / p.n_rep;
    if (batch < 1) return fail(VPMC_ERR_STATE, "hand-off buffer smaller than one record per scenario");
    p.phase = c->d_phase;
    p.phase_cap = c->phase_cap;
    p.phase_count = c->d_phase_count;
    p.rep_cap = batch;
    p.rep_hist = p.n_rep > 1 ? p.rep_hist : total;
    p.mid = c->d_mid;
    p.mid_cap = batch;
    p.mid_count = c->d_mid_count;
    p.aggregate = t.aggregate;
    p.chunk = t.chunk;
    if (p.surrogate) {
        if (!c->d_sq || c->sq_cap < c->phase_cap) return fail(VPMC_ERR_STATE, "surrogate query buffer not sized");
        p.sq = c->d_sq;
        p.sq_cap = c->sq_cap;
        p.sq_count = c->d_sq_count;
    }
    // the batch events are recorded as event nodes when the transport is
    // captured into a graph (external records), or directly otherwise
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CUDA_TRY(cudaStreamIsCapturing(c->stream, &cap));
    const unsigned rec_flags = cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
    c->kev_batches = 0;
    for (long long h0 = 0; h0 < total; h0 += batch) {
        const int b = c->kev_batches < vpmc_ctx::kTimedBatches ? c->kev_batches++ : -1;
        p.hist_begin = h0;
        p.total = std::min(total, h0 + batch);
        CUDA_TRY(cudaMemsetAsync(c->d_counter, 0, sizeof(unsigned long long), c->stream));
        CUDA_TRY(cudaMemsetAsync(c->d_phase_count, 0, sizeof(unsigned long long), c->stream));
        if (p.surrogate) CUDA_TRY(cudaMemsetAsync(c->d_sq_count, 0, sizeof(unsigned long long), c->stream));
        if (b >= 0) CUDA_TRY(cudaEventRecordWithFlags(c->kev[3 * b], c->stream, rec_flags));
        CUDA_TRY(launch_devices(p, c->num_sms, t.dev_block, c->stream));
        if (p.surrogate) {
            // brass entries in the surrogate's domain: one network draw each
            CUDA_TRY(launch_sur_infer(c->sur, p, c->num_sms, c->stream));
            c->launches += 1;
        }
        CUDA_TRY(cudaMemsetAsync(c->d_counter, 0, sizeof(unsigned long long), c->stream));
        if (b >= 0) CUDA_TRY(cudaEventRecordWithFlags(c->kev[3 * b + 1], c->stream, rec_flags));
        CUDA_TRY(launch_patient(p, c->num_sms, t.block, c->stream));
        if (b >= 0) CUDA_TRY(cudaEventRecordWithFlags(c->kev[3 * b + 2], c->stream, rec_flags));
        c->launches += 3;
    }
    return VPMC_OK;
}

float time_launch(vpmc_ctx* c, cudaError_t (*fn)(const TransportParams&, int, int, cudaStream_t),
                  const TransportParams& p, int block, int kernels)
{
    cudaMemsetAsync(c->d_counter, 0, sizeof(unsigned long long), c->stream);
    cudaEventRecord(c->ev0, c->stream);
    cudaError_t e = fn(p, c->num_sms, block, c->stream);
    cudaEventRecord(c->ev1, c->stream);
    if (e != cudaSuccess || cudaEventSynchronize(c->ev1) != cudaSuccess) return 1e30f;
    c->launches += kernels;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    return ms;
}

// Chooses the two kernels' block sizes, warp aggregation and refill chunk by
// timing launches over a prefix of the work (results are discarded; the
// caller zeroes the scoring buffers afterwards).  The prefix gives every lane
// of the largest block about 24 histories: in a launch of only a few
// histories per lane the tail (the last long histories of each warp) decides
// the time and favours small blocks, which lose on long launches (13-scenario
// head set: 768 threads chosen on 4 histories per lane, 4.7 % slower than the
// 896 chosen on 24).
vpmc_status autotune(vpmc_ctx* c, TransportParams p, TuneResult* out, const vpmc_opts& o)
{
    const long long sample = std::min<long long>(p.total, (long long)c->num_sms * patient_max_block() * 24);
    TuneResult best;
    best.valid = true;
    if (o.block_size) best.block = o.block_size;
    if (o.aggregate >= 0) best.aggregate = o.aggregate;
    if (o.chunk) best.chunk = o.chunk;
    if (sample <= 0) { *out = best; return VPMC_OK; }
    p.records = nullptr;
    p.rec_cap = 0;
    p.hist_begin = 0;
    p.total = sample;
    p.surrogate = 0;            // timed on the plain beam-line path
    p.chunk = best.chunk;
    p.aggregate = best.aggregate;
    // devices kernel block size (its output is identical for every choice)
    float t_best = 1e30f;
    for (int rep = 0; rep < 2; ++rep)
        for (int block : {384, 512, 640}) {
            CUDA_TRY(cudaMemsetAsync(c->d_phase_count, 0, sizeof(unsigned long long), c->stream));
            vpmc_status st = reset_counters(c);
            if (st != VPMC_OK) return st;
            const float ms = time_launch(c, launch_devices, p, block, 2);
            if (rep == 1 && ms < t_best) { t_best = ms; best.dev_block = block; }
        }
    // patient kernel on the histories the last devices launch handed over
    t_best = 1e30f;
    for (int rep = 0; rep < 2; ++rep)
        for (int block : {512, 640, 768, 896})
            for (int agg : {0, 1})
                for (int chunk : {32, 128}) {
                    if (block > patient_max_block() || (o.block_size && block != o.block_size)) continue;
                    if (o.aggregate >= 0 && agg != o.aggregate) continue;
                    if (o.chunk && chunk != o.chunk) continue;
                    p.aggregate = agg;
                    p.chunk = chunk;
                    vpmc_status st = reset_counters(c);
                    if (st != VPMC_OK) return st;
                    const float ms = time_launch(c, launch_patient, p, block, 1);
                    if (rep == 1 && ms < t_best) {
                        t_best = ms;
                        best.block = block;
                        best.aggregate = agg;
                        best.chunk = chunk;
                    }
                }
    *out = best;
    return VPMC_OK;
}

// Process-wide cache of tuned launch configurations.  The launch choices
// change speed only (results are identical for every choice), so a context
// whose device, grids, field devices and fixed launch options match an
// earlier one reuses that tuning instead of timing ~30 launches again.
struct TuneKey {
    int device, kind;                 // kind 0: dose path, 1: influence matrices
    int ct[3], sg[3];
    unsigned long long fields;        // per set beam: range shifter, aperture, divergent walls, vertex count
    int block, aggregate, chunk;      // launch options the caller fixed
    bool operator==(const TuneKey& o) const
    {
        return device == o.device && kind == o.kind && ct[0] == o.ct[0] && ct[1] == o.ct[1] && ct[2] == o.ct[2] &&
               sg[0] == o.sg[0] && sg[1] == o.sg[1] && sg[2] == o.sg[2] && fields == o.fields &&
               block == o.block && aggregate == o.aggregate && chunk == o.chunk;
    }
};

std::mutex g_tune_mu;
std::vector<std::pair<TuneKey, TuneResult>> g_tune_cache;

TuneKey tune_key(const vpmc_ctx* c, int kind, const vpmc_opts& o)
{
    TuneKey k{};
    k.device = c->device;
    k.kind = kind;
    for (int i = 0; i < 3; ++i) {
        k.ct[i] = c->ctg.n[i];
        k.sg[i] = c->sg.n[i];
    }
    unsigned long long h = 1469598103934665603ull;             // FNV-1a over the fields' device kinds
    for (int b = 0; b < kMaxBeams; ++b) {
        const unsigned long long v = !c->beam_set[b] ? 0ull
                                     : 1ull | (unsigned long long)c->beams[b].rs << 1 |
                                           (unsigned long long)c->beams[b].ap << 2 |
                                           (unsigned long long)(c->beams[b].ap_sad > 0.0f) << 3 |
                                           (unsigned long long)c->beams[b].nvert << 4;
        h = (h ^ v) * 1099511628211ull;
    }
    k.fields = h;
    k.block = o.block_size;
    k.aggregate = o.aggregate;
    k.chunk = o.chunk;
    return k;
}

bool tune_cache_get(const TuneKey& k, TuneResult* out)
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (const auto& e : g_tune_cache)
        if (e.first == k) {
            *out = e.second;
            return true;
        }
    return false;
}

void tune_cache_put(const TuneKey& k, const TuneResult& t)
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (auto& e : g_tune_cache)
        if (e.first == k) {
            e.second = t;
            return;
        }
    g_tune_cache.emplace_back(k, t);
}

TuneResult resolve_launch(const vpmc_opts& o, const TuneResult& t)
{
    TuneResult r = t;
    if (o.block_size) r.block = o.block_size;
    if (o.aggregate >= 0) r.aggregate = o.aggregate;
    if (o.chunk) r.chunk = o.chunk;
    if (!t.valid) r.dev_block = 512;
    return r;
}

// Device time of the beam-line kernels and of the patient kernel over the
// batches the last transport recorded (its work has completed).
vpmc_status add_kernel_times(vpmc_ctx* c, vpmc_stats* acc)
{
    for (int b = 0; b < c->kev_batches; ++b) {
        float a = 0.0f, p = 0.0f;
        CUDA_TRY(cudaEventElapsedTime(&a, c->kev[3 * b], c->kev[3 * b + 1]));
        CUDA_TRY(cudaEventElapsedTime(&p, c->kev[3 * b + 1], c->kev[3 * b + 2]));
        acc->ms_devices += a;
        acc->ms_patient += p;
    }
    return VPMC_OK;
}

vpmc_status read_stats(vpmc_ctx* c, int frac_bits, vpmc_stats* acc, bool add)
{
    unsigned long long h[kNStats];
    CUDA_TRY(cudaMemcpy(h, c->d_stats, sizeof h, cudaMemcpyDeviceToHost));
    const double sc = std::ldexp(1.0, -frac_bits);
    if (!add) *acc = vpmc_stats{};
    acc->e_dep += h[kStDep] * sc;
    acc->e_leak += h[kStLeak] * sc;
    acc->e_rs += h[kStRS] * sc;
    acc->e_aperture += h[kStAp] * sc;
    acc->e_nuc += h[kStNuc] * sc;
    acc->steps += (int64_t)h[kStSteps];
    acc->errors += (int64_t)h[kStErr];
    acc->steps_rs += (int64_t)h[kStStepsRS];
    acc->steps_aperture += (int64_t)h[kStStepsAp];
    return VPMC_OK;
}

}  // namespace

extern "C" {

void vpmc_default_opts(vpmc_opts* o)
{
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->seed = 1234;
    o->mcs = 1;
    o->straggling = 1;
    o->nuclear = 1;
    o->frac_bits = 24;
    o->aggregate = -1;
    o->range_rejection = 1;
    o->surrogate = 0;
}

const char* vpmc_last_error(void) { return g_error.c_str(); }

vpmc_status vpmc_create_geometry(vpmc_ctx** out, const int16_t* hu, int hu_on_device, const vpmc_grid* ct,
                                 const vpmc_hu_curve* curve, const vpmc_grid* dose_grid, void* cuda_stream)
{
    g_error.clear();
    (void)cudaGetLastError();   // a failed call elsewhere in this thread must not leak into ours
    if (!out) return fail(VPMC_ERR_ARG, "out is null");
    *out = nullptr;
    if (!hu || !ct || !curve || !dose_grid) return fail(VPMC_ERR_ARG, "null argument");
    for (const vpmc_grid* g : {ct, dose_grid}) {
        if (g->nx <= 0 || g->ny <= 0 || g->nz <= 0 || !(g->dx > 0) || !(g->dy > 0) || !(g->dz > 0))
            return fail(VPMC_ERR_ARG, "grid with non-positive size or spacing");
        if ((long long)g->nx * g->ny * g->nz > (1ll << 31))
            return fail(VPMC_ERR_ARG, "grid larger than 2^31 voxels");
    }
    const double cd[3] = {ct->dx, ct->dy, ct->dz}, sd[3] = {dose_grid->dx, dose_grid->dy, dose_grid->dz};
    const int cn[3] = {ct->nx, ct->ny, ct->nz}, sn[3] = {dose_grid->nx, dose_grid->ny, dose_grid->nz};
    for (int k = 0; k < 3; ++k) {
        const double ext = cn[k] * cd[k];
        if (std::fabs(sn[k] * sd[k] - ext) > 1e-6 * ext || std::fabs(ct->origin[k] - dose_grid->origin[k]) > 1e-6 * ext)
            return fail(VPMC_ERR_ARG, "dose grid must share the CT's origin and extent (axis %d)", k);
    }
    for (int i = 0; i < 4; ++i)
        if (!(curve->hu[i + 1] > curve->hu[i])) return fail(VPMC_ERR_ARG, "HU knots must be ascending");
    for (int i = 0; i < 5; ++i)
        if (!(curve->density[i] > 0) || !(curve->spr[i] > 0))
            return fail(VPMC_ERR_ARG, "HU curve densities and SPRs must be positive");

    vpmc_ctx* c = new vpmc_ctx();
    auto cleanup = [&](vpmc_status st) {
        vpmc_destroy(c);
        return st;
    };
    if (cudaGetDevice(&c->device) != cudaSuccess) return cleanup(fail(VPMC_ERR_CUDA, "no CUDA device"));
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    int smem_optin = 0;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
    const size_t smem_need = std::max(devices_smem_bytes(), patient_smem_bytes());
    if ((size_t)smem_optin < smem_need)
        return cleanup(fail(VPMC_ERR_CUDA, "device allows %d B shared memory per block, kernels need %zu", smem_optin,
                            smem_need));
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreate(&c->stream) != cudaSuccess) return cleanup(fail(VPMC_ERR_CUDA, "stream creation"));
        c->own_stream = true;
    }
    c->ctg = to_grid3(*ct);
    c->sg = to_grid3(*dose_grid);
    for (int k = 0; k < 3; ++k) { c->ct_spacing[k] = cd[k]; c->sg_spacing[k] = sd[k]; }
    // nested axes: the scoring grid's faces are CT faces (same FP32 origin,
    // FP32 spacing 2^sh x the CT's, 2^sh CT voxels per scoring voxel)
    for (int k = 0; k < 3; ++k) {
        c->nest_shift[k] = -1;
        for (int sh = 0; sh <= 3; ++sh)
            if (c->sg.lo[k] == c->ctg.lo[k] && c->sg.d[k] == std::ldexp(c->ctg.d[k], sh) &&
                (long long)sn[k] << sh == (long long)cn[k]) {
                c->nest_shift[k] = sh;
                break;
            }
    }
    c->nvox = (long long)sn[0] * sn[1] * sn[2];
    for (int i = 0; i < 5; ++i) {
        c->curve15[i] = curve->hu[i];
        c->curve15[5 + i] = curve->density[i];
        c->curve15[10 + i] = curve->spr[i];
    }
    const long long nct = (long long)cn[0] * cn[1] * cn[2];
    vpmc_status st = VPMC_OK;
#define CTX_TRY(expr)                                                                                   \
    do {                                                                                                \
        cudaError_t e_ = (expr);                                                                        \
        if (e_ != cudaSuccess)                                                                          \
            return cleanup(fail(e_ == cudaErrorMemoryAllocation ? VPMC_ERR_OOM : VPMC_ERR_CUDA, "%s: %s", #expr, \
                                cudaGetErrorString(e_)));                                               \
    } while (0)
    CTX_TRY(dev_alloc(&c->d_ct, nct));
    CTX_TRY(cudaMemcpyAsync(c->d_ct, hu, nct * sizeof(int16_t),
                            hu_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    std::vector<unsigned char> img_bytes(sizeof(TablesImage));
    TablesImage* img = reinterpret_cast<TablesImage*>(img_bytes.data());
    build_tables(c->curve15, img);
    c->water_mat = img->mat[kWater];
    c->range_water.assign(img->R[kWater], img->R[kWater] + kNEPad);
    CTX_TRY(dev_alloc(&c->d_tables, 1));
    CTX_TRY(cudaMemcpyAsync(c->d_tables, img, sizeof(TablesImage), cudaMemcpyHostToDevice, c->stream));
    CTX_TRY(dev_alloc(&c->d_curve, 15));
    CTX_TRY(cudaMemcpyAsync(c->d_curve, c->curve15, sizeof(c->curve15), cudaMemcpyHostToDevice, c->stream));
    CTX_TRY(dev_alloc(&c->d_rho, c->nvox));
    CTX_TRY(launch_scoring_density(c->d_ct, c->ctg, c->sg, c->d_curve, c->ct_spacing, c->sg_spacing, c->d_rho,
                                   c->stream));
    CTX_TRY(dev_alloc(&c->d_inv_rho, c->nvox));
    CTX_TRY(dev_alloc(&c->d_inv_rho_f, c->nvox));
    CTX_TRY(launch_reciprocal(c->d_rho, c->nvox, c->d_inv_rho, c->d_inv_rho_f, c->stream));
    // from here on the CT holds the kernels' table index per voxel
    CTX_TRY(launch_ct_lut_index(c->d_ct, nct, c->stream));
    CTX_TRY(dev_alloc(&c->d_beams, kMaxBeams));
    CTX_TRY(dev_alloc(&c->d_counter, 1));
    CTX_TRY(dev_alloc(&c->d_phase_count, 1));
    CTX_TRY(dev_alloc(&c->d_mid_count, 1));
    CTX_TRY(dev_alloc(&c->d_stats, kNStats));
    CTX_TRY(dev_alloc(&c->d_status, 1));
    CTX_TRY(dev_alloc(&c->d_scens, kMaxScen));
    CTX_TRY(cudaEventCreate(&c->ev0));
    CTX_TRY(cudaEventCreate(&c->ev1));
    for (cudaEvent_t& e : c->kev) CTX_TRY(cudaEventCreate(&e));
    CTX_TRY(cudaStreamSynchronize(c->stream));
#undef CTX_TRY
    st = upload_beams(c);
    if (st != VPMC_OK) return cleanup(st);
    *out = c;
    return VPMC_OK;
}

vpmc_status vpmc_set_aperture(vpmc_ctx* c, int beam_id, const vpmc_beam* b)
{
    g_error.clear();
    (void)cudaGetLastError();   // a failed call elsewhere in this thread must not leak into ours
    if (!c || !b) return fail(VPMC_ERR_ARG, "null argument");
    if (beam_id < 0 || beam_id >= kMaxBeams) return fail(VPMC_ERR_ARG, "beam_id %d outside [0, %d)", beam_id, kMaxBeams);
    const double nw = std::sqrt(b->dir[0] * b->dir[0] + b->dir[1] * b->dir[1] + b->dir[2] * b->dir[2]);
    const double nu = std::sqrt(b->bev_x[0] * b->bev_x[0] + b->bev_x[1] * b->bev_x[1] + b->bev_x[2] * b->bev_x[2]);
    const double dot = b->dir[0] * b->bev_x[0] + b->dir[1] * b->bev_x[1] + b->dir[2] * b->bev_x[2];
    if (std::fabs(nw - 1.0) > 1e-6 || std::fabs(nu - 1.0) > 1e-6 || std::fabs(dot) > 1e-6)
        return fail(VPMC_ERR_ARG, "dir and bev_x must be orthonormal");
    DevBeam d{};
    for (int k = 0; k < 3; ++k) {
        d.w[k] = (float)b->dir[k];
        d.u[k] = (float)b->bev_x[k];
        d.iso[k] = (float)b->iso[k];
    }
    const double v[3] = {b->dir[1] * b->bev_x[2] - b->dir[2] * b->bev_x[1],
                         b->dir[2] * b->bev_x[0] - b->dir[0] * b->bev_x[2],
                         b->dir[0] * b->bev_x[1] - b->dir[1] * b->bev_x[0]};
    for (int k = 0; k < 3; ++k) d.v[k] = (float)v[k];
    d.t_src = (float)(-b->source_to_iso_mm);
    double first_device = 1e300;
    d.rs = b->rs_present ? 1 : 0;
    if (d.rs) {
        if (!(b->rs_wet_mm > 0) || !(b->rs_radius_mm > 0)) return fail(VPMC_ERR_ARG, "range shifter: bad WET or radius");
        const double thick = b->rs_wet_mm / pmma_stopping_power_ratio(150.0);
        d.rs_tdn = (float)(-b->rs_down_to_iso_mm);
        d.rs_tup = (float)(-b->rs_down_to_iso_mm - thick);
        d.rs_r2 = (float)(b->rs_radius_mm * b->rs_radius_mm);
        first_device = std::min(first_device, -b->rs_down_to_iso_mm - thick);
    }
    d.ap = b->ap_present ? 1 : 0;
    std::vector<double> poly;
    std::vector<unsigned char> ras;
    std::vector<float> ras_lb;
    if (d.ap) {
        if (!b->poly_xy || b->n_vertices < 3) return fail(VPMC_ERR_ARG, "aperture needs a polygon of >= 3 vertices");
        if (!(b->ap_thickness_mm > 0)) return fail(VPMC_ERR_ARG, "aperture thickness must be positive");
        d.ap_tdn = (float)(-b->ap_down_to_iso_mm);
        d.ap_tup = (float)(-b->ap_down_to_iso_mm - b->ap_thickness_mm);
        first_device = std::min(first_device, -b->ap_down_to_iso_mm - b->ap_thickness_mm);
        if (d.rs && -b->rs_down_to_iso_mm > -b->ap_down_to_iso_mm - b->ap_thickness_mm + 1e-9)
            return fail(VPMC_ERR_ARG, "range shifter must lie upstream of the aperture");
        poly.assign(b->poly_xy, b->poly_xy + 2 * b->n_vertices);
        for (double x : poly)
            if (!std::isfinite(x)) return fail(VPMC_ERR_ARG, "aperture polygon has a non-finite vertex");
        int e1 = 0, e2 = 0;
        if (!polygon_is_simple(poly.data(), b->n_vertices, &e1, &e2))
            return fail(VPMC_ERR_ARG, "aperture polygon is not simple: edges %d and %d meet or overlap", e1, e2);
        double rc = 0.0;
        for (int i = 0; i < b->n_vertices; ++i) rc = std::max(rc, std::hypot(poly[2 * i], poly[2 * i + 1]));
        d.r_circ = (float)rc;
        // divergent walls: the raster is in the downstream face's (projected)
        // coordinates, where a real distance is the projected one x the scale
        // at that depth (>= the entrance's) x the cosine of the wall tilt
        double margin_scale = 1.0;
        if (!(b->ap_sad_mm >= 0.0) || !std::isfinite(b->ap_sad_mm)) return fail(VPMC_ERR_ARG, "ap_sad_mm must be >= 0");
        if (b->ap_sad_mm > 0.0) {
            const double K = -b->ap_down_to_iso_mm + b->ap_sad_mm;
            const double k_up = -b->ap_down_to_iso_mm - b->ap_thickness_mm + b->ap_sad_mm;
            if (!(k_up > 0.0)) return fail(VPMC_ERR_ARG, "the virtual source must lie upstream of the aperture");
            d.ap_sad = (float)b->ap_sad_mm;
            d.ap_K = (float)K;
            d.ap_cos = (float)(K / std::sqrt(K * K + rc * rc));
            margin_scale = 1.0 / ((k_up / K) * (K / std::sqrt(K * K + rc * rc)));
        } else {
            d.ap_sad = 0.0f;
            d.ap_K = 1.0f;
            d.ap_cos = 1.0f;
        }
        ras.resize(kRaster * kRaster);
        ras_lb.resize(kRaster * kRaster);
        // range rejection needs wall distances up to half the block thickness only
        build_raster(poly.data(), b->n_vertices, (0.5 * b->ap_thickness_mm + 1.0) * margin_scale, ras.data(),
                     ras_lb.data(), d.ras_lo, d.ras_inv, &d.ras_diag);
        d.nvert = b->n_vertices;
    }
    if (first_device < 1e300 && !(-b->source_to_iso_mm < first_device))
        return fail(VPMC_ERR_ARG, "source plane must lie upstream of every device");
    const bool prev_set = c->beam_set[beam_id];
    const DevBeam prev = c->beams[beam_id];
    std::vector<double> prev_poly = c->poly[beam_id];
    std::vector<unsigned char> prev_ras = c->raster[beam_id];
    std::vector<float> prev_lb = c->raster_lb[beam_id];
    c->beams[beam_id] = d;
    c->poly[beam_id] = poly;
    c->raster[beam_id] = ras;
    c->raster_lb[beam_id] = ras_lb;
    c->beam_set[beam_id] = true;
    vpmc_status st = upload_beams(c);
    if (st != VPMC_OK) {
        c->beams[beam_id] = prev;
        c->poly[beam_id] = prev_poly;
        c->raster[beam_id] = prev_ras;
        c->raster_lb[beam_id] = prev_lb;
        c->beam_set[beam_id] = prev_set;
        return st;
    }
    c->tune_dose.valid = c->tune_im.valid = false;
    return VPMC_OK;
}

vpmc_status vpmc_run_spots(vpmc_ctx* c, const vpmc_spot* spots, int n_spots, const vpmc_scenario* scen,
                           const vpmc_opts* opts_in, float* dose_dev, vpmc_stats* stats_out)
{
    g_error.clear();
    (void)cudaGetLastError();   // a failed call elsewhere in this thread must not leak into ours
    if (!c || !dose_dev) return fail(VPMC_ERR_ARG, "null context or dose buffer");
    const long long launches0 = c->launches;
    vpmc_opts o;
    vpmc_default_opts(&o);
    if (opts_in) o = *opts_in;
    vpmc_status st = check_opts(&o);
    if (st != VPMC_OK) return st;
    if (o.surrogate && !c->sur_ready) return fail(VPMC_ERR_STATE, "surrogate requested before its weights were set");
    st = check_spots(c, spots, n_spots);
    if (st != VPMC_OK) return st;
    st = check_surrogate_walls(c, spots, n_spots, o.surrogate);
    if (st != VPMC_OK) return st;
    st = pending_status(c);
    if (st != VPMC_OK) return st;
    DevScen sc{{0.0f, 0.0f, 0.0f}, 1.0f};
    if (scen) {
        if (!(scen->spr_scale > 0)) return fail(VPMC_ERR_ARG, "scenario spr_scale must be positive");
        for (int k = 0; k < 3; ++k) sc.shift[k] = (float)scen->shift_mm[k];
        sc.spr_scale = (float)scen->spr_scale;
    }
    // work items: one per spot with histories
    std::vector<DevItem> items;
    long long total = 0;
    double qmax = 0.0, e_in = 0.0;
    const double fs = std::ldexp(1.0, o.frac_bits);
    for (int i = 0; i < n_spots; ++i) {
        const vpmc_spot& s = spots[i];
        if (s.n_hist == 0) continue;
        DevItem it{};
        it.hist_off = total;
        it.E0 = (float)s.energy_mev;
        it.x = (float)s.x_mm;
        it.y = (float)s.y_mm;
        it.sigma = (float)s.sigma_mm;
        it.div_rad = (float)(s.div_mrad * 1e-3);
        it.wscale = (float)(s.weight * fs);
        it.spot = i;
        it.scen = 0;
        it.beam = s.beam;
        it.box = 0;
        if (!(s.weight >= 0.0)) return fail(VPMC_ERR_ARG, "spot %d: negative weight", i);
        items.push_back(it);
        total += s.n_hist;
        qmax += (double)s.n_hist * s.energy_mev * std::max(s.weight, 1.0) * fs;
        e_in += (double)s.n_hist * s.energy_mev;
    }
    if (qmax >= 9.0e18) return fail(VPMC_ERR_ARG, "fixed-point range exceeded: lower frac_bits or weights");
    CUDA_TRY(cudaMemsetAsync(dose_dev, 0, c->nvox * sizeof(float), c->stream));
    if (!c->d_acc) CUDA_TRY(dev_alloc(&c->d_acc, c->nvox));
    CUDA_TRY(cudaMemsetAsync(c->d_acc, 0, c->nvox * sizeof(unsigned long long), c->stream));
    vpmc_stats stats{};
    if (!items.empty()) {
        // sentinel keeps hist_off lookups in range
        st = grow(c, &c->d_items, &c->items_cap, items.size());
        if (st != VPMC_OK) return st;
        st = grow_boxes(c, 1);
        if (st != VPMC_OK) return st;
        DevBox box{};
        box.base = 0;
        for (int k = 0; k < 3; ++k) { box.lo[k] = 0; box.n[k] = c->sg.n[k]; }
        CUDA_TRY(cudaMemcpyAsync(c->d_items, items.data(), items.size() * sizeof(DevItem), cudaMemcpyHostToDevice,
                                 c->stream));
        CUDA_TRY(cudaMemcpyAsync(c->d_boxes, &box, sizeof box, cudaMemcpyHostToDevice, c->stream));
        CUDA_TRY(cudaMemcpyAsync(c->d_scens, &sc, sizeof sc, cudaMemcpyHostToDevice, c->stream));
        TransportParams p = base_params(c, o);
        p.items = c->d_items;
        p.n_items = (int)items.size();
        p.boxes = c->d_boxes;
        p.n_scen = 1;
        p.total = total;
        p.scratch = c->d_acc;
        st = ensure_phase(c, total, p.surrogate != 0);
        if (st != VPMC_OK) return st;
        const bool want_tune = o.block_size == 0 || o.aggregate < 0 || o.chunk == 0;
        if (want_tune && !c->tune_dose.valid) {
            const TuneKey key = tune_key(c, 0, o);
            if (!tune_cache_get(key, &c->tune_dose)) {
                st = autotune(c, p, &c->tune_dose, o);
                if (st != VPMC_OK) return st;
                CUDA_TRY(cudaMemsetAsync(c->d_acc, 0, c->nvox * sizeof(unsigned long long), c->stream));
                tune_cache_put(key, c->tune_dose);
            }
        }
        const TuneResult t = resolve_launch(o, c->tune_dose);
        st = reset_counters(c);
        if (st != VPMC_OK) return st;
        CUDA_TRY(cudaEventRecord(c->ev0, c->stream));
        st = enqueue_transport(c, p, total, t);
        if (st != VPMC_OK) return st;
        CUDA_TRY(cudaEventRecord(c->ev1, c->stream));
        if (!stats_out) c->status_pending = p.surrogate ? 2 : 1;
    }
    const double scale = std::ldexp(1.0, -o.frac_bits) * 1.602176634e-10 /
                         (c->sg_spacing[0] * c->sg_spacing[1] * c->sg_spacing[2] * 1e-3);
    CUDA_TRY(launch_dose_normalise(c->d_acc, c->d_rho, c->nvox, scale, dose_dev, c->stream));
    ++c->launches;
    if (stats_out) {
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        if (!items.empty()) {
            st = read_stats(c, o.frac_bits, &stats, false);
            if (st != VPMC_OK) return st;
            float ms = 0.0f;
            CUDA_TRY(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
            stats.ms = ms;
            st = add_kernel_times(c, &stats);
            if (st != VPMC_OK) return st;
            int status = 0;
            CUDA_TRY(cudaMemcpy(&status, c->d_status, sizeof status, cudaMemcpyDeviceToHost));
            stats.histories = total;
            stats.e_in = e_in;
            stats.launches = c->launches - launches0;
            *stats_out = stats;
            if (status & 1) return fail(VPMC_ERR_TIMEOUT, "%lld histories reached the iteration cap", (long long)stats.errors);
            if (status & 6) return fail(VPMC_ERR_DEVICE_FLAG, "hand-off or query buffer overflow (status %d)", status);
            if (o.surrogate) {
                int ss = 0;
                CUDA_TRY(cudaMemcpy(&ss, c->sur.status, sizeof ss, cudaMemcpyDeviceToHost));
                if (ss) return fail(VPMC_ERR_TIMEOUT, "surrogate: a tensor-core wait timed out");
            }
        } else {
            stats.launches = c->launches - launches0;
            *stats_out = stats;
        }
    }
    return VPMC_OK;
}

namespace {

struct BoxSpec { int lo[3], n[3]; };

// Beam b's field in scenario sc, in the beam frame (origin base = isocentre +
// shift, axes u, v across and w along the beam): the lateral extent of the
// aperture opening (or of the spots, 4 sigma) and the depth range [t0, t1] of
// the scoring grid along w.
struct FieldFrame {
    double a0, a1, b0, b1;
    double base[3];
    double t0, t1;
};

FieldFrame field_frame(vpmc_ctx* c, int b, const vpmc_scenario& sc, const vpmc_spot* spots, int n_spots)
{
    const DevBeam& B = c->beams[b];
    FieldFrame f;
    f.a0 = f.b0 = 1e300;
    f.a1 = f.b1 = -1e300;
    if (B.ap) {
        const std::vector<double>& p = c->poly[b];
        for (size_t i = 0; i + 1 < p.size(); i += 2) {
            f.a0 = std::min(f.a0, p[i]); f.a1 = std::max(f.a1, p[i]);
            f.b0 = std::min(f.b0, p[i + 1]); f.b1 = std::max(f.b1, p[i + 1]);
        }
    } else {
        for (int i = 0; i < n_spots; ++i)
            if (spots[i].beam == b) {
                const double r = 4.0 * spots[i].sigma_mm;
                f.a0 = std::min(f.a0, spots[i].x_mm - r); f.a1 = std::max(f.a1, spots[i].x_mm + r);
                f.b0 = std::min(f.b0, spots[i].y_mm - r); f.b1 = std::max(f.b1, spots[i].y_mm + r);
            }
    }
    double lo[3], hi[3];
    for (int k = 0; k < 3; ++k) {
        lo[k] = c->sg.lo[k];
        hi[k] = c->sg.lo[k] + c->sg.n[k] * c->sg_spacing[k];
        f.base[k] = (double)B.iso[k] + sc.shift_mm[k];
    }
    // depth range: projections of the grid corners on the beam axis
    f.t0 = 1e300;
    f.t1 = -1e300;
    for (int m = 0; m < 8; ++m) {
        double t = 0.0;
        for (int k = 0; k < 3; ++k) t += (((m >> k) & 1 ? hi[k] : lo[k]) - f.base[k]) * (double)B.w[k];
        f.t0 = std::min(f.t0, t);
        f.t1 = std::max(f.t1, t);
    }
    return f;
}

// Axis-aligned box (scoring voxels) that holds the field's lateral extent plus
// a margin over the depths [t0, min(t1, t_cap)].
BoxSpec frame_box(vpmc_ctx* c, int b, const FieldFrame& f, double margin, double t_cap)
{
    const DevBeam& B = c->beams[b];
    const double a0 = f.a0 - margin, a1 = f.a1 + margin, b0 = f.b0 - margin, b1 = f.b1 + margin;
    const double t_hi = std::max(std::min(f.t1, t_cap), f.t0);
    double plo[3] = {1e300, 1e300, 1e300}, phi[3] = {-1e300, -1e300, -1e300};
    for (int m = 0; m < 8; ++m) {
        const double a = m & 1 ? a1 : a0, bb = m & 2 ? b1 : b0, t = m & 4 ? t_hi : f.t0;
        for (int k = 0; k < 3; ++k) {
            const double x = f.base[k] + a * B.u[k] + bb * B.v[k] + t * B.w[k];
            plo[k] = std::min(plo[k], x);
            phi[k] = std::max(phi[k], x);
        }
    }
    BoxSpec s;
    for (int k = 0; k < 3; ++k) {
        const double lo = c->sg.lo[k];
        int i0 = (int)std::floor((plo[k] - lo) / c->sg_spacing[k]);
        int i1 = (int)std::ceil((phi[k] - lo) / c->sg_spacing[k]);
        i0 = std::max(i0, 0);
        i1 = std::min(i1, c->sg.n[k]);
        s.lo[k] = i0;
        s.n[k] = std::max(i1 - i0, 0);
    }
    return s;
}

// Residual range in water (mm) at energy e, from the host copy of the table
// the kernels interpolate.
double water_range(const vpmc_ctx* c, double e)
{
    const double x = std::max(e, 0.0) * 10.0;
    const int i = std::min((int)x, kNE - 1);
    const float2 v = c->range_water[i];
    return (double)v.x + (x - i) * (double)v.y;
}

// A run: consecutive spots of one beam whose column boxes share a shape (one
// energy layer, or several merged).  r_lim: water-equivalent path (mm) beyond
// which none of the run's protons deposits -- the water range behind the
// range shifter, with 5 % + 3 mm for range straggling and table rounding.
struct Run {
    int first, count, beam;
    double r_lim;
};

long long box_elems(const BoxSpec& s) { return (long long)s.n[0] * s.n[1] * s.n[2]; }

}  // namespace

vpmc_status vpmc_influence_matrix(vpmc_ctx* c, const vpmc_spot* spots, int n_spots, const vpmc_scenario* scen,
                                  int n_scen, const vpmc_opts* opts_in, float rel_threshold, vpmc_csr* out,
                                  vpmc_stats* stats_out)
{
    g_error.clear();
    (void)cudaGetLastError();   // a failed call elsewhere in this thread must not leak into ours
    if (!c || !out || !scen || n_scen <= 0) return fail(VPMC_ERR_ARG, "null argument or no scenario");
    const long long launches0 = c->launches;
    if (n_scen > kMaxScen) return fail(VPMC_ERR_ARG, "at most %d scenarios per call", kMaxScen);
    if (!(rel_threshold >= 0.0f && rel_threshold < 1.0f)) return fail(VPMC_ERR_ARG, "rel_threshold outside [0, 1)");
    for (int s = 0; s < n_scen; ++s) out[s] = vpmc_csr{};
    vpmc_opts o;
    vpmc_default_opts(&o);
    if (opts_in) o = *opts_in;
    vpmc_status st = check_opts(&o);
    if (st != VPMC_OK) return st;
    if (o.surrogate && !c->sur_ready) return fail(VPMC_ERR_STATE, "surrogate requested before its weights were set");
    st = check_spots(c, spots, n_spots);
    if (st != VPMC_OK) return st;
    st = check_surrogate_walls(c, spots, n_spots, o.surrogate);
    if (st != VPMC_OK) return st;
    if (n_spots == 0) return fail(VPMC_ERR_ARG, "no spots");
    st = pending_status(c);
    if (st != VPMC_OK) return st;
    for (int i = 1; i < n_spots; ++i)
        if (spots[i].beam < spots[i - 1].beam) return fail(VPMC_ERR_ARG, "spots must be sorted by beam id");
    for (int s = 0; s < n_scen; ++s)
        if (!(scen[s].spr_scale > 0)) return fail(VPMC_ERR_ARG, "scenario %d: spr_scale must be positive", s);
    const double fs = std::ldexp(1.0, o.frac_bits);
    for (int i = 0; i < n_spots; ++i)
        if ((double)spots[i].n_hist * spots[i].energy_mev * fs >= 9.0e18)
            return fail(VPMC_ERR_ARG, "spot %d: fixed-point range exceeded, lower frac_bits", i);

    // beams in use: spots of beam b are the contiguous range [beam_first, +beam_count)
    int nb = 0;
    for (int i = 0; i < n_spots; ++i) nb = std::max(nb, spots[i].beam + 1);
    std::vector<int> beam_first(nb, 0), beam_count(nb, 0);
    for (int i = n_spots - 1; i >= 0; --i) beam_first[spots[i].beam] = i;
    for (int i = 0; i < n_spots; ++i) beam_count[spots[i].beam] += 1;
    std::vector<DevScen> dscen(n_scen);
    for (int s = 0; s < n_scen; ++s) {
        for (int k = 0; k < 3; ++k) dscen[s].shift[k] = (float)scen[s].shift_mm[k];
        dscen[s].spr_scale = (float)scen[s].spr_scale;
    }
    // runs: consecutive spots of one beam and one energy, at most kMaxRuns per
    // beam (adjacent runs merged beyond that)
    constexpr int kMaxRuns = 64;
    std::vector<Run> runs;
    for (int b = 0; b < nb; ++b) {
        if (!beam_count[b]) continue;
        const DevBeam& B = c->beams[b];
        const double rs_wet = B.rs ? (double)(B.rs_tdn - B.rs_tup) * pmma_stopping_power_ratio(150.0) : 0.0;
        std::vector<Run> br;
        for (int j = beam_first[b]; j < beam_first[b] + beam_count[b]; ++j) {
            const double r = std::max(water_range(c, spots[j].energy_mev) - 0.97 * rs_wet, 0.0) * 1.05 + 3.0;
            if (br.empty() || spots[j].energy_mev != spots[br.back().first].energy_mev)
                br.push_back(Run{j, 0, b, 0.0});
            br.back().count += 1;
            br.back().r_lim = std::max(br.back().r_lim, r);
        }
        const int merge = ((int)br.size() + kMaxRuns - 1) / kMaxRuns;
        for (size_t i = 0; i < br.size(); i += merge) {
            Run m = br[i];
            for (size_t k = i + 1; k < std::min(br.size(), i + merge); ++k) {
                m.count += br[k].count;
                m.r_lim = std::max(m.r_lim, br[k].r_lim);
            }
            runs.push_back(m);
        }
    }
    const int nr = (int)runs.size();
    // each run's reach along its field's axis in each scenario (one kernel
    // marching rays through the CT), then its box: the field plus a lateral
    // margin, from the grid's near end to the reach plus a margin
    std::vector<FieldFrame> frames((size_t)n_scen * nb);
    std::vector<float> reach((size_t)n_scen * nr, 0.0f);
    {
        std::vector<DepthJob> jobs;
        std::vector<float> rl;
        std::vector<int> slot((size_t)n_scen * nr);     // (scenario, run) -> entry of rl / reach
        for (int s = 0; s < n_scen; ++s)
            for (int b = 0; b < nb; ++b) {
                if (!beam_count[b]) continue;
                const FieldFrame f = field_frame(c, b, scen[s], spots, n_spots);
                frames[(size_t)s * nb + b] = f;
                const DevBeam& B = c->beams[b];
                std::vector<int> mine;
                for (int r = 0; r < nr; ++r)
                    if (runs[r].beam == b) mine.push_back(r);
                std::sort(mine.begin(), mine.end(), [&](int x, int y) { return runs[x].r_lim < runs[y].r_lim; });
                DepthJob J{};
                for (int k = 0; k < 3; ++k) {
                    J.base[k] = (float)f.base[k];
                    J.u[k] = B.u[k]; J.v[k] = B.v[k]; J.w[k] = B.w[k];
                }
                const double lat = 10.0, da = 2.0;
                J.a0 = (float)(f.a0 - lat);
                J.b0 = (float)(f.b0 - lat);
                J.da = (float)da;
                J.na = std::max(1, (int)std::ceil((f.a1 - f.a0 + 2 * lat) / da) + 1);
                J.nb = std::max(1, (int)std::ceil((f.b1 - f.b0 + 2 * lat) / da) + 1);
                J.t0 = (float)f.t0;
                J.t1 = (float)f.t1;
                J.dt = 0.5f;
                J.spr_scale = (float)scen[s].spr_scale;
                J.run_off = (int)rl.size();
                J.run_n = (int)mine.size();
                for (int r : mine) {
                    slot[(size_t)s * nr + r] = (int)rl.size();
                    rl.push_back((float)runs[r].r_lim);
                }
                jobs.push_back(J);
            }
        DepthJob* d_jobs = nullptr;
        float* d_rl = nullptr;
        unsigned* d_reach = nullptr;
        std::vector<unsigned> h_reach(rl.size(), 0u);
        cudaError_t e = ensure(c->im_jobs, jobs.size(), &d_jobs);
        if (e == cudaSuccess) e = ensure(c->im_rlim, rl.size(), &d_rl);
        if (e == cudaSuccess) e = ensure(c->im_reach, rl.size(), &d_reach);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_jobs, jobs.data(), jobs.size() * sizeof(DepthJob), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_rl, rl.data(), rl.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(d_reach, 0, rl.size() * sizeof(unsigned), c->stream);
        if (e == cudaSuccess)
            e = launch_depth_bounds(reinterpret_cast<const uint16_t*>(c->d_ct), c->d_tables, c->ctg, d_jobs,
                                    (int)jobs.size(), d_rl, d_reach, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h_reach.data(), d_reach, rl.size() * sizeof(unsigned), cudaMemcpyDeviceToHost,
                                c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess)
            return fail(e == cudaErrorMemoryAllocation ? VPMC_ERR_OOM : VPMC_ERR_CUDA, "column-box depths: %s",
                        cudaGetErrorString(e));
        ++c->launches;
        for (size_t i = 0; i < slot.size(); ++i) {
            unsigned bits = h_reach[slot[i]];
            float v;
            std::memcpy(&v, &bits, sizeof v);
            reach[i] = v;
        }
    }
    std::vector<BoxSpec> spec((size_t)n_scen * nr);
    std::vector<long long> scen_elems(n_scen, 0);
    long long per_scen_elems_max = 0;
    for (int s = 0; s < n_scen; ++s) {
        for (int r = 0; r < nr; ++r) {
            const FieldFrame& f = frames[(size_t)s * nb + runs[r].beam];
            spec[(size_t)s * nr + r] = frame_box(c, runs[r].beam, f, 25.0, f.t0 + reach[(size_t)s * nr + r] + 5.0);
            scen_elems[s] += box_elems(spec[(size_t)s * nr + r]) * runs[r].count;
        }
        per_scen_elems_max = std::max(per_scen_elems_max, scen_elems[s]);
    }
    size_t free_b = 0, total_b = 0;
    CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    long long budget = (long long)((double)(free_b + c->scratch_cap * 8) * 0.80 / 8.0);
    if (per_scen_elems_max > budget)
        return fail(VPMC_ERR_OOM, "one scenario needs %.1f GB of column scratch, %.1f GB available",
                    per_scen_elems_max * 8e-9, budget * 8e-9);

    std::vector<double> item_scale(n_spots);
    const double vol_cm3 = c->sg_spacing[0] * c->sg_spacing[1] * c->sg_spacing[2] * 1e-3;
    for (int j = 0; j < n_spots; ++j)
        item_scale[j] = spots[j].n_hist > 0 ? std::ldexp(1.0, -o.frac_bits) * 1.602176634e-10 / vol_cm3 /
                                                  (double)spots[j].n_hist
                                            : 0.0;
    // per-call buffers
    double* d_colmax = nullptr;
    double* d_item_scale = nullptr;
    long long* d_rowcnt = nullptr;
    long long* d_nnz = nullptr;
    long long* d_scan_tmp = nullptr;
    int* d_beam_meta = nullptr;
    long long* d_bucket_off = nullptr;
    long long* d_bucket_cur = nullptr;
    int* d_bucket_len = nullptr;
    OvfRec* d_ovf_sorted = nullptr;
    unsigned long long* d_ovf_count = nullptr;
    // the work arrays are the context's (kept between calls); on failure the
    // library's own CSR buffers are freed, a caller allocator's are left to it
    auto release = [&]() {};
    auto drop_outputs = [&]() {
        if (c->csr_alloc) {
            for (int s = 0; s < n_scen; ++s) out[s] = vpmc_csr{};
        } else {
            vpmc_free_csr(out, n_scen);
        }
    };
    auto out_alloc = [&](void** p, size_t bytes) -> cudaError_t {
        *p = nullptr;
        if (!c->csr_alloc) return cudaMalloc(p, bytes == 0 ? 1 : bytes);
        if (bytes == 0) return cudaSuccess;
        *p = c->csr_alloc(bytes, c->csr_alloc_user);
        return *p ? cudaSuccess : cudaErrorMemoryAllocation;
    };
#define IM_TRY(expr)                                                                                    \
    do {                                                                                                \
        cudaError_t e_ = (expr);                                                                        \
        if (e_ != cudaSuccess) {                                                                        \
            release();                                                                                  \
            drop_outputs();                                                                             \
            return fail(e_ == cudaErrorMemoryAllocation ? VPMC_ERR_OOM : VPMC_ERR_CUDA, "%s: %s", #expr, \
                        cudaGetErrorString(e_));                                                        \
        }                                                                                               \
    } while (0)
#define IM_ST(expr)                                                                                     \
    do {                                                                                                \
        vpmc_status s_ = (expr);                                                                        \
        if (s_ != VPMC_OK) { release(); drop_outputs(); return s_; }                                    \
    } while (0)
    IM_TRY(ensure(c->im_item_scale, n_spots, &d_item_scale));
    IM_TRY(cudaMemcpy(d_item_scale, item_scale.data(), n_spots * sizeof(double), cudaMemcpyHostToDevice));
    IM_TRY(ensure(c->im_rowcnt, (size_t)n_scen * (c->nvox + 1), &d_rowcnt));
    IM_TRY(ensure(c->im_nnz, (size_t)n_scen, &d_nnz));
    IM_TRY(ensure(c->im_scan_tmp, scan_tmp_elems((long long)n_scen * c->nvox + 1), &d_scan_tmp));
    IM_TRY(ensure(c->im_meta, (4 * (size_t)nr + 1) * n_scen, &d_beam_meta));
    IM_TRY(ensure(c->im_ovf_count, 1, &d_ovf_count));
    IM_TRY(cudaMemcpy(c->d_scens, dscen.data(), n_scen * sizeof(DevScen), cudaMemcpyHostToDevice));

    vpmc_stats stats{};
    float total_ms = 0.0f;
    int s0 = 0;
    while (s0 < n_scen) {
        // a wave = consecutive scenarios whose column scratch fits the budget
        int s1 = s0;
        long long wave_elems = 0;
        while (s1 < n_scen && wave_elems + scen_elems[s1] <= budget) wave_elems += scen_elems[s1++];
        const int ns = s1 - s0;
        {
            vpmc_status gs = grow_scratch(c, (size_t)wave_elems);
            if (gs == VPMC_ERR_OOM && ns > 1) {
                budget = std::max(per_scen_elems_max, wave_elems / 2);
                (void)cudaGetLastError();
                continue;
            }
            if (gs != VPMC_OK) {
                size_t fb = 0, tb = 0;
                cudaMemGetInfo(&fb, &tb);
                IM_ST(fail(VPMC_ERR_OOM, "column scratch of %.1f GB for %d scenario(s) does not fit (%.1f GB free)",
                           wave_elems * 8e-9, ns, fb * 1e-9));
            }
        }
        // items (scenario-major, spot order) and their boxes
        std::vector<DevItem> items((size_t)ns * n_spots);
        std::vector<DevBox> boxes;
        std::vector<int> run_box((size_t)ns * nr, 0);
        boxes.reserve(items.size() + (size_t)ns * nr);
        long long base = 0, total = 0;
        for (int s = s0; s < s1; ++s) {
            for (int r = 0; r < nr; ++r) {
                const BoxSpec& sp = spec[(size_t)s * nr + r];
                DevBox bx{};
                for (int k = 0; k < 3; ++k) { bx.lo[k] = sp.lo[k]; bx.n[k] = sp.n[k]; }
                bx.base = base;
                run_box[(size_t)(s - s0) * nr + r] = (int)boxes.size();
                boxes.push_back(bx);
                for (int j = runs[r].first; j < runs[r].first + runs[r].count; ++j) {
                    const vpmc_spot& sp_j = spots[j];
                    DevItem it{};
                    it.hist_off = total;
                    it.E0 = (float)sp_j.energy_mev;
                    it.x = (float)sp_j.x_mm;
                    it.y = (float)sp_j.y_mm;
                    it.sigma = (float)sp_j.sigma_mm;
                    it.div_rad = (float)(sp_j.div_mrad * 1e-3);
                    it.wscale = (float)fs;
                    it.spot = j;
                    it.scen = s;
                    it.beam = runs[r].beam;
                    DevBox ib = bx;
                    ib.base = base;
                    base += box_elems(sp);
                    it.box = (int)boxes.size();
                    boxes.push_back(ib);
                    items[(size_t)(s - s0) * n_spots + j] = it;
                    total += sp_j.n_hist;
                }
            }
        }
        IM_ST(grow(c, &c->d_items, &c->items_cap, items.size()));
        IM_ST(grow_boxes(c, boxes.size()));
        IM_TRY(cudaMemcpy(c->d_items, items.data(), items.size() * sizeof(DevItem), cudaMemcpyHostToDevice));
        IM_TRY(cudaMemcpy(c->d_boxes, boxes.data(), boxes.size() * sizeof(DevBox), cudaMemcpyHostToDevice));
        if (!c->d_ovf) IM_ST(grow_ovf(c, 1ll << 24));
        IM_ST(ensure_phase(c, total, o.surrogate && c->sur_ready));
        TransportParams p = base_params(c, o);
        p.items = c->d_items;
        // the wave's scenarios share the beam-line transport (the random
        // numbers do not depend on the scenario): the beam-line kernels run
        // over the first scenario's items, and each survivor is handed to the
        // patient kernel once per scenario
        const long long per_scen = total / ns;
        p.n_items = n_spots;
        p.n_rep = ns;
        p.rep_items = n_spots;
        p.rep_hist = per_scen;
        p.rep_cap = c->phase_cap / ns;
        p.boxes = c->d_boxes;
        p.n_scen = n_scen;
        p.total = per_scen;
        p.scratch = c->d_scratch;
        p.unit_weight = 1;              // every item's wscale is 2^F
        p.records = nullptr;
        p.rec_cap = 0;
        p.ovf_count = d_ovf_count;
        const bool want_tune = o.block_size == 0 || o.aggregate < 0 || o.chunk == 0;
        if (want_tune && !c->tune_im.valid) {
            const TuneKey key = tune_key(c, 1, o);
            if (!tune_cache_get(key, &c->tune_im)) {
                p.ovf = c->d_ovf;
                p.ovf_cap = c->ovf_cap;
                IM_TRY(cudaMemsetAsync(d_ovf_count, 0, sizeof(unsigned long long), c->stream));
                IM_ST(autotune(c, p, &c->tune_im, o));
                tune_cache_put(key, c->tune_im);
            }
        }
        const TuneResult tr = resolve_launch(o, c->tune_im);
        unsigned long long n_ovf = 0;
        for (int attempt = 0;; ++attempt) {
            p.ovf = c->d_ovf;
            p.ovf_cap = c->ovf_cap;
            // zero the wave's columns and counters; the transport batches run as one CUDA graph
            IM_TRY(cudaMemsetAsync(c->d_scratch, 0, (size_t)wave_elems * sizeof(unsigned long long), c->stream));
            IM_TRY(cudaMemsetAsync(d_ovf_count, 0, sizeof(unsigned long long), c->stream));
            IM_ST(reset_counters(c));
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            IM_TRY(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
            vpmc_status qs = enqueue_transport(c, p, per_scen, tr);
            cudaError_t ce = cudaStreamEndCapture(c->stream, &graph);
            IM_ST(qs);
            IM_TRY(ce);
            cudaError_t ge = cudaGraphInstantiate(&exec, graph, 0);
            if (ge == cudaSuccess) ge = cudaEventRecord(c->ev0, c->stream);
            if (ge == cudaSuccess) ge = cudaGraphLaunch(exec, c->stream);
            if (ge == cudaSuccess) ge = cudaEventRecord(c->ev1, c->stream);
            if (ge == cudaSuccess) ge = cudaStreamSynchronize(c->stream);
            if (exec) cudaGraphExecDestroy(exec);
            if (graph) cudaGraphDestroy(graph);
            IM_TRY(ge);
            IM_TRY(cudaMemcpy(&n_ovf, d_ovf_count, sizeof n_ovf, cudaMemcpyDeviceToHost));
            if ((long long)n_ovf <= c->ovf_cap) break;
            // the tail records did not fit: enlarge the buffer and run the wave again
            if (attempt > 0) IM_ST(fail(VPMC_ERR_OOM, "out-of-box records keep overflowing (%llu)", n_ovf));
            IM_ST(grow_ovf(c, (long long)(n_ovf * 1.25) + 1024));
        }
        float ms = 0.0f;
        IM_TRY(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
        total_ms += ms;
        IM_ST(read_stats(c, o.frac_bits, &stats, true));
        IM_ST(add_kernel_times(c, &stats));
        int status = 0;
        IM_TRY(cudaMemcpy(&status, c->d_status, sizeof status, cudaMemcpyDeviceToHost));
        if (status & 1) {
            release();
            drop_outputs();
            return fail(VPMC_ERR_TIMEOUT, "histories reached the iteration cap");
        }
        if (status & 6) {
            release();
            drop_outputs();
            return fail(VPMC_ERR_DEVICE_FLAG, "hand-off or query buffer overflow (status %d)", status);
        }
        if (o.surrogate && c->sur_ready) {
            int ss = 0;
            IM_TRY(cudaMemcpy(&ss, c->sur.status, sizeof ss, cudaMemcpyDeviceToHost));
            if (ss) {
                release();
                drop_outputs();
                return fail(VPMC_ERR_TIMEOUT, "surrogate: a tensor-core wait timed out");
            }
        }
        stats.ovf_records += (long long)n_ovf;
        stats.scratch_bytes += wave_elems * (long long)sizeof(unsigned long long);
        // column maxima over boxes, then bucket the out-of-box records and raise the maxima
        IM_TRY(ensure(c->im_colmax, items.size(), &d_colmax));
        IM_TRY(launch_column_max(c->d_scratch, c->d_items, c->d_boxes, c->d_inv_rho, c->d_inv_rho_f, c->sg, 0,
                                 (int)items.size(), d_colmax, c->stream));
        ++c->launches;
        const long long n_buckets = (long long)ns * c->nvox;
        if (n_ovf) {
            IM_TRY(ensure(c->im_bucket_off, n_buckets + 1, &d_bucket_off));
            IM_TRY(ensure(c->im_bucket_cur, n_buckets + 1, &d_bucket_cur));
            IM_TRY(ensure(c->im_bucket_len, n_buckets, &d_bucket_len));
            IM_TRY(ensure(c->im_ovf_sorted, n_ovf, &d_ovf_sorted));
            IM_TRY(cudaMemsetAsync(d_bucket_cur, 0, (n_buckets + 1) * sizeof(long long), c->stream));
            IM_TRY(launch_ovf_count(c->d_ovf, (long long)n_ovf, n_spots, c->nvox, d_bucket_cur, c->stream));
            IM_TRY(launch_exclusive_scan(d_bucket_cur, d_bucket_off, n_buckets + 1, d_scan_tmp, c->stream));
            IM_TRY(cudaMemsetAsync(d_bucket_cur, 0, (n_buckets + 1) * sizeof(long long), c->stream));
            IM_TRY(launch_ovf_scatter(c->d_ovf, (long long)n_ovf, n_spots, c->nvox, d_bucket_off, d_bucket_cur,
                                      d_ovf_sorted, c->stream));
            IM_TRY(launch_ovf_merge(d_ovf_sorted, d_bucket_off, n_buckets, c->nvox, c->d_rho, d_bucket_len, d_colmax,
                                    c->stream));
            c->launches += 3 + scan_launches(n_buckets + 1);
        }
        // per column: the threshold in FP64 and FP32 (the row passes' screen)
        double* d_thr = nullptr;
        float* d_thr_f = nullptr;
        IM_TRY(ensure(c->im_thr, items.size(), &d_thr));
        IM_TRY(ensure(c->im_thr_f, items.size(), &d_thr_f));
        IM_TRY(launch_column_threshold(d_colmax, (int)items.size(), (double)rel_threshold, d_thr, d_thr_f, c->stream));
        ++c->launches;
        // CSR per scenario: every scenario's count pass and row-pointer scan,
        // one read of the entry counts, then the fill passes
        const size_t meta_stride = 4 * (size_t)nr + 1;
        std::vector<int> meta(meta_stride * ns, 0);
        std::vector<int> count_blocks(ns, 0);
        for (int s = s0; s < s1; ++s) {
            int* m = meta.data() + meta_stride * (s - s0);
            int blocks = 0;
            for (int r = 0; r < nr; ++r) {
                m[r] = runs[r].first;
                m[nr + r] = runs[r].count;
                m[2 * nr + r] = run_box[(size_t)(s - s0) * nr + r];
                m[3 * nr + r] = blocks;
                blocks += (int)((box_elems(spec[(size_t)s * nr + r]) + kCountBlock - 1) / kCountBlock);
            }
            m[4 * nr] = blocks;
            count_blocks[s - s0] = blocks;
        }
        IM_TRY(cudaMemcpyAsync(d_beam_meta, meta.data(), meta.size() * sizeof(int), cudaMemcpyHostToDevice,
                               c->stream));
        // one slot per box-major thread of every scenario of the wave
        std::vector<size_t> slot0(ns + 1, 0);
        for (int k = 0; k < ns; ++k) slot0[k + 1] = slot0[k] + (size_t)count_blocks[k] * kCountBlock;
        unsigned* d_box_slot = nullptr;
        IM_TRY(ensure(c->im_box_slot, slot0[ns], &d_box_slot));
        std::vector<CsrBuildParams> cps(ns);
        for (int s = s0; s < s1; ++s) {
            const int first = (s - s0) * n_spots;
            const int* m = d_beam_meta + meta_stride * (s - s0);
            long long* rowcnt = d_rowcnt + (size_t)(s - s0) * (c->nvox + 1);
            CsrBuildParams& cp = cps[s - s0];
            cp = CsrBuildParams{};
            cp.scratch = c->d_scratch;
            cp.items = c->d_items + first;
            cp.boxes = c->d_boxes;
            cp.inv_rho = c->d_inv_rho;
            cp.thr = d_thr + first;
            cp.thr_f = d_thr_f + first;
            cp.run_first = m;
            cp.run_count = m + nr;
            cp.run_box = m + 2 * nr;
            cp.run_block0 = m + 3 * nr;
            cp.box_slot = d_box_slot + slot0[s - s0];
            cp.n_runs = nr;
            cp.ovf = n_ovf ? d_ovf_sorted : nullptr;
            cp.bucket_off = n_ovf ? d_bucket_off + (long long)(s - s0) * c->nvox : nullptr;
            cp.bucket_len = n_ovf ? d_bucket_len + (long long)(s - s0) * c->nvox : nullptr;
            cp.item_base = first;
            cp.sg = c->sg;
            cp.nvox = c->nvox;
            cp.item_scale = d_item_scale;
            cp.row_count = rowcnt;
            IM_TRY(cudaMemsetAsync(rowcnt, 0, (c->nvox + 1) * sizeof(long long), c->stream));
            IM_TRY(launch_csr_count(cp, count_blocks[s - s0], c->stream));
            c->launches += n_ovf ? 2 : 1;
            vpmc_csr& csr = out[s];
            csr.n_rows = c->nvox;
            csr.n_cols = n_spots;
            IM_TRY(out_alloc(reinterpret_cast<void**>(&csr.row_ptr), (c->nvox + 1) * sizeof(int64_t)));
            IM_TRY(launch_exclusive_scan(rowcnt, reinterpret_cast<long long*>(csr.row_ptr), c->nvox + 1, d_scan_tmp,
                                         c->stream));
            c->launches += scan_launches(c->nvox + 1);
            IM_TRY(cudaMemcpyAsync(d_nnz + (s - s0), csr.row_ptr + c->nvox, sizeof(long long),
                                   cudaMemcpyDeviceToDevice, c->stream));
        }
        std::vector<long long> nnz(ns, 0);
        IM_TRY(cudaMemcpyAsync(nnz.data(), d_nnz, ns * sizeof(long long), cudaMemcpyDeviceToHost, c->stream));
        IM_TRY(cudaStreamSynchronize(c->stream));
        for (int s = s0; s < s1; ++s) {
            vpmc_csr& csr = out[s];
            CsrBuildParams& cp = cps[s - s0];
            csr.nnz = nnz[s - s0];
            IM_TRY(out_alloc(reinterpret_cast<void**>(&csr.col), csr.nnz * sizeof(int32_t)));
            IM_TRY(out_alloc(reinterpret_cast<void**>(&csr.val), csr.nnz * sizeof(float)));
            cp.row_ptr = reinterpret_cast<const long long*>(csr.row_ptr);
            cp.col = csr.col;
            cp.val = csr.val;
            IM_TRY(launch_csr_fill(cp, count_blocks[s - s0], c->stream));
            c->launches += 2;
        }
        IM_TRY(cudaStreamSynchronize(c->stream));
        s0 = s1;
    }
    release();
#undef IM_TRY
#undef IM_ST
    if (stats_out) {
        double e_in = 0.0;
        long long h = 0;
        for (int j = 0; j < n_spots; ++j) {
            e_in += (double)spots[j].n_hist * spots[j].energy_mev;
            h += spots[j].n_hist;
        }
        stats.e_in = e_in * n_scen;
        stats.histories = h * n_scen;
        stats.ms = total_ms;
        stats.launches = c->launches - launches0;
        *stats_out = stats;
    }
    return VPMC_OK;
}

vpmc_status vpmc_set_csr_allocator(vpmc_ctx* c, vpmc_alloc_fn alloc, void* user)
{
    g_error.clear();
    if (!c) return fail(VPMC_ERR_ARG, "null context");
    c->csr_alloc = alloc;
    c->csr_alloc_user = alloc ? user : nullptr;
    return VPMC_OK;
}

vpmc_status vpmc_free_csr(vpmc_csr* csr, int n)
{
    if (!csr || n < 0) return fail(VPMC_ERR_ARG, "null csr array");
    for (int i = 0; i < n; ++i) {
        cudaFree(csr[i].row_ptr);
        cudaFree(csr[i].col);
        cudaFree(csr[i].val);
        csr[i] = vpmc_csr{};
    }
    return VPMC_OK;
}

void vpmc_destroy(vpmc_ctx* c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    cudaFree(c->d_ct);
    cudaFree(c->d_tables);
    cudaFree(c->d_curve);
    cudaFree(c->d_rho);
    cudaFree(c->d_inv_rho);
    cudaFree(c->d_inv_rho_f);
    cudaFree(c->d_acc);
    cudaFree(c->d_beams);
    cudaFree(c->d_poly);
    cudaFree(c->d_raster);
    cudaFree(c->d_raster_lb);
    cudaFree(c->d_counter);
    cudaFree(c->d_stats);
    cudaFree(c->d_status);
    cudaFree(c->d_scens);
    cudaFree(c->d_items);
    cudaFree(c->d_boxes);
    cudaFree(c->d_ovf);
    cudaFree(c->d_phase);
    cudaFree(c->d_phase_count);
    cudaFree(c->d_mid);
    cudaFree(c->d_mid_count);
    cudaFree(c->d_scratch);
    cudaFree(c->d_poly_kappa);
    cudaFree(c->d_sq);
    cudaFree(c->d_sq_count);
    cudaFree(c->sur.params);
    cudaFree(c->sur.grad);
    cudaFree(c->sur.gpart);
    cudaFree(c->sur.m);
    cudaFree(c->sur.v);
    cudaFree(c->sur.img);
    cudaFree(c->sur.loss);
    cudaFree(c->sur.status);
    for (DevBuf* b : {&c->im_colmax, &c->im_item_scale, &c->im_rowcnt, &c->im_nnz, &c->im_scan_tmp, &c->im_meta,
                      &c->im_bucket_off, &c->im_bucket_cur, &c->im_bucket_len, &c->im_ovf_sorted, &c->im_ovf_count,
                      &c->im_jobs, &c->im_rlim, &c->im_reach, &c->im_thr, &c->im_thr_f, &c->im_box_slot})
        free_buf(*b);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    for (cudaEvent_t e : c->kev)
        if (e) cudaEventDestroy(e);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Learned aperture surrogate.
// ---------------------------------------------------------------------------
namespace {

vpmc_status ensure_surrogate(vpmc_ctx* c)
{
    if (c->sur.params) return VPMC_OK;
    SurNet& n = c->sur;
    CUDA_TRY(dev_alloc(&n.params, sur::kNParams));
    CUDA_TRY(dev_alloc(&n.grad, sur::kNParams));
    n.n_part_cap = c->num_sms;
    CUDA_TRY(dev_alloc(&n.gpart, (size_t)n.n_part_cap * sur::kNParams));
    CUDA_TRY(dev_alloc(&n.m, sur::kNParams));
    CUDA_TRY(dev_alloc(&n.v, sur::kNParams));
    CUDA_TRY(dev_alloc(&n.img, sur::kImgBytes));
    CUDA_TRY(dev_alloc(&n.loss, 2));
    CUDA_TRY(dev_alloc(&n.status, 1));
    CUDA_TRY(cudaMemset(n.img, 0, sur::kImgBytes));   // padding rows and columns stay zero
    return VPMC_OK;
}

vpmc_status reset_optimizer(vpmc_ctx* c)
{
    const size_t b = sur::kNParams * sizeof(float);
    CUDA_TRY(cudaMemsetAsync(c->sur.grad, 0, b, c->stream));
    CUDA_TRY(cudaMemsetAsync(c->sur.m, 0, b, c->stream));
    CUDA_TRY(cudaMemsetAsync(c->sur.v, 0, b, c->stream));
    CUDA_TRY(cudaMemsetAsync(c->sur.status, 0, sizeof(int), c->stream));
    c->sur_step = 0;
    return VPMC_OK;
}

vpmc_status surrogate_status(vpmc_ctx* c)
{
    int ss = 0;
    CUDA_TRY(cudaMemcpy(&ss, c->sur.status, sizeof ss, cudaMemcpyDeviceToHost));
    if (ss) return fail(VPMC_ERR_TIMEOUT, "surrogate: a tensor-core wait timed out");
    return VPMC_OK;
}

}  // namespace

extern "C" {

vpmc_status vpmc_surrogate_set_weights(vpmc_ctx* c, const float* params)
{
    g_error.clear();
    (void)cudaGetLastError();
    if (!c || !params) return fail(VPMC_ERR_ARG, "null argument");
    for (int i = 0; i < sur::kNParams; ++i)
        if (!std::isfinite(params[i])) return fail(VPMC_ERR_ARG, "parameter %d is not finite", i);
    vpmc_status st = ensure_surrogate(c);
    if (st != VPMC_OK) return st;
    CUDA_TRY(cudaMemcpyAsync(c->sur.params, params, sur::kNParams * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    st = reset_optimizer(c);
    if (st != VPMC_OK) return st;
    CUDA_TRY(launch_sur_pack(c->sur, c->stream));
    ++c->launches;
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->sur_ready = true;
    return VPMC_OK;
}

vpmc_status vpmc_surrogate_init(vpmc_ctx* c, uint64_t seed)
{
    g_error.clear();
    if (!c) return fail(VPMC_ERR_ARG, "null context");
    // He-normal weights (std sqrt(2 / fan_in); the output layer 0.1 sqrt(1 /
    // fan_in), so the mixture starts near unit widths), zero biases; normals
    // from splitmix64 uniforms by Box-Muller.
    std::vector<float> w(sur::kNParams, 0.0f);
    uint64_t state = seed;
    auto next_u = [&]() {
        uint64_t z = (state += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return ((double)(z >> 11) + 0.5) * 0x1p-53;
    };
    auto fill = [&](int off, int count, double sd) {
        for (int i = 0; i < count; i += 2) {
            const double r = std::sqrt(-2.0 * std::log(next_u())), a = 6.283185307179586 * next_u();
            w[off + i] = (float)(sd * r * std::cos(a));
            if (i + 1 < count) w[off + i + 1] = (float)(sd * r * std::sin(a));
        }
    };
    fill(sur::oW1, sur::kH * sur::kIn, std::sqrt(2.0 / sur::kIn));
    fill(sur::oW2, sur::kH * sur::kH, std::sqrt(2.0 / sur::kH));
    fill(sur::oW3, sur::kOut * sur::kH, 0.1 * std::sqrt(1.0 / sur::kH));
    return vpmc_surrogate_set_weights(c, w.data());
}

vpmc_status vpmc_surrogate_get_weights(vpmc_ctx* c, float* params)
{
    g_error.clear();
    (void)cudaGetLastError();
    if (!c || !params) return fail(VPMC_ERR_ARG, "null argument");
    if (!c->sur_ready) return fail(VPMC_ERR_STATE, "no surrogate weights");
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    CUDA_TRY(cudaMemcpy(params, c->sur.params, sur::kNParams * sizeof(float), cudaMemcpyDeviceToHost));
    return VPMC_OK;
}

vpmc_status vpmc_surrogate_forward(vpmc_ctx* c, const float* feat_dev, int64_t n, float* z_dev)
{
    g_error.clear();
    (void)cudaGetLastError();
    if (!c || (n > 0 && (!feat_dev || !z_dev)) || n < 0) return fail(VPMC_ERR_ARG, "bad argument");
    if ((reinterpret_cast<uintptr_t>(feat_dev) | reinterpret_cast<uintptr_t>(z_dev)) & 15u)
        return fail(VPMC_ERR_ARG, "feat_dev and z_dev must be 16-byte aligned");
    if (!c->sur_ready) return fail(VPMC_ERR_STATE, "no surrogate weights");
    CUDA_TRY(launch_sur_forward(c->sur, feat_dev, n, z_dev, c->num_sms, c->stream));
    ++c->launches;
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return surrogate_status(c);
}

vpmc_status vpmc_surrogate_gradient(vpmc_ctx* c, const float* feat_dev, const float* target_dev,
                                    const int32_t* label_dev, int64_t n, float* grad_dev, double* loss)
{
    g_error.clear();
    (void)cudaGetLastError();
    if (!c || n <= 0 || !feat_dev || !target_dev || !label_dev || !grad_dev) return fail(VPMC_ERR_ARG, "bad argument");
    if (!c->sur_ready) return fail(VPMC_ERR_STATE, "no surrogate weights");
    CUDA_TRY(cudaMemsetAsync(c->sur.grad, 0, sur::kNParams * sizeof(float), c->stream));
    CUDA_TRY(cudaMemsetAsync(c->sur.loss, 0, 2 * sizeof(double), c->stream));
    int parts = 0;
    CUDA_TRY(launch_sur_train(c->sur, feat_dev, target_dev, label_dev, 0, n, n, (float)(1.0 / (double)n), c->num_sms,
                              &parts, c->stream));
    CUDA_TRY(launch_sur_reduce(c->sur, parts, c->stream));
    c->launches += 2;
    CUDA_TRY(cudaMemcpyAsync(grad_dev, c->sur.grad, sur::kNParams * sizeof(float), cudaMemcpyDeviceToDevice,
                             c->stream));
    CUDA_TRY(cudaMemsetAsync(c->sur.grad, 0, sur::kNParams * sizeof(float), c->stream));
    double h[2] = {0.0, 0.0};
    CUDA_TRY(cudaMemcpyAsync(h, c->sur.loss, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (loss) *loss = h[0] / (double)n;
    return surrogate_status(c);
}

vpmc_status vpmc_surrogate_train(vpmc_ctx* c, const float* feat_dev, const float* target_dev, const int32_t* label_dev,
                                 int64_t n, int batch, int epochs, float lr, float lr_min, float* epoch_loss)
{
    g_error.clear();
    (void)cudaGetLastError();
    if (!c || n <= 0 || !feat_dev || !target_dev || !label_dev) return fail(VPMC_ERR_ARG, "bad argument");
    if (batch <= 0 || epochs <= 0 || !(lr > 0.0f) || !(lr_min >= 0.0f) || lr_min > lr)
        return fail(VPMC_ERR_ARG, "batch and epochs must be positive, 0 <= lr_min <= lr, lr > 0");
    if (!c->sur_ready) return fail(VPMC_ERR_STATE, "no surrogate weights (set them first)");
    const long long nb = (n + batch - 1) / batch;
    const long long steps = nb * (long long)epochs;
    long long t = 0;
    for (int e = 0; e < epochs; ++e) {
        CUDA_TRY(cudaMemsetAsync(c->sur.loss, 0, 2 * sizeof(double), c->stream));
        // batch order of this epoch: an affine permutation j -> (a j + b) mod nb
        long long a = (2654435761ll + 2ll * e) % nb;
        if (a == 0) a = 1;
        while (std::gcd(a, nb) != 1) ++a;
        const long long b = (40503ll * (e + 1)) % nb;
        for (long long j = 0; j < nb; ++j, ++t) {
            const long long bj = (a * j + b) % nb;
            const long long first = bj * batch;
            const long long rows = std::min<long long>(batch, n - first);
            int parts = 0;
            CUDA_TRY(launch_sur_train(c->sur, feat_dev, target_dev, label_dev, first, rows, n,
                                      (float)(1.0 / (double)rows), c->num_sms, &parts, c->stream));
            ++c->sur_step;
            const double cosw = 0.5 * (1.0 + std::cos(3.14159265358979323846 * (double)t / (double)steps));
            const float lr_t = (float)(lr_min + (lr - lr_min) * cosw);
            CUDA_TRY(launch_sur_adam(c->sur, c->sur_step, lr_t, parts, c->stream));
            c->launches += 2;
        }
        double h[2] = {0.0, 0.0};
        CUDA_TRY(cudaMemcpyAsync(h, c->sur.loss, sizeof h, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        if (epoch_loss) epoch_loss[e] = (float)(h[0] / (double)n);
        vpmc_status st = surrogate_status(c);
        if (st != VPMC_OK) return st;
        if (!std::isfinite(h[0]))
            return fail(VPMC_ERR_STATE, "training diverged in epoch %d (non-finite loss); lower lr or fewer steps", e);
    }
    return VPMC_OK;
}

vpmc_status vpmc_surrogate_tracks(vpmc_ctx* c, const int* beam_ids, int n_beams, int64_t tracks_per_beam,
                                  const vpmc_opts* opts_in, int use_surrogate, float* feat_dev, float* target_dev,
                                  int32_t* label_dev)
{
    g_error.clear();
    (void)cudaGetLastError();
    if (!c || !beam_ids || n_beams <= 0 || n_beams > kMaxBeams || tracks_per_beam <= 0 || !feat_dev || !target_dev ||
        !label_dev)
        return fail(VPMC_ERR_ARG, "bad argument");
    if (tracks_per_beam >= (1ll << 32)) return fail(VPMC_ERR_ARG, "tracks_per_beam must be below 2^32");
    vpmc_opts o;
    vpmc_default_opts(&o);
    if (opts_in) o = *opts_in;
    vpmc_status st = check_opts(&o);
    if (st != VPMC_OK) return st;
    if (use_surrogate && !c->sur_ready) return fail(VPMC_ERR_STATE, "no surrogate weights");
    st = pending_status(c);
    if (st != VPMC_OK) return st;
    std::vector<DevItem> items(n_beams);
    for (int g = 0; g < n_beams; ++g) {
        const int b = beam_ids[g];
        if (b < 0 || b >= kMaxBeams || !c->beam_set[b]) return fail(VPMC_ERR_STATE, "beam %d is not set", b);
        if (!c->beams[b].ap || c->beams[b].rs || c->beams[b].ap_sad > 0.0f)
            return fail(VPMC_ERR_ARG, "beam %d: training tracks need a parallel-wall aperture and no range shifter", b);
        DevItem it{};
        it.hist_off = (long long)g * tracks_per_beam;
        it.spot = g;
        it.beam = b;
        items[g] = it;
    }
    const long long total = (long long)n_beams * tracks_per_beam;
    float* d_frame = nullptr;
    CUDA_TRY(dev_alloc(&d_frame, (size_t)total * 8));
    if (cudaMemsetAsync(d_frame, 0, (size_t)total * 8 * sizeof(float), c->stream) != cudaSuccess) {
        cudaFree(d_frame);
        return fail(VPMC_ERR_CUDA, "frame buffer reset failed");
    }
    auto done = [&](vpmc_status s) {
        cudaFree(d_frame);
        return s;
    };
    st = grow(c, &c->d_items, &c->items_cap, items.size());
    if (st != VPMC_OK) return done(st);
    const DevScen sc{{0.0f, 0.0f, 0.0f}, 1.0f};
    const long long batch = std::min<long long>(total, kMaxBatch);
    st = ensure_phase(c, batch, use_surrogate != 0);
    if (st != VPMC_OK) return done(st);
    if (cudaMemcpyAsync(c->d_items, items.data(), items.size() * sizeof(DevItem), cudaMemcpyHostToDevice, c->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(c->d_scens, &sc, sizeof sc, cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
        return done(fail(VPMC_ERR_CUDA, "upload of the track items failed"));
    TransportParams p = base_params(c, o);
    p.items = c->d_items;
    p.n_items = n_beams;
    p.n_scen = 1;
    p.records = nullptr;
    p.rec_cap = 0;
    p.track_mode = 1;
    p.trk_feat = feat_dev;
    p.trk_y = target_dev;
    p.trk_label = label_dev;
    p.trk_frame = d_frame;
    p.surrogate = use_surrogate ? 1 : 0;
    p.sq = c->d_sq;
    p.sq_cap = c->sq_cap;
    p.sq_count = c->d_sq_count;
    p.phase = c->d_phase;
    p.phase_cap = c->phase_cap;
    p.phase_count = c->d_phase_count;
    p.mid = c->d_mid;
    p.mid_cap = c->phase_cap;
    p.mid_count = c->d_mid_count;
    p.aggregate = 0;
    p.chunk = 32;
    st = reset_counters(c);
    if (st != VPMC_OK) return done(st);
    if (use_surrogate && cudaMemsetAsync(c->sur.status, 0, sizeof(int), c->stream) != cudaSuccess)
        return done(fail(VPMC_ERR_CUDA, "status reset failed"));
    const int block = c->tune_dose.valid ? c->tune_dose.dev_block : 512;
    for (long long h0 = 0; h0 < total; h0 += batch) {
        p.hist_begin = h0;
        p.total = std::min(total, h0 + batch);
        cudaError_t e = cudaMemsetAsync(c->d_counter, 0, sizeof(unsigned long long), c->stream);
        if (e == cudaSuccess && use_surrogate) e = cudaMemsetAsync(c->d_sq_count, 0, sizeof(unsigned long long), c->stream);
        if (e == cudaSuccess) e = launch_devices(p, c->num_sms, block, c->stream);
        if (e == cudaSuccess && use_surrogate) e = launch_sur_infer(c->sur, p, c->num_sms, c->stream);
        if (e != cudaSuccess) return done(fail(VPMC_ERR_CUDA, "track launch: %s", cudaGetErrorString(e)));
        c->launches += use_surrogate ? 2 : 1;
    }
    if (cudaStreamSynchronize(c->stream) != cudaSuccess)
        return done(fail(VPMC_ERR_CUDA, "track transport: %s", cudaGetErrorString(cudaGetLastError())));
    int status = 0;
    if (cudaMemcpy(&status, c->d_status, sizeof status, cudaMemcpyDeviceToHost) != cudaSuccess)
        return done(fail(VPMC_ERR_CUDA, "status read failed"));
    if (status & 1) return done(fail(VPMC_ERR_TIMEOUT, "tracks reached the iteration cap"));
    if (status & 6) return done(fail(VPMC_ERR_DEVICE_FLAG, "query buffer overflow (status %d)", status));
    if (use_surrogate) {
        st = surrogate_status(c);
        if (st != VPMC_OK) return done(st);
    }
    return done(VPMC_OK);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Robust spot-weight optimisation.
// ---------------------------------------------------------------------------
namespace {

struct OptInputs {
    std::vector<const long long*> rp;
    std::vector<const int*> col;
    std::vector<const float*> val;
    long long n_rows = 0;
    int n_cols = 0;
    long long n_target = 0, n_ring = 0;
    std::vector<unsigned char> cls;         // host copy of the voxel classes
};

vpmc_status check_opt_inputs(const vpmc_csr* mats, int n_scen, const uint8_t* cls, OptInputs* in)
{
    if (!mats || n_scen <= 0 || n_scen > kMaxScen || !cls) return fail(VPMC_ERR_ARG, "bad matrices or classes");
    in->n_rows = mats[0].n_rows;
    in->n_cols = (int)mats[0].n_cols;
    for (int s = 0; s < n_scen; ++s) {
        if (mats[s].n_rows != in->n_rows || mats[s].n_cols != mats[0].n_cols)
            return fail(VPMC_ERR_ARG, "scenario %d: matrix shape differs", s);
        if (!mats[s].row_ptr || (mats[s].nnz > 0 && (!mats[s].col || !mats[s].val)))
            return fail(VPMC_ERR_ARG, "scenario %d: null CSR buffer", s);
        in->rp.push_back(reinterpret_cast<const long long*>(mats[s].row_ptr));
        in->col.push_back(mats[s].col);
        in->val.push_back(mats[s].val);
    }
    if (in->n_rows <= 0 || mats[0].n_cols <= 0) return fail(VPMC_ERR_ARG, "empty matrices");
    if (mats[0].n_cols > 28000) return fail(VPMC_ERR_ARG, "%lld columns: at most 28,000", (long long)mats[0].n_cols);
    if (in->n_rows > INT32_MAX) return fail(VPMC_ERR_ARG, "more than 2^31 - 1 rows");
    std::vector<unsigned char>& h = in->cls;
    h.resize((size_t)in->n_rows);
    if (cudaMemcpy(h.data(), cls, h.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(VPMC_ERR_CUDA, "reading the voxel classes: %s", cudaGetErrorString(cudaGetLastError()));
    for (unsigned char c : h) {
        in->n_target += c == 1;
        in->n_ring += c == 2;
    }
    return VPMC_OK;
}

int current_sms()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

}  // namespace

extern "C" {

vpmc_status vpmc_robust_optimize(const vpmc_csr* mats, int n_scen, const uint8_t* voxel_class_dev,
                                 const vpmc_opt_params* prm, float* x_dev, float* history, float* ms, void* stream)
{
    g_error.clear();
    (void)cudaGetLastError();
    if (!prm || !x_dev) return fail(VPMC_ERR_ARG, "null params or weights");
    if (prm->iterations < 0 || !(prm->prescription > 0.0f) || !(prm->lr > 0.0f) || !(prm->over_frac >= 1.0f) ||
        !(prm->ring_frac > 0.0f) || prm->w_under < 0.0f || prm->w_over < 0.0f || prm->w_ring < 0.0f)
        return fail(VPMC_ERR_ARG, "invalid optimisation parameters");
    OptInputs in;
    vpmc_status st = check_opt_inputs(mats, n_scen, voxel_class_dev, &in);
    if (st != VPMC_OK) return st;
    if (in.n_target == 0) return fail(VPMC_ERR_ARG, "no target voxels (class 1)");
    std::vector<float> x0((size_t)in.n_cols);
    CUDA_TRY(cudaMemcpy(x0.data(), x_dev, x0.size() * sizeof(float), cudaMemcpyDeviceToHost));
    double mean = 0.0;
    for (float v : x0) {
        if (!(v >= 0.0f) || !std::isfinite(v)) return fail(VPMC_ERR_ARG, "initial weights must be finite and >= 0");
        mean += v;
    }
    mean /= (double)x0.size();
    OptSpec spec;
    spec.dp = prm->prescription;
    spec.w_u = prm->w_under;
    spec.w_o = prm->w_over;
    spec.w_r = prm->w_ring;
    spec.over = prm->over_frac;
    spec.ring = prm->ring_frac;
    spec.n_target = in.n_target;
    spec.n_ring = in.n_ring;
    spec.step = (float)(prm->lr * (mean > 0.0 ? mean : 1.0));
    spec.eps = 1e-8f;
    spec.iterations = prm->iterations;
    float t[2] = {0.0f, 0.0f};
    CUDA_TRY(run_robust_optimize(in.rp.data(), in.col.data(), in.val.data(), n_scen, in.n_rows, in.n_cols,
                                 in.cls.data(), spec, x_dev, history, (cudaStream_t)stream, t, nullptr));
    if (ms) {
        ms[0] = t[0];
        ms[1] = t[1];
    }
    return VPMC_OK;
}

vpmc_status vpmc_weights_dose(const vpmc_csr* mat, const float* x_dev, float* dose_dev, void* stream)
{
    g_error.clear();
    (void)cudaGetLastError();
    if (!mat || !x_dev || !dose_dev || !mat->row_ptr || mat->n_rows <= 0 || mat->n_cols <= 0 ||
        mat->n_cols > INT32_MAX || (mat->nnz > 0 && (!mat->col || !mat->val)))
        return fail(VPMC_ERR_ARG, "bad argument");
    CUDA_TRY(run_weights_dose(reinterpret_cast<const long long*>(mat->row_ptr), mat->col, mat->val, mat->n_rows,
                              (int)mat->n_cols, x_dev, dose_dev, (cudaStream_t)stream, current_sms()));
    return VPMC_OK;
}

vpmc_status vpmc_target_indices(const vpmc_csr* mats, int n_scen, const uint8_t* voxel_class_dev,
                                float prescription, const float* x_dev, double* out, void* stream)
{
    g_error.clear();
    (void)cudaGetLastError();
    if (!x_dev || !out || !(prescription > 0.0f)) return fail(VPMC_ERR_ARG, "bad argument");
    OptInputs in;
    vpmc_status st = check_opt_inputs(mats, n_scen, voxel_class_dev, &in);
    if (st != VPMC_OK) return st;
    CUDA_TRY(run_target_indices(in.rp.data(), in.col.data(), in.val.data(), n_scen, in.n_rows, in.n_cols,
                                voxel_class_dev, prescription, x_dev, out, (cudaStream_t)stream, current_sms()));
    return VPMC_OK;
}

}  // extern "C"
