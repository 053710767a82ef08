// Dose entry point that allocates no memory of its own.
//
// vpmc_run_spots takes its scratch (64-bit accumulator, work items, hand-off
// buffer, counters) from the context, which grows it with cudaMalloc when a
// call needs more.  Some callers cannot let a call allocate: serving loops
// where the implicit device synchronisation of cudaMalloc/cudaFree would
// stall other streams, and hosts whose memory pool owns all device memory.
// vpmc_run_spots_noalloc gives them the same dose with its scratch in one
// file-scope device array of fixed size, resolved once per device.  The
// context must already exist (vpmc_create_geometry and vpmc_set_aperture
// allocate, once, at set-up).
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/vpmc.h"
#include "context.h"
#include "vpmc_internal.cuh"

using namespace vpmc;

namespace {

constexpr long long kMaxVoxels = 1ll << 21;      // 2,097,152 scoring voxels
constexpr int kMaxItems = 16384;                 // spots with histories per call
constexpr long long kBatch = 1ll << 17;          // histories per batch (two hand-off buffers of this size)
constexpr int kMaxDevices = 64;

constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t kOffAcc = 0;
constexpr size_t kOffItems = kOffAcc + align256(sizeof(unsigned long long) * kMaxVoxels);
constexpr size_t kOffBox = kOffItems + align256(sizeof(DevItem) * kMaxItems);
constexpr size_t kOffScen = kOffBox + align256(sizeof(DevBox));
constexpr size_t kOffPhase = kOffScen + align256(sizeof(DevScen));
constexpr size_t kOffMid = kOffPhase + align256(sizeof(PhaseRec) * kBatch);
constexpr size_t kOffCount = kOffMid + align256(sizeof(PhaseRec) * kBatch);      // counter, two hand-off counts, stats
constexpr size_t kOffStatus = kOffCount + align256(sizeof(unsigned long long) * (3 + kNStats));
constexpr size_t kScratchBytes = kOffStatus + 256;                              // about 29 MiB

// The scratch of every call on a device (each GPU that loads the library
// holds it until the process exits).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {};
// per device: an asynchronous call (no stats_out) left the array's status
// word unread, with the stream it ran on; the next call on the device reads it
struct Pending {
    bool set = false;
    cudaStream_t stream = nullptr;
};
Pending g_pending[kMaxDevices];

// Device address of the scratch array on the current device; resolved by the
// first call on that device.
vpmc_status scratch_address(int device, unsigned char** out)
{
    if (device < 0 || device >= kMaxDevices) return report_error(VPMC_ERR_CUDA, "device ordinal %d out of range", device);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[device]) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess)
            return report_error(VPMC_ERR_CUDA, "cudaGetSymbolAddress of the scratch array: %s", cudaGetErrorString(e));
        g_addr[device] = static_cast<unsigned char*>(ptr);
    }
    *out = g_addr[device];
    return VPMC_OK;
}

#define NA_TRY(expr)                                                                               \
    do {                                                                                           \
        const cudaError_t e_ = (expr);                                                             \
        if (e_ != cudaSuccess) return report_error(VPMC_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)

}  // namespace

namespace {

// Reads the status word that an earlier asynchronous call on this device
// left unread and reports its error.  It first waits for that call's work:
// the stream, when the earlier call ran on this call's stream, else the
// whole device (that stream may belong to another context, or be gone).
vpmc_status pending_status(int device, cudaStream_t stream)
{
    cudaStream_t s = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_pending[device].set) return VPMC_OK;
        g_pending[device].set = false;
        s = g_pending[device].stream;
    }
    int st_word = 0;
    if (s == stream) NA_TRY(cudaStreamSynchronize(stream));
    else NA_TRY(cudaDeviceSynchronize());
    NA_TRY(cudaMemcpyAsync(&st_word, g_addr[device] + kOffStatus, sizeof st_word, cudaMemcpyDeviceToHost, stream));
    NA_TRY(cudaStreamSynchronize(stream));
    if (st_word & 1)
        return report_error(VPMC_ERR_TIMEOUT, "an earlier asynchronous call: histories reached the iteration cap");
    if (st_word & 6)
        return report_error(VPMC_ERR_DEVICE_FLAG, "an earlier asynchronous call: hand-off buffer overflow (status %d)",
                            st_word);
    return VPMC_OK;
}

}  // namespace

extern "C" vpmc_status vpmc_run_spots_noalloc(vpmc_ctx* c, const vpmc_spot* spots, int n_spots,
                                              const vpmc_scenario* scen, const vpmc_opts* opts_in, float* dose_dev,
                                              vpmc_stats* stats_out)
{
    clear_error();
    (void)cudaGetLastError();
    if (!c || !dose_dev) return report_error(VPMC_ERR_ARG, "null context or dose buffer");
    if (c->nvox > kMaxVoxels)
        return report_error(VPMC_ERR_ARG, "scoring grid has %lld voxels; this entry point holds at most %lld",
                            c->nvox, kMaxVoxels);
    if (n_spots < 0 || (n_spots > 0 && !spots)) return report_error(VPMC_ERR_ARG, "spots: null pointer or negative count");
    vpmc_opts o;
    vpmc_default_opts(&o);
    if (opts_in) o = *opts_in;
    if (o.frac_bits < 0 || o.frac_bits > 40) return report_error(VPMC_ERR_ARG, "frac_bits %d outside [0, 40]", o.frac_bits);
    if (o.block_size != 0 && (o.block_size < 32 || o.block_size > patient_max_block() || o.block_size % 32))
        return report_error(VPMC_ERR_ARG, "block_size %d: must be 0 or a multiple of 32 up to %d", o.block_size,
                            patient_max_block());
    if (o.chunk < 0 || o.chunk > 4096) return report_error(VPMC_ERR_ARG, "chunk %d outside [0, 4096]", o.chunk);
    if (o.history_cap < 0 || (o.history_cap > 0 && !o.history_out))
        return report_error(VPMC_ERR_ARG, "history_cap > 0 needs history_out");
    if (o.surrogate) return report_error(VPMC_ERR_ARG, "this entry point runs the plain aperture transport only");
    if (o.timeout_iters < 0 || o.timeout_iters > 0x7fffffffll)
        return report_error(VPMC_ERR_ARG, "timeout_iters outside [0, 2^31 - 1]");
    DevScen sc{{0.0f, 0.0f, 0.0f}, 1.0f};
    if (scen) {
        if (!(scen->spr_scale > 0)) return report_error(VPMC_ERR_ARG, "scenario spr_scale must be positive");
        for (int k = 0; k < 3; ++k) sc.shift[k] = (float)scen->shift_mm[k];
        sc.spr_scale = (float)scen->spr_scale;
    }
    int device = 0;
    NA_TRY(cudaGetDevice(&device));
    if (device != c->device) return report_error(VPMC_ERR_STATE, "the context belongs to device %d, current is %d",
                                                 c->device, device);
    // the work list below is copied from host stack memory during the call
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    NA_TRY(cudaStreamIsCapturing(c->stream, &cap));
    if (cap != cudaStreamCaptureStatusNone)
        return report_error(VPMC_ERR_STATE, "the context's stream is capturing; this call copies host stack memory");
    unsigned char* base = nullptr;
    const vpmc_status sa = scratch_address(device, &base);
    if (sa != VPMC_OK) return sa;
    const vpmc_status ps = pending_status(device, c->stream);
    if (ps != VPMC_OK) return ps;
    unsigned long long* acc = reinterpret_cast<unsigned long long*>(base + kOffAcc);
    DevItem* items = reinterpret_cast<DevItem*>(base + kOffItems);
    DevBox* box = reinterpret_cast<DevBox*>(base + kOffBox);
    DevScen* dscen = reinterpret_cast<DevScen*>(base + kOffScen);
    PhaseRec* phase = reinterpret_cast<PhaseRec*>(base + kOffPhase);
    PhaseRec* mid = reinterpret_cast<PhaseRec*>(base + kOffMid);
    unsigned long long* counters = reinterpret_cast<unsigned long long*>(base + kOffCount);
    int* status = reinterpret_cast<int*>(base + kOffStatus);

    // work items, uploaded from a small stack buffer (pageable copies are
    // staged before cudaMemcpyAsync returns, so the buffer can be reused)
    const double fs = std::ldexp(1.0, o.frac_bits);
    DevItem chunk[128];
    int n_items = 0, in_chunk = 0;
    long long total = 0;
    double qmax = 0.0, e_in = 0.0;
    for (int i = 0; i < n_spots; ++i) {
        const vpmc_spot& s = spots[i];
        if (s.beam < 0 || s.beam >= kMaxBeams || !c->beam_set[s.beam])
            return report_error(VPMC_ERR_STATE, "spot %d: beam %d was not set with vpmc_set_aperture", i, s.beam);
        if (!(s.energy_mev > 0.5 && s.energy_mev <= 250.0))
            return report_error(VPMC_ERR_ARG, "spot %d: energy %g MeV outside (0.5, 250]", i, s.energy_mev);
        if (s.n_hist < 0 || s.n_hist >= (1ll << 32))
            return report_error(VPMC_ERR_ARG, "spot %d: n_hist outside [0, 2^32)", i);
        if (!(s.sigma_mm >= 0.0) || !(s.div_mrad >= 0.0) || !std::isfinite(s.x_mm) || !std::isfinite(s.y_mm) ||
            !(s.weight >= 0.0))
            return report_error(VPMC_ERR_ARG, "spot %d: invalid position, sigma, divergence or weight", i);
        if (s.n_hist == 0) continue;
        if (n_items == kMaxItems)
            return report_error(VPMC_ERR_ARG, "more than %d spots with histories; this entry point holds %d", kMaxItems,
                                kMaxItems);
        DevItem& it = chunk[in_chunk++];
        it = DevItem{};
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
        total += s.n_hist;
        qmax += (double)s.n_hist * s.energy_mev * (s.weight > 1.0 ? s.weight : 1.0) * fs;
        e_in += (double)s.n_hist * s.energy_mev;
        if (in_chunk == 128) {
            NA_TRY(cudaMemcpyAsync(items + n_items, chunk, sizeof chunk, cudaMemcpyHostToDevice, c->stream));
            n_items += in_chunk;
            in_chunk = 0;
        }
    }
    if (in_chunk) {
        NA_TRY(cudaMemcpyAsync(items + n_items, chunk, in_chunk * sizeof(DevItem), cudaMemcpyHostToDevice, c->stream));
        n_items += in_chunk;
    }
    if (qmax >= 9.0e18) return report_error(VPMC_ERR_ARG, "fixed-point range exceeded: lower frac_bits or weights");
    DevBox full{};
    for (int k = 0; k < 3; ++k) full.n[k] = c->sg.n[k];
    NA_TRY(cudaMemcpyAsync(box, &full, sizeof full, cudaMemcpyHostToDevice, c->stream));
    NA_TRY(cudaMemcpyAsync(dscen, &sc, sizeof sc, cudaMemcpyHostToDevice, c->stream));
    // the array keeps the previous call's contents: clear what must start at zero
    NA_TRY(cudaMemsetAsync(acc, 0, (size_t)c->nvox * sizeof(unsigned long long), c->stream));
    NA_TRY(cudaMemsetAsync(counters, 0, sizeof(unsigned long long) * (3 + kNStats), c->stream));
    NA_TRY(cudaMemsetAsync(status, 0, sizeof(int), c->stream));
    NA_TRY(cudaMemsetAsync(dose_dev, 0, (size_t)c->nvox * sizeof(float), c->stream));

    TransportParams p{};
    p.tables = c->d_tables;
    p.water = c->water_mat;
    p.ct_lut = reinterpret_cast<const uint16_t*>(c->d_ct);
    p.ctg = c->ctg;
    p.sg = c->sg;
    for (int k = 0; k < 3; ++k) p.nest_shift[k] = c->nest_shift[k];
    p.beams = c->d_beams;
    p.n_beams = kMaxBeams;
    p.scens = dscen;
    p.n_scen = 1;
    p.poly = c->d_poly;
    p.n_poly = c->n_poly;
    p.raster = c->d_raster;
    p.raster_lb = c->d_raster_lb;
    p.range_rejection = o.range_rejection;
    p.items = items;
    p.n_items = n_items;
    p.boxes = box;
    p.counter = counters;
    p.phase_count = counters + 1;
    p.mid_count = counters + 2;
    p.stats = counters + 3;
    p.status = status;
    p.scratch = acc;
    p.phase = phase;
    p.phase_cap = kBatch;
    p.n_rep = 1;
    p.rep_cap = kBatch;
    p.mid = mid;
    p.mid_cap = kBatch;
    p.ovf = nullptr;
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
    const TuneResult& t = c->tune_dose;
    const int dev_block = t.valid ? t.dev_block : 512;
    const int block = o.block_size ? o.block_size : (t.valid ? t.block : 640);
    p.aggregate = o.aggregate >= 0 ? o.aggregate : (t.valid ? t.aggregate : 0);
    p.chunk = o.chunk ? o.chunk : (t.valid ? t.chunk : 32);
    if (n_items) NA_TRY(cudaEventRecord(c->ev0, c->stream));
    for (long long h0 = 0; h0 < total; h0 += kBatch) {
        p.hist_begin = h0;
        p.total = h0 + kBatch < total ? h0 + kBatch : total;
        NA_TRY(cudaMemsetAsync(p.counter, 0, sizeof(unsigned long long), c->stream));
        NA_TRY(cudaMemsetAsync(p.phase_count, 0, sizeof(unsigned long long), c->stream));
        NA_TRY(launch_devices(p, c->num_sms, dev_block, c->stream));
        NA_TRY(cudaMemsetAsync(p.counter, 0, sizeof(unsigned long long), c->stream));
        NA_TRY(launch_patient(p, c->num_sms, block, c->stream));
        c->launches += 3;
    }
    if (n_items) NA_TRY(cudaEventRecord(c->ev1, c->stream));
    const double scale = std::ldexp(1.0, -o.frac_bits) * 1.602176634e-10 /
                         (c->sg_spacing[0] * c->sg_spacing[1] * c->sg_spacing[2] * 1e-3);
    NA_TRY(launch_dose_normalise(acc, c->d_rho, c->nvox, scale, dose_dev, c->stream));
    ++c->launches;
    if (!stats_out && n_items) {
        std::lock_guard<std::mutex> lock(g_mu);
        g_pending[device].set = true;
        g_pending[device].stream = c->stream;
    }
    if (stats_out) {
        NA_TRY(cudaStreamSynchronize(c->stream));
        unsigned long long h[3 + kNStats];
        int st_word = 0;
        NA_TRY(cudaMemcpy(h, counters, sizeof h, cudaMemcpyDeviceToHost));
        NA_TRY(cudaMemcpy(&st_word, status, sizeof st_word, cudaMemcpyDeviceToHost));
        const unsigned long long* v = h + 3;
        const double q = std::ldexp(1.0, -o.frac_bits);
        vpmc_stats r;
        std::memset(&r, 0, sizeof r);
        r.histories = total;
        r.steps = (int64_t)v[kStSteps];
        r.errors = (int64_t)v[kStErr];
        r.steps_rs = (int64_t)v[kStStepsRS];
        r.steps_aperture = (int64_t)v[kStStepsAp];
        r.e_in = e_in;
        r.e_dep = v[kStDep] * q;
        r.e_leak = v[kStLeak] * q;
        r.e_rs = v[kStRS] * q;
        r.e_aperture = v[kStAp] * q;
        r.e_nuc = v[kStNuc] * q;
        if (n_items) NA_TRY(cudaEventElapsedTime(&r.ms, c->ev0, c->ev1));
        r.launches = 3 * ((total + kBatch - 1) / kBatch) + 1;
        *stats_out = r;
        if (st_word & 1) return report_error(VPMC_ERR_TIMEOUT, "%lld histories reached the iteration cap",
                                             (long long)r.errors);
        if (st_word & 6) return report_error(VPMC_ERR_DEVICE_FLAG, "hand-off buffer overflow (status %d)", st_word);
    }
    return VPMC_OK;
}
