// Finalisation kernels: scoring-voxel density, fixed-point -> dose, and the
// influence-matrix columns -> CSR (paper Sec. 2.C: sparse matrix storage).
//
// FP64 appears only here (dose normalisation and thresholds); transport is FP32.
#include "vpmc_internal.cuh"

namespace vpmc {
namespace {

__device__ double curve_density(const double* c, double hu)
{
    const double h = fmin(fmax(hu, c[0]), 3071.0);
    int s = 0;
    while (s < 3 && h >= c[s + 1]) ++s;
    const double t = (h - c[s]) / (c[s + 1] - c[s]);
    return c[5 + s] + t * (c[5 + s + 1] - c[5 + s]);
}

// Volume-weighted mean density of the CT voxels overlapping each scoring voxel.
__global__ void k_scoring_density(const int16_t* __restrict__ ct, Grid3 ctg, Grid3 sg, const double* __restrict__ c15,
                                  double ctd0, double ctd1, double ctd2, double sgd0, double sgd1, double sgd2,
                                  double* __restrict__ rho_out)
{
    const long long nv = (long long)sg.n[0] * sg.n[1] * sg.n[2];
    const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const double dct[3] = {ctd0, ctd1, ctd2}, dsg[3] = {sgd0, sgd1, sgd2};
    const int S[3] = {(int)(v % sg.n[0]), (int)((v / sg.n[0]) % sg.n[1]), (int)(v / ((long long)sg.n[0] * sg.n[1]))};
    int c0[3], c1[3];
    for (int k = 0; k < 3; ++k) {
        c0[k] = max((int)floor(S[k] * dsg[k] / dct[k]), 0);
        c1[k] = min((int)ceil((S[k] + 1) * dsg[k] / dct[k]), ctg.n[k]);
    }
    double acc = 0.0, vol = 0.0;
    for (int z = c0[2]; z < c1[2]; ++z)
        for (int y = c0[1]; y < c1[1]; ++y)
            for (int x = c0[0]; x < c1[0]; ++x) {
                const int C[3] = {x, y, z};
                double ov = 1.0;
                for (int k = 0; k < 3; ++k) {
                    const double a = S[k] * dsg[k], b = (S[k] + 1) * dsg[k];
                    const double lo = fmax(a, C[k] * dct[k]), hi = fmin(b, (C[k] + 1) * dct[k]);
                    ov *= fmax(hi - lo, 0.0);
                }
                if (ov <= 0.0) continue;
                const double rho = curve_density(c15, (double)ct[x + (long long)ctg.n[0] * (y + (long long)ctg.n[1] * z)]);
                acc += ov * rho;
                vol += ov;
            }
    rho_out[v] = acc / vol;
}

__global__ void k_dose_normalise(const unsigned long long* __restrict__ acc, const double* __restrict__ rho,
                                 long long nvox, double scale, float* __restrict__ dose)
{
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox;
         v += (long long)gridDim.x * blockDim.x)
        dose[v] = (float)((double)acc[v] * scale / rho[v]);
}

// FP32 screen of the FP64 quotient q / rho: q's two 32-bit halves converted
// (64-bit conversions would take the FP64 pipe), times the FP32 reciprocal
// density.  Its relative error against the FP64 value is below 2^-21, so a
// comparison decided by more than kScreen (2^-19) in FP32 has the same
// outcome in FP64; only the rest is redone in FP64.
constexpr float kScreen = 1.0f / 524288.0f;

__device__ __forceinline__ float quotient_f32(unsigned long long q, float inv_rho_f)
{
    const float qf = fmaf(__uint2float_rn((unsigned)(q >> 32)), 4294967296.0f, __uint2float_rn((unsigned)q));
    return qf * inv_rho_f;
}

// One block per item: maximum over the item's box of q / rho, as q x (1 / rho)
// with the same FP64 reciprocal the row pass uses.  The box is contiguous in
// the scratch, so the block streams it as one array, eight coalesced loads in
// flight per thread; only a non-zero entry (a few per cent) needs its voxel's
// coordinates and 1 / rho.  Each thread tracks its maximum in FP32 and
// evaluates in FP64 only the entries within the screen of it: the column's
// FP64 maximum is among them (it is at least the running FP32 maximum x
// (1 - 2^-19)), so the result is the FP64 maximum over all entries.
__global__ void k_column_max(const unsigned long long* __restrict__ scratch, const DevItem* __restrict__ items,
                             const DevBox* __restrict__ boxes, const double* __restrict__ inv_rho,
                             const float* __restrict__ inv_rho_f, Grid3 sg, int first_item,
                             double* __restrict__ colmax)
{
    constexpr int kU = 8;
    const int it = first_item + blockIdx.x;
    const DevBox b = boxes[items[it].box];
    const long long size = (long long)b.n[0] * b.n[1] * b.n[2];
    const unsigned long long* src = scratch + b.base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    double m = 0.0;
    float mf = 0.0f;
    for (long long i0 = threadIdx.x; i0 < size; i0 += (long long)kU * blockDim.x) {
        unsigned long long q[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const long long i = i0 + (long long)u * blockDim.x;
            q[u] = i < size ? __ldcs(src + i) : 0ull;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            if (q[u] == 0ull) continue;
            const long long i = i0 + (long long)u * blockDim.x;
            const int row = (int)(i / b.n[0]);
            const int lx = (int)(i - (long long)row * b.n[0]);
            const int ly = row % b.n[1], lz = row / b.n[1];
            const long long v = (b.lo[0] + lx) + (long long)sg.n[0] * ((b.lo[1] + ly) + (long long)sg.n[1] * (b.lo[2] + lz));
            const float rf = quotient_f32(q[u], inv_rho_f[v]);
            if (rf >= mf * (1.0f - kScreen)) {
                m = fmax(m, (double)q[u] * inv_rho[v]);
                mf = fmaxf(mf, rf);
            }
        }
    }
    __shared__ double red[32];
    for (int o = 16; o >= 1; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) red[warp] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < nwarp ? red[threadIdx.x] : 0.0;
        for (int o = 16; o >= 1; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) colmax[blockIdx.x] = m;
    }
}

// Per item: the FP64 threshold rel x column maximum and its FP32 value.
__global__ void k_column_threshold(const double* __restrict__ colmax, int n, double rel, double* __restrict__ thr,
                                   float* __restrict__ thr_f)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double t = rel * colmax[i];
    thr[i] = t;
    thr_f[i] = (float)t;
}

__global__ void k_reciprocal(const double* __restrict__ x, long long n, double* __restrict__ out,
                             float* __restrict__ out_f)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double r = 1.0 / x[i];
        out[i] = r;
        out_f[i] = (float)r;
    }
}

// Keep q / rho unless it is below the column's threshold: decided by the FP32
// screen and, within its margin, in FP64 (the FP64 rule's outcome).
__device__ __forceinline__ bool keep_entry(unsigned long long q, double inv_rho, float inv_rho_f, double thr,
                                           float thr_f)
{
    const float rf = quotient_f32(q, inv_rho_f);
    if (rf < thr_f * (1.0f - kScreen)) return false;
    if (rf > thr_f * (1.0f + kScreen)) return true;
    return !((double)q * inv_rho < thr);
}

// Count pass, box-major: one thread per (run, voxel of the run's box), a run
// being consecutive items of one field whose boxes have one shape and origin.
// The blocks of a run take consecutive voxels of its box, so each of its
// columns is read with coalesced loads and no thread waits outside a box.
// The kept entries of a (voxel, run) go to the voxel's row count with one
// atomic add (a count does not depend on the order); the voxel's out-of-box
// records are counted by k_csr_count_records.
__global__ void k_csr_count_box(const CsrBuildParams p)
{
    __shared__ int s_run;
    if (threadIdx.x == 0) {
        int lo = 0, hi = p.n_runs;                  // run_block0[lo] <= blockIdx.x < run_block0[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (p.run_block0[mid] <= (int)blockIdx.x) lo = mid; else hi = mid;
        }
        s_run = lo;
    }
    __syncthreads();
    const int r = s_run;
    const int cnt = p.run_count[r];
    if (cnt == 0) return;
    const DevBox bb = p.boxes[p.run_box[r]];
    const long long size = (long long)bb.n[0] * bb.n[1] * bb.n[2];
    const long long l = (long long)(blockIdx.x - p.run_block0[r]) * blockDim.x + threadIdx.x;
    if (l >= size) return;
    const int first = p.run_first[r];
    const int row = (int)(l / bb.n[0]);
    const int lx = (int)(l - (long long)row * bb.n[0]), ly = row % bb.n[1], lz = row / bb.n[1];
    const long long v = (bb.lo[0] + lx) + (long long)p.sg.n[0] * ((bb.lo[1] + ly) + (long long)p.sg.n[1] * (bb.lo[2] + lz));
    const double inv_rho = p.inv_rho[v];
    const float inv_rho_f = (float)inv_rho;
    const unsigned long long* col0 = p.scratch + p.boxes[p.items[first].box].base + l;
    long long count = 0;
    for (int t0 = 0; t0 < cnt; t0 += 8) {
        unsigned long long q[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) q[u] = t0 + u < cnt ? __ldcs(col0 + (long long)(t0 + u) * size) : 0ull;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (q[u] == 0ull) continue;
            const int it = first + t0 + u;
            count += keep_entry(q[u], inv_rho, inv_rho_f, p.thr[it], p.thr_f[it]) ? 1 : 0;
        }
    }
    if (count) atomicAdd(reinterpret_cast<unsigned long long*>(p.row_count + v), (unsigned long long)count);
    p.box_slot[blockIdx.x * (long long)blockDim.x + threadIdx.x] = (unsigned)count;
}

// Count pass of the out-of-box records: one thread per voxel.
__global__ void k_csr_count_records(const CsrBuildParams p)
{
    const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= p.nvox) return;
    const int nrec = p.bucket_len[v];
    if (nrec == 0) return;
    const OvfRec* rec = p.ovf + p.bucket_off[v];
    const double inv_rho = p.inv_rho[v];
    const float inv_rho_f = (float)inv_rho;
    long long count = 0;
    for (int j = 0; j < nrec; ++j) {
        const int it = rec[j].item - p.item_base;
        count += keep_entry(rec[j].q, inv_rho, inv_rho_f, p.thr[it], p.thr_f[it]) ? 1 : 0;
    }
    if (count) atomicAdd(reinterpret_cast<unsigned long long*>(p.row_count + v), (unsigned long long)count);
}

// A run's shape, origin and column range, staged in shared memory: every
// thread of a block tests the same runs in the same order.
struct RunRow {
    int lo[3], n[3];
    int first, cnt;
    int block0;                      // the run's first block in the box-major passes
};
constexpr int kRunsPerStage = 512;

// Fill pass, box-major, first part: one thread per voxel walks the runs in
// column order.  For each run whose box holds the voxel it turns the
// (voxel, run) count of the count pass into that segment's first position in
// the row; the voxel's out-of-box records (sorted by item; their items' boxes
// do not hold the voxel) are written in between, in column order.
__global__ void k_csr_offsets(const CsrBuildParams p)
{
    __shared__ RunRow runs[kRunsPerStage];
    const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const bool row = v < p.nvox;
    const long long vv = row ? v : 0;
    const int x = (int)(vv % p.sg.n[0]);
    const int y = (int)((vv / p.sg.n[0]) % p.sg.n[1]);
    const int z = (int)(vv / ((long long)p.sg.n[0] * p.sg.n[1]));
    long long pos = row ? p.row_ptr[vv] : 0;
    const OvfRec* rec = (p.ovf && row) ? p.ovf + p.bucket_off[vv] : nullptr;
    const int nrec = (p.ovf && row) ? p.bucket_len[vv] : 0;
    const double inv_rho = (row && nrec) ? p.inv_rho[vv] : 0.0;
    const float inv_rho_f = (float)inv_rho;
    int j = 0;
    auto emit_records_before = [&](int item_end) {
        for (; j < nrec && rec[j].item - p.item_base < item_end; ++j) {
            const int it = rec[j].item - p.item_base;
            if (!keep_entry(rec[j].q, inv_rho, inv_rho_f, p.thr[it], p.thr_f[it])) continue;
            p.col[pos] = p.items[it].spot;
            p.val[pos] = (float)((double)rec[j].q * inv_rho * p.item_scale[it]);
            ++pos;
        }
    };
    for (int r0 = 0; r0 < p.n_runs; r0 += kRunsPerStage) {
        const int nst = min(kRunsPerStage, p.n_runs - r0);
        __syncthreads();
        for (int i = threadIdx.x; i < nst; i += blockDim.x) {
            const DevBox bb = p.boxes[p.run_box[r0 + i]];
            RunRow rr;
            for (int k = 0; k < 3; ++k) { rr.lo[k] = bb.lo[k]; rr.n[k] = bb.n[k]; }
            rr.first = p.run_first[r0 + i];
            rr.cnt = p.run_count[r0 + i];
            rr.block0 = p.run_block0[r0 + i];
            runs[i] = rr;
        }
        __syncthreads();
        if (!row) continue;
        for (int b = 0; b < nst; ++b) {
            const RunRow& rr = runs[b];
            const int lx = x - rr.lo[0], ly = y - rr.lo[1], lz = z - rr.lo[2];
            if (rr.cnt == 0 || (unsigned)lx >= (unsigned)rr.n[0] || (unsigned)ly >= (unsigned)rr.n[1] ||
                (unsigned)lz >= (unsigned)rr.n[2])
                continue;
            emit_records_before(rr.first);
            const long long l = lx + (long long)rr.n[0] * (ly + (long long)rr.n[1] * lz);
            unsigned* slot = p.box_slot + (long long)rr.block0 * kCountBlock + l;
            const unsigned c = *slot;
            *slot = (unsigned)(pos - p.row_ptr[vv]);      // the segment's offset within the row
            pos += c;
        }
    }
    if (!row) return;
    emit_records_before(0x7fffffff);
}

// Fill pass, box-major, second part: one thread per (run, voxel of the run's
// box), as in the count pass, writes the segment's kept entries from the
// position the first part left.
__global__ void k_csr_fill_box(const CsrBuildParams p)
{
    __shared__ int s_run;
    if (threadIdx.x == 0) {
        int lo = 0, hi = p.n_runs;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (p.run_block0[mid] <= (int)blockIdx.x) lo = mid; else hi = mid;
        }
        s_run = lo;
    }
    __syncthreads();
    const int r = s_run;
    const int cnt = p.run_count[r];
    if (cnt == 0) return;
    const DevBox bb = p.boxes[p.run_box[r]];
    const long long size = (long long)bb.n[0] * bb.n[1] * bb.n[2];
    const long long l = (long long)(blockIdx.x - p.run_block0[r]) * blockDim.x + threadIdx.x;
    if (l >= size) return;
    const int first = p.run_first[r];
    const int row = (int)(l / bb.n[0]);
    const int lx = (int)(l - (long long)row * bb.n[0]), ly = row % bb.n[1], lz = row / bb.n[1];
    const long long v = (bb.lo[0] + lx) + (long long)p.sg.n[0] * ((bb.lo[1] + ly) + (long long)p.sg.n[1] * (bb.lo[2] + lz));
    long long pos = p.row_ptr[v] + p.box_slot[blockIdx.x * (long long)blockDim.x + threadIdx.x];
    const double inv_rho = p.inv_rho[v];
    const float inv_rho_f = (float)inv_rho;
    const unsigned long long* col0 = p.scratch + p.boxes[p.items[first].box].base + l;
    for (int t0 = 0; t0 < cnt; t0 += 8) {
        unsigned long long q[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) q[u] = t0 + u < cnt ? __ldcs(col0 + (long long)(t0 + u) * size) : 0ull;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (q[u] == 0ull) continue;
            const int it = first + t0 + u;
            if (!keep_entry(q[u], inv_rho, inv_rho_f, p.thr[it], p.thr_f[it])) continue;
            p.col[pos] = p.items[it].spot;
            p.val[pos] = (float)((double)q[u] * inv_rho * p.item_scale[it]);
            ++pos;
        }
    }
}

__global__ void k_ovf_count(const OvfRec* __restrict__ rec, long long n, int n_spots, long long nvox,
                            unsigned long long* __restrict__ cnt)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const OvfRec r = rec[i];
        atomicAdd(cnt + (long long)(r.item / n_spots) * nvox + r.voxel, 1ull);
    }
}

__global__ void k_ovf_scatter(const OvfRec* __restrict__ rec, long long n, int n_spots, long long nvox,
                              const long long* __restrict__ off, unsigned long long* __restrict__ cursor,
                              OvfRec* __restrict__ sorted)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const OvfRec r = rec[i];
        const long long b = (long long)(r.item / n_spots) * nvox + r.voxel;
        sorted[off[b] + (long long)atomicAdd(cursor + b, 1ull)] = r;
    }
}

// One thread per bucket: insertion sort by item, sum records of the same
// item, and raise that item's column maximum (q / rho as FP64 bits).
__global__ void k_ovf_merge(OvfRec* __restrict__ sorted, const long long* __restrict__ off, long long n_buckets,
                            long long nvox, const double* __restrict__ rho, int* __restrict__ len,
                            double* __restrict__ colmax)
{
    const long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (b >= n_buckets) return;
    const long long o = off[b], n = off[b + 1] - o;
    if (n == 0) { len[b] = 0; return; }
    OvfRec* r = sorted + o;
    for (long long i = 1; i < n; ++i) {
        const OvfRec key = r[i];
        long long k = i - 1;
        while (k >= 0 && r[k].item > key.item) { r[k + 1] = r[k]; --k; }
        r[k + 1] = key;
    }
    long long m = 0;
    for (long long i = 0; i < n; ++i) {
        if (m > 0 && r[m - 1].item == r[i].item) r[m - 1].q += r[i].q;
        else r[m++] = r[i];
    }
    len[b] = (int)m;
    const double inv_rho = 1.0 / rho[b % nvox];
    for (long long i = 0; i < m; ++i)
        atomicMax(reinterpret_cast<unsigned long long*>(colmax + r[i].item),
                  (unsigned long long)__double_as_longlong((double)r[i].q * inv_rho));
}

constexpr int kScanBlock = 1024;
constexpr int kScanItems = 4;

// Exclusive scan of each 4096-element tile; tile totals to block_sums.
__global__ void k_scan_tiles(const long long* __restrict__ in, long long* __restrict__ out, long long n,
                             long long* __restrict__ block_sums)
{
    __shared__ long long warp_tot[32];
    const long long base = (long long)blockIdx.x * kScanBlock * kScanItems + (long long)threadIdx.x * kScanItems;
    long long v[kScanItems];
    long long run = 0;
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = base + i < n ? in[base + i] : 0;
        run += v[i];
    }
    // inclusive warp scan of per-thread totals
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long inc = run;
    for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        long long w = lane < (kScanBlock >> 5) ? warp_tot[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const long long t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        warp_tot[lane] = w;   // inclusive
    }
    __syncthreads();
    long long excl = inc - run + (warp > 0 ? warp_tot[warp - 1] : 0);
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = excl;
        excl += v[i];
    }
    if (threadIdx.x == kScanBlock - 1) block_sums[blockIdx.x] = excl;
}

__global__ void k_scan_add(long long* __restrict__ out, long long n, const long long* __restrict__ offsets)
{
    const long long base = (long long)blockIdx.x * kScanBlock * kScanItems;
    const long long add = offsets[blockIdx.x];
    for (int i = threadIdx.x; i < kScanBlock * kScanItems; i += kScanBlock)
        if (base + i < n) out[base + i] += add;
}

}  // namespace

cudaError_t launch_scoring_density(const int16_t* ct, Grid3 ctg, Grid3 sg, const double* curve15_dev,
                                   const double ct_spacing[3], const double sg_spacing[3], double* rho_out,
                                   cudaStream_t s)
{
    const long long nv = (long long)sg.n[0] * sg.n[1] * sg.n[2];
    const int block = 256;
    const long long grid = (nv + block - 1) / block;
    k_scoring_density<<<(unsigned)grid, block, 0, s>>>(ct, ctg, sg, curve15_dev, ct_spacing[0], ct_spacing[1],
                                                        ct_spacing[2], sg_spacing[0], sg_spacing[1], sg_spacing[2],
                                                        rho_out);
    return cudaGetLastError();
}

cudaError_t launch_dose_normalise(const unsigned long long* acc, const double* rho, long long nvox, double scale,
                                  float* dose, cudaStream_t s)
{
    const int block = 256;
    long long grid = (nvox + block - 1) / block;
    if (grid > 152 * 64) grid = 152 * 64;
    k_dose_normalise<<<(unsigned)grid, block, 0, s>>>(acc, rho, nvox, scale, dose);
    return cudaGetLastError();
}

cudaError_t launch_column_max(const unsigned long long* scratch, const DevItem* items, const DevBox* boxes,
                              const double* inv_rho, const float* inv_rho_f, const Grid3 sg, int first_item,
                              int n_items, double* colmax, cudaStream_t s)
{
    if (n_items <= 0) return cudaSuccess;
    k_column_max<<<n_items, 512, 0, s>>>(scratch, items, boxes, inv_rho, inv_rho_f, sg, first_item, colmax);
    return cudaGetLastError();
}

cudaError_t launch_column_threshold(const double* colmax, int n, double rel, double* thr, float* thr_f, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_column_threshold<<<(n + 255) / 256, 256, 0, s>>>(colmax, n, rel, thr, thr_f);
    return cudaGetLastError();
}

cudaError_t launch_reciprocal(const double* x, long long n, double* out, float* out_f, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const long long blocks = (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096;
    k_reciprocal<<<(int)blocks, 256, 0, s>>>(x, n, out, out_f);
    return cudaGetLastError();
}

cudaError_t launch_csr_count(const CsrBuildParams& p, int box_blocks, cudaStream_t s)
{
    if (box_blocks > 0) k_csr_count_box<<<box_blocks, kCountBlock, 0, s>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !p.ovf) return e;
    const int block = 256;
    k_csr_count_records<<<(unsigned)((p.nvox + block - 1) / block), block, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_csr_fill(const CsrBuildParams& p, int box_blocks, cudaStream_t s)
{
    const int block = 128;
    const long long grid = (p.nvox + block - 1) / block;
    k_csr_offsets<<<(unsigned)grid, block, 0, s>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || box_blocks <= 0) return e;
    k_csr_fill_box<<<box_blocks, kCountBlock, 0, s>>>(p);
    return cudaGetLastError();
}

int scan_launches(long long n)
{
    const long long tile = (long long)kScanBlock * kScanItems;
    const long long nb = (n + tile - 1) / tile;
    if (nb <= 0) return 0;
    if (nb == 1) return 1;
    return 2 + scan_launches(nb);
}

cudaError_t launch_ovf_count(const OvfRec* rec, long long n, int n_spots, long long nvox, long long* bucket_cnt,
                             cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_ovf_count<<<152 * 8, 256, 0, s>>>(rec, n, n_spots, nvox, reinterpret_cast<unsigned long long*>(bucket_cnt));
    return cudaGetLastError();
}

cudaError_t launch_ovf_scatter(const OvfRec* rec, long long n, int n_spots, long long nvox, const long long* bucket_off,
                               long long* cursor, OvfRec* sorted, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_ovf_scatter<<<152 * 8, 256, 0, s>>>(rec, n, n_spots, nvox, bucket_off,
                                          reinterpret_cast<unsigned long long*>(cursor), sorted);
    return cudaGetLastError();
}

cudaError_t launch_ovf_merge(OvfRec* sorted, const long long* bucket_off, long long n_buckets, long long nvox,
                             const double* rho, int* bucket_len, double* colmax, cudaStream_t s)
{
    const int block = 256;
    const long long grid = (n_buckets + block - 1) / block;
    k_ovf_merge<<<(unsigned)grid, block, 0, s>>>(sorted, bucket_off, n_buckets, nvox, rho, bucket_len, colmax);
    return cudaGetLastError();
}

size_t scan_tmp_elems(long long n)
{
    size_t total = 0;
    const long long tile = (long long)kScanBlock * kScanItems;
    while (n > 1) {
        const long long nb = (n + tile - 1) / tile;
        total += (size_t)(2 * nb + 1);
        n = nb;
    }
    return total + 2;
}

// Exclusive scan of n int64 values (out may not alias in); out[n] is not written.
cudaError_t launch_exclusive_scan(const long long* in, long long* out, long long n, long long* tmp, cudaStream_t s)
{
    const long long tile = (long long)kScanBlock * kScanItems;
    const long long nb = (n + tile - 1) / tile;
    if (nb <= 0) return cudaSuccess;
    long long* sums = tmp;
    long long* sums_scan = tmp + nb;
    k_scan_tiles<<<(unsigned)nb, kScanBlock, 0, s>>>(in, out, n, sums);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || nb == 1) return e;
    e = launch_exclusive_scan(sums, sums_scan, nb, tmp + 2 * nb + 1, s);
    if (e != cudaSuccess) return e;
    k_scan_add<<<(unsigned)nb, kScanBlock, 0, s>>>(out, n, sums_scan);
    return cudaGetLastError();
}

}  // namespace vpmc
