// Robust spot-weight optimisation over the scenarios' influence matrices
// (Sec. 2.E: robust optimisation over 13 scenarios against the target
// constraints of Table 3).  The paper's optimiser is an in-house
// trial-and-error procedure; the objective here is a worst case over the
// scenarios of quadratic target under- and overdose and ring-overdose
// penalties, minimised by Adam with non-negative weights.
//
// Only target and ring voxels enter the objective and its gradient, so one
// setup pass per call copies those rows of every scenario into
//   a compact CSR (16-bit spot indices, rows padded to 8 entries: one
//   16-byte load of columns, two of values per lane and step), and
//   its transpose (CSC over the same rows, columns padded to 4 entries),
// and each iteration then runs two kernels, with no host synchronisation:
//   k_fwd        d_s = A_s x on the compact rows of every scenario (a warp per
//                row) and the scenario's objective f_s (FP64 block sums);
//   k_bwd_adam   s* = first s with the largest f_s (every block), records it;
//                g_j = sum_i A_s*,ij f'(d_i) down spot j's transposed column
//                (a warp per 512-entry chunk; the chunks' partial sums are
//                added in a fixed order), then Adam on x_j, clamped at zero,
//                by the last chunk of spot j.
// Both stream their compact arrays once per iteration: HBM-bound.
// Full-matrix products (dose of the weights, target indices over all
// voxels) use k_spmv_obj: a sub-warp per row of the caller's CSR.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "vpmc_internal.cuh"

namespace vpmc {
namespace {

constexpr unsigned kFullMask = 0xffffffffu;
constexpr int kLanesPerRow = 8;                 // 4 rows per warp

struct Csr {
    const long long* row_ptr;
    const int* col;
    const float* val;
};

struct ObjParams {
    float dp, w_u, w_o, w_r, over, ring;       // prescription and weights
    float inv_nt, inv_nr;                       // 1 / |T|, 1 / |R|
};

__device__ __forceinline__ float obj_term(float d, unsigned char c, const ObjParams& q)
{
    if (c == 1) {
        const float u = fmaxf(q.dp - d, 0.0f), o = fmaxf(d - q.over * q.dp, 0.0f);
        return q.inv_nt * (q.w_u * u * u + q.w_o * o * o);
    }
    if (c == 2) {
        const float r = fmaxf(d - q.ring * q.dp, 0.0f);
        return q.inv_nr * q.w_r * r * r;
    }
    return 0.0f;
}

__device__ __forceinline__ float obj_grad(float d, unsigned char c, const ObjParams& q)
{
    if (c == 1) {
        const float u = fmaxf(q.dp - d, 0.0f), o = fmaxf(d - q.over * q.dp, 0.0f);
        return 2.0f * q.inv_nt * (q.w_o * o - q.w_u * u);
    }
    if (c == 2) return 2.0f * q.inv_nr * q.w_r * fmaxf(d - q.ring * q.dp, 0.0f);
    return 0.0f;
}

// d_s = A_s x and f_s, grid (row blocks, scenario).
__global__ void k_spmv_obj(const Csr* __restrict__ mats, long long n_rows, int n_cols, const float* __restrict__ x,
                           const unsigned char* __restrict__ cls, ObjParams q, float* __restrict__ dose,
                           double* __restrict__ fsum)
{
    const int s = blockIdx.y;
    const Csr A = mats[s];
    const int lane = threadIdx.x & 31, sub = lane & (kLanesPerRow - 1);
    constexpr int kRowsPerWarp = 32 / kLanesPerRow;
    // warp-uniform loop over groups of kRowsPerWarp rows (the shuffles below
    // need every lane of the warp in every iteration)
    const long long wstride = (long long)gridDim.x * (blockDim.x >> 5) * kRowsPerWarp;
    float f = 0.0f;
    for (long long base = ((long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * kRowsPerWarp;
         base < n_rows; base += wstride) {
        const long long row = base + (lane / kLanesPerRow);
        float acc = 0.0f;
        if (row < n_rows) {
            const long long b = __ldg(A.row_ptr + row), e = __ldg(A.row_ptr + row + 1);
            for (long long k = b + sub; k < e; k += kLanesPerRow) {
                const int j = __ldg(A.col + k);
                if ((unsigned)j < (unsigned)n_cols) acc = fmaf(__ldg(A.val + k), __ldg(x + j), acc);
            }
        }
#pragma unroll
        for (int o = kLanesPerRow / 2; o >= 1; o >>= 1) acc += __shfl_xor_sync(kFullMask, acc, o);
        if (sub == 0 && row < n_rows) {
            dose[(long long)s * n_rows + row] = acc;
            f += obj_term(acc, __ldg(cls + row), q);
        }
    }
    // block sum of the objective
    __shared__ float part[32];
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) f += __shfl_xor_sync(kFullMask, f, o);
    if (lane == 0) part[threadIdx.x >> 5] = f;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0f;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(kFullMask, v, o);
        if (threadIdx.x == 0 && v != 0.0f) atomicAdd(fsum + s, (double)v);
    }
}

// Per scenario: [count(d >= D_p in T), count(T), count(d >= D_p), min_T d, max_T d]
// (min/max as FP32 bit patterns of non-negative doses, atomicMin/Max on ints).
__global__ void k_indices(const float* __restrict__ dose, long long n_rows, const unsigned char* __restrict__ cls,
                          float dp, unsigned long long* __restrict__ counts, int* __restrict__ minmax)
{
    const int s = blockIdx.y;
    const float* d = dose + (long long)s * n_rows;
    unsigned long long a = 0, b = 0, c = 0;
    int mn = 0x7f7fffff, mx = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_rows;
         i += (long long)gridDim.x * blockDim.x) {
        const float di = fmaxf(d[i], 0.0f);
        const bool t = cls[i] == 1;
        const bool hi = di >= dp;
        a += (t && hi) ? 1 : 0;
        b += t ? 1 : 0;
        c += hi ? 1 : 0;
        if (t) {
            mn = min(mn, __float_as_int(di));
            mx = max(mx, __float_as_int(di));
        }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        a += __shfl_xor_sync(kFullMask, a, o);
        b += __shfl_xor_sync(kFullMask, b, o);
        c += __shfl_xor_sync(kFullMask, c, o);
        mn = min(mn, __shfl_xor_sync(kFullMask, mn, o));
        mx = max(mx, __shfl_xor_sync(kFullMask, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (a) atomicAdd(counts + 3 * s, a);
        if (b) atomicAdd(counts + 3 * s + 1, b);
        if (c) atomicAdd(counts + 3 * s + 2, c);
        atomicMin(minmax + 2 * s, mn);
        atomicMax(minmax + 2 * s + 1, mx);
    }
}

__global__ void k_init_minmax(int* minmax, int n_scen)
{
    const int i = threadIdx.x;
    if (i < n_scen) {
        minmax[2 * i] = 0x7f7fffff;
        minmax[2 * i + 1] = 0;
    }
}

constexpr int kPadRow = 8;                      // compact CSR row padding (entries)
constexpr int kPadCol = 4;                      // CSC column padding (entries)
constexpr int kSetupSmemCols = 25600;           // ordered transpose (shared-memory cursors) up to this many spots

// len[s n_tr + i] = entries of target/ring row tr_rows[i] in scenario s.
__global__ void k_tr_len(const Csr* __restrict__ mats, const int* __restrict__ tr_rows, int n_tr,
                         long long* __restrict__ len)
{
    const int s = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_tr) return;
    const long long* rp = mats[s].row_ptr;
    const int r = __ldg(tr_rows + i);
    len[(long long)s * n_tr + i] = __ldg(rp + r + 1) - __ldg(rp + r);
}

constexpr int kSetupRows = 32;                  // compact rows per setup block (8 warps x 4)

// Copies the target/ring rows into the compact CSR (a warp per row and
// scenario; pads and entries with an out-of-range spot become (0, 0.0)) and
// counts, per spot, the entries the transpose will hold (every entry but a
// (0, 0.0) one).  kBlockCounts: the block counts in shared memory (n_cols
// ints) and stores its whole count row, bcnt[(s nb + block) n_cols + j];
// otherwise it adds to the per-scenario totals ccount with global atomics.
template <bool kBlockCounts>
__global__ void __launch_bounds__(256) k_tr_gather(const Csr* __restrict__ mats, const int* __restrict__ tr_rows,
                                                   int n_tr, int n_cols, const long long* __restrict__ crp,
                                                   unsigned short* __restrict__ ccol, float* __restrict__ cval,
                                                   int* __restrict__ ccount, int* __restrict__ bcnt)
{
    extern __shared__ int hist_s[];
    const int s = blockIdx.y, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (kBlockCounts) {
        for (int j = threadIdx.x; j < n_cols; j += blockDim.x) hist_s[j] = 0;
        __syncthreads();
    }
    const Csr A = mats[s];
    int* cnt = kBlockCounts ? hist_s : ccount + (long long)s * n_cols;
    for (int r = 0; r < kSetupRows / 8; ++r) {
        const int i = blockIdx.x * kSetupRows + r * 8 + warp;
        if (i >= n_tr) break;
        const int row = __ldg(tr_rows + i);
        const long long b = __ldg(A.row_ptr + row), len = __ldg(A.row_ptr + row + 1) - b;
        const long long dst = crp[(long long)s * (n_tr + 1) + i];
        const long long plen = crp[(long long)s * (n_tr + 1) + i + 1] - dst;
        for (long long k = lane; k < plen; k += 32) {
            int j = 0;
            float v = 0.0f;
            if (k < len) {
                j = __ldg(A.col + b + k);
                if ((unsigned)j < (unsigned)n_cols) {
                    v = __ldg(A.val + b + k);
                    if (j != 0 || v != 0.0f) atomicAdd(cnt + j, 1);
                } else {
                    j = 0;
                }
            }
            ccol[dst + k] = (unsigned short)j;
            cval[dst + k] = v;
        }
    }
    if (kBlockCounts) {
        __syncthreads();
        int* out = bcnt + ((long long)s * gridDim.x + blockIdx.x) * n_cols;
        for (int j = threadIdx.x; j < n_cols; j += blockDim.x) out[j] = hist_s[j];
    }
}

// Per scenario and spot: the blocks' counts become exclusive prefixes over
// the blocks (in block order) and their sum the spot's total.
__global__ void k_col_scan(int* __restrict__ bcnt, int nb, int n_cols, int* __restrict__ ccount)
{
    const int s = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_cols) return;
    int run = 0;
    int* c = bcnt + (long long)s * nb * n_cols + j;
    for (int b = 0; b < nb; ++b) {
        const int v = c[(long long)b * n_cols];
        c[(long long)b * n_cols] = run;
        run += v;
    }
    ccount[(long long)s * n_cols + j] = run;
}

// Transpose in row order: block b of scenario s places its rows one after
// the other; spot j's entries of this block start at tcp[j] + (entries of j
// in the blocks before), so every segment is sorted by compact row index and
// the layout does not depend on scheduling (a row that repeats a spot places
// its repeats in atomic order).
__global__ void __launch_bounds__(256) k_csc_fill_ordered(const long long* __restrict__ crp,
                                                          const unsigned short* __restrict__ ccol,
                                                          const float* __restrict__ cval, int n_tr, int n_cols,
                                                          const long long* __restrict__ tcp,
                                                          const int* __restrict__ bprefix, int* __restrict__ trow,
                                                          float* __restrict__ tval)
{
    extern __shared__ int cursor[];
    const int s = blockIdx.y;
    const long long* cp = tcp + (long long)s * (n_cols + 1);
    const int* pre = bprefix + ((long long)s * gridDim.x + blockIdx.x) * n_cols;
    for (int j = threadIdx.x; j < n_cols; j += blockDim.x) cursor[j] = pre[j];
    __syncthreads();
    for (int r = 0; r < kSetupRows; ++r) {
        const int i = blockIdx.x * kSetupRows + r;
        if (i >= n_tr) break;                             // block-uniform
        const long long b = crp[(long long)s * (n_tr + 1) + i], e = crp[(long long)s * (n_tr + 1) + i + 1];
        for (long long k = b + threadIdx.x; k < e; k += blockDim.x) {
            const int j = ccol[k];
            const float v = cval[k];
            if (j == 0 && v == 0.0f) continue;
            const long long pos = __ldg(cp + j) + atomicAdd(cursor + j, 1);
            trow[pos] = i;
            tval[pos] = v;
        }
        __syncthreads();
    }
}

// The same placement with one global cursor per spot (atomics): for more
// spots than shared memory holds.  The order inside a segment follows the
// atomics.
__global__ void __launch_bounds__(256) k_csc_fill_atomic(const long long* __restrict__ crp,
                                                         const unsigned short* __restrict__ ccol,
                                                         const float* __restrict__ cval, int n_tr, int n_cols,
                                                         const long long* __restrict__ tcp, int* __restrict__ fill,
                                                         int* __restrict__ trow, float* __restrict__ tval)
{
    const int s = blockIdx.y, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long* cp = tcp + (long long)s * (n_cols + 1);
    int* fl = fill + (long long)s * n_cols;
    for (int r = 0; r < kSetupRows / 8; ++r) {
        const int i = blockIdx.x * kSetupRows + r * 8 + warp;
        if (i >= n_tr) break;
        const long long b = crp[(long long)s * (n_tr + 1) + i], e = crp[(long long)s * (n_tr + 1) + i + 1];
        for (long long k = b + lane; k < e; k += 32) {
            const int j = ccol[k];
            const float v = cval[k];
            if (j == 0 && v == 0.0f) continue;
            const long long pos = cp[j] + atomicAdd(fl + j, 1);
            trow[pos] = i;
            tval[pos] = v;
        }
    }
}

// d_s on the compact rows and f_s; grid (rows / 8, scenarios), 256 threads.
__global__ void __launch_bounds__(256) k_fwd(const long long* __restrict__ crp, const unsigned short* __restrict__ ccol,
                                             const float* __restrict__ cval, int n_tr, const float* __restrict__ x,
                                             const unsigned char* __restrict__ tr_cls, ObjParams q,
                                             float* __restrict__ dose_tr, double* __restrict__ fsum)
{
    const int s = blockIdx.y, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = blockIdx.x * 8 + warp;
    float f = 0.0f;
    if (i < n_tr) {                                   // warp-uniform
        const long long b = __ldg(crp + (long long)s * (n_tr + 1) + i);
        const long long e = __ldg(crp + (long long)s * (n_tr + 1) + i + 1);
        float acc = 0.0f;
#pragma unroll 2
        for (long long k = b + lane * kPadRow; k < e; k += 32 * kPadRow) {
            const uint4 c = __ldcs(reinterpret_cast<const uint4*>(ccol + k));
            const float4 v0 = __ldcs(reinterpret_cast<const float4*>(cval + k));
            const float4 v1 = __ldcs(reinterpret_cast<const float4*>(cval + k + 4));
            acc = fmaf(v0.x, __ldg(x + (c.x & 0xffffu)), acc);
            acc = fmaf(v0.y, __ldg(x + (c.x >> 16)), acc);
            acc = fmaf(v0.z, __ldg(x + (c.y & 0xffffu)), acc);
            acc = fmaf(v0.w, __ldg(x + (c.y >> 16)), acc);
            acc = fmaf(v1.x, __ldg(x + (c.z & 0xffffu)), acc);
            acc = fmaf(v1.y, __ldg(x + (c.z >> 16)), acc);
            acc = fmaf(v1.z, __ldg(x + (c.w & 0xffffu)), acc);
            acc = fmaf(v1.w, __ldg(x + (c.w >> 16)), acc);
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) acc += __shfl_xor_sync(kFullMask, acc, o);
        if (lane == 0) {
            dose_tr[(long long)s * n_tr + i] = acc;
            f = obj_term(acc, __ldg(tr_cls + i), q);
        }
    }
    __shared__ float part[8];
    if (lane == 0) part[warp] = f;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
#pragma unroll
        for (int w = 0; w < 8; ++w) t += part[w];
        if (t != 0.0f) atomicAdd(fsum + s, (double)t);
    }
}

// A piece of one spot's transposed column: entries [b, b + n) of the
// transpose (n a multiple of 4, at most kChunk; n = 0 for a spot without
// entries, which still takes its Adam step with g = 0).  first: index of the
// spot's first chunk in the scenario's list; total: the spot's chunk count.
struct Chunk {
    long long b;
    int j, n, first, total;
};
constexpr int kChunk = 512;

// Worst scenario, gradient and Adam step (Kingma & Ba 2015) clamped at zero.
// A warp per chunk of the worst scenario's transpose: FP32 sums per lane (at
// most 16 terms), an FP64 warp sum stored as the chunk's partial; the last
// of spot j's chunks to arrive (counter per spot) adds the spot's partials
// in chunk order (the same sum whatever the arrival order), resets the
// counter and updates x_j, m_j, v_j.  Grid: the largest chunk count over the
// scenarios / 8, 256 threads.
__global__ void __launch_bounds__(256) k_bwd_adam(const Chunk* __restrict__ chunks,
                                                  const long long* __restrict__ chunk_off,
                                                  const int* __restrict__ trow, const float* __restrict__ tval,
                                                  int n_tr, const float* __restrict__ dose_tr,
                                                  const unsigned char* __restrict__ tr_cls, ObjParams q,
                                                  const double* __restrict__ fsum_cur, double* __restrict__ fsum_next,
                                                  int n_scen, float* __restrict__ hist, int it,
                                                  double* __restrict__ partial, int* __restrict__ arrived,
                                                  float* __restrict__ x, float* __restrict__ m, float* __restrict__ v,
                                                  float step, float c1, float c2, float eps)
{
    __shared__ int s_star;
    if (threadIdx.x == 0) {
        int w = 0;
        for (int k = 1; k < n_scen; ++k)
            if (fsum_cur[k] > fsum_cur[w]) w = k;
        s_star = w;
        if (blockIdx.x == 0 && hist) hist[it] = (float)fsum_cur[w];
    }
    if (blockIdx.x == 0 && threadIdx.x < n_scen) fsum_next[threadIdx.x] = 0.0;
    __syncthreads();
    const int s = s_star, lane = threadIdx.x & 31;
    const long long c = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
    const long long c0 = __ldg(chunk_off + s), c1n = __ldg(chunk_off + s + 1);
    if (c >= c1n - c0) return;                        // warp-uniform
    const Chunk ch = chunks[c0 + c];
    const float* d = dose_tr + (long long)s * n_tr;
    float accf = 0.0f;
    for (int k = lane * 4; k < ch.n; k += 128) {
        const int4 r = __ldcs(reinterpret_cast<const int4*>(trow + ch.b + k));
        const float4 a = __ldcs(reinterpret_cast<const float4*>(tval + ch.b + k));
        accf = fmaf(a.x, obj_grad(__ldg(d + r.x), __ldg(tr_cls + r.x), q), accf);
        accf = fmaf(a.y, obj_grad(__ldg(d + r.y), __ldg(tr_cls + r.y), q), accf);
        accf = fmaf(a.z, obj_grad(__ldg(d + r.z), __ldg(tr_cls + r.z), q), accf);
        accf = fmaf(a.w, obj_grad(__ldg(d + r.w), __ldg(tr_cls + r.w), q), accf);
    }
    double acc = (double)accf;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) acc += __shfl_xor_sync(kFullMask, acc, o);
    if (lane == 0) {
        const int j = ch.j;
        partial[c] = acc;
        __threadfence();
        if (atomicAdd(arrived + j, 1) == ch.total - 1) {
            __threadfence();
            double gsum = 0.0;
            for (int k = 0; k < ch.total; ++k) gsum += __ldcg(partial + ch.first + k);
            arrived[j] = 0;
            const float gj = (float)gsum;
            const float mj = fmaf(0.9f, m[j], 0.1f * gj), vj = fmaf(0.999f, v[j], 0.001f * gj * gj);
            m[j] = mj;
            v[j] = vj;
            x[j] = fmaxf(x[j] - step * (mj * c1) / (sqrtf(vj * c2) + eps), 0.0f);
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side (called from api.cu).
// ---------------------------------------------------------------------------
// Device buffers of the full-matrix target indices.
struct OptWorkspace {
    Csr* mats = nullptr;
    float* dose = nullptr;          // [S x n_rows]
    double* fsum = nullptr;         // [S]
    unsigned long long* counts = nullptr;
    int* minmax = nullptr;
};

static void free_ws(OptWorkspace& w)
{
    cudaFree(w.mats); cudaFree(w.dose); cudaFree(w.fsum); cudaFree(w.counts); cudaFree(w.minmax);
    w = OptWorkspace{};
}

static cudaError_t alloc_ws(OptWorkspace& w, const long long* const* rp, const int* const* col,
                            const float* const* val, int n_scen, long long n_rows)
{
    std::vector<Csr> h(n_scen);
    for (int s = 0; s < n_scen; ++s) h[s] = Csr{rp[s], col[s], val[s]};
    cudaError_t e;
    if ((e = cudaMalloc(&w.mats, sizeof(Csr) * n_scen)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(w.mats, h.data(), sizeof(Csr) * n_scen, cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&w.dose, sizeof(float) * n_scen * n_rows)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&w.fsum, sizeof(double) * n_scen)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&w.counts, sizeof(unsigned long long) * 3 * n_scen)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&w.minmax, sizeof(int) * 2 * n_scen)) != cudaSuccess) return e;
    return cudaSuccess;
}

// Device buffers of one robust optimisation call.
struct RobustWs {
    Csr* mats = nullptr;
    int* tr_rows = nullptr;
    unsigned char* tr_cls = nullptr;
    long long* len = nullptr;
    long long* crp = nullptr;
    unsigned short* ccol = nullptr;
    float* cval = nullptr;
    int* ccount = nullptr;
    long long* tcp = nullptr;
    int* fill = nullptr;
    int* trow = nullptr;
    float* tval = nullptr;
    Chunk* chunks = nullptr;                    // every scenario's transpose chunks
    long long* chunk_off = nullptr;             // [S + 1]
    int* bcnt = nullptr;                        // [S x blocks x n_cols] setup counts
    double* partial = nullptr;                  // [largest chunk count]
    int* arrived = nullptr;
    float* dose_tr = nullptr;
    double* fsum = nullptr;                     // [2 x S]: this iteration's sums, the next one's
    float* m = nullptr;
    float* v = nullptr;
    float* hist = nullptr;
    ~RobustWs()
    {
        cudaFree(mats); cudaFree(tr_rows); cudaFree(tr_cls); cudaFree(len); cudaFree(crp); cudaFree(ccol);
        cudaFree(cval); cudaFree(ccount); cudaFree(tcp); cudaFree(fill); cudaFree(trow); cudaFree(tval);
        cudaFree(chunks); cudaFree(chunk_off); cudaFree(bcnt); cudaFree(partial); cudaFree(arrived);
        cudaFree(dose_tr); cudaFree(fsum); cudaFree(m); cudaFree(v); cudaFree(hist);
    }
};

template <class T>
static cudaError_t dalloc(T** p, size_t n)
{
    return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * std::max<size_t>(n, 1));
}

cudaError_t run_robust_optimize(const long long* const* rp, const int* const* col, const float* const* val, int n_scen,
                                long long n_rows, int n_cols, const unsigned char* cls_host, const OptSpec& spec,
                                float* x, float* hist_host, cudaStream_t st, float* ms_out, OptSetupInfo* info)
{
    RobustWs w;
    cudaError_t e;
#define OPT_TRY(expr) do { if ((e = (expr)) != cudaSuccess) return e; } while (0)
    // target and ring rows, in voxel order
    std::vector<int> rows;
    std::vector<unsigned char> rcls;
    for (long long r = 0; r < n_rows; ++r)
        if (cls_host[r] == 1 || cls_host[r] == 2) {
            rows.push_back((int)r);
            rcls.push_back(cls_host[r]);
        }
    const int n_tr = (int)rows.size();
    const int S = n_scen;
    std::vector<Csr> h(S);
    for (int s = 0; s < S; ++s) h[s] = Csr{rp[s], col[s], val[s]};
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    for (auto& q : ev) OPT_TRY(cudaEventCreate(&q));
    struct EvFree {
        cudaEvent_t* e;
        ~EvFree() { for (int k = 0; k < 3; ++k) if (e[k]) cudaEventDestroy(e[k]); }
    } evfree{ev};
    OPT_TRY(cudaEventRecord(ev[0], st));
    OPT_TRY(dalloc(&w.mats, S));
    OPT_TRY(cudaMemcpyAsync(w.mats, h.data(), sizeof(Csr) * S, cudaMemcpyHostToDevice, st));
    OPT_TRY(dalloc(&w.tr_rows, n_tr));
    OPT_TRY(dalloc(&w.tr_cls, n_tr));
    OPT_TRY(cudaMemcpyAsync(w.tr_rows, rows.data(), sizeof(int) * n_tr, cudaMemcpyHostToDevice, st));
    OPT_TRY(cudaMemcpyAsync(w.tr_cls, rcls.data(), n_tr, cudaMemcpyHostToDevice, st));
    // compact row layout
    OPT_TRY(dalloc(&w.len, (size_t)S * n_tr));
    k_tr_len<<<dim3((unsigned)((n_tr + 255) / 256), (unsigned)S), 256, 0, st>>>(w.mats, w.tr_rows, n_tr, w.len);
    OPT_TRY(cudaGetLastError());
    std::vector<long long> len((size_t)S * n_tr), crp((size_t)S * (n_tr + 1));
    OPT_TRY(cudaMemcpyAsync(len.data(), w.len, sizeof(long long) * len.size(), cudaMemcpyDeviceToHost, st));
    OPT_TRY(cudaStreamSynchronize(st));
    long long total_c = 0, nnz_tr = 0;
    for (int s = 0; s < S; ++s) {
        for (int i = 0; i < n_tr; ++i) {
            crp[(size_t)s * (n_tr + 1) + i] = total_c;
            const long long l = len[(size_t)s * n_tr + i];
            nnz_tr += l;
            total_c += (l + kPadRow - 1) / kPadRow * kPadRow;
        }
        crp[(size_t)s * (n_tr + 1) + n_tr] = total_c;
    }
    OPT_TRY(dalloc(&w.crp, crp.size()));
    OPT_TRY(cudaMemcpyAsync(w.crp, crp.data(), sizeof(long long) * crp.size(), cudaMemcpyHostToDevice, st));
    OPT_TRY(dalloc(&w.ccol, (size_t)total_c));
    OPT_TRY(dalloc(&w.cval, (size_t)total_c));
    OPT_TRY(dalloc(&w.ccount, (size_t)S * n_cols));
    OPT_TRY(cudaMemsetAsync(w.ccount, 0, sizeof(int) * (size_t)S * n_cols, st));
    const int nb = (n_tr + kSetupRows - 1) / kSetupRows;
    const dim3 gw((unsigned)nb, (unsigned)S);
    // ordered transpose when the per-block counts and the cursors fit
    const bool ordered = n_cols <= kSetupSmemCols && (size_t)S * nb * n_cols * sizeof(int) <= ((size_t)1 << 30);
    if (ordered) {
        OPT_TRY(dalloc(&w.bcnt, (size_t)S * nb * n_cols));
        const int sm1 = (int)(sizeof(int) * n_cols);
        OPT_TRY(cudaFuncSetAttribute(k_tr_gather<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm1));
        k_tr_gather<true><<<gw, 256, sm1, st>>>(w.mats, w.tr_rows, n_tr, n_cols, w.crp, w.ccol, w.cval, w.ccount,
                                                w.bcnt);
        OPT_TRY(cudaGetLastError());
        k_col_scan<<<dim3((unsigned)((n_cols + 255) / 256), (unsigned)S), 256, 0, st>>>(w.bcnt, nb, n_cols,
                                                                                        w.ccount);
    } else {
        k_tr_gather<false><<<gw, 256, 0, st>>>(w.mats, w.tr_rows, n_tr, n_cols, w.crp, w.ccol, w.cval, w.ccount,
                                               nullptr);
    }
    OPT_TRY(cudaGetLastError());
    // transpose layout
    std::vector<int> cnt((size_t)S * n_cols);
    std::vector<long long> tcp((size_t)S * (n_cols + 1));
    OPT_TRY(cudaMemcpyAsync(cnt.data(), w.ccount, sizeof(int) * cnt.size(), cudaMemcpyDeviceToHost, st));
    OPT_TRY(cudaStreamSynchronize(st));
    long long total_t = 0;
    for (int s = 0; s < S; ++s) {
        for (int j = 0; j < n_cols; ++j) {
            tcp[(size_t)s * (n_cols + 1) + j] = total_t;
            total_t += ((long long)cnt[(size_t)s * n_cols + j] + kPadCol - 1) / kPadCol * kPadCol;
        }
        tcp[(size_t)s * (n_cols + 1) + n_cols] = total_t;
    }
    std::vector<Chunk> chunks;
    std::vector<long long> chunk_off(S + 1, 0);
    long long max_chunks = 0;
    for (int s = 0; s < S; ++s) {
        chunk_off[s] = (long long)chunks.size();
        for (int j = 0; j < n_cols; ++j) {
            const long long b = tcp[(size_t)s * (n_cols + 1) + j], e = tcp[(size_t)s * (n_cols + 1) + j + 1];
            const int first = (int)((long long)chunks.size() - chunk_off[s]);
            const int total = e > b ? (int)((e - b + kChunk - 1) / kChunk) : 1;
            for (int k = 0; k < total; ++k) {
                const long long c = b + (long long)k * kChunk;
                chunks.push_back(Chunk{c, j, (int)std::max<long long>(0, std::min<long long>(kChunk, e - c)), first,
                                       total});
            }
        }
        max_chunks = std::max(max_chunks, (long long)chunks.size() - chunk_off[s]);
    }
    chunk_off[S] = (long long)chunks.size();
    OPT_TRY(dalloc(&w.chunks, chunks.size()));
    OPT_TRY(dalloc(&w.chunk_off, chunk_off.size()));
    OPT_TRY(cudaMemcpyAsync(w.chunks, chunks.data(), sizeof(Chunk) * chunks.size(), cudaMemcpyHostToDevice, st));
    OPT_TRY(cudaMemcpyAsync(w.chunk_off, chunk_off.data(), sizeof(long long) * chunk_off.size(),
                            cudaMemcpyHostToDevice, st));
    OPT_TRY(dalloc(&w.tcp, tcp.size()));
    OPT_TRY(cudaMemcpyAsync(w.tcp, tcp.data(), sizeof(long long) * tcp.size(), cudaMemcpyHostToDevice, st));
    OPT_TRY(dalloc(&w.trow, (size_t)total_t));
    OPT_TRY(dalloc(&w.tval, (size_t)total_t));
    OPT_TRY(cudaMemsetAsync(w.trow, 0, sizeof(int) * (size_t)std::max<long long>(total_t, 1), st));
    OPT_TRY(cudaMemsetAsync(w.tval, 0, sizeof(float) * (size_t)std::max<long long>(total_t, 1), st));
    if (ordered) {
        const int sm2 = (int)(sizeof(int) * n_cols);
        OPT_TRY(cudaFuncSetAttribute(k_csc_fill_ordered, cudaFuncAttributeMaxDynamicSharedMemorySize, sm2));
        k_csc_fill_ordered<<<gw, 256, sm2, st>>>(w.crp, w.ccol, w.cval, n_tr, n_cols, w.tcp, w.bcnt, w.trow, w.tval);
    } else {
        OPT_TRY(dalloc(&w.fill, (size_t)S * n_cols));
        OPT_TRY(cudaMemsetAsync(w.fill, 0, sizeof(int) * (size_t)S * n_cols, st));
        k_csc_fill_atomic<<<gw, 256, 0, st>>>(w.crp, w.ccol, w.cval, n_tr, n_cols, w.tcp, w.fill, w.trow, w.tval);
    }
    OPT_TRY(cudaGetLastError());
    // iteration state
    OPT_TRY(dalloc(&w.dose_tr, (size_t)S * n_tr));
    OPT_TRY(dalloc(&w.fsum, (size_t)2 * S));
    OPT_TRY(dalloc(&w.m, (size_t)n_cols));
    OPT_TRY(dalloc(&w.v, (size_t)n_cols));
    OPT_TRY(dalloc(&w.partial, (size_t)max_chunks));
    OPT_TRY(dalloc(&w.arrived, (size_t)n_cols));
    OPT_TRY(cudaMemsetAsync(w.arrived, 0, sizeof(int) * n_cols, st));
    OPT_TRY(dalloc(&w.hist, (size_t)std::max(spec.iterations, 1)));
    OPT_TRY(cudaMemsetAsync(w.fsum, 0, sizeof(double) * 2 * S, st));
    OPT_TRY(cudaMemsetAsync(w.m, 0, sizeof(float) * n_cols, st));
    OPT_TRY(cudaMemsetAsync(w.v, 0, sizeof(float) * n_cols, st));
    OPT_TRY(cudaEventRecord(ev[1], st));
    const ObjParams q{spec.dp, spec.w_u, spec.w_o, spec.w_r, spec.over, spec.ring,
                      1.0f / (float)std::max<long long>(spec.n_target, 1),
                      1.0f / (float)std::max<long long>(spec.n_ring, 1)};
    const dim3 gf((unsigned)std::max((n_tr + 7) / 8, 1), (unsigned)S);
    const unsigned gb = (unsigned)((max_chunks + 7) / 8);
    for (int it = 0; it < spec.iterations; ++it) {
        double* cur = w.fsum + (it & 1) * S;
        double* nxt = w.fsum + ((it + 1) & 1) * S;
        k_fwd<<<gf, 256, 0, st>>>(w.crp, w.ccol, w.cval, n_tr, x, w.tr_cls, q, w.dose_tr, cur);
        const double t = it + 1;
        k_bwd_adam<<<gb, 256, 0, st>>>(w.chunks, w.chunk_off, w.trow, w.tval, n_tr, w.dose_tr, w.tr_cls, q, cur, nxt,
                                       S, w.hist, it, w.partial, w.arrived, x, w.m, w.v, spec.step,
                                       (float)(1.0 / (1.0 - std::pow(0.9, t))),
                                       (float)(1.0 / (1.0 - std::pow(0.999, t))), spec.eps);
    }
    OPT_TRY(cudaGetLastError());
    OPT_TRY(cudaEventRecord(ev[2], st));
    OPT_TRY(cudaStreamSynchronize(st));
    float setup = 0.0f, iters = 0.0f;
    cudaEventElapsedTime(&setup, ev[0], ev[1]);
    cudaEventElapsedTime(&iters, ev[1], ev[2]);
    if (ms_out) {
        ms_out[0] = iters;
        ms_out[1] = setup;
    }
    if (info) {
        info->n_tr = n_tr;
        info->nnz_tr = nnz_tr;
        info->compact_entries = total_c;
        info->transpose_entries = total_t;
    }
    if (hist_host && spec.iterations > 0)
        OPT_TRY(cudaMemcpy(hist_host, w.hist, sizeof(float) * spec.iterations, cudaMemcpyDeviceToHost));
#undef OPT_TRY
    return cudaSuccess;
}

cudaError_t run_weights_dose(const long long* rp, const int* col, const float* val, long long n_rows, int n_cols,
                             const float* x, float* dose, cudaStream_t st, int num_sms)
{
    Csr h{rp, col, val};
    Csr* d_m = nullptr;
    double* d_f = nullptr;
    unsigned char* d_c = nullptr;
    cudaError_t e = cudaMalloc(&d_m, sizeof(Csr));
    if (e == cudaSuccess) e = cudaMalloc(&d_f, sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&d_c, (size_t)n_rows);
    if (e == cudaSuccess) e = cudaMemcpy(d_m, &h, sizeof(Csr), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_c, 0, (size_t)n_rows, st);
    if (e == cudaSuccess) {
        ObjParams q{1, 0, 0, 0, 1, 1, 0, 0};
        k_spmv_obj<<<dim3((unsigned)(num_sms * 8), 1), 256, 0, st>>>(d_m, n_rows, n_cols, x, d_c, q, dose, d_f);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d_m);
    cudaFree(d_f);
    cudaFree(d_c);
    return e;
}

cudaError_t run_target_indices(const long long* const* rp, const int* const* col, const float* const* val, int n_scen,
                               long long n_rows, int n_cols, const unsigned char* cls, float dp, const float* x,
                               double* out, cudaStream_t st, int num_sms)
{
    OptWorkspace w;
    cudaError_t e = alloc_ws(w, rp, col, val, n_scen, n_rows);
    auto done = [&](cudaError_t r) { free_ws(w); return r; };
    if (e != cudaSuccess) return done(e);
    ObjParams q{dp, 0, 0, 0, 1, 1, 0, 0};
    cudaMemsetAsync(w.fsum, 0, sizeof(double) * n_scen, st);
    cudaMemsetAsync(w.counts, 0, sizeof(unsigned long long) * 3 * n_scen, st);
    k_init_minmax<<<1, 64, 0, st>>>(w.minmax, n_scen);
    k_spmv_obj<<<dim3((unsigned)(num_sms * 8), (unsigned)n_scen), 256, 0, st>>>(w.mats, n_rows, n_cols, x, cls, q, w.dose,
                                                                                 w.fsum);
    k_indices<<<dim3((unsigned)(num_sms * 4), (unsigned)n_scen), 256, 0, st>>>(w.dose, n_rows, cls, dp, w.counts,
                                                                               w.minmax);
    if ((e = cudaGetLastError()) != cudaSuccess) return done(e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return done(e);
    std::vector<unsigned long long> cnt(3 * n_scen);
    std::vector<int> mm(2 * n_scen);
    if ((e = cudaMemcpy(cnt.data(), w.counts, sizeof(unsigned long long) * cnt.size(), cudaMemcpyDeviceToHost)) !=
        cudaSuccess)
        return done(e);
    if ((e = cudaMemcpy(mm.data(), w.minmax, sizeof(int) * mm.size(), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return done(e);
    for (int s = 0; s < n_scen; ++s) {
        const double nt = (double)std::max<unsigned long long>(cnt[3 * s + 1], 1);
        float mn, mx;
        std::memcpy(&mn, &mm[2 * s], 4);
        std::memcpy(&mx, &mm[2 * s + 1], 4);
        out[4 * s + 0] = (double)cnt[3 * s] / nt;
        out[4 * s + 1] = cnt[3 * s + 1] ? mn / dp : 0.0;
        out[4 * s + 2] = (double)cnt[3 * s + 2] / nt;
        out[4 * s + 3] = cnt[3 * s + 1] ? mx / dp : 0.0;
    }
    return done(cudaSuccess);
}

}  // namespace vpmc
