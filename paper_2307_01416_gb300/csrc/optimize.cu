// Robust spot-weight optimisation over the scenarios' influence matrices
// (Sec. 2.E: robust optimisation over 13 scenarios against the target
// constraints of Table 3).  The paper's optimiser is an in-house
// trial-and-error procedure; the objective here is a worst case over the
// scenarios of quadratic target under- and overdose and ring-overdose
// penalties, minimised by Adam with non-negative weights.
//
// Only target and ring voxels enter the objective and its gradient, so one
// setup pass per call copies those rows of every scenario into a compact CSR
// (16-bit spot indices, rows padded to 8 entries: one 16-byte load of
// columns and two of values per lane and step).  Each iteration then runs,
// with no host synchronisation:
//   k_fwd         d_s = A_s x on the compact rows of every scenario (a warp
//                 per row) and the scenario's objective f_s (FP64 block sums);
//   k_bwd_rows    s* = first s with the largest f_s (every block), recorded;
//                 each block adds f'(d_i) A_s*,i. over its 8 rows, in row
//                 order, into a shared-memory gradient (rows with f'(d_i) = 0
//                 are skipped) and stores it as the block's partial;
//   k_reduce_adam g_j = the partials summed in a fixed order, then the Adam
//                 step on x_j, clamped at zero.
// Every sum has a fixed order, so repeated calls give the same bits.  The
// iteration is HBM-bound.  Full-matrix products (dose of the weights, target
// indices over all voxels) use k_spmv_obj: a sub-warp per row of the
// caller's CSR.
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
constexpr size_t kBwdSmemMax = 227 * 1024;      // shared memory of one gradient block

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

// Copies the target/ring rows into the compact CSR: a warp per row and
// scenario; pads and entries with an out-of-range spot become (0, 0.0).
// Sets *unordered if a row's spot indices are not strictly increasing (a
// row may then repeat a spot).
__global__ void __launch_bounds__(256) k_tr_gather(const Csr* __restrict__ mats, const int* __restrict__ tr_rows,
                                                   int n_tr, int n_cols, const long long* __restrict__ crp,
                                                   unsigned short* __restrict__ ccol, float* __restrict__ cval,
                                                   int* __restrict__ unordered)
{
    const int s = blockIdx.y, lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= n_tr) return;
    const Csr A = mats[s];
    const int row = __ldg(tr_rows + i);
    const long long b = __ldg(A.row_ptr + row), len = __ldg(A.row_ptr + row + 1) - b;
    const long long dst = crp[(long long)s * (n_tr + 1) + i];
    const long long plen = crp[(long long)s * (n_tr + 1) + i + 1] - dst;
    for (long long k = lane; k < plen; k += 32) {
        int j = 0;
        float v = 0.0f;
        if (k < len) {
            j = __ldg(A.col + b + k);
            if (k > 0 && j <= __ldg(A.col + b + k - 1)) *unordered = 1;
            if ((unsigned)j < (unsigned)n_cols)
                v = __ldg(A.val + b + k);
            else
                j = 0;
        }
        ccol[dst + k] = (unsigned short)j;
        cval[dst + k] = v;
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

constexpr int kBwdRows = 8;                     // compact rows per gradient block

// Worst scenario and the blocks' gradient partials: each block adds
// f'(d_i) A_s*,ij over its rows, one row after the other (a barrier after
// each), into a shared-memory gradient.  Pads and zero values add nothing
// and are skipped.  kAtomic = false when every row's spots are strictly
// increasing: a row's adds then touch distinct spots and are plain
// read-add-writes; kAtomic = true for rows that may repeat a spot (shared
// atomics; the repeats of a row add in atomic order).  Either way the sum
// order of every spot is the row order.  Grid: compact rows / kBwdRows, 256
// threads, n_cols floats of shared memory.
template <bool kAtomic>
__global__ void __launch_bounds__(256) k_bwd_rows(const long long* __restrict__ crp,
                                                  const unsigned short* __restrict__ ccol,
                                                  const float* __restrict__ cval, int n_tr, int n_cols,
                                                  const float* __restrict__ dose_tr,
                                                  const unsigned char* __restrict__ tr_cls, ObjParams q,
                                                  const double* __restrict__ fsum_cur, double* __restrict__ fsum_next,
                                                  int n_scen, float* __restrict__ hist, int it,
                                                  float* __restrict__ partial)
{
    extern __shared__ float gs[];
    __shared__ int s_star;
    __shared__ double s_f[kMaxScen];
    __shared__ float s_ri[kBwdRows];
    __shared__ long long s_b[kBwdRows], s_e[kBwdRows];
    if (threadIdx.x < n_scen) s_f[threadIdx.x] = fsum_cur[threadIdx.x];
    for (int j = threadIdx.x; j < n_cols; j += blockDim.x) gs[j] = 0.0f;
    __syncthreads();
    if (threadIdx.x == 0) {
        int w = 0;
        for (int k = 1; k < n_scen; ++k)
            if (s_f[k] > s_f[w]) w = k;
        s_star = w;
        if (blockIdx.x == 0 && hist) hist[it] = (float)s_f[w];
    }
    if (blockIdx.x == 0 && threadIdx.x < n_scen) fsum_next[threadIdx.x] = 0.0;
    __syncthreads();
    const int s = s_star;
    // the block's rows: f'(d_i) and entry range, loaded together
    if (threadIdx.x < kBwdRows) {
        const int i = blockIdx.x * kBwdRows + threadIdx.x;
        float ri = 0.0f;
        long long b = 0, e = 0;
        if (i < n_tr) {
            ri = obj_grad(__ldg(dose_tr + (long long)s * n_tr + i), __ldg(tr_cls + i), q);
            b = __ldg(crp + (long long)s * (n_tr + 1) + i);
            e = __ldg(crp + (long long)s * (n_tr + 1) + i + 1);
        }
        s_ri[threadIdx.x] = ri;
        s_b[threadIdx.x] = b;
        s_e[threadIdx.x] = ri != 0.0f ? e : b;          // rows with f' = 0 add nothing: empty
    }
    __syncthreads();
    auto add = [&](unsigned j, float a, float ri) {
        if (a != 0.0f) {
            if (kAtomic)
                atomicAdd(gs + j, a * ri);
            else
                gs[j] = fmaf(a, ri, gs[j]);
        }
    };
    auto add8 = [&](const uint4& c, const float4& v0, const float4& v1, float ri) {
        add(c.x & 0xffffu, v0.x, ri);
        add(c.x >> 16, v0.y, ri);
        add(c.y & 0xffffu, v0.z, ri);
        add(c.y >> 16, v0.w, ri);
        add(c.z & 0xffffu, v1.x, ri);
        add(c.z >> 16, v1.y, ri);
        add(c.w & 0xffffu, v1.z, ri);
        add(c.w >> 16, v1.w, ri);
    };
    const long long lane8 = (long long)threadIdx.x * kPadRow, stride = (long long)blockDim.x * kPadRow;
    // first step of row 0 in registers; each iteration loads the next row's
    // first step before adding the current one
    uint4 c = make_uint4(0u, 0u, 0u, 0u);
    float4 v0 = make_float4(0.f, 0.f, 0.f, 0.f), v1 = v0;
    if (s_b[0] + lane8 < s_e[0]) {
        c = __ldcs(reinterpret_cast<const uint4*>(ccol + s_b[0] + lane8));
        v0 = __ldcs(reinterpret_cast<const float4*>(cval + s_b[0] + lane8));
        v1 = __ldcs(reinterpret_cast<const float4*>(cval + s_b[0] + lane8 + 4));
    }
    for (int r = 0; r < kBwdRows; ++r) {
        uint4 cn = make_uint4(0u, 0u, 0u, 0u);
        float4 w0 = make_float4(0.f, 0.f, 0.f, 0.f), w1 = w0;
        if (r + 1 < kBwdRows && s_b[r + 1] + lane8 < s_e[r + 1]) {
            cn = __ldcs(reinterpret_cast<const uint4*>(ccol + s_b[r + 1] + lane8));
            w0 = __ldcs(reinterpret_cast<const float4*>(cval + s_b[r + 1] + lane8));
            w1 = __ldcs(reinterpret_cast<const float4*>(cval + s_b[r + 1] + lane8 + 4));
        }
        const float ri = s_ri[r];
        const long long b = s_b[r], e = s_e[r];
        if (b + lane8 < e) add8(c, v0, v1, ri);
        for (long long k = b + lane8 + stride; k < e; k += stride) {          // rows longer than one step
            add8(__ldcs(reinterpret_cast<const uint4*>(ccol + k)), __ldcs(reinterpret_cast<const float4*>(cval + k)),
                 __ldcs(reinterpret_cast<const float4*>(cval + k + 4)), ri);
        }
        if (b < e) __syncthreads();                       // block-uniform
        c = cn;
        v0 = w0;
        v1 = w1;
    }
    __syncthreads();
    float* out = partial + (long long)blockIdx.x * n_cols;
    for (int j = threadIdx.x; j < n_cols; j += blockDim.x) out[j] = gs[j];
}

// g_j = the blocks' partials in a fixed order: slice t of 32 sums (FP32) the
// partials of blocks t, t + 32, ..., then the 32 slice sums are added in
// order (FP64); then Adam (Kingma & Ba 2015) on x_j, clamped at zero.
// Grid: n_cols / 16, 512 threads (16 spots x 32 slices).
__global__ void __launch_bounds__(512) k_reduce_adam(const float* __restrict__ partial, int nb, int n_cols,
                                                      float* __restrict__ x, float* __restrict__ m,
                                                      float* __restrict__ v, float step, float c1, float c2,
                                                      float eps)
{
    __shared__ float red[32][17];
    const int c = threadIdx.x & 15, sl = threadIdx.x >> 4;
    const int j = blockIdx.x * 16 + c;
    float a = 0.0f;
    if (j < n_cols) {
#pragma unroll 8
        for (int b = sl; b < nb; b += 32) a += __ldcs(partial + (long long)b * n_cols + j);
    }
    red[sl][c] = a;
    __syncthreads();
    if (sl != 0 || j >= n_cols) return;
    double acc = 0.0;
#pragma unroll 8
    for (int k = 0; k < 32; ++k) acc += (double)red[k][c];
    const float g = (float)acc;
    const float mj = fmaf(0.9f, m[j], 0.1f * g), vj = fmaf(0.999f, v[j], 0.001f * g * g);
    m[j] = mj;
    v[j] = vj;
    x[j] = fmaxf(x[j] - step * (mj * c1) / (sqrtf(vj * c2) + eps), 0.0f);
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
    float* partial = nullptr;                   // [gradient blocks x n_cols]
    int* unordered = nullptr;
    float* dose_tr = nullptr;
    double* fsum = nullptr;                     // [2 x S]: this iteration's sums, the next one's
    float* m = nullptr;
    float* v = nullptr;
    float* hist = nullptr;
    ~RobustWs()
    {
        cudaFree(mats); cudaFree(tr_rows); cudaFree(tr_cls); cudaFree(len); cudaFree(crp); cudaFree(ccol);
        cudaFree(cval); cudaFree(partial); cudaFree(unordered); cudaFree(dose_tr); cudaFree(fsum); cudaFree(m); cudaFree(v);
        cudaFree(hist);
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
    if ((size_t)n_cols * sizeof(float) > kBwdSmemMax) return cudaErrorInvalidValue;
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
    OPT_TRY(dalloc(&w.unordered, 1));
    OPT_TRY(cudaMemsetAsync(w.unordered, 0, sizeof(int), st));
    k_tr_gather<<<dim3((unsigned)((n_tr + 7) / 8), (unsigned)S), 256, 0, st>>>(w.mats, w.tr_rows, n_tr, n_cols,
                                                                               w.crp, w.ccol, w.cval, w.unordered);
    OPT_TRY(cudaGetLastError());
    int unordered = 0;
    OPT_TRY(cudaMemcpyAsync(&unordered, w.unordered, sizeof(int), cudaMemcpyDeviceToHost, st));
    OPT_TRY(cudaStreamSynchronize(st));
    // iteration state
    const int nb = (n_tr + kBwdRows - 1) / kBwdRows;
    OPT_TRY(dalloc(&w.partial, (size_t)nb * n_cols));
    OPT_TRY(dalloc(&w.dose_tr, (size_t)S * n_tr));
    OPT_TRY(dalloc(&w.fsum, (size_t)2 * S));
    OPT_TRY(dalloc(&w.m, (size_t)n_cols));
    OPT_TRY(dalloc(&w.v, (size_t)n_cols));
    OPT_TRY(dalloc(&w.hist, (size_t)std::max(spec.iterations, 1)));
    OPT_TRY(cudaMemsetAsync(w.fsum, 0, sizeof(double) * 2 * S, st));
    OPT_TRY(cudaMemsetAsync(w.m, 0, sizeof(float) * n_cols, st));
    OPT_TRY(cudaMemsetAsync(w.v, 0, sizeof(float) * n_cols, st));
    const int smem = (int)(sizeof(float) * n_cols);
    auto* bwd = unordered ? k_bwd_rows<true> : k_bwd_rows<false>;
    OPT_TRY(cudaFuncSetAttribute(bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    OPT_TRY(cudaEventRecord(ev[1], st));
    const ObjParams q{spec.dp, spec.w_u, spec.w_o, spec.w_r, spec.over, spec.ring,
                      1.0f / (float)std::max<long long>(spec.n_target, 1),
                      1.0f / (float)std::max<long long>(spec.n_ring, 1)};
    const dim3 gf((unsigned)std::max((n_tr + 7) / 8, 1), (unsigned)S);
    for (int it = 0; it < spec.iterations; ++it) {
        double* cur = w.fsum + (it & 1) * S;
        double* nxt = w.fsum + ((it + 1) & 1) * S;
        k_fwd<<<gf, 256, 0, st>>>(w.crp, w.ccol, w.cval, n_tr, x, w.tr_cls, q, w.dose_tr, cur);
        bwd<<<(unsigned)nb, 256, smem, st>>>(w.crp, w.ccol, w.cval, n_tr, n_cols, w.dose_tr, w.tr_cls, q, cur, nxt, S,
                                             w.hist, it, w.partial);
        const double t = it + 1;
        k_reduce_adam<<<(unsigned)((n_cols + 15) / 16), 512, 0, st>>>(
            w.partial, nb, n_cols, x, w.m, w.v, spec.step, (float)(1.0 / (1.0 - std::pow(0.9, t))),
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
