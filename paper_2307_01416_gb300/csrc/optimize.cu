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
//                 per row), the scenario's objective f_s (FP64 block sums) and
//                 max_i |f'(d_i)|;
//   k_bwd_fixed   s* = first s with the largest f_s (every block), recorded;
//                 g = A_s*^T f'(d_s*) over the compact rows (a warp per row)
//                 as 64-bit fixed-point sums: shared-memory atomics per
//                 block, one global atomic per spot and block;
//   k_adam_fixed  g_j back to floating point, then the Adam step on x_j,
//                 clamped at zero.
// Integer sums do not depend on the order of the adds, so repeated calls
// give the same bits.  The iteration is HBM-bound.  Full-matrix products
// (dose of the weights, target indices over all voxels) use k_spmv_obj: a
// sub-warp per row of the caller's CSR.
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
                                                   int* __restrict__ unordered, unsigned* __restrict__ max_abs)
{
    const int s = blockIdx.y, lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= n_tr) return;                            // warp-uniform
    const Csr A = mats[s];
    const int row = __ldg(tr_rows + i);
    const long long b = __ldg(A.row_ptr + row), len = __ldg(A.row_ptr + row + 1) - b;
    const long long dst = crp[(long long)s * (n_tr + 1) + i];
    const long long plen = crp[(long long)s * (n_tr + 1) + i + 1] - dst;
    unsigned amax = 0u;                               // |a| as bits: non-negative floats order as integers
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
        amax = max(amax, __float_as_uint(fabsf(v)));
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) amax = max(amax, __shfl_xor_sync(kFullMask, amax, o));
    if (lane == 0 && amax) atomicMax(max_abs + s, amax);
}

// d_s on the compact rows, f_s and max_i |f'(d_i)| (as float bits); grid
// (rows / 8, scenarios), 256 threads.
__global__ void __launch_bounds__(256) k_fwd(const long long* __restrict__ crp, const unsigned short* __restrict__ ccol,
                                             const float* __restrict__ cval, int n_tr, const float* __restrict__ x,
                                             const unsigned char* __restrict__ tr_cls, ObjParams q,
                                             float* __restrict__ dose_tr, double* __restrict__ fsum,
                                             unsigned* __restrict__ max_r)
{
    const int s = blockIdx.y, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = blockIdx.x * 8 + warp;
    float f = 0.0f, rabs = 0.0f;
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
            const unsigned char c = __ldg(tr_cls + i);
            f = obj_term(acc, c, q);
            rabs = fabsf(obj_grad(acc, c, q));
        }
    }
    __shared__ float part[8], pmax[8];
    if (lane == 0) {
        part[warp] = f;
        pmax[warp] = rabs;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f, mx = 0.0f;
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            t += part[w];
            mx = fmaxf(mx, pmax[w]);
        }
        if (t != 0.0f) atomicAdd(fsum + s, (double)t);
        if (mx > 0.0f) atomicMax(max_r + s, __float_as_uint(mx));
    }
}

// p 2^k as a 64-bit integer, truncated toward zero (p a binary32 with
// |p| 2^k < 2^63; zero and subnormal p give 0).  Integer operations only.
__device__ __forceinline__ long long to_fixed_pow2(float p, int k)
{
    const unsigned bits = __float_as_uint(p);
    const int ex = (int)((bits >> 23) & 0xffu);
    if (ex == 0) return 0;
    const long long mant = (long long)((bits & 0x7fffffu) | 0x800000u);
    const int sh = ex - 150 + k;                      // p 2^k = mant 2^sh
    long long v;
    if (sh >= 0)
        v = mant << sh;
    else
        v = sh > -24 ? (mant >> -sh) : 0;
    return (bits >> 31) ? -v : v;
}

// Rows are cut into pieces of at most kRowChunk entries so that the
// gradient's warps get work of similar length: piece c of the worst
// scenario is row c / per_row, entries [k kRowChunk, (k + 1) kRowChunk) of it
// with k = c % per_row (empty when the row is shorter).
constexpr int kRowChunk = 1024;

// Worst scenario and the gradient in 64-bit fixed point.  The scale 2^k,
// k = 62 - ceil(log2 B) with B = max_i |f'(d_i)| x (compact rows) x max |a|
// of the worst scenario, bounds every partial sum by 2^62 (the row count is
// replaced by the scenario's entry count when a row may repeat a spot).
// Each warp takes row pieces (consecutive pieces go to different blocks;
// rows with f'(d_i) = 0 add nothing and are skipped) and adds a f'(d_i) 2^k to a
// shared-memory copy of g per block, held as two 32-bit words per spot: the
// low word by a native 32-bit atomic whose returned old value gives the
// carry, the high word by a second one (exact, whatever the order).  The
// block adds its copy to g with one 64-bit atomic per spot.  Grid: number of
// SMs, 1024 threads, n_cols x 8 bytes of shared memory.
__global__ void __launch_bounds__(1024) k_bwd_fixed(const long long* __restrict__ crp, int per_row,
                                                    const unsigned short* __restrict__ ccol,
                                                    const float* __restrict__ cval, int n_tr, int n_cols,
                                                    const float* __restrict__ dose_tr,
                                                    const unsigned char* __restrict__ tr_cls, ObjParams q,
                                                    const double* __restrict__ fsum_cur,
                                                    const unsigned* __restrict__ max_r_cur,
                                                    double* __restrict__ fsum_next, unsigned* __restrict__ max_r_next,
                                                    const unsigned* __restrict__ max_abs,
                                                    const float* __restrict__ count_bound, int n_scen,
                                                    float* __restrict__ hist, int it,
                                                    unsigned long long* __restrict__ g, int* __restrict__ g_shift)
{
    extern __shared__ unsigned gsw[];
    unsigned* lo = gsw;
    unsigned* hi = gsw + n_cols;
    __shared__ double s_f[kMaxScen];
    __shared__ int s_star, s_k;
    if (threadIdx.x < n_scen) s_f[threadIdx.x] = fsum_cur[threadIdx.x];
    for (int j = threadIdx.x; j < 2 * n_cols; j += blockDim.x) gsw[j] = 0u;
    __syncthreads();
    if (threadIdx.x == 0) {
        int w = 0;
        for (int k = 1; k < n_scen; ++k)
            if (s_f[k] > s_f[w]) w = k;
        const float bound = __uint_as_float(max_r_cur[w]) * count_bound[w] * __uint_as_float(max_abs[w]);
        int e = 129;                                  // an overflowed bound: above any binary32
        if (bound <= 3.4028235e38f) frexpf(bound, &e);  // bound < 2^e
        s_star = w;
        s_k = bound > 0.0f ? 62 - e : 0;
        if (blockIdx.x == 0) {
            if (hist) hist[it] = (float)s_f[w];
            *g_shift = s_k;
        }
    }
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x < n_scen) {
        fsum_next[threadIdx.x] = 0.0;
        max_r_next[threadIdx.x] = 0u;
    }
    const int s = s_star, kq = s_k, lane = threadIdx.x & 31;
    const float* d = dose_tr + (long long)s * n_tr;
    const int warps = blockDim.x >> 5;
    const long long* rp = crp + (long long)s * (n_tr + 1);
    const long long nc = (long long)n_tr * per_row;
    for (long long ci = blockIdx.x + (long long)gridDim.x * (threadIdx.x >> 5); ci < nc;
         ci += (long long)gridDim.x * warps) {
        const int i = (int)(ci / per_row);
        const long long rb = __ldg(rp + i), re = __ldg(rp + i + 1);
        const long long b = rb + (ci - (long long)i * per_row) * kRowChunk;
        if (b >= re) continue;                        // warp-uniform: the row is shorter
        const float ri = obj_grad(__ldg(d + i), __ldg(tr_cls + i), q);
        if (ri == 0.0f) continue;                     // warp-uniform
        const long long e = min(b + kRowChunk, re);
#pragma unroll 2
        for (long long k = b + lane * kPadRow; k < e; k += 32 * kPadRow) {
            const uint4 c = __ldcs(reinterpret_cast<const uint4*>(ccol + k));
            const float4 v0 = __ldcs(reinterpret_cast<const float4*>(cval + k));
            const float4 v1 = __ldcs(reinterpret_cast<const float4*>(cval + k + 4));
            const unsigned js[8] = {c.x & 0xffffu, c.x >> 16, c.y & 0xffffu, c.y >> 16,
                                    c.z & 0xffffu, c.z >> 16, c.w & 0xffffu, c.w >> 16};
            const float as[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const unsigned long long fx = (unsigned long long)to_fixed_pow2(as[t] * ri, kq);
                if (fx != 0ull) {
                    const unsigned l = (unsigned)fx;
                    const unsigned old = atomicAdd(lo + js[t], l);
                    const unsigned h = (unsigned)(fx >> 32) + (old + l < old ? 1u : 0u);
                    if (h) atomicAdd(hi + js[t], h);
                }
            }
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < n_cols; j += blockDim.x) {
        const unsigned long long t = ((unsigned long long)hi[j] << 32) | lo[j];
        if (t != 0ull) atomicAdd(g + j, t);
    }
}

// g_j = (fixed-point sum) 2^-k, reset for the next iteration, then Adam
// (Kingma & Ba 2015) on x_j, clamped at zero.
__global__ void k_adam_fixed(unsigned long long* __restrict__ g, const int* __restrict__ g_shift, int n_cols,
                             float* __restrict__ x, float* __restrict__ m, float* __restrict__ v, float step,
                             float c1, float c2, float eps)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_cols) return;
    const long long gi = (long long)g[j];
    g[j] = 0ull;
    const float gj = (float)ldexp((double)gi, -*g_shift);
    const float mj = fmaf(0.9f, m[j], 0.1f * gj), vj = fmaf(0.999f, v[j], 0.001f * gj * gj);
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
    unsigned long long* g = nullptr;            // [n_cols] fixed-point gradient
    int* g_shift = nullptr;
    unsigned* max_abs = nullptr;                // [S] max |a| (float bits)
    unsigned* max_r = nullptr;                  // [2 x S] max |f'(d)| (float bits)
    float* count_bound = nullptr;               // [S] entries of a spot over the compact rows, at most
    int* unordered = nullptr;
    float* dose_tr = nullptr;
    double* fsum = nullptr;                     // [2 x S]: this iteration's sums, the next one's
    float* m = nullptr;
    float* v = nullptr;
    float* hist = nullptr;
    ~RobustWs()
    {
        cudaFree(mats); cudaFree(tr_rows); cudaFree(tr_cls); cudaFree(len); cudaFree(crp); cudaFree(ccol);
        cudaFree(cval); cudaFree(g); cudaFree(g_shift); cudaFree(max_abs); cudaFree(max_r); cudaFree(count_bound);
        cudaFree(unordered);
        cudaFree(dose_tr); cudaFree(fsum); cudaFree(m); cudaFree(v);
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
    if ((size_t)n_cols * sizeof(unsigned long long) > kBwdSmemMax) return cudaErrorInvalidValue;
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
    long long longest = 0;
    for (int s = 0; s < S; ++s)
        for (int i = 0; i < n_tr; ++i)
            longest = std::max(longest, crp[(size_t)s * (n_tr + 1) + i + 1] - crp[(size_t)s * (n_tr + 1) + i]);
    const int per_row = (int)std::max<long long>(1, (longest + kRowChunk - 1) / kRowChunk);
    OPT_TRY(dalloc(&w.ccol, (size_t)total_c));
    OPT_TRY(dalloc(&w.cval, (size_t)total_c));
    OPT_TRY(dalloc(&w.unordered, 1));
    OPT_TRY(dalloc(&w.max_abs, S));
    OPT_TRY(cudaMemsetAsync(w.unordered, 0, sizeof(int), st));
    OPT_TRY(cudaMemsetAsync(w.max_abs, 0, sizeof(unsigned) * S, st));
    k_tr_gather<<<dim3((unsigned)((n_tr + 7) / 8), (unsigned)S), 256, 0, st>>>(
        w.mats, w.tr_rows, n_tr, n_cols, w.crp, w.ccol, w.cval, w.unordered, w.max_abs);
    OPT_TRY(cudaGetLastError());
    int unordered = 0;
    OPT_TRY(cudaMemcpyAsync(&unordered, w.unordered, sizeof(int), cudaMemcpyDeviceToHost, st));
    OPT_TRY(cudaStreamSynchronize(st));
    std::vector<float> cb(S);
    for (int s = 0; s < S; ++s) {
        long long nz = 0;
        for (int i = 0; i < n_tr; ++i) nz += len[(size_t)s * n_tr + i];
        cb[s] = (float)(unordered ? std::max<long long>(nz, 1) : n_tr);
    }
    OPT_TRY(dalloc(&w.count_bound, S));
    OPT_TRY(cudaMemcpyAsync(w.count_bound, cb.data(), sizeof(float) * S, cudaMemcpyHostToDevice, st));
    // iteration state
    OPT_TRY(dalloc(&w.g, (size_t)n_cols));
    OPT_TRY(dalloc(&w.g_shift, 1));
    OPT_TRY(dalloc(&w.max_r, (size_t)2 * S));
    OPT_TRY(dalloc(&w.dose_tr, (size_t)S * n_tr));
    OPT_TRY(dalloc(&w.fsum, (size_t)2 * S));
    OPT_TRY(dalloc(&w.m, (size_t)n_cols));
    OPT_TRY(dalloc(&w.v, (size_t)n_cols));
    OPT_TRY(dalloc(&w.hist, (size_t)std::max(spec.iterations, 1)));
    OPT_TRY(cudaMemsetAsync(w.g, 0, sizeof(unsigned long long) * n_cols, st));
    OPT_TRY(cudaMemsetAsync(w.max_r, 0, sizeof(unsigned) * 2 * S, st));
    OPT_TRY(cudaMemsetAsync(w.fsum, 0, sizeof(double) * 2 * S, st));
    OPT_TRY(cudaMemsetAsync(w.m, 0, sizeof(float) * n_cols, st));
    OPT_TRY(cudaMemsetAsync(w.v, 0, sizeof(float) * n_cols, st));
    const int smem = (int)(sizeof(unsigned long long) * n_cols);
    OPT_TRY(cudaFuncSetAttribute(k_bwd_fixed, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int dev = 0, nsm = 0;
    OPT_TRY(cudaGetDevice(&dev));
    OPT_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    OPT_TRY(cudaEventRecord(ev[1], st));
    const ObjParams q{spec.dp, spec.w_u, spec.w_o, spec.w_r, spec.over, spec.ring,
                      1.0f / (float)std::max<long long>(spec.n_target, 1),
                      1.0f / (float)std::max<long long>(spec.n_ring, 1)};
    const dim3 gf((unsigned)std::max((n_tr + 7) / 8, 1), (unsigned)S);
    for (int it = 0; it < spec.iterations; ++it) {
        const int cu = it & 1, nx = (it + 1) & 1;
        k_fwd<<<gf, 256, 0, st>>>(w.crp, w.ccol, w.cval, n_tr, x, w.tr_cls, q, w.dose_tr, w.fsum + cu * S,
                                  w.max_r + cu * S);
        k_bwd_fixed<<<(unsigned)nsm, 1024, smem, st>>>(w.crp, per_row, w.ccol, w.cval, n_tr, n_cols, w.dose_tr,
                                                       w.tr_cls, q,
                                                       w.fsum + cu * S, w.max_r + cu * S, w.fsum + nx * S,
                                                       w.max_r + nx * S, w.max_abs, w.count_bound, S, w.hist, it, w.g,
                                                       w.g_shift);
        const double t = it + 1;
        k_adam_fixed<<<(unsigned)((n_cols + 255) / 256), 256, 0, st>>>(
            w.g, w.g_shift, n_cols, x, w.m, w.v, spec.step, (float)(1.0 / (1.0 - std::pow(0.9, t))),
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
