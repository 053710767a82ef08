// Robust spot-weight optimisation over the scenarios' influence matrices
// (Sec. 2.E: robust optimisation over 13 scenarios against the target
// constraints of Table 3).  The paper's optimiser is an in-house
// trial-and-error procedure; the objective here is a worst case over the
// scenarios of quadratic target under- and overdose and ring-overdose
// penalties, minimised by Adam with non-negative weights.
//
// One iteration, all on the device (no host synchronisation):
//   k_spmv_obj   d_s = A_s x for every scenario s (sub-warp per row, CSR) and
//                the scenario's objective f_s (block sums, FP64 atomics);
//   k_select     s* = first s with the largest f_s; records the worst case;
//   k_spmvT      g = A_s*^T f'(d_s*): each block accumulates its rows'
//                contributions per spot in shared memory (FP64), then adds
//                them to g with one atomic per spot;
//   k_adam_proj  Adam step on x, clamped at zero; clears g.
// Every kernel streams the matrices once per use: the iteration is bound by
// HBM (13 SpMV + 1 transposed SpMV over ~0.35 GB of CSR each).
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

__global__ void k_select(const double* __restrict__ fsum, int n_scen, int* __restrict__ worst,
                         float* __restrict__ hist, int it)
{
    int s = 0;
    for (int k = 1; k < n_scen; ++k)
        if (fsum[k] > fsum[s]) s = k;
    *worst = s;
    if (hist) hist[it] = (float)fsum[s];
}

// g += A_s*^T f'(d_s*): shared-memory FP64 accumulation per spot, then one
// global atomic per spot and block.
__global__ void k_spmvT(const Csr* __restrict__ mats, long long n_rows, int n_cols, const int* __restrict__ worst,
                        const float* __restrict__ dose, const unsigned char* __restrict__ cls, ObjParams q,
                        double* __restrict__ g)
{
    extern __shared__ double gs[];
    for (int j = threadIdx.x; j < n_cols; j += blockDim.x) gs[j] = 0.0;
    __syncthreads();
    const int s = *worst;
    const Csr A = mats[s];
    const float* d = dose + (long long)s * n_rows;
    const int sub = threadIdx.x & (kLanesPerRow - 1);
    const long long groups = (long long)gridDim.x * (blockDim.x / kLanesPerRow);
    for (long long row = (long long)blockIdx.x * (blockDim.x / kLanesPerRow) + threadIdx.x / kLanesPerRow;
         row < n_rows; row += groups) {
        const unsigned char c = __ldg(cls + row);
        if (c != 1 && c != 2) continue;
        const float r = obj_grad(__ldg(d + row), c, q);
        if (r == 0.0f) continue;
        const long long b = __ldg(A.row_ptr + row), e = __ldg(A.row_ptr + row + 1);
        for (long long k = b + sub; k < e; k += kLanesPerRow) {
            const int j = __ldg(A.col + k);
            if ((unsigned)j < (unsigned)n_cols) atomicAdd(gs + j, (double)(__ldg(A.val + k) * r));
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < n_cols; j += blockDim.x)
        if (gs[j] != 0.0) atomicAdd(g + j, gs[j]);
}

// Adam (Kingma & Ba 2015) with the weights clamped at zero; clears g.
__global__ void k_adam_proj(float* __restrict__ x, double* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float step, float c1, float c2, float eps)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const float gj = (float)g[j];
    g[j] = 0.0;
    const float mj = fmaf(0.9f, m[j], 0.1f * gj), vj = fmaf(0.999f, v[j], 0.001f * gj * gj);
    m[j] = mj;
    v[j] = vj;
    x[j] = fmaxf(x[j] - step * (mj * c1) / (sqrtf(vj * c2) + eps), 0.0f);
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

}  // namespace

// ---------------------------------------------------------------------------
// Host side (called from api.cu).
// ---------------------------------------------------------------------------
struct OptWorkspace {
    Csr* mats = nullptr;
    float* dose = nullptr;          // [S x n_rows]
    double* fsum = nullptr;         // [S]
    int* worst = nullptr;
    double* g = nullptr;            // [n_cols]
    float* m = nullptr;
    float* v = nullptr;
    float* hist = nullptr;
    unsigned long long* counts = nullptr;
    int* minmax = nullptr;
};

static void free_ws(OptWorkspace& w)
{
    cudaFree(w.mats); cudaFree(w.dose); cudaFree(w.fsum); cudaFree(w.worst); cudaFree(w.g);
    cudaFree(w.m); cudaFree(w.v); cudaFree(w.hist); cudaFree(w.counts); cudaFree(w.minmax);
    w = OptWorkspace{};
}

static cudaError_t alloc_ws(OptWorkspace& w, const long long* const* rp, const int* const* col,
                            const float* const* val, int n_scen, long long n_rows, int n_cols, int iterations)
{
    std::vector<Csr> h(n_scen);
    for (int s = 0; s < n_scen; ++s) h[s] = Csr{rp[s], col[s], val[s]};
    cudaError_t e;
    if ((e = cudaMalloc(&w.mats, sizeof(Csr) * n_scen)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(w.mats, h.data(), sizeof(Csr) * n_scen, cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&w.dose, sizeof(float) * n_scen * n_rows)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&w.fsum, sizeof(double) * n_scen)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&w.worst, sizeof(int))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&w.g, sizeof(double) * std::max(n_cols, 1))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&w.m, sizeof(float) * std::max(n_cols, 1))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&w.v, sizeof(float) * std::max(n_cols, 1))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&w.hist, sizeof(float) * std::max(iterations, 1))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&w.counts, sizeof(unsigned long long) * 3 * n_scen)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&w.minmax, sizeof(int) * 2 * n_scen)) != cudaSuccess) return e;
    return cudaSuccess;
}

size_t opt_spmvT_smem(int n_cols) { return sizeof(double) * (size_t)n_cols; }

cudaError_t run_robust_optimize(const long long* const* rp, const int* const* col, const float* const* val, int n_scen,
                                long long n_rows, int n_cols, const unsigned char* cls, const OptSpec& spec, float* x,
                                float* hist_host, cudaStream_t st, int num_sms, float* ms_out)
{
    OptWorkspace w;
    cudaError_t e = alloc_ws(w, rp, col, val, n_scen, n_rows, n_cols, spec.iterations);
    auto done = [&](cudaError_t r) { free_ws(w); return r; };
    if (e != cudaSuccess) return done(e);
    ObjParams q{spec.dp, spec.w_u, spec.w_o, spec.w_r, spec.over, spec.ring,
                1.0f / (float)std::max<long long>(spec.n_target, 1), 1.0f / (float)std::max<long long>(spec.n_ring, 1)};
    const size_t smem = opt_spmvT_smem(n_cols);
    if ((e = cudaFuncSetAttribute(k_spmvT, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return done(e);
    if ((e = cudaMemsetAsync(w.g, 0, sizeof(double) * n_cols, st)) != cudaSuccess) return done(e);
    if ((e = cudaMemsetAsync(w.m, 0, sizeof(float) * n_cols, st)) != cudaSuccess) return done(e);
    if ((e = cudaMemsetAsync(w.v, 0, sizeof(float) * n_cols, st)) != cudaSuccess) return done(e);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
    const dim3 gs((unsigned)(num_sms * 8), (unsigned)n_scen);
    for (int it = 0; it < spec.iterations; ++it) {
        cudaMemsetAsync(w.fsum, 0, sizeof(double) * n_scen, st);
        k_spmv_obj<<<gs, 256, 0, st>>>(w.mats, n_rows, n_cols, x, cls, q, w.dose, w.fsum);
        k_select<<<1, 1, 0, st>>>(w.fsum, n_scen, w.worst, w.hist, it);
        k_spmvT<<<num_sms * 2, 512, smem, st>>>(w.mats, n_rows, n_cols, w.worst, w.dose, cls, q, w.g);
        const double t = it + 1;
        k_adam_proj<<<(n_cols + 255) / 256, 256, 0, st>>>(x, w.g, w.m, w.v, n_cols, spec.step,
                                                         (float)(1.0 / (1.0 - std::pow(0.9, t))),
                                                         (float)(1.0 / (1.0 - std::pow(0.999, t))), spec.eps);
    }
    cudaEventRecord(e1, st);
    if ((e = cudaGetLastError()) != cudaSuccess) return done(e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return done(e);
    if (ms_out) cudaEventElapsedTime(ms_out, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (hist_host && spec.iterations > 0)
        e = cudaMemcpy(hist_host, w.hist, sizeof(float) * spec.iterations, cudaMemcpyDeviceToHost);
    return done(e);
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
    cudaError_t e = alloc_ws(w, rp, col, val, n_scen, n_rows, 1, 1);
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
