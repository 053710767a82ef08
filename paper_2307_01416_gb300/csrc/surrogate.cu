// Learned aperture surrogate on the fifth-generation tensor cores (sm_103a).
//
// The network (6 -> 128 -> 128 -> 45, ReLU) maps a proton entering the brass
// block near the opening to a transmission logit and a 4-component diagonal
// Gaussian mixture over its state on the block's exit plane.  It is not part
// of the paper.  It replaces the in-brass stepping of the aperture module
// (Sec. 2.B), which the paper reads from pre-computed brass transport data.
//
// Every layer is one 128-row tile GEMM D[128 x N] (+)= A[128 x K] B[N x K]^T:
// BF16 operands in shared memory in the canonical no-swizzle K-major layout
// (8 x 8 core matrices of 128 contiguous bytes), FP32 accumulators in tensor
// memory, issued by one thread with tcgen05.mma and completed through an
// mbarrier; the epilogues read the accumulators back with tcgen05.ld, one
// thread per row.  Training keeps the whole forward and backward of a tile in
// one CTA: the weight gradients accumulate in tensor memory over the CTA's
// tiles and the bias gradients ride along as an extra all-ones operand row.
#include <algorithm>
#include <cmath>

#include <cuda_bf16.h>

#include "device_common.cuh"
#include "vpmc_internal.cuh"

namespace vpmc {
namespace {

using namespace dev;
using namespace sur;

constexpr int kRows = 128;                // rows (tracks) per tile, one thread each
constexpr int kWaitLimit = 1 << 22;       // mbarrier polls before a wait is declared failed

// Byte offset of element (r, k) of an R x K operand in the no-swizzle
// K-major layout: core matrix (r / 8, k / 8) of 8 rows x 16 bytes.
__host__ __device__ constexpr int kmaj(int r, int k, int K)
{
    return ((((r >> 3) * (K >> 3)) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1);
}

// ---- tensor-core, tensor-memory and mbarrier primitives (inline PTX) ----
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading-dimension byte
// offset (next core matrix along K), stride byte offset (next 8-row group),
// descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        :: "r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void umma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t mbar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Bounded wait for the completion of the mbarrier phase with the given parity.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity)
{
    for (int i = 0; i < kWaitLimit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tmem_alloc(uint32_t slot_saddr, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(slot_saddr), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(ncols) : "memory");
}

// 16 consecutive FP32 columns of this thread's tensor-memory lane, waited for.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
        "[%16];\n\ttcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 consecutive FP32 columns of this thread's tensor-memory lane, waited for.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);   // a in the low half (lower address)
    return *reinterpret_cast<uint32_t*>(&h);
}

__device__ __forceinline__ unsigned short bf16_bits(float a) { return __bfloat16_as_ushort(__float2bfloat16_rn(a)); }

// D[128 x N] (+)= A[128 x K] B[N x K]^T from K-major shared-memory operands.
__device__ __forceinline__ void mma_tile(uint32_t d_tmem, uint32_t a_saddr, uint32_t b_saddr, int K, int N,
                                         bool accumulate)
{
    const uint32_t idesc = idesc_bf16(kRows, N);
    const uint32_t sbo = (uint32_t)(K >> 3) << 7;
    for (int kc = 0; kc < (K >> 4); ++kc) {
        const uint64_t a = sdesc(a_saddr + (uint32_t)kc * 256u, 128u, sbo);
        const uint64_t b = sdesc(b_saddr + (uint32_t)kc * 256u, 128u, sbo);
        umma(d_tmem, a, b, idesc, (accumulate || kc > 0) ? 1u : 0u);
    }
}

// Make this thread's generic-proxy shared-memory writes and tensor-memory
// reads visible to the next tensor-core operation, then synchronise.
__device__ __forceinline__ void publish()
{
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
}

// Wait (all threads) for the tensor-core work committed to mbar; the CTA
// agrees on the outcome.
__device__ __forceinline__ bool complete(uint32_t mbar, uint32_t& phase)
{
    const bool ok = mbar_wait(mbar, phase);
    phase ^= 1u;
    const bool all = __syncthreads_and(ok) != 0;
    tc_fence_after();
    return all;
}

// Barrier of one 128-thread warpgroup (named barrier 1 + g): the forward
// kernels run one tile pipeline per warpgroup, so their steps synchronise
// the group, not the CTA.
__device__ __forceinline__ void group_sync(int g)
{
    asm volatile("bar.sync %0, %1;" :: "r"(1 + g), "r"(kRows) : "memory");
}

// The same barrier, returning whether every thread of the group passed ok.
__device__ __forceinline__ bool group_sync_and(int g, bool ok)
{
    uint32_t all;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, %2, %3, p;\n\tselp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(all) : "r"(ok ? 1u : 0u), "r"(1 + g), "r"(kRows) : "memory");
    return all != 0u;
}

// publish / complete for one warpgroup's tile pipeline.
__device__ __forceinline__ void publish_group(int g)
{
    fence_async_smem();
    tc_fence_before();
    group_sync(g);
}

__device__ __forceinline__ bool complete_group(int g, uint32_t mbar, uint32_t& phase)
{
    const bool ok = mbar_wait(mbar, phase);
    phase ^= 1u;
    const bool all = group_sync_and(g, ok);
    tc_fence_after();
    return all;
}

__device__ __forceinline__ void copy_to_smem(unsigned char* dst, const unsigned char* src, int bytes)
{
    const uint4* s = reinterpret_cast<const uint4*>(src);
    uint4* d = reinterpret_cast<uint4*>(dst);
    for (int i = threadIdx.x; i < (bytes >> 4); i += blockDim.x) d[i] = __ldg(s + i);
}

__device__ __forceinline__ void zero_smem(unsigned char* dst, int bytes)
{
    uint4* d = reinterpret_cast<uint4*>(dst);
    for (int i = threadIdx.x; i < (bytes >> 4); i += blockDim.x) d[i] = make_uint4(0u, 0u, 0u, 0u);
}

// Row r of a [128 x 16] input tile: the 6 features, then zeros.
__device__ __forceinline__ void store_input_row(unsigned char* X, int r, const float f[6])
{
    uint4 lo = make_uint4(pack_bf16(f[0], f[1]), pack_bf16(f[2], f[3]), pack_bf16(f[4], f[5]), 0u);
    *reinterpret_cast<uint4*>(X + kmaj(r, 0, kInPad)) = lo;
    *reinterpret_cast<uint4*>(X + kmaj(r, 8, kInPad)) = make_uint4(0u, 0u, 0u, 0u);
}

// 16 consecutive FP32 columns of this thread's tensor-memory lane, issued and
// not waited for: the registers are valid after tmem_wait16 on them.
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
        "[%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}

// Wait for this thread's outstanding tensor-memory loads; the registers pass
// through the wait so that no use of them moves above it.
__device__ __forceinline__ void tmem_wait16(uint32_t (&r)[16])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
}

// relu(D + b) of 16 columns [c0, c0 + 16) of row r, rounded to BF16 into the
// K-major [128 x 128] tile dst.
__device__ __forceinline__ void relu_pack16(const uint32_t (&v)[16], const float* __restrict__ bias, int c0,
                                            unsigned char* dst, int r)
{
    uint32_t w[8];
#pragma unroll
    for (int j = 0; j < 16; j += 2) {
        const float a0 = __uint_as_float(v[j]) + __ldg(bias + c0 + j);
        const float a1 = __uint_as_float(v[j + 1]) + __ldg(bias + c0 + j + 1);
        w[j >> 1] = pack_bf16(fmaxf(a0, 0.0f), fmaxf(a1, 0.0f));
    }
    *reinterpret_cast<uint4*>(dst + kmaj(r, c0, kH)) = make_uint4(w[0], w[1], w[2], w[3]);
    *reinterpret_cast<uint4*>(dst + kmaj(r, c0 + 8, kH)) = make_uint4(w[4], w[5], w[6], w[7]);
}

// Calls f(v, c) for the ncols (a multiple of 32) FP32 columns of this
// thread's tensor-memory lane from t_row, 16 at a time: the load of the next
// 16 is in flight while f works on the current ones, so one load round trip
// is exposed per call, not one per chunk.
template <class F>
__device__ __forceinline__ void tmem_cols_pipelined(uint32_t t_row, int ncols, F&& f)
{
    uint32_t a[16], b[16];
    tmem_ld16_async(t_row, a);
    tmem_wait16(a);
#pragma unroll
    for (int c0 = 0; c0 < ncols; c0 += 32) {
        tmem_ld16_async(t_row + (uint32_t)(c0 + 16), b);
        f(a, c0);
        tmem_wait16(b);
        if (c0 + 32 < ncols) tmem_ld16_async(t_row + (uint32_t)(c0 + 32), a);
        f(b, c0 + 16);
        if (c0 + 32 < ncols) tmem_wait16(a);
    }
}

// Hidden-layer epilogue of the forward path: relu(D + b) to BF16 into the
// K-major [128 x 128] tile dst.
__device__ __forceinline__ void hidden_epilogue_fwd(uint32_t t_row, const float* __restrict__ bias,
                                                    unsigned char* dst, int r)
{
    tmem_cols_pipelined(t_row, kH, [&](const uint32_t (&v)[16], int c0) { relu_pack16(v, bias, c0, dst, r); });
}

// Hidden-layer epilogue of training: relu(D + b) to BF16 into the K-major
// tile dst and its transposed copy dstT (rows = units, K = tile rows), and the
// ReLU mask (bit c of mask[c / 32]: D + b > 0; the caller zeroes mask).
__device__ __forceinline__ void hidden_epilogue_train(uint32_t t_row, const float* __restrict__ bias,
                                                      unsigned char* dst, unsigned char* dstT, int r,
                                                      uint32_t (&mask)[4])
{
    tmem_cols_pipelined(t_row, kH, [&](const uint32_t (&v)[16], int c0) {
        uint32_t w[8];
        uint32_t mbits = 0u;
#pragma unroll
        for (int j = 0; j < 16; j += 2) {
            const float a0 = __uint_as_float(v[j]) + __ldg(bias + c0 + j);
            const float a1 = __uint_as_float(v[j + 1]) + __ldg(bias + c0 + j + 1);
            mbits |= (a0 > 0.0f ? 1u : 0u) << j;
            mbits |= (a1 > 0.0f ? 1u : 0u) << (j + 1);
            w[j >> 1] = pack_bf16(fmaxf(a0, 0.0f), fmaxf(a1, 0.0f));
            *reinterpret_cast<unsigned short*>(dstT + kmaj(c0 + j, r, kRows)) = (unsigned short)(w[j >> 1] & 0xFFFFu);
            *reinterpret_cast<unsigned short*>(dstT + kmaj(c0 + j + 1, r, kRows)) = (unsigned short)(w[j >> 1] >> 16);
        }
        *reinterpret_cast<uint4*>(dst + kmaj(r, c0, kH)) = make_uint4(w[0], w[1], w[2], w[3]);
        *reinterpret_cast<uint4*>(dst + kmaj(r, c0 + 8, kH)) = make_uint4(w[4], w[5], w[6], w[7]);
        mask[c0 >> 5] |= mbits << (c0 & 31);
    });
}

// z = D3 + b3 for row r (48 columns, 45 used).
__device__ __forceinline__ void output_epilogue(uint32_t t_d3, const float* __restrict__ b3, float (&z)[kOutPad])
{
    float v[32], u[16];
    tmem_ld32(t_d3, v);
    tmem_ld16(t_d3 + 32u, u);
#pragma unroll
    for (int j = 0; j < 32; ++j) z[j] = v[j] + __ldg(b3 + j);
#pragma unroll
    for (int j = 0; j < 16; ++j) z[32 + j] = u[j] + (32 + j < kOut ? __ldg(b3 + 32 + j) : 0.0f);
}

// ============================================================================
// Forward: network outputs of n feature rows, and the same network drawing
// exit states for the transport's queries.
// ============================================================================
// A CTA runs kGroups tile pipelines, one per 128-thread warpgroup, sharing
// one copy of the weight images: while one group's epilogue runs on the CUDA
// cores, another group's GEMMs run on the tensor core.  Per group: its input,
// hidden and staging tiles, its queries and its mbarrier; in tensor memory,
// 128 columns (D1, then D2 over it once D1 is read, then D3).
constexpr int kGroups = 3;
constexpr int kFwdThreads = kGroups * kRows;
struct FwdSmem {
    static constexpr int W = 0;                                   // W1, W2, W3 images
    static constexpr int G0 = kImgW2T;                            // the groups' regions
    // offsets within a group's region
    static constexpr int X = 0;                                   // [128 x 16]
    static constexpr int H = X + kRows * kInPad * 2;              // [128 x 128]; also the output staging
    static constexpr int XS = H + kRows * kH * 2;                 // FP32 inputs of a tile, [128 x 6]
    static constexpr int QS = XS + kRows * kIn * 4;               // a tile's queries (inference)
    static constexpr int Bar = QS + kRows * (int)sizeof(SurQuery);
    static constexpr int GBytes = (Bar + 8 + 127) / 128 * 128;
    static constexpr int Slot = G0 + kGroups * GBytes;
    static constexpr int Bytes = Slot + 8;
};
static_assert(FwdSmem::Bytes <= 232448, "forward CTA exceeds the shared memory of one SM");
static_assert(FwdSmem::G0 % 128 == 0 && FwdSmem::GBytes % 128 == 0, "operand tiles 128-byte aligned");
constexpr uint32_t kFwdCols = 512;        // allocation (a power of two); group g uses columns [128 g, 128 g + 128)

// The three GEMMs of one tile whose inputs are in the group's X; returns
// false when a tensor-core wait failed.  On return the group's accumulator
// columns hold z - b3.
__device__ __forceinline__ bool forward_tile(unsigned char* sm, unsigned char* gs, uint32_t tcol, uint32_t t_row,
                                             const SurNet& net, uint32_t bar, uint32_t& phase, int r, int g)
{
    const uint32_t s0 = smem_addr(sm), gs0 = smem_addr(gs);
    publish_group(g);
    if (r == 0) {
        tc_fence_after();
        mma_tile(tcol, gs0 + FwdSmem::X, s0 + FwdSmem::W + kImgW1, kInPad, kH, false);
        umma_commit(bar);
    }
    if (!complete_group(g, bar, phase)) return false;
    hidden_epilogue_fwd(t_row, net.params + ob1, gs + FwdSmem::H, r);
    publish_group(g);
    if (r == 0) {
        tc_fence_after();
        mma_tile(tcol, gs0 + FwdSmem::H, s0 + FwdSmem::W + kImgW2, kH, kH, false);
        umma_commit(bar);
    }
    if (!complete_group(g, bar, phase)) return false;
    hidden_epilogue_fwd(t_row, net.params + ob2, gs + FwdSmem::H, r);
    publish_group(g);
    if (r == 0) {
        tc_fence_after();
        mma_tile(tcol, gs0 + FwdSmem::H, s0 + FwdSmem::W + kImgW3, kH, kOutPad, false);
        umma_commit(bar);
    }
    return complete_group(g, bar, phase);
}

__device__ __forceinline__ void fwd_prologue(unsigned char* sm, const SurNet& net, uint32_t& tbase)
{
    copy_to_smem(sm + FwdSmem::W, net.img, kImgW2T);
    if (threadIdx.x < kGroups) mbar_init(smem_addr(sm + FwdSmem::G0 + threadIdx.x * FwdSmem::GBytes + FwdSmem::Bar));
    if ((threadIdx.x >> 5) == 0) tmem_alloc(smem_addr(sm + FwdSmem::Slot), kFwdCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    tbase = *reinterpret_cast<volatile uint32_t*>(sm + FwdSmem::Slot);
}

__device__ __forceinline__ void fwd_epilogue_free(unsigned char* sm, uint32_t tbase, uint32_t bar, uint32_t phase,
                                                  bool ok, const SurNet& net)
{
    if (!ok) {
        // a wait failed: latch the error and give the tensor core a last
        // bounded chance to finish this group's work before the memory is
        // released
        if ((threadIdx.x & (kRows - 1)) == 0) atomicOr(net.status, 1);
        (void)mbar_wait(bar, phase);
    }
    tc_fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        tc_fence_after();
        tmem_dealloc(tbase, kFwdCols);
    }
}

__global__ void __launch_bounds__(kFwdThreads, 1) k_sur_forward(const SurNet net, const float* __restrict__ x,
                                                                 long long n, float* __restrict__ z)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    uint32_t tbase;
    fwd_prologue(sm, net, tbase);
    const int g = threadIdx.x / kRows, r = threadIdx.x % kRows;
    unsigned char* gs = sm + FwdSmem::G0 + g * FwdSmem::GBytes;
    const uint32_t tcol = tbase + (uint32_t)(g * kRows);
    const uint32_t t_row = tcol + ((uint32_t)((r >> 5) * 32) << 16);
    const uint32_t bar = smem_addr(gs + FwdSmem::Bar);
    uint32_t phase = 0u;
    bool ok = true;
    float* xs = reinterpret_cast<float*>(gs + FwdSmem::XS);
    float* zs = reinterpret_cast<float*>(gs + FwdSmem::H);
    for (long long tile = (long long)blockIdx.x * kGroups + g; tile * kRows < n && ok;
         tile += (long long)gridDim.x * kGroups) {
        const long long row0 = tile * kRows;
        const int rows = (int)min((long long)kRows, n - row0);
        // the tile's inputs, rows x 6 contiguous floats: coalesced 16-byte loads
        // (row0 * 24 bytes is a multiple of 16 when row0 is a multiple of 128)
        const float4* xg = reinterpret_cast<const float4*>(x + kIn * row0);
        const int nx = rows * kIn;
        for (int i = r; i < (nx >> 2); i += kRows) reinterpret_cast<float4*>(xs)[i] = __ldg(xg + i);
        for (int i = (nx & ~3) + r; i < nx; i += kRows) xs[i] = __ldg(x + kIn * row0 + i);
        group_sync(g);
        float f[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        if (r < rows) {
#pragma unroll
            for (int k = 0; k < 6; ++k) f[k] = xs[kIn * r + k];
        }
        store_input_row(gs + FwdSmem::X, r, f);
        ok = forward_tile(sm, gs, tcol, t_row, net, bar, phase, r, g);
        if (!ok) break;
        float zz[kOutPad];
        output_epilogue(t_row, net.params + ob3, zz);
        // outputs through shared memory (h2 is consumed): rows x 45 contiguous
        // floats leave with coalesced 16-byte stores (row0 * 180 bytes is a
        // multiple of 16)
#pragma unroll
        for (int j = 0; j < kOut; ++j) zs[kOut * r + j] = zz[j];
        group_sync(g);
        float4* zg = reinterpret_cast<float4*>(z + kOut * row0);
        const int nz = rows * kOut;
        for (int i = r; i < (nz >> 2); i += kRows) zg[i] = reinterpret_cast<const float4*>(zs)[i];
        for (int i = (nz & ~3) + r; i < nz; i += kRows) z[kOut * row0 + i] = zs[i];
        tc_fence_before();
        group_sync(g);
    }
    fwd_epilogue_free(sm, tbase, bar, phase, ok, net);
}

// Draw of one query from the network output z (see the sampler in the oracle):
// transmitted = u0 < sigmoid(z0); component = first c with u1 < sum pi;
// y_j = mu_cj + exp(clamp(s_cj)) xi_j with xi from three Box-Muller pairs.
__device__ __forceinline__ bool sample_exit(const float (&z)[kOutPad], uint4 ua, uint4 ub, float (&y)[kDY])
{
    const float p = 1.0f / (1.0f + expf(-z[0]));
    const bool trans = u01(ua.x) < p;
    float amax = fmaxf(fmaxf(z[1], z[2]), fmaxf(z[3], z[4]));
    float e[kNComp], sum = 0.0f;
#pragma unroll
    for (int c = 0; c < kNComp; ++c) { e[c] = expf(z[1 + c] - amax); sum += e[c]; }
    const float u1 = u01(ua.y);
    int comp = kNComp - 1;
    float cum = 0.0f;
#pragma unroll
    for (int c = 0; c < kNComp; ++c) {
        cum += e[c] / sum;
        if (comp == kNComp - 1 && c < kNComp - 1 && u1 < cum) comp = c;
    }
    // the loop above takes the first c with u1 < cum_c; the last component otherwise
    const float2 x01 = box_muller(u01(ua.z), u01(ua.w));
    const float2 x23 = box_muller(u01(ub.x), u01(ub.y));
    const float2 x45 = box_muller(u01(ub.z), u01(ub.w));
    const float xi[kDY] = {x01.x, x01.y, x23.x, x23.y, x45.x};
#pragma unroll
    for (int j = 0; j < kDY; ++j) {
        float mu = 0.0f, s = 0.0f;
#pragma unroll
        for (int c = 0; c < kNComp; ++c) {
            if (c == comp) { mu = z[5 + 5 * c + j]; s = z[25 + 5 * c + j]; }
        }
        y[j] = fmaf(expf(fminf(fmaxf(s, kSMin), kSMax)), xi[j], mu);
    }
    return trans;
}

__global__ void __launch_bounds__(kFwdThreads, 1) k_sur_infer(const SurNet net, const TransportParams P)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    uint32_t tbase;
    fwd_prologue(sm, net, tbase);
    const int g = threadIdx.x / kRows, r = threadIdx.x % kRows;
    const int lane = r & 31;
    unsigned char* gs = sm + FwdSmem::G0 + g * FwdSmem::GBytes;
    const uint32_t tcol = tbase + (uint32_t)(g * kRows);
    const uint32_t t_row = tcol + ((uint32_t)((r >> 5) * 32) << 16);
    const uint32_t bar = smem_addr(gs + FwdSmem::Bar);
    uint32_t phase = 0u;
    bool ok = true;
    const long long nq = min((long long)*P.sq_count, P.sq_cap);
    unsigned long long acc_ap = 0ull;
    SurQuery* qs = reinterpret_cast<SurQuery*>(gs + FwdSmem::QS);
    static_assert(sizeof(SurQuery) % 16 == 0, "query records are copied in 16-byte pieces");
    for (long long tile = (long long)blockIdx.x * kGroups + g; tile * kRows < nq && ok;
         tile += (long long)gridDim.x * kGroups) {
        const long long row = tile * kRows + r;
        const int rows = (int)min((long long)kRows, nq - tile * kRows);
        // the tile's query records, contiguous: coalesced 16-byte loads
        {
            const uint4* src = reinterpret_cast<const uint4*>(P.sq + tile * kRows);
            uint4* dst = reinterpret_cast<uint4*>(qs);
            const int n16 = rows * (int)(sizeof(SurQuery) / 16);
            for (int i = r; i < n16; i += kRows) dst[i] = src[i];
        }
        group_sync(g);
        float f[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        if (r < rows) {
#pragma unroll
            for (int k = 0; k < 6; ++k) f[k] = qs[r].x[k];
        }
        store_input_row(gs + FwdSmem::X, r, f);
        ok = forward_tile(sm, gs, tcol, t_row, net, bar, phase, r, g);
        if (!ok) break;
        float zz[kOutPad];
        output_epilogue(t_row, net.params + ob3, zz);
        tc_fence_before();
        group_sync(g);

        bool emit = false;
        PhaseRec rec;
        float pb[3] = {0.0f, 0.0f, 0.0f};       // exit point, BEV frame
        int scen0 = 0;
        const DevBeam* Bp = P.beams;
        if (row < nq) {
            const SurQuery q = qs[r];
            const DevItem& I = P.items[q.item];
            const DevBeam& B = P.beams[I.beam];
            const uint32_t hist = (uint32_t)(q.g - I.hist_off);
            const uint2 key = make_uint2(P.key0, P.key1_hi ^ (uint32_t)I.spot);
            const uint4 ua = philox(make_uint4(hist, q.step, 4u, 0u), key);
            const uint4 ub = philox(make_uint4(hist, q.step, 5u, 0u), key);
            float y[kDY];
            const bool trans = sample_exit(zz, ua, ub, y);
            if (P.track_mode) {
                if (q.g < P.total) {
                    P.trk_label[q.g] = trans ? 1 : 0;
#pragma unroll
                    for (int j = 0; j < kDY; ++j) P.trk_y[5 * q.g + j] = trans ? y[j] : 0.0f;
                }
            } else {
                const float T = B.ap_tdn - B.ap_tup;
                const float un = q.dx * q.nx + q.dy * q.ny, ut = q.dy * q.nx - q.dx * q.ny;
                const float E1 = q.E * (1.0f - 0.2f * y[0]);
                const float dn = y[1] + T * un / q.dz, dt = y[2] + T * ut / q.dz;
                float vn = fmaf(kDirScale, y[3], un), vt = fmaf(kDirScale, y[4], ut);
                const float r2 = vn * vn + vt * vt;
                if (r2 > 0.75f) {
                    const float sc = sqrtf(0.75f / r2);
                    vn *= sc;
                    vt *= sc;
                }
                if (trans && E1 > kEcut && E1 <= q.E && isfinite(dn + dt + vn + vt)) {
                    scen0 = I.scen;
                    Bp = &B;
                    pb[0] = q.px + dn * q.nx - dt * q.ny;
                    pb[1] = q.py + dn * q.ny + dt * q.nx;
                    pb[2] = B.ap_tdn;
                    const float db[3] = {vn * q.nx - vt * q.ny, vn * q.ny + vt * q.nx, sqrtf(1.0f - vn * vn - vt * vt)};
#pragma unroll
                    for (int k = 0; k < 3; ++k) rec.d[k] = db[0] * B.u[k] + db[1] * B.v[k] + db[2] * B.w[k];
                    rec.E = E1;
                    if (P.nuclear) {
                        const uint4 un6 = philox(make_uint4(hist, q.step, 6u, 0u), key);
                        rec.nlam = -logf(u01(un6.x));
                    } else {
                        rec.nlam = __int_as_float(0x7f800000);
                    }
                    rec.step = q.step + 1u;
                    rec.item = q.item;
                    rec.g = q.g;
                    emit = true;
                    acc_ap += __float2ull_rn((q.E - E1) * P.fscale) * (unsigned long long)P.n_rep;
                } else {
                    acc_ap += __float2ull_rn(q.E * P.fscale) * (unsigned long long)P.n_rep;
                    if (P.records && q.g < P.rec_cap) {
                        HistRecord hr;
                        hr.q_dep = 0;
                        hr.fate = kAbsAp;
                        hr.steps = (int)q.step;
                        hr.e_dep = 0.0f;
                        hr.e_end = 0.0f;
                        const float pe[3] = {q.px, q.py, B.ap_tup};
                        bev_to_patient(B, P.scens[I.scen], pe, hr.pos);
                        hr.pad = 0.0f;
                        P.records[q.g] = hr;
                    }
                }
            }
        }
        // hand-off into the slot the beam-line kernel reserved for this proton;
        // an absorbed proton leaves the slot empty (item -1)
        if (row < nq && !P.track_mode) {
            const long long slot = qs[r].slot;
            if (slot >= 0 && slot < P.rep_cap) {
                if (!emit) {
                    rec = PhaseRec{};
                    rec.item = -1;
                }
                // one copy per scenario sharing the beam-line transport
                const int item0 = rec.item;
                const long long g0 = rec.g;
                for (int s = 0; s < P.n_rep; ++s) {
                    if (emit) {
                        bev_to_patient(*Bp, P.scens[scen0 + s], pb, rec.p);
                        rec.item = item0 + s * P.rep_items;
                        rec.g = g0 + s * P.rep_hist;
                    }
                    P.phase[s * P.rep_cap + slot] = rec;
                }
            } else {
                atomicOr(P.status, 2);
            }
        }
        group_sync(g);                              // qs is refilled by the next tile
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) acc_ap += __shfl_xor_sync(kFull, acc_ap, o);
    if (lane == 0 && acc_ap) atomicAdd(P.stats + kStAp, acc_ap);
    fwd_epilogue_free(sm, tbase, bar, phase, ok, net);
}

// ============================================================================
// Training: forward, loss, backward and weight-gradient accumulation of the
// CTA's tiles in one kernel.
// ============================================================================
struct TrainSmem {
    static constexpr int Img = 0;                                  // all five weight images
    static constexpr int X = kImgBytes;                            // [128 x 16]
    static constexpr int XT = X + kRows * kInPad * 2;              // [16 x 128]: features, row 6 = ones
    static constexpr int A = XT + kInPad * kRows * 2;              // [128 x 128]: h1, h2, then da2
    static constexpr int Bt = A + kRows * kH * 2;                  // [144 x 128]: h1^T, row 128 = ones
    static constexpr int C = Bt + 144 * kRows * 2;                 // [128 x 128]: h2^T, da2^T, da1^T
    static constexpr int DZ = C + kH * kRows * 2;                  // [128 x 48]
    static constexpr int DZT = DZ + kRows * kOutPad * 2;           // [48 x 128]
    static constexpr int Bar = DZT + kOutPad * kRows * 2;
    static constexpr int Slot = Bar + 8;
    static constexpr int Bytes = Slot + 8;
};
static_assert(TrainSmem::Bytes <= 232448, "training tile exceeds the shared memory of one CTA");
// tensor-memory columns: D1/D3/D4 at 0, D2/D5 at 128, dW2 (with db2) at 256,
// dW3^T at 400, dW1 (with db1) at 448
constexpr uint32_t kTrainCols = 512, kColW2 = 256, kColW3T = 400, kColW1 = 448;

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Loss of one row and its gradient with respect to z (written out from the
// loss: BCE of the transmission logit plus, for transmitted tracks, the
// negative log-likelihood of the mixture).
__device__ __forceinline__ float row_loss_grad(const float (&z)[kOutPad], float t, const float* __restrict__ yv,
                                               float (&g)[kOutPad])
{
#pragma unroll
    for (int j = 0; j < kOutPad; ++j) g[j] = 0.0f;
    const float logit = z[0];
    const float sig = 1.0f / (1.0f + expf(-logit));
    g[0] = sig - t;
    float loss = fmaxf(logit, 0.0f) + log1pf(expf(-fabsf(logit))) - t * logit;
    if (t > 0.0f) {
        float y[kDY];
#pragma unroll
        for (int j = 0; j < kDY; ++j) y[j] = yv[j];
        const float amax = fmaxf(fmaxf(z[1], z[2]), fmaxf(z[3], z[4]));
        float asum = 0.0f;
#pragma unroll
        for (int c = 0; c < kNComp; ++c) asum += expf(z[1 + c] - amax);
        const float lse_a = amax + logf(asum);
        float lc[kNComp];
#pragma unroll
        for (int c = 0; c < kNComp; ++c) {
            float acc = z[1 + c] - lse_a;
#pragma unroll
            for (int j = 0; j < kDY; ++j) {
                const float s = z[25 + 5 * c + j];
                const float rr = (y[j] - z[5 + 5 * c + j]) * expf(-s);
                acc += -0.5f * rr * rr - s - 0.91893853320467274f;
            }
            lc[c] = acc;
        }
        const float lmax = fmaxf(fmaxf(lc[0], lc[1]), fmaxf(lc[2], lc[3]));
        float lsum = 0.0f;
#pragma unroll
        for (int c = 0; c < kNComp; ++c) lsum += expf(lc[c] - lmax);
        const float L = lmax + logf(lsum);
        loss -= L;
#pragma unroll
        for (int c = 0; c < kNComp; ++c) {
            const float resp = expf(lc[c] - L);
            const float pi = expf(z[1 + c] - lse_a);
            g[1 + c] = pi - resp;
#pragma unroll
            for (int j = 0; j < kDY; ++j) {
                const float s = z[25 + 5 * c + j];
                const float inv2 = expf(-2.0f * s);
                const float diff = y[j] - z[5 + 5 * c + j];
                g[5 + 5 * c + j] = -resp * diff * inv2;
                g[25 + 5 * c + j] = -resp * (diff * diff * inv2 - 1.0f);
            }
        }
    }
    return loss;
}

__global__ void __launch_bounds__(kRows, 1) k_sur_train(const SurNet net, const float* __restrict__ x,
                                                        const float* __restrict__ yt, const int* __restrict__ label,
                                                        long long first, long long rows, long long n, float inv_rows)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ float s_db3[kOutPad];              // the CTA's b3 gradient
    const uint32_t s0 = smem_addr(sm);
    const int r = threadIdx.x;
    const int lane = r & 31;
    if (r < kOutPad) s_db3[r] = 0.0f;
    copy_to_smem(sm + TrainSmem::Img, net.img, kImgBytes);
    zero_smem(sm + TrainSmem::XT, kInPad * kRows * 2);
    zero_smem(sm + TrainSmem::Bt + kmaj(128, 0, kRows), 16 * kRows * 2);
    zero_smem(sm + TrainSmem::DZT, kOutPad * kRows * 2);
    __syncthreads();
    // constant operand rows: XT row 6 and h1^T row 128 are all ones (bias gradients)
    {
        const unsigned short one = bf16_bits(1.0f);
        *reinterpret_cast<unsigned short*>(sm + TrainSmem::XT + kmaj(6, r, kRows)) = one;
        *reinterpret_cast<unsigned short*>(sm + TrainSmem::Bt + kmaj(128, r, kRows)) = one;
    }
    if (r == 0) mbar_init(s0 + TrainSmem::Bar);
    if ((r >> 5) == 0) tmem_alloc(s0 + TrainSmem::Slot, kTrainCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *reinterpret_cast<volatile uint32_t*>(sm + TrainSmem::Slot);
    const uint32_t t_row = tbase + ((uint32_t)((r >> 5) * 32) << 16);
    const uint32_t bar = s0 + TrainSmem::Bar;
    uint32_t phase = 0u;
    bool ok = true;
    int tiles_done = 0;
    double loss_acc = 0.0;
    const long long end = min(first + rows, n);
    for (long long tile = blockIdx.x; first + tile * kRows < end && ok; tile += gridDim.x) {
        const long long row = first + tile * kRows + r;
        const bool valid = row < end;
        // ---- inputs ----
        float f[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        if (valid) {
#pragma unroll
            for (int k = 0; k < 6; ++k) f[k] = __ldg(x + 6 * row + k);
        }
        store_input_row(sm + TrainSmem::X, r, f);
#pragma unroll
        for (int k = 0; k < 6; ++k)
            *reinterpret_cast<unsigned short*>(sm + TrainSmem::XT + kmaj(k, r, kRows)) = bf16_bits(f[k]);
        uint32_t m1[4] = {0u, 0u, 0u, 0u}, m2[4] = {0u, 0u, 0u, 0u};
        // ---- layer 1 ----
        publish();
        if (r == 0) {
            tc_fence_after();
            mma_tile(tbase, s0 + TrainSmem::X, s0 + TrainSmem::Img + kImgW1, kInPad, kH, false);
            umma_commit(bar);
        }
        if (!(ok = complete(bar, phase))) break;
        hidden_epilogue_train(t_row, net.params + ob1, sm + TrainSmem::A, sm + TrainSmem::Bt, r, m1);
        // ---- layer 2 ----
        publish();
        if (r == 0) {
            tc_fence_after();
            mma_tile(tbase + 128u, s0 + TrainSmem::A, s0 + TrainSmem::Img + kImgW2, kH, kH, false);
            umma_commit(bar);
        }
        if (!(ok = complete(bar, phase))) break;
        hidden_epilogue_train(t_row + 128u, net.params + ob2, sm + TrainSmem::A, sm + TrainSmem::C, r, m2);
        // ---- output layer ----
        publish();
        if (r == 0) {
            tc_fence_after();
            mma_tile(tbase, s0 + TrainSmem::A, s0 + TrainSmem::Img + kImgW3, kH, kOutPad, false);
            umma_commit(bar);
        }
        if (!(ok = complete(bar, phase))) break;
        float zz[kOutPad], g[kOutPad];
        output_epilogue(t_row, net.params + ob3, zz);
        float lrow = 0.0f;
        if (valid) {
            lrow = row_loss_grad(zz, label[row] > 0 ? 1.0f : 0.0f, yt + 5 * row, g);
#pragma unroll
            for (int j = 0; j < kOutPad; ++j) g[j] *= inv_rows;
        } else {
#pragma unroll
            for (int j = 0; j < kOutPad; ++j) g[j] = 0.0f;
        }
        loss_acc += (double)lrow;
        // dz: K-major [128 x 48] and transposed [48 x 128]; b3 gradient by warp sums
#pragma unroll
        for (int c0 = 0; c0 < kOutPad; c0 += 8) {
            uint32_t w[4];
#pragma unroll
            for (int j = 0; j < 8; j += 2) w[j >> 1] = pack_bf16(g[c0 + j], g[c0 + j + 1]);
            *reinterpret_cast<uint4*>(sm + TrainSmem::DZ + kmaj(r, c0, kOutPad)) = make_uint4(w[0], w[1], w[2], w[3]);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (c0 + j < kOut) {
                    const unsigned short b = (unsigned short)((w[j >> 1] >> (16 * (j & 1))) & 0xFFFFu);
                    *reinterpret_cast<unsigned short*>(sm + TrainSmem::DZT + kmaj(c0 + j, r, kRows)) = b;
                }
            }
        }
#pragma unroll 1
        for (int j = 0; j < kOut; ++j) {
            const float s = warp_sum(g[j]);
            if (lane == 0 && s != 0.0f) atomicAdd(s_db3 + j, s);
        }
        // ---- dh2 = dz W3 and dW3^T += h2^T dz ----
        publish();
        if (r == 0) {
            tc_fence_after();
            mma_tile(tbase, s0 + TrainSmem::DZ, s0 + TrainSmem::Img + kImgW3T, kOutPad, kH, false);
            mma_tile(tbase + kColW3T, s0 + TrainSmem::C, s0 + TrainSmem::DZT, kRows, kOutPad, tiles_done > 0);
            umma_commit(bar);
        }
        if (!(ok = complete(bar, phase))) break;
        // ---- da2 = dh2 * relu'(a2): K-major into A, transposed into C ----
        tmem_cols_pipelined(t_row, kH, [&](const uint32_t (&v)[16], int c0) {
            const uint32_t mb = m2[c0 >> 5] >> (c0 & 31);
            uint32_t w[8];
#pragma unroll
            for (int j = 0; j < 16; j += 2) {
                const float a0 = ((mb >> j) & 1u) ? __uint_as_float(v[j]) : 0.0f;
                const float a1 = ((mb >> (j + 1)) & 1u) ? __uint_as_float(v[j + 1]) : 0.0f;
                w[j >> 1] = pack_bf16(a0, a1);
                *reinterpret_cast<unsigned short*>(sm + TrainSmem::C + kmaj(c0 + j, r, kRows)) =
                    (unsigned short)(w[j >> 1] & 0xFFFFu);
                *reinterpret_cast<unsigned short*>(sm + TrainSmem::C + kmaj(c0 + j + 1, r, kRows)) =
                    (unsigned short)(w[j >> 1] >> 16);
            }
            *reinterpret_cast<uint4*>(sm + TrainSmem::A + kmaj(r, c0, kH)) = make_uint4(w[0], w[1], w[2], w[3]);
            *reinterpret_cast<uint4*>(sm + TrainSmem::A + kmaj(r, c0 + 8, kH)) = make_uint4(w[4], w[5], w[6], w[7]);
        });
        // ---- dh1 = da2 W2 and [dW2 | db2] += da2^T [h1 | 1] ----
        publish();
        if (r == 0) {
            tc_fence_after();
            mma_tile(tbase + 128u, s0 + TrainSmem::A, s0 + TrainSmem::Img + kImgW2T, kH, kH, false);
            mma_tile(tbase + kColW2, s0 + TrainSmem::C, s0 + TrainSmem::Bt, kRows, 144, tiles_done > 0);
            umma_commit(bar);
        }
        if (!(ok = complete(bar, phase))) break;
        // ---- da1 = dh1 * relu'(a1), transposed into C ----
        tmem_cols_pipelined(t_row + 128u, kH, [&](const uint32_t (&v)[16], int c0) {
            const uint32_t mb = m1[c0 >> 5] >> (c0 & 31);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float a = ((mb >> j) & 1u) ? __uint_as_float(v[j]) : 0.0f;
                *reinterpret_cast<unsigned short*>(sm + TrainSmem::C + kmaj(c0 + j, r, kRows)) = bf16_bits(a);
            }
        });
        // ---- [dW1 | db1] += da1^T [x | 1] ----
        publish();
        if (r == 0) {
            tc_fence_after();
            mma_tile(tbase + kColW1, s0 + TrainSmem::C, s0 + TrainSmem::XT, kRows, kInPad, tiles_done > 0);
            umma_commit(bar);
        }
        if (!(ok = complete(bar, phase))) break;
        ++tiles_done;
    }
    // ---- loss and the accumulated weight gradients ----
    const float ls = warp_sum((float)loss_acc);
    if (lane == 0 && ls != 0.0f) atomicAdd(net.loss, (double)ls);
    // the CTA's partial gradient, every parameter written once (plain stores;
    // the Adam step sums the CTAs' partials: no contended atomics)
    float* part = net.gpart + (long long)blockIdx.x * kNParams;
    const bool have = ok && tiles_done > 0;
    __syncthreads();                                // s_db3 complete
    {
        const int h = r;
#pragma unroll 1
        for (int c0 = 0; c0 < 144; c0 += 16) {
            float v[16];
            if (have) tmem_ld16(t_row + kColW2 + (uint32_t)c0, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int i = c0 + j;
                const float gv = have ? v[j] : 0.0f;
                if (i < kH) part[oW2 + h * kH + i] = gv;
                else if (i == kH) part[ob2 + h] = gv;
            }
        }
#pragma unroll 1
        for (int c0 = 0; c0 < kOutPad; c0 += 16) {
            float v[16];
            if (have) tmem_ld16(t_row + kColW3T + (uint32_t)c0, v);
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (c0 + j < kOut) part[oW3 + (c0 + j) * kH + h] = have ? v[j] : 0.0f;
        }
        {
            float v[16];
            if (have) tmem_ld16(t_row + kColW1, v);
#pragma unroll
            for (int j = 0; j < kIn; ++j) part[oW1 + h * kIn + j] = have ? v[j] : 0.0f;
            part[ob1 + h] = have ? v[kIn] : 0.0f;
        }
        if (r < kOut) part[ob3 + r] = have ? s_db3[r] : 0.0f;
    }
    if (!ok) {
        if (r == 0) atomicOr(net.status, 1);
        (void)mbar_wait(bar, phase);
    }
    tc_fence_before();
    __syncthreads();
    if ((r >> 5) == 0) {
        tc_fence_after();
        tmem_dealloc(tbase, kTrainCols);
    }
}

// ============================================================================
// Parameter update and BF16 operand images.
// ============================================================================
__device__ __forceinline__ void write_images(unsigned char* img, int k, float w)
{
    const unsigned short b = bf16_bits(w);
    if (k >= oW1 && k < ob1) {
        const int h = (k - oW1) / kIn, f = (k - oW1) % kIn;
        *reinterpret_cast<unsigned short*>(img + kImgW1 + kmaj(h, f, kInPad)) = b;
    } else if (k >= oW2 && k < ob2) {
        const int h = (k - oW2) / kH, i = (k - oW2) % kH;
        *reinterpret_cast<unsigned short*>(img + kImgW2 + kmaj(h, i, kH)) = b;
        *reinterpret_cast<unsigned short*>(img + kImgW2T + kmaj(i, h, kH)) = b;
    } else if (k >= oW3 && k < ob3) {
        const int o = (k - oW3) / kH, h = (k - oW3) % kH;
        *reinterpret_cast<unsigned short*>(img + kImgW3 + kmaj(o, h, kH)) = b;
        *reinterpret_cast<unsigned short*>(img + kImgW3T + kmaj(h, o, kOutPad)) = b;
    }
}

__global__ void k_sur_pack(const SurNet net)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < kNParams) write_images(net.img, k, net.params[k]);
}

// Adam (Kingma & Ba 2015): moments, bias corrections c1 = 1 / (1 - beta1^t),
// c2 = 1 / (1 - beta2^t); the gradient is cleared for the next step.
// Sum of the parts CTAs' partial gradients of parameter k (coalesced over k).
__device__ __forceinline__ float summed_grad(const SurNet& net, int k, int parts)
{
    float g = 0.0f;
    for (int c = 0; c < parts; ++c) g += net.gpart[(long long)c * kNParams + k];
    return g;
}

__global__ void k_sur_reduce(const SurNet net, int parts)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < kNParams) net.grad[k] = summed_grad(net, k, parts);
}

__global__ void k_sur_adam(const SurNet net, float lr, float c1, float c2, int parts)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= kNParams) return;
    const float g = summed_grad(net, k, parts);
    const float m = fmaf(0.9f, net.m[k], 0.1f * g);
    const float v = fmaf(0.999f, net.v[k], 0.001f * g * g);
    net.m[k] = m;
    net.v[k] = v;
    const float w = net.params[k] - lr * (m * c1) / (sqrtf(v * c2) + 1e-8f);
    net.params[k] = w;
    write_images(net.img, k, w);
}

}  // namespace

size_t sur_forward_smem_bytes() { return FwdSmem::Bytes; }
size_t sur_train_smem_bytes() { return TrainSmem::Bytes; }

cudaError_t launch_sur_pack(const SurNet& net, cudaStream_t s)
{
    k_sur_pack<<<(kNParams + 255) / 256, 256, 0, s>>>(net);
    return cudaGetLastError();
}

cudaError_t launch_sur_forward(const SurNet& net, const float* x, long long n, float* z, int grid, cudaStream_t s)
{
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_sur_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, FwdSmem::Bytes);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    if (n <= 0) return cudaSuccess;
    const long long tiles = (n + kRows - 1) / kRows;
    const long long ctas = (tiles + kGroups - 1) / kGroups;
    k_sur_forward<<<(int)std::min<long long>(ctas, grid), kFwdThreads, FwdSmem::Bytes, s>>>(net, x, n, z);
    return cudaGetLastError();
}

cudaError_t launch_sur_infer(const SurNet& net, const TransportParams& p, int grid, cudaStream_t s)
{
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_sur_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, FwdSmem::Bytes);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_sur_infer<<<grid, kFwdThreads, FwdSmem::Bytes, s>>>(net, p);
    return cudaGetLastError();
}

cudaError_t launch_sur_train(const SurNet& net, const float* x, const float* y, const int* label, long long first,
                             long long rows, long long n, float inv_rows, int grid, int* parts, cudaStream_t s)
{
    *parts = 0;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_sur_train, cudaFuncAttributeMaxDynamicSharedMemorySize, TrainSmem::Bytes);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const long long tiles = (rows + kRows - 1) / kRows;
    if (tiles <= 0) return cudaSuccess;
    const int ctas = (int)std::min<long long>(tiles, std::min(grid, net.n_part_cap));
    k_sur_train<<<ctas, kRows, TrainSmem::Bytes, s>>>(net, x, y, label, first, rows, n, inv_rows);
    *parts = ctas;
    return cudaGetLastError();
}

cudaError_t launch_sur_reduce(const SurNet& net, int parts, cudaStream_t s)
{
    k_sur_reduce<<<(kNParams + 255) / 256, 256, 0, s>>>(net, parts);
    return cudaGetLastError();
}

cudaError_t launch_sur_adam(const SurNet& net, int step, float lr, int parts, cudaStream_t s)
{
    const float c1 = (float)(1.0 / (1.0 - pow(0.9, step)));
    const float c2 = (float)(1.0 / (1.0 - pow(0.999, step)));
    k_sur_adam<<<(kNParams + 255) / 256, 256, 0, s>>>(net, lr, c1, c2, parts);
    return cudaGetLastError();
}

}  // namespace vpmc
