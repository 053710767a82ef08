// Persistent proton transport kernel for sm_103a.
//
// One history per thread (paper Sec. 2.A: every history follows one identical
// model, so no secondary particles are spawned).  Warps are persistent: a warp
// takes chunks of consecutive global history indices from one counter and hands
// them to lanes whose history has ended, so dead lanes are refilled at once.
// Each history crosses, in order, an optional range shifter, the brass aperture
// (Sec. 2.B: at every step inside the aperture slab a crossing-number test
// decides opening -> straight flight, or brass -> condensed-history step with
// brass physics), and the voxelised patient, where every step's deposit is
// scored into a 64-bit fixed-point accumulator (optionally aggregated over the
// lanes of a warp that hit the same voxel, then one atomic per voxel).
//
// Physics of one condensed-history step (same definition as the CPU oracle):
//   step = min(1 mm, 1 % energy-loss length, geometry limit, nuclear point);
//   mean loss from the residual range carried with the particle,
//   E' = E(R - s * kappa); Bohr straggling; Highland scattering with the PDG
//   correlated (angle, offset) pair in two planes; nuclear removal at
//   0.0012 / mm x density with the removed energy deposited locally.
// Random numbers: Philox4x32-10, key = (seed lo, spot ^ seed hi), counter =
// (history, step, slot, 0): slot 0 source, 1 scattering, 2 straggling,
// 3 nuclear free path.
#include "vpmc_internal.cuh"

namespace vpmc {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr float kMp = 938.272f;

__device__ __forceinline__ uint4 philox(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// ((x >> 9) + 1/2) * 2^-23: 23-bit uniform in (0, 1), exact in FP32.
__device__ __forceinline__ float u01(uint32_t x) { return fmaf(__uint2float_rn(x >> 9), 0x1p-23f, 0x1p-24f); }

// Box-Muller with accurate functions (source sampling, once per history).
__device__ __forceinline__ float2 box_muller(float u1, float u2)
{
    const float r = sqrtf(-2.0f * logf(u1));
    float s, c;
    sincospif(2.0f * u2, &s, &c);
    return make_float2(r * c, r * s);
}

// Box-Muller with hardware approximations (per-step physics).  u1 <= 1 - 2^-24,
// so -2 ln u1 > 0; the clamp only guards the approximate logarithm.
__device__ __forceinline__ float2 box_muller_fast(float u1, float u2)
{
    const float l = fmaxf(-2.0f * __logf(u1), 0.0f);
    const float r = l * rsqrtf(fmaxf(l, 1e-30f));
    float s, c;
    __sincosf(6.28318530717958647f * u2, &s, &c);
    return make_float2(r * c, r * s);
}

__device__ __forceinline__ float fast_sqrt(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }

// Two Philox4x32-10 blocks with the same key, rounds interleaved for ILP.
__device__ __forceinline__ void philox_pair(uint4& a, uint4& b, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t ah0 = __umulhi(0xD2511F53u, a.x), al0 = 0xD2511F53u * a.x;
        const uint32_t ah1 = __umulhi(0xCD9E8D57u, a.z), al1 = 0xCD9E8D57u * a.z;
        const uint32_t bh0 = __umulhi(0xD2511F53u, b.x), bl0 = 0xD2511F53u * b.x;
        const uint32_t bh1 = __umulhi(0xCD9E8D57u, b.z), bl1 = 0xCD9E8D57u * b.z;
        a = make_uint4(ah1 ^ a.y ^ k.x, al1, ah0 ^ a.w ^ k.y, al0);
        b = make_uint4(bh1 ^ b.y ^ k.x, bl1, bh0 ^ b.w ^ k.y, bl0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
}

__device__ __forceinline__ float range_of(const float* __restrict__ R, float E)
{
    if (E <= 0.0f) return 0.0f;
    const float x = E * 10.0f;
    const int i = min((int)x, kNE - 2);
    const float f = x - (float)i;
    const float r0 = R[i];
    return fmaf(f, R[i + 1] - r0, r0);
}

__device__ __forceinline__ float energy_of(const float* __restrict__ Et, float inv_dR, float R)
{
    if (R <= 0.0f) return kEcut;
    const float x = R * inv_dR;
    const int j = min((int)x, kNR - 2);
    const float f = x - (float)j;
    const float e0 = Et[j];
    return fmaf(f, Et[j + 1] - e0, e0);
}

// Crossing-number (ray casting) point-in-polygon test, half-open edge rule.
__device__ __forceinline__ bool point_in_polygon(const float2* __restrict__ poly, int n, float x, float y)
{
    bool inside = false;
    float2 pj = poly[n - 1];
    for (int i = 0; i < n; ++i) {
        const float2 pi = poly[i];
        if ((pi.y > y) != (pj.y > y)) {
            const float xc = pi.x + (y - pi.y) * (pj.x - pi.x) / (pj.y - pi.y);
            if (x < xc) inside = !inside;
        }
        pj = pi;
    }
    return inside;
}

// Smallest s > 0 at which (x, y) + s (dx, dy) crosses an edge.
__device__ __forceinline__ float first_wall_hit(const float2* __restrict__ poly, int n, float x, float y, float dx,
                                                float dy)
{
    float best = __int_as_float(0x7f800000);
    for (int i = 0; i < n; ++i) {
        const float2 a = poly[i];
        const float2 b = poly[i + 1 < n ? i + 1 : 0];
        const float ex = b.x - a.x, ey = b.y - a.y;
        const float den = dx * ey - dy * ex;
        if (den == 0.0f) continue;
        const float wx = a.x - x, wy = a.y - y;
        const float s = (wx * ey - wy * ex) / den;
        const float lam = (wx * dy - wy * dx) / den;
        if (s > 0.0f && lam >= 0.0f && lam <= 1.0f && s < best) best = s;
    }
    return best;
}

// Opening test accelerated by the beam's BEV raster: cells that no edge comes
// near are wholly inside (1) or outside (0); edge cells (2) run the exact test.
__device__ __forceinline__ bool in_opening(const DevBeam& B, const float2* __restrict__ poly,
                                           const unsigned char* __restrict__ raster, float a, float b)
{
    const float fx = (a - B.ras_lo[0]) * B.ras_inv[0];
    const float fy = (b - B.ras_lo[1]) * B.ras_inv[1];
    if (!(fx >= 0.0f && fx < (float)kRaster && fy >= 0.0f && fy < (float)kRaster)) return false;
    const int c = __ldg(raster + B.ras_off + (int)fy * kRaster + (int)fx);
    if (c != 2) return c == 1;
    return point_in_polygon(poly + B.poly_off, B.nvert, a, b);
}

// Duff et al. 2017, "Building an orthonormal basis, revisited".
__device__ __forceinline__ void orthonormal_basis(const float n[3], float b1[3], float b2[3])
{
    const float sign = copysignf(1.0f, n[2]);
    const float a = __fdividef(-1.0f, sign + n[2]);
    const float b = n[0] * n[1] * a;
    b1[0] = 1.0f + sign * n[0] * n[0] * a;
    b1[1] = sign * b;
    b1[2] = -sign * n[0];
    b2[0] = b;
    b2[1] = sign + n[1] * n[1] * a;
    b2[2] = -n[1];
}

// n-th (0-based) set bit of m; m must have more than n bits set.
__device__ __forceinline__ int nth_set_bit(unsigned m, int n)
{
    int pos = 0;
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const unsigned low = (unsigned)((1ull << (pos + w)) - 1ull);
        if (__popc(m & low) <= n) pos += w;
    }
    return pos;
}

// Every lane of the warp calls this.  key < 0: no deposit.  Lanes with the
// same key are summed (tree over the peer group) and the lowest peer issues
// one 64-bit atomic.
__device__ __forceinline__ void deposit_aggregated(unsigned long long* __restrict__ dst, long long key,
                                                   unsigned long long q)
{
    const unsigned peers = __match_any_sync(kFull, key);
    const int lane = threadIdx.x & 31;
    const int rank = __popc(peers & ((1u << lane) - 1u));
    const int cnt = __popc(peers);
    const unsigned maxcnt = __reduce_max_sync(kFull, (unsigned)cnt);
    unsigned long long sum = q;
    for (int k = 1; k < (int)maxcnt; k <<= 1) {
        const int src_rank = rank + k;
        const int src = src_rank < cnt ? nth_set_bit(peers, src_rank) : lane;
        const unsigned long long other = __shfl_sync(kFull, sum, src);
        if ((rank & (2 * k - 1)) == 0 && src_rank < cnt) sum += other;
    }
    if (rank == 0 && key >= 0 && sum != 0ull) atomicAdd(dst + key, sum);
}

struct Medium {
    int table;
    float kappa, rho, za, inv_x0;
};

struct StepResult {
    float s, dE;
    float disp[3];
    int lim;        // 0 none, 1 geometry, 2 nuclear
    int killed;     // 1 stopped, 2 nuclear
};

struct Lane {
    float p[3], d[3];
    float E, R, nlam;
    uint32_t step;
    uint32_t hist;
    int stage;      // 0 range shifter, 1 aperture, 2 patient
    int forced;     // aperture: the next step is in brass (after a wall hit)
    int ic[3], is[3];
    int item;
    int iters, nsteps;
    long long g;
    unsigned long long qdep;
};

struct Smem {
    const float* R;
    const float* Et;
    const float2* hu;
    const MatConst* mat;
    const DevBeam* beams;
    const DevScen* scens;
    const float2* poly;
};

__device__ __forceinline__ void ch_step(const Smem& S, const Medium& m, float s_geom, Lane& L,
                                        const TransportParams& P, uint2 key, StepResult& o)
{
    const float* Rt = S.R + m.table * kNEPad;
    const float* Et = S.Et + m.table * kNR;
    const float inv_dR = S.mat[m.table].inv_dR;
    const float E = L.E;
    const float R0 = L.R;
    const float inv_kappa = __fdividef(1.0f, m.kappa);
    float s1 = (R0 - range_of(Rt, 0.99f * E)) * inv_kappa;
    if (!(s1 > 0.0f)) s1 = R0 * inv_kappa;
    const float mu = P.nuclear ? 0.0012f * m.rho : 0.0f;
    float s = 1.0f;
    int lim = 0;
    if (s1 < s) s = s1;
    if (s_geom < s) { s = s_geom; lim = 1; }
    if (mu > 0.0f) {
        const float sn = __fdividef(L.nlam, mu);
        if (sn < s) { s = sn; lim = 2; }
    }
    L.step += 1;
    if (lim == 2) L.nlam = 0.0f; else L.nlam -= mu * s;

    // random numbers of this step: slot 1 (scattering) and slot 2 (straggling)
    uint4 r1 = make_uint4(L.hist, L.step, 1u, 0u), r2 = make_uint4(L.hist, L.step, 2u, 0u);
    if (P.mcs || P.straggling) philox_pair(r1, r2, key);

    const float R1 = R0 - s * m.kappa;
    const float Emean = R1 > 0.0f ? energy_of(Et, inv_dR, R1) : kEcut;
    float dE = E - Emean;
    const float etot = E + kMp;
    const float pc2 = E * (E + 2.0f * kMp);               // (pc)^2
    const float inv_etot = __fdividef(1.0f, etot);
    if (P.straggling) {
        const float beta2 = pc2 * inv_etot * inv_etot;
        const float2 z = box_muller_fast(u01(r2.x), u01(r2.y));
        const float var = 0.01569f * m.rho * m.za * s * __fdividef(1.0f - 0.5f * beta2, 1.0f - beta2);
        dE += fast_sqrt(var) * z.x;
    }
    dE = fminf(fmaxf(dE, 0.0f), E);
    const float Enew = E - dE;
    float Rnew = R1;
    if (P.straggling) {
        Rnew = R1 + (range_of(Rt, Enew) - range_of(Rt, Emean));
        if (!(Rnew > 0.0f)) Rnew = range_of(Rt, Enew);
    }
    L.R = Rnew;

    o.s = s;
    o.lim = lim;
    o.disp[0] = o.disp[1] = o.disp[2] = 0.0f;
    o.killed = lim == 2 ? 2 : (Enew <= kEcut ? 1 : 0);
    if (o.killed) { o.dE = E; L.E = 0.0f; }
    else { o.dE = dE; L.E = Enew; }

#pragma unroll
    for (int k = 0; k < 3; ++k) L.p[k] = fmaf(s, L.d[k], L.p[k]);

    if (P.mcs && !o.killed) {
        const float x = s * m.rho * m.inv_x0;
        float th0 = 0.0f;
        if (x >= 1e-6f) {
            const float bcp = pc2 * inv_etot;                 // beta c p
            th0 = __fdividef(13.6f, bcp) * fast_sqrt(x) * (1.0f + 0.038f * __logf(x));
        }
        const float2 za = box_muller_fast(u01(r1.x), u01(r1.y));
        const float2 zb = box_muller_fast(u01(r1.z), u01(r1.w));
        const float th1 = za.y * th0, th2 = zb.y * th0;
        const float dx1 = s * th0 * fmaf(za.x, 0.28867513459481287f, 0.5f * za.y);
        const float dx2 = s * th0 * fmaf(zb.x, 0.28867513459481287f, 0.5f * zb.y);
        float e1[3], e2[3];
        orthonormal_basis(L.d, e1, e2);
        const float th2sq = th1 * th1 + th2 * th2;
        const float th = fast_sqrt(th2sq);
        float sn, c;
        __sincosf(th, &sn, &c);
        const float sc = th > 0.0f ? __fdividef(sn, th) : 1.0f;
        float nd[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            o.disp[k] = dx1 * e1[k] + dx2 * e2[k];
            nd[k] = c * L.d[k] + sc * (th1 * e1[k] + th2 * e2[k]);
        }
        const float inv = rsqrtf(nd[0] * nd[0] + nd[1] * nd[1] + nd[2] * nd[2]);
#pragma unroll
        for (int k = 0; k < 3; ++k) L.d[k] = nd[k] * inv;
    }
}

__device__ __forceinline__ void bev_to_patient(const DevBeam& B, const DevScen& sc, const float pb[3], float out[3])
{
#pragma unroll
    for (int k = 0; k < 3; ++k)
        out[k] = B.iso[k] + sc.shift[k] + pb[0] * B.u[k] + pb[1] * B.v[k] + pb[2] * B.w[k];
}

// Move the history into the next stage after `from` (-1: just born).  Returns
// a fate >= 0 if the history ends here (left the geometry), else -1.
__device__ int enter_next_stage(const Smem& S, const TransportParams& P, const DevBeam& B, const DevScen& sc,
                                Lane& L, int from)
{
    if (from < 0 && B.rs) {   // just born
        const float sdr = (B.rs_tup - L.p[2]) / L.d[2];
#pragma unroll
        for (int k = 0; k < 3; ++k) L.p[k] = fmaf(sdr, L.d[k], L.p[k]);
        L.R = range_of(S.R + kPMMA * kNEPad, L.E);
        L.stage = 0;
        return -1;
    }
    if (from < 1 && B.ap) {
        if (!(L.d[2] > 0.0f)) return kLeak;
        const float sdr = (B.ap_tup - L.p[2]) / L.d[2];
#pragma unroll
        for (int k = 0; k < 3; ++k) L.p[k] = fmaf(sdr, L.d[k], L.p[k]);
        L.R = range_of(S.R + kBrass * kNEPad, L.E);
        L.stage = 1;
        L.forced = 0;
        return -1;
    }
    // patient: BEV -> patient frame, ray / grid box entry
    float Pp[3], D[3];
    bev_to_patient(B, sc, L.p, Pp);
#pragma unroll
    for (int k = 0; k < 3; ++k) D[k] = L.d[0] * B.u[k] + L.d[1] * B.v[k] + L.d[2] * B.w[k];
    float tmin = -__int_as_float(0x7f800000), tmax = __int_as_float(0x7f800000);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float lo = P.ctg.lo[k], hi = P.ctg.lo[k] + P.ctg.n[k] * P.ctg.d[k];
        if (D[k] != 0.0f) {
            float t1 = (lo - Pp[k]) / D[k], t2 = (hi - Pp[k]) / D[k];
            if (t1 > t2) { const float tt = t1; t1 = t2; t2 = tt; }
            tmin = fmaxf(tmin, t1);
            tmax = fminf(tmax, t2);
        } else if (Pp[k] < lo || Pp[k] > hi) {
            tmax = -__int_as_float(0x7f800000);
        }
    }
    const float tin = fmaxf(tmin, 0.0f);
#pragma unroll
    for (int k = 0; k < 3; ++k) { L.p[k] = Pp[k]; L.d[k] = D[k]; }
    L.stage = 2;
    if (!(tmax > tin)) return kLeak;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        L.p[k] = fmaf(tin, D[k], Pp[k]);
        const int a = (int)floorf((L.p[k] - P.ctg.lo[k]) / P.ctg.d[k]);
        L.ic[k] = min(max(a, 0), P.ctg.n[k] - 1);
        const int b = (int)floorf((L.p[k] - P.sg.lo[k]) / P.sg.d[k]);
        L.is[k] = min(max(b, 0), P.sg.n[k] - 1);
    }
    L.R = range_of(S.R + kWater * kNEPad, L.E);
    return -1;
}

// Largest i with items[i].hist_off <= g, searched by the whole warp: each
// round the 32 lanes probe 32 evenly spaced entries (g is warp-uniform).
__device__ __forceinline__ int find_item_warp(const DevItem* __restrict__ items, int n, long long g, int lane)
{
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int step = (hi - lo + 31) >> 5;
        const int idx = lo + lane * step;
        const bool le = idx < hi && __ldg(&items[idx].hist_off) <= g;
        const unsigned m = __ballot_sync(kFull, le);
        const int last = 31 - __clz(m);
        lo = lo + last * step;
        hi = min(lo + step, hi);
    }
    return lo;
}

}  // namespace

__global__ void __launch_bounds__(640, 1) k_transport(const TransportParams P)
{
    extern __shared__ __align__(16) unsigned char smem[];
    // stage the tables, beams, scenarios and polygons into shared memory
    {
        const int4* src = reinterpret_cast<const int4*>(P.tables);
        int4* dst = reinterpret_cast<int4*>(smem);
        constexpr int n16 = (int)(SharedLayout::Beams / 16);
        static_assert(SharedLayout::Beams % 16 == 0, "table image must be a 16-byte multiple");
        static_assert(sizeof(TablesImage) == SharedLayout::Beams, "table image layout");
        for (int i = threadIdx.x; i < n16; i += blockDim.x) dst[i] = __ldg(src + i);
        DevBeam* bm = reinterpret_cast<DevBeam*>(smem + SharedLayout::Beams);
        for (int i = threadIdx.x; i < P.n_beams; i += blockDim.x) bm[i] = P.beams[i];
        DevScen* sc = reinterpret_cast<DevScen*>(smem + SharedLayout::Scens);
        for (int i = threadIdx.x; i < P.n_scen; i += blockDim.x) sc[i] = P.scens[i];
        float2* pl = reinterpret_cast<float2*>(smem + SharedLayout::Poly);
        for (int i = threadIdx.x; i < P.n_poly; i += blockDim.x) pl[i] = P.poly[i];
    }
    __syncthreads();
    Smem S;
    S.R = reinterpret_cast<const float*>(smem + SharedLayout::R);
    S.Et = reinterpret_cast<const float*>(smem + SharedLayout::Einv);
    S.hu = reinterpret_cast<const float2*>(smem + SharedLayout::HU);
    S.mat = reinterpret_cast<const MatConst*>(smem + SharedLayout::Mat);
    S.beams = reinterpret_cast<const DevBeam*>(smem + SharedLayout::Beams);
    S.scens = reinterpret_cast<const DevScen*>(smem + SharedLayout::Scens);
    S.poly = reinterpret_cast<const float2*>(smem + SharedLayout::Poly);

    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    long long pool_next = 0, pool_end = 0;      // warp-uniform
    int pool_item = 0;                          // item of pool_next (warp-uniform)
    bool alive = false, done = false;
    Lane L;
    L.item = 0; L.g = 0; L.hist = 0; L.qdep = 0ull; L.iters = 0; L.nsteps = 0; L.stage = 0; L.forced = 0;
    L.step = 0; L.E = 0.0f; L.R = 0.0f; L.nlam = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) { L.p[k] = 0.0f; L.d[k] = 0.0f; L.ic[k] = 0; L.is[k] = 0; }
    unsigned long long acc_dep = 0, acc_leak = 0, acc_rs = 0, acc_ap = 0, acc_nuc = 0;
    unsigned acc_steps = 0, acc_err = 0;
    uint2 key = make_uint2(0u, 0u);

    for (;;) {
        // ---- hand new histories to lanes whose history has ended ----
        unsigned need = __ballot_sync(kFull, !alive && !done);
        while (need) {
            if (pool_next >= pool_end) {
                // take the next chunk; stop taking work once any history has
                // hit the iteration cap (a latched error ends the launch early)
                unsigned long long base = 0;
                int abort = 0;
                if (lane == 0) {
                    base = atomicAdd(P.counter, (unsigned long long)P.chunk);
                    abort = *reinterpret_cast<volatile int*>(P.status);
                }
                base = __shfl_sync(kFull, base, 0);
                abort = __shfl_sync(kFull, abort, 0);
                if (abort || (long long)base >= P.total) {
                    if (!alive) done = true;
                    break;
                }
                pool_next = (long long)base;
                pool_end = min((long long)base + P.chunk, P.total);
                pool_item = find_item_warp(P.items, P.n_items, pool_next, lane);
            }
            const int take = (int)min((long long)__popc(need), pool_end - pool_next);
            const bool mine = ((need >> lane) & 1u) && __popc(need & lt_mask) < take;
            if (mine) {
                const long long g = pool_next + __popc(need & lt_mask);
                int it = pool_item;
                while (it + 1 < P.n_items && __ldg(&P.items[it + 1].hist_off) <= g) ++it;
                const DevItem I = P.items[it];
                const DevBeam& B = S.beams[I.beam];
                L.item = it;
                L.g = g;
                L.hist = (uint32_t)(g - I.hist_off);
                L.step = 0;
                L.iters = 0;
                L.nsteps = 0;
                L.qdep = acc_dep;
                key = make_uint2(P.key0, P.key1_hi ^ (uint32_t)I.spot);
                // source: slot 0 -> (x, y) at the isocentre plane and two projected angles
                const uint4 x = philox(make_uint4(L.hist, 0u, 0u, 0u), key);
                const float2 z01 = box_muller(u01(x.x), u01(x.y));
                const float2 z23 = box_muller(u01(x.z), u01(x.w));
                const float a0 = fmaf(I.sigma, z01.x, I.x), b0 = fmaf(I.sigma, z01.y, I.y);
                const float tha = I.div_rad * z23.x, thb = I.div_rad * z23.y;
                const float nrm = rsqrtf(1.0f + tha * tha + thb * thb);
                L.d[0] = tha * nrm; L.d[1] = thb * nrm; L.d[2] = nrm;
                L.p[0] = fmaf(B.t_src, tha, a0); L.p[1] = fmaf(B.t_src, thb, b0); L.p[2] = B.t_src;
                L.E = I.E0;
                if (P.nuclear) {
                    const uint4 y = philox(make_uint4(L.hist, 0u, 3u, 0u), key);
                    L.nlam = -logf(u01(y.x));
                } else {
                    L.nlam = __int_as_float(0x7f800000);
                }
                L.stage = -1;                       // enters its first stage in the next iteration
                alive = true;
            }
            pool_next += take;
            need = __ballot_sync(kFull, !alive && !done);
        }
        if (!__any_sync(kFull, alive)) {
            if (__all_sync(kFull, done || alive)) break;
            continue;
        }

        // ---- one iteration of every live history ----
        long long dep_key = -1;
        unsigned long long dep_q = 0ull;
        if (alive) {
            int fate = -1;
            bool advance = false;                   // move to the next stage after this iteration
            const int from = L.stage;
            const DevItem& I = P.items[L.item];
            const int beam = __ldg(&I.beam);
            const int scn = __ldg(&I.scen);
            const DevBeam& B = S.beams[beam];
            const DevScen& SC = S.scens[scn];
            Medium m;
            float s_geom = __int_as_float(0x7f800000);
            bool do_ch = false, down = true;
            float dc[3], ds[3];
            if (++L.iters > kMaxIter) {
                fate = kErr;
            } else if (L.stage < 0) {
                advance = true;
            } else if (L.stage == 0) {
                // ---- range shifter ----
                if (L.p[0] * L.p[0] + L.p[1] * L.p[1] > B.rs_r2) {
                    if (!(L.d[2] > 0.0f)) fate = kLeak;
                    else {
                        const float sf = (B.rs_tdn - L.p[2]) / L.d[2];
#pragma unroll
                        for (int k = 0; k < 3; ++k) L.p[k] = fmaf(sf, L.d[k], L.p[k]);
                        advance = true;
                    }
                } else {
                    if (L.d[2] > 0.0f) s_geom = (B.rs_tdn - L.p[2]) / L.d[2];
                    else if (L.d[2] < 0.0f) { s_geom = (B.rs_tup - L.p[2]) / L.d[2]; down = false; }
                    s_geom = fmaxf(s_geom, 0.0f);   // scattering offsets can leave it past the plane
                    m.table = kPMMA; m.kappa = S.mat[kPMMA].rho; m.rho = m.kappa; m.za = S.mat[kPMMA].za;
                    m.inv_x0 = S.mat[kPMMA].inv_x0;
                    do_ch = true;
                }
            } else if (L.stage == 1) {
                // ---- aperture block ----
                if (L.d[2] > 0.0f) s_geom = (B.ap_tdn - L.p[2]) / L.d[2];
                else if (L.d[2] < 0.0f) { s_geom = (B.ap_tup - L.p[2]) / L.d[2]; down = false; }
                s_geom = fmaxf(s_geom, 0.0f);       // scattering offsets can leave it past the plane
                const bool open = !L.forced && in_opening(B, S.poly, P.raster, L.p[0], L.p[1]);
                if (open) {
                    const float sw = first_wall_hit(S.poly + B.poly_off, B.nvert, L.p[0], L.p[1], L.d[0], L.d[1]);
                    if (sw < s_geom) {
#pragma unroll
                        for (int k = 0; k < 3; ++k) L.p[k] = fmaf(sw, L.d[k], L.p[k]);
                        L.forced = 1;
                    } else if (!isfinite(s_geom)) {
                        fate = kErr;
                    } else {
#pragma unroll
                        for (int k = 0; k < 3; ++k) L.p[k] = fmaf(s_geom, L.d[k], L.p[k]);
                        if (down) advance = true; else fate = kLeak;
                    }
                } else {
                    L.forced = 0;
                    m.table = kBrass; m.kappa = S.mat[kBrass].rho; m.rho = m.kappa; m.za = S.mat[kBrass].za;
                    m.inv_x0 = S.mat[kBrass].inv_x0;
                    do_ch = true;
                }
            } else {
                // ---- patient ----
                const long long cidx = L.ic[0] + (long long)P.ctg.n[0] * (L.ic[1] + (long long)P.ctg.n[1] * L.ic[2]);
                const int h = min(max((int)__ldg(P.ct + cidx), kHULo), kHULo + kNHU - 1);
                const float2 rs = S.hu[h - kHULo];
                m.table = kWater; m.kappa = rs.y * SC.spr_scale; m.rho = rs.x; m.za = S.mat[kWater].za;
                m.inv_x0 = S.mat[kWater].inv_x0;
                do_ch = true;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    dc[k] = ds[k] = __int_as_float(0x7f800000);
                    const float Dk = L.d[k];
                    if (Dk != 0.0f) {
                        const float inv = __fdividef(1.0f, Dk);
                        const int up = Dk > 0.0f ? 1 : 0;
                        const float bc = P.ctg.lo[k] + (float)(L.ic[k] + up) * P.ctg.d[k];
                        dc[k] = fmaxf((bc - L.p[k]) * inv, 0.0f);
                        if (P.same_grid) ds[k] = dc[k];
                        else {
                            const float bs = P.sg.lo[k] + (float)(L.is[k] + up) * P.sg.d[k];
                            ds[k] = fmaxf((bs - L.p[k]) * inv, 0.0f);
                        }
                    }
                    s_geom = fminf(s_geom, fminf(dc[k], ds[k]));
                }
            }

            if (do_ch) {
                StepResult o;
                const float d_old[3] = {L.d[0], L.d[1], L.d[2]};
                const int is_old[3] = {L.is[0], L.is[1], L.is[2]};
                ch_step(S, m, s_geom, L, P, key, o);
                L.nsteps += 1;
                acc_steps += 1;
                const unsigned long long qs = __float2ull_rn(o.dE * P.fscale);
                if (L.stage == 0) {
                    acc_rs += qs;
                    if (o.killed) { if (o.killed == 2) acc_nuc += qs; fate = kAbsRS; }
                } else if (L.stage == 1) {
                    acc_ap += qs;
                    if (o.killed) { if (o.killed == 2) acc_nuc += qs; fate = kAbsAp; }
                } else {
                    // score into the scoring voxel where the step started
                    const DevBox bx = P.boxes[__ldg(&I.box)];
                    const int lx = is_old[0] - bx.lo[0], ly = is_old[1] - bx.lo[1], lz = is_old[2] - bx.lo[2];
                    const float wsc = __ldg(&I.wscale);
                    const unsigned long long q = wsc == P.fscale ? qs : __float2ull_rn(o.dE * wsc);
                    if (lx >= 0 && ly >= 0 && lz >= 0 && lx < bx.n[0] && ly < bx.n[1] && lz < bx.n[2]) {
                        dep_key = bx.base + lx + (long long)bx.n[0] * (ly + (long long)bx.n[1] * lz);
                        dep_q = q;
                    } else if (o.dE > 0.0f && P.ovf) {
                        // rare tail outside the item's box: append a record
                        const unsigned long long slot = atomicAdd(P.ovf_count, 1ull);
                        if ((long long)slot < P.ovf_cap) {
                            OvfRec r;
                            r.voxel = is_old[0] + P.sg.n[0] * (is_old[1] + P.sg.n[1] * is_old[2]);
                            r.item = L.item;
                            r.q = q;
                            P.ovf[slot] = r;
                        }
                    }
                    acc_dep += qs;
                    if (o.killed) {
                        if (o.killed == 2) acc_nuc += qs;
                        fate = o.killed == 2 ? kNuc : kStop;
                    }
                }
                if (fate < 0) {
                    if (L.stage <= 1) {
#pragma unroll
                        for (int k = 0; k < 3; ++k) L.p[k] += o.disp[k];
                        if (o.lim == 1) { if (down) advance = true; else fate = kLeak; }
                    } else {
                        if (o.lim == 1) {
                            bool out = false;
#pragma unroll
                            for (int k = 0; k < 3; ++k) {
                                const int sg = d_old[k] > 0.0f ? 1 : -1;
                                if (d_old[k] != 0.0f && dc[k] == o.s) L.ic[k] += sg;
                                if (d_old[k] != 0.0f && ds[k] == o.s) L.is[k] += sg;
                                out |= L.ic[k] < 0 || L.ic[k] >= P.ctg.n[k] || L.is[k] < 0 || L.is[k] >= P.sg.n[k];
                            }
                            if (out) fate = kLeak;
                        }
                        if (fate < 0) {
                            // lateral displacement, confined to the current voxel of both grids
#pragma unroll
                            for (int k = 0; k < 3; ++k) {
                                const float vlo = fmaxf(P.ctg.lo[k] + (float)L.ic[k] * P.ctg.d[k],
                                                        P.sg.lo[k] + (float)L.is[k] * P.sg.d[k]);
                                const float vhi = fminf(P.ctg.lo[k] + (float)(L.ic[k] + 1) * P.ctg.d[k],
                                                        P.sg.lo[k] + (float)(L.is[k] + 1) * P.sg.d[k]);
                                L.p[k] = fminf(fmaxf(L.p[k] + o.disp[k], vlo), vhi);
                            }
                        }
                    }
                }
            }
            // the single place where a history changes stage
            if (advance && fate < 0) fate = enter_next_stage(S, P, B, SC, L, from);
            // the single place where a history ends
            if (fate >= 0) {
                if (fate == kLeak || fate == kErr) acc_leak += __float2ull_rn(L.E * P.fscale);
                if (fate == kErr) { acc_err += 1; atomicOr(P.status, 1); }
                if (P.records && L.g < P.rec_cap) {
                    HistRecord r;
                    float pos[3] = {L.p[0], L.p[1], L.p[2]};
                    if (L.stage < 2) bev_to_patient(B, SC, L.p, pos);
                    r.q_dep = (long long)(acc_dep - L.qdep);
                    r.fate = fate;
                    r.steps = L.nsteps;
                    r.e_dep = (float)((double)(acc_dep - L.qdep) / (double)P.fscale);
                    r.e_end = (fate == kLeak || fate == kErr) ? L.E : 0.0f;
                    r.pos[0] = pos[0]; r.pos[1] = pos[1]; r.pos[2] = pos[2];
                    r.pad = 0.0f;
                    P.records[L.g] = r;
                }
                alive = false;
            }
        }
        // ---- scoring (all lanes together) ----
        if (P.aggregate) deposit_aggregated(P.scratch, dep_key, dep_q);
        else if (dep_key >= 0 && dep_q) atomicAdd(P.scratch + dep_key, dep_q);
    }

    // ---- per-warp totals ----
    unsigned long long v[kNStats] = {acc_dep, acc_leak, acc_rs, acc_ap, acc_nuc, acc_steps, acc_err};
#pragma unroll
    for (int k = 0; k < kNStats; ++k) {
        unsigned long long x = v[k];
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
        if (lane == 0 && x) atomicAdd(P.stats + k, x);
    }
}

size_t transport_smem_bytes() { return SharedLayout::Bytes; }

cudaError_t transport_func_attributes(int* regs, int* max_threads)
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, k_transport);
    if (e != cudaSuccess) return e;
    *regs = a.numRegs;
    *max_threads = a.maxThreadsPerBlock;
    return cudaSuccess;
}

cudaError_t launch_transport(const TransportParams& p, int grid, int block, cudaStream_t s)
{
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_transport, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)SharedLayout::Bytes);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    k_transport<<<grid, block, SharedLayout::Bytes, s>>>(p);
    return cudaGetLastError();
}

}  // namespace vpmc
