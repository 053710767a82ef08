// Device code shared by the transport kernels (beam-line devices and the
// voxelised patient): the condensed-history step, the interpolated tables,
// the lane state, the persistent work pool and the scoring primitives.
//
// Physics of one condensed-history step (same definition as the CPU oracle):
//   step = min(1 mm, 1 % energy-loss length, geometry limit, nuclear point);
//   mean loss from the residual range carried with the particle,
//   E' = E(R - s * kappa); Bohr straggling; Highland scattering with the PDG
//   correlated (angle, offset) pair in two planes; nuclear removal at
//   0.0012 / mm x density with the removed energy deposited locally.
// Random numbers: Philox4x32-10, key = (seed lo, spot ^ seed hi), counter =
// (history, step, slot, 0): slot 0 source (23-bit uniforms), slot 1 one
// condensed-history step (six 21-bit uniforms for scattering and
// straggling), slot 3 nuclear free path; the surrogate uses slots 4-6.
#pragma once

#include "device_common.cuh"
#include "vpmc_internal.cuh"

namespace vpmc {
namespace tr {

using namespace dev;

constexpr float kMp = 938.272f;

// Hardware square root (approximate, relative error about 2^-22), 0 for x <= 0.
__device__ __forceinline__ float sqrt_approx(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Box-Muller with hardware approximations (per-step physics).  u1 <= 1 - 2^-22,
// so -2 ln u1 > 0; the clamp only guards the approximate logarithm.
__device__ __forceinline__ float2 box_muller_fast(float u1, float u2)
{
    const float l = fmaxf(__log2f(u1) * -1.38629436111989061f, 0.0f);      // -2 ln u1
    const float r = sqrt_approx(l);
    float s, c;
    __sincosf(6.28318530717958647f * u2, &s, &c);
    return make_float2(r * c, r * s);
}

__device__ __forceinline__ float fast_sqrt(float x) { return sqrt_approx(fmaxf(x, 0.0f)); }

// Residual range R(E) by linear interpolation on the 0.1 MeV grid.  Each
// entry holds (R_k, R_{k+1} - R_k) (the last one a zero difference), so a
// lookup is one 8-byte load.  E >= 0 (energies only decrease, from at most
// 250 MeV); the index clamp keeps any other input inside the table.
__device__ __forceinline__ float range_of(const float2* __restrict__ R, float E)
{
    const float x = E * 10.0f;
    const unsigned i = min((unsigned)(int)x, (unsigned)(kNE - 1));
    const float2 v = R[i];
    return fmaf(x - (float)i, v.y, v.x);
}

// Energy E(R) on the uniform residual-range grid, R > 0 (entries as above).
__device__ __forceinline__ float energy_of(const float2* __restrict__ Et, float inv_dR, float R)
{
    const float x = R * inv_dR;
    const unsigned j = min((unsigned)(int)x, (unsigned)(kNR - 1));
    const float2 v = Et[j];
    return fmaf(x - (float)j, v.y, v.x);
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
    const float2* Rt;  // residual range table: (R_k, R_{k+1} - R_k)
    const float2* Et;  // energy table on the uniform range grid: (E_j, E_{j+1} - E_j)
    float inv_dR, kappa, rho, za, inv_x0;
};

struct StepResult {
    float s, dE;
    float disp[3];
    int lim;        // 0 none, 1 geometry, 2 nuclear
    int killed;     // 1 stopped, 2 nuclear
};

// State of the history a lane carries.
struct Lane {
    float p[3], d[3];
    float E, R, nlam;
    uint32_t step;  // condensed-history steps so far (RNG counter)
    uint32_t hist;  // history index within its spot
    int stage;      // devices: -1 just born, 0 range shifter, 1 aperture
    int forced;     // aperture: 1 the next step is in brass (after a wall hit), -1 on the entrance plane
    int ic[3], is[3];
    int item;
    int beam;       // the item's beam entry (kept so that each iteration reads it from a register)
    int iters;
    long long g;
    unsigned long long qdep;
};

// State of the history a patient lane carries.  Its global index and work
// item stay in shared memory: they are read only when the history ends.
struct PatientLane {
    float p[3], d[3];
    float E, R, nlam;
    uint32_t step;              // condensed-history steps so far (RNG counter)
    uint32_t hist;              // history index within its spot
    int iters;
    int ic[3], is[3];
    unsigned long long hdep;    // fixed-point energy the history deposited in the patient
};

// kAllPhysics: scattering, straggling and nuclear removal all on, known at
// compile time, so that the step carries none of their switches; otherwise
// the launch's switches decide.
template <bool kAllPhysics, class LaneT>
__device__ __forceinline__ void ch_step(const Medium& m, float s_geom, LaneT& L, const TransportParams& P, uint2 key,
                                        StepResult& o)
{
    const bool mcs = kAllPhysics || P.mcs, straggling = kAllPhysics || P.straggling,
               nuclear = kAllPhysics || P.nuclear;
    const float E = L.E;
    const float R0 = L.R;
    const float inv_kappa = __fdividef(1.0f, m.kappa);
    float s1 = (R0 - range_of(m.Rt, 0.99f * E)) * inv_kappa;
    if (!(s1 > 0.0f)) s1 = R0 * inv_kappa;
    const float mu = nuclear ? 0.0012f * m.rho : 0.0f;
    float s = 1.0f;
    int lim = 0;
    if (s1 < s) s = s1;
    if (s_geom < s) { s = s_geom; lim = 1; }
    // (with mu = 0 the quotient is +inf or NaN and never limits the step)
    if (kAllPhysics || mu > 0.0f) {
        const float sn = __fdividef(L.nlam, mu);
        if (sn < s) { s = sn; lim = 2; }
    }
    L.step += 1;
    if (lim == 2) L.nlam = 0.0f; else L.nlam -= mu * s;

    // random numbers of this step: one block, counter (history, step, 1, 0),
    // six 21-bit uniforms -- the top 21 bits of each word (scattering) and the
    // low bits of words 0|1 and 2|3 (straggling)
    uint4 r = make_uint4(L.hist, L.step, 1u, 0u);
    if (mcs || straggling) r = philox(r, key);

    const float R1 = R0 - s * m.kappa;
    // (looked up whatever the sign of R1, the index being clamped, so that the
    // step selects instead of branching)
    const float Eint = energy_of(m.Et, m.inv_dR, R1);
    const float Emean = R1 > 0.0f ? Eint : kEcut;
    float dE = E - Emean;
    const float pc2 = E * (E + 2.0f * kMp);               // (pc)^2
    const float etot = E + kMp;
    const float inv_etot = __fdividef(1.0f, etot);
    if (straggling) {
        // (1 - beta^2 / 2) / (1 - beta^2) = gamma^2 - (beta gamma)^2 / 2 = (Etot^2 - (pc)^2 / 2) / Mp^2
        const float2 z = box_muller_fast(u21(((r.x & 0x7FFu) << 10) | (r.y & 0x3FFu)),
                                         u21(((r.z & 0x7FFu) << 10) | (r.w & 0x3FFu)));
        const float rel = fmaf(etot, etot, -0.5f * pc2) * (0.01569f / (kMp * kMp));
        const float var = m.rho * m.za * s * rel;
        dE += fast_sqrt(var) * z.x;
    }
    dE = fminf(fmaxf(dE, 0.0f), E);
    const float Enew = E - dE;
    float Rnew = R1;
    if (straggling) {
        Rnew = R1 + (range_of(m.Rt, Enew) - range_of(m.Rt, Emean));
        if (!(Rnew > 0.0f)) Rnew = range_of(m.Rt, Enew);
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

    // (also on the step that ends the history: the new direction and offset
    // are then never read, and the step needs no branch around this block)
    if (mcs) {
        const float x = s * m.rho * m.inv_x0;
        // 1 + 0.038 ln x = 1 + (0.038 ln 2) log2 x; evaluated for any x and
        // selected (a NaN or infinity at x ~ 0 is discarded), without a branch
        const float th0v = __fdividef(13.6f, pc2 * inv_etot) * fast_sqrt(x) * fmaf(0.02633959f, __log2f(x), 1.0f);
        const float th0 = x >= 1e-6f ? th0v : 0.0f;
        const float2 za = box_muller_fast(u21(r.x >> 11), u21(r.y >> 11));
        const float2 zb = box_muller_fast(u21(r.z >> 11), u21(r.w >> 11));
        const float th1 = za.y * th0, th2 = zb.y * th0;
        const float dx1 = s * th0 * fmaf(za.x, 0.28867513459481287f, 0.5f * za.y);
        const float dx2 = s * th0 * fmaf(zb.x, 0.28867513459481287f, 0.5f * zb.y);
        float e1[3], e2[3];
        orthonormal_basis(L.d, e1, e2);
        // deflection by theta = |(th1, th2)|: cos(theta) and sin(theta)/theta.
        // Up to theta^2 = 0.09 their Taylor series in theta^2, cut after the
        // theta^6 terms, are exact to a few 1e-9 -- below FP32 rounding
        // (almost every step: theta0 is a few mrad); beyond, the functions
        const float t = fmaf(th1, th1, th2 * th2);
        float c, sc;
        if (t <= 0.09f) {
            c = fmaf(t, fmaf(t, fmaf(t, -1.0f / 720.0f, 1.0f / 24.0f), -0.5f), 1.0f);
            sc = fmaf(t, fmaf(t, fmaf(t, -1.0f / 5040.0f, 1.0f / 120.0f), -1.0f / 6.0f), 1.0f);
        } else {
            const float th = sqrt_approx(t);
            float sn;
            __sincosf(th, &sn, &c);
            sc = __fdividef(sn, th);
        }
        float nd[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            o.disp[k] = dx1 * e1[k] + dx2 * e2[k];
            nd[k] = c * L.d[k] + sc * (th1 * e1[k] + th2 * e2[k]);
        }
        // |nd| = 1 to rounding: one Newton step of 1/sqrt(n2) from 1 renormalises
        const float n2 = fmaf(nd[0], nd[0], fmaf(nd[1], nd[1], nd[2] * nd[2]));
        const float inv = fmaf(-0.5f, n2, 1.5f);
#pragma unroll
        for (int k = 0; k < 3; ++k) L.d[k] = nd[k] * inv;
    }
}

// Fixed-point value round-half-even(e * scale) of an energy.  Below 2^32 (any
// energy up to 250 MeV at scales up to 2^24) the 32-bit conversion gives the
// same integer as the 64-bit one, which would occupy the FP64 pipe.
__device__ __forceinline__ unsigned long long to_fixed(float e, float scale, bool fits32)
{
    return fits32 ? (unsigned long long)__float2uint_rn(e * scale) : __float2ull_rn(e * scale);
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

// Warp-uniform pool of work indices [pool_next, pool_end) taken from a global
// counter in chunks.  Returns false once the work (or the launch) has ended.
struct WorkPool {
    long long next = 0, end = 0;
    __device__ __forceinline__ bool refill(const TransportParams& P, long long begin, long long total, int lane)
    {
        unsigned long long base = 0;
        int abort = 0;
        if (lane == 0) {
            base = atomicAdd(P.counter, (unsigned long long)P.chunk);
            abort = *reinterpret_cast<volatile int*>(P.status);   // a latched error ends the launch early
        }
        base = __shfl_sync(kFull, base, 0);
        abort = __shfl_sync(kFull, abort, 0);
        const long long b = begin + (long long)base;
        if (abort || b >= total) return false;
        next = b;
        end = min(b + P.chunk, total);
        return true;
    }
};

__device__ __forceinline__ void put_record(const TransportParams& P, long long g, int fate, uint32_t steps,
                                           unsigned long long q, float e, const float pos[3])
{
    HistRecord r;
    r.q_dep = (long long)q;
    r.fate = fate;
    r.steps = (int)steps;
    r.e_dep = (float)((double)q / (double)P.fscale);
    r.e_end = (fate == kLeak || fate == kErr) ? e : 0.0f;
    r.pos[0] = pos[0]; r.pos[1] = pos[1]; r.pos[2] = pos[2];
    r.pad = 0.0f;
    P.records[g] = r;
}

__device__ __forceinline__ void write_record(const TransportParams& P, const Lane& L, int fate, const float pos[3],
                                             unsigned long long acc_dep)
{
    put_record(P, L.g, fate, L.step, acc_dep - L.qdep, L.E, pos);
}

__device__ __forceinline__ void warp_add_stats(const TransportParams& P, unsigned long long (&v)[kNStats], int lane)
{
#pragma unroll
    for (int k = 0; k < kNStats; ++k) {
        unsigned long long x = v[k];
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
        if (lane == 0 && x) atomicAdd(P.stats + k, x);
    }
}

}  // namespace tr
}  // namespace vpmc
