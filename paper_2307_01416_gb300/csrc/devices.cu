// Persistent transport kernels of the beam-line devices for sm_103a.
//
// One history per thread (paper Sec. 2.A: every history follows one identical
// model, so no secondary particles are spawned).  Warps are persistent: a warp
// takes chunks of consecutive work indices from one counter and hands them to
// lanes whose history has ended, so dead lanes are refilled at once.
// Transport runs in three kernels so that the lanes of a warp execute the same
// geometry, each handing its survivors' phase space to the next:
// k_source_rs samples the source and carries each history through the
// optional range shifter; k_aperture takes it through the brass aperture
// (Sec. 2.B: at every step inside the aperture slab a crossing-number test
// decides opening -> straight flight, or brass -> condensed-history step with
// brass physics); k_patient (patient.cu) transports it through the voxelised
// patient.  Each kernel is compiled twice: with the physics switches read
// from the launch, and with full physics known at compile time.
#include "transport_common.cuh"

namespace vpmc {
namespace {

using namespace dev;
using namespace tr;

// Lower bound of the distance from (a, b) to the polygon boundary from the
// raster (0 outside it or in a cell an edge passes through).
__device__ __forceinline__ float wall_lower_bound(const DevBeam& B, const float* __restrict__ lower, float a, float b)
{
    const float fx = (a - B.ras_lo[0]) * B.ras_inv[0];
    const float fy = (b - B.ras_lo[1]) * B.ras_inv[1];
    if (!(fx >= 0.0f && fx < (float)kRaster && fy >= 0.0f && fy < (float)kRaster)) return 0.0f;
    return __ldg(lower + B.ras_off + (int)fy * kRaster + (int)fx);
}

// ---- warp-cooperative exact polygon queries --------------------------------
// Lanes that need an exact test post a request; the converged warp then serves
// the requests one by one, each lane evaluating every 32nd edge with the same
// per-edge arithmetic as a serial loop, and the warp reduces the results.
// Every lane of the warp must call these (need = false for non-requesters).

// Raster class of (a, b): 0 outside the opening, 1 inside, 2 near an edge.
__device__ __forceinline__ int raster_class(const DevBeam& B, const unsigned char* __restrict__ raster, float a, float b)
{
    const float fx = (a - B.ras_lo[0]) * B.ras_inv[0];
    const float fy = (b - B.ras_lo[1]) * B.ras_inv[1];
    if (!(fx >= 0.0f && fx < (float)kRaster && fy >= 0.0f && fy < (float)kRaster)) return 0;
    return __ldg(raster + B.ras_off + (int)fy * kRaster + (int)fx);
}

// Crossing number (half-open edge rule) of the requesting lane's point.
__device__ __forceinline__ bool coop_point_in_polygon(bool need, float x, float y, const float2* __restrict__ poly,
                                                      int off, int n, int lane)
{
    bool result = false;
    unsigned m = __ballot_sync(kFull, need);
    while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1u;
        const float qx = __shfl_sync(kFull, x, src), qy = __shfl_sync(kFull, y, src);
        const int qo = __shfl_sync(kFull, off, src), qn = __shfl_sync(kFull, n, src);
        bool c = false;
        for (int i = lane; i < qn; i += 32) {
            const float2 pi = poly[qo + i];
            const float2 pj = poly[qo + (i == 0 ? qn - 1 : i - 1)];
            if ((pi.y > qy) != (pj.y > qy)) {
                const float xc = pi.x + (qy - pi.y) * (pj.x - pi.x) / (pj.y - pi.y);
                if (qx < xc) c = !c;
            }
        }
        const bool in = (__popc(__ballot_sync(kFull, c)) & 1) != 0;
        if (lane == src) result = in;
    }
    return result;
}

__device__ __forceinline__ float warp_min(float v)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v = fminf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

// Smallest s > 0 at which the requester's ray (x, y) + s (dx, dy) crosses an edge.
__device__ __forceinline__ float coop_first_wall_hit(bool need, float x, float y, float dx, float dy,
                                                     const float2* __restrict__ poly, int off, int n, int lane)
{
    float result = __int_as_float(0x7f800000);
    unsigned m = __ballot_sync(kFull, need);
    while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1u;
        const float qx = __shfl_sync(kFull, x, src), qy = __shfl_sync(kFull, y, src);
        const float qdx = __shfl_sync(kFull, dx, src), qdy = __shfl_sync(kFull, dy, src);
        const int qo = __shfl_sync(kFull, off, src), qn = __shfl_sync(kFull, n, src);
        float best = __int_as_float(0x7f800000);
        for (int i = lane; i < qn; i += 32) {
            const float2 a = poly[qo + i];
            const float2 b = poly[qo + (i + 1 < qn ? i + 1 : 0)];
            const float ex = b.x - a.x, ey = b.y - a.y;
            const float den = qdx * ey - qdy * ex;
            if (den == 0.0f) continue;
            const float wx = a.x - qx, wy = a.y - qy;
            const float sh = (wx * ey - wy * ex) / den;
            const float lam = (wx * qdy - wy * qdx) / den;
            if (sh > 0.0f && lam >= 0.0f && lam <= 1.0f && sh < best) best = sh;
        }
        best = warp_min(best);
        if (lane == src) result = best;
    }
    return result;
}

// Distance from the requester's point to the polygon boundary.
__device__ __forceinline__ float coop_wall_distance(bool need, float x, float y, const float2* __restrict__ poly,
                                                    int off, int n, int lane)
{
    float result = 0.0f;
    unsigned m = __ballot_sync(kFull, need);
    while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1u;
        const float qx = __shfl_sync(kFull, x, src), qy = __shfl_sync(kFull, y, src);
        const int qo = __shfl_sync(kFull, off, src), qn = __shfl_sync(kFull, n, src);
        float best = __int_as_float(0x7f800000);
        for (int i = lane; i < qn; i += 32) {
            const float2 a = poly[qo + i];
            const float2 b = poly[qo + (i + 1 < qn ? i + 1 : 0)];
            const float ex = b.x - a.x, ey = b.y - a.y;
            float t = __fdividef((qx - a.x) * ex + (qy - a.y) * ey, ex * ex + ey * ey);
            t = fminf(fmaxf(t, 0.0f), 1.0f);
            const float ddx = a.x + t * ex - qx, ddy = a.y + t * ey - qy;
            best = fminf(best, ddx * ddx + ddy * ddy);
        }
        best = warp_min(best);
        if (lane == src) result = sqrtf(best);
    }
    return result;
}

// Nearest boundary point of the requester's (x, y): (distance, nearest x,
// nearest y, curvature there).  Ties between edges go to the lower edge index;
// the curvature is interpolated along the nearest edge between its vertices'
// curvatures, so either of two equidistant edges gives the same value.
__device__ __forceinline__ float4 coop_nearest_edge(bool need, float x, float y, const float2* __restrict__ poly,
                                                    const float* __restrict__ kappa, int off, int n, int lane)
{
    // Returns (distance, p - q, curvature at q) for the nearest boundary point
    // q of the query p.  Every difference is taken between nearby points
    // (a - p, b - a: exact when within a factor two), never as a + t e at the
    // opening's radius: near the corner between an edge region and a vertex
    // region two candidates' distances can differ by ~1e-7 mm, below the
    // rounding of a coordinate of tens of mm.
    float4 result = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    unsigned m = __ballot_sync(kFull, need);
    while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1u;
        const float qx = __shfl_sync(kFull, x, src), qy = __shfl_sync(kFull, y, src);
        const int qo = __shfl_sync(kFull, off, src), qn = __shfl_sync(kFull, n, src);
        float best = __int_as_float(0x7f800000), bt = 0.0f;
        int bi = 0x7fffffff;
        for (int i = lane; i < qn; i += 32) {
            const float2 a = poly[qo + i];
            const float2 b = poly[qo + (i + 1 < qn ? i + 1 : 0)];
            const float ex = b.x - a.x, ey = b.y - a.y;
            const float ax = a.x - qx, ay = a.y - qy;
            float t = -(ax * ex + ay * ey) / (ex * ex + ey * ey);
            t = fminf(fmaxf(t, 0.0f), 1.0f);
            const float ddx = fmaf(t, ex, ax), ddy = fmaf(t, ey, ay);
            const float d2 = ddx * ddx + ddy * ddy;
            if (d2 < best) { best = d2; bi = i; bt = t; }
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            const float ob = __shfl_xor_sync(kFull, best, o);
            const int oi = __shfl_xor_sync(kFull, bi, o);
            const float ot = __shfl_xor_sync(kFull, bt, o);
            if (ob < best || (ob == best && oi < bi)) { best = ob; bi = oi; bt = ot; }
        }
        if (lane == src && bi < qn) {
            const int bj = bi + 1 < qn ? bi + 1 : 0;
            const float2 a = poly[qo + bi], b = poly[qo + bj];
            const float k0 = __ldg(kappa + qo + bi), k1 = __ldg(kappa + qo + bj);
            result = make_float4(sqrtf(best), -fmaf(bt, b.x - a.x, a.x - qx), -fmaf(bt, b.y - a.y, a.y - qy),
                                 fmaf(bt, k1 - k0, k0));
        }
    }
    return result;
}

}  // namespace

// ============================================================================
// Source and range shifter.
// ============================================================================
// Samples each history's source state (slot 0 of its stream) and carries it
// through the optional range shifter, a homogeneous PMMA slab of finite
// radius: outside the radius a proton flies straight to the slab's exit plane.
// Survivors go to the aperture kernel in the beam's-eye frame.  Every lane of
// a warp runs the same slab step, so the warps stay converged.
template <bool kAllPhysics>
__global__ void __launch_bounds__(768, 1) k_source_rs(const TransportParams P)
{
    extern __shared__ __align__(16) unsigned char smem[];
    {
        float2* R = reinterpret_cast<float2*>(smem + SourceSmem::R);
        float2* Et = reinterpret_cast<float2*>(smem + SourceSmem::Einv);
        for (int i = threadIdx.x; i < kNEPad; i += blockDim.x) R[i] = P.tables->R[kPMMA][i];
        for (int i = threadIdx.x; i < kNR; i += blockDim.x) Et[i] = P.tables->Einv[kPMMA][i];
        MatConst* mt = reinterpret_cast<MatConst*>(smem + SourceSmem::Mat);
        if (threadIdx.x < kNMat) mt[threadIdx.x] = P.tables->mat[threadIdx.x];
        DevBeam* bm = reinterpret_cast<DevBeam*>(smem + SourceSmem::Beams);
        for (int i = threadIdx.x; i < P.n_beams; i += blockDim.x) bm[i] = P.beams[i];
    }
    __syncthreads();
    const MatConst* mat = reinterpret_cast<const MatConst*>(smem + SourceSmem::Mat);
    const DevBeam* beams = reinterpret_cast<const DevBeam*>(smem + SourceSmem::Beams);
    Medium pmma;
    pmma.Rt = reinterpret_cast<const float2*>(smem + SourceSmem::R);
    pmma.Et = reinterpret_cast<const float2*>(smem + SourceSmem::Einv);
    pmma.inv_dR = mat[kPMMA].inv_dR; pmma.kappa = mat[kPMMA].rho;
    pmma.rho = mat[kPMMA].rho; pmma.za = mat[kPMMA].za; pmma.inv_x0 = mat[kPMMA].inv_x0;

    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    WorkPool pool;
    int pool_item = 0;
    bool alive = false, done = false;
    Lane L;
    L.item = 0; L.beam = 0; L.g = 0; L.hist = 0; L.qdep = 0ull; L.iters = 0; L.stage = 0; L.forced = 0;
    L.step = 0; L.E = 0.0f; L.R = 0.0f; L.nlam = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) { L.p[k] = 0.0f; L.d[k] = 0.0f; }
    unsigned long long acc_leak = 0, acc_rs = 0, acc_nuc = 0, acc_steps = 0, acc_err = 0;
    uint2 key = make_uint2(0u, 0u);

    for (;;) {
        // ---- new histories for lanes whose history has ended ----
        unsigned need = __ballot_sync(kFull, !alive && !done);
        while (need) {
            if (pool.next >= pool.end) {
                if (!pool.refill(P, P.hist_begin, P.total, lane)) {
                    if (!alive) done = true;
                    break;
                }
                pool_item = find_item_warp(P.items, P.n_items, pool.next, lane);
            }
            const int take = (int)min((long long)__popc(need), pool.end - pool.next);
            const bool mine = ((need >> lane) & 1u) && __popc(need & lt_mask) < take;
            if (mine) {
                const long long g = pool.next + __popc(need & lt_mask);
                int it = pool_item;
                while (it + 1 < P.n_items && __ldg(&P.items[it + 1].hist_off) <= g) ++it;
                const DevItem I = P.items[it];
                const DevBeam& B = beams[I.beam];
                L.item = it;
                L.beam = I.beam;
                L.g = g;
                L.hist = (uint32_t)(g - I.hist_off);
                L.step = 0;
                L.iters = 0;
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
                if (kAllPhysics || P.nuclear) {
                    const uint4 y = philox(make_uint4(L.hist, 0u, 3u, 0u), key);
                    L.nlam = -logf(u01(y.x));
                } else {
                    L.nlam = __int_as_float(0x7f800000);
                }
                L.stage = -1;                       // enters the slab (if any) in the next iteration
                alive = true;
            }
            pool.next += take;
            need = __ballot_sync(kFull, !alive && !done);
        }
        if (!__any_sync(kFull, alive)) {
            if (__all_sync(kFull, done || alive)) break;
            continue;
        }

        // ---- one iteration of every live history ----
        bool handoff = false;
        int fate = -1;
        if (alive) {
            const DevBeam& B = beams[L.beam];
            if (++L.iters > P.max_iter) {
                fate = kErr;
            } else if (L.stage < 0) {
                if (B.rs) {
                    const float sdr = __fdividef(B.rs_tup - L.p[2], L.d[2]);
#pragma unroll
                    for (int k = 0; k < 3; ++k) L.p[k] = fmaf(sdr, L.d[k], L.p[k]);
                    L.R = range_of(pmma.Rt, L.E);
                    L.stage = 0;
                } else {
                    handoff = true;                 // no range shifter
                }
            } else if (L.p[0] * L.p[0] + L.p[1] * L.p[1] > B.rs_r2) {
                // outside the slab's radius: straight flight to its exit plane
                if (!(L.d[2] > 0.0f)) fate = kLeak;
                else {
                    const float sf = __fdividef(B.rs_tdn - L.p[2], L.d[2]);
#pragma unroll
                    for (int k = 0; k < 3; ++k) L.p[k] = fmaf(sf, L.d[k], L.p[k]);
                    handoff = true;
                }
            } else {
                float s_geom = __int_as_float(0x7f800000);
                bool down = true;
                if (L.d[2] > 0.0f) s_geom = __fdividef(B.rs_tdn - L.p[2], L.d[2]);
                else if (L.d[2] < 0.0f) { s_geom = __fdividef(B.rs_tup - L.p[2], L.d[2]); down = false; }
                s_geom = fmaxf(s_geom, 0.0f);       // scattering offsets can leave it past the plane
                StepResult o;
                ch_step<kAllPhysics>(pmma, s_geom, L, P, key, o);
                acc_steps += 1;
                const unsigned long long qs = to_fixed(o.dE, P.fscale, P.fx32);
                acc_rs += qs;
                if (o.killed) {
                    if (o.killed == 2) acc_nuc += qs;
                    fate = kAbsRS;
                } else {
#pragma unroll
                    for (int k = 0; k < 3; ++k) L.p[k] += o.disp[k];
                    if (o.lim == 1) { if (down) handoff = true; else fate = kLeak; }
                }
            }
            if (fate >= 0) {
                if (fate == kLeak || fate == kErr) acc_leak += to_fixed(L.E, P.fscale, P.fx32);
                if (fate == kErr) { acc_err += 1; atomicOr(P.status, 1); }
                if (P.records && L.g < P.rec_cap) {
                    float pos[3];
                    bev_to_patient(B, P.scens[__ldg(&P.items[L.item].scen)], L.p, pos);
                    write_record(P, L, fate, pos, 0ull);
                }
                alive = false;
            }
        }
        // ---- hand-off to the aperture kernel (one atomic per warp) ----
        const unsigned hmask = __ballot_sync(kFull, handoff);
        if (hmask) {
            unsigned long long base = 0;
            const int leader = __ffs(hmask) - 1;
            if (lane == leader) base = atomicAdd(P.mid_count, (unsigned long long)__popc(hmask));
            base = __shfl_sync(kFull, base, leader);
            if (handoff) {
                const long long slot = (long long)base + __popc(hmask & lt_mask);
                if (slot < P.mid_cap) {
                    PhaseRec r;
#pragma unroll
                    for (int k = 0; k < 3; ++k) { r.p[k] = L.p[k]; r.d[k] = L.d[k]; }
                    r.E = L.E;
                    r.nlam = L.nlam;
                    r.step = L.step;
                    r.item = L.item;
                    r.g = L.g;
                    P.mid[slot] = r;
                } else {
                    atomicOr(P.status, 2);          // hand-off buffer too small (host sizes it to the batch)
                }
                alive = false;
            }
        }
    }
    // energies and errors count once per scenario sharing the transport; steps as taken
    const unsigned long long nr = (unsigned long long)P.n_rep;
    unsigned long long v[kNStats] = {0ull, acc_leak * nr, acc_rs * nr, 0ull, acc_nuc * nr, acc_steps, acc_err * nr,
                                     acc_steps, 0ull};
    warp_add_stats(P, v, lane);
}

// ============================================================================
// Aperture block.
// ============================================================================
// Takes the histories the source kernel hands over (or, for training tracks,
// births them on the block's entrance plane) through the aperture block and
// hands the survivors to the patient kernel.
// kMode bit 0: brass entries in the surrogate's domain become queries;
// bit 1: training tracks (histories start on the aperture entrance plane and
// record the surrogate's inputs and targets).
template <int kMode, bool kAllPhysics>
__global__ void __launch_bounds__(640, 1) k_aperture(const TransportParams P)
{
    constexpr bool kSur = (kMode & 1) != 0;
    constexpr bool kTrack = (kMode & 2) != 0;
    extern __shared__ __align__(16) unsigned char smem[];
    {
        // brass rows of the tables, material constants, beams, scenarios, polygons
        float2* R = reinterpret_cast<float2*>(smem + ApertureSmem::R);
        float2* Et = reinterpret_cast<float2*>(smem + ApertureSmem::Einv);
        for (int i = threadIdx.x; i < kNEPad; i += blockDim.x) R[i] = P.tables->R[kBrass][i];
        for (int i = threadIdx.x; i < kNR; i += blockDim.x) Et[i] = P.tables->Einv[kBrass][i];
        MatConst* mt = reinterpret_cast<MatConst*>(smem + ApertureSmem::Mat);
        if (threadIdx.x < kNMat) mt[threadIdx.x] = P.tables->mat[threadIdx.x];
        DevBeam* bm = reinterpret_cast<DevBeam*>(smem + ApertureSmem::Beams);
        for (int i = threadIdx.x; i < P.n_beams; i += blockDim.x) bm[i] = P.beams[i];
        DevScen* sc = reinterpret_cast<DevScen*>(smem + ApertureSmem::Scens);
        for (int i = threadIdx.x; i < P.n_scen; i += blockDim.x) sc[i] = P.scens[i];
        float2* pl = reinterpret_cast<float2*>(smem + ApertureSmem::Poly);
        for (int i = threadIdx.x; i < P.n_poly; i += blockDim.x) pl[i] = P.poly[i];
    }
    __syncthreads();
    const MatConst* mat = reinterpret_cast<const MatConst*>(smem + ApertureSmem::Mat);
    const DevBeam* beams = reinterpret_cast<const DevBeam*>(smem + ApertureSmem::Beams);
    const DevScen* scens = reinterpret_cast<const DevScen*>(smem + ApertureSmem::Scens);
    const float2* poly = reinterpret_cast<const float2*>(smem + ApertureSmem::Poly);
    Medium brass;
    brass.Rt = reinterpret_cast<const float2*>(smem + ApertureSmem::R);
    brass.Et = reinterpret_cast<const float2*>(smem + ApertureSmem::Einv);
    brass.inv_dR = mat[kBrass].inv_dR; brass.kappa = mat[kBrass].rho;
    brass.rho = mat[kBrass].rho; brass.za = mat[kBrass].za; brass.inv_x0 = mat[kBrass].inv_x0;
    // histories handed over by the source kernel (training tracks: born here)
    const long long n_in = kTrack ? P.total : min((long long)*P.mid_count, P.mid_cap);

    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    WorkPool pool;
    int pool_item = 0;
    bool alive = false, done = false;
    Lane L;
    L.item = 0; L.beam = 0; L.g = 0; L.hist = 0; L.qdep = 0ull; L.iters = 0; L.stage = 0; L.forced = 0;
    L.step = 0; L.E = 0.0f; L.R = 0.0f; L.nlam = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) { L.p[k] = 0.0f; L.d[k] = 0.0f; }
    unsigned long long acc_leak = 0, acc_ap = 0, acc_nuc = 0, acc_steps = 0, acc_err = 0;
    uint2 key = make_uint2(0u, 0u);

    for (;;) {
        // ---- new histories for lanes whose history has ended ----
        unsigned need = __ballot_sync(kFull, !alive && !done);
        while (need) {
            if (pool.next >= pool.end) {
                if (!pool.refill(P, kTrack ? P.hist_begin : 0ll, n_in, lane)) {
                    if (!alive) done = true;
                    break;
                }
                if (kTrack) pool_item = find_item_warp(P.items, P.n_items, pool.next, lane);
            }
            const int take = (int)min((long long)__popc(need), pool.end - pool.next);
            const bool mine = ((need >> lane) & 1u) && __popc(need & lt_mask) < take;
            if (mine) {
                const long long g = pool.next + __popc(need & lt_mask);
                if (kTrack) {
                    int it = pool_item;
                    while (it + 1 < P.n_items && __ldg(&P.items[it + 1].hist_off) <= g) ++it;
                    const DevItem I = P.items[it];
                    const DevBeam& B = beams[I.beam];
                    L.item = it;
                    L.beam = I.beam;
                    L.g = g;
                    L.hist = (uint32_t)(g - I.hist_off);
                    L.step = 0;
                    L.iters = 0;
                    key = make_uint2(P.key0, P.key1_hi ^ (uint32_t)I.spot);
                    {
                        // training track: born on the aperture's entrance plane near
                        // the opening (slot 0: energy, angle, edge distance; slot 5:
                        // incidence angles along the radial and tangential directions)
                        const uint4 x = philox(make_uint4(L.hist, 0u, 0u, 0u), key);
                        const float E = fmaf(sur::kEHi - sur::kELo, u01(x.x), sur::kELo);
                        float sph, cph;
                        sincospif(2.0f * u01(x.y), &sph, &cph);
                        const float r12 = 1.2f * range_of(brass.Rt, E) / brass.rho;
                        const float dhi = r12 < B.ap_tdn - B.ap_tup ? fminf(sur::kDCap, r12) : sur::kDCap;
                        const float uz = u01(x.z);
                        const float rr = fmaf(dhi * uz, uz, B.r_circ);   // d = d_hi u^2: denser near the edge
                        const uint4 a = philox(make_uint4(L.hist, 0u, 5u, 0u), key);
                        const float2 zz = box_muller(u01(a.x), u01(a.y));
                        const float tn = fminf(fmaxf(sur::kAngSigma * zz.x, -sur::kAngMax), sur::kAngMax);
                        const float tt = fminf(fmaxf(sur::kAngSigma * zz.y, -sur::kAngMax), sur::kAngMax);
                        L.d[0] = tn * cph - tt * sph;
                        L.d[1] = tn * sph + tt * cph;
                        L.d[2] = sqrtf(1.0f - tn * tn - tt * tt);
                        L.p[0] = rr * cph; L.p[1] = rr * sph; L.p[2] = B.ap_tup;
                        L.E = E;
                    }
                    if (kAllPhysics || P.nuclear) {
                        const uint4 y = philox(make_uint4(L.hist, 0u, 3u, 0u), key);
                        L.nlam = -logf(u01(y.x));
                    } else {
                        L.nlam = __int_as_float(0x7f800000);
                    }
                } else {
                    const PhaseRec r = P.mid[g];
                    const DevItem I = P.items[r.item];
                    L.item = r.item;
                    L.beam = I.beam;
                    L.g = r.g;
                    L.hist = (uint32_t)(r.g - I.hist_off);
                    L.step = r.step;
                    L.iters = 0;
                    key = make_uint2(P.key0, P.key1_hi ^ (uint32_t)I.spot);
#pragma unroll
                    for (int k = 0; k < 3; ++k) { L.p[k] = r.p[k]; L.d[k] = r.d[k]; }
                    L.E = r.E;
                    L.nlam = r.nlam;
                }
                L.stage = -1;                       // enters the block (if any) in the next iteration
                alive = true;
            }
            pool.next += take;
            need = __ballot_sync(kFull, !alive && !done);
        }
        if (!__any_sync(kFull, alive)) {
            if (__all_sync(kFull, done || alive)) break;
            continue;
        }

        // ---- one iteration of every live history ----
        bool handoff = false;
        int fate = -1;
        bool advance = false;
        Medium m;
        bool do_ch = false;
        float s_geom = __int_as_float(0x7f800000);
        bool down = true;
        bool ap_pending = false, was_forced = false, at_entry = false, need_pip = false;
        int cls = 0, q_off = 0, q_n = 0;
        // opening coordinates: the point projected from the virtual source onto
        // the downstream face (divergent walls; the point itself for parallel
        // walls) and the opening's scale at the point's depth
        float pu = 0.0f, pv = 0.0f, sc = 1.0f;
        if (alive) {
            const DevBeam& B = beams[L.beam];
            if (++L.iters > P.max_iter) {
                fate = kErr;
            } else if (L.stage < 0) {
                advance = true;
            } else {
                // ---- aperture block: geometry needing exact polygon tests is
                // requested here and served below by the whole warp ----
                if (L.d[2] > 0.0f) s_geom = __fdividef(B.ap_tdn - L.p[2], L.d[2]);
                else if (L.d[2] < 0.0f) { s_geom = __fdividef(B.ap_tup - L.p[2], L.d[2]); down = false; }
                s_geom = fmaxf(s_geom, 0.0f);       // scattering offsets can leave it past the plane
                ap_pending = true;
                was_forced = L.forced > 0;
                at_entry = L.forced < 0;
                pu = L.p[0];
                pv = L.p[1];
                if (B.ap_sad > 0.0f) {
                    sc = (L.p[2] + B.ap_sad) / B.ap_K;
                    const float inv = 1.0f / sc;
                    pu *= inv;
                    pv *= inv;
                }
                cls = was_forced ? 0 : raster_class(B, P.raster, pu, pv);
                need_pip = cls == 2;
                q_off = B.poly_off;
                q_n = B.nvert;
            }
        }
        // ---- exact opening test for lanes near an edge (warp-cooperative) ----
        const bool pip_in = coop_point_in_polygon(need_pip, pu, pv, poly, q_off, q_n, lane);
        bool open = false, need_hit = false, need_dist = false, absorb = false;
        float rmax = 0.0f;
        // flight direction in opening coordinates: along p + s d the projected
        // point moves as q(0) + g(s) (hx, hy) with g(s) = s c / (c + s d_t),
        // c = t + sad (parallel walls: g = s and (hx, hy) = d_xy)
        float hx = L.d[0], hy = L.d[1], cdiv = 0.0f;
        if (ap_pending) {
            const DevBeam& B = beams[L.beam];
            open = cls == 1 || (cls == 2 && pip_in);
            if (open) {
                float g_exit = s_geom;
                if (B.ap_sad > 0.0f) {
                    cdiv = L.p[2] + B.ap_sad;
                    const float f = B.ap_K / (cdiv * cdiv);
                    hx = f * (L.d[0] * cdiv - L.p[0] * L.d[2]);
                    hy = f * (L.d[1] * cdiv - L.p[1] * L.d[2]);
                    g_exit = s_geom * cdiv / (cdiv + s_geom * L.d[2]);
                }
                // a flight whose lateral travel (opening coordinates) stays below the
                // wall-distance bound of its start cell cannot meet a wall
                const float lat = g_exit * sqrtf(hx * hx + hy * hy);
                need_hit = !(lat < wall_lower_bound(B, P.raster_lb, pu, pv));
            } else if (P.range_rejection && !was_forced) {
                // a proton whose longest possible remaining path (1.2 x its residual
                // CSDA range) cannot reach the opening or a face of the block is
                // absorbed now -- its energy stays in the brass either way
                rmax = 1.2f * L.R * __fdividef(1.0f, brass.rho);
                const float dpl = fminf(L.p[2] - B.ap_tup, B.ap_tdn - L.p[2]);
                if (rmax < dpl) {
                    const float fx = (pu - B.ras_lo[0]) * B.ras_inv[0];
                    const float fy = (pv - B.ras_lo[1]) * B.ras_inv[1];
                    if (!(fx >= 0.0f && fx < (float)kRaster && fy >= 0.0f && fy < (float)kRaster)) {
                        absorb = true;              // beyond the raster: farther than half the thickness
                    } else {
                        // real distances: opening-coordinate ones x scale x cos(largest tilt)
                        const float to_real = sc * B.ap_cos;
                        const float lb = __ldg(P.raster_lb + B.ras_off + (int)fy * kRaster + (int)fx) * to_real;
                        if (rmax < lb) absorb = true;
                        else if (rmax < lb + B.ras_diag * to_real) need_dist = true;
                    }
                }
            }
        }
        // ---- brass entry: edge frame and surrogate inputs (warp-cooperative) ----
        // training tracks record their inputs at birth whatever the opening
        // test says (a start that rounds onto the opening's boundary can test
        // inside); the surrogate draws only for brass entries
        const bool entry_q = ap_pending && at_entry && (kTrack || (kSur && !open));
        const float4 ne = coop_nearest_edge(entry_q, L.p[0], L.p[1], poly, P.poly_kappa, q_off, q_n, lane);
        bool sur_emit = false;
        float feat[6], fnx = 0.0f, fny = 0.0f;
        if (entry_q) {
            const DevBeam& B = beams[L.beam];
            const float T = B.ap_tdn - B.ap_tup;
            const float dist = ne.x;
            const float inv = dist > 0.0f ? 1.0f / dist : 0.0f;
            fnx = ne.y * inv;
            fny = ne.z * inv;
            const float un = L.d[0] * fnx + L.d[1] * fny, ut = L.d[1] * fnx - L.d[0] * fny;
            const float rmm = L.R / brass.rho;
            feat[0] = fminf(dist, sur::kDCap) * (2.0f / sur::kDCap) - 1.0f;
            feat[1] = (L.E - 0.5f * (sur::kELo + sur::kEHi)) * (2.0f / (sur::kEHi - sur::kELo));
            feat[2] = un * (1.0f / sur::kAngSigma);
            feat[3] = ut * (1.0f / sur::kAngSigma);
            feat[4] = fmaf(8.0f, ne.w, -1.0f);
            feat[5] = rmm / T - 1.0f;
            if (kTrack && L.g < P.total) {
#pragma unroll
                for (int k = 0; k < 6; ++k) P.trk_feat[6 * L.g + k] = feat[k];
                float* fr = P.trk_frame + 8 * L.g;
                fr[0] = L.p[0]; fr[1] = L.p[1]; fr[2] = L.d[2]; fr[3] = fnx;
                fr[4] = fny; fr[5] = un; fr[6] = ut; fr[7] = L.E;
            }
            if (kSur && !open) {
                if (1.2f * rmm < fminf(dist, T)) {
                    absorb = true;                  // cannot reach the opening or the exit face
                } else if (L.E >= sur::kELo && L.E <= sur::kEHi && fabsf(un) <= sur::kAngMax &&
                           fabsf(ut) <= sur::kAngMax && ne.w >= sur::kKappaLo && ne.w <= sur::kKappaHi &&
                           fabsf(T - sur::kThickness) < 1e-3f && dist > 0.0f &&
                           fabsf(feat[5]) >= sur::kNearThreshold && (kTrack || B.rs)) {
                    sur_emit = true;                // in the training domain: one network draw
                }
            }
        }
        // ---- surrogate queries of the brass entries in its domain (one atomic per warp) ----
        // Each query also reserves its hand-off slot now, in arrival order, so
        // that the patient kernel meets the protons in the same order as on the
        // plain path (the influence-matrix columns it scores into stay in L2).
        const unsigned smask = __ballot_sync(kFull, sur_emit);
        if (smask) {
            unsigned long long base = 0, pbase = 0;
            const int leader = __ffs(smask) - 1;
            if (lane == leader) {
                base = atomicAdd(P.sq_count, (unsigned long long)__popc(smask));
                if (!kTrack) pbase = atomicAdd(P.phase_count, (unsigned long long)__popc(smask));
            }
            base = __shfl_sync(kFull, base, leader);
            pbase = __shfl_sync(kFull, pbase, leader);
            if (sur_emit) {
                const long long slot = (long long)base + __popc(smask & lt_mask);
                if (slot < P.sq_cap) {
                    SurQuery q;
#pragma unroll
                    for (int k = 0; k < 6; ++k) q.x[k] = feat[k];
                    q.px = L.p[0]; q.py = L.p[1];
                    q.dx = L.d[0]; q.dy = L.d[1]; q.dz = L.d[2];
                    q.E = L.E;
                    q.nx = fnx; q.ny = fny;
                    q.step = L.step;
                    q.item = L.item;
                    q.g = L.g;
                    q.slot = kTrack ? -1ll : (long long)pbase + __popc(smask & lt_mask);
                    P.sq[slot] = q;
                } else {
                    atomicOr(P.status, 4);          // query buffer too small (host sizes it to the batch)
                }
                alive = false;
            }
        }
        // ---- exact wall hit and wall distance (warp-cooperative) ----
        float sw = coop_first_wall_hit(need_hit, pu, pv, hx, hy, poly, q_off, q_n, lane);
        const float dw = coop_wall_distance(need_dist, pu, pv, poly, q_off, q_n, lane) * sc *
                         (ap_pending ? beams[L.beam].ap_cos : 1.0f);
        if (cdiv > 0.0f && isfinite(sw)) {
            // back from g to the path length: s = g c / (c - g d_t)
            const float den = cdiv - sw * L.d[2];
            sw = den > 0.0f ? sw * cdiv / den : __int_as_float(0x7f800000);
        }
        if (alive) {
            const DevBeam& B = beams[L.beam];
            if (ap_pending) {
                if (open) {
                    // opening: keep velocity and direction up to a wall or the exit
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
                } else if (sur_emit) {
                    // handed to the surrogate below
                } else {
                    L.forced = 0;
                    if (need_dist) absorb = rmax < dw;
                    if (absorb) {
                        acc_ap += to_fixed(L.E, P.fscale, P.fx32);
                        L.E = 0.0f;
                        fate = kAbsAp;
                    } else {
                        m = brass;
                        do_ch = true;
                    }
                }
            }
            if (do_ch) {
                StepResult o;
                ch_step<kAllPhysics>(m, s_geom, L, P, key, o);
                acc_steps += 1;
                const unsigned long long qs = to_fixed(o.dE, P.fscale, P.fx32);
                acc_ap += qs;
                if (o.killed) {
                    if (o.killed == 2) acc_nuc += qs;
                    fate = kAbsAp;
                } else {
#pragma unroll
                    for (int k = 0; k < 3; ++k) L.p[k] += o.disp[k];
                    if (o.lim == 1) { if (down) advance = true; else fate = kLeak; }
                }
            }
            if (advance && fate < 0) {
                // the single place where a history changes stage
                const int from = L.stage;
                if (from < 1 && B.ap) {
                    if (!(L.d[2] > 0.0f)) fate = kLeak;
                    else {
                        const float sdr = __fdividef(B.ap_tup - L.p[2], L.d[2]);
#pragma unroll
                        for (int k = 0; k < 3; ++k) L.p[k] = fmaf(sdr, L.d[k], L.p[k]);
                        L.R = range_of(brass.Rt, L.E);
                        L.stage = 1;
                        L.forced = -1;              // on the entrance plane
                    }
                } else {
                    handoff = true;                 // leaves the beam line: on to the patient kernel
                }
            }
            if (fate >= 0) {
                // the single place where a history ends in this kernel
                if (fate == kLeak || fate == kErr) acc_leak += to_fixed(L.E, P.fscale, P.fx32);
                if (fate == kErr) { acc_err += 1; atomicOr(P.status, 1); }
                if (P.records && L.g < P.rec_cap) {
                    float pos[3];
                    bev_to_patient(B, scens[__ldg(&P.items[L.item].scen)], L.p, pos);
                    write_record(P, L, fate, pos, 0ull);
                }
                if (kTrack && L.g < P.total) {
                    P.trk_label[L.g] = 0;
#pragma unroll
                    for (int k = 0; k < 5; ++k) P.trk_y[5 * L.g + k] = 0.0f;
                }
                alive = false;
            }
        }
        // ---- hand-off of the histories that left the beam line (one atomic per warp) ----
        if (kTrack) {
            if (handoff) {
                // training track: targets from the exit state against the entry frame
                const DevBeam& B = beams[L.beam];
                const float T = B.ap_tdn - B.ap_tup;
                const float* fr = P.trk_frame + 8 * L.g;
                const float nx = fr[3], ny = fr[4], un = fr[5], ut = fr[6], E0 = fr[7];
                const float dx = L.p[0] - fr[0], dy = L.p[1] - fr[1];
                float* y = P.trk_y + 5 * L.g;
                y[0] = 5.0f * (E0 - L.E) / E0;
                y[1] = dx * nx + dy * ny - T * un / fr[2];
                y[2] = dy * nx - dx * ny - T * ut / fr[2];
                y[3] = (L.d[0] * nx + L.d[1] * ny - un) * (1.0f / sur::kDirScale);
                y[4] = (L.d[1] * nx - L.d[0] * ny - ut) * (1.0f / sur::kDirScale);
                P.trk_label[L.g] = 1;
                alive = false;
            }
            handoff = false;
        }
        const unsigned hmask = __ballot_sync(kFull, handoff);
        if (hmask) {
            unsigned long long base = 0;
            const int leader = __ffs(hmask) - 1;
            if (lane == leader) base = atomicAdd(P.phase_count, (unsigned long long)__popc(hmask));
            base = __shfl_sync(kFull, base, leader);
            if (handoff) {
                const long long slot = (long long)base + __popc(hmask & lt_mask);
                const DevBeam& B = beams[L.beam];
                if (slot < P.rep_cap) {
                    // one copy per scenario sharing the transport, with that scenario's shift
                    const int scen0 = __ldg(&P.items[L.item].scen);
                    PhaseRec r;
#pragma unroll
                    for (int k = 0; k < 3; ++k) r.d[k] = L.d[0] * B.u[k] + L.d[1] * B.v[k] + L.d[2] * B.w[k];
                    r.E = L.E;
                    r.nlam = L.nlam;
                    r.step = L.step;
                    for (int s = 0; s < P.n_rep; ++s) {
                        bev_to_patient(B, scens[scen0 + s], L.p, r.p);
                        r.item = L.item + s * P.rep_items;
                        r.g = L.g + s * P.rep_hist;
                        P.phase[s * P.rep_cap + slot] = r;
                    }
                } else {
                    atomicOr(P.status, 2);          // hand-off buffer too small (host sizes it to the batch)
                }
                alive = false;
            }
        }
    }
    // energies and errors count once per scenario sharing the transport; steps as taken
    const unsigned long long nr = (unsigned long long)P.n_rep;
    unsigned long long v[kNStats] = {0ull, acc_leak * nr, 0ull, acc_ap * nr, acc_nuc * nr, acc_steps, acc_err * nr,
                                     0ull, acc_steps};
    warp_add_stats(P, v, lane);
}

size_t devices_smem_bytes() { return SourceSmem::Bytes > ApertureSmem::Bytes ? SourceSmem::Bytes : ApertureSmem::Bytes; }
int devices_max_block() { return 640; }

template <int kMode, bool kAllPhysics>
static cudaError_t launch_aperture_variant(const TransportParams& p, int grid, int block, cudaStream_t s)
{
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_aperture<kMode, kAllPhysics>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ApertureSmem::Bytes);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    k_aperture<kMode, kAllPhysics><<<grid, block, ApertureSmem::Bytes, s>>>(p);
    return cudaGetLastError();
}

template <int kMode>
static cudaError_t launch_aperture_mode(const TransportParams& p, int grid, int block, cudaStream_t s)
{
    if (p.mcs && p.straggling && p.nuclear) return launch_aperture_variant<kMode, true>(p, grid, block, s);
    return launch_aperture_variant<kMode, false>(p, grid, block, s);
}

template <bool kAllPhysics>
static cudaError_t launch_source_rs(const TransportParams& p, int grid, cudaStream_t s)
{
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_source_rs<kAllPhysics>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)SourceSmem::Bytes);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    k_source_rs<kAllPhysics><<<grid, 768, SourceSmem::Bytes, s>>>(p);      // 78 registers: 768 threads fit
    return cudaGetLastError();
}

cudaError_t launch_devices(const TransportParams& p, int grid, int block, cudaStream_t s)
{
    const int mode = (p.surrogate ? 1 : 0) | (p.track_mode ? 2 : 0);
    if (!p.track_mode) {
        cudaError_t e = cudaMemsetAsync(p.mid_count, 0, sizeof(unsigned long long), s);
        if (e != cudaSuccess) return e;
        e = (p.mcs && p.straggling && p.nuclear) ? launch_source_rs<true>(p, grid, s) : launch_source_rs<false>(p, grid, s);
        if (e != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(p.counter, 0, sizeof(unsigned long long), s)) != cudaSuccess) return e;
    }
    switch (mode) {
    case 1: return launch_aperture_mode<1>(p, grid, block, s);
    case 2: return launch_aperture_mode<2>(p, grid, block, s);
    case 3: return launch_aperture_mode<3>(p, grid, block, s);
    default: return launch_aperture_mode<0>(p, grid, block, s);
    }
}

}  // namespace vpmc
