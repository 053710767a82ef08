// Persistent transport kernel of the voxelised patient for sm_103a.
//
// k_patient takes the histories that the beam-line kernels (devices.cu) hand
// over on the block's exit plane, transports them through the CT with
// condensed-history steps (paper Sec. 2.A: one identical model per history)
// and scores every step's deposit into a 64-bit fixed-point accumulator: the
// dose grid, or the influence-matrix column of the history's spot (Sec. 2.C),
// optionally aggregated over the lanes of a warp that hit the same voxel.
//
// Steps end on the faces of two grids, the CT (materials) and the scoring
// grid, so that every step deposits in one scoring voxel.  Where an axis of
// the scoring grid is nested in the CT's -- the same origin and a spacing of
// 2^sh CT voxels -- every scoring face is a CT face: that axis needs no
// second face distance and the scoring index is the CT index shifted right
// by sh.  The kernel is compiled for three nestings (kNest bit k: axis k
// nested): none, x and y (the 2 mm scoring grid over a 1 x 1 x 1.5 mm CT),
// and all three (one grid).  Each is compiled for three modes: the launch's
// switches read at run time; full physics known at compile time; and full
// physics with influence-matrix scoring (unit item weights, 32-bit
// fixed-point conversion, plain atomics) known at compile time.  The results
// do not depend on the variant.
#include "transport_common.cuh"

namespace vpmc {
namespace {

using namespace dev;
using namespace tr;

constexpr int kModeAllPhysics = 1;   // scattering, straggling and nuclear removal on
constexpr int kModeIMScoring = 2;    // unit item weights, fx32, plain atomics

template <int kNest, int kMode>
__global__ void __launch_bounds__(kPatientMaxBlock, 1) k_patient(const TransportParams P)
{
    constexpr bool kIM = (kMode & kModeIMScoring) != 0;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    long long* s_g = reinterpret_cast<long long*>(smem + PatientSmem::G);
    long long* s_pool = reinterpret_cast<long long*>(smem + PatientSmem::Pool) + 2 * warp;
    int* s_item = reinterpret_cast<int*>(smem + PatientSmem::Item);
    {
        float2* R = reinterpret_cast<float2*>(smem + PatientSmem::R);
        float2* Et = reinterpret_cast<float2*>(smem + PatientSmem::Einv);
        for (int i = threadIdx.x; i < kNEPad; i += blockDim.x) R[i] = P.tables->R[kWater][i];
        for (int i = threadIdx.x; i < kNR; i += blockDim.x) Et[i] = P.tables->Einv[kWater][i];
        float2* hu = reinterpret_cast<float2*>(smem + PatientSmem::HU);
        for (int i = threadIdx.x; i < kNHU; i += blockDim.x) hu[i] = P.tables->hu[i];
        DevScen* sc = reinterpret_cast<DevScen*>(smem + PatientSmem::Scens);
        for (int i = threadIdx.x; i < P.n_scen; i += blockDim.x) sc[i] = P.scens[i];
        if (lane == 0) { s_pool[0] = 0; s_pool[1] = 0; }
        s_g[threadIdx.x] = 0;
        s_item[threadIdx.x] = 0;
    }
    __syncthreads();
    Medium water;
    water.Rt = reinterpret_cast<const float2*>(smem + PatientSmem::R);
    water.Et = reinterpret_cast<const float2*>(smem + PatientSmem::Einv);
    const float2* hu_lut = reinterpret_cast<const float2*>(smem + PatientSmem::HU);
    const DevScen* scens = reinterpret_cast<const DevScen*>(smem + PatientSmem::Scens);
    water.inv_dR = P.water.inv_dR;
    water.za = P.water.za;
    water.inv_x0 = P.water.inv_x0;

    bool alive = false, done = false;
    PatientLane L;
    L.hist = 0; L.hdep = 0ull; L.iters = 0; L.step = 0; L.E = 0.0f; L.R = 0.0f; L.nlam = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) { L.p[k] = 0.0f; L.d[k] = 0.0f; L.ic[k] = 0; L.is[k] = 0; }
    uint32_t key1 = 0u;
    float spr_scale = 1.0f;
    DevBox bx;
    unsigned long long* box_q = nullptr;
    bx.base = 0; bx.lo[0] = bx.lo[1] = bx.lo[2] = 0; bx.n[0] = bx.n[1] = bx.n[2] = 0;
    float wsc = 0.0f;

    for (;;) {
        // ---- histories handed over by the devices kernel ----
        unsigned need = __ballot_sync(kFull, !alive && !done);
        if (need) {
            // the warp's pool lives in shared memory between refills, so that
            // it holds no registers across the step
            WorkPool pool;
            pool.next = s_pool[0];
            pool.end = s_pool[1];
            const unsigned lt_mask = (1u << lane) - 1u;
            while (need) {
                // the work is n_rep regions (one per scenario sharing the
                // beam-line transport) of cnt records each
                const long long cnt = min((long long)*P.phase_count, P.rep_cap);
                if (pool.next >= pool.end) {
                    if (!pool.refill(P, 0, cnt * P.n_rep, lane)) {
                        if (!alive) done = true;
                        break;
                    }
                }
                const int take = (int)min((long long)__popc(need), pool.end - pool.next);
                const bool mine = ((need >> lane) & 1u) && __popc(need & lt_mask) < take;
                if (mine) {
                    const long long w = pool.next + __popc(need & lt_mask);
                    const long long reg = w / cnt;
                    const PhaseRec r = P.phase[reg * P.rep_cap + (w - reg * cnt)];
                    if (r.item >= 0) {        // item -1: a slot the aperture surrogate left empty
                        const DevItem I = P.items[r.item];
                        s_item[threadIdx.x] = r.item;
                        s_g[threadIdx.x] = r.g;
                        L.hist = (uint32_t)(r.g - I.hist_off);
                        L.step = r.step;
                        L.iters = 0;
                        L.E = r.E;
                        L.nlam = r.nlam;
                        L.hdep = 0ull;
                        key1 = P.key1_hi ^ (uint32_t)I.spot;
                        spr_scale = scens[I.scen].spr_scale;
                        bx = P.boxes[I.box];
                        box_q = P.scratch + bx.base;
                        wsc = I.wscale;
                        // ray / grid box entry
                        float tmin = -__int_as_float(0x7f800000), tmax = __int_as_float(0x7f800000);
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            const float lo = P.ctg.lo[k], hi = P.ctg.lo[k] + P.ctg.n[k] * P.ctg.d[k];
                            if (r.d[k] != 0.0f) {
                                const float inv = __fdividef(1.0f, r.d[k]);
                                float t1 = (lo - r.p[k]) * inv, t2 = (hi - r.p[k]) * inv;
                                if (t1 > t2) { const float tt = t1; t1 = t2; t2 = tt; }
                                tmin = fmaxf(tmin, t1);
                                tmax = fminf(tmax, t2);
                            } else if (r.p[k] < lo || r.p[k] > hi) {
                                tmax = -__int_as_float(0x7f800000);
                            }
                        }
                        const float tin = fmaxf(tmin, 0.0f);
#pragma unroll
                        for (int k = 0; k < 3; ++k) { L.p[k] = r.p[k]; L.d[k] = r.d[k]; }
                        if (!(tmax > tin)) {
                            // misses the grid
                            atomicAdd(P.stats + kStLeak, to_fixed(L.E, P.fscale, P.fx32));
                            if (P.records && r.g < P.rec_cap) put_record(P, r.g, kLeak, L.step, 0ull, L.E, L.p);
                        } else {
#pragma unroll
                            for (int k = 0; k < 3; ++k) {
                                L.p[k] = fmaf(tin, L.d[k], L.p[k]);
                                const int a = (int)floorf(__fdividef(L.p[k] - P.ctg.lo[k], P.ctg.d[k]));
                                L.ic[k] = min(max(a, 0), P.ctg.n[k] - 1);
                                if (!((kNest >> k) & 1)) {
                                    const int b = (int)floorf(__fdividef(L.p[k] - P.sg.lo[k], P.sg.d[k]));
                                    L.is[k] = min(max(b, 0), P.sg.n[k] - 1);
                                }
                            }
                            L.R = range_of(water.Rt, L.E);
                            alive = true;
                        }
                    }
                }
                pool.next += take;
                need = __ballot_sync(kFull, !alive && !done);
            }
            __syncwarp();
            if (lane == 0) { s_pool[0] = pool.next; s_pool[1] = pool.end; }
            __syncwarp();
            // every lane is now alive or done: a warp without a live lane has
            // finished.  A warp that needed no work has a live lane, since a
            // history ends only in a step and its lane then needs work
            if (!__any_sync(kFull, alive)) break;
        }

        // ---- one condensed-history step of every live history ----
        long long dep_key = -1;                  // voxel of the scratch (dose scoring)
        unsigned long long* dep_ptr = nullptr;   // its address (influence-matrix scoring)
        unsigned long long dep_q = 0ull;
        if (alive) {
            int fate = -1;
            if (++L.iters > P.max_iter) {
                fate = kErr;
            } else {
                // material: the CT holds each voxel's index into the (density,
                // SPR) table, clamped when the context was created
                const int cidx = L.ic[0] + P.ctg.n[0] * (L.ic[1] + P.ctg.n[1] * L.ic[2]);   // CT < 2^31 voxels
                const float2 rs = hu_lut[__ldg(P.ct_lut + cidx)];
                water.kappa = rs.y * spr_scale;
                water.rho = rs.x;
                // the faces of the current voxel of each grid (the scoring
                // grid's only on axes that are not nested), shared by the
                // lateral confinement and the face distances.  The previous
                // step's lateral displacement is confined here, to the voxel
                // the step ended in, so that the faces are computed once per
                // step (not again after a crossing); nothing reads the
                // position in between.  The first step confines the entry
                // point to its voxel (a move of a rounding error at most).
                // The far face's index converts exactly as i + 1 (indices are
                // far below 2^24).  The position then lies in the voxel, so
                // each face distance along the direction is >= 0 (or -0)
                float f0[3], f1[3], g0[3], g1[3];
                float dc[3], ds[3], s_geom = __int_as_float(0x7f800000);
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const bool nested = (kNest >> k) & 1;
                    const float fc = (float)L.ic[k];
                    f0[k] = P.ctg.lo[k] + fc * P.ctg.d[k];
                    f1[k] = P.ctg.lo[k] + (fc + 1.0f) * P.ctg.d[k];
                    if (!nested) {
                        const float fs = (float)L.is[k];
                        g0[k] = P.sg.lo[k] + fs * P.sg.d[k];
                        g1[k] = P.sg.lo[k] + (fs + 1.0f) * P.sg.d[k];
                    }
                    const float vlo = nested ? f0[k] : fmaxf(f0[k], g0[k]);
                    const float vhi = nested ? f1[k] : fminf(f1[k], g1[k]);
                    L.p[k] = fminf(fmaxf(L.p[k], vlo), vhi);
                    dc[k] = ds[k] = __int_as_float(0x7f800000);
                    const float Dk = L.d[k];
                    if (Dk != 0.0f) {
                        const float inv = __fdividef(1.0f, Dk);
                        const bool up = Dk > 0.0f;
                        dc[k] = ((up ? f1[k] : f0[k]) - L.p[k]) * inv;
                        if (nested) ds[k] = dc[k];
                        else ds[k] = ((up ? g1[k] : g0[k]) - L.p[k]) * inv;
                    }
                    s_geom = fminf(s_geom, nested ? dc[k] : fminf(dc[k], ds[k]));
                }
                StepResult o;
                const float d_old[3] = {L.d[0], L.d[1], L.d[2]};
                int sv[3];                  // scoring voxel where the step starts
#pragma unroll
                for (int k = 0; k < 3; ++k) sv[k] = ((kNest >> k) & 1) ? (L.ic[k] >> P.nest_shift[k]) : L.is[k];
                ch_step<(kMode & kModeAllPhysics) != 0>(water, s_geom, L, P, make_uint2(P.key0, key1), o);
                const unsigned long long qs = to_fixed(o.dE, P.fscale, kIM || P.fx32);
                unsigned long long q = qs;
                if (!kIM && !P.unit_weight && wsc != P.fscale) q = to_fixed(o.dE, wsc, false);
                // score into the scoring voxel where the step started
                const int lx = sv[0] - bx.lo[0], ly = sv[1] - bx.lo[1], lz = sv[2] - bx.lo[2];
                if ((unsigned)lx < (unsigned)bx.n[0] && (unsigned)ly < (unsigned)bx.n[1] &&
                    (unsigned)lz < (unsigned)bx.n[2]) {
                    if (kIM) dep_ptr = box_q + (lx + bx.n[0] * (ly + bx.n[1] * lz));
                    else dep_key = bx.base + (long long)(lx + bx.n[0] * (ly + bx.n[1] * lz));   // box < 2^31 voxels
                    dep_q = q;
                } else if (o.dE > 0.0f && P.ovf) {
                    // rare tail outside the item's box: append a record
                    const unsigned long long slot = atomicAdd(P.ovf_count, 1ull);
                    if ((long long)slot < P.ovf_cap) {
                        OvfRec rr;
                        rr.voxel = sv[0] + P.sg.n[0] * (sv[1] + P.sg.n[1] * sv[2]);
                        rr.item = s_item[threadIdx.x];
                        rr.q = q;
                        P.ovf[slot] = rr;
                    }
                }
                L.hdep += qs;
                if (o.killed) {
                    if (o.killed == 2) atomicAdd(P.stats + kStNuc, qs);
                    fate = o.killed == 2 ? kNuc : kStop;
                } else {
                    if (o.lim == 1) {
                        // the step ended on a face: move to the next voxel of
                        // each grid whose face it reached
                        bool out = false;
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            const bool nested = (kNest >> k) & 1;
                            // (dc and ds are +inf on an axis the direction does not move along)
                            const int sg = d_old[k] > 0.0f ? 1 : -1;
                            if (dc[k] == o.s) {
                                L.ic[k] += sg;
                            }
                            out |= (unsigned)L.ic[k] >= (unsigned)P.ctg.n[k];
                            if (!nested) {
                                if (ds[k] == o.s) {
                                    L.is[k] += sg;
                                }
                                out |= (unsigned)L.is[k] >= (unsigned)P.sg.n[k];
                            }
                        }
                        if (out) fate = kLeak;
                    }
                    if (fate < 0) {
                        // lateral displacement (confined at the next step's start)
#pragma unroll
                        for (int k = 0; k < 3; ++k) L.p[k] += o.disp[k];
                    }
                }
            }
            if (fate >= 0) {
                // the history's totals go straight to the launch's counters
                // (one history ends every few hundred steps of a lane)
                if (L.hdep) atomicAdd(P.stats + kStDep, L.hdep);
                atomicAdd(P.stats + kStSteps, (unsigned long long)min(L.iters, P.max_iter));
                if (fate == kLeak || fate == kErr) atomicAdd(P.stats + kStLeak, to_fixed(L.E, P.fscale, P.fx32));
                if (fate == kErr) { atomicAdd(P.stats + kStErr, 1ull); atomicOr(P.status, 1); }
                if (P.records) {
                    const long long g = s_g[threadIdx.x];
                    if (g < P.rec_cap) put_record(P, g, fate, L.step, L.hdep, L.E, L.p);
                }
                alive = false;
            }
        }
        // ---- scoring (all lanes together) ----
        if (kIM) { if (dep_ptr && dep_q) atomicAdd(dep_ptr, dep_q); }
        else if (P.aggregate) deposit_aggregated(P.scratch, dep_key, dep_q);
        else if (dep_key >= 0 && dep_q) atomicAdd(P.scratch + dep_key, dep_q);
    }
}

// CT hounsfield units -> index into the kernels' (density, SPR) table, in place.
__global__ void k_ct_lut_index(int16_t* ct, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int h = min(max((int)ct[i], kHULo), kHULo + kNHU - 1);
        reinterpret_cast<uint16_t*>(ct)[i] = (uint16_t)(h - kHULo);
    }
}

template <int kNest, int kMode>
cudaError_t launch_patient_variant(const TransportParams& p, int grid, int block, cudaStream_t s)
{
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_patient<kNest, kMode>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)PatientSmem::Bytes);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    k_patient<kNest, kMode><<<grid, block, PatientSmem::Bytes, s>>>(p);
    return cudaGetLastError();
}

template <int kNest>
cudaError_t launch_patient_nest(const TransportParams& p, int grid, int block, cudaStream_t s)
{
    if (!(p.mcs && p.straggling && p.nuclear)) return launch_patient_variant<kNest, 0>(p, grid, block, s);
    if (p.unit_weight && p.fx32 && !p.aggregate)
        return launch_patient_variant<kNest, kModeAllPhysics | kModeIMScoring>(p, grid, block, s);
    return launch_patient_variant<kNest, kModeAllPhysics>(p, grid, block, s);
}

}  // namespace

size_t patient_smem_bytes() { return PatientSmem::Bytes; }
int patient_max_block() { return kPatientMaxBlock; }

int patient_nest_variant(const int nest_shift[3])
{
    const int mask = (nest_shift[0] >= 0 ? 1 : 0) | (nest_shift[1] >= 0 ? 2 : 0) | (nest_shift[2] >= 0 ? 4 : 0);
    return mask == 7 ? 7 : ((mask & 3) == 3 ? 3 : 0);
}

cudaError_t launch_patient(const TransportParams& p, int grid, int block, cudaStream_t s)
{
    switch (patient_nest_variant(p.nest_shift)) {
    case 7: return launch_patient_nest<7>(p, grid, block, s);
    case 3: return launch_patient_nest<3>(p, grid, block, s);
    default: return launch_patient_nest<0>(p, grid, block, s);
    }
}

cudaError_t launch_ct_lut_index(int16_t* ct, long long n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const long long blocks = (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096;
    k_ct_lut_index<<<(int)blocks, 256, 0, s>>>(ct, n);
    return cudaGetLastError();
}

}  // namespace vpmc
