// Reach of each energy layer along its field's axis, for the influence-matrix
// column boxes.
//
// The influence matrix (paper Sec. 2.C) stores each spot's dose per primary
// as a sparse column.  The transport scores a spot's deposits into a dense
// box of the scoring grid first; a box that covers the field's whole depth
// holds, beyond the spots' Bragg peaks, voxels that no proton reaches, and
// each of them is cleared and read by every pass that builds the CSR.  This
// kernel finds, per (scenario, field, layer), the depth where a proton with
// the layer's largest residual range must have stopped: it marches rays
// parallel to the field's axis through the CT, one per lateral column of the
// opening, sums the water-equivalent path (SPR x scenario scale x length),
// and keeps, over the columns, the largest depth at which the sum reaches the
// layer's range.  A deposit beyond it (a bound that was too tight) is not
// lost: the transport records deposits outside an item's box one by one and
// the CSR build merges them.
#include <cstddef>

#include "vpmc_internal.cuh"

namespace vpmc {
namespace {

// One block per job; threads stride over the job's lateral columns.  Run
// ranges are ascending within a job, so one pointer walks them as the sum
// grows.  Depths are stored as t - t0 >= 0, whose FP32 bit patterns order as
// the values do, so an integer maximum over the columns is the float maximum.
__global__ void k_depth_bounds(const uint16_t* __restrict__ ct, const float2* __restrict__ hu, Grid3 ctg,
                               const DepthJob* __restrict__ jobs, const float* __restrict__ r_lim,
                               unsigned* __restrict__ reach)
{
    const DepthJob J = jobs[blockIdx.x];
    const int ncol = J.na * J.nb;
    const int nstep = (int)ceilf((J.t1 - J.t0) / J.dt);
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
        const float a = J.a0 + (float)(c % J.na) * J.da, b = J.b0 + (float)(c / J.na) * J.da;
        float q[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) q[k] = J.base[k] + a * J.u[k] + b * J.v[k];
        float wet = 0.0f;
        int r = 0;
        for (int i = 0; i < nstep && r < J.run_n; ++i) {
            const float t = J.t0 + ((float)i + 0.5f) * J.dt;
            long long idx = 0;
            bool inside = true;
#pragma unroll
            for (int k = 2; k >= 0; --k) {
                const int v = (int)floorf((q[k] + t * J.w[k] - ctg.lo[k]) / ctg.d[k]);
                inside = inside && v >= 0 && v < ctg.n[k];
                idx = idx * ctg.n[k] + v;
            }
            if (!inside) continue;
            wet += hu[ct[idx]].y * J.spr_scale * J.dt;
            while (r < J.run_n && wet >= r_lim[J.run_off + r]) {
                atomicMax(reach + J.run_off + r, __float_as_uint(t + 0.5f * J.dt - J.t0));
                ++r;
            }
        }
        // a range the column never exhausts: the field's far end
        for (; r < J.run_n; ++r) atomicMax(reach + J.run_off + r, __float_as_uint(J.t1 - J.t0));
    }
}

}  // namespace

cudaError_t launch_depth_bounds(const uint16_t* ct, const TablesImage* tables, Grid3 ctg, const DepthJob* jobs,
                                int n_jobs, const float* r_lim, unsigned* reach, cudaStream_t s)
{
    if (n_jobs <= 0) return cudaSuccess;
    const float2* hu = reinterpret_cast<const float2*>(reinterpret_cast<const char*>(tables) + offsetof(TablesImage, hu));
    k_depth_bounds<<<n_jobs, 256, 0, s>>>(ct, hu, ctg, jobs, r_lim, reach);
    return cudaGetLastError();
}

}  // namespace vpmc
