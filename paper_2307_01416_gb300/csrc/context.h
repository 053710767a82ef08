// Library-internal definition of the context behind the C ABI's opaque
// vpmc_ctx handle (shared by the translation units of the library).
#pragma once

#include <string>
#include <vector>

#include "../../include/vpmc.h"
#include "vpmc_internal.cuh"

namespace vpmc {

// Launch configuration of the two transport kernels chosen by the autotuner.
struct TuneResult {
    bool valid = false;
    int dev_block = 512;     // k_devices threads per block
    int block = 640;         // k_patient threads per block
    int aggregate = 0;
    int chunk = 32;
};

// Grow-only device buffer a context keeps between calls (the influence
// matrix's work arrays), so that repeated calls of one size allocate nothing.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

}  // namespace vpmc

struct vpmc_ctx {
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    vpmc::Grid3 ctg{}, sg{};
    double ct_spacing[3]{}, sg_spacing[3]{};
    int nest_shift[3]{-1, -1, -1};      // per axis: scoring spacing = CT spacing << shift, same origin (-1: not)
    long long nvox = 0;
    double curve15[15]{};
    int16_t* d_ct = nullptr;                  // CT: HU until the scoring densities are built, then table indices
    vpmc::TablesImage* d_tables = nullptr;
    vpmc::MatConst water_mat{};          // the tables image's water entry (a launch constant)
    std::vector<float2> range_water;         // host copy of the water range table (column-box depths)
    double* d_curve = nullptr;
    double* d_rho = nullptr;
    double* d_inv_rho = nullptr;               // 1 / rho per scoring voxel (FP64)
    float* d_inv_rho_f = nullptr;              // the same in FP32 (screens of the influence-matrix passes)
    unsigned long long* d_acc = nullptr;       // dose accumulator (scoring grid)
    // fields
    bool beam_set[vpmc::kMaxBeams]{};
    vpmc::DevBeam beams[vpmc::kMaxBeams]{};
    std::vector<double> poly[vpmc::kMaxBeams];
    std::vector<unsigned char> raster[vpmc::kMaxBeams];
    std::vector<float> raster_lb[vpmc::kMaxBeams];
    vpmc::DevBeam* d_beams = nullptr;
    float2* d_poly = nullptr;
    int n_poly = 0;
    unsigned char* d_raster = nullptr;
    float* d_raster_lb = nullptr;
    // per-launch buffers
    unsigned long long* d_counter = nullptr;
    unsigned long long* d_stats = nullptr;
    int* d_status = nullptr;
    vpmc::DevScen* d_scens = nullptr;
    vpmc::DevItem* d_items = nullptr;
    size_t items_cap = 0;
    vpmc::DevBox* d_boxes = nullptr;
    size_t boxes_cap = 0;
    vpmc::OvfRec* d_ovf = nullptr;                   // out-of-box deposit records
    long long ovf_cap = 0;
    vpmc::PhaseRec* d_phase = nullptr;               // hand-off from the aperture to the patient kernel
    vpmc::PhaseRec* d_mid = nullptr;                 // hand-off from the range-shifter to the aperture kernel
    long long phase_cap = 0;                         // records of each hand-off buffer
    unsigned long long* d_phase_count = nullptr;
    unsigned long long* d_mid_count = nullptr;
    unsigned long long* d_scratch = nullptr;
    size_t scratch_cap = 0;                    // elements
    float* d_poly_kappa = nullptr;             // per polygon vertex: signed curvature (surrogate inputs)
    // learned aperture surrogate
    vpmc::SurNet sur{};
    bool sur_ready = false;                    // weights loaded or trained
    int sur_step = 0;                          // Adam steps taken since the weights were set
    vpmc::SurQuery* d_sq = nullptr;            // brass entries handed to the surrogate
    long long sq_cap = 0;
    unsigned long long* d_sq_count = nullptr;
    vpmc::TuneResult tune_dose, tune_im;
    long long launches = 0;                    // kernels launched since creation
    // per transport batch: events before the beam-line kernels, between them
    // and the patient kernel, and after it (the first kTimedBatches batches)
    static constexpr int kTimedBatches = 64;
    cudaEvent_t kev[3 * kTimedBatches]{};
    int kev_batches = 0;                       // batches the last enqueued transport recorded
    // an asynchronous dose call left its status word unread (1; 2: with the
    // surrogate's status word too): the next call reads it first
    int status_pending = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // influence-matrix work arrays (kept, grown on demand)
    vpmc::DevBuf im_colmax, im_item_scale, im_rowcnt, im_nnz, im_scan_tmp, im_meta, im_bucket_off, im_bucket_cur,
        im_bucket_len, im_ovf_sorted, im_ovf_count, im_jobs, im_rlim, im_reach, im_thr, im_thr_f, im_box_slot;
    // allocator of the influence matrices' CSR buffers (NULL: the library's)
    vpmc_alloc_fn csr_alloc = nullptr;
    void* csr_alloc_user = nullptr;
};

namespace vpmc {
// Records an error message for vpmc_last_error() on the calling thread and
// returns st (printf-style message).
vpmc_status report_error(vpmc_status st, const char* fmt, ...);
// Clears the calling thread's message (at the start of every entry point).
void clear_error();
}  // namespace vpmc
