// Internal types of the GB300 transport library (not part of the C ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace vpmc {

// Physics tables (built in FP64 on the host, stored FP32; staged in shared memory).
constexpr int kNE = 2501;            // E_k = 0.1 k MeV, k = 0..2500
constexpr int kNEPad = 2504;         // row stride (16-byte multiple)
constexpr int kNR = 4096;            // uniform residual-range grid
constexpr int kNMat = 3;             // 0 water (patient media, SPR-scaled), 1 PMMA, 2 brass
constexpr int kHULo = -1024;
constexpr int kNHU = 4096;           // HU -1024..3071
constexpr int kMaxBeams = 64;            // beam entries: fields, or (field, energy layer) pairs
constexpr int kMaxScen = 64;
constexpr int kMaxPolyVerts = 4096;
constexpr int kRaster = 256;         // BEV raster per beam (cells per side): opening class, wall-distance bound
constexpr float kEcut = 0.5f;        // MeV
constexpr int kMaxIter = 200000;     // default cap on a history's iterations in one kernel (then it is an error)

enum Material { kWater = 0, kPMMA = 1, kBrass = 2 };
enum Fate { kStop = 0, kNuc = 1, kLeak = 2, kAbsRS = 3, kAbsAp = 4, kErr = 5 };
// kStSteps counts condensed-history steps in every medium; kStStepsRS and
// kStStepsAp the range shifter's and the brass block's share of them.
enum Stat { kStDep = 0, kStLeak, kStRS, kStAp, kStNuc, kStSteps, kStErr, kStStepsRS, kStStepsAp, kNStats };

struct MatConst {
    float za;          // Z/A
    float rho;         // g/cc (PMMA, brass); 1 for water
    float inv_x0;      // 1 / radiation length in mm * g/cc
    float inv_dR;      // 1 / (uniform R-grid step)
};

struct TablesImage {                 // global-memory image, copied to shared memory
    float2 R[kNMat][kNEPad];         // (R(E_k), R(E_{k+1}) - R(E_k)): residual range, mm * g/cc
    float2 Einv[kNMat][kNR];         // (E(R_j), E(R_{j+1}) - E(R_j)) at R_j = j * dR
    float2 hu[kNHU];                 // (density, SPR) per HU
    MatConst mat[kNMat];
};

struct DevBeam {
    float w[3], u[3], v[3], iso[3];
    float t_src;
    int rs;
    float rs_tup, rs_tdn, rs_r2;
    int ap;
    float ap_tup, ap_tdn;
    int poly_off, nvert;
    float ras_lo[2], ras_inv[2];     // raster origin and 1/cell size
    int ras_off;                     // offset into the raster arrays (class bytes, distance bounds)
    float ras_diag;                  // raster cell diagonal
    float r_circ;                    // largest vertex distance from the beam axis (training tracks)
    float ap_sad;                    // divergent walls: virtual source at t = -ap_sad (0: parallel walls)
    float ap_K;                      // ap_tdn + ap_sad: opening scale at depth t = (t + ap_sad) / ap_K
    float ap_cos;                    // cosine of the largest wall tilt (1 for parallel walls)
};

struct DevScen {
    float shift[3];
    float spr_scale;
};

// One work item = one (scenario, spot) pair: a contiguous range of global
// history indices and the box of the scoring grid its deposits go to.
struct DevItem {
    long long hist_off;              // global index of the item's first history
    float E0, x, y, sigma;
    float div_rad, wscale;           // wscale = 2^F (x weight in the dose path)
    int spot;                        // spot index: RNG key and CSR column
    int scen;
    int beam;
    int box;                         // index into the box table
};

struct DevBox {
    long long base;                  // element offset into the uint64 scratch
    int lo[3];                       // first scoring voxel of the box
    int n[3];                        // box extent in voxels
};

struct Grid3 {
    int n[3];
    float d[3];
    float lo[3];
};

// Deposit that fell outside its item's box (rare tails of the lateral
// spread); bucketed by voxel after transport and merged into the CSR rows.
struct OvfRec {
    int voxel;                       // scoring-grid voxel
    int item;                        // item index within the launch
    unsigned long long q;
};

// A history at the end of the beam-line devices, handed to the patient
// kernel: position and direction in the patient frame (scenario shift applied).
struct PhaseRec {
    float p[3], d[3];
    float E, nlam;
    uint32_t step;                   // condensed-history steps so far (RNG counter)
    int item;                        // -1: an empty slot (absorbed by the aperture surrogate)
    long long g;                     // global history index
};

// ---- learned aperture surrogate (not in the paper: a network drawing the
// state on the block's exit plane in place of in-brass stepping) ----
namespace sur {
constexpr int kIn = 6, kInPad = 16, kH = 128, kOut = 45, kOutPad = 48, kNComp = 4, kDY = 5;
// FP32 parameter vector: W1 [128 x 6], b1, W2 [128 x 128], b2, W3 [45 x 128], b3 (row-major, out x in)
constexpr int oW1 = 0, ob1 = oW1 + kH * kIn, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, oW3 = ob2 + kH,
              ob3 = oW3 + kOut * kH;
constexpr int kNParams = ob3 + kOut;
// BF16 operand images in the canonical no-swizzle K-major layout of the
// tensor-core instructions (byte offsets): W1 [128 x 16], W2 [128 x 128],
// W3 [48 x 128], and the transposes W2^T [128 x 128], W3^T [128 x 48].
constexpr int kImgW1 = 0;
constexpr int kImgW2 = kImgW1 + kH * kInPad * 2;
constexpr int kImgW3 = kImgW2 + kH * kH * 2;
constexpr int kImgW2T = kImgW3 + kOutPad * kH * 2;
constexpr int kImgW3T = kImgW2T + kH * kH * 2;
constexpr int kImgBytes = kImgW3T + kH * kOutPad * 2;
// Input and target scales, training domain.
constexpr float kDCap = 12.0f;       // mm: edge distance clip
constexpr float kELo = 40.0f, kEHi = 230.0f;
constexpr float kAngSigma = 0.04f, kAngMax = 0.12f;
constexpr float kDirScale = 0.05f;
constexpr float kSMin = -8.0f, kSMax = 4.0f;
constexpr float kThickness = 30.0f;  // block thickness of the training geometries, mm
constexpr float kKappaLo = -1e-3f, kKappaHi = 0.26f;
// The network serves beams with a range shifter only (the test domain in
// which its dose error stays below 1 % of the maximum).
// Near the stopping threshold (brass CSDA range within 6 % of the thickness)
// a proton leaves the block with a few MeV or not at all: the exit energy
// distribution has a sharp edge that the mixture does not follow.  Those
// entries take the plain path.
constexpr float kNearThreshold = 0.06f;
}  // namespace sur

// One proton handed from the beam-line kernel to the surrogate: its state on
// the block's entrance plane and its edge frame.
struct SurQuery {
    float x[6];                      // network inputs
    float px, py, dx, dy, dz, E;     // BEV position (entrance plane), direction, energy
    float nx, ny;                    // unit vector from the nearest edge point into the brass
    uint32_t step;
    int item;
    long long g;
    long long slot;                  // hand-off slot reserved in arrival order (-1: none)
};

struct HistRecord {                  // mirrors vpmc_history_record
    long long q_dep;
    int fate;
    int steps;
    float e_dep;
    float e_end;
    float pos[3];
    float pad;
};

struct TransportParams {
    const TablesImage* tables;
    const uint16_t* ct_lut;          // per CT voxel: index into the (density, SPR) table
    Grid3 ctg, sg;
    int nest_shift[3];               // per axis: scoring spacing = CT spacing << shift, same origin (-1: not nested)
    const DevBeam* beams;
    int n_beams;
    const DevScen* scens;
    int n_scen;
    const float2* poly;
    int n_poly;
    const unsigned char* raster;
    const float* raster_lb;          // per raster cell: lower bound of the distance to the opening's boundary
    int range_rejection;             // absorb brass protons that cannot leave the block
    const DevItem* items;
    int n_items;
    const DevBox* boxes;
    long long total;                 // total histories
    unsigned long long* counter;     // global work counter
    unsigned long long* scratch;     // deposit target
    long long hist_begin;            // beam-line kernels: first global history of the batch
    PhaseRec* mid;                   // histories handed from the range-shifter to the aperture kernel (BEV)
    unsigned long long* mid_count;
    long long mid_cap;
    PhaseRec* phase;                 // histories handed from the aperture to the patient kernel
    unsigned long long* phase_count;
    long long phase_cap;
    // Scenarios share the beam-line transport: the random numbers do not
    // depend on the scenario, so a history's source, range shifter and
    // aperture are the same in all of them.  The beam-line kernels run over
    // the first scenario's items only and hand each survivor to the patient
    // kernel once per scenario, copy s into region s of the hand-off buffer.
    int n_rep;                       // scenarios sharing the beam-line transport (1: none)
    int rep_items;                   // items per scenario: copy s refers to item + s * rep_items
    long long rep_hist;              // histories per scenario: copy s has global index g + s * rep_hist
    long long rep_cap;               // records of one region of the hand-off buffer
    OvfRec* ovf;                     // out-of-box deposits (NULL: none expected)
    unsigned long long* ovf_count;   // records appended (may exceed ovf_cap: then re-run)
    long long ovf_cap;
    unsigned long long* stats;       // kNStats counters
    int* status;                     // device status word (bit 0: iteration cap)
    int max_iter;                    // iterations a history may take in one kernel
    HistRecord* records;
    long long rec_cap;
    uint32_t key0, key1_hi;
    int mcs, straggling, nuclear;
    float fscale;                    // 2^F
    int fx32;                        // 2^F <= 2^24: every energy x 2^F fits 32 bits (E <= 250 MeV)
    int unit_weight;                 // every item's wscale is 2^F (influence-matrix columns)
    MatConst water;                  // the patient medium's constants (the tables image's water entry)
    int aggregate;
    int chunk;
    // learned aperture surrogate
    int surrogate;                   // brass entries in its domain become queries
    SurQuery* sq;
    unsigned long long* sq_count;
    long long sq_cap;
    const float* poly_kappa;         // per polygon vertex: signed curvature, 1/mm
    // training tracks: histories start on the aperture entrance plane and
    // record the surrogate's inputs and targets, indexed by global history
    int track_mode;
    float* trk_feat;                 // [n x 6]
    float* trk_y;                    // [n x 5]
    int* trk_label;                  // [n]
    float* trk_frame;                // [n x 8] entry: x, y, w, n_x, n_y, u_n, u_t, E
};

// Shared-memory layouts of the two transport kernels.
struct SourceSmem {                  // source and range shifter
    static constexpr size_t R = 0;                                            // PMMA
    static constexpr size_t Einv = R + sizeof(float2) * kNEPad;
    static constexpr size_t Mat = Einv + sizeof(float2) * kNR;
    static constexpr size_t Beams = Mat + sizeof(MatConst) * kNMat;
    static constexpr size_t Bytes = Beams + sizeof(DevBeam) * kMaxBeams;
};
struct ApertureSmem {                // aperture block
    static constexpr size_t R = 0;                                            // brass
    static constexpr size_t Einv = R + sizeof(float2) * kNEPad;
    static constexpr size_t Mat = Einv + sizeof(float2) * kNR;
    static constexpr size_t Beams = Mat + sizeof(MatConst) * kNMat;
    static constexpr size_t Scens = Beams + sizeof(DevBeam) * kMaxBeams;
    static constexpr size_t Poly = Scens + sizeof(DevScen) * kMaxScen;
    static constexpr size_t Bytes = Poly + sizeof(float2) * kMaxPolyVerts;
};
constexpr int kPatientMaxBlock = 896;
struct PatientSmem {                 // voxelised patient
    static constexpr size_t R = 0;                                            // water
    static constexpr size_t Einv = R + sizeof(float2) * kNEPad;
    static constexpr size_t HU = Einv + sizeof(float2) * kNR;
    static constexpr size_t Scens = HU + sizeof(float2) * kNHU;
    // per thread: global index and work item of the history it carries (read
    // only when a history ends); per warp: the work pool [next, end)
    static constexpr size_t G = (Scens + sizeof(DevScen) * kMaxScen + 15) & ~size_t(15);
    static constexpr size_t Pool = G + sizeof(long long) * kPatientMaxBlock;
    static constexpr size_t Item = Pool + 2 * sizeof(long long) * (kPatientMaxBlock / 32);
    static constexpr size_t Bytes = Item + sizeof(int) * kPatientMaxBlock;
};
// One block per SM of each transport kernel: every layout fits the 227 KB a
// block may opt in to.
static_assert(SourceSmem::Bytes <= 227 * 1024, "source kernel shared memory");
static_assert(ApertureSmem::Bytes <= 227 * 1024, "aperture kernel shared memory");
static_assert(PatientSmem::Bytes <= 227 * 1024, "patient kernel shared memory");
static_assert(kPatientMaxBlock % 32 == 0, "whole warps");

// Host-side launchers (transport.cu, finalize.cu).
// Transport of histories [p.hist_begin, p.total): the beam-line kernels
// (source and range shifter, then the aperture: launch_devices, which resets
// p.counter between them), then the patient kernel on the histories they hand
// over (p.mid and p.phase must each hold p.total - p.hist_begin records).
// All launches are persistent grids of one block per SM.
cudaError_t launch_devices(const TransportParams& p, int grid, int block, cudaStream_t s);
cudaError_t launch_patient(const TransportParams& p, int grid, int block, cudaStream_t s);
// Which compiled nesting of the patient kernel serves these grids (bit k: axis k nested).
int patient_nest_variant(const int nest_shift[3]);
// Converts a device CT of hounsfield units, in place, to indices into the
// kernels' (density, SPR) table (HU clamped to [-1024, 3071]).
cudaError_t launch_ct_lut_index(int16_t* ct, long long n, cudaStream_t s);
size_t devices_smem_bytes();
size_t patient_smem_bytes();
int patient_max_block();
int devices_max_block();

// Learned aperture surrogate (surrogate.cu).
struct SurNet {
    float* params;                   // FP32 master parameters [kNParams]
    float* grad;                     // [kNParams]: the summed gradient (gradient entry point)
    float* gpart;                    // [n_part_cap x kNParams]: one partial gradient per CTA of a training launch
    int n_part_cap;
    float* m;                        // Adam moments
    float* v;
    unsigned char* img;              // BF16 operand images [kImgBytes]
    double* loss;                    // [2]: summed loss, rows
    int* status;                     // bit 0: a tensor-core wait timed out
};
cudaError_t launch_sur_pack(const SurNet& net, cudaStream_t s);
cudaError_t launch_sur_forward(const SurNet& net, const float* x, long long n, float* z, int grid, cudaStream_t s);
// One training launch over rows [first, first + rows); each of its *parts
// CTAs writes its partial gradient into net.gpart.
cudaError_t launch_sur_train(const SurNet& net, const float* x, const float* y, const int* label, long long first,
                             long long rows, long long n, float inv_rows, int grid, int* parts, cudaStream_t s);
// Adam step on the sum of the parts partial gradients.
cudaError_t launch_sur_adam(const SurNet& net, int step, float lr, int parts, cudaStream_t s);
// net.grad = the sum of the parts partial gradients.
cudaError_t launch_sur_reduce(const SurNet& net, int parts, cudaStream_t s);
cudaError_t launch_sur_infer(const SurNet& net, const TransportParams& p, int grid, cudaStream_t s);
size_t sur_forward_smem_bytes();
size_t sur_train_smem_bytes();

// Robust spot-weight optimisation (optimize.cu).  Matrices: n_scen CSR of
// n_rows x n_cols (device pointers); cls: uint8 voxel classes (1 target,
// 2 ring); x: device weights, optimised in place.
struct OptSpec {
    float dp, w_u, w_o, w_r, over, ring;    // prescription, weights, over- and ring-dose fractions
    long long n_target, n_ring;
    float step, eps;                        // Adam step (absolute) and epsilon
    int iterations;
};
struct OptSetupInfo {
    long long n_tr, nnz_tr;                 // target + ring rows; their entries over all scenarios
    long long compact_entries;              // padded size of the compact CSR
};
cudaError_t run_robust_optimize(const long long* const* rp, const int* const* col, const float* const* val, int n_scen,
                                long long n_rows, int n_cols, const unsigned char* cls_host, const OptSpec& spec,
                                float* x, float* hist_host, cudaStream_t st, float* ms_out, OptSetupInfo* info);
cudaError_t run_weights_dose(const long long* rp, const int* col, const float* val, long long n_rows, int n_cols,
                             const float* x, float* dose, cudaStream_t st, int num_sms);
cudaError_t run_target_indices(const long long* const* rp, const int* const* col, const float* const* val, int n_scen,
                               long long n_rows, int n_cols, const unsigned char* cls, float dp, const float* x,
                               double* out, cudaStream_t st, int num_sms);

cudaError_t launch_scoring_density(const int16_t* ct, Grid3 ctg, Grid3 sg, const double* curve15_dev,
                                   const double ct_spacing[3], const double sg_spacing[3], double* rho_out,
                                   cudaStream_t s);
cudaError_t launch_dose_normalise(const unsigned long long* acc, const double* rho, long long nvox, double scale,
                                  float* dose, cudaStream_t s);
// colmax[i] = max over item first_item + i's box of q x inv_rho (inv_rho: 1 / rho per scoring voxel, FP64;
// inv_rho_f: the same in FP32, for the screen).
cudaError_t launch_column_max(const unsigned long long* scratch, const DevItem* items, const DevBox* boxes,
                              const double* inv_rho, const float* inv_rho_f, const Grid3 sg, int first_item,
                              int n_items, double* colmax, cudaStream_t s);
// out = 1 / x in FP64, out_f its FP32 value.
cudaError_t launch_reciprocal(const double* x, long long n, double* out, float* out_f, cudaStream_t s);

struct CsrBuildParams {
    const unsigned long long* scratch;
    const DevItem* items;            // items of one scenario, in spot order (spots sorted by beam)
    const DevBox* boxes;
    const double* inv_rho;           // per scoring voxel: 1 / density (FP64)
    const double* thr;               // per item: rel_threshold x max of q / rho (FP64)
    const float* thr_f;              // the same in FP32 (the screen)
    const int* run_first;            // per run of items sharing one box: first item index (relative)
    const int* run_count;
    const int* run_box;              // per run: the box shared by its items (shape and origin)
    const int* run_block0;           // [n_runs + 1]: first block of each run in the box-major passes (kCountBlock threads)
    unsigned* box_slot;              // per box-major thread: its (voxel, run) count, then that segment's offset in the row
    int n_runs;
    const OvfRec* ovf;               // out-of-box deposits bucketed by voxel, sorted by item, merged
    const long long* bucket_off;     // per voxel of this scenario: first record
    const int* bucket_len;           // per voxel: merged records
    int item_base;                   // item index of this scenario's first item in the launch
    Grid3 sg;
    long long nvox;
    const double* item_scale;        // per item: 2^-F * (MeV/g -> Gy) / (V(cm^3) * n_hist)
    long long* row_count;            // [nvox + 1]
    const long long* row_ptr;        // for the fill pass
    int* col;
    float* val;
};
constexpr int kCountBlock = 256;      // threads per block of the box-major count pass
// Row counts (p.row_count, zeroed by the caller) of one scenario: box entries
// box-major over box_blocks blocks (each (voxel, run) count kept in
// p.box_slot), then the out-of-box records.
cudaError_t launch_csr_count(const CsrBuildParams& p, int box_blocks, cudaStream_t s);
// Column indices and values into p.col / p.val at p.row_ptr: the segments'
// offsets and the out-of-box records per voxel, then the box entries
// box-major over the same box_blocks blocks.
cudaError_t launch_csr_fill(const CsrBuildParams& p, int box_blocks, cudaStream_t s);
// thr[i] = rel x colmax[i] and its FP32 value, for the row passes' screen.
cudaError_t launch_column_threshold(const double* colmax, int n, double rel, double* thr, float* thr_f, cudaStream_t s);

// Rays parallel to one field's axis (beam frame base + a u + b v + t w) over
// a lateral grid of na x nb columns at spacing da, marched from t0 to t1 in
// steps dt; runs [run_off, run_off + run_n) of r_lim (ascending) are the
// water-equivalent ranges whose reach the job finds.
struct DepthJob {
    float base[3], u[3], v[3], w[3];
    float a0, b0, da;
    int na, nb;
    float t0, t1, dt;
    float spr_scale;
    int run_off, run_n;
};
// reach[run] (FP32 bits, zeroed by the caller): the largest t - t0 over the
// columns at which the water-equivalent path reaches r_lim[run].
cudaError_t launch_depth_bounds(const uint16_t* ct, const TablesImage* tables, Grid3 ctg, const DepthJob* jobs,
                                int n_jobs, const float* r_lim, unsigned* reach, cudaStream_t s);
// Counting sort of out-of-box records into per-(scenario, voxel) buckets,
// then per bucket: sort by item, merge duplicates, raise the column maxima.
cudaError_t launch_ovf_count(const OvfRec* rec, long long n, int n_spots, long long nvox, long long* bucket_cnt,
                             cudaStream_t s);
cudaError_t launch_ovf_scatter(const OvfRec* rec, long long n, int n_spots, long long nvox, const long long* bucket_off,
                               long long* cursor, OvfRec* sorted, cudaStream_t s);
cudaError_t launch_ovf_merge(OvfRec* sorted, const long long* bucket_off, long long n_buckets, long long nvox,
                             const double* rho, int* bucket_len, double* colmax, cudaStream_t s);
cudaError_t launch_exclusive_scan(const long long* in, long long* out, long long n, long long* block_tmp,
                                  cudaStream_t s);
size_t scan_tmp_elems(long long n);
int scan_launches(long long n);

}  // namespace vpmc
