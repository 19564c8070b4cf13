// Internal types shared by the host plan builder, the engine and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "speckle.h"

namespace smi {

// Bispectrum tile geometry (Sect. 2 / 3.2 speckle masking): a CTA owns a
// block of WBX x WBY target frequencies w and a block of VBX x VBY offsets v.
// Warp q of the CTA owns offset row vy0 + q; lane (wyl, gx) owns the four
// targets (wx0 + 4 gx + j, wy0 + wyl), j = 0..3, and the eight offsets
// (vx0 + kk, vy0 + q), kk = 0..7.  Four warps per CTA let four CTAs share
// an SM, so warps of different tiles fill each other's idle issue slots.
constexpr int WBX = 16, WBY = 8, VBX = 8, VBY = 4;
constexpr int TILE_W = WBX * WBY;            // 128 targets
constexpr int TILE_V = VBX * VBY;            // 32 offsets
constexpr int TILE_PAIRS = TILE_W * TILE_V;  // 4096 (w, v) slots
constexpr int BISPEC_THREADS = 32 * VBY;     // one warp per offset row
static_assert(TILE_V == 32, "a tile row of offsets maps onto the 32 lanes of a warp");

// Least-squares refinement partials per bispectrum tile: one per target w
// (128), per difference u = w - v of the tile's 11 x 23 rectangle (253) and
// per offset v (32).
constexpr int REF_W = TILE_W, REF_U = (WBY + VBY - 1) * (WBX + VBX - 1), REF_V = TILE_V;
constexpr int REF_SLOTS = REF_W + REF_U + REF_V;   // 413

constexpr float FP16_SCALE = 16384.0f;       // |I_n| <= 1 -> fits half with margin
constexpr float FP16_INV_SCALE = 1.0f / 16384.0f;

// Everything a kernel needs to know about a plan, passed by value.
struct PlanDev {
    int N, logN, K, R;
    int W, H, stride, taper;
    int n_sub, nsx, nsy;
    int box_rows, box_cols, box_pitch, hb_rows;
    int r2i;                 // floor((fc N)^2): |k|^2 <= r2i  <=>  |k| <= fc N
    int n_tiles, n_rings, n_points;
    int n_wbx, n_wby;
    int v_org;               // x origin of the offset-block grid (odd: -R, or -R - 7 for even R),
                             //   so that every difference rectangle starts at an even box column
    int prec, weight;
    int acc_mode, phase_prec;
    int phase_iters;         // least-squares sweeps after the recursion
    int mosaic_mode;         // SM_MOSAIC_BLEND / SM_MOSAIC_CENTRAL
    double photon_gain;      // photons per count (> 0: photon-noise bias removal)
    const int* ref_start;    // [n_points + 1] CSR: refinement partial slots of each point
    const int* ref_idx;      //   tile * REF_SLOTS + slot, bit 31 = conjugate (lower-half occurrence)
    const int4* subs;        // [n_sub] x0, y0, w, h
    const float* winx;       // [n_sub][N] window along x (0 beyond the extent)
    const float* winy;       // [n_sub][N]
    const double* winsum;    // [n_sub] sum of the 2-D window
    const float2* winft;     // [n_sub][K+1] DFT of the x window at kx = 0..K
    const float2* tw;        // [N] exp(-2 pi i k / N)
    const int4* tiles;       // [n_tiles] wx0, wy0, vx0, vy0
    const unsigned* tile_masks;  // [n_tiles] byte q (offset row q, one warp of a tile's CTA): bit e
                                 //   set when column e holds a used pair of some target
    const int* ring_start;   // [n_rings + 1]
    const int2* points;      // [n_points] (wx, wy), ring-ordered
    const int* wb_start;     // [n_wbx * n_wby + 1] CSR: tiles of each w-block
    const int* wb_tiles;
    // phase recursion work items: (point, tile) pairs holding at least one
    // pair the point reads, grouped by point, points in ring order
    const int4* items;          // [n_items] packed (w, offset origin) bytes, B offset
                                //   within the subfield, mask of lanes whose pair is read
    const int* ring_items;      // [n_rings + 1] first item of each ring
    const int* point_items;     // [n_points + 1] first item of each point
    const int4* point_rec;      // [n_points] (wx, wy, first item, end item), items counted
                                //   from the first item of the point's ring
    int n_items, max_ring_items, max_ring_points;
    // seeing (Sect. 3.1): the non-overlapping N x N cubes among the
    // subfields and the annuli of unit width over the half-plane domain
    int n_cubes;
    double rcut, ck;         // cutoff radius fc N in DFT bins; Korff constant of the model STF
    const int* cube_of_sub;  // [n_sub] cube index or -1
    int n_bins;              // K + 2 annuli b = 0..K+1 (nearest integer |k|)
    const int* ann_start;    // [n_bins + 1] CSR over ann_idx
    const int* ann_idx;      // half-box element index (ky * box_pitch + kx + K), row-major per annulus
    const double* t0;        // [hb_rows][box_pitch] diffraction OTF on the half box
};

constexpr int MAX_BATCH = 8;

// One burst of a batched launch (k_batch.cu): its channel's plan, its frames
// and the workspace buffers of all of its subfields (one chunk).
struct BatchBurst {
    PlanDev p;
    const void* frames;
    int frame_type, F;
    void* spec;
    float* flux;
    float* mu;
    float2* B;
    int cnt_base;            // first of the burst's per-subfield dependency counters
    int need;                // counter value a tile waits for: F when the launch
                             //   transforms the frames, 0 when they were transformed before
};
// Buffers of the bursts of one plan in the batched tile grid.
struct BatchPtrs {
    const void* spec[MAX_BATCH];
    float2* B[MAX_BATCH];
    int F[MAX_BATCH];
    int n;
};
// Kernel argument of the batched launch (passed by value, so a captured
// graph holds it).
struct BatchArgs {
    BatchBurst b[MAX_BATCH];
    int n;
};

}  // namespace smi

// ---- kernel launchers (defined in the .cu files) ---------------------------
namespace smk {
cudaError_t launch_spectra(const smi::PlanDev& p, const void* frames, int frame_type, int F,
                           int sub0, int nsub, void* spec, float* flux, float* mu,
                           cudaStream_t st);
cudaError_t launch_stats(const smi::PlanDev& p, const void* spec, int F, int nsub, float* P,
                         float2* M, float* noise, cudaStream_t st);
cudaError_t launch_amplitude(const smi::PlanDev& p, int nsub, const double* stf, const float* P,
                             const float* noise, float* A, cudaStream_t st);
cudaError_t launch_gain(const smi::PlanDev& p, const float* flat, const float* dark, float* gain, cudaStream_t st);
cudaError_t launch_calibrate(const smi::PlanDev& p, const void* raw, int frame_type, int F, const float* dark,
                             const float* gain, float* out, cudaStream_t st);
int track_max_search();   // largest search half-width S of the tracking kernel
cudaError_t launch_track(const smi::PlanDev& p, const void* frames, int frame_type, int F, int ref, int G, int S,
                         float* rw, double* cc, int* shifts, cudaStream_t st);
cudaError_t launch_shift(const smi::PlanDev& p, const void* frames, int frame_type, int F, const int* shifts,
                         float* out, cudaStream_t st);
cudaError_t launch_seeing(const smi::PlanDev& p, int F, int sub0, int nsub, const float* P, const float2* M,
                          const float* noise, double* seeing, cudaStream_t st);
cudaError_t launch_seeing_stf(const smi::PlanDev& p, double* seeing, double* stf, cudaStream_t st);
int seeing_max_bins();   // annuli the seeing kernel holds in shared memory
cudaError_t launch_unbias(const smi::PlanDev& p, int F, int nsub, const float* flux, const float* P, float2* B,
                          cudaStream_t st);
cudaError_t launch_bispectrum(const smi::PlanDev& p, const void* spec, int F, int nsub,
                              float2* B, cudaStream_t st);
cudaError_t launch_refine(const smi::PlanDev& p, int nsub, const float2* B, const float* P, double2* z,
                          float2* partials, cudaStream_t st);
cudaError_t launch_phase(const smi::PlanDev& p, int nsub, const float2* B, const float2* M, const float* P,
                         double2* z, cudaStream_t st, int threads = 512);
cudaError_t launch_inverse(const smi::PlanDev& p, int F, int sub0, int nsub, const float* A,
                           const double2* z, const float* flux, const float* mu, float* rec,
                           cudaStream_t st);
cudaError_t launch_mosaic(const smi::PlanDev& p, const float* rec, float* out, uint8_t* valid,
                          cudaStream_t st);
cudaError_t launch_batch_grid(const smi::PlanDev& p, const smi::BatchPtrs& q, cudaStream_t st);
size_t spectra_smem_bytes(int N, int K);
size_t batch_smem_bytes(int N, int K, int prec);
int batch_blocks_per_sm(size_t smem, int prec, int minb);
cudaError_t launch_batch(const smi::BatchArgs& a, int prec, int minb, const int4* items, int n_items, int* head,
                         int* cnt, int* status, float2* scratch, size_t scr_elems, int grid, size_t smem,
                         cudaStream_t st);
size_t phase_smem_bytes(int hb_rows, int box_pitch, int max_ring_items, int max_ring_points,
                        int phase_prec);
}  // namespace smk
