// Mean bispectrum accumulation (Sect. 2 and Sect. 3.2: speckle masking,
// Weigelt 1977): for every pair (w, v) that the phase recursion reads,
//
//     B(w - v, v) = (1/F) sum_i I_i(w - v) I_i(v) conj I_i(w),
//
// with w in the upper half plane, 0 < |v| <= R, |v| < |w| and |w - v| < |w|.
//
// Work decomposition: a CTA owns a tile = 16 x 8 targets w x 8 x 4 offsets v
// of one subfield.  Warp q owns offset row vy0 + q; lane (wyl, gx) owns
// targets (wx0 + 4 gx + j, wy0 + wyl), j = 0..3, and offsets
// (vx0 + kk, vy0 + q), kk = 0..7: 32 complex accumulators in registers for
// the whole burst.  Per frame the CTA stages three rectangles of the frame
// spectrum in shared memory: the targets W (8 x 16), the offsets V (4 x 8)
// and U = W - V (11 x 23, staged 24 wide).  For its 32 pairs a thread reads
// 4 values of W, 8 broadcast values of V and an 11-wide sliding window of U
// (12 shared loads of 16 bytes for 32 pairs), so each triple product costs
// 8 FP32 FMA-pipe instructions.
//
// Spectra are staged by cp.async, four frames per barrier, while the
// previous four frames are multiplied out (half-precision spectra at half
// the bytes, converted to FP32 once per stage in shared memory).  W and U start at even box
// columns (the plan places the offset grid so that they do), so they move in
// 16-byte copies of two spectrum values, and so does V when the box's
// centre column K is odd: 212 copies per frame, two per thread (otherwise V
// takes 32 8-byte copies).  A last, partial stage is padded with zero-filled
// frames, which add nothing to the sums.  A warp skips the offset columns
// (and so whole tiles) in which none of its lanes owns a used pair; warps
// that own a used pair in every column run a copy of the frame loop without
// the column tests.  Accumulators are written once per burst.
#include "sm_bispec_tile.cuh"

namespace {

using smi::PlanDev;
using smb::BUF;
using smb::THREADS;

// Four CTAs per SM (128 registers a thread); the compensated sums keep a
// partial, a running sum and a correction per pair and take three (168).
template <int PREC, bool VCH, bool KAHAN>
__global__ void __launch_bounds__(THREADS, KAHAN ? 3 : 4)
k_bispectrum(PlanDev p, const void* __restrict__ spec, int F, float2* __restrict__ B) {
    __shared__ __align__(16) float2 S[smb::staging_float2<PREC>()];
    smb::bispec_tile<PREC, VCH, KAHAN>(p, spec, F, B, blockIdx.x, blockIdx.y, S);
}

}  // namespace

namespace smk {

cudaError_t launch_bispectrum(const smi::PlanDev& p, const void* spec, int F, int nsub, float2* B,
                              cudaStream_t st) {
    dim3 grid(p.n_tiles, nsub);
    const bool vch = ((p.v_org + p.K) & 1) == 0;     // every tile's V starts at an even column
    if (p.acc_mode == SM_ACC_KAHAN) {
        if (p.prec == SM_FP32) {
            if (vch) k_bispectrum<SM_FP32, true, true><<<grid, THREADS, 0, st>>>(p, spec, F, B);
            else k_bispectrum<SM_FP32, false, true><<<grid, THREADS, 0, st>>>(p, spec, F, B);
        } else if (p.prec == SM_FP16) {
            if (vch) k_bispectrum<SM_FP16, true, true><<<grid, THREADS, 0, st>>>(p, spec, F, B);
            else k_bispectrum<SM_FP16, false, true><<<grid, THREADS, 0, st>>>(p, spec, F, B);
        } else {
            if (vch) k_bispectrum<SM_BF16, true, true><<<grid, THREADS, 0, st>>>(p, spec, F, B);
            else k_bispectrum<SM_BF16, false, true><<<grid, THREADS, 0, st>>>(p, spec, F, B);
        }
    } else if (p.prec == SM_FP32) {
        if (vch) k_bispectrum<SM_FP32, true, false><<<grid, THREADS, 0, st>>>(p, spec, F, B);
        else k_bispectrum<SM_FP32, false, false><<<grid, THREADS, 0, st>>>(p, spec, F, B);
    } else if (p.prec == SM_FP16) {
        if (vch) k_bispectrum<SM_FP16, true, false><<<grid, THREADS, 0, st>>>(p, spec, F, B);
        else k_bispectrum<SM_FP16, false, false><<<grid, THREADS, 0, st>>>(p, spec, F, B);
    } else {
        if (vch) k_bispectrum<SM_BF16, true, false><<<grid, THREADS, 0, st>>>(p, spec, F, B);
        else k_bispectrum<SM_BF16, false, false><<<grid, THREADS, 0, st>>>(p, spec, F, B);
    }
    return cudaGetLastError();
}

}  // namespace smk
