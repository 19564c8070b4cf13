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
// and U = W - V (11 x 23).  For its 32 pairs a thread reads 4 values of W,
// 8 broadcast values of V and an 11-wide sliding window of U, so each
// triple product costs 8 FP32 FMA-pipe instructions and ~0.7 shared loads.
// The next frame's rectangles are prefetched into registers while the
// current frame is multiplied out.  A warp skips the offset columns (and so
// whole tiles) in which none of its lanes owns a used pair.  Accumulators are
// written once per burst.
#include "sm_internal.h"

namespace {

using smi::PlanDev;
using smi::TILE_PAIRS;
using smi::TILE_V;
using smi::TILE_W;

constexpr int PW = 17;                  // row pitch of W in smem (conflict-free, see below)
constexpr int PU = 25;                  // row pitch of U in smem
constexpr int UR = smi::WBY + smi::VBY - 1;     // 15 rows of U
constexpr int UC = smi::WBX + smi::VBX - 1;     // 23 cols of U
constexpr int OFF_W = 0;
constexpr int OFF_V = smi::WBY * PW;                      // 136
constexpr int OFF_U = OFF_V + smi::VBY * smi::VBX;        // 168
constexpr int BUF = OFF_U + UR * PU;                      // 443 float2 per frame buffer
constexpr int NLOAD = smi::WBY * smi::WBX + smi::VBY * smi::VBX + UR * UC;  // 413
constexpr int THREADS = smi::BISPEC_THREADS;
constexpr int LPT = (NLOAD + THREADS - 1) / THREADS;      // 4 elements per thread

// Bank check (64-bit accesses, half-warp phases): lanes 0..15 hold
// wyl = 0..3, gx = 0..3 and read element wyl*P + 4*gx + m; with P = 17 or
// 25 the 16 word-pairs 2*(wyl*P + 4*gx) mod 32 are all distinct.

template <int PREC>
__device__ __forceinline__ float2 load_spec(const void* spec, size_t idx) {
    if (PREC == SM_FP32) {
        return __ldg(reinterpret_cast<const float2*>(spec) + idx);
    } else if (PREC == SM_FP16) {
        const __half2 h = reinterpret_cast<const __half2*>(spec)[idx];
        const float2 v = __half22float2(h);
        return make_float2(v.x * smi::FP16_INV_SCALE, v.y * smi::FP16_INV_SCALE);
    } else {
        const __nv_bfloat162 h = reinterpret_cast<const __nv_bfloat162*>(spec)[idx];
        return __bfloat1622float2(h);
    }
}

__device__ __forceinline__ bool pair_used(int wx, int wy, int vx, int vy, int r2i, int R2) {
    const int w2 = wx * wx + wy * wy, v2 = vx * vx + vy * vy;
    const int ux = wx - vx, uy = wy - vy, u2 = ux * ux + uy * uy;
    const bool inH = wy > 0 || (wy == 0 && wx > 0);
    return inH && w2 >= 2 && w2 <= r2i && v2 > 0 && v2 <= R2 && v2 < w2 && u2 < w2;
}

template <int PREC>
__global__ void __launch_bounds__(THREADS, 4)
k_bispectrum(PlanDev p, const void* __restrict__ spec, int F, float2* __restrict__ B) {
    __shared__ __align__(16) float2 S[2 * BUF];
    const int tile = blockIdx.x, sl = blockIdx.y;
    const int4 T = p.tiles[tile];
    const int wx0 = T.x, wy0 = T.y, vx0 = T.z, vy0 = T.w;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int wyl = lane >> 2, gx = lane & 3;

    // Which spectrum element each thread stages, and where it goes.
    int src[LPT], dst[LPT];
#pragma unroll
    for (int i = 0; i < LPT; ++i) {
        const int e = tid + i * THREADS;
        int kx = 0, ky = 0, d = -1;
        if (e < smi::WBY * smi::WBX) {
            const int r = e / smi::WBX, c = e - r * smi::WBX;
            kx = wx0 + c; ky = wy0 + r; d = OFF_W + r * PW + c;
        } else if (e < smi::WBY * smi::WBX + smi::VBY * smi::VBX) {
            const int e2 = e - smi::WBY * smi::WBX;
            const int r = e2 / smi::VBX, c = e2 - r * smi::VBX;
            kx = vx0 + c; ky = vy0 + r; d = OFF_V + r * smi::VBX + c;
        } else if (e < NLOAD) {
            const int e2 = e - smi::WBY * smi::WBX - smi::VBY * smi::VBX;
            const int r = e2 / UC, c = e2 - r * UC;
            kx = wx0 - vx0 - (smi::VBX - 1) + c; ky = wy0 - vy0 - (smi::VBY - 1) + r;
            d = OFF_U + r * PU + c;
        }
        dst[i] = d;
        const bool inbox = d >= 0 && ky >= -p.R && ky <= p.K && kx >= -p.K && kx <= p.K;
        src[i] = inbox ? (ky + p.R) * p.box_pitch + (kx + p.K) : -1;
    }

    // Offset columns kk for which some lane of this warp owns a used pair:
    // a warp-uniform mask, so the warp skips columns (and whole tiles) it
    // does not need without diverging.
    unsigned kkmask = 0;
#pragma unroll
    for (int kk = 0; kk < smi::VBX; ++kk) {
        bool mine = false;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            mine |= pair_used(wx0 + 4 * gx + j, wy0 + wyl, vx0 + kk, vy0 + warp, p.r2i, p.R * p.R);
        if (__any_sync(0xffffffffu, mine)) kkmask |= 1u << kk;
    }
    const bool active = kkmask != 0;

    const size_t box = (size_t)p.box_rows * p.box_pitch;
    const size_t sbase = (size_t)sl * F * box;
    float2 pre[LPT];
#pragma unroll
    for (int i = 0; i < LPT; ++i)
        pre[i] = src[i] >= 0 ? load_spec<PREC>(spec, sbase + src[i]) : make_float2(0.f, 0.f);

    float2 acc[4][smi::VBX];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int kk = 0; kk < smi::VBX; ++kk) acc[j][kk] = make_float2(0.f, 0.f);

    for (int f = 0; f < F; ++f) {
        float2* Sb = S + (f & 1) * BUF;
#pragma unroll
        for (int i = 0; i < LPT; ++i)
            if (dst[i] >= 0) Sb[dst[i]] = pre[i];
        __syncthreads();
        if (f + 1 < F) {
            const size_t fb = sbase + (size_t)(f + 1) * box;
#pragma unroll
            for (int i = 0; i < LPT; ++i)
                pre[i] = src[i] >= 0 ? load_spec<PREC>(spec, fb + src[i]) : make_float2(0.f, 0.f);
        }
        if (active) {
            float2 a[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float2 t = Sb[OFF_W + wyl * PW + 4 * gx + j];
                a[j] = make_float2(t.x, -t.y);          // conj I(w)
            }
            float2 c[11];
            const float2* up = Sb + OFF_U + (wyl - warp + smi::VBY - 1) * PU + 4 * gx;
#pragma unroll
            for (int m = 0; m < 11; ++m) c[m] = up[m];  // I(w - v), m = j - kk + 7
            const float2* vp = Sb + OFF_V + warp * smi::VBX;
#pragma unroll
            for (int kk = 0; kk < smi::VBX; ++kk) {
                if (!(kkmask & (1u << kk))) continue;    // warp-uniform
                const float2 b = vp[kk];                 // I(v), warp broadcast
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float2 u = c[j - kk + 7];
                    const float px = fmaf(u.x, b.x, -u.y * b.y);
                    const float py = fmaf(u.x, b.y, u.y * b.x);
                    acc[j][kk].x = fmaf(px, a[j].x, fmaf(-py, a[j].y, acc[j][kk].x));
                    acc[j][kk].y = fmaf(px, a[j].y, fmaf(py, a[j].x, acc[j][kk].y));
                }
            }
        }
    }

    if (!active) return;
    const float sc = 1.0f / (float)F;
    float2* out = B + (size_t)(sl * p.n_tiles + tile) * TILE_PAIRS;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float4* o = reinterpret_cast<float4*>(out + (wyl * smi::WBX + 4 * gx + j) * TILE_V +
                                              warp * smi::VBX);
#pragma unroll
        for (int q = 0; q < smi::VBX / 2; ++q)
            o[q] = make_float4(acc[j][2 * q].x * sc, acc[j][2 * q].y * sc,
                               acc[j][2 * q + 1].x * sc, acc[j][2 * q + 1].y * sc);
    }
}


}  // namespace

namespace smk {

cudaError_t launch_bispectrum(const smi::PlanDev& p, const void* spec, int F, int nsub, float2* B,
                              cudaStream_t st) {
    dim3 grid(p.n_tiles, nsub);
    if (p.prec == SM_FP32) k_bispectrum<SM_FP32><<<grid, THREADS, 0, st>>>(p, spec, F, B);
    else if (p.prec == SM_FP16) k_bispectrum<SM_FP16><<<grid, THREADS, 0, st>>>(p, spec, F, B);
    else k_bispectrum<SM_BF16><<<grid, THREADS, 0, st>>>(p, spec, F, B);
    return cudaGetLastError();
}

}  // namespace smk
