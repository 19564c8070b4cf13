// Least-squares refinement of the recursive phase (Sect. 3.2: the phase from
// the bispectrum "recursively or iteratively").
//
// Every split w = u + v the recursion reads ties three phases:
// arg B(u, v) = phi(u) + phi(v) - phi(w).  A sweep maximises
// sum g Re[conj B z(u) z(v) conj z(w)] one phase at a time from the previous
// sweep's phases (Jacobi): z(k) = S_k / |S_k| with
//   S_k = sum_{w=k} g z(u) z(v) conj B + sum_{u=k} g z(w) conj z(v) B
//       + sum_{v=k} g z(w) conj z(u) B
// (g = 1, 1/|B| or 1/(P(u) P(v) P(w)) by the channel's weighting; lower-half
// occurrences fold onto k conjugated; the anchors stay fixed).
//
// k_refine_tiles: one CTA per (bispectrum tile, subfield), laid out like
// the bispectrum kernel (warp = offset row, lane = 4 targets), reads each
// stored B once and reduces the three contributions of its 4096 slots into
// 413 partials in fixed orders: per target over the warps in shared memory,
// per difference over the tile's splits in shared memory, per offset along
// a warp shuffle tree.  The tile touches 413 distinct frequencies (its
// targets, offsets and differences); their phasors (and powers, for the SNR
// weighting) are staged in shared memory first, and each thread issues the
// loads of its 32 stored values before using any.
//
// k_refine_gather: eight CTAs per subfield, one warp per recursion point,
// sums the point's partials from the plan's list along a fixed tree and
// renormalises.  No atomics: the result does not depend on scheduling.
#include "sm_internal.h"

namespace {

using smi::PlanDev;
using smi::REF_SLOTS;
using smi::REF_U;
using smi::REF_V;
using smi::REF_W;
using smi::TILE_PAIRS;
using smi::TILE_V;

constexpr int RT_THREADS = smi::BISPEC_THREADS;     // 128: 4 warps = 4 offset rows
constexpr int UCOLS = smi::WBX + smi::VBX - 1;      // 23 difference columns
constexpr int RG_THREADS = 512;
// contributions to the differences, one row of 32 slots per target padded
// to 33: lanes of a warp hold different targets, so an unpadded row pitch
// of 32 float2 put all 32 lanes on one shared-memory bank
constexpr int CU_PITCH = TILE_V + 1;
constexpr int RG_BLOCKS = 8;                        // gather CTAs per subfield

__device__ __forceinline__ bool pair_used(int wx, int wy, int vx, int vy, int r2i, int R2) {
    const int w2 = wx * wx + wy * wy, v2 = vx * vx + vy * vy;
    const int ux = wx - vx, uy = wy - vy, u2 = ux * ux + uy * uy;
    const bool inH = wy > 0 || (wy == 0 && wx > 0);
    return inH && w2 >= 2 && w2 <= r2i && v2 > 0 && v2 <= R2 && v2 < w2 && u2 < w2;
}

// z of any frequency inside the disk from the FP64 half-box table.
__device__ __forceinline__ float2 zget(const double2* z, int pitch, int K, int kx, int ky) {
    if (ky >= 0) {
        const double2 t = z[ky * pitch + kx + K];
        return make_float2((float)t.x, (float)t.y);
    }
    const double2 t = z[(-ky) * pitch - kx + K];
    return make_float2((float)t.x, -(float)t.y);
}

// P of any frequency (P(-k) = P(k)).
__device__ __forceinline__ float pget(const float* P, int pitch, int K, int kx, int ky) {
    return ky >= 0 ? __ldg(P + ky * pitch + kx + K) : __ldg(P + (-ky) * pitch - kx + K);
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

__global__ void __launch_bounds__(RT_THREADS)
k_refine_tiles(PlanDev p, const float2* __restrict__ B, const float* __restrict__ P,
               const double2* __restrict__ z, float2* __restrict__ partials) {
    __shared__ float2 cu[smi::TILE_W * CU_PITCH]; // contributions to u = w - v: [target][offset slot]
    __shared__ float2 cw[smi::VBY][REF_W];        // per offset row: contributions to each target
    __shared__ float2 zt[REF_SLOTS];              // phasors of the tile's targets | differences | offsets
    __shared__ float pt[REF_SLOTS];               // their powers (SNR weighting)
    const int tile = blockIdx.x, sl = blockIdx.y;
    const int4 T = p.tiles[tile];
    const int wx0 = T.x, wy0 = T.y, vx0 = T.z, vy0 = T.w;
    const int tid = threadIdx.x, q = tid >> 5, lane = tid & 31;
    const int wyl = lane >> 2, gx = lane & 3;
    const int K = p.K, pitch = p.box_pitch, R2 = p.R * p.R;
    const size_t hb = (size_t)p.hb_rows * pitch;
    const double2* zs = z + sl * hb;
    const float* Ps = P + sl * hb;
    const float2* Bt = B + (size_t)(sl * p.n_tiles + tile) * TILE_PAIRS;
    const int ux0 = wx0 - vx0 - (smi::VBX - 1), uy0 = wy0 - vy0 - (smi::VBY - 1);
    const bool snr = p.weight == SM_W_SNR;
    for (int e = tid; e < REF_SLOTS; e += RT_THREADS) {
        int kx, ky;
        if (e < REF_W) { kx = wx0 + e % smi::WBX; ky = wy0 + e / smi::WBX; }
        else if (e < REF_W + REF_U) { const int c = e - REF_W; kx = ux0 + c % UCOLS; ky = uy0 + c / UCOLS; }
        else { const int c = e - REF_W - REF_U; kx = vx0 + c % smi::VBX; ky = vy0 + c / smi::VBX; }
        // only frequencies inside the disk are read by used pairs
        const bool in = kx * kx + ky * ky <= p.r2i;
        zt[e] = in ? zget(zs, pitch, K, kx, ky) : make_float2(0.f, 0.f);
        pt[e] = (in && snr) ? pget(Ps, pitch, K, kx, ky) : 1.f;
    }
    __syncthreads();
    const int wy = wy0 + wyl, vy = vy0 + q;
    float2 sv[smi::VBX];                          // this lane's targets' contributions to each offset
#pragma unroll
    for (int kk = 0; kk < smi::VBX; ++kk) sv[kk] = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int wcol = 4 * gx + j, wx = wx0 + wcol;
        const int wslot = wyl * smi::WBX + wcol;
        float2 sw = make_float2(0.f, 0.f);
        const float2 zw = zt[wslot];
        const float pw = pt[wslot];
        // the 8 stored values of this target's offset row are 64 contiguous
        // bytes: four independent 16-byte loads, issued before any use (a
        // slot of an unused pair may hold anything; it is never used)
        const float4* b4 = reinterpret_cast<const float4*>(Bt + wslot * TILE_V + q * smi::VBX);
        float4 bq[smi::VBX / 2];
#pragma unroll
        for (int h = 0; h < smi::VBX / 2; ++h) bq[h] = __ldg(b4 + h);
#pragma unroll
        for (int kk = 0; kk < smi::VBX; ++kk) {
            const int vx = vx0 + kk;
            float2 tu = make_float2(0.f, 0.f);
            if (pair_used(wx, wy, vx, vy, p.r2i, R2)) {
                const float2 b = (kk & 1) ? make_float2(bq[kk >> 1].z, bq[kk >> 1].w)
                                          : make_float2(bq[kk >> 1].x, bq[kk >> 1].y);
                const int ucell = REF_W + (wyl - q + smi::VBY - 1) * UCOLS + 4 * gx + j - kk + smi::VBX - 1;
                const int vcell = REF_W + REF_U + q * smi::VBX + kk;
                const float2 zu = zt[ucell];
                const float2 zv = zt[vcell];
                float g = 1.f;
                if (p.weight == SM_W_UNIT) {
                    const float m = sqrtf(b.x * b.x + b.y * b.y);
                    g = m > 0.f ? 1.f / m : 0.f;
                } else if (snr) {
                    const float den = pt[ucell] * pt[vcell] * pw;
                    g = den > 0.f ? 1.f / den : 0.f;
                }
                const float2 a = cmul(cmul(zu, zv), cconj(b));                 // as w
                sw.x += g * a.x;
                sw.y += g * a.y;
                const float2 c1 = cmul(cmul(zw, cconj(zv)), b);               // as u
                tu = make_float2(g * c1.x, g * c1.y);
                const float2 c2 = cmul(cmul(zw, cconj(zu)), b);               // as v
                sv[kk].x += g * c2.x;
                sv[kk].y += g * c2.y;
            }
            cu[wslot * CU_PITCH + q * smi::VBX + kk] = tu;
        }
        cw[q][wslot] = sw;
    }
    __syncthreads();
    float2* out = partials + (size_t)(sl * p.n_tiles + tile) * REF_SLOTS;
    // targets: the four offset rows in order
    {
        const int t = tid;   // 128 targets
        float2 s = cw[0][t];
#pragma unroll
        for (int r = 1; r < smi::VBY; ++r) { s.x += cw[r][t].x; s.y += cw[r][t].y; }
        out[t] = s;
    }
    // differences: cell (ur, uc) collects the splits with w = u + v in the tile,
    // offsets in row-major order
    for (int cell = tid; cell < REF_U; cell += RT_THREADS) {
        const int ur = cell / UCOLS, uc = cell - ur * UCOLS;
        float2 s = make_float2(0.f, 0.f);
#pragma unroll
        for (int qq = 0; qq < smi::VBY; ++qq) {
            const int tr = ur + qq - (smi::VBY - 1);
            if (tr < 0 || tr >= smi::WBY) continue;
#pragma unroll
            for (int kk = 0; kk < smi::VBX; ++kk) {
                const int tc = uc + kk - (smi::VBX - 1);
                if (tc < 0 || tc >= smi::WBX) continue;
                const float2 c = cu[(tr * smi::WBX + tc) * CU_PITCH + qq * smi::VBX + kk];
                s.x += c.x;
                s.y += c.y;
            }
        }
        out[REF_W + cell] = s;
    }
    // offsets: every lane of warp q holds the same 8 offsets; sum over the
    // 32 lanes (128 targets) along a fixed butterfly
#pragma unroll
    for (int kk = 0; kk < smi::VBX; ++kk) {
        float2 s = sv[kk];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
            s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
        }
        if (lane == 0) out[REF_W + REF_U + q * smi::VBX + kk] = s;
    }
}

__global__ void __launch_bounds__(RG_THREADS)
k_refine_gather(PlanDev p, const float2* __restrict__ partials, double2* __restrict__ z) {
    const int sl = blockIdx.x, lane = threadIdx.x & 31;
    const int gwarp = blockIdx.y * (RG_THREADS / 32) + (threadIdx.x >> 5);
    const int nwarp = gridDim.y * (RG_THREADS / 32);
    const int K = p.K, pitch = p.box_pitch;
    double2* zs = z + (size_t)sl * p.hb_rows * pitch;
    const float2* part = partials + (size_t)sl * p.n_tiles * REF_SLOTS;
    for (int pi = gwarp; pi < p.n_points; pi += nwarp) {
        double sx = 0.0, sy = 0.0;
        const int a0 = p.ref_start[pi], a1 = p.ref_start[pi + 1];
        // two entries per lane per step, both loads in flight together
        for (int a = a0 + lane; a < a1; a += 64) {
            const bool two = a + 32 < a1;
            const int e0 = p.ref_idx[a];
            const int e1 = two ? p.ref_idx[a + 32] : 0;
            const float2 c0 = part[e0 & 0x7fffffff];
            const float2 c1 = two ? part[e1 & 0x7fffffff] : make_float2(0.f, 0.f);
            sx += (double)c0.x + (double)c1.x;
            sy += (e0 < 0 ? -(double)c0.y : (double)c0.y) + (e1 < 0 ? -(double)c1.y : (double)c1.y);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sx += __shfl_xor_sync(0xffffffffu, sx, o);
            sy += __shfl_xor_sync(0xffffffffu, sy, o);
        }
        if (lane == 0) {
            const double n = sqrt(sx * sx + sy * sy);
            if (n > 0.0) {
                const int2 w = p.points[pi];
                const double2 zz = make_double2(sx / n, sy / n);
                zs[w.y * pitch + w.x + K] = zz;
                if (w.y == 0) zs[-w.x + K] = make_double2(zz.x, -zz.y);
            }
        }
    }
}

}  // namespace

namespace smk {

cudaError_t launch_refine(const smi::PlanDev& p, int nsub, const float2* B, const float* P, double2* z,
                          float2* partials, cudaStream_t st) {
    for (int it = 0; it < p.phase_iters; ++it) {
        k_refine_tiles<<<dim3(p.n_tiles, nsub), RT_THREADS, 0, st>>>(p, B, P, z, partials);
        k_refine_gather<<<dim3(nsub, RG_BLOCKS), RG_THREADS, 0, st>>>(p, partials, z);
    }
    return cudaGetLastError();
}

}  // namespace smk
