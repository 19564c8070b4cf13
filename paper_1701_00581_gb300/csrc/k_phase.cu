// Recursive Fourier phase from the mean bispectrum (Sect. 3.2: speckle
// masking phase, Lohmann, Weigelt & Wirnitzer 1983).
//
// Since arg B(w - v, v) = phi(w - v) + phi(v) - phi(w), each split of a
// target w into two already known frequencies gives a phasor estimate of
// exp(i phi(w)).  One CTA per subfield walks the rings of equal |w|^2 in
// ascending order (points of one ring never depend on each other); warp q
// takes points q, q + 16, ... of the ring, its lanes sum
// exp(i(phi(w-v) + phi(v))) conj B over the offsets v in FP32 products and
// FP64 sums, and lane 0 stores z(w) = S / |S|.  The known phasors live in
// shared memory (FP32 copy for the products); the FP64 result goes to HBM.
#include "sm_internal.h"

namespace {

using smi::PlanDev;
using smi::TILE_PAIRS;
using smi::TILE_V;

constexpr int PH_THREADS = 512;
constexpr int PH_WARPS = PH_THREADS / 32;

__device__ __forceinline__ bool pair_used(int wx, int wy, int vx, int vy, int r2i, int R2) {
    const int w2 = wx * wx + wy * wy, v2 = vx * vx + vy * vy;
    const int ux = wx - vx, uy = wy - vy, u2 = ux * ux + uy * uy;
    const bool inH = wy > 0 || (wy == 0 && wx > 0);
    return inH && w2 >= 2 && w2 <= r2i && v2 > 0 && v2 <= R2 && v2 < w2 && u2 < w2;
}

// z of any frequency from the half-box copy (row 0 holds both signs).
__device__ __forceinline__ float2 zget(const float2* zs, int pitch, int K, int kx, int ky) {
    if (ky >= 0) return zs[ky * pitch + kx + K];
    const float2 t = zs[(-ky) * pitch - kx + K];
    return make_float2(t.x, -t.y);
}

__global__ void __launch_bounds__(PH_THREADS, 1)
k_phase(PlanDev p, const float2* __restrict__ B, const float2* __restrict__ M,
        double2* __restrict__ z) {
    extern __shared__ __align__(16) unsigned char smem[];
    float2* zs = reinterpret_cast<float2*>(smem);
    const int sl = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int K = p.K, pitch = p.box_pitch;
    const size_t hb = (size_t)p.hb_rows * pitch;
    double2* zo = z + (size_t)sl * hb;
    for (int e = tid; e < (int)hb; e += PH_THREADS) zs[e] = make_float2(0.f, 0.f);
    __syncthreads();
    if (tid == 0) {
        zs[K] = make_float2(1.f, 0.f);
        zo[K] = make_double2(1.0, 0.0);
        // anchors: z(e_x) = M(e_x)/|M(e_x)|, z(e_y) = M(e_y)/|M(e_y)|
        const float2 mx = M[(size_t)sl * hb + K + 1];
        const float2 my = M[(size_t)sl * hb + pitch + K];
        double n = hypot((double)mx.x, (double)mx.y);
        double2 ax = n > 0 ? make_double2(mx.x / n, mx.y / n) : make_double2(1.0, 0.0);
        n = hypot((double)my.x, (double)my.y);
        double2 ay = n > 0 ? make_double2(my.x / n, my.y / n) : make_double2(1.0, 0.0);
        zs[K + 1] = make_float2((float)ax.x, (float)ax.y);
        zs[K - 1] = make_float2((float)ax.x, -(float)ax.y);
        zs[pitch + K] = make_float2((float)ay.x, (float)ay.y);
        zo[K + 1] = ax;
        zo[K - 1] = make_double2(ax.x, -ax.y);
        zo[pitch + K] = ay;
    }
    __syncthreads();

    const int R2 = p.R * p.R;
    const bool unit = p.weight == SM_W_UNIT;
    for (int r = 0; r < p.n_rings; ++r) {
        const int pe = p.ring_start[r + 1];
        for (int pt = p.ring_start[r] + warp; pt < pe; pt += PH_WARPS) {
            const int2 w = p.points[pt];
            const int wbx = (w.x + K) / smi::WBX, wxl = (w.x + K) - wbx * smi::WBX;
            const int wby = w.y / smi::WBY, wyl = w.y - wby * smi::WBY;
            const int wb = wby * p.n_wbx + wbx;
            double sx = 0.0, sy = 0.0;
            const int t1 = p.wb_start[wb + 1];
            for (int ti = p.wb_start[wb]; ti < t1; ++ti) {
                const int t = p.wb_tiles[ti];
                const int4 Tt = p.tiles[t];
                const float2* bp = B + (size_t)(sl * p.n_tiles + t) * TILE_PAIRS +
                                   (wyl * smi::WBX + wxl) * TILE_V;
#pragma unroll
                for (int h = 0; h < TILE_V / 32; ++h) {
                    const int vl = lane + 32 * h;
                    const int vx = Tt.z + (vl % smi::VBX), vy = Tt.w + (vl / smi::VBX);
                    if (!pair_used(w.x, w.y, vx, vy, p.r2i, R2)) continue;
                    const float2 b = bp[vl];
                    const float2 zu = zget(zs, pitch, K, w.x - vx, w.y - vy);
                    const float2 zv = zget(zs, pitch, K, vx, vy);
                    const float2 q = make_float2(zu.x * zv.x - zu.y * zv.y, zu.x * zv.y + zu.y * zv.x);
                    float tx = q.x * b.x + q.y * b.y;      // q * conj(b)
                    float ty = q.y * b.x - q.x * b.y;
                    if (unit) {
                        const float m = sqrtf(b.x * b.x + b.y * b.y);
                        if (m > 0.f) {
                            tx /= m;
                            ty /= m;
                        } else {
                            tx = ty = 0.f;
                        }
                    }
                    sx += tx;
                    sy += ty;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                sx += __shfl_xor_sync(0xffffffffu, sx, o);
                sy += __shfl_xor_sync(0xffffffffu, sy, o);
            }
            if (lane == 0) {
                const double n = hypot(sx, sy);
                const double2 zz = n > 0 ? make_double2(sx / n, sy / n) : make_double2(1.0, 0.0);
                const int o = w.y * pitch + w.x + K;
                zs[o] = make_float2((float)zz.x, (float)zz.y);
                zo[o] = zz;
                if (w.y == 0) {
                    zs[-w.x + K] = make_float2((float)zz.x, -(float)zz.y);
                    zo[-w.x + K] = make_double2(zz.x, -zz.y);
                }
            }
        }
        __syncthreads();
    }
}

}  // namespace

namespace smk {

size_t phase_smem_bytes(int hb_rows, int box_pitch) {
    return (size_t)hb_rows * box_pitch * sizeof(float2);
}

cudaError_t launch_phase(const smi::PlanDev& p, int nsub, const float2* B, const float2* M,
                         double2* z, cudaStream_t st) {
    const size_t sm = phase_smem_bytes(p.hb_rows, p.box_pitch);
    cudaError_t e = cudaFuncSetAttribute(k_phase, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_phase<<<nsub, PH_THREADS, sm, st>>>(p, B, M, z);
    return cudaGetLastError();
}

}  // namespace smk
