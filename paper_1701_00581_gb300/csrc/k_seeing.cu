// Seeing estimate (Sect. 3.1: spectral ratio technique, von der Luehe 1984).
//
// The burst is cut into non-overlapping N x N cubes; each cube's spectral
// ratio |<I>|^2 / <|I|^2>, averaged over annuli of unit width, is fitted by
// the model ratio |T_LE|^2 / STF of a seeing D/r0 (Fried's long-exposure OTF
// T0 exp(-3.44 (rho D/r0)^(5/3)) squared over the model STF
// T0^2 exp(-6.88 (rho D/r0)^(5/3)) + ck (r0/D)^2 T0, both 1 at k = 0), and the
// cubes' r0 are averaged.  The cubes are subfields of the reconstruction
// grid, so their P, M and noise floor come from the stats stage.
//
// k_seeing: one CTA per subfield of the chunk (non-cubes return at once).
// Warps sum the annuli from the plan's index lists in FP64 (a fixed shuffle
// tree, so the result does not depend on scheduling), thread 0 picks the
// fitted annuli, each thread evaluates the least-squares cost of one of 256
// log-spaced D/r0 candidates, and thread 0 takes the first minimum and
// refines it by a parabola in log D/r0.  k_seeing_stf: the mean r0 and the
// model STF table at it, on the centred N x N grid.  All FP64: the work is
// a few thousand transcendental evaluations per cube.
#include <algorithm>

#include "sm_internal.h"

namespace {

using smi::PlanDev;

constexpr int SE_THREADS = 256;
constexpr int SE_GRID = 256;                  // D/r0 candidates, log-spaced
constexpr double SE_LO = 1.0, SE_HI = 64.0;   // candidate range
constexpr double SE_STOP = 0.05;              // fit annuli until the observed ratio drops below this
constexpr int SE_MAXB = 136;                  // annuli held in shared memory (K + 2 for fc N < 134)
static_assert(SE_GRID == SE_THREADS, "one candidate per thread");

__device__ __forceinline__ double otf_t0(double rho) {
    return (2.0 / M_PI) * (acos(rho) - rho * sqrt(1.0 - rho * rho));
}

// |T_LE|^2 / STF at rho = |k| / r < 1 and D/r0 = x, both normalised at k = 0.
__device__ __forceinline__ double ratio_model(double rho, double x, double ck) {
    const double T0 = otf_t0(rho);
    const double e = exp(-6.88 * pow(rho * x, 5.0 / 3.0));
    return T0 * T0 * e * (1.0 + ck / (x * x)) / (T0 * T0 * e + ck * T0 / (x * x));
}

__device__ __forceinline__ double log_candidate(double llo, double lhi, int i) {
    return llo + (lhi - llo) * ((double)i / (double)(SE_GRID - 1));
}

__global__ void __launch_bounds__(SE_THREADS)
k_seeing(PlanDev p, int F, int sub0, const float* __restrict__ P, const float2* __restrict__ M,
         const float* __restrict__ noise, double* __restrict__ seeing) {
    const int sl = blockIdx.x;
    const int cube = p.cube_of_sub[sub0 + sl];
    if (cube < 0) return;
    __shared__ double num[SE_MAXB], den[SE_MAXB], eps[SE_MAXB], J[SE_GRID];
    __shared__ int nfit;
    const size_t hb = (size_t)p.hb_rows * p.box_pitch;
    const float* Ps = P + sl * hb;
    const float2* Ms = M + sl * hb;
    const double nz = noise[sl], fF = (double)F;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // annulus sums: num_b = sum (F |M|^2 - P) / (F - 1), den_b = sum (P - noise)
    for (int b = warp; b < p.n_bins; b += SE_THREADS / 32) {
        double a = 0.0, c = 0.0;
        for (int i = p.ann_start[b] + lane; i < p.ann_start[b + 1]; i += 32) {
            const int e = p.ann_idx[i];
            const double pv = Ps[e];
            const float2 m = Ms[e];
            const double m2 = (double)m.x * m.x + (double)m.y * m.y;
            a += (fF * m2 - pv) / (fF - 1.0);
            c += pv - nz;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            c += __shfl_xor_sync(0xffffffffu, c, o);
        }
        if (lane == 0) { num[b] = a; den[b] = c; }
    }
    __syncthreads();
    // fitted annuli: b = 1, 2, ... inside the cutoff while den_b > 0 and the
    // observed ratio stays at or above SE_STOP
    if (threadIdx.x == 0) {
        int n = 0;
        for (int b = 1; b < p.n_bins; ++b) {
            if (!((double)b < p.rcut) || !(den[b] > 0.0) || num[b] / den[b] < SE_STOP) break;
            eps[n++] = num[b] / den[b];
        }
        nfit = n;
    }
    __syncthreads();
    const int n = nfit;
    const double llo = log(SE_LO), lhi = log(SE_HI);
    {
        const int i = threadIdx.x;
        const double x = exp(log_candidate(llo, lhi, i));
        double s = 0.0;
        for (int k = 0; k < n; ++k) {
            const double d = eps[k] - ratio_model((double)(k + 1) / p.rcut, x, p.ck);
            s += d * d;
        }
        J[i] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double xhat = SE_HI;
        if (n > 0) {
            int im = 0;
            for (int i = 1; i < SE_GRID; ++i)
                if (J[i] < J[im]) im = i;
            double t = log_candidate(llo, lhi, im);
            if (im > 0 && im < SE_GRID - 1) {
                const double curv = J[im - 1] - 2.0 * J[im] + J[im + 1];
                if (curv > 0.0) {
                    const double h = log_candidate(llo, lhi, 1) - log_candidate(llo, lhi, 0);
                    t += 0.5 * h * (J[im - 1] - J[im + 1]) / curv;
                }
            }
            xhat = exp(t);
        }
        seeing[cube] = xhat;
    }
}

__global__ void __launch_bounds__(SE_THREADS)
k_seeing_stf(PlanDev p, double* __restrict__ seeing, double* __restrict__ stf) {
    __shared__ double xs;
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int c = 0; c < p.n_cubes; ++c) s += 1.0 / seeing[c];
        xs = 1.0 / (s / (double)p.n_cubes);     // D over the mean r0
        if (blockIdx.x == 0) seeing[p.n_cubes] = xs;
    }
    __syncthreads();
    const double x = xs, ck = p.ck;
    const int N = p.N;
    const double norm = 1.0 + ck / (x * x);      // the model at k = 0
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < N * N; e += gridDim.x * blockDim.x) {
        const int ky = e / N - N / 2, kx = e % N - N / 2;
        const double rho = hypot((double)kx, (double)ky) / p.rcut;
        double v = 0.0;
        if (rho <= 1.0) {
            const double T0 = otf_t0(rho);
            v = T0 * T0 * exp(-6.88 * pow(rho * x, 5.0 / 3.0)) + ck * T0 / (x * x);
        }
        stf[e] = v / norm;
    }
}

}  // namespace

namespace smk {

cudaError_t launch_seeing(const smi::PlanDev& p, int F, int sub0, int nsub, const float* P, const float2* M,
                          const float* noise, double* seeing, cudaStream_t st) {
    k_seeing<<<nsub, SE_THREADS, 0, st>>>(p, F, sub0, P, M, noise, seeing);
    return cudaGetLastError();
}

cudaError_t launch_seeing_stf(const smi::PlanDev& p, double* seeing, double* stf, cudaStream_t st) {
    const int blocks = std::min(256, (p.N * p.N + SE_THREADS - 1) / SE_THREADS);
    k_seeing_stf<<<blocks, SE_THREADS, 0, st>>>(p, seeing, stf);
    return cudaGetLastError();
}

int seeing_max_bins() { return SE_MAXB; }

}  // namespace smk
