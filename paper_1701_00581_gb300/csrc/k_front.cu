// Front end (Table 2's first row: flat-field and dark-field preprocessing).
//
// k_gain: the detector's normalised gain g = (flat - dark) / mean(flat - dark),
// the mean over the pixels where flat > dark (g = 0 elsewhere).  Computed
// once per flat field, by one CTA: each thread sums its pixels in order in
// FP64, a fixed tree combines the threads, then the same CTA writes the map.
// k_calibrate: every frame sample (raw - dark) / g, 0 where g = 0; an
// elementwise pass bound by HBM (2 or 4 bytes read, 4 written per sample).
#include <algorithm>

#include "sm_internal.h"

namespace {

using smi::PlanDev;

constexpr int GAIN_THREADS = 1024;
constexpr int CAL_THREADS = 256;

__global__ void __launch_bounds__(GAIN_THREADS)
k_gain(int npx, const float* __restrict__ flat, const float* __restrict__ dark, float* __restrict__ gain) {
    __shared__ double ssum[GAIN_THREADS];
    __shared__ long long scnt[GAIN_THREADS];
    double s = 0.0;
    long long c = 0;
    for (int i = threadIdx.x; i < npx; i += GAIN_THREADS) {
        const double d = (double)flat[i] - (double)dark[i];
        if (d > 0.0) { s += d; ++c; }
    }
    ssum[threadIdx.x] = s;
    scnt[threadIdx.x] = c;
    __syncthreads();
    for (int h = GAIN_THREADS / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            ssum[threadIdx.x] += ssum[threadIdx.x + h];
            scnt[threadIdx.x] += scnt[threadIdx.x + h];
        }
        __syncthreads();
    }
    const double mean = scnt[0] > 0 ? ssum[0] / (double)scnt[0] : 0.0;
    for (int i = threadIdx.x; i < npx; i += GAIN_THREADS) {
        const double d = (double)flat[i] - (double)dark[i];
        gain[i] = (d > 0.0 && mean > 0.0) ? (float)(d / mean) : 0.f;
    }
}

template <typename In>
__global__ void __launch_bounds__(CAL_THREADS)
k_calibrate(size_t n, int npx, const In* __restrict__ raw, const float* __restrict__ dark,
            const float* __restrict__ gain, float* __restrict__ out) {
    for (size_t i = (size_t)blockIdx.x * CAL_THREADS + threadIdx.x; i < n; i += (size_t)gridDim.x * CAL_THREADS) {
        const int px = (int)(i % (size_t)npx);
        const float g = __ldg(gain + px);
        out[i] = g > 0.f ? ((float)raw[i] - __ldg(dark + px)) / g : 0.f;
    }
}

}  // namespace

namespace smk {

cudaError_t launch_gain(const smi::PlanDev& p, const float* flat, const float* dark, float* gain, cudaStream_t st) {
    k_gain<<<1, GAIN_THREADS, 0, st>>>(p.W * p.H, flat, dark, gain);
    return cudaGetLastError();
}

cudaError_t launch_calibrate(const smi::PlanDev& p, const void* raw, int frame_type, int F, const float* dark,
                             const float* gain, float* out, cudaStream_t st) {
    const int npx = p.W * p.H;
    const size_t n = (size_t)F * npx;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = (int)std::min<size_t>((size_t)sms * 8, (n + CAL_THREADS - 1) / CAL_THREADS);
    if (frame_type == SM_U16)
        k_calibrate<uint16_t><<<blocks, CAL_THREADS, 0, st>>>(n, npx, static_cast<const uint16_t*>(raw), dark, gain, out);
    else
        k_calibrate<float><<<blocks, CAL_THREADS, 0, st>>>(n, npx, static_cast<const float*>(raw), dark, gain, out);
    return cudaGetLastError();
}

}  // namespace smk
