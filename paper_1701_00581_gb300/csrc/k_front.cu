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

// Correlation tracking (Table 2's correlation-tracking row): per frame the
// integer shift s = (sx, sy), |sx|, |sy| <= S, maximising
// C(s) = sum over the central G x G window of a(x + s) (r(x) - mean r),
// r the reference frame, the first maximum in row-major (sy, sx) order;
// then the frames shifted by s with edge pixels replicated.
//
// k_track_ref: the reference window minus its mean (FP64 mean, one CTA).
// k_track_cc: one CTA per (sy, frame), one thread per sx; each window row
// of the frame (G + 2S samples) is staged in shared memory and every thread
// sums its products in FP32 over 32-sample chunks, the chunks in FP64.
// k_track_pick: the first maximum per frame.  k_shift: elementwise copy.
namespace {

constexpr int TRACK_MAX_S = 31;        // 2S + 1 <= 63 threads per CTA
constexpr int TRACK_REF_THREADS = 1024;

template <typename In>
__device__ __forceinline__ float sample(const In* f, size_t i) { return (float)f[i]; }

template <typename In>
__global__ void __launch_bounds__(TRACK_REF_THREADS)
k_track_ref(const In* __restrict__ frames, int W, int H, int ref, int x0, int y0, int G, float* __restrict__ rw) {
    __shared__ double red[TRACK_REF_THREADS];
    const In* r = frames + (size_t)ref * W * H;
    double s = 0.0;
    for (int i = threadIdx.x; i < G * G; i += TRACK_REF_THREADS)
        s += (double)sample(r, (size_t)(y0 + i / G) * W + x0 + i % G);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = TRACK_REF_THREADS / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    const float mean = (float)(red[0] / ((double)G * G));
    for (int i = threadIdx.x; i < G * G; i += TRACK_REF_THREADS)
        rw[i] = sample(r, (size_t)(y0 + i / G) * W + x0 + i % G) - mean;
}

template <typename In>
__global__ void k_track_cc(const In* __restrict__ frames, int W, int H, int x0, int y0, int G, int S,
                           const float* __restrict__ rw, double* __restrict__ cc) {
    extern __shared__ float trow[];     // [G + 2S] frame row, then [G] reference row
    float* rrow = trow + G + 2 * S;
    const int syi = blockIdx.x, f = blockIdx.y, sxi = threadIdx.x, n = 2 * S + 1;
    const int sy = syi - S;
    const In* a = frames + (size_t)f * W * H;
    double acc = 0.0;
    for (int y = 0; y < G; ++y) {
        __syncthreads();
        const size_t row = (size_t)(y0 + y + sy) * W + (x0 - S);
        for (int i = threadIdx.x; i < G + 2 * S; i += blockDim.x) trow[i] = sample(a, row + i);
        for (int i = threadIdx.x; i < G; i += blockDim.x) rrow[i] = rw[y * G + i];
        __syncthreads();
        if (sxi < n) {
            for (int c = 0; c < G; c += 32) {
                float part = 0.f;
                const int e = min(c + 32, G);
                for (int x = c; x < e; ++x) part = fmaf(trow[x + sxi], rrow[x], part);
                acc += (double)part;
            }
        }
    }
    if (sxi < n) cc[((size_t)f * n + syi) * n + sxi] = acc;
}

__global__ void k_track_pick(int F, int S, const double* __restrict__ cc, int* __restrict__ shifts) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    const int n = 2 * S + 1;
    const double* c = cc + (size_t)f * n * n;
    int best = 0;
    for (int k = 1; k < n * n; ++k)
        if (c[k] > c[best]) best = k;
    shifts[2 * f] = best % n - S;
    shifts[2 * f + 1] = best / n - S;
}

template <typename In>
__global__ void k_shift(size_t total, int W, int H, const In* __restrict__ frames, const int* __restrict__ shifts,
                        float* __restrict__ out) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t npx = (size_t)W * H;
        const int f = (int)(i / npx);
        const int p = (int)(i - (size_t)f * npx), y = p / W, x = p - y * W;
        const int yy = min(max(y + shifts[2 * f + 1], 0), H - 1);
        const int xx = min(max(x + shifts[2 * f], 0), W - 1);
        out[i] = sample(frames, (size_t)f * npx + (size_t)yy * W + xx);
    }
}

template <typename In>
cudaError_t track(const smi::PlanDev& p, const In* frames, int F, int ref, int G, int S, float* rw, double* cc,
                  int* shifts, cudaStream_t st) {
    const int x0 = (p.W - G) / 2, y0 = (p.H - G) / 2;
    k_track_ref<In><<<1, TRACK_REF_THREADS, 0, st>>>(frames, p.W, p.H, ref, x0, y0, G, rw);
    const int n = 2 * S + 1;
    const size_t sm = (size_t)(2 * G + 2 * S) * sizeof(float);
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_track_cc<In>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    k_track_cc<In><<<dim3(n, F), 64, sm, st>>>(frames, p.W, p.H, x0, y0, G, S, rw, cc);
    k_track_pick<<<(F + 127) / 128, 128, 0, st>>>(F, S, cc, shifts);
    return cudaGetLastError();
}

}  // namespace

namespace smk {

int track_max_search() { return TRACK_MAX_S; }

cudaError_t launch_track(const smi::PlanDev& p, const void* frames, int frame_type, int F, int ref, int G, int S,
                         float* rw, double* cc, int* shifts, cudaStream_t st) {
    if (frame_type == SM_U16)
        return track(p, static_cast<const uint16_t*>(frames), F, ref, G, S, rw, cc, shifts, st);
    return track(p, static_cast<const float*>(frames), F, ref, G, S, rw, cc, shifts, st);
}

cudaError_t launch_shift(const smi::PlanDev& p, const void* frames, int frame_type, int F, const int* shifts,
                         float* out, cudaStream_t st) {
    const size_t total = (size_t)F * p.W * p.H;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = (int)std::min<size_t>((size_t)sms * 8, (total + 255) / 256);
    if (frame_type == SM_U16)
        k_shift<uint16_t><<<blocks, 256, 0, st>>>(total, p.W, p.H, static_cast<const uint16_t*>(frames), shifts, out);
    else
        k_shift<float><<<blocks, 256, 0, st>>>(total, p.W, p.H, static_cast<const float*>(frames), shifts, out);
    return cudaGetLastError();
}

}  // namespace smk
