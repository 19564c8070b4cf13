// Device helpers of the subfield transforms (Sect. 2: Fourier transform of
// every subimage), shared by the per-stage kernels (k_fft.cu) and the batched
// persistent launch (k_batch.cu): an in-register radix-2 FFT and the
// four-step split of an N-point transform over a group of threads.
#pragma once
#include "sm_internal.h"

namespace smf {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// In-register radix-2 FFT of length L (decimation in time, bit-reversed
// input order resolved at compile time).  tw[m] = exp(-2 pi i m / N) for the
// transform size N of the kernel; W_L^k = tw[k N / L].  INV conjugates.
__host__ __device__ constexpr int bitrev(int i, int bits) {
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
    return r;
}
__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }

template <int L, int N, bool INV>
__device__ __forceinline__ void reg_fft(float2 (&v)[L], const float2* tw) {
    constexpr int LB = ilog2(L);
#pragma unroll
    for (int i = 0; i < L; ++i) {
        const int j = bitrev(i, LB);
        if (j > i) {
            const float2 t = v[i];
            v[i] = v[j];
            v[j] = t;
        }
    }
#pragma unroll
    for (int len = 2; len <= L; len <<= 1) {
        const int half = len / 2;
#pragma unroll
        for (int j = 0; j < half; ++j) {
            float2 w = tw[j * (N / len)];
            if (INV) w.y = -w.y;
#pragma unroll
            for (int i = 0; i < L; i += len) {
                const float2 a = v[i + j];
                const float2 b = v[i + j + half];
                const float2 t = j == 0 ? b : cmul(b, w);
                v[i + j] = make_float2(a.x + t.x, a.y + t.y);
                v[i + j + half] = make_float2(a.x - t.x, a.y - t.y);
            }
        }
    }
}

// Four-step split of an N-point transform: N = P * Q, thread n1 < P of a
// group holds x[n1 + P n2] (n2 < Q) on entry; on exit thread k2 < Q holds
// X[k2 + Q k1] (k1 < P) in out[].  T is the group's [Q][P+1] exchange tile.
template <int N> struct Split;
template <> struct Split<64> { static constexpr int P = 8, Q = 8; };
template <> struct Split<128> { static constexpr int P = 8, Q = 16; };
template <> struct Split<256> { static constexpr int P = 16, Q = 16; };

template <int N, bool INV>
__device__ __forceinline__ void four_step(float2 (&v)[Split<N>::Q], float2 (&out)[Split<N>::P],
                                          float2* T, const float2* tw, int g) {
    constexpr int P = Split<N>::P, Q = Split<N>::Q;
    if (g < P) {
        reg_fft<Q, N, INV>(v, tw);
#pragma unroll
        for (int k2 = 0; k2 < Q; ++k2) {
            float2 w = tw[g * k2];
            if (INV) w.y = -w.y;
            T[k2 * (P + 1) + g] = k2 == 0 ? v[k2] : cmul(v[k2], w);
        }
    }
    __syncwarp();
    if (g < Q) {
#pragma unroll
        for (int n1 = 0; n1 < P; ++n1) out[n1] = T[g * (P + 1) + n1];
        reg_fft<P, N, INV>(out, tw);
    }
    __syncwarp();
}

__device__ __forceinline__ float load_sample(const uint16_t* p) { return (float)__ldg(p); }
__device__ __forceinline__ float load_sample(const float* p) { return __ldg(p); }

template <int PREC>
__device__ __forceinline__ void store_spec(void* spec, size_t idx, float2 v) {
    if (PREC == SM_FP32) {
        reinterpret_cast<float2*>(spec)[idx] = v;
    } else if (PREC == SM_FP16) {
        reinterpret_cast<__half2*>(spec)[idx] =
            __floats2half2_rn(v.x * smi::FP16_SCALE, v.y * smi::FP16_SCALE);
    } else {
        reinterpret_cast<__nv_bfloat162*>(spec)[idx] = __floats2bfloat162_rn(v.x, v.y);
    }
}


}  // namespace smf
