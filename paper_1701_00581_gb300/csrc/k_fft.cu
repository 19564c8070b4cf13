// Subfield spectra (Sect. 2: Fourier transform of every subimage) and the
// inverse transform of modulus and phase (Sect. 2, Sect. 3.2).
//
// One CTA per (frame, subfield): the tile is cut from the frame, apodised by
// the separable window, its windowed mean is removed, and the 2-D DFT is
// taken as real row FFTs (two rows packed per complex FFT) followed by
// column FFTs of only the K+1 non-negative columns inside the cutoff box.
// The forward transforms are four-step FFTs (N = P x Q) computed in
// registers by groups of 16 threads with one shared-memory exchange; the
// inverse (one CTA per subfield, off the critical path) uses warp-wide
// radix-2 Stockham FFTs in shared memory.
#include "sm_fft_dev.cuh"

namespace {

using smi::PlanDev;
using smf::cmul;
using smf::four_step;
using smf::load_sample;
using smf::Split;
using smf::store_spec;

// Radix-2 Stockham FFT of length N by one warp.  a holds the input, b is
// scratch; returns the buffer holding the output in natural order.
// INV = true uses exp(+2 pi i k / N) (unnormalised inverse).
template <int N, bool INV>
__device__ __forceinline__ float2* warp_fft(float2* a, float2* b, const float2* tw, int lane) {
#pragma unroll
    for (int Ns = 1; Ns < N; Ns <<= 1) {
#pragma unroll
        for (int j = lane; j < N / 2; j += 32) {
            const int k = j & (Ns - 1);
            float2 w = tw[k * (N / (2 * Ns))];
            if (INV) w.y = -w.y;
            const float2 a0 = a[j];
            const float2 t = cmul(a[j + N / 2], w);
            const int o = 2 * j - k;
            b[o] = make_float2(a0.x + t.x, a0.y + t.y);
            b[o + Ns] = make_float2(a0.x - t.x, a0.y - t.y);
        }
        __syncwarp();
        float2* t = a;
        a = b;
        b = t;
    }
    return a;
}

constexpr int FFT_THREADS = 256;
constexpr int FFT_WARPS = FFT_THREADS / 32;
// Forward transforms: 32 groups of 16 threads for N >= 128 (one CTA per SM
// fits in shared memory, so latency is hidden by warps within the CTA).
template <int N> struct SpecThreads { static constexpr int T = N >= 128 ? 512 : 256; };

// Thread groups of the four-step transform: G threads per transform.
template <int N> struct Grp {
    static constexpr int P = Split<N>::P, Q = Split<N>::Q;
    static constexpr int G = P > Q ? P : Q;
    static constexpr int NG = SpecThreads<N>::T / G;                 // groups per CTA
    static constexpr int TB = (Q * (P + 1) > N ? Q * (P + 1) : N);   // exchange buffer
};

// scratch area (float2): per-warp ping-pong of the inverse, per-group
// exchange tiles of the forward transform
template <int N>
__host__ __device__ constexpr int scratch_elems() {
    return FFT_WARPS * 2 * N > Grp<N>::NG * Grp<N>::TB ? FFT_WARPS * 2 * N : Grp<N>::NG * Grp<N>::TB;
}
__host__ __device__ constexpr int scratch_elems_rt(int N) {
    return N == 64 ? scratch_elems<64>() : (N == 128 ? scratch_elems<128>() : scratch_elems<256>());
}

__host__ __device__ constexpr size_t fft_smem(int N, int K) {
    return (size_t)(K + 1) * (N + 1) * sizeof(float2)        // column buffer
           + (size_t)scratch_elems_rt(N) * sizeof(float2)    // scratch
           + (size_t)N * sizeof(float2)                      // twiddles
           + (size_t)(K + 1) * sizeof(float2)                // window transform
           + (size_t)2 * N * sizeof(float)                   // windows
           + (size_t)(FFT_WARPS * 2 + 2) * sizeof(double);   // reductions and scalars
}

// Spectra of one (frame, subfield): the tile times the window is transformed
// row by row (two real rows per complex transform), the windowed mean mu is
// read off the row transforms' DC terms, mu * window is removed through the
// window's own transform, and the K+1 non-negative columns are transformed.
template <int N, typename TIn, int PREC>
__global__ void __launch_bounds__(SpecThreads<N>::T, 1)
k_spectra(PlanDev p, const TIn* __restrict__ frames, int F, int sub0, void* __restrict__ spec,
          float* __restrict__ flux, float* __restrict__ mu) {
    using GP = Grp<N>;
    constexpr int P = GP::P, Q = GP::Q, G = GP::G, NG = GP::NG, TB = GP::TB;
    constexpr int TS = SpecThreads<N>::T, WS = TS / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    const int K1 = p.K + 1, CP = N + 1;
    float2* C = reinterpret_cast<float2*>(smem);
    float2* scratch = C + (size_t)K1 * CP;
    float2* stw = scratch + scratch_elems<N>();
    float2* swf = stw + N;
    float* swx = reinterpret_cast<float*>(swf + K1);
    float* swy = swx + N;
    double* red = reinterpret_cast<double*>(swy + N);

    // frame-major grid: consecutive CTAs cut neighbouring subfields of one
    // frame, whose tiles overlap, so most tile reads hit L2
    const int sl = blockIdx.x, f = blockIdx.y, s = sub0 + sl;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int grp = tid / G, g = tid - grp * G;
    float2* T = scratch + grp * TB;
    const int4 sb = p.subs[s];
    const int x0 = sb.x, y0 = sb.y, w = sb.z, h = sb.w;
    {
        // the whole tile towards L2 now, so the row rounds after the first
        // do not wait on DRAM: one prefetch per 128-byte line of each row
        const char* fb = reinterpret_cast<const char*>(frames + (size_t)f * p.H * p.W + (size_t)y0 * p.W);
        const size_t b0 = (size_t)x0 * sizeof(TIn), b1 = (size_t)(x0 + w) * sizeof(TIn);
        const int l0 = (int)(b0 >> 7), nl = (int)(((b1 - 1) >> 7) - (b0 >> 7)) + 1;
        for (int e = tid; e < h * nl; e += TS) {
            const int y = e / nl, l = e - y * nl;
            const size_t off = (size_t)y * p.W * sizeof(TIn) + ((size_t)(l0 + l) << 7);
            const size_t lo = (size_t)y * p.W * sizeof(TIn) + b0;   // stay inside the tile's row
            asm volatile("prefetch.global.L2 [%0];" :: "l"(fb + (off > lo ? off : lo)));
        }
    }
    for (int i = tid; i < N; i += TS) {
        stw[i] = p.tw[i];
        swx[i] = p.winx[(size_t)s * N + i];
        swy[i] = p.winy[(size_t)s * N + i];
    }
    for (int i = tid; i < K1; i += TS) swf[i] = p.winft[(size_t)s * K1 + i];
    __syncthreads();

    const TIn* fr = frames + (size_t)f * p.H * p.W + (size_t)y0 * p.W + x0;
    // row transforms: group grp of round r handles rows 2(r NG + grp), +1
    float raw[2][Q];
    auto fetch = [&](int pr) {
        const int y1 = 2 * pr, y2 = y1 + 1;
#pragma unroll
        for (int n2 = 0; n2 < Q; ++n2) {
            const int x = g + P * n2;
            const bool inx = g < P && x < w;
            raw[0][n2] = inx && y1 < h ? load_sample(fr + (size_t)y1 * p.W + x) : 0.f;
            raw[1][n2] = inx && y2 < h ? load_sample(fr + (size_t)y2 * p.W + x) : 0.f;
        }
    };
    for (int pr0 = 0; pr0 < N / 2; pr0 += NG) {
        fetch(pr0 + grp);
        const int pr = pr0 + grp, y1 = 2 * pr, y2 = y1 + 1;
        float2 v[Q], X[P];
#pragma unroll
        for (int n2 = 0; n2 < Q; ++n2) {
            const float wx = swx[(g + P * n2) & (N - 1)];
            v[n2] = make_float2(wx * swy[y1] * raw[0][n2], wx * swy[y2] * raw[1][n2]);
        }
        four_step<N, false>(v, X, T, stw, g);
        if (g < Q) {
#pragma unroll
            for (int k1 = 0; k1 < P; ++k1) T[g + Q * k1] = X[k1];
        }
        __syncwarp();
        for (int kx = g; kx < K1; kx += G) {
            const float2 za = T[kx], zb = T[(N - kx) & (N - 1)];
            C[kx * CP + y1] = make_float2(0.5f * (za.x + zb.x), 0.5f * (za.y - zb.y));
            C[kx * CP + y2] = make_float2(0.5f * (za.y + zb.y), -0.5f * (za.x - zb.x));
        }
        __syncwarp();
    }
    __syncthreads();

    // windowed mean from the DC terms of the row transforms: the warps
    // holding DC terms reduce them, thread 0 forms the scalars once
    if (tid < N) {
        double dacc = 0.0;
        for (int y = tid; y < N; y += TS) dacc += (double)C[y].x;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dacc += __shfl_xor_sync(0xffffffffu, dacc, o);
        if (lane == 0) red[warp] = dacc;
    }
    __syncthreads();
    if (tid == 0) {
        double tot = 0.0;
        for (int i = 0; i < (N < TS ? N : TS) / 32; ++i) tot += red[i];
        const double wsum = p.winsum[s];
        const float m = (float)(tot / wsum);
        const double fl = (double)m * wsum;
        red[WS] = fl;                                  // flux, then its reciprocal and the mean
        reinterpret_cast<float*>(red + WS + 1)[0] = (float)(1.0 / fl);
        reinterpret_cast<float*>(red + WS + 1)[1] = m;
    }
    __syncthreads();
    const float mean = reinterpret_cast<const float*>(red + WS + 1)[1];
    // remove mean * window: row transform of w_x(x) w_y(y) mu is mu w_y(y) Wx(kx)
    // (a warp per column, lanes along it: no index division per element)
    for (int kx = warp; kx < K1; kx += WS) {
        const float2 wf = swf[kx];
        for (int y = lane; y < h; y += 32) {
            const float a = mean * swy[y];
            float2& c = C[kx * CP + y];
            c.x -= a * wf.x;
            c.y -= a * wf.y;
        }
    }
    __syncthreads();

    // column transforms of kx = 0..K (groups past K transform column K and drop it)
    for (int c0 = 0; c0 < K1; c0 += NG) {
        const int kx = c0 + grp;
        const int kc = kx < K1 ? kx : K1 - 1;
        float2 v[Q], X[P];
#pragma unroll
        for (int n2 = 0; n2 < Q; ++n2) v[n2] = g < P ? C[kc * CP + g + P * n2] : make_float2(0.f, 0.f);
        four_step<N, false>(v, X, T, stw, g);
        if (kx < K1 && g < Q) {
#pragma unroll
            for (int k1 = 0; k1 < P; ++k1) C[kx * CP + g + Q * k1] = X[k1];
        }
        __syncwarp();
    }
    __syncthreads();

    // normalise by the windowed flux and store the box ky = -R..K (a warp
    // per box row, coalesced along it)
    const double fl = red[WS];
    const float inv = reinterpret_cast<const float*>(red + WS + 1)[0];
    const size_t base = ((size_t)sl * F + f) * p.box_rows * p.box_pitch;
    for (int row = warp; row < p.box_rows; row += WS)
    for (int col = lane; col < p.box_cols; col += 32) {
        const int ky = row - p.R, kx = col - p.K;
        float2 v;
        if (kx >= 0) {
            v = C[kx * CP + (ky & (N - 1))];
        } else {
            v = C[(-kx) * CP + ((-ky) & (N - 1))];
            v.y = -v.y;
        }
        v.x *= inv;
        v.y *= inv;
        if (kx == 0 && ky == 0) v = make_float2(1.f, 0.f);
        store_spec<PREC>(spec, base + (size_t)row * p.box_pitch + col, v);
    }
    if (tid == 0) {
        flux[(size_t)sl * F + f] = (float)fl;
        mu[(size_t)sl * F + f] = mean;
    }
}

// Inverse: O = A z on the disk (Hermitian), DC removed; columns first, then
// pairs of Hermitian rows packed into one complex inverse FFT.
template <int N>
__global__ void __launch_bounds__(FFT_THREADS, 1)
k_inverse(PlanDev p, int F, int sub0, const float* __restrict__ A, const double2* __restrict__ z,
          const float* __restrict__ flux, const float* __restrict__ mu, float* __restrict__ rec) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int K = p.K, K1 = K + 1, CP = N + 1;
    float2* C = reinterpret_cast<float2*>(smem);
    float2* scratch = C + (size_t)K1 * CP;
    float2* stw = scratch + scratch_elems<N>();
    float* swx = reinterpret_cast<float*>(stw + N + K1);
    float* swy = swx + N;
    double* red = reinterpret_cast<double*>(swy + N);

    const int sl = blockIdx.x, s = sub0 + sl;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < N; i += FFT_THREADS) {
        stw[i] = p.tw[i];
        swx[i] = p.winx[(size_t)s * N + i];
        swy[i] = p.winy[(size_t)s * N + i];
    }
    if (tid == 0) {
        double fs = 0.0, ms = 0.0;
        for (int f = 0; f < F; ++f) {
            fs += flux[(size_t)sl * F + f];
            ms += mu[(size_t)sl * F + f];
        }
        red[0] = fs / F;
        red[1] = ms / F;
    }
    const size_t hb = (size_t)p.hb_rows * p.box_pitch;
    const float* As = A + (size_t)sl * hb;
    const double2* zs = z + (size_t)sl * hb;
    for (int e = tid; e < K1 * N; e += FFT_THREADS) {
        const int kx = e / N, j = e - kx * N;
        const int ky = j < N / 2 ? j : j - N;
        float2 v = make_float2(0.f, 0.f);
        if (kx * kx + ky * ky <= p.r2i && (kx | ky) != 0 && ky >= -K && ky <= K) {
            if (ky > 0 || (ky == 0 && kx > 0)) {
                const size_t o = (size_t)ky * p.box_pitch + kx + K;
                const double2 zz = zs[o];
                v = make_float2((float)(As[o] * zz.x), (float)(As[o] * zz.y));
            } else {
                const size_t o = (size_t)(-ky) * p.box_pitch + (-kx) + K;
                const double2 zz = zs[o];
                v = make_float2((float)(As[o] * zz.x), (float)(-As[o] * zz.y));
            }
        }
        C[kx * CP + j] = v;
    }
    __syncthreads();
    const double fmean = red[0];
    const float mmean = (float)red[1];
    const float scale = (float)(fmean / ((double)N * N));

    float2* fa = scratch + warp * 2 * N;
    float2* fb = fa + N;
    for (int kx = warp; kx < K1; kx += FFT_WARPS) {
        float2* col = C + (size_t)kx * CP;
        for (int y = lane; y < N; y += 32) fa[y] = col[y];
        __syncwarp();
        const float2* Zc = warp_fft<N, true>(fa, fb, stw, lane);
        for (int y = lane; y < N; y += 32) col[y] = Zc[y];
        __syncwarp();
    }
    __syncthreads();

    float* out = rec + (size_t)s * N * N;
    for (int pr = warp; pr < N / 2; pr += FFT_WARPS) {
        const int y1 = 2 * pr, y2 = y1 + 1;
        for (int kx = lane; kx < N; kx += 32) fa[kx] = make_float2(0.f, 0.f);
        __syncwarp();
        for (int kx = lane; kx < K1; kx += 32) {
            const float2 a = C[kx * CP + y1], b = C[kx * CP + y2];
            fa[kx] = make_float2(a.x - b.y, a.y + b.x);
            if (kx > 0) fa[N - kx] = make_float2(a.x + b.y, -a.y + b.x);
        }
        __syncwarp();
        const float2* Zr = warp_fft<N, true>(fa, fb, stw, lane);
        for (int x = lane; x < N; x += 32) {
            const float2 v = Zr[x];
            out[(size_t)y1 * N + x] = v.x * scale + mmean * swx[x] * swy[y1];
            out[(size_t)y2 * N + x] = v.y * scale + mmean * swx[x] * swy[y2];
        }
        __syncwarp();
    }
}

template <int N>
cudaError_t spectra_n(const PlanDev& p, const void* frames, int frame_type, int F, int sub0,
                      int nsub, void* spec, float* flux, float* mu, cudaStream_t st) {
    const size_t sm = fft_smem(N, p.K);
    dim3 grid(nsub, F);
    cudaError_t e = cudaSuccess;
#define SM_LAUNCH(TIN, PREC)                                                                    \
    do {                                                                                        \
        e = cudaFuncSetAttribute(k_spectra<N, TIN, PREC>,                                       \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);         \
        if (e != cudaSuccess) return e;                                                         \
        k_spectra<N, TIN, PREC><<<grid, SpecThreads<N>::T, sm, st>>>(                                 \
            p, reinterpret_cast<const TIN*>(frames), F, sub0, spec, flux, mu);                  \
    } while (0)
    if (frame_type == SM_U16) {
        if (p.prec == SM_FP32) SM_LAUNCH(uint16_t, SM_FP32);
        else if (p.prec == SM_FP16) SM_LAUNCH(uint16_t, SM_FP16);
        else SM_LAUNCH(uint16_t, SM_BF16);
    } else {
        if (p.prec == SM_FP32) SM_LAUNCH(float, SM_FP32);
        else if (p.prec == SM_FP16) SM_LAUNCH(float, SM_FP16);
        else SM_LAUNCH(float, SM_BF16);
    }
#undef SM_LAUNCH
    return cudaGetLastError();
}

template <int N>
cudaError_t inverse_n(const PlanDev& p, int F, int sub0, int nsub, const float* A, const double2* z,
                      const float* flux, const float* mu, float* rec, cudaStream_t st) {
    const size_t sm = fft_smem(N, p.K);
    cudaError_t e = cudaFuncSetAttribute(k_inverse<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
    k_inverse<N><<<nsub, FFT_THREADS, sm, st>>>(p, F, sub0, A, z, flux, mu, rec);
    return cudaGetLastError();
}

}  // namespace

namespace smk {

size_t spectra_smem_bytes(int N, int K) { return fft_smem(N, K); }

cudaError_t launch_spectra(const smi::PlanDev& p, const void* frames, int frame_type, int F,
                           int sub0, int nsub, void* spec, float* flux, float* mu,
                           cudaStream_t st) {
    switch (p.N) {
        case 64: return spectra_n<64>(p, frames, frame_type, F, sub0, nsub, spec, flux, mu, st);
        case 128: return spectra_n<128>(p, frames, frame_type, F, sub0, nsub, spec, flux, mu, st);
        case 256: return spectra_n<256>(p, frames, frame_type, F, sub0, nsub, spec, flux, mu, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_inverse(const smi::PlanDev& p, int F, int sub0, int nsub, const float* A,
                           const double2* z, const float* flux, const float* mu, float* rec,
                           cudaStream_t st) {
    switch (p.N) {
        case 64: return inverse_n<64>(p, F, sub0, nsub, A, z, flux, mu, rec, st);
        case 128: return inverse_n<128>(p, F, sub0, nsub, A, z, flux, mu, rec, st);
        case 256: return inverse_n<256>(p, F, sub0, nsub, A, z, flux, mu, rec, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace smk
