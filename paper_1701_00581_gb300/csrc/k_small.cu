// Per-subfield statistics (Eq. 1 numerator and the noise floor), the
// Labeyrie modulus (Eq. 1) and the mosaic merge (Sect. 3.2).
#include "sm_internal.h"

namespace {

using smi::PlanDev;

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

constexpr int STAT_THREADS = 1024;

// P = <|I_i|^2>, M = <I_i> over the F frames on the half box ky = 0..K;
// noise = mean of P over {ky >= 1, |k|^2 > r^2} (the half-box corners).
// HBM bound: one 1024-thread CTA per subfield streams its F spectra once,
// each thread summing two neighbouring values over the frames in order
// (16-byte loads, four frames in flight).
template <int PREC>
__global__ void __launch_bounds__(STAT_THREADS)
k_stats(PlanDev p, const void* __restrict__ spec, int F, float* __restrict__ P,
        float2* __restrict__ M, float* __restrict__ noise) {
    __shared__ double red_s[STAT_THREADS / 32];
    __shared__ int red_n[STAT_THREADS / 32];
    const int sl = blockIdx.x, tid = threadIdx.x;
    const size_t box = (size_t)p.box_rows * p.box_pitch;
    const size_t hb = (size_t)p.hb_rows * p.box_pitch;
    const size_t sbase = (size_t)sl * F * box;
    const int ne = p.hb_rows * p.box_cols;
    const float invF = 1.0f / (float)F;
    double cs = 0.0;
    int cn = 0;
    if constexpr (PREC == SM_FP32) {
        // two neighbouring spectrum values per thread, 16-byte loads (the
        // pitch is a multiple of 4 and the last value of a row pairs with
        // the row's padding, which is read but not stored)
        const int hp = p.box_pitch / 2, ne2 = p.hb_rows * hp;
        const float4* s4 = reinterpret_cast<const float4*>(spec);
        for (int e = tid; e < ne2; e += STAT_THREADS) {
            const int ky = e / hp, c2 = e - ky * hp, col = 2 * c2;
            const size_t off = ((size_t)(ky + p.R) * p.box_pitch + col) / 2;
            float ps0 = 0.f, ps1 = 0.f;
            float2 m0 = make_float2(0.f, 0.f), m1 = make_float2(0.f, 0.f);
#pragma unroll 4
            for (int f = 0; f < F; ++f) {
                const float4 v = __ldg(s4 + (sbase + (size_t)f * box) / 2 + off);
                ps0 = fmaf(v.x, v.x, fmaf(v.y, v.y, ps0));
                ps1 = fmaf(v.z, v.z, fmaf(v.w, v.w, ps1));
                m0.x += v.x; m0.y += v.y;
                m1.x += v.z; m1.y += v.w;
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int cc = col + h, kx = cc - p.K;
                if (cc >= p.box_cols) break;
                const float pm = (h ? ps1 : ps0) * invF;
                const float2 ms = h ? m1 : m0;
                const size_t o = (size_t)sl * hb + (size_t)ky * p.box_pitch + cc;
                P[o] = pm;
                M[o] = make_float2(ms.x * invF, ms.y * invF);
                if (ky >= 1 && kx * kx + ky * ky > p.r2i) {
                    cs += pm;
                    ++cn;
                }
            }
        }
    } else {
        for (int e = tid; e < ne; e += STAT_THREADS) {
            const int ky = e / p.box_cols, col = e - ky * p.box_cols, kx = col - p.K;
            const size_t off = (size_t)(ky + p.R) * p.box_pitch + col;
            float ps = 0.f;
            float2 ms = make_float2(0.f, 0.f);
#pragma unroll 4
            for (int f = 0; f < F; ++f) {
                const float2 v = load_spec<PREC>(spec, sbase + (size_t)f * box + off);
                ps = fmaf(v.x, v.x, fmaf(v.y, v.y, ps));
                ms.x += v.x;
                ms.y += v.y;
            }
            const float pm = ps * invF;
            const size_t o = (size_t)sl * hb + (size_t)ky * p.box_pitch + col;
            P[o] = pm;
            M[o] = make_float2(ms.x * invF, ms.y * invF);
            if (ky >= 1 && kx * kx + ky * ky > p.r2i) {
                cs += pm;
                ++cn;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        cs += __shfl_xor_sync(0xffffffffu, cs, o);
        cn += __shfl_xor_sync(0xffffffffu, cn, o);
    }
    if ((tid & 31) == 0) {
        red_s[tid >> 5] = cs;
        red_n[tid >> 5] = cn;
    }
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        int n = 0;
        for (int i = 0; i < STAT_THREADS / 32; ++i) {
            s += red_s[i];
            n += red_n[i];
        }
        noise[sl] = n > 0 ? (float)(s / n) : 0.f;
    }
}

// A = sqrt(max(P - noise, 0) / max(STF, 1e-4)) * T0 on U, A(0) = 1, 0 outside.
__global__ void k_amplitude(PlanDev p, const double* __restrict__ stf, const float* __restrict__ P,
                            const float* __restrict__ noise, float* __restrict__ A) {
    const int sl = blockIdx.y;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int ne = p.hb_rows * p.box_cols;
    if (e >= ne) return;
    const int ky = e / p.box_cols, col = e - ky * p.box_cols, kx = col - p.K;
    const size_t hb = (size_t)p.hb_rows * p.box_pitch;
    const size_t o = (size_t)ky * p.box_pitch + col;
    const double t0 = p.t0[o];
    float a = 0.f;
    if (kx == 0 && ky == 0) {
        a = 1.f;
    } else if (t0 > 0.0) {
        const double s = stf[(size_t)(ky + p.N / 2) * p.N + kx + p.N / 2];
        const double num = fmax((double)P[(size_t)sl * hb + o] - (double)noise[sl], 0.0);
        a = (float)(sqrt(num / fmax(s, 1e-4)) * t0);
    }
    A[(size_t)sl * hb + o] = a;
}

// out(x) = sum_s rec_s(x - o_s) / sum_s window_s(x - o_s); a gather over the
// (at most ceil(N/stride)^2) subfields covering the pixel, no atomics.
__global__ void k_mosaic(PlanDev p, const float* __restrict__ rec, float* __restrict__ out,
                         uint8_t* __restrict__ valid) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= p.W || y >= p.H) return;
    if (p.mosaic_mode == SM_MOSAIC_CENTRAL) {
        // the one subfield whose central stride x stride block holds (x, y)
        const int h0 = (p.N - p.stride) / 2;
        const int i = x >= h0 ? (x - h0) / p.stride : -1, j = y >= h0 ? (y - h0) / p.stride : -1;
        const bool ok = i >= 0 && i < p.nsx && j >= 0 && j < p.nsy;
        float v = 0.f;
        if (ok) {
            const int s = j * p.nsx + i;
            const int4 sb = p.subs[s];
            const int lx = x - sb.x, ly = y - sb.y;       // in [h0, h0 + stride)
            v = rec[((size_t)s * p.N + ly) * p.N + lx] /
                (p.winx[(size_t)s * p.N + lx] * p.winy[(size_t)s * p.N + ly]);
        }
        out[(size_t)y * p.W + x] = v;
        if (valid) valid[(size_t)y * p.W + x] = ok ? 1 : 0;
        return;
    }
    const int ilo = x - p.N + 1 > 0 ? (x - p.N + p.stride) / p.stride : 0;
    const int ihi = min(p.nsx - 1, x / p.stride);
    const int jlo = y - p.N + 1 > 0 ? (y - p.N + p.stride) / p.stride : 0;
    const int jhi = min(p.nsy - 1, y / p.stride);
    float num = 0.f, den = 0.f;
    for (int j = jlo; j <= jhi; ++j) {
        for (int i = ilo; i <= ihi; ++i) {
            const int s = j * p.nsx + i;
            const int4 sb = p.subs[s];
            const int lx = x - sb.x, ly = y - sb.y;
            if (lx < 0 || ly < 0 || lx >= sb.z || ly >= sb.w) continue;
            num += rec[((size_t)s * p.N + ly) * p.N + lx];
            den += p.winx[(size_t)s * p.N + lx] * p.winy[(size_t)s * p.N + ly];
        }
    }
    const bool ok = den >= 0.25f;
    out[(size_t)y * p.W + x] = ok ? num / den : 0.f;
    if (valid) valid[(size_t)y * p.W + x] = ok ? 1 : 0;
}

// Photon-noise bias of the mean bispectrum (Wirnitzer 1985), removed in
// place at every used pair of every tile: B -= (P(u) + P(v) + P(w)) <1/N>
// - 2 <1/N^2> (real), u = w - v, P(-k) = P(k) from the half box, N_f the
// photon count of frame f's windowed tile.  One CTA per (tile, subfield),
// laid out as the bispectrum kernel's tiles.
__global__ void __launch_bounds__(smi::BISPEC_THREADS)
k_unbias(PlanDev p, int F, const float* __restrict__ flux, const float* __restrict__ P, float2* __restrict__ B) {
    __shared__ float a12[2];
    const int tile = blockIdx.x, sl = blockIdx.y;
    const int4 T = p.tiles[tile];
    const int q = threadIdx.x >> 5, lane = threadIdx.x & 31, wyl = lane >> 2, gx = lane & 3;
    const float* Ps = P + (size_t)sl * p.hb_rows * p.box_pitch;
    if (threadIdx.x == 0) {             // <1/N_f>, <1/N_f^2>, N_f = photon_gain * flux_f
        double a1 = 0.0, a2 = 0.0;
        for (int f = 0; f < F; ++f) {
            const double nf = p.photon_gain * (double)flux[(size_t)sl * F + f];
            if (nf > 0.0) {
                a1 += 1.0 / nf;
                a2 += 1.0 / (nf * nf);
            }
        }
        a12[0] = (float)(a1 / F);
        a12[1] = (float)(a2 / F);
    }
    __syncthreads();
    const float a1 = a12[0], a2 = a12[1];
    float2* Bt = B + (size_t)(sl * p.n_tiles + tile) * smi::TILE_PAIRS;
    auto pget = [&](int kx, int ky) -> float {
        return ky >= 0 ? Ps[ky * p.box_pitch + kx + p.K] : Ps[(-ky) * p.box_pitch - kx + p.K];
    };
    const int wy = T.y + wyl, vy = T.w + q;
    for (int j = 0; j < 4; ++j) {
        const int wx = T.x + 4 * gx + j;
        for (int kk = 0; kk < smi::VBX; ++kk) {
            const int vx = T.z + kk;
            const int w2 = wx * wx + wy * wy, v2 = vx * vx + vy * vy;
            const int ux = wx - vx, uy = wy - vy, u2 = ux * ux + uy * uy;
            const bool inH = wy > 0 || (wy == 0 && wx > 0);
            if (!(inH && w2 >= 2 && w2 <= p.r2i && v2 > 0 && v2 <= p.R * p.R && v2 < w2 && u2 < w2)) continue;
            float2& b = Bt[((wyl * smi::WBX + 4 * gx + j) * smi::TILE_V) + q * smi::VBX + kk];
            b.x -= (pget(ux, uy) + pget(vx, vy) + pget(wx, wy)) * a1 - 2.f * a2;
        }
    }
}

}  // namespace

namespace smk {

cudaError_t launch_stats(const smi::PlanDev& p, const void* spec, int F, int nsub, float* P,
                         float2* M, float* noise, cudaStream_t st) {
    if (p.prec == SM_FP32) k_stats<SM_FP32><<<nsub, STAT_THREADS, 0, st>>>(p, spec, F, P, M, noise);
    else if (p.prec == SM_FP16) k_stats<SM_FP16><<<nsub, STAT_THREADS, 0, st>>>(p, spec, F, P, M, noise);
    else k_stats<SM_BF16><<<nsub, STAT_THREADS, 0, st>>>(p, spec, F, P, M, noise);
    return cudaGetLastError();
}

cudaError_t launch_amplitude(const smi::PlanDev& p, int nsub, const double* stf, const float* P,
                             const float* noise, float* A, cudaStream_t st) {
    const int ne = p.hb_rows * p.box_cols;
    dim3 grid((ne + 255) / 256, nsub);
    k_amplitude<<<grid, 256, 0, st>>>(p, stf, P, noise, A);
    return cudaGetLastError();
}

cudaError_t launch_unbias(const smi::PlanDev& p, int F, int nsub, const float* flux, const float* P, float2* B,
                          cudaStream_t st) {
    k_unbias<<<dim3(p.n_tiles, nsub), smi::BISPEC_THREADS, 0, st>>>(p, F, flux, P, B);
    return cudaGetLastError();
}

cudaError_t launch_mosaic(const smi::PlanDev& p, const float* rec, float* out, uint8_t* valid,
                          cudaStream_t st) {
    dim3 grid((p.W + 255) / 256, p.H);
    k_mosaic<<<grid, 256, 0, st>>>(p, rec, out, valid);
    return cudaGetLastError();
}

}  // namespace smk
