// Bispectrum tile body (Sect. 2 and Sect. 3.2: speckle masking, Weigelt 1977),
// shared by the per-stage kernel (k_bispec.cu) and the batched persistent
// launch (k_batch.cu).
#pragma once
#include <type_traits>

#include "sm_internal.h"

namespace smb {

using smi::PlanDev;
using smi::TILE_PAIRS;
using smi::TILE_V;
using smi::TILE_W;

constexpr int PW = 18;                  // row pitch of W in smem (float2)
constexpr int PU = 26;                  // row pitch of U in smem (float2)
constexpr int UR = smi::WBY + smi::VBY - 1;     // 11 rows of U
constexpr int UC = smi::WBX + smi::VBX - 1;     // 23 cols of U
constexpr int OFF_W = 0;
constexpr int OFF_V = smi::WBY * PW;                      // 144
constexpr int OFF_U = OFF_V + smi::VBY * smi::VBX;        // 176
constexpr int BUF = OFF_U + UR * PU;                      // 462 float2 per frame buffer
constexpr int NLOAD = smi::WBY * smi::WBX + smi::VBY * smi::VBX + UR * UC;  // 413 values staged per frame
constexpr int THREADS = smi::BISPEC_THREADS;
static_assert(OFF_V % 2 == 0 && OFF_U % 2 == 0 && BUF % 2 == 0 && PW % 2 == 0 && PU % 2 == 0,
              "16-byte shared accesses need even float2 offsets");

// 16-byte staging of FP32 spectra: W as 8 rows x 8 chunks, U as 11 rows x 12
// chunks (24 columns; the 24th is read by no used pair) and, with VCH, V as
// 4 rows x 4 chunks; chunk c of W|V|U (VCH) or W|U goes to copy slot c / 128
// of thread c % 128.  Without VCH, slot 1 of warp 0 copies V value `lane`
// (8 bytes) and W|U chunks 128.. go to threads 32.., so the copy width is
// uniform across each warp.
constexpr int UCH = (UC + 1) / 2;                         // 12 chunks per U row
constexpr int NCH_W = smi::WBY * smi::WBX / 2;            // 64
constexpr int NCH_V = smi::VBY * smi::VBX / 2;            // 16
constexpr int NCH_U = UR * UCH;                           // 132
constexpr int NV = smi::VBY * smi::VBX;                   // 32
static_assert(NCH_W + NCH_V + NCH_U <= 2 * THREADS && NCH_W + NCH_U <= 2 * THREADS - NV && NV == 32,
              "two copy slots per thread");
static_assert(smi::WBX % 2 == 0, "targets start at even box columns");

// Bank check (16-byte loads, 8-lane phases): lanes 0..7 hold wyl = 0, 1 and
// gx = 0..3.  Targets: 16-byte slot 9 wyl + 2 gx (+ j/2) -> {0,2,4,6} + {0,1}
// mod 8, distinct.  Differences: slot 13 row + 2 gx + q, rows of lanes 0..7
// differ by 1 -> {0,2,4,6} + {0,5} mod 8, distinct.  Offsets: broadcast.

// Asynchronous copies global -> shared of 8 or 16 bytes; the first `bytes`
// bytes come from global memory, the rest of the copy is zero-filled.
__device__ __forceinline__ void cp_async8(unsigned smem_addr, const void* gmem, int bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" :: "r"(smem_addr), "l"(gmem), "r"(bytes));
}
__device__ __forceinline__ void cp_async16(unsigned smem_addr, const void* gmem, int bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" :: "r"(smem_addr), "l"(gmem), "r"(bytes));
}
__device__ __forceinline__ void cp_async4(unsigned smem_addr, const void* gmem, int bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" :: "r"(smem_addr), "l"(gmem), "r"(bytes));
}
// Chunk copies of E-byte spectrum values: two values (2E bytes) or one (E).
template <int E> __device__ __forceinline__ void cp_pair(unsigned s, const void* g, int bytes) {
    if (E == 8) cp_async16(s, g, bytes); else cp_async8(s, g, bytes);
}
template <int E> __device__ __forceinline__ void cp_one(unsigned s, const void* g, int bytes) {
    if (E == 8) cp_async8(s, g, bytes); else cp_async4(s, g, bytes);
}

// acc += t with Kahan compensation (c carries the rounding error of the sum);
// explicit round-to-nearest intrinsics keep the compiler from fusing or
// reassociating the correction away.
__device__ __forceinline__ void kahan_add(float& acc, float& c, float t) {
    const float y = __fsub_rn(t, c);
    const float s = __fadd_rn(acc, y);
    c = __fsub_rn(__fsub_rn(s, acc), y);
    acc = s;
}

// One frame of the thread's 4 targets x NC offset columns col0 .. col0+NC-1
// from the staged rectangles, added into acc; kkmask holds those columns'
// bits (bit k = column col0 + k).  FULL: the warp owns a used pair in every
// one of them, so no column is tested.
template <bool FULL, int NC>
__device__ __forceinline__ void accumulate_frame(const float2* __restrict__ Sb, int wyl, int gx, int warp,
                                                 unsigned kkmask, int col0, float2 (&acc)[4][NC]) {
    const float4* w4 = reinterpret_cast<const float4*>(Sb + OFF_W + wyl * PW + 4 * gx);
    const float4 w01 = w4[0], w23 = w4[1];
    const float2 a[4] = {make_float2(w01.x, -w01.y), make_float2(w01.z, -w01.w),   // conj I(w)
                         make_float2(w23.x, -w23.y), make_float2(w23.z, -w23.w)};
    const float4* u4 = reinterpret_cast<const float4*>(Sb + OFF_U + (wyl - warp + smi::VBY - 1) * PU + 4 * gx);
    float2 c[12];                                    // I(w - v), m = j - kk + 7
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const float4 t = u4[q];
        c[2 * q] = make_float2(t.x, t.y);
        c[2 * q + 1] = make_float2(t.z, t.w);
    }
    const float4* v4 = reinterpret_cast<const float4*>(Sb + OFF_V + warp * smi::VBX + col0);
#pragma unroll
    for (int k2 = 0; k2 < NC / 2; ++k2) {
        if (!FULL && !(kkmask & (3u << (2 * k2)))) continue;   // warp-uniform
        const float4 bb = v4[k2];                               // I(v) for two columns (broadcast)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int kl = 2 * k2 + e, kk = col0 + kl;
            if (!FULL && !(kkmask & (1u << kl))) continue;      // warp-uniform
            const float2 b = e == 0 ? make_float2(bb.x, bb.y) : make_float2(bb.z, bb.w);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float2 u = c[j - kk + 7];
                const float px = fmaf(u.x, b.x, -u.y * b.y);
                const float py = fmaf(u.x, b.y, u.y * b.x);
                acc[j][kl].x = fmaf(px, a[j].x, fmaf(-py, a[j].y, acc[j][kl].x));
                acc[j][kl].y = fmaf(px, a[j].y, fmaf(py, a[j].x, acc[j][kl].y));
            }
        }
    }
}

// Staging: spectra go from global to shared memory by cp.async (zero-filled
// outside the box), FB frames per stage in a two-stage ring, so one barrier
// serves FB frames.  FP32 values (E = 8 bytes) are multiplied out from the
// ring itself.  Half-precision values (E = 4: half2 or bfloat162) are
// copied raw, at half the bytes, and converted to FP32 once per stage into
// one of two compute buffers, a stage ahead of the products, so the inner
// loop and the barrier count are those of FP32.  Shared memory per CTA:
// 2 FB BUF float2 (FP32 ring), or a 2 FB BUF raw ring and 2 FB BUF float2
// of compute buffers (half precision).
template <int PREC> struct Staging;
template <> struct Staging<SM_FP32> { static constexpr int FB = 4, E = 8; };
template <> struct Staging<SM_FP16> { static constexpr int FB = 4, E = 4; };
template <> struct Staging<SM_BF16> { static constexpr int FB = 4, E = 4; };

template <int PREC>
__device__ __forceinline__ float2 raw_to_float2(unsigned w) {
    if (PREC == SM_FP16) {
        const float2 v = __half22float2(*reinterpret_cast<const __half2*>(&w));
        return make_float2(v.x * smi::FP16_INV_SCALE, v.y * smi::FP16_INV_SCALE);
    } else {
        return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w));
    }
}

// Box index of spectrum value (kx, ky), or -1 outside the stored box.
__device__ __forceinline__ int box_index(const PlanDev& p, int kx, int ky) {
    const bool in = ky >= -p.R && ky <= p.K && kx >= -p.K && kx <= p.K;
    return in ? (ky + p.R) * p.box_pitch + (kx + p.K) : -1;
}

// Source, destination and size of chunk c of W|V|U (VCH) or W|U of a tile:
// two spectrum values from an even box column, both, the first or neither
// inside the box (the box's last column 2K is even, so a chunk never starts
// outside it and ends inside).
template <bool VCH>
__device__ __forceinline__ void chunk_copy(const PlanDev& p, int c, int wx0, int wy0, int vx0, int vy0,
                                           int& src, int& dst, int& bytes) {
    int kx, ky;
    if (c < NCH_W) {
        const int r = c >> 3, h = c & 7;
        kx = wx0 + 2 * h; ky = wy0 + r; dst = OFF_W + r * PW + 2 * h;
    } else if (VCH && c < NCH_W + NCH_V) {
        const int c2 = c - NCH_W, r = c2 >> 2, h = c2 & 3;
        kx = vx0 + 2 * h; ky = vy0 + r; dst = OFF_V + r * smi::VBX + 2 * h;
    } else {
        const int c2 = c - NCH_W - (VCH ? NCH_V : 0), r = c2 / UCH, h = c2 - r * UCH;
        kx = wx0 - vx0 - (smi::VBX - 1) + 2 * h; ky = wy0 - vy0 - (smi::VBY - 1) + r;
        dst = OFF_U + r * PU + 2 * h;
    }
    const int i0 = box_index(p, kx, ky), i1 = box_index(p, kx + 1, ky);
    src = i0 >= 0 ? i0 : 0;
    bytes = i0 < 0 ? 0 : (i1 >= 0 ? 16 : 8);
}

// One tile (blockIdx-free) of subfield slot `sl`: B of spec[sl] into
// B[sl][tile]; S is the CTA's staging area, staging_float2<PREC>() float2 of
// 16-byte aligned shared memory (2 FB BUF for FP32 spectra, 3 FB BUF for
// half precision).  Runs on 128 threads; uses __syncthreads, so the
// whole CTA must call it.  VCH: V moves in 16-byte chunks (every tile's
// vx0 + K is even).  KAHAN: blocked compensated sums -- each block of two
// stages (2 FB frames) is summed plainly into a partial, which is then added
// to the running sum with Kahan compensation; partial, sum and correction
// fill the registers of 4 columns three times over, so the frames stream
// twice, 4 columns per pass.
template <int PREC, bool VCH, bool KAHAN>
__device__ __forceinline__ void bispec_tile(const PlanDev& p, const void* __restrict__ spec, int F,
                                            float2* __restrict__ B, int tile, int sl, float2* __restrict__ S) {
    constexpr int FB = Staging<PREC>::FB, E = Staging<PREC>::E;
    constexpr bool RAW = E == 4;                  // half precision: raw ring + FP32 compute buffer
    const int4 T = p.tiles[tile];
    const int wx0 = T.x, wy0 = T.y, vx0 = T.z, vy0 = T.w;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int wyl = lane >> 2, gx = lane & 3;

    // Offset columns kk for which some lane of this warp owns a used pair
    // (from the plan), rebuilt from warp votes so that the compiler treats
    // the mask as warp-uniform: the warp skips columns (and whole tiles) it
    // does not need with uniform branches.
    const unsigned planned = (__ldg(p.tile_masks + tile) >> (8 * warp)) & 0xFFu;
    unsigned kkmask = 0;
#pragma unroll
    for (int kk = 0; kk < smi::VBX; ++kk)
        if (__any_sync(0xffffffffu, (planned >> kk) & 1u)) kkmask |= 1u << kk;

    constexpr int NP = KAHAN ? 2 : 1;                // passes over the frames
    constexpr int NC = smi::VBX / NP;                // offset columns per pass
    const size_t box = (size_t)p.box_rows * p.box_pitch;
    const size_t sbase = (size_t)sl * F * box;
    float2* out = B + (size_t)(sl * p.n_tiles + tile) * TILE_PAIRS;
    const float sc = 1.0f / (float)F;
    auto write_out = [&](int col0, const float2 (&acc)[4][NC]) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float4* o = reinterpret_cast<float4*>(out + (wyl * smi::WBX + 4 * gx + j) * TILE_V +
                                                  warp * smi::VBX + col0);
#pragma unroll
            for (int q = 0; q < NC / 2; ++q)
                o[q] = make_float4(acc[j][2 * q].x * sc, acc[j][2 * q].y * sc,
                                   acc[j][2 * q + 1].x * sc, acc[j][2 * q + 1].y * sc);
        }
    };
    // spectrum values as E-byte words: float2, or half2 / bfloat162
    using Word = typename std::conditional<E == 8, float2, unsigned>::type;
    const Word* sp = reinterpret_cast<const Word*>(spec) + sbase;
    const int nst = (F + FB - 1) / FB;
    // The ring: E-byte slots, 2 stages x FB frames x BUF; the half-
    // precision compute buffers (2 x FB x BUF float2) follow it.
    Word* ring = reinterpret_cast<Word*>(S);
    float2* cbuf = S + FB * BUF;
    // Copy slots, fixed for the CTA: global source at frame 0, shared
    // destination in buffer 0 and size (chunk_copy counts 8-byte values).
    int src, dst, nb0, nb1 = 0;
    chunk_copy<VCH>(p, tid, wx0, wy0, vx0, vy0, src, dst, nb0);
    nb0 = nb0 * E / 8;
    const Word* g0 = sp + src;
    const unsigned s0 = (unsigned)__cvta_generic_to_shared(ring + dst);
    const bool v8 = !VCH && warp == 0;                  // warp 0 copies V by single values
    const int c1 = VCH ? tid + THREADS : tid + THREADS - NV;
    const bool has1 = v8 || c1 < NCH_W + NCH_U + (VCH ? NCH_V : 0);
    if (v8) {
        const int r = lane >> 3, c = lane & 7;
        const int i = box_index(p, vx0 + c, vy0 + r);
        src = i >= 0 ? i : 0; dst = OFF_V + r * smi::VBX + c; nb1 = i >= 0 ? E : 0;
    } else if (has1) {
        chunk_copy<VCH>(p, c1, wx0, wy0, vx0, vy0, src, dst, nb1);
        nb1 = nb1 * E / 8;
    } else {
        src = 0; dst = 0;
    }
    const Word* g1 = sp + src;
    const unsigned s1 = (unsigned)__cvta_generic_to_shared(ring + dst);
    auto copy = [&](unsigned soff, size_t goff, int n0, int n1) {
        cp_pair<E>(s0 + soff, g0 + goff, n0);
        if (v8) cp_one<E>(s1 + soff, g1 + goff, n1);
        else if (has1) cp_pair<E>(s1 + soff, g1 + goff, n1);
    };
    // Stage st holds frames FB st .. FB st + FB - 1; frames past F are
    // zero-filled (no global read) so that every stage is multiplied out whole.
    auto issue = [&](int st) {
        if (st < nst) {
            const unsigned sb = (unsigned)((st & 1) * FB * BUF * E);
            if (st * FB + FB <= F) {
#pragma unroll
                for (int ff = 0; ff < FB; ++ff)
                    copy(sb + ff * BUF * E, (size_t)(st * FB + ff) * box, nb0, nb1);
            } else {
#pragma unroll
                for (int ff = 0; ff < FB; ++ff) {
                    const bool in = st * FB + ff < F;
                    copy(sb + ff * BUF * E, in ? (size_t)(st * FB + ff) * box : 0, in ? nb0 : 0, in ? nb1 : 0);
                }
            }
        }
        asm volatile("cp.async.commit_group;");
    };
#pragma unroll
    for (int pass = 0; pass < NP; ++pass) {
        const int col0 = pass * NC;
        const unsigned pm = (kkmask >> col0) & ((1u << NC) - 1u);
        float2 acc[4][NC];                         // the sums (KAHAN: the running sums)
        float2 part[4][KAHAN ? NC : 1];            // KAHAN: this block's plain partial sums
        float2 comp[4][KAHAN ? NC : 1];            // KAHAN: the running sums' corrections
#pragma unroll
        for (int j = 0; j < 4; ++j) {
#pragma unroll
            for (int k = 0; k < NC; ++k) acc[j][k] = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < (KAHAN ? NC : 1); ++k) {
                comp[j][k] = make_float2(0.f, 0.f);
                part[j][k] = make_float2(0.f, 0.f);
            }
        }
        if (pass > 0) __syncthreads();             // the previous pass is done with the ring
        // Half precision converts stage st + 1 while stage st is
        // multiplied out, so one barrier per stage serves both: at the
        // barrier of iteration st the raw stage st + 1 has landed, the
        // conversion of stage st (into compute buffer st & 1) is complete
        // and the products of stage st - 1 are done with compute buffer
        // (st + 1) & 1.  The raw ring slot st & 1 is refilled with stage
        // st + 2, its conversion having finished before the barrier.
        auto convert = [&](int st) {
            const unsigned* rs = reinterpret_cast<const unsigned*>(ring) + (st & 1) * FB * BUF;
            float2* cb = cbuf + (st & 1) * FB * BUF;
            for (int e = tid; e < FB * BUF; e += THREADS) cb[e] = raw_to_float2<PREC>(rs[e]);
        };
        issue(0);
        if constexpr (RAW) {
            issue(1);
            asm volatile("cp.async.wait_group 1;");
            __syncthreads();                      // raw stage 0 visible
            convert(0);
        }
        for (int st = 0; st < nst; ++st) {
            asm volatile("cp.async.wait_group 0;");
            __syncthreads();          // stage st visible to all; stage st-1 fully consumed
            const float2* Sst;
            if constexpr (RAW) {
                issue(st + 2);
                if (st + 1 < nst) convert(st + 1);
                Sst = cbuf + (st & 1) * FB * BUF;
            } else {
                issue(st + 1);
                Sst = reinterpret_cast<const float2*>(ring) + (st & 1) * FB * BUF;
            }
            if (!pm) continue;
            auto& dst = [&]() -> float2 (&)[4][NC] {
                if constexpr (KAHAN) return part; else return acc;
            }();
            if (pm == (1u << NC) - 1u) {
#pragma unroll
                for (int ff = 0; ff < FB; ++ff)
                    accumulate_frame<true, NC>(Sst + ff * BUF, wyl, gx, warp, pm, col0, dst);
            } else {
#pragma unroll 1
                for (int ff = 0; ff < FB; ++ff)
                    accumulate_frame<false, NC>(Sst + ff * BUF, wyl, gx, warp, pm, col0, dst);
            }
            // KAHAN: every second stage (8 frames) and after the last one,
            // the partial sums go into the running sums
            if constexpr (KAHAN) if ((st & 1) == 1 || st + 1 == nst) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int k = 0; k < NC; ++k)
                        if (pm & (1u << k)) {                   // warp-uniform
                            kahan_add(acc[j][k].x, comp[j][k].x, part[j][k].x);
                            kahan_add(acc[j][k].y, comp[j][k].y, part[j][k].y);
                            part[j][k] = make_float2(0.f, 0.f);
                        }
            }
        }
        asm volatile("cp.async.wait_group 0;");
        if (pm) write_out(col0, acc);
    }
}


// float2 elements of the staging area bispec_tile<PREC> takes
template <int PREC> __host__ __device__ constexpr int staging_float2() {
    return Staging<PREC>::E == 8 ? 2 * Staging<PREC>::FB * BUF : 3 * Staging<PREC>::FB * BUF;
}
__host__ __device__ constexpr size_t staging_bytes(int prec) {
    return (size_t)(prec == SM_FP32 ? staging_float2<SM_FP32>() : staging_float2<SM_FP16>()) * 8;
}

}  // namespace smb
