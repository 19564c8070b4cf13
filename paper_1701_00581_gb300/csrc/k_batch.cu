// Batched persistent launch: the subfield spectra (Sect. 2: Fourier transform
// of every subimage) and the mean bispectrum (Sect. 2, Sect. 3.2: speckle
// masking) of several bursts -- of one or several channels, with subfields of
// different sizes -- in one kernel.
//
// The launch is persistent: one grid of 128-thread CTAs, as many as fit on
// the GPU, takes work items from one device queue by an atomic counter until
// the queue is empty.  Two kinds of item:
//
//   FFT  (burst, subfield, frame): cut, apodise, mean-subtract, 2-D DFT and
//        normalise one frame tile (the transform of k_spectra, computed by
//        128 threads: the row transforms go to the column transforms through
//        a per-CTA scratch tile in global memory, which stays in L2);
//   BIS  (burst, subfield, tile):  one bispectrum tile of the subfield over
//        all of the burst's frames (the tile body of k_bispectrum).
//
// A BIS item needs every frame spectrum of its subfield: each FFT item, once
// its spectrum is stored, increments the subfield's counter (release), and a
// BIS item waits until the counter reaches F (acquire).  The host orders the
// queue so that a subfield's FFT items precede its BIS items; an item is only
// ever waited on after it has been taken by a running CTA, so every wait
// ends.  The wait is still bounded: after SPIN_LIMIT polls the CTA records
// the error in the status word and skips the item.  Because the spectra of
// later subfields are transformed while earlier subfields' tiles are
// accumulated, the latency-bound transforms share the SMs with the
// ALU-bound bispectrum instead of running as a stage of their own.
//
// Every result depends only on its item's inputs, in a fixed order of
// operations: a burst's spectra and bispectrum are bitwise the same whatever
// other bursts share the launch and in whatever order the CTAs take items.
#include "sm_bispec_tile.cuh"
#include "sm_fft_dev.cuh"

namespace {

using smi::BatchArgs;
using smi::BatchBurst;
using smi::PlanDev;

constexpr int BT = 128;                       // threads per CTA (the bispectrum tile's)
constexpr long long SPIN_LIMIT = 1ll << 23;   // polls of a dependency counter (>= ~2 s) before giving up

// Thread groups of the 128-thread four-step transform.
template <int N> struct BGrp {
    static constexpr int P = smf::Split<N>::P, Q = smf::Split<N>::Q;
    static constexpr int G = P > Q ? P : Q;                         // threads per transform
    static constexpr int NG = BT / G;                                // transforms in flight
    static constexpr int TB = (Q * (P + 1) > N ? Q * (P + 1) : N);   // exchange tile (holds a row)
    static constexpr int RR = 2 * NG;                                // rows per round (two per transform)
    static_assert((N / 2) % NG == 0, "whole rounds of row pairs");
};

// Shared memory of one FFT item (bytes), for K1 = K + 1 columns.
__host__ __device__ constexpr int rs_pitch(int K1) { return K1 | 1; }
template <int N>
__host__ __device__ constexpr size_t fft_item_smem(int K1) {
    using GP = BGrp<N>;
    const size_t stage = (size_t)GP::RR * rs_pitch(K1) > (size_t)GP::NG * (N + 1)
                             ? (size_t)GP::RR * rs_pitch(K1) : (size_t)GP::NG * (N + 1);
    return ((size_t)N + (size_t)K1 + (size_t)GP::NG * GP::TB + stage) * sizeof(float2)   // tw, wf, T, stage
           + (size_t)2 * N * sizeof(float)                                               // windows
           + 4 * sizeof(double);                                                         // scalars
}

// Spectrum of frame f of subfield s (workspace slot s): the transform of
// k_spectra -- rows of the windowed tile (two real rows per complex FFT),
// the windowed mean from the rows' DC terms, the mean times the window
// removed through the window's own transform, the K+1 non-negative columns,
// normalisation by the windowed flux and the box ky = -R..K stored.  scr is
// this CTA's [K+1][N] scratch tile.
template <int N, typename TIn, int PREC>
__device__ __forceinline__ void fft_item(const PlanDev& p, const TIn* __restrict__ frames, int F, int s, int f,
                                         void* __restrict__ spec, float* __restrict__ flux, float* __restrict__ mu,
                                         float2* __restrict__ scr, unsigned char* smem) {
    using GP = BGrp<N>;
    constexpr int P = GP::P, Q = GP::Q, G = GP::G, NG = GP::NG, TB = GP::TB, RR = GP::RR;
    const int K = p.K, K1 = K + 1, RP = rs_pitch(K1), CP = N + 1;
    float2* stw = reinterpret_cast<float2*>(smem);
    float2* swf = stw + N;
    float2* Tall = swf + K1;
    float2* stage = Tall + NG * TB;
    const size_t nstage = (size_t)RR * RP > (size_t)NG * CP ? (size_t)RR * RP : (size_t)NG * CP;
    float* swx = reinterpret_cast<float*>(stage + nstage);
    float* swy = swx + N;
    double* red = reinterpret_cast<double*>(swy + N);

    const int tid = threadIdx.x, grp = tid / G, g = tid - grp * G;
    float2* T = Tall + grp * TB;
    const int4 sb = p.subs[s];
    const int x0 = sb.x, y0 = sb.y, w = sb.z, h = sb.w;
    for (int i = tid; i < N; i += BT) {
        stw[i] = p.tw[i];
        swx[i] = p.winx[(size_t)s * N + i];
        swy[i] = p.winy[(size_t)s * N + i];
    }
    for (int i = tid; i < K1; i += BT) swf[i] = p.winft[(size_t)s * K1 + i];
    __syncthreads();

    // rows: round r, group grp transforms rows 2 (r NG + grp) and +1; the
    // round's RR rows of K+1 columns go through `stage` to scr[kx][y]
    const TIn* fr = frames + (size_t)f * p.H * p.W + (size_t)y0 * p.W + x0;
    double dc = 0.0;                                   // thread 0: sum of the rows' DC terms
    for (int pr0 = 0; pr0 < N / 2; pr0 += NG) {
        const int y1 = 2 * (pr0 + grp), y2 = y1 + 1;
        float2 v[Q], X[P];
#pragma unroll
        for (int n2 = 0; n2 < Q; ++n2) {
            const int x = g + P * n2;
            const bool inx = g < P && x < w;
            const float r1 = inx && y1 < h ? smf::load_sample(fr + (size_t)y1 * p.W + x) : 0.f;
            const float r2 = inx && y2 < h ? smf::load_sample(fr + (size_t)y2 * p.W + x) : 0.f;
            const float wx = swx[x & (N - 1)];
            v[n2] = make_float2(wx * swy[y1] * r1, wx * swy[y2] * r2);
        }
        smf::four_step<N, false>(v, X, T, stw, g);
        if (g < Q) {
#pragma unroll
            for (int k1 = 0; k1 < P; ++k1) T[g + Q * k1] = X[k1];
        }
        __syncwarp();
        for (int kx = g; kx < K1; kx += G) {
            const float2 za = T[kx], zb = T[(N - kx) & (N - 1)];
            stage[(2 * grp) * RP + kx] = make_float2(0.5f * (za.x + zb.x), 0.5f * (za.y - zb.y));
            stage[(2 * grp + 1) * RP + kx] = make_float2(0.5f * (za.y + zb.y), -0.5f * (za.x - zb.x));
        }
        __syncthreads();
        if (tid == 0)
            for (int r = 0; r < RR; ++r) dc += (double)stage[r * RP].x;
        for (int e = tid; e < K1 * RR; e += BT) {
            const int kx = e / RR, r = e - kx * RR;
            scr[(size_t)kx * N + 2 * pr0 + r] = stage[r * RP + kx];
        }
        __syncthreads();
    }
    if (tid == 0) {
        const double wsum = p.winsum[s];
        const float m = (float)(dc / wsum);
        const double fl = (double)m * wsum;
        red[0] = fl;
        reinterpret_cast<float*>(red + 1)[0] = (float)(1.0 / fl);
        reinterpret_cast<float*>(red + 1)[1] = m;
        flux[(size_t)s * F + f] = (float)fl;
        mu[(size_t)s * F + f] = m;
    }
    __syncthreads();
    const float mean = reinterpret_cast<const float*>(red + 1)[1];
    const float inv = reinterpret_cast<const float*>(red + 1)[0];

    // columns kx = 0..K, NG at a time, with mean * window removed on the way
    // in (row transform of w_x w_y mu is mu w_y(y) Wx(kx)); each round's
    // columns are written to the box rows from `stage` (64-byte row runs)
    const size_t base = ((size_t)s * F + f) * p.box_rows * p.box_pitch;
    for (int c0 = 0; c0 < K1; c0 += NG) {
        const int kx = c0 + grp;
        const int kc = kx < K1 ? kx : K1 - 1;
        const float2 wf = swf[kc];
        float2 v[Q], X[P];
#pragma unroll
        for (int n2 = 0; n2 < Q; ++n2) {
            const int y = g + P * n2;
            float2 c = make_float2(0.f, 0.f);
            if (g < P) {
                c = __ldcg(scr + (size_t)kc * N + y);
                const float a = mean * swy[y];
                c.x -= a * wf.x;
                c.y -= a * wf.y;
            }
            v[n2] = c;
        }
        smf::four_step<N, false>(v, X, T, stw, g);
        if (g < Q) {
#pragma unroll
            for (int k1 = 0; k1 < P; ++k1) stage[grp * CP + g + Q * k1] = X[k1];
        }
        __syncthreads();
        const int ncol = K1 - c0 < NG ? K1 - c0 : NG;
        for (int e = tid; e < p.box_rows * ncol; e += BT) {
            const int row = e / ncol, j = e - row * ncol, cx = c0 + j, ky = row - p.R;
            float2 a = stage[j * CP + (ky & (N - 1))];
            a.x *= inv;
            a.y *= inv;
            if (cx == 0 && ky == 0) a = make_float2(1.f, 0.f);
            smf::store_spec<PREC>(spec, base + (size_t)row * p.box_pitch + cx + K, a);
            if (cx > 0) {
                float2 b = stage[j * CP + ((-ky) & (N - 1))];
                b.x *= inv;
                b.y = -b.y * inv;
                smf::store_spec<PREC>(spec, base + (size_t)row * p.box_pitch + K - cx, b);
            }
        }
        __syncthreads();
    }
}

template <typename TIn, int PREC>
__device__ __forceinline__ void fft_dispatch(const BatchBurst& b, int s, int f, float2* scr, unsigned char* smem) {
    const TIn* fr = reinterpret_cast<const TIn*>(b.frames);
    switch (b.p.N) {
        case 64: fft_item<64, TIn, PREC>(b.p, fr, b.F, s, f, b.spec, b.flux, b.mu, scr, smem); break;
        case 128: fft_item<128, TIn, PREC>(b.p, fr, b.F, s, f, b.spec, b.flux, b.mu, scr, smem); break;
        default: fft_item<256, TIn, PREC>(b.p, fr, b.F, s, f, b.spec, b.flux, b.mu, scr, smem); break;
    }
}

__device__ __forceinline__ int load_acquire(const int* a) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
    return v;
}

// One bispectrum tile as a call of its own, so that its register allocation
// does not share the persistent loop's live values.
template <int PREC, bool VCH>
__device__ __noinline__ void tile_call(const PlanDev& p, const void* spec, int F, float2* B, int tile, int sl,
                                       float2* S) {
    smb::bispec_tile<PREC, VCH, false>(p, spec, F, B, tile, sl, S);
}

// MINB: CTAs per SM the register allocation is sized for (4: 128 registers
// per thread; 3: 168, so the tile body does not spill).
template <int PREC, int MINB>
__global__ void __launch_bounds__(BT, MINB)
k_batch(const __grid_constant__ BatchArgs a, const int4* __restrict__ items, int n_items, int* head, int* cnt,
        int* status, float2* __restrict__ scratch, size_t scr_elems) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_cur, s_next, s_skip;
    const int tid = threadIdx.x;
    if (tid == 0) s_cur = atomicAdd(head, 1);
    // No value lives across an item in registers: the item's work needs all
    // of them, so the current index is re-read from shared memory.
    for (;;) {
        __syncthreads();                             // s_cur visible; smem free for the next item
        // the item index and record through warp reductions: the same in
        // every lane, and known so to the compiler, which keeps the item's
        // dispatch and loops uniform
        const int cur = (int)__reduce_or_sync(0xffffffffu, (unsigned)s_cur);
        if (cur >= n_items) break;
        if (tid == 0) s_next = atomicAdd(head, 1);   // the next item, fetched while this one runs
        const int4 rec = items[cur];
        const int4 it = make_int4((int)__reduce_or_sync(0xffffffffu, (unsigned)rec.x),
                                  (int)__reduce_or_sync(0xffffffffu, (unsigned)rec.y),
                                  (int)__reduce_or_sync(0xffffffffu, (unsigned)rec.z),
                                  (int)__reduce_or_sync(0xffffffffu, (unsigned)rec.w));
        const BatchBurst& b = a.b[it.y];
        const int s = it.z;
        if (it.x == 0) {
            float2* scr = scratch + (size_t)blockIdx.x * scr_elems;
            if (b.frame_type == SM_U16) fft_dispatch<uint16_t, PREC>(b, s, it.w, scr, smem);
            else fft_dispatch<float, PREC>(b, s, it.w, scr, smem);
            __syncthreads();                         // the whole spectrum is stored
            if (tid == 0) {
                __threadfence();
                atomicAdd(cnt + b.cnt_base + s, 1);  // release: one more frame of subfield s
            }
        } else {
            if (tid == 0) {
                int skip = 0;
                long long n = 0;
                while (load_acquire(cnt + b.cnt_base + s) < b.need) {
                    if (++n > SPIN_LIMIT) {
                        atomicOr(status, 1);         // dependency wait gave up
                        skip = 1;
                        break;
                    }
                    __nanosleep(256);
                }
                s_skip = skip;
            }
            __syncthreads();
            if (!s_skip) {
                float2* S = reinterpret_cast<float2*>(smem);
                const bool vch = ((b.p.v_org + b.p.K) & 1) == 0;
                if (vch) tile_call<PREC, true>(b.p, b.spec, b.F, b.B, it.w, s, S);
                else tile_call<PREC, false>(b.p, b.spec, b.F, b.B, it.w, s, S);
            }
        }
        __syncthreads();                             // s_next visible, the item's work done
        if (tid == 0) s_cur = s_next;
    }
}

// SM_BATCH_GRID: for the bursts of the batch that share one plan, one CTA
// per (tile, subfield, burst) -- grid (n_tiles, n_sub, bursts) -- scheduled
// by the hardware like the per-stage bispectrum kernel.  The plan is a
// by-value argument, as there, so its fields stay constant-bank operands;
// only the bursts' buffers are looked up by blockIdx.z.
template <int PREC, bool VCH>
__global__ void __launch_bounds__(BT, 4) k_batch_grid(PlanDev p, const __grid_constant__ smi::BatchPtrs q) {
    __shared__ __align__(16) float2 S[smb::staging_float2<PREC>()];
    const int z = blockIdx.z;
    smb::bispec_tile<PREC, VCH, false>(p, q.spec[z], q.F[z], q.B[z], blockIdx.x, blockIdx.y, S);
}

size_t fft_smem_for(int N, int K) {
    switch (N) {
        case 64: return fft_item_smem<64>(K + 1);
        case 128: return fft_item_smem<128>(K + 1);
        default: return fft_item_smem<256>(K + 1);
    }
}

}  // namespace

namespace smk {

size_t batch_smem_bytes(int N, int K, int prec) {
    const size_t bis = smb::staging_bytes(prec);
    const size_t fft = N > 0 ? fft_smem_for(N, K) : 0;
    return bis > fft ? bis : fft;
}

namespace {

// The dynamic shared memory limit is an attribute of the function, shared by
// every batch: it is set to the device's largest opt-in size once, so a batch
// built later with smaller subfields cannot lower it under an earlier batch.
template <int PREC, int MINB>
int fit(size_t smem) {
    int n = 0, dev = 0, optin = 0;
    cudaFuncAttributes fa;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_batch<PREC, MINB>);
    const int dyn_max = optin - (int)fa.sharedSizeBytes;
    if (e == cudaSuccess && smem > (size_t)dyn_max) return 0;
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_batch<PREC, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch<PREC, MINB>, BT, smem);
    return e == cudaSuccess ? n : -1;
}

template <int PREC, int MINB>
void go(const BatchArgs& a, const int4* items, int n_items, int* head, int* cnt, int* status, float2* scratch,
        size_t scr_elems, int grid, size_t smem, cudaStream_t st) {
    k_batch<PREC, MINB><<<grid, BT, smem, st>>>(a, items, n_items, head, cnt, status, scratch, scr_elems);
}

}  // namespace

int batch_blocks_per_sm(size_t smem, int prec, int minb) {
    if (minb == 3) return prec == SM_FP32 ? fit<SM_FP32, 3>(smem) : prec == SM_FP16 ? fit<SM_FP16, 3>(smem)
                                                                                   : fit<SM_BF16, 3>(smem);
    return prec == SM_FP32 ? fit<SM_FP32, 4>(smem) : prec == SM_FP16 ? fit<SM_FP16, 4>(smem) : fit<SM_BF16, 4>(smem);
}

cudaError_t launch_batch(const BatchArgs& a, int prec, int minb, const int4* items, int n_items, int* head, int* cnt,
                         int* status, float2* scratch, size_t scr_elems, int grid, size_t smem, cudaStream_t st) {
    if (minb == 3) {
        if (prec == SM_FP32) go<SM_FP32, 3>(a, items, n_items, head, cnt, status, scratch, scr_elems, grid, smem, st);
        else if (prec == SM_FP16) go<SM_FP16, 3>(a, items, n_items, head, cnt, status, scratch, scr_elems, grid, smem, st);
        else go<SM_BF16, 3>(a, items, n_items, head, cnt, status, scratch, scr_elems, grid, smem, st);
    } else {
        if (prec == SM_FP32) go<SM_FP32, 4>(a, items, n_items, head, cnt, status, scratch, scr_elems, grid, smem, st);
        else if (prec == SM_FP16) go<SM_FP16, 4>(a, items, n_items, head, cnt, status, scratch, scr_elems, grid, smem, st);
        else go<SM_BF16, 4>(a, items, n_items, head, cnt, status, scratch, scr_elems, grid, smem, st);
    }
    return cudaGetLastError();
}

cudaError_t launch_batch_grid(const PlanDev& p, const smi::BatchPtrs& q, cudaStream_t st) {
    const dim3 grid(p.n_tiles, p.n_sub, q.n);
    const bool vch = ((p.v_org + p.K) & 1) == 0;
    if (p.prec == SM_FP32) {
        if (vch) k_batch_grid<SM_FP32, true><<<grid, BT, 0, st>>>(p, q);
        else k_batch_grid<SM_FP32, false><<<grid, BT, 0, st>>>(p, q);
    } else if (p.prec == SM_FP16) {
        if (vch) k_batch_grid<SM_FP16, true><<<grid, BT, 0, st>>>(p, q);
        else k_batch_grid<SM_FP16, false><<<grid, BT, 0, st>>>(p, q);
    } else {
        if (vch) k_batch_grid<SM_BF16, true><<<grid, BT, 0, st>>>(p, q);
        else k_batch_grid<SM_BF16, false><<<grid, BT, 0, st>>>(p, q);
    }
    return cudaGetLastError();
}

}  // namespace smk
