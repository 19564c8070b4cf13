// Recursive Fourier phase from the mean bispectrum (Sect. 3.2: speckle
// masking phase, Lohmann, Weigelt & Wirnitzer 1983).
//
// Since arg B(w - v, v) = phi(w - v) + phi(v) - phi(w), each split of a
// target w into two already known frequencies gives a phasor estimate of
// exp(i phi(w)).  One CTA per subfield walks the rings of equal |w|^2 in
// ascending order (points of one ring never depend on each other).  The
// ring's work is a list of (point, bispectrum tile) items; the 16 warps
// take items round-robin, eight at a time so that their B loads are in
// flight together, and sum exp(i(phi(w-v) + phi(v))) conj B over the
// offsets of the tile into one partial per item.  Then one warp per point
// adds its partials along a fixed tree and stores z(w) = S / |S|: the
// result does not depend on scheduling.  Arithmetic is FP32 by default
// (GB300's FP64 unit is shared by the SM's warps and a small fraction of its
// FP32 rate), or FP64 throughout when the channel asks for it; the known
// phasors live in shared memory in that type and the result is stored as FP64.
#include "sm_internal.h"

namespace {

using smi::PlanDev;
using smi::TILE_PAIRS;
using smi::TILE_V;

// Items are spread over 16 virtual warps whatever the CTA size: each item
// then lands in the same slot of the same batch, and its sum runs along the
// same shuffle tree, in the 512-thread kernel (two CTAs per SM, the stage
// path) and in the 256-thread one (64 registers a thread, so it fits beside
// three bispectrum CTAs on an SM): the two give bitwise the same phasors.
constexpr int PH_VWARPS = 16;

// Complex values of the recursion's arithmetic type T.
template <typename T> struct Cx;
template <> struct Cx<float> {
    using T2 = float2;
    __device__ static float2 make(float x, float y) { return make_float2(x, y); }
    __device__ static float rnorm(float n2) { return rsqrtf(n2); }
};
template <> struct Cx<double> {
    using T2 = double2;
    __device__ static double2 make(double x, double y) { return make_double2(x, y); }
    __device__ static double rnorm(double n2) { return 1.0 / sqrt(n2); }
};

// Float-float ("double-single") numbers: an unevaluated sum hi + lo of two
// floats, |lo| <= ulp(hi) / 2, with about 48 significant bits, computed on
// the FP32 pipe -- GB300's FP64 unit runs at a small fraction of its FP32
// rate.  The error-free transformations are Knuth's two-sum, Dekker's
// fast-two-sum and the FMA-based two-product (the product's exact low part
// is fma(a, b, -a b)); addition and multiplication are the classical
// double-single ones, division and the reciprocal square root one Newton
// correction of the float estimate.  The type and its functions live in a
// namespace of their own: argument-dependent lookup adds them to the
// overloads of sqrt and __shfl_xor_sync without hiding the built-in ones.
namespace ffa {
struct ff {
    float hi, lo;
    __device__ ff() : hi(0.f), lo(0.f) {}
    __device__ ff(int v) : hi((float)v), lo(0.f) {}
    __device__ ff(float v) : hi(v), lo(0.f) {}
    __device__ ff(float h, float l) : hi(h), lo(l) {}
    __device__ explicit ff(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
    __device__ explicit operator double() const { return (double)hi + (double)lo; }
};
__device__ __forceinline__ ff fast_two_sum(float a, float b) {       // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return ff(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float v = __fsub_rn(s, a);
    return ff(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v)));
}
__device__ __forceinline__ ff operator+(ff a, ff b) {
    ff s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ff operator-(ff a) { return ff(-a.hi, -a.lo); }
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }
__device__ __forceinline__ ff operator*(ff a, ff b) {
    const float p = __fmul_rn(a.hi, b.hi);
    const float e = __fmaf_rn(a.hi, b.hi, -p);
    return fast_two_sum(p, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e)));
}
__device__ __forceinline__ ff operator/(ff a, ff b) {
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const ff r = a - b * ff(q1);
    return fast_two_sum(q1, __fdiv_rn(r.hi, b.hi));
}
__device__ __forceinline__ ff& operator+=(ff& a, ff b) { return a = a + b; }
__device__ __forceinline__ ff& operator/=(ff& a, ff b) { return a = a / b; }
__device__ __forceinline__ bool operator>(ff a, ff b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
__device__ __forceinline__ ff sqrt(ff a) {
    if (!(a.hi > 0.f)) return ff(0.f);
    const float s = sqrtf(a.hi);
    const ff r = a - ff(s) * ff(s);                  // exact residual of s^2
    return fast_two_sum(s, __fdiv_rn(r.hi, 2.f * s));
}
__device__ __forceinline__ ff __shfl_xor_sync(unsigned mask, ff v, int o) {
    return ff(::__shfl_xor_sync(mask, v.hi, o), ::__shfl_xor_sync(mask, v.lo, o));
}
}  // namespace ffa
using ffa::ff;
struct ff2 { ff x, y; };
template <> struct Cx<ff> {
    using T2 = ff2;
    __device__ static ff2 make(ff x, ff y) { return ff2{x, y}; }
    // 1 / sqrt(n2): the float estimate r, then r (3 - n2 r^2) / 2 in float-float
    __device__ static ff rnorm(ff n2) {
        const ff r(rsqrtf(n2.hi));
        return r * (ff(3.f) - n2 * r * r) * ff(0.5f);
    }
};

// z of any frequency from the half-box copy (row 0 holds both signs).
template <typename T2>
__device__ __forceinline__ T2 zget(const T2* zs, int pitch, int K, int kx, int ky) {
    if (ky >= 0) return zs[ky * pitch + kx + K];
    T2 t = zs[(-ky) * pitch - kx + K];
    t.y = -t.y;
    return t;
}

constexpr int PH_ITEMS = 8;           // items per warp batch (all loads in flight together)

// Eight per-lane values -> eight warp sums, by recursive halving: after the
// exchanges at distances 16, 8 and 4 each lane holds one item's partial sum
// over 8 lanes (item = lane >> 2), then two xor steps finish it.  18 shuffles
// instead of 8 full reductions (80).
template <typename T2>
__device__ __forceinline__ T2 reduce8(T2 (&s)[PH_ITEMS], int lane) {
#pragma unroll
    for (int lvl = 0, o = 16, n = PH_ITEMS / 2; lvl < 3; ++lvl, o >>= 1, n >>= 1) {
        const bool hi = lane & o;
#pragma unroll
        for (int q = 0; q < n; ++q) {
            const T2 keep = hi ? s[q + n] : s[q];
            const T2 give = hi ? s[q] : s[q + n];
            s[q].x = keep.x + __shfl_xor_sync(0xffffffffu, give.x, o);
            s[q].y = keep.y + __shfl_xor_sync(0xffffffffu, give.y, o);
        }
    }
    T2 r = s[0];
#pragma unroll
    for (int o = 2; o > 0; o >>= 1) {
        r.x += __shfl_xor_sync(0xffffffffu, r.x, o);
        r.y += __shfl_xor_sync(0xffffffffu, r.y, o);
    }
    return r;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(sa), "l"(gmem));
}

// Shared memory: item partial sums of the ring and the phasor table (complex
// values of e2 bytes), the item records of the next ring and the point
// records of this and the next ring.
__host__ __device__ inline size_t phase_layout(int hb_rows, int pitch, int mri, int mrp, size_t e2, size_t* o_zs,
                                               size_t* o_itm, size_t* o_prc) {
    size_t o = 0;
    o += ((size_t)mri * e2 + 15) & ~(size_t)15;
    *o_zs = o;
    o += ((size_t)hb_rows * pitch * e2 + 15) & ~(size_t)15;
    *o_itm = o;
    o += (size_t)mri * sizeof(int4);
    *o_prc = o;
    o += (size_t)2 * mrp * sizeof(int4);
    return o;
}

template <typename T, int TH>
__global__ void __launch_bounds__(TH, TH == 512 ? (sizeof(T) == 4 ? 2 : 1) : 4)
k_phase(PlanDev p, const float2* __restrict__ B, const float2* __restrict__ M, const float* __restrict__ P,
        double2* __restrict__ z) {
    constexpr int PH_THREADS = TH, PH_WARPS = TH / 32;
    using T2 = typename Cx<T>::T2;
    extern __shared__ __align__(16) unsigned char smem[];
    const int K = p.K, pitch = p.box_pitch;
    const size_t hb = (size_t)p.hb_rows * pitch;
    size_t o_zs, o_itm, o_prc;
    phase_layout(p.hb_rows, pitch, p.max_ring_items, p.max_ring_points, sizeof(T2), &o_zs, &o_itm, &o_prc);
    T2* part = reinterpret_cast<T2*>(smem);
    T2* zs = reinterpret_cast<T2*>(smem + o_zs);
    int4* const itm = reinterpret_cast<int4*>(smem + o_itm);
    int4* const prc = reinterpret_cast<int4*>(smem + o_prc);
    // the warp index through a warp reduction, so that the compiler knows it
    // is the same in every lane and keeps the loops over it uniform
    const int sl = blockIdx.x, tid = threadIdx.x, lane = tid & 31;
    const int warp = (int)__reduce_or_sync(0xffffffffu, (unsigned)(tid >> 5));
    double2* zo = z + (size_t)sl * hb;
    for (int e = tid; e < (int)hb; e += PH_THREADS) zs[e] = Cx<T>::make(0, 0);
    __syncthreads();
    if (tid == 0) {
        zs[K] = Cx<T>::make(1, 0);
        zo[K] = make_double2(1.0, 0.0);
        // anchors: z(e_x) = M(e_x)/|M(e_x)|, z(e_y) = M(e_y)/|M(e_y)|
        const float2 mx = M[(size_t)sl * hb + K + 1];
        const float2 my = M[(size_t)sl * hb + pitch + K];
        double n = hypot((double)mx.x, (double)mx.y);
        const double2 ax = n > 0 ? make_double2(mx.x / n, mx.y / n) : make_double2(1.0, 0.0);
        n = hypot((double)my.x, (double)my.y);
        const double2 ay = n > 0 ? make_double2(my.x / n, my.y / n) : make_double2(1.0, 0.0);
        zs[K + 1] = Cx<T>::make((T)ax.x, (T)ax.y);
        zs[K - 1] = Cx<T>::make((T)ax.x, -(T)ax.y);
        zs[pitch + K] = Cx<T>::make((T)ay.x, (T)ay.y);
        zo[K + 1] = ax;
        zo[K - 1] = make_double2(ax.x, -ax.y);
        zo[pitch + K] = ay;
    }

    const bool unit = p.weight == SM_W_UNIT, snr = p.weight == SM_W_SNR;
    const float* Ps = P + (size_t)sl * hb;         // power spectrum, for the SNR weighting
    auto pget = [&](int kx, int ky) -> T {          // P(-k) = P(k)
        return (T)(ky >= 0 ? __ldg(Ps + ky * pitch + kx + K) : __ldg(Ps + (-ky) * pitch - kx + K));
    };
    const float2* Bs = B + (size_t)sl * p.n_tiles * TILE_PAIRS;
    // Stage the item and point records of ring q (< n_rings) into shared
    // memory: items into itm, points into prc[q & 1].
    auto stage = [&](int q) {
        if (q < p.n_rings) {
            const int i0 = p.ring_items[q], ni = p.ring_items[q + 1] - i0;
            const int p0 = p.ring_start[q], np = p.ring_start[q + 1] - p0;
            for (int e = tid; e < ni; e += PH_THREADS) cp_async16(itm + e, p.items + i0 + e);
            int4* pr = prc + (q & 1) * p.max_ring_points;
            for (int e = tid; e < np; e += PH_THREADS) cp_async16(pr + e, p.point_rec + p0 + e);
        }
        asm volatile("cp.async.commit_group;");
    };
    // A batch is up to PH_ITEMS items of one warp: per item the packed
    // coordinates (w and the tile's offset origin as signed bytes) and this
    // lane's B value (when the lane's (w, v) pair is read).
    float2 bv[PH_ITEMS];
    unsigned pk[PH_ITEMS];
    unsigned okm = 0;
    auto load_batch = [&](const int4* recs, int base, int ni) {
        okm = 0;
#pragma unroll
        for (int q = 0; q < PH_ITEMS; ++q) {
            const int e = base + q * PH_VWARPS;
            bv[q] = make_float2(0.f, 0.f);
            pk[q] = 0;
            if (e < ni) {
                const int4 item = recs[e];
                pk[q] = (unsigned)item.x;
                if ((unsigned)item.z & (1u << lane)) {
                    okm |= 1u << q;
                    bv[q] = Bs[(size_t)item.y + lane];
                }
            }
        }
    };
    // Per ring r: (0) stage ring r+1's records; (1) items of ring r -> one
    // FP32 partial per item; barrier; (2) load ring r+1's first batch from the
    // staged records (its B loads overlap step 3); (3) one warp per point sums
    // its items and stores z = S / |S|; barrier.
    int i0 = p.ring_items[0];
    int ni = (int)__reduce_or_sync(0xffffffffu, (unsigned)(p.ring_items[1] - i0));
    int np = (int)__reduce_or_sync(0xffffffffu, (unsigned)(p.ring_start[1] - p.ring_start[0]));
    stage(0);
    asm volatile("cp.async.wait_group 0;");
    __syncthreads();                              // anchors and ring 0 records visible
    load_batch(itm, warp, ni);
    __syncthreads();                              // staging buffer free again
    for (int r = 0; r < p.n_rings; ++r) {
        const bool more = r + 1 < p.n_rings;
        const int i0n = more ? p.ring_items[r + 1] : 0;
        const int nin = (int)__reduce_or_sync(0xffffffffu, (unsigned)(more ? p.ring_items[r + 2] - i0n : 0));
        const int npn = (int)__reduce_or_sync(0xffffffffu,
                                              (unsigned)(more ? p.ring_start[r + 2] - p.ring_start[r + 1] : 0));
        stage(r + 1);
        // (1) items: products in T, one term per lane, item sums in T
        // One batch of up to PH_ITEMS items of a (virtual) warp: 512 threads
        // give one virtual warp per warp, 256 two, one after the other.
        auto item_batch = [&](int base, bool first) {
            if (!first) load_batch(p.items + i0, base, ni);
            T2 t[PH_ITEMS];
#pragma unroll
            for (int q = 0; q < PH_ITEMS; ++q) {
                t[q] = Cx<T>::make(0, 0);
                if (okm & (1u << q)) {
                    const int wx = (signed char)(pk[q] & 255), wy = (signed char)((pk[q] >> 8) & 255);
                    const int vx = (signed char)((pk[q] >> 16) & 255) + (lane % smi::VBX);
                    const int vy = (signed char)((pk[q] >> 24) & 255) + (lane / smi::VBX);
                    const T bx = (T)bv[q].x, by = (T)bv[q].y;
                    const T2 zu = zget(zs, pitch, K, wx - vx, wy - vy);
                    const T2 zv = zget(zs, pitch, K, vx, vy);
                    const T2 c = Cx<T>::make(zu.x * zv.x - zu.y * zv.y, zu.x * zv.y + zu.y * zv.x);
                    T tx = c.x * bx + c.y * by;            // c * conj(b)
                    T ty = c.y * bx - c.x * by;
                    if (unit) {
                        const T m = sqrt(bx * bx + by * by);
                        if (m > (T)0) {
                            tx /= m;
                            ty /= m;
                        } else {
                            tx = ty = (T)0;
                        }
                    } else if (snr) {                   // |B|^2 over the speckle-noise variance of B
                        const T den = pget(wx - vx, wy - vy) * pget(vx, vy) * pget(wx, wy);
                        if (den > (T)0) {
                            tx /= den;
                            ty /= den;
                        } else {
                            tx = ty = (T)0;
                        }
                    }
                    t[q] = Cx<T>::make(tx, ty);
                }
            }
            const T2 sum = reduce8(t, lane);
            const int e = base + (lane >> 2) * PH_VWARPS;
            if ((lane & 3) == 0 && e < ni) part[e] = sum;
        };
        if constexpr (TH == 512) {
            for (int base = warp; base < ni; base += PH_VWARPS * PH_ITEMS) item_batch(base, base == warp);
        } else {
            bool first = true;
            for (int vw = warp; vw < PH_VWARPS; vw += PH_WARPS)
                for (int base = vw; base < ni; base += PH_VWARPS * PH_ITEMS) {
                    item_batch(base, first);
                    first = false;
                }
        }
        asm volatile("cp.async.wait_group 0;");
        __syncthreads();                          // partials complete, ring r+1 records visible
        if (more) {
            load_batch(itm, warp, nin);
            // the B values of ring r+1's later batches towards L2 while this
            // ring's points are summed: two 128-byte lines per item
            for (int e = tid; e < nin; e += PH_THREADS) {
                if (e < PH_VWARPS * PH_ITEMS && e % PH_VWARPS < PH_WARPS) continue;   // in the first batch
                const char* a = reinterpret_cast<const char*>(Bs + itm[e].y);
                asm volatile("prefetch.global.L2 [%0];" :: "l"(a));
                asm volatile("prefetch.global.L2 [%0];" :: "l"(a + 128));
            }
        }
        // (3) one warp per point: sum of its items along a fixed shuffle
        // tree, then z = S / |S|, in T (with T = float GB300's shared FP64
        // unit no longer serialises this step across warps).  The stored
        // state is FP64.
        const int4* pr = prc + (r & 1) * p.max_ring_points;
        for (int pl = warp; pl < np; pl += PH_WARPS) {
            const int4 rec = pr[pl];
            T sx = 0, sy = 0;
            for (int a = rec.z + lane; a < rec.w; a += 32) {
                const T2 v = part[a];
                sx += v.x;
                sy += v.y;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                sx += __shfl_xor_sync(0xffffffffu, sx, o);
                sy += __shfl_xor_sync(0xffffffffu, sy, o);
            }
            if (lane == 0) {
                const T n2 = sx * sx + sy * sy;
                T2 zz = Cx<T>::make(1, 0);
                if (n2 > (T)0) {
                    const T inv = Cx<T>::rnorm(n2);
                    zz = Cx<T>::make(sx * inv, sy * inv);
                }
                const int o = rec.y * pitch + rec.x + K;
                zs[o] = zz;
                zo[o] = make_double2((double)zz.x, (double)zz.y);
                if (rec.y == 0) {
                    zs[-rec.x + K] = Cx<T>::make(zz.x, -zz.y);
                    zo[-rec.x + K] = make_double2((double)zz.x, -(double)zz.y);
                }
            }
        }
        __syncthreads();                          // phasors visible, staging buffers free
        i0 = i0n;
        ni = nin;
        np = npn;
    }
}

}  // namespace

namespace smk {

size_t phase_smem_bytes(int hb_rows, int box_pitch, int max_ring_items, int max_ring_points, int phase_prec) {
    size_t a, b, c;
    return phase_layout(hb_rows, box_pitch, max_ring_items, max_ring_points,
                        phase_prec == SM_PHASE_FP32 ? sizeof(float2) : 16, &a, &b, &c);
}

cudaError_t launch_phase(const smi::PlanDev& p, int nsub, const float2* B, const float2* M, const float* P,
                         double2* z, cudaStream_t st, int threads) {
    const size_t sm = phase_smem_bytes(p.hb_rows, p.box_pitch, p.max_ring_items, p.max_ring_points, p.phase_prec);
    cudaError_t e;
    if (p.phase_prec == SM_PHASE_FP64) {
        e = cudaFuncSetAttribute(k_phase<double, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_phase<double, 512><<<nsub, 512, sm, st>>>(p, B, M, P, z);
    } else if (p.phase_prec == SM_PHASE_FF) {
        e = cudaFuncSetAttribute(k_phase<ff, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_phase<ff, 512><<<nsub, 512, sm, st>>>(p, B, M, P, z);
    } else if (threads == 256) {
        e = cudaFuncSetAttribute(k_phase<float, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_phase<float, 256><<<nsub, 256, sm, st>>>(p, B, M, P, z);
    } else {
        e = cudaFuncSetAttribute(k_phase<float, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_phase<float, 512><<<nsub, 512, sm, st>>>(p, B, M, P, z);
    }
    return cudaGetLastError();
}

}  // namespace smk
