// Plan construction: every table that depends only on the channel, built on
// the host in double precision and uploaded once.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "sm_plan.h"

namespace smi {

thread_local std::string g_last_error = "";

void set_error(const std::string& msg) { g_last_error = msg; }

int cuda_fail(cudaError_t e, const char* where) {
    set_error(std::string(where) + ": " + cudaGetErrorString(e));
    return SM_ECUDA;
}

// Sect. 2: partially overlapping subfields; ragged edge tiles keep their
// true extent, or (drop) only full tiles are kept, as in the paper's 1110
// cubes (Sect. 3.2).
static std::vector<int> tile_starts(int L, int N, int stride, bool drop) {
    int n = drop ? (L - N) / stride + 1 : (L <= N ? 1 : (int)std::ceil((double)(L - N) / stride) + 1);
    std::vector<int> s(n);
    for (int k = 0; k < n; ++k) s[k] = k * stride;
    return s;
}

// Raised-cosine ramps of `taper` px at both ends; the smaller of the two.
static double tukey_at(int x, int L, int taper) {
    if (taper <= 0) return 1.0;
    auto ramp = [&](int q) {
        return q < taper ? 0.5 * (1.0 - std::cos(M_PI * (q + 0.5) / taper)) : 1.0;
    };
    return std::min(ramp(x), ramp(L - 1 - x));
}

bool pair_used_host(int wx, int wy, int vx, int vy, int r2i, int R2) {
    const int w2 = wx * wx + wy * wy, v2 = vx * vx + vy * vy;
    const int ux = wx - vx, uy = wy - vy, u2 = ux * ux + uy * uy;
    const bool inH = wy > 0 || (wy == 0 && wx > 0);
    return inH && w2 >= 2 && w2 <= r2i && v2 > 0 && v2 <= R2 && v2 < w2 && u2 < w2;
}

int validate_channel(const sm_channel* ch) {
    if (!ch) { set_error("channel is NULL"); return SM_EINVAL; }
    if (ch->N != 64 && ch->N != 128 && ch->N != 256) {
        set_error("N must be 64, 128 or 256"); return SM_EINVAL;
    }
    if (ch->W < 1 || ch->H < 1 || ch->W > 65536 || ch->H > 65536) {
        set_error("frame size out of range"); return SM_EINVAL;
    }
    if (ch->stride < 1 || ch->stride > ch->N) { set_error("stride must be in 1..N"); return SM_EINVAL; }
    if (!(ch->fc > 0.0 && ch->fc < 0.5)) { set_error("fc must be in (0, 0.5)"); return SM_EINVAL; }
    const double r = ch->fc * ch->N;
    const int K = (int)std::floor(r);
    if (K < 2) { set_error("cutoff radius fc*N must be >= 2"); return SM_EINVAL; }
    if (ch->R < 1 || ch->R > K) { set_error("R must be in 1..floor(fc*N)"); return SM_EINVAL; }
    if (ch->R + VBX > 127) { set_error("R must be below 120 (offset tiles use byte coordinates)"); return SM_EINVAL; }
    if (ch->taper < 0 || ch->taper > ch->N / 4) { set_error("taper must be in 0..N/4"); return SM_EINVAL; }
    if (ch->spectra_prec < SM_FP32 || ch->spectra_prec > SM_BF16) {
        set_error("spectra_prec must be SM_FP32, SM_FP16 or SM_BF16"); return SM_EINVAL;
    }
    if (ch->phase_weight != SM_W_BISPEC && ch->phase_weight != SM_W_UNIT && ch->phase_weight != SM_W_SNR) {
        set_error("phase_weight must be SM_W_BISPEC, SM_W_UNIT or SM_W_SNR"); return SM_EINVAL;
    }
    if (ch->max_frames < 1 || ch->max_frames > 65535) { set_error("max_frames must be in 1..65535"); return SM_EINVAL; }
    if (ch->acc_mode != SM_ACC_PLAIN && ch->acc_mode != SM_ACC_KAHAN) {
        set_error("acc_mode must be SM_ACC_PLAIN or SM_ACC_KAHAN"); return SM_EINVAL;
    }
    if (ch->phase_iters < 0 || ch->phase_iters > 64) { set_error("phase_iters must be in 0..64"); return SM_EINVAL; }
    if (!(ch->photon_gain >= 0.0)) { set_error("photon_gain must be >= 0"); return SM_EINVAL; }
    if (ch->edge_mode != SM_EDGE_PAD && ch->edge_mode != SM_EDGE_DROP) {
        set_error("edge_mode must be SM_EDGE_PAD or SM_EDGE_DROP"); return SM_EINVAL;
    }
    if (ch->edge_mode == SM_EDGE_DROP && (ch->W < ch->N || ch->H < ch->N)) {
        set_error("SM_EDGE_DROP needs a frame of at least N x N"); return SM_EINVAL;
    }
    if (ch->mosaic_mode != SM_MOSAIC_BLEND && ch->mosaic_mode != SM_MOSAIC_CENTRAL) {
        set_error("mosaic_mode must be SM_MOSAIC_BLEND or SM_MOSAIC_CENTRAL"); return SM_EINVAL;
    }
    if (ch->mosaic_mode == SM_MOSAIC_CENTRAL && (ch->edge_mode != SM_EDGE_DROP || (ch->N - ch->stride) % 2)) {
        set_error("SM_MOSAIC_CENTRAL needs SM_EDGE_DROP and N - stride even"); return SM_EINVAL;
    }
    if (ch->phase_prec != SM_PHASE_FP32 && ch->phase_prec != SM_PHASE_FP64 && ch->phase_prec != SM_PHASE_FF) {
        set_error("phase_prec must be SM_PHASE_FP32, SM_PHASE_FP64 or SM_PHASE_FF"); return SM_EINVAL;
    }
    if (!(ch->ck >= 0.0)) { set_error("ck must be >= 0"); return SM_EINVAL; }
    if (smk::spectra_smem_bytes(ch->N, K) > 227 * 1024) {
        set_error("fc*N too large for the shared-memory FFT at this N"); return SM_EINVAL;
    }
    const int pitch = ((2 * K + 1) + 3) / 4 * 4;
    if (smk::phase_smem_bytes(K + 1, pitch, 0, 0, ch->phase_prec) > 200 * 1024) {
        set_error("phase table exceeds shared memory"); return SM_EINVAL;
    }
    return SM_OK;
}

}  // namespace smi

using namespace smi;

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

extern "C" int sm_plan_create(const sm_channel* ch, int device, sm_plan** out) {
    if (!out) { set_error("out is NULL"); return SM_EINVAL; }
    *out = nullptr;
    int rc = validate_channel(ch);
    if (rc != SM_OK) return rc;
    cudaError_t ce = cudaSetDevice(device);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaSetDevice");

    sm_plan* pl = new (std::nothrow) sm_plan();
    if (!pl) { set_error("host allocation failed"); return SM_ENOMEM; }
    pl->ch = *ch;
    pl->device = device;
    const int N = ch->N, R = ch->R;
    const double r = ch->fc * N;
    const int K = (int)std::floor(r);
    const int r2i = (int)std::floor(r * r);
    PlanDev& d = pl->dev;
    std::memset(&d, 0, sizeof(d));
    d.N = N; d.K = K; d.R = R; d.W = ch->W; d.H = ch->H; d.stride = ch->stride; d.taper = ch->taper;
    d.logN = N == 64 ? 6 : (N == 128 ? 7 : 8);
    d.r2i = r2i;
    d.prec = ch->spectra_prec; d.weight = ch->phase_weight;
    d.acc_mode = ch->acc_mode; d.phase_prec = ch->phase_prec;
    d.phase_iters = ch->phase_iters;
    d.mosaic_mode = ch->mosaic_mode;
    d.photon_gain = ch->photon_gain;
    d.box_rows = K + R + 1;
    d.box_cols = 2 * K + 1;
    d.box_pitch = (d.box_cols + 3) / 4 * 4;
    d.hb_rows = K + 1;

    // subfield grid
    const bool drop = ch->edge_mode == SM_EDGE_DROP;
    auto xs = tile_starts(ch->W, N, ch->stride, drop), ys = tile_starts(ch->H, N, ch->stride, drop);
    d.nsx = (int)xs.size(); d.nsy = (int)ys.size(); d.n_sub = d.nsx * d.nsy;
    pl->subs.resize(d.n_sub);
    std::vector<float> winx((size_t)d.n_sub * N, 0.f), winy((size_t)d.n_sub * N, 0.f);
    std::vector<double> winsum(d.n_sub);
    std::vector<float2> winft((size_t)d.n_sub * (K + 1));
    for (int j = 0; j < d.nsy; ++j)
        for (int i = 0; i < d.nsx; ++i) {
            const int s = j * d.nsx + i;
            const int w = std::min(N, ch->W - xs[i]), h = std::min(N, ch->H - ys[j]);
            pl->subs[s] = make_int4(xs[i], ys[j], w, h);
            double sx = 0, sy = 0;
            for (int x = 0; x < w; ++x) { double v = tukey_at(x, w, ch->taper); winx[(size_t)s * N + x] = (float)v; sx += v; }
            for (int y = 0; y < h; ++y) { double v = tukey_at(y, h, ch->taper); winy[(size_t)s * N + y] = (float)v; sy += v; }
            winsum[s] = sx * sy;
            for (int kx = 0; kx <= K; ++kx) {
                double re = 0, im = 0;
                for (int x = 0; x < w; ++x) {
                    const double v = tukey_at(x, w, ch->taper), a = -2.0 * M_PI * kx * x / N;
                    re += v * std::cos(a);
                    im += v * std::sin(a);
                }
                winft[(size_t)s * (K + 1) + kx] = make_float2((float)re, (float)im);
            }
        }

    // twiddles exp(-2 pi i k / N)
    std::vector<float2> tw(N);
    for (int k = 0; k < N; ++k)
        tw[k] = make_float2((float)std::cos(-2.0 * M_PI * k / N), (float)std::sin(-2.0 * M_PI * k / N));

    // diffraction OTF T0 on the half box
    const size_t hb = (size_t)d.hb_rows * d.box_pitch;
    std::vector<double> t0(hb, 0.0);
    int nU = 0;
    for (int ky = -K; ky <= K; ++ky)
        for (int kx = -K; kx <= K; ++kx) {
            const int q = kx * kx + ky * ky;
            if (q > r2i) continue;
            ++nU;
            if (ky < 0) continue;
            const double rho = std::sqrt((double)q) / r;
            t0[(size_t)ky * d.box_pitch + kx + K] =
                rho <= 1.0 ? (2.0 / M_PI) * (std::acos(rho) - rho * std::sqrt(1.0 - rho * rho)) : 0.0;
        }
    int nV = 0;
    for (int vy = -R; vy <= R; ++vy)
        for (int vx = -R; vx <= R; ++vx)
            if ((vx | vy) != 0 && vx * vx + vy * vy <= R * R) ++nV;
    pl->n_U = nU; pl->n_V = nV;

    // bispectrum tiles: every (w-block, v-block) holding a used pair
    d.n_wbx = (2 * K + 1 + WBX - 1) / WBX;
    d.n_wby = (K + 1 + WBY - 1) / WBY;
    // The difference rectangle of a tile starts at box column
    // wx0 - vx0 - (VBX - 1) + K = WBX wbx - vx0 - (VBX - 1); an odd vx0 makes it even
    // (VBX - 1 is odd), so the bispectrum kernel can stage it in 16-byte copies.
    // For even R the grid ends at column R (origin -R - (VBX - 1)), for odd R it
    // starts at -R: either way no block reaches past the offset disk on one side.
    d.v_org = (R % 2 == 0) ? -R - (VBX - 1) : -R;
    pl->n_vbx = (R - d.v_org + 1 + VBX - 1) / VBX;
    pl->n_vby = (2 * R + 1 + VBY - 1) / VBY;
    const int nwb = d.n_wbx * d.n_wby, nvb = pl->n_vbx * pl->n_vby;
    pl->tile_of.assign((size_t)nwb * nvb, -1);
    std::vector<int> wb_count(nwb, 0);
    long long npairs = 0;
    for (int wby = 0; wby < d.n_wby; ++wby)
        for (int wbx = 0; wbx < d.n_wbx; ++wbx) {
            const int wb = wby * d.n_wbx + wbx;
            const int wx0 = -K + WBX * wbx, wy0 = WBY * wby;
            for (int vby = 0; vby < pl->n_vby; ++vby)
                for (int vbx = 0; vbx < pl->n_vbx; ++vbx) {
                    const int vx0 = d.v_org + VBX * vbx, vy0 = -R + VBY * vby;
                    // used pairs of the tile, and per offset row c (one warp
                    // of the bispectrum CTA) the columns e holding one
                    long long cnt = 0;
                    unsigned mask = 0;
                    for (int a = 0; a < WBY; ++a)
                        for (int b = 0; b < WBX; ++b)
                            for (int c = 0; c < VBY; ++c)
                                for (int e = 0; e < VBX; ++e)
                                    if (pair_used_host(wx0 + b, wy0 + a, vx0 + e, vy0 + c, r2i, R * R)) {
                                        ++cnt;
                                        mask |= 1u << (8 * c + e);
                                    }
                    if (cnt == 0) continue;
                    npairs += cnt;
                    pl->tile_of[(size_t)wb * nvb + vby * pl->n_vbx + vbx] = (int)pl->tiles.size();
                    pl->tiles.push_back(make_int4(wx0, wy0, vx0, vy0));
                    pl->tile_masks.push_back(mask);
                    wb_count[wb]++;
                }
        }
    d.n_tiles = (int)pl->tiles.size();

    // seeing cubes (Sect. 3.1): non-overlapping N x N tiles from the image
    // origin, i.e. the full-size subfields whose corner lies on the N grid
    pl->cube_of_sub.assign(d.n_sub, -1);
    for (int s = 0; s < d.n_sub; ++s) {
        const int4 q = pl->subs[s];
        if (q.x % N == 0 && q.y % N == 0 && q.z == N && q.w == N) {
            pl->cube_of_sub[s] = (int)pl->cubes.size();
            pl->cubes.push_back(s);
        }
    }
    d.n_cubes = (int)pl->cubes.size();
    d.rcut = r;
    d.ck = ch->ck;
    // annuli b = nearest integer |k| over U n H: (2b - 1)^2 <= 4|k|^2 < (2b + 1)^2
    d.n_bins = K + 2;
    if (d.n_bins > smk::seeing_max_bins()) { delete pl; set_error("fc*N too large for the seeing annuli"); return SM_EINVAL; }
    {
        std::vector<std::vector<int>> ann(d.n_bins);
        for (int ky = 0; ky <= K; ++ky)
            for (int kx = -K; kx <= K; ++kx) {
                const int q = kx * kx + ky * ky;
                if (q > r2i || !(ky > 0 || (ky == 0 && kx > 0))) continue;
                int sq = (int)std::sqrt((double)(4 * q));
                while (sq * sq > 4 * q) --sq;
                while ((sq + 1) * (sq + 1) <= 4 * q) ++sq;
                ann[(sq + 1) / 2].push_back(ky * d.box_pitch + kx + K);
            }
        pl->ann_start.assign(d.n_bins + 1, 0);
        for (int b = 0; b < d.n_bins; ++b) {
            pl->ann_start[b + 1] = pl->ann_start[b] + (int)ann[b].size();
            pl->ann_idx.insert(pl->ann_idx.end(), ann[b].begin(), ann[b].end());
        }
    }
    // The bispectrum kernel stages W and U = W - V in 16-byte copies from even
    // box columns of an even-pitched box.
    for (const int4& T : pl->tiles)
        if (((T.x + K) & 1) || ((T.x - T.z - (VBX - 1) + K) & 1) || (d.box_pitch & 1)) {
            set_error("internal: bispectrum tile not on an even box column"); return SM_EINVAL;
        }
    pl->n_pairs = npairs;
    pl->wb_start.assign(nwb + 1, 0);
    for (int b = 0; b < nwb; ++b) pl->wb_start[b + 1] = pl->wb_start[b] + wb_count[b];
    pl->wb_tiles.resize(d.n_tiles);
    {
        std::vector<int> fill(pl->wb_start.begin(), pl->wb_start.end() - 1);
        for (int t = 0; t < d.n_tiles; ++t) {
            const int4 T = pl->tiles[t];
            const int wb = (T.y / WBY) * d.n_wbx + (T.x + K) / WBX;
            pl->wb_tiles[fill[wb]++] = t;
        }
    }

    // recursion schedule: points of the half-plane disk with |w|^2 >= 2,
    // rings of equal |w|^2 in ascending order
    std::vector<int2> pts;
    for (int wy = 0; wy <= K; ++wy)
        for (int wx = -K; wx <= K; ++wx) {
            const int q = wx * wx + wy * wy;
            const bool inH = wy > 0 || (wy == 0 && wx > 0);
            if (inH && q >= 2 && q <= r2i) pts.push_back(make_int2(wx, wy));
        }
    std::stable_sort(pts.begin(), pts.end(), [](const int2& a, const int2& b) {
        return a.x * a.x + a.y * a.y < b.x * b.x + b.y * b.y;
    });
    pl->points = pts;
    pl->ring_start.clear();
    for (size_t i = 0; i < pts.size(); ++i) {
        const int q = pts[i].x * pts[i].x + pts[i].y * pts[i].y;
        if (i == 0 || q != pts[i - 1].x * pts[i - 1].x + pts[i - 1].y * pts[i - 1].y)
            pl->ring_start.push_back((int)i);
    }
    pl->ring_start.push_back((int)pts.size());
    d.n_points = (int)pts.size();
    d.n_rings = (int)pl->ring_start.size() - 1;

    // recursion work items: for each point (ring order), the tiles of its
    // w-block that hold at least one pair the point reads
    pl->point_items.assign(d.n_points + 1, 0);
    pl->items.clear();
    for (int pi = 0; pi < d.n_points; ++pi) {
        const int wx = pts[pi].x, wy = pts[pi].y;
        const int wb = (wy / WBY) * d.n_wbx + (wx + K) / WBX;
        pl->point_items[pi] = (int)pl->items.size();
        for (int ti = pl->wb_start[wb]; ti < pl->wb_start[wb + 1]; ++ti) {
            const int t = pl->wb_tiles[ti];
            const int4 T = pl->tiles[t];
            unsigned mask = 0;
            for (int l = 0; l < TILE_V; ++l)
                if (pair_used_host(wx, wy, T.z + l % VBX, T.w + l / VBX, r2i, R * R)) mask |= 1u << l;
            if (!mask) continue;
            const unsigned packed = (unsigned)(wx & 255) | ((unsigned)(wy & 255) << 8) |
                                    ((unsigned)(T.z & 255) << 16) | ((unsigned)(T.w & 255) << 24);
            const int wxl = (wx + K) % WBX, wyl = wy % WBY;
            const int boff = t * TILE_PAIRS + (wyl * WBX + wxl) * TILE_V;
            pl->items.push_back(make_int4((int)packed, boff, (int)mask, 0));
        }
    }
    pl->point_items[d.n_points] = (int)pl->items.size();
    pl->ring_items.resize(d.n_rings + 1);
    d.max_ring_items = 0;
    for (int rr = 0; rr <= d.n_rings; ++rr) {
        pl->ring_items[rr] = pl->point_items[pl->ring_start[rr]];
        if (rr > 0) d.max_ring_items = std::max(d.max_ring_items, pl->ring_items[rr] - pl->ring_items[rr - 1]);
    }
    d.n_items = (int)pl->items.size();
    d.max_ring_points = 0;
    pl->point_rec.resize(d.n_points);
    for (int rr = 0; rr < d.n_rings; ++rr) {
        d.max_ring_points = std::max(d.max_ring_points, pl->ring_start[rr + 1] - pl->ring_start[rr]);
        for (int pi = pl->ring_start[rr]; pi < pl->ring_start[rr + 1]; ++pi)
            pl->point_rec[pi] = make_int4(pts[pi].x, pts[pi].y, pl->point_items[pi] - pl->ring_items[rr],
                                          pl->point_items[pi + 1] - pl->ring_items[rr]);
    }
    if (smk::phase_smem_bytes(d.hb_rows, d.box_pitch, d.max_ring_items, d.max_ring_points, d.phase_prec) >
        227 * 1024) {
        delete pl;
        set_error("phase recursion tables exceed shared memory");
        return SM_EINVAL;
    }

    // least-squares refinement: for every recursion point, the partial-sum
    // slots of the refinement's tile pass that hold one of its occurrences
    // (as w, as u = w - v or as v; lower-half occurrences conjugated), in
    // tile and slot order, so the gather sums them in a fixed order
    pl->ref_start.assign(d.n_points + 1, 0);
    if (ch->phase_iters > 0) {
        std::vector<int> pt_of((size_t)d.hb_rows * d.box_pitch, -1);
        for (int pi = 0; pi < d.n_points; ++pi) pt_of[(size_t)pts[pi].y * d.box_pitch + pts[pi].x + K] = pi;
        std::vector<std::vector<int>> lists(d.n_points);
        std::vector<char> hit(REF_SLOTS);
        auto add = [&](int t, int slot, int kx, int ky) {
            bool conj = false;
            if (!(ky > 0 || (ky == 0 && kx > 0))) { kx = -kx; ky = -ky; conj = true; }
            if (ky > K || kx < -K || kx > K) return;
            const int pi = pt_of[(size_t)ky * d.box_pitch + kx + K];
            if (pi < 0) return;                                     // anchor or outside the domain
            lists[pi].push_back((t * REF_SLOTS + slot) | (conj ? (int)0x80000000u : 0));
        };
        for (int t = 0; t < d.n_tiles; ++t) {
            const int4 T = pl->tiles[t];
            std::fill(hit.begin(), hit.end(), 0);
            for (int row = 0; row < WBY; ++row)
                for (int col = 0; col < WBX; ++col)
                    for (int q = 0; q < VBY; ++q)
                        for (int kk = 0; kk < VBX; ++kk) {
                            if (!pair_used_host(T.x + col, T.y + row, T.z + kk, T.w + q, r2i, R * R)) continue;
                            hit[row * WBX + col] = 1;
                            hit[REF_W + (row - q + VBY - 1) * (WBX + VBX - 1) + col - kk + VBX - 1] = 1;
                            hit[REF_W + REF_U + q * VBX + kk] = 1;
                        }
            for (int sl = 0; sl < REF_SLOTS; ++sl) {
                if (!hit[sl]) continue;
                if (sl < REF_W) {
                    add(t, sl, T.x + sl % WBX, T.y + sl / WBX);
                } else if (sl < REF_W + REF_U) {
                    const int c = sl - REF_W, ur = c / (WBX + VBX - 1), uc = c % (WBX + VBX - 1);
                    add(t, sl, T.x - T.z - (VBX - 1) + uc, T.y - T.w - (VBY - 1) + ur);
                } else {
                    const int c = sl - REF_W - REF_U;
                    add(t, sl, T.z + c % VBX, T.w + c / VBX);
                }
            }
        }
        for (int pi = 0; pi < d.n_points; ++pi) {
            pl->ref_start[pi + 1] = pl->ref_start[pi] + (int)lists[pi].size();
            pl->ref_idx.insert(pl->ref_idx.end(), lists[pi].begin(), lists[pi].end());
        }
    }

    // upload all tables in one allocation
    struct Piece { const void* src; size_t bytes; size_t off; };
    std::vector<Piece> pcs = {
        {pl->subs.data(), pl->subs.size() * sizeof(int4), 0},
        {winx.data(), winx.size() * sizeof(float), 0},
        {winy.data(), winy.size() * sizeof(float), 0},
        {winsum.data(), winsum.size() * sizeof(double), 0},
        {tw.data(), tw.size() * sizeof(float2), 0},
        {pl->tiles.data(), pl->tiles.size() * sizeof(int4), 0},
        {pl->ring_start.data(), pl->ring_start.size() * sizeof(int), 0},
        {pl->points.data(), pl->points.size() * sizeof(int2), 0},
        {pl->wb_start.data(), pl->wb_start.size() * sizeof(int), 0},
        {pl->wb_tiles.data(), pl->wb_tiles.size() * sizeof(int), 0},
        {t0.data(), t0.size() * sizeof(double), 0},
        {pl->items.data(), pl->items.size() * sizeof(int4), 0},
        {pl->ring_items.data(), pl->ring_items.size() * sizeof(int), 0},
        {pl->point_items.data(), pl->point_items.size() * sizeof(int), 0},
        {winft.data(), winft.size() * sizeof(float2), 0},
        {pl->point_rec.data(), pl->point_rec.size() * sizeof(int4), 0},
        {pl->cube_of_sub.data(), pl->cube_of_sub.size() * sizeof(int), 0},
        {pl->ann_start.data(), pl->ann_start.size() * sizeof(int), 0},
        {pl->ann_idx.data(), pl->ann_idx.size() * sizeof(int), 0},
        {pl->ref_start.data(), pl->ref_start.size() * sizeof(int), 0},
        {pl->ref_idx.data(), pl->ref_idx.size() * sizeof(int), 0},
        {pl->tile_masks.data(), pl->tile_masks.size() * sizeof(unsigned), 0},
    };
    size_t total = 0;
    for (auto& p : pcs) { p.off = total; total += align256(std::max<size_t>(p.bytes, 1)); }
    void* dm = nullptr;
    ce = cudaMalloc(&dm, total);
    if (ce != cudaSuccess) { delete pl; return cuda_fail(ce, "cudaMalloc(plan tables)"); }
    for (auto& p : pcs) {
        if (p.bytes == 0) continue;
        ce = cudaMemcpy((char*)dm + p.off, p.src, p.bytes, cudaMemcpyHostToDevice);
        if (ce != cudaSuccess) { cudaFree(dm); delete pl; return cuda_fail(ce, "cudaMemcpy(plan tables)"); }
    }
    pl->dmem = dm;
    auto at = [&](int i) { return (const void*)((char*)dm + pcs[i].off); };
    d.subs = (const int4*)at(0);
    d.winx = (const float*)at(1);
    d.winy = (const float*)at(2);
    d.winsum = (const double*)at(3);
    d.tw = (const float2*)at(4);
    d.tiles = (const int4*)at(5);
    d.ring_start = (const int*)at(6);
    d.points = (const int2*)at(7);
    d.wb_start = (const int*)at(8);
    d.wb_tiles = (const int*)at(9);
    d.t0 = (const double*)at(10);
    d.items = (const int4*)at(11);
    d.ring_items = (const int*)at(12);
    d.point_items = (const int*)at(13);
    d.winft = (const float2*)at(14);
    d.point_rec = (const int4*)at(15);
    d.cube_of_sub = (const int*)at(16);
    d.ann_start = (const int*)at(17);
    d.ann_idx = (const int*)at(18);
    d.ref_start = (const int*)at(19);
    d.ref_idx = (const int*)at(20);
    d.tile_masks = (const unsigned*)at(21);
    *out = pl;
    return SM_OK;
}

extern "C" int sm_plan_destroy(sm_plan* plan) {
    if (!plan) return SM_OK;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaSetDevice(plan->device);
    if (plan->dmem) cudaFree(plan->dmem);
    cudaSetDevice(dev);
    delete plan;
    return SM_OK;
}

extern "C" int sm_plan_get_info(const sm_plan* plan, sm_plan_info* info) {
    if (!plan || !info) { set_error("NULL argument"); return SM_EINVAL; }
    const PlanDev& d = plan->dev;
    info->n_sub = d.n_sub; info->nsx = d.nsx; info->nsy = d.nsy;
    info->N = d.N; info->K = d.K; info->R = d.R;
    info->box_rows = d.box_rows; info->box_cols = d.box_cols; info->box_pitch = d.box_pitch;
    info->hb_rows = d.hb_rows;
    info->n_tiles = d.n_tiles; info->tile_pairs = TILE_PAIRS;
    info->n_pairs = plan->n_pairs;
    info->n_rings = d.n_rings; info->n_points = d.n_points;
    info->n_U = plan->n_U; info->n_V = plan->n_V;
    info->n_cubes = d.n_cubes;
    return SM_OK;
}

extern "C" int sm_plan_cubes(const sm_plan* plan, int* sub_idx) {
    if (!plan || (!sub_idx && plan->dev.n_cubes > 0)) { set_error("NULL argument"); return SM_EINVAL; }
    for (int c = 0; c < plan->dev.n_cubes; ++c) sub_idx[c] = plan->cubes[c];
    return SM_OK;
}

extern "C" int sm_plan_subfields(const sm_plan* plan, int* xywh) {
    if (!plan || !xywh) { set_error("NULL argument"); return SM_EINVAL; }
    for (int s = 0; s < plan->dev.n_sub; ++s) {
        xywh[4 * s] = plan->subs[s].x; xywh[4 * s + 1] = plan->subs[s].y;
        xywh[4 * s + 2] = plan->subs[s].z; xywh[4 * s + 3] = plan->subs[s].w;
    }
    return SM_OK;
}

extern "C" int sm_plan_pair_index(const sm_plan* plan, long long n, const int* wv, long long* idx) {
    if (!plan || (n > 0 && (!wv || !idx)) || n < 0) { set_error("bad argument"); return SM_EINVAL; }
    const PlanDev& d = plan->dev;
    const int K = d.K, R = d.R, nvb = plan->n_vbx * plan->n_vby;
    for (long long i = 0; i < n; ++i) {
        const int wx = wv[4 * i], wy = wv[4 * i + 1], vx = wv[4 * i + 2], vy = wv[4 * i + 3];
        idx[i] = -1;
        if (!pair_used_host(wx, wy, vx, vy, d.r2i, R * R)) continue;
        const int wbx = (wx + K) / WBX, wby = wy / WBY;
        const int vbx = (vx - d.v_org) / VBX, vby = (vy + R) / VBY;
        const int t = plan->tile_of[(size_t)(wby * d.n_wbx + wbx) * nvb + vby * plan->n_vbx + vbx];
        if (t < 0) continue;
        const int wl = (wy - wby * WBY) * WBX + (wx + K - wbx * WBX);
        const int vl = (vy + R - vby * VBY) * VBX + (vx - d.v_org - vbx * VBX);
        idx[i] = (long long)t * TILE_PAIRS + (long long)wl * TILE_V + vl;
    }
    return SM_OK;
}

extern "C" int sm_model_stf(const sm_channel* ch, int F, const double* d_over_r0, double* stf) {
    if (!ch || !d_over_r0 || !stf || F < 1) { set_error("bad argument"); return SM_EINVAL; }
    if (!(ch->fc > 0.0) || ch->N < 2) { set_error("bad channel"); return SM_EINVAL; }
    for (int i = 0; i < F; ++i)
        if (!(d_over_r0[i] > 0.0)) { set_error("d_over_r0 must be > 0"); return SM_EINVAL; }
    const int N = ch->N;
    const double r = ch->fc * N;
    // The model depends on |k| only and vanishes with T0 outside the cutoff
    // disk, so it is evaluated once per distinct |k|^2 inside the disk.
    std::vector<double> a(F), b(F);
    for (int f = 0; f < F; ++f) {
        a[f] = 6.88 * std::pow(d_over_r0[f], 5.0 / 3.0);
        b[f] = ch->ck / (d_over_r0[f] * d_over_r0[f]);
    }
    const int qmax = (N / 2) * (N / 2) * 2;
    std::vector<double> byq(qmax + 1, -1.0);
    std::vector<double> acc((size_t)N * N, 0.0);
    for (int iy = 0; iy < N; ++iy)
        for (int ix = 0; ix < N; ++ix) {
            const int ky = iy - N / 2, kx = ix - N / 2, q = kx * kx + ky * ky;
            if (byq[q] < 0.0) {
                const double rho = std::sqrt((double)q) / r;
                double s = 0.0;
                if (rho <= 1.0) {
                    const double t0 = (2.0 / M_PI) * (std::acos(rho) - rho * std::sqrt(1.0 - rho * rho));
                    const double t = std::pow(rho, 5.0 / 3.0);
                    for (int f = 0; f < F; ++f) s += t0 * t0 * std::exp(-a[f] * t) + b[f] * t0;
                }
                byq[q] = s / F;
            }
            acc[(size_t)iy * N + ix] = byq[q];
        }
    const double c = acc[(size_t)(N / 2) * N + N / 2];
    for (size_t i = 0; i < acc.size(); ++i) stf[i] = acc[i] / c;
    return SM_OK;
}
