// Batched reconstruction: several bursts (of one or several channels) whose
// spectra and bispectra run in one persistent launch (k_batch.cu), then the
// per-burst stages.  The work queue depends only on the batch's composition
// (the channels' plans and the bursts' frame counts), so it is built on the
// host once, when the batch object is created, and reused by every run.
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "sm_plan.h"
#include "sm_tune.h"

using namespace smi;

struct sm_batch {
    int n = 0, device = 0, prec = SM_FP32, blocks_per_sm = 0;
    sm_batch_opts opts{};
    std::vector<const sm_plan*> plans;
    std::vector<int> F, frame_type, cnt_base;
    int n_cnt = 0, n_items = 0, grid = 0, max_tiles = 0;
    size_t smem = 0, scr_elems = 0;
    int4* d_items = nullptr;
    int* d_state = nullptr;             // [0] queue head, [1] status, [2..] per-subfield counters
    float2* d_scratch = nullptr;        // per-CTA [K+1][N] transform scratch
    int* h_status = nullptr;            // pinned copy of the status word
    // each burst's remaining stages run on a stream of their own, forked
    // from and joined back to the caller's stream by events
    std::vector<cudaStream_t> side;
    cudaEvent_t ev_fork = nullptr;
    std::vector<cudaEvent_t> ev_join;
};

namespace {

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

// Cost of a bispectrum tile: the CTA lasts as long as its busiest warp, which
// runs once per offset column holding a used pair of its row.
std::vector<int> tiles_by_cost(const sm_plan* pl) {
    const PlanDev& d = pl->dev;
    std::vector<int> cost(d.n_tiles, 0), order(d.n_tiles);
    for (int t = 0; t < d.n_tiles; ++t) {
        const int4 T = pl->tiles[t];
        for (int q = 0; q < VBY; ++q) {
            int cols = 0;
            for (int kk = 0; kk < VBX; ++kk) {
                bool any = false;
                for (int a = 0; a < WBY && !any; ++a)
                    for (int b = 0; b < WBX && !any; ++b)
                        any = pair_used_host(T.x + b, T.y + a, T.z + kk, T.w + q, d.r2i, d.R * d.R);
                cols += any;
            }
            cost[t] = std::max(cost[t], cols);
        }
    }
    for (int t = 0; t < d.n_tiles; ++t) order[t] = t;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    return order;
}

void release(sm_batch* bt) {
    if (!bt) return;
    if (bt->d_items) cudaFree(bt->d_items);
    if (bt->d_state) cudaFree(bt->d_state);
    if (bt->d_scratch) cudaFree(bt->d_scratch);
    if (bt->h_status) cudaFreeHost(bt->h_status);
    for (cudaStream_t st : bt->side)
        if (st) cudaStreamDestroy(st);
    if (bt->ev_fork) cudaEventDestroy(bt->ev_fork);
    for (cudaEvent_t ev : bt->ev_join)
        if (ev) cudaEventDestroy(ev);
    delete bt;
}

}  // namespace

extern "C" int sm_batch_create(int n, const sm_plan* const* plans, const int* F, const int* frame_type,
                               const sm_batch_opts* opts_in, sm_batch** out) {
    if (!out) { set_error("out is NULL"); return SM_EINVAL; }
    *out = nullptr;
    if (n < 1 || n > MAX_BATCH || !plans || !F || !frame_type) {
        set_error("a batch holds 1.." + std::to_string(MAX_BATCH) + " bursts"); return SM_EINVAL;
    }
    for (int i = 0; i < n; ++i)
        if (!plans[i]) { set_error("NULL plan"); return SM_EINVAL; }
    sm_batch_opts opts = opts_in ? *opts_in : sm_batch_opts{};
    {
        int N = 0, R = 0;
        for (int i = 0; i < n; ++i)
            if (plans[i]->dev.N > N || (plans[i]->dev.N == N && plans[i]->dev.R > R)) {
                N = plans[i]->dev.N;
                R = plans[i]->dev.R;
            }
        const smt::TuneEntry t = smt::tune_for(N, R, opts.launch);
        if (opts.lookahead == 0) opts.lookahead = t.lookahead;
        if (opts.ctas_per_sm == 0) opts.ctas_per_sm = t.ctas_per_sm;
        if (opts.launch == 0) opts.launch = t.launch;
        if (opts.tile_order == 0) opts.tile_order = t.tile_order;
    }
    if (opts.tile_order != 1 && opts.tile_order != 2) { set_error("tile_order must be 1 or 2"); return SM_EINVAL; }
    if (opts.lookahead < 1) { set_error("lookahead must be >= 1"); return SM_EINVAL; }
    if (opts.ctas_per_sm != 3 && opts.ctas_per_sm != 4) { set_error("ctas_per_sm must be 3 or 4"); return SM_EINVAL; }
    if (opts.launch < SM_BATCH_FUSED || opts.launch > SM_BATCH_GRID) {
        set_error("launch must be SM_BATCH_FUSED, SM_BATCH_TILES or SM_BATCH_GRID"); return SM_EINVAL;
    }
    const int lookahead = opts.lookahead;
    const bool fused = opts.launch == SM_BATCH_FUSED, queued = opts.launch != SM_BATCH_GRID;
    for (int i = 0; i < n; ++i) {
        const sm_plan* p = plans[i];
        if (!p) { set_error("NULL plan"); return SM_EINVAL; }
        if (p->device != plans[0]->device) { set_error("a batch runs on one device"); return SM_EINVAL; }
        if (p->dev.prec != plans[0]->dev.prec) { set_error("a batch shares one spectra precision"); return SM_EINVAL; }
        if (p->dev.acc_mode != SM_ACC_PLAIN) {
            set_error("the batched launch accumulates plain FP32 sums (acc_mode SM_ACC_PLAIN)"); return SM_EINVAL;
        }
        if (F[i] < 1 || F[i] > p->ch.max_frames) { set_error("F out of range 1..max_frames"); return SM_EINVAL; }
        if (frame_type[i] != SM_U16 && frame_type[i] != SM_F32) { set_error("bad frame_type"); return SM_EINVAL; }
    }
    sm_batch* bt = new (std::nothrow) sm_batch();
    if (!bt) { set_error("host allocation failed"); return SM_ENOMEM; }
    bt->n = n;
    bt->device = plans[0]->device;
    bt->prec = plans[0]->dev.prec;
    bt->opts = opts;
    bt->plans.assign(plans, plans + n);
    bt->F.assign(F, F + n);
    bt->frame_type.assign(frame_type, frame_type + n);
    int maxN = 0, maxK = 0;
    for (int i = 0; i < n; ++i) {
        bt->cnt_base.push_back(bt->n_cnt);
        bt->n_cnt += plans[i]->dev.n_sub;
        maxN = std::max(maxN, plans[i]->dev.N);
        maxK = std::max(maxK, plans[i]->dev.K);
        bt->smem = std::max(bt->smem, smk::batch_smem_bytes(plans[i]->dev.N, plans[i]->dev.K, bt->prec));
    }

    // The queue: subfield units (burst, subfield) in the order of their
    // relative position in their burst, so the bursts advance together; the
    // FFT items of a unit `lookahead` units ahead of its BIS items; a unit's
    // tiles costliest first.
    struct Unit { double pos; int b, s; };
    std::vector<Unit> units;
    for (int i = 0; i < n; ++i)
        for (int s = 0; s < plans[i]->dev.n_sub; ++s)
            units.push_back({(s + 0.5) / plans[i]->dev.n_sub, i, s});
    std::stable_sort(units.begin(), units.end(), [](const Unit& a, const Unit& b) { return a.pos < b.pos; });
    std::vector<std::vector<int>> order(n);
    for (int i = 0; i < n; ++i) {
        if (opts.tile_order == 2) {
            order[i] = tiles_by_cost(plans[i]);
        } else {
            order[i].resize(plans[i]->dev.n_tiles);
            for (int t = 0; t < plans[i]->dev.n_tiles; ++t) order[i][t] = t;
        }
    }
    std::vector<int4> items;
    auto ffts = [&](const Unit& u) {
        if (fused)
            for (int f = 0; f < F[u.b]; ++f) items.push_back(make_int4(0, u.b, u.s, f));
    };
    const int nu = (int)units.size();
    if (queued) {
        for (int k = 0; k < std::min(lookahead, nu); ++k) ffts(units[k]);
        for (int k = 0; k < nu; ++k) {
            for (int t : order[units[k].b]) items.push_back(make_int4(1, units[k].b, units[k].s, t));
            if (k + lookahead < nu) ffts(units[k + lookahead]);
        }
    }
    bt->n_items = (int)items.size();

    int old = 0;
    cudaGetDevice(&old);
    cudaError_t e = cudaSetDevice(bt->device);
    auto fail = [&](cudaError_t ce, const char* where) {
        release(bt);
        cudaSetDevice(old);
        return cuda_fail(ce, where);
    };
    if (e != cudaSuccess) return fail(e, "cudaSetDevice");
    int nsm = 0;
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, bt->device);
    if (e != cudaSuccess) return fail(e, "cudaDeviceGetAttribute");
    if (!fused) bt->smem = smk::batch_smem_bytes(0, 0, bt->prec);      // tiles only
    bt->blocks_per_sm = std::min(smk::batch_blocks_per_sm(bt->smem, bt->prec, opts.ctas_per_sm), opts.ctas_per_sm);
    if (bt->blocks_per_sm < 1) {
        release(bt);
        cudaSetDevice(old);
        set_error("the batched kernel does not fit on an SM");
        return SM_ECUDA;
    }
    bt->grid = nsm * bt->blocks_per_sm;
    for (int i = 0; i < n; ++i) bt->max_tiles = std::max(bt->max_tiles, plans[i]->dev.n_tiles);
    if (!queued) bt->grid = 0;             // a grid over (tile, subfield of every burst) per run
    bt->scr_elems = fused ? (size_t)(maxK + 1) * maxN : 0;
    if (!items.empty()) {
        e = cudaMalloc(&bt->d_items, items.size() * sizeof(int4));
        if (e == cudaSuccess)
            e = cudaMemcpy(bt->d_items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMalloc(&bt->d_state, (size_t)(2 + bt->n_cnt) * sizeof(int));
    if (e == cudaSuccess && fused) e = cudaMalloc(&bt->d_scratch, (size_t)bt->grid * bt->scr_elems * sizeof(float2));
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&bt->h_status, sizeof(int), cudaHostAllocDefault);
    if (e != cudaSuccess) return fail(e, "allocating the batch queue");
    *bt->h_status = 0;
    bt->side.assign(n, nullptr);
    bt->ev_join.assign(n, nullptr);
    e = cudaEventCreateWithFlags(&bt->ev_fork, cudaEventDisableTiming);
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&bt->side[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bt->ev_join[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return fail(e, "creating the batch's streams");
    cudaSetDevice(old);
    *out = bt;
    return SM_OK;
}

extern "C" int sm_batch_destroy(sm_batch* bt) {
    if (!bt) return SM_OK;
    int old = 0;
    cudaGetDevice(&old);
    cudaSetDevice(bt->device);
    release(bt);
    cudaSetDevice(old);
    return SM_OK;
}

extern "C" int sm_batch_get_opts(const sm_batch* bt, sm_batch_opts* opts) {
    if (!bt || !opts) { set_error("NULL argument"); return SM_EINVAL; }
    *opts = bt->opts;
    return SM_OK;
}

extern "C" int sm_batch_info(const sm_batch* bt, int* n_items, int* grid, size_t* device_bytes) {
    if (!bt) { set_error("NULL batch"); return SM_EINVAL; }
    if (n_items) *n_items = bt->n_items;
    if (grid) *grid = bt->grid;
    if (device_bytes)
        *device_bytes = (size_t)bt->n_items * sizeof(int4) + (size_t)(2 + bt->n_cnt) * sizeof(int) +
                        (size_t)bt->grid * bt->scr_elems * sizeof(float2);
    return SM_OK;
}

namespace {

int ret(cudaError_t e, const char* where) { return e == cudaSuccess ? SM_OK : cuda_fail(e, where); }

template <typename T>
T* at(void* ws, size_t off) { return reinterpret_cast<T*>(static_cast<char*>(ws) + off); }

}  // namespace

extern "C" int sm_batch_spectra_bispectrum(sm_batch* bt, const sm_batch_io* io, void* stream) {
    if (!bt || !io) { set_error("NULL batch or io"); return SM_EINVAL; }
    BatchArgs a;
    std::memset(&a, 0, sizeof(a));
    a.n = bt->n;
    for (int i = 0; i < bt->n; ++i) {
        const sm_plan* p = bt->plans[i];
        const sm_batch_io& b = io[i];
        if (!b.frames || !b.ws || !b.lay) { set_error("NULL frames, workspace or layout"); return SM_EINVAL; }
        if ((reinterpret_cast<uintptr_t>(b.ws) & 255) != 0) { set_error("workspace must be 256-byte aligned"); return SM_EINVAL; }
        sm_workspace_layout want;
        int rc = sm_workspace_query(p, bt->F[i], p->dev.n_sub, &want);
        if (rc) return rc;
        if (std::memcmp(&want, b.lay, sizeof(want)) != 0) {
            set_error("a batched burst needs the workspace layout of all its subfields in one chunk");
            return SM_EINVAL;
        }
        BatchBurst& d = a.b[i];
        d.p = p->dev;
        d.frames = b.frames;
        d.frame_type = bt->frame_type[i];
        d.F = bt->F[i];
        d.spec = at<void>(b.ws, b.lay->spec);
        d.flux = at<float>(b.ws, b.lay->flux);
        d.mu = at<float>(b.ws, b.lay->mu);
        d.B = at<float2>(b.ws, b.lay->B);
        d.cnt_base = bt->cnt_base[i];
        d.need = bt->opts.launch == SM_BATCH_FUSED ? bt->F[i] : 0;
    }
    int old = 0;
    cudaGetDevice(&old);
    if (old != bt->device) cudaSetDevice(bt->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = SM_OK;
    if (bt->opts.launch != SM_BATCH_FUSED)          // the transforms first, as the per-stage kernel
        for (int i = 0; i < bt->n && !rc; ++i)
            rc = sm_stage_spectra(bt->plans[i], io[i].frames, bt->frame_type[i], bt->F[i], 0,
                                  bt->plans[i]->dev.n_sub, io[i].ws, io[i].lay, stream);
    if (!rc)
        rc = ret(cudaMemsetAsync(bt->d_state, 0, (size_t)(2 + bt->n_cnt) * sizeof(int), st), "cudaMemsetAsync(batch)");
    if (!rc && bt->opts.launch == SM_BATCH_GRID) {
        // one grid per distinct plan, over all of that plan's bursts
        std::vector<bool> done(bt->n, false);
        for (int i = 0; i < bt->n && !rc; ++i) {
            if (done[i]) continue;
            BatchPtrs q;
            std::memset(&q, 0, sizeof(q));
            for (int j = i; j < bt->n; ++j)
                if (!done[j] && bt->plans[j] == bt->plans[i]) {
                    q.spec[q.n] = a.b[j].spec;
                    q.B[q.n] = a.b[j].B;
                    q.F[q.n] = a.b[j].F;
                    ++q.n;
                    done[j] = true;
                }
            rc = ret(smk::launch_batch_grid(bt->plans[i]->dev, q, st), "batched bispectrum grid");
        }
    } else if (!rc)
        rc = ret(smk::launch_batch(a, bt->prec, bt->opts.ctas_per_sm, bt->d_items, bt->n_items, bt->d_state,
                                   bt->d_state + 2, bt->d_state + 1, bt->d_scratch, bt->scr_elems, bt->grid,
                                   bt->smem, st),
                 "batched spectra and bispectrum kernel");
    // the status word goes back with the work, so a poll can read it
    if (!rc)
        rc = ret(cudaMemcpyAsync(bt->h_status, bt->d_state + 1, sizeof(int), cudaMemcpyDeviceToHost, st),
                 "cudaMemcpyAsync(batch status)");
    if (old != bt->device) cudaSetDevice(old);
    return rc;
}

extern "C" int sm_batch_status(const sm_batch* bt) {
    if (!bt) { set_error("NULL batch"); return SM_EINVAL; }
    if (*bt->h_status) {
        set_error("batched launch: a bispectrum tile gave up waiting for its subfield's spectra");
        return SM_ECUDA;
    }
    return SM_OK;
}

extern "C" int sm_batch_reconstruct(sm_batch* bt, const sm_batch_io* io, void* stream) {
    if (!bt || !io) { set_error("NULL argument"); return SM_EINVAL; }
    for (int i = 0; i < bt->n; ++i) {
        if (!io[i].stf && (bt->plans[i]->dev.n_cubes < 1 || bt->F[i] < 2)) {
            set_error("no STF given and the seeing cannot be estimated (needs a cube and F >= 2)");
            return SM_EINVAL;
        }
    }
    int rc = sm_batch_spectra_bispectrum(bt, io, stream);
    if (rc) return rc;
    // Each burst's remaining stages (statistics, seeing, modulus, phase,
    // inverse, mosaic) on its own stream, forked from the caller's stream
    // after the batched launch and joined back to it: small bursts, whose
    // phase recursion is a handful of CTAs, then run side by side.  The
    // fork and join are stream-ordered, so the whole call can be captured.
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaEventRecord(bt->ev_fork, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    int forked = 0;
    for (; forked < bt->n; ++forked) {
        e = cudaStreamWaitEvent(bt->side[forked], bt->ev_fork, 0);
        if (e != cudaSuccess) break;
    }
    for (int i = 0; i < forked && !rc; ++i) {
        const sm_plan* p = bt->plans[i];
        const sm_batch_io& b = io[i];
        void* si = bt->side[i];
        const int F = bt->F[i], n = p->dev.n_sub;
        const double* stf = b.stf;
        rc = sm_stage_stats(p, F, n, b.ws, b.lay, si);
        if (!rc && !stf) {
            rc = sm_stage_seeing(p, F, 0, n, b.ws, b.lay, si);
            if (!rc) rc = sm_stage_seeing_stf(p, b.ws, b.lay, si);
            stf = at<double>(b.ws, b.lay->stf);
        }
        if (!rc) rc = sm_stage_amplitude(p, n, stf, b.ws, b.lay, si);
        if (!rc && p->dev.photon_gain > 0.0)
            rc = ret(smk::launch_unbias(p->dev, F, n, at<float>(b.ws, b.lay->flux), at<float>(b.ws, b.lay->P),
                                        at<float2>(b.ws, b.lay->B), bt->side[i]),
                     "photon-noise bias kernel");
        if (!rc) rc = sm_stage_phase(p, n, b.ws, b.lay, si);
        if (!rc) rc = sm_stage_inverse(p, F, 0, n, b.ws, b.lay, si);
        if (!rc) rc = sm_stage_mosaic(p, b.ws, b.lay, b.out, b.valid, si);
    }
    // join every forked stream, whatever happened above
    for (int i = 0; i < forked; ++i) {
        cudaError_t j = cudaEventRecord(bt->ev_join[i], bt->side[i]);
        if (j == cudaSuccess) j = cudaStreamWaitEvent(st, bt->ev_join[i], 0);
        if (j != cudaSuccess && e == cudaSuccess) e = j;
    }
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "forking the bursts' streams");
    return SM_OK;
}
