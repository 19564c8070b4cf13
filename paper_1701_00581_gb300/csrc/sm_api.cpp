// C ABI: workspace layout, stage entry points, the whole-burst path and the
// serving engine.  No exception crosses the ABI; every call returns a status.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <map>
#include <tuple>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "sm_plan.h"

using namespace smi;

namespace {

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

size_t spec_elem_bytes(int prec) { return prec == SM_FP32 ? 8 : 4; }

class DeviceGuard {
  public:
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&old_);
        if (old_ != dev) cudaSetDevice(dev);
        dev_ = dev;
    }
    ~DeviceGuard() {
        if (old_ != dev_) cudaSetDevice(old_);
    }

  private:
    int old_ = 0, dev_ = 0;
};

int check_lay(const sm_plan* plan, const void* ws, const sm_workspace_layout* lay) {
    if (!plan || !ws || !lay) { set_error("NULL plan, workspace or layout"); return SM_EINVAL; }
    if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0) {
        set_error("workspace must be 256-byte aligned"); return SM_EINVAL;
    }
    return SM_OK;
}

template <typename T>
T* at(void* ws, size_t off) { return reinterpret_cast<T*>(static_cast<char*>(ws) + off); }

int ret(cudaError_t e, const char* where) { return e == cudaSuccess ? SM_OK : cuda_fail(e, where); }

}  // namespace

extern "C" const char* sm_strerror(int s) {
    switch (s) {
        case SM_OK: return "ok";
        case SM_PENDING: return "pending";
        case SM_EINVAL: return "invalid argument";
        case SM_ENOMEM: return "request exceeds the memory budget";
        case SM_EBUSY: return "no free slot, retry later";
        case SM_ETIMEDOUT: return "timed out";
        case SM_ECUDA: return "CUDA error";
        case SM_ECANCELED: return "cancelled";
        case SM_ENOTFOUND: return "unknown ticket";
        default: return "unknown status";
    }
}

extern "C" const char* sm_last_error(void) { return g_last_error.c_str(); }

// Workspace sizing.  The per-chunk buffers are sized for nsub_chunk
// subfields; rec holds all subfields so the mosaic can run at the end.
extern "C" int sm_workspace_query(const sm_plan* plan, int F, int nsub_chunk, sm_workspace_layout* lay) {
    if (!plan || !lay) { set_error("NULL argument"); return SM_EINVAL; }
    const PlanDev& d = plan->dev;
    if (F < 1 || F > plan->ch.max_frames) { set_error("F out of range 1..max_frames"); return SM_EINVAL; }
    if (nsub_chunk < 1 || nsub_chunk > d.n_sub) { set_error("nsub_chunk out of range"); return SM_EINVAL; }
    const size_t n = (size_t)nsub_chunk;
    const size_t box = (size_t)d.box_rows * d.box_pitch, hb = (size_t)d.hb_rows * d.box_pitch;
    size_t o = 0;
    lay->spec = o; o += al(n * F * box * spec_elem_bytes(d.prec));
    lay->flux = o; o += al(n * F * sizeof(float));
    lay->mu = o; o += al(n * F * sizeof(float));
    lay->P = o; o += al(n * hb * sizeof(float));
    lay->M = o; o += al(n * hb * sizeof(float2));
    lay->noise = o; o += al(n * sizeof(float));
    lay->A = o; o += al(n * hb * sizeof(float));
    lay->B = o; o += al(n * d.n_tiles * (size_t)TILE_PAIRS * sizeof(float2));
    lay->z = o; o += al(n * hb * sizeof(double2));
    lay->rec = o; o += al((size_t)d.n_sub * d.N * d.N * sizeof(float));
    lay->seeing = o; o += al((size_t)(d.n_cubes + 1) * sizeof(double));
    lay->stf = o; o += al((size_t)d.N * d.N * sizeof(double));
    lay->refine = o;
    if (d.phase_iters > 0) o += al(n * d.n_tiles * (size_t)REF_SLOTS * sizeof(float2));
    lay->bytes = o;
    return SM_OK;
}

extern "C" int sm_stage_gain(const sm_plan* plan, const float* flat, const float* dark, float* gain, void* stream) {
    if (!plan || !flat || !dark || !gain) { set_error("NULL argument"); return SM_EINVAL; }
    DeviceGuard g(plan->device);
    return ret(smk::launch_gain(plan->dev, flat, dark, gain, (cudaStream_t)stream), "gain kernel");
}

extern "C" int sm_stage_calibrate(const sm_plan* plan, const void* raw, int frame_type, int F, const float* dark,
                                  const float* gain, float* out, void* stream) {
    if (!plan || !raw || !dark || !gain || !out) { set_error("NULL argument"); return SM_EINVAL; }
    if (frame_type != SM_U16 && frame_type != SM_F32) { set_error("bad frame_type"); return SM_EINVAL; }
    if (F < 1) { set_error("F must be >= 1"); return SM_EINVAL; }
    if ((const void*)out == raw) { set_error("out may not alias raw"); return SM_EINVAL; }
    DeviceGuard g(plan->device);
    return ret(smk::launch_calibrate(plan->dev, raw, frame_type, F, dark, gain, out, (cudaStream_t)stream),
               "calibrate kernel");
}

extern "C" int sm_stage_track(const sm_plan* plan, const void* frames, int frame_type, int F, int ref, int G, int S,
                              float* ref_window, double* cc, int* shifts, void* stream) {
    if (!plan || !frames || !ref_window || !cc || !shifts) { set_error("NULL argument"); return SM_EINVAL; }
    if (frame_type != SM_U16 && frame_type != SM_F32) { set_error("bad frame_type"); return SM_EINVAL; }
    if (F < 1 || ref < 0 || ref >= F) { set_error("need F >= 1 and 0 <= ref < F"); return SM_EINVAL; }
    const int W = plan->dev.W, H = plan->dev.H;
    const int x0 = (W - G) / 2, y0 = (H - G) / 2;
    if (S < 0 || S > smk::track_max_search() || G < 1 || x0 < S || y0 < S || x0 + G + S > W || y0 + G + S > H) {
        set_error("tracking window plus search range does not fit the frame (or S > 31)"); return SM_EINVAL;
    }
    DeviceGuard g(plan->device);
    return ret(smk::launch_track(plan->dev, frames, frame_type, F, ref, G, S, ref_window, cc, shifts,
                                 (cudaStream_t)stream),
               "tracking kernels");
}

extern "C" int sm_stage_shift(const sm_plan* plan, const void* frames, int frame_type, int F, const int* shifts,
                              float* out, void* stream) {
    if (!plan || !frames || !shifts || !out) { set_error("NULL argument"); return SM_EINVAL; }
    if (frame_type != SM_U16 && frame_type != SM_F32) { set_error("bad frame_type"); return SM_EINVAL; }
    if (F < 1) { set_error("F must be >= 1"); return SM_EINVAL; }
    if ((const void*)out == frames) { set_error("out may not alias frames"); return SM_EINVAL; }
    DeviceGuard g(plan->device);
    return ret(smk::launch_shift(plan->dev, frames, frame_type, F, shifts, out, (cudaStream_t)stream),
               "shift kernel");
}

extern "C" int sm_stage_spectra(const sm_plan* plan, const void* frames, int frame_type, int F, int sub0,
                                int nsub, void* ws, const sm_workspace_layout* lay, void* stream) {
    int rc = check_lay(plan, ws, lay);
    if (rc) return rc;
    if (!frames) { set_error("frames is NULL"); return SM_EINVAL; }
    if (frame_type != SM_U16 && frame_type != SM_F32) { set_error("bad frame_type"); return SM_EINVAL; }
    if (F < 1 || F > plan->ch.max_frames) { set_error("F out of range"); return SM_EINVAL; }
    if (sub0 < 0 || nsub < 1 || sub0 + nsub > plan->dev.n_sub) { set_error("subfield range"); return SM_EINVAL; }
    DeviceGuard g(plan->device);
    return ret(smk::launch_spectra(plan->dev, frames, frame_type, F, sub0, nsub, at<void>(ws, lay->spec),
                                   at<float>(ws, lay->flux), at<float>(ws, lay->mu), (cudaStream_t)stream),
               "spectra kernel");
}

extern "C" int sm_stage_stats(const sm_plan* plan, int F, int nsub, void* ws, const sm_workspace_layout* lay,
                              void* stream) {
    int rc = check_lay(plan, ws, lay);
    if (rc) return rc;
    if (F < 1 || nsub < 1 || nsub > plan->dev.n_sub) { set_error("bad F or nsub"); return SM_EINVAL; }
    DeviceGuard g(plan->device);
    return ret(smk::launch_stats(plan->dev, at<void>(ws, lay->spec), F, nsub, at<float>(ws, lay->P),
                                 at<float2>(ws, lay->M), at<float>(ws, lay->noise), (cudaStream_t)stream),
               "stats kernel");
}

extern "C" int sm_stage_amplitude(const sm_plan* plan, int nsub, const double* stf, void* ws,
                                  const sm_workspace_layout* lay, void* stream) {
    int rc = check_lay(plan, ws, lay);
    if (rc) return rc;
    if (!stf || nsub < 1 || nsub > plan->dev.n_sub) { set_error("bad stf or nsub"); return SM_EINVAL; }
    DeviceGuard g(plan->device);
    return ret(smk::launch_amplitude(plan->dev, nsub, stf, at<float>(ws, lay->P), at<float>(ws, lay->noise),
                                     at<float>(ws, lay->A), (cudaStream_t)stream),
               "amplitude kernel");
}

extern "C" int sm_stage_seeing(const sm_plan* plan, int F, int sub0, int nsub, void* ws,
                               const sm_workspace_layout* lay, void* stream) {
    int rc = check_lay(plan, ws, lay);
    if (rc) return rc;
    if (F < 2) { set_error("the spectral ratio needs F >= 2"); return SM_EINVAL; }
    if (plan->dev.n_cubes < 1) {
        set_error("no seeing cube: the stride must divide N and the image hold an N x N cube"); return SM_EINVAL;
    }
    if (sub0 < 0 || nsub < 1 || sub0 + nsub > plan->dev.n_sub) { set_error("subfield range"); return SM_EINVAL; }
    DeviceGuard g(plan->device);
    return ret(smk::launch_seeing(plan->dev, F, sub0, nsub, at<float>(ws, lay->P), at<float2>(ws, lay->M),
                                  at<float>(ws, lay->noise), at<double>(ws, lay->seeing), (cudaStream_t)stream),
               "seeing kernel");
}

extern "C" int sm_stage_seeing_stf(const sm_plan* plan, void* ws, const sm_workspace_layout* lay, void* stream) {
    int rc = check_lay(plan, ws, lay);
    if (rc) return rc;
    if (plan->dev.n_cubes < 1) {
        set_error("no seeing cube: the stride must divide N and the image hold an N x N cube"); return SM_EINVAL;
    }
    DeviceGuard g(plan->device);
    return ret(smk::launch_seeing_stf(plan->dev, at<double>(ws, lay->seeing), at<double>(ws, lay->stf),
                                      (cudaStream_t)stream),
               "seeing STF kernel");
}

extern "C" int sm_stage_bispectrum(const sm_plan* plan, int F, int nsub, void* ws,
                                   const sm_workspace_layout* lay, void* stream) {
    int rc = check_lay(plan, ws, lay);
    if (rc) return rc;
    if (F < 1 || nsub < 1 || nsub > plan->dev.n_sub) { set_error("bad F or nsub"); return SM_EINVAL; }
    DeviceGuard g(plan->device);
    if (plan->dev.photon_gain > 0.0) {
        rc = ret(smk::launch_bispectrum(plan->dev, at<void>(ws, lay->spec), F, nsub, at<float2>(ws, lay->B),
                                        (cudaStream_t)stream),
                 "bispectrum kernel");
        if (rc) return rc;
        return ret(smk::launch_unbias(plan->dev, F, nsub, at<float>(ws, lay->flux), at<float>(ws, lay->P),
                                      at<float2>(ws, lay->B), (cudaStream_t)stream),
                   "photon-noise bias kernel");
    }
    return ret(smk::launch_bispectrum(plan->dev, at<void>(ws, lay->spec), F, nsub, at<float2>(ws, lay->B),
                                      (cudaStream_t)stream),
               "bispectrum kernel");
}

extern "C" int sm_stage_phase(const sm_plan* plan, int nsub, void* ws, const sm_workspace_layout* lay,
                              void* stream) {
    int rc = check_lay(plan, ws, lay);
    if (rc) return rc;
    if (nsub < 1 || nsub > plan->dev.n_sub) { set_error("bad nsub"); return SM_EINVAL; }
    DeviceGuard g(plan->device);
    rc = ret(smk::launch_phase(plan->dev, nsub, at<float2>(ws, lay->B), at<float2>(ws, lay->M),
                               at<float>(ws, lay->P), at<double2>(ws, lay->z), (cudaStream_t)stream),
             "phase kernel");
    if (rc || plan->dev.phase_iters == 0) return rc;
    return ret(smk::launch_refine(plan->dev, nsub, at<float2>(ws, lay->B), at<float>(ws, lay->P),
                                  at<double2>(ws, lay->z), at<float2>(ws, lay->refine), (cudaStream_t)stream),
               "least-squares phase sweeps");
}

extern "C" int sm_stage_inverse(const sm_plan* plan, int F, int sub0, int nsub, void* ws,
                                const sm_workspace_layout* lay, void* stream) {
    int rc = check_lay(plan, ws, lay);
    if (rc) return rc;
    if (F < 1 || sub0 < 0 || nsub < 1 || sub0 + nsub > plan->dev.n_sub) { set_error("subfield range"); return SM_EINVAL; }
    DeviceGuard g(plan->device);
    return ret(smk::launch_inverse(plan->dev, F, sub0, nsub, at<float>(ws, lay->A), at<double2>(ws, lay->z),
                                   at<float>(ws, lay->flux), at<float>(ws, lay->mu), at<float>(ws, lay->rec),
                                   (cudaStream_t)stream),
               "inverse kernel");
}

extern "C" int sm_stage_mosaic(const sm_plan* plan, void* ws, const sm_workspace_layout* lay, float* out,
                               uint8_t* valid, void* stream) {
    int rc = check_lay(plan, ws, lay);
    if (rc) return rc;
    if (!out) { set_error("out is NULL"); return SM_EINVAL; }
    DeviceGuard g(plan->device);
    return ret(smk::launch_mosaic(plan->dev, at<float>(ws, lay->rec), out, valid, (cudaStream_t)stream),
               "mosaic kernel");
}

namespace {

// One stage launch of a whole-burst reconstruction: which stage, over which
// subfields.  The reconstruction is this list run in order on one stream.
enum StageId { ST_SPECTRA, ST_STATS, ST_SEEING, ST_SEEING_STF, ST_AMPLITUDE, ST_BISPECTRUM, ST_PHASE,
               ST_INVERSE, ST_MOSAIC };
struct StageCall {
    StageId stage;
    int s0, ns;
};

// Reported stage of each StageId (sm_result.stage_ms): the seeing estimate
// and its STF table count as one stage.
int reported_stage(StageId s) {
    static const int map[] = {0, 1, 2, 2, 3, 4, 5, 6, 7};
    return map[s];
}

// The stage sequence of sm_reconstruct.  Seeing from the burst itself
// (Sect. 3.1) when no STF is given: with one chunk the cubes are estimated
// inside it; otherwise a first pass over the chunks holding cubes estimates
// them before any modulus is formed.
std::vector<StageCall> burst_schedule(const sm_plan* plan, bool est, int nsub_chunk) {
    std::vector<StageCall> c;
    const int n = plan->dev.n_sub;
    if (est && nsub_chunk < n) {
        for (int s0 = 0; s0 < n; s0 += nsub_chunk) {
            const int ns = std::min(nsub_chunk, n - s0);
            bool cubes = false;
            for (int s = s0; s < s0 + ns; ++s) cubes |= plan->cube_of_sub[s] >= 0;
            if (!cubes) continue;
            c.push_back({ST_SPECTRA, s0, ns});
            c.push_back({ST_STATS, s0, ns});
            c.push_back({ST_SEEING, s0, ns});
        }
        c.push_back({ST_SEEING_STF, 0, 0});
    }
    for (int s0 = 0; s0 < n; s0 += nsub_chunk) {
        const int ns = std::min(nsub_chunk, n - s0);
        c.push_back({ST_SPECTRA, s0, ns});
        c.push_back({ST_STATS, s0, ns});
        if (est && nsub_chunk >= n) {
            c.push_back({ST_SEEING, s0, ns});
            c.push_back({ST_SEEING_STF, 0, 0});
        }
        c.push_back({ST_AMPLITUDE, s0, ns});
        c.push_back({ST_BISPECTRUM, s0, ns});
        c.push_back({ST_PHASE, s0, ns});
        c.push_back({ST_INVERSE, s0, ns});
    }
    c.push_back({ST_MOSAIC, 0, n});
    return c;
}

// Checks of sm_reconstruct's arguments; on success *stf_used is the STF
// table the amplitude stage reads (the workspace's own when estimated).
int reconstruct_check(const sm_plan* plan, int F, const double* stf, int nsub_chunk, void* ws,
                      const sm_workspace_layout* lay, const double** stf_used) {
    int rc = check_lay(plan, ws, lay);
    if (rc) return rc;
    const int n = plan->dev.n_sub;
    if (nsub_chunk < 1 || nsub_chunk > n) { set_error("nsub_chunk out of range"); return SM_EINVAL; }
    *stf_used = stf;
    if (stf == nullptr) {
        if (plan->dev.n_cubes < 1) {
            set_error("no STF given and no seeing cube to estimate it (the stride must divide N)");
            return SM_EINVAL;
        }
        if (F < 2) { set_error("no STF given and F < 2: the seeing estimate needs two frames"); return SM_EINVAL; }
        *stf_used = at<double>(ws, lay->stf);
    }
    return SM_OK;
}

// Run a schedule; with `marks`, marks[i] is recorded on the stream before
// call i and marks[calls.size()] after the last (timing of each call).
// The phase stage with the recursion kernel at `threads` threads a CTA (512:
// the stage path; 256: small enough to share an SM with three bispectrum
// CTAs; bitwise the same phasors).
int stage_phase_threads(const sm_plan* plan, int nsub, void* ws, const sm_workspace_layout* lay, void* stream,
                        int threads) {
    if (threads == 512 || plan->dev.phase_prec != SM_PHASE_FP32) return sm_stage_phase(plan, nsub, ws, lay, stream);
    DeviceGuard g(plan->device);
    int rc = ret(smk::launch_phase(plan->dev, nsub, at<float2>(ws, lay->B), at<float2>(ws, lay->M),
                                   at<float>(ws, lay->P), at<double2>(ws, lay->z), (cudaStream_t)stream, threads),
                 "phase kernel");
    if (rc || plan->dev.phase_iters == 0) return rc;
    return ret(smk::launch_refine(plan->dev, nsub, at<float2>(ws, lay->B), at<float>(ws, lay->P),
                                  at<double2>(ws, lay->z), at<float2>(ws, lay->refine), (cudaStream_t)stream),
               "least-squares phase sweeps");
}

int run_schedule(const sm_plan* plan, const std::vector<StageCall>& calls, const void* frames, int frame_type,
                 int F, const double* stf, void* ws, const sm_workspace_layout* lay, float* out, uint8_t* valid,
                 void* stream, const std::vector<cudaEvent_t>* marks, int phase_threads = 512) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    auto mark = [&](size_t i) -> int {
        if (!marks) return SM_OK;
        return ret(cudaEventRecordWithFlags((*marks)[i], st, cudaEventRecordExternal), "cudaEventRecordWithFlags");
    };
    int rc = SM_OK;
    for (size_t i = 0; i < calls.size(); ++i) {
        const StageCall& c = calls[i];
        if ((rc = mark(i))) return rc;
        switch (c.stage) {
        case ST_SPECTRA: rc = sm_stage_spectra(plan, frames, frame_type, F, c.s0, c.ns, ws, lay, stream); break;
        case ST_STATS: rc = sm_stage_stats(plan, F, c.ns, ws, lay, stream); break;
        case ST_SEEING: rc = sm_stage_seeing(plan, F, c.s0, c.ns, ws, lay, stream); break;
        case ST_SEEING_STF: rc = sm_stage_seeing_stf(plan, ws, lay, stream); break;
        case ST_AMPLITUDE: rc = sm_stage_amplitude(plan, c.ns, stf, ws, lay, stream); break;
        case ST_BISPECTRUM: rc = sm_stage_bispectrum(plan, F, c.ns, ws, lay, stream); break;
        case ST_PHASE: rc = stage_phase_threads(plan, c.ns, ws, lay, stream, phase_threads); break;
        case ST_INVERSE: rc = sm_stage_inverse(plan, F, c.s0, c.ns, ws, lay, stream); break;
        case ST_MOSAIC: rc = sm_stage_mosaic(plan, ws, lay, out, valid, stream); break;
        }
        if (rc) return rc;
    }
    return mark(calls.size());
}

}  // namespace

extern "C" int sm_reconstruct(const sm_plan* plan, const void* frames, int frame_type, int F,
                              const double* stf, int nsub_chunk, void* ws, const sm_workspace_layout* lay,
                              float* out, uint8_t* valid, void* stream) {
    const double* stf_used = nullptr;
    int rc = reconstruct_check(plan, F, stf, nsub_chunk, ws, lay, &stf_used);
    if (rc) return rc;
    return run_schedule(plan, burst_schedule(plan, stf == nullptr, nsub_chunk), frames, frame_type, F, stf_used,
                        ws, lay, out, valid, stream, nullptr);
}

// ============================================================================
// Serving engine
// ============================================================================
namespace {

using Clock = std::chrono::steady_clock;

// First-fit allocator over one device arena (host-side bookkeeping only).
class Arena {
  public:
    void init(char* base, size_t bytes) {
        base_ = base;
        free_.clear();
        free_[0] = bytes;
    }
    bool alloc(size_t bytes, size_t* off) {
        bytes = al(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = al(bytes);
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    char* base() const { return base_; }

  private:
    char* base_ = nullptr;
    std::map<size_t, size_t> free_;
};

struct Job {
    uint64_t ticket = 0;
    int channel = 0, F = 0, slot = -1;
    size_t off = 0, bytes = 0;
    float* host_out = nullptr;
    uint8_t* host_valid = nullptr;
    float* d_out = nullptr;
    uint8_t* d_valid = nullptr;
    const double* d_seeing = nullptr;     // the burst's D / mean r0 when estimated
    double* d_seeing_io = nullptr;        // its copy in the burst's own buffers (shared workspace)
    cudaEvent_t ev_start = nullptr, ev_done = nullptr;
    cudaEvent_t ev_mid = nullptr;         // pipelined: the burst's front half done
    const std::vector<cudaEvent_t>* marks = nullptr;   // the burst graph's stage marks
    const std::vector<int>* mark_stage = nullptr;
    const std::vector<cudaEvent_t>* marks2 = nullptr;  // pipelined: the back half's marks
    const std::vector<int>* mark_stage2 = nullptr;
    const std::vector<cudaEvent_t>* marks3 = nullptr;  // pipelined: the bispectrum's marks
    const std::vector<int>* mark_stage3 = nullptr;
    cudaEvent_t ev_bis = nullptr;         // pipelined: the burst's bispectrum done
    // pipelined: the back half is launched later (next submit or poll)
    bool back_pending = false;
    sm_burst bcopy{};
    const void* d_frames = nullptr;
    const double* d_stf = nullptr;
    void* ws = nullptr;
    sm_workspace_layout lay{};
    int wsi = 0;
    bool staged = false;                  // the mosaic went to the slot's pinned staging, not to out
    const sm_batch* batch = nullptr;      // batched mode: the batch object the burst ran in
    double t_submit = 0.0;
    int status = SM_PENDING;
};

}  // namespace

struct sm_handle {
    sm_config cfg;
    std::vector<sm_channel> ch;
    std::vector<sm_plan*> plans;
    std::vector<int> chunk;               // subfields per chunk, per channel
    std::vector<cudaStream_t> streams;
    std::vector<bool> stream_busy;
    std::vector<double*> stf_pinned;      // per slot: pinned host staging of the STF table
    Arena arena;
    void* dmem = nullptr;
    std::mutex mu;
    std::map<uint64_t, Job> jobs;
    uint64_t next_ticket = 1;
    Clock::time_point t0;
    // Instantiated launch graphs of whole bursts, keyed by (channel, F,
    // arena offset, stream slot): every pointer a burst's kernels take is
    // fixed by that key, so a burst that lands where an earlier one did
    // replays its graph instead of issuing the launches again.
    struct Graph {
        cudaGraphExec_t exec = nullptr;
        std::vector<cudaEvent_t> marks;   // recorded before each stage call and after the last
        std::vector<int> stage;           // reported stage of each call
    };
    std::map<std::tuple<int, int, size_t, int>, Graph> graphs;
    std::map<std::vector<size_t>, Graph> bgraphs;     // batched mode: by composition and placement
    // Device order of the bursts' kernels (overlap_kernels == 0): re-recorded
    // on the launching stream after every burst, and waited on by the next
    // burst's stream before its graph, under launch_mu so that the wait,
    // the launch and the record of one burst are not interleaved with
    // another's.
    cudaEvent_t order = nullptr;
    bool ordered = false;                 // `order` has been recorded at least once
    std::mutex launch_mu;
    // With the bursts' kernels in submission order one workspace serves
    // every burst (only one burst computes at a time): it sits at the start
    // of the arena, and a burst holds only its frames, mosaic, mask, STF
    // table and seeing value.  Concurrent kernels: one workspace per burst.
    void* shared_ws = nullptr;
    size_t shared_ws_bytes = 0;
    size_t arena_bytes = 0;               // what the bursts' arena holds
    // Pipelined (overlap_kernels = 2): two workspaces, bursts alternating;
    // each burst's front half (transforms .. bispectrum) after the previous
    // burst's front half and after the back half of the burst that used the
    // workspace before; the back half (phase .. mosaic) on a high-priority
    // stream beside the next burst's front half.
    int mode = 0;
    void* ws2[2] = {nullptr, nullptr};
    cudaEvent_t ev_front = nullptr, ev_free[2] = {nullptr, nullptr};
    bool front_recorded = false, free_recorded[2] = {false, false};
    uint64_t n_launched = 0;
    uint64_t pending_back = 0;            // ticket whose back half waits for the next burst (0: none)
    // Batched (overlap_kernels = 3): one batch object per composition
    // (channel, F, frame type of each burst, in order).
    std::map<std::vector<int>, sm_batch*> batches;
    std::vector<cudaStream_t> pstreams;   // per slot, middle priority (pipelined back halves)
    std::vector<cudaStream_t> lstreams;   // per slot, lowest priority (pipelined bispectra)
    // Per slot: pinned staging for the mosaic, mask and seeing value, copied
    // back on the burst's own stream so that sm_poll need not wait for it.
    std::vector<char*> pin_out;
    size_t pin_out_bytes = 0;
    // Host-side failure injection (SM_FAULT=alloc:N at sm_open): admission
    // number fault_alloc_at (from 1) fails as if its arena allocation had.
    long long fault_alloc_at = 0;
    long long n_admitted = 0;
};

namespace {

double ms_since(const Clock::time_point& t0) {
    return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
}

// Diagnostics on stderr: SM_LOG=2 prints the phase timings of every submit.
int log_level() {
    static const int lvl = [] {
        const char* e = getenv("SM_LOG");
        return e ? atoi(e) : 0;
    }();
    return lvl;
}

// Device bytes of one burst's own buffers: frames (room for FP32), mosaic,
// mask, STF table and the seeing value.
size_t io_bytes(const sm_handle* h, int c, int F) {
    const sm_channel& ch = h->ch[c];
    const size_t fb = (size_t)F * ch.W * ch.H * 2;   // uint16 frames
    return al(fb * 2) + al((size_t)ch.W * ch.H * 4) + al((size_t)ch.W * ch.H) +
           al((size_t)ch.N * ch.N * sizeof(double)) + al(sizeof(double));
}

// Device bytes one burst of channel c takes from the arena: its own buffers,
// plus its workspace unless the engine shares one.
size_t burst_bytes(const sm_handle* h, int c, int F, sm_workspace_layout* lay) {
    sm_workspace_query(h->plans[c], F, h->chunk[c], lay);
    return (h->shared_ws_bytes ? 0 : al(lay->bytes)) + io_bytes(h, c, F);
}

void finish_job(sm_handle* h, Job& j) {
    if (j.ev_start) cudaEventDestroy(j.ev_start);
    if (j.ev_done) cudaEventDestroy(j.ev_done);
    if (j.ev_mid) cudaEventDestroy(j.ev_mid);
    if (j.ev_bis) cudaEventDestroy(j.ev_bis);
    j.ev_start = j.ev_done = j.ev_mid = j.ev_bis = nullptr;
    if (j.bytes) h->arena.release(j.off, j.bytes);
    j.bytes = 0;
    if (j.slot >= 0) h->stream_busy[j.slot] = false;
    j.slot = -1;
}

}  // namespace

namespace {

// Launch one burst's stage sequence on its slot stream through a cached
// CUDA graph (captured on first use of the key).  The frame type and the
// STF mode (given, or estimated on the device when d_stf is NULL) are part
// of the captured kernels, so they join the key through the F slot.
// part 0: the whole schedule; pipelined: 1 the stages before the bispectrum,
// 3 the bispectrum, 2 the back half (phase .. mosaic, with the 256-thread
// phase kernel); wsi: the pipelined workspace the burst uses.
int launch_burst(sm_handle* h, const sm_burst* b, Job& j, const void* d_frames, const double* d_stf,
                 void* ws, sm_workspace_layout& lay, cudaStream_t st, int part = 0, int wsi = 0) {
    const auto key = std::make_tuple(b->channel, b->F * 4 + (d_stf ? 0 : 2) + (b->frame_type == SM_F32 ? 1 : 0),
                                     j.off, j.slot * 16 + part * 4 + wsi);
    sm_handle::Graph* g = nullptr;
    {
        std::lock_guard<std::mutex> lk(h->mu);
        auto it = h->graphs.find(key);
        if (it != h->graphs.end()) g = &it->second;
    }
    if (!g) {
        const sm_plan* plan = h->plans[b->channel];
        const double* stf_used = nullptr;
        int rc = reconstruct_check(plan, b->F, d_stf, h->chunk[b->channel], ws, &lay, &stf_used);
        if (rc) return rc;
        std::vector<StageCall> calls = burst_schedule(plan, d_stf == nullptr, h->chunk[b->channel]);
        if (part) {
            // the schedule of an unchunked burst, cut before the bispectrum
            // and before the phase
            size_t cb = 0, cp = 0;
            while (cb < calls.size() && calls[cb].stage != ST_BISPECTRUM) ++cb;
            while (cp < calls.size() && calls[cp].stage != ST_PHASE) ++cp;
            if (part == 1) calls = std::vector<StageCall>(calls.begin(), calls.begin() + cb);
            else if (part == 3) calls = std::vector<StageCall>(calls.begin() + cb, calls.begin() + cp);
            else calls = std::vector<StageCall>(calls.begin() + cp, calls.end());
        }
        sm_handle::Graph ng;
        for (const StageCall& c : calls) ng.stage.push_back(reported_stage(c.stage));
        ng.marks.assign(calls.size() + 1, nullptr);
        auto drop = [&](cudaGraph_t graph) {
            if (graph) cudaGraphDestroy(graph);
            for (auto ev : ng.marks) if (ev) cudaEventDestroy(ev);
        };
        for (auto& ev : ng.marks) {
            cudaError_t e = cudaEventCreate(&ev);
            if (e != cudaSuccess) { drop(nullptr); return cuda_fail(e, "cudaEventCreate"); }
        }
        cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) { drop(nullptr); return cuda_fail(e, "cudaStreamBeginCapture"); }
        rc = run_schedule(plan, calls, d_frames, b->frame_type, b->F, stf_used, ws, &lay, j.d_out, j.d_valid, st,
                          &ng.marks, part == 2 ? 256 : 512);
        if (rc == SM_OK && j.d_seeing_io && (part == 0 || part == 2))
            rc = ret(cudaMemcpyAsync(j.d_seeing_io, j.d_seeing, sizeof(double), cudaMemcpyDeviceToDevice, st),
                     "cudaMemcpyAsync(seeing)");
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(st, &graph);
        if (rc != SM_OK) { drop(graph); return rc; }
        if (e != cudaSuccess) { drop(graph); return cuda_fail(e, "cudaStreamEndCapture"); }
        e = cudaGraphInstantiate(&ng.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) { drop(nullptr); return cuda_fail(e, "cudaGraphInstantiate"); }
        std::lock_guard<std::mutex> lk(h->mu);
        g = &(h->graphs[key] = std::move(ng));
    }
    if (part == 2) {
        j.marks2 = &g->marks;
        j.mark_stage2 = &g->stage;
    } else if (part == 3) {
        j.marks3 = &g->marks;
        j.mark_stage3 = &g->stage;
    } else {
        j.marks = &g->marks;
        j.mark_stage = &g->stage;
    }
    return ret(cudaGraphLaunch(g->exec, st), "cudaGraphLaunch");
}

// The burst's results back to the host on its own stream: straight into the
// caller's buffers when they are page-locked host memory, otherwise into the
// slot's pinned staging, which sm_poll copies out.  The seeing value always
// goes to the staging.
int copy_back(sm_handle* h, Job& j, const sm_channel& ch, cudaStream_t st) {
    const size_t npx = (size_t)ch.W * ch.H;
    char* pin = h->pin_out[j.slot];
    auto pinned = [](const void* p) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        return a.type == cudaMemoryTypeHost;
    };
    j.staged = !pinned(j.host_out) || (j.host_valid && !pinned(j.host_valid));
    float* out = j.staged ? reinterpret_cast<float*>(pin) : j.host_out;
    uint8_t* valid = j.staged ? reinterpret_cast<uint8_t*>(pin + al(npx * 4)) : j.host_valid;
    cudaError_t e = cudaMemcpyAsync(out, j.d_out, npx * sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && j.host_valid) e = cudaMemcpyAsync(valid, j.d_valid, npx, cudaMemcpyDeviceToHost, st);
    double* sv = reinterpret_cast<double*>(pin + al(npx * 4) + al(npx));
    *sv = 0.0;
    if (e == cudaSuccess && j.d_seeing)
        e = cudaMemcpyAsync(sv, j.d_seeing_io ? j.d_seeing_io : j.d_seeing, sizeof(double), cudaMemcpyDeviceToHost, st);
    return ret(e, "copying the mosaic back");
}

// A pipelined burst's back half (phase .. mosaic and the copies back) on its
// slot's middle-priority stream, after its bispectrum and after `after` (the
// next burst's stages before the bispectrum, so that the spectra kernel,
// which takes whole SMs, does not wait for phase CTAs; or nullptr).  The
// caller holds launch_mu but not mu.
int launch_back(sm_handle* h, Job& j, cudaEvent_t after) {
    cudaStream_t ph = h->pstreams[j.slot];
    j.back_pending = false;
    cudaError_t e = cudaStreamWaitEvent(ph, j.ev_bis, 0);
    if (e == cudaSuccess && after) e = cudaStreamWaitEvent(ph, after, 0);
    if (e != cudaSuccess) return cuda_fail(e, "ordering burst");
    int rc = launch_burst(h, &j.bcopy, j, j.d_frames, j.d_stf, j.ws, j.lay, ph, 2, j.wsi);
    if (rc == SM_OK) {
        e = cudaEventRecord(h->ev_free[j.wsi], ph);
        h->free_recorded[j.wsi] = e == cudaSuccess;
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaEventRecord");
    }
    if (rc == SM_OK) rc = copy_back(h, j, h->ch[j.channel], ph);
    if (rc == SM_OK) rc = ret(cudaEventRecord(j.ev_done, ph), "cudaEventRecord");
    return rc;
}

}  // namespace

extern "C" int sm_open(const sm_config* cfg, sm_handle** out) {
    if (!cfg || !out || cfg->n_channels < 1 || !cfg->ch || cfg->max_inflight < 1) {
        set_error("bad sm_config"); return SM_EINVAL;
    }
    if ((cfg->dev_alloc == nullptr) != (cfg->dev_free == nullptr)) {
        set_error("dev_alloc and dev_free must be given together"); return SM_EINVAL;
    }
    *out = nullptr;
    sm_handle* h = new (std::nothrow) sm_handle();
    if (!h) { set_error("host allocation failed"); return SM_ENOMEM; }
    h->cfg = *cfg;
    if (const char* f = getenv("SM_FAULT")) {
        long long n = 0;
        if (sscanf(f, "alloc:%lld", &n) == 1 && n > 0) h->fault_alloc_at = n;
    }
    h->ch.assign(cfg->ch, cfg->ch + cfg->n_channels);
    h->cfg.ch = h->ch.data();
    h->t0 = Clock::now();
    DeviceGuard g(cfg->device);
    for (int c = 0; c < cfg->n_channels; ++c) {
        sm_plan* p = nullptr;
        int rc = sm_plan_create(&h->ch[c], cfg->device, &p);
        if (rc) { for (auto* q : h->plans) sm_plan_destroy(q); delete h; return rc; }
        h->plans.push_back(p);
    }
    // chunk: all subfields if the channel's workspace fits, otherwise the
    // largest count that does.  Concurrent kernels: each burst's workspace
    // and buffers in an equal share of the budget.  In order: one shared
    // workspace beside max_inflight bursts' own buffers.
    if (cfg->overlap_kernels < 0 || cfg->overlap_kernels > 3) {
        for (auto* q : h->plans) sm_plan_destroy(q);
        delete h;
        set_error("overlap_kernels must be 0, 1, 2 or 3");
        return SM_EINVAL;
    }
    h->mode = cfg->overlap_kernels;
    const bool shared = h->mode == 0 || h->mode == 2;
    size_t io_max = 0;
    for (int c = 0; c < cfg->n_channels; ++c) io_max = std::max(io_max, io_bytes(h, c, h->ch[c].max_frames));
    const size_t io_all = io_max * (size_t)cfg->max_inflight;
    for (int c = 0; c < cfg->n_channels; ++c) {
        const sm_plan* p = h->plans[c];
        int lo = 1, hi = p->dev.n_sub;
        h->chunk.push_back(hi);
        sm_workspace_layout lay;
        auto fits = [&](int chunk) {
            h->chunk[c] = chunk;
            if (shared) {
                sm_workspace_query(p, h->ch[c].max_frames, chunk, &lay);
                return io_all + al(lay.bytes) <= cfg->hbm_budget_bytes;
            }
            return burst_bytes(h, c, h->ch[c].max_frames, &lay) <= cfg->hbm_budget_bytes / (size_t)cfg->max_inflight;
        };
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (fits(mid)) lo = mid; else hi = mid - 1;
        }
        h->chunk[c] = lo;
        if (h->mode == 3) {
            // a batched burst holds every subfield's workspace (one chunk)
            h->chunk[c] = p->dev.n_sub;
            if (burst_bytes(h, c, h->ch[c].max_frames, &lay) > cfg->hbm_budget_bytes) {
                for (auto* q : h->plans) sm_plan_destroy(q);
                delete h;
                set_error("batched mode: hbm_budget_bytes cannot hold one whole burst");
                return SM_ENOMEM;
            }
        } else if (h->mode == 2) {
            // two unchunked workspaces (a burst's back half reads its whole
            // workspace while the next burst's front half fills the other)
            h->chunk[c] = p->dev.n_sub;
            sm_workspace_query(p, h->ch[c].max_frames, p->dev.n_sub, &lay);
            h->shared_ws_bytes = std::max(h->shared_ws_bytes, 2 * al(lay.bytes));
        } else if (shared) {
            sm_workspace_query(p, h->ch[c].max_frames, lo, &lay);
            h->shared_ws_bytes = std::max(h->shared_ws_bytes, al(lay.bytes));
        }
    }
    if (h->mode == 2 && h->shared_ws_bytes + io_all > cfg->hbm_budget_bytes) {
        for (auto* q : h->plans) sm_plan_destroy(q);
        delete h;
        set_error("pipelined mode: hbm_budget_bytes cannot hold two whole-burst workspaces and the bursts' buffers");
        return SM_ENOMEM;
    }
    if (shared && h->shared_ws_bytes + io_all > cfg->hbm_budget_bytes) {
        for (auto* q : h->plans) sm_plan_destroy(q);
        delete h;
        set_error("hbm_budget_bytes cannot hold one subfield's workspace and the bursts' buffers");
        return SM_ENOMEM;
    }
    cudaError_t e = cudaSuccess;
    if (cfg->dev_alloc) {
        h->dmem = cfg->dev_alloc(cfg->hbm_budget_bytes, cfg->alloc_ctx);
        if (!h->dmem || (reinterpret_cast<uintptr_t>(h->dmem) & 255)) {
            if (h->dmem) cfg->dev_free(h->dmem, cfg->alloc_ctx);
            h->dmem = nullptr;
            for (auto* q : h->plans) sm_plan_destroy(q);
            delete h;
            set_error("dev_alloc returned NULL or a pointer not aligned to 256 bytes");
            return SM_ENOMEM;
        }
    } else {
        e = cudaMalloc(&h->dmem, cfg->hbm_budget_bytes);
    }
    if (e != cudaSuccess) {
        for (auto* q : h->plans) sm_plan_destroy(q);
        delete h;
        return cuda_fail(e, "cudaMalloc(engine arena)");
    }
    h->arena_bytes = cfg->hbm_budget_bytes - h->shared_ws_bytes;
    h->shared_ws = shared ? h->dmem : nullptr;
    if (h->mode == 2) {
        h->ws2[0] = h->dmem;
        h->ws2[1] = static_cast<char*>(h->dmem) + h->shared_ws_bytes / 2;
    }
    h->arena.init(static_cast<char*>(h->dmem) + h->shared_ws_bytes, h->arena_bytes);
    e = cudaEventCreateWithFlags(&h->order, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_front, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_free[0], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_free[1], cudaEventDisableTiming);
    if (e != cudaSuccess) { *out = h; sm_close(h); *out = nullptr; return cuda_fail(e, "cudaEventCreate"); }
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    for (const auto& c : h->ch)
        h->pin_out_bytes = std::max(h->pin_out_bytes, al((size_t)c.W * c.H * 4) + al((size_t)c.W * c.H) + 256);
    for (int i = 0; i < cfg->max_inflight; ++i) {
        cudaStream_t s;
        e = h->mode == 2 ? cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, prio_hi)
                         : cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e != cudaSuccess) { *out = h; sm_close(h); *out = nullptr; return cuda_fail(e, "cudaStreamCreate"); }
        h->streams.push_back(s);
        h->stream_busy.push_back(false);
        cudaStream_t ps, ls;
        e = cudaStreamCreateWithPriority(&ps, cudaStreamNonBlocking, (prio_hi + prio_lo) / 2);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&ls, cudaStreamNonBlocking, prio_lo);
        if (e != cudaSuccess) { *out = h; sm_close(h); *out = nullptr; return cuda_fail(e, "cudaStreamCreateWithPriority"); }
        h->pstreams.push_back(ps);
        h->lstreams.push_back(ls);
        char* po = nullptr;
        e = cudaHostAlloc((void**)&po, h->pin_out_bytes, cudaHostAllocDefault);
        if (e != cudaSuccess) { *out = h; sm_close(h); *out = nullptr; return cuda_fail(e, "cudaHostAlloc"); }
        h->pin_out.push_back(po);
        size_t nmax = 0;
        for (const auto& c : h->ch) nmax = std::max(nmax, (size_t)c.N * c.N);
        double* pin = nullptr;
        e = cudaHostAlloc((void**)&pin, nmax * sizeof(double), cudaHostAllocDefault);
        if (e != cudaSuccess) { *out = h; sm_close(h); *out = nullptr; return cuda_fail(e, "cudaHostAlloc"); }
        h->stf_pinned.push_back(pin);
    }
    *out = h;
    return SM_OK;
}

extern "C" int sm_submit_burst(sm_handle* h, const sm_burst* b, uint64_t* ticket) {
    if (!h || !b || !ticket) { set_error("NULL argument"); return SM_EINVAL; }
    if (h->mode == 3) return sm_submit_batch(h, 1, b, ticket);
    if (b->channel < 0 || b->channel >= (int)h->ch.size()) { set_error("bad channel"); return SM_EINVAL; }
    const sm_channel& ch = h->ch[b->channel];
    if (b->F < 1 || b->F > ch.max_frames || !b->frames || !b->out) { set_error("bad burst"); return SM_EINVAL; }
    if (b->frame_type != SM_U16 && b->frame_type != SM_F32) { set_error("bad frame_type"); return SM_EINVAL; }
    const bool est = !b->stf && !b->d_over_r0;     // seeing estimated on the device (Sect. 3.1)
    if (est && (h->plans[b->channel]->dev.n_cubes < 1 || b->F < 2)) {
        set_error("no stf or d_over_r0, and the seeing cannot be estimated (needs a cube and F >= 2)");
        return SM_EINVAL;
    }
    const auto t_in = Clock::now();
    std::vector<double> stf;
    if (!b->stf && !est) {
        stf.resize((size_t)ch.N * ch.N);
        int rc = sm_model_stf(&ch, b->F, b->d_over_r0, stf.data());
        if (rc) return rc;
    }
    const double t_stf = ms_since(t_in);
    const double* stf_src = b->stf ? b->stf : (est ? nullptr : stf.data());
    DeviceGuard g(h->cfg.device);
    sm_workspace_layout lay;
    const size_t need = burst_bytes(h, b->channel, b->F, &lay);
    if (need > h->arena_bytes) { set_error("burst exceeds the HBM budget"); return SM_ENOMEM; }

    Job j;
    {
        std::lock_guard<std::mutex> lk(h->mu);
        if (h->fault_alloc_at > 0 && ++h->n_admitted == h->fault_alloc_at) {
            // injected allocation failure: the burst gets a ticket that
            // reports SM_ENOMEM, nothing is queued, no slot or budget is held
            j.ticket = h->next_ticket++;
            j.channel = b->channel;
            j.F = b->F;
            j.status = SM_ENOMEM;
            j.t_submit = ms_since(h->t0);
            *ticket = j.ticket;
            h->jobs[j.ticket] = j;
            return SM_OK;
        }
        int slot = -1;
        for (size_t i = 0; i < h->streams.size(); ++i)
            if (!h->stream_busy[i]) { slot = (int)i; break; }
        if (slot < 0) { set_error("all in-flight slots busy"); return SM_EBUSY; }
        size_t off = 0;
        if (!h->arena.alloc(need, &off)) { set_error("budget full"); return SM_EBUSY; }
        h->stream_busy[slot] = true;
        j.slot = slot;
        j.off = off;
        j.bytes = need;
        j.ticket = h->next_ticket++;
    }
    cudaStream_t st = h->streams[j.slot];
    char* base = h->arena.base() + j.off;
    void* ws = h->shared_ws ? h->shared_ws : base;       // pipelined: chosen at launch
    const size_t fbytes = (size_t)b->F * ch.W * ch.H * (b->frame_type == SM_U16 ? 2 : 4);
    char* d_frames = h->shared_ws ? base : base + al(lay.bytes);
    j.d_out = reinterpret_cast<float*>(d_frames + al((size_t)b->F * ch.W * ch.H * 2 * 2));
    j.d_valid = reinterpret_cast<uint8_t*>(reinterpret_cast<char*>(j.d_out) + al((size_t)ch.W * ch.H * 4));
    double* d_stf = reinterpret_cast<double*>(reinterpret_cast<char*>(j.d_valid) + al((size_t)ch.W * ch.H));
    j.channel = b->channel;
    j.F = b->F;
    if (est) {
        j.d_seeing = at<double>(ws, lay.seeing) + h->plans[b->channel]->dev.n_cubes;
        if (h->shared_ws) {
            // the next burst reuses the workspace before this one is polled:
            // the graph copies the value into the burst's own buffers
            j.d_seeing_io = reinterpret_cast<double*>(reinterpret_cast<char*>(d_stf) +
                                                      al((size_t)ch.N * ch.N * sizeof(double)));
        }
    }
    j.host_out = b->out;
    j.host_valid = b->valid;
    cudaError_t e = cudaEventCreate(&j.ev_start);
    if (e == cudaSuccess) e = cudaEventCreate(&j.ev_done);
    if (e == cudaSuccess) {
        if (b->frames_on_device)
            e = cudaMemcpyAsync(d_frames, b->frames, fbytes, cudaMemcpyDeviceToDevice, st);
        else
            e = cudaMemcpyAsync(d_frames, b->frames, fbytes, cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess && !est) {
        // from pinned staging: a pageable source would make the copy wait
        // behind the frame transfer and other pageable traffic
        double* pin = h->stf_pinned[j.slot];
        std::memcpy(pin, stf_src, (size_t)ch.N * ch.N * sizeof(double));
        e = cudaMemcpyAsync(d_stf, pin, (size_t)ch.N * ch.N * sizeof(double), cudaMemcpyHostToDevice, st);
    }
    const double t_copy = ms_since(t_in);
    if (e == cudaSuccess) e = cudaEventRecord(j.ev_start, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(j.ev_start);   // input staged: caller may reuse frames
    const double t_staged = ms_since(t_in);
    int rc = SM_OK;
    if (e != cudaSuccess) {
        rc = cuda_fail(e, "staging burst");
    } else if (h->mode == 2) {
        std::lock_guard<std::mutex> lk(h->launch_mu);
        const int w = (int)(h->n_launched++ & 1);
        // stages before the bispectrum on the slot's high-priority stream
        // (the spectra kernel takes whole SMs: it must not wait for phase
        // CTAs), the bispectrum on the lowest, the back half in between (its
        // CTAs are admitted first as the bispectrum's retire)
        cudaStream_t ph = h->pstreams[j.slot], lo = h->lstreams[j.slot];
        void* wsw = h->ws2[w];
        if (h->front_recorded) e = cudaStreamWaitEvent(st, h->ev_front, 0);
        if (e == cudaSuccess && h->free_recorded[w]) e = cudaStreamWaitEvent(st, h->ev_free[w], 0);
        if (e == cudaSuccess) e = cudaEventRecord(j.ev_start, st);
        if (e == cudaSuccess && !j.ev_mid) e = cudaEventCreateWithFlags(&j.ev_mid, cudaEventDisableTiming);
        if (e == cudaSuccess && !j.ev_bis) e = cudaEventCreateWithFlags(&j.ev_bis, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "ordering burst");
        } else {
            if (j.d_seeing) j.d_seeing = at<double>(wsw, lay.seeing) + h->plans[b->channel]->dev.n_cubes;
            rc = launch_burst(h, b, j, d_frames, est ? nullptr : d_stf, wsw, lay, st, 1, w);
        }
        if (rc == SM_OK) {
            e = cudaEventRecord(j.ev_mid, st);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(lo, j.ev_mid, 0);
            if (e != cudaSuccess) rc = cuda_fail(e, "ordering burst");
        }
        if (rc == SM_OK) rc = launch_burst(h, b, j, d_frames, est ? nullptr : d_stf, wsw, lay, lo, 3, w);
        if (rc == SM_OK) {
            e = cudaEventRecord(j.ev_bis, lo);
            if (e == cudaSuccess) e = cudaEventRecord(h->ev_front, lo);
            h->front_recorded = e == cudaSuccess;
            if (e != cudaSuccess) rc = cuda_fail(e, "ordering burst");
        }
        (void)ph;
        // the previous burst's back half now goes after this burst's early
        // stages; this burst's waits for the next burst (or its poll)
        if (rc == SM_OK && h->pending_back) {
            Job* pj = nullptr;
            {
                std::lock_guard<std::mutex> lk2(h->mu);
                auto it = h->jobs.find(h->pending_back);
                if (it != h->jobs.end() && it->second.back_pending) pj = &it->second;
            }
            h->pending_back = 0;
            if (pj) {
                const int brc = launch_back(h, *pj, j.ev_mid);
                if (brc != SM_OK) pj->status = brc;
            }
        }
        if (rc == SM_OK) {
            j.back_pending = true;
            j.bcopy = *b;
            j.d_frames = d_frames;
            j.d_stf = est ? nullptr : d_stf;
            j.ws = wsw;
            j.lay = lay;
            j.wsi = w;
            h->pending_back = j.ticket;
        }
    } else {
        std::lock_guard<std::mutex> lk(h->launch_mu);
        if (!h->cfg.overlap_kernels && h->ordered) {
            // queue behind the previous burst's kernels; ev_start is taken
            // again after the wait so that gpu_ms counts this burst's own
            // kernels only
            e = cudaStreamWaitEvent(st, h->order, 0);
            if (e == cudaSuccess) e = cudaEventRecord(j.ev_start, st);
        }
        if (e != cudaSuccess) rc = cuda_fail(e, "ordering burst");
        else rc = launch_burst(h, b, j, d_frames, est ? nullptr : d_stf, ws, lay, st);
        if (rc == SM_OK && !h->cfg.overlap_kernels) {
            // the next burst's kernels need not wait for this one's copies
            e = cudaEventRecord(h->order, st);
            h->ordered = e == cudaSuccess;
            if (e != cudaSuccess) rc = cuda_fail(e, "cudaEventRecord");
        }
        if (rc == SM_OK) rc = copy_back(h, j, ch, st);
        if (rc == SM_OK) rc = ret(cudaEventRecord(j.ev_done, st), "cudaEventRecord");
    }
    std::lock_guard<std::mutex> lk(h->mu);
    if (rc != SM_OK) {
        cudaStreamSynchronize(st);
        finish_job(h, j);
        return rc;
    }
    j.t_submit = ms_since(h->t0);
    if (log_level() >= 2)
        fprintf(stderr, "[speckle] submit ticket %llu ch %d slot %d off %zu: stf %.2f ms, copies issued %.2f ms, "
                        "staged %.2f ms, launched %.2f ms\n", (unsigned long long)j.ticket, j.channel, j.slot, j.off,
                t_stf, t_copy, t_staged, ms_since(t_in));
    *ticket = j.ticket;
    h->jobs[j.ticket] = j;
    return SM_OK;
}

// Batched mode: n bursts staged together and run as one batch.  Staging is
// the per-burst staging of sm_submit_burst (own slot stream, frames and STF
// copied in, the caller's buffers free on return); the batch then runs on
// the first burst's stream after every burst's copies, in submission order.
extern "C" int sm_submit_batch(sm_handle* h, int n, const sm_burst* bs, uint64_t* tickets) {
    if (!h || !bs || !tickets) { set_error("NULL argument"); return SM_EINVAL; }
    if (h->mode != 3) { set_error("sm_submit_batch needs an engine opened with overlap_kernels = 3"); return SM_EINVAL; }
    if (n < 1 || n > MAX_BATCH) { set_error("a batch holds 1..8 bursts"); return SM_EINVAL; }
    std::vector<sm_workspace_layout> lays(n);
    std::vector<size_t> need(n);
    std::vector<std::vector<double>> stfs(n);
    for (int i = 0; i < n; ++i) {
        const sm_burst* b = bs + i;
        if (b->channel < 0 || b->channel >= (int)h->ch.size()) { set_error("bad channel"); return SM_EINVAL; }
        const sm_channel& ch = h->ch[b->channel];
        if (b->F < 1 || b->F > ch.max_frames || !b->frames || !b->out) { set_error("bad burst"); return SM_EINVAL; }
        if (b->frame_type != SM_U16 && b->frame_type != SM_F32) { set_error("bad frame_type"); return SM_EINVAL; }
        const bool est = !b->stf && !b->d_over_r0;
        if (est && (h->plans[b->channel]->dev.n_cubes < 1 || b->F < 2)) {
            set_error("no stf or d_over_r0, and the seeing cannot be estimated (needs a cube and F >= 2)");
            return SM_EINVAL;
        }
        if (!b->stf && !est) {
            stfs[i].resize((size_t)ch.N * ch.N);
            int rc = sm_model_stf(&ch, b->F, b->d_over_r0, stfs[i].data());
            if (rc) return rc;
        }
        need[i] = burst_bytes(h, b->channel, b->F, &lays[i]);
        if (need[i] > h->arena_bytes) { set_error("burst exceeds the HBM budget"); return SM_ENOMEM; }
    }
    DeviceGuard g(h->cfg.device);
    std::vector<Job> js(n);
    {
        // all or nothing: n slots and n arena blocks, or none
        std::lock_guard<std::mutex> lk(h->mu);
        std::vector<int> slots;
        for (size_t i = 0; i < h->streams.size() && (int)slots.size() < n; ++i)
            if (!h->stream_busy[i]) slots.push_back((int)i);
        if ((int)slots.size() < n) { set_error("not enough free in-flight slots for the batch"); return SM_EBUSY; }
        std::vector<size_t> offs;
        for (int i = 0; i < n; ++i) {
            size_t off = 0;
            if (!h->arena.alloc(need[i], &off)) {
                for (int k = 0; k < i; ++k) h->arena.release(offs[k], need[k]);
                set_error("budget full");
                return SM_EBUSY;
            }
            offs.push_back(off);
        }
        for (int i = 0; i < n; ++i) {
            h->stream_busy[slots[i]] = true;
            js[i].slot = slots[i];
            js[i].off = offs[i];
            js[i].bytes = need[i];
            js[i].ticket = h->next_ticket++;
        }
    }
    std::vector<sm_batch_io> io(n);
    std::vector<const sm_plan*> plans(n);
    std::vector<int> Fs(n), fts(n), key;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        const sm_burst* b = bs + i;
        const sm_channel& ch = h->ch[b->channel];
        Job& j = js[i];
        cudaStream_t st = h->streams[j.slot];
        char* base = h->arena.base() + j.off;
        void* ws = base;
        char* d_frames = base + al(lays[i].bytes);
        const size_t fbytes = (size_t)b->F * ch.W * ch.H * (b->frame_type == SM_U16 ? 2 : 4);
        j.d_out = reinterpret_cast<float*>(d_frames + al((size_t)b->F * ch.W * ch.H * 2 * 2));
        j.d_valid = reinterpret_cast<uint8_t*>(reinterpret_cast<char*>(j.d_out) + al((size_t)ch.W * ch.H * 4));
        double* d_stf = reinterpret_cast<double*>(reinterpret_cast<char*>(j.d_valid) + al((size_t)ch.W * ch.H));
        const bool est = !b->stf && !b->d_over_r0;
        j.channel = b->channel;
        j.F = b->F;
        if (est) j.d_seeing = at<double>(ws, lays[i].seeing) + h->plans[b->channel]->dev.n_cubes;
        j.host_out = b->out;
        j.host_valid = b->valid;
        e = cudaEventCreate(&j.ev_start);
        if (e == cudaSuccess) e = cudaEventCreate(&j.ev_done);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_frames, b->frames, fbytes,
                                b->frames_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && !est) {
            double* pin = h->stf_pinned[j.slot];
            std::memcpy(pin, b->stf ? b->stf : stfs[i].data(), (size_t)ch.N * ch.N * sizeof(double));
            e = cudaMemcpyAsync(d_stf, pin, (size_t)ch.N * ch.N * sizeof(double), cudaMemcpyHostToDevice, st);
        }
        if (e == cudaSuccess) e = cudaEventRecord(j.ev_start, st);
        io[i] = sm_batch_io{d_frames, est ? nullptr : d_stf, ws, nullptr, j.d_out, j.d_valid};
        plans[i] = h->plans[b->channel];
        Fs[i] = b->F;
        fts[i] = b->frame_type;
        key.insert(key.end(), {b->channel, b->F, b->frame_type, est ? 1 : 0});
    }
    for (int i = 0; i < n; ++i) io[i].lay = &lays[i];
    for (int i = 0; i < n && e == cudaSuccess; ++i) e = cudaEventSynchronize(js[i].ev_start);   // frames reusable
    int rc = e == cudaSuccess ? SM_OK : cuda_fail(e, "staging batch");
    if (rc == SM_OK) {
        std::lock_guard<std::mutex> lk(h->launch_mu);
        cudaStream_t st = h->streams[js[0].slot];
        if (h->ordered) e = cudaStreamWaitEvent(st, h->order, 0);
        for (int i = 1; i < n && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(st, js[i].ev_start, 0);
        for (int i = 0; i < n && e == cudaSuccess; ++i) e = cudaEventRecord(js[i].ev_start, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "ordering batch");
        sm_batch* bt = nullptr;
        if (rc == SM_OK) {
            std::vector<int> ckey(key.begin(), key.end());
            for (int i = 0; i < n; ++i) ckey[4 * i + 3] = 0;       // the STF mode does not change the queue
            auto it = h->batches.find(ckey);
            if (it != h->batches.end()) {
                bt = it->second;
            } else {
                rc = sm_batch_create(n, plans.data(), Fs.data(), fts.data(), nullptr, &bt);
                if (rc == SM_OK) h->batches[ckey] = bt;
            }
        }
        // one graph per batch composition and placement (every pointer its
        // kernels take is fixed by the bursts' arena offsets)
        if (rc == SM_OK) {
            std::vector<size_t> gk(key.begin(), key.end());
            for (int i = 0; i < n; ++i) gk.push_back(js[i].off);
            gk.push_back((size_t)js[0].slot);
            sm_handle::Graph* gr = nullptr;
            {
                std::lock_guard<std::mutex> lk2(h->mu);
                auto it = h->bgraphs.find(gk);
                if (it != h->bgraphs.end()) gr = &it->second;
            }
            if (!gr) {
                sm_handle::Graph ng;
                e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
                if (e != cudaSuccess) {
                    rc = cuda_fail(e, "cudaStreamBeginCapture");
                } else {
                    rc = sm_batch_reconstruct(bt, io.data(), st);
                    cudaGraph_t graph = nullptr;
                    e = cudaStreamEndCapture(st, &graph);
                    if (rc == SM_OK && e != cudaSuccess) rc = cuda_fail(e, "cudaStreamEndCapture");
                    if (rc == SM_OK) {
                        e = cudaGraphInstantiate(&ng.exec, graph, 0);
                        if (e != cudaSuccess) rc = cuda_fail(e, "cudaGraphInstantiate");
                    }
                    if (graph) cudaGraphDestroy(graph);
                }
                if (rc == SM_OK) {
                    std::lock_guard<std::mutex> lk2(h->mu);
                    gr = &(h->bgraphs[gk] = std::move(ng));
                }
            }
            if (rc == SM_OK) rc = ret(cudaGraphLaunch(gr->exec, st), "cudaGraphLaunch");
        }
        if (rc == SM_OK) {
            e = cudaEventRecord(h->order, st);
            h->ordered = e == cudaSuccess;
            if (e != cudaSuccess) rc = cuda_fail(e, "cudaEventRecord");
        }
        for (int i = 0; i < n && rc == SM_OK; ++i) {
            js[i].batch = bt;
            rc = copy_back(h, js[i], h->ch[bs[i].channel], st);
            if (rc == SM_OK) rc = ret(cudaEventRecord(js[i].ev_done, st), "cudaEventRecord");
        }
    }
    std::lock_guard<std::mutex> lk(h->mu);
    if (rc != SM_OK) {
        for (auto& j : js) {
            if (j.slot >= 0) cudaStreamSynchronize(h->streams[j.slot]);
            finish_job(h, j);
        }
        return rc;
    }
    const double now = ms_since(h->t0);
    for (int i = 0; i < n; ++i) {
        js[i].t_submit = now;
        tickets[i] = js[i].ticket;
        h->jobs[js[i].ticket] = js[i];
    }
    return SM_OK;
}

extern "C" int sm_poll(sm_handle* h, uint64_t ticket, int timeout_ms, sm_result* res) {
    if (!h) { set_error("NULL handle"); return SM_EINVAL; }
    const auto start = Clock::now();
    if (h->mode == 2) {
        // a pipelined burst whose back half still waits for a next burst:
        // the caller wants it now
        std::lock_guard<std::mutex> lk0(h->launch_mu);
        Job* pj = nullptr;
        {
            std::lock_guard<std::mutex> lk(h->mu);
            auto it = h->jobs.find(ticket);
            if (it != h->jobs.end() && it->second.back_pending) pj = &it->second;
        }
        if (pj) {
            if (h->pending_back == ticket) h->pending_back = 0;
            DeviceGuard g(h->cfg.device);
            const int brc = launch_back(h, *pj, nullptr);
            if (brc != SM_OK) pj->status = brc;
        }
    }
    for (;;) {
        cudaEvent_t ev = nullptr;
        {
            std::lock_guard<std::mutex> lk(h->mu);
            auto it = h->jobs.find(ticket);
            if (it == h->jobs.end()) { set_error("unknown ticket"); return SM_ENOTFOUND; }
            if (it->second.status < 0) {
                // a burst that failed before it was queued reports once
                const int rc = it->second.status;
                set_error(rc == SM_ENOMEM ? "burst allocation failed (injected by SM_FAULT)" : "burst failed");
                if (res) {
                    std::memset(res, 0, sizeof(*res));
                    res->status = rc;
                    res->t_submit_ms = it->second.t_submit;
                    res->t_done_ms = ms_since(h->t0);
                }
                finish_job(h, it->second);
                h->jobs.erase(it);
                return rc;
            }
            ev = it->second.ev_done;
        }
        DeviceGuard g(h->cfg.device);
        cudaError_t q = cudaEventQuery(ev);
        if (q == cudaSuccess) break;
        if (q != cudaErrorNotReady) {
            std::lock_guard<std::mutex> lk(h->mu);
            auto it = h->jobs.find(ticket);
            int rc = cuda_fail(q, "burst execution");
            if (res) { std::memset(res, 0, sizeof(*res)); res->status = rc; }
            finish_job(h, it->second);
            h->jobs.erase(it);
            return rc;
        }
        const double waited = std::chrono::duration<double, std::milli>(Clock::now() - start).count();
        if (timeout_ms == 0 || (timeout_ms > 0 && waited >= timeout_ms)) {
            if (res) { std::memset(res, 0, sizeof(*res)); res->status = timeout_ms == 0 ? SM_PENDING : SM_ETIMEDOUT; }
            return timeout_ms == 0 ? SM_PENDING : SM_ETIMEDOUT;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(100));
    }
    std::lock_guard<std::mutex> lk(h->mu);
    auto it = h->jobs.find(ticket);
    if (it == h->jobs.end()) { set_error("unknown ticket"); return SM_ENOTFOUND; }
    Job& j = it->second;
    const double t_done = ms_since(h->t0);
    DeviceGuard g(h->cfg.device);
    const sm_channel& ch = h->ch[j.channel];
    const size_t npx = (size_t)ch.W * ch.H;
    const char* pin = h->pin_out[j.slot];
    if (j.staged) {            // the caller's buffers are pageable: from the pinned staging
        std::memcpy(j.host_out, pin, npx * sizeof(float));
        if (j.host_valid) std::memcpy(j.host_valid, pin + al(npx * 4), npx);
    }
    double dr0 = 0.0;
    if (j.d_seeing) std::memcpy(&dr0, pin + al(npx * 4) + al(npx), sizeof(double));
    float gms = 0.f;
    cudaEventElapsedTime(&gms, j.ev_start, j.ev_done);
    double stage_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int part = 0; part < 3; ++part) {
        const std::vector<cudaEvent_t>* mk = part == 0 ? j.marks : part == 1 ? j.marks2 : j.marks3;
        const std::vector<int>* ms_of = part == 0 ? j.mark_stage : part == 1 ? j.mark_stage2 : j.mark_stage3;
        if (!mk) continue;
        for (size_t i = 0; i + 1 < mk->size(); ++i) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, (*mk)[i], (*mk)[i + 1]) == cudaSuccess) stage_ms[(*ms_of)[i]] += ms;
        }
    }
    int rc = SM_OK;
    if (j.batch && sm_batch_status(j.batch) != SM_OK) rc = SM_ECUDA;
    if (res) {
        res->status = rc;
        res->t_submit_ms = j.t_submit;
        res->t_done_ms = t_done;
        res->gpu_ms = gms;
        res->bytes_admitted = j.bytes;
        res->d_over_r0 = dr0;
        for (int i = 0; i < 8; ++i) res->stage_ms[i] = stage_ms[i];
    }
    finish_job(h, j);
    h->jobs.erase(it);
    return rc;
}

extern "C" int sm_close(sm_handle* h) {
    if (!h) return SM_OK;
    DeviceGuard g(h->cfg.device);
    for (auto s : h->streams) cudaStreamSynchronize(s);
    {
        std::lock_guard<std::mutex> lk(h->mu);
        for (auto& kv : h->jobs) finish_job(h, kv.second);
        h->jobs.clear();
    }
    for (auto& kv : h->bgraphs) cudaGraphExecDestroy(kv.second.exec);
    h->bgraphs.clear();
    for (auto& kv : h->batches) sm_batch_destroy(kv.second);
    h->batches.clear();
    for (auto& kv : h->graphs) {
        cudaGraphExecDestroy(kv.second.exec);
        for (auto ev : kv.second.marks) cudaEventDestroy(ev);
    }
    h->graphs.clear();
    for (auto s : h->pstreams) cudaStreamSynchronize(s);
    for (auto s : h->lstreams) cudaStreamSynchronize(s);
    for (auto s : h->streams) cudaStreamDestroy(s);
    for (auto s : h->pstreams) cudaStreamDestroy(s);
    for (auto s : h->lstreams) cudaStreamDestroy(s);
    if (h->order) cudaEventDestroy(h->order);
    if (h->ev_front) cudaEventDestroy(h->ev_front);
    for (auto ev : h->ev_free) if (ev) cudaEventDestroy(ev);
    for (auto p : h->stf_pinned) cudaFreeHost(p);
    for (auto p : h->pin_out) cudaFreeHost(p);
    if (h->dmem) {
        if (h->cfg.dev_free) h->cfg.dev_free(h->dmem, h->cfg.alloc_ctx);
        else cudaFree(h->dmem);
    }
    for (auto* p : h->plans) sm_plan_destroy(p);
    delete h;
    return SM_OK;
}
