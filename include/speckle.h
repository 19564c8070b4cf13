/*
 * speckle.h -- C ABI of the GB300 speckle-masking reconstruction library.
 *
 * The library reconstructs one diffraction-limited image from a burst of F
 * short-exposure frames by speckle masking, subfield by subfield, as the
 * paper describes it (Li et al., "High Performance Parallel Image
 * Reconstruction for New Vacuum Solar Telescope"):
 *
 *   Sect. 2      frames are cut into partially overlapping subfields (the
 *                isoplanatic patch) that are processed independently;
 *   Sect. 2, 3.2 every subfield frame is Fourier transformed; the object's
 *                Fourier modulus comes from the mean power spectrum over
 *                the speckle transfer function (Eq. 1); its Fourier phase
 *                comes from the mean bispectrum by speckle masking;
 *   Sect. 2, 3.2 modulus and phase are transformed back and the overlapping
 *                sub-images are merged into one mosaic.
 *
 * Every step runs in hand-written CUDA kernels for sm_103a.  All entry
 * points return an int status (SM_OK = 0, SM_PENDING = 1, negative =
 * error); none throws or aborts.  Device pointers are plain CUDA device
 * addresses on the plan's / engine's device; a "stream" argument is a
 * cudaStream_t passed as void* (NULL = the legacy default stream).
 *
 * Frequency conventions used by every layout below:
 *   k = (kx, ky) in DFT bins of the N-point transform, centred in
 *   [-N/2, N/2); r = fc * N is the optics cutoff radius; K = floor(r);
 *   U = {|k| <= r}; H = upper half plane {ky > 0 or (ky == 0 and kx > 0)};
 *   V = {0 < |v| <= R}.
 */
#ifndef SPECKLE_GB300_H
#define SPECKLE_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define SM_OK         0
#define SM_PENDING    1   /* sm_poll: ticket not finished yet                */
#define SM_EINVAL    -1   /* bad argument or configuration                    */
#define SM_ENOMEM    -2   /* request larger than the memory budget            */
#define SM_EBUSY     -3   /* no free slot now; retry after a poll             */
#define SM_ETIMEDOUT -4   /* sm_poll timeout elapsed                          */
#define SM_ECUDA     -5   /* a CUDA call failed (message: sm_last_error)      */
#define SM_ECANCELED -6   /* ticket cancelled by sm_close                     */
#define SM_ENOTFOUND -7   /* unknown ticket                                   */

/* ---- enums ------------------------------------------------------------- */
#define SM_FP32 0         /* frame spectra stored as float2                   */
#define SM_FP16 1         /* frame spectra stored as half2 (scaled by 2^14)   */
#define SM_BF16 2         /* frame spectra stored as bfloat162                */

#define SM_W_BISPEC 0     /* phase terms weighted by |B| (plain phasor sum)   */
#define SM_W_UNIT   1     /* unit-modulus phase terms                         */
#define SM_W_SNR    2     /* terms weighted by |B| / (P(u) P(v) P(w)): |B|^2
                           * over the speckle-noise variance of B            */

#define SM_U16 0          /* frame samples: uint16 counts                     */
#define SM_F32 1          /* frame samples: float32                           */

#define SM_ACC_PLAIN 0    /* bispectrum sums: FP32, one rounding per frame    */
#define SM_ACC_KAHAN 1    /* bispectrum sums: FP32, blocked compensated: each
                           * group of 8 frames summed plainly, the group sums
                           * added with Kahan compensation; each subfield
                           * streams its frames twice (half of the offsets
                           * per pass)                                        */

#define SM_EDGE_PAD  0     /* ragged last subfields kept, zero-padded to N     */
#define SM_EDGE_DROP 1     /* full N x N subfields only (the paper's layout)   */

#define SM_MOSAIC_BLEND   0 /* out = sum rec / sum window, valid where >= 0.25 */
#define SM_MOSAIC_CENTRAL 1 /* each pixel from the central stride x stride block
                             * of one sub-image (the paper's 2368 x 1920 mosaic
                             * from 1110 cubes at stride 64); needs
                             * SM_EDGE_DROP and N - stride even               */

#define SM_PHASE_FP32 0   /* phase recursion arithmetic FP32, phasors stored FP64 */
#define SM_PHASE_FP64 1   /* phase recursion arithmetic FP64 throughout       */
#define SM_PHASE_FF   2   /* phase recursion arithmetic float-float (about 48
                           * significant bits) on the FP32 pipe               */

/* ---- one camera channel ------------------------------------------------ */
typedef struct {
    int    W, H;          /* frame size in px (Table 1: 2560x2160, 1024x1024)  */
    int    N;             /* subfield size = DFT size: 64, 128 or 256          */
    int    stride;        /* subfield step in px (N/2 = 50 % overlap)          */
    int    R;             /* bispectrum offset radius, DFT bins, 1 <= R <= K   */
    double fc;            /* optics cutoff in cycles/px (0 < fc < 0.5)         */
    int    taper;         /* apodisation ramp width in px (0 = none, <= N/4)   */
    int    spectra_prec;  /* SM_FP32 / SM_FP16 / SM_BF16                       */
    int    phase_weight;  /* SM_W_BISPEC / SM_W_UNIT                           */
    double ck;            /* Korff constant of the model STF (e.g. 0.435)      */
    int    max_frames;    /* largest burst length F accepted (>= 1)            */
    int    acc_mode;      /* SM_ACC_PLAIN / SM_ACC_KAHAN                       */
    int    phase_prec;    /* SM_PHASE_FP32 / SM_PHASE_FP64 / SM_PHASE_FF       */
    int    phase_iters;   /* least-squares sweeps after the recursion (0..64);
                           * see sm_stage_phase                               */
    int    edge_mode;     /* SM_EDGE_PAD / SM_EDGE_DROP                        */
    int    mosaic_mode;   /* SM_MOSAIC_BLEND / SM_MOSAIC_CENTRAL               */
    double photon_gain;   /* photons per frame count; > 0 removes the photon-
                           * noise bias from the bispectrum (see
                           * sm_stage_bispectrum), 0 = off                   */
} sm_channel;

/* ======================================================================== *
 *  Plan: everything that depends only on the channel (subfield grid, pair  *
 *  tiles, recursion schedule, twiddles, windows), built once on the host   *
 *  and uploaded to the device.                                             *
 * ======================================================================== */
typedef struct sm_plan sm_plan;

typedef struct {
    int    n_sub;          /* subfields per frame (Sect. 2 division)           */
    int    nsx, nsy;       /* subfield grid, row-major: s = j * nsx + i        */
    int    N, K, R;        /* DFT size, floor(fc*N), offset radius             */
    int    box_rows;       /* spectrum box rows: ky = -R .. K                  */
    int    box_cols;       /* 2K+1 columns: kx = -K .. K                       */
    int    box_pitch;      /* row pitch of every box, elements                 */
    int    hb_rows;        /* half box rows: ky = 0 .. K (pitch box_pitch)     */
    int    n_tiles;        /* bispectrum tiles per subfield                    */
    int    tile_pairs;     /* (w, v) slots per tile                            */
    long long n_pairs;     /* used (w, v) pairs per subfield                   */
    int    n_rings;        /* recursion rings (|w|^2 >= 2)                     */
    int    n_points;       /* recursion points in H with |w|^2 >= 2            */
    int    n_U;            /* |U|                                              */
    int    n_V;            /* |V|                                              */
    int    n_cubes;        /* seeing cubes: full-size subfields on the N grid  */
} sm_plan_info;

/* Build a plan on `device`.  Validates every field of *ch (SM_EINVAL). */
int sm_plan_create(const sm_channel* ch, int device, sm_plan** out);
int sm_plan_destroy(sm_plan* plan);
int sm_plan_get_info(const sm_plan* plan, sm_plan_info* info);
/* Subfield rectangles (x0, y0, w, h) in host memory, [n_sub][4] ints. */
int sm_plan_subfields(const sm_plan* plan, int* xywh);

/* Seeing cubes (Sect. 3.1): the burst cut into non-overlapping N x N cubes
 * from the image origin (80 for a 2560 x 2160 burst of N = 256).  They are
 * the full-size subfields whose corner lies on the N grid, so there are
 * some only when the stride divides N.  sub_idx: host int[n_cubes] gets
 * their subfield indices, in cube order.                                    */
int sm_plan_cubes(const sm_plan* plan, int* sub_idx);

/* Position of the bispectrum value B(w - v, v) of pair (w, v) in the per-
 * subfield B buffer (units of complex values), for n host pairs given as
 * int[4] = (wx, wy, vx, vy); -1 where the pair is not stored.  Host only. */
int sm_plan_pair_index(const sm_plan* plan, long long n, const int* wv, long long* idx);

/* ======================================================================== *
 *  Workspace: one device allocation holding the per-chunk buffers of the   *
 *  stage entry points.  The caller allocates ws_bytes (256-B aligned) and  *
 *  owns it; the library never allocates on these paths.                    *
 * ======================================================================== */
typedef struct {
    /* byte offsets into the workspace of each buffer, for `nsub_chunk`
     * subfields of F frames (layouts documented per field)                  */
    size_t spec;   /* [nsub][F][box_rows][box_pitch] complex (prec-sized)    */
    size_t flux;   /* [nsub][F] float: windowed flux of each frame tile       */
    size_t mu;     /* [nsub][F] float: windowed mean of each frame tile       */
    size_t P;      /* [nsub][hb_rows][box_pitch] float: mean power (Eq. 1)    */
    size_t M;      /* [nsub][hb_rows][box_pitch] float2: mean spectrum        */
    size_t noise;  /* [nsub] float: additive-noise floor of P                 */
    size_t A;      /* [nsub][hb_rows][box_pitch] float: object modulus        */
    size_t B;      /* [nsub][n_tiles][tile_pairs] float2: mean bispectrum     */
    size_t z;      /* [nsub][hb_rows][box_pitch] double2: unit phasors        */
    size_t rec;    /* [n_sub total][N][N] float: sub-images of all subfields  */
    size_t seeing; /* [n_cubes + 1] double: D/r0 of every seeing cube, then the
                    * burst's D / mean r0                                    */
    size_t stf;    /* [N][N] double, centred: model STF at the burst's seeing */
    size_t refine; /* [nsub][n_tiles][413] float2: least-squares sweep partials
                    * (0 bytes when the channel's phase_iters is 0)         */
    size_t bytes;  /* total workspace size                                    */
} sm_workspace_layout;

/* Workspace layout for chunks of `nsub_chunk` subfields of F frames. */
int sm_workspace_query(const sm_plan* plan, int F, int nsub_chunk, sm_workspace_layout* lay);

/* ---- stage entry points (device pointers, asynchronous on `stream`) ----
 * `sub0` is the first subfield of the chunk (0 .. n_sub-1), `nsub` its
 * length (<= nsub_chunk of the layout); per-chunk buffers start at the
 * chunk's first subfield, `rec` is indexed by absolute subfield.           */

/* ---- front end (Table 2: flat/dark preprocessing), device pointers ----- */

/* Normalised detector gain g = (flat - dark) / mean(flat - dark), the mean
 * over the pixels where flat > dark (FP64, fixed order); g = 0 where
 * flat <= dark.  flat, dark, gain: device float [H][W] of the plan's frame
 * size.  Meant to run once per flat field (one CTA: about a millisecond
 * for 2560 x 2160).                                                        */
int sm_stage_gain(const sm_plan* plan, const float* flat, const float* dark, float* gain, void* stream);

/* Flat/dark-corrected frames: out = (raw - dark) / g, 0 where g = 0.  raw:
 * device [F][H][W] of frame_type; out: device float [F][H][W] (may not
 * alias raw), which sm_stage_spectra / sm_reconstruct take as SM_F32.      */
int sm_stage_calibrate(const sm_plan* plan, const void* raw, int frame_type, int F, const float* dark,
                       const float* gain, float* out, void* stream);

/* Correlation tracking (Table 2): for every frame the integer shift
 * (sx, sy), |sx|, |sy| <= S, maximising
 * C(s) = sum over the central G x G window of a(x + s) (r(x) - mean r),
 * r the frame `ref` of the burst, the first maximum in row-major (sy, sx)
 * order (products in FP32 over 32-sample chunks, summed in FP64).
 * ref_window: device float [G][G] scratch; cc: device double
 * [F][2S+1][2S+1] receives C; shifts: device int [F][2] receives (sx, sy).
 * SM_EINVAL unless 0 <= S <= 31 and the window moved by +-S fits the frame
 * ((W-G)/2 >= S, (W-G)/2 + G + S <= W, and likewise in y).                */
int sm_stage_track(const sm_plan* plan, const void* frames, int frame_type, int F, int ref, int G, int S,
                   float* ref_window, double* cc, int* shifts, void* stream);

/* Aligned frames: out_f(x, y) = a_f(x + sx_f, y + sy_f) with the
 * coordinates clamped to the frame (edges replicated).  out: device float
 * [F][H][W], not aliasing frames.                                          */
int sm_stage_shift(const sm_plan* plan, const void* frames, int frame_type, int F, const int* shifts,
                   float* out, void* stream);

/* Sect. 2: cut, apodise, mean-subtract, 2-D DFT and normalise every frame
 * tile of subfields sub0..sub0+nsub-1.  frames: device [F][H][W] samples of
 * `frame_type`.  Writes spec, flux, mu.                                     */
int sm_stage_spectra(const sm_plan* plan, const void* frames, int frame_type, int F,
                     int sub0, int nsub, void* ws, const sm_workspace_layout* lay,
                     void* stream);

/* Eq. 1 numerator: P = <|I_i|^2>, M = <I_i> over the frames on the half box;
 * noise = mean P over the half-box corners outside the cutoff.             */
int sm_stage_stats(const sm_plan* plan, int F, int nsub, void* ws,
                   const sm_workspace_layout* lay, void* stream);

/* Eq. 1: A = sqrt(max(P - noise, 0) / max(STF, 1e-4)) * T0 on U.  stf is a
 * device double [N][N] table, centred (index (ky+N/2)*N + kx+N/2).        */
int sm_stage_amplitude(const sm_plan* plan, int nsub, const double* stf, void* ws,
                       const sm_workspace_layout* lay, void* stream);

/* Sect. 3.1 (spectral ratio technique, von der Luehe 1984): D/r0 of every
 * seeing cube among subfields sub0..sub0+nsub-1 (after sm_stage_stats of
 * that chunk), into seeing[cube].  Per cube, over annuli b of unit width
 * in the half-plane domain: num_b = sum (F |M|^2 - P) / (F - 1) and
 * den_b = sum (P - noise); annuli b = 1, 2, ... are used until the first
 * with den_b <= 0 or num_b / den_b < 0.05; D/r0 = x minimises
 * sum_b (num_b/den_b - |T_LE(b/r; x)|^2 / STF(b/r; x))^2 over 256
 * log-spaced candidates in [1, 64] (Fried long-exposure OTF, the model STF
 * of sm_model_stf, both 1 at k = 0), refined by a parabola in log x; 64
 * when no annulus qualifies.  FP64.  Needs F >= 2 and a plan with cubes.   */
int sm_stage_seeing(const sm_plan* plan, int F, int sub0, int nsub, void* ws,
                    const sm_workspace_layout* lay, void* stream);

/* Sect. 3.1: the burst's seeing is the mean r0 of the cubes,
 * seeing[n_cubes] = 1 / mean_c (1 / seeing[c]), and stf gets the model STF
 * of sm_model_stf at that D/r0 (device double [N][N], centred) for
 * sm_stage_amplitude.  Every cube's seeing must be written first.          */
int sm_stage_seeing_stf(const sm_plan* plan, void* ws, const sm_workspace_layout* lay, void* stream);

/* Sect. 2, 3.2 (speckle masking): mean bispectrum
 * B(w-v, v) = (1/F) sum_i I_i(w-v) I_i(v) conj I_i(w) on every pair the
 * phase recursion reads.  With photon_gain > 0 the photon-noise bias is
 * removed (Wirnitzer 1985): B - (P(w-v) + P(v) + P(w)) <1/N> + 2 <1/N^2>,
 * N_f = photon_gain * flux_f the photon count of frame f's windowed tile,
 * from this chunk's P (sm_stage_stats first) and flux.                      */
int sm_stage_bispectrum(const sm_plan* plan, int F, int nsub, void* ws,
                        const sm_workspace_layout* lay, void* stream);

/* Sect. 3.2 (LWW recursion): unit phasors z on the half box, ring by ring
 * from the anchors z(e_x), z(e_y) = M/|M|; each point sums
 * z(w-v) z(v) conj B(w-v, v) times the channel's weighting (1, 1/|B|, or
 * 1/(P(w-v) P(v) P(w))).  With phase_iters > 0, that many least-squares
 * sweeps follow ("or iteratively"): every split w = u + v then updates all
 * three of its phases, z(k) = S_k / |S_k| with
 * S_k = sum_{w=k} g z(u) z(v) conj B + sum_{u=k} g z(w) conj z(v) B
 *     + sum_{v=k} g z(w) conj z(u) B   (g the weighting factor),
 * from the previous sweep's phases (Jacobi), anchors fixed, a point with
 * S_k = 0 keeping its phase.  The sweeps use a workspace buffer of
 * 413 complex partial sums per bispectrum tile.                             */
int sm_stage_phase(const sm_plan* plan, int nsub, void* ws,
                   const sm_workspace_layout* lay, void* stream);

/* Sect. 2: sub-image rec = Re IDFT(A z) * <flux> + <mu> * window, for
 * subfields sub0..sub0+nsub-1, into rec[sub].                              */
int sm_stage_inverse(const sm_plan* plan, int F, int sub0, int nsub, void* ws,
                     const sm_workspace_layout* lay, void* stream);

/* Sect. 3.2 merge: out = sum_s rec_s / sum_s window_s over all subfields;
 * valid = (sum window >= 0.25), out = 0 elsewhere.  With SM_MOSAIC_CENTRAL
 * each pixel inside the central stride x stride block of a subfield
 * [x0 + (N-s)/2, x0 + (N+s)/2)^2 is rec / window of that subfield, valid;
 * every other pixel 0, invalid.  out: device float [H][W]; valid: device
 * uint8 [H][W] or NULL.                                                     */
int sm_stage_mosaic(const sm_plan* plan, void* ws, const sm_workspace_layout* lay,
                    float* out, uint8_t* valid, void* stream);

/* Whole path on device data: chunks of lay->... subfields through every
 * stage, then the mosaic.  Asynchronous on `stream`.  stf: device
 * [N][N] centred table, or NULL to estimate the seeing from the burst
 * (Sect. 3.1: sm_stage_seeing on every chunk holding cubes, then
 * sm_stage_seeing_stf; when the chunks do not cover every subfield at once
 * the spectra of the cube chunks are computed twice).  SM_EINVAL when
 * stf is NULL and the plan has no cube or F < 2.                           */
int sm_reconstruct(const sm_plan* plan, const void* frames, int frame_type, int F,
                   const double* stf, int nsub_chunk, void* ws,
                   const sm_workspace_layout* lay, float* out, uint8_t* valid, void* stream);

/* Allocation-free whole path.  The paper has no counterpart: this entry
 * point exists for callers that may not allocate device memory once they
 * are running, such as a camera or telescope control loop that fixes all of
 * its device memory at start-up (an allocation can synchronise the device
 * and stall frame acquisition), or a plug-in whose host framework owns every
 * device allocation.  Same arguments and result as sm_reconstruct (stf may
 * be NULL: the seeing is then estimated from the burst, Sect. 3.1), but the
 * workspace is a fixed array of SM_NOALLOC_SCRATCH_BYTES in the library's
 * own device image (every GPU that loads the library holds it until the
 * process exits), so the call allocates nothing.  Subfields go through in
 * the largest chunks that fit; a channel whose workspace does not fit even
 * one subfield at a time gets SM_ENOMEM (the message states both sizes).
 * The first call on a device looks up the array's device address; make that
 * first call before any stream capture.  All calls share the one array:
 * calls that overlap on the GPU (other streams or threads) race, and the
 * caller must serialise them.  Nothing in the array has to start at zero:
 * every value a call reads is written earlier in the same call.            */
#define SM_NOALLOC_SCRATCH_BYTES (64u << 20)
int sm_reconstruct_noalloc(const sm_plan* plan, const void* frames, int frame_type, int F,
                           const double* stf, float* out, uint8_t* valid, void* stream);

/* ======================================================================== *
 *  Batched launch: the subfields of several bursts -- of one channel or of  *
 *  several, with subfields of different sizes -- through one persistent     *
 *  launch of the spectra (Sect. 2: the Fourier transform of every           *
 *  subimage) and the mean bispectrum (Sect. 2, 3.2: speckle masking), then  *
 *  each burst's remaining stages.  The subfields are independent (Sect. 2), *
 *  so a burst's result is bitwise the same alone or in any batch.           *
 * ======================================================================== */
typedef struct sm_batch sm_batch;

/* One burst of a batch run.  Device pointers on the batch's device. */
typedef struct {
    const void*                frames;  /* [F][H][W] of the burst's frame_type   */
    const double*              stf;     /* [N][N] centred model STF, or NULL: the
                                           seeing is estimated from the burst
                                           (Sect. 3.1, sm_stage_seeing)          */
    void*                      ws;      /* the burst's workspace, 256-B aligned   */
    const sm_workspace_layout* lay;     /* sm_workspace_query(plan, F, n_sub):
                                           every subfield in one chunk           */
    float*                     out;     /* [H][W] mosaic                          */
    uint8_t*                   valid;   /* [H][W] or NULL                         */
} sm_batch_io;

#define SM_BATCH_FUSED 1
#define SM_BATCH_TILES 2
#define SM_BATCH_GRID  3

/* Shape of the batched launch; a field left 0 takes the tuned value for the
 * batch's largest subfield size N and its R (the table the library's
 * autotuner wrote, autotune.py).                                            */
typedef struct {
    int lookahead;      /* subfields whose transforms run ahead of the tiles  */
    int ctas_per_sm;    /* persistent CTAs per SM: 3 (168 registers a thread)
                           or 4 (128)                                          */
    int launch;         /* SM_BATCH_FUSED: one persistent launch whose items
                           are the transforms and the tiles; SM_BATCH_TILES:
                           the transforms first (per-stage spectra kernel),
                           then one persistent launch of the tiles;
                           SM_BATCH_GRID: the transforms first, then one grid
                           of CTAs over every tile of every burst (scheduled
                           by the hardware, not a queue)                      */
    int tile_order;     /* order of a subfield's tiles in the queue: 1 as the
                           plan lists them (by target block), 2 costliest
                           first                                               */
} sm_batch_opts;

/* Build the work queue of a batch of n (1..8) bursts: burst i has the plan
 * plans[i], F[i] frames of frame_type[i].  The plans may differ (channel,
 * frame size, N, R) but share the device and the spectra precision, and
 * accumulate plain FP32 sums (SM_ACC_PLAIN).  The queue holds one item per
 * (burst, subfield, frame) transform (SM_BATCH_FUSED) and per (burst,
 * subfield, tile) of the bispectrum (SM_BATCH_FUSED, SM_BATCH_TILES); a
 * subfield's transforms come `lookahead` subfields ahead of its tiles.  The
 * SM_BATCH_GRID launch needs no queue.  opts may be NULL
 * (all tuned).  Allocates the queue, the dependency counters and a
 * transform scratch tile per persistent CTA on the device (sm_batch_info
 * reports the bytes), and one stream per burst for the stages after the
 * batched launch; SM_EINVAL on a bad batch.  A batch serves one run at a
 * time: its queue, counters and status word are reused by every run, so
 * runs issued on different streams must be ordered by the caller (runs on
 * one stream are).                                                          */
int sm_batch_create(int n, const sm_plan* const* plans, const int* F, const int* frame_type,
                    const sm_batch_opts* opts, sm_batch** out);
/* The shape the batch was built with (the tuned values filled in).         */
int sm_batch_get_opts(const sm_batch* bt, sm_batch_opts* opts);
int sm_batch_destroy(sm_batch* bt);
/* Items in the queue, persistent CTAs of the launch, device bytes held.    */
int sm_batch_info(const sm_batch* bt, int* n_items, int* grid, size_t* device_bytes);

/* The batched transforms and bispectrum alone: spectra, flux and mean of
 * every subfield of every burst, and the bispectrum, into each burst's
 * workspace.  io: [n].  Asynchronous on `stream`; capturable in a CUDA
 * graph.  In SM_BATCH_FUSED a bispectrum tile waits for its subfield's F
 * transforms with a bounded poll; if a wait ever gives up, the tile is
 * skipped and sm_batch_status reports it.                                  */
int sm_batch_spectra_bispectrum(sm_batch* bt, const sm_batch_io* io, void* stream);
/* The whole path for every burst of the batch: the persistent launch, then
 * per burst P/M/noise, the seeing estimate when io[i].stf is NULL, the
 * modulus (Eq. 1), the photon-noise correction when the channel asks for it,
 * the phase, the inverse transforms and the mosaic.  Each burst's stages
 * after the batched launch run on a stream of the batch's own, forked from
 * `stream` and joined back to it, so bursts' recursions run side by side;
 * the call stays asynchronous on `stream` and capturable in a CUDA graph.
 * SM_EINVAL (before any launch) when a burst has no STF and its seeing
 * cannot be estimated.                                                      */
int sm_batch_reconstruct(sm_batch* bt, const sm_batch_io* io, void* stream);
/* Status of the last run's persistent launch, after the caller has
 * synchronised its stream: SM_OK, or SM_ECUDA when a dependency wait gave up. */
int sm_batch_status(const sm_batch* bt);

/* Model STF (Sect. 3.2, calibrated by r0): per frame
 * T0^2 exp(-6.88 (rho D/r0)^(5/3)) + ck (r0/D)^2 T0, averaged over the F
 * frames' D/r0 and normalised to 1 at k = 0.  Host only; stf_out is host
 * double [N][N], centred.                                                   */
int sm_model_stf(const sm_channel* ch, int F, const double* d_over_r0, double* stf_out);

/* ======================================================================== *
 *  Serving engine: bursts from several channels admitted as device slots   *
 *  free up, results polled by ticket.  Each slot has its own stream: one  *
 *  burst's host-to-device copy overlaps another's kernels, and by default  *
 *  the kernels themselves run one burst at a time in submission order     *
 *  (overlap_kernels = 0).  A burst's stage sequence is captured once as a *
 *  CUDA graph per (channel, F, frame type, STF mode, arena offset, slot)  *
 *  and replayed for later bursts with the same key.                        *
 * ======================================================================== */
typedef struct sm_handle sm_handle;

typedef struct {
    int               n_channels;
    const sm_channel* ch;               /* [n_channels]                         */
    size_t            hbm_budget_bytes; /* device memory the engine may hold     */
    int               max_inflight;     /* bursts on the device at once (>= 1)   */
    int               device;
    int               overlap_kernels;  /* 0: the kernels of admitted bursts run
                                           in submission order, one burst at a
                                           time, while the next bursts' frame
                                           copies proceed on their own streams;
                                           1: bursts' kernels run concurrently;
                                           2: pipelined -- two whole-burst
                                           workspaces; the bursts' transforms
                                           and bispectra run in submission
                                           order, and each burst's phase,
                                           inverse and mosaic run on a
                                           high-priority stream beside the
                                           next burst's transforms and
                                           bispectrum (the recursion takes a
                                           quarter of an SM and fills the
                                           issue slots the ALU-bound
                                           bispectrum leaves);
                                           3: batched -- bursts submitted
                                           together (sm_submit_batch) run
                                           through one batched launch
                                           (sm_batch_*), batches in
                                           submission order; every burst
                                           holds a whole-burst workspace     */
    /* Optional device allocator for the engine's one arena of
     * hbm_budget_bytes (both NULL: cudaMalloc / cudaFree).  dev_alloc is
     * called once by sm_open and must return device memory of `device`
     * aligned to 256 bytes, or NULL (sm_open then fails with SM_ENOMEM);
     * dev_free is called once by sm_close (or by a failing sm_open) with
     * that pointer.  Both receive alloc_ctx.  Giving one without the other
     * is SM_EINVAL.                                                          */
    void*           (*dev_alloc)(size_t bytes, void* ctx);
    void            (*dev_free)(void* ptr, void* ctx);
    void*             alloc_ctx;
} sm_config;

typedef struct {
    int            channel;
    int            F;                   /* frames in this burst (<= max_frames)  */
    const void*    frames;              /* [F][H][W] of frame_type               */
    int            frame_type;          /* SM_U16 / SM_F32                        */
    int            frames_on_device;    /* 1: frames is a device pointer          */
    const double*  stf;                 /* host [N][N] centred, or NULL           */
    const double*  d_over_r0;           /* host [F]; used when stf == NULL; with
                                         * both NULL the seeing is estimated on
                                         * the device (sm_stage_seeing)           */
    float*         out;                 /* host [H][W], caller-owned              */
    uint8_t*       valid;               /* host [H][W] or NULL                    */
} sm_burst;

typedef struct {
    int    status;                      /* SM_OK, SM_PENDING or an error          */
    double t_submit_ms;                 /* engine clock at submit return          */
    double t_done_ms;                   /* engine clock when the result was ready */
    double gpu_ms;                      /* device time of the burst's work        */
    size_t bytes_admitted;              /* device bytes held by the burst         */
    double d_over_r0;                   /* the burst's estimated D / mean r0, or 0
                                         * when the STF or D/r0 was given         */
    double stage_ms[8];                 /* device time of each stage, summed over
                                         * chunks: spectra, P/M/noise, seeing
                                         * estimate (0 when not estimated),
                                         * modulus, bispectrum, phase, inverse,
                                         * mosaic                                 */
} sm_result;

/* The serving calls restate the paper's statement of the problem for a
 * stream of bursts: a burst of F >= 100 short exposures of one channel
 * (Sect. 2, Table 1: H-alpha 1024 x 1024, TiO and G-band 2560 x 2160, each at
 * 10 frames/s) goes in, and one reconstructed mosaic comes out, computed
 * subfield by subfield and merged (Sect. 2, Sect. 3.2), with the seeing
 * estimated from the burst itself (Sect. 3.1) unless given.  The paper runs
 * one burst at a time on an MPI cluster; admission of bursts by a device
 * memory budget, tickets, overlap of one burst's copies with another's
 * kernels and the latency record are this library's serving design, not the
 * paper's.
 *
 * sm_open: create an engine: one plan per channel and one device arena of
 * hbm_budget_bytes.  With overlap_kernels = 0 (the default) the arena starts
 * with one workspace that every burst uses in turn, sized for the largest
 * channel's max_frames and the largest subfield chunk that leaves room for
 * max_inflight bursts' own buffers (frames, mosaic, mask, STF table); with
 * overlap_kernels = 1 each burst holds its own workspace in an equal share
 * of the budget; with 2 the arena starts with two whole-burst workspaces
 * (SM_ENOMEM when they and the bursts' buffers do not fit).  SM_ENOMEM when
 * the budget cannot hold one subfield's workspace beside those buffers
 * (shared workspace), or at submit when one burst does not fit its share.
 * *out is NULL on any failure.                                               */
int sm_open(const sm_config* cfg, sm_handle** out);
/* sm_submit_burst: stage one burst (Sect. 2: the frames of one burst of one
 * channel) -- copies the frames to the device (the caller may reuse them on
 * return) and queues its whole reconstruction (Sect. 2, 3.1, 3.2).  The
 * returned ticket names the burst for sm_poll.  SM_EBUSY when no slot or no
 * budget is free now (retry after a poll), SM_ENOMEM when the burst can never
 * fit the budget, SM_EINVAL for a bad burst.  With the environment variable
 * SM_FAULT=alloc:N set when the engine is opened, the N-th admission of that
 * engine (counting from 1) fails as if its arena allocation had failed: the
 * burst gets a ticket, nothing is queued, and sm_poll reports SM_ENOMEM for
 * it; the engine stays usable (a host-side failure injection for tests).   */
int sm_submit_burst(sm_handle* h, const sm_burst* b, uint64_t* ticket);
/* sm_submit_batch: stage n bursts (1..8, of any of the engine's channels)
 * and queue them as one batch: their transforms and bispectra in one batched
 * launch, then each burst's remaining stages (sm_batch_reconstruct, with the
 * autotuned launch shape), captured once per batch composition and arena
 * placement as a CUDA graph.  Needs an engine opened with
 * overlap_kernels = 3.  tickets: [n], one per burst, polled as usual
 * (stage_ms is not split for batched bursts).  All-or-nothing: SM_EBUSY
 * when the slots or the budget cannot take the whole batch now.            */
int sm_submit_batch(sm_handle* h, int n, const sm_burst* b, uint64_t* tickets);

/* sm_poll: the mosaic of one burst (Sect. 3.2: the merged image) -- wait
 * up to timeout_ms (0 = test and return SM_PENDING, > 0 = return SM_ETIMEDOUT
 * when it elapses, < 0 = forever).  SM_OK once the mosaic (and mask) are in
 * the burst's out (and valid) buffers; res gets the latency record and
 * per-stage device times; then the ticket is released.  The device copies
 * the results back at the end of the burst's own work: straight into out
 * and valid when they are page-locked host memory (so they may change while
 * the ticket is pending), otherwise into a pinned staging buffer from which
 * this call copies them.  A ticket whose work failed reports that status
 * once and is released.                                                      */
int sm_poll(sm_handle* h, uint64_t ticket, int timeout_ms, sm_result* res);
/* sm_close: end the engine -- cancel pending tickets, wait for the device,
 * free everything.  (The paper's master process ends after the mosaic is
 * written, Sect. 3.2; here the engine outlives any number of bursts.)      */
int sm_close(sm_handle* h);

/* sm_strerror: text of a status code of this library (no paper
 * counterpart).                                                             */
const char* sm_strerror(int status);
/* Last CUDA or validation message of this thread (never NULL). */
const char* sm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SPECKLE_GB300_H */
