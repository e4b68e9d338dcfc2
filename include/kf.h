/*
 * kf.h -- C ABI of the GB300 batched Kalman-step library (libkf.so).
 *
 * What it computes (paper section 2, "The p2r and p2z program"): for every
 * track of a batch, propagate the helix state and its covariance to a
 * detector surface -- a plane at fixed z (propagateToZ, "p2z") or a cylinder
 * at fixed r (propagateToR, "p2r") -- then Kalman-update the propagated track
 * against the track's hit on that surface (KalmanUpdate).  The paper gives no
 * formulas; the operations are the exact helix motion in a uniform field
 * B = (0, 0, bz), the transport Jacobian J and C' = J C J^T, and the textbook
 * linear Kalman update with a two-dimensional measurement:
 *   p2z: m = (x, y) of the hit, H = [e_x; e_y], V = top-left 2x2 of the hit
 *        covariance;
 *   p2r: m = (r*phi, z) at the hit, i.e. residual (u . (hit - x'), z_hit - z')
 *        with u = (-sin phi_h, cos phi_h), phi_h the azimuth of the hit, and
 *        V = P V_hit P^T, P = [[-sin phi_h, cos phi_h, 0], [0, 0, 1]].
 *
 * Units and conventions.  State p = (x, y, z, k, phi, theta): cm, cm, cm,
 * k = 1/pT in 1/GeV (k > 0), azimuth of the momentum in rad wrapped to
 * (-pi, pi], polar angle in rad.  Charge q = +1/-1 (int8) is separate.  The
 * signed curvature is omega = -q * 0.299792458e-2 * bz * k [1/cm] (a positive
 * charge turns clockwise seen from +z).  Symmetric 6x6 covariances are packed
 * lower-triangular, 21 floats in the order 00,10,11,20,21,22,30,...,55; the
 * 3x3 hit covariance is packed the same way, 6 floats (xx,xy,yy,xz,yz,zz).
 * p2r takes the first outward crossing of a track that starts strictly
 * inside the cylinder; p2z allows negative path (a plane behind the track).
 *
 * Layouts (paper section 2: an array of MPTRK blocks, each a structure of
 * arrays of bsize tracks).  Every per-track float array with C components
 * is either
 *   KF_SOA:   [C][n]            element (c, i) at c*n + i
 *   KF_AOSOA: [ceil(n/W)][C][W] element (c, i) at (i/W)*C*W + c*W + i%W,
 *             W = layout.width in {16, 32, 64, 128}; the last block is
 *             padded (allocate ceil(n/W)*W*C floats; padding is never read
 *             into a result and never written).
 * The components are: state 6, covariance 21, hit 3, hit covariance 6.
 * charge [n] and status [n] are plain arrays in both layouts; per-track
 * surfaces are a plain [n] float array.
 *
 * Ownership and execution.  Every data pointer is a DEVICE pointer owned by
 * the caller (allocated e.g. by PyTorch); the library allocates nothing per
 * call and keeps no reference after the call returns.  Managed memory and
 * page-locked host memory are accepted too (each array is checked against
 * its allocation); calls with such an array run the one-thread-per-track
 * kernels, whose plain loads and stores reach them, never the bulk copies
 * of the staged kernels.  Workspaces and arenas must be device memory.  Calls are enqueued on
 * `stream` (a cudaStream_t; NULL = the legacy default stream) and return
 * without synchronising.  Input and output may alias exactly (in place:
 * state_in == state_out and/or cov_in == cov_out); any other overlap is
 * undefined.  Float arrays must be 16-byte aligned.
 *
 * Errors.  Functions return KF_OK (0) or an error code; nothing is launched
 * when an argument is rejected.  KF_ERR_CUDA carries the CUDA message,
 * available from kf_last_error_string() (per calling thread).  Per-track
 * numerical problems never fail a call: they set bits in status[i]
 * (status may be NULL) and leave that track as described for each bit.
 */
#ifndef KF_H
#define KF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ return codes */
#define KF_OK              0
#define KF_ERR_ARG         1  /* null/misaligned pointer, n < 0, bad layout  */
#define KF_ERR_CUDA        2  /* a CUDA call or launch failed                */
#define KF_ERR_UNSUPPORTED 3  /* valid but not provided (e.g. a variant)     */
#define KF_ERR_TIMEOUT     4  /* a bounded device wait gave up               */

/* ------------------------------------------------------- per-track status */
#define KF_NO_INTERSECT 1u /* surface not reached: track copied unchanged    */
#define KF_S_NOT_PD     2u /* H C' H^T + V not positive definite: the track
                              is propagated but not updated                  */
#define KF_BAD_K        4u /* updated 1/pT <= 0 (kept as computed)           */
#define KF_NONFINITE    8u /* a non-finite value in the written result       */

/* ---------------------------------------------------------------- layouts */
#define KF_SOA   0
#define KF_AOSOA 1

typedef struct {
    int32_t kind;  /* KF_SOA or KF_AOSOA                                  */
    int32_t width; /* AoSoA block width W (16, 32, 64, 128); ignored for SoA */
    int64_t n;     /* number of tracks (>= 0; 0 launches nothing)         */
} kf_layout;

/* ------------------------------------------------------- update variants */
#define KF_FP32           0 /* all arithmetic in FP32                       */
#define KF_FP64_UPDATE    1 /* FP32 propagation; S^-1, K and C'' in FP64     */
#define KF_JOSEPH         2 /* FP32, Joseph-form C'' = (I-KH)C'(I-KH)^T+KVK^T */
#define KF_FP64           3 /* every operation of the step in FP64 (in the
                               chain the state also stays in FP64 between
                               layers)                                       */
#define KF_ADAPTIVE       4 /* FP32, and the whole step redone in FP64 for a
                               track whose FP32 step is ill-conditioned: the
                               hit shrinks a measured variance by more than
                               1e4, a cylinder is crossed at an incidence
                               cosine below 0.3, or the update leaves 1/pT
                               at or below 0 (a hit far off the track).
                               There the covariance update
                               C' - K H C' loses more digits than FP32 holds
                               (the propagated covariance is rounded element
                               by element, which breaks the near-perfect
                               correlations the update divides out).  In the
                               chain such a track reruns the whole chain with
                               its state in FP64.  Other
                               tracks run at the FP32 cost.  The single-step
                               entry points on device arrays (and the
                               compressed one) and the chain need a status
                               array with it: the FP32 kernel marks
                               ill-conditioned tracks there and a second,
                               short kernel redoes just those (KF_ERR_ARG
                               when status is NULL).  The host-array entry
                               points and the server use their own (the
                               host-array direct path: the workspace, or
                               the no-allocation call's staging buffer).    */
#define KF_DF_UPDATE      5 /* FP32 propagation; S^-1, K and C'' in
                               double-float: each quantity an unevaluated sum
                               of two floats (about 48 significant bits) with
                               error-free sums and products (Knuth's two-sum,
                               the FMA two-product, the double-word add and
                               multiply of Joldes, Muller and Popescu 2017,
                               compensated two-term dot products after Ogita,
                               Rump and Oishi 2005).  Same algebra as
                               KF_FP64_UPDATE at FP32 instruction rates
                               (GB300 issues FP64 at 1/64 of FP32).  In the
                               chain the state is rounded to FP32 between
                               layers, as for KF_FP64_UPDATE.                */

typedef struct {
    float    bz;        /* field along +z in tesla                          */
    int32_t  precision; /* KF_FP32, KF_FP64_UPDATE, KF_JOSEPH, KF_FP64,
                           KF_ADAPTIVE or KF_DF_UPDATE                      */
    uint32_t flags;     /* reserved, must be 0                              */
} kf_params;

/*
 * kf_p2z_propagate_update -- one p2z step for n tracks (paper section 2:
 * propagateToZ followed by KalmanUpdate).
 *   params          field and update variant (host pointer, read in call)
 *   layout          layout of every per-track float array (see above)
 *   state_in/out    [6 comps] track states in / out
 *   cov_in/out      [21 comps] packed covariances in / out
 *   charge          [n] int8, +1 or -1
 *   hit             [3 comps] hit position (x, y, z); z is not measured
 *   hit_cov         [6 comps] packed 3x3 hit covariance (xx, xy, yy used)
 *   z_surf          plane position(s): z_surf[0] for every track when
 *                   surf_per_track == 0, else z_surf[i] (plain [n] array)
 *   status          [n] uint8 per-track status bits, or NULL (not NULL
 *                   with KF_ADAPTIVE)
 *   stream          cudaStream_t
 * A track with |cos(theta)| <= 1e-4 is treated as parallel to the plane
 * (KF_NO_INTERSECT).
 */
int kf_p2z_propagate_update(const kf_params *params, kf_layout layout,
                            const float *state_in, const float *cov_in,
                            float *state_out, float *cov_out,
                            const int8_t *charge, const float *hit,
                            const float *hit_cov, const float *z_surf,
                            int32_t surf_per_track, uint8_t *status,
                            void *stream);

/*
 * kf_p2r_propagate_update -- one p2r step for n tracks (paper section 2:
 * propagateToR followed by KalmanUpdate).  Arguments as for p2z, with
 * r_surf the cylinder radius (or radii).  All six hit-covariance entries
 * are used (V = P V_hit P^T).  A track that starts on or outside the
 * cylinder, or whose helix stays inside it, gets KF_NO_INTERSECT.
 */
int kf_p2r_propagate_update(const kf_params *params, kf_layout layout,
                            const float *state_in, const float *cov_in,
                            float *state_out, float *cov_out,
                            const int8_t *charge, const float *hit,
                            const float *hit_cov, const float *r_surf,
                            int32_t surf_per_track, uint8_t *status,
                            void *stream);

/*
 * kf_p2z_propagate_update_host / kf_p2r_propagate_update_host -- the same
 * steps on HOST arrays, the host<->device transfers included (the paper's
 * p2z throughput counts the transfers: section 4, Figure 6).
 *   state_in ... status   HOST pointers with the layouts and sizes of the
 *                         device call (AoSoA arrays padded to whole blocks;
 *                         the padding of the output arrays may be
 *                         overwritten).  surf is a host scalar
 *                         (surf_per_track == 0) or host [n] array.
 *   workspace             DEVICE buffer owned by the caller, 256-byte
 *                         aligned, of at least
 *                         kf_host_workspace_bytes(layout, chunk_tracks)
 *                         bytes; used by the copy path only (and by the
 *                         direct path for KF_ADAPTIVE's redo marks when
 *                         status is NULL: n bytes), else may be NULL
 *   chunk_tracks          copy path: tracks per pipeline chunk (rounded up
 *                         to the AoSoA width); 0 selects 262144
 *   stream                the work starts after what is already queued on
 *                         `stream`, and work queued on `stream` afterwards
 *                         starts after it: synchronise `stream` before
 *                         reading the host outputs.
 * Two paths (kf_set_host_path chooses; by default the direct one wherever
 * it applies):
 *   direct  every array is reachable in place from the GPU -- page-locked
 *           (pinned) memory, or any mapped host memory on a device that
 *           walks the host page tables (cudaDevAttrPageableMemoryAccess-
 *           UsesHostPageTables: Grace-Blackwell, Grace-Hopper) -- and every
 *           float array 4-byte aligned: the kernel reads the inputs from and
 *           writes the results to the caller's arrays over the CPU-GPU link,
 *           on `stream`; no copies, no workspace.  Output arrays must be
 *           writable memory (a read-only mapping faults the kernel).
 *   copy    otherwise: the batch is processed in chunks alternating between
 *           two streams the library creates once per device (kept until
 *           exit); while one chunk runs its kernel and copies out, the next
 *           copies in.  Page-locked memory lets the copies run
 *           asynchronously; pageable memory works but the driver stages it.
 *           Calls on one device are serialised by a lock while they enqueue.
 * Errors as for the device calls.  Page-locked and device arrays are range-
 * checked against their allocations; pageable arrays only against the
 * process's mappings (KF_ERR_ARG when a range holds unmapped pages): their
 * sizes are otherwise the caller's duty.
 */
int kf_p2z_propagate_update_host(const kf_params *params, kf_layout layout,
                                 const float *state_in, const float *cov_in,
                                 float *state_out, float *cov_out,
                                 const int8_t *charge, const float *hit,
                                 const float *hit_cov, const float *z_surf,
                                 int32_t surf_per_track, uint8_t *status,
                                 void *workspace, int64_t workspace_bytes,
                                 int64_t chunk_tracks, void *stream);

int kf_p2r_propagate_update_host(const kf_params *params, kf_layout layout,
                                 const float *state_in, const float *cov_in,
                                 float *state_out, float *cov_out,
                                 const int8_t *charge, const float *hit,
                                 const float *hit_cov, const float *r_surf,
                                 int32_t surf_per_track, uint8_t *status,
                                 void *workspace, int64_t workspace_bytes,
                                 int64_t chunk_tracks, void *stream);

/* Device workspace bytes the host-array calls' copy path needs for `layout`
 * and `chunk_tracks` (0 = default chunk); -1 for an invalid layout. */
int64_t kf_host_workspace_bytes(kf_layout layout, int64_t chunk_tracks);

/*
 * kf_set_host_path -- how the host-array calls (the _host pair,
 * kf_propagate_update_host_noalloc and kf_server_submit) move data, for all
 * later calls in this process:
 *   KF_HOST_AUTO    (default) direct where every array allows it, else copy;
 *   KF_HOST_COPY    always the chunked copy path;
 *   KF_HOST_DIRECT  always direct: KF_ERR_ARG when an array is not reachable
 *                   in place (or, for KF_ADAPTIVE without a status array,
 *                   when there is no device scratch for the redo marks).
 * The results are the same on either path, bit for bit.  Returns KF_ERR_ARG
 * for an unknown mode.
 */
#define KF_HOST_AUTO   0
#define KF_HOST_COPY   1
#define KF_HOST_DIRECT 2
int kf_set_host_path(int32_t mode);

/* Step kinds for entry points that take the kind as an argument. */
#define KF_P2Z 0
#define KF_P2R 1

/*
 * kf_propagate_update_compressed -- the single step (kind KF_P2Z or KF_P2R)
 * on a compressed covariance store: per track six FP32 standard deviations
 * sigma_i = sqrt(C_ii) and fifteen FP16 correlations
 * rho_ij = C_ij / (sigma_i sigma_j), stored as IEEE binary16 bit patterns, in
 * packed off-diagonal order (10, 20, 21, 30, 31, 32, 40, ..., 54: rho_0 .. rho_14).
 *   sigma_in/out   [6 comps] float in the layout
 *   rho_in/out     15 uint16 per track, in pairs: per block of W tracks
 *                  (AoSoA; SoA is one block of W = n tracks) seven rows of
 *                  W pairs -- elements 2 (p W + r) and 2 (p W + r) + 1 hold
 *                  rho_2p and rho_2p+1 of the block's track r, p = 0..6 --
 *                  then one row of W values rho_14 (element 14 W + r); 15 W
 *                  values per block, the size of a [15 comps] array
 *   other arguments as for kf_p2z_propagate_update / kf_p2r_propagate_update.
 * The step decodes C_ii = sigma_i^2, C_ij = rho_ij sigma_i sigma_j, runs the
 * FP32 step and encodes the result (sigma = sqrt(max(C_ii, 0)), rho clamped
 * to [-1, 1], 0 where a sigma is 0, round to nearest).  FP16 keeps each
 * correlation to 2^-12, i.e. each covariance element to about 2.4e-4 of
 * sqrt(C_ii C_jj).  A track that is not propagated (KF_NO_INTERSECT) keeps
 * its input sigma and rho bit for bit.  Traffic per p2r track: 193 B instead
 * of 253 B.  No paper counterpart: a storage option of this library.
 */
int kf_propagate_update_compressed(int32_t kind, const kf_params *params,
                                   kf_layout layout, const float *state_in,
                                   const float *sigma_in,
                                   const uint16_t *rho_in, float *state_out,
                                   float *sigma_out, uint16_t *rho_out,
                                   const int8_t *charge, const float *hit,
                                   const float *hit_cov, const float *surf,
                                   int32_t surf_per_track, uint8_t *status,
                                   void *stream);

/* ------------------------------------------------------------ the chain */
#define KF_MAX_LAYERS 64

typedef struct {
    int32_t kind; /* KF_P2Z (plane at z = pos) or KF_P2R (cylinder r = pos) */
    float   pos;  /* z of the plane or radius of the cylinder, cm          */
} kf_layer;

/*
 * kf_kalman_chain -- the multi-layer track fit of the mini-apps (paper
 * section 2 and the layer loop of Figs. 3-5: for every layer, propagateToZ or
 * propagateToR, then KalmanUpdate), fused: each track runs through all L
 * layers in one kernel with its state and covariance in registers.
 *   params          field and update variant
 *   layout          layout of the per-track arrays (as for the single step)
 *   state, cov      [6 comps], [21 comps]: the start track on input, the
 *                   track after the last layer on output (in place)
 *   charge          [n] int8
 *   hits            L consecutive hit arrays, layer l at
 *                   hits + l * F3 floats, F3 = floats of a 3-component array
 *                   in the layout (3n for SoA, 3 W ceil(n/W) for AoSoA)
 *   hit_covs        L consecutive packed 3x3 hit-covariance arrays, layer l
 *                   at hit_covs + l * F6 floats
 *   layers          HOST array of L layer descriptors, 0 <= L <= KF_MAX_LAYERS
 *   status          [n] uint8: OR of the per-layer status bits, or NULL
 *                   (not NULL with KF_ADAPTIVE)
 *   stream          cudaStream_t
 * A layer the track does not reach is skipped (KF_NO_INTERSECT is set, the
 * track is left as it was) and the chain goes on with the next layer; a
 * layer whose update is rejected (KF_S_NOT_PD) leaves the propagated track.
 * Same arithmetic as the single-step calls: chain over one layer equals the
 * single step bit for bit.
 * Under KF_ADAPTIVE the second pass (the marked tracks' whole chain in
 * double) takes 4 (n + 1) bytes of device scratch, stream-ordered on
 * `stream`, from a memory pool the library creates per device on first use
 * and keeps (its memory included) for the life of the process; when that
 * allocation fails, or n >= 2^32 - 1, or the pool does not exist yet while
 * `stream` is being captured into a graph, the pass runs without it, with
 * the same results.  Under capture the allocation becomes a node of the
 * graph.
 */
int kf_kalman_chain(const kf_params *params, kf_layout layout, float *state,
                    float *cov, const int8_t *charge, const float *hits,
                    const float *hit_covs, const kf_layer *layers, int32_t L,
                    uint8_t *status, void *stream);

/* Capacity of the staging buffer of kf_propagate_update_host_noalloc. */
#define KF_NOALLOC_MAX_CHUNK     32768    /* tracks per staged chunk        */
#define KF_NOALLOC_STAGING_BYTES 8454144  /* device bytes held per GPU      */

/*
 * kf_propagate_update_host_noalloc -- the host-array step (as
 * kf_p2z_propagate_update_host / kf_p2r_propagate_update_host) for callers
 * that cannot allocate device memory.  The paper has no counterpart; this
 * entry point exists for deployment.
 *
 * Some callers cannot call cudaMalloc: a plugin or module whose process owns
 * the device allocator and forbids others from allocating, or a latency-
 * critical loop where cudaMalloc/cudaFree would synchronise the device.
 * Such callers pass only host arrays.  This call stages them through a
 * buffer of KF_NOALLOC_STAGING_BYTES (about 8 MiB) that the library itself
 * declares in device memory: every GPU that loads the library holds that
 * buffer until the process exits.  The call allocates nothing -- no
 * cudaMalloc, no cudaFree, no stream or event creation.
 *
 *   kind            KF_P2Z or KF_P2R
 *   params, layout, state_in ... status
 *                   as for the _host calls: HOST pointers, the same layouts
 *                   and sizes; status may be NULL; surf is a host scalar or a
 *                   host [n] array.
 *   chunk_tracks    tracks per staged chunk, 0 = KF_NOALLOC_MAX_CHUNK; a
 *                   value above KF_NOALLOC_MAX_CHUNK is rejected with
 *                   KF_ERR_ARG.  Any n is accepted: the batch is processed
 *                   chunk by chunk.
 *   stream          all copies and kernels run on this stream, in order;
 *                   synchronise it before reading the host outputs.
 * The direct path of the _host calls applies here too (kf_set_host_path):
 * where every array is reachable in place the kernel works on the caller's
 * arrays and the staging buffer is not used, except as the redo marks of
 * KF_ADAPTIVE without a status array (n <= KF_NOALLOC_STAGING_BYTES; larger
 * such calls take the copy path under KF_HOST_AUTO and are refused with
 * KF_ERR_ARG under KF_HOST_DIRECT).  Outputs that partially overlap the
 * inputs (not exactly in place) are refused with KF_ERR_ARG.
 *
 * Set-up: the first call on a device looks up the device address of the
 * staging buffer with that device current (cudaGetSymbolAddress) and keeps
 * it for the life of the process.  Make that first call before any stream
 * capture.  cudaDeviceReset is not supported while the library is in use:
 * the library keeps device addresses (this buffer's, the device error
 * word's) that a reset invalidates.
 * Sharing: every call on a device uses the same staging buffer, which keeps
 * the last call's contents (nothing in it needs to start at zero).  Calls
 * whose work overlaps on the GPU -- on different streams, or from different
 * host threads without ordering between them -- race on the buffer and
 * corrupt each other's results: keep them on one stream or order them.
 */
int kf_propagate_update_host_noalloc(int32_t kind, const kf_params *params,
                                     kf_layout layout, const float *state_in,
                                     const float *cov_in, float *state_out,
                                     float *cov_out, const int8_t *charge,
                                     const float *hit, const float *hit_cov,
                                     const float *surf, int32_t surf_per_track,
                                     uint8_t *status, int64_t chunk_tracks,
                                     void *stream);

/* -------------------------------------------------------------- tuning */
/*
 * The autotuner measures candidate launch shapes on the caller's arrays and
 * keeps the fastest per (GPU model, operation, kind, precision, layout,
 * n bucket = floor(log2 n)); later calls in KF_STEP_AUTO mode use it.  No
 * paper counterpart (the paper fixes bsize and launch shapes by hand).
 * Single-step candidates: one thread per track with 128 or 256 threads per
 * CTA; for AoSoA (and SoA with n a multiple of 4) also the persistent staged
 * kernel with 1, 2 or 3 CTAs per
 * SM (3: two pipeline stages per CTA instead of three, FP32-arithmetic
 * variants only; the others run it as 2).
 * Chain candidates: 64, 128 or 256 threads per CTA.
 */
typedef struct {
    int32_t step_kernel;  /* KF_STEP_DIRECT or KF_STEP_STAGED               */
    int32_t threads;      /* threads per CTA (one-thread-per-track kernels) */
    int32_t ctas_per_sm;  /* persistent CTAs per SM (staged kernel), 1-3    */
    float   ms;           /* measured time per call of the chosen shape     */
} kf_tuning;

/* Time every candidate with the arguments of kf_p2z/p2r_propagate_update
 * (synchronous; candidates take turns over 5 rounds of 10 timed calls after
 * 3 warm-up calls, each judged by its median round), store and return the
 * best.
 * Outputs are written repeatedly; with in == out the step is applied more
 * than once, so pass separate output arrays. */
int kf_autotune_step(int32_t kind, const kf_params *params, kf_layout layout,
                     const float *state_in, const float *cov_in,
                     float *state_out, float *cov_out, const int8_t *charge,
                     const float *hit, const float *hit_cov, const float *surf,
                     int32_t surf_per_track, uint8_t *status, void *stream,
                     kf_tuning *out);

/* The same for kf_kalman_chain (1 warm-up + 3 timed calls per candidate).
 * The chain runs in place, so the start state is saved into the caller's
 * device arrays state_scratch / cov_scratch (same sizes as state / cov),
 * restored before every call and once more at the end: state and cov are
 * unchanged when the call returns. */
int kf_autotune_chain(const kf_params *params, kf_layout layout, float *state,
                      float *cov, const int8_t *charge, const float *hits,
                      const float *hit_covs, const kf_layer *layers, int32_t L,
                      uint8_t *status, float *state_scratch, float *cov_scratch,
                      void *stream, kf_tuning *out);

/* The cache as text, one entry per line (*len = bytes without the final
 * NUL; buf may be NULL to ask for the size), and back.  Entries name the GPU
 * model, so a file written on one GB300 serves another. */
int kf_autotune_export(char *buf, int64_t cap, int64_t *len);
int kf_autotune_import(const char *text);
int kf_autotune_clear(void);

/* ----------------------------------------------------- the serving loop */
/*
 * A kf_server serves the multi-layer chain to a stream of events (requests)
 * with continuous batching.  No paper counterpart: the paper's mini-apps run
 * one fixed batch; this is the deployment form of the same chain.
 *
 * Events are submitted from any host thread at any time.  The server's
 * scheduler thread admits pending events in submission order while an event
 * slot (max_events_in_flight) and space in the caller's device arena are
 * free, copies each one in, and whenever the device is not already computing
 * a batch launches ONE kernel over every admitted event whose copies have
 * landed (at most 128).  Events submitted while a batch runs join the next
 * batch; results are copied out while the next batch computes.  Each track
 * runs the same arithmetic as kf_kalman_chain (SoA layout, one event per
 * submission), so an event's results do not depend on what else is in its
 * batch.  Creating a server creates its thread, three streams and
 * max_events_in_flight + 1 CUDA events; submitting and serving allocate
 * nothing (event memory comes from the arena).
 *
 * Direct events: where the server's GPU reaches every array of an event in
 * place -- page-locked memory, or any mapped host memory on a device that
 * walks the host page tables (the host-array calls' direct path; the
 * kf_set_host_path mode in force at submission decides) -- the batch kernel
 * reads the event's inputs from and writes its results to the caller's
 * arrays itself.  Such an event is ready for the next batch as soon as it is
 * admitted and done as soon as its batch completes: no copy-in, no
 * copy-out; the arena holds only its status marks (n bytes rounded up to
 * 256).  Other events are copied in and out through the arena.  The results
 * are the same either way, bit for bit.
 */
typedef struct kf_server kf_server;

typedef struct {
    float    bz;                       /* field, T                              */
    int32_t  precision;                /* any KF_* precision variant; KF_ADAPTIVE
                                          redoes the marked tracks of a batch
                                          in FP64 before the copy-out      */
    int32_t  L;                        /* layers of every event, 1..KF_MAX_LAYERS */
    kf_layer layers[KF_MAX_LAYERS];
    void    *arena;                    /* DEVICE memory owned by the caller,
                                          256-byte aligned, untouched outside
                                          the server until kf_server_destroy */
    int64_t  arena_bytes;
    int32_t  max_events_in_flight;     /* admitted and not yet finished, >= 1 */
    int32_t  device;                   /* CUDA device of the arena             */
} kf_server_config;

typedef struct {
    int64_t events_done;
    int64_t tracks_done;
    int64_t batches;                   /* kernel launches                      */
    int64_t max_batch_events;          /* most events in one launch            */
    double  p50_ms, p99_ms, max_ms, mean_ms; /* submit -> results in host memory */
    /* The same latency split into phases, p50 and p99 of each (ms, as the
     * scheduler thread observes them): queue = submit -> admitted (copy-in
     * issued); ready = admitted -> its batch launched (copy-in, then waiting
     * for the running batch); compute = launched -> batch seen finished;
     * out = copy-out issued -> landed in host memory. */
    double  queue_p50_ms, queue_p99_ms, ready_p50_ms, ready_p99_ms;
    double  compute_p50_ms, compute_p99_ms, out_p50_ms, out_p99_ms;
    /* the copy-in part of 'ready': admitted -> its copies seen landed (the
     * rest of 'ready' is waiting for the batch in flight to finish) */
    double  copyin_p50_ms, copyin_p99_ms;
    /* The device's own durations, from timing events recorded in the
     * streams around the work (0 where an event has no such work: a direct
     * event copies nothing): its copies in, its batch's kernel(s), its copies
     * out.  The host-observed phase minus the device duration is time the
     * work waited in its stream or the scheduler took to notice it. */
    double  gpu_copyin_p50_ms, gpu_copyin_p99_ms;
    double  gpu_compute_p50_ms, gpu_compute_p99_ms;
    double  gpu_out_p50_ms, gpu_out_p99_ms;
    /* host time the scheduler spent in the calls that enqueue the copies in
     * (part of copyin; 0 for a direct event) */
    double  copyin_issue_p50_ms, copyin_issue_p99_ms;
    /* the scheduler thread's longest pass, and its longest absence between
     * passes while GPU work was in flight (ms) */
    double  sched_pass_max_ms, sched_gap_max_ms;
} kf_server_stats;

/* Arena bytes one copied event of n tracks and L layers occupies (-1 if
 * invalid); a direct event occupies n bytes rounded up to 256. */
int64_t kf_server_event_bytes(int64_t n, int32_t L);

/* Create a server (starts its thread).  KF_ERR_ARG for a bad config or an
 * arena that is not device memory of the stated size. */
int kf_server_create(const kf_server_config *cfg, kf_server **out);

/*
 * Submit one event of n tracks.  HOST arrays, SoA per event: state [6][n],
 * cov [21][n] packed, charge [n], hits [L][3][n], hit_covs [L][6][n]; results
 * are written to state_out [6][n], cov_out [21][n] and status_out [n]
 * (status_out may be NULL).  The arrays must stay valid, and the inputs
 * unchanged, until the event is done; page-locked memory lets the copies
 * overlap, or the event go direct.  Returns at once with a ticket.
 * KF_ERR_ARG if the event can never fit the arena, if an array is pageable
 * memory with unmapped pages or page-locked memory shorter than the event,
 * or (under KF_HOST_DIRECT) if the event cannot go direct.
 */
int kf_server_submit(kf_server *s, int64_t n, const float *state,
                     const float *cov, const int8_t *charge, const float *hits,
                     const float *hit_covs, float *state_out, float *cov_out,
                     uint8_t *status_out, uint64_t *ticket);

/* *done = 1 once the event's results are in host memory.  Polling does not
 * release the ticket. */
int kf_server_poll(kf_server *s, uint64_t ticket, int32_t *done);

/* Block until the event is done (KF_OK; the ticket is then released) or
 * timeout_s seconds pass (KF_ERR_TIMEOUT; the ticket stays valid).  A
 * ticket's record (a few hundred bytes of host memory) is freed only by a
 * successful wait or by kf_server_destroy, so a long-running caller waits on
 * every ticket it is given, polled or not. */
int kf_server_wait(kf_server *s, uint64_t ticket, double timeout_s);

/* paused != 0: admit and launch nothing new (work already on the device
 * finishes); 0: resume. */
int kf_server_pause(kf_server *s, int32_t paused);

int kf_server_get_stats(kf_server *s, kf_server_stats *out);
int kf_server_reset_stats(kf_server *s);

/* Finish admitted and pending work (up to 30 s), stop the thread, release
 * the server's streams and events.  The arena is the caller's again. */
int kf_server_destroy(kf_server *s);

/*
 * kf_set_step_kernel -- choose the single-step kernel for all later calls in
 * this process (a tuning knob; the results are the same, bit for bit):
 *   KF_STEP_AUTO    (default) the autotuner's choice where it has one, else
 *                   the direct kernel in 128-thread CTAs (on GB300 it leads
 *                   or ties the staged kernel from 240,000 to 3.84 M tracks
 *                   and at every layout measured), and for the FP64-pipe-
 *                   bound variants (KF_FP64_UPDATE, KF_FP64) the staged
 *                   kernel at 2 CTAs/SM where it applies;
 *   KF_STEP_DIRECT  one thread per track with direct global loads (any
 *                   layout), 128-thread CTAs;
 *   KF_STEP_STAGED  a persistent kernel in which a producer warp streams
 *                   tiles into shared memory with bulk asynchronous copies
 *                   while eight warps compute: any AoSoA layout, and SoA when
 *                   n is a multiple of 4 (otherwise the direct kernel runs).
 * Returns KF_ERR_ARG for an unknown mode.
 */
#define KF_STEP_AUTO   0
#define KF_STEP_DIRECT 1
#define KF_STEP_STAGED 2
int kf_set_step_kernel(int32_t mode);

/*
 * kf_set_staged_ctas_per_sm -- resident CTAs per SM of the staged kernel
 * under KF_STEP_STAGED (the autotuner's choice applies under KF_STEP_AUTO):
 * 1 or 2 (three pipeline stages per CTA), 3 (two stages per CTA, more
 * compute warps per SM; FP32-arithmetic variants, the others run 2), or 0
 * for the default 2.  Results are the same, bit for bit.  Returns
 * KF_ERR_ARG outside 0..3.
 */
int kf_set_staged_ctas_per_sm(int32_t ctas);

/*
 * kf_set_chain_redo -- how kf_kalman_chain's KF_ADAPTIVE second pass runs
 * the marked tracks, for all later calls in this process (results are the
 * same, bit for bit):
 *   KF_CHAIN_REDO_LIST  (default) the whole batch's marked tracks in one
 *                       compacted list, 32 to a warp (device scratch from
 *                       the library's pool; per span when it cannot be had)
 *   KF_CHAIN_REDO_SPAN  each 4,096-track span's marked tracks by one block
 * Returns KF_ERR_ARG for any other value.
 */
#define KF_CHAIN_REDO_LIST 0
#define KF_CHAIN_REDO_SPAN 1
int kf_set_chain_redo(int32_t mode);

/*
 * kf_set_device_wait_limit -- how long the compute warps of the staged
 * kernels (KF_STEP_STAGED and the compressed store's staged kernel) wait for
 * a tile before they give up, in polls of the tile's barrier (each poll
 * backs off by about 0.1 us): 0 .. 16,777,216, or -1 for the default
 * (16,777,216: seconds, far beyond any healthy wait, which lasts
 * microseconds).  A wait that runs out sets KF_DEVERR_TIMEOUT in the device
 * error word (kf_take_device_error); that CTA then stops, lets the copies it
 * has in flight land and exits, so the call returns with its results
 * incomplete and the GPU context stays usable.  A limit of 0 makes every
 * such wait give up at once: every staged launch then reports
 * KF_DEVERR_TIMEOUT, which exercises the error path.  The producer warp's
 * own waits keep the default limit.  Process-wide, read at each launch;
 * results of launches that do not time out are unchanged.  Returns
 * KF_ERR_ARG outside the range.
 */
int kf_set_device_wait_limit(int64_t polls);

/*
 * kf_take_device_error -- read and clear the library's device error word
 * (synchronous).  Kernels that wait on barriers bound every wait; a wait
 * that gives up sets KF_DEVERR_TIMEOUT here and the kernel ends early, so
 * its results are incomplete.  *error_bits = 0 means no kernel gave up.
 */
#define KF_DEVERR_TIMEOUT 1u
int kf_take_device_error(unsigned int *error_bits);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH (0.3.1 = 301; the
 * minor number grows with every change of a declared struct or function, the
 * patch number with a change of behaviour behind the same declarations). */
#define KF_VERSION 400
int kf_version(void);

/* Message of the last KF_ERR_* returned on the calling thread ("" if none). */
const char *kf_last_error_string(void);

#ifdef __cplusplus
}
#endif

#endif /* KF_H */
