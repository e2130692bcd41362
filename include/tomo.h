/*
 * tomo.h - C ABI of the GB300 (sm_103a) library for decentralized ADMM
 * tomographic reconstruction with quantized messages
 * ("Distributed Tomographic Reconstruction with Quantization", Miao, Aslan,
 * Koyuncu, Gursoy, arXiv 2410.06106).
 *
 * Conventions shared by every call
 * --------------------------------
 * - All functions return tomo_status: TOMO_OK (0) or a negative error code.
 *   tomo_last_error() gives a message for the calling thread's last error.
 * - Argument errors (null pointers, sizes out of range, a geometry used on a
 *   different device) are detected on the host BEFORE anything is launched;
 *   the call then returns TOMO_ERR_INVALID_ARG and has no effect.
 * - Array arguments are caller-owned DEVICE pointers unless stated otherwise
 *   (PyTorch or cudaMalloc memory of the current device); the library never
 *   frees them and keeps no reference after the call returns, except the
 *   state pointers captured by dadmm_step (see there). Opaque handles are
 *   library-owned and released by their destroy call.
 * - Work is enqueued asynchronously on `stream` (NULL = legacy default
 *   stream); no call synchronizes unless documented.
 * - Handles (geometries, solvers) may be used from several host threads
 *   only one call at a time: the caller serializes calls on one handle.
 *   Distinct handles are independent (the process-wide cache of autotuned
 *   launch shapes is locked internally).
 * - Images are float32 [N][N] row-major, pixel (i, j) centred at
 *   x = j - (N-1)/2, y = (N-1)/2 - i (row 0 at the top, y up), unit pixels.
 *   Sinograms are float32 [angles][B] row-major; ray (a, b) is the line
 *   x cos(theta_a) + y sin(theta_a) = t_b, t_b = b - (B-1)/2.
 * - The system matrix entry P[(a,b),(i,j)] is the length of the
 *   intersection of ray (a, b) with pixel (i, j) (Sec. 2.1, Eq. 2); a ray
 *   lying exactly on the edge between two pixels gives each half the length.
 */
#ifndef TOMO_H
#define TOMO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define TOMO_API __attribute__((visibility("default")))
#else
#define TOMO_API
#endif

struct CUstream_st;
typedef struct CUstream_st* tomo_stream_t; /* same type as cudaStream_t */

typedef int tomo_status;
#define TOMO_OK 0
#define TOMO_ERR_INVALID_ARG -1 /* bad argument, nothing launched */
#define TOMO_ERR_CUDA -2        /* a CUDA runtime call failed */
#define TOMO_ERR_WORKSPACE -3   /* workspace / constant table too small */
#define TOMO_ERR_TIMEOUT -4     /* a bounded device wait gave up (see *_sync_status) */
#define TOMO_ERR_NUMERIC -5     /* non-finite values reached the statistics */

/* Message of the calling thread's most recent error ("" if none). The string
 * stays valid until the next failing call on the same thread. */
TOMO_API const char* tomo_last_error(void);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
TOMO_API int tomo_version(void);

/* ------------------------------------------------------------------ */
/* Geometry and the discrete x-ray transform (Sec. 2.1, Eq. 1-4)      */
/* ------------------------------------------------------------------ */

typedef struct tomo_geometry* tomo_geometry_t;

/* Create a parallel-beam geometry: N x N unit pixels, n_bins unit detector
 * bins, n_angles projection angles. angles_rad: HOST array of n_angles
 * radians, or NULL for theta_a = a pi / n_angles (uniform on [0, pi)).
 * Angles within 1e-12 rad of a multiple of pi/2 are snapped so that their
 * cosine and sine are exactly 0 or +-1.
 * The per-angle operator constants (fixed-point ray and pixel steps, trapezoid
 * weight constants) are derived on the host in FP64 and copied into device
 * tables owned by the geometry, on the current device.
 * Limits: 1 <= N <= 8192, 1 <= n_bins <= 16384, 1 <= n_angles <= 4096. */
TOMO_API tomo_status tomo_geometry_create(int N, int n_bins, int n_angles, const double* angles_rad,
                                 tomo_geometry_t* out);
TOMO_API tomo_status tomo_geometry_destroy(tomo_geometry_t g);

/* Forward projection, Eq. 4 restricted to a subset of angles:
 *   sino[k][q][b] = sum_{i,j} P[(angle_idx[q], b), (i,j)] img[k][i][j]
 *                   - (subtract ? subtract[k][q][b] : 0)
 * img      [batch][N][N]      device, read
 * sino     [batch][n_sel][B]  device, written (every element)
 * angle_idx[n_sel]            HOST int32 angle indices (NULL = all angles,
 *                             then n_sel must equal n_angles); read during
 *                             the call only
 * subtract [batch][n_sel][B]  device or NULL (the data term d of Alg. 2)
 * Requires 1 <= n_sel <= 65536 and batch >= 1 (an empty request is an
 * argument error, TOMO_ERR_INVALID_ARG, with nothing launched).
 * Ray-driven kernel, FP32 arithmetic, FP32 accumulation. */
TOMO_API tomo_status tomo_project(tomo_geometry_t g, const float* img, float* sino,
                         const int32_t* angle_idx, int n_sel, int batch,
                         const float* subtract, tomo_stream_t stream);

/* Forward projection that allocates no device memory. The paper has no
 * counterpart: this is a service for callers that cannot call cudaMalloc
 * (code running while a CUDA graph is being captured elsewhere in the
 * process, code bound to a fixed memory budget or pool, real-time loops that
 * forbid allocation after start-up). Same arguments, layouts and result as
 * tomo_project; the work list lives in a fixed array inside the library's
 * device image instead of memory the library allocates, so the call performs
 * no cudaMalloc/cudaFree and no allocating library routine.
 * Limits: n_sel <= 8192 angles and at most 16384 work items (about
 * batch * ceil(n_sel / 4) * ceil(B / 128); up to batch * n_sel * ceil(B / 128)
 * when consecutive angles cannot share an item); larger requests return
 * TOMO_ERR_WORKSPACE with a message and launch nothing. The array (576 KiB)
 * is held on every GPU that loads the library until the process exits.
 * Every call looks up the array's device address on the current device (the
 * first lookup may load the library's module on that device) and copies its
 * work list there from host memory that lives only during the call, so a
 * stream that is capturing a CUDA graph is refused with TOMO_ERR_INVALID_ARG
 * and nothing is enqueued. Every call reuses the same array and leaves its
 * work list there: calls that overlap on the GPU (other streams, or other host
 * threads) race and must be serialized by the caller. */
TOMO_API tomo_status tomo_project_noalloc(tomo_geometry_t g, const float* img, float* sino,
                                          const int32_t* angle_idx, int n_sel, int batch,
                                          const float* subtract, tomo_stream_t stream);

/* Matched backprojection (the exact transpose of tomo_project's matrix):
 *   img[k][i][j] = beta * img[k][i][j] + sum_{q,b} P[(angle_idx[q], b),(i,j)] sino[k][q][b]
 * beta must be 0 or 1 (0: img is not read). Same layouts and ownership as
 * tomo_project. Pixel-driven kernel, FP32. */
TOMO_API tomo_status tomo_backproject(tomo_geometry_t g, const float* sino, float* img,
                             const int32_t* angle_idx, int n_sel, int batch, float beta,
                             tomo_stream_t stream);

/* Work lists of the standalone operator calls. tomo_project, tomo_backproject
 * and tomo_opnorm_sq need, per (angle selection, batch), the work items of the
 * persistent kernels and the per-angle constants of the selection. The first
 * call with a selection builds them on the host and copies them into ONE
 * device allocation that the geometry keeps; every later call with the same
 * selection and batch allocates nothing. The geometry keeps at most 256 MiB
 * and 4096 selections of such lists and drops the least recently used beyond
 * that (cudaFree, which waits for the device). tomo_geometry_plan builds the
 * lists of a selection ahead of time (same angle_idx, n_sel and batch rules
 * as tomo_project; synchronous copy), so that the operator calls that use it
 * allocate nothing afterwards, e.g. before a stream capture or a loop that
 * must not allocate. tomo_geometry_cache_stats reports the device
 * allocations and frees of the geometry's lists so far and the selections
 * and bytes it holds (each output may be NULL). Neither launches a kernel. */
TOMO_API tomo_status tomo_geometry_plan(tomo_geometry_t g, const int32_t* angle_idx, int n_sel, int batch);
TOMO_API tomo_status tomo_geometry_cache_stats(tomo_geometry_t g, int64_t* allocs, int64_t* frees, int64_t* entries,
                                               int64_t* bytes);

/* Squared spectral norm ||P_sel||_2^2 by `iters` power iterations on
 * P_sel^T P_sel from a seeded start vector. work: device scratch of at least
 * tomo_opnorm_workspace_size() bytes. Synchronizes the stream; result in
 * *out (host). Used to choose the Algorithm 2 step eta1 = 1/(L + rho). */
TOMO_API size_t tomo_opnorm_workspace_size(tomo_geometry_t g, int n_sel);
TOMO_API tomo_status tomo_opnorm_sq(tomo_geometry_t g, const int32_t* angle_idx, int n_sel, int iters,
                           uint64_t seed, void* work, size_t work_bytes, double* out,
                           tomo_stream_t stream);

/* Device status of the standalone operator calls of geometry g
 * (tomo_project, tomo_project_noalloc and the projections inside
 * tomo_opnorm_sq): enqueues a read and a reset of g's status word on
 * `stream`, synchronizes the stream and returns TOMO_ERR_TIMEOUT if a
 * projector block stopped waiting for a staged image band (its bounded wait
 * gave up; those outputs are incomplete), TOMO_ERR_CUDA on an internal
 * staging-extent error, else TOMO_OK. Operator calls themselves are
 * asynchronous and cannot report device-side failures; the word is shared by
 * every call on g since the previous read. */
TOMO_API tomo_status tomo_sync_status(tomo_geometry_t g, tomo_stream_t stream);

/* Self test of the failure detection above, with no fault: launches one
 * block that waits, with the projector's bounded wait, on a barrier that
 * nothing completes; after timeout_ms (1..2000) of GPU time it sets the
 * timeout bit of g's status word and returns, leaving the context usable.
 * The next tomo_sync_status(g) returns TOMO_ERR_TIMEOUT. The projector's
 * own waits give up after one second. */
TOMO_API tomo_status tomo_selftest_wait(tomo_geometry_t g, int timeout_ms, tomo_stream_t stream);

/* ------------------------------------------------------------------ */
/* Measurement: the FP32 ceiling of the operators                      */
/* ------------------------------------------------------------------ */

/* Measured FP32 FMA throughput of the current GPU, the roofline denominator
 * of the projector and backprojector: both evaluate the system matrix of
 * Eq. 2 on the fly (Sec. 2.1), so their bound is the FP32 pipe, not memory.
 * Launches a grid that fills every SM (occupancy API) whose threads run 8
 * independent chains of dependent FMAs, once with scalar fmaf and once with
 * packed two-lane FMAs, each timed with CUDA events over one launch of about
 * target_ms (1..2000) after a warm-up. Outputs (HOST, each may be NULL):
 * TFLOP/s of the scalar and of the packed form (one FMA = 2 FLOP), and the
 * SM clock in MHz that the scalar launch ran at (SM cycle counter over the
 * global nanosecond timer of one thread). Synchronizes the stream; refuses a
 * stream that is capturing a CUDA graph (TOMO_ERR_INVALID_ARG). */
TOMO_API tomo_status tomo_fp32_peak(int target_ms, double* tflops_scalar, double* tflops_packed, double* sm_mhz,
                                    tomo_stream_t stream);

/* Measured shared-memory load bandwidth of the current GPU (GB/s over all
 * SMs): the other ceiling of both operators, which read 8 bytes of staged data
 * from shared memory per pixel-angle update (two FP32 image values per ray and
 * row in the projector, one (r_b, r_b+1) pair per pixel and angle in the
 * backprojector). Conflict-free 8-byte loads (a warp reads 256 consecutive
 * bytes) on a grid that fills every SM, timed with CUDA events over one launch
 * of about target_ms (1..2000) after a warm-up. Synchronizes the stream;
 * refuses a capturing stream (TOMO_ERR_INVALID_ARG). */
TOMO_API tomo_status tomo_smem_peak(int target_ms, double* gbs, tomo_stream_t stream);

/* ------------------------------------------------------------------ */
/* Elementwise building blocks of the differentiable unrolled ADMM      */
/* (Algorithm 2 step, Algorithm 3 closed form, Eq. 18; their adjoints)  */
/* ------------------------------------------------------------------ */

/* out[i] = sum_{j<k} coef[j] * x[j][i], i < n. x: HOST array of k device
 * pointers (float32, n each); coef: HOST array of k floats; 1 <= k <= 4.
 * out may alias any x[j] (every element is read before it is written). */
TOMO_API tomo_status tomo_lincomb(int64_t n, int k, const float* const* x, const float* coef, float* out,
                                  tomo_stream_t stream);

/* FP64 dot product sum_i x[i] y[i] (fixed reduction order: deterministic).
 * out: DEVICE float64 array of at least TOMO_DOT_SCRATCH entries; out[0]
 * receives the result, the rest is scratch. */
#define TOMO_DOT_SCRATCH 257
TOMO_API tomo_status tomo_dot(int64_t n, const float* x, const float* y, double* out, tomo_stream_t stream);

/* ------------------------------------------------------------------ */
/* Message quantizers (Sec. 2.7)                                       */
/* ------------------------------------------------------------------ */

/* Scalar K-means quantizer of one vector (Algorithm 5, Eq. 23).
 * in [n] device float32; codes [n] uint8 (centre index); centroids [k]
 * float32; deq [n] float32 = centroids[codes]; objective [iters+1] float64
 * or NULL (distortion after each assignment step).
 * Initial centres: the values at k indices drawn by the splitmix64 counter
 * key `key` (an index whose value is already a centre moves to the next
 * index, at most 64 times), sorted ascending. Then `iters` Lloyd
 * iterations: assign every value to the nearest centre by FP32 distance
 * (ties to the lower index); move each centre to the mean of its members
 * (exact 64-bit fixed-point sums at scale 2^sh, |v| 2^sh < 2^(62 - lg n),
 * so that the sum does not depend on its order; the mean in FP64); empty
 * clusters keep their centre.
 * A final assignment produces codes and deq. 1 <= k <= 32, n >= 1. */
TOMO_API tomo_status quant_kmeans(const float* in, int64_t n, int k, int iters, uint64_t key,
                         uint8_t* codes, float* centroids, float* deq, double* objective,
                         tomo_stream_t stream);

/* Counter key of the K-means initialisation for (seed, slice, owner,
 * iteration), as used by dadmm_step. Host function. */
TOMO_API uint64_t quant_kmeans_key(uint64_t seed, int slice, int owner, int iteration);

/* JPEG-style quantizer of one rows x cols segment (Sec. 2.7 "standard
 * JPEG"; rows, cols multiples of 8). Per segment lo = min, hi = max; FP32
 * sample map s = round(255 (v - lo) / (hi - lo)) - 128; orthonormal 8x8
 * DCT-II in registers; q = round(F / Qt) with the ITU-T T.81 Annex K
 * luminance table scaled to `quality` (IJG rule); dequantize, inverse DCT,
 * +128, round, clamp to [0, 255]; v' = lo + s'' (hi - lo) / 255 (hi for
 * s'' = 255). Rounding is half away from zero. A constant segment is sent
 * exactly (all coefficients 0). in, deq [rows][cols] float32; coefs
 * [rows/8][cols/8][64] int16 natural order (may be NULL); lohi [2] float32
 * (may be NULL); nnz: device int64 counter INCREMENTED by the number of
 * non-zero coefficients (may be NULL). 1 <= quality <= 100. */
TOMO_API tomo_status quant_jpeg(const float* in, int rows, int cols, int quality, int16_t* coefs,
                       float* lohi, float* deq, int64_t* nnz, tomo_stream_t stream);

/* Baseline sequential Huffman coding of the quantized blocks of one image
 * (ITU-T T.81 Annex F.1.2: DC differences by category with extra bits, AC
 * run/size symbols with ZRL and EOB in the zig-zag order of Figure A.6),
 * with the luminance tables of Annex K (Table K.3 DC, Table K.5 AC), codes
 * assigned as in Annex C, one DC predictor over the image, the last byte
 * padded with 1-bits and a 0x00 stuffed after every 0xFF byte: the
 * entropy-coded segment of a single-component baseline scan.
 *   coefs [rows/8][cols/8][64] int16, device, natural order within a block
 *     (the layout quant_jpeg writes); |AC| <= 1023, |DC difference| <= 2047;
 *   stream: device buffer of stream_cap >= quant_jpeg_entropy_bound() bytes
 *     for the stuffed segment, or NULL to count only;
 *   nbytes: device int64, set to the segment's length in bytes, or to -1 when
 *     a coefficient is outside the baseline range (nothing meaningful is
 *     written then);
 *   workspace: device scratch of quant_jpeg_entropy_workspace_size() bytes.
 * Asynchronous on `stream_`; one CTA codes the image. */
TOMO_API size_t quant_jpeg_entropy_bound(int rows, int cols);
TOMO_API size_t quant_jpeg_entropy_workspace_size(int rows, int cols);
TOMO_API tomo_status quant_jpeg_entropy(const int16_t* coefs, int rows, int cols, uint8_t* stream,
                                        size_t stream_cap, int64_t* nbytes, void* workspace,
                                        size_t workspace_bytes, tomo_stream_t stream_);

/* ------------------------------------------------------------------ */
/* Decentralized ADMM with quantized messages (Sec. 2.4-2.7, Alg. 2-4)  */
/* ------------------------------------------------------------------ */

#define DADMM_Q_NONE 0
#define DADMM_Q_KMEANS 1
#define DADMM_Q_JPEG 2

#define DADMM_MODE_BATCHED 0 /* one persistent launch per phase, CUDA graph */
#define DADMM_MODE_PLAIN 1   /* one launch per node and phase, no graph */

/* Problem description (all pointers are HOST arrays, copied by dadmm_create).
 * S independent slices share the geometry, the node split and the graph.
 *   node_ang_ptr [M+1], node_ang [n_angles]: CSR list of the angles each node
 *     holds (every angle belongs to exactly one node);
 *   seg_row_ptr [M+1]: segment m of x is the row band
 *     [seg_row_ptr[m], seg_row_ptr[m+1]); 0 = seg_row_ptr[0] < ... = N;
 *   adj [M*M]: symmetric 0/1 adjacency of the message graph (connected);
 *   edge_q [M*M]: quantizer kind of each edge (ignored where adj = 0);
 *   home_q [M]: quantizer of each node's own copy of its segment;
 *   eta1 [M]: Algorithm 2 step per node; eta2: Algorithm 3 step;
 *   E1, E2: inner GD steps; rho: penalty (Eq. 7);
 *   km_k, km_iters: K-means centres (<= 32) and Lloyd iterations;
 *   jpeg_quality: 1..100 (JPEG segments need rows and N multiples of 8);
 *   seed: K-means initialisation seed; mode: DADMM_MODE_*. */
typedef struct {
    int N, n_bins, n_angles, S, M;
    const int32_t* node_ang_ptr;
    const int32_t* node_ang;
    const int32_t* seg_row_ptr;
    const int32_t* adj;
    const int32_t* edge_q;
    const int32_t* home_q;
    const double* eta1;
    double eta2, rho;
    int E1, E2;
    int km_k, km_iters, jpeg_quality;
    uint64_t seed;
    int mode;
    int max_stale; /* >= 0: extra iterations a held message may age through losses
                      (dadmm_step_lossy); deepens the message ring by as many planes */
    int variant;   /* DADMM_VARIANT_SEGMENTS (Algorithm 4) or DADMM_VARIANT_CONSENSUS */
    int tune;      /* launch shapes: DADMM_TUNE_WIDE, _AUTO, _NARROW, _PAIRS, _QUADS or _WIDE_PAIRS */
} dadmm_config;

/* Launch shapes of the two operators. Wide: 64 x 64-pixel backprojector tiles
 * and 128-bin projector items; narrow: 32 x 64 tiles and 64-bin items for
 * runs of 4 angles (twice the work items, for problems with few of them).
 * With an even number of slices, both operators may also take slice-pair
 * items (two slices of one node per item, sharing the position and weight
 * arithmetic): the batched backprojector on narrow tiles (the plain form then
 * runs single-slice narrow tiles, with identical results), and the projector
 * in both forms (chunks of 16 rows; groups of 4 slices with chunks of 8 rows
 * when S is divisible by 4). Auto: the first dadmm_step of the solver times the shapes of each
 * operator on its own state and keeps the fastest (synchronizing the stream once; do not
 * make that first call while the stream is being captured); the choice is
 * cached per device and problem shape for the life of the process, so solvers
 * of the same problem, batched or plain, run the same shapes. Results differ
 * between shapes by FP32 rounding only (tile origins and chunk boundaries
 * move); for a given shape every run is deterministic. */
#define DADMM_TUNE_WIDE 0
#define DADMM_TUNE_AUTO 1
#define DADMM_TUNE_NARROW 2
/* slice pairs: narrow backprojector tiles with slice-pair items in the
 * batched form, and slice-pair projector items (128 bins) in both forms
 * (needs an even S) */
#define DADMM_TUNE_PAIRS 3
/* wide backprojector tiles, projector items of 4 slices of one node in both
 * forms (needs S divisible by 4) */
#define DADMM_TUNE_QUADS 4
/* wide backprojector tiles in slice pairs (batched form), projector items of 4
 * slices (needs S divisible by 4) */
#define DADMM_TUNE_WIDE_PAIRS 5

/* Algorithm 4: every node owns a segment of x and the segments travel over the
 * graph (the paper's decentralized ADMM). */
#define DADMM_VARIANT_SEGMENTS 0
/* Neighbour-averaged consensus, the decentralized analogue of the standard
 * ADMM x-update (Eq. 9): every node keeps its own x_m and sets it to the mean,
 * over its closed neighbourhood, of the messages Q(u_j + lambda_j / rho)
 * (full images; the edge's quantizer, the home quantizer for its own term);
 * messages travel one hop per iteration. The state's xseg is then x
 * [S][M][N][N] and hist the message planes [3][S][M][N][N]; seg_row_ptr,
 * eta2, E2 and max_stale are not used. On a complete graph without
 * quantization this is Eq. 8-10. */
#define DADMM_VARIANT_CONSENSUS 1

typedef struct dadmm* dadmm_t;

/* Create a solver for geometry g (which must outlive it). Builds the relay
 * tables (hop distance and first edge of the lowest-id shortest path from
 * every owner to every node), the persistent-kernel work lists and the
 * launch shapes (persistent grids sized by the occupancy API). Allocates only
 * small device tables owned by the handle. */
TOMO_API tomo_status dadmm_create(tomo_geometry_t g, const dadmm_config* cfg, dadmm_t* out);
TOMO_API tomo_status dadmm_destroy(dadmm_t h);

/* Depth D of the message ring (maximum hop distance + 1). */
TOMO_API int dadmm_ring_depth(dadmm_t h);

/* The launch shapes in use: backprojector tile width in pixels (64 or 32),
 * slices per batched backprojector item (1, or 2: two slices of one node and
 * tile share the position and weight arithmetic; even S), bins
 * per angle of 4-angle projector items (128 or 64), and slices per projector
 * item (1, 2 or 4: the rays of that many slices of one node share their
 * arithmetic; both forms, S divisible by it). With DADMM_TUNE_AUTO these are the wide single-slice
 * shapes until the first dadmm_step. */
TOMO_API tomo_status dadmm_launch_shape(dadmm_t h, int* bp_tile_x, int* bp_slices, int* proj_item_bins,
                                        int* proj_slices);

/* Device state, all caller-owned float32 unless noted:
 *   u, lam  [S][M][N][N]    local images u_m and duals lambda_m
 *   xseg    [S][N][N]       every owner's unquantized segment x[m]
 *   hist    [D][3][S][N][N] dequantized messages by (iteration mod D, kind)
 *   iter    int32 [1]       completed iterations k
 * dadmm_state_init zeroes all of it (Algorithm 4 starts from zero). */
typedef struct {
    float* u;
    float* lam;
    float* xseg;
    float* hist;
    int32_t* iter;
} dadmm_state;

TOMO_API size_t dadmm_state_size(dadmm_t h); /* bytes of u+lam+xseg+hist+iter, for sizing */
TOMO_API tomo_status dadmm_state_init(dadmm_t h, const dadmm_state* st, tomo_stream_t stream);

/* Report that the caller wrote the state (u, lambda, x, history or the
 * iteration counter) other than through dadmm_step / dadmm_state_init, e.g.
 * when restoring a checkpoint. The library keeps two arrays derived from the
 * state in the workspace: a transposed copy of u (read by the projector for
 * steep rays) and, per node, w_m = lambda_m - rho x_m^k, the part of the
 * Algorithm 2 step that stays fixed during its E1 inner steps (written by the
 * dual update of the previous iteration). It rebuilds both at the next
 * dadmm_step only after this call, after dadmm_state_init, or when the state
 * or workspace pointers change. Host-only; never fails for a valid h. */
TOMO_API tomo_status dadmm_state_modified(dadmm_t h);

/* Scratch for dadmm_step (residuals, the transposed copy of u and w of every
 * node, each [S][M][N][N] float32, codec scratch, partial sums); device,
 * caller-owned, at least dadmm_workspace_size() bytes, 256-byte aligned. */
TOMO_API size_t dadmm_workspace_size(dadmm_t h);

/* Per-iteration, per-slice statistics (float64), in this order:
 *   0 gap2   sum_m ||u_m - x_m^{k+1}||^2 (primal residual)
 *   1 chg2   ||x_0^{k+1} - x_0^k||^2 (node 0's view)
 *   2 nrm2   ||x_0^k||^2 (stopping test chg2 / nrm2 < 1e-12, i.e. 1e-6 rel.)
 *   3 res2   sum_m ||P_m u_m - d_m||^2 at the last inner step
 *   4 bytes  message bytes sent over the graph in this iteration */
#define DADMM_NSTAT 5

/* Run n_iters iterations of Algorithm 4 on sinograms sino [S][n_angles][B]
 * (device, natural angle order). Each iteration: E1 x {projector + residual,
 * matched backprojector + fused u step} for every node and slice; E2 segment
 * steps + K-means / JPEG messages for every owner; assembly of every node's
 * view through the message ring + dual update + FP64 norms.
 * BATCHED mode captures one iteration as a CUDA graph (re-captured when the
 * state/workspace/sino pointers or the stream change) and replays it.
 * stats: HOST [n_iters][S][DADMM_NSTAT] or NULL; when non-NULL the call
 * synchronizes the stream, fills it and checks the device status word:
 * TOMO_ERR_NUMERIC if a statistic is not finite (the state is still
 * advanced), TOMO_ERR_TIMEOUT if a bounded device wait gave up.
 * Right after dadmm_step_lossy calls that left some node holding an old
 * message version, the first iteration still reads that version (the
 * exchange then brings every node up to date); that call synchronizes once. */
TOMO_API tomo_status dadmm_step(dadmm_t h, const dadmm_state* st, const float* sino, int n_iters,
                       void* workspace, size_t workspace_bytes, double* stats,
                       tomo_stream_t stream);

/* Device status of the iterations run with this workspace since the last
 * read (dadmm_step with stats reads and resets it itself): reads and resets
 * the word on `stream`, synchronizes, and returns TOMO_ERR_TIMEOUT (a bounded
 * device wait gave up; the iterate is incomplete), TOMO_ERR_NUMERIC
 * (non-finite statistics), TOMO_ERR_CUDA (internal error) or TOMO_OK. The
 * word lives in the workspace; the first call of this handle on a workspace
 * (step or status read) zeroes it, so fresh memory needs no initialisation. */
TOMO_API tomo_status dadmm_sync_status(dadmm_t h, void* workspace, size_t workspace_bytes,
                                       tomo_stream_t stream);

/* dadmm_step with lost messages (a decentralized extension of Algorithm 4):
 * drop is a HOST array [n_iters][M][M] (n_iters <= DADMM_MAX_LOSSY_ITERS);
 * drop[i][s][m] != 0 means node m loses owner s's message in the exchange of
 * the i-th iteration of this call and keeps the version it holds; otherwise
 * it receives the newest version that has reached it over the relay. A
 * node's own segment is never lost (drop[i][m][m] is ignored). The versions
 * every node holds are tracked on the host, starting from the lossless ones
 * whenever the iteration counter differs from where the previous lossy call
 * ended. Requires a handle created with max_stale > 0; a mask that would make
 * a held version older than the message ring (max_stale extra iterations) is
 * refused with TOMO_ERR_INVALID_ARG before anything is launched. Reads the
 * iteration counter (synchronizes the stream once); otherwise as dadmm_step. */
#define DADMM_MAX_LOSSY_ITERS 256
TOMO_API tomo_status dadmm_step_lossy(dadmm_t h, const dadmm_state* st, const float* sino, int n_iters,
                                      const uint8_t* drop, void* workspace, size_t workspace_bytes,
                                      double* stats, tomo_stream_t stream);

/* Per-phase timing of the iterations. When enabled, dadmm_step records a
 * CUDA event (timing enabled) before and after every phase launch of an
 * iteration, inside the captured graph in BATCHED mode; phases are, in
 * order: E1 x (projector, backprojector + u-step), x-step, K-means, JPEG,
 * dual update + norms, statistics. Enabling or disabling forces a new
 * capture. dadmm_phase_times synchronizes on the most recent iteration's
 * last event and writes min(n, dadmm_num_phases()) durations in ms. */
TOMO_API tomo_status dadmm_set_profiling(dadmm_t h, int enable);
TOMO_API int dadmm_num_phases(dadmm_t h);
TOMO_API tomo_status dadmm_phase_times(dadmm_t h, float* ms, int n);

/* x as reconstructed by the owners: rows of segment m taken from the
 * home-quantized message of owner m at the current iteration (zero before
 * the first iteration). out [S][N][N] device. */
TOMO_API tomo_status dadmm_home_view(dadmm_t h, const dadmm_state* st, float* out, tomo_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* TOMO_H */
