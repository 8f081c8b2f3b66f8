/*
 * bl.h -- C ABI of the GB300 beamline tracking library (libbl.so).
 *
 * The library tracks a 6D electron bunch, in coordinates relative to a
 * reference particle, through a beamline of linear transport elements and
 * plasma accelerator stages. Each element is a per-particle transfer map
 * f: R^6 -> R^6 (paper Sec. 1, valid without collective effects). A plasma
 * stage is either a classical RK4 push through a prescribed linear wake or a
 * learned MLP surrogate of that push (Sec. 3, Sec. 4.3). Particle arrays live
 * on the device and are owned by the caller; every call updates them in
 * place, as the paper's zero-copy views let the ML framework and the tracking
 * code share device memory (Sec. 2).
 *
 * Coordinates (all six arrays of one bunch have the same dtype and length n):
 *   x, y  [m]                transverse offsets
 *   px, py                   p_x / p_ref, p_y / p_ref
 *   t     [m]                c * (arrival-time offset), t = zeta_ref - zeta
 *   pt                       -(gamma - gamma_ref) / (beta gamma)_ref
 *
 * Conventions for every call:
 *   - Returns a bl_status; BL_OK on success. No exception crosses the ABI.
 *     bl_last_error_message() returns a per-thread description of the last
 *     failure.
 *   - Work is enqueued on the given CUDA stream (NULL = legacy default
 *     stream). Outputs that the call states are "host" are written before the
 *     call returns (the call synchronises the stream); all other outputs are
 *     valid after the stream is synchronised.
 *   - Pointers documented as "device" must be device (or managed) memory of
 *     the current device; "host" pointers are ordinary host memory.
 *   - Arguments are checked on the host before any work is enqueued; an
 *     invalid argument returns BL_ERR_INVALID_ARG and enqueues nothing.
 *   - The library keeps a scratch workspace per (device, stream). Calls on the
 *     same stream are ordered; calls on different streams use different
 *     workspaces and may run concurrently if they touch different particles.
 *   - Kernels that wait on the tensor core give up after a bounded spin and
 *     raise a device flag; bl_poll_device_errors() reports it as
 *     BL_ERR_TIMEOUT.
 */
#ifndef BL_H
#define BL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *bl_stream; /* same type as cudaStream_t */

typedef enum {
  BL_OK = 0,
  BL_ERR_INVALID_ARG = 1,
  BL_ERR_CUDA = 2,
  BL_ERR_OOM = 3,
  BL_ERR_UNSUPPORTED_ARCH = 4,
  BL_ERR_NONFINITE = 5,
  BL_ERR_TIMEOUT = 6,
  BL_ERR_STATE = 7
} bl_status;

typedef enum { BL_F32 = 0, BL_F64 = 1 } bl_dtype;

/* Objectives of bl_track_grad (final beam quantities, Sec. 4 moments). */
typedef enum {
  BL_OBJ_EPS_N_X = 0, /* normalised emittance, x plane */
  BL_OBJ_SIGMA_X = 1, /* rms beam size, x plane */
  BL_OBJ_EPS_N_Y = 2,
  BL_OBJ_SIGMA_Y = 3
} bl_objective;

/* A bunch, or a batch of independent bunches stored back to back.
 * Particle arrays: device, dtype `dtype`, n elements each, caller-owned.
 * Bunch b occupies particles [offsets[b], offsets[b+1]); offsets has
 * n_bunch+1 entries with offsets[0] = 0 and offsets[n_bunch] = n. When
 * n_bunch == 1 both offset pointers may be NULL. offsets_dev is device
 * memory and offsets_host the same values in host memory (the host copy lets
 * the library plan its grids without a device round trip).
 * gamma_ref is the reference particle's Lorentz factor (host value, shared by
 * all bunches); bl_track advances it through every plasma stage. */
typedef struct {
  void *x, *px, *y, *py, *t, *pt;
  int64_t n;
  int32_t n_bunch;
  int32_t dtype;
  const int64_t *offsets_dev;
  const int64_t *offsets_host;
  double gamma_ref;
} bl_bunch;

typedef enum { BL_DRIFT = 0, BL_QUAD = 1, BL_SBEND = 2, BL_PLASMA = 3, BL_PLASMA_LENS = 4 } bl_kind;

struct bl_surrogate_s;
typedef struct bl_surrogate_s bl_surrogate;
struct bl_lattice_s;
typedef struct bl_lattice_s bl_lattice;

/* One beamline element.
 *   BL_DRIFT:  L [m]
 *   BL_QUAD:   L [m], k [1/m^2] (k > 0 focuses x); per_bunch_k: host array of
 *              n_bunch_k strengths that override k bunch by bunch, or NULL
 *   BL_SBEND:  L [m] arc length, angle [rad] (sector bend, no edge focusing)
 *   BL_PLASMA: L [m], nsteps RK4 steps, n0_cm3 plasma density [1/cm^3],
 *              E0_Vpm wake amplitude [V/m], phi0 reference phase [rad];
 *              surrogate: trained stage surrogate, or NULL for the RK4 push;
 *              wide_surrogate: one of the paper's wide PReLU networks as the
 *              stage's surrogate instead (at most one of the two is set; the
 *              wide stage maps every particle and has no training domain).
 *   BL_PLASMA_LENS: L [m], k [1/m^2] focusing both planes alike (k > 0
 *              focuses): the linear map of an active plasma lens, whose
 *              azimuthal field gradient g = dB/dr [T/m] gives k = e g / p_ref
 *              (Sec. 4: plasma lenses between stages). per_bunch_k must be
 *              NULL; lens strengths are not among the strengths that
 *              bl_track_grad differentiates.
 * The linear maps are the solutions of the linear equations of motion of
 * H = px^2/2 + py^2/2 + pt^2/(2 b^2 g^2) + h^2 x^2/2 + h x pt/b + k (x^2-y^2)/2
 * (h = angle/L in a bend; k (x^2+y^2)/2 in a plasma lens); the paper (Sec. 1,
 * Sec. 4) treats them as given conventional elements. */
typedef struct {
  int32_t kind;
  int32_t nsteps;
  double L, k, angle;
  double n0_cm3, E0_Vpm, phi0;
  const bl_surrogate *surrogate;
  const double *per_bunch_k;
  const struct bl_wide_mlp_s *wide_surrogate; /* BL_PLASMA: a wide PReLU surrogate of the
                                                 stage (see bl_wide_mlp), or NULL */
} bl_element;

/* Compile a beamline. elements: host array of n_elements entries (copied).
 * n_bunch_k: length of every non-NULL per_bunch_k array (0 if none).
 * Consecutive linear elements are fused into one segment map per bunch. The
 * lattice keeps pointers to the surrogates it names: they must outlive it. */
bl_status bl_lattice_create(const bl_element *elements, int32_t n_elements,
                            int32_t n_bunch_k, bl_lattice **out);
bl_status bl_lattice_destroy(bl_lattice *lat);
int32_t bl_lattice_num_elements(const bl_lattice *lat);
int32_t bl_lattice_num_quads(const bl_lattice *lat);

/* Track the bunch through the lattice (Sec. 2/4.3: conventional elements and
 * plasma stages in one s-based loop, particles never leaving the device).
 * moments_out: host, n_elements * n_bunch * 28 doubles, or NULL. Entry
 * [e][b] holds the moments of bunch b after element e as
 * [N, 6 means, 21 central second moments S_ab, a <= b, row-major over
 * (x, px, y, py, t, pt)] with normalisation 1/N (Sec. 4 moments). Linear
 * elements' moments are propagated in FP64 (mu <- M mu, S <- M S M^T) from a
 * reduction at each segment's entry. When moments_out is non-NULL the call
 * synchronises the stream. nonfinite_out: host, or NULL; receives the number
 * of non-finite coordinates seen by the moment reductions (the particles are
 * kept). bunch->gamma_ref is advanced to the reference energy at the exit. */
bl_status bl_track(bl_bunch *bunch, const bl_lattice *lat, double *moments_out,
                   int64_t *nonfinite_out, bl_stream stream);

/* Track one FP32 bunch that lives in HOST memory (Sec. 4.3 at scale: the
 * beamline applied to a bunch streamed through the GPU; bunches larger than
 * device memory work too). in_host[c] / out_host[c] (c = x, px, y, py, t,
 * pt): n floats each in host memory; out may alias in. Page-locked buffers
 * let the copies overlap the tracking; pageable ones work but serialise.
 * The bunch is copied in chunks of `chunk` particles (0: 2^21 in the
 * whole-bunch mode below, 2^22 otherwise) on internal
 * streams (one per copy direction, two for compute). When the bunch fits in
 * half the free device memory and the lattice has two plasma stages or more,
 * the groups up to the first stage run chunk by chunk as the chunks arrive,
 * the groups in between run once on the whole device-resident bunch, and
 * the groups from the last stage on run chunk by chunk, each chunk copied
 * back as soon as it is done. Otherwise every chunk is copied in, tracked
 * through the whole lattice and copied back in a ring of four device chunk
 * buffers, so bunches larger than device memory work. Particles are tracked
 * by the same kernels as bl_track, one by one, so out_host equals bl_track's
 * result on a device copy of the bunch bit for bit. moments_out (host,
 * n_elements * 28 doubles, or NULL) and nonfinite_out (host, or NULL) are
 * bl_track's for the whole bunch: chunked reductions are pooled in FP64
 * (counts add, means pool, central moments gain the parallel-axis term),
 * equal to bl_track's up to FP64 rounding order. gamma_ref: in, the
 * reference Lorentz factor at the entrance; out, at the exit. The lattice may
 * carry per-bunch strengths for one bunch at most. Work already on `stream`
 * completes first; the call returns when out_host is written (synchronous).
 * Calls in one process run one at a time. Errors: BL_ERR_INVALID_ARG for bad
 * arguments (checked before any work), BL_ERR_NONFINITE as bl_track,
 * BL_ERR_CUDA / BL_ERR_OOM from the runtime (no copy is in flight on return). */
bl_status bl_track_host(const float *const in_host[6], float *const out_host[6], int64_t n,
                        double *gamma_ref, const bl_lattice *lat, int64_t chunk,
                        double *moments_out, int64_t *nonfinite_out, bl_stream stream);

/* bl_track split for CUDA-graph capture: bl_track_async enqueues the same
 * work without synchronising, allocating or touching host memory, writing
 * the raw reductions to reduced_dev (device, or NULL for none):
 * R * n_bunch * 28 doubles (R = bl_track_num_reductions(lat); reduction r is
 * taken at the entry of a segment or the exit of a stage not followed by
 * one), followed by one uint64 count of non-finite coordinates. The lattice's
 * plan for this bunch (reference energy, dtype, bunch count) and the
 * library's work buffers must exist before a stream capture: call bl_track or
 * bl_track_async once on the same bunch shape first (a capture without them
 * returns BL_ERR_INVALID_ARG). bunch->gamma_ref is advanced on the host at
 * enqueue time; a replayed graph is valid for the captured entry energy.
 * bl_track_expand_moments turns copied-back reductions into bl_track's
 * moments_out (host FP64 propagation through the segments' elements). */
int32_t bl_track_num_reductions(const bl_lattice *lat);
bl_status bl_track_async(bl_bunch *bunch, const bl_lattice *lat, double *reduced_dev,
                         bl_stream stream);
bl_status bl_track_expand_moments(const bl_lattice *lat, int32_t n_bunch,
                                  const double *reduced_host, double *moments_out);

/* Per-bunch moments of the current particles (Sec. 4 moments, definitions as
 * in bl_track). out: host or device, n_bunch * 28 doubles; valid after the
 * stream is synchronised. Accumulation (FP32 bunches): per thread, biased
 * FP32 sums whose rounding errors (products included) are recovered exactly
 * and folded into float-float pairs; FP64 across threads. FP64 bunches: FP64
 * sums. Uses library scratch memory. */
bl_status bl_moments(const bl_bunch *bunch, double *out, bl_stream stream);

/* Size of the fixed scratch used by bl_moments_noalloc, in partial-sum
 * slots of 28 doubles (about 7.3 MB): one slot per 4096-particle block plus
 * one per bunch, so one call handles up to about (32768 - n_bunch) * 4096
 * particles. */
#define BL_NOALLOC_SCRATCH_SLOTS 32768

/* bl_moments without any device allocation by the library, for callers that
 * cannot allocate device memory: a framework whose caching allocator owns the
 * GPU's memory, real-time or embedded code that reserves all memory up front,
 * or a pipeline that cannot tolerate the device-wide synchronisation that
 * cudaMalloc/cudaFree may imply. The paper has no counterpart.
 * Results are those of bl_moments. out: device-accessible memory (device,
 * managed or mapped pinned host), n_bunch * 28 doubles, valid after the
 * stream is synchronised. The per-block partial sums live in one fixed device
 * array of BL_NOALLOC_SCRATCH_SLOTS slots that the library defines at file
 * scope; every GPU that loads the library keeps it until the process exits.
 * Inputs larger than that scratch are rejected with BL_ERR_INVALID_ARG.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress), so make that first call before any stream capture;
 * the lookup is repeated when the device's context has changed (after a
 * cudaDeviceReset). An `out` that the GPU cannot store to through this very
 * pointer (plain pageable host memory, for instance) is rejected with
 * BL_ERR_INVALID_ARG before any work is enqueued.
 * All calls share the one array and every call overwrites what it reads, so
 * no state carries over from call to call; calls whose work overlaps on the
 * GPU (different streams or threads at the same time) race on it. */
bl_status bl_moments_noalloc(const bl_bunch *bunch, double *out, bl_stream stream);

/* Beam quantities of one 28-moment vector (host computation, Sec. 4):
 * out[0] eps_n,x = (beta gamma)_ref sqrt(S_xx S_pxpx - S_xpx^2), out[1] eps_n,y,
 * out[2] sigma_x = sqrt(S_xx), out[3] sigma_y, out[4] <gamma> =
 * gamma_ref - (beta gamma)_ref <pt>, out[5] relative energy spread
 * (beta gamma)_ref sigma_pt / <gamma>. moments28 and out: host. */
bl_status bl_beam_quantities(const double *moments28, double gamma_ref, double *out);

/* Apply one 6x6 matrix (host, row-major, 36 doubles, or n_bunch*36 for one
 * matrix per bunch when per_bunch != 0) to every particle: z <- M z. */
bl_status bl_apply_linear(bl_bunch *bunch, const double *M, int32_t per_bunch,
                          bl_stream stream);

/* Push every particle through one prescribed-wake plasma stage with classical
 * RK4 (the plain method a surrogate replaces, Sec. 4). The stage is given by
 * an element of kind BL_PLASMA (its surrogate field is ignored).
 * bunch->gamma_ref is advanced to the reference energy at the exit (FP64
 * reference particle on the host). FP32 bunches are integrated in
 * a deviation form relative to the FP64 reference trajectory; FP64 bunches in
 * FP64. */
bl_status bl_push_stage(bl_bunch *bunch, const bl_element *stage, bl_stream stream);

/* FP64 transfer matrix of a run of linear elements (host computation, no
 * device work): M_out (36 doubles, row-major) = M_{n-1} ... M_1 M_0 for the
 * elements' own strengths k (per_bunch_k is ignored) at reference
 * gamma_ref > 1. Elements must be BL_DRIFT, BL_QUAD, BL_SBEND or
 * BL_PLASMA_LENS; n = 0 gives the identity. The same matrices that bl_track
 * composes into segment maps, exposed for matching and optimisation on the
 * host (Sec. 4: the transport between stages is set from measured moments). */
bl_status bl_segment_matrix(const bl_element *elements, int32_t n, double gamma_ref,
                            double *M_out);

/* FP64 on-axis reference particle through one stage (host computation).
 * Returns gamma at the exit given gamma at the entry. */
bl_status bl_reference_exit(const bl_element *stage, double gamma_in,
                            double *gamma_out);

/* ---------------------------------------------------------------- MLP ---- */

/* Surrogate network F = L4 o s o L3 o s o L2 o s o L1 o s o L0 (Sec. 3, Eq.
 * for F) with widths 6 -> 128 -> 128 -> 128 -> 128 -> 6 and s = GELU
 * (tanh form). Weights W[l] are (out x in) row-major FP32 masters; the
 * device computes with BF16 copies and FP32 accumulation. mu/sd: FP64
 * per-coordinate normalisation of inputs and outputs (Sec. 3 data
 * preparation). All pointers are host memory and are copied. */
typedef struct {
  int32_t n_layers;          /* must be 5 */
  const int32_t *widths;     /* n_layers + 1 entries: 6,128,128,128,128,6 */
  const float *const *W;     /* n_layers pointers */
  const float *const *b;     /* n_layers pointers */
  const double *mu_in, *sd_in, *mu_out, *sd_out; /* 6 each */
} bl_mlp_desc;

/* ---- the paper's wide surrogate networks (Sec. 4.2) ----
 * F = L_{n-1} o prelu o ... o prelu o L_0 with PReLU (one learned slope per
 * hidden layer): widths[0] = widths[n_layers] = 6, hidden widths 1..4096
 * (e.g. five layers of 900 or three of 700 units). Weights are rounded to
 * BF16, activations are BF16 between layers, sums FP32; inputs and outputs
 * are normalised as for bl_surrogate. Weights W[l] are host FP32 row-major
 * [widths[l+1]][widths[l]], b[l] host FP32, slopes host FP32 (n_layers - 1).
 * Hidden widths are padded on the device with zero weights to multiples of
 * 64. */
typedef struct {
  int32_t n_layers;
  const int32_t *widths;
  const float *const *W;
  const float *const *b;
  const float *slopes;
  const double *mu_in, *sd_in, *mu_out, *sd_out;
} bl_wide_mlp_desc;

struct bl_wide_mlp_s;
typedef struct bl_wide_mlp_s bl_wide_mlp;

bl_status bl_wide_mlp_create(const bl_wide_mlp_desc *desc, bl_wide_mlp **out);
bl_status bl_wide_mlp_destroy(bl_wide_mlp *m);
/* Apply the network to every particle of an FP32 bunch in place, `chunk`
 * particles at a time (0: 2^21); the library keeps two activation buffers
 * of chunk x (widest padded layer) BF16 values per stream. */
bl_status bl_wide_mlp_apply(const bl_wide_mlp *m, bl_bunch *bunch, int64_t chunk,
                            bl_stream stream);

bl_status bl_surrogate_create(const bl_mlp_desc *desc, bl_surrogate **out);
bl_status bl_surrogate_destroy(bl_surrogate *s);
/* Training-input domain of a surrogate: the box [lo_c, hi_c] (host, 6 doubles
 * each, raw coordinates) of the inputs it was trained on; lo = hi = NULL
 * clears it. Inside bl_track, a particle entering this surrogate's stage
 * outside the box is not mapped by the network but pushed through the stage
 * by the plain RK4 method (the surrogate's fallback; the learned map is
 * trusted only where it was trained). bl_surrogate_apply and bl_track_grad
 * map every particle with the network. */
bl_status bl_surrogate_set_domain(bl_surrogate *s, const double *lo, const double *hi);
/* Surrogate files, so that training can resume: the FP64 normalisation
 * constants, the training domain, the FP32 master parameters, the Adam
 * moments and step count (binary, with a checksum; the BF16 image is rebuilt
 * on load). save synchronises the device; load validates the whole file
 * (magic, version, widths, finiteness, checksum) before it allocates. */
bl_status bl_surrogate_save(const bl_surrogate *s, const char *path);
bl_status bl_surrogate_load(const char *path, bl_surrogate **out);
bl_status bl_surrogate_get_norm(const bl_surrogate *s, double *mu_in, double *sd_in,
                                double *mu_out, double *sd_out);
/* The training domain as the kernels use it (FP32 bounds widened to contain
 * the box given to bl_surrogate_set_domain); *has = 0 when none is set. */
bl_status bl_surrogate_get_domain(const bl_surrogate *s, double *lo, double *hi, int32_t *has);

/* Read back the FP32 master parameters (after synchronising the device):
 * W_out[l] and b_out[l] are host buffers sized like the descriptor's. */
bl_status bl_surrogate_get_params(const bl_surrogate *s, float *const *W_out,
                                  float *const *b_out);

/* Replace relative coordinates at the stage entry by the surrogate's
 * prediction at the stage exit (Sec. 4.3 in-situ inference): FP64 normalise,
 * tcgen05 BF16 MLP with FP32 accumulation, FP64 de-normalise. FP32 bunches
 * only. Does not change bunch->gamma_ref. */
bl_status bl_surrogate_apply(const bl_surrogate *s, bl_bunch *bunch, bl_stream stream);

typedef struct {
  double lr, beta1, beta2, eps;
} bl_adam_cfg;

/* One Adam step (Sec. 3: MSE loss, Adam, minibatches) on a minibatch of
 * (input, target) pairs. in, out: device FP32, coordinate-major [6][ld];
 * idx: device int64 array of `batch` column indices, or NULL for columns
 * 0..batch-1. Inputs and targets are normalised with the surrogate's FP64
 * constants; the loss is the MSE over the normalised targets.
 * loss_out: device float, or NULL; receives the minibatch loss before the
 * update. The step counter t used for bias correction is kept in the
 * surrogate and advanced by one. 1 <= batch <= 2^24; a batch above 2^17
 * samples is processed in launches of 2^17 whose partial gradients are
 * summed in FP64, so the library's work buffers stay near 320 MB however
 * large the batch (BL_ERR_OOM if they cannot be allocated). */
bl_status bl_surrogate_train_step(bl_surrogate *s, const float *in, const float *out,
                                  int64_t ld, const int64_t *idx, int64_t batch,
                                  const bl_adam_cfg *cfg, float *loss_out,
                                  bl_stream stream);

/* Gradient of the minibatch MSE (same data layout as bl_surrogate_train_step)
 * without an update, for optimisers or data-parallel reductions outside the
 * library. grad_out: device, BL_MLP_NPARAM floats in the flat layout
 * [W0 (128x6), b0 (128), W1 (128x128), b1, W2, b2, W3, b3, W4 (6x128), b4 (6)],
 * weights row-major (out x in). loss_out: device float, or NULL. */
#define BL_MLP_NPARAM 51206
bl_status bl_surrogate_grad(const bl_surrogate *s, const float *in, const float *out,
                            int64_t ld, const int64_t *idx, int64_t batch, float *grad_out,
                            float *loss_out, bl_stream stream);

/* MSE of the surrogate on `count` pairs (test loss of the 70/30 split, Sec. 3)
 * with the same layout as bl_surrogate_train_step. loss_out: device double. */
bl_status bl_surrogate_loss(const bl_surrogate *s, const float *in, const float *out,
                            int64_t ld, const int64_t *idx, int64_t count,
                            double *loss_out, bl_stream stream);

/* ---- training the wide PReLU networks (Sec. 3 and 4.2: MSE on normalised
 * data, Adam, minibatches; every weight, bias and the slope of every hidden
 * layer is learned) ----
 * Parameters form one flat FP32 vector: W_0 (widths[1] x widths[0],
 * row-major), b_0, W_1, b_1, ..., W_{n-1}, b_{n-1}, then the n-1 slopes. The
 * forward pass is the inference datapath (tcgen05 BF16 layers, FP32
 * pre-activations kept); the backward pass (dW = dZ^T X, dX = dZ W with the
 * BF16-valued weights, the PReLU derivative and the slopes' gradient
 * sum min(pre, 0) dX) runs in FP32 on the CUDA cores. in, out, idx, ld and
 * batch as for bl_surrogate_train_step; batch <= BL_WIDE_MAX_BATCH. */
#define BL_WIDE_MAX_BATCH 65536
bl_status bl_wide_mlp_num_params(const bl_wide_mlp *m, int64_t *nparam);
/* Minibatch gradient into grad_out (device, num_params floats, flat layout)
 * and loss (device float, or NULL), without an update. */
bl_status bl_wide_mlp_grad(const bl_wide_mlp *m, const float *in, const float *out, int64_t ld,
                           const int64_t *idx, int64_t batch, float *grad_out, float *loss_out,
                           bl_stream stream);
/* One Adam step (bias-corrected, the step counter kept in the network);
 * loss_out: device float, or NULL, the minibatch loss before the update. */
bl_status bl_wide_mlp_train_step(bl_wide_mlp *m, const float *in, const float *out, int64_t ld,
                                 const int64_t *idx, int64_t batch, const bl_adam_cfg *cfg,
                                 float *loss_out, bl_stream stream);
/* The FP32 masters (after synchronising the device): W_out[l], b_out[l] host
 * buffers sized like the descriptor's, slopes_out n_layers - 1 floats. */
bl_status bl_wide_mlp_get_params(const bl_wide_mlp *m, float *const *W_out, float *const *b_out,
                                 float *slopes_out);

/* ------------------------------------------------------------ adjoint ---- */

/* Objective J of the final beam (Sec. 4.4: lens strengths tuned against final
 * beam quality) and its gradient with respect to every quadrupole strength of
 * the lattice, in element order, by reverse mode: segment maps transposed,
 * surrogate stages through the MLP's vector-Jacobian product recomputed from
 * stage-entry checkpoints. Plasma stages must be surrogates. The bunch is
 * tracked to the exit (its arrays and gamma_ref are updated as by bl_track).
 * J_out, dJ_dk: host (n_bunch and n_bunch * n_quads doubles, bunch-major).
 * The call synchronises the stream. */
bl_status bl_track_grad(bl_bunch *bunch, const bl_lattice *lat, int32_t objective,
                        double *J_out, double *dJ_dk, bl_stream stream);

/* -------------------------------------------------------------- misc ---- */

const char *bl_last_error_message(void);
const char *bl_version(void);

/* Read and clear the device-side error flags of the current device (bounded
 * waits that gave up). Synchronises the device. */
bl_status bl_poll_device_errors(void);

#ifdef __cplusplus
}
#endif

#endif /* BL_H */
