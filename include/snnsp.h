/*
 * snnsp.h — C ABI of the GB300 (sm_103a) structural-plasticity library.
 *
 * Implements the data-parallel hot path of Knight, Senk & Nowotny, "A flexible framework
 * for structural plasticity in GPU-accelerated sparse spiking neural networks":
 * spike propagation through ragged sparse matrices (Sec. 2.1, Fig. 1), the LIF/ALIF
 * recurrent classifier with e-prop learning and Adam (Sec. 2.2.1), DEEP R rewiring
 * (Sec. 2.1.2, Fig. 2) and the topographic-map rewiring rule with STDP
 * (Sec. 2.1.3, Sec. 2.2.2, Fig. 3, Tab. 1-2).
 *
 * Conventions that hold for every entry point:
 *  - Every pointer named "device" is CUDA device memory owned by the CALLER; the library
 *    never frees it.  Opaque handles (snn_ragged, snn_classifier) and the fixed scratch
 *    they hold are owned by the library and released by the matching destroy call.
 *  - Every compute call is asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *    default stream), allocates nothing and never synchronises, unless its comment says
 *    otherwise (the create calls validate inputs and do synchronise).
 *  - Argument errors are returned synchronously (SNN_EINVAL, with a message from
 *    snn_last_error()).  Errors that only the device can see (capacity overflow,
 *    out-of-range index, a wait that gave up) are recorded in the handle's device
 *    status word and returned by snn_ragged_status(); no device code traps.
 *  - Ragged layout (Fig. 1): row i = presynaptic neuron i, slot (i, s) at i*C + s,
 *    s < row_len[i] are synapses, slots >= row_len[i] are padding for growth.  Rows
 *    are unsorted and contain no duplicate targets.
 *  - Bitfields: row i of a P x Q bitfield is ceil(Q/32) uint32 words; bit j of the row
 *    is bit (j & 31) of word (j >> 5).
 *  - Random numbers: Philox4x64-10 (Salmon et al., SC'11) keyed by (seed, purpose),
 *    with purpose-specific counters; Bernoulli(p) is "word < floor(p * 2^64)" and a
 *    uniform index in [0, n) is the high 64 bits of word * n.  The classifier's
 *    Poisson input is the one exception: 32-bit halves of the words against
 *    floor(p * 2^32) (see snn_step_neurons).
 *  - Spike accumulators (snn_propagate) are int64 fixed point with 40 fractional bits,
 *    so their sums do not depend on the order of the atomic additions.
 */
#ifndef SNNSP_H
#define SNNSP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t snn_status;
#define SNN_OK         0
#define SNN_EINVAL    (-1)   /* bad argument (sizes, NULL, alignment, unsupported dtype) */
#define SNN_ENOMEM    (-2)   /* library-owned scratch could not be allocated at create time */
#define SNN_ECAPACITY (-3)   /* a row ran out of padding, or activations were left over */
#define SNN_ECUDA     (-4)   /* a CUDA runtime call failed (message has the CUDA error) */
#define SNN_ETIMEOUT  (-5)   /* a bounded device-side wait gave up */
#define SNN_ESTATE    (-6)   /* device-detected invariant violation (bad index, bad row) */

#define SNN_F32 0
#define SNN_F64 1

#define SNN_FIXED_FRAC_BITS 40   /* fractional bits of the int64 spike accumulators */

typedef void* snn_stream;        /* cudaStream_t */

/* Message for the most recent failing call on this host thread ("" if none). */
const char* snn_last_error(void);
/* ABI version of this header (bumped on any incompatible change). */
int32_t snn_abi_version(void);   /* 8 */

/* ==================================================================================
 * Ragged sparse matrix (Sec. 2.1, Fig. 1; DEEP R bitfields Sec. 2.1.2, Fig. 2)
 * ================================================================================== */
typedef struct {
    int32_t P;            /* rows = presynaptic neurons */
    int32_t Q;            /* postsynaptic neurons (targets are 0..Q-1) */
    int32_t C;            /* capacity = maximum row length, padding included */
    int32_t dtype;        /* SNN_F32 or SNN_F64: element type of w, m, v, grad */
    int32_t no_autapse;   /* 1: target j == i is forbidden (recurrent projection) */
    int32_t reserved;     /* must be 0 */
    int32_t* row_len;     /* device [P] */
    int32_t* ind;         /* device [P*C] target indices */
    void* w;              /* device [P*C] weights / conductances */
    void* m;              /* device [P*C] Adam first moment, or NULL */
    void* v;              /* device [P*C] Adam second moment, or NULL */
    void* grad;           /* device [P*C] gradient (written by snn_eprop_update), or NULL */
    uint32_t* sign_bits;  /* device [P*ceil(Q/32)] DEEP R fixed signs, or NULL */
    uint32_t* conn_bits;  /* device [P*ceil(Q/32)] DEEP R connectivity mirror, or NULL */
    uint64_t seed;        /* Philox seed of this projection's structural plasticity */
} snn_ragged_desc;

typedef struct snn_ragged snn_ragged;

/* Counts of one rewiring call, written to DEVICE memory by the rewire calls
 * (accumulated: the caller zeroes it when it wants per-call numbers). */
typedef struct {
    int64_t removed;      /* synapses eliminated */
    int64_t formed;       /* synapses created */
    int64_t overflow;     /* formations skipped because a row was full / activations left over */
    int64_t attempts;     /* rewiring attempts processed (topographic rule) */
} snn_rewire_stats;

/* Validate a ragged matrix and wrap it in a handle.  Checks on the device (and waits
 * for the result): 0 <= row_len <= C, 0 <= ind < Q for live slots, no duplicate
 * targets in a row, no self target when no_autapse.  If init_deepr_bitfields != 0,
 * sign_bits and conn_bits must be given and are initialised as in Fig. 2A: all
 * connectivity bits cleared, all sign bits drawn from Philox (purpose SIGN, counter
 * (row, word, 0, 0), low 32 bits of word 0), then for every synapse its connectivity
 * bit set and its sign bit forced to the sign of its weight (w > 0: set, w < 0: clear,
 * w == 0: unchanged).  Allocates the handle's fixed scratch (O(P) words; with sign_bits
 * also a P*C word array in which DEEP R caches each live slot's sign bit, tagged with the
 * slot's target: a slot whose target changed outside the library reads the bitfield
 * again, so callers may rewrite row_len and ind freely, but the sign bit of a potential
 * connection must stay fixed, as the method has it, Sec. 2.1.2).  Returns SNN_EINVAL for
 * bad sizes/pointers, SNN_ESTATE if the contents are invalid. */
snn_status snn_create_ragged(const snn_ragged_desc* desc, int32_t init_deepr_bitfields,
                             snn_stream stream, snn_ragged** out);
snn_status snn_destroy_ragged(snn_ragged* r);
/* Wait for `stream`, then return and clear the handle's device status word
 * (SNN_OK, SNN_ECAPACITY, SNN_ESTATE or SNN_ETIMEOUT). */
snn_status snn_ragged_status(snn_ragged* r, snn_stream stream);

/* Spike propagation (Fig. 1): for every instance b < B and every row i whose bit is set
 * in pre_bits[b] (device [B][ceil(P/32)]), add w[i][s] to post_acc[b][ind[i][s]] for
 * s < row_len[i].  post_acc: device int64 [B][Q], fixed point (SNN_FIXED_FRAC_BITS),
 * accumulated into (the caller zeroes it).  Weights are shared by all instances. */
snn_status snn_propagate(const snn_ragged* r, const uint32_t* pre_bits, int32_t B,
                         int64_t* post_acc, snn_stream stream);

/* Target-tiled propagation (Fig. 1's operation, regrouped for shared-memory
 * accumulation).  A plan holds a copy of a handle's synapses grouped by target tile (W
 * consecutive targets; W chosen at create time so that the tiles spread over the GPU):
 * within tile k, entry (row i << 12 | j - kW, w_ij in fixed point) for every synapse i -> j.  One CTA per
 * (tile, group of 16 instances) reads its tile's entries once for all those instances,
 * adds the weights of rows spiking in each instance into exact 64-bit shared-memory
 * accumulators (two 32-bit reductions with an explicit carry) and adds them to post_acc
 * once: the result is the same int64 value snn_propagate gives (fixed-point sums do not
 * depend on order), with no global atomics.
 *  snn_create_prop_plan: allocates the plan's arrays (P*C entries, per-tile offsets, a
 *    per-row instance mask for max_B instances); P <= 2^20.  The plan refers to the
 *    handle, which must outlive it.  SNN_EINVAL / SNN_ENOMEM.
 *  snn_prop_plan_pack: rebuilds the tiles from the handle's current row_len, ind and w
 *    (asynchronous, capturable; call again after anything changes the synapses: an
 *    optimiser step, a rewiring, a caller edit).  A row length outside [0, C] or a
 *    target outside [0, Q) is skipped and sets SNN_ESTATE in the handle's status word.
 *  snn_propagate_tiled: as snn_propagate (same pre_bits, post_acc and result) from the
 *    last pack; B <= max_B.
 *  snn_destroy_prop_plan: frees the plan (NULL is a no-op). */
typedef struct snn_prop_plan snn_prop_plan;
snn_status snn_create_prop_plan(snn_ragged* r, int32_t max_B, snn_prop_plan** out);
snn_status snn_prop_plan_pack(snn_prop_plan* plan, snn_stream stream);
snn_status snn_propagate_tiled(const snn_prop_plan* plan, const uint32_t* pre_bits, int32_t B,
                               int64_t* post_acc, snn_stream stream);
snn_status snn_destroy_prop_plan(snn_prop_plan* plan);

/* DEEP R rewiring after the optimiser step (Sec. 2.1.2, Fig. 2B-C).
 *  elimination: slot s of row i is removed iff its weight's sign is strictly opposite
 *    to sign bit (i, ind); rows are compacted stably (survivors keep their order;
 *    w, m, v move with them); connectivity bits of removed synapses are cleared;
 *  redistribution: D = sum of removed counts is spread over rows in rounds
 *    r = 0..63: round r draws its remaining activations' rows (purpose DEEPR_DIST,
 *    counter (rewire_idx, r, k/4, 0), word k%4, row = mulhi(u, P)); a row takes at most
 *    min(C - row_len, free targets) in total; rejected activations go to round r+1;
 *  formation: the k-th activation of row i appends the m-th free target (ascending;
 *    the self target counts as taken when no_autapse), m = mulhi(u, n_free),
 *    u = Philox(DEEPR_FORM, (rewire_idx, i, k, 0)) word 0, with w = m = v = 0.
 * Needs w, m, v, sign_bits, conn_bits.  stats: device pointer or NULL.  Leftover
 * activations after 64 rounds are counted in stats->overflow and set SNN_ECAPACITY in
 * the status word. */
snn_status snn_rewire_deepr(snn_ragged* r, int64_t rewire_idx, snn_rewire_stats* stats,
                            snn_stream stream);
/* Same as snn_rewire_deepr with the rewiring index read from device memory when the
 * kernels run (rewire_idx_dev: device int64), so a captured CUDA graph can advance it. */
snn_status snn_rewire_deepr_dev(snn_ragged* r, const int64_t* rewire_idx_dev, snn_rewire_stats* stats,
                                snn_stream stream);

/* Distance-guided DEEP R formation.  The paper's Discussion proposes guiding DEEP R's
 * regrowth by the distance-dependent formation rule of the topographic map (Tab. 1-2)
 * instead of choosing new targets uniformly.  Neurons of both populations sit on sites
 * of an L x L torus; the k-th activation of row i picks free target j with probability
 * proportional to the integer weight q[d^2] = floor(2^24 exp(-d^2 / (2 sigma^2))), d the
 * torus distance between the sites of i and j (q computed on the host in double
 * precision): with S the weight total over the row's free targets and u the uniform
 * rule's draw, r = mulhi(u, S) picks the first free target in ascending order whose
 * running weight sum exceeds r.  A row whose free targets all weigh 0 falls back to the
 * uniform rule.  Elimination and the redistribution of activations over rows are
 * unchanged. */
typedef struct {
    int32_t L;                  /* side of the site grid (sites 0 .. L*L - 1) */
    int32_t reserved;           /* must be 0 */
    double sigma;               /* Gaussian width in grid units, > 0 */
    const int32_t* pre_site;    /* device [P]: site of each presynaptic neuron (row) */
    const int32_t* post_site;   /* device [Q]: site of each postsynaptic neuron (target) */
} snn_deepr_guide;
/* Attach a guide to a handle; g = NULL detaches it (uniform formation again).  Builds
 * the weight table in device memory that the handle allocates on the first call (its
 * only allocation after snn_create_ragged), checks every site on the device and waits
 * for the result: SNN_ESTATE if a site lies outside [0, L*L) (the guide stays off).  The
 * site arrays remain the caller's and must stay valid while attached.  snn_rewire_deepr
 * and snn_rewire_deepr_dev then form with the guide; snn_rewire_deepr_noalloc (no
 * handle) always forms uniformly.  Cost: two passes over a row's bitfield per
 * activation (the uniform rule needs one chunk scan). */
snn_status snn_ragged_set_deepr_guide(snn_ragged* r, const snn_deepr_guide* g, snn_stream stream);

/* Row updates, the two custom connectivity updates the paper lists (Sec. 2.1: add the
 * diagonal synapse to every row; remove from every row the synapse to a target the host
 * drew).  One optional edit per row, rows in parallel (a warp each).  targets: device
 * int32 [P], -1 = no edit.
 *  snn_ragged_add_row: appends synapse i -> targets[i] at slot row_len[i] with weight
 *    w_new[i] (device array of the matrix dtype, or NULL for 0), zero m, v and grad where
 *    the handle has them, and its connectivity bit where it has bitfields.  A target
 *    already in the row or a full row is skipped (stats->overflow).
 *  snn_ragged_remove_row: removes synapse i -> targets[i] if the row has it; the later
 *    slots move down one and keep their order (the paper moves the last synapse into the
 *    hole, which leaves the same set), and its connectivity bit is cleared
 *    (stats->removed).
 * A target outside [0, Q), or a self target of a no_autapse matrix, is skipped and sets
 * the invalid-state flag (SNN_ESTATE at the next snn_ragged_status).  Sign bits are not
 * touched.  stats: device or NULL (formed counts the adds).  Asynchronous. */
snn_status snn_ragged_add_row(snn_ragged* r, const int32_t* targets, const void* w_new, snn_rewire_stats* stats,
                              snn_stream stream);
snn_status snn_ragged_remove_row(snn_ragged* r, const int32_t* targets, snn_rewire_stats* stats,
                                 snn_stream stream);

/* DEEP R rewiring that allocates nothing (the paper has no counterpart; this entry
 * exists for callers that cannot allocate device memory).  Some callers cannot call
 * cudaMalloc: a serving process that reserved its whole device-memory budget at start-up
 * and must not grow it, a host framework whose own allocator owns every device buffer,
 * or a latency-critical loop where an allocation could synchronise the device.  They
 * cannot create an snn_ragged handle either, because that allocates its scratch.
 *
 * Same computation, inputs and outputs as snn_rewire_deepr, but on a plain descriptor
 * (the caller's device arrays; no handle) and with its scratch taken from a fixed array
 * of 16384 rows inside the library (static device memory that every GPU which loads the
 * library holds until the process exits).
 *  - desc->P must be <= 16384; larger matrices get SNN_EINVAL (use the handle API).
 *  - status: optional device int32 that receives the OR of the error flags
 *    (1 = leftover activations, 2 = invalid state); NULL discards them.
 *  - The first call on a device looks up the scratch's device address (once per
 *    device, with that device current); make that first call before any stream capture.
 *    The address is kept for the life of the process: after cudaDeviceReset (or any
 *    teardown of the device's primary context) this entry point must not be called
 *    again on that device in the same process.
 *  - desc->reserved must be 0, as for snn_create_ragged.
 *  - Every call shares the one scratch array and leaves its contents behind; the
 *    kernels re-initialise what they read.  Calls that overlap on the GPU (different
 *    streams, or different host threads, without ordering between them) race on it and
 *    give wrong results: serialise them.
 *  - Calls no cudaMalloc, cudaFree or allocating library routine. */
snn_status snn_rewire_deepr_noalloc(const snn_ragged_desc* desc, int64_t rewire_idx,
                                    snn_rewire_stats* stats, int32_t* status, snn_stream stream);

/* ==================================================================================
 * Recurrent LIF/ALIF classifier with e-prop (Sec. 2.2.1)
 * ================================================================================== */
typedef struct {
    int32_t n_in, N, K;   /* input channels, hidden ALIF/LIF neurons, readouts (K <= 32) */
    int32_t dtype;        /* SNN_F32 or SNN_F64 (all real arrays below and in the ragged
                             handles use it) */
    double tau_m;         /* membrane / readout / trace time constant (ms) */
    double v_thr;         /* baseline threshold */
    double beta;          /* adaptation strength (0 for LIF) */
    double tau_a;         /* adaptation time constant (ms); <= 0 means LIF (rho = 0) */
    double dt;            /* step (ms) */
    int32_t n_classes, n_bins;
    const uint32_t* in_thr;  /* device [n_classes][n_bins][n_in] Poisson thresholds:
                                floor(p * 2^32), saturated at 2^32 - 1 */
    uint64_t in_seed;        /* Philox seed of the input spikes (purpose INPUT) */
    snn_ragged* w_in;        /* P = n_in, Q = N */
    snn_ragged* w_rec;       /* P = N, Q = N, no_autapse = 1 */
    void* W_out;             /* device [K][N] readout weights */
    void* b_out;             /* device [K] readout biases */
    void* W_out_m; void* W_out_v;   /* device [K][N] Adam moments, or NULL */
    void* b_m; void* b_v;           /* device [K] Adam moments, or NULL */
    void* G_out;             /* device [K][N] readout weight gradient (written) */
    void* G_b;               /* device [K] readout bias gradient (written) */
    int32_t max_B, max_T;    /* largest batch and trial length the scratch is sized for */
} snn_classifier_desc;

typedef struct snn_classifier snn_classifier;

/* Per-batch state, records and workspace (all caller-owned device memory).
 * Win = ceil(n_in/32), Wh = ceil(N/32), Kp = roundup(K, 4). */
typedef struct {
    int32_t B, T;              /* trials in the batch, steps per trial */
    const int32_t* labels;     /* [B] class of each trial */
    const int32_t* bin_len;    /* [B] steps per template bin (time warp), >= 1 */
    const int64_t* trial_ids;  /* [B] Philox counter field of each trial's input */
    void* v; void* a; void* y; /* [B][N], [B][N], [B][K] state (zero before step 0) */
    uint32_t* x_bits;          /* [B][Win] input spikes of the last simulated step */
    uint32_t* z_bits;          /* [B][Wh] hidden spikes of the last simulated step */
    uint32_t* x_rec;           /* [B][T][Win] recorded input spikes */
    uint32_t* z_rec;           /* [B][T][Wh] recorded hidden spikes */
    void* psi_rec;             /* [B][T][N] recorded surrogate derivatives, or NULL (inference) */
    void* d_rec;               /* [B][T][K] recorded softmax(y) - onehot(label), or NULL */
    void* ysum;                /* [B][K] sum over steps of y (prediction = argmax) */
    void* v_rec; void* a_rec;  /* optional [B][T][N] voltage / adaptation records (NULL = off) */
    void* y_rec;               /* optional [B][T][K] readout records (NULL = off) */
    void* delta;               /* workspace [B][T][N] (e-prop adjoint) */
    void* Dout;                /* workspace [B][T][Kp] (filtered readout error) */
    const int32_t* trial_T;    /* [B] per-trial lengths (<= T) or NULL (all run T steps);
                                  forward only: trials stop at their own length */
} snn_batch;

/* Adam (Kingma & Ba; the optimiser of Sec. 3.1) with bias corrections 1 - beta1^t,
 * 1 - beta2^t.  The library forms beta^t itself, as a running product (beta^t = beta^(t-1)
 * x beta, starting from beta^0 = 1, in double precision: snn_adam_bias gives the values
 * it uses); the caller passes the step count t only. */
typedef struct {
    double lr, beta1, beta2, eps;
    int64_t step;             /* t >= 1: this is the t-th Adam step */
    const int64_t* step_dev;  /* optional device int64 holding t, read when the kernels run
                                 (lets a captured CUDA graph advance the step count on the
                                 device; the running products then live in the classifier
                                 handle's device scratch); NULL: use step */
    double l1;                /* DEEP R L1 strength (0: off); needs sign_bits */
    /* DEEP R noise term (Bellec et al. 2018; Sec. 2.1.2 notes that the paper leaves it
     * out, as Bellec et al. 2020 did): temperature > 0 adds sqrt(2 lr temperature) nu to
     * every active ragged weight after its Adam step (not to the dense readout), with
     * nu ~ N(0, 1) from the Box-Muller transform of Philox (purpose DEEPR_NOISE, key =
     * the matrix's seed, counter (noise_idx, row, slot, 0)):
     *   u1 = ((word0 >> 11) + 1) 2^-53 in (0, 1],  u2 = (word1 >> 11) 2^-53 in [0, 1),
     *   nu = sqrt(-2 ln u1) cos(2 pi u2)   (evaluated in double precision).
     * temperature = 0: off (the paper's setting). */
    double temperature;
    int64_t noise_idx;            /* counter field of this step's draws (e.g. the batch index) */
    const int64_t* noise_idx_dev; /* optional device copy of noise_idx, read by the kernel
                                     (graph replay); NULL: use noise_idx */
} snn_adam;

#define SNN_EPROP_GRAD  0
#define SNN_EPROP_APPLY 1

/* beta1^t and beta2^t exactly as the Adam step of snn_eprop_update forms them (running
 * products in double precision); out: host double[2].  Host only: needs no GPU.
 * SNN_EINVAL if step < 0 or a beta is outside [0, 1). */
snn_status snn_adam_bias(double beta1, double beta2, int64_t step, double* out);

/* Create a classifier handle; validates sizes (0 < K <= 32, N <= 2048, n_in <= 1024,
 * row capacities <= 2048) and allocates fixed scratch: the e-prop gradient partial sums
 * (sized from max_B, max_T and the two ragged handles), the packed forward rows and the
 * gather order of each row.  The forward sums each neuron's synaptic input of a step
 * exactly in integers (see snn_step_neurons for the grids) while its incoming |weight|
 * sum stays below 2^11 (2048 in weight units). */
snn_status snn_create_classifier(const snn_classifier_desc* desc, snn_classifier** out);
/* Row schedule of snn_step_neurons: how many warps (4, 8 or 16) share one trial's
 * spiking rows and neurons (default 8).  Results do not depend on it (integer
 * accumulation); an autotuner picks it per (N, row length, spike rate). */
snn_status snn_classifier_set_schedule(snn_classifier* c, int32_t warps_per_trial);
/* How the warps of a trial share the spiking rows of a step (results do not depend on
 * it): SNN_ROWS_PAIRS (default) a warp per row, two rows in flight per warp, 160 slots
 * of each per round trip; SNN_ROWS_PER_WARP one row at a time; SNN_ROWS_PER_BLOCK all
 * warps on each row, a 32-slot chunk each; SNN_ROWS_WIDE two rows, 256 slots of each per
 * round trip (long rows); SNN_ROWS_QUAD four rows, 128 slots each.  The last two keep 16
 * loads per thread in flight and exist in the persistent multi-instance kernel only
 * (its CTAs have the registers): snn_step_neurons runs them as SNN_ROWS_PAIRS.  The
 * persistent kernel reads the mode when its plan is created (snn_multi_create). */
#define SNN_ROWS_PAIRS     0
#define SNN_ROWS_PER_WARP  1
#define SNN_ROWS_PER_BLOCK 2
#define SNN_ROWS_WIDE      3
#define SNN_ROWS_QUAD      4
snn_status snn_classifier_set_row_schedule(snn_classifier* c, int32_t mode);
snn_status snn_destroy_classifier(snn_classifier* c);

/* Advance every trial of the batch by n_steps steps, t0 .. t0+n_steps-1 (t0 + n_steps
 * <= T), with all steps in one forward launch (one CTA per trial; the input spikes are
 * drawn by a launch before it and d by a launch after it).  Per step t (Sec. 2.2.1 equations with the
 * one-step synaptic delay):
 *   x^t    : input spikes, channel c fires iff the 32-bit half c%2 (0 low, 1 high) of
 *            Philox(INPUT; (trial_id, t, c/8, 0))[(c%8)/2]
 *            < in_thr[label][min(n_bins-1, t / bin_len)][c]
 *   I^t    : ragged propagation of x^{t-1} through w_in and z^{t-1} through w_rec
 *   v, a, z, psi : v = alpha (v - z v_thr) + I, a = rho a + z_prev, A = v_thr + beta a,
 *            z = [v >= A], psi = (0.3/v_thr) max(0, 1 - |v - A|/v_thr)
 *   y^t    : alpha y + W_out z^{t-1} + b ;  d^t = softmax(y^t) - onehot(label)
 * and records x, z, psi, d (and v, a, y when those pointers are set).  A label outside
 * [0, n_classes) or a bin_len < 1 sets SNN_ESTATE in w_in's status word and the trial
 * runs with the value clamped into range.  The synaptic sums are exact integer sums,
 * so their order does not matter: FP64 on the fixed-point grid 2^-40 (weights below
 * 2^-17 in magnitude are rounded to it); FP32 in 32 bits on a grid per neuron or readout,
 * 2^(sh - 40) with sh = max(0, bits(S 2^40) - 30) for its incoming |weight| sum S
 * (input, recurrent and readout weights, the bound on any step's sum), each weight
 * rounded (half up) to its target's grid: an error of at most S 2^-30 per weight (1.3e-8
 * at S = 14).  A neuron or readout whose S reaches 2^11 sets SNN_ESTATE (beyond it the
 * FP64 sums could wrap). */
snn_status snn_step_neurons(snn_classifier* c, const snn_batch* b, int32_t t0, int32_t n_steps,
                            snn_stream stream);

/* Draw the input spikes x^t of steps t0 .. t0+n_steps-1 into b->x_rec (the first part
 * of snn_step_neurons, as its own launch).  Needs labels, bin_len, trial_ids (and
 * trial_T when set) of b; touches nothing else.  A caller can draw the next batch's
 * inputs on another stream while the current batch trains, since they depend on
 * (trial, step, channel) only. */
snn_status snn_draw_inputs(snn_classifier* c, const snn_batch* b, int32_t t0, int32_t n_steps,
                           snn_stream stream);

#define SNN_STEP_INPUTS_READY 1   /* x_rec already holds the steps' inputs (snn_draw_inputs) */
#define SNN_STEP_PACKED_READY 2   /* the packed forward rows are current (snn_classifier_pack) */
/* snn_step_neurons with flags: SNN_STEP_INPUTS_READY skips the input draw;
 * SNN_STEP_PACKED_READY skips rebuilding the handle's packed forward rows from the
 * weights (the caller ran snn_classifier_pack after the last change of the weights);
 * every other flag bit is SNN_EINVAL.  Results are identical to snn_step_neurons when
 * x_rec holds what snn_draw_inputs wrote for the same batch and steps and the packed
 * rows are current.
 * Concurrency: a classifier handle's scratch (packed rows, their |weight| sums, gather
 * order, gradient partials) is written by snn_step_neurons and snn_eprop_update, so calls
 * on one handle must not overlap on the GPU -- except forward calls with
 * SNN_STEP_PACKED_READY, which only read it (e.g. several batches of requests of one
 * served model on different streams). */
snn_status snn_step_neurons_ex(snn_classifier* c, const snn_batch* b, int32_t t0, int32_t n_steps,
                               int32_t flags, snn_stream stream);
/* Rebuild the handle's packed forward rows (and the |weight| sums of the range check)
 * from the current weights on `stream`; what every snn_step_neurons call does first
 * unless it passes SNN_STEP_PACKED_READY. */
snn_status snn_classifier_pack(snn_classifier* c, snn_stream stream);

/* e-prop learning (Sec. 2.2.1 eligibility-trace equations, summed over trials).
 * SNN_EPROP_GRAD: from the records of a finished batch (all T steps) computes
 *   G^in, G^rec (into the ragged handles' grad arrays), G_out and G_b with the pairing
 *   G_ji = sum_t L_j^{t+1} ebar_ji^t.  It evaluates the traces in adjoint form: a
 *   reverse-time scan per hidden neuron builds delta_j^t such that
 *   G_ji = sum over presynaptic spikes (b, t) of neuron i of delta_j^{b,t}, which is the
 *   same sum reordered (equal up to rounding).
 * SNN_EPROP_APPLY: adds L1 (l1 * (sign bit ? +1 : -1)) to ragged gradients of
 *   projections with sign bits, then one Adam step on active ragged slots and on
 *   W_out, b_out (needs the moment arrays). */
snn_status snn_eprop_update(snn_classifier* c, const snn_batch* b, int32_t phase,
                            const snn_adam* adam, snn_stream stream);

/* ==================================================================================
 * Batched form: many classifier instances trained in one persistent launch
 * ================================================================================== */
/* One instance of the batched form: its own classifier (FP32; ragged handles with Adam
 * moments, gradient and DEEP R bitfields, no distance guide), one trial per iteration.
 * Iteration it of the instance runs exactly what these per-call steps run, in order:
 *   trial_ids[0] = it, labels[0] = label_table[it % n_label],
 *   bin_len[0] = bin_table[it % n_bin], state (v, a, y, ysum, x_bits, z_bits) zeroed;
 *   snn_step_neurons(cls, &batch, 0, T);  snn_eprop_update(GRAD);
 *   snn_eprop_update(APPLY) with Adam step it + 1, L1 l1, DEEP R noise (temperature,
 *     Philox counter it);
 *   snn_rewire_deepr on the input then the recurrent projection with rewire index it,
 *     counts added to stats[0] and stats[1];
 *   *iter = it + 1.
 * The results are bit-identical to those calls (same device functions). */
typedef struct {
    snn_classifier* cls;
    snn_batch batch;                /* B = 1, T <= min(max_T, 4096); state, records and workspace
                                       (no trial_T) in caller memory */
    const int32_t* label_table;     /* device [n_label] */
    int32_t n_label;
    const int32_t* bin_table;       /* device [n_bin]: steps per template bin */
    int32_t n_bin;
    int64_t* iter;                  /* device: iterations done (advanced by each run) */
    double lr, beta1, beta2, eps, l1, temperature;
    snn_rewire_stats* stats;        /* device [2] (input, recurrent), accumulated; or NULL */
} snn_multi_instance;

typedef struct snn_multi snn_multi;

/* Build the work plan of n instances (n distinct classifiers) and allocate its queue,
 * the instance table and a small mapped-host mailbox; synchronises.  SNN_EINVAL for an
 * unsupported instance. */
snn_status snn_multi_create(const snn_multi_instance* inst, int32_t n, snn_multi** out);
snn_status snn_multi_destroy(snn_multi* m);

#define SNN_MULTI_HOST_POSTS 1
/* One training iteration of every instance in ONE kernel launch on `stream`: a
 * persistent grid (as many CTAs as fit on the GPU) takes work items (instance, phase,
 * index) from a device queue; an instance's phases (input and packing, the trial's
 * forward, readout scan, adjoint scan, gradient gather, L1 + Adam, DEEP R elimination,
 * redistribution and formation) follow one another and interleave with the other
 * instances'.  Every wait of the kernel (for queue work, and for the mailbox) gives up
 * after wait_limit_ns (0 < limit <= 60 s): the kernel then leaves, the iteration is
 * incomplete and snn_multi_status returns SNN_ETIMEOUT.
 * flags = SNN_MULTI_HOST_POSTS: the kernel starts no instance by itself; it waits for a
 * host producer to name the instances of this iteration with snn_multi_post (called
 * after snn_multi_run; such runs cannot be replayed from a captured graph).  Without the
 * flag every instance runs (graph capture allowed: the run's queue stamp lives on the
 * device).  Runs of one plan must not overlap on the GPU. */
snn_status snn_multi_run(snn_multi* m, int32_t flags, int64_t wait_limit_ns, snn_stream stream);
/* Phase timing of later runs (tracing): times = device int64 [n][12] (NULL: off).  Each
 * run writes, per instance in the order given to snn_multi_create, the global timer (ns)
 * when its iteration was seeded ([i][0]) and when each of its 11 phases completed
 * ([i][1 + phase]: bookkeeping, inputs and accumulator weight sums, packing, forward
 * (with the gather order beside it), readout scan, adjoint scan, gather, Adam, DEEP R
 * elimination, redistribution, formation).  The caller keeps the buffer alive while it
 * is set. */
snn_status snn_multi_set_trace(snn_multi* m, int64_t* times);
/* Host producer for a SNN_MULTI_HOST_POSTS run: the instances (indices into the array
 * given to snn_multi_create, no repeats) that the running iteration should train.
 * Writes the plan's mapped mailbox; the kernel picks it up while it runs. */
snn_status snn_multi_post(snn_multi* m, const int32_t* instances, int32_t n);
/* Wait for `stream`, then return and clear the plan's status: SNN_ETIMEOUT if a wait
 * gave up, SNN_ESTATE for an invalid post, else SNN_OK.  The instances' own device
 * errors stay in their ragged handles' status words. */
snn_status snn_multi_status(snn_multi* m, snn_stream stream);

/* ==================================================================================
 * Topographic map (Sec. 2.1.3, Sec. 2.2.2, Tab. 1-2): conductance LIF target sheet,
 * correlated Poisson source sheet, STDP and distance-dependent rewiring on a torus
 * ================================================================================== */
typedef struct {
    int32_t L;            /* grid side; N = L*L neurons per sheet */
    int32_t L_f;          /* stimulus tile side (L for a single focus) */
    int32_t radius2;      /* squared focus radius (sites^2) */
    int32_t t_stim;       /* steps between focus re-draws */
    double dt, tau_m, V_rest, E_exc, V_theta, V_reset, tau_s, g_leak;
    double tau_ref;       /* absolute refractory period (ms, Tab. 2D): V is held at V_reset
                             for round(tau_ref / dt) steps after a spike */
    double f_base, f_in;             /* Hz outside / inside the focus (disc profile); with
                                        sigma_stim > 0: base and peak rate */
    double g_max, tau_plus, tau_minus;
    /* STDP rates as Tab. 2F defines them: A_+ = A_plus_rel g_max (A_plus_rel = 0.1 in the
     * paper) and A_- = B A_+ tau_+ / tau_- (B = 1.2, the ratio of potentiation to
     * depression); the library derives A_+ and A_- (snn_topo_derive shows the values). */
    double A_plus_rel, B;
    /* Input profile.  sigma_stim = 0: disc, channel rate f_in within squared torus
     * distance radius2 of its tile's focus, f_base outside.  sigma_stim > 0: the Gaussian
     * of Tab. 1 "Input", rate f_base + f_in exp(-d^2 / (2 sigma_stim^2)) (f_in is f_peak).
     * Either way a channel fires iff its Philox word is below thr(d^2) =
     * floor(rate dt 1e-3 2^64), computed on the host in double precision from the
     * expression in that order.  The thresholds of d^2 >= 1024 must all equal
     * thr(1023) (true for the disc with radius2 < 1023 and for any Gaussian whose
     * tail has fallen below the rounding of f_base by then, e.g. sigma_stim = 2);
     * otherwise the calls return SNN_EINVAL. */
    double sigma_stim;
} snn_topo_params;

/* The quantities the library derives from snn_topo_params (Tab. 2D, 2F). */
typedef struct {
    int32_t n_ref;        /* refractory steps: round(tau_ref / dt) */
    int32_t reserved;
    double A_plus;        /* A_plus_rel g_max */
    double A_minus;       /* B A_plus tau_plus / tau_minus */
} snn_topo_derived;
/* Fills *out with the values every topographic call uses for p (host only: needs no
 * GPU).  SNN_EINVAL for parameters the calls refuse. */
snn_status snn_topo_derive(const snn_topo_params* p, snn_topo_derived* out);

typedef struct {
    double p_form, sigma;            /* Gaussian formation probability */
    double p_elim_dep, p_elim_pot;   /* elimination probabilities (clamped to [0,1]) */
    double g_max;                    /* maximum conductance (Tab. 2F, 2G): a new synapse
                                        starts at g_max, and a synapse is depressed (uses
                                        p_elim_dep) iff g < g_theta = g_max / 2 */
    int32_t L;                       /* torus side used for distances */
    int32_t n_att;                   /* attempts per call */
    /* Optional event histograms for the connectivity-evolution analysis of Sec. 3.2
     * (eliminations and formations by spatial separation, Figs. 8-9 A-B): device int64
     * arrays of 2*(L/2)^2 + 1 bins, bin = squared torus distance d^2 between the
     * source and target grid positions.  Each elimination adds 1 to elim_d2[d^2], each
     * synapse created (not the overflowed ones) 1 to form_d2[d^2].  The library only
     * adds: the caller zeroes them and reads them (e.g. once per time bin).  NULL: not
     * recorded.  Squared distances keep the bins exact; unit-width distance bins are
     * floor(sqrt(d^2)) on the host. */
    int64_t* elim_d2;
    int64_t* form_d2;
} snn_topo_rewire;

/* Topographic network state (caller-owned device memory), N = L*L, Nw = ceil(N/32). */
typedef struct {
    float* V; float* gs; int32_t* ref;       /* [N] target sheet */
    float* x_src; float* x_tgt;              /* [N] presynaptic STDP traces */
    float* y; float* ydec;                   /* [N] postsynaptic trace, decayed copy */
    uint32_t* src_bits; uint32_t* tgt_bits;  /* [2][Nw] spikes, parity t & 1 */
    int64_t* acc;                            /* [N] conductance input (fixed point) */
} snn_topo_state;

/* Source sheet spikes of step t into src_bits[t&1] and x_src <- x_src e^{-dt/tau+} + s. */
snn_status snn_topo_input(const snn_topo_params* p, const snn_topo_state* st, uint64_t seed,
                          int64_t t, snn_stream stream);
/* Target sheet step t: g <- g e^{-dt/tau_s} + acc (acc consumed and zeroed); refractory
 * hold or exponential Euler; spikes into tgt_bits[t&1]; x_tgt, y, ydec traces. */
snn_status snn_topo_neurons(const snn_topo_params* p, const snn_topo_state* st, int64_t t,
                            snn_stream stream);
/* All-to-all STDP for step t on one projection: depression of rows whose pre spiked
 * (pre_bits) by A_- ydec[post], then potentiation of slots whose target spiked
 * (post_bits) by A_+ x_pre[row], clamped to [0, g_max]. */
snn_status snn_stdp_update(snn_ragged* r, const snn_topo_params* p, const uint32_t* pre_bits,
                           const uint32_t* post_bits, const float* x_pre, const float* ydec,
                           snn_stream stream);
/* One rewiring update (Sec. 2.1.3): n_att attempts to rows (purpose TOPO_ATT, counter
 * (rewire_idx, k/4, 0, 0), word k%4); per row a_r distinct candidates, the k-th being the
 * m-th unselected target, m = mulhi(Philox(TOPO_CAND; (rewire_idx, i, k, 0)), Q - k);
 * candidates with a synapse are eliminated iff R < thr(p_elim_dep if g < g_theta else
 * p_elim_pot), the others formed iff R < thr(p_form exp(-d^2/2 sigma^2)) with g = g_new,
 * R = Philox(TOPO_DRAW; (rewire_idx, i, j, 0)) word 0; rows compact stably; formations are
 * appended in ascending target order; a full row counts overflow.  F32 only.  The first
 * call with a new (L, p_form, sigma) builds the handle's formation-threshold table on
 * the host and copies it synchronously; later calls with the same parameters do not
 * synchronise. */
snn_status snn_rewire_topo(snn_ragged* r, const snn_topo_rewire* p, int64_t rewire_idx,
                           snn_rewire_stats* stats, snn_stream stream);
/* Run steps t0 .. t0+n_steps-1 of the full topographic network: input, propagation of
 * the previous step's spikes (ff and lateral), neurons, STDP on both projections and,
 * after every step with (t+1) % rewire_every == 0, snn_rewire_topo on ff then lateral
 * with rewire index (t+1)/rewire_every - 1.  Runs as one thread-block-cluster launch
 * per (up to) 1000 steps, with results identical to that sequence of per-step calls;
 * networks too large for one cluster use the per-step launches.  No host sync except
 * when a projection's formation-threshold table has to be (re)built. */
snn_status snn_topo_run(const snn_topo_params* p, const snn_topo_state* st, snn_ragged* ff,
                        snn_ragged* lat, const snn_topo_rewire* rw_ff, const snn_topo_rewire* rw_lat,
                        uint64_t input_seed, int32_t rewire_every, int64_t t0, int32_t n_steps,
                        snn_rewire_stats* stats_ff, snn_rewire_stats* stats_lat, snn_stream stream);

/* Connectivity profile of a topographic projection (the state analysed in Sec. 3.2,
 * Figs. 8-9 C-D): for every synapse i -> j of the L*L x L*L matrix, its displacement on
 * the torus dx = (x_j - x_i) mod L, dy = (y_j - y_i) mod L (x = index % L, y = index / L)
 * and its target.  Outputs (device arrays, each optional, zeroed by the call and then
 * filled):
 *   disp_count [L*L] int64: synapses with displacement (dx, dy) at dy*L + dx; divided by
 *              L*L it is the connection probability at that displacement (panel D);
 *   disp_wsum  [L*L] double: sum of their weights (mean weight = wsum / count; summed
 *              with atomics, so the rounding order varies between runs);
 *   in_degree  [L*L] int32: synapses onto each target (panel C; the out-degree of row i
 *              is row_len[i]).
 * F32 matrices with P = Q = L*L.  Asynchronous on `stream`; no allocation. */
snn_status snn_topo_connectivity(const snn_ragged* r, int32_t L, int64_t* disp_count, double* disp_wsum,
                                 int32_t* in_degree, snn_stream stream);

/* ==================================================================================
 * Test hook
 * ================================================================================== */
/* Failure-detection probe: one warp waits, with the library's bounded mbarrier wait (the
 * one the adjoint scan's bulk-copy stages use), for a barrier that completes only if
 * arrive != 0.  After `limit` polls (1 .. 2^24) the wait gives up and sets the timeout
 * flag in r's status word, so snn_ragged_status then returns SNN_ETIMEOUT; no copy is in
 * flight and nothing traps, so the context stays usable.  Asynchronous on `stream`. */
snn_status snn_test_wait_timeout(snn_ragged* r, int32_t arrive, int32_t limit, snn_stream stream);
/* out[k*4 + q] = word q of Philox4x64-10(key = (seed, purpose), counter = ctr[4k..4k+3])
 * for k < n; ctr and out are device arrays. */
snn_status snn_philox(uint64_t seed, uint64_t purpose, const uint64_t* ctr, int64_t n,
                      uint64_t* out, snn_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* SNNSP_H */
