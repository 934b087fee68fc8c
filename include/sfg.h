/*
 * sfg.h -- C ABI of the GB300 self-gravity library (libsfg.so).
 *
 * The library evaluates the self-gravity field of gas cells and sink
 * particles as the STARFORGE methods paper defines it (Grudic et al. 2021,
 * Sec. 2.2 "Gravity" and Sec. 2.2.1 "Softening"): an oct-tree over the
 * particles, Barnes-Hut opening angle theta = L/r (node side over distance to
 * the node centre of mass, Sec. 2.2), monopole + quadrupole node fields, and
 * per-pair M4 cubic-spline softening of compact support: the adaptive gas
 * softening S_i = H_i with the two kernels averaged for gas-gas pairs, and a
 * single kernel of support max(S_i, S_j) for any pair that involves a sink
 * (Sec. 2.2.1).  The field is evaluated only for the "active" particles of a
 * timestep bin (Sec. 2.3), and the library also provides the adjoint
 * (vector-Jacobian product) of that evaluation with the interaction lists
 * frozen, built from the softened tidal tensor T = -grad grad Phi of the same
 * kernel (Sec. 2.2).
 *
 * Conventions (every entry point):
 *   - All array pointers are DEVICE pointers unless stated otherwise, in
 *     row-major layout: positions are [n][3] float64 (x, y, z interleaved).
 *   - Calls are asynchronous and ordered on the CUDA stream passed as
 *     `stream` (a cudaStream_t; NULL = the legacy default stream), except
 *     sfg_build, which synchronizes `stream` once at its end to size the tree.
 *   - Inputs are owned by the caller and may be freed once the stream has
 *     passed the call.  sfg_build copies what the tree needs.  Outputs are
 *     allocated by the caller.
 *   - A tree must be used from one stream at a time (it keeps a workspace).
 *   - CUDA graphs: a tree allocates its grow-only workspaces on the first call
 *     of each kind (sfg_accel, sfg_accel_vjp, per-cloud timing) that needs
 *     them.  Make one such call eagerly before capturing a stream into a
 *     graph; a call that would allocate while its stream is being captured
 *     returns SFG_EINVAL instead (the memory would belong to the graph).
 *   - Return value: SFG_OK or an SFG_E* status.  Nothing aborts or exits.
 *     Errors that only the device can see (non-finite inputs, an index out
 *     of range, a traversal buffer overflow that survived its retry) are
 *     recorded in the tree's status word and returned by sfg_get_status,
 *     which synchronizes the tree's last stream.
 *   - Particle indices are int64 in [0, n); n must be < 2^31.
 */
#ifndef SFG_H
#define SFG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SFG_OK 0
#define SFG_EINVAL 1    /* bad argument: n <= 0, NULL pointer, h <= 0, m < 0, non-finite, index out of range */
#define SFG_ENOMEM 2    /* device allocation failed */
#define SFG_ECUDA 3     /* a CUDA runtime call or launch failed */
#define SFG_EOVERFLOW 4 /* a traversal buffer overflowed even after the automatic retry */
#define SFG_ETIMEOUT 5  /* a bounded device-side wait gave up */

typedef struct sfg_tree sfg_tree; /* opaque; owns its device memory */

/* Numerical and launch parameters of a tree. */
typedef struct sfg_params {
    double G;        /* gravitational constant multiplying every term */
    double theta;    /* maximum opening angle Theta of Sec. 2.2 (the paper uses 0.5); 0 = always open */
    int leaf_size;   /* N_leaf: a node with <= N_leaf particles (or at the 21st level) is a leaf; 1..256 */
    int group_size;  /* G_group: <= G_group active targets share one walk; 1..32 */
    int list_depth;  /* depth of the evaluation's shared-memory list buffer: the interaction-list
                        sources each active lane stages per chunk (1, 2 or 4; 0 = 1) */
    int quadrupole;  /* 1: monopole + quadrupole node fields; 0: monopole only (Sec. 2.2) */
    int precision;   /* 0: FP32 pair/multipole arithmetic on node-centred offsets, FP64
                        frame/moments/potential sums; 1: all-FP64 evaluation */
    int store_lists; /* 1: walk once per call into stored interaction lists (one walk that
                        stages each group's lists and places them, or, when they outgrow the
                        sizing hint, a sizes-first walk and a list-writing walk), evaluate
                        from them, and let the adjoint reuse the forward's lists when
                        called with the same active set;
                        0: every evaluation walks the tree itself.  Ignored (0) with
                        precision = 1 and while the stream is captured into a CUDA graph
                        (sizing the lists synchronizes the stream once). */
    /* Optional device allocator (stream-ordered).  NULL alloc => cudaMallocAsync. */
    void *(*alloc)(size_t bytes, void *stream, void *ctx);
    void (*free)(void *ptr, void *stream, void *ctx);
    void *alloc_ctx;
} sfg_params;

/* Summary of a tree and of the last sfg_accel / sfg_accel_vjp call. */
typedef struct sfg_stats {
    int64_t n;            /* particles */
    int64_t n_nodes;      /* tree nodes */
    int32_t depth;        /* deepest level (root = 0) */
    int32_t n_levels;     /* depth + 1 */
    double x0[3];         /* frame origin: per-axis minimum position */
    double L0;            /* root cube side: smallest power of two >= the largest extent */
    int64_t n_groups;     /* groups of the last call */
    int64_t n_targets;    /* distinct active particles of the last call */
    int64_t n_p2p;        /* particle-particle interactions of the last call (self excluded) */
    int64_t n_p2m;        /* particle-node interactions of the last call */
    int64_t n_overflow;   /* groups that needed the spill traversal buffer */
    int32_t n_clouds;     /* independent clouds in the tree (sfg_build_batch), 1 otherwise */
    int64_t n_launches;   /* kernels this tree has launched since it was built (build included) */
    /* with timing on (sfg_set_timing), milliseconds of the last call of each kind,
     * from CUDA events on the call's stream (0 when off) */
    float build_ms;       /* whole sfg_build */
    float fwd_ms;         /* whole sfg_accel */
    float fwd_walk_ms;    /* its evaluation launch (k_eval from stored lists, or the walking
                             evaluation when lists are off), after the list passes */
    float vjp_ms;         /* whole sfg_accel_vjp */
    float vjp_walk_ms;    /* its adjoint evaluation launch, likewise */
    int64_t n_p2p_newton; /* of n_p2p: pairs from stored Newtonian range lists (opened leaves wholly
                             outside both softening supports; 0 without stored lists) */
    int32_t list_walks;   /* walks the last stored-list build took: 1 = one pass (lists staged and
                             placed as walked), 2 = sizes first, then the lists (the first build
                             of the process, or one whose lists outgrew the sizing hint) */
} sfg_stats;

/* Fill *p with the defaults: G = 1, theta = 0.5, leaf_size = 16, group_size = 32,
 * quadrupole = 1, precision = 0, list_depth = 0, store_lists = 1, no allocator. */
void sfg_default_params(sfg_params *p);

/* Build the tree of n particles (Sec. 2.2: the oct-tree over every gas cell and
 * sink): frame, 63-bit Morton keys on a 2^21-per-axis grid, stable radix sort,
 * octree, FP64 node moments (mass, centre of mass, traceless quadrupole about
 * it), and the FP32 node/particle records of the walk.
 *   pos     [n][3] float64, device
 *   mass    [n]    float64 >= 0, device
 *   soft    [n]    float64 > 0, device: kernel radius of compact support (H for
 *                  gas, S_* for sinks, Sec. 2.2.1)
 *   is_sink [n]    uint8 (nonzero = sink particle), device, or NULL (all gas)
 *   params  host pointer, or NULL for the defaults; copied into the tree
 *   out     host pointer receiving the new tree (NULL on failure)
 * Synchronizes `stream` once (the node count sizes the tree).  Errors:
 * SFG_EINVAL (n <= 0, n >= 2^31, NULL pointer, bad params, non-finite or
 * out-of-domain inputs), SFG_ENOMEM, SFG_ECUDA. */
int sfg_build(const double *pos, const double *mass, const double *soft, const uint8_t *is_sink, int64_t n,
              const sfg_params *params, void *stream, sfg_tree **out);

/* Build one forest over an ensemble of independent clouds (no gravity acts
 * between clouds): cloud c is the particle range [offsets[c], offsets[c+1])
 * of the concatenated arrays, with its own frame and root; every later call
 * (sfg_accel, sfg_accel_vjp and the *_batch aliases below) solves all clouds
 * together in one walk launch, with particle indices over the concatenation.
 *   offsets [n_clouds + 1] int64, HOST: offsets[0] = 0, strictly increasing
 *           (no empty cloud), offsets[n_clouds] = n < 2^31; 1 <= n_clouds <= 65535
 * Other arguments and errors as sfg_build (which is the one-cloud case). */
int sfg_build_batch(const double *pos, const double *mass, const double *soft, const uint8_t *is_sink,
                    const int64_t *offsets, int n_clouds, const sfg_params *params, void *stream, sfg_tree **out);

/* Field at the active particles (Sec. 2.2, the active set of a timestep bin,
 * Sec. 2.3): for row k, the particle i = active_idx[k] gets
 *   accel[k][3] = g_i = -grad Phi (x_i)   and   phi[k] = Phi(x_i),
 * summing softened pair terms over the particles of opened leaves (self
 * excluded) and multipole terms over accepted nodes.
 *   active_idx [n_active] int64, device, or NULL for all particles in order;
 *              duplicates are allowed (rows are independent)
 *   accel      [n_active][3] float64, device, overwritten
 *   phi        [n_active]    float64, device, overwritten (may be NULL)
 * n_active == 0 is a no-op.  An index outside [0, n) is reported through
 * sfg_get_status as SFG_EINVAL and its row is left unwritten. */
int sfg_accel(sfg_tree *tree, const int64_t *active_idx, int64_t n_active, double *accel, double *phi,
              void *stream);

/* Field, potential and tidal tensor at the active particles (Sec. 2.2: the
 * tidal tensor T = -grad grad Phi is summed in the same pass and with the same
 * opening criterion as g; Sec. 2.2.1: pairs use spatial derivatives of the
 * same softened kernel with the same symmetrisation).  accel and phi are as
 * for sfg_accel; for row k
 *   tidal[k][6] = (T_xx, T_yy, T_zz, T_xy, T_xz, T_yz) at x_{active_idx[k]}:
 * each softened pair adds -G m_j [K I + (dK/dr / r) d d^T] (d = x_j - x_i,
 * a = G m_j K d), each accepted node the derivative of its monopole (+
 * quadrupole) field, so T is the derivative of accel with respect to the
 * target's own position with the lists fixed.  Sums are FP32 per lane and
 * per work item, written as float64.
 *   tidal [n_active][6] float64, device, overwritten
 * Always walks stored interaction lists (whatever store_lists says) and keeps
 * them for a following sfg_accel_vjp of the same active set.  Errors as for
 * sfg_accel, and SFG_EINVAL for a tree built with precision = 1 or while
 * `stream` is being captured into a CUDA graph (sizing the lists
 * synchronizes the stream). */
int sfg_accel_tidal(sfg_tree *tree, const int64_t *active_idx, int64_t n_active, double *accel, double *phi,
                    double *tidal, void *stream);

/* Relative (acceleration-based) opening criterion of Sec. 2.2, which the
 * paper applies together with the geometric rule: a node is accepted only if
 * its quadrupole-order error scale stays below a fraction alpha of the field
 * of the previous step,
 *   G M L^2 / r^4 <= alpha |g_prev,i|  for every target i of the group,
 * tested conservatively per group (r bounded below by the whole-cell gap
 * between the node's centre-of-mass cell and the group's box, |g_prev| by the
 * group's minimum) in fixed FP64 products.
 *   g_prev [n] float64, device: |g| of every particle (input order) from the
 *          previous step; copied (gathered into the sorted order), so it may
 *          be freed once the stream has passed the call.  NULL switches the
 *          criterion off.
 *   alpha  >= 0, finite (alpha = 0 opens every node of positive mass)
 * It applies to every following sfg_accel / sfg_accel_tidal / sfg_accel_vjp
 * walk of this tree; kept interaction lists are dropped.  Errors: SFG_EINVAL
 * (NULL tree, bad alpha), SFG_ENOMEM, SFG_ECUDA. */
int sfg_set_relative_criterion(sfg_tree *tree, const double *g_prev, double alpha, void *stream);

/* Field, potential and gravitational jerk j = dg/dt at the active particles
 * (Sec. 2.2: j is summed in the same pass and with the same opening
 * criterion as g; pairs use spatial derivatives of the same softened kernel
 * with the same symmetrisation, nodes their monopole contributions).  With
 * d = x_j - x_i and w = v_j - v_i, a pair adds
 *   G m_j [K w + (dK/dr / r) (d . w) d]      (a = G m_j K d),
 * an accepted node G M [w / r^3 - 3 (d . w) d / r^5] with d from the target
 * to its centre of mass and w from the target's velocity to the node's
 * mass-weighted velocity (FP64 sums, members in sorted order, children in
 * octant order).  accel and phi are as for sfg_accel.
 *   vel  [n][3] float64, device: every particle's velocity (input order)
 *   jerk [n_active][3] float64, device, overwritten
 * Sums are FP32 per lane and per work item.  Stored lists, precision and
 * capture rules and errors as for sfg_accel_tidal. */
int sfg_accel_jerk(sfg_tree *tree, const double *vel, const int64_t *active_idx, int64_t n_active, double *accel,
                   double *phi, double *jerk, void *stream);

/* Sink two-body timestep of Sec. 2.3 with its minima taken in the tree pass,
 * masses within an accepted node combined (the paper's sink criterion,
 * evaluated on a tree of the sinks alone):
 *   dt[k] = sqrt(eta) / (1 / t_c,min + 1 / t_dyn,min),
 *   t_c = sqrt(r^2 + eps^2) / |v_s' - v_s|,  t_dyn = sqrt((r^2 + eps^2)^{3/2} / (G (m_s + m_s'))),
 * minimised over the particles of opened leaves (eps = max(h_s, h_s') / 2.8,
 * the Plummer-equivalent softening) and the accepted nodes (total mass at the
 * centre of mass, mass-weighted velocity, eps = h_s / 2.8).  FP32 terms, FP64
 * output; +infinity when no other particle limits the step.
 *   vel [n][3] float64, device (input order); dt [n_active] float64, device;
 *   eta > 0 the tolerance parameter.
 * Stored lists, precision and capture rules and errors as for sfg_accel_tidal. */
int sfg_sink_timestep(sfg_tree *tree, const double *vel, const int64_t *active_idx, int64_t n_active, double eta,
                      double *dt, void *stream);

/* One step of the modified 4th-order Hermite integrator for sink particles
 * (Sec. 2.3, the predictor and corrector equations), with both field and
 * jerk evaluations done by the library on a tree of the n particles alone
 * (the paper's sinks-only pass; every particle is treated as a sink, so
 * every pair takes one kernel of support max(S_i, S_j), Sec. 2.2.1):
 *   a0, j0 at (pos, vel);
 *   x_p = pos + dt vel + dt^2/2 a0 + dt^3/6 j0,  v_p = vel + dt a0 + dt^2/2 j0;
 *   a1, j1 at (x_p, v_p);
 *   vel_out = vel + dt/2 (a1 + a0) + dt^2/12 (j0 - j1),
 *   pos_out = pos + dt/2 (vel_out + vel) + dt^2/12 (a0 - a1)
 * (the velocity is corrected first and the position uses it).  Field and
 * jerk are as sfg_accel_jerk computes them (FP32 terms, FP64 sums and
 * outputs); the predictor and corrector run in FP64.
 *   pos, vel  [n][3] float64, device: the state at the start of the step
 *   mass, soft [n] float64, device: masses and softening radii S_*
 *   params    as for sfg_build (G, theta, leaf and group size; precision must be 0), or NULL
 *   dt        the step (finite; the caller chooses it, e.g. from sfg_sink_timestep)
 *   pos_out, vel_out [n][3] float64, device, overwritten (may not alias pos or vel)
 * Builds two trees and frees them; allocates its temporaries with
 * cudaMallocAsync on `stream` and synchronizes it.  Errors: SFG_EINVAL (NULL
 * pointer, n <= 0 or >= 2^31, dt not finite, bad params, or an error the
 * device reported for the inputs), SFG_ENOMEM, SFG_ECUDA, SFG_EOVERFLOW,
 * SFG_ETIMEOUT. */
int sfg_hermite_step(const double *pos, const double *vel, const double *mass, const double *soft, int64_t n,
                     const sfg_params *params, double dt, double *pos_out, double *vel_out, void *stream);

/* Tidal timestep constraint of Sec. 2.3:
 *   dt[k] = sqrt(eta) * (|T_k|^2 / 6)^(-1/4),
 * |T| the Frobenius norm of the symmetric tensor given by its six components
 * (as sfg_accel_tidal writes them); +infinity where T = 0.
 *   tidal [n][6] float64, device;  dt [n] float64, device, overwritten;
 *   eta > 0 the tolerance parameter.
 * Errors: SFG_EINVAL (n < 0, NULL pointer with n > 0, eta <= 0 or not finite),
 * SFG_ECUDA. */
int sfg_tidal_timestep(const double *tidal, int64_t n, double eta, double *dt, void *stream);

/* Adjoint of sfg_accel with the interaction lists frozen (recomputed by the
 * same walk): with L = sum_k cot_a[k] . accel[k] + cot_phi[k] * phi[k],
 *   d_pos[n][3] = dL/dpos  and  d_mass[n] = dL/dmass
 * (original particle order, overwritten), including the dependence of node
 * moments on member positions and masses.  The softening radii are constants.
 * The adjoint always uses the FP32 pair/multipole arithmetic on node-centred
 * offsets (with FP64 node-gradient and particle-gradient accumulation), under
 * either precision setting of the tree.
 *   cot_a   [n_active][3] float64, device
 *   cot_phi [n_active]    float64, device, or NULL (zero)
 * Duplicate rows sum.  Errors as for sfg_accel. */
int sfg_accel_vjp(sfg_tree *tree, const int64_t *active_idx, int64_t n_active, const double *cot_a,
                  const double *cot_phi, double *d_pos, double *d_mass, void *stream);

/* Split the evaluation of one tree across `world` processes (one per GPU):
 * later sfg_accel, sfg_accel_vjp, sfg_accel_tidal, sfg_accel_jerk and
 * sfg_sink_timestep calls of this tree evaluate only share `rank` of the
 * groups of their active set -- the contiguous run of groups
 * [floor(ng rank / world), floor(ng (rank + 1) / world)) in Morton order,
 * ng the call's group count -- so that every group is evaluated by exactly
 * one process.  Rows of targets in other shares come out as zeros (+inf for
 * sfg_sink_timestep), and the adjoint's d_pos, d_mass hold this share's
 * part of the sums, so the sum over all processes of each output (one
 * all-reduce) is the unsplit result.  The paper's runs split the tree work
 * over MPI ranks by domain decomposition (Sec. 2.2); here every process
 * holds the whole tree (built from the same particles) and the split is
 * over groups of targets.  Interaction counts in sfg_get_stats cover this
 * share.  (rank, world) = (0, 1) evaluates everything (the default).
 * Errors: SFG_EINVAL (NULL tree, world < 1 or > 65536, rank outside [0, world)). */
int sfg_set_group_share(sfg_tree *tree, int rank, int world);

/* Turn per-phase CUDA-event timing of later calls on (1) or off (0).  Timing
 * records a few events per call on the call's stream; it does not synchronize. */
int sfg_set_timing(sfg_tree *tree, int on);

/* The same calls under the names of the ensemble interface (a batched tree
 * is an ordinary tree; these forward to sfg_accel / sfg_accel_vjp). */
int sfg_accel_batch(sfg_tree *tree, const int64_t *active_idx, int64_t n_active, double *accel, double *phi,
                    void *stream);
int sfg_accel_vjp_batch(sfg_tree *tree, const int64_t *active_idx, int64_t n_active, const double *cot_a,
                        const double *cot_phi, double *d_pos, double *d_mass, void *stream);

/* Per-cloud completion times of the last walk launches while timing was on:
 * fwd_ms[c] / vjp_ms[c] = milliseconds from the first warp start of the last
 * sfg_accel / sfg_accel_vjp walk launch to the end of cloud c's last work
 * item (0 if that call ran with timing off).  Host arrays of n_clouds
 * floats, either may be NULL.  Synchronizes. */
int sfg_cloud_times(sfg_tree *tree, float *fwd_ms, float *vjp_ms);

/* Statistics of the tree and of its last call (host pointer).  Synchronizes. */
int sfg_get_stats(sfg_tree *tree, sfg_stats *out);

/* Device-side status accumulated since the last call of this function
 * (SFG_OK if none); synchronizes the tree's last stream and clears it. */
int sfg_get_status(sfg_tree *tree);

/* Release the tree and all its device memory (synchronizes its last stream). */
void sfg_free(sfg_tree *tree);

/* Static string naming a status code. */
const char *sfg_status_string(int status);

/* Name of the CUDA runtime error behind the last SFG_ECUDA that a call of
 * this library returned on the calling thread ("cudaSuccess" if none).  The
 * compute entry points clear a non-sticky CUDA error left pending by earlier,
 * unrelated calls before they start, so SFG_ECUDA names an error of their own. */
const char *sfg_last_cuda_error(void);

/* ---- measurement ----
 * FP32 fused multiply-add throughput of the current device, measured: a
 * launch of FMA-only threads (8 independent chains each, 4 blocks of 256
 * threads per SM), timed with CUDA events on `stream` after a warm-up
 * launch.  The roofline of the evaluation kernels (bound by the FP32 pipes)
 * is taken against it.  *tflops receives 2 x FMAs / time in TFLOP/s and, if
 * ms is not NULL, *ms the timed launch's milliseconds.  Synchronizes the
 * stream.  SFG_EINVAL for a NULL tflops, SFG_ENOMEM, SFG_ECUDA. */
int sfg_fp32_peak(double *tflops, double *ms, void *stream);

/* ---- inspection (tests and tools; copies to HOST memory, synchronizing) ----
 * field ids and layouts:
 *   SFG_FIELD_KEYS      uint64 [n]        sorted Morton keys
 *   SFG_FIELD_ORDER     int32  [n]        sorted rank -> original index
 *   SFG_FIELD_NODE_INT  int32  [nn][16]   level, first, count, parent, child_first,
 *                                         nchild, lo[3], hi[3], cq[3], cloud
 *   SFG_FIELD_NODE_HQ   uint64 [nn]       ceil((h_max / cell)^2), capped at 2^62
 *   SFG_FIELD_NODE_F64  float64 [nn][11]  M, com[3], Q[6] (xx yy zz xy xz yz), h_max
 *   SFG_FIELD_FRAMES    float64 [n_clouds][4]  x0[3], L0 of every cloud
 *   SFG_FIELD_PARTICLE_F32 float32 [n][4] the evaluation's particle records, sorted:
 *                                         x - c_leaf (c_leaf = centre of the particle's
 *                                         leaf cell), m; each the FP32 rounding (to
 *                                         nearest, even) of the FP64 value
 *   SFG_FIELD_NODE_F32  float32 [nn][9]   the evaluation's node records: com - c_node,
 *                                         M, Q xx yy xy xz yz; roundings as above
 * `bytes` must equal the field's size.  With several clouds, node ids are
 * breadth-first over the whole forest (the roots are nodes 0..n_clouds-1). */
#define SFG_FIELD_FRAMES 6
#define SFG_FIELD_KEYS 1
#define SFG_FIELD_ORDER 2
#define SFG_FIELD_NODE_INT 3
#define SFG_FIELD_NODE_HQ 4
#define SFG_FIELD_NODE_F64 5
#define SFG_FIELD_PARTICLE_F32 7
#define SFG_FIELD_NODE_F32 8
int sfg_export(sfg_tree *tree, int field, void *host_dst, size_t bytes);

/* Interaction lists of every group for the given active set (same walk as
 * sfg_accel), copied to HOST memory.  First call with NULL arrays to get
 * *n_groups, *n_p2m_total and *n_p2p_total; then call again with
 *   groups [n_groups][4] int64: first target (rank in the sorted list of
 *          distinct active particles), target count, P2M list length, P2P
 *          list length (entries)
 *   p2m    [n_p2m_total] int32 accepted node ids, group after group
 *   p2p    [n_p2p_total] int32 node ids whose whole particle range is summed
 *          pair by pair: opened leaves, and internal nodes that lie entirely
 *          inside the group's softening reach (all their leaves would be
 *          opened), group after group
 * Each group's entries come in walk order. */
int sfg_debug_lists(sfg_tree *tree, const int64_t *active_idx, int64_t n_active, int64_t *n_groups,
                    int64_t *n_p2m_total, int64_t *n_p2p_total, int64_t *groups, int32_t *p2m, int32_t *p2p,
                    void *stream);

/* ---- allocation-free variant ----
 * The paper has no counterpart to this call; it serves callers that cannot
 * allocate device memory at call time, e.g. an application whose device
 * memory is entirely reserved up front by its own pool, or a latency-bound
 * loop that must not run cudaMalloc (which can block the host and serialize
 * work on the device).
 *
 * sfg_sort_keys_static computes what sfg_build computes first -- the frame,
 * the 63-bit Morton keys and their stable sort -- for n <= SFG_STATIC_MAX_N
 * particles without allocating anything:
 *   pos       [n][3] float64, device, finite, with a largest per-axis extent
 *             that is 0 or a normal double below 2^1023 (not checked: other
 *             inputs give unspecified keys, where sfg_build reports SFG_EINVAL)
 *   key_out   [n] uint64, device: the sorted keys (as SFG_FIELD_KEYS)
 *   order_out [n] int32, device: sorted rank -> original index (as SFG_FIELD_ORDER)
 * Temporary buffers live in one fixed array of 6,556,928 bytes (6.25 MiB) that every GPU
 * loading the library holds until the process exits.  The first call on a
 * device looks up that array's device address (make it before any stream
 * capture); later calls reuse it.  All calls share the array, so calls that
 * overlap on the GPU (different streams or threads) race: serialize them.
 * Returns SFG_EINVAL for NULL pointers, n <= 0 or n > SFG_STATIC_MAX_N, and
 * SFG_ECUDA if the address lookup or a launch fails. */
#define SFG_STATIC_MAX_N (1 << 19)
int sfg_sort_keys_static(const double *pos, int64_t n, uint64_t *key_out, int32_t *order_out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SFG_H */
