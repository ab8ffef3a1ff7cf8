/*
 * pfm.h -- C ABI of libpfm, a single-GPU (GB300, sm_103a) solver for the
 * pseudo-flow continuous max-flow method of Baxter, Rajchl, Yuan and Peters,
 * "A Proximal Bregman Projection Approach to Continuous Max-Flow Problems
 * Using Entropic Distances" (arXiv 1501.07844).
 *
 * What one iteration computes (Algorithm 1 for the Potts model, Algorithm 2
 * for DAG-structured and hierarchical models, Section 3):
 *   excess      d_L(x) = D_L(x) + div q_L(x) + sum_{P in L.P} w_(P,L) d_P(x)
 *               (Potts: d_L = D_L + div q_L)
 *   label prox  u_L <- u_L exp(-d_L / c) / sum_L' u_L' exp(-d_L' / c)
 *               over end-labels (Eq. potts_labelupdate, both forms)
 *   flow step   q_A <- Proj_{|q_A| <= S_A} (q_A - c tau grad g_A),
 *               g_A = sum_{L end-label} W_(A,L) u_L (Eq. potts_flowupdate and
 *               the DAG flow update of Section 3.3)
 * Discretisation (not fixed by the paper): unit grid, forward-difference
 * gradient that is zero at the last index of each axis, divergence = minus
 * its adjoint, capacity set the Euclidean ball (PFM_NORM_ISO) or the box
 * (PFM_NORM_ANISO).  The source S carries no flow and d_S = 0.
 *
 * Conventions for every entry point:
 *   - Spatial arrays are x fastest: index (z*ny + y)*nx + x; a 2-D problem
 *     has ndim = 2 and dims[2] = 1.
 *   - Per-label and per-node arrays are label-major: D and u are
 *     [n_leaf][z][y][x]; flows are [n_nodes][ndim][z][y][x] with component 0
 *     along x.  End-labels (nodes without children) are numbered in
 *     ascending node id.
 *   - "Host or device" pointers are copied with cudaMemcpyDefault (unified
 *     addressing), so either kind works; pinned host memory is fastest.
 *   - The library owns every device buffer of a problem.  Inputs are copied
 *     at the call; the caller may free them afterwards.  Outputs go to
 *     caller-owned memory.
 *   - Work is queued on the CUDA stream given at creation (NULL = the legacy
 *     default stream).  Entry points marked (sync) wait for that stream.
 *   - No entry point aborts or traps.  Failures return a status and set a
 *     thread-local message readable with pfm_last_error().  A CUDA error
 *     returns PFM_ECUDA; the problem should then be destroyed.
 */
#ifndef PFM_H
#define PFM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PFM_VERSION 1

/* Symbols of the C ABI are the only ones the shared library exports. */
#if defined(__GNUC__)
#define PFM_API __attribute__((visibility("default")))
#else
#define PFM_API
#endif

typedef enum {
    PFM_OK = 0,
    PFM_EINVAL = 1,         /* bad argument, size or parameter */
    PFM_EDAG = 2,           /* malformed label DAG */
    PFM_ENOMEM = 3,         /* device allocation failed */
    PFM_ECUDA = 4,          /* CUDA runtime or launch error */
    PFM_ENONFINITE = 5,     /* NaN or Inf in inputs, energy or dual */
    PFM_ETIMEOUT = 6,       /* a bounded device-side wait expired */
    PFM_ENOTCONVERGED = 7,  /* gap target not met within max_iters */
    PFM_EUNSUPPORTED = 8    /* valid request the library does not implement */
} pfm_status;

enum { PFM_NORM_ISO = 0, PFM_NORM_ANISO = 1 };

/* Which labelling the flow step differentiates.  NORMALISED: the normalised
 * u after the prox step (the gradient of the smoothed objective
 * Eq. potts_bregmanopt with respect to div q_L).  PAPER_LITERAL: the
 * unnormalised u exp(-d/c) as Algorithms 1 and 2 print it. */
enum { PFM_GRAD_NORMALISED = 0, PFM_GRAD_PAPER_LITERAL = 1 };

/* Storage type of the labelling u and the flows q (arithmetic is FP32;
 * D and S are always stored in FP32).  BF16 keeps FP32's exponent range
 * with 8 significant bits; F16 has 11 significant bits but its smallest
 * positive value is 2^-24, below which the multiplicative label update
 * would store an exact zero that never recovers: with F16 storage every
 * labelling value is stored as max(u, 2^-24) (a deviation from the method,
 * at most n_leaf * 2^-24 in the simplex sum), and flows saturate at the
 * largest finite F16, +-65504. */
enum { PFM_STORAGE_F32 = 0, PFM_STORAGE_BF16 = 1, PFM_STORAGE_F16 = 2 };

/* PFM_SCHEDULE_FUSED: one kernel per iteration, u and q double-buffered
 * (fewest bytes moved); operands are staged by TMA when the problem allows
 * it (Potts, <= 8 labels, row pitch a multiple of 16 bytes).
 * PFM_SCHEDULE_INPLACE: two kernels per iteration updating u and q in place
 * (fewest buffers: the paper's memory argument).
 * PFM_SCHEDULE_FUSED_PLAIN: the fused schedule without TMA staging (operands
 * loaded into registers), for comparison. */
enum { PFM_SCHEDULE_FUSED = 0, PFM_SCHEDULE_INPLACE = 1, PFM_SCHEDULE_FUSED_PLAIN = 2 };

typedef struct {
    double c;          /* entropic weight c > 0 (Eq. potts_bregmanopt) */
    double tau;        /* gradient step tau > 0; the applied step is c*tau */
    int norm;          /* PFM_NORM_* */
    int grad_source;   /* PFM_GRAD_* */
    int storage;       /* PFM_STORAGE_* */
    int schedule;      /* PFM_SCHEDULE_* */
    int check_every;   /* iterations between gap checks in pfm_run_to_gap */
    double gap_tol;    /* relative gap target (E - P) / |E| */
} pfm_params;

/* Problem description.  Nodes 0..n_nodes-1 are the non-source labels; edge e
 * goes from edge_parent[e] (-1 = the source S) to edge_child[e] with weight
 * edge_w[e] > 0 (w_(parent,child) of Eq. dagmf_original).  The Potts model is
 * the flat DAG (S -> every label, w = 1).  Requirements checked at creation
 * (PFM_EDAG otherwise): indices in range, no self loop or cycle, every node
 * has a parent, every end-label has path weight W_(S,L) = 1 (so that the
 * end-label simplex of Section 3.3 is the constraint u_S = 1).
 * Capacity of node A at voxel x: s_node[A] * S_field[x]; either may be NULL
 * (then 1); values must be finite and >= 0.  D must be finite.  Data terms
 * exist on end-labels only (Eq. dagmf_primal). */
typedef struct {
    int ndim;               /* 2 or 3 */
    int64_t dims[3];        /* nx, ny, nz (nz = 1 for ndim = 2) */
    int n_nodes;
    int n_edges;
    const int32_t* edge_parent;   /* host [n_edges] */
    const int32_t* edge_child;    /* host [n_edges] */
    const double* edge_w;         /* host [n_edges] */
    const float* D;               /* host or device [n_leaf][z][y][x] */
    const float* S_field;         /* host or device [z][y][x], or NULL */
    const float* s_node;          /* host [n_nodes], or NULL */
} pfm_desc;

typedef struct pfm_problem pfm_problem;

/* Library version (PFM_VERSION) and the last error message of this thread. */
PFM_API int pfm_version(void);
PFM_API const char* pfm_last_error(void);

/* Fills *p with defaults: c = 0.5, tau = 0.11, ISO, NORMALISED, F32, FUSED,
 * check_every = 10, gap_tol = 1e-4. */
PFM_API void pfm_params_default(pfm_params* p);

/* Host-only query (no GPU needed): device bytes and number of full-grid
 * buffers (one value per voxel each) that pfm_create would allocate.  The
 * device arrays store rows of nx values at a pitch of nx rounded up to a
 * multiple of 8 (every row starts on a 16-byte boundary for the TMA
 * kernels); the bytes include that padding.  Caller-side arrays are always
 * dense.  n_leaf_out may be NULL.  Returns PFM_EDAG / PFM_EINVAL like
 * pfm_create. */
PFM_API pfm_status pfm_footprint(const pfm_desc* desc, const pfm_params* params,
                         size_t* device_bytes, int64_t* n_grid_buffers, int* n_leaf_out);

/* Validates desc and params, allocates device state on the current device,
 * copies D and S, and initialises u_L = 1/#leaves, q = 0 (Algorithm 1 and
 * Algorithm 2, first line; q is not initialised by the paper and is read as
 * zero).  stream is a cudaStream_t (may be NULL).  (sync) */
PFM_API pfm_status pfm_create(const pfm_desc* desc, const pfm_params* params, void* stream,
                      pfm_problem** out);

/* Frees every device buffer of the problem (after a stream sync).  NULL ok. */
PFM_API void pfm_destroy(pfm_problem* pb);

/* Replaces D (and S_field when the problem has one; pass NULL otherwise),
 * host or device pointers, same shapes as at creation.  Does not reset u, q.
 * Asynchronous on the problem's stream. */
PFM_API pfm_status pfm_set_data(pfm_problem* pb, const float* D, const float* S_field);

/* Double-buffered data upload (no counterpart in the paper; for callers that
 * stream new data terms while the solver runs).  pfm_prefetch_data starts
 * copying D (and S_field, as for pfm_set_data) into a library-owned staging
 * buffer on a copy stream of its own and returns at once, so the copy
 * overlaps the iterations already queued; the caller keeps the source
 * buffers unchanged (pinned host memory for a truly asynchronous copy) until
 * pfm_commit_data.  The staged data is validated like pfm_set_data's, on the
 * copy stream.  pfm_commit_data makes the problem's stream wait for the copy
 * and puts the staged data in place: the staging buffers and the problem's
 * D / S trade places (no device work; the next prefetch waits for the work
 * queued before the commit, which still reads the old buffers), except for a
 * member of a batch, whose buffers the batch's kernel arguments hold, where
 * the staged data is copied into place on the problem's stream.  A failed
 * validation shows at the next call that checks the problem's flags.  A
 * second prefetch before the commit replaces the first; pfm_commit_data
 * without a prefetch returns PFM_EINVAL.  The staging buffers (D and S
 * sized) are allocated on the first prefetch and freed with the problem. */
PFM_API pfm_status pfm_prefetch_data(pfm_problem* pb, const float* D, const float* S_field);
PFM_API pfm_status pfm_commit_data(pfm_problem* pb);

/* u_L = 1/#leaves, q = 0, iteration counter = 0.  Asynchronous. */
PFM_API pfm_status pfm_reset(pfm_problem* pb);

/* Sets the entropic weight c and the step tau used by the following
 * iterations (c > 0, tau > 0; the applied flow step is c*tau).  Lowering c
 * between blocks of iterations is the continuation toward the c -> 0 limit
 * of Section 3.2, where the label update tends to the per-voxel argmin of
 * the excess and the smoothed objective to the pseudo-flow dual.  Problems
 * in a batch keep the batch's parameters. */
PFM_API pfm_status pfm_set_step(pfm_problem* pb, double c, double tau);

/* Queues n_iters >= 0 iterations (Algorithm 1 / Algorithm 2 loop body) on
 * the problem's stream.  Asynchronous; errors of the launches are reported
 * here, device-side non-finite values by the next pfm_energy. */
PFM_API pfm_status pfm_iterate(pfm_problem* pb, int n_iters);

/* Primal energy E(u) (Eq. potts_original / Eq. dagmf_original, inner-node
 * labellings u_A = sum_L W_(A,L) u_L, TV norm matching params.norm) and
 * pseudo-flow dual P(q) = sum_x min_L d_L(x) (Eq. potts_pseudo /
 * Eq. dagmf_pseudo), accumulated in FP64.  P <= E for every feasible pair
 * (weak duality).  (sync)  PFM_ENONFINITE if either is not finite. */
PFM_API pfm_status pfm_energy(pfm_problem* pb, double* primal, double* dual);

/* Runs n_iters >= 1 iterations and returns E and P (as pfm_energy) of the
 * state the LAST of them started from, i.e. after n_iters - 1 iterations.
 * On the TMA-staged fused path that reduction happens inside the last
 * iteration's kernel, which streams that state anyway (no extra pass);
 * otherwise a separate reduction is queued just before it.  (sync) */
PFM_API pfm_status pfm_iterate_energy(pfm_problem* pb, int n_iters, double* primal, double* dual);

/* Iterates in blocks of params.check_every (each block through
 * pfm_iterate_energy) until (E - P)/|E| <= gap_tol or max_iters iterations
 * were run; reports iterations run and the last gap.  The gap is that of
 * the state one iteration before the returned state.  Returns
 * PFM_ENOTCONVERGED (with valid outputs) if the target was missed.  (sync) */
PFM_API pfm_status pfm_run_to_gap(pfm_problem* pb, int max_iters, int* iters_done, double* rel_gap);

/* Copies of the state into caller memory (host or device).  (sync)
 *   labels: FP32 [n_leaf][z][y][x]
 *   argmax: int32 [z][y][x], index of the largest u_L (ties: lowest index)
 *   flows : FP32 [n_nodes][ndim][z][y][x] */
PFM_API pfm_status pfm_get_labels(pfm_problem* pb, float* dst);
PFM_API pfm_status pfm_get_argmax(pfm_problem* pb, int32_t* dst);
PFM_API pfm_status pfm_get_flows(pfm_problem* pb, float* dst);

/* Asynchronous copy of the state (u, q; either may be NULL) into DEVICE
 * memory, layouts as above, ordered on the problem's stream and not waited
 * for (no counterpart in the paper: it serves callers that keep many states
 * on the device, e.g. the recomputation of the adjoint).  Host pointers are
 * rejected with PFM_EINVAL. */
PFM_API pfm_status pfm_get_state_async(pfm_problem* pb, float* u_dst, float* q_dst);

/* Asynchronous thresholded read-back (no counterpart in the paper): the
 * argmax of the current labelling is formed on the problem's stream in a
 * library buffer and copied to dst (host, pinned for a truly asynchronous
 * copy, or device) on the library's copy stream, overlapping whatever is
 * queued next; pfm_readback_wait blocks until the last such copy has
 * landed.  A second call waits (on the device) for the previous copy before
 * reusing the buffer.  dst must stay valid until the wait. */
PFM_API pfm_status pfm_get_argmax_async(pfm_problem* pb, int32_t* dst);
PFM_API pfm_status pfm_readback_wait(pfm_problem* pb);

/* Overwrites the state from caller memory (host or device), same layouts as
 * the getters, converted to the storage type.  Flows are projected onto the
 * capacity set and the normal component at the last index of each axis is
 * set to zero (a feasible flow is stored unchanged).  Labellings must be
 * finite and >= 0 with a positive sum per voxel (PFM_EINVAL otherwise) and
 * are stored as given: the next label update normalises them, and a
 * labelling read with pfm_get_labels resumes bit for bit.  (sync) */
PFM_API pfm_status pfm_set_labels(pfm_problem* pb, const float* src);
PFM_API pfm_status pfm_set_flows(pfm_problem* pb, const float* src);

/* Checkpoint / resume as one caller-held blob (the paper's state between
 * iterations of Algorithms 1-3 is the pair (u, q); the blob adds what a
 * resumed run needs to continue exactly: the iteration counter and the
 * current c, tau, which continuation schedules change).  Layout: a
 * pfm_state_header of PFM_STATE_HEADER_BYTES bytes, then u and q in the
 * problem's STORAGE type (F32: 4 bytes, BF16: 2 bytes per value) as dense
 * arrays in the getters' layouts (u [n_leaf][z][y][x], then q
 * [n_nodes][ndim][z][y][x]) -- bit for bit what the solver holds.
 * pfm_get_state: with dst == NULL only writes the blob size to *size;
 * otherwise *size must be at least that size (PFM_EINVAL otherwise) and the
 * blob is written to dst (host or device memory).  (sync)
 * pfm_set_state: imports a blob written by pfm_get_state of a problem with
 * the same grid, n_leaf, n_nodes and storage (PFM_EINVAL on a size, magic,
 * version, shape or storage mismatch, before anything is changed): u and q
 * are copied bit for bit, the iteration counter, c and tau restored, so the
 * iterations that follow equal those the saved problem would have run.
 * The data terms D, S are not part of the state.  (sync) */
#define PFM_STATE_HEADER_BYTES 128
typedef struct {
    char magic[8];          /* "PFMSTATE" */
    int32_t version;        /* PFM_VERSION of the writer */
    int32_t storage;        /* PFM_STORAGE_* of u and q in the blob */
    int32_t ndim;
    int32_t n_leaf;
    int32_t n_nodes;
    int32_t reserved0;
    int64_t dims[3];        /* nx, ny, nz */
    int64_t iterations;     /* pfm_iterations_done at the save */
    double c, tau;          /* the step parameters in force at the save */
    uint8_t reserved[48];   /* zero */
} pfm_state_header;
PFM_API pfm_status pfm_get_state(pfm_problem* pb, void* dst, size_t* size);
PFM_API pfm_status pfm_set_state(pfm_problem* pb, const void* src, size_t size);

/* Problem shape queries. */
PFM_API pfm_status pfm_shape(const pfm_problem* pb, int* ndim, int64_t dims[3], int* n_leaf, int* n_nodes);

/* Kernel family pfm_iterate launches for this problem: "fused_tma"
 * (TMA-staged fused Potts iteration), "fused_tma_ishikawa",
 * "fused_tma_tree", "fused_tma_dag" (TMA-staged DAG iterations: Ishikawa
 * chain, two-level tree, general DAG), "fused" (register-staged fused
 * iteration), "inplace_tma" or "inplace" (two in-place kernels).  Static
 * string; "" for NULL. */
PFM_API const char* pfm_kernel_variant(const pfm_problem* pb);

/* Iterations run since creation or the last reset, and kernels this problem
 * has launched since creation (for launch accounting). */
PFM_API int64_t pfm_iterations_done(const pfm_problem* pb);
/* Failure-detection self-test: runs, on the problem's stream, one bounded
 * mbarrier wait of the kind every TMA pipeline uses (the same primitive with
 * a twentieth of the pipelines' cycle budget of about 2 s), on a barrier
 * nothing arrives on.  The wait gives up after its budget (about 0.1 s),
 * raises the timeout flag and the kernel returns; the call then restores the
 * problem's flags and returns PFM_ETIMEOUT (PFM_ECUDA if the wait did not
 * report).  The problem and the CUDA context stay usable.  Not part of the
 * paper's method. */
PFM_API pfm_status pfm_selftest_timeout(pfm_problem* pb);
PFM_API int64_t pfm_launch_count(const pfm_problem* pb);

/* Autotuner of the plane-marching kernels (the iteration kernels walk their
 * tile through a chunk of consecutive z-planes; one CTA per tile and chunk):
 * times trial_iters iterations (after one warm-up iteration) for each chunk
 * length in {4, 8, 16, 32, 64, 128} and the cost model's choice made at
 * create (all clamped to nz), keeps the fastest and writes it to *zc_out
 * (may be NULL).  The trials advance the state, so the problem is reset to
 * its initial state (as pfm_reset) afterwards: tune before pfm_set_labels /
 * pfm_set_flows.  Synchronises the stream.  Not part of the paper's method
 * (a launch-configuration search): the iterates u, q do not depend on the
 * chunk length (every voxel's arithmetic is the same), the energy's
 * summation order does. */
PFM_API pfm_status pfm_tune(pfm_problem* pb, int trial_iters, int* zc_out);
/* Sets the z-chunk length (zc >= 1, clamped to nz; PFM_EINVAL otherwise)
 * for the following launches; may reallocate the energy partials (and then
 * synchronises the stream).  pfm_chunk_length returns it (-1 for NULL). */
PFM_API pfm_status pfm_set_chunk_length(pfm_problem* pb, int zc);
PFM_API int pfm_chunk_length(const pfm_problem* pb);

/* Forces the kernel family of the fused schedule (a launch choice, not part
 * of the paper's method; the iterates agree to FP32 rounding across
 * families): "fused_tma" (Potts), "fused_tma_ishikawa" (Ishikawa chains),
 * "fused_tma_tree" (two-level label trees: source, inner nodes, end-labels),
 * "fused_tma_dag" (the general TMA-staged DAG kernel) or "fused" (the
 * register-staged kernel).  pfm_create picks the most specialised family the
 * problem allows; this call serves comparisons.  Resets the chunk length to
 * the cost model's choice for the family's tile.  PFM_EUNSUPPORTED if the
 * problem cannot run the family or uses the in-place schedule. */
PFM_API pfm_status pfm_select_kernel(pfm_problem* pb, const char* family);

/* Reverse-mode step of one Potts iteration (the paper has no gradient; this differentiates the unrolled iteration of
 * Algorithm 1, NORMALISED gradient source, ISO or ANISO, flat label set).
 * Given the forward input state (u_k, q_k) of an iteration, its output
 * labelling u_k1, and the adjoints (ubar_k1, qbar_k1) of its outputs
 * (u_k1, q_k1), writes the adjoints (ubar_k, qbar_k) of its inputs and
 * ADDS this iteration's contribution to Dbar (gradient w.r.t. D) and Sbar
 * (gradient w.r.t. S_field; ignored if the problem has no field).  All
 * buffers are caller-owned FP32 device memory in the getters' layouts;
 * ubar_k may alias ubar_k1 and qbar_k may alias qbar_k1; Dbar, Sbar and
 * work overlap no other argument.  work: device scratch of
 * (ndim + 1) * n_leaf * n floats.  D, S, c, tau, the capacities
 * and the norm are the problem's.  Asynchronous on the problem's stream.
 * PFM_EUNSUPPORTED for DAG problems, PAPER_LITERAL or more than 16 labels. */
PFM_API pfm_status pfm_adjoint_step(pfm_problem* pb, const float* u_k, const float* q_k, const float* u_k1,
                                    const float* ubar_k1, const float* qbar_k1, float* ubar_k, float* qbar_k,
                                    float* Dbar, float* Sbar, float* work);

/* The reverse-mode steps of n_steps consecutive iterations in one call (a
 * checkpoint segment): u_states is a host array of n_steps + 1 device
 * pointers (the labelling entering iteration 0, ..., leaving the last) and
 * q_states one of n_steps (the flows entering each iteration).  On entry
 * ubar / qbar hold the adjoints of the last iteration's outputs; on return
 * those of iteration 0's inputs.  Dbar and Sbar accumulate as with
 * pfm_adjoint_step, work as there.  Equal, bit for bit, to applying
 * pfm_adjoint_step to the iterations from the last to the first; the
 * divergence adjoint of each iteration and the projection adjoint of the one
 * before it share a pass, so the flow adjoints between iterations never go
 * to memory (2 n_steps + 1 launches instead of 3 n_steps).  Errors as
 * pfm_adjoint_step; PFM_EINVAL for n_steps < 1 or a NULL pointer. */
PFM_API pfm_status pfm_adjoint_steps(pfm_problem* pb, int n_steps, const float* const* u_states,
                                     const float* const* q_states, float* ubar, float* qbar, float* Dbar,
                                     float* Sbar, float* work);

/* ---- Batches (many independent problems, one persistent kernel per
 * iteration) ----
 * A batch advances n problems of possibly different grid sizes and label
 * DAGs in lockstep: each pfm_batch_iterate iteration is ONE launch of a
 * persistent kernel whose CTAs walk a work list of (member, x tile, y tile,
 * z chunk) items, and runs of 20 iterations are replayed from a captured
 * CUDA graph.  All members share params and ndim.  With the default
 * PFM_SCHEDULE_FUSED, batches with label DAGs run the TMA-staged DAG kernel
 * when every member fits it (at most 16 end-labels and nodes, three stages
 * within shared memory), else, and with PFM_SCHEDULE_FUSED_PLAIN, the
 * register-staged one; Potts-only batches run the register-staged kernel.
 * The state is always double-buffered.  Each member is an ordinary pfm_problem
 * owned by the batch: read it back with pfm_get_* through
 * pfm_batch_member, but advance it only through pfm_batch_iterate.  stream
 * NULL makes the batch create its own stream (capture needs one other than
 * the legacy default stream).  Errors of member creation are reported with
 * the member index. */
typedef struct pfm_batch pfm_batch;
PFM_API pfm_status pfm_batch_create(int n, const pfm_desc* descs, const pfm_params* params, void* stream,
                                    pfm_batch** out);
PFM_API void pfm_batch_destroy(pfm_batch* b);
PFM_API int pfm_batch_size(const pfm_batch* b);
/* "batched_tma_dag4", "batched_tma_dag" or "batched": the kernel family of
 * pfm_batch_iterate. */
PFM_API const char* pfm_batch_kernel_variant(const pfm_batch* b);
PFM_API pfm_status pfm_batch_member(pfm_batch* b, int index, pfm_problem** out);
/* n_iters >= 0 iterations of every member (asynchronous). */
PFM_API pfm_status pfm_batch_iterate(pfm_batch* b, int n_iters);
/* E and P of every member (arrays of pfm_batch_size entries), as
 * pfm_energy gives them; the four-inner-node batch reduces every member in
 * one launch over its work items (the members' sums agree with pfm_energy's
 * up to their order).  Returns the first member error.  (sync) */
PFM_API pfm_status pfm_batch_energy(pfm_batch* b, double* primal, double* dual);
/* Autotuner: times trial_iters iterations for each z-chunk length in
 * {8, 16, 32, 64} and persistent grid sizes (resident CTAs, twice that, one
 * CTA per item), keeps the fastest, then RESETS every member to the initial
 * state (u = 1/#leaves, q = 0).  Reports the choice.  (sync) */
PFM_API pfm_status pfm_batch_tune(pfm_batch* b, int trial_iters, int* zc_out, int* grid_out);
PFM_API int64_t pfm_batch_launch_count(const pfm_batch* b);

/* ---- Explicit-flow ("full-flow") solver, the comparison path ----
 * The augmented-Lagrangian continuous max-flow of the Potts model with every
 * flow stored (source flow p_S, sink flows p_L, spatial flows q_L, labels as
 * multipliers u_L): the primal of Section 3.2 and the formulation the
 * pseudo-flow method replaces.  One iteration: f_L = u_L - gamma G_L with
 * G_L = div q_L - p_S + p_L; q_L <- Proj(q_L - step grad f_L);
 * p_L <- min(D_L, p_S - div q_L + u_L/gamma);
 * p_S <- (sum_L (div q_L + p_L - u_L/gamma) + 1/gamma)/#L;
 * u_L <- u_L - gamma G_L.  Potts problems (flat label set), FP32.  Kept to
 * measure the paper's memory and time claims on the same GPU.
 * pfm_alm_energy reports E(u) and P(q) as pfm_energy does for the current
 * (u, q), and flow = sum_x p_S, the primal objective. */
typedef struct pfm_alm pfm_alm;
PFM_API pfm_status pfm_alm_footprint(const pfm_desc* desc, size_t* device_bytes, int64_t* n_grid_buffers);
PFM_API pfm_status pfm_alm_create(const pfm_desc* desc, double gamma, double step, int norm, void* stream,
                                  pfm_alm** out);
PFM_API void pfm_alm_destroy(pfm_alm* m);
PFM_API pfm_status pfm_alm_iterate(pfm_alm* m, int n_iters);
PFM_API pfm_status pfm_alm_energy(pfm_alm* m, double* primal, double* dual, double* flow);
PFM_API pfm_status pfm_alm_get_labels(pfm_alm* m, float* dst);
PFM_API int64_t pfm_alm_iterations_done(const pfm_alm* m);

/* Allocation-free energy evaluation.  The paper has no counterpart: this is
 * a service for callers that cannot call cudaMalloc -- code whose device
 * memory belongs to an outer allocator that has already claimed the budget
 * (a framework's caching allocator, a plugin host), or latency-critical
 * loops where an allocation, which can synchronise the device, is not
 * acceptable.  It computes what pfm_energy computes for a Potts problem
 * (flat label set), but on caller-held FP32 device buffers and without
 * allocating or freeing anything:
 *   u  [n_labels][z][y][x], q [n_labels][ndim][z][y][x], D [n_labels][z][y][x],
 *   S_field [z][y][x] or NULL (device); s_label [n_labels] or NULL (host);
 *   out: device double[2] receiving (E, P); norm: PFM_NORM_*.
 * The per-block partial sums live in a fixed 1 MiB device array compiled
 * into the library (held on every GPU that loads it until the process
 * exits), so the grid may have at most PFM_NOALLOC_MAX_VOXELS voxels;
 * larger grids are rejected with PFM_EINVAL.  Nothing in the array needs to
 * start at zero: each call overwrites the partials it reads.  Every call on
 * a device shares that array, so calls that overlap on the GPU (different
 * streams, or threads) race and give wrong results; serialise them.  The
 * first call on each device looks up the array's device address (with that
 * device current) and keeps it for the life of the process; make that first
 * call before any stream capture, and do not call this entry point after
 * cudaDeviceReset or anything else that destroys the device's primary
 * context (the kept address is then stale).
 * Asynchronous on `stream` (a cudaStream_t, NULL = legacy default): the
 * status covers the arguments and the launches only, so a non-finite E or P
 * is not reported as PFM_ENONFINITE -- it appears as NaN or Inf in out. */
#define PFM_NOALLOC_MAX_VOXELS 16777216LL
PFM_API pfm_status pfm_potts_energy_noalloc(int ndim, const int64_t dims[3], int n_labels, const float* u,
                                            const float* q, const float* D, const float* S_field,
                                            const float* s_label, int norm, double* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PFM_H */
