/*
 * bg.h -- C-ABI of libbg.so: batched Berends-Giele recursion for
 * colour-ordered n-gluon tree amplitudes on GB300 (sm_103a).
 *
 * Method: arXiv:2502.07060.  Sec. 2.2 defines the off-shell currents
 *   J(i,j) = (-i / P_{i,j}^2) [ sum V3(P_A,P_B) J_A J_B + sum V4 J_A J_B J_C ],
 * the three- and four-gluon vertices V3, V4 and the range momenta
 * P_{i,j} = k_i + ... + k_j; the amplitude is the (n-1)-leg current with its
 * propagator removed, contracted with the last polarisation.  Sec. 2.3 fixes
 * the d-dimensional setting (momenta in d dimensions, states embedded by zero
 * padding, mostly-minus metric); Sec. 3 the number types (F_p with p < 2^31,
 * complex double) and the parallelisation along the event dimension; Sec. 3.1
 * the alternating metric diag(1,-1,1,-1,...).
 *
 * Value returned for each point and state assignment:
 *     A = eps_n . R_top,     R_top = i^-1 x (bracket of the (n-1)-leg current)
 * i.e. the paper's amplitude divided by i (no factor of i is needed, so the
 * same code serves p = 3 mod 4).  With the states eps1/eps2 of Sec. 2.3,
 * A(1-,2-,3+..n+) = (-1)^n 2^(n-3) <12>^4 / (<12><23>...<n1>).
 *
 * Conventions: all momenta outgoing, sum_i k_i = 0; array leg index l <-> leg
 * l+1 in colour order; leg n (index n-1) is the contracted leg.  F_p values are
 * canonical residues in [0, p) stored as uint32; complex values are FP64
 * (re, im) pairs (16 bytes, CUDA double2 / torch.complex128).
 *
 * Ownership: the caller owns every buffer passed to bg_eval; bg_eval allocates
 * nothing.  A plan holds host memory and, when n_assign > 1, one small device
 * copy of the state-assignment table, made on the device current at
 * bg_plan_create and freed by bg_plan_destroy.
 *
 * Errors: every entry point returns a bg_status.  Argument errors are detected
 * on the host before any launch (BG_ERR_INVALID_ARG / BG_ERR_UNSUPPORTED) and
 * leave all buffers untouched; CUDA launch errors return BG_ERR_CUDA.
 * Data-dependent failures never trap: a singular propagator (P_{i,j}^2 = 0 for
 * an internal range) sets status[e] = 1 and out = 0 for that point.  A library
 * built with BG_CHECKED also tests each point's inputs against the
 * preconditions of bg_eval and sets status[e] = 2 and out = 0 for a point
 * that breaks one.
 * bg_last_error() returns a thread-local message for the last failure.
 */
#ifndef BG_H
#define BG_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BG_VERSION 3

typedef enum {
    BG_OK = 0,
    BG_ERR_INVALID_ARG = 1,   /* null pointer, size or parameter out of range  */
    BG_ERR_UNSUPPORTED = 2,   /* valid request this build has no kernel for    */
    BG_ERR_NOMEM = 3,         /* host or device allocation failed              */
    BG_ERR_CUDA = 4,          /* CUDA runtime error (launch, device mismatch)  */
    BG_ERR_TIMEOUT = 5,       /* serving: the wait's deadline passed           */
    BG_ERR_BUSY = 6           /* serving: the server is shutting down          */
} bg_status;

typedef enum {
    BG_FIELD_C64 = 0,         /* complex FP64 (Sec. 3, double precision)        */
    BG_FIELD_FP = 1,          /* prime field F_p, odd prime p < 2^31 (Sec. 3)  */
    BG_FIELD_C64_REAL = 2     /* complex FP64 with REAL momenta: the physical
                                 phase-space points of Sec. 3.  Momenta are
                                 double [E][n][d]; polarisations and amplitudes
                                 are double2 as for BG_FIELD_C64.  Same values
                                 as BG_FIELD_C64 on momenta with zero imaginary
                                 part, with fewer FP64 operations.             */
} bg_field;

typedef enum {
    BG_METRIC_MOSTLY_MINUS = 0,   /* diag(+,-,...,-)      (Sec. 2.3)           */
    BG_METRIC_ALTERNATING = 1     /* diag(+,-,+,-,...)    (Sec. 3.1)           */
} bg_metric;

typedef struct bg_plan bg_plan;   /* opaque; immutable after creation; may be
                                     shared by threads and streams            */

/*
 * bg_plan_create -- validate and fix one (n, d, D_s, field, p, metric, states)
 * configuration.  Host-side work, plus one device copy of `assign` when
 * n_assign > 1.
 *
 *   n        number of gluons, 4 <= n <= 12
 *   d        momentum dimension, 4 <= d <= 8 (Sec. 2.3)
 *   D_s      polarisation dimension, d <= D_s <= 8 (zero-padding embedding)
 *   field    BG_FIELD_FP, BG_FIELD_C64 or BG_FIELD_C64_REAL
 *   p        the prime for BG_FIELD_FP (odd prime, 3 <= p < 2^31, checked by
 *            a deterministic Miller-Rabin test); must be 0 for the complex
 *            fields
 *   metric   BG_METRIC_*
 *   n_states S >= 1: states supplied per leg (eps layout [E][n][S][D_s])
 *   n_assign H >= 1: state assignments evaluated per point (out [E][H]);
 *            H * n <= 2^20
 *   assign   host array [H][n] of state indices < S, copied by the call; or
 *            NULL with H == 1 (every leg uses state 0); or NULL with
 *            H == S^n, S >= 2: every assignment, leg l taking state
 *            (h / S^l) mod S in output column h.  That form evaluates all
 *            assignments of a point in one recursion whose sub-currents are
 *            shared between the assignments that agree on their legs (one
 *            warp per point); bg_eval_noalloc and bg_batch_* reject it.
 *   out      receives the plan
 */
bg_status bg_plan_create(int n, int d, int D_s, bg_field field, uint32_t p,
                         bg_metric metric, int n_states, int n_assign,
                         const uint8_t* assign, bg_plan** out);

/*
 * bg_plan_create_product -- a plan over every assignment of a product of
 * per-leg state sets: leg l takes states 0 .. states_per_leg[l]-1 (of the
 * n_states slots per leg in eps).  H = prod states_per_leg; output column
 * h = sum_l s_l * prod_{l' < l} states_per_leg[l'] (leg 0 fastest).  All
 * assignments of a point are evaluated in one recursion whose sub-currents
 * are shared between the assignments that agree on their legs (Sec. 2.2
 * memoisation carried across assignments): the helicity sums of Sec. 2.3
 * (all legs two states) and the cut trees of Sec. 2.1 (only the internal
 * legs with several states; see bg_cut_trace).  1 <= states_per_leg[l] <=
 * n_states <= 255, H * n <= 2^20.  Other arguments and errors as
 * bg_plan_create; bg_eval_noalloc and bg_batch_* reject such plans.
 */
bg_status bg_plan_create_product(int n, int d, int D_s, bg_field field, uint32_t p,
                                 bg_metric metric, int n_states,
                                 const uint8_t* states_per_leg, bg_plan** out);

/*
 * bg_plan_create_mixed -- a plan whose legs are partly four-dimensional: the
 * loop-level situation of Sec. 2.3, where only some external states are
 * d-dimensional and the others are four-dimensional states zero-padded into
 * d (resp. D_s) dimensions.  Bit l of four_dim_legs marks leg l (array index
 * l) as four-dimensional: its momentum components 4..d-1 and polarisation
 * components 4..D_s-1 are zero (precondition, not checked on the device).
 * A current whose range holds only such legs lies in the first four
 * components (the vertices of Sec. 2.2 combine currents and momenta
 * linearly), so it is computed with four components instead of D_s -- the
 * specialised four-dimensional recursion the paper leaves for future work.
 * The values are those bg_plan_create gives on the same inputs (identical
 * over F_p: only products with exact zeros are skipped).
 *   four_dim_legs  bits 0..n-1 (higher bits: BG_ERR_INVALID_ARG); 0 gives the
 *                  ordinary plan
 *   assign         an explicit [H][n] table or NULL with H == 1; the
 *                  all-assignment form (NULL with H > 1) is BG_ERR_UNSUPPORTED
 * Other arguments and errors as bg_plan_create.  bg_batch_* evaluates such a
 * plan at full width (same values).
 */
bg_status bg_plan_create_mixed(int n, int d, int D_s, bg_field field, uint32_t p,
                               bg_metric metric, int n_states, int n_assign,
                               const uint8_t* assign, uint32_t four_dim_legs,
                               bg_plan** out);

/* bg_plan_destroy -- free a plan (NULL is accepted).  No kernel of this plan
 * may still be running. */
bg_status bg_plan_destroy(bg_plan* plan);

/*
 * bg_workspace_size -- device workspace bytes bg_eval needs for E points
 * (0 when the plan's kernel keeps its current table in shared memory, or when
 * the batch is small enough for the lane-group kernel described at bg_eval).
 * The size is at most the value for E = INT64_MAX and is independent of E
 * once E exceeds the number of resident threads.
 */
bg_status bg_workspace_size(const bg_plan* plan, int64_t E, size_t* bytes);

/*
 * bg_eval -- evaluate E points on `stream` (asynchronous, one kernel launch;
 * the results are valid once the stream reaches the call).  The data-parallel
 * evaluation of Sec. 3: one independent recursion (Sec. 2.2) per point and
 * state assignment.  Large batches run one work item (point x assignment)
 * per thread; small ones -- up to 16 (complex) or 24 (F_p, n >= 7) work
 * items per SM or half a resident wave of the lane kernel, whichever is
 * larger: bg_plan_describe's lanes_max_items -- run each item on a
 * group of 4 or 8 lanes, one vector component per lane, which shortens the
 * call when most of the GPU would otherwise idle (the flat part of the
 * time-against-points curve of Sec. 3.2); the smallest -- up to
 * team_max_items, about 5 (F_p) or n - 5 (complex) items per warp scheduler
 * -- on a team of the groups of one warp, which evaluate the ranges of each
 * length in parallel.  All give the same F_p residues; complex results agree
 * to rounding (the two lane forms bit for bit).  The environment variable
 * BG_LANES=0 (never), 1 (always, one item per group) or 2 (always, one item
 * per team) read at plan creation overrides the choice.
 * bg_eval_host and bg_eval_noalloc take the same kernel as bg_eval for the
 * same batch (bg_eval_host chooses by the whole batch, not by chunk).
 *
 *   E          number of phase-space points, E >= 0 (E == 0: no launch)
 *   momenta    device [E][n][d]: uint32 residues (FP), double2 (C64) or
 *              double (C64_REAL)
 *   eps        device [E][n][S][D_s]: uint32 (FP) or double2 (complex
 *              fields) (S = n_states)
 *   out        device [E][H]: uint32 in [0,p) (FP) or double2 (complex)
 *   status     device [E] uint8 or NULL: 0 ok, 1 singular propagator,
 *              2 precondition broken (checked builds only, see below)
 *   workspace  device buffer of >= bg_workspace_size(plan, E) bytes, 256-byte
 *              aligned, or NULL when that size is 0; concurrent calls need
 *              distinct workspaces.  Scratch: its contents are undefined after
 *              the call (the kernel drops its dead lines from L2 unwritten)
 *   stream     CUDA stream (0 = legacy default stream)
 *
 * Buffers must be on the device that is current at the call, and momenta,
 * eps and out must be aligned to their element size.
 *
 * Preconditions of the inputs (Sec. 2.2: currents of on-shell legs, momentum
 * conservation imposed at the amplitude): canonical F_p residues (< p),
 * sum k = 0, k_i^2 = 0, and eps_i . k_i = 0 for every state slot of every
 * leg.  The kernels use the current conservation these imply (P_X . J_X = 0
 * for every internal current, so the three-gluon coefficients are formed
 * with the range momentum).  The ordinary build does not test them: on inputs
 * that break them the results are unspecified (non-canonical F_p states can
 * also overflow the kernels' unreduced sums), though every access stays
 * inside the caller's buffers.  A build with BG_CHECKED tests every point
 * (exactly over F_p; for the complex fields within 1e-8 of the point's
 * momentum scale) and reports a point that breaks one with status 2 and
 * amplitude 0.
 */
bg_status bg_eval(const bg_plan* plan, int64_t E, const void* momenta,
                  const void* eps, void* out, uint8_t* status,
                  void* workspace, size_t workspace_bytes, cudaStream_t stream);

/*
 * bg_host_staging_size -- device staging bytes that bg_eval_host needs when
 * it moves the batch in chunks of `chunk` points (two input/output slots plus
 * the kernel workspace).
 */
bg_status bg_host_staging_size(const bg_plan* plan, int64_t chunk, size_t* bytes);

/*
 * bg_eval_host -- evaluate E points whose inputs and outputs live in HOST
 * memory (the data-parallel evaluation of Sec. 3 with the host-device
 * transfers included).  The batch moves in chunks of `chunk` points through
 * two staging slots in the caller's device buffer `staging` (>=
 * bg_host_staging_size bytes, 256-byte aligned): the copy of chunk c+1 to the
 * device, the kernel on chunk c and the copy of chunk c-1 back to the host
 * overlap on separate streams.  When all four host buffers are page-locked
 * and mapped into the device's address space (cudaHostAlloc/cudaMallocHost
 * under unified addressing) and the batch's arithmetic per point hides the
 * host-link traffic -- batches of at most 64 MiB of host data, or heavier
 * ones such as complex FP64 at n = 8 -- one kernel instead reads the inputs
 * and writes the results in place, with no copies and the workspace at the
 * start of `staging`; light, large batches (F_p) keep the copies, which move
 * data faster than the kernels' scattered loads.  The rate of those loads
 * over the host link is measured once per device, on the first such batch
 * larger than 64 MiB (a probe kernel reads 32 MiB of page-locked memory;
 * freeing it waits for the device, so that first call may wait for work
 * already queued).  Results are identical on both paths.  Asynchronous: the
 * host buffers hold the results once `stream` reaches the call.  Host buffers
 * should be page-locked (pageable memory works but the copies serialise).
 *
 *   momenta, eps  host arrays with the layouts of bg_eval
 *   out, status   host arrays [E][H] and [E] (status is required here)
 *   chunk         points per chunk, >= 1
 * Returns BG_ERR_INVALID_ARG for device pointers in place of host buffers, a
 * too small or misaligned staging buffer, or E < 0; BG_ERR_CUDA when a copy
 * or launch cannot be enqueued -- such a call returns after the copies it had
 * already enqueued have finished, and the contents of out and status are then
 * unspecified.  Calls from several host threads are serialised while they
 * enqueue.
 */
bg_status bg_eval_host(const bg_plan* plan, int64_t E, const void* momenta,
                       const void* eps, void* out, uint8_t* status, int64_t chunk,
                       void* staging, size_t staging_bytes, cudaStream_t stream);

/*
 * bg_eval_noalloc -- the same evaluation as bg_eval, for callers that cannot
 * allocate device memory: a framework that owns the device-memory budget
 * through its own allocator, a latency-critical loop that cannot afford the
 * implicit synchronisation of cudaMalloc, or code running where CUDA
 * allocation calls are not permitted.  The paper has no counterpart; this is
 * an interface convenience of this library.
 *
 * The call allocates nothing.  Its scratch table is a statically sized
 * device array of 64 MiB inside libbg.so, present on every device that loads
 * the library until the process exits.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress, with that device
 * current); make that first call before any stream capture.  The address is
 * kept for the life of the process, so it goes stale if the device's primary
 * context is torn down (cudaDeviceReset): do not call this entry point after
 * such a reset in the same process.  All calls share the array: calls whose
 * kernels overlap on the GPU race, so order them on one stream.  Nothing in
 * the array needs to start at zero.
 *
 *   plan, E, momenta, eps, out, status, stream: as for bg_eval (buffers on
 *   the current device, caller-owned).  Returns BG_ERR_INVALID_ARG when
 *   E * n_assign exceeds 2^40 work items, BG_ERR_UNSUPPORTED when one thread
 *   block's table would not fit in the 64 MiB array; fewer blocks run at once
 *   than with bg_eval when the array limits residency.
 */
bg_status bg_eval_noalloc(const bg_plan* plan, int64_t E, const void* momenta,
                          const void* eps, void* out, uint8_t* status,
                          cudaStream_t stream);

/*
 * Uneven batches: groups of points with different n, d, D_s, metric and
 * number type evaluated by ONE CUDA-graph launch (the data-parallel method of
 * Sec. 3 over a mixed workload; Sec. 3.2 notes that the per-configuration
 * launch overhead dominates small batches).  The groups are ordered by cost,
 * cut into tiles and consumed by two persistent kernels (F_p and complex)
 * that run as parallel branches of the graph.
 */
typedef struct {
    const bg_plan* plan;      /* the group's configuration (n, d, D_s, field, p, ...) */
    int64_t E;                /* points in the group (0: group skipped)           */
    const void* momenta;      /* device buffers with the layouts of bg_eval       */
    const void* eps;
    void* out;
    uint8_t* status;          /* may be NULL                                       */
} bg_group;

typedef struct {
    int tile_points;          /* work items per tile; 0 = 1024                     */
    int fp_blocks_per_sm;     /* residency cap of the F_p kernel; 0 = all that fit.
                                 The F_p kernel has two builds: caps 1-2 take the
                                 one built for few resident blocks (up to 255
                                 registers, two blocks fit), 0 and 3-4 the one
                                 built for four (at most 128 registers)         */
    int c64_blocks_per_sm;    /* residency cap of the complex kernel; 0 = all      */
    int lanes_max_items;      /* groups of at most this many work items run one
                                 item per group of 4 or 8 lanes (the lane-group
                                 body of bg_eval's small batches); 0 = none       */
} bg_batch_config;

typedef struct bg_batch bg_batch;   /* opaque: tables in the workspace + a graph */

/* bg_batch_workspace_size -- device bytes the batch needs (group and tile
 * tables, tile counters, table scratch).  cfg == NULL: the largest size any
 * bg_batch_autotune candidate needs. */
bg_status bg_batch_workspace_size(const bg_group* groups, int n_groups,
                                  const bg_batch_config* cfg, size_t* bytes);

/* bg_batch_create -- order, tile, upload the tables into `workspace` (device,
 * 256-byte aligned, owned by the batch until bg_batch_destroy) and capture the
 * graph.  The groups' buffers are bound into the graph: each launch evaluates
 * whatever they hold.  cfg may be NULL: 256-point tiles, lane groups for
 * groups of at most 2048 work items, and the F_p kernel held to 2 blocks per
 * SM when most of its F_p work items run on lane groups (otherwise all that
 * fit).  Synchronous. */
bg_status bg_batch_create(const bg_group* groups, int n_groups, const bg_batch_config* cfg,
                          void* workspace, size_t workspace_bytes, bg_batch** out);

/* bg_batch_launch -- one graph launch on `stream` (asynchronous). */
bg_status bg_batch_launch(const bg_batch* batch, cudaStream_t stream);

/* bg_batch_describe -- one-line summary (groups, tiles, grids, workspace). */
bg_status bg_batch_describe(const bg_batch* batch, char* buf, size_t len);

/* bg_batch_destroy -- free the batch (not the workspace); NULL accepted. */
bg_status bg_batch_destroy(bg_batch* batch);

/* bg_batch_autotune -- time every candidate configuration (tile size x
 * residency caps of the two kernels, which also choose the F_p kernel's
 * build, x lane groups for small groups or not) on this batch, `reps`
 * launches each on `stream`, and return the fastest in *best (and its time
 * per launch in *best_ms if non-NULL).  Needs bg_batch_workspace_size(groups, n, NULL)
 * bytes of workspace.  Synchronises the stream.  When the environment
 * variable BG_AUTOTUNE_CACHE names a file, a result stored there for the same
 * device, library version and group mix (each group's configuration and its
 * size rounded up to a power of two) is returned without timing, and a newly
 * timed result is appended to the file.  Setting BG_LOG (to anything but 0)
 * logs plan choices and autotune results to stderr. */
bg_status bg_batch_autotune(const bg_group* groups, int n_groups, void* workspace,
                            size_t workspace_bytes, int reps, cudaStream_t stream,
                            bg_batch_config* best, double* best_ms);

/*
 * Serving: evaluation requests of mixed size and configuration, submitted
 * from host threads (the request stream of a finite-field reconstruction or
 * Monte Carlo consumer, Sec. 1) and run with continuous admission.
 *
 * bg_serve_create allocates one device arena of `budget_bytes` on the current
 * device and starts a dispatcher thread with `max_inflight` stream slots
 * (1..64).  A submitted request is admitted as soon as a slot and arena
 * memory for its inputs, outputs and workspace are free -- while earlier
 * requests are still running -- so the copies and kernels of concurrent
 * requests overlap on the device.  Admission is first-come-first-served, but
 * a request that does not fit may be overtaken by later ones until it has
 * waited 50 ms.  Each buffer (momenta, eps, out, status, layouts as for
 * bg_eval) is one of:
 *   - device memory of the server's device, used in place with no copy and
 *     no arena bytes (momenta and states kept resident on the device across
 *     requests, outputs left on the device);
 *   - page-locked host memory mapped into the device's address space (as
 *     cudaHostAlloc / cudaMallocHost give under unified addressing), also
 *     used in place: the kernel reads the inputs and writes the results over
 *     the host link, without copy-engine transfers (unless the request is
 *     large and light per point; the decision of bg_eval_host, with the
 *     host-link rate measured when the server is created);
 *   - pageable host memory, staged through the arena by copies.
 * All buffers must stay valid, and inputs unchanged, until bg_serve_wait
 * returns.  Every result equals what bg_eval gives for the request alone.
 */
typedef struct bg_server bg_server;

bg_status bg_serve_create(size_t budget_bytes, int max_inflight, bg_server** out);

/* bg_serve_submit -- queue E >= 1 points of `plan`; returns a ticket.
 * BG_ERR_INVALID_ARG when the request can never fit the budget or a buffer
 * lives on another device; BG_ERR_BUSY after bg_serve_destroy has begun. */
bg_status bg_serve_submit(bg_server* srv, const bg_plan* plan, int64_t E, const void* momenta,
                          const void* eps, void* out, uint8_t* status, uint64_t* ticket);

/* bg_serve_wait -- block until the ticket's results are in its host buffers
 * (BG_OK, the ticket is then retired), or until timeout_ms elapsed
 * (BG_ERR_TIMEOUT, the ticket stays valid); timeout_ms < 0 waits forever.
 * BG_ERR_CUDA when the request's copies or kernel failed, including an
 * asynchronous error raised on the device after they were enqueued.  Several
 * threads may wait on the same ticket at once: each returns the request's
 * result; a wait that starts after the ticket was retired returns
 * BG_ERR_INVALID_ARG (unknown ticket). */
bg_status bg_serve_wait(bg_server* srv, uint64_t ticket, int64_t timeout_ms);

/* bg_serve_stats -- counters (any pointer may be NULL). */
bg_status bg_serve_stats(bg_server* srv, uint64_t* submitted, uint64_t* completed,
                         uint64_t* pending, size_t* bytes_in_use, size_t* peak_bytes);

/* bg_serve_destroy -- finish every queued and running request, then free the
 * arena, streams and thread.  No call on `srv` may follow. */
bg_status bg_serve_destroy(bg_server* srv);

/*
 * bg_cut_trace -- state sum over a ring of k tree amplitudes (the leading pole
 * of a one-loop cut, Sec. 2.1): for every point e,
 *     out[e] = sum_{s_1..s_k} prod_{i=1..k} M_i[e][s_{i+1}][s_i],  s_{k+1} = s_1,
 * i.e. trace(M_k ... M_2 M_1).  M is a HOST array of k device pointers, each
 * [E][S][S] (row = outgoing internal state, column = incoming), uint32
 * residues in [0, p) for BG_FIELD_FP or double2 for the complex fields: the
 * output of a product plan whose only legs with S states are leg 0 (the
 * incoming internal leg, with the dual "tilde" states of Sec. 2.3) and leg
 * n-1 (the outgoing one), the others one state.  out: device [E], same
 * element type.  1 <= k <= 16, 1 <= S <= 8, p < 2^31 for F_p (ignored
 * otherwise).  Asynchronous on `stream`; errors as bg_eval.
 */
bg_status bg_cut_trace(bg_field field, uint32_t p, int64_t E, int k, int S,
                       const void* const* M, void* out, cudaStream_t stream);

/* bg_plan_describe -- NUL-terminated one-line description of the kernel the
 * plan launches (variant, block size, shared memory, workspace per thread)
 * written to buf[0..len); returns BG_ERR_INVALID_ARG when it does not fit. */
bg_status bg_plan_describe(const bg_plan* plan, char* buf, size_t len);

/* bg_strerror -- static string for a status code. */
const char* bg_strerror(bg_status s);

/* bg_last_error -- thread-local detail of the last failing call on this
 * thread ("" if none). */
const char* bg_last_error(void);

/* bg_version -- BG_VERSION of the library binary. */
int bg_version(void);

/*
 * bg_debug_bounds_report -- testing aid for memory safety (no counterpart in
 * the paper).  A library compiled with BG_CHECKED compares every index into
 * the recursion tables with the extent of its region before the access; a
 * violation is recorded as (site << 32 | index) -- the first one since the
 * last report -- and the access is redirected to slot 0 of the thread's own
 * table.  This call returns *checked = 1 and that record (0 = none) for the
 * current device in such a build and clears it; in an ordinary build it
 * returns *checked = 0 and *first_violation = 0 (no checks are compiled).
 * Call it after the evaluations have completed (synchronise first).
 */
bg_status bg_debug_bounds_report(int* checked, uint64_t* first_violation);

/*
 * bg_debug_in_place_pays -- testing aid (no counterpart in the paper): the
 * decision bg_eval_host and the server take for a batch of E points of a plan
 * with (field, n, d, D_s) and H amplitudes per point whose host buffers,
 * host_bytes in all, are page-locked and mapped.  *in_place = 1 when one
 * kernel should read and write them over the host link (batches of at most
 * 64 MiB, or batches whose arithmetic per point hides the link traffic), 0
 * when copies should move them; *ops = the field multiplications per
 * amplitude of the literal recursion that the estimate uses.  Pure host
 * arithmetic for a 152-SM GB300 with a host-link probe rate of 135 GB/s (the
 * library's own decision scales the kernels' rates by the plan device's SM
 * count and uses the read rate measured on the device): needs no device.
 * BG_ERR_INVALID_ARG for arguments out of the ranges of bg_plan_create,
 * H < 1, E < 0 or NULL outputs.
 */
bg_status bg_debug_in_place_pays(bg_field field, int n, int d, int D_s, int H, int64_t E,
                                 size_t host_bytes, int* in_place, double* ops);

typedef enum {
    BG_FAULT_DEVICE_ALLOC = 1,
    BG_FAULT_LAUNCH = 2,
    BG_FAULT_COPY = 3
} bg_fault_site;

/*
 * bg_debug_inject_fault -- testing aid for the failure paths (no counterpart
 * in the paper).  Operations at `site` number 0, 1, 2, ... from this call on;
 * operations skip .. skip+count-1 fail as if the CUDA runtime had refused
 * them, without calling it (nothing reaches the GPU, so nothing can fault
 * there), and every later one runs normally.  count = 0 disarms the site.
 * Process-wide; not meant for production use.
 *   BG_FAULT_DEVICE_ALLOC  device allocations: the assignment table of
 *                          bg_plan_create*, the arena of bg_serve_create ->
 *                          BG_ERR_NOMEM
 *   BG_FAULT_LAUNCH        kernel and graph launches of bg_eval,
 *                          bg_eval_noalloc, bg_batch_launch, bg_cut_trace ->
 *                          BG_ERR_CUDA, outputs untouched
 *   BG_FAULT_COPY          asynchronous copies of bg_eval_host (per chunk)
 *                          and of served requests -> BG_ERR_CUDA (for a
 *                          served request, from its bg_serve_wait)
 * Returns BG_ERR_INVALID_ARG for an unknown site or negative skip / count.
 */
bg_status bg_debug_inject_fault(bg_fault_site site, int skip, int count);

#ifdef __cplusplus
}
#endif

#endif /* BG_H */
