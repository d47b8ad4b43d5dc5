/*
 * llp.h — C ABI of libllp.so, the single-GPU (sm_103a) lattice-linear
 * predicate (LLP) sweep engine.
 *
 * Method (paper Sec. 3, Algorithm LLP): a problem is a state vector G, a
 * predicate forbidden(G, j) and a monotone advance(G, j).  Starting from the
 * bottom of the lattice, every forbidden index is advanced, in parallel and in
 * any order, until no index is forbidden; the result is the least G that
 * satisfies the problem's predicate.  Each entry point below is one problem of
 * the paper's Sec. 4 run to that fixed point on the GPU.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Pointers are DEVICE pointers unless their name starts with h_.  The caller
 *    owns every buffer; the library keeps no pointer after a call returns.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Calls only enqueue work on it: no allocation, no host synchronisation.
 *    Exception: llp_get_status() synchronises `stream`.
 *  - Scratch memory comes from the caller's `ws` (`ws_bytes` long, 256-byte
 *    aligned), sized by the matching *_workspace_size() query.  A workspace may
 *    be reused by consecutive calls on one stream; two calls in flight at the
 *    same time must not share one.
 *  - The return value is the HOST-side status: argument validation and launch
 *    errors (LLP_ERR_INVALID_ARG, LLP_ERR_WORKSPACE_TOO_SMALL, LLP_ERR_CUDA).
 *    On a non-OK return nothing was enqueued (LLP_ERR_CUDA: possibly partly).
 *  - DEVICE-side outcomes (LLP_ERR_TIMEOUT, LLP_ERR_INFEASIBLE,
 *    LLP_ERR_OVERFLOW) are written to a status word in the workspace header;
 *    read it with llp_get_status().  Every device-side wait (grid barrier,
 *    work queue) is bounded by `deadline_ns`; when it expires the kernel stops
 *    cleanly and reports LLP_ERR_TIMEOUT, outputs are then undefined.
 *  - `sched` (may be NULL = built-in heuristic) only changes HOW the sweep
 *    runs, never the result: every schedule reaches the same least fixed point.
 *  - All results are integers and independent of scheduling, bit for bit.
 */
#ifndef LLP_H
#define LLP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t llp_status_t;

#define LLP_OK 0
#define LLP_ERR_INVALID_ARG 1
#define LLP_ERR_WORKSPACE_TOO_SMALL 2
#define LLP_ERR_CUDA 3
#define LLP_ERR_TIMEOUT 4
#define LLP_ERR_INFEASIBLE 5 /* Algorithm LLP returns null: an advance passes the top T[j] */
#define LLP_ERR_OVERFLOW 6
#define LLP_ERR_UNSUPPORTED 7

/* Sweep modes (llp_sched_t.mode). */
#define LLP_MODE_AUTO 0   /* per sweep: dense when the worklist is large */
#define LLP_MODE_SPARSE 1 /* always walk the worklist (paper's bag / shared work bag) */
#define LLP_MODE_DENSE 2  /* always scan every index's "changed" stamp (paper's all-indices solver) */

#define LLP_DELTA_INF 0xFFFFFFFFu /* no priority buckets: one worklist (Bellman-Ford order) */

/* Compressed sparse rows of OUT-arcs.  offsets has n+1 entries, int32 if
 * offsets_64 == 0 else int64, non-decreasing, offsets[0] == 0, offsets[n] == m;
 * indices[m] are target vertices in [0, n); weights[m] (may be NULL where the
 * problem ignores them).  Self-loops and parallel arcs are allowed. */
typedef struct llp_csr {
    int32_t n;
    int32_t offsets_64;
    int64_t m;
    const void *offsets;
    const int32_t *indices;
    const uint32_t *weights;
} llp_csr_t;

/* Schedule.  Fields never change results.  Every field 0 = heuristic choice,
 * so a zero-initialised struct (or sched == NULL) is the default schedule. */
typedef struct llp_sched {
    int32_t mode;           /* LLP_MODE_* (0 = AUTO) */
    uint32_t delta;         /* SSSP/BFS priority-bucket width in distance units; 0 = auto,
                               LLP_DELTA_INF = no buckets */
    int32_t block_cfg;      /* work-block configuration 1..LLP_BLOCK_CFGS (see below); 0 = auto */
    int32_t dense_permille; /* AUTO mode: the next sweep is dense when this one examines more than
                               m * dense_permille / 1000 arcs (0 = 50) */
    int32_t use_mlp;        /* 1: the learned scheduler model chooses mode, delta and block_cfg */
    int32_t threads;        /* threads per CTA: 0 = auto, else 256 or 512 */
    int64_t deadline_ns;    /* device wait limit of one call; 0 = default (10 s) */
    const float *mlp_params;/* device pointer to the scheduler network's parameters when use_mlp = 1 */
    int32_t local_chain;    /* graph sweep: a warp expands the small vertices it has just advanced
                               itself within the same sweep (LIFO, the paper's recency-biased per-thread
                               bags), up to local_chain batches of 32 per worklist item;
                               0 = heuristic (off), -1 = off */
    int32_t pull_permille;  /* llp_bfs_pull: a sweep runs pull-style over the in-arcs when its frontier
                               holds more than about m * pull_permille / 1000 out-arcs (0 = 200);
                               < 0 = never pull */
    int32_t group_words;    /* graph sweep: bitmap words (32 vertices each) per work item of a dense
                               sweep, 1, 2, 4 or 8; 0 = auto (the widest that still gives every warp
                               of the grid about three items) */
    int32_t fixed_memo;     /* SSSP with finite delta: 1 = fixed-state memoization (paper Sec. 3,
                               "memoization through fixed states"): once a bucket empties, every
                               vertex below its bound is final; a relaxation that meets such a
                               vertex marks it in a bitmap, and later relaxations test the bit
                               instead of reading d(v).  0 = off */
} llp_sched_t;

/* Work-block configurations of the graph sweep: (small-vertex degree limit,
 * arcs per chunk of a large vertex), selected by block_cfg:
 *   1: (32, 256)   2: (64, 256)   3: (128, 512) */
#define LLP_BLOCK_CFGS 3

/* Device-side outcome and counters of the last call that used a workspace. */
typedef struct llp_stats {
    int32_t status;     /* LLP_OK or a device-side LLP_ERR_* */
    int32_t sweeps;     /* forbidden/advance sweeps executed (grid barriers) */
    int64_t items;      /* worklist items evaluated */
    int64_t edges;      /* arcs / dependents examined by forbidden() */
    int64_t advances;   /* successful advances (monotone updates that changed G) */
    int64_t aux;        /* problem-specific: SSSP bucket advances, marriage proposals, ... */
    int64_t elapsed_ns; /* device time of the sweep loop (%globaltimer) */
    int32_t mode_used;  /* schedule actually used */
    uint32_t delta_used;
    int32_t block_cfg_used;
    int32_t dense_sweeps; /* sweeps run in dense mode */
    int32_t local_chain_used;
    int32_t pull_sweeps;  /* llp_bfs_pull: sweeps run pull-style over the in-arcs */
} llp_stats_t;

const char *llp_version(void);
const char *llp_status_string(llp_status_t code);

/* Synchronises `stream`, then copies the workspace header of the last call
 * that used `ws` into *out.  Returns out->status, or LLP_ERR_CUDA. */
llp_status_t llp_get_status(const void *ws, void *stream, llp_stats_t *out);

/* Synchronises `stream`, then copies up to max_records per-sweep records of
 * the last graph-engine call (SSSP/BFS) that used `ws` into out, 4 uint32 per
 * record: device ns since the call started, small-vertex worklist size, chunk
 * worklist size, flags (bit 0 dense sweep, bit 1 bucket advance, bits 2..31
 * arcs examined by the sweep / 1024).  Returns the
 * number of records, or -LLP_ERR_* on error.  Diagnostics and the learned
 * scheduler's training data; not needed for results. */
int32_t llp_sweep_log(const void *ws, void *stream, uint32_t *out, int32_t max_records);

/* ------------------------------------------------------------------ SSSP
 * Paper Sec. 4.1: G[v] = d(v); v is forbidden iff some arc (u,v) has
 * d(v) > d(u) + w(u,v); advance sets d(v) to the minimum over such arcs.
 * Implemented push-style on out-arcs with atomicMin (the same least fixed
 * point).  Result: dist[v] = length of a shortest path from `source`, or
 * 0xFFFFFFFF if v is unreachable.  Path lengths are formed in 64 bits; a finite
 * length >= 0xFFFFFFFF sets LLP_ERR_OVERFLOW (device status).
 * dist: uint32[n], written in place (it is the state vector G). */
size_t llp_sssp_workspace_size(int32_t n, int64_t m);
llp_status_t llp_sssp(const llp_csr_t *g, int32_t source, uint32_t *dist, const llp_sched_t *sched,
                      void *ws, size_t ws_bytes, void *stream);

/* SSSP on a graph in HOST memory: h_g's offsets/indices/weights and h_dist
 * are host pointers (pinned memory gives the full copy bandwidth; pageable
 * memory works but the copies are staged by the driver).  Enqueues on `stream`
 * the copies of the graph into the workspace (cudaMemcpyAsync, 64 MiB pieces),
 * llp_sssp on them, and the copy of the distances into h_dist; h_dist is
 * valid once the stream has been synchronised.  The workspace holds the sweep's
 * scratch followed by the device copy of the graph and of dist:
 * llp_sssp_host_workspace_size(n, m, offsets_64) bytes.  Same result as
 * llp_sssp; device status via llp_get_status(ws). */
size_t llp_sssp_host_workspace_size(int32_t n, int64_t m, int32_t offsets_64);
llp_status_t llp_sssp_host(const llp_csr_t *h_g, int32_t source, uint32_t *h_dist, const llp_sched_t *sched,
                           void *ws, size_t ws_bytes, void *stream);

/* Warm start (incremental re-solve).  Algorithm LLP (Sec. 3) reaches the same
 * least solution from any state below it in the lattice order, so a previous
 * result can be the starting state after the graph changed in a way that only
 * shortens paths: arc weights decreased and/or arcs inserted (same n).  dist
 * (in/out): on entry, for every v, a length of some path from `source` to v in
 * the new graph, or 0xFFFFFFFF; the previous result of llp_sssp on the old
 * graph is such a state.  seeds[0..n_seeds): every vertex with an out-arc that
 * is new or whose weight decreased (duplicates allowed; vertices with an
 * infinite distance are ignored): only their arcs can make an index forbidden
 * in the entry state, so they are the initial_states_to_process of the run.
 * On return dist holds the new shortest distances, bit-exact as llp_sssp on the
 * new graph.  n_seeds = 0 returns dist unchanged (d[source] set to 0).  A seed
 * outside [0, n) is skipped and sets LLP_ERR_INVALID_ARG (device status).
 * If the entry state is not as stated (e.g. a finite value below a true
 * distance) the result is the least fixed point above it, not the distances.
 * Workspace: llp_sssp_workspace_size. */
llp_status_t llp_sssp_warm(const llp_csr_t *g, int32_t source, uint32_t *dist, const int32_t *seeds,
                           int32_t n_seeds, const llp_sched_t *sched, void *ws, size_t ws_bytes, void *stream);

/* SSSP for callers that cannot allocate device memory.
 * Same computation and result as llp_sssp, but the scratch space comes from a
 * fixed 64 MiB array inside this library instead of a caller workspace, so the
 * caller only provides the graph and dist[].  Meant for code that has no device
 * allocator of its own or must not call one: a plain C or Fortran client
 * without a CUDA memory pool, a plugin whose host owns all device memory, or a
 * latency-critical loop where cudaMalloc's implicit device synchronisation is
 * not acceptable.  The paper has no counterpart; it is an interface addition.
 *  - Limit: graphs whose llp_sssp_workspace_size(n, m) exceeds
 *    llp_sssp_noalloc_max_workspace() (64 MiB; e.g. n = 1M vertices with
 *    m = 16M arcs fits) are rejected with LLP_ERR_WORKSPACE_TOO_SMALL.
 *  - The array exists once per GPU that loads the library and stays allocated
 *    until the process exits.  The first call on a device looks up its device
 *    address (cudaGetSymbolAddress); make that first call before any stream
 *    capture on that device.
 *  - All calls on a device share the one array: calls that overlap on the GPU
 *    (different streams, or another thread) race and give undefined results.
 *    Serialise them, e.g. on one stream.
 *  - The array is a module global: under CUDA's lazy module loading it may be
 *    reserved only when this module first loads on a device, which can be the
 *    first llp_sssp_noalloc call; that call then fails with LLP_ERR_CUDA when
 *    the device has no 64 MiB left.  Every process that loads the library pays
 *    the 64 MiB on each device where the module is loaded, whether or not it
 *    calls llp_sssp_noalloc.
 *  - The return value is the host-side outcome only.  The device-side outcome
 *    of the last call on the device (LLP_OK, or LLP_ERR_TIMEOUT /
 *    LLP_ERR_OVERFLOW / LLP_ERR_INVALID_ARG raised during the sweep, in which
 *    case dist[] is not the distances) is read with llp_sssp_noalloc_status;
 *    llp_get_status()/llp_sweep_log() cannot be pointed at this scratch.
 *  - Allocates nothing: no cudaMalloc/cudaFree or allocating library call. */
size_t llp_sssp_noalloc_max_workspace(void);
llp_status_t llp_sssp_noalloc(const llp_csr_t *g, int32_t source, uint32_t *dist, const llp_sched_t *sched,
                              void *stream);
/* Device status word of the last llp_sssp_noalloc call on the current device:
 * copies it into *status after the work queued on `stream` (synchronises the
 * stream).  Calls from other streams that may still run race with it, as for
 * llp_sssp_noalloc itself.  Allocates nothing.  LLP_ERR_INVALID_ARG if status
 * is NULL. */
llp_status_t llp_sssp_noalloc_status(int32_t *status, void *stream);

/* Measurement helper with no counterpart in the paper: the access-pattern floor of
 * a push sweep.  One pass over all m arcs of g that streams indices[] and
 * weights[] (16-byte loads; both arrays 16-byte aligned) and reads state[v] at
 * random for every arc's target v (state: n uint32 values, any contents), with
 * 8 reads per lane in flight.  Its device time is the time any push sweep needs
 * to touch every arc once; the benchmark reports it beside the sweep kernel's.
 * sink: llp_gather_floor_sink_size() bytes of device memory, overwritten.
 * Stream-ordered; allocates nothing. */
size_t llp_gather_floor_sink_size(void);
llp_status_t llp_gather_floor(const llp_csr_t *g, const uint32_t *state, void *sink, size_t sink_bytes, void *stream);

/* ------------------------------------------------------------------- BFS
 * Paper Sec. 4.2: G[v] = level; v is forbidden iff an in-neighbour u has
 * G[u] < G[v] - 1; advance sets G[v] = 1 + min G[u].  level[v] = hop distance
 * from `source`, 0xFFFFFFFF if unreachable.  g->weights is ignored. */
size_t llp_bfs_workspace_size(int32_t n, int64_t m);
llp_status_t llp_bfs(const llp_csr_t *g, int32_t source, uint32_t *level, const llp_sched_t *sched,
                     void *ws, size_t ws_bytes, void *stream);

/* BFS warm start after arc insertions: as llp_sssp_warm with unit weights
 * (level in/out; seeds = sources of the inserted arcs).  Push sweeps only. */
llp_status_t llp_bfs_warm(const llp_csr_t *g, int32_t source, uint32_t *level, const int32_t *seeds,
                          int32_t n_seeds, const llp_sched_t *sched, void *ws, size_t ws_bytes, void *stream);

/* BFS with direction switching.  Same result as llp_bfs; g_in is the
 * transpose of g (CSR of IN-arcs: row v lists the sources u of the arcs (u,v),
 * any order within a row; same n, m and offsets_64 as g; weights ignored),
 * e.g. built by llp_csr_transpose.  A sweep whose frontier is narrow runs
 * push-style as in llp_bfs.  A sweep whose frontier is wide (see
 * llp_sched_t.pull_permille) evaluates the predicate of Sec. 4.2 in its own
 * direction, over in-neighbours: every vertex not yet reached scans its
 * in-arcs and stops at the first one whose source is in the frontier, which
 * gives it the next level.  The paper states the predicate this way; switching
 * by frontier width is the hybrid its Conclusion (Future work) proposes for
 * dense frontiers.  Pull sweeps are used only when the run keeps exact
 * levels per sweep, i.e. without a local chain (llp_sched_t.local_chain);
 * with a chain every sweep is push-style.  Workspace: llp_bfs_workspace_size. */
llp_status_t llp_bfs_pull(const llp_csr_t *g, const llp_csr_t *g_in, int32_t source, uint32_t *level,
                          const llp_sched_t *sched, void *ws, size_t ws_bytes, void *stream);

/* ------------------------------------------------------------ Transpose
 * Input preparation for llp_bfs_pull (not a step of the method): writes the
 * transpose of g.  in_offsets: n+1 entries of g's offset type (int32 if
 * g->offsets_64 == 0, else int64); in_indices[m]: row v holds the sources u of
 * the arcs (u,v); in_weights[m] (may be NULL; needs g->weights) the matching
 * weights.  The order of the arcs within a row is unspecified (it depends on
 * timing); the rows as multisets and in_offsets are exact.  An arc whose
 * target is outside [0, n) is skipped and sets LLP_ERR_INVALID_ARG as the
 * device status. */
size_t llp_csr_transpose_workspace_size(int32_t n, int64_t m);
llp_status_t llp_csr_transpose(const llp_csr_t *g, void *in_offsets, int32_t *in_indices, uint32_t *in_weights,
                               void *ws, size_t ws_bytes, void *stream);

/* ------------------------------------------------------- Stable marriage
 * Paper Sec. 4.3: G[m] = index into man m's preference list; m is forbidden
 * iff the woman he targets prefers another man who targets her; advance
 * moves to his next choice.  The fixed point is the man-optimal stable
 * matching.  men_pref[m*n + k] = k-th choice of man m; women_rank[w*n + m] =
 * rank of m for woman w (0 = best; each row a permutation of 0..n-1).
 * Outputs: wife[m]; husband[w] and next[m] (= G, the final list index) if not
 * NULL.  A list exhausted (malformed input) gives LLP_ERR_INFEASIBLE.
 * 1 <= n <= 2^24. */
size_t llp_stable_marriage_workspace_size(int32_t n);
llp_status_t llp_stable_marriage(int32_t n, const int32_t *men_pref, const int32_t *women_rank, int32_t *wife,
                                 int32_t *husband, int32_t *next, const llp_sched_t *sched, void *ws,
                                 size_t ws_bytes, void *stream);

/* --------------------------------------------------------- 0-1 knapsack
 * Paper Sec. 4.7: cell G[k,c] = best value of items 0..k-1 within capacity c;
 * forbidden iff G[k,c] < max(G[k-1,c], v_k + G[k-1,c-w_k]); advance raises it
 * to that bound.  best[0] = G[n, capacity]; final_row (optional, int32[capacity+1])
 * = G[n, 0..capacity].  Requires w[i] >= 1, v[i] >= 0, sum(v) < 2^31,
 * 0 <= capacity <= 2^26.  Large instances run as a wavefront over capacity
 * slices whose rows pass through a ring of up to 256 rows of (capacity + 1)
 * 8-byte words in the workspace (cleared by the call), so the workspace size
 * grows with both arguments; a workspace sized for (n, capacity) serves every
 * instance with at most n items and at most that capacity.  A wait of the
 * wavefront that passes the schedule's deadline ends the call with
 * LLP_ERR_TIMEOUT in the status word. */
size_t llp_knapsack_workspace_size(int32_t n_items, int32_t capacity);
llp_status_t llp_knapsack(int32_t n_items, const int32_t *w, const int32_t *v, int32_t capacity, int32_t *best,
                          int32_t *final_row, const llp_sched_t *sched, void *ws, size_t ws_bytes, void *stream);

/* --------------------------------------------------- Transitive closure
 * Paper Sec. 4.6: G[u,v] boolean; (u,v) is forbidden iff not G[u,v] and
 * G[u,w] and G[w,v] for some w; advance sets G[u,v].  reach: n rows of
 * W = ceil(n/32) uint32 words; bit (v & 31) of reach[u*W + v/32] (least
 * significant bit first) is 1 iff a path of >= 1 arcs leads from u to v.
 * g->weights is ignored.  n <= 65536. */
size_t llp_transitive_closure_workspace_size(int32_t n, int64_t m);
llp_status_t llp_transitive_closure(const llp_csr_t *g, uint32_t *reach, const llp_sched_t *sched, void *ws,
                                    size_t ws_bytes, void *stream);

/* ------------------------------------------------------- Job scheduling
 * Paper Sec. 4.4: G[j] = completion time, initially t_j; j is forbidden iff
 * all predecessors are fixed and G[j] < max_p G[p] + t_j; advance raises it
 * and fixes j.  completion[j] = t_j + max over predecessors (0 if none).
 * succ: CSR of successor arcs (weights ignored).  duration[j] >= 0.
 * A cycle leaves some job never ready: LLP_ERR_INFEASIBLE. */
size_t llp_job_schedule_workspace_size(int32_t n, int64_t m);
llp_status_t llp_job_schedule(const llp_csr_t *succ, const int32_t *duration, int32_t *completion,
                              const llp_sched_t *sched, void *ws, size_t ws_bytes, void *stream);

/* ------------------------------------------------------------ Reduction
 * Paper Sec. 4.5: nodes of a reduction tree; a node is forbidden once all its
 * children have published and it has not combined them.  sum[0] = sum of x
 * modulo 2^64.  n >= 0. */
size_t llp_reduce_workspace_size(int64_t n);
llp_status_t llp_reduce(int64_t n, const uint64_t *x, uint64_t *sum, const llp_sched_t *sched, void *ws,
                        size_t ws_bytes, void *stream);

/* ---------------------------------------------------------------- Batched
 * Many independent instances of four families solved in ONE persistent
 * launch (plus a one-CTA planning kernel): each CTA takes the next instance
 * from a device queue, most expensive first, and runs that instance's LLP
 * sweeps on its own (shared-memory state, CTA barriers).  Results are the same
 * as the single-instance entry points, bit for bit.  Counts may be 0.  The
 * *_max_* fields are host-known upper bounds used to size the workspace;
 * an instance above its bound sets LLP_ERR_INVALID_ARG (device status).
 * Every call is stream-ordered and capturable in a CUDA graph. */
typedef struct llp_batch {
    /* 0-1 knapsack: items of instance i are [knap_item_off[i], knap_item_off[i+1]) of knap_w/knap_v */
    int32_t knap_count;
    int32_t knap_max_capacity;
    const int64_t *knap_item_off; /* [knap_count + 1] */
    const int32_t *knap_w;
    const int32_t *knap_v;
    const int32_t *knap_capacity; /* [knap_count] */
    int32_t *knap_best;           /* [knap_count] out: optimum of each instance */
    /* job DAGs: jobs of DAG i are [job_off[i], job_off[i+1]) of the concatenated arrays;
     * job_succ_offsets (total_jobs + 1 entries) are positions in job_succ_indices, whose
     * entries are LOCAL job ids of the same DAG */
    int32_t job_count;
    int32_t job_max_n;
    const int64_t *job_off;          /* [job_count + 1] */
    const int64_t *job_succ_offsets; /* [total_jobs + 1] */
    const int32_t *job_succ_indices;
    const int32_t *job_duration;     /* [total_jobs] */
    int32_t *job_completion;         /* [total_jobs] out */
    /* stable marriage: instance i has n = sm_n[i]; its n*n preference entries start at
     * sm_pref_off[i] in sm_men_pref / sm_women_rank (layouts as llp_stable_marriage);
     * its wife[] output starts at sm_man_off[i] */
    int32_t sm_count;
    int32_t sm_max_n;
    const int32_t *sm_n;
    const int64_t *sm_pref_off;
    const int64_t *sm_man_off;
    const int32_t *sm_men_pref;
    const int32_t *sm_women_rank;
    int32_t *sm_wife;
    /* small SSSP / BFS (Sec. 4.1 / 4.2): graph i has vertices [gr_off[i], gr_off[i+1]) of the
     * concatenated arrays; gr_arc_offsets (total_vertices + 1 entries) are positions in gr_indices /
     * gr_weights, whose entries are LOCAL vertex ids of the same graph; gr_source[i] is local;
     * gr_unit (may be NULL = every instance SSSP): gr_unit[i] != 0 makes instance i a BFS (levels,
     * weights ignored); gr_weights may be NULL when every instance is a BFS.  gr_dist[total_vertices]
     * receives distances / levels, 0xFFFFFFFF = unreachable; a finite path length >= 0xFFFFFFFF sets
     * LLP_ERR_OVERFLOW.  The CTA keeps d[] and two frontier bitmaps in shared memory when
     * 4.25 * n bytes fit, else it works on gr_dist in place. */
    int32_t gr_count;
    int32_t gr_max_n;
    const int64_t *gr_off;         /* [gr_count + 1] */
    const int64_t *gr_arc_offsets; /* [total_vertices + 1] */
    const int32_t *gr_indices;
    const uint32_t *gr_weights;
    const int32_t *gr_source;      /* [gr_count] */
    const int32_t *gr_unit;        /* [gr_count] or NULL */
    uint32_t *gr_dist;             /* [total_vertices] out */
} llp_batch_t;

/* Launch shape of the batched engine (never changes results); 0 = default. */
typedef struct llp_batch_cfg {
    int32_t threads;     /* threads per CTA: 256, 512 or 1024 (default 1024) */
    int32_t knap_unroll; /* knapsack cells per thread per chunk: 4, 8 (default) or 16 */
    int32_t ctas_per_sm; /* resident CTAs per SM: 1 (default) or 2 (threads <= 512; each CTA then has
                            half the shared memory, so larger instances keep their state in the
                            per-CTA global scratch) */
    int32_t reserved;
} llp_batch_cfg_t;

size_t llp_batch_workspace_size(const llp_batch_t *b);
llp_status_t llp_batch_solve(const llp_batch_t *b, const llp_batch_cfg_t *cfg, const llp_sched_t *sched, void *ws,
                             size_t ws_bytes, void *stream);

/* Autotuner: runs the batch once untimed and once timed (CUDA events) for every
 * candidate launch shape (threads 1024/512 at one CTA per SM, 512/256 at two, each
 * with knapsack blocking 4, 8, 16: 12 candidates) and writes the fastest to *best.  Synchronises
 * `stream`.  h_ms (may be NULL) receives up to max_tried timings; *n_tried the
 * number of candidates run.  Outputs of the batch hold the last run's result. */
llp_status_t llp_batch_autotune(const llp_batch_t *b, void *ws, size_t ws_bytes, void *stream,
                                llp_batch_cfg_t *best, float *h_ms, int32_t max_tried, int32_t *n_tried);

/* ------------------------------------------------------ Learned scheduler
 * Not in the paper (its conclusion asks for an adaptive runtime choice of
 * solver): a small fp32 MLP maps instance features of a graph to a schedule
 * of the graph sweep.  Setting llp_sched_t.use_mlp = 1 and mlp_params makes
 * llp_sssp / llp_bfs run a feature kernel and an inference kernel on the device
 * before the sweep, which then uses the chosen schedule.  Results never depend
 * on the schedule.  The scheduler network is features(16) -> 64 -> 64 -> 23
 * logits = heads {mode: 3 (AUTO, SPARSE, DENSE), bucket-width class: 8
 * (0 = none, c >= 1: width = max sampled weight * 2^(c-1)), block_cfg: 3,
 * local chain: 4 (off, 4, 16, 64 batches), dense-sweep group width: 5 (the
 * grid-size rule, 1, 2, 4, 8 words)}.
 * Parameters: one fp32 vector, row-major W1[F,H1] b1 W2[H1,H2] b2 W3[H2,O] b3. */
typedef struct llp_mlp_dims {
    int32_t F, H1, H2, O; /* each 1..128 */
    int32_t nheads;       /* 1..8, sum of heads[] == O */
    int32_t heads[8];
} llp_mlp_dims_t;

size_t llp_mlp_param_count(const llp_mlp_dims_t *dims);
size_t llp_mlp_workspace_size(const llp_mlp_dims_t *dims, int32_t batch);

/* logits[batch, O] = MLP(X[batch, F]).  All device pointers. */
llp_status_t llp_mlp_forward(const llp_mlp_dims_t *dims, const float *params, const float *X, int32_t batch,
                             float *logits, void *stream);

/* loss[0] = mean over the batch of the sum over heads of the softmax
 * cross-entropy with labels Y[batch, nheads] (class index within each head; a
 * label outside its head contributes nothing); grad = d loss / d params (same
 * layout as params).  The gradient reduction is deterministic. */
llp_status_t llp_mlp_loss_grad(const llp_mlp_dims_t *dims, const float *params, const float *X, const int32_t *Y,
                               int32_t batch, float *loss, float *grad, void *ws, size_t ws_bytes, void *stream);

/* One Adam step (Kingma and Ba 2015) in place; step >= 1. */
llp_status_t llp_mlp_adam(float *params, const float *grad, float *m, float *v, size_t n, int32_t step, float lr,
                          float beta1, float beta2, float eps, void *stream);

/* Runs only the feature and inference kernels for graph g (the default
 * 16-64-64-18 network) into the header of ws.  If h_chosen / h_features are not
 * NULL, synchronises the stream and copies the choice / the 16 features out. */
llp_status_t llp_graph_schedule(const llp_csr_t *g, int32_t source, int32_t unit_weights, const float *params,
                                void *ws, size_t ws_bytes, void *stream, llp_sched_t *h_chosen, float *h_features);

#ifdef __cplusplus
}
#endif

#endif /* LLP_H */
