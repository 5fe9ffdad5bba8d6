/*
 * napspmv.h -- C ABI of the GB300 node-aware parallel SpMV library.
 *
 * The library computes w <- A v (Sec. 1 of Bienz, Gropp, Olson, "Node aware
 * sparse matrix-vector multiplication", arXiv 1612.08060) the way the paper's
 * node-aware algorithm NAPSpMV (Sec. 4, Algorithm "NAPSpMV") does, with every
 * simulated process and node living on one GPU:
 *
 *   - the rows of the N x N matrix A are split into n_p contiguous blocks, one
 *     per simulated process (Sec. 2, Eq. R; or strided, row i on process
 *     i mod n_p, with NAPSPMV_PARTITION_STRIDED), and the processes are grouped
 *     ppn per simulated node, process r being (r mod ppn, floor(r / ppn));
 *   - each process's rows are split into on-process, on-node and off-node
 *     column blocks (Sec. 2, Eqs. on_proc, on_node, off_node);
 *   - napspmv_plan builds, on the GPU, the standard communication plan
 *     (Sec. 2.1, Eqs. P, D) and the node-aware plan (Sec. 4.1, Eqs. N, E, T,
 *     U, G, I; Sec. 4.2, Eqs. L0/IL0, L1_send/IL1, L2/IL2), and the three-block
 *     CSR with each block's columns pointing into that block's receive buffer;
 *   - napspmv_apply runs, on the GPU, every message of the node-aware
 *     algorithm as a device gather or copy in HBM (on_node -> on_node and
 *     on_node -> off_node local exchanges, packing of g_send, the inter-node
 *     transfer g_send -> g_recv, the off_node -> on_node forwarding) and the
 *     three-block SpMV, for all simulated processes at once: by default as a
 *     CUDA graph of kernels in which the on_process part of the SpMV overlaps
 *     the message steps (NAPSPMV_ENGINE_OVERLAP), or in one persistent launch
 *     (NAPSPMV_ENGINE_FUSED).
 *
 * Conventions for every call:
 *   - Return value: NAPSPMV_OK (0) or a negative NAPSPMV_ERR_* code; the
 *     message of the last error of the calling thread is napspmv_last_error().
 *   - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Work is queued on it asynchronously unless stated otherwise.
 *   - Vectors are FP64, N entries, contiguous.  Device pointers must be device
 *     memory of the plan's device (the device current at napspmv_plan).
 *   - A plan owns all its device memory.  It is not thread-safe: calls on one
 *     plan (or one workspace) must not overlap on the host, and applies that
 *     use the same workspace must be ordered on one stream.
 *   - Limits: N < 2^30, nnz < 2^31, and every receive buffer < 2^30 values.
 *     Larger inputs are rejected with NAPSPMV_ERR_UNSUPPORTED, as are the
 *     engine / plan combinations documented with the plan flags.
 *   - There is no CPU fallback: without a usable CUDA device every call that
 *     needs one fails with NAPSPMV_ERR_CUDA.
 */
#ifndef NAPSPMV_H
#define NAPSPMV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ return codes */
#define NAPSPMV_OK 0
#define NAPSPMV_ERR_ARG (-1)         /* invalid argument or malformed CSR        */
#define NAPSPMV_ERR_OOM (-2)         /* device or host allocation failed         */
#define NAPSPMV_ERR_CUDA (-3)        /* a CUDA runtime call failed               */
#define NAPSPMV_ERR_TIMEOUT (-4)     /* a bounded device-side wait gave up       */
#define NAPSPMV_ERR_STATE (-5)       /* call not valid in the object's state     */
#define NAPSPMV_ERR_UNSUPPORTED (-6) /* size beyond the limits above, or an
                                        engine a plan's flags exclude            */

/* ------------------------------------------------------------ memory kinds */
#define NAPSPMV_HOST 0
#define NAPSPMV_DEVICE 1

/* -------------------------------------------------------------- plan flags */
/* Keep an FP32 copy of A's values for NAPSPMV_PREC_F32 applies. */
#define NAPSPMV_F32_VALUES (1u << 0)
/* Map the receiving side of every node pair by |E(n,m)| descending, as the
 * prose after Eq. U states, instead of the default that reproduces the
 * paper's Tables U and G (ascending |E|, last process first). */
#define NAPSPMV_MAP_TEXT (1u << 1)
/* Strided row partition: row i belongs to process i mod n_p (the partition of
 * the paper's SuiteSparse runs, Sec. 5) instead of contiguous blocks (Eq. R).
 * A node's rows then interleave with every other node's.  Every engine runs
 * such plans (the staged remote pass of the overlapped engine is not used). */
#define NAPSPMV_PARTITION_STRIDED (1u << 2)
/* Majority mapping, the alternative the text names after Eq. U: node pair
 * (n,m) is sent by the process of n that owns the most values of E(n,m) and
 * received by the process of m whose rows use the most of them (ties: the
 * lowest local process), which minimises per pair the values that reach the
 * sender through the on->off step and those the receiver only forwards.
 * Excludes NAPSPMV_MAP_TEXT (ERR_ARG). */
#define NAPSPMV_MAP_MAJORITY (1u << 3)
/* Node splitting, the mapping the text after Eq. U describes for a node with
 * fewer partner nodes than processes: each partner gets a group of the node's
 * processes so that all of them communicate.  On a node with P processes and
 * K < P partners (ordered as by the default rule), partner k gets
 * floor(P/K) + (k < P mod K) consecutive processes, counted up from process 0
 * on the sending side and down from process P-1 on the receiving side.  For
 * the pair (n,m) with sending group S and receiving group R, E(n,m) (ascending
 * j) is cut into max(|S|,|R|) contiguous pieces, piece i holding positions
 * floor(i e / c) .. floor((i+1) e / c) - 1, sent by S[i mod |S|] to
 * R[i mod |R|]; empty pieces are no message.  Nodes with at least P partners
 * map as without the flag.  NAPSPMV_LIST_TU then reports the first process of
 * each group.  Excludes NAPSPMV_MAP_MAJORITY (ERR_ARG). */
#define NAPSPMV_MAP_SPLIT (1u << 5)
/* Composed gathers, an ablation with no counterpart in the paper: each
 * process's receive buffers are gathered straight from v (b_{l->l} as in the
 * on->on step, b_{nl->l} from the owners' values), skipping the on->off
 * gather, pack, transfer and off->on hops of Algorithm NAPSpMV.  The plan and
 * its statistics are unchanged; the result has the same bits as the literal
 * exchange.  Every engine, batches and the no-allocation entry run such
 * plans. */
#define NAPSPMV_COMPOSED_GATHERS (1u << 4)

/* ------------------------------------------------------------- apply modes */
#define NAPSPMV_PREC_F64 0 /* FP64 values, FP64 products and sums            */
#define NAPSPMV_PREC_F32 1 /* FP32-stored values, FP32 products, FP64 sums   */

#define NAPSPMV_ENGINE_DEFAULT 0 /* the plan's default engine               */
#define NAPSPMV_ENGINE_FUSED 1   /* one persistent, cooperative launch for all
                                    phases and all chained applies, in levels
                                    separated by grid barriers               */
#define NAPSPMV_ENGINE_PHASED 2  /* one kernel per phase; chains of applies
                                    are captured once into a CUDA graph      */
#define NAPSPMV_ENGINE_OVERLAP 3 /* as PHASED, with the on_process part of
                                    the SpMV on a second stream while the
                                    message steps run (Algorithm NAPSpMV's
                                    overlap); the remote part then continues
                                    each row's sum (with vec = 1 the same
                                    bits as PHASED and FUSED)                */

#define NAPSPMV_PIPELINE_CTA 1
#define NAPSPMV_PIPELINE_WARP 2
/* Sliced rows: every process's rows sorted by length and packed 32 to a
 * chunk, column-major, one lane per row (no shared-memory stage; the chunk's
 * columns and values are read coalesced straight from global memory).  Each
 * row is summed in its stored order, so the bits are those of vec = 1; the
 * vec field is ignored.  The fused engine always sums rows this way; the
 * phased and overlapped engines do by default where rows average more than
 * 12 entries. */
#define NAPSPMV_PIPELINE_SELL 3

#define NAPSPMV_HALO_ON 1  /* overlapped engine: stage each process's receive
                              buffers in shared memory for its remote rows when
                              they fit (the default)                        */
#define NAPSPMV_HALO_OFF 2 /* gather the receive buffers from global memory   */

typedef struct napspmv_plan_s napspmv_plan_t;
typedef struct napspmv_ws_s napspmv_ws_t;

/* A CSR matrix.  row_ptr[0] = 0, row_ptr non-decreasing, row_ptr[n] = nnz,
 * 0 <= col[k] < n, no (i, j) stored twice.  Every stored entry counts as a
 * nonzero, zero values included (the paper's "A_ij != 0" is read as
 * structural).  `mem` says whether the three arrays are host or device
 * memory; they are only read during napspmv_plan and may be freed after. */
typedef struct {
    int64_t n;
    int64_t nnz;
    const int64_t *row_ptr;
    const int32_t *col;
    const double *val;
    int32_t mem; /* NAPSPMV_HOST or NAPSPMV_DEVICE */
} napspmv_csr;

/* Launch options of an apply.  Zero fields take the plan's defaults (which
 * napspmv_set_default_opts, e.g. from an autotuner, may change). */
typedef struct {
    int32_t precision;   /* NAPSPMV_PREC_F64 or NAPSPMV_PREC_F32               */
    int32_t engine;      /* NAPSPMV_ENGINE_DEFAULT, _FUSED, _PHASED, _OVERLAP  */
    int32_t vec;         /* lanes per matrix row: 1, 2, 4, 8, 16 or 32         */
    int32_t ctas_per_sm; /* resident CTAs per SM: the persistent CTAs of the
                            fused engine; a cap on the SpMV grid of the
                            phased / overlapped engines                       */
    int32_t chunk;       /* elements per message-step unit of the fused engine
                            (32 .. 2^24; the plan default is 2048)             */
    int32_t tile_rows;   /* at most this many matrix rows per SpMV work item   */
    int32_t tile_nnz;    /* at most this many stored entries per SpMV work item
                            (staged in shared memory by bulk copies); a longer
                            single row gets a tile of its own                  */
    int32_t stages;      /* shared-memory stages of the CTA and warp tile
                            pipelines (2..4)                                   */
    int32_t pipeline;    /* SpMV tiles of the phased / overlapped engines:
                            NAPSPMV_PIPELINE_CTA (a CTA per tile),
                            NAPSPMV_PIPELINE_WARP (each warp its own stages and
                            tiles of tile_rows / 8 rows, tile_nnz / 8 entries;
                            a CTA takes a contiguous run of tiles either way)
                            or NAPSPMV_PIPELINE_SELL (sliced rows, above)     */
    int32_t halo;        /* NAPSPMV_HALO_ON / _OFF (overlapped engine)         */
    int32_t timeout_ms;  /* limit of every device-side wait                    */
    int32_t debug_stall; /* test hook (fused engine): 1 makes the CTA of job
                            0's first unit wait on a counter nothing
                            increments, so the
                            launch ends with NAPSPMV_ERR_TIMEOUT after
                            timeout_ms.  After any device-side error every
                            kernel of the workspace skips its work until
                            napspmv_status clears the flag.                    */
} napspmv_opts;

/* Communication statistics of a plan.  Counts are numbers of messages and
 * of vector values; "max ... proc" is the maximum over sending processes (the
 * per-process figures the paper plots in Sec. 5).  Standard plan: the messages
 * of Eqs. P, D.  Node-aware plan: inter-node = the messages of Eq. I, one per
 * node pair; intra-node = J0 + J1 + J2 (Eqs. IL0, IL1, IL2), each step
 * counted on its own. */
typedef struct {
    int64_t std_msgs, std_vals, std_intra_msgs, std_intra_vals;
    int64_t std_inter_msgs, std_inter_vals;
    int64_t std_max_inter_msgs_proc, std_max_inter_vals_proc;
    int64_t std_max_intra_msgs_proc, std_max_intra_vals_proc;
    int64_t std_max_msg_vals;
    int64_t nap_inter_msgs, nap_inter_vals;
    int64_t j0_msgs, j0_vals, j1_msgs, j1_vals, j2_msgs, j2_vals;
    int64_t nap_intra_msgs, nap_intra_vals;
    int64_t nap_max_inter_msgs_proc, nap_max_inter_vals_proc;
    int64_t nap_max_intra_msgs_proc, nap_max_intra_vals_proc;
    int64_t nap_max_inter_msg_vals;
    int64_t node_pairs, bll_total, bnl_total, lbuf_total;
    int64_t nnz_on_process, nnz_on_node, nnz_off_node;
    /* Algorithmic bytes of one apply: the plain-SpMV stream
     * 4(N+1) + nnz (4 + s_val) + 8N (v) + 8N (w), and the message part: every
     * value moved by a gather (J2, J0, pack, unpack) costs 8 B read + 8 B
     * write + 4 B index, every value of the transfer g_send -> g_recv 8 + 8 + 4
     * (its destination index). */
    double bytes_csr_f64, bytes_csr_f32, bytes_msg;
    double plan_ms; /* wall time of napspmv_plan on the host clock */
} napspmv_stats;

/* Build the plans of A for n_p simulated processes, ppn per node.
 *   A      CSR (host or device memory), see napspmv_csr.
 *   n_p    1 <= n_p <= N;  ppn >= 1 (the last node may hold fewer processes).
 *   flags  NAPSPMV_F32_VALUES | NAPSPMV_MAP_TEXT or NAPSPMV_MAP_MAJORITY |
 *          NAPSPMV_MAP_SPLIT (not with MAJORITY) | NAPSPMV_PARTITION_STRIDED |
 *          NAPSPMV_COMPOSED_GATHERS; other bits: ERR_ARG.
 *   out    receives the plan; the caller frees it with napspmv_plan_destroy.
 * Runs on the current device and synchronises it.  Errors: ERR_ARG for a
 * malformed CSR or bad n_p / ppn, ERR_UNSUPPORTED beyond the size limits,
 * ERR_OOM, ERR_CUDA.  Paper: Secs. 2, 2.1, 4.1, 4.2 (all plan equations). */
int napspmv_plan(const napspmv_csr *A, int32_t n_p, int32_t ppn, uint32_t flags,
                 napspmv_plan_t **out);

/* w <- A v with the plan's default options (FP64).  v, w: device, N values,
 * must not overlap.  Asynchronous on `stream`.  Device-side failures (a wait
 * that timed out) are sticky and reported by napspmv_status.
 * Paper: Algorithm NAPSpMV (Sec. 4) with local_comm (Sec. 4.2). */
int napspmv_apply(napspmv_plan_t *P, const double *v, double *w, void *stream);

/* reps chained applies in one launch: x_0 = v, x_{k+1} = scale * A x_k, and
 * w <- x_reps.  v is not modified; the plan's workspace holds the
 * intermediate vector.  reps >= 1. */
int napspmv_apply_n(napspmv_plan_t *P, const double *v, double *w, int32_t reps, double scale,
                    void *stream);

/* As napspmv_apply_n with explicit options (NULL = defaults) and workspace
 * (NULL = the plan's own).  A workspace holds the receive buffers and the
 * fused engine's barrier words of one in-flight apply. */
int napspmv_apply_ex(napspmv_plan_t *P, napspmv_ws_t *ws, const double *v, double *w,
                     int32_t reps, double scale, const napspmv_opts *opts, void *stream);

/* The three-block SpMV step alone (the three local_spmv calls of Algorithm
 * NAPSpMV, Sec. 4): w <- scale (A_on_process v + A_on_node b_{l->l} +
 * A_off_node b_{nl->l}) with the receive buffers the workspace (NULL = the
 * plan's own) holds from its last apply.  For measuring the step on its own;
 * after an apply of v it reproduces that apply's w.  Asynchronous. */
int napspmv_spmv_step(napspmv_plan_t *P, napspmv_ws_t *ws, const double *v, double *w,
                      double scale, const napspmv_opts *opts, void *stream);

/* End-to-end variant on HOST vectors (pageable or pinned): copies v in,
 * runs reps chained applies, copies w out and synchronises `stream`.
 * Returns the device-side status like napspmv_status. */
int napspmv_apply_host(napspmv_plan_t *P, const double *v_host, double *w_host, int32_t reps,
                       double scale, void *stream);

/* Persistent launches over `count` independent applies (each with its own
 * plan, workspace, vectors, reps and scale): the batched form used by the
 * request server.  ws[i] may be NULL only if no other entry uses the same
 * plan's own workspace.  count <= 64; all plans on one device.  count = 1
 * runs as napspmv_apply_ex with the given options; count > 1 runs on the
 * fused engine, whatever engine `opts` names.  Options: each entry resolves
 * the fields of `opts` left 0 (or opts NULL) against its own plan's
 * defaults.  Entries whose resolved launch options agree share one fused
 * launch; the launches are issued on `stream` in order of each option set's
 * first entry.  Each entry's result is bit-identical to napspmv_apply_ex of
 * its plan on the fused engine with its resolved options, whatever else is
 * in the batch.  Errors stay per entry: an entry whose wait times out sets
 * its workspace's error flag (napspmv_ws_status) and its remaining work is
 * skipped; the other entries complete.  An invalid entry (NULL vector,
 * reps < 1, a shared workspace, options its plan cannot run) fails the whole
 * call before anything is launched. */
int napspmv_apply_batch(int32_t count, napspmv_plan_t *const *plans, napspmv_ws_t *const *ws,
                        const double *const *v, double *const *w, const int32_t *reps,
                        const double *scale, const napspmv_opts *opts, void *stream);

/* w <- A v (reps chained applies, as napspmv_apply_n) without allocating any
 * memory.  The paper has no counterpart: this serves callers that cannot
 * allocate device memory when they need a product, because another allocator
 * (a framework's memory pool) owns the device's free memory or because
 * cudaMalloc's implicit device synchronisation is not acceptable on their
 * path.  The plan must already exist (napspmv_plan allocates).
 *   - Receive buffers, the chain vector and barrier words come from one
 *     fixed array of 2^20 doubles (8 MiB) that this library reserves on every
 *     device that loads it, until the process exits.  Plans needing more
 *     (see below) are rejected with NAPSPMV_ERR_UNSUPPORTED and a message
 *     giving both sizes.
 *   - Every call shares that array and it keeps the last call's contents;
 *     the barrier words are cleared by each call.  Calls that overlap on the GPU
 *     (on different streams, or on different plans) race on it: order them.
 *   - The first call on a device looks the array's device address up (with
 *     that device current) and caches it for the life of the process: the
 *     cached address does not survive cudaDeviceReset on that device.
 *   - Scratch needed: 2 barrier words + b_{l->l} + b_{l->nl} + 2 g_send + b_{nl->l}
 *     values, plus N for the chain vector when reps > 1.
 *   - Uses the fused engine with the plan's default options and FP64
 *     values; device-side timeouts are reported by napspmv_status(P). */
int napspmv_apply_noalloc(napspmv_plan_t *P, const double *v, double *w, int32_t reps,
                          double scale, void *stream);

/* Synchronise `stream`, return and clear the plan's device-side status
 * (NAPSPMV_OK or NAPSPMV_ERR_TIMEOUT) of its own workspace. */
int napspmv_status(napspmv_plan_t *P, void *stream);
int napspmv_ws_status(napspmv_ws_t *ws, void *stream);

/* Extra workspaces for concurrent applies of one plan. */
int napspmv_ws_create(napspmv_plan_t *P, napspmv_ws_t **out);
void napspmv_ws_destroy(napspmv_ws_t *ws);

/* Statistics of the plan (host copy; no device work). */
int napspmv_plan_stats(const napspmv_plan_t *P, napspmv_stats *out);

/* Canonical plan arrays for comparison with an independent implementation.
 * which: NAPSPMV_LIST_* below.  buf: host int64 array of *count entries; with
 * buf == NULL, *count receives the required length.  Message lists are laid
 * out as [m, total, src[m], dst[m], ptr[m+1], idx[total]] with messages in
 * ascending (src, dst) and idx ascending within a message; src / dst are
 * processes (nodes for NAPSPMV_LIST_NODE).  BLL / BNL / LBUF hold one
 * "message" per process with a non-empty buffer, src = dst = process, idx
 * the global columns in buffer order.  NAPSPMV_LIST_TU is [m, send_proc[m],
 * recv_proc[m]]: the local process on the sending and receiving node that
 * carries node pair k of the NODE list.  NAPSPMV_LIST_SPLIT is [n, then 3
 * counts per row: on_process, on_node, off_node].  Synchronous. */
#define NAPSPMV_LIST_STD 0   /* P(r), D(r,t)               Eqs. P, D        */
#define NAPSPMV_LIST_NODE 1  /* N(n), E(n,m)               Eqs. N, E        */
#define NAPSPMV_LIST_INTER 2 /* G, I((p,n),(q,m))          Eqs. G, I        */
#define NAPSPMV_LIST_J0 3    /* on_node -> off_node        Eqs. L0, IL0     */
#define NAPSPMV_LIST_J1 4    /* off_node -> on_node        Eqs. L1, IL1     */
#define NAPSPMV_LIST_J2 5    /* on_node -> on_node         Eqs. L2, IL2     */
#define NAPSPMV_LIST_BLL 6   /* on-node receive buffer b_{l->l} per process */
#define NAPSPMV_LIST_BNL 7   /* off-node receive buffer b_{nl->l}           */
#define NAPSPMV_LIST_LBUF 8  /* aggregator buffer b_{l->nl}                 */
#define NAPSPMV_LIST_TU 9    /* T, U assignment            Eqs. T, U        */
#define NAPSPMV_LIST_SPLIT 10
int napspmv_plan_export(const napspmv_plan_t *P, int32_t which, int64_t *buf, int64_t *count);

/* Default options of the plan (used where a napspmv_opts field is 0). */
int napspmv_get_default_opts(const napspmv_plan_t *P, napspmv_opts *out);
int napspmv_set_default_opts(napspmv_plan_t *P, const napspmv_opts *opts);

/* Conjugate gradients with iterative refinement for SPD A.
 * Outer loop in FP64: r = b - A x with the FP64 apply, stop when
 * ||r|| / ||b|| <= rtol; otherwise solve A d = r approximately by CG whose
 * applies use the FP32-stored values (NAPSPMV_PREC_F32; the plan needs
 * NAPSPMV_F32_VALUES) with FP64 vectors and FP64 dot products, to relative
 * residual inner_rtol or inner_max iterations, then x += d.
 *   b, x   device, N values; x holds the initial guess on entry.
 *   info   optional: iterations and final relative residual.
 * Synchronous (polls the residual on the host every few iterations).
 * Errors: ERR_ARG, ERR_STATE (plan without FP32 values), ERR_TIMEOUT. */
typedef struct {
    int32_t outer_iters;
    int32_t inner_iters; /* total over all outer iterations */
    double relres;       /* ||b - A x|| / ||b||, FP64 */
    int32_t converged;
} napspmv_cg_info;
int napspmv_cg_ir(napspmv_plan_t *P, const double *b, double *x, double rtol, double inner_rtol,
                  int32_t max_outer, int32_t inner_max, napspmv_cg_info *info, void *stream);

/* Plain FP64 CG (no refinement), same conventions; for comparison. */
int napspmv_cg(napspmv_plan_t *P, const double *b, double *x, double rtol, int32_t max_it,
               napspmv_cg_info *info, void *stream);

/* One conjugate-gradient solve among several served together: its plan and
 * workspace (NULL = the plan's own; slots of one call must not share one),
 * the right-hand side b and device vectors x, r, p, q of N values, and 8
 * device doubles of scalars: [0] r.r, [1] p.q, [2] alpha, [3] beta,
 * [4] latest r.r, [5] b.b.  Not in the paper: the batched form of the
 * request server.  Each slot's arithmetic does not depend on the others in
 * the call: its dot products use a partition fixed by its own N (one block
 * per 1,024 values, at most 4,096) and a fixed-order final sum, and its
 * products run with its own plan's default options (slots whose options
 * differ go into separate fused launches). */
/* Slots (and served SpMV requests) whose matrix holds at least this many
 * stored entries are applied on their own with the phased engine: there one
 * product costs less than its share of a fused-engine launch. */
#define NAPSPMV_SOLO_NNZ (1ll << 19)

typedef struct {
    napspmv_plan_t *plan;
    napspmv_ws_t *ws;
    const double *b;
    double *x, *r, *p, *q;
    double *scal;
} napspmv_cg_slot;

/* For every slot: r = b - A x (apply at `precision`), p = r, scal[0] = r.r,
 * scal[5] = b.b.  With x_is_zero the apply is skipped and x is set to 0.
 * count <= 64.  Asynchronous. */
int napspmv_cg_batch_init(int32_t count, const napspmv_cg_slot *slots, int32_t precision,
                          int32_t x_is_zero, void *stream);

/* `iters` CG iterations for every slot: q = A p, alpha = r.r / p.q,
 * x += alpha p, r -= alpha q, beta = r.r_new / r.r, p = r + beta p.
 * Asynchronous; the caller reads scal[0] to decide convergence.
 * The products q = A p (and r = b - A x of napspmv_cg_batch_init): slots whose
 * matrix holds at least NAPSPMV_SOLO_NNZ stored entries are applied one by one
 * on the phased engine, the others together in one fused-engine launch.  The
 * choice depends on the slot's own matrix, not on the rest of the batch. */
int napspmv_cg_batch_iterate(int32_t count, const napspmv_cg_slot *slots, int32_t precision,
                             int32_t iters, void *stream);

/* y_i += x_i for count <= 64 pairs of device vectors of n_i values (the
 * refinement update x += d of served CG-IR solves).  Asynchronous. */
int napspmv_batch_add(int32_t count, double *const *y, const double *const *x, const int64_t *n,
                      void *stream);

/* Deterministic FP64 dot product of two device vectors of length n (fixed
 * partition and summation order, so the result does not depend on timing).
 * result: device pointer to one double.  Asynchronous. */
int napspmv_dot(const double *x, const double *y, int64_t n, double *result, void *stream);

void napspmv_plan_destroy(napspmv_plan_t *P);
const char *napspmv_strerror(int code);
const char *napspmv_last_error(void);
/* Number of kernel launches this thread queued through the library so far
 * (for the benchmark's launch count). */
int64_t napspmv_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* NAPSPMV_H */
