/*
 * kg.h -- C ABI of libkg.so: reverse-mode gradients of data-parallel functions
 * on one GB300 GPU (sm_103a).
 *
 * The method is that of Liegeois et al., "Performance Portable Gradient
 * Computations Using Source Transformation" (arXiv 2507.13204):
 *   - a gradient call runs the forward pass of the function and then its
 *     reverse pass (Sec. 3, opening paragraph of "Methodology");
 *   - the reverse of a sum reduction is a broadcast of the output adjoint
 *     (Sec. 3.2, reverse of deep_copy(view, scalar) and the parallel_sum
 *     helper); the output adjoint ("seed") defaults to 1 as in the paper's
 *     generated gradient (Sec. 4, Fig. "grad_f");
 *   - a read through an index map becomes a scatter-add of adjoints, which the
 *     paper makes atomic (Sec. 3.3, race-detection rules); this library offers
 *     that atomic scatter and an atomic-free gather over the transposed
 *     connectivity, the rescheduling the paper proposes as future work
 *     (Sec. 5, first restriction);
 *   - forward values needed by the reverse pass are recomputed or read from a
 *     tape allocated once outside the kernels (Sec. 5, third restriction).
 *
 * Problems ("kinds"):
 *   KG_QUADFORM   f(x; A) = ||A x||^2, A dense m x n, row-major.  Forward is a
 *                 team-per-row parallel_reduce then a sum reduction.
 *   KG_TETENERGY  f(u; conn, G) = sum_e log1p(|G_e u_e|^2): u_e gathers the 4
 *                 vertex values of tet e through conn (an index map), G_e is
 *                 the 3x4 matrix of P1 barycentric gradients.
 *   KG_SPQUADFORM f(x; A) = ||A x||^2, A sparse m x n in compressed sparse
 *                 rows (rowptr, col, val): the row loop runs over the stored
 *                 entries only and reads x through the index map col, so the
 *                 reverse pass is a scatter-add (or, rescheduled, a gather
 *                 over the transpose).
 *   KG_LAPLACE1D  the paper's example (Sec. 4, Fig. "function_f"):
 *                 f(x, b) = ||A (3 x) - b||^2, A = tridiag(-1, 2, -1).
 *
 * Conventions for every entry point:
 *   - All data pointers are DEVICE pointers unless the name ends in _host.
 *   - Element type is the problem's dtype (double for KG_F64, float for
 *     KG_F32); index arrays are int32.  Scalars such as f and the seed are
 *     single elements of that dtype, in device memory.
 *   - Inputs given to kg_create (A, conn, G, b) are BORROWED: the caller owns
 *     them and keeps them alive and unchanged until kg_destroy (kg_create
 *     scans them and may derive prepared copies from them, see
 *     tape_budget_bytes).
 *     All workspaces (partial sums, tape, transposed connectivity, error word)
 *     are allocated by kg_create / kg_batch_create; the per-call entry points
 *     kg_eval, kg_grad, kg_eval_tape, kg_grad_from_tape and kg_grad_batched
 *     allocate nothing.
 *   - Calls are asynchronous on the given stream (NULL = legacy default
 *     stream) and do not synchronise the host, except kg_create,
 *     kg_batch_create, kg_sync and the *_host entry points, which do.
 *   - Calls on one problem must be ordered on one stream: they share the
 *     problem's workspace.
 *   - Every entry point returns a kg_status and never aborts; on failure a
 *     message is kept per host thread and returned by kg_last_error().
 *     Device-side failures (out-of-range connectivity when checks are on, a
 *     bounded wait that ran out) set a sticky error word that kg_sync reads.
 */
#ifndef KG_H
#define KG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same object as cudaStream_t; NULL selects the legacy default stream. */
typedef struct CUstream_st *kg_stream;

typedef enum {
  KG_OK = 0,
  KG_ERR_INVALID_ARG = 1, /* bad size, NULL pointer, misaligned pointer, bad enum */
  KG_ERR_OOM = 2,         /* a workspace allocation failed (nothing is leaked) */
  KG_ERR_CUDA = 3,        /* a CUDA runtime call failed; message has the CUDA error */
  KG_ERR_BOUNDS = 4,      /* connectivity entry outside [0, N_v) */
  KG_ERR_TIMEOUT = 5,     /* a bounded device wait gave up */
  KG_ERR_UNSUPPORTED = 6, /* option combination not implemented for this kind */
  KG_ERR_STATE = 7,       /* call out of order (e.g. kg_grad_from_tape before a tape exists) */
  KG_ERR_RANGE = 8        /* PAIR arithmetic: an input outside 0 or [2^-60, 2^40) in magnitude;
                             the results of that call are invalid (rerun with KG_ARITH_NATIVE) */
} kg_status;

typedef enum { KG_QUADFORM = 1, KG_TETENERGY = 2, KG_LAPLACE1D = 3, KG_SPQUADFORM = 4 } kg_kind;
typedef enum { KG_F64 = 0, KG_F32 = 1 } kg_dtype;

/* Reverse-pass schedule for gathers (Sec. 3.3 and Sec. 5).
 *   ATOMIC    reuse the forward schedule; scatter-adds are atomic adds.
 *   CSR       (tet) atomic-free and bitwise run-to-run reproducible: the
 *             element adjoints of each tile of 32 consecutive elements are
 *             summed per tile vertex in a fixed order (the tiles of
 *             KG_STRATEGY_TILE, built at kg_create) into a partials buffer,
 *             then each vertex adds its tiles' partials in ascending order.
 *             FP64 problems in NATIVE arithmetic and bounds-checked problems
 *             reach the tile sums through the tape (per-element adjoints).
 *   TRANSPOSE (dense) a second kernel reads A by columns: xbar = A^T ybar.
 *             (sparse) atomic-free: a row kernel stores y, then a team per
 *             column of the transpose (built at kg_create) gathers
 *             xbar_j = 2 fbar sum_i a_ij y_i in ascending i; reproducible.
 *   FUSED     (dense) one pass over A: each team computes y_i, broadcasts
 *             ybar_i and accumulates ybar_i A_i,: into private partials that are
 *             summed in a fixed order; reproducible.  The TMA-streamed kernels
 *             (FP32, and FP64 in PAIR arithmetic with the prepared A for
 *             2048 < n <= 10240) sum them in their own tail after a bounded
 *             grid barrier, as one cooperative launch; the others (and these
 *             when the grid cannot be resident at once) in a second small
 *             kernel, with the same bits.
 *   SHARED    (tet) the forward schedule with the scatter-adds of each tile of
 *             elements first combined per vertex in a shared-memory table, then
 *             one global atomic per distinct vertex (Sec. 5: shared memory for
 *             temporaries to reduce atomics).
 *   WARP      (tet) the forward schedule with the scatter-adds combined within
 *             each warp: lanes whose element shares a vertex (in the same local
 *             slot) add their values by shuffles and one lane issues the
 *             atomic.  FP64 data combines runs of consecutive lanes (elements
 *             numbered along the mesh); FP32 data combines equal vertices
 *             anywhere in the warp.  The result holds for any element order.
 *   TILE      (tet) the reverse pass rescheduled per tile of 32 consecutive
 *             elements (Sec. 5: rescheduling the reverse pass): kg_create
 *             sorts each tile's 128 incidences by vertex, giving the tile's
 *             distinct vertices and their incidence lists; the gradient
 *             stores a warp's 32 element adjoints in shared memory, then one
 *             lane per tile vertex adds its incidences in ascending order and
 *             issues one global atomic.  Value-and-gradient and Hessian-vector
 *             products; FP32, or FP64 in PAIR arithmetic with the prepared G;
 *             no bounds checks (else KG_ERR_UNSUPPORTED).
 *   AUTO      FUSED for dense; for tets TILE with FP32 data (no bounds checks)
 *             and WARP otherwise; ATOMIC for sparse; the stencil transpose for
 *             1-D. */
typedef enum {
  KG_STRATEGY_AUTO = 0,
  KG_STRATEGY_ATOMIC = 1,
  KG_STRATEGY_CSR = 2,
  KG_STRATEGY_TRANSPOSE = 3,
  KG_STRATEGY_FUSED = 4,
  KG_STRATEGY_SHARED = 5,
  KG_STRATEGY_WARP = 6,
  KG_STRATEGY_TILE = 7
} kg_strategy;

/* Forward values for the reverse pass (Sec. 5, taping restriction).
 *   RECOMPUTE  kg_grad reruns the forward pass inside the gradient kernel.
 *   TAPE       kg_create allocates a tape (tet: the per-element adjoint
 *              c_e = G_e^T (2 g_e / (1 + |g_e|^2)), N_e x 4 values; 1-D:
 *              the chain's intermediate y = A (3x) - b, n values);
 *              kg_eval_tape fills it and kg_grad_from_tape consumes it.
 *   AUTO       tet: TAPE when the tape fits tape_budget_bytes, else
 *              RECOMPUTE; other kinds: RECOMPUTE. */
typedef enum { KG_MODE_AUTO = 0, KG_MODE_RECOMPUTE = 1, KG_MODE_TAPE = 2 } kg_mode;

/* FP64 arithmetic.  GB300 has few FP64 units (about 2 FMA per clock per SM),
 * so FP64 kernels can run their arithmetic as pairs of FP32 values
 * (hi + lo, at least 47 significant bits) on the FP32 units.
 *   NATIVE  FP64 instructions throughout.
 *   PAIR    FP32-pair arithmetic for the streamed products and sums
 *           (results within 1e-12 relative L2 of exact FP64 arithmetic for
 *           inputs in the normal FP32 exponent range); kernels that have no
 *           pair variant use NATIVE.
 *   AUTO    PAIR where a pair variant exists. */
typedef enum { KG_ARITH_AUTO = 0, KG_ARITH_NATIVE = 1, KG_ARITH_PAIR = 2 } kg_arith;

typedef struct {
  int dtype;                /* kg_dtype */
  int strategy;             /* kg_strategy */
  int mode;                 /* kg_mode */
  int arith;                /* kg_arith (FP64 only) */
  int check;                /* 1: kernels bounds-check conn and set KG_ERR_BOUNDS */
  int block;                /* threads per CTA; 0 = tuned default */
  int team;                 /* dense: threads per row team (32 or block); 0 = tuned */
  int tile;                 /* elements (tet) or rows (dense) per work tile; 0 = tuned */
  size_t tape_budget_bytes; /* cap on optional create-time workspaces; 0 = 1 GiB.
                             * FP64 problems in PAIR arithmetic first take a copy
                             * of A (QUADFORM, 8 m n bytes), G (TETENERGY,
                             * 96 N_e bytes) or the stored values (SPQUADFORM,
                             * 8 nnz bytes; required by its pair kernels, so
                             * AUTO stays NATIVE without it) split into float
                             * pairs, which the kernels stream instead of
                             * splitting on every call; KG_MODE_AUTO then takes
                             * the tet tape if it fits what is left */
} kg_options;

typedef struct kg_problem kg_problem;
typedef struct kg_batch kg_batch;

/* Fills *opt with defaults: KG_F64, AUTO strategy/mode/arith, check = 0.
 * No passage: library infrastructure. */
void kg_options_default(kg_options *opt);

/* Environment overrides, applied by kg_create on top of the caller's options
 * (so a run can switch schedules without a rebuild):
 *   KG_STRATEGY = auto | atomic | csr | transpose | fused | shared | warp | tile
 *   KG_MODE     = auto | recompute | tape
 *   KG_ARITH    = auto | native | pair
 *   KG_CHECK    = 0 | 1
 * Unset or empty variables leave the field alone.  An unknown value returns
 * KG_ERR_INVALID_ARG (message names the variable) and leaves *opt unchanged.
 * Host only; usable without a GPU.  No passage: library infrastructure. */
kg_status kg_options_apply_env(kg_options *opt);

/* Create a problem (Sec. 3.1: shadow storage for every intermediate is
 * allocated once, here, never inside the per-call entry points).
 *   kind   kg_kind.
 *   sizes  KG_QUADFORM: {n} (square) or {m, n};  KG_TETENERGY: {N_e, N_v};
 *          KG_LAPLACE1D: {n};  KG_SPQUADFORM: {m, n, nnz}.  All sizes >= 1
 *          and < 2^31 (nnz may be 0).
 *   data   device pointers, borrowed: KG_QUADFORM {A (m*n, row-major)};
 *          KG_TETENERGY {conn (int32, N_e*4), G (N_e*12, row-major 3x4 per
 *          element: G[e*12 + r*4 + k] = d lambda_k / d x_r)};
 *          KG_LAPLACE1D {b (n)};  KG_SPQUADFORM {rowptr (int32, m+1),
 *          col (int32, nnz, each in [0, n), repeats add), val (nnz)}.  A, conn,
 *          G and b must be 16-byte aligned; the sparse arrays element-aligned.
 *   opt    NULL for defaults.
 * Validates conn against [0, N_v) and the CSR structure (rowptr[0] = 0,
 * rowptr[m] = nnz, non-decreasing, columns in [0, n)) (KG_ERR_BOUNDS), builds
 * the transposed connectivity (tet CSR strategy) or the transposed matrix
 * (sparse TRANSPOSE strategy, values copied in column order), and synchronises
 * `s`.  The environment overrides of kg_options_apply_env are applied to opt
 * first. */
kg_status kg_create(kg_problem **out, int kind, const int64_t *sizes, int nsizes,
                    const void *const *data, int ndata, const kg_options *opt, kg_stream s);

/* Forward pass only (the primal function: Sec. 4, Fig. "function_f", whose
 * parallel_for / parallel_reduce kernels compute the value): *f = f(x).
 * x: n (QUADFORM, SPQUADFORM, LAPLACE1D) or N_v (TET); f: device scalar. */
kg_status kg_eval(kg_problem *p, const void *x, void *f, kg_stream s);

/* Value and gradient (the paper's gradient function: forward pass, seed,
 * reverse pass; Sec. 4, Fig. "grad_f").
 *   x      input (device), length n or N_v.
 *   f      nullable; receives f(x).
 *   gx     gradient w.r.t. x, length n or N_v.
 *   gdata  nullable; gradient w.r.t. the first data operand: A (m*n,
 *          QUADFORM), b (n, LAPLACE1D) or the stored values val (nnz,
 *          SPQUADFORM).  KG_ERR_UNSUPPORTED for TET.
 *   seed   nullable device scalar: the output adjoint fbar (NULL means 1).
 *   accumulate  0: gx/gdata are overwritten; 1: the gradient is added to
 *          them (the "_d_x +=" convention of the generated code). */
kg_status kg_grad(kg_problem *p, const void *x, void *f, void *gx, void *gdata,
                  const void *seed, int accumulate, kg_stream s);

/* TET and LAPLACE1D, TAPE mode: forward pass that also records, in the
 * problem's tape, the per-element adjoint factors c_e for fbar = 1 (TET) or the
 * intermediate y of the chain x -> y -> y^2 -> sum (LAPLACE1D).  f nullable. */
kg_status kg_eval_tape(kg_problem *p, const void *x, void *f, kg_stream s);

/* TAPE mode: reverse pass from the tape as the last call that wrote it left
 * it: kg_eval_tape, or (TET, CSR strategy in NATIVE arithmetic or with bounds
 * checks) kg_grad, whose reverse pass goes through the same tape.
 * kg_tape_generation tells the two apart.
 * TET: gx[v] (+)= fbar * sum over incidences (e,k) of v of c_e[k], by atomic
 * scatter, per-tile sums (TILE: one atomic per tile vertex; CSR: the
 * reproducible partials and vertex gather) (the problem's strategy); reads
 * no G.
 * LAPLACE1D: the reverse chain from y alone, ybar = 2 fbar y and
 * gx_j (+)= 3 (2 ybar_j - ybar_{j-1} - ybar_{j+1}); reads neither x nor b.
 * KG_ERR_STATE if no tape was recorded. */
kg_status kg_grad_from_tape(kg_problem *p, void *gx, const void *seed, int accumulate,
                            kg_stream s);

/* Number of launches so far that wrote the problem's tape (kg_eval_tape, and
 * kg_grad of a TET problem with the CSR strategy in NATIVE arithmetic or with
 * bounds checks).  A caller that records a
 * tape and replays it later (e.g. an autograd backward) compares the value
 * taken after its kg_eval_tape with the current one: if they differ, another
 * call overwrote the tape in between and the reverse pass must recompute.
 * Host-side counter; no synchronisation.  Tape restriction of Sec. 5. */
kg_status kg_tape_generation(const kg_problem *p, uint64_t *gen);

/* Hessian-vector product (forward mode over the reverse pass; the paper's
 * Sec. 5 lists forward mode as future work): hv (+)= fbar * H(x) v with H the
 * Hessian of f w.r.t. x.  TETENERGY: per element the tangent of the reverse
 * pass in direction v, scatter-added like the gradient (the problem's
 * scatter strategy; CSR uses atomics here); x is needed.  QUADFORM and
 * SPQUADFORM: f is a homogeneous quadratic, so H v is the gradient at v (x
 * unused, may be NULL).  LAPLACE1D: 18 fbar A^T A v (x unused).  v and hv:
 * length n or N_v; seed nullable (fbar = 1).  Allocates nothing. */
kg_status kg_hvp(kg_problem *p, const void *x, const void *v, void *hv, const void *seed,
                 int accumulate, kg_stream s);

/* End-to-end variant of kg_grad on HOST buffers (the paper's gradient
 * function returns its value to the host, Sec. 4, Fig. "grad_f"): copies x
 * (pageable or pinned host memory) to the device, runs kg_grad with seed 1 on
 * `s`, copies f and gx back and synchronises `s`.  f_host nullable. */
kg_status kg_grad_host(kg_problem *p, const void *x_host, void *f_host, void *gx_host,
                       kg_stream s);

/* Batched value-and-gradient of many independent problems (QUADFORM and
 * TETENERGY, FP64 or FP32, all of one dtype) in ONE persistent kernel launch
 * driven by a device work queue of (instance, tile) items, captured once in a
 * CUDA graph and replayed (Sec. 5, second restriction: fewer launches and
 * host synchronisation points).  kg_batch_create autotunes the tile and team
 * sizes (cached in $KG_TUNE_CACHE, default ~/.cache/kg_tune.json, keyed by GPU
 * name, kind and size bucket), builds the work table and synchronises `s`.
 * opt->strategy picks the tet scatter: AUTO or ATOMIC (one atomic per
 * contribution) or WARP (warp-combined atomics, see KG_STRATEGY_WARP); others
 * are KG_ERR_UNSUPPORTED.
 * FP64 batches in PAIR arithmetic stream float-pair copies of the data: the
 * instances' own (kg_create's), and for dense instances that have none (n <
 * 1024) one the batch makes at create, largest first, within
 * opt->tape_budget_bytes (0 = 1 GiB); the others split their FP64 data on
 * every load.  Like kg_create's, these copies are taken once: A must not
 * change while the batch lives.
 * The problems are borrowed and must outlive the batch. */
kg_status kg_batch_create(kg_batch **out, kg_problem *const *probs, int count,
                          const kg_options *opt, kg_stream s);

/* Batched value and gradient in one launch (Sec. 5, second restriction: the
 * gradient doubles the kernel launches and host synchronisation points, which
 * fewer, larger launches avoid).
 * x[i], f[i], gx[i]: device pointers for instance i (f[i] nullable).  The
 * pointer tables are host arrays of `count` entries; they are copied into the
 * batch's device table (a graph replay if unchanged since the last call). */
kg_status kg_grad_batched(kg_batch *b, const void *const *x, void *const *f, void *const *gx,
                          kg_stream s);

/* The batch's resolved FP64 arithmetic (kg_arith), number of work items in
 * its device table and persistent grid size.  Any pointer may be NULL.
 * No passage: library infrastructure. */
kg_status kg_batch_get_config(const kg_batch *b, int *arith, int *items, int *grid);

/* Same work as kg_grad_batched, issued as one kg_grad launch sequence per
 * instance on `s` (the per-instance launch loop the batch is compared with:
 * the launch pattern Sec. 5, second restriction, describes). */
kg_status kg_grad_batched_loop(kg_batch *b, const void *const *x, void *const *f,
                               void *const *gx, kg_stream s);

/* Allocation-free value and gradient of f(x) = ||A x||^2 in FP64 (the paper
 * has no counterpart: this entry point exists for callers that cannot
 * allocate device memory, e.g. code under a memory manager that owns the
 * whole device heap, or a loop that must never enter the allocator).
 *   A   m x n, row-major, device; x (n) device; f (device scalar, nullable);
 *   gx  (n) device, overwritten with the gradient (output adjoint 1).
 *   Limits: FP64 only, 1 <= m < 2^31, 1 <= n <= 12288; larger sizes return
 *   KG_ERR_INVALID_ARG with a message.  No handle, no cudaMalloc/cudaFree.
 * Scratch: a fixed 16 MiB array compiled into libkg.so, present on every GPU
 * that loads the library until the process exits.  The first call on a
 * device looks up its address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  Every call
 * shares the array and leaves its contents behind (the kernels overwrite
 * what they read, so nothing has to be cleared); calls that overlap on the
 * GPU race on it and must be serialised by the caller.  Asynchronous on `s`. */
kg_status kg_quadform_grad_noalloc(const double *A, int64_t m, int64_t n, const double *x,
                                   double *f, double *gx, kg_stream s);

/* Synchronises the problem's (batch's) last stream and reads its sticky
 * device error word (cleared by the read): KG_ERR_BOUNDS, KG_ERR_TIMEOUT,
 * KG_ERR_RANGE or KG_OK.  No passage: library infrastructure. */
kg_status kg_sync(kg_problem *p);
kg_status kg_batch_sync(kg_batch *b);

/* Check of the failure path of the bounded device waits: one warp waits,
 * through the same bounded mbarrier wait the TMA pipelines use, on an
 * mbarrier that nothing arrives at and no copy completes, with a limit of
 * limit_ns nanoseconds (0 < limit_ns <= 2e9) instead of the kernels' one
 * second.  The wait gives up, the kernel sets KG_ERR_TIMEOUT in the problem's
 * sticky error word and returns normally (no copy is in flight, no trap), so
 * the context stays usable; the next kg_sync returns KG_ERR_TIMEOUT.
 * Asynchronous on `s`.  No passage: library infrastructure (failure
 * detection of the waits every pipelined kernel uses). */
kg_status kg_check_bounded_wait(kg_problem *p, uint64_t limit_ns, kg_stream s);

/* Rates of this GPU that set the ALU rooflines of the native-FP64 kernels
 * (and motivate the float-pair arithmetic), measured by small kernels of the
 * library: eight independent register FMA chains per thread over 4 CTAs of
 * 256 threads per SM (FP64, FP32; FP64 log1p and division in the same
 * pattern), red.global.add to pseudo-random slots of an 8 MiB array
 * (FP64, FP32), and independent loads from the same slots (FP64, FP32; eight
 * in flight a thread).  Best of three timed launches each, after a
 * warm-up.  Allocates and frees an 8 MiB scratch array and synchronises `s`
 * (a characterisation call, not a per-call entry point).  No passage: device
 * characterisation for the roofline. */
typedef struct {
  double fp64_fma_tflops; /* FP64 FMA rate, 2 flops per FMA, 1e12 flop/s */
  double fp32_fma_tflops; /* FP32 FMA rate, 1e12 flop/s */
  double fp64_red_gops;   /* FP64 red.global.add to random L2-resident slots, 1e9/s */
  double fp32_red_gops;   /* FP32 red.global.add, same pattern, 1e9/s */
  double fp64_log1p_gops; /* FP64 log1p (CUDA's), eight dependent chains a thread, 1e9/s */
  double fp64_div_gops;   /* FP64 division, the same pattern, 1e9/s */
  int sms;                /* streaming multiprocessors */
  int l2_bytes;           /* L2 cache size */
  double fp64_gather_gops; /* FP64 loads from random L2-resident slots, 1e9/s */
  double fp32_gather_gops; /* FP32 loads, same pattern, 1e9/s */
} kg_box_rates;
kg_status kg_measure_box(kg_box_rates *out, kg_stream s);

/* Message for the last failure on this host thread ("" if none).
 * No passage: library infrastructure. */
const char *kg_last_error(void);

/* The configuration kg_create resolved from the options (AUTO replaced by the
 * choice made): kg_strategy, kg_mode and kg_arith.  Any pointer may be NULL.
 * No passage: library infrastructure. */
kg_status kg_get_config(const kg_problem *p, int *strategy, int *mode, int *arith);

/* Bytes of device workspace owned by the problem (tape, CSR, partials).
 * No passage: library infrastructure. */
size_t kg_workspace_bytes(const kg_problem *p);

/* Number of kernel launches the last per-call entry point issued on this
 * host thread (for launch accounting in benchmarks).
 * No passage: library infrastructure. */
int kg_last_launch_count(void);

/* Main-kernel timing for benchmarks.  While enabled (on this host thread),
 * every per-call entry point brackets its main kernel (the fused forward /
 * reverse kernel; not the small reduction or zero-fill launches) with CUDA
 * events recorded on the launch stream.  kg_profile_read waits for the
 * recorded events and returns the summed kernel time in milliseconds and the
 * number of bracketed launches since the last kg_profile_enable(1); name
 * receives a static string naming the last bracketed kernel.  Up to 65536
 * launches are kept; later ones are not timed.  Not for use inside CUDA graph
 * capture.  No passage: library infrastructure. */
kg_status kg_profile_enable(int on);
kg_status kg_profile_read(double *ms, int *launches, const char **name);

/* Free a problem's (batch's) workspaces; NULL is a no-op.  The borrowed
 * inputs are not freed.  No passage: library infrastructure. */
void kg_destroy(kg_problem *p);
void kg_batch_destroy(kg_batch *b);

#ifdef __cplusplus
}
#endif
#endif /* KG_H */
