/*
 * tbsweep -- exact amplitudes of open-boundary 1D brickwork circuits by the
 * temporal-boundary sweep, on one NVIDIA GB300 (sm_103a).
 *
 * The method (arXiv 2608.13110, Sec. 3.1, Algorithm 1 and Proposition 1):
 * the circuit's tensor network (Sec. 2.2) is contracted one qubit row at a
 * time. The running "temporal state" B holds 2^h complex64 entries,
 * h = ceil(d/2), one address bit per CZ layer in which the last absorbed row
 * still waits for its partner. Absorbing a row is a staircase of h paired
 * steps (consume one stored bit, create the next one), each a controlled 2x2
 * complex gate on two adjacent address bits; rows alternate time direction
 * (snake order) so that the width stays h. For odd d the odd rows wait in
 * h - 1 layers only (Proposition 1, odd case): a forward row's last step sums
 * it out and leaves the top address bit 0, and the next row's first step
 * creates its value of layer d-1 there; both are steps of the same form.
 *
 * Circuit convention: qubits q = 0..n-1, CZ layers l = 0..d-1, layer l acts
 * on (i, i+1) for every i = l (mod 2) with i+1 < n (Sec. 2.1); one-qubit
 * slots t = 0..d, slot t < d before CZ layer t and slot d after the last
 * layer; the gate of slot t on qubit q is U = E . T^tau . C, with C one of the
 * 24 Cliffords C_k = P_(k mod 4) . R_(k div 4), P in (I, X, Y, Z),
 * Y = [[0,-i],[i,0]], R in (I, H, S, S.H, H.S, H.S.H), T = diag(1, e^(i pi/4))
 * and E an optional arbitrary extra gate. Output: psi(x) = <x|U|0^n>, with
 * bit q of a bitstring the value of qubit q (Sec. 2.2).
 *
 * All functions return a tb_status code and never throw. Unless stated
 * otherwise, every pointer argument must be non-NULL.
 */
#ifndef TBSWEEP_H
#define TBSWEEP_H

#include <stdint.h>

#if defined(__GNUC__)
#define TB_API __attribute__((visibility("default")))
#else
#define TB_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
enum tb_status {
    TB_OK = 0,
    TB_EINVAL = 1,   /* NULL pointer, bit not in {0,1}, Clifford index > 23, bad size */
    TB_EDOMAIN = 2,  /* circuit outside what this build contracts: n < 2, d < 2,
                        ceil(d/2) > 40 for a plan, > 35 for evaluation */
    TB_ENOMEM = 3,   /* workspace smaller than tb_workspace_bytes() or host allocation failed */
    TB_ECUDA = 4,    /* a CUDA runtime call failed; tb_last_error() has the message */
    TB_ETIMEOUT = 5  /* a bounded device wait gave up, or a server wait timed out */
};

/* Opaque plan: the folded gates, the step tables and the pass schedule of one
 * circuit. Immutable after creation; safe to share between threads. */
typedef struct tb_plan tb_plan;

/* One arbitrary one-qubit gate, applied after the Clifford and T of its slot.
 * m: row-major 2x2 complex matrix as (re, im) pairs: m[0..1] = (0,0),
 * m[2..3] = (0,1), m[4..5] = (1,0), m[6..7] = (1,1). */
typedef struct {
    int32_t qubit; /* 0..n-1 */
    int32_t slot;  /* 0..d   */
    double m[8];
} tb_gate1q;

/* Pass arithmetic (tb_opts.precision). The split forms compose several
 * paired steps into a dense block so that tensor cores can apply them (the
 * paper's production code also combines small tensors before the boundary
 * contraction, Sec. 5.2, and compares complex64 with complex128 precision,
 * Sec. 5.1). */
enum {
    TB_PRECISION_FP32 = 0,
    TB_PRECISION_TF32X3 = 1,
    TB_PRECISION_BF16X3 = 2
};

/* Plan options. A zeroed struct (or NULL) selects the defaults. */
typedef struct {
    int32_t window_bits;  /* largest number of address bits one boundary pass
                             covers (5..10; 0 = default 10) */
    int32_t bottom_bits;  /* size of the window at address bit 0 (5..10; 0 = auto) */
    int32_t top_bits;     /* size of the window ending at bit h-1 (5..10; 0 = auto) */
    int32_t precision;    /* arithmetic of the boundary passes (boundaries wider
                             than 12 bits; narrower ones always use the first):
                             TB_PRECISION_FP32 (0, default): the staircase of
                               controlled 2x2 steps in FP32 FMA;
                             TB_PRECISION_TF32X3 / TB_PRECISION_BF16X3: the steps
                               of each pass composed on the host into one dense
                               complex matrix over 5 (TF32) or 6 (BF16) address
                               bits and applied with tensor-core MMAs as three
                               split products hi.hi + hi.lo + lo.hi accumulated
                               in FP32 (window options are then ignored). */
    int64_t hbm_budget_bytes; /* cap on the boundary batch a call keeps on the
                                 device (0 = no cap beyond the workspace); an
                                 open plan whose budget cannot hold two
                                 boundaries works in place (see
                                 tb_plan_create_open) */
} tb_opts;

/* Plan summary. */
typedef struct {
    int32_t n, d;
    int32_t width;          /* W of Algorithm 1's path, log2 of the largest
                               intermediate (Sec. 2.2 contraction width) */
    int32_t boundary_bits;  /* h: the device boundary holds 2^h complex64 */
    double log2_cost;       /* log2 C, C = sum over Algorithm 1's pairwise
                               contractions of |I||J||K| (Sec. 2.2) */
    int64_t boundary_bytes; /* 8 * 2^h */
    int32_t n_steps;        /* paired steps on the device (rows 1..n-2) */
    int32_t n_passes;       /* HBM passes over the boundary per amplitude
                               (0 when the whole boundary fits one CTA) */
    int64_t table_bytes;    /* device bytes of the plan's tables */
    int32_t open_k;         /* open output bits of an open plan, 0 otherwise */
    int32_t open_width;     /* open plans: width of Algorithm 2's path,
                               max(h, 2k) (Proposition 2: h for k <= d/4) */
    int32_t pass_madds;     /* real multiply-adds per boundary entry that
                               the FP32 pass kernels spend per amplitude: 8
                               per paired step, 16 per row turn, whose four
                               steps on two address bits run as one 4x4
                               block; 0 without passes */
} tb_plan_info_t;

/* Create a plan (host only: no CUDA call is made): the circuit of Sec. 2.1
 * folded into the network of Sec. 2.2 (one-qubit gates absorbed into the
 * neighbouring tensors), the paired steps of Algorithm 1 for every absorbed
 * row (Sec. 3.1, Proposition 1), the pass schedule that fuses consecutive
 * steps of a window of address bits, and the counters W and C.
 *   n, d   : qubits and CZ layers; n >= 2, 2 <= d, ceil(d/2) <= 40 (odd or
 *            even d)
 *            (else TB_EDOMAIN). Plans wider than 35 bits (2^35 complex64 =
 *            256 GiB, the most one GPU's HBM holds) only report their
 *            counters: evaluating them returns TB_EDOMAIN and
 *            tb_workspace_bytes returns -1.
 *   cliff  : (d+1)*n Clifford indices 0..23, slot-major (cliff[t*n + q]);
 *            NULL means identity everywhere.
 *   tmask  : d*n bytes in {0,1}, tmask[t*n + q] = 1 puts a T after the
 *            Clifford of slot t < d; NULL means no T gate.
 *   extra  : n_extra arbitrary gates (may be NULL when n_extra == 0).
 *   opts   : NULL or a tb_opts (zero fields = defaults).
 *   out    : receives the plan; release it with tb_plan_destroy.
 * The input arrays are copied; the caller keeps ownership. */
TB_API int tb_plan_create(int n, int d, const uint8_t* cliff, const uint8_t* tmask,
                   const tb_gate1q* extra, int n_extra, const tb_opts* opts,
                   tb_plan** out);

/* Create an open plan: the output bits of the last k qubits stay open and
 * one evaluation returns all 2^k amplitudes <a,b|U|0^n> sharing the prefix a
 * (Algorithm 2, Sec. 4 "Constructive path for batched sampling"): the sweep of
 * Algorithm 1 absorbs rows 0..n-k-1 (the fixed region), the early region (the
 * open band's first 2k CZ layers) is contracted on the host in FP64 into a
 * 2^k x 2^k matrix and joined with the boundary over the k shared bits on the
 * device, then the late region is absorbed layer by layer, each crossing CZ
 * with row n-k-1 contracting one boundary bit.
 *   k: 1 <= k <= min(floor(d/4), 10, n-1) (else TB_EDOMAIN); ceil(d/2) >= 13.
 * Other arguments as tb_plan_create. Evaluate with tb_amplitudes /
 * tb_amplitudes_device, where a row of the input is the prefix
 * a = (x_0..x_(n-k-1)) (n-k bytes) and the output holds 2^k amplitudes per
 * prefix, index y = sum_j b_j 2^j with b_j the output bit of qubit n-k+j. The
 * workspace holds two boundaries per prefix evaluated concurrently: for
 * k >= 4 the join runs on the tensor cores and writes its product out of
 * place. When the boundary is wider than 2^33 entries, or the plan's
 * hbm_budget_bytes cannot hold two boundaries, the plan works in place: the
 * join runs in FP32 over the boundary itself and each late crossing writes
 * its output rows over its input rows (one boundary per prefix; 2^35
 * entries = 256 GiB at most). tb_workspace_bytes accounts for either.
 * tb_amplitudes_noalloc, batches and servers reject open plans (TB_EINVAL). */
TB_API int tb_plan_create_open(int n, int d, const uint8_t* cliff, const uint8_t* tmask,
                               const tb_gate1q* extra, int n_extra, const tb_opts* opts, int k,
                               tb_plan** out);

/* Create a plan whose entanglers are controlled phases. Sec. 2.1 admits any
 * two-qubit entangler of operator Schmidt rank 2 in the brickwork; the sweep
 * only ever uses the diagonal factor w^(s s') that such a gate contributes for
 * the two qubits' values s, s' in its layer (w = -1 is CZ), so each entangler
 * here is diag(1, 1, 1, e^(i phi)).
 *   cphase: NULL (every entangler is CZ) or d*(n-1) angles in radians,
 *           cphase[l*(n-1) + i] for the pair (i, i+1) in layer l; entries of
 *           pairs a layer does not couple (i != l mod 2) are ignored. A
 *           non-finite angle of a coupled pair returns TB_EINVAL; phi = pi
 *           exactly gives the same plan as CZ. The array is copied.
 *   open_k: 0 for a plain plan (as tb_plan_create), else the open bits of
 *           tb_plan_create_open with its domain.
 * Other arguments, evaluation and errors as tb_plan_create. Width and cost
 * counters do not depend on the angles. With one-qubit gates on either side
 * (folded into the neighbouring slots through extra) this covers every gate
 * of operator Schmidt rank 2: in the canonical form (A x B) exp(i(c1 XX +
 * c2 YY + c3 ZZ)) (C x D) rank 2 leaves one nonzero c, which local gates turn
 * into exp(i c ZZ) = e^(-ic) (Rz(-2c) x Rz(-2c)) diag(1, 1, 1, e^(4ic)),
 * Rz(t) = diag(e^(-it/2), e^(it/2)). */
TB_API int tb_plan_create_cphase(int n, int d, const uint8_t* cliff, const uint8_t* tmask,
                                 const tb_gate1q* extra, int n_extra, const double* cphase,
                                 const tb_opts* opts, int open_k, tb_plan** out);

/* Batched sampling from open-plan amplitudes (Sec. 4, "Batched sampling"):
 * for each of na prefixes with amplitudes amps[a*2^k .. (a+1)*2^k) ((re, im)
 * pairs, host FP64), Q_a = sum_b |amp|^2 and the suffix b drawn from
 * p(b | a) = |amp(a, b)|^2 / Q_a by inverting its distribution function at the
 * uniform variate u[a] in [0, 1) (the smallest b whose cumulative mass exceeds
 * u[a] Q_a; the random numbers are inputs). Writes b[a] and, if q is not NULL,
 * q[a] = Q_a. Host only. Returns TB_EINVAL for NULL pointers, k outside 0..30 or
 * u outside [0, 1). */
TB_API int tb_batched_sample(const double* amps, int k, int64_t na, const double* u, int32_t* b,
                             double* q);

/* Fill *info: sizes of the plan and Algorithm 1's counters (Sec. 2.2). */
TB_API int tb_plan_info(const tb_plan* plan, tb_plan_info_t* info);

/* Device workspace bytes that tb_amplitudes / tb_amplitudes_device need to
 * evaluate nb bitstrings (tables, rescaling state, partial sums and one
 * boundary per bitstring evaluated concurrently: the temporal state of
 * Sec. 3.1 is 2^h complex64). Returns -1 on a bad
 * argument. The batch a call evaluates concurrently is the largest that fits
 * the workspace given (and the plan's hbm_budget_bytes). */
TB_API int64_t tb_workspace_bytes(const tb_plan* plan, int64_t nb);

/* Smallest workspace that can evaluate any number of bitstrings (one
 * boundary at a time). */
TB_API int64_t tb_workspace_min_bytes(const tb_plan* plan);

/* Copy the plan's tables into the head of a device workspace, on stream
 * (asynchronous with respect to the host for pinned memory; the plan's host
 * tables must outlive the copy, which they do while the plan lives).
 *   d_ws  : caller-owned device memory, at least tb_workspace_min_bytes().
 *   stream: a cudaStream_t, or NULL for the legacy default stream. */
TB_API int tb_plan_upload(const tb_plan* plan, void* d_ws, int64_t ws_bytes, void* stream);

/* Amplitudes psi(x) = <x|U|0^n> (Sec. 2.2) by Algorithm 1 (Sec. 3.1) from
 * device-resident inputs, fully asynchronous on stream.
 *   d_bits: device, nb*n bytes, d_bits[i*n + q] = x_q in {0,1} (values are
 *           not checked on the device; anything nonzero counts as 1).
 *   d_ws  : workspace that tb_plan_upload filled for this plan.
 *   d_out : device, 2*nb doubles, (re, im) of psi(x_i) in FP64.
 * Work is enqueued only; no synchronisation. */
TB_API int tb_amplitudes_device(const tb_plan* plan, const uint8_t* d_bits, int64_t nb,
                         void* d_ws, int64_t ws_bytes, double* d_out, void* stream);

/* Amplitudes psi(x) = <x|U|0^n> (Sec. 2.2, Algorithm 1) end to end from host
 * buffers: uploads the tables, copies the
 * bitstrings host->device, runs the sweep, copies the amplitudes back and
 * synchronises the stream before returning.
 *   bits : host, nb*n bytes in {0,1} (checked: TB_EINVAL otherwise).
 *   d_ws : caller-owned device workspace of at least
 *          tb_workspace_min_bytes() + nb*(n + 16) bytes rounded up; it also
 *          holds the staged inputs and outputs.
 *   out  : host, 2*nb doubles (re, im). */
TB_API int tb_amplitudes(const tb_plan* plan, const uint8_t* bits, int64_t nb, void* d_ws,
                  int64_t ws_bytes, double* out, void* stream);

/* The pass schedule (the windows in which Algorithm 1's paired steps are
 * fused into one HBM pass each; the fusion is this library's): for pass i, sched[3*i] = shape (0 forward window,
 * 1 reversed window, 2 turn at the top, 3 turn at address bit 0, 4 first
 * window of the first absorbed row, 5 last window of a reversed last row,
 * 6 last window of a forward last row, 7 dense tensor-core block of a
 * TF32X3 / BF16X3 plan), sched[3*i+1] = window bits M,
 * sched[3*i+2] = address bit of the window's lowest bit. Writes at most cap
 * passes (sched may be NULL when cap == 0) and returns the number of passes,
 * or -1 for a NULL plan. */
TB_API int tb_plan_schedule(const tb_plan* plan, int32_t* sched, int cap);

/* ---- Batches of circuits -------------------------------------------------
 * Many independent circuits (the paper evaluates many contractions of one
 * topology as independent jobs, Sec. 5.2; here n and d may differ) recorded
 * once into a CUDA graph and replayed with one launch. Narrow circuits
 * (width <= 12) share a single kernel launch, one CTA per bitstring; wider
 * ones evaluate all their bitstrings side by side and run on parallel graph
 * branches balanced by estimated cost. */
typedef struct {
    const tb_plan* plan;   /* must outlive the batch */
    const uint8_t* d_bits; /* device, nb*n bytes (x_q at [i*n + q]) */
    int64_t nb;
    double* d_out;         /* device, 2*nb doubles (re, im) */
} tb_batch_item;

typedef struct tb_batch tb_batch;

/* Workspace bytes a batch of these items needs (-1 on a bad item). */
TB_API int64_t tb_batch_workspace_bytes(const tb_batch_item* items, int nitems);

/* Upload every plan's tables into d_ws (synchronously on stream), then
 * record the batch's work into a graph. nbranches: parallel branches for the
 * wide circuits (0 = 4, at most 16). Device pointers of the items are baked
 * into the graph: rewrite the buffers, not the pointers, between launches. */
TB_API int tb_batch_create(const tb_batch_item* items, int nitems, void* d_ws, int64_t ws_bytes,
                           int nbranches, void* stream, tb_batch** out);

/* Replay the recorded batch on stream (asynchronous). */
TB_API int tb_batch_launch(tb_batch* batch, void* stream);

/* Release a batch (NULL is ignored). */
TB_API void tb_batch_destroy(tb_batch* batch);

/* ---- Serving -------------------------------------------------------------
 * A server keeps plans' tables resident on the device and admits amplitude
 * requests of any size while others run: it owns one device arena (its HBM
 * budget, allocated once at creation) and `slots` CUDA streams; a dispatcher
 * thread starts queued requests in arrival order whenever a slot is free and
 * the arena holds the request's tables plus at least one boundary (tables no
 * running request uses are evicted least recently used first), polls their
 * completion events and copies the amplitudes to the caller's buffer. The
 * paper reuses plan and workspace caches across its contractions (Sec. 5.2);
 * this applies the same reuse to a stream of independent requests. */
typedef struct tb_server tb_server;

typedef struct {
    int64_t hbm_budget_bytes; /* device arena (0 = 16 GiB) */
    int32_t slots;            /* concurrent requests (0 = 4, at most 64) */
    int32_t device;           /* CUDA device ordinal */
    int64_t pinned_bytes;     /* pinned host staging (0 = 64 MiB) */
} tb_server_opts;

typedef struct {
    double latency_s; /* submit -> amplitudes in the caller's buffer */
    double queue_s;   /* submit -> admitted to a slot */
    double run_s;     /* admitted -> done */
    int32_t status;
    int32_t slot;
} tb_request_stats;

typedef struct {
    int64_t completed, amplitudes, peak_concurrent, peak_bytes_in_use, queued;
    double p50_latency_s, p99_latency_s, mean_latency_s;
} tb_server_stats_t;

/* Create a server (allocates its arena and pinned staging, starts the
 * dispatcher thread). */
TB_API int tb_server_create(const tb_server_opts* opts, tb_server** out);

/* Queue nb host bitstrings (nb*n bytes in {0,1}, copied during the call) of
 * plan; the amplitudes go to out (host, 2*nb doubles) when the request
 * completes. The plan and out must stay valid until tb_server_wait returns.
 * A request that cannot fit the budget even alone returns TB_ENOMEM. */
TB_API int tb_server_submit(tb_server* server, const tb_plan* plan, const uint8_t* bits, int64_t nb,
                            double* out, int64_t* ticket);

/* Wait for a request (timeout_s < 0: no limit; TB_ETIMEOUT when it runs out,
 * stats untouched and the ticket still valid). Once the request has finished,
 * returns its status (TB_ETIMEOUT there means a bounded device wait of its
 * kernels gave up and out is not written; stats->status says the same) and
 * consumes the ticket; fills stats. */
TB_API int tb_server_wait(tb_server* server, int64_t ticket, double timeout_s, tb_request_stats* stats);

/* Counters and latency percentiles of completed requests. */
TB_API int tb_server_stats(tb_server* server, tb_server_stats_t* out);

/* Finish every queued request, stop the dispatcher, free the server. */
TB_API void tb_server_destroy(tb_server* server);

/* Kernel timing (tracing aid). While enabled, every kernel this library
 * launches is bracketed by CUDA events on its stream. Classes: 0 boundary
 * passes, 1 row-0 writer, 2 last-row reduction, 3 finalisation, 4 narrow
 * (whole boundary in shared memory), 5 open-plan join, 6 open-plan late
 * crossings. bytes[c] is the algorithmic HBM traffic of those launches: a
 * pass or a join reads and writes every boundary entry once (16 bytes per
 * entry), the writer writes 8, the reduction reads 8, a late crossing reads
 * two entries and writes one (24 bytes per output entry). */
#define TB_PROFILE_CLASSES 7
typedef struct {
    int64_t launches[TB_PROFILE_CLASSES];
    double ms[TB_PROFILE_CLASSES];
    double bytes[TB_PROFILE_CLASSES];
} tb_profile_t;

/* Start recording (clears earlier records). Process-wide; not reentrant. */
TB_API int tb_profile_begin(void);

/* Stop recording, wait for the recorded events and sum them into *out. */
TB_API int tb_profile_end(tb_profile_t* out);

/* Amplitudes without allocating: like tb_amplitudes_device, but the tables,
 * rescaling state and boundary live in a fixed 64 MiB scratch array compiled
 * into this library, so the call needs no workspace and calls no cudaMalloc.
 * The paper has no counterpart; this entry exists for callers that cannot
 * allocate device memory at the point of use: processes whose device memory is
 * capped by a quota someone else owns, and plugins or libraries embedded in a
 * host application that tracks every device allocation and must not see
 * untracked ones.
 *   d_bits: device, nb*n bytes; d_out: device, 2*nb doubles (re, im).
 * Limits and behaviour:
 *   - plans whose tables plus one boundary exceed 64 MiB (for n = 70: width
 *     above 22) return TB_ENOMEM;
 *   - the first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream capture;
 *   - every call on a device shares the one array and leaves its contents
 *     behind; calls that overlap on the GPU (other streams, other threads)
 *     race and corrupt each other's results: serialise them;
 *   - work is enqueued on stream; no synchronisation. */
TB_API int tb_amplitudes_noalloc(const tb_plan* plan, const uint8_t* d_bits, int64_t nb, double* d_out,
                                 void* stream);

/* log-XEB estimator F = gamma + n ln 2 + (1/N) sum_i ln |amp_i|^2 (Sec. 5.2,
 * normalized log-XEB equation), host FP64. amp: 2*nb doubles (re, im).
 * A zero amplitude gives -inf. */
TB_API int tb_log_xeb(const double* amp, int64_t nb, int n, double* out);

/* The same estimator on the device, in FP64 (Sec. 5.2, normalized log-XEB
 * equation; the final reduction of the sweep's amplitudes stays on the GPU).
 *   d_amp : device, 2*nb doubles (re, im), e.g. the d_out of
 *           tb_amplitudes_device; read only.
 *   nb    : number of amplitudes, >= 1.
 *   n     : number of qubits (the n ln 2 term).
 *   d_out : device, one double; receives F.
 *   stream: cudaStream_t (NULL: legacy default stream). The reduction is
 *           enqueued after the work already on the stream and the call returns
 *           without synchronising.
 * One CTA sums ln |amp|^2 in a fixed order (deterministic); a zero amplitude
 * gives -inf. Returns TB_OK, TB_EINVAL (NULL pointer, nb < 1, n < 1) or
 * TB_ECUDA (launch failure). */
TB_API int tb_log_xeb_device(const double* d_amp, int64_t nb, int n, double* d_out, void* stream);

/* The Clifford table this library uses: m receives C_k as in tb_gate1q. */
TB_API int tb_clifford_matrix(int k, double m[8]);

/* Release a plan (NULL is ignored). */
TB_API void tb_plan_destroy(tb_plan* plan);

/* Static description of a status code. */
TB_API const char* tb_status_str(int status);

/* Message of the last failed call on this host thread ("" if none). */
TB_API const char* tb_last_error(void);

/* Device-side wait failures (no counterpart in the paper). Every spin-wait in
 * the library's kernels (the FP32 passes wait for their tile copies and for
 * their consumer warps, the tensor-core passes for their MMAs) gives up after
 * a bounded number of tries; a kernel that gives up counts it in a fault word,
 * writes nothing more for the affected tiles (the amplitudes of that call are
 * not valid) and exits cleanly, so the context stays usable.
 *   - tb_amplitudes and server requests use a fault word of their own and
 *     return TB_ETIMEOUT when it is nonzero;
 *   - tb_amplitudes_device, tb_amplitudes_noalloc and batches are
 *     asynchronous: their kernels count in the library-wide word, which the
 *     caller reads here after synchronising.
 * A tensor-core pass that cannot confirm that its last MMAs completed keeps
 * its tensor memory rather than free it under a running MMA; after that the
 * library refuses further split-precision evaluations in this process
 * (TB_ECUDA).
 * *count receives the number of failed waits since the last call on the
 * current device, and the word is cleared. Synchronises the device.
 * Returns TB_OK, TB_EINVAL (NULL count) or TB_ECUDA. */
TB_API int tb_device_faults(int32_t* count);

/* Self-test of the bounded device waits (no counterpart in the paper), with
 * no fault of any kind: (1) one small split-precision evaluation (n = 3,
 * d = 26, 3xBF16, asynchronous entry) whose tensor-core kernels wait for MMAs
 * that are never issued; (2) one FP32 evaluation of the same size through
 * tb_amplitudes whose pass kernels wait for tile copies that are never issued
 * and must return TB_ETIMEOUT. Each wait gives up after a short bounded number
 * of tries and is counted; the kernels stop and exit, so the device stays
 * usable. *faults receives the number of CTAs whose waits gave up in both
 * parts (positive when the mechanism works); the results are discarded.
 * Allocates and frees small workspaces; synchronises the device. Returns
 * TB_OK, TB_EINVAL (NULL faults) or TB_ECUDA (including: the synchronous entry
 * did not report the give-up). */
TB_API int tb_selftest_bounded_wait(int32_t* faults);

#ifdef __cplusplus
}
#endif

#endif /* TBSWEEP_H */
