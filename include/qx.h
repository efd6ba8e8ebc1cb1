/*
 * qx.h -- C ABI of libqx: sliced contraction of a quantum-circuit tensor
 * network to output amplitudes on one GB300 (sm_103a).
 *
 * The calls follow the paper's statement of the problem (arXiv 2110.09894):
 *   - build the tensor network of a circuit (Sec. II: |0> inputs, gate tensors
 *     attached to the open legs of their qubits in circuit order, outputs
 *     closed by <x_q| except on qubits left open);
 *   - take a contraction plan: a pairwise order (Sec. III-A) and a set of
 *     sliced bonds (Sec. III-A, Eq. 2);
 *   - contract for a list of bitstrings to get amplitudes <x|C|0> (Sec. II),
 *     summing the sliced sub-networks in FP64 with compensated summation.
 *
 * Canonical labels, so that a plan made elsewhere addresses this network:
 *   tensor ids  0..n-1        input |0> of qubit q
 *               n..n+G-1      gates in list order
 *               n+G..         one output <x_q| per CLOSED qubit, increasing q
 *   bond ids    0..n-1        the input wires
 *               n..           each gate's output legs in creation order
 *                             (gate g on (q0,q1) creates q0's leg, then q1's)
 *   plan        order[t] = {i, j}: step t contracts tensors i and j (each id
 *               used once) into the new tensor with id N_tensors + t; a full
 *               plan has N_tensors - 1 steps.
 *   slices      slice s fixes sliced[j] to bit j of s, s in [0, 2^n_sliced).
 *
 * Amplitude layout: out[b][o] (complex128 as {re, im} doubles) for bitstring
 * b and open-qubit assignment o, the first open qubit (lowest qubit index)
 * being the most significant bit of o.  Bit order of a state: qubit 0 is the
 * most significant bit; a bitstring is n bytes, byte q = value of qubit q.
 *
 * Memory and streams: every device buffer the library touches is either
 * caller-owned (qx_bind_workspace, qx_contract_device) or, only when the
 * caller passes NULL to qx_bind_workspace, allocated once there.  No
 * call allocates inside qx_contract / qx_contract_device.  All device work
 * is issued on the stream given to qx_create (NULL = legacy default stream).
 *
 * Errors: every int-returning call gives QX_OK (0) or a negative code and
 * leaves a message for qx_last_error; on error no partial result is written.
 * Handles are not thread-safe: one host thread drives a handle at a time.
 */
#ifndef QX_H
#define QX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QX_OK        0
#define QX_EINVAL   -1  /* malformed circuit, plan, bitstring or argument */
#define QX_ENOMEM   -2  /* the bound workspace is too small for the request */
#define QX_ECUDA    -3  /* a CUDA runtime call or kernel launch failed */
#define QX_ETIMEOUT -4  /* a bounded device wait expired */
#define QX_ESTATE   -5  /* call out of order (e.g. contract before plan) */

/* Precision forms of the contraction (the cross-slice sum is always FP64). */
#define QX_PREC_C64         0  /* complex64 operands, FP32 FMA (plain form)   */
#define QX_PREC_3XTF32      1  /* tcgen05 TF32, 3-product compensated split   */
#define QX_PREC_SPLIT_BF16  2  /* tcgen05 BF16, 3-way split, 6 products       */
#define QX_PREC_FP16_SCALED 3  /* tcgen05 FP16 with per-tensor power-2 scale  */
/* The tensor-core forms apply to contraction steps with M >= 128, N >= 64 and
 * K >= 32 (complex; the larger free side is taken as M); every other step runs
 * in the complex64 SIMT kernels. */

typedef struct qx_ctx* qx_handle;

/* One gate: nq = 1 or 2 target qubits q[0] (, q[1]); explicit unitary,
 * row-major, 2x2 or 4x4 in the basis |q0 q1> (row = 2*b(q0) + b(q1)).
 * Entries beyond nq's matrix are ignored.  272 bytes. */
typedef struct {
    int32_t nq;
    int32_t q[2];
    int32_t pad;
    double re[16];
    double im[16];
} qx_gate;

typedef struct {
    int32_t precision;       /* QX_PREC_*                                     */
    int32_t max_items;       /* (slice, bitstring) pairs per batch; 0 = fill  */
    int32_t gemm_min_bits;   /* steps with k, m, n >= this run as GEMM; 0 = 5 */
    int32_t executor;        /* 0 auto (= 1), 1 one launch per step over a
                                batch of pairs, 2 persistent (one launch, one
                                pair per CTA at a time; plans without
                                tensor-core steps), 3 member of a group (see
                                qx_group_*; contracts only through the group).
                                Read by qx_set_plan: plans compiled for 0 / 1
                                may store products in the layout the next
                                GEMM reads and fuse the last permute into the
                                dot, which only the batched launches do, so
                                set 2 or 3 before qx_set_plan */
    int64_t timeout_cycles;  /* bound on each device spin-wait, in SM clock
                                cycles; 0 = default (2e9).  An expired wait
                                makes the call report QX_ETIMEOUT (through
                                qx_device_status for the enqueue-only calls);
                                a new value drops a captured graph */
    int32_t no_slice_level;  /* read by qx_set_plan.  0 (default): with
                                executor 0 / 1, intermediates that depend on
                                the slice but on no output bit are computed
                                once per slice and shared by the slice's
                                bitstrings; 1: once per (slice, bitstring)
                                pair, as executors 2 and 3 always do.  The
                                amplitudes agree to FP32 rounding (launches
                                over fewer items may pick other tiles). */
    int32_t pad;
} qx_options;

/* Create a handle on CUDA device `device`; `cuda_stream` is a cudaStream_t
 * (may be NULL).  device = -1 gives a host-only handle that can build
 * networks, check plans and size workspaces but not contract.  opt may be
 * NULL for defaults.  *h is owned by the caller and released by qx_destroy.
 * QX_ECUDA for a device that does not exist, QX_EINVAL for bad options. */
int qx_create(qx_handle* h, int device, void* cuda_stream, const qx_options* opt);
void qx_destroy(qx_handle h);
const char* qx_last_error(qx_handle h);
int qx_set_options(qx_handle h, const qx_options* opt);

/* Build the network of a circuit (Sec. II).  gates: n_gates records, host
 * memory, copied.  open_mask: n_qubits bytes, 1 = leave that qubit's output
 * leg open (may be NULL = all closed).  Drops any previous plan.
 * QX_EINVAL on qubit indices out of range or nq not in {1, 2}. */
int qx_build_network(qx_handle h, int32_t n_qubits, const qx_gate* gates, int64_t n_gates,
                     const uint8_t* open_mask);

/* Number of tensors and bonds of the built network (for plan makers). */
int qx_network_info(qx_handle h, int64_t* n_tensors, int64_t* n_bonds);

/* Set the contraction plan (Sec. III-A): order = n_steps x 2 SSA ids (host,
 * copied), sliced = n_sliced bond ids (host, copied; each must join two
 * tensors and must not be the final wire of a qubit).  *peak_entries_out
 * (may be NULL) receives the largest intermediate of one slice in complex
 * entries.  QX_EINVAL on a malformed plan. */
int qx_set_plan(qx_handle h, const int64_t* order, int64_t n_steps, const int64_t* sliced,
                int32_t n_sliced, int64_t* peak_entries_out);

/* Device bytes a workspace needs to contract up to max_bits bitstrings per
 * call with batches of `items` (slice, bitstring) pairs (items <= 0: one
 * pair).  Requires a plan. */
int qx_workspace_size(qx_handle h, int64_t max_bits, int64_t items, int64_t* bytes_out);

/* Bind device memory (256-byte aligned) of `bytes` bytes as the workspace for
 * calls of up to max_bits bitstrings; batches are sized to fill it.  The
 * caller keeps ownership and must keep it alive until the next bind or
 * qx_destroy.  dptr = NULL asks the library to cudaMalloc `bytes` itself
 * (freed on the next bind or by qx_destroy).  Requires a plan; setting a new
 * plan unbinds.  QX_ENOMEM if not even one pair fits. */
int qx_bind_workspace(qx_handle h, void* dptr, int64_t bytes, int64_t max_bits);

/* A workspace in two parts, so that handles whose calls never overlap on the
 * GPU (enqueued one after another on one stream) can share the larger one
 * (the paper has no counterpart; a batch of uneven circuits contracted in
 * turn needs the batch regions of only one circuit at a time).
 *   fixed part  what a handle keeps between calls: its network's tensors,
 *               bitstrings, FP64 accumulators, invariant intermediates and
 *               programs (its own buffer);
 *   batch part  the per-slice and per-pair intermediates of one batch of
 *               (slice, bitstring) pairs, which a call overwrites from the
 *               start: it may be shared by handles whose calls run in stream
 *               order, never by calls that overlap.
 * qx_workspace_parts gives both sizes for calls of up to max_bits
 * bitstrings in batches of `items` pairs (items <= 0: one pair);
 * qx_bind_workspace_parts binds caller-owned device buffers (256-byte
 * aligned, kept alive by the caller until the next bind or qx_destroy;
 * batches are sized to fill the batch part).  Batched executor only
 * (QX_EINVAL otherwise); QX_ENOMEM when the fixed part is too small or the
 * batch part holds no pair.  Requires a plan; setting a new plan unbinds. */
int qx_workspace_parts(qx_handle h, int64_t max_bits, int64_t items, int64_t* fixed_bytes, int64_t* batch_bytes);
int qx_bind_workspace_parts(qx_handle h, void* d_fixed, int64_t fixed_bytes, void* d_batch, int64_t batch_bytes,
                            int64_t max_bits);

/* Contract for n_bits bitstrings (host, n_bits x n_qubits bytes of 0/1; bytes
 * at open qubits are ignored) and write amplitudes to amps_out (host,
 * caller-owned, n_bits x 2^n_open x {re, im} doubles).  Copies the
 * bitstrings to the device, runs every slice, copies the result back and
 * synchronises the stream.  QX_EINVAL on a non-0/1 byte, QX_ENOMEM when
 * n_bits exceeds what the workspace was sized for. */
int qx_contract(qx_handle h, const uint8_t* bitstrings, int64_t n_bits, double* amps_out);

/* As qx_contract, but both buffers are device memory and the call only
 * enqueues work on the stream (no synchronisation, no host copies).
 * Bitstring bytes are not validated on this path. */
int qx_contract_device(qx_handle h, const uint8_t* d_bitstrings, int64_t n_bits, double* d_amps_out);

/* Partial sums for multi-process slice sharding (Sec. IV-A: slices are
 * balanced over processes and recombined): as qx_contract /
 * qx_contract_device, but only slices s in [s_begin, s_end) are contracted
 * and summed (FP64, compensated).  QX_EINVAL for an empty or out-of-range
 * slice range. */
int qx_contract_slices(qx_handle h, const uint8_t* bitstrings, int64_t n_bits, int64_t s_begin, int64_t s_end,
                       double* amps_out);
int qx_contract_slices_device(qx_handle h, const uint8_t* d_bitstrings, int64_t n_bits, int64_t s_begin,
                              int64_t s_end, double* d_amps_out);

/* Asynchronous requests for serving (the paper states the problem as a batch
 * call; the request loop of the serving workload needs to overlap requests).
 * qx_submit enqueues what qx_contract_slices_device does (device bitstrings
 * d_bitstrings [n_bits][n_qubits], slices [s_begin, s_end), FP64 partial sums
 * into d_amps_out [n_bits][2^n_open][2]) on the handle's stream, then, when
 * h_amps_out is not NULL, a device-to-host copy of those amplitudes into it
 * (pinned host memory for the copy to be asynchronous), and records a
 * completion event; it returns at once with *req_out, a request number that
 * increases per handle.  The buffers must stay valid until the request is
 * done.  qx_poll sets *done = 1 once everything of request req has finished
 * (then the number is forgotten) and 0 while it runs; unknown numbers give
 * QX_EINVAL.  A device-side timeout shows in qx_device_status. */
int qx_submit(qx_handle h, const uint8_t* d_bitstrings, int64_t n_bits, int64_t s_begin, int64_t s_end,
              double* d_amps_out, double* h_amps_out, int64_t* req_out);
int qx_poll(qx_handle h, int64_t req, int32_t* done);

/* One sum over all slices (Eq. 2) submitted in parts, so that a server can
 * interleave other work between the parts of a long request: as qx_submit,
 * but the FP64 compensated accumulators of the handle carry the running sum
 * from one part to the next, so the parts add exactly as one call over their
 * slices would (the same per-slice results, summed in the same slice order).
 *   first != 0  starts a new sum (clears the accumulators); first == 0
 *               continues the handle's open sum: d_bitstrings and n_bits must
 *               be those of its first part and s_begin the s_end of its last
 *               part, else QX_ESTATE;
 *   last != 0   ends the sum: the amplitudes are written to d_amps_out (and
 *               copied to h_amps_out when it is not NULL); parts with
 *               last == 0 write nothing to either buffer.
 * The completion event of every part is polled with qx_poll.  Any other
 * contraction on the handle ends an open sum (its parts must be submitted
 * again from first != 0).  The batched executor only (executor 0 or 1; else
 * QX_EINVAL). */
int qx_submit_part(qx_handle h, const uint8_t* d_bitstrings, int64_t n_bits, int64_t s_begin, int64_t s_end,
                   int32_t first, int32_t last, double* d_amps_out, double* h_amps_out, int64_t* req_out);

/* Graph replay (on by default): a call of qx_contract / qx_contract_device /
 * qx_contract_slices[_device] that repeats the previous call's device
 * buffers, bitstring count and slice range is captured once as a CUDA graph
 * and replayed afterwards (the contents of the buffers may change; the
 * pointers and sizes may not).  Not used on the legacy default stream or
 * while profiling.  enable = 0 turns it off and drops the captured graph. */
int qx_set_graphs(qx_handle h, int enable);

/* Memoised invariant intermediates (the checkpoint reuse the paper's outlook
 * proposes, after Pan et al. 2021: parts of the contraction that no sliced
 * bond and no output bit touch are the same for every slice and every
 * bitstring, so they can be kept between samples).  enable = 1: the first
 * contraction after this call (or after a new plan or workspace) computes
 * them into the bound workspace as usual, later calls of the batched
 * executor skip those steps and read the kept tensors.  Same amplitudes
 * (the kept tensors are the ones the skipped steps would write again).
 * enable = 0 (default): every call computes them.  qx_contract_device_static
 * always computes them.  A device timeout reported by qx_device_status
 * drops the kept tensors.  Drops a captured graph.  QX_EINVAL unless enable
 * is 0 or 1. */
int qx_set_memo(qx_handle h, int enable);

/* Concurrent issue of independent contraction steps (the paper has no
 * counterpart; Sec. IV-A's levels of parallelism stop at one contraction per
 * GPU kernel).  The plan compiler records, for every kernel launch, the
 * earlier launches it must follow: those writing what it reads, reading or
 * writing what it writes (storages of dead tensors are reused).  The batched
 * executor then issues launches over n_streams streams: the handle's own
 * stream plus n_streams - 1 streams the handle creates on its device, with
 * event waits for the dependencies, and joins them back into the handle's
 * stream before the slice sum of every batch, so the call stays ordered on
 * the handle's stream as before.  Results are bit-identical for every
 * n_streams (each launch computes the same values; only the overlap of
 * independent launches changes).  n_streams = 1 issues everything on the
 * handle's stream in plan order.  Default 8; range 1 .. 32 (QX_EINVAL
 * otherwise).  Profiling runs everything on the handle's stream.  Drops a
 * captured graph. */
int qx_set_streams(qx_handle h, int32_t n_streams);

/* A text listing of the compiled plan, one line per kernel launch of a
 * contraction (kind, whether it runs per pair or once, M/K/N bits, operand
 * layouts).  Writes at most len bytes (NUL-terminated) to buf; *needed (may be
 * NULL) receives the full size.  Works on host-only handles. */
int qx_describe_plan(qx_handle h, char* buf, int64_t len, int64_t* needed);

/* Statistics of the last contraction (host values, any pointer may be NULL):
 * algorithmic complex flops (8 M K N per step, per pair), kernel launches,
 * batches. */
int qx_last_stats(qx_handle h, double* flops, int64_t* launches, int64_t* batches);

/* Synchronise the handle's stream and report a device-side failure of the
 * work enqueued since the last contraction started: QX_OK, or QX_ETIMEOUT if
 * a bounded wait inside a kernel expired (the kernel then returned early and
 * the amplitudes are invalid).  qx_contract checks this itself. */
int qx_device_status(qx_handle h);

/* qx_contract_device without allocation (the paper has no counterpart; this
 * serves host programs, not the method).  Some callers cannot allocate device
 * memory for the library: programs whose own pool allocator owns the whole
 * GPU, and code that must not call cudaMalloc / cudaFree because those calls
 * can synchronise the device.  This entry point needs no bound workspace:
 * its scratch is a fixed array of QX_STATIC_SCRATCH_BYTES compiled into the
 * library (every GPU that loads libqx holds it until the process exits), and
 * it calls no cudaMalloc, cudaFree or allocating library routine.  The caller
 * passes device bitstrings (n_bits x n_qubits bytes, not validated) and the
 * device output (n_bits x 2^n_open x {re, im} doubles); work is enqueued on
 * the handle's stream, as for qx_contract_device, and gives the same
 * amplitudes.
 *   - Each call first copies the network's tensors and the compiled programs
 *     from host memory into the array and synchronises the handle's stream
 *     (the array may hold another plan's data), so the call returns only once
 *     earlier work on that stream is done; the contraction itself is then
 *     enqueued.
 *   - A bounded device wait that expires is reported by the next
 *     qx_device_status on this handle (QX_ETIMEOUT), as for
 *     qx_contract_device.
 *   - The first call on each device also looks up the array's device address
 *     (once per device); make that first call before any stream capture.
 *   - QX_ENOMEM when the network's tensors, n_bits bitstrings, their
 *     accumulators and one (slice, bitstring) pair's intermediates do not fit
 *     in QX_STATIC_SCRATCH_BYTES; use qx_bind_workspace + qx_contract_device
 *     for such plans.
 *   - All calls on a device share the one array, which keeps the last call's
 *     contents (each call clears its own accumulators).  Calls whose work
 *     overlaps on the GPU -- other streams, handles or host threads -- race on
 *     it and give wrong results; serialise them. */
#define QX_STATIC_SCRATCH_BYTES (64ll << 20)
int qx_contract_device_static(qx_handle h, const uint8_t* d_bitstrings, int64_t n_bits, double* d_amps_out);

/* Empirical-supremum rejection sampling of output bitstrings (Sec. III-B;
 * the method of Caffo, Booth and Davison, 2002).  Target law p(x) =
 * |<x|C|0>|^2 over the N = 2^n_qubits bitstrings, uniform proposal, density
 * ratio w(x) = p(x) N.  Iteration i takes candidate X_i and uniform U_i
 * (both drawn by the caller, so the run is reproducible), accepts X_i when
 * U_i * M < w(X_i) (FP64, the test U < w / M without a division, p = re*re
 * + im*im rounded term by term, M the bound BEFORE this iteration), then
 * sets M = max(M, w(X_i)); a NaN w is never accepted and never raises M.
 * Iterations i < n_warmup only move M.  The run stops right after its
 * max_out-th acceptance (later candidates are not consumed and do not touch
 * M) or when the candidates run out.  A fresh run starts with *m_inout = 1;
 * to continue a run, pass back the returned bound, the candidates from
 * *n_consumed on, and the warm-up still left.  Results are exactly those of
 * the one-at-a-time algorithm (the batch is scanned on the GPU: a prefix
 * maximum and a stream compaction).
 *
 * qx_esup_accept takes the candidates' amplitudes:
 *   d_amps      device, n_cand x {re, im} doubles (amplitude of candidate i)
 *   d_uniforms  device, n_cand doubles
 *   n_qubits    N = 2^n_qubits, 1 .. 62
 *   d_accepted  device, room for min(max_out, n_cand) int64: the accepted
 *               iterations' indices in [0, n_cand), increasing
 *   m_inout, n_accepted, n_consumed: host values
 * It runs on the handle's stream and synchronises it (the counts come back
 * to the host).  Needs no network, plan or workspace.
 *
 * qx_esup_sample first contracts the candidates with the handle's network,
 * plan and bound workspace (every qubit closed, else QX_EINVAL), in pieces
 * of at most the workspace's bitstring count, then runs the tests of each
 * piece, stopping early once max_out are accepted:
 *   d_candidates  device, n_cand x n_qubits bytes of 0/1 (not validated)
 *   d_amps        device, n_cand x {re, im} doubles, receives the
 *                 amplitudes of the pieces contracted (all of
 *                 [0, *n_consumed) at least)
 * Other arguments as above.  QX_ESTATE without a network, plan or
 * workspace; QX_ETIMEOUT if a bounded device wait expired.
 *
 * Both: n_cand == 0 or max_out == 0 consumes nothing (M unchanged);
 * negative counts and NULL pointers give QX_EINVAL. */
int qx_esup_accept(qx_handle h, const double* d_amps, const double* d_uniforms, int64_t n_cand, int32_t n_qubits,
                   int64_t n_warmup, int64_t max_out, double* m_inout, int64_t* d_accepted, int64_t* n_accepted,
                   int64_t* n_consumed);
int qx_esup_sample(qx_handle h, const uint8_t* d_candidates, const double* d_uniforms, int64_t n_cand,
                   int64_t n_warmup, int64_t max_out, double* m_inout, double* d_amps, int64_t* d_accepted,
                   int64_t* n_accepted, int64_t* n_consumed);

/* Groups: the pairs of many networks in one persistent launch (uneven
 * circuits and slice counts side by side; Sec. IV-A's slice and bitstring
 * levels of parallelism across several circuits).  Every member handle must be
 * created with executor = 3, have a plan without tensor-core steps and a
 * bound workspace on the same device; the group uses member 0's stream.
 *   qx_group_create  takes, per member, device bitstrings (n_bits[i] x
 *                    n_qubits bytes) and a device output (n_bits[i] x 2^open x
 *                    {re, im} doubles) that stay fixed for the group's life;
 *                    ctas_per_sm (0 = 2) sets the persistent grid.  On error
 *                    *g may still be returned for qx_group_last_error.
 *   qx_group_bind    takes caller-owned device scratch of at least
 *                    qx_group_scratch_size bytes, uploads the members' tensors
 *                    and programs and synchronises the stream.
 *   qx_group_run     only enqueues: one launch for all members' invariant
 *                    tensors, one persistent launch for all (slice, bitstring)
 *                    pairs (largest programs first), one FP64 compensated sum
 *                    into the outputs.  No allocation, no host copies, no
 *                    synchronisation, so a CUDA graph can capture it.
 * A group does not own its members; destroy it before them. */
typedef struct qx_group* qx_group_t;
int qx_group_create(qx_group_t* g, qx_handle* hs, int32_t n, const uint8_t* const* d_bitstrings,
                    const int64_t* n_bits, double* const* d_amps_out, int32_t ctas_per_sm);
int qx_group_scratch_size(qx_group_t g, int64_t* bytes_out);
int qx_group_bind(qx_group_t g, void* d_scratch, int64_t bytes);
int qx_group_run(qx_group_t g);
const char* qx_group_last_error(qx_group_t g);
void qx_group_destroy(qx_group_t g);

/* Kernel timing for roofline reports.  With profiling on, every kernel launch
 * of a contraction is bracketed by CUDA events on the handle's stream;
 * qx_profile_read synchronises the stream and returns, for one kernel kind,
 * the summed event time (ms), launches, algorithmic complex flops (8 M K N
 * per pair) and algorithmic bytes (operands read once, result written once)
 * since profiling was last switched.  qx_set_profiling resets the totals. */
#define QX_KERNEL_PERMUTE 0
#define QX_KERNEL_SMALL   1  /* gathers, small operand staged in shared memory (k_small) */
#define QX_KERNEL_GEMM    2
#define QX_KERNEL_SUM     3
#define QX_KERNEL_TC_PREP 4  /* operand split / expansion for the tensor-core forms */
#define QX_KERNEL_TC_GEMM 5  /* tcgen05 complex GEMM on pre-split operands (k_gemm_tc) */
#define QX_KERNEL_PERSIST 6  /* persistent executor (whole contractions) */
#define QX_KERNEL_WAVE    7  /* batched executor: the small invariant steps, one CTA per chain */
#define QX_KERNEL_SMALL_FLAT 8  /* gathers of short per-pair rows, one thread per row (k_small_flat) */
#define QX_KERNEL_TC_DIRECT 9  /* tcgen05 3xTF32 GEMM splitting raw complex64 slabs itself (k_gemm_tc2) */
#define QX_KERNEL_TC_DIRECT_KB 10  /* the same with B' built once per CTA and kept (k_gemm_tc2kb): B
                                    * shared by every item and one tile wide */
#define QX_KERNEL_KINDS   11
int qx_set_profiling(qx_handle h, int enable);
int qx_profile_read(qx_handle h, int kind, double* ms, int64_t* launches, double* flops, double* bytes);

#ifdef __cplusplus
}
#endif
#endif /* QX_H */
