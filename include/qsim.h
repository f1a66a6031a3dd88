/*
 * qsim.h -- C ABI of libqsim, a single-GPU (GB300, sm_103a) state-vector simulator.
 *
 * The simulated object is the state vector of the paper (arXiv 2511.14664, Sec. 2.1 "State-Vector
 * Simulation"): 2^n complex amplitudes, one per computational basis state, on which each gate acts as
 * a tensor-product operator. Its hot path -- applying gates to all 2^n amplitudes -- runs in the
 * library's own CUDA kernels; PyTorch (or any other caller) only provides device memory and a stream.
 *
 * Conventions used by every entry point:
 *   - qubit q is bit q of the amplitude index (little-endian);
 *   - for a gate on targets (t_0, ..., t_{k-1}) the matrix row/column index is m = sum_j bit_{t_j} 2^j;
 *   - gate matrices are 2^k x 2^k complex128, row-major, interleaved (re, im), in HOST memory; the
 *     library copies them before the call returns, so the caller may free them at once;
 *   - controls fire on |1>;
 *   - amplitudes are stored interleaved (re, im): complex64 = 2 x float32 (8 B), complex128 =
 *     2 x float64 (16 B), amplitude x at byte offset x * sizeof(amplitude).
 *
 * Return codes: QSIM_OK (0) on success, otherwise one of the QSIM_E* codes below; a thread-local
 * message describing the failure is available from qsim_last_error(). No C++ exception crosses the ABI.
 * Argument errors (QSIM_EINVAL) are detected before any work is enqueued, so the state is unchanged.
 * After QSIM_ECUDA or QSIM_ETIMEOUT the state contents are undefined.
 *
 * Threading and streams: a handle is bound to one CUDA stream and is not thread-safe. Gate and run
 * calls are asynchronous on that stream. Calls that write host outputs (norm, probabilities,
 * expectations, samples, get_state to host) synchronise the stream before returning.
 */
#ifndef QSIM_H
#define QSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QSIM_ABI_VERSION 2

/* Status codes. */
#define QSIM_OK 0
#define QSIM_EINVAL 1       /* bad qubit index, duplicate qubit, control that is also a target, NULL, size */
#define QSIM_ENOMEM 2       /* device or host allocation failed, or the caller's buffer is too small */
#define QSIM_ECUDA 3        /* a CUDA runtime call or kernel launch failed */
#define QSIM_ETIMEOUT 4     /* a bounded device-side wait expired; the kernel stopped and reported it */
#define QSIM_EUNSUPPORTED 5 /* valid request that the library does not implement (e.g. k too large) */

/* Amplitude types. */
#define QSIM_C64 0  /* complex64: float32 real and imaginary parts */
#define QSIM_C128 1 /* complex128: float64 real and imaginary parts */

/* Arithmetic used for fused dense blocks (Sec. 2.1: fusion trades flops for arithmetic intensity). */
#define QSIM_PREC_SIMT 0   /* CUDA-core FMA in the state's own precision */
#define QSIM_PREC_TF32X3 1 /* tensor cores: 3 TF32 products (hi*hi + hi*lo + lo*hi), FP32 accumulation */
#define QSIM_PREC_BF16X3 2 /* tensor cores: 2-way BF16 split, 3 products, FP32 accumulation. REDUCED
                              accuracy (~16 significant bits per product, not complex64 level): ~1e-8
                              infidelity per block on a random state, 7.9e-10 after the 64 blocks of the
                              20-qubit depth-40 brickwork; never reported as a complex64-accuracy result */
#define QSIM_PREC_BF16X6 3 /* tensor cores: 3-way BF16 split, 6 products, FP32 accumulation */
/* tensor cores: FP16 split products with fixed scales -- amplitudes x 2^15 (the state must be normalised,
   |amplitude| <= 1), matrix entries x 2^14, each split into two FP16 parts (22 significant bits, as 3xTF32),
   three products, FP32 accumulation. Half the tensor cycles and A-operand traffic of 3xTF32. In plans,
   blocks whose 3xTF32 form has the line-group or pair-rows data path (low qubits among the targets) run as
   QSIM_PREC_TF32X3; see also qsim_run_opts.pair_blocks. The one precision with 7-qubit tensor-core blocks
   (qsim_apply_fused with k = 7, plans with max_fused = 7). */
#define QSIM_PREC_FP16X3 4

/* Run modes. */
#define QSIM_RUN_PLAIN 0 /* one device pass per gate (diagonal gates touch only their non-unit entries) */
#define QSIM_RUN_FUSED 1 /* gates merged into dense or diagonal blocks of at most max_fused qubits */

#define QSIM_MAX_TARGETS 8
#define QSIM_MAX_CONTROLS 8
#define QSIM_MAX_QUBITS 36

typedef struct qsim_state* qsim_h;
typedef struct qsim_plan* qsim_plan_h;

/* One gate: U (2^k x 2^k, FP64 complex, host) on `targets`, applied where all `controls` are 1. */
typedef struct {
    int32_t k;                            /* number of targets, 1..QSIM_MAX_TARGETS */
    int32_t nc;                           /* number of controls, 0..QSIM_MAX_CONTROLS */
    int32_t targets[QSIM_MAX_TARGETS];    /* target j <-> bit j of the matrix index */
    int32_t controls[QSIM_MAX_CONTROLS];
    const double* matrix;                 /* interleaved complex128, row-major, host */
} qsim_gate;

/* A circuit: gates applied in array order. */
typedef struct {
    int32_t n;                /* number of qubits */
    int32_t num_gates;
    const qsim_gate* gates;   /* host array of num_gates gates */
} qsim_circuit;

/* Options for planning a circuit. Zero-initialise, then set fields. */
typedef struct {
    int32_t mode;       /* QSIM_RUN_PLAIN or QSIM_RUN_FUSED */
    int32_t max_fused;  /* fusion width k for QSIM_RUN_FUSED: 1..6 (0 = 5); 7 with QSIM_PREC_FP16X3 on a
                           complex64 state (7-qubit tensor-core blocks; plans of < 14 qubits or with global
                           qubits keep 6); dry runs also 7, 8 at any precision (pass counts) */
    int32_t precision;  /* QSIM_PREC_* for dense blocks of >= tc_min_k qubits (complex64 states only) */
    int32_t tc_min_k;   /* smallest dense block sent to the tensor-core kernel (0 = 5) */
    int32_t use_graph;  /* 1: replay the plan's launches from a CUDA graph captured on first execution */
    /* > 0: treat qubits >= local_qubits as "global" index bits, as a state split over 2^(n - local_qubits)
       devices would (Sec. 2.1: gates on the n - log2(m) local qubits need no exchange). Before a pass that
       touches a global qubit, a reorder pass swaps it with an idle local qubit (least recently used) and
       the plan tracks the logical -> physical qubit map; the identity order is restored at the end.
       0 = off (every qubit is addressed in place). */
    int32_t local_qubits;
    /* 1 (qsim_plan_create only): plan on the host and stop before any device work (no device needed):
       the plan lists its passes (qsim_plan_num_passes, qsim_plan_pass_info, qsim_plan_info) but cannot be
       executed (QSIM_EINVAL). */
    int32_t dry_run;
    /* Batches only (qsim_batch_plan_create): with a tensor-core precision, circuits of at least this many
       qubits run as fused tensor-core plans (6-qubit blocks, or up to 7 with QSIM_PREC_FP16X3; every pass on
       the whole GPU) inside the same
       enqueue, instead of on one cluster of the persistent launch (0 = 20; at least 13). Ignored for
       QSIM_PREC_SIMT. */
    int32_t batch_tc_min_n;
    /* Planning effort: 0 = greedy fusion (the largest candidate block at each step); 1 = also fuse with
       one block of look-ahead and keep the grouping with fewer blocks (planning about 4x slower; e.g. the
       33-qubit triangular-lattice TFIM goes from 63 to 58 passes); 2 / 3 = also a beam search over
       groupings (beam 8 / 32: the partial groupings that placed the most gates), fewest blocks kept
       (30-qubit brickwork 64 -> 62 passes, 33-qubit paper random circuit 45 -> 44 / 42; planning 5-20x
       slower than greedy). */
    int32_t plan_effort;
    /* QSIM_PREC_FP16X3 plans only: 1 = also run consecutive 6-qubit blocks whose targets together span at most
       12 qubits as ONE pass (both products per tile while it is on chip). Correct, but measured slower than
       two single passes on GB300 (the pass is bound by instruction issue, not memory); for study. */
    int32_t pair_blocks;
    /* Plans of states of at most 16 qubits whose passes are all CUDA-core dense blocks (k <= 5), diagonals
       (k <= 6) or phase passes run every pass inside ONE cooperative launch, one CTA per SM resident over the plan and a grid
       barrier between passes (Sec. 2.1: the passes applied in order; at these sizes a pass is a few
       microseconds of arithmetic, less than a launch costs). Only a whole-plan execution does; a pass range
       launches per pass. 1 = always one launch per pass (and the CUDA graph of use_graph). */
    int32_t launch_per_pass;
} qsim_run_opts;

/* What a plan does per execution (filled by qsim_plan_create). */
typedef struct {
    int64_t input_gates;     /* unfused gates in the circuit */
    int64_t passes;          /* device passes over the state (kernel launches on the state) */
    int64_t dense_blocks;    /* passes applying a dense matrix on CUDA cores */
    int64_t tc_blocks;       /* passes applying a dense matrix on tensor cores */
    int64_t diag_blocks;     /* passes applying a diagonal */
    int64_t reorders;        /* qubit-reorder passes */
    double algorithmic_bytes;/* HBM bytes the passes must move at minimum (read + write) */
    double host_plan_ms;     /* host time spent planning */
    int64_t resident;        /* 1: a whole-plan execution is one cooperative launch (launch_per_pass) */
} qsim_plan_info;

/* ---- version and errors ------------------------------------------------------------------------------ */

/* Version of this ABI (library service, no passage). */
int qsim_abi_version(void);

/* Message of the last failed call on this thread ("" if none). Valid until the next call. Library service, no
   passage. */
const char* qsim_last_error(void);

/* Bytes of a 2^n state of `dtype` (8 or 16 bytes per amplitude; Sec. 1: 2^(n-27) GiB at FP32). */
int qsim_state_bytes(int n, int dtype, size_t* out);

/* ---- state lifetime ---------------------------------------------------------------------------------- */

/*
 * Create a handle for an n-qubit state (1 <= n <= QSIM_MAX_QUBITS) of `dtype` (Sec. 2.1 "State-Vector
 * Simulation": the 2^n-amplitude vector the simulation stores; Sec. 1: its memory doubles per qubit).
 * dev_buf: device buffer of at least qsim_state_bytes(n, dtype) bytes, 256-byte aligned, owned by the
 *          caller, who keeps it alive until qsim_destroy; or NULL, in which case the library allocates
 *          (and later frees) the state with cudaMalloc.
 * stream:  the cudaStream_t every call on this handle is enqueued on (NULL = legacy default stream).
 * The state is NOT initialised; call qsim_set_basis or qsim_set_state. The library also allocates a
 * small device workspace for reductions (about 2^(n-9) bytes + 4 MiB).
 */
int qsim_create(int n, int dtype, void* dev_buf, size_t buf_bytes, void* stream, qsim_h* out);
/* Release the handle (after its stream completes) and the state if the library allocated it. Library
   service, no passage. NULL is accepted. */
int qsim_destroy(qsim_h h);
/* Bind later calls to another cudaStream_t. Library service, no passage. */
int qsim_set_stream(qsim_h h, void* stream);
/* The handle's n (Sec. 2.1: the number of qubits fixes the vector length 2^n). */
int qsim_num_qubits(qsim_h h, int* n);
/* Device address of amplitude 0 (layout above). Library service, no passage. */
int qsim_device_ptr(qsim_h h, void** out);

/* |x>: amplitude x = 1, all others 0 (Sec. 2.1: a basis state). x < 2^n. */
int qsim_set_basis(qsim_h h, uint64_t x);
/* Copy a whole state in (src) or out (dst); *_on_device = 1 for device pointers, 0 for host (Sec. 2.1
   "State-Vector Simulation": the full amplitude vector; also a checkpoint of a run). Copies to the host
   synchronise and report a set device error word. */
int qsim_set_state(qsim_h h, const void* src, int src_on_device);
int qsim_get_state(qsim_h h, void* dst, int dst_on_device);
/* Wait for all work enqueued on h's stream and report any device-side error (QSIM_ETIMEOUT when a
   bounded wait expired, QSIM_ECUDA for a CUDA error). Library service, no passage. */
int qsim_synchronize(qsim_h h);
/* Failure injection for tests of a caller's recovery path (a library service; the paper has no counterpart).
   After the work already enqueued on h's stream completes, `code` (nonzero; bit 0 = "a bounded device-side
   wait expired") is written into h's device error word from the host, exactly as a kernel whose bounded wait
   ran out would leave it. No kernel runs and nothing waits on the GPU. The next call that checks the word
   (qsim_synchronize, a readout, qsim_get_state to host) returns QSIM_ETIMEOUT and clears it; the handle stays
   usable. Synchronises. */
int qsim_inject_device_error(qsim_h h, unsigned code);

/* ---- gate application (the hot path; Sec. 2.1, cost O(g 2^n)) --------------------------------------- */

/*
 * Apply U on `targets` (k of them, 1 <= k <= QSIM_MAX_TARGETS = 8) controlled on `controls` (nc of them,
 * may be NULL when nc = 0). All qubits distinct and < n. Asynchronous.
 * Diagonal matrices (every off-diagonal entry exactly 0, k <= 6) touch only the amplitudes whose factor is
 * not exactly 1; single-qubit gates use vectorised streaming or warp-shuffle butterflies; k <= 4 gathers
 * 2^k amplitudes per thread (spread over several lanes for small states); k = 5, 6 use a shared-memory
 * tile kernel and k = 7, 8 a kernel that streams U from L2 in column chunks, both in the state's precision.
 */
int qsim_apply_gate(qsim_h h, const int* targets, int k, const int* controls, int nc, const double* matrix);

/*
 * Apply a dense 2^k x 2^k block (1 <= k <= 8) on `targets` with the given QSIM_PREC_* arithmetic.
 * Tensor-core precisions (TF32X3, BF16X3, BF16X6, FP16X3) need a complex64 state of n >= k + 7 qubits and
 * k in 5..6, or k = 7 with FP16X3 (QSIM_EUNSUPPORTED otherwise);
 * QSIM_PREC_SIMT works for both types and every k.
 * This is the single-block form of what QSIM_RUN_FUSED plans produce.
 */
int qsim_apply_fused(qsim_h h, const int* targets, int k, const double* matrix, int precision);

/*
 * Qubit reorder (the on-device analogue of the paper's global/local index-bit exchange, Sec. 2.1 and
 * Sec. 2.5): exchange qubit a[i] with qubit b[i] for i < p, i.e. amplitude x moves to the index with
 * bits a[i] and b[i] swapped. All 2p qubits distinct, p <= 8. In place, one pass over the state.
 */
int qsim_swap_qubits(qsim_h h, const int* a, const int* b, int p);

/* ---- circuits and plans ---------------------------------------------------------------------------- */

/*
 * Plan a circuit (Sec. 2.1: gate fusion merges gates into larger matrices; Sec. 2.2: the fusion level is
 * tuned per architecture and precision) for states of c->n qubits and `dtype`: fusion into blocks (QSIM_RUN_FUSED), choice of
 * kernel per block, and FP64 composition of each fused block on the device (enqueued on `stream`).
 * The plan owns its device buffers; it can be executed on any handle with matching n and dtype.
 * info may be NULL.
 */
int qsim_plan_create(const qsim_circuit* c, int dtype, const qsim_run_opts* opts, void* stream,
                     qsim_plan_h* out, qsim_plan_info* info);
/* Enqueue every pass of the plan on h's stream (Sec. 2.1: the gates applied to the state in order).
   Asynchronous. */
int qsim_plan_execute(qsim_h h, qsim_plan_h plan);
/* qsim_set_basis(h, x) then passes [0, count) of the plan (count < 0: all of them), on h's stream (no
   graph). When the plan starts with a tensor-core block (3xTF32 or BF16x3) that block generates |x> as its
   input instead of reading the state, and writes every amplitude, so neither the set-up pass nor the
   block's reads happen. QSIM_EINVAL for x >= 2^n or count > the number of passes. */
int qsim_plan_execute_from_basis(qsim_h h, qsim_plan_h plan, uint64_t x, int64_t count);
/* Release a plan and its device buffers. Library service, no passage. NULL is accepted. */
int qsim_plan_destroy(qsim_plan_h plan);

/*
 * Library service (no passage). Plans group gates into blocks by the circuit's structure alone (each gate's
 * qubits, whether it is diagonal, the planning options), so groupings are cached process-wide by structure
 * (at most 1024, thread-safe): circuits that repeat a structure -- a batch of chains of one width and depth,
 * one circuit planned again with new angles -- are grouped once. Matrices are composed anew every time.
 * This empties the cache (for timing cold planning, or to release its host memory).
 */
int qsim_plan_cache_clear(void);

/* One pass of a plan, for per-kernel timing and roofline accounting. */
#define QSIM_PASS_DENSE_SMALL 0 /* dense k <= 4 on CUDA cores (register gather or warp-shuffle butterfly) */
#define QSIM_PASS_DIAG 1        /* diagonal factors, non-unit entries only */
#define QSIM_PASS_DENSE_TILE 2  /* dense k = 5, 6 on CUDA cores through shared memory */
#define QSIM_PASS_TC 3          /* dense block on tensor cores (complex64) */
#define QSIM_PASS_REORDER 4     /* qubit reorder (exchange of index-bit pairs) */
#define QSIM_PASS_PHASE 5       /* any number of 1- and 2-qubit diagonal gates on any qubits, one phase per
                                   amplitude (a quadratic form of its index bits) */
#define QSIM_PASS_TC_PAIR 6     /* two 6-qubit tensor-core blocks in one pass (QSIM_PREC_FP16X3): targets[] holds
                                   the first block's targets, controls[] (nc = 6) the second's */
typedef struct {
    int32_t kind;             /* QSIM_PASS_* */
    int32_t k;                /* qubits the pass's matrix acts on (a reorder pass: exchanged pairs) */
    int32_t nc;               /* control qubits (not part of the matrix; a reorder pass: = k) */
    int32_t precision;        /* QSIM_PREC_* used by the pass */
    int64_t gates;            /* input gates merged into this pass */
    double algorithmic_bytes; /* HBM bytes the pass must read + write */
    int32_t targets[QSIM_MAX_TARGETS];   /* index bits the matrix acts on, in the order of its index bits
                                            (k of them; k = 0 for a phase pass; a reorder pass exchanges
                                            index bit targets[i] with controls[i], i < k) */
    int32_t controls[QSIM_MAX_CONTROLS]; /* control bits (nc of them) */
    int32_t launches;         /* kernel launches one execution of the pass makes (2 for a tensor-core block
                                 with a phase epilogue: a small kernel computes its per-tile factors first) */
    int32_t reserved;
} qsim_pass_info;
/* Number of passes and the description of pass i (Sec. 2.1: after fusion, each pass is one application of a
   fused matrix to the whole vector). Host only; also for dry-run plans. */
int qsim_plan_num_passes(qsim_plan_h plan, int64_t* out);
int qsim_plan_pass_info(qsim_plan_h plan, int64_t i, qsim_pass_info* out);
/* Enqueue passes [first, first + count) of the plan on h's stream (no graph; Sec. 2.1, gates in order). */
int qsim_plan_execute_range(qsim_h h, qsim_plan_h plan, int64_t first, int64_t count);
/* Plan, execute and destroy in one call (Sec. 2.1: fusion, then the fused gates applied in order; the plan's
   device buffers are released after the stream completes the run). */
int qsim_run(qsim_h h, const qsim_circuit* c, const qsim_run_opts* opts, qsim_plan_info* info);

/* ---- readout (Sec. 2.1 "Measurement and Sampling"; Sec. 2.5 expectation values) --------------------- */

/* sum_x |a_x|^2, accumulated with compensated (float-float, then FP64 TwoSum) sums. Synchronises. */
int qsim_norm(qsim_h h, double* out);

/*
 * Marginal probabilities over `qubits` (1 <= nq <= min(30, n), distinct): out[m] = sum of |a_x|^2 over the
 * x whose bit qubits[j] equals bit j of m. out has 2^nq doubles (host, caller-owned). Compensated sums
 * (float-float per segment, FP64 across segments). For nq > 12 the bins are formed in a temporary device
 * buffer of 8 * 2^nq bytes from the stream-ordered allocator, released before return (QSIM_ECUDA if it
 * cannot be had). Synchronises.
 */
int qsim_probs(qsim_h h, const int* qubits, int nq, double* out);

/*
 * <psi|P|psi> for the Pauli string `paulis` (n characters from "IXYZ"; character q acts on qubit q).
 * out[0] = real part, out[1] = imaginary part (0 up to rounding). Compensated sums. Synchronises.
 */
int qsim_expect_pauli(qsim_h h, const char* paulis, double* out);

/*
 * All single-qubit and nearest-neighbour Z correlators in one pass: zi[i] = <Z_i> (n values) and
 * zz[i] = <Z_i Z_{i+1}> (n - 1 values), host arrays. Compensated sums. Synchronises.
 */
int qsim_expect_z(qsim_h h, double* zi, double* zz);

/*
 * Draw `shots` samples x ~ |a_x|^2 / sum |a|^2 (inverse CDF: the smallest x whose inclusive prefix
 * sum exceeds u * total). Uniform u_i is the i-th SplitMix64 output for `seed` (top 53 bits); the CDF
 * is never materialised: block sums of 4096 amplitudes, their FP64 prefix sums, then a search inside
 * one block per sample. out: `shots` uint64 indices, host, in the order of the uniforms. Synchronises.
 */
int qsim_sample(qsim_h h, uint64_t seed, int64_t shots, uint64_t* out);
/* Same with caller-supplied uniforms u[0..shots) in [0, 1) (host). */
int qsim_sample_uniforms(qsim_h h, const double* u, int64_t shots, uint64_t* out);
/*
 * qsim_expect_z followed by qsim_sample (same outputs, same seed convention) with one read of the state:
 * the <Z> pass also leaves the probability of every segment of 1024 amplitudes, and the sampler searches
 * those instead of summing the state again (Sec. 2.1: sampling and expectation values are the readouts of
 * a run). Samples equal qsim_sample's up to rounding at segment boundaries. Synchronises.
 */
int qsim_expect_z_and_sample(qsim_h h, double* zi, double* zz, uint64_t seed, int64_t shots, uint64_t* out);

/*
 * Sampling for callers that cannot allocate device memory (the paper has no counterpart; this is a library
 * service). A framework that has reserved all GPU memory in its own pool, or a latency-critical path that
 * cannot afford an allocation's implicit synchronisation, can draw samples from a state it owns without
 * creating a handle: dev_state is its complex64 (dtype 0) or complex128 (dtype 1) state of 2^n amplitudes
 * in device memory, dev_out a device buffer of `shots` uint64 that receives the indices, both owned by the
 * caller. Results are those of qsim_sample with the same seed. The call only enqueues work on `stream`
 * (a cudaStream_t; NULL = legacy default stream) and returns; dev_out is valid once the stream completes.
 * It allocates nothing: its scratch is one fixed 8 MiB array inside the library image, present on every
 * GPU that loads the library until the process exits. Requests needing more scratch than that (8 bytes
 * per shot plus 8 bytes per 4096 amplitudes, each region rounded up to 256 bytes) fail with QSIM_EINVAL
 * before any work: so n >= 32 is always refused (the 2^(n-12) segment sums alone fill the array), n = 31
 * allows 523 776 shots, n = 30 786 176, n = 22 1 047 520, and no n more than 2^20 = 1 048 576.
 * dev_state must be 256-byte aligned (like a state buffer given to qsim_create) and dev_out 8-byte
 * aligned; QSIM_EINVAL otherwise, before any work.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress); make that first
 * call before any stream capture. All calls share the array: calls whose work overlaps on the GPU race,
 * so serialise them (one stream, one host thread at a time).
 */
int qsim_sample_noalloc(const void* dev_state, int n, int dtype, uint64_t seed, int64_t shots,
                        uint64_t* dev_out, void* stream);

/* <a|b> = sum_x conj(a_x) b_x for two handles of equal n and dtype on the same device (Sec. 2.1: the
   amplitudes of the two state vectors; the overlap behind a fidelity). out[0..1] = (re, im). Synchronises. */
int qsim_inner(qsim_h a, qsim_h b, double* out);

/* ---- states in host memory (Sec. 2.5: host memory supplements GPU memory) ------------------------------ */

/*
 * Out-of-core execution for states larger than the device can hold (Sec. 2.5: host memory can supplement GPU
 * memory, at 4x or more per two extra qubits; Sec. 2.1: a state cut by its top index bits needs no exchange
 * for gates on the other qubits). The state stays in HOST memory (caller-owned, 2^n amplitudes in the
 * layout above; page-locked memory -- cudaHostAlloc, torch pin_memory -- lets the copies run asynchronously
 * and overlap, pageable memory works but serialises them). It is cut into slices of 2^L amplitudes by its top
 * n - L index bits, L = window_qubits - global_slots. The circuit is split into segments, each a set of
 * gates (dependencies kept) touching at most global_slots of those top bits; for every value of the other
 * top bits, the slices that differ only in the segment's bits are copied into a device window of
 * 2^window_qubits amplitudes, the segment's plan (made once per segment by the ordinary planner with
 * opts->run) runs there, and the window is copied back. Each segment reads and writes the whole state over
 * the host link once. Three windows are allocated (3 x 2^window_qubits amplitudes of device memory) and
 * rotate so that copies in, passes and copies out overlap.
 */
typedef struct {
    int32_t window_qubits;  /* W: index bits of a device window (14 <= W; W >= n: the state fits one window) */
    int32_t global_slots;   /* h: top index bits a window holds (0 = min(4, W - 12); 1..8, W - h >= 10) */
    qsim_run_opts run;      /* planning options for every segment (use_graph, dry_run, local_qubits ignored) */
} qsim_spill_opts;
typedef struct {
    int64_t segments;       /* stream-throughs of the whole state */
    int64_t windows;        /* window loads in all */
    int64_t passes;         /* kernel passes run on windows, summed over windows */
    double host_bytes;      /* bytes copied between host and device (in + out) */
    double elapsed_ms;      /* wall time of the call (it synchronises) */
    double host_plan_ms;    /* host time spent segmenting and planning */
    int32_t window_qubits;  /* W actually used (min(W, n)) */
    int32_t global_slots;   /* h actually used (0 when the state fits one window) */
} qsim_spill_info;
/* Run circuit c (c->n qubits) on the host state in place. The work is ordered after earlier work on `stream`
   (a cudaStream_t) and the call returns when it has completed. QSIM_EUNSUPPORTED when a gate has more than
   h qubits among the top n - L index bits. info may be NULL. */
int qsim_spill_run(void* host_state, const qsim_circuit* c, int dtype, const qsim_spill_opts* opts, void* stream,
                   qsim_spill_info* info);
/* The segmentation qsim_spill_run would use, on the host only (no device): seg_of_gate[i] = segment of gate i
   (c->num_gates entries); used_global (may be NULL; room for c->num_gates masks) = per segment, the qubit mask
   of the top index bits its gates touch; *nseg = number of segments. Gates of one segment run in their
   input order; any two gates sharing a qubit run in input order. */
int qsim_spill_segments(const qsim_circuit* c, int window_qubits, int global_slots, int32_t* seg_of_gate,
                        uint64_t* used_global, int64_t* nseg);
/* Sampling from a host state (Sec. 2.1 "Measurement and Sampling"): slices of 2^min(window_qubits, n)
   amplitudes are streamed through the device to sum |a_x|^2 per slice (compensated sums); each shot's uniform
   (the SplitMix64 stream of qsim_sample for `seed`) picks its slice by the FP64 prefix sums of the slice
   totals and is rescaled into that slice, which is then sampled on the device as qsim_sample_uniforms does.
   out: `shots` uint64 indices (host); *norm (may be NULL) = sum_x |a_x|^2. Synchronises. */
int qsim_spill_sample(const void* host_state, int n, int dtype, int window_qubits, uint64_t seed, int64_t shots,
                      uint64_t* out, double* norm);

/* ---- roofline calibration -------------------------------------------------------------------------------- */

/*
 * Dense tensor-core rate of the current GPU (a measurement service for roofline accounting; the paper has no
 * counterpart, its fusion level is chosen per architecture and precision, Sec. 2.2). Every SM runs one CTA
 * that issues tcgen05 MMAs back to back in the form the fused-block kernels use (A in tensor memory, B in
 * shared memory, M = 128, N = n_cols, FP32 accumulation) on resident operands, for about `seconds` seconds.
 * kind: 0 = TF32, 1 = BF16, 2 = FP16; n_cols: 128 or 256. *tflops receives 2 M N K x MMAs / elapsed time
 * (CUDA events); *ms (may be NULL) the elapsed time. Runs on a private stream, allocates 4 bytes, and
 * synchronises; QSIM_ETIMEOUT if a bounded wait of the probe expired.
 */
int qsim_tc_peak(int kind, int n_cols, double seconds, double* tflops, double* ms);

/*
 * Measured FP64 FMA rate of this GPU (library service, no passage: the denominator against which the
 * resident small-state runner's FP64 arithmetic is reported). Independent FP64 FMA chains on 32 warps per SM
 * for about `seconds` seconds (0 < seconds <= 30); *tflops receives 2 x FMAs / elapsed time (CUDA events),
 * *ms (may be NULL) the elapsed time. Runs on a private stream, allocates 8 bytes, and synchronises.
 */
int qsim_fp64_peak(double seconds, double* tflops, double* ms);

/* ---- batches of independent circuits (one persistent launch) ---------------------------------------- */

/*
 * Many independent circuits in one launch (Sec. 1: many circuits, e.g. for iterative algorithms, are one
 * reason to need large GPU resources). Every circuit starts from |0...0> (complex64); widths 1..26, gates on
 * at most 4 qubits (targets plus controls). Each circuit is fused with width k (opts->max_fused; 0 = the
 * width chosen for its qubit count by qsim_batch_autotune, default 4), composed in FP64 on the device, and
 * run by one persistent launch of thread-block clusters: a cluster per circuit of more than 13 qubits (its
 * state in the caller's workspace, passes separated by cluster barriers), then one CTA per smaller circuit
 * with the whole state in shared memory. With opts->precision a tensor-core precision, circuits of at
 * least opts->batch_tc_min_n qubits (default 20) are planned as fused tensor-core plans instead (k = 6
 * blocks, or up to 7 with QSIM_PREC_FP16X3; their state in the workspace) and enqueued after the persistent
 * launch, with their <Z> values reduced on the device: one cluster streams a wide state at a fraction of the
 * GPU's bandwidth, a plan's passes use all of it (below 24 qubits a half, below 22 a quarter of the SMs, so
 * that several run side by side). Those plans run on eight streams the batch owns, forked from the caller's stream
 * and joined back into it, so all work of an execution is ordered before later work on that stream. For circuit i, <Z_q> lands at zi[zi_off(i) + q] (q < n_i) and
 * <Z_q Z_{q+1}> at zz[zz_off(i) + q] (q < n_i - 1), the offsets being the running sums of n_i and n_i - 1
 * in input order; sums are compensated (float-float per thread, double-double across threads), and the
 * values are those of the normalised state (divided by the computed squared norm, which FP32 arithmetic
 * moves away from 1 by up to ~1e-5 over hundreds of tensor-core blocks).
 */
typedef struct qsim_batch* qsim_batch_h;
/* Device workspace (bytes) the circuits of more than 13 qubits need: sum of 2^n x 8 B, 256-byte aligned. */
int qsim_batch_workspace_bytes(const qsim_circuit* cs, int count, size_t* out);
/* Plan (fusion, FP64 composition on `stream`); the plan owns its device buffers. info may be NULL. */
int qsim_batch_plan_create(const qsim_circuit* cs, int count, const qsim_run_opts* opts, void* stream,
                           qsim_batch_h* out, qsim_plan_info* info);
/* Enqueue the batch on `stream` (asynchronous). dev_ws: device workspace of at least the bytes above,
   256-byte aligned, owned by the caller. use_graph = 1 replays a CUDA graph captured on first use. */
int qsim_batch_execute(qsim_batch_h b, void* dev_ws, size_t ws_bytes, void* stream, int use_graph);
/* Copy the last execution's <Z> values to host arrays zi, zz (see above for the layout). Synchronises. */
int qsim_batch_results(qsim_batch_h b, void* stream, double* zi, double* zz);
/* Release a batch plan and its device buffers. Library service, no passage. NULL is accepted. */
int qsim_batch_destroy(qsim_batch_h b);
/*
 * Plan, execute, fetch results and destroy in one call (Sec. 1: many circuits for iterative algorithms). The
 * work overlaps: the persistent launch of the narrower circuits goes out as soon as they are planned, and each
 * tensor-core plan of a wide circuit is enqueued as soon as it is made, while the host plans the others. The
 * results (zi, zz: host arrays laid out as for qsim_batch_results) are those of qsim_batch_plan_create +
 * qsim_batch_execute + qsim_batch_results, bit for bit. dev_ws: at least qsim_batch_workspace_bytes,
 * 256-byte aligned (QSIM_ENOMEM / QSIM_EINVAL otherwise, before any launch); every circuit is validated before
 * any launch. Synchronises `stream`.
 */
int qsim_batch_run(const qsim_circuit* cs, int count, const qsim_run_opts* opts, void* dev_ws,
                   size_t ws_bytes, void* stream, double* zi, double* zz, qsim_plan_info* info);
/*
 * Fusion-width tuner: for every width present in cs, time k = 1..4 on the first circuit of that width
 * (median of three launches after a warm-up; a trial workspace is allocated and released here) and keep
 * the fastest for later plans made with max_fused = 0 (process-wide). chosen (may be NULL) receives the k
 * each circuit would now get.
 */
int qsim_batch_autotune(const qsim_circuit* cs, int count, void* stream, int* chosen);
/*
 * Tuner for the width from which batched circuits run as tensor-core plans (a library service beside the
 * fusion-width tuner; Sec. 2.2: the fusion setting is tuned per architecture and precision): the whole batch
 * cs is planned and replayed (graph, median of three after a warm-up) with batch_tc_min_n = 14, 16, ..., 24
 * and 27 (no circuit leaves the persistent launch), for `precision` (a tensor-core one); the fastest
 * threshold is kept process-wide for plans made with batch_tc_min_n = 0 and returned in *best_min_n (may be
 * NULL). Allocates a trial workspace and releases it.
 */
int qsim_batch_autotune_threshold(const qsim_circuit* cs, int count, int precision, void* stream, int* best_min_n);
/*
 * The process-wide tuning (fusion width per circuit width, tensor-core threshold per precision) to and from a
 * small JSON file (library service). Load validates every entry (QSIM_EINVAL for a file that is not such a
 * table; nothing is changed then). With the environment variable QSIM_TUNE_CACHE set to a path, the table is
 * read from it before the first batch plan or tuning of the process (if the file exists) and written to it
 * after every successful tuning.
 */
int qsim_batch_tune_save(const char* path);
int qsim_batch_tune_load(const char* path);

#ifdef __cplusplus
}
#endif

#endif /* QSIM_H */
