// internal.h -- host-side declarations shared by the libqsim translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/qsim.h"

namespace qsim {

constexpr int kMaxFixed = QSIM_MAX_TARGETS + QSIM_MAX_CONTROLS;

struct DevInfo {
    int device = 0;
    int num_sms = 1;
    size_t smem_optin = 0;
};

// Per-call error message (thread-local) used by qsim_last_error().
void set_error(const char* fmt, ...);
// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) once per kernel, device and size (the largest asked so far
// covers smaller launches): the call is a driver round trip, which a plan's passes would otherwise make before
// every launch.
cudaError_t smem_optin(const void* kern, int bytes);
int cuda_fail(cudaError_t e, const char* what);

// ---- gate kernels (k_gates.cu) ------------------------------------------------------------------------------
// Dense U on k <= 4 targets with controls; `mat` is 2^k x 2^k interleaved complex128 (host), converted to
// the state precision and passed by value.
cudaError_t launch_dense_small(int dtype, void* psi, int n, int k, const int* targets, int nc,
                               const int* controls, const double* mat, cudaStream_t s, const DevInfo& d);
// Diagonal gate: diag (host, 2^k complex128) on targets; only patterns listed in `touch` are updated.
cudaError_t launch_diag(int dtype, void* psi, int n, int k, const int* targets, int nc, const int* controls,
                        const double* diag, const std::vector<int>& touch, cudaStream_t s, const DevInfo& d);
// Dense U on k = 5, 6 targets with controls; `dmat` is a DEVICE buffer of 2^k x 2^k complex in the state
// precision (interleaved, row-major).
cudaError_t launch_dense_tile(int dtype, void* psi, int n, int k, const int* targets, int nc,
                              const int* controls, const void* dmat, cudaStream_t s, const DevInfo& d);
// Exchange qubits a[i] <-> b[i] (i < p) in place; splits into several passes when one tile cannot hold
// all swapped bits. Returns the number of passes through *passes when non-NULL.
cudaError_t launch_swap(int dtype, void* psi, int n, const int* a, const int* b, int p, cudaStream_t s,
                        const DevInfo& d, int* passes);
cudaError_t launch_set_basis(int dtype, void* psi, int n, uint64_t x, cudaStream_t s, const DevInfo& d);
// Convert a device FP64 matrix (2^k x 2^k complex) into the state precision (device -> device).
cudaError_t launch_convert_matrix(int dtype, const double* src, void* dst, int64_t count, cudaStream_t s);

// ---- every pass of a small-state plan in one cooperative launch (k_small.cu) --------------------------------
constexpr int kSmallMaxQubits = 16;  // states of at most 2^16 amplitudes (1 MiB complex128): L2-resident
struct PhaseForm;
// One pass of such a plan: a dense U on k <= 5 targets or a diagonal on k <= 6 targets, with any controls, or a
// phase pass (form).
struct SmallOpDesc {
    bool diag = false;
    int k = 0, nc = 0;
    const int* targets = nullptr;
    const int* controls = nullptr;
    const double* mat = nullptr;               // dense: 2^k x 2^k; diagonal: 2^k entries (interleaved, FP64)
    const std::vector<int>* touch = nullptr;   // diagonal: entries with a factor other than 1
    const PhaseForm* form = nullptr;           // phase pass: its combined phase (the other fields unused)
};
// Device bytes of the program of npass passes (a barrier word, then one fixed-size record per pass).
size_t small_program_bytes(int dtype, int npass);
// Write the program into host memory `out` (small_program_bytes bytes); false if a pass is outside the limits.
bool small_program_build(int dtype, const std::vector<SmallOpDesc>& ops, unsigned char* out);
// Run the uploaded program (16-byte aligned device copy) on the state in one cooperative launch, grid
// barriers between passes; with from_basis the state is first set to |*from_basis>.
cudaError_t launch_small_run(int dtype, void* psi, int n, void* dprog, int npass, unsigned* dev_err, cudaStream_t s,
                             const DevInfo& d, const uint64_t* from_basis);

// ---- phase pass: any number of 1- and 2-qubit diagonal gates (k_phase.cu) -----------------------------------
// The combined phase c + sum_a h_a x_a + sum_{a<b} lam_ab x_a x_b (radians) of a run of diagonal gates.
struct PhaseForm {
    struct Pair { int a, b; double lam; };
    double c = 0.0;
    std::vector<double> h;     // per qubit
    std::vector<Pair> pairs;   // a < b, one entry per pair
};
// Launch parameters of a packed form: 64-bit fixed-point constants and byte offsets of the device tables.
struct PhasePacked {
    uint64_t c = 0;
    int nb = 0, ntt = 0;
    int lt_off[15] = {};
    size_t off_tt_ab = 0, off_tt_l = 0, off_lt_a = 0, off_lt_l = 0, off_small = 0, off_tmid = 0;
};
// A phase in radians as 64-bit fixed-point turns (2^64 = one turn), reduced to [0, 1) turn.
uint64_t phase_turns(double phi);
// A diagonal gate the phase pass takes: 1 or 2 qubits in all (targets plus controls).
bool phase_gate_ok(const qsim_gate& g);
// The form of gates[0..count) (each diagonal, phase_gate_ok); false if one is not acceptable.
bool phase_form_build(const qsim_gate* const* gates, int count, int n, PhaseForm& f);
// Device tables of a form (bytes to upload as they are) and its launch parameters.
void phase_pack(const PhaseForm& f, int dtype, std::vector<unsigned char>& out, PhasePacked& pk);
// Multiply every amplitude by exp(i phi(x)); dtab is the uploaded table block; n >= 10.
cudaError_t launch_phase(int dtype, void* psi, int n, const void* dtab, const PhasePacked& pk, cudaStream_t s,
                         const DevInfo& d);

// ---- tensor-core fused block (k_tc.cu) ----------------------------------------------------------------------
// Launch parameters of a phase epilogue (a phase form applied to the block's output): byte offsets of the
// device tables and the counts.
struct TcEpiPacked {
    uint64_t c = 0;
    int ntt = 0;
    int off[14] = {};
    size_t off_rowphase = 0, off_tt_ab = 0, off_tt_l = 0, off_tb_t = 0, off_tb_l = 0, off_thr = 0;
};
// Tables of a phase epilogue for a k-qubit block on `targets` (the order launch_tc_apply gets) in an n-qubit
// state. The terms on target bits alone become row phases of U (off_rowphase, for launch_tc_prepare); each
// launch writes the per-tile factors to a scratch of tc_epi_scratch_bytes.
void tc_epi_pack(int n, int k, const int* targets, const PhaseForm& f, std::vector<unsigned char>& out,
                 TcEpiPacked& pk);
size_t tc_epi_scratch_bytes(int n, int k);
// Bytes of the prepared B operand for a k-qubit block at `precision`.
size_t tc_operand_bytes(int k, int precision);
// Build the B operand (tensor-core layout) from a device FP64 matrix U (2^k x 2^k complex) for a block on
// `targets` (their order decides the data path, and with it the column order of B).
// cudaErrorInvalidValue for an unsupported k or precision, or `lines` with a precision or epilogue that has
// no line-group path.
cudaError_t launch_tc_prepare(const double* dU, int k, int precision, bool lines, void* dB, cudaStream_t s,
                              const double* rowphase = nullptr);
// True when a block on `targets` may run the line-group data path (qubits 0..3 are targets 0..3, 3xTF32, no
// phase epilogue). The operand must then be prepared with lines = true and applied with lines = true.
bool tc_line_groups(int k, const int* targets, int precision, bool epi);
// Apply the prepared block to a complex64 state. dev_err receives DEVERR_* bits on a bounded-wait expiry.
// With from_basis the block's input is the basis state |*from_basis>, generated instead of read (the block
// writes the whole state). lines: the operand was prepared for the line-group path (tc_line_groups must hold
// for these targets, else cudaErrorInvalidValue).
cudaError_t launch_tc_apply(void* psi, int n, int k, const int* targets, const void* dB, int precision,
                            unsigned* dev_err, cudaStream_t s, const DevInfo& d, const void* epi_tab = nullptr,
                            const TcEpiPacked* epi = nullptr, void* epi_scratch = nullptr,
                            const uint64_t* from_basis = nullptr, bool lines = false);
bool tc_supported(int k, int precision);

// ---- 7-qubit blocks (k_tc7.cu, FP16 split products; reached through the tensor-core entry points above
// with k = 7 and QSIM_PREC_FP16X3) ----------------------------------------------------------------------------
size_t tc7_operand_bytes();
cudaError_t launch_tc7_prepare(const double* dU, void* dB, cudaStream_t s);
cudaError_t launch_tc7_apply(void* psi, int n, const int* targets, const void* dB, unsigned* dev_err, cudaStream_t s,
                             const DevInfo& d, const uint64_t* from_basis);

// ---- two 6-qubit blocks in one pass (k_tc_pair.cu, FP16 split products) -------------------------------------
// True when blocks on t1 and then t2 (6 targets each, in their matrices' index order) fit one 13-bit tile of
// an n-qubit state (|t1 u t2| <= 12, n >= 13).
bool tc_pair_supported(int n, const int* t1, int k1, const int* t2, int k2);
// Bytes of a pair's prepared operands: the real forms of U1 and U2 as FP16 hi / lo planes (4 x 32 KiB).
size_t tc_pair_operand_bytes();
// Prepare the operands from device FP64 matrices U1, U2 (64 x 64 complex each) into dops.
cudaError_t launch_tc_pair_prepare(const double* dU1, const double* dU2, void* dops, cudaStream_t s);
// Apply U1 on t1, then U2 on t2, to a complex64 state in one pass. from_basis: the input is that basis state.
cudaError_t launch_tc_pair(void* psi, int n, const int* t1, const int* t2, const void* dops, unsigned* dev_err,
                           cudaStream_t s, const DevInfo& d, const uint64_t* from_basis = nullptr);

// ---- fused-block composition (k_compose.cu) -------------------------------------------------------------------
struct ComposeGate {
    int k, nc;
    int targets[QSIM_MAX_TARGETS];   // local indices within the block's qubit list
    int controls[QSIM_MAX_CONTROLS]; // local indices
    int64_t mat_off;                 // offset (in complex entries) into the gate-matrix pool
};
struct ComposeBlock {
    int kb;         // block width (local qubits 0..kb-1)
    int first_gate; // index into the ComposeGate array
    int num_gates;
    int64_t out_off; // offset (in complex entries) of the 2^kb x 2^kb output
};
// For every block: U_block = G_last ... G_first on kb local qubits, in FP64, on the device.
cudaError_t launch_compose(const ComposeBlock* dblocks, int nblocks, const ComposeGate* dgates,
                           const double* dpool, double* dout, int max_kb, cudaStream_t s);

// ---- reductions and sampling (k_reduce.cu) ------------------------------------------------------------------------
struct ReduceScratch {
    double* partials = nullptr;  // kPartialDoubles doubles
    double* seg = nullptr;       // 2 * 2^(n-10) doubles: segment sums (doubles, then float-float pairs)
    double* scan = nullptr;      // max(1, 2^(n-12)) + 4096 doubles
    double* result = nullptr;    // 256 doubles (device)
    double* hresult = nullptr;   // 256 doubles (pinned host)
};
constexpr int64_t kPartialDoubles = 1 << 21;
constexpr int kSegBits = 12;

cudaError_t run_norm(int dtype, const void* psi, int n, ReduceScratch& r, cudaStream_t s, const DevInfo& d,
                     double* out);
cudaError_t run_probs(int dtype, const void* psi, int n, const int* qubits, int nq, ReduceScratch& r,
                      cudaStream_t s, const DevInfo& d, double* out);
cudaError_t run_pauli(int dtype, const void* psi, int n, const char* paulis, ReduceScratch& r, cudaStream_t s,
                      const DevInfo& d, double* out);
cudaError_t run_zstats(int dtype, const void* psi, int n, ReduceScratch& r, cudaStream_t s, const DevInfo& d,
                       double* zi, double* zz);
// The same values written to device arrays zi_dev[n], zz_dev[n - 1] on `s` (no host synchronisation);
// normalise: divided by the squared norm (the values of the normalised state).
cudaError_t run_zstats_device(int dtype, const void* psi, int n, ReduceScratch& r, cudaStream_t s,
                              const DevInfo& d, double* zi_dev, double* zz_dev, bool normalise);
cudaError_t run_inner(int dtype, const void* a, const void* b, int n, ReduceScratch& r, cudaStream_t s,
                      const DevInfo& d, double* out);
// Samples: u_dev (device, shots doubles) -> out_dev (device, shots uint64).
cudaError_t run_sample(int dtype, const void* psi, int n, const double* u_dev, int64_t shots, uint64_t* out_dev,
                       ReduceScratch& r, cudaStream_t s, const DevInfo& d,
                       int seg_ready_bits = 0);
// Bits of the segments whose sums run_zstats leaves in r.seg (0: none).
int zstats_segment_bits(int n);
cudaError_t launch_uniforms(uint64_t seed, int64_t count, double* out_dev, cudaStream_t s);

}  // namespace qsim
