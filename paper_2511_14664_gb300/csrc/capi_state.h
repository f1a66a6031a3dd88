// capi_state.h -- the handle behind qsim_h and helpers shared by capi.cu and plan.cu.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "internal.h"

namespace qsim {

constexpr size_t kDevMatBytes = 1 << 20;  // per-handle device scratch for one gate / block operand

}  // namespace qsim

struct qsim_state {
    int n = 0;
    int dtype = QSIM_C64;
    void* psi = nullptr;
    size_t bytes = 0;
    bool owns = false;
    cudaStream_t stream = nullptr;
    qsim::DevInfo dev;
    qsim::ReduceScratch red;
    void* dmat = nullptr;       // kDevMatBytes: a gate matrix in state precision or a tensor-core operand
    double* dmat64 = nullptr;   // 64 KiB FP64 staging for a block matrix
    unsigned* derr = nullptr;   // device error word (DEVERR_* bits)
    uint64_t* dsamples = nullptr;
    double* du = nullptr;
    size_t samples_cap = 0;
};

namespace qsim {

bool is_diagonal(const double* m, int k);
bool is_unitary(const double* m, int k, double tol);
int validate_qubits(int n, const int* targets, int k, const int* controls, int nc, int kmax);
std::vector<int> nonunit_patterns(const double* diag, int k);
int check_device_error(qsim_state* h);
int apply_gate_plain(qsim_state* h, const int* targets, int k, const int* controls, int nc, const double* m);

// Greedy fusion (plan.cu): starting from the earliest unplaced gate, collect every later gate that is not
// blocked by an earlier unplaced gate on a shared qubit (diagonal gates are blocked only by non-diagonal
// ones) and keeps the block within kmax qubits. gmask[i] = qubits of gate i (targets and controls). With
// gwide, the diagonal gates it marks may also form one block of any width (a phase pass), chosen when it
// holds more than wide_factor times the gates of the best other candidate. lookahead > 0: choose among the
// `lookahead` largest candidates by their size plus that of the best block after them. *wide_used (if given) is
// set when a block was the phase candidate.
std::vector<std::vector<int>> group_gates(const std::vector<uint64_t>& gmask, const std::vector<char>& gdiag, int n,
                                          int kmax, const std::vector<char>* gwide = nullptr, int wide_factor = 1,
                                          int lookahead = 0, uint64_t narrow = 0, bool* wide_used = nullptr);
// Groupings cached by structure (plan.cu): key words describe the request (options, each gate's qubit mask and
// flags); the first word tells the requester apart (0 plans, 1 batch circuits).
bool group_cache_get(const std::vector<uint64_t>& key, std::vector<std::vector<int>>& out);
void group_cache_put(const std::vector<uint64_t>& key, const std::vector<std::vector<int>>& blocks);

}  // namespace qsim

extern "C" int qsim_synchronize(qsim_h h);
