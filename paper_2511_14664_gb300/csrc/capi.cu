// capi.cu -- the C ABI of libqsim (declared in include/qsim.h): handles, argument validation, dispatch of
// each gate to its kernel, and the readout entry points. No exception or CUDA error crosses the ABI: every
// failure becomes a QSIM_E* code plus a thread-local message.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "capi_state.h"
#include "internal.h"

namespace qsim {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

cudaError_t smem_optin(const void* kern, int bytes) {
    struct Entry { const void* kern; int device; int bytes; };
    static std::mutex mu;
    static std::vector<Entry> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    for (Entry& x : done)
        if (x.kern == kern && x.device == dev) {
            if (x.bytes >= bytes) return cudaSuccess;
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
            if (e == cudaSuccess) x.bytes = bytes;
            return e;
        }
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done.push_back({kern, dev, bytes});
    return e;
}

int cuda_fail(cudaError_t e, const char* what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return QSIM_ECUDA;
}

bool is_diagonal(const double* m, int k) {
    const int D = 1 << k;
    for (int r = 0; r < D; ++r)
        for (int c = 0; c < D; ++c)
            if (r != c && (m[2 * (r * D + c)] != 0.0 || m[2 * (r * D + c) + 1] != 0.0)) return false;
    return true;
}

bool is_unitary(const double* m, int k, double tol) {
    const int D = 1 << k;
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
            double re = 0, im = 0;  // (U U^dagger)_{ij} = sum_c U_ic conj(U_jc)
            for (int c = 0; c < D; ++c) {
                const double ar = m[2 * (i * D + c)], ai = m[2 * (i * D + c) + 1];
                const double br = m[2 * (j * D + c)], bi = m[2 * (j * D + c) + 1];
                re += ar * br + ai * bi;
                im += ai * br - ar * bi;
            }
            if (std::fabs(re - (i == j ? 1.0 : 0.0)) > tol || std::fabs(im) > tol) return false;
        }
    return true;
}

int validate_qubits(int n, const int* targets, int k, const int* controls, int nc, int kmax) {
    if (k < 1 || k > kmax) { set_error("number of targets %d outside 1..%d", k, kmax); return QSIM_EINVAL; }
    if (nc < 0 || nc > QSIM_MAX_CONTROLS) { set_error("number of controls %d outside 0..%d", nc, QSIM_MAX_CONTROLS); return QSIM_EINVAL; }
    if (!targets || (nc > 0 && !controls)) { set_error("NULL qubit list"); return QSIM_EINVAL; }
    uint64_t seen = 0;
    for (int j = 0; j < k + nc; ++j) {
        const int q = j < k ? targets[j] : controls[j - k];
        if (q < 0 || q >= n) { set_error("qubit %d outside 0..%d", q, n - 1); return QSIM_EINVAL; }
        if ((seen >> q) & 1) { set_error("qubit %d listed twice (targets and controls must be distinct)", q); return QSIM_EINVAL; }
        seen |= 1ull << q;
    }
    return QSIM_OK;
}

// Patterns m (over the targets) whose diagonal factor is not exactly 1.
std::vector<int> nonunit_patterns(const double* diag, int k) {
    std::vector<int> t;
    const int D = 1 << k;
    for (int m = 0; m < D; ++m)
        if (diag[2 * m] != 1.0 || diag[2 * m + 1] != 0.0) t.push_back(m);
    return t;
}

// Check the handle's device error word (after the stream has been synchronised).
int check_device_error(qsim_state* h) {
    unsigned v = 0;
    cudaError_t e = cudaMemcpy(&v, h->derr, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "reading the device error word");
    if (v) {
        cudaMemset(h->derr, 0, sizeof(unsigned));
        set_error("a device-side bounded wait expired (code 0x%x); the state is undefined", v);
        return QSIM_ETIMEOUT;
    }
    return QSIM_OK;
}

// Apply one gate through the plain per-gate kernels (shared by qsim_apply_gate and plan execution).
int apply_gate_plain(qsim_state* h, const int* targets, int k, const int* controls, int nc, const double* m) {
    cudaError_t e;
    if (k <= 6 && is_diagonal(m, k)) {
        std::vector<double> dg(2 << k);
        const int D = 1 << k;
        for (int i = 0; i < D; ++i) { dg[2 * i] = m[2 * (i * D + i)]; dg[2 * i + 1] = m[2 * (i * D + i) + 1]; }
        e = launch_diag(h->dtype, h->psi, h->n, k, targets, nc, controls, dg.data(), nonunit_patterns(dg.data(), k),
                        h->stream, h->dev);
        return e == cudaSuccess ? QSIM_OK : cuda_fail(e, "diagonal gate launch");
    }
    if (k <= 4) {
        e = launch_dense_small(h->dtype, h->psi, h->n, k, targets, nc, controls, m, h->stream, h->dev);
        return e == cudaSuccess ? QSIM_OK : cuda_fail(e, "dense gate launch");
    }
    // k = 5..8: matrix to device scratch in the state precision
    const int D = 1 << k;
    const size_t cnt = 2 * (size_t)D * D;
    if (h->dtype == QSIM_C64) {
        std::vector<float> f(cnt);
        for (size_t i = 0; i < cnt; ++i) f[i] = (float)m[i];
        e = cudaMemcpyAsync(h->dmat, f.data(), cnt * sizeof(float), cudaMemcpyHostToDevice, h->stream);
    } else {
        e = cudaMemcpyAsync(h->dmat, m, cnt * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "matrix upload");
    // pageable host memory: wait for the copy so the temporary above may be released
    if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return cuda_fail(e, "matrix upload");
    e = launch_dense_tile(h->dtype, h->psi, h->n, k, targets, nc, controls, h->dmat, h->stream, h->dev);
    return e == cudaSuccess ? QSIM_OK : cuda_fail(e, "dense tile launch");
}

}  // namespace qsim

using namespace qsim;

#define QSIM_CHECK_HANDLE(h)                                  \
    do {                                                      \
        if (!(h)) { set_error("NULL handle"); return QSIM_EINVAL; } \
        set_error("%s", "");                                  \
    } while (0)

extern "C" {

int qsim_abi_version(void) { return QSIM_ABI_VERSION; }

const char* qsim_last_error(void) { return g_err; }

int qsim_state_bytes(int n, int dtype, size_t* out) {
    if (!out) { set_error("NULL output"); return QSIM_EINVAL; }
    if (n < 1 || n > QSIM_MAX_QUBITS) { set_error("n = %d outside 1..%d", n, QSIM_MAX_QUBITS); return QSIM_EINVAL; }
    if (dtype != QSIM_C64 && dtype != QSIM_C128) { set_error("unknown dtype %d", dtype); return QSIM_EINVAL; }
    *out = (size_t)(dtype == QSIM_C64 ? 8 : 16) << n;
    return QSIM_OK;
}

int qsim_create(int n, int dtype, void* dev_buf, size_t buf_bytes, void* stream, qsim_h* out) {
    set_error("%s", "");
    if (!out) { set_error("NULL output handle"); return QSIM_EINVAL; }
    *out = nullptr;
    size_t need = 0;
    int rc = qsim_state_bytes(n, dtype, &need);
    if (rc) return rc;
    if (dev_buf && buf_bytes < need) { set_error("buffer of %zu bytes < %zu needed", buf_bytes, need); return QSIM_ENOMEM; }
    if (dev_buf && (reinterpret_cast<uintptr_t>(dev_buf) & 255)) { set_error("state buffer must be 256-byte aligned"); return QSIM_EINVAL; }
    qsim_state* h = new (std::nothrow) qsim_state();
    if (!h) { set_error("out of host memory"); return QSIM_ENOMEM; }
    h->n = n;
    h->dtype = dtype;
    h->bytes = need;
    h->stream = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaGetDevice(&h->dev.device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->dev.num_sms, cudaDevAttrMultiProcessorCount, h->dev.device);
    int optin = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->dev.device);
    h->dev.smem_optin = (size_t)optin;
    if (e != cudaSuccess) { delete h; return cuda_fail(e, "querying the device"); }
    if (dev_buf) {
        h->psi = dev_buf;
    } else {
        e = cudaMalloc(&h->psi, need);
        if (e != cudaSuccess) { delete h; set_error("cudaMalloc of %zu state bytes failed", need); return QSIM_ENOMEM; }
        h->owns = true;
    }
    const uint64_t nseg = n > kSegBits ? (1ull << (n - kSegBits)) : 1ull;
    bool ok = cudaMalloc(&h->red.partials, sizeof(double) * kPartialDoubles) == cudaSuccess;
    const uint64_t nseg10 = n > 10 ? (1ull << (n - 10)) : 1ull;  // 1024-amplitude segments of the <Z> pass
    ok = ok && cudaMalloc(&h->red.seg, sizeof(double) * std::max<uint64_t>(2 * nseg, 2 * nseg10)) == cudaSuccess;
    ok = ok && cudaMalloc(&h->red.scan, sizeof(double) * (nseg + 8192)) == cudaSuccess;
    ok = ok && cudaMalloc(&h->red.result, sizeof(double) * 256) == cudaSuccess;
    ok = ok && cudaMallocHost(&h->red.hresult, sizeof(double) * 256) == cudaSuccess;
    ok = ok && cudaMalloc(&h->dmat, kDevMatBytes) == cudaSuccess;
    ok = ok && cudaMalloc(&h->dmat64, sizeof(double) * 2 * 16384) == cudaSuccess;  // a 7-qubit block
    ok = ok && cudaMalloc(&h->derr, sizeof(unsigned)) == cudaSuccess;
    ok = ok && cudaMemset(h->derr, 0, sizeof(unsigned)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        qsim_destroy(h);
        set_error("workspace allocation failed");
        return QSIM_ENOMEM;
    }
    *out = h;
    return QSIM_OK;
}

int qsim_destroy(qsim_h h) {
    if (!h) return QSIM_OK;
    if (h->stream || true) cudaStreamSynchronize(h->stream);
    if (h->owns && h->psi) cudaFree(h->psi);
    cudaFree(h->red.partials);
    cudaFree(h->red.seg);
    cudaFree(h->red.scan);
    cudaFree(h->red.result);
    if (h->red.hresult) cudaFreeHost(h->red.hresult);
    cudaFree(h->dmat);
    cudaFree(h->dmat64);
    cudaFree(h->derr);
    cudaFree(h->dsamples);
    cudaFree(h->du);
    delete h;
    return QSIM_OK;
}

int qsim_set_stream(qsim_h h, void* stream) {
    QSIM_CHECK_HANDLE(h);
    h->stream = reinterpret_cast<cudaStream_t>(stream);
    return QSIM_OK;
}

int qsim_num_qubits(qsim_h h, int* n) {
    QSIM_CHECK_HANDLE(h);
    if (!n) { set_error("NULL output"); return QSIM_EINVAL; }
    *n = h->n;
    return QSIM_OK;
}

int qsim_device_ptr(qsim_h h, void** out) {
    QSIM_CHECK_HANDLE(h);
    if (!out) { set_error("NULL output"); return QSIM_EINVAL; }
    *out = h->psi;
    return QSIM_OK;
}

int qsim_set_basis(qsim_h h, uint64_t x) {
    QSIM_CHECK_HANDLE(h);
    if (x >> h->n) { set_error("basis index %llu >= 2^%d", (unsigned long long)x, h->n); return QSIM_EINVAL; }
    cudaError_t e = launch_set_basis(h->dtype, h->psi, h->n, x, h->stream, h->dev);
    return e == cudaSuccess ? QSIM_OK : cuda_fail(e, "set_basis launch");
}

int qsim_set_state(qsim_h h, const void* src, int src_on_device) {
    QSIM_CHECK_HANDLE(h);
    if (!src) { set_error("NULL source"); return QSIM_EINVAL; }
    cudaError_t e = cudaMemcpyAsync(h->psi, src, h->bytes, src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && !src_on_device) e = cudaStreamSynchronize(h->stream);
    return e == cudaSuccess ? QSIM_OK : cuda_fail(e, "set_state copy");
}

int qsim_get_state(qsim_h h, void* dst, int dst_on_device) {
    QSIM_CHECK_HANDLE(h);
    if (!dst) { set_error("NULL destination"); return QSIM_EINVAL; }
    cudaError_t e = cudaMemcpyAsync(dst, h->psi, h->bytes, dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && !dst_on_device) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "get_state copy");
    return dst_on_device ? QSIM_OK : check_device_error(h);
}

int qsim_synchronize(qsim_h h) {
    QSIM_CHECK_HANDLE(h);
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    return check_device_error(h);
}

int qsim_inject_device_error(qsim_h h, unsigned code) {
    QSIM_CHECK_HANDLE(h);
    if (!code) { set_error("code must be nonzero"); return QSIM_EINVAL; }
    // after the work already enqueued, so that the word is not cleared or overwritten behind the caller
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess) e = cudaMemcpy(h->derr, &code, sizeof(unsigned), cudaMemcpyHostToDevice);
    return e == cudaSuccess ? QSIM_OK : cuda_fail(e, "writing the device error word");
}

int qsim_apply_gate(qsim_h h, const int* targets, int k, const int* controls, int nc, const double* matrix) {
    QSIM_CHECK_HANDLE(h);
    int rc = validate_qubits(h->n, targets, k, controls, nc, QSIM_MAX_TARGETS);
    if (rc) return rc;
    if (!matrix) { set_error("NULL matrix"); return QSIM_EINVAL; }
    if (!is_unitary(matrix, k, 1e-8 * (1 << k))) { set_error("matrix is not unitary (|U U^dagger - I| > %g)", 1e-8 * (1 << k)); return QSIM_EINVAL; }
    return apply_gate_plain(h, targets, k, controls, nc, matrix);
}

int qsim_apply_fused(qsim_h h, const int* targets, int k, const double* matrix, int precision) {
    QSIM_CHECK_HANDLE(h);
    int rc = validate_qubits(h->n, targets, k, nullptr, 0, QSIM_MAX_TARGETS);
    if (rc) return rc;
    if (!matrix) { set_error("NULL matrix"); return QSIM_EINVAL; }
    if (precision < QSIM_PREC_SIMT || precision > QSIM_PREC_FP16X3) { set_error("unknown precision %d", precision); return QSIM_EINVAL; }
    if (precision == QSIM_PREC_SIMT) {
        if (k <= 4) {
            cudaError_t e = launch_dense_small(h->dtype, h->psi, h->n, k, targets, 0, nullptr, matrix, h->stream, h->dev);
            return e == cudaSuccess ? QSIM_OK : cuda_fail(e, "dense gate launch");
        }
        return apply_gate_plain(h, targets, k, nullptr, 0, matrix);
    }
    if (h->dtype != QSIM_C64) { set_error("tensor-core precisions need a complex64 state"); return QSIM_EUNSUPPORTED; }
    if (!tc_supported(k, precision)) { set_error("tensor-core block of %d qubits is not supported", k); return QSIM_EUNSUPPORTED; }
    if (h->n < k + 7) { set_error("tensor-core block needs n >= k + 7"); return QSIM_EUNSUPPORTED; }
    const size_t cnt = (size_t)2 << (2 * k);
    cudaError_t e = cudaMemcpyAsync(h->dmat64, matrix, cnt * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    const bool lines = tc_line_groups(k, targets, precision, false);
    if (e == cudaSuccess) e = launch_tc_prepare(h->dmat64, k, precision, lines, h->dmat, h->stream);
    if (e == cudaSuccess)
        e = launch_tc_apply(h->psi, h->n, k, targets, h->dmat, precision, h->derr, h->stream, h->dev, nullptr, nullptr,
                            nullptr, nullptr, lines);
    return e == cudaSuccess ? QSIM_OK : cuda_fail(e, "tensor-core block");
}

int qsim_swap_qubits(qsim_h h, const int* a, const int* b, int p) {
    QSIM_CHECK_HANDLE(h);
    if (p == 0) return QSIM_OK;
    if (p < 0 || p > 8 || !a || !b) { set_error("need 1..8 qubit pairs"); return QSIM_EINVAL; }
    uint64_t seen = 0;
    for (int i = 0; i < 2 * p; ++i) {
        const int q = i < p ? a[i] : b[i - p];
        if (q < 0 || q >= h->n || ((seen >> q) & 1)) { set_error("swap qubits must be distinct and < n"); return QSIM_EINVAL; }
        seen |= 1ull << q;
    }
    cudaError_t e = launch_swap(h->dtype, h->psi, h->n, a, b, p, h->stream, h->dev, nullptr);
    return e == cudaSuccess ? QSIM_OK : cuda_fail(e, "swap launch");
}

int qsim_norm(qsim_h h, double* out) {
    QSIM_CHECK_HANDLE(h);
    if (!out) { set_error("NULL output"); return QSIM_EINVAL; }
    cudaError_t e = run_norm(h->dtype, h->psi, h->n, h->red, h->stream, h->dev, out);
    if (e != cudaSuccess) return cuda_fail(e, "norm");
    return check_device_error(h);
}

int qsim_probs(qsim_h h, const int* qubits, int nq, double* out) {
    QSIM_CHECK_HANDLE(h);
    if (!out || !qubits) { set_error("NULL argument"); return QSIM_EINVAL; }
    if (nq < 1 || nq > 30 || nq > h->n) { set_error("nq = %d outside 1..min(30, n)", nq); return QSIM_EINVAL; }
    uint64_t seen = 0;
    for (int j = 0; j < nq; ++j) {
        if (qubits[j] < 0 || qubits[j] >= h->n || ((seen >> qubits[j]) & 1)) { set_error("bad marginal qubit list"); return QSIM_EINVAL; }
        seen |= 1ull << qubits[j];
    }
    cudaError_t e = run_probs(h->dtype, h->psi, h->n, qubits, nq, h->red, h->stream, h->dev, out);
    if (e != cudaSuccess) return cuda_fail(e, "probs");
    return check_device_error(h);
}

int qsim_expect_pauli(qsim_h h, const char* paulis, double* out) {
    QSIM_CHECK_HANDLE(h);
    if (!paulis || !out) { set_error("NULL argument"); return QSIM_EINVAL; }
    for (int q = 0; q < h->n; ++q) {
        const char c = paulis[q];
        if (c != 'I' && c != 'X' && c != 'Y' && c != 'Z') { set_error("Pauli string must have n characters from IXYZ"); return QSIM_EINVAL; }
    }
    if (paulis[h->n] != '\0') { set_error("Pauli string longer than n"); return QSIM_EINVAL; }
    cudaError_t e = run_pauli(h->dtype, h->psi, h->n, paulis, h->red, h->stream, h->dev, out);
    if (e != cudaSuccess) return cuda_fail(e, "expect_pauli");
    return check_device_error(h);
}

int qsim_expect_z(qsim_h h, double* zi, double* zz) {
    QSIM_CHECK_HANDLE(h);
    if (!zi || (!zz && h->n > 1)) { set_error("NULL output"); return QSIM_EINVAL; }
    std::vector<double> zz_dummy(1);
    cudaError_t e = run_zstats(h->dtype, h->psi, h->n, h->red, h->stream, h->dev, zi, zz ? zz : zz_dummy.data());
    if (e != cudaSuccess) return cuda_fail(e, "expect_z");
    return check_device_error(h);
}

static int sample_common(qsim_h h, int64_t shots, uint64_t* out, const double* u_host, uint64_t seed,
                         int seg_ready_bits = 0) {
    if (!out) { set_error("NULL output"); return QSIM_EINVAL; }
    if (shots < 0 || shots > (1ll << 31)) { set_error("shots outside 0..2^31"); return QSIM_EINVAL; }
    if (shots == 0) return QSIM_OK;
    if ((size_t)shots > h->samples_cap) {
        cudaFree(h->dsamples);
        cudaFree(h->du);
        h->dsamples = nullptr;
        h->du = nullptr;
        h->samples_cap = 0;
        if (cudaMalloc(&h->dsamples, sizeof(uint64_t) * shots) != cudaSuccess ||
            cudaMalloc(&h->du, sizeof(double) * shots) != cudaSuccess) {
            cudaGetLastError();
            set_error("sample buffers");
            return QSIM_ENOMEM;
        }
        h->samples_cap = (size_t)shots;
    }
    cudaError_t e;
    if (u_host) e = cudaMemcpyAsync(h->du, u_host, sizeof(double) * shots, cudaMemcpyHostToDevice, h->stream);
    else e = launch_uniforms(seed, shots, h->du, h->stream);
    if (e == cudaSuccess)
        e = run_sample(h->dtype, h->psi, h->n, h->du, shots, h->dsamples, h->red, h->stream, h->dev, seg_ready_bits);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, h->dsamples, sizeof(uint64_t) * shots, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "sample");
    return check_device_error(h);
}

int qsim_sample(qsim_h h, uint64_t seed, int64_t shots, uint64_t* out) {
    QSIM_CHECK_HANDLE(h);
    return sample_common(h, shots, out, nullptr, seed);
}

int qsim_expect_z_and_sample(qsim_h h, double* zi, double* zz, uint64_t seed, int64_t shots, uint64_t* out) {
    QSIM_CHECK_HANDLE(h);
    if (!zi || (!zz && h->n > 1) || (!out && shots > 0)) { set_error("NULL output"); return QSIM_EINVAL; }
    if (shots < 0 || shots > (1ll << 31)) { set_error("shots outside 0..2^31"); return QSIM_EINVAL; }
    std::vector<double> zz_dummy(1);
    cudaError_t e = run_zstats(h->dtype, h->psi, h->n, h->red, h->stream, h->dev, zi, zz ? zz : zz_dummy.data());
    if (e != cudaSuccess) return cuda_fail(e, "expect_z_and_sample");
    const int rc = check_device_error(h);
    if (rc) return rc;
    return sample_common(h, shots, out, nullptr, seed, zstats_segment_bits(h->n));
}

int qsim_sample_uniforms(qsim_h h, const double* u, int64_t shots, uint64_t* out) {
    QSIM_CHECK_HANDLE(h);
    if (!u && shots > 0) { set_error("NULL uniforms"); return QSIM_EINVAL; }
    for (int64_t i = 0; i < shots; ++i)
        if (!(u[i] >= 0.0 && u[i] < 1.0)) { set_error("uniform %lld outside [0, 1)", (long long)i); return QSIM_EINVAL; }
    return sample_common(h, shots, out, u, 0);
}

int qsim_inner(qsim_h a, qsim_h b, double* out) {
    QSIM_CHECK_HANDLE(a);
    QSIM_CHECK_HANDLE(b);
    if (!out) { set_error("NULL output"); return QSIM_EINVAL; }
    if (a->n != b->n || a->dtype != b->dtype) { set_error("handles differ in n or dtype"); return QSIM_EINVAL; }
    if (a->stream != b->stream) {
        cudaError_t e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return cuda_fail(e, "inner: synchronising the second stream");
    }
    cudaError_t e = run_inner(a->dtype, a->psi, b->psi, a->n, a->red, a->stream, a->dev, out);
    if (e != cudaSuccess) return cuda_fail(e, "inner");
    return check_device_error(a);
}

}  // extern "C"
