// k_noalloc.cu -- measurement sampling that allocates no device memory.
//
// Some callers cannot call cudaMalloc: a host framework that has reserved the GPU's memory up front in its
// own pool (a raw allocation would fail or fragment that pool), or a latency-critical path that cannot
// accept the implicit device synchronisation an allocation may cause. For them this entry point samples
// from a state they own, using only buffers they pass in plus one fixed scratch array that is part of the
// library image itself.
//
// The scratch is a file-scope __device__ array of kNoAllocBytes (8 MiB). Every GPU that loads libqsim holds
// it until the process exits. In host code the array's name is only a host-side stand-in, so its device
// address is looked up once per device with cudaGetSymbolAddress (with that device current) and cached.
// All calls share the array and it keeps the last call's contents: calls whose work overlaps on the GPU
// (different streams, or several host threads) race and must be serialised by the caller.
#include <mutex>

#include "capi_state.h"
#include "internal.h"

namespace {

constexpr size_t kNoAllocBytes = size_t(8) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch on the current device (looked up on the first call per device).
int noalloc_scratch(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return qsim::cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) {
        qsim::set_error("device %d beyond the %d devices this entry point tracks", dev, kMaxDevices);
        return QSIM_EUNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return qsim::cuda_fail(e, "cudaGetSymbolAddress of the sampling scratch");
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return QSIM_OK;
}

}  // namespace

extern "C" int qsim_sample_noalloc(const void* dev_state, int n, int dtype, uint64_t seed, int64_t shots,
                                   uint64_t* dev_out, void* stream) {
    using namespace qsim;
    set_error("%s", "");
    if (!dev_state || (!dev_out && shots > 0)) { set_error("NULL state or output"); return QSIM_EINVAL; }
    if (n < 1 || n > QSIM_MAX_QUBITS) { set_error("n = %d outside 1..%d", n, QSIM_MAX_QUBITS); return QSIM_EINVAL; }
    if (dtype != QSIM_C64 && dtype != QSIM_C128) { set_error("unknown dtype %d", dtype); return QSIM_EINVAL; }
    if (shots < 0) { set_error("negative number of shots"); return QSIM_EINVAL; }
    // Before any size arithmetic: a request for more shots than the scratch holds uniforms fails here, so
    // 8 * shots below cannot wrap around.
    if ((uint64_t)shots > kNoAllocBytes / 8) {
        set_error("%lld shots exceed the %zu uniforms the static scratch can hold", (long long)shots,
                  kNoAllocBytes / 8);
        return QSIM_EINVAL;
    }
    // The sampling kernels read the state with 16-byte vector loads and write 8-byte indices.
    if (reinterpret_cast<uintptr_t>(dev_state) & 255) {
        set_error("dev_state must be 256-byte aligned (as a state buffer given to qsim_create)");
        return QSIM_EINVAL;
    }
    if (reinterpret_cast<uintptr_t>(dev_out) & 7) { set_error("dev_out must be 8-byte aligned"); return QSIM_EINVAL; }
    if (shots == 0) return QSIM_OK;
    // Scratch layout: uniforms (shots doubles) | segment sums (nseg) | chunk prefix sums (nchunk), each
    // region 256-byte aligned.
    const int SB = n < kSegBits ? n : kSegBits;
    const uint64_t nseg = 1ull << (n - SB);
    const uint64_t nchunk = (nseg + 1023) / 1024;
    auto up = [](uint64_t bytes) { return (bytes + 255) & ~uint64_t(255); };
    const uint64_t need = up(8ull * (uint64_t)shots) + up(8ull * nseg) + up(8ull * nchunk);
    if (need > kNoAllocBytes) {
        set_error("sampling %lld shots from %d qubits needs %llu bytes of scratch (8 per shot plus 8 per 4096 "
                  "amplitudes); the static scratch holds %zu",
                  (long long)shots, n, (unsigned long long)need, kNoAllocBytes);
        return QSIM_EINVAL;
    }
    void* base = nullptr;
    int rc = noalloc_scratch(&base);
    if (rc) return rc;
    DevInfo d;
    cudaError_t e = cudaGetDevice(&d.device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, d.device);
    if (e != cudaSuccess) return cuda_fail(e, "querying the device");
    unsigned char* p = static_cast<unsigned char*>(base);
    double* u = reinterpret_cast<double*>(p);
    ReduceScratch r;
    r.seg = reinterpret_cast<double*>(p + up(8ull * (uint64_t)shots));
    r.scan = reinterpret_cast<double*>(p + up(8ull * (uint64_t)shots) + up(8ull * nseg));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // Every scratch word is written before it is read (uniforms, segment sums, chunk sums), so nothing needs
    // clearing between calls.
    e = launch_uniforms(seed, shots, u, s);
    if (e == cudaSuccess) e = run_sample(dtype, dev_state, n, u, shots, dev_out, r, s, d);
    return e == cudaSuccess ? QSIM_OK : cuda_fail(e, "sampling launch");
}
