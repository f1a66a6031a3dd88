// k_tc_peak.cu -- the dense tensor-core rate of this GPU, measured with a loop of MMAs and nothing else.
//
// The fused-block roofline needs the tensor rate of the exact MMA form the block kernels issue (A in tensor
// memory, B in shared memory in the SWIZZLE_128B K-major layout, M = 128, FP32 accumulation). Only the BF16
// rate of a library GEMM is known beforehand, and the TF32 / FP16 rates are not fixed multiples of it on
// every part, so this kernel measures them: every SM runs one CTA whose single issuing thread keeps the
// tensor core busy with back-to-back MMAs on resident operands (no global memory traffic), in chunks of
// 256 K-loops; at most two chunks are in flight, each tracked by a tcgen05.commit on its own mbarrier, so
// every wait is short and bounded (2 s; on expiry the kernel records DEVERR_TIMEOUT, waits once more for
// the MMAs it issued, frees its tensor memory and returns).
#include <algorithm>

#include "capi_state.h"
#include "common.cuh"
#include "internal.h"
#include "tc_ptx.cuh"

namespace qsim {
namespace tc {

constexpr int kPeakThreads = 128;  // four warps: one per TMEM lane quadrant to write A
constexpr int kPeakKSteps = 16;    // MMAs per K-loop: 512 bytes of K per row (4 SW128 atoms)
constexpr uint64_t kPeakChunk = 256;

// KIND: 0 = TF32 (kind::tf32), 1 = BF16, 2 = FP16 (kind::f16). N: 128 (the block kernels' shape) or 256.
template <int KIND, int N>
__global__ void __launch_bounds__(kPeakThreads, 1) k_tc_peak(uint64_t chunks, unsigned* __restrict__ err) {
    constexpr bool F16KIND = KIND != 0;
    constexpr int ATOM = N * 128;
    constexpr int BBYTES = 4 * ATOM;
    constexpr uint32_t FMT = KIND == 0 ? 2u : (KIND == 1 ? 1u : 0u);
    constexpr uint32_t IDESC = (1u << 4) | (FMT << 7) | (FMT << 10) | ((uint32_t)(N >> 3) << 17) |
                               ((uint32_t)(128 >> 4) << 24);
    constexpr uint32_t A0 = 256;  // A at TMEM columns [256, 384): K = 128 TF32 or 256 16-bit values per row
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sb = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sb + BBYTES);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // Operand values: finite numbers in [0.5, 1) of the operand type with pseudo-random mantissas and signs
    // (the tensor core's power, and so its clock, depends on the data it multiplies).
    auto word = [](uint32_t i) -> uint32_t {
        uint32_t h = i * 0x9E3779B9u;
        h ^= h >> 15;
        h *= 0x85EBCA6Bu;
        h ^= h >> 13;
        if constexpr (KIND == 0) return 0x3F000000u | (h & 0x807FE000u);
        else if constexpr (KIND == 1) return (0x3F003F00u | (h & 0x807F807Fu));
        else return (0x38003800u | (h & 0x83FF83FFu));
    };
    for (int i = tid; i < BBYTES / 4; i += kPeakThreads) reinterpret_cast<uint32_t*>(sb)[i] = word((uint32_t)i);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic-proxy writes -> tensor-core reads
    if (tid == 0) {
        for (int j = 0; j < 2; ++j)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(mbar + j)), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(tslot)), "r"(512) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tbase = *tslot;
    {
        const uint32_t tlane = (uint32_t)(warp * 32) << 16;
#pragma unroll 1
        for (int c = 0; c < 128; c += 16) {
            uint32_t v[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = word((uint32_t)(0x10000 + (warp * 32 + lane) * 128 + c + j));
            tmem_st_x16(tbase + tlane + A0 + (uint32_t)c, v);
        }
        wait_st();
    }
    fence_before();
    __syncthreads();
    fence_after();

    if (tid == 0) {
        const uint64_t desc0 = sdesc_sw128(smem_u32(sb));
        const uint32_t dlo0 = (uint32_t)desc0, dhi = (uint32_t)(desc0 >> 32);
        const uint32_t bar0 = smem_u32(mbar);
        bool bad = false;
        uint32_t acc = 0;
        for (uint64_t c = 0; c < chunks && !bad; ++c) {
#pragma unroll 1
            for (uint64_t it = 0; it < kPeakChunk; ++it) {
                uint32_t dlo = dlo0, tb = tbase;
                asm volatile("" : "+r"(dlo), "+r"(tb));
#pragma unroll
                for (int s = 0; s < kPeakKSteps; ++s) {
                    const uint32_t off = (uint32_t)((s >> 2) * ATOM + (s & 3) * 32);
                    mma_ts_lohi<F16KIND>(tb, tb + A0 + 8 * s, dlo + (off >> 4), dhi, IDESC, acc);
                    acc = 1;
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(bar0 + 8u * (uint32_t)(c & 1)) : "memory");
            if (c > 0 && !mbar_wait_bounded(bar0 + 8u * (uint32_t)((c - 1) & 1), (uint32_t)(((c - 1) >> 1) & 1)))
                bad = true;
        }
        if (chunks > 0) {
            const uint64_t l = chunks - 1;
            if (!mbar_wait_bounded(bar0 + 8u * (uint32_t)(l & 1), (uint32_t)((l >> 1) & 1))) {
                bad = true;
                mbar_wait_bounded(bar0 + 8u * (uint32_t)(l & 1), (uint32_t)((l >> 1) & 1));
            }
        }
        if (bad) atomicOr(err, DEVERR_TIMEOUT);
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tbase), "r"(512) : "memory");
    }
}

template <int KIND, int N>
cudaError_t launch_peak(uint64_t chunks, unsigned* err, int sms, cudaStream_t s) {
    // B operand + barriers + alignment, and at least 120 KiB so that one CTA (one TMEM owner) runs per SM
    const size_t smem = std::max<size_t>((size_t)4 * N * 128 + 64 + 1024, 120 * 1024);
    cudaError_t e = cudaFuncSetAttribute(k_tc_peak<KIND, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_tc_peak<KIND, N><<<sms, kPeakThreads, smem, s>>>(chunks, err);
    return cudaGetLastError();
}

cudaError_t launch_peak_any(int kind, int n_cols, uint64_t chunks, unsigned* err, int sms, cudaStream_t s) {
    switch (kind * 2 + (n_cols == 256 ? 1 : 0)) {
        case 0: return launch_peak<0, 128>(chunks, err, sms, s);
        case 1: return launch_peak<0, 256>(chunks, err, sms, s);
        case 2: return launch_peak<1, 128>(chunks, err, sms, s);
        case 3: return launch_peak<1, 256>(chunks, err, sms, s);
        case 4: return launch_peak<2, 128>(chunks, err, sms, s);
        default: return launch_peak<2, 256>(chunks, err, sms, s);
    }
}

}  // namespace tc
}  // namespace qsim

using namespace qsim;

extern "C" int qsim_tc_peak(int kind, int n_cols, double seconds, double* tflops, double* ms) {
    set_error("%s", "");
    if (kind < 0 || kind > 2) { set_error("kind %d: 0 = TF32, 1 = BF16, 2 = FP16", kind); return QSIM_EINVAL; }
    if (n_cols != 128 && n_cols != 256) { set_error("n_cols must be 128 or 256"); return QSIM_EINVAL; }
    if (!(seconds > 0.0 && seconds <= 30.0)) { set_error("seconds outside (0, 30]"); return QSIM_EINVAL; }
    if (!tflops) { set_error("NULL output"); return QSIM_EINVAL; }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "querying the device");
    unsigned* derr = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = QSIM_OK;
    auto done = [&](int r) {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (s) cudaStreamDestroy(s);
        if (derr) cudaFree(derr);
        return r;
    };
    if ((e = cudaMalloc(&derr, sizeof(unsigned))) != cudaSuccess) return done(cuda_fail(e, "error word"));
    if ((e = cudaMemset(derr, 0, sizeof(unsigned))) != cudaSuccess) return done(cuda_fail(e, "error word"));
    if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) return done(cuda_fail(e, "stream"));
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess)
        return done(cuda_fail(e, "events"));
    // flops of one chunk on one CTA: 256 K-loops x 16 MMAs x 2 M N K (K = 8 for TF32, 16 for 16-bit types)
    const double kmma = kind == 0 ? 8.0 : 16.0;
    const double chunk_flops = (double)tc::kPeakChunk * tc::kPeakKSteps * 2.0 * 128.0 * n_cols * kmma;
    auto timed = [&](uint64_t chunks, float* out_ms) -> int {
        cudaError_t x = cudaEventRecord(e0, s);
        if (x == cudaSuccess) x = tc::launch_peak_any(kind, n_cols, chunks, derr, sms, s);
        if (x == cudaSuccess) x = cudaEventRecord(e1, s);
        if (x == cudaSuccess) x = cudaStreamSynchronize(s);
        if (x == cudaSuccess) x = cudaEventElapsedTime(out_ms, e0, e1);
        if (x != cudaSuccess) return cuda_fail(x, "tensor-core rate probe");
        unsigned v = 0;
        if ((x = cudaMemcpy(&v, derr, sizeof(unsigned), cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(x, "error word");
        if (v) { set_error("a bounded wait of the rate probe expired (code 0x%x)", v); return QSIM_ETIMEOUT; }
        return QSIM_OK;
    };
    float t = 0.0f;
    // warm-up and calibration (~10 ms), then the measured run of the requested length
    if ((rc = timed(8, &t)) != QSIM_OK) return done(rc);
    if ((rc = timed(8, &t)) != QSIM_OK) return done(rc);
    const double per_chunk_ms = std::max(1e-6, (double)t / 8.0);
    const uint64_t chunks = (uint64_t)std::max(8.0, std::min(1e7, seconds * 1000.0 / per_chunk_ms));
    if ((rc = timed(chunks, &t)) != QSIM_OK) return done(rc);
    *tflops = chunk_flops * (double)chunks * sms / ((double)t * 1e-3) / 1e12;
    if (ms) *ms = t;
    return done(QSIM_OK);
}
