// k_small.cu -- every pass of a small-state plan in ONE cooperative launch (paper Sec. 2.1 "State-Vector
// Simulation": the gates, or fused blocks, applied one after another to the state vector).
//
// For a state of up to 2^16 amplitudes a pass is a few microseconds of arithmetic (at 14 qubits and a
// complex128 state, a 4-qubit dense block is 2^14 x 64 FP64 FMAs, about 2 us at GB300's FP64 rate spread
// over every SM), so one launch per pass spends more time starting and draining kernels than computing. Here
// one CTA per SM stays resident over the whole plan and the passes are separated by a grid barrier: every
// CTA counts its arrival on a device word and waits until all have arrived (bounded: 2 s, then
// DEVERR_TIMEOUT and return). A cooperative launch guarantees that the CTAs are co-resident, so the barrier
// cannot wait on a CTA that has not started. The state stays in L2 (at most 1 MiB); loads of it bypass L1
// (.cg) so that a pass reads what other SMs wrote in the pass before.
//
// Each pass is described by a fixed-size record holding its matrix (dense U on k <= 5 targets with any
// controls, the non-unit entries of a diagonal on k <= 6 targets, or the terms of a phase pass), copied into
// shared memory one pass ahead (two buffers) so that the copy hides behind the barrier. Dense passes of up to
// 4 targets and diagonal passes do the arithmetic of the per-pass kernels (k_dense_small / k_dense_split and
// k_diag in k_gates.cu): the same FMA chains in the same order, so the two paths give identical states. A
// phase pass (any run of
// commuting 1- and 2-qubit diagonal gates: exp(i phi(x)) with phi a quadratic form of the index bits) sums
// its terms per amplitude in 64-bit fixed-point turns (exact, wrapping mod 2 pi) and takes one FP64
// sine/cosine of the sum. Work is spread warp by warp over the CTAs (warp w of the grid is warp w / G of CTA
// w mod G), so that a pass with a few hundred warps of work still occupies every SM's FP64 units.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>

#include "common.cuh"
#include "internal.h"

namespace qsim {
namespace small {

constexpr int kThreads = 256;
constexpr int kMaxDense = 5;   // dense targets
constexpr int kMaxDiag = 6;    // diagonal targets
constexpr int kMaxTerms = 1 + kSmallMaxQubits + kSmallMaxQubits * (kSmallMaxQubits - 1) / 2;  // phase terms
constexpr size_t kHeader = 256;  // the barrier word, padded
enum Kind { kDense = 0, kDiag = 1, kPhase = 2 };

template <typename R>
struct alignas(16) Pass {
    int32_t kind;                 // Kind
    int32_t k, nf, np;            // targets; fixed bits (targets + controls); diagonal entries / phase terms
    int32_t next16;               // 16-byte chunks of the next record that hold data (what is copied of it)
    int32_t pad[3];
    int32_t fixed[kMaxFixed];     // fixed bit positions, ascending
    uint64_t cmask;               // control bits, set in every group's base index
    uint64_t off[kMaxTerms];      // dense: offset of matrix index m; diagonal: offset of non-unit entry p;
                                  // phase: the index bits of term t (none, one or two)
    R m[2 << (2 * kMaxDense)];    // dense: U row-major (re, im); diagonal: the np factors (re, im); phase:
                                  // the terms' angles as 64-bit fixed-point turns (reinterpreted)
};
static_assert(sizeof(uint64_t) * kMaxTerms <= sizeof(float) * (2 << (2 * kMaxDense)), "phase terms fit");

__device__ __forceinline__ float fmar(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmar(double a, double b, double c) { return __fma_rn(a, b, c); }

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid barrier number `epoch` (1, 2, ...): the word counts arrivals and never resets within a launch; every
// CTA waits until it reaches epoch x G. False when the wait expired (the error word is set); the caller
// returns. (Measured on GB300: cheaper than a last-arrival flag on its own line, which needs the count back.)
__device__ __forceinline__ bool grid_sync(unsigned* bar, unsigned epoch, unsigned G, unsigned* err, int* s_stop) {
    __syncthreads();
    if (threadIdx.x == 0) {
        // release: this CTA's writes of the pass (ordered before this thread by the CTA barrier) are visible
        // to whoever acquires the count
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" :: "l"(bar) : "memory");
        const unsigned target = epoch * G;
        const uint64_t t0 = gtimer();
        int stop = 0;
        for (;;) {
            unsigned v;
            asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
            if ((int)(v - target) >= 0) break;
            if (gtimer() - t0 > 2000000000ull) {
                atomicOr(err, DEVERR_TIMEOUT);
                stop = 1;
                break;
            }
        }
        asm volatile("fence.acq_rel.gpu;" ::: "memory");  // acquire: the other CTAs' writes before our reads
        *s_stop = stop;
    }
    __syncthreads();
    return *s_stop == 0;
}

// The next pass's record (its first `chunks` 16-byte chunks: the header and the entries its kind uses), copied
// into shared memory by asynchronous copies (no registers, no wait): the copies run during this pass and are
// waited for just before the grid barrier.
template <typename R>
__device__ __forceinline__ void copy_pass(Pass<R>* dst, const Pass<R>* src, int chunks) {
    const char* s = reinterpret_cast<const char*>(src);
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    for (int i = threadIdx.x; i < chunks; i += kThreads)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(d + 16 * i), "l"(s + 16 * i) : "memory");
    asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void copy_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Dense pass: D lanes share a group (the fixed bits masked out of the index); every lane loads the group's D
// amplitudes (same-address loads are broadcast), the warp synchronises (all reads before any write: the update
// is in place), and lane r of the group computes and stores row r. Items are rounded up to whole warps so
// that every lane of a warp reaches the warp barrier.
template <typename R, int K>
__device__ __forceinline__ void dense_pass(typename Amp<R>::T* psi, int n, const Pass<R>& P, uint64_t first,
                                           uint64_t stride) {
    using T = typename Amp<R>::T;
    constexpr int D = 1 << K;
    const uint64_t items = (1ull << (n - P.nf)) << K;
    const uint64_t nit = (items + 31) & ~31ull;
    for (uint64_t it = first; it < nit; it += stride) {
        const bool act = it < items;
        const uint64_t base = insert_zeros(it >> K, P.fixed, P.nf) | P.cmask;
        T v[D];
        if (act) {
#pragma unroll
            for (int m = 0; m < D; ++m) v[m] = __ldcg(psi + base + P.off[m]);
        }
        __syncwarp();
        if (act) {
            const int r = (int)(it & (D - 1));
            R re = 0, im = 0;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const R ur = P.m[2 * (r * D + c)], ui = P.m[2 * (r * D + c) + 1];
                re = fmar(ur, v[c].x, re);
                re = fmar(-ui, v[c].y, re);
                im = fmar(ur, v[c].y, im);
                im = fmar(ui, v[c].x, im);
            }
            psi[base + P.off[r]] = make_amp<R>(re, im);
        }
    }
}

// Dense pass on 5 targets: a group is one warp; lane c loads amplitude c of the group and lane r computes
// row r, taking the other amplitudes from the lanes that hold them (shuffles, column order as above) rather
// than loading all 32 of them (which would take 128 registers a thread in complex128). U is stored column-major
// for this width, so that the lanes read consecutive entries. A lane's store follows shuffles that need every
// lane's load, so all reads precede all writes without a warp barrier.
template <typename R>
__device__ __forceinline__ void dense_pass5(typename Amp<R>::T* psi, int n, const Pass<R>& P, uint64_t first,
                                            uint64_t stride) {
    using T = typename Amp<R>::T;
    constexpr int D = 32;
    const uint64_t items = (1ull << (n - P.nf)) << 5;  // whole warps
    for (uint64_t it = first; it < items; it += stride) {
        const uint64_t base = insert_zeros(it >> 5, P.fixed, P.nf) | P.cmask;
        const int r = (int)(it & 31);  // this lane
        const T v = __ldcg(psi + base + P.off[r]);
        R re = 0, im = 0;
#pragma unroll 8
        for (int c = 0; c < D; ++c) {
            const R vx = __shfl_sync(0xffffffffu, v.x, c), vy = __shfl_sync(0xffffffffu, v.y, c);
            const R ur = P.m[2 * (c * D + r)], ui = P.m[2 * (c * D + r) + 1];
            re = fmar(ur, vx, re);
            re = fmar(-ui, vy, re);
            im = fmar(ur, vy, im);
            im = fmar(ui, vx, im);
        }
        psi[base + P.off[r]] = make_amp<R>(re, im);
    }
}

// Diagonal pass: one group per item; the non-unit entries of the diagonal multiply their amplitudes.
template <typename R>
__device__ __forceinline__ void diag_pass(typename Amp<R>::T* psi, int n, const Pass<R>& P, uint64_t first,
                                          uint64_t stride) {
    using T = typename Amp<R>::T;
    const uint64_t items = 1ull << (n - P.nf);
    for (uint64_t it = first; it < items; it += stride) {
        const uint64_t base = insert_zeros(it, P.fixed, P.nf) | P.cmask;
        for (int p = 0; p < P.np; ++p) {
            const R dr = P.m[2 * p], di = P.m[2 * p + 1];
            T* q = psi + base + P.off[p];
            const T v = __ldcg(q);
            *q = make_amp<R>(fmar(dr, v.x, -di * v.y), fmar(dr, v.y, di * v.x));
        }
    }
}

// Phase pass: every amplitude x times exp(i phi(x)), phi(x) = the sum of the terms whose index bits are all set
// in x (64-bit fixed-point turns: the sum wraps exactly at one turn).
template <typename R>
__device__ __forceinline__ void phase_pass(typename Amp<R>::T* psi, int n, const Pass<R>& P, uint64_t first,
                                           uint64_t stride) {
    using T = typename Amp<R>::T;
    const uint64_t N = 1ull << n;
    const uint64_t* turn = reinterpret_cast<const uint64_t*>(P.m);
    for (uint64_t i = first; i < N; i += stride) {
        uint64_t acc = 0;
        for (int t = 0; t < P.np; ++t) acc += (i & P.off[t]) == P.off[t] ? turn[t] : 0ull;
        double sn, cs;
        sincospi((double)(int64_t)acc * 0x1p-63, &sn, &cs);  // angle 2 pi acc / 2^64, taken in [-pi, pi)
        const R c = (R)cs, s = (R)sn;
        const T v = __ldcg(psi + i);
        psi[i] = make_amp<R>(fmar(c, v.x, -s * v.y), fmar(c, v.y, s * v.x));
    }
}

template <typename R>
__global__ void __launch_bounds__(kThreads)
k_small_run(typename Amp<R>::T* __restrict__ psi, int n, const Pass<R>* __restrict__ prog, int npass,
            unsigned* bar, unsigned* err, int from_basis, uint64_t basis) {
    __shared__ Pass<R> sp[2];
    __shared__ int s_stop;
    const unsigned G = gridDim.x;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    // warp w of the grid = warp w / G of CTA w mod G
    const uint64_t first = ((uint64_t)wib * G + blockIdx.x) * 32 + lane;
    const uint64_t stride = (uint64_t)G * kThreads;
    unsigned epoch = 0;
    auto sync = [&]() -> bool { ++epoch; return grid_sync(bar, epoch, G, err, &s_stop); };

    if (npass > 0) {
        copy_pass(&sp[0], prog, (int)(sizeof(Pass<R>) / 16));
        copy_wait();
    }
    if (from_basis) {
        const uint64_t N = 1ull << n;
        for (uint64_t i = first; i < N; i += stride) psi[i] = make_amp<R>(i == basis ? R(1) : R(0), R(0));
        if (npass > 0 && !sync()) return;
    } else {
        __syncthreads();
    }
    for (int p = 0; p < npass; ++p) {
        const Pass<R>& P = sp[p & 1];
        // the other buffer was last read in pass p - 1, which every thread of this CTA has finished
        if (p + 1 < npass) copy_pass(&sp[(p + 1) & 1], prog + p + 1, P.next16);
        if (P.kind == kDiag) {
            diag_pass<R>(psi, n, P, first, stride);
        } else if (P.kind == kPhase) {
            phase_pass<R>(psi, n, P, first, stride);
        } else {
            switch (P.k) {
                case 1: dense_pass<R, 1>(psi, n, P, first, stride); break;
                case 2: dense_pass<R, 2>(psi, n, P, first, stride); break;
                case 3: dense_pass<R, 3>(psi, n, P, first, stride); break;
                case 4: dense_pass<R, 4>(psi, n, P, first, stride); break;
                default: dense_pass5<R>(psi, n, P, first, stride); break;
            }
        }
        if (p + 1 < npass) {
            copy_wait();  // the next record is in shared memory before the barrier (which orders it for all)
            if (!sync()) return;
        }
    }
}

// An angle in radians as 64-bit fixed-point turns (2^64 = one turn).
inline uint64_t fixed_turns(double rad) {
    double t = rad / (2.0 * 3.14159265358979323846);
    t -= std::floor(t);                   // [0, 1)
    const double v = std::ldexp(t, 64);   // [0, 2^64]
    return v >= 18446744073709551616.0 ? 0ull : (uint64_t)v;
}

template <typename R>
bool build_t(const std::vector<SmallOpDesc>& ops, unsigned char* out) {
    std::memset(out, 0, kHeader + sizeof(Pass<R>) * ops.size());
    Pass<R>* P = reinterpret_cast<Pass<R>*>(out + kHeader);
    for (size_t i = 0; i < ops.size(); ++i) {
        const SmallOpDesc& o = ops[i];
        Pass<R>& q = P[i];
        if (o.form) {  // phase pass: the constant, one term per qubit, one per pair
            q.kind = kPhase;
            uint64_t* turn = reinterpret_cast<uint64_t*>(q.m);
            auto add = [&](uint64_t mask, double rad) {
                if (q.np >= kMaxTerms) return false;
                q.off[q.np] = mask;
                turn[q.np++] = fixed_turns(rad);
                return true;
            };
            if (!add(0, o.form->c)) return false;
            for (size_t a = 0; a < o.form->h.size(); ++a)
                if (o.form->h[a] != 0.0 && (a >= 64 || !add(1ull << a, o.form->h[a]))) return false;
            for (const PhaseForm::Pair& pr : o.form->pairs)
                if (pr.a < 0 || pr.b < 0 || pr.a >= 64 || pr.b >= 64 || !add((1ull << pr.a) | (1ull << pr.b), pr.lam))
                    return false;
            continue;
        }
        if (o.k < 1 || o.nc < 0 || o.k + o.nc > kMaxFixed || (o.diag ? o.k > kMaxDiag : o.k > kMaxDense)) return false;
        q.kind = o.diag ? kDiag : kDense;
        q.k = o.k;
        q.nf = o.k + o.nc;
        for (int j = 0; j < o.k; ++j) q.fixed[j] = o.targets[j];
        for (int j = 0; j < o.nc; ++j) {
            q.fixed[o.k + j] = o.controls[j];
            q.cmask |= 1ull << o.controls[j];
        }
        std::sort(q.fixed, q.fixed + q.nf);
        auto offset = [&](int m) {
            uint64_t off = 0;
            for (int j = 0; j < o.k; ++j) off |= (uint64_t)((m >> j) & 1) << o.targets[j];
            return off;
        };
        if (o.diag) {
            if (!o.touch || o.touch->size() > 64) return false;
            q.np = (int)o.touch->size();
            for (int p = 0; p < q.np; ++p) {
                const int m = (*o.touch)[p];
                q.off[p] = offset(m);
                q.m[2 * p] = (R)o.mat[2 * m];
                q.m[2 * p + 1] = (R)o.mat[2 * m + 1];
            }
        } else {
            const int D = 1 << o.k;
            for (int m = 0; m < D; ++m) q.off[m] = offset(m);
            if (o.k == 5) {  // column-major (dense_pass5)
                for (int r = 0; r < D; ++r)
                    for (int c = 0; c < D; ++c) {
                        q.m[2 * (c * D + r)] = (R)o.mat[2 * (r * D + c)];
                        q.m[2 * (c * D + r) + 1] = (R)o.mat[2 * (r * D + c) + 1];
                    }
            } else {
                for (int e = 0; e < 2 * D * D; ++e) q.m[e] = (R)o.mat[e];
            }
        }
    }
    // what the kernel copies of each record: the header and offsets, and the entries of m its kind uses
    auto chunks = [](const Pass<R>& q) {
        size_t mb = q.kind == kPhase ? sizeof(uint64_t) * q.np
                    : q.kind == kDiag ? sizeof(R) * 2 * q.np
                                      : sizeof(R) * ((size_t)2 << (2 * q.k));
        return (int)((offsetof(Pass<R>, m) + mb + 15) / 16);
    };
    for (size_t i = 0; i + 1 < ops.size(); ++i) P[i].next16 = chunks(P[i + 1]);
    return true;
}

template <typename R>
cudaError_t run_t(void* psi, int n, void* dprog, int npass, unsigned* dev_err, cudaStream_t s, const DevInfo& d,
                  const uint64_t* from_basis) {
    auto kern = k_small_run<R>;
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, 0);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const unsigned grid = (unsigned)std::max(1, d.num_sms);  // one CTA per SM (co-resident: occ >= 1)
    if ((uint64_t)(npass + 1) * grid >= (1ull << 31)) return cudaErrorInvalidValue;
    unsigned* bar = static_cast<unsigned*>(dprog);
    e = cudaMemsetAsync(bar, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    using T = typename Amp<R>::T;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<T*>(psi), n,
                              reinterpret_cast<const Pass<R>*>(static_cast<char*>(dprog) + kHeader), npass, bar,
                              dev_err, from_basis ? 1 : 0, from_basis ? *from_basis : (uint64_t)0);
}

}  // namespace small

size_t small_program_bytes(int dtype, int npass) {
    const size_t rec = dtype == QSIM_C64 ? sizeof(small::Pass<float>) : sizeof(small::Pass<double>);
    return small::kHeader + rec * (size_t)npass;
}

bool small_program_build(int dtype, const std::vector<SmallOpDesc>& ops, unsigned char* out) {
    return dtype == QSIM_C64 ? small::build_t<float>(ops, out) : small::build_t<double>(ops, out);
}

cudaError_t launch_small_run(int dtype, void* psi, int n, void* dprog, int npass, unsigned* dev_err, cudaStream_t s,
                             const DevInfo& d, const uint64_t* from_basis) {
    if (n < 1 || n > kSmallMaxQubits || npass < 0 || !dev_err || (reinterpret_cast<uintptr_t>(dprog) & 15) != 0)
        return cudaErrorInvalidValue;
    return dtype == QSIM_C64 ? small::run_t<float>(psi, n, dprog, npass, dev_err, s, d, from_basis)
                             : small::run_t<double>(psi, n, dprog, npass, dev_err, s, d, from_basis);
}

// ---- FP64 rate probe: the denominator of the small-state runner's roofline -----------------------------------
namespace small {

constexpr int kPeakChains = 8;      // independent FMA chains per thread
constexpr int kPeakUnroll = 64;     // FMAs per chain per loop iteration

// Every thread runs kPeakChains independent FP64 FMA chains for `iters` iterations; the result is stored only
// if it equals a value it cannot take, so the chains are not removed.
__global__ void __launch_bounds__(kThreads) k_fp64_peak(uint64_t iters, double seed, double* sink) {
    double a[kPeakChains];
#pragma unroll
    for (int j = 0; j < kPeakChains; ++j) a[j] = seed + threadIdx.x * 1e-9 + j * 1e-7;
    const double m = 0.999999, c = 1e-9;
    for (uint64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kPeakUnroll; ++u)
#pragma unroll
            for (int j = 0; j < kPeakChains; ++j) a[j] = __fma_rn(a[j], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kPeakChains; ++j) s += a[j];
    if (s == -1.0) *sink = s;
}

}  // namespace small
}  // namespace qsim

extern "C" int qsim_fp64_peak(double seconds, double* tflops, double* ms) {
    using namespace qsim;
    set_error("%s", "");
    if (!(seconds > 0.0 && seconds <= 30.0)) { set_error("seconds outside (0, 30]"); return QSIM_EINVAL; }
    if (!tflops) { set_error("NULL output"); return QSIM_EINVAL; }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "querying the device");
    double* sink = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto done = [&](int r) {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (s) cudaStreamDestroy(s);
        if (sink) cudaFree(sink);
        return r;
    };
    if ((e = cudaMalloc(&sink, sizeof(double))) != cudaSuccess) return done(cuda_fail(e, "probe output"));
    if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) return done(cuda_fail(e, "stream"));
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess)
        return done(cuda_fail(e, "events"));
    const unsigned grid = (unsigned)sms * 4;  // 32 warps per SM
    auto timed = [&](uint64_t iters, float* out_ms) -> int {
        cudaError_t x = cudaEventRecord(e0, s);
        if (x == cudaSuccess) {
            small::k_fp64_peak<<<grid, small::kThreads, 0, s>>>(iters, 1.0, sink);
            x = cudaGetLastError();
        }
        if (x == cudaSuccess) x = cudaEventRecord(e1, s);
        if (x == cudaSuccess) x = cudaStreamSynchronize(s);
        if (x == cudaSuccess) x = cudaEventElapsedTime(out_ms, e0, e1);
        return x == cudaSuccess ? QSIM_OK : cuda_fail(x, "FP64 rate probe");
    };
    float t = 0.0f;
    int rc;
    if ((rc = timed(16, &t)) != QSIM_OK) return done(rc);  // warm-up
    if ((rc = timed(16, &t)) != QSIM_OK) return done(rc);
    const double per_iter_ms = std::max(1e-6, (double)t / 16.0);
    const uint64_t iters = (uint64_t)std::max(16.0, std::min(1e8, seconds * 1000.0 / per_iter_ms));
    if ((rc = timed(iters, &t)) != QSIM_OK) return done(rc);
    const double flops = 2.0 * small::kPeakChains * small::kPeakUnroll * (double)iters * grid * small::kThreads;
    *tflops = flops / ((double)t * 1e-3) / 1e12;
    if (ms) *ms = t;
    return done(QSIM_OK);
}
