// k_reduce.cu -- readout of the state (paper Sec. 2.1 "Measurement and Sampling"; Sec. 2.5: sampling and
// expectation values): norm, marginal probabilities, Pauli-string expectations, the Z / ZZ correlators of
// a chain in one pass, overlaps, and inverse-CDF sampling without materialising the 2^n CDF.
//
// Precision: each thread accumulates exact |a|^2 (or exact products) in float-float (~48 bits, FP32 ops);
// warps reduce in float-float; per-block partials are combined in double-double (FP64 TwoSum). GB300's FP64
// rate is far below its FP32 rate, so FP64 is kept off the per-amplitude path. complex128 states use
// double-double throughout.
#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace qsim {

// ---- accumulator traits -----------------------------------------------------------------------------------
template <typename R> struct Acc;
template <> struct Acc<float> {
    using A = ff;
    __device__ static A zero() { return {0.f, 0.f}; }
    __device__ static A abs2(float re, float im) { return ff_abs2(re, im); }
    __device__ static A prod(float x, float y) { return two_prod(x, y); }
    __device__ static A add(A a, A b) { return ff_add(a, b); }
    __device__ static A neg(A a) { return ff_neg(a); }
    __device__ static A warp_sum(A a) { return warp_sum_ff(a); }
    __device__ static dd to_dd(A a) { return {(double)a.hi + (double)a.lo, 0.0}; }
};
__device__ __forceinline__ dd two_prod_d(double x, double y) {
    double p = __dmul_rn(x, y);
    return {p, __fma_rn(x, y, -p)};
}
template <> struct Acc<double> {
    using A = dd;
    __device__ static A zero() { return {0.0, 0.0}; }
    __device__ static A abs2(double re, double im) { return dd_add(two_prod_d(re, re), two_prod_d(im, im)); }
    __device__ static A prod(double x, double y) { return two_prod_d(x, y); }
    __device__ static A add(A a, A b) { return dd_add(a, b); }
    __device__ static A neg(A a) { return {-a.hi, -a.lo}; }
    __device__ static A warp_sum(A a) { return warp_sum_dd(a); }
    __device__ static dd to_dd(A a) { return a; }
};

// Sum of one dd value per thread over the block; result valid in thread 0. `sm` holds >= 32 dd.
__device__ dd block_sum_dd(dd v, dd* sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum_dd(v);
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    dd r = {0.0, 0.0};
    if (warp == 0) {
        r = lane < nw ? sm[lane] : dd{0.0, 0.0};
        r = warp_sum_dd(r);
    }
    __syncthreads();
    return r;
}

template <typename R>
__device__ dd block_sum_acc(typename Acc<R>::A v, dd* sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = Acc<R>::warp_sum(v);
    if (lane == 0) sm[warp] = Acc<R>::to_dd(v);
    __syncthreads();
    dd r = {0.0, 0.0};
    if (warp == 0) {
        r = lane < nw ? sm[lane] : dd{0.0, 0.0};
        r = warp_sum_dd(r);
    }
    __syncthreads();
    return r;
}

// partials layout: quantity q, block b -> partials[2 * (q * nblocks + b)] (hi, lo).
__global__ void __launch_bounds__(256) k_final_dd(const double* __restrict__ partials, int nblocks, double* __restrict__ out) {
    __shared__ dd sm[32];
    const int q = blockIdx.x;
    dd acc = {0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        const double* p = partials + 2 * ((int64_t)q * nblocks + b);
        acc = dd_add(acc, dd{p[0], p[1]});
    }
    acc = block_sum_dd(acc, sm);
    if (threadIdx.x == 0) {
        out[2 * q] = acc.hi;
        out[2 * q + 1] = acc.lo;
    }
}

// Amplitudes 2i and 2i+1 as float-float |a|^2 values (one 16-byte load for complex64).
template <typename R>
__device__ __forceinline__ void load_p2(const typename Amp<R>::T* psi, uint64_t i, ff& p0, ff& p1) {
    if constexpr (sizeof(R) == 4) {
        const float4 v = reinterpret_cast<const float4*>(psi)[i];
        p0 = ff_abs2(v.x, v.y);
        p1 = ff_abs2(v.z, v.w);
    } else {
        const double2 a = psi[2 * i], b = psi[2 * i + 1];
        const dd qa = Acc<double>::abs2(a.x, a.y), qb = Acc<double>::abs2(b.x, b.y);
        const float ha = (float)qa.hi, hb = (float)qb.hi;
        p0 = {ha, (float)(qa.hi - (double)ha + qa.lo)};
        p1 = {hb, (float)(qb.hi - (double)hb + qb.lo)};
    }
}

// Sum of N float-float values as a pairwise tree (depth log2 N instead of a serial chain of N adds).
template <int N>
__device__ __forceinline__ ff ff_tree_sum(ff (&q)[N]) {
#pragma unroll
    for (int w = N / 2; w >= 1; w >>= 1) {
#pragma unroll
        for (int i = 0; i < w; ++i) q[i] = ff_add(q[i], q[i + w]);
    }
    return q[0];
}

// ============================================================================================================
// Norm and overlap
// ============================================================================================================
// sum |a|^2 over npairs amplitude pairs. Each block reads one contiguous slice of the state (so the blocks
// in flight spread over the whole vector rather than sweeping it as one narrow window), eight independent
// 16-byte loads in flight per thread, summed as a tree.
template <typename R>
__global__ void __launch_bounds__(256) k_norm_pairs(const typename Amp<R>::T* __restrict__ psi, uint64_t npairs,
                                                    double* partials) {
    __shared__ dd sm[32];
    ff acc = {0.f, 0.f};
    const uint64_t per = (npairs + gridDim.x - 1) / gridDim.x;
    const uint64_t lo = (uint64_t)blockIdx.x * per, hi = min(npairs, lo + per);
    for (uint64_t i = lo + threadIdx.x; i < hi; i += 4 * blockDim.x) {
        ff q[8];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint64_t k = i + u * blockDim.x;
            if (k < hi) load_p2<R>(psi, k, q[2 * u], q[2 * u + 1]);
            else q[2 * u] = q[2 * u + 1] = ff{0.f, 0.f};
        }
        acc = ff_add(acc, ff_tree_sum(q));
    }
    const dd r = block_sum_acc<float>(acc, sm);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = r.hi;
        partials[2 * blockIdx.x + 1] = r.lo;
    }
}

// <a|b> = sum conj(a_x) b_x: quantity 0 = real part, 1 = imaginary part.
template <typename R>
__global__ void __launch_bounds__(256) k_inner_partial(const typename Amp<R>::T* __restrict__ a,
                                                       const typename Amp<R>::T* __restrict__ b, uint64_t N,
                                                       double* partials) {
    __shared__ dd sm[32];
    using A = typename Acc<R>::A;
    A re = Acc<R>::zero(), im = Acc<R>::zero();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        const auto x = a[i];
        const auto y = b[i];
        re = Acc<R>::add(re, Acc<R>::add(Acc<R>::prod(x.x, y.x), Acc<R>::prod(x.y, y.y)));
        im = Acc<R>::add(im, Acc<R>::add(Acc<R>::prod(x.x, y.y), Acc<R>::neg(Acc<R>::prod(x.y, y.x))));
    }
    const dd r0 = block_sum_acc<R>(re, sm);
    const dd r1 = block_sum_acc<R>(im, sm);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = r0.hi;
        partials[2 * blockIdx.x + 1] = r0.lo;
        partials[2 * (gridDim.x + blockIdx.x)] = r1.hi;
        partials[2 * (gridDim.x + blockIdx.x) + 1] = r1.lo;
    }
}

// ============================================================================================================
// Pauli strings: <P> = i^{nY} sum_x s(x) conj(psi_{x^f}) psi_x, s(x) = (-1)^{popcount(x & (Y|Z mask))}.
// With f != 0, x and x^f are visited together (x has the top flip bit h clear), so every amplitude is read
// once: their two terms are s(x) w + s(x^f) conj(w), w = conj(psi_{x^f}) psi_x.
// ============================================================================================================
template <typename R>
__global__ void __launch_bounds__(256) k_pauli_partial(const typename Amp<R>::T* __restrict__ psi, int n, uint64_t fmask,
                                                       uint64_t smask, int h, double* partials) {
    __shared__ dd sm[32];
    using A = typename Acc<R>::A;
    A sre = Acc<R>::zero(), sim = Acc<R>::zero();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    if (fmask == 0) {
        const uint64_t N = 1ull << n;
        for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < N; x += stride) {
            const auto a = psi[x];
            A p = Acc<R>::abs2(a.x, a.y);
            if (__popcll(x & smask) & 1) p = Acc<R>::neg(p);
            sre = Acc<R>::add(sre, p);
        }
    } else {
        const uint64_t G = 1ull << (n - 1);
        for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < G; g += stride) {
            const uint64_t x = insert_zero(g, h), y = x ^ fmask;
            const auto a = psi[x];
            const auto b = psi[y];
            // w = conj(b) a
            A wr = Acc<R>::add(Acc<R>::prod(b.x, a.x), Acc<R>::prod(b.y, a.y));
            A wi = Acc<R>::add(Acc<R>::prod(b.x, a.y), Acc<R>::neg(Acc<R>::prod(b.y, a.x)));
            const bool sx = __popcll(x & smask) & 1, sy = __popcll(y & smask) & 1;
            // s(x) w + s(y) conj(w): real = (s(x)+s(y)) wr, imag = (s(x)-s(y)) wi
            if (sx == sy) {
                A t = Acc<R>::add(wr, wr);
                sre = Acc<R>::add(sre, sx ? Acc<R>::neg(t) : t);
            } else {
                A t = Acc<R>::add(wi, wi);
                sim = Acc<R>::add(sim, sx ? Acc<R>::neg(t) : t);
            }
        }
    }
    const dd r0 = block_sum_acc<R>(sre, sm);
    const dd r1 = block_sum_acc<R>(sim, sm);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = r0.hi;
        partials[2 * blockIdx.x + 1] = r0.lo;
        partials[2 * (gridDim.x + blockIdx.x)] = r1.hi;
        partials[2 * (gridDim.x + blockIdx.x) + 1] = r1.lo;
    }
}

// ============================================================================================================
// Marginal probabilities
// ============================================================================================================
struct ProbsArgs {
    int nq;
};

// Marginals for n >= 12, every nq (1..30), in one pass at close to the norm's cost. Warp segments of 1024
// amplitudes: lane l holds amplitudes 2 (32 j + l) + h of a segment (h = bit 0, l = bits 1..5, j = bits 6..9).
// A work item is a bin group (the marginal bits >= 10 fixed: mh) and one of S chunks of the segments that
// differ only in non-marginal bits >= 10. WPI warps share an item and stride over its segments, each lane
// adding |a|^2 into registers indexed by (h, j) -- 16 float-float values, 32 when qubit 0 is marginal --
// regardless of the marginal set. Only at the end of the item are the non-marginal bits among 0..9 folded
// (register pairs for bits 6..9, lane shuffles for bits 1..5), the item's warps merged into shared-memory
// bins, and its 2^nlow sums written: final values (S = 1) or per-chunk partials for k_probs_warp_final.
struct ProbsWArgs {
    int nlow;            // marginal bits among 0..9
    int lowj[10];        // user index j of the r-th smallest of them
    uint32_t lowmask;    // their positions, as a mask over bits 0..9
    int nhigh;
    int highpos[32];     // marginal positions >= 10, ascending
    int highj[32];       // their user index j
    int nfh;
    int fhpos[32];       // non-marginal positions >= 10, ascending
    uint64_t S;          // chunks per bin group (a power of two dividing 2^nfh)
    uint64_t nitems;     // 2^nhigh * S
    int wpi;             // warps per item (a power of two, <= warps per block)
};

__device__ __forceinline__ uint64_t probs_bin(const ProbsWArgs& a, uint64_t i, uint64_t mh) {
    uint64_t m = 0;
    for (int r = 0; r < a.nlow; ++r) m |= ((i >> r) & 1) << a.lowj[r];
    for (int j = 0; j < a.nhigh; ++j) m |= ((mh >> j) & 1) << a.highj[j];
    return m;
}

template <typename R, bool M0>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 2 : 1) k_probs_warp(const typename Amp<R>::T* __restrict__ psi,
                                                       const __grid_constant__ ProbsWArgs a,
                                                       double* __restrict__ partials, double* __restrict__ out) {
    constexpr int NV = M0 ? 32 : 16;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ff* bins = reinterpret_cast<ff*>(smem_raw);  // [items per block][2^nlow]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int ipb = nwarps / a.wpi;               // items per block
    const int sub = warp % a.wpi, slot = warp / a.wpi;
    const int NL = 1 << a.nlow;
    const uint64_t per = (1ull << a.nfh) / a.S;
    for (uint64_t it0 = (uint64_t)blockIdx.x * ipb; it0 < a.nitems; it0 += (uint64_t)gridDim.x * ipb) {
        const uint64_t it = it0 + slot;
        const bool active = it < a.nitems;
        const uint64_t mh = active ? it / a.S : 0, sc = active ? it % a.S : 0;
        uint64_t hbits = 0;  // segment-index bits (position - 10)
        for (int j = 0; j < a.nhigh; ++j) hbits |= ((mh >> j) & 1) << (a.highpos[j] - 10);
        ff v[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] = {0.f, 0.f};
        if (active) {
            for (uint64_t f = sc * per + sub; f < (sc + 1) * per; f += a.wpi) {
                uint64_t sidx = hbits;
                for (int j = 0; j < a.nfh; ++j) sidx |= ((f >> j) & 1) << (a.fhpos[j] - 10);
                const uint64_t base = sidx * 512 + lane;  // amplitude-pair index
                constexpr int NB = M0 ? 4 : 8;  // loads per batch (registers: NV accumulators + 4 NB values)
#pragma unroll
                for (int hh = 0; hh < 16 / NB; ++hh) {
                    ff p[NB], q[NB];
#pragma unroll
                    for (int j = 0; j < NB; ++j) load_p2<R>(psi, base + 32 * (NB * hh + j), p[j], q[j]);
#pragma unroll
                    for (int j = 0; j < NB; ++j) {
                        if constexpr (M0) {
                            v[NB * hh + j] = ff_add(v[NB * hh + j], p[j]);
                            v[16 + NB * hh + j] = ff_add(v[16 + NB * hh + j], q[j]);
                        } else {
                            v[NB * hh + j] = ff_add(v[NB * hh + j], ff_add(p[j], q[j]));
                        }
                    }
                }
            }
        }
        // fold the non-marginal bits 6..9 (register index bits), then 1..5 (lane bits)
#pragma unroll
        for (int bb = 0; bb < 4; ++bb) {
            if (!((a.lowmask >> (6 + bb)) & 1)) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    if ((j >> bb) & 1) continue;
                    v[j] = ff_add(v[j], v[j | (1 << bb)]);
                    if constexpr (M0) v[16 + j] = ff_add(v[16 + j], v[16 + (j | (1 << bb))]);
                }
            }
        }
#pragma unroll
        for (int b = 0; b < 5; ++b) {
            if (!((a.lowmask >> (1 + b)) & 1)) {
#pragma unroll
                for (int k = 0; k < NV; ++k) v[k] = ff_add(v[k], shfl_xor_ff(v[k], 1 << b));
            }
        }
        // merge the item's warps into its bins (index = the marginal bits among 0..9, in position order)
        ff* mybins = bins + (size_t)slot * NL;
        for (int i = threadIdx.x; i < ipb * NL; i += blockDim.x) bins[i] = {0.f, 0.f};
        __syncthreads();
        const uint32_t lbits = (uint32_t)lane << 1;
        for (int r = 0; r < a.wpi; ++r) {
            if (sub == r && active && (lbits & ~a.lowmask & 0x3Eu) == 0) {
#pragma unroll
                for (int k = 0; k < NV; ++k) {
                    const uint32_t x = ((uint32_t)(k & 15) << 6) | lbits | (uint32_t)(k >> 4);
                    if ((x & ~a.lowmask & 0x3C0u) != 0) continue;  // a register folded into another
                    int idx = 0, o = 0;
                    for (int b = 0; b < 10; ++b)
                        if ((a.lowmask >> b) & 1) { idx |= (int)((x >> b) & 1) << o; ++o; }
                    mybins[idx] = ff_add(mybins[idx], v[k]);
                }
            }
            __syncthreads();
        }
        for (int i = threadIdx.x; i < ipb * NL; i += blockDim.x) {
            const uint64_t its = it0 + (uint64_t)(i / NL);
            if (its >= a.nitems) continue;
            const uint64_t mhs = its / a.S, scs = its % a.S, bi = (uint64_t)(i % NL);
            const double val = (double)bins[i].hi + (double)bins[i].lo;
            if (a.S == 1) out[probs_bin(a, bi, mhs)] = val;
            else partials[((mhs << a.nlow) + bi) * a.S + scs] = val;
        }
        __syncthreads();  // the bins are reused by the next items
    }
}

__global__ void __launch_bounds__(256) k_probs_warp_final(const double* __restrict__ partials,
                                                          const __grid_constant__ ProbsWArgs a,
                                                          double* __restrict__ out) {
    const uint64_t NL = 1ull << a.nlow, nbins = NL << a.nhigh;
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < nbins; p += (uint64_t)gridDim.x * blockDim.x) {
        dd acc = {0.0, 0.0};
        for (uint64_t sc = 0; sc < a.S; ++sc) acc = dd_add(acc, dd{partials[p * a.S + sc], 0.0});
        out[probs_bin(a, p % NL, p / NL)] = acc.hi + acc.lo;
    }
}

// Small states (n < 12): one CTA; out[m] directly (dd), each bin summing its 2^(n-nq) amplitudes.
template <typename R>
__global__ void __launch_bounds__(256) k_probs_small(const typename Amp<R>::T* __restrict__ psi, int n,
                                                     const __grid_constant__ ProbsArgs a, const int* __restrict__ qpos,
                                                     double* out) {
    // qpos: the nq marginal positions (user order) followed by the n-nq other positions, ascending.
    const int nq = a.nq;
    const int NB = 1 << nq, nr = n - nq;
    for (int m = threadIdx.x; m < NB; m += blockDim.x) {
        uint64_t fixedbits = 0;
        for (int j = 0; j < nq; ++j) fixedbits |= (uint64_t)((m >> j) & 1) << qpos[j];
        dd acc = {0.0, 0.0};
        for (uint64_t r = 0; r < (1ull << nr); ++r) {
            const uint64_t x = fixedbits | deposit(r, qpos + nq, nr);
            const auto v = psi[x];
            acc = dd_add(acc, Acc<double>::abs2((double)v.x, (double)v.y));
        }
        out[2 * m] = acc.hi;
        out[2 * m + 1] = acc.lo;
    }
}

template <typename R>
__device__ __forceinline__ ff load_p(const typename Amp<R>::T* psi, uint64_t i) {
    const auto v = psi[i];
    if constexpr (sizeof(R) == 4) {
        return ff_abs2(v.x, v.y);
    } else {
        const dd p = Acc<double>::abs2(v.x, v.y);
        const float hi = (float)p.hi;
        return {hi, (float)(p.hi - (double)hi + p.lo)};
    }
}

// ---- <Z> statistics with one warp per 1024-amplitude segment -------------------------------------------------
// Lane l reads pairs l + 32 j (j < 16) of segment s, i.e. amplitudes x = 1024 s + 2 (l + 32 j) + e: index bit 0
// is e, bits 1..5 are the lane, bits 6..9 are j. Each lane keeps, across all its segments (no barrier per
// segment), V[j] = sum of |a|^2 over its amplitudes with that j, plus S_0 (e = 1); the quantities of bits 6..9
// follow from V at the end. Per segment, two 8-term trees give the halves split by bit 9 (for X_9, bits 9 and
// 10) and the segment total, which goes to W[s] for the quantities of bits >= 10 (k_zstats_hi). Quantities per
// block at the end: 0: T, 1..10: S_0..S_9, 11..20: X_0..X_9.
constexpr int kZW = 21;

template <typename R>
__global__ void __launch_bounds__(256) k_zstats_warp(const typename Amp<R>::T* __restrict__ psi, uint64_t nseg,
                                                     double* __restrict__ W, float2* __restrict__ Wf,
                                                     double* __restrict__ partials) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const ff Z = {0.f, 0.f};
    ff V[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) V[j] = Z;
    ff S0 = Z, X9 = Z;
    for (uint64_t s = warp0; s < nseg; s += nwarps) {
        ff pj[16], qj[16];
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            ff P[8], Q[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) load_p2<R>(psi, s * 512 + lane + 32 * (8 * hh + j), P[j], Q[j]);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                pj[8 * hh + j] = ff_add(P[j], Q[j]);
                qj[8 * hh + j] = Q[j];
                V[8 * hh + j] = ff_add(V[8 * hh + j], pj[8 * hh + j]);
            }
        }
        S0 = ff_add(S0, ff_tree_sum(qj));
        ff lo8[8], hi8[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) { lo8[j] = pj[j]; hi8[j] = pj[8 + j]; }
        const ff lo = ff_tree_sum(lo8), hi = ff_tree_sum(hi8);  // bit 9 clear / set
        X9 = ff_add(X9, (s & 1) ? lo : hi);
        const ff tot = warp_sum_ff(ff_add(lo, hi));
        if (lane == 0) {
            W[s] = (double)tot.hi + (double)tot.lo;  // for the sampler
            Wf[s] = make_float2(tot.hi, tot.lo);     // for k_zstats_hi (no FP64 arithmetic there)
        }
    }
    // bits 6..9 from V: S_{6+b} = sum over j with bit b set; X_{6+b} = sum over j with bits b, b+1 different
    ff T = Z, S6 = Z, S7 = Z, S8 = Z, S9 = Z, X6 = Z, X7 = Z, X8 = Z;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        T = ff_add(T, V[j]);
        if (j & 1) S6 = ff_add(S6, V[j]);
        if (j & 2) S7 = ff_add(S7, V[j]);
        if (j & 4) S8 = ff_add(S8, V[j]);
        if (j & 8) S9 = ff_add(S9, V[j]);
        if ((j ^ (j >> 1)) & 1) X6 = ff_add(X6, V[j]);
        if (((j >> 1) ^ (j >> 2)) & 1) X7 = ff_add(X7, V[j]);
        if (((j >> 2) ^ (j >> 3)) & 1) X8 = ff_add(X8, V[j]);
    }
    // per-thread contributions; lane bit b is index bit b + 1
    ff c[kZW];
    c[0] = T;
    c[1] = S0;
#pragma unroll
    for (int i = 1; i <= 5; ++i) c[1 + i] = ((lane >> (i - 1)) & 1) ? T : Z;
    c[7] = S6; c[8] = S7; c[9] = S8; c[10] = S9;
    c[11] = (lane & 1) ? ff_add(T, ff_neg(S0)) : S0;
#pragma unroll
    for (int i = 1; i <= 4; ++i) c[11 + i] = (((lane >> (i - 1)) ^ (lane >> i)) & 1) ? T : Z;
    c[16] = ((lane >> 4) & 1) ? ff_add(T, ff_neg(S6)) : S6;
    c[17] = X6; c[18] = X7; c[19] = X8; c[20] = X9;
    __shared__ ff sm[8][kZW];
    const int warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kZW; ++q) {
        const ff v = warp_sum_ff(c[q]);
        if (lane == 0) sm[warp][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < kZW) {
        dd acc = {0.0, 0.0};
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            acc = dd_add(acc, dd{(double)sm[w][threadIdx.x].hi + (double)sm[w][threadIdx.x].lo, 0.0});
        double* p = partials + 2 * ((int64_t)threadIdx.x * gridDim.x + blockIdx.x);
        p[0] = acc.hi;
        p[1] = acc.lo;
    }
}

// Quantities of bits >= B from the segment totals Wf (float-float; nh = n - B), as partial sums: CTA (p, q) takes the p-th of
// gridDim.x equal contiguous ranges of segments and quantity q:
//   q < nh: S_{B+q} = sum_s W[s] bit_q(s);   nh <= q < 2 nh - 1: X_{B+r}, r = q - nh (bits r, r+1 of s).
// The partial goes to partials[q * gridDim.x + p] (hi, lo), for k_final_dd.
__global__ void __launch_bounds__(256) k_zstats_hi(const float2* __restrict__ Wf, uint64_t nseg, int nh,
                                                   double* __restrict__ partials) {
    __shared__ ff smf[8];
    const int q = blockIdx.y;
    const uint64_t len = nseg / gridDim.x, s0 = (uint64_t)blockIdx.x * len;
    ff acc = {0.f, 0.f};
    constexpr int U = 8;  // loads in flight per thread
    for (uint64_t s = s0 + threadIdx.x; s < s0 + len; s += U * blockDim.x) {
        float2 w[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t su = s + (uint64_t)u * blockDim.x;
            bool use = su < s0 + len;
            if (q < nh) use = use && ((su >> q) & 1);
            else { const int r = q - nh; use = use && (((su >> r) ^ (su >> (r + 1))) & 1); }
            w[u] = use ? Wf[su] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) acc = ff_add(acc, ff{w[u].x, w[u].y});
    }
    // block sum in float-float (FP64 is a small fraction of GB300's FP32 rate); partials combine in FP64
    acc = warp_sum_ff(acc);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) smf[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        ff v = smf[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v = ff_add(v, smf[w]);
        double* o = partials + 2 * ((int64_t)q * gridDim.x + blockIdx.x);
        o[0] = (double)v.hi;
        o[1] = (double)v.lo;
    }
}

// n < 12: one CTA; quantity q: 0 -> T, 1..n -> S_{q-1}, n+1..2n-1 -> X_{q-n-1}.
template <typename R>
__global__ void __launch_bounds__(256) k_zstats_small(const typename Amp<R>::T* __restrict__ psi, int n, double* out) {
    __shared__ double p[4096];
    const int N = 1 << n;
    for (int x = threadIdx.x; x < N; x += blockDim.x) {
        const ff v = load_p<R>(psi, x);
        p[x] = (double)v.hi + (double)v.lo;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < 2 * n; q += blockDim.x) {
        dd acc = {0.0, 0.0};
        for (int x = 0; x < N; ++x) {
            bool use;
            if (q == 0) use = true;
            else if (q <= n) use = (x >> (q - 1)) & 1;
            else { const int i = q - n - 1; use = ((x >> i) ^ (x >> (i + 1))) & 1; }
            if (use) acc = dd_add(acc, dd{p[x], 0.0});
        }
        out[2 * q] = acc.hi;
        out[2 * q + 1] = acc.lo;
    }
}

// ============================================================================================================
// Sampling: W[s] segment sums (2^SB amplitudes each), chunk sums of 1024 segments, inclusive scan of the
// chunk sums; then one warp per uniform walks chunk -> segment -> amplitude.
// ============================================================================================================
// W[s] = sum of |a|^2 over segment s (2^SB amplitudes), one warp per segment, 16-byte loads eight at a time.
template <typename R>
__global__ void __launch_bounds__(256) k_segsum(const typename Amp<R>::T* __restrict__ psi, int SB, uint64_t nseg,
                                                double* __restrict__ W) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    if (SB == 0) {  // one amplitude per segment (n = 0 never happens; kept for completeness)
        for (uint64_t s = warp0 * 32 + lane; s < nseg; s += nwarps * 32) {
            const ff p = load_p<R>(psi, s);
            W[s] = (double)p.hi + (double)p.lo;
        }
        return;
    }
    const uint64_t pairs = 1ull << (SB - 1);
    for (uint64_t s = warp0; s < nseg; s += nwarps) {
        ff acc = {0.f, 0.f};
        for (uint64_t j = lane; j < pairs; j += 8 * 32) {
            ff q[16];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const uint64_t k = j + 32 * u;
                if (k < pairs) load_p2<R>(psi, s * pairs + k, q[2 * u], q[2 * u + 1]);
                else q[2 * u] = q[2 * u + 1] = ff{0.f, 0.f};
            }
            acc = ff_add(acc, ff_tree_sum(q));
        }
        const ff tot = warp_sum_ff(acc);
        if (lane == 0) W[s] = (double)tot.hi + (double)tot.lo;
    }
}

__global__ void __launch_bounds__(256) k_chunksum(const double* __restrict__ W, uint64_t nseg, double* __restrict__ C) {
    __shared__ dd sm[32];
    const uint64_t c = blockIdx.x;
    dd acc = {0.0, 0.0};
    for (uint64_t i = c * 1024 + threadIdx.x; i < min(nseg, (c + 1) * 1024); i += blockDim.x)
        acc = dd_add(acc, dd{W[i], 0.0});
    acc = block_sum_dd(acc, sm);
    if (threadIdx.x == 0) C[c] = acc.hi + acc.lo;
}

// Inclusive scan of C[0..m) in place, one CTA of 1024 threads (double-double). Thread t owns the
// contiguous run [t * per, (t + 1) * per), per = ceil(m / 1024).
__global__ void __launch_bounds__(1024) k_scan_small(double* __restrict__ C, int m) {
    __shared__ dd sh[1024];
    const int t = threadIdx.x;
    const int per = (m + 1023) / 1024;
    const int i0 = t * per, i1 = min(m, i0 + per);
    dd run = {0.0, 0.0};
    for (int i = i0; i < i1; ++i) run = dd_add(run, dd{C[i], 0.0});
    sh[t] = run;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const dd v = t >= off ? sh[t - off] : dd{0.0, 0.0};
        __syncthreads();
        sh[t] = dd_add(sh[t], v);
        __syncthreads();
    }
    dd acc = t > 0 ? sh[t - 1] : dd{0.0, 0.0};
    for (int i = i0; i < i1; ++i) {
        acc = dd_add(acc, dd{C[i], 0.0});
        C[i] = acc.hi + acc.lo;
    }
}

__device__ __forceinline__ double warp_incl_scan_d(double v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

__device__ __forceinline__ ff warp_incl_scan_ff(ff v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const ff u = {__shfl_up_sync(0xffffffffu, v.hi, o), __shfl_up_sync(0xffffffffu, v.lo, o)};
        if (lane >= o) v = ff_add(v, u);
    }
    return v;
}

template <typename R>
__global__ void __launch_bounds__(256) k_sample(const typename Amp<R>::T* __restrict__ psi, int SB, uint64_t nseg,
                                                const double* __restrict__ W, const double* __restrict__ C,
                                                int nchunk, const double* __restrict__ u, int64_t shots,
                                                uint64_t* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const double total = C[nchunk - 1];
    for (int64_t i = warp0; i < shots; i += nwarps) {
        const double target = u[i] * total;
        // chunk: first c with C[c] > target
        int lo = 0, hi = nchunk;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (C[mid] > target) hi = mid; else lo = mid + 1;
        }
        int c = lo < nchunk ? lo : nchunk - 1;
        double r = target - (c > 0 ? C[c - 1] : 0.0);
        // segment inside the chunk
        const uint64_t s0 = (uint64_t)c * 1024, s1 = min(nseg, s0 + 1024);
        double run = 0.0;
        uint64_t seg = ~0ull, last_nz = s0;
        for (uint64_t sb = s0; sb < s1 && seg == ~0ull; sb += 32) {
            const uint64_t s = sb + lane;
            const double w = s < s1 ? W[s] : 0.0;
            const double pre = warp_incl_scan_d(w);
            const unsigned hit = __ballot_sync(0xffffffffu, s < s1 && run + pre > r);
            const unsigned nz = __ballot_sync(0xffffffffu, w > 0.0);
            if (nz) last_nz = sb + 31 - __clz(nz);
            if (hit) {
                const int l = __ffs(hit) - 1;
                seg = sb + l;
                const double before = __shfl_sync(0xffffffffu, pre - w, l);
                r -= run + before;
            } else {
                run += __shfl_sync(0xffffffffu, pre, 31);
            }
        }
        if (seg == ~0ull) { seg = last_nz; r = W[seg]; }
        // amplitude inside the segment
        const uint64_t a0 = seg << SB, a1 = a0 + (1ull << SB);
        ff frun = {0.f, 0.f};
        uint64_t x = ~0ull, lastx = a0;
        for (uint64_t xb = a0; xb < a1 && x == ~0ull; xb += 32) {
            const uint64_t xi = xb + lane;
            const ff p = xi < a1 ? load_p<R>(psi, xi) : ff{0.f, 0.f};
            const ff pre = warp_incl_scan_ff(p);
            const ff tot = ff_add(frun, pre);
            const unsigned hit = __ballot_sync(0xffffffffu, xi < a1 && ((double)tot.hi + (double)tot.lo) > r);
            const unsigned nz = __ballot_sync(0xffffffffu, p.hi > 0.f);
            if (nz) lastx = xb + 31 - __clz(nz);
            if (hit) x = xb + (__ffs(hit) - 1);
            else frun = ff_add(frun, ff{__shfl_sync(0xffffffffu, pre.hi, 31), __shfl_sync(0xffffffffu, pre.lo, 31)});
        }
        if (x == ~0ull) x = lastx;
        if (lane == 0) out[i] = x;
    }
}

__global__ void k_uniforms(uint64_t seed, int64_t count, double* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        // SplitMix64 (Steele, Lea, Flood 2014): the (i+1)-th state of the golden-ratio Weyl sequence, finalised.
        uint64_t z = seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        out[i] = (double)(z >> 11) * 0x1.0p-53;
    }
}

// ============================================================================================================
// Host drivers
// ============================================================================================================
static cudaError_t fetch(ReduceScratch& r, int nvals, cudaStream_t s) {
    cudaError_t e = cudaMemcpyAsync(r.hresult, r.result, sizeof(double) * nvals, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

static int reduce_blocks(const DevInfo& d, uint64_t N, int nq) {
    int64_t b = std::min<int64_t>((int64_t)d.num_sms * 8, (int64_t)((N + 255) / 256));
    b = std::min<int64_t>(b, kPartialDoubles / (2 * std::max(1, nq)));
    return (int)std::max<int64_t>(1, b);
}

cudaError_t run_norm(int dtype, const void* psi, int n, ReduceScratch& r, cudaStream_t s, const DevInfo& d, double* out) {
    const uint64_t N = 1ull << n;
    const int nb = reduce_blocks(d, N / 2, 1);
    if (dtype == QSIM_C64) k_norm_pairs<float><<<nb, 256, 0, s>>>((const float2*)psi, N / 2, r.partials);
    else k_norm_pairs<double><<<nb, 256, 0, s>>>((const double2*)psi, N / 2, r.partials);
    k_final_dd<<<1, 256, 0, s>>>(r.partials, nb, r.result);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = fetch(r, 2, s)) != cudaSuccess) return e;
    *out = r.hresult[0] + r.hresult[1];
    return cudaSuccess;
}

cudaError_t run_inner(int dtype, const void* a, const void* b, int n, ReduceScratch& r, cudaStream_t s,
                      const DevInfo& d, double* out) {
    const uint64_t N = 1ull << n;
    const int nb = reduce_blocks(d, N, 2);
    if (dtype == QSIM_C64) k_inner_partial<float><<<nb, 256, 0, s>>>((const float2*)a, (const float2*)b, N, r.partials);
    else k_inner_partial<double><<<nb, 256, 0, s>>>((const double2*)a, (const double2*)b, N, r.partials);
    k_final_dd<<<2, 256, 0, s>>>(r.partials, nb, r.result);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = fetch(r, 4, s)) != cudaSuccess) return e;
    out[0] = r.hresult[0] + r.hresult[1];
    out[1] = r.hresult[2] + r.hresult[3];
    return cudaSuccess;
}

cudaError_t run_pauli(int dtype, const void* psi, int n, const char* paulis, ReduceScratch& r, cudaStream_t s,
                      const DevInfo& d, double* out) {
    uint64_t f = 0, sm = 0;
    int ny = 0;
    for (int q = 0; q < n; ++q) {
        const char c = paulis[q];
        if (c == 'X' || c == 'Y') f |= 1ull << q;
        if (c == 'Y' || c == 'Z') sm |= 1ull << q;
        if (c == 'Y') ++ny;
    }
    const int h = f ? 63 - __builtin_clzll(f) : 0;
    const uint64_t work = f ? (1ull << (n - 1)) : (1ull << n);
    const int nb = reduce_blocks(d, work, 2);
    if (dtype == QSIM_C64) k_pauli_partial<float><<<nb, 256, 0, s>>>((const float2*)psi, n, f, sm, h, r.partials);
    else k_pauli_partial<double><<<nb, 256, 0, s>>>((const double2*)psi, n, f, sm, h, r.partials);
    k_final_dd<<<2, 256, 0, s>>>(r.partials, nb, r.result);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = fetch(r, 4, s)) != cudaSuccess) return e;
    const double sr = r.hresult[0] + r.hresult[1], si = r.hresult[2] + r.hresult[3];
    // multiply by i^{ny}
    switch (ny & 3) {
        case 0: out[0] = sr; out[1] = si; break;
        case 1: out[0] = -si; out[1] = sr; break;
        case 2: out[0] = -sr; out[1] = -si; break;
        default: out[0] = si; out[1] = -sr; break;
    }
    return cudaSuccess;
}

// n >= 12: k_probs_warp (see above); the 2^nq results go to r.scan (nq <= 12) or to a temporary device
// buffer of 8 x 2^nq bytes from the stream-ordered allocator, then one copy to the host.
static cudaError_t run_probs_warp(int dtype, const void* psi, int n, const int* qubits, int nq, ReduceScratch& r,
                                  cudaStream_t s, const DevInfo& d, double* out) {
    ProbsWArgs a;
    std::memset(&a, 0, sizeof(a));
    std::vector<std::pair<int, int>> low, high;  // (position, user index)
    uint64_t marg = 0;
    for (int j = 0; j < nq; ++j) {
        marg |= 1ull << qubits[j];
        (qubits[j] < 10 ? low : high).push_back({qubits[j], j});
    }
    std::sort(low.begin(), low.end());
    std::sort(high.begin(), high.end());
    a.nlow = (int)low.size();
    for (int k = 0; k < a.nlow; ++k) { a.lowj[k] = low[k].second; a.lowmask |= 1u << low[k].first; }
    a.nhigh = (int)high.size();
    for (int k = 0; k < a.nhigh; ++k) { a.highpos[k] = high[k].first; a.highj[k] = high[k].second; }
    for (int b = 10; b < n; ++b)
        if (!((marg >> b) & 1)) a.fhpos[a.nfh++] = b;
    // chunks per bin group: split while the items alone keep too few warps busy, each item still spans
    // at least 16 segments, and the partials (2^nq x S doubles) fit the scratch buffer
    const uint64_t F = 1ull << a.nfh, target_warps = (uint64_t)d.num_sms * 32;
    uint64_t S = 1;
    while (F / S >= 16 && ((S << a.nhigh) * 8) < target_warps && ((S * 2) << nq) <= (uint64_t)kPartialDoubles) S <<= 1;
    a.S = S;
    a.nitems = S << a.nhigh;
    a.wpi = (int)std::min<uint64_t>(8, F / S);
    const int ipb = 8 / a.wpi;
    const size_t smem = sizeof(ff) * (size_t)ipb << a.nlow;
    const int nb = (int)std::max<uint64_t>(1, std::min<uint64_t>((a.nitems + ipb - 1) / ipb, (uint64_t)d.num_sms * 2));
    const size_t bytes = sizeof(double) << nq;
    double* dout = r.scan;
    cudaError_t e = cudaSuccess;
    const bool tmp = nq > kSegBits;
    if (tmp && (e = cudaMallocAsync(reinterpret_cast<void**>(&dout), bytes, s)) != cudaSuccess) return e;
    const bool m0 = (a.lowmask & 1u) != 0;
    auto launch = [&](auto kern, auto typed_psi) {
        cudaError_t err = smem_optin(reinterpret_cast<const void*>(kern), (int)smem);
        if (err == cudaSuccess) {
            kern<<<nb, 256, smem, s>>>(typed_psi, a, r.partials, dout);
            err = cudaGetLastError();
        }
        return err;
    };
    const float2* p32 = static_cast<const float2*>(psi);
    const double2* p64 = static_cast<const double2*>(psi);
    if (dtype == QSIM_C64) e = m0 ? launch(k_probs_warp<float, true>, p32) : launch(k_probs_warp<float, false>, p32);
    else e = m0 ? launch(k_probs_warp<double, true>, p64) : launch(k_probs_warp<double, false>, p64);
    if (e == cudaSuccess && S > 1) {
        k_probs_warp_final<<<(unsigned)std::min<uint64_t>(((1ull << nq) + 255) / 256, 4096), 256, 0, s>>>(r.partials, a, dout);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, bytes, cudaMemcpyDeviceToHost, s);
    const cudaError_t ef = tmp ? cudaFreeAsync(dout, s) : cudaSuccess;
    const cudaError_t es = cudaStreamSynchronize(s);
    return e != cudaSuccess ? e : (ef != cudaSuccess ? ef : es);
}

cudaError_t run_probs(int dtype, const void* psi, int n, const int* qubits, int nq, ReduceScratch& r,
                      cudaStream_t s, const DevInfo& d, double* out) {
    ProbsArgs a;
    std::memset(&a, 0, sizeof(a));
    a.nq = nq;
    const int NB = 1 << nq;
    cudaError_t e;
    if (n < kSegBits) {
        // positions: marginal qubits in user order, then the others ascending
        std::vector<int> qpos(qubits, qubits + nq);
        for (int q = 0; q < n; ++q)
            if (std::find(qubits, qubits + nq, q) == qubits + nq) qpos.push_back(q);
        int* dq = reinterpret_cast<int*>(r.partials + kPartialDoubles - 64);
        if ((e = cudaMemcpyAsync(dq, qpos.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
        if (dtype == QSIM_C64) k_probs_small<float><<<1, 256, 0, s>>>((const float2*)psi, n, a, dq, r.partials);
        else k_probs_small<double><<<1, 256, 0, s>>>((const double2*)psi, n, a, dq, r.partials);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        std::vector<double> h(2 * (size_t)NB);  // up to 2 x 2^11 values: more than the pinned result buffer
        if ((e = cudaMemcpyAsync(h.data(), r.partials, sizeof(double) * 2 * NB, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
        for (int m = 0; m < NB; ++m) out[m] = h[2 * m] + h[2 * m + 1];
        return cudaSuccess;
    }
    return run_probs_warp(dtype, psi, n, qubits, nq, r, s, d, out);
}

int zstats_segment_bits(int n) { return n < kSegBits ? 0 : 10; }

// The <Z> kernels: r.result receives, as (hi, lo) pairs, T, S_0..S_{n-1}, X_0..X_{n-2} for n < 12 (one CTA),
// else the kZW warp-segment quantities (T, S_0..S_9, X_0..X_9) followed by S_10..S_{n-1}, X_10..X_{n-2}.
static cudaError_t enqueue_zstats(int dtype, const void* psi, int n, ReduceScratch& r, cudaStream_t s,
                                  const DevInfo& d) {
    if (n < kSegBits) {
        if (dtype == QSIM_C64) k_zstats_small<float><<<1, 256, 0, s>>>((const float2*)psi, n, r.result);
        else k_zstats_small<double><<<1, 256, 0, s>>>((const double2*)psi, n, r.result);
        return cudaGetLastError();
    }
    // warp segments of 1024 amplitudes (n >= 12 here): bits 0..9 per thread, bits >= 10 from W
    const uint64_t nseg = 1ull << (n - 10);
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)d.num_sms * 8, (int64_t)((nseg + 7) / 8)));
    double* W = r.seg;                                   // 2^(n-10) doubles
    float2* Wf = reinterpret_cast<float2*>(r.seg + nseg);  // then the same sums as float-float
    if (dtype == QSIM_C64) k_zstats_warp<float><<<nb, 256, 0, s>>>((const float2*)psi, nseg, W, Wf, r.partials);
    else k_zstats_warp<double><<<nb, 256, 0, s>>>((const double2*)psi, nseg, W, Wf, r.partials);
    k_final_dd<<<kZW, 256, 0, s>>>(r.partials, nb, r.result);
    const int nh = n - 10;
    // after k_final_dd above has consumed the warp partials (same stream), the buffer takes the high bits'
    const unsigned P = (unsigned)std::min<uint64_t>(32, nseg);
    k_zstats_hi<<<dim3(P, 2 * nh - 1), 256, 0, s>>>(Wf, nseg, nh, r.partials);
    k_final_dd<<<2 * nh - 1, 256, 0, s>>>(r.partials, (int)P, r.result + 2 * kZW);
    return cudaGetLastError();
}

static int zstats_result_values(int n) { return n < kSegBits ? 4 * n : 2 * kZW + 2 * (2 * (n - 10) - 1); }

// <Z_i> = T - 2 S_i and <Z_i Z_{i+1}> = T - 2 X_i from the quantities enqueue_zstats leaves (h: (hi, lo) pairs).
__host__ __device__ inline double zstats_value(const double* h, int q) { return h[2 * q] + h[2 * q + 1]; }
__host__ __device__ inline double zstats_zi(const double* h, int n, int i) {
    const double T = zstats_value(h, 0);
    if (n < kSegBits) return T - 2.0 * zstats_value(h, 1 + i);
    return T - 2.0 * (i < 10 ? zstats_value(h, 1 + i) : zstats_value(h, kZW + (i - 10)));
}
__host__ __device__ inline double zstats_zz(const double* h, int n, int i) {
    const double T = zstats_value(h, 0);
    if (n < kSegBits) return T - 2.0 * zstats_value(h, n + 1 + i);
    return T - 2.0 * (i < 10 ? zstats_value(h, 11 + i) : zstats_value(h, kZW + (n - 10) + (i - 10)));
}

// normalise: divide by T (the squared norm), i.e. report the values of the normalised state
__global__ void k_zstats_finish(const double* __restrict__ h, int n, int normalise, double* __restrict__ zi,
                                double* __restrict__ zz) {
    const double inv = normalise ? 1.0 / zstats_value(h, 0) : 1.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        zi[i] = normalise ? zstats_zi(h, n, i) * inv : zstats_zi(h, n, i);
        if (i + 1 < n) zz[i] = normalise ? zstats_zz(h, n, i) * inv : zstats_zz(h, n, i);
    }
}

cudaError_t run_zstats(int dtype, const void* psi, int n, ReduceScratch& r, cudaStream_t s, const DevInfo& d,
                       double* zi, double* zz) {
    cudaError_t e = enqueue_zstats(dtype, psi, n, r, s, d);
    if (e != cudaSuccess) return e;
    if ((e = fetch(r, zstats_result_values(n), s)) != cudaSuccess) return e;
    for (int i = 0; i < n; ++i) zi[i] = zstats_zi(r.hresult, n, i);
    for (int i = 0; i + 1 < n; ++i) zz[i] = zstats_zz(r.hresult, n, i);
    return cudaSuccess;
}

cudaError_t run_zstats_device(int dtype, const void* psi, int n, ReduceScratch& r, cudaStream_t s,
                              const DevInfo& d, double* zi_dev, double* zz_dev, bool normalise) {
    cudaError_t e = enqueue_zstats(dtype, psi, n, r, s, d);
    if (e != cudaSuccess) return e;
    k_zstats_finish<<<1, 64, 0, s>>>(r.result, n, normalise ? 1 : 0, zi_dev, zz_dev);
    return cudaGetLastError();
}

cudaError_t launch_uniforms(uint64_t seed, int64_t count, double* out_dev, cudaStream_t s) {
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((count + 255) / 256, 4096));
    k_uniforms<<<blocks, 256, 0, s>>>(seed, count, out_dev);
    return cudaGetLastError();
}

cudaError_t run_sample(int dtype, const void* psi, int n, const double* u_dev, int64_t shots, uint64_t* out_dev,
                       ReduceScratch& r, cudaStream_t s, const DevInfo& d, int seg_ready_bits) {
    // seg_ready_bits > 0: r.seg already holds the sums of segments of 2^seg_ready_bits amplitudes (from the
    // <Z> pass), so the state is read again only inside the sampled segments
    const int SB = seg_ready_bits > 0 ? seg_ready_bits : std::min(n, kSegBits);
    const uint64_t nseg = 1ull << (n - SB);
    const int nchunk = (int)((nseg + 1023) / 1024);
    double* W = r.seg;
    double* C = r.scan;
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)d.num_sms * 8, (int64_t)((nseg + 7) / 8)));
    if (seg_ready_bits <= 0) {
        if (dtype == QSIM_C64) k_segsum<float><<<nb, 256, 0, s>>>((const float2*)psi, SB, nseg, W);
        else k_segsum<double><<<nb, 256, 0, s>>>((const double2*)psi, SB, nseg, W);
    }
    k_chunksum<<<nchunk, 256, 0, s>>>(W, nseg, C);
    k_scan_small<<<1, 1024, 0, s>>>(C, nchunk);
    const int sb = (int)std::max<int64_t>(1, std::min<int64_t>((shots * 32 + 255) / 256, (int64_t)d.num_sms * 8));
    if (dtype == QSIM_C64) k_sample<float><<<sb, 256, 0, s>>>((const float2*)psi, SB, nseg, W, C, nchunk, u_dev, shots, out_dev);
    else k_sample<double><<<sb, 256, 0, s>>>((const double2*)psi, SB, nseg, W, C, nchunk, u_dev, shots, out_dev);
    return cudaGetLastError();
}

}  // namespace qsim
