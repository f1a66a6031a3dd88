// k_gates.cu -- per-gate passes over the state vector (the hot loop of paper Sec. 2.1 "State-Vector
// Simulation": every gate is a tensor-product operator, applied at O(2^n) cost per gate).
//
//   k_dense_small  dense U on k <= 4 targets (+ controls): each thread gathers the 2^k amplitudes of one
//                  group (targets and controls masked out of the index), multiplies, scatters. With qubit 0
//                  untouched, a complex64 thread handles two adjacent groups with 16-byte loads.
//   k_dense_split  the same for small states: 2..16 lanes of a warp share one group, so that the
//                  (complex128) arithmetic of a few thousand groups still spreads over every SM.
//   k_butterfly    single-qubit dense U on a low target (1..4, complex64): every lane streams one
//                  contiguous 16-byte pair of amplitudes and receives its partners by warp shuffles.
//   k_diag         diagonal U: multiplies only the amplitudes whose diagonal factor is not exactly 1
//                  (CZ / controlled phase touch a quarter of the state).
//   k_dense_tile   dense U on k = 5, 6 targets through shared memory (CUDA-core arithmetic).
//   k_dense_big    dense U on k = 7, 8 targets: U streamed from L2 in column chunks, 32 groups per CTA.
//   k_swap_tile    in-place qubit reorder through shared-memory tiles.
//   k_set_basis    |x>.
#include <algorithm>
#include <type_traits>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace qsim {

__device__ __forceinline__ float fmar(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmar(double a, double b, double c) { return __fma_rn(a, b, c); }

// ============================================================================================================
// Dense k <= 4
// ============================================================================================================
template <typename R, int K>
struct DenseSmallArgs {
    int nf;                 // fixed bits (targets + controls), ascending
    int fixed[kMaxFixed];
    uint64_t cmask;         // control bits, set in every base index
    uint64_t off[1 << K];   // index offset of matrix index m: sum_j bit_j(m) << targets[j]
    R m[2 << (2 * K)];      // U, row-major, interleaved (re, im)
};

template <typename R, int K, int V>
__global__ void __launch_bounds__(256)
k_dense_small(typename Amp<R>::T* __restrict__ psi, uint64_t nitems, const __grid_constant__ DenseSmallArgs<R, K> a) {
    using T = typename Amp<R>::T;
    constexpr int D = 1 << K;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t it = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; it < nitems; it += stride) {
        const uint64_t base = insert_zeros(it * V, a.fixed, a.nf) | a.cmask;
        if constexpr (V == 1) {
            T v[D];
#pragma unroll
            for (int m = 0; m < D; ++m) v[m] = psi[base + a.off[m]];
#pragma unroll
            for (int r = 0; r < D; ++r) {
                R re = 0, im = 0;
#pragma unroll
                for (int c = 0; c < D; ++c) {
                    const R ur = a.m[2 * (r * D + c)], ui = a.m[2 * (r * D + c) + 1];
                    re = fmar(ur, v[c].x, re);
                    re = fmar(-ui, v[c].y, re);
                    im = fmar(ur, v[c].y, im);
                    im = fmar(ui, v[c].x, im);
                }
                psi[base + a.off[r]] = make_amp<R>(re, im);
            }
        } else {
            // complex64 only: groups (it*2, it*2+1) have bases base and base+1, one float4 per matrix index.
            float4 v[D];
#pragma unroll
            for (int m = 0; m < D; ++m) v[m] = *reinterpret_cast<const float4*>(psi + base + a.off[m]);
#pragma unroll
            for (int r = 0; r < D; ++r) {
                float r0 = 0, i0 = 0, r1 = 0, i1 = 0;
#pragma unroll
                for (int c = 0; c < D; ++c) {
                    const float ur = a.m[2 * (r * D + c)], ui = a.m[2 * (r * D + c) + 1];
                    r0 = fmar(ur, v[c].x, r0); r0 = fmar(-ui, v[c].y, r0);
                    i0 = fmar(ur, v[c].y, i0); i0 = fmar(ui, v[c].x, i0);
                    r1 = fmar(ur, v[c].z, r1); r1 = fmar(-ui, v[c].w, r1);
                    i1 = fmar(ur, v[c].w, i1); i1 = fmar(ui, v[c].z, i1);
                }
                *reinterpret_cast<float4*>(psi + base + a.off[r]) = make_float4(r0, i0, r1, i1);
            }
        }
    }
}

// Small states (too few groups to fill the GPU; the complex128 arithmetic is then the limit): TPG lanes of
// one warp share a group. Every lane loads the group's 2^K amplitudes (same-address loads are broadcast),
// the warp synchronises (all reads before any write: the update is in place), and each lane computes and
// stores the rows r = sub + j * TPG. nitems = groups * TPG is a multiple of 32, so warps run in lockstep.
template <typename R, int K, int TPG>
__global__ void __launch_bounds__(256)
k_dense_split(typename Amp<R>::T* __restrict__ psi, uint64_t nitems, const __grid_constant__ DenseSmallArgs<R, K> a) {
    using T = typename Amp<R>::T;
    constexpr int D = 1 << K, RPL = D / TPG;
    static_assert(TPG >= 2 && TPG <= D && 32 % TPG == 0, "a group's lanes sit in one warp");
    // lanes of a warp read different rows of U: from shared memory (banked), not the constant bank
    // (which serialises divergent addresses)
    __shared__ R sU[2 * D * D];
    for (int i = threadIdx.x; i < 2 * D * D; i += blockDim.x) sU[i] = a.m[i];
    __syncthreads();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const int sub = threadIdx.x % TPG;
    for (uint64_t it = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; it < nitems; it += stride) {
        const uint64_t base = insert_zeros(it / TPG, a.fixed, a.nf) | a.cmask;
        T v[D];
#pragma unroll
        for (int m = 0; m < D; ++m) v[m] = psi[base + a.off[m]];
        __syncwarp();
#pragma unroll
        for (int j = 0; j < RPL; ++j) {
            const int r = sub + j * TPG;
            R re = 0, im = 0;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const R ur = sU[2 * (r * D + c)], ui = sU[2 * (r * D + c) + 1];
                re = fmar(ur, v[c].x, re);
                re = fmar(-ui, v[c].y, re);
                im = fmar(ur, v[c].y, im);
                im = fmar(ui, v[c].x, im);
            }
            psi[base + a.off[r]] = make_amp<R>(re, im);
        }
    }
}

// ============================================================================================================
// Single-qubit butterfly on a low target t in 1..4 (complex64, no controls): lane l holds amplitudes
// 2l, 2l+1 of a 64-amplitude warp chunk; the partner of amplitude i is i ^ 2^t, held by lane l ^ 2^(t-1).
// ============================================================================================================
struct ButterflyArgs {
    int t;
    float m[8];
};

__global__ void __launch_bounds__(256)
k_butterfly(float4* __restrict__ psi4, uint64_t n4, const __grid_constant__ ButterflyArgs a) {
    const int lane = threadIdx.x & 31;
    const int sh = 1 << (a.t - 1);
    const bool upper = (lane >> (a.t - 1)) & 1;  // this lane's amplitudes have bit t set
    // Row of U this lane produces and which operand is "own" vs "partner":
    //   bit t clear: out = u00 * own + u01 * partner;  bit t set: out = u10 * partner + u11 * own.
    const float ow_r = upper ? a.m[6] : a.m[0], ow_i = upper ? a.m[7] : a.m[1];
    const float pa_r = upper ? a.m[4] : a.m[2], pa_i = upper ? a.m[5] : a.m[3];
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    // n4 is a multiple of 32 (n >= 6), so every warp iterates in lock-step.
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
        const float4 v = psi4[i];
        float4 p;
        p.x = __shfl_xor_sync(0xffffffffu, v.x, sh);
        p.y = __shfl_xor_sync(0xffffffffu, v.y, sh);
        p.z = __shfl_xor_sync(0xffffffffu, v.z, sh);
        p.w = __shfl_xor_sync(0xffffffffu, v.w, sh);
        float4 o;
        o.x = fmar(ow_r, v.x, fmar(-ow_i, v.y, fmar(pa_r, p.x, -pa_i * p.y)));
        o.y = fmar(ow_r, v.y, fmar(ow_i, v.x, fmar(pa_r, p.y, pa_i * p.x)));
        o.z = fmar(ow_r, v.z, fmar(-ow_i, v.w, fmar(pa_r, p.z, -pa_i * p.w)));
        o.w = fmar(ow_r, v.w, fmar(ow_i, v.z, fmar(pa_r, p.w, pa_i * p.z)));
        psi4[i] = o;
    }
}

// ============================================================================================================
// Diagonal
// ============================================================================================================
template <typename R>
struct DiagArgs {
    int nf;
    int fixed[kMaxFixed];
    uint64_t cmask;
    int np;              // number of diagonal patterns touched
    uint64_t off[64];    // index offset of each touched pattern
    R d[128];            // its factor (re, im)
};

template <typename R, int V>
__global__ void __launch_bounds__(256)
k_diag(typename Amp<R>::T* __restrict__ psi, uint64_t nitems, const __grid_constant__ DiagArgs<R> a) {
    using T = typename Amp<R>::T;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t it = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; it < nitems; it += stride) {
        const uint64_t base = insert_zeros(it * V, a.fixed, a.nf) | a.cmask;
        for (int p = 0; p < a.np; ++p) {
            const R dr = a.d[2 * p], di = a.d[2 * p + 1];
            if constexpr (V == 1) {
                T* q = psi + base + a.off[p];
                const T v = *q;
                *q = make_amp<R>(fmar(dr, v.x, -di * v.y), fmar(dr, v.y, di * v.x));
            } else {
                float4* q = reinterpret_cast<float4*>(psi + base + a.off[p]);
                const float4 v = *q;
                *q = make_float4(fmar(dr, v.x, -di * v.y), fmar(dr, v.y, di * v.x),
                                 fmar(dr, v.z, -di * v.w), fmar(dr, v.w, di * v.z));
            }
        }
    }
}

// ============================================================================================================
// Dense k = 5, 6 through shared memory
// ============================================================================================================
struct TileArgs {
    int nf;
    int fixed[kMaxFixed];
    uint64_t cmask;
    uint64_t off[64];
};

template <typename R, int K>
__global__ void __launch_bounds__(256)
k_dense_tile(typename Amp<R>::T* __restrict__ psi, uint64_t ngroups, const __grid_constant__ TileArgs a,
             const typename Amp<R>::T* __restrict__ U) {
    using T = typename Amp<R>::T;
    constexpr int D = 1 << K, ROWS = 64, OUTS = D / 4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sU = reinterpret_cast<T*>(smem_raw);  // D x D
    T* sX = sU + D * D;                      // column-major: sX[c * ROWS + r]
    for (int i = threadIdx.x; i < D * D; i += blockDim.x) sU[i] = U[i];
    const int r = threadIdx.x & (ROWS - 1), q = threadIdx.x / ROWS;
    const uint64_t ntiles = (ngroups + ROWS - 1) / ROWS;
    __syncthreads();
    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint64_t g = tile * ROWS + r;
        const bool act = g < ngroups;
        const uint64_t base = act ? (insert_zeros(g, a.fixed, a.nf) | a.cmask) : 0;
        if (act) {
#pragma unroll
            for (int j = 0; j < OUTS; ++j) {
                const int c = q * OUTS + j;
                sX[c * ROWS + r] = psi[base + a.off[c]];
            }
        }
        __syncthreads();
        R ar[OUTS], ai[OUTS];
#pragma unroll
        for (int j = 0; j < OUTS; ++j) ar[j] = ai[j] = 0;
        for (int c = 0; c < D; ++c) {
            const T x = sX[c * ROWS + r];
#pragma unroll
            for (int j = 0; j < OUTS; ++j) {
                const T u = sU[(q * OUTS + j) * D + c];
                ar[j] = fmar(u.x, x.x, ar[j]);
                ar[j] = fmar(-u.y, x.y, ar[j]);
                ai[j] = fmar(u.x, x.y, ai[j]);
                ai[j] = fmar(u.y, x.x, ai[j]);
            }
        }
        __syncthreads();
        if (act) {
#pragma unroll
            for (int j = 0; j < OUTS; ++j) psi[base + a.off[q * OUTS + j]] = make_amp<R>(ar[j], ai[j]);
        }
    }
}

// ============================================================================================================
// Qubit reorder: tile = 2^L contiguous amplitudes x the combinations of the swapped bits above L. Inside a
// tile the exchange of bit pairs is a permutation of tile positions (an involution), applied through smem.
// ============================================================================================================
struct SwapArgs {
    int nS;          // tile bits
    int L;           // tile bits 0..L-1 are index bits 0..L-1
    int nH;          // nS - L
    int hbits[16];   // index positions of tile bits L.. (ascending)
    int perm[16];    // tile bit b moves to tile bit perm[b]
};

template <typename R>
__global__ void __launch_bounds__(256)
k_swap_tile(typename Amp<R>::T* __restrict__ psi, uint64_t ntiles, const __grid_constant__ SwapArgs a) {
    using T = typename Amp<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sT = reinterpret_cast<T*>(smem_raw);
    __shared__ uint64_t hoff[1 << 9];
    const int TS = 1 << a.nS;
    const int lmask = (1 << a.L) - 1;
    for (int i = threadIdx.x; i < (1 << a.nH); i += blockDim.x) hoff[i] = deposit((uint64_t)i, a.hbits, a.nH);
    __syncthreads();
    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint64_t base = insert_zeros(tile << a.L, a.hbits, a.nH);
        for (int j = threadIdx.x; j < TS; j += blockDim.x) sT[j] = psi[base + (j & lmask) + hoff[j >> a.L]];
        __syncthreads();
        for (int j = threadIdx.x; j < TS; j += blockDim.x) {
            int src = 0;
            for (int b = 0; b < a.nS; ++b) src |= ((j >> b) & 1) << a.perm[b];
            psi[base + (j & lmask) + hoff[j >> a.L]] = sT[src];
        }
        __syncthreads();
    }
}

// Direct exchange when every swapped bit is >= 1 (complex64 16-byte vectors of two groups) or any (V = 1):
// only amplitudes whose index changes are read and written. Items enumerate (moving pattern pair, group);
// groups vary fastest, so a warp streams contiguous runs for a fixed pattern pair.
struct SwapDirectArgs {
    int nb;               // 2p swapped bit positions, ascending
    int bits[16];
    int npairs;           // moving pattern pairs (u, sigma(u)), u < sigma(u)
    uint64_t off_u[120], off_v[120];
};

template <typename R, int V>
__global__ void __launch_bounds__(256)
k_swap_direct(typename Amp<R>::T* __restrict__ psi, uint64_t groups_v, const __grid_constant__ SwapDirectArgs a) {
    using T = typename Amp<R>::T;
    using X = typename std::conditional<V == 2, float4, T>::type;  // one access: V adjacent amplitudes
    constexpr int U = 4;  // items per thread and round: every load of a round is issued before its stores
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t total = groups_v * (uint64_t)a.npairs;
    for (uint64_t it0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; it0 < total; it0 += U * stride) {
        X* pu[U];
        X* pv[U];
        X x[U], y[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const uint64_t it = it0 + (uint64_t)k * stride;
            pu[k] = pv[k] = nullptr;
            if (it < total) {
                const uint64_t m = it / groups_v, gv = it - m * groups_v;
                const uint64_t base = insert_zeros(gv * V, a.bits, a.nb);
                pu[k] = reinterpret_cast<X*>(psi + base + a.off_u[m]);
                pv[k] = reinterpret_cast<X*>(psi + base + a.off_v[m]);
                x[k] = *pu[k];
                y[k] = *pv[k];
            }
        }
#pragma unroll
        for (int k = 0; k < U; ++k)
            if (pu[k]) {
                *pu[k] = y[k];
                *pv[k] = x[k];
            }
    }
}

// ============================================================================================================
// |x>
// ============================================================================================================
template <typename R>
__global__ void __launch_bounds__(256)
k_set_basis(typename Amp<R>::T* __restrict__ psi, uint64_t namps, uint64_t x) {
    using T = typename Amp<R>::T;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < namps; i += stride)
        psi[i] = (i == x) ? make_amp<R>(1, 0) : make_amp<R>(0, 0);
}

__global__ void k_convert_matrix(const double* __restrict__ src, float* __restrict__ dst, int64_t count) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (float)src[i];
}

// ============================================================================================================
// Dense k = 7, 8 (CUDA cores). The matrix (up to 256 x 256 complex, L2-resident) does not fit in shared
// memory next to the amplitudes, so it is streamed in column chunks of C through a padded shared buffer;
// each chunk serves the G = 32 groups a CTA holds in shared memory. Thread (row r, half h) accumulates row
// r of its G / H groups in registers and writes them back after the last chunk (the update is in place;
// every input of the iteration is in shared memory by then).
// ============================================================================================================
struct BigArgs {
    int nf;
    int fixed[kMaxFixed];
    uint64_t cmask;
    int tpos[8];
};

template <typename R, int K> struct BigCfg {
    static constexpr int D = 1 << K, G = 32, C = K == 7 ? 32 : 16, H = 256 / D, GPT = G / H;
    static constexpr size_t smem = sizeof(typename Amp<R>::T) * ((size_t)G * D + (size_t)D * (C + 1)) +
                                   sizeof(uint64_t) * D;
};

template <typename R, int K>
__global__ void __launch_bounds__(256)
k_dense_big(typename Amp<R>::T* __restrict__ psi, uint64_t ngroups, const __grid_constant__ BigArgs a,
            const typename Amp<R>::T* __restrict__ U) {
    using T = typename Amp<R>::T;
    using B = BigCfg<R, K>;
    constexpr int D = B::D, G = B::G, C = B::C, GPT = B::GPT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* V = reinterpret_cast<T*>(smem_raw);                             // [G][D] amplitudes
    T* UC = V + G * D;                                                 // [D][C + 1] column chunk of U
    uint64_t* offs = reinterpret_cast<uint64_t*>(UC + D * (C + 1));    // [D] index offset of column c
    for (int i = threadIdx.x; i < D; i += blockDim.x) offs[i] = deposit((uint64_t)i, a.tpos, K);
    const int r = threadIdx.x % D, h = threadIdx.x / D;
    for (uint64_t g0 = (uint64_t)blockIdx.x * G; g0 < ngroups; g0 += (uint64_t)gridDim.x * G) {
        __syncthreads();  // offsets ready; the previous iteration's reads of V and UC are done
        for (int i = threadIdx.x; i < G * D; i += blockDim.x) {
            const uint64_t g = g0 + (uint64_t)(i / D);
            if (g < ngroups) V[i] = psi[(insert_zeros(g, a.fixed, a.nf) | a.cmask) + offs[i % D]];
        }
        R re[GPT], im[GPT];
#pragma unroll
        for (int j = 0; j < GPT; ++j) re[j] = im[j] = 0;
        for (int c0 = 0; c0 < D; c0 += C) {
            __syncthreads();  // V loaded; the previous chunk consumed
            for (int i = threadIdx.x; i < D * C; i += blockDim.x) {
                const int rr = i / C, cc = i % C;
                UC[rr * (C + 1) + cc] = U[(size_t)rr * D + c0 + cc];
            }
            __syncthreads();
#pragma unroll 4
            for (int cc = 0; cc < C; ++cc) {
                const T u = UC[r * (C + 1) + cc];
#pragma unroll
                for (int j = 0; j < GPT; ++j) {
                    const T v = V[(h * GPT + j) * D + c0 + cc];  // same address across the warp: broadcast
                    re[j] = fmar(u.x, v.x, re[j]);
                    re[j] = fmar(-u.y, v.y, re[j]);
                    im[j] = fmar(u.x, v.y, im[j]);
                    im[j] = fmar(u.y, v.x, im[j]);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < GPT; ++j) {
            const uint64_t g = g0 + (uint64_t)(h * GPT + j);
            if (g < ngroups) psi[(insert_zeros(g, a.fixed, a.nf) | a.cmask) + offs[r]] = make_amp<R>(re[j], im[j]);
        }
    }
}

// ============================================================================================================
// Host launchers
// ============================================================================================================
namespace {

struct Fixed {
    int nf = 0;
    int pos[kMaxFixed];
    uint64_t cmask = 0;
    int lowest = 64;
};

Fixed make_fixed(int k, const int* targets, int nc, const int* controls) {
    Fixed f;
    for (int j = 0; j < k; ++j) f.pos[f.nf++] = targets[j];
    for (int j = 0; j < nc; ++j) {
        f.pos[f.nf++] = controls[j];
        f.cmask |= 1ull << controls[j];
    }
    std::sort(f.pos, f.pos + f.nf);
    f.lowest = f.nf ? f.pos[0] : 64;
    return f;
}

uint64_t target_offset(int m, int k, const int* targets) {
    uint64_t off = 0;
    for (int j = 0; j < k; ++j) off |= (uint64_t)((m >> j) & 1) << targets[j];
    return off;
}

template <typename R, int K>
cudaError_t dense_small_t(void* psi, int n, const int* targets, const Fixed& f, const double* mat,
                          cudaStream_t s, const DevInfo& d) {
    DenseSmallArgs<R, K> a;
    std::memset(&a, 0, sizeof(a));
    a.nf = f.nf;
    std::memcpy(a.fixed, f.pos, sizeof(int) * f.nf);
    a.cmask = f.cmask;
    constexpr int D = 1 << K;
    for (int m = 0; m < D; ++m) a.off[m] = target_offset(m, K, targets);
    for (int i = 0; i < 2 * D * D; ++i) a.m[i] = (R)mat[i];
    const uint64_t ngroups = 1ull << (n - f.nf);
    using T = typename Amp<R>::T;
    // Small states: spread each group over TPG lanes until about 1024 threads per SM are busy.
    if (ngroups < (uint64_t)d.num_sms * 512) {
        int tpg = 1;
        while (tpg < D && ngroups * (uint64_t)tpg < (uint64_t)d.num_sms * 1024) tpg <<= 1;
        const uint64_t items = ngroups * (uint64_t)tpg;
        if (tpg > 1 && items % 32 == 0) {
            const unsigned grid = grid_for((int64_t)items, 256, d.num_sms, 8);
            T* p = reinterpret_cast<T*>(psi);
            switch (tpg) {
                case 2: k_dense_split<R, K, 2><<<grid, 256, 0, s>>>(p, items, a); break;
                case 4: if constexpr (D >= 4) k_dense_split<R, K, 4><<<grid, 256, 0, s>>>(p, items, a); break;
                case 8: if constexpr (D >= 8) k_dense_split<R, K, 8><<<grid, 256, 0, s>>>(p, items, a); break;
                default: if constexpr (D >= 16) k_dense_split<R, K, 16><<<grid, 256, 0, s>>>(p, items, a); break;
            }
            return cudaGetLastError();
        }
    }
    if constexpr (sizeof(R) == 4) {
        if (f.lowest >= 1 && ngroups >= 2) {
            const uint64_t items = ngroups / 2;
            k_dense_small<R, K, 2><<<grid_for((int64_t)items, 256, d.num_sms, 8), 256, 0, s>>>(
                reinterpret_cast<T*>(psi), items, a);
            return cudaGetLastError();
        }
    }
    k_dense_small<R, K, 1><<<grid_for((int64_t)ngroups, 256, d.num_sms, 8), 256, 0, s>>>(
        reinterpret_cast<T*>(psi), ngroups, a);
    return cudaGetLastError();
}

template <typename R>
cudaError_t dense_small_r(void* psi, int n, int k, const int* targets, const Fixed& f, const double* mat,
                          cudaStream_t s, const DevInfo& d) {
    switch (k) {
        case 1: return dense_small_t<R, 1>(psi, n, targets, f, mat, s, d);
        case 2: return dense_small_t<R, 2>(psi, n, targets, f, mat, s, d);
        case 3: return dense_small_t<R, 3>(psi, n, targets, f, mat, s, d);
        case 4: return dense_small_t<R, 4>(psi, n, targets, f, mat, s, d);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_dense_small(int dtype, void* psi, int n, int k, const int* targets, int nc,
                               const int* controls, const double* mat, cudaStream_t s, const DevInfo& d) {
    const Fixed f = make_fixed(k, targets, nc, controls);
    // Low single-qubit targets without controls: warp-shuffle butterfly with fully contiguous 16-byte lanes.
    if (dtype == QSIM_C64 && k == 1 && nc == 0 && targets[0] >= 1 && targets[0] <= 5 && n >= 6) {
        ButterflyArgs a;
        a.t = targets[0];
        for (int i = 0; i < 8; ++i) a.m[i] = (float)mat[i];
        const uint64_t n4 = 1ull << (n - 1);
        k_butterfly<<<grid_for((int64_t)n4, 256, d.num_sms, 8), 256, 0, s>>>(reinterpret_cast<float4*>(psi), n4, a);
        return cudaGetLastError();
    }
    if (dtype == QSIM_C64) return dense_small_r<float>(psi, n, k, targets, f, mat, s, d);
    return dense_small_r<double>(psi, n, k, targets, f, mat, s, d);
}

template <typename R>
static cudaError_t diag_t(void* psi, int n, int k, const int* targets, const Fixed& f, const double* diag,
                          const std::vector<int>& touch, cudaStream_t s, const DevInfo& d) {
    DiagArgs<R> a;
    std::memset(&a, 0, sizeof(a));
    a.nf = f.nf;
    std::memcpy(a.fixed, f.pos, sizeof(int) * f.nf);
    a.cmask = f.cmask;
    a.np = (int)touch.size();
    for (int i = 0; i < a.np; ++i) {
        const int m = touch[i];
        a.off[i] = target_offset(m, k, targets);
        a.d[2 * i] = (R)diag[2 * m];
        a.d[2 * i + 1] = (R)diag[2 * m + 1];
    }
    const uint64_t ngroups = 1ull << (n - f.nf);
    using T = typename Amp<R>::T;
    if constexpr (sizeof(R) == 4) {
        if (f.lowest >= 1 && ngroups >= 2) {
            const uint64_t items = ngroups / 2;
            k_diag<R, 2><<<grid_for((int64_t)items, 256, d.num_sms, 8), 256, 0, s>>>(reinterpret_cast<T*>(psi), items, a);
            return cudaGetLastError();
        }
    }
    k_diag<R, 1><<<grid_for((int64_t)ngroups, 256, d.num_sms, 8), 256, 0, s>>>(reinterpret_cast<T*>(psi), ngroups, a);
    return cudaGetLastError();
}

cudaError_t launch_diag(int dtype, void* psi, int n, int k, const int* targets, int nc, const int* controls,
                        const double* diag, const std::vector<int>& touch, cudaStream_t s, const DevInfo& d) {
    if (touch.empty()) return cudaSuccess;
    if (k > 6 || touch.size() > 64) return cudaErrorInvalidValue;
    const Fixed f = make_fixed(k, targets, nc, controls);
    if (dtype == QSIM_C64) return diag_t<float>(psi, n, k, targets, f, diag, touch, s, d);
    return diag_t<double>(psi, n, k, targets, f, diag, touch, s, d);
}

template <typename R, int K>
static cudaError_t dense_tile_t(void* psi, int n, const int* targets, const Fixed& f, const void* dmat,
                                cudaStream_t s, const DevInfo& d) {
    using T = typename Amp<R>::T;
    TileArgs a;
    std::memset(&a, 0, sizeof(a));
    a.nf = f.nf;
    std::memcpy(a.fixed, f.pos, sizeof(int) * f.nf);
    a.cmask = f.cmask;
    constexpr int D = 1 << K;
    for (int m = 0; m < D; ++m) a.off[m] = target_offset(m, K, targets);
    const size_t smem = (size_t)(D * D + D * 64) * sizeof(T);
    cudaError_t e = smem_optin(reinterpret_cast<const void*>(k_dense_tile<R, K>), (int)smem);
    if (e != cudaSuccess) return e;
    const uint64_t ngroups = 1ull << (n - f.nf);
    const uint64_t ntiles = (ngroups + 63) / 64;
    const int per_sm = smem > 100 * 1024 ? 1 : 3;
    k_dense_tile<R, K><<<grid_for((int64_t)ntiles, 1, d.num_sms, per_sm), 256, smem, s>>>(
        reinterpret_cast<T*>(psi), ngroups, a, reinterpret_cast<const T*>(dmat));
    return cudaGetLastError();
}

template <typename R, int K>
static cudaError_t dense_big_t(void* psi, int n, const int* targets, const Fixed& f, const void* dmat,
                               cudaStream_t s, const DevInfo& d) {
    using T = typename Amp<R>::T;
    BigArgs a;
    std::memset(&a, 0, sizeof(a));
    a.nf = f.nf;
    std::memcpy(a.fixed, f.pos, sizeof(int) * f.nf);
    a.cmask = f.cmask;
    std::memcpy(a.tpos, targets, sizeof(int) * K);
    const size_t smem = BigCfg<R, K>::smem;
    cudaError_t e = smem_optin(reinterpret_cast<const void*>(k_dense_big<R, K>), (int)smem);
    if (e != cudaSuccess) return e;
    const uint64_t ngroups = 1ull << (n - f.nf);
    const uint64_t nchunks = (ngroups + BigCfg<R, K>::G - 1) / BigCfg<R, K>::G;
    k_dense_big<R, K><<<grid_for((int64_t)nchunks, 1, d.num_sms, smem > 110 * 1024 ? 1 : 2), 256, smem, s>>>(
        reinterpret_cast<T*>(psi), ngroups, a, reinterpret_cast<const T*>(dmat));
    return cudaGetLastError();
}

cudaError_t launch_dense_tile(int dtype, void* psi, int n, int k, const int* targets, int nc,
                              const int* controls, const void* dmat, cudaStream_t s, const DevInfo& d) {
    const Fixed f = make_fixed(k, targets, nc, controls);
    if (k == 7 || k == 8) {
        if (dtype == QSIM_C64) return k == 7 ? dense_big_t<float, 7>(psi, n, targets, f, dmat, s, d)
                                             : dense_big_t<float, 8>(psi, n, targets, f, dmat, s, d);
        return k == 7 ? dense_big_t<double, 7>(psi, n, targets, f, dmat, s, d)
                      : dense_big_t<double, 8>(psi, n, targets, f, dmat, s, d);
    }
    if (dtype == QSIM_C64) {
        if (k == 5) return dense_tile_t<float, 5>(psi, n, targets, f, dmat, s, d);
        if (k == 6) return dense_tile_t<float, 6>(psi, n, targets, f, dmat, s, d);
    } else {
        if (k == 5) return dense_tile_t<double, 5>(psi, n, targets, f, dmat, s, d);
        if (k == 6) return dense_tile_t<double, 6>(psi, n, targets, f, dmat, s, d);
    }
    return cudaErrorInvalidValue;
}

// One swap pass: all pair bits must fit in a single tile.
template <typename R>
static cudaError_t swap_pass(void* psi, int n, const int* a, const int* b, int p, int max_tile_bits,
                             cudaStream_t s, const DevInfo& d, bool* fits) {
    using T = typename Amp<R>::T;
    bool inpair[64] = {false};
    int partner[64];
    for (int i = 0; i < p; ++i) {
        inpair[a[i]] = inpair[b[i]] = true;
        partner[a[i]] = b[i];
        partner[b[i]] = a[i];
    }
    // Choose L (contiguous low block) minimising the tile, preferring larger L at equal size.
    int bestL = -1, bestS = 1 << 30;
    const int Lmin = std::min(n, 4);
    for (int L = Lmin; L <= n; ++L) {
        int nS = L;
        for (int q = L; q < n; ++q) nS += inpair[q] ? 1 : 0;
        if (nS > max_tile_bits) continue;
        const int want = std::min(10, n);
        const int score = (nS < want ? want : nS);
        if (score < bestS || (score == bestS && L > bestL)) { bestS = score; bestL = L; }
    }
    if (bestL < 0) { *fits = false; return cudaSuccess; }
    *fits = true;
    SwapArgs sa;
    std::memset(&sa, 0, sizeof(sa));
    sa.L = bestL;
    int tb[64];  // index bit -> tile bit
    for (int q = 0; q < bestL; ++q) tb[q] = q;
    sa.nH = 0;
    for (int q = bestL; q < n; ++q)
        if (inpair[q]) { tb[q] = bestL + sa.nH; sa.hbits[sa.nH++] = q; }
    sa.nS = bestL + sa.nH;
    for (int bt = 0; bt < sa.nS; ++bt) {
        const int q = bt < bestL ? bt : sa.hbits[bt - bestL];
        sa.perm[bt] = inpair[q] ? tb[partner[q]] : bt;
    }
    const size_t smem = sizeof(T) << sa.nS;
    cudaError_t e = smem_optin(reinterpret_cast<const void*>(k_swap_tile<R>), (int)smem);
    if (e != cudaSuccess) return e;
    const uint64_t ntiles = 1ull << (n - sa.nS);
    const int per_sm = std::max(1, std::min(8, (int)((200 * 1024) / std::max<size_t>(smem, 1))));
    k_swap_tile<R><<<grid_for((int64_t)ntiles, 1, d.num_sms, per_sm), 256, smem, s>>>(
        reinterpret_cast<T*>(psi), ntiles, sa);
    return cudaGetLastError();
}

// Direct exchange of p <= 4 pairs whose bits are all >= minbit; false if not applicable.
template <typename R>
static bool swap_direct(void* psi, int n, const int* a, const int* b, int p, cudaStream_t s, const DevInfo& d,
                        cudaError_t* err) {
    using T = typename Amp<R>::T;
    if (p > 4) return false;
    SwapDirectArgs sa;
    std::memset(&sa, 0, sizeof(sa));
    int lo = 64;
    for (int i = 0; i < p; ++i) {
        sa.bits[sa.nb++] = a[i];
        sa.bits[sa.nb++] = b[i];
        lo = std::min(lo, std::min(a[i], b[i]));
    }
    const int minbit = sizeof(R) == 4 ? 4 : 3;  // runs of >= 128 bytes
    if (lo < minbit) return false;
    std::sort(sa.bits, sa.bits + sa.nb);
    // pattern u: bit 2i <-> a[i], bit 2i+1 <-> b[i]; sigma exchanges the two bits of every pair
    for (int u = 0; u < (1 << (2 * p)); ++u) {
        int v = 0;
        for (int i = 0; i < p; ++i) v |= (((u >> (2 * i)) & 1) << (2 * i + 1)) | (((u >> (2 * i + 1)) & 1) << (2 * i));
        if (u < v) {
            uint64_t ou = 0, ov = 0;
            for (int i = 0; i < p; ++i) {
                ou |= (uint64_t)((u >> (2 * i)) & 1) << a[i] | (uint64_t)((u >> (2 * i + 1)) & 1) << b[i];
                ov |= (uint64_t)((v >> (2 * i)) & 1) << a[i] | (uint64_t)((v >> (2 * i + 1)) & 1) << b[i];
            }
            sa.off_u[sa.npairs] = ou;
            sa.off_v[sa.npairs] = ov;
            ++sa.npairs;
        }
    }
    const uint64_t groups = 1ull << (n - sa.nb);
    if constexpr (sizeof(R) == 4) {
        const uint64_t gv = groups / 2;
        k_swap_direct<R, 2><<<grid_for((int64_t)(gv * sa.npairs), 256, d.num_sms, 8), 256, 0, s>>>(
            reinterpret_cast<T*>(psi), gv, sa);
    } else {
        k_swap_direct<R, 1><<<grid_for((int64_t)(groups * sa.npairs), 256, d.num_sms, 8), 256, 0, s>>>(
            reinterpret_cast<T*>(psi), groups, sa);
    }
    *err = cudaGetLastError();
    return true;
}

cudaError_t launch_swap(int dtype, void* psi, int n, const int* a, const int* b, int p, cudaStream_t s,
                        const DevInfo& d, int* passes) {
    {
        cudaError_t e = cudaSuccess;
        const bool done = dtype == QSIM_C64 ? swap_direct<float>(psi, n, a, b, p, s, d, &e)
                                            : swap_direct<double>(psi, n, a, b, p, s, d, &e);
        if (done) {
            if (passes) *passes = 1;
            return e;
        }
    }
    const int max_bits = dtype == QSIM_C64 ? 13 : 12;
    int done = 0, np = 0;
    while (done < p) {
        // Largest prefix of the remaining pairs that fits in one tile.
        int take = p - done;
        for (; take >= 1; --take) {
            bool fits = false;
            cudaError_t e = dtype == QSIM_C64
                ? swap_pass<float>(psi, n, a + done, b + done, take, max_bits, s, d, &fits)
                : swap_pass<double>(psi, n, a + done, b + done, take, max_bits, s, d, &fits);
            if (e != cudaSuccess) return e;
            if (fits) break;
        }
        if (take < 1) return cudaErrorInvalidValue;
        done += take;
        ++np;
    }
    if (passes) *passes = np;
    return cudaSuccess;
}

cudaError_t launch_set_basis(int dtype, void* psi, int n, uint64_t x, cudaStream_t s, const DevInfo& d) {
    const uint64_t N = 1ull << n;
    if (dtype == QSIM_C64)
        k_set_basis<float><<<grid_for((int64_t)N, 256, d.num_sms, 8), 256, 0, s>>>(reinterpret_cast<float2*>(psi), N, x);
    else
        k_set_basis<double><<<grid_for((int64_t)N, 256, d.num_sms, 8), 256, 0, s>>>(reinterpret_cast<double2*>(psi), N, x);
    return cudaGetLastError();
}

cudaError_t launch_convert_matrix(int dtype, const double* src, void* dst, int64_t count, cudaStream_t s) {
    if (dtype == QSIM_C128)
        return cudaMemcpyAsync(dst, src, (size_t)count * sizeof(double), cudaMemcpyDeviceToDevice, s);
    const int blocks = (int)std::min<int64_t>((count + 255) / 256, 1024);
    k_convert_matrix<<<std::max(1, blocks), 256, 0, s>>>(src, reinterpret_cast<float*>(dst), count);
    return cudaGetLastError();
}

}  // namespace qsim
