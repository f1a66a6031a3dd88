// k_tc_pair.cu -- two fused 6-qubit blocks applied in one pass over the state, on the tensor cores.
//
// Paper Sec. 2.1: fusion raises arithmetic intensity; each pass over the 2^n amplitudes costs a full read and
// write of the state, so applying two consecutive fused blocks while their amplitudes are on chip halves the
// memory traffic of the pair. Blocks U1 (targets T1) and then U2 (targets T2) with |T1 u T2| <= 12 share a
// tile of 13 index bits S (T1 u T2 plus the lowest other qubits): 8192 amplitudes, read once and written once.
//
// Per tile (one CTA per SM, 16 data warps + 1 MMA-issuing warp):
//   1. The data warps load the tile as X[r1][c1] -- rows r1 over the 7 bits R1 = S \ T1 (TMEM lanes), columns
//      over T1 -- and store its FP16 planes (below) in tensor memory as the A operand.
//   2. MMA 1: D1 = A1 . B1^T with B1 the real form of U1 in shared memory: D1[r1][i] = (U1 x_{r1})_i.
//   3. The data warps read D1 and write it into shared memory as the B operand of the second product, with
//      the roles of the bits exchanged: row n2 over R2 = S \ T2, K over T2 (x its real / imaginary part). This
//      is where the tile changes which of its bits are rows, without a separate transpose.
//   4. MMA 2: D2 = A2 . B2^T with A2 the real form of U2 in shared memory: D2[2i + ro][n2] = part ro of
//      (U2 y_{n2})_i. The data warps pair real and imaginary parts (adjacent lanes, one shuffle each) and
//      store the amplitudes back in place.
// Numbers: FP16 split products with FP32 accumulation. An amplitude of a normalised state has |a| <= 1, so
// every operand value is scaled by a fixed power of two (2^15 for amplitudes, 2^14 for matrix entries) and
// split into hi = fp16(v) and lo = fp16(v - hi): 22 significant bits for values down to 2^-17 of the
// largest possible one, and an absolute error of 2^-40 below that; the three products hi.hi + hi.lo + lo.hi
// give 3xTF32-level accuracy at the FP16 tensor rate (FP16 runs at twice the TF32 rate), and two blocks'
// operands fit in shared memory (2 x 64 KiB, where TF32 planes would need 2 x 128 KiB).
// Every mbarrier wait is bounded (2 s); on expiry the kernel records DEVERR_TIMEOUT, waits once more for
// the MMAs it issued, frees its tensor memory and returns.
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "internal.h"
#include "tc_ptx.cuh"

namespace qsim {
namespace tcp {

using namespace qsim::tc;

constexpr int kTileBits = 13;
constexpr int kRowBits = 7;
constexpr int kDataWarps = 16;                    // four per TMEM lane quadrant
constexpr int kCPT = 64 / (kDataWarps / 4);       // complex columns of the first product per thread (16)
constexpr int kNPT = 128 / (kDataWarps / 4);      // accumulator columns of the second product per thread (32)
constexpr int kDataThreads = kDataWarps * 32;
constexpr int kThreads = (kDataWarps + 1) * 32;
constexpr int kPlane = 128 * 128 * 2;             // one FP16 plane of a 128 x 128 real-form operand (32 KiB)
constexpr int kAtom = 128 * 128;                  // bytes of one 128-byte-wide K atom of a 128-row operand
constexpr int kKSteps = 8;                        // 128 K values / 16 per MMA
constexpr float kScaleX = 32768.0f;               // 2^15: amplitudes into the FP16 range
constexpr double kScaleU = 16384.0;               // 2^14: matrix entries
constexpr float kX1toX2 = 1.0f / 16384.0f;        // D1 (2^29 x value) -> 2^15 x value
constexpr float kOut = 1.0f / (32768.0f * 16384.0f);  // D2 -> value
// shared memory: [B1 hi, lo][A2 hi, lo][B2 hi, lo] (1024-aligned), then tables and barriers
constexpr int kOffB1 = 0, kOffA2 = 2 * kPlane, kOffB2 = 4 * kPlane, kOffTab = 6 * kPlane;

struct PairArgs {
    int spos[kTileBits];  // tile bits, ascending (zeros inserted there form a tile's base index)
    int r1pos[kRowBits];  // R1 = S \ T1, ascending: row bit j of the first product
    int t1pos[6];         // T1 in U1's index order
    int t2pos[6];         // T2 in U2's index order
    int r2pos[kRowBits];  // R2 = S \ T2, ascending
    // where each bit of (r1, i1) goes in the second product's coordinates: < 8: bit of t2; >= 8: bit
    // (value - 8) of n2
    uint8_t r1_to[kRowBits];
    uint8_t t1_to[6];
    // output staging: amplitude at tile index t (13 bits, S order) goes to the 8-byte word t ^ f(t >> 4) of
    // the staging buffer, f linear with f(bit j) = fmask[j]: chosen per pair so that the scattered writes of
    // a warp fall in distinct bank groups
    uint8_t t2s[6];       // position in S of t2pos[j]
    uint8_t r2s[kRowBits];// position in S of r2pos[j]
    uint8_t fmask[kTileBits - 4];
    uint64_t ntiles;
    int from_basis;
    uint64_t basis;
};

// Byte offset of element (row, kk) of a 128-row FP16 K-major operand in the SWIZZLE_128B layout.
__host__ __device__ inline uint32_t sw128_f16(int row, int kk) {
    const int atom = kk >> 6, b = (kk & 63) * 2;
    const int chunk = b >> 4, within = b & 15, g = row >> 3, r8 = row & 7;
    return (uint32_t)(atom * kAtom + g * 1024 + r8 * 128 + ((chunk ^ r8) << 4) + within);
}

// Real form of U (64 x 64 complex, FP64, row-major interleaved) as a 128 x 128 K-major operand, scaled by 2^14,
// split into FP16 hi / lo planes: R[2i + ro][2c + ri] = (ro, ri) = (0,0): Re U_ic, (0,1): -Im U_ic,
// (1,0): Im U_ic, (1,1): Re U_ic.
__global__ void k_tcp_prepare(const double* __restrict__ U, unsigned char* __restrict__ out) {
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < 128 * 128; idx += gridDim.x * blockDim.x) {
        const int row = idx >> 7, kk = idx & 127;
        const int i = row >> 1, ro = row & 1, c = kk >> 1, ri = kk & 1;
        const double ur = U[2 * (i * 64 + c)], ui = U[2 * (i * 64 + c) + 1];
        const double v = kScaleU * (ro == 0 ? (ri == 0 ? ur : -ui) : (ri == 0 ? ui : ur));
        const __half hi = __float2half_rn((float)v);
        const __half lo = __float2half_rn((float)(v - (double)__half2float(hi)));
        const uint32_t off = sw128_f16(row, kk);
        *reinterpret_cast<__half*>(out + off) = hi;
        *reinterpret_cast<__half*>(out + kPlane + off) = lo;
    }
}

// (re, im) scaled amplitude -> FP16 hi and lo pairs, packed with the real part in the low half.
__device__ __forceinline__ void split_f16x2(float re, float im, uint32_t& hi, uint32_t& lo) {
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(im), "f"(re));
    const float2 h = __half22float2(*reinterpret_cast<const __half2*>(&hi));
    const float rr = re - h.x, ri = im - h.y;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(ri), "f"(rr));
}

// MMA with both operands in shared memory (descriptors given as 32-bit halves).
__device__ __forceinline__ void mma_ss_f16(uint32_t d_tmem, uint32_t a_lo, uint32_t a_hi, uint32_t b_lo, uint32_t b_hi,
                                           uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t.reg .b64 ad, bd;\n\tsetp.ne.b32 p, %6, 0;\n\tmov.b64 ad, {%1, %2};\n\t"
        "mov.b64 bd, {%3, %4};\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], ad, bd, %5, p;\n}"
        :: "r"(d_tmem), "r"(a_lo), "r"(a_hi), "r"(b_lo), "r"(b_hi), "r"(idesc), "r"(acc) : "memory");
}

__device__ __forceinline__ void commit_to(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(bar) : "memory");
}

// TMEM: two slots of 256 columns; slot s holds A1 hi (cols 0..63), A1 lo (64..127) and the accumulator
// (128..255), which MMA 1 and MMA 2 use in turn. A tile j lives in slot j & 1 from its load to its store.
__global__ void __launch_bounds__(kThreads, 1)
k_tc_pair(float2* __restrict__ psi, const __grid_constant__ PairArgs a, const uint4* __restrict__ ops,
          unsigned* __restrict__ err) {
    constexpr uint32_t IDESC = (1u << 4) | ((uint32_t)(128 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);  // F16 in, F32 out
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sb = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* sCol1 = reinterpret_cast<uint64_t*>(sb + kOffTab);  // [64] index offset of T1 column c
    uint64_t* sDepLo = sCol1 + 64;                                // [512] index offset of tile bits 0..8
    uint64_t* sDepHi = sDepLo + 512;                              // [16] index offset of tile bits 9..12
    uint32_t* sP2 = reinterpret_cast<uint32_t*>(sDepHi + 16);     // [64] T1 column c: B2 byte offset part | xor part << 16
    uint32_t* sStN2 = sP2 + 64;                                   // [128] staging word part of R2 column n2
    uint32_t* sFj = sStN2 + 128;                                  // [16] f of tile bits 9..12
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sFj + 16);       // full1[2] done1[2] full2 done2[2] bops
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 8);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    auto fswz = [&](uint32_t hi9) {  // f of tile bits 4..12 (given shifted down by 4)
        uint32_t f = 0;
        for (int b = 0; b < kTileBits - 4; ++b) if ((hi9 >> b) & 1) f ^= a.fmask[b];
        return f;
    };
    // B2 byte offset of (n2, t2) = additive part + ((xor part) << 4): the SWIZZLE_128B offset of element
    // (n2, 2 t2) splits over disjoint bit sets of (n2, t2), and the row's and the column's parts combine so
    // (the 16-byte chunk index is t2 bits 2..4 XOR n2 bits 0..2)
    auto b2part = [](uint32_t n2, uint32_t t2, uint32_t& add, uint32_t& x) {
        add = (t2 >> 5) * (uint32_t)kAtom + (n2 >> 3) * 1024u + (n2 & 7u) * 128u + 4u * (t2 & 3u);
        x = ((t2 >> 2) & 7u) ^ (n2 & 7u);
    };
    for (int c = tid; c < 64; c += kThreads) {
        sCol1[c] = deposit((uint64_t)c, a.t1pos, 6);
        uint32_t t2 = 0, n2 = 0;
        for (int j = 0; j < 6; ++j)
            if ((c >> j) & 1) { if (a.t1_to[j] < 8) t2 |= 1u << a.t1_to[j]; else n2 |= 1u << (a.t1_to[j] - 8); }
        uint32_t add, x;
        b2part(n2, t2, add, x);
        sP2[c] = add | (x << 16);
    }
    for (int c = tid; c < 512; c += kThreads) sDepLo[c] = deposit((uint64_t)c, a.spos, 9);
    for (int c = tid; c < 16; c += kThreads) {
        sDepHi[c] = deposit((uint64_t)c, a.spos + 9, kTileBits - 9);
        sFj[c] = fswz((uint32_t)c << 5);
    }
    for (int c = tid; c < 128; c += kThreads) {
        uint32_t t = 0;
        for (int j = 0; j < kRowBits; ++j) if ((c >> j) & 1) t |= 1u << a.r2s[j];
        sStN2[c] = t ^ fswz(t >> 4);
    }
    if (tid == 0) {
        for (int j = 0; j < 8; ++j) {
            const uint32_t cnt = (j < 2 || j == 4) ? kDataWarps : 1;  // full1[0..1], full2: one arrival per data warp
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(mbar + j)), "r"(cnt) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(tslot)), "r"(512) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tbase = *tslot;
    const uint32_t bar0 = smem_u32(mbar);
    auto full1 = [&](int s) { return bar0 + 8u * (uint32_t)s; };
    auto done1 = [&](int s) { return bar0 + 8u * (uint32_t)(2 + s); };
    const uint32_t full2 = bar0 + 8u * 4;
    auto done2 = [&](int s) { return bar0 + 8u * (uint32_t)(5 + s); };
    const uint32_t bbar = bar0 + 8u * 7;
    // a programmatic dependent of the kernel before it: its writes are visible from here on
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (tid == 0) {  // B1 and A2 planes (prepared in the swizzled byte layout): four 32 KiB bulk copies
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bbar), "r"(4 * kPlane) : "memory");
        for (int q = 0; q < 4; ++q)
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         :: "r"(smem_u32(sb) + q * kPlane), "l"(reinterpret_cast<const char*>(ops) + q * kPlane),
                            "r"(kPlane), "r"(bbar) : "memory");
    }
    const uint64_t t0 = blockIdx.x, G = gridDim.x;
    const uint64_t m = t0 < a.ntiles ? (a.ntiles - t0 + G - 1) / G : 0;

    if (warp == kDataWarps) {
        // ---- MMA issuer: MMA 1 of tile i, then MMA 2 of tile i - 1 ----
        if (lane == 0) {
            const uint64_t dB1 = sdesc_sw128(smem_u32(sb + kOffB1)), dA2 = sdesc_sw128(smem_u32(sb + kOffA2)),
                           dB2 = sdesc_sw128(smem_u32(sb + kOffB2));
            const uint32_t hiB1 = (uint32_t)(dB1 >> 32), hiA2 = (uint32_t)(dA2 >> 32), hiB2 = (uint32_t)(dB2 >> 32);
            auto mma1 = [&](int s) {
                uint32_t lo = (uint32_t)dB1, tb = tbase;
                asm volatile("" : "+r"(lo), "+r"(tb));
                const uint32_t d = tb + 256u * s + 128u, aHi = tb + 256u * s, aLo = aHi + 64u;
                uint32_t acc = 0;
#pragma unroll
                for (int pr = 0; pr < 3; ++pr) {  // lo.hi, hi.lo, hi.hi: small products first
                    const uint32_t at = pr == 0 ? aLo : aHi;
                    const uint32_t bp = pr == 1 ? (uint32_t)kPlane : 0u;
#pragma unroll
                    for (int k = 0; k < kKSteps; ++k) {
                        const uint32_t off = bp + (uint32_t)((k >> 2) * kAtom + (k & 3) * 32);
                        mma_ts_lohi<true>(d, at + 8u * k, lo + (off >> 4), hiB1, IDESC, acc);
                        acc = 1;
                    }
                }
            };
            auto mma2 = [&](int s) {
                uint32_t la = (uint32_t)dA2, lb = (uint32_t)dB2, tb = tbase;
                asm volatile("" : "+r"(la), "+r"(lb), "+r"(tb));
                const uint32_t d = tb + 256u * s + 128u;
                uint32_t acc = 0;
#pragma unroll
                for (int pr = 0; pr < 3; ++pr) {  // U lo . y hi, U hi . y lo, U hi . y hi
                    const uint32_t ap = pr == 0 ? (uint32_t)kPlane : 0u, bp = pr == 1 ? (uint32_t)kPlane : 0u;
#pragma unroll
                    for (int k = 0; k < kKSteps; ++k) {
                        const uint32_t off = (uint32_t)((k >> 2) * kAtom + (k & 3) * 32);
                        mma_ss_f16(d, la + ((ap + off) >> 4), hiA2, lb + ((bp + off) >> 4), hiB2, IDESC, acc);
                        acc = 1;
                    }
                }
            };
            uint32_t last_bar = 0, last_par = 0;
            bool bad = !mbar_wait_bounded(bbar, 0);
            if (bad) mbar_wait_bounded(bbar, 0);  // once more for the copy in flight
            for (uint64_t i = 0; i <= m && !bad; ++i) {
                if (i < m) {
                    const int s = (int)(i & 1);
                    if (!mbar_wait_bounded(full1(s), (uint32_t)((i >> 1) & 1))) { bad = true; break; }
                    fence_after();
                    mma1(s);
                    commit_to(done1(s));
                    last_bar = done1(s);
                    last_par = (uint32_t)((i >> 1) & 1);
                }
                if (i >= 1) {
                    const uint64_t j = i - 1;
                    const int s = (int)(j & 1);
                    if (!mbar_wait_bounded(full2, (uint32_t)(j & 1))) { bad = true; break; }
                    fence_after();
                    mma2(s);
                    commit_to(done2(s));
                    last_bar = done2(s);
                    last_par = (uint32_t)((j >> 1) & 1);
                }
            }
            if (bad) {
                atomicOr(err, DEVERR_TIMEOUT);
                if (last_bar) mbar_wait_bounded(last_bar, last_par);  // the latest commit tracks every MMA issued
            }
        }
        __syncwarp();
    } else {
        // ---- data warps: thread = TMEM lane r of its quadrant; four warps per quadrant split the columns ----
        const int quad = warp & 3, grp = warp >> 2;
        const int r = quad * 32 + lane;
        const uint32_t tlane = (uint32_t)(quad * 32) << 16;
        const int c0 = grp * kCPT;  // first-product columns c0 .. c0 + 15
        const uint64_t rowoff1 = deposit((uint64_t)r, a.r1pos, kRowBits);
        uint32_t t2r = 0, n2r = 0;  // this row's bits in the second product's coordinates
        for (int j = 0; j < kRowBits; ++j)
            if ((r >> j) & 1) { if (a.r1_to[j] < 8) t2r |= 1u << a.r1_to[j]; else n2r |= 1u << (a.r1_to[j] - 8); }
        uint32_t addr_r, xr;
        b2part(n2r, t2r, addr_r, xr);
        const int ro = r & 1;
        uint32_t wi2 = 0;  // staging word part of this lane's output row i2 = r / 2
        for (int j = 0; j < 6; ++j) if (((r >> 1) >> j) & 1) wi2 |= 1u << a.t2s[j];
        wi2 ^= fswz(wi2 >> 4);
        const int k = tid;  // 0..511: this thread's staging reads are tile indices k + 512 jj
        const uint64_t deplo = sDepLo[k];
        const uint32_t fk = fswz((uint32_t)k >> 4);
        const volatile uint64_t* vCol = sCol1 + c0;
        const uint32_t sB2 = smem_u32(sb + kOffB2);
        auto wait = [&](uint32_t bar, uint32_t par) -> bool {
            const bool ok = !__any_sync(0xffffffffu, !mbar_wait_bounded(bar, par));
            fence_after();
            return ok;
        };
        auto data_sync = [&]() { asm volatile("bar.sync 1, %0;" :: "r"(kDataThreads) : "memory"); };
        float2 X[kCPT];
        auto load = [&](uint64_t t) {
            const uint64_t b = insert_zeros(t, a.spos, kTileBits) + rowoff1;
#pragma unroll
            for (int j = 0; j < kCPT; ++j) {
                const uint64_t o = b + vCol[j];
                X[j] = a.from_basis ? make_float2(o == a.basis ? 1.0f : 0.0f, 0.0f) : psi[o];
                asm volatile("" ::: "memory");
            }
        };
        // FP16 planes of the tile in X into A1 of slot s (arrival on full1[s] comes later: the slot's
        // accumulator may still hold the previous tile's output)
        auto p1_write = [&](int s) {
            uint32_t hi[kCPT], lo[kCPT];
#pragma unroll
            for (int j = 0; j < kCPT; ++j) split_f16x2(X[j].x * kScaleX, X[j].y * kScaleX, hi[j], lo[j]);
            tmem_st_x16(tbase + tlane + 256u * s + (uint32_t)c0, hi);
            tmem_st_x16(tbase + tlane + 256u * s + 64u + (uint32_t)c0, lo);
            wait_st();
        };
        auto p1_arrive = [&](int s) {
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(full1(s));
        };
        // D1 of slot s into the B operand of the second product (rows n2, K = 2 t2 + part)
        auto p2 = [&](int s, uint32_t par) -> bool {
            if (!wait(done1(s), par)) return false;
            uint32_t v[2 * kCPT];
            tmem_ld_x32(tbase + tlane + 256u * s + 128u + 2u * c0, v);
            wait_ld();
#pragma unroll
            for (int j = 0; j < kCPT; ++j) {
                const uint32_t mp = sP2[c0 + j];
                const uint32_t off = addr_r + (mp & 0xFFFFu) + ((xr ^ (mp >> 16)) << 4);
                uint32_t hi, lo;
                split_f16x2(__uint_as_float(v[2 * j]) * kX1toX2, __uint_as_float(v[2 * j + 1]) * kX1toX2, hi, lo);
                asm volatile("st.shared.u32 [%0], %1;" :: "r"(sB2 + off), "r"(hi) : "memory");
                asm volatile("st.shared.u32 [%0], %1;" :: "r"(sB2 + (uint32_t)kPlane + off), "r"(lo) : "memory");
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor-core reads
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(full2);
            return true;
        };
        // D2 of slot s to the state: real and imaginary parts paired across adjacent lanes, staged in tile
        // order in the (now free) B2 buffer, then stored in tile order so that a warp writes the longest
        // contiguous runs the tile has
        auto p3 = [&](int s, uint32_t par, uint64_t t) -> bool {
            if (!wait(done2(s), par)) return false;
            uint32_t w[kNPT];
            tmem_ld_x32(tbase + tlane + 256u * s + 128u + (uint32_t)(kNPT * grp), w);
            wait_ld();
            fence_before();
            constexpr int H = kNPT / 2;
            const int nb = kNPT * grp + (ro ? H : 0);  // this lane's 16 columns after the exchange
#pragma unroll
            for (int j = 0; j < H; ++j) {
                const float mine = __uint_as_float(ro ? w[H + j] : w[j]);
                const float got = __shfl_xor_sync(0xffffffffu, __uint_as_float(ro ? w[j] : w[H + j]), 1);
                const float re = ro ? got : mine, im = ro ? mine : got;
                const uint32_t word = wi2 ^ sStN2[nb + j];
                asm volatile("st.shared.v2.f32 [%0], {%1, %2};" :: "r"(sB2 + 8u * word), "f"(re * kOut), "f"(im * kOut)
                             : "memory");
            }
            data_sync();
            const uint64_t b = insert_zeros(t, a.spos, kTileBits) + deplo;
#pragma unroll 8
            for (int jj = 0; jj < 16; ++jj) {
                const uint32_t word = ((uint32_t)(k + 512 * jj)) ^ (fk ^ sFj[jj]);
                float2 y;
                asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(y.x), "=f"(y.y) : "r"(sB2 + 8u * word) : "memory");
                psi[b + sDepHi[jj]] = y;
            }
            data_sync();  // the staging buffer is the next tile's B2
            return true;
        };
        // Tile j lives in TMEM slot j & 1. Per iteration: finish MMA 1 of tile j (p2), fill tile j + 2's A1
        // while MMA 2 of tile j runs, store tile j (p3), then release slot j & 1 to tile j + 2.
        bool bad = false;
        for (uint64_t j = 0; j < 2 && j < m; ++j) {
            load(t0 + j * G);
            p1_write((int)j);
            p1_arrive((int)j);
        }
        if (m > 2) load(t0 + 2 * G);
        for (uint64_t j = 0; j < m && !bad; ++j) {
            const int s = (int)(j & 1);
            const uint32_t par = (uint32_t)((j >> 1) & 1);
            if (!p2(s, par)) { bad = true; break; }
            if (j + 2 < m) p1_write(s);
            if (!p3(s, par, t0 + j * G)) { bad = true; break; }
            if (j + 2 < m) {
                p1_arrive(s);
                if (j + 3 < m) load(t0 + (j + 3) * G);
            }
        }
        if (bad && lane == 0) atomicOr(err, DEVERR_TIMEOUT);
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tbase), "r"(512) : "memory");
    }
}

}  // namespace tcp

// ---- host side --------------------------------------------------------------------------------------------
namespace {

// The tile of a pair: T1 u T2 plus the lowest other qubits up to 13 bits. false if the pair does not fit.
bool pair_geometry(int n, const int* t1, const int* t2, tcp::PairArgs& a) {
    if (n < tcp::kTileBits) return false;
    uint64_t m1 = 0, m2 = 0;
    for (int j = 0; j < 6; ++j) { m1 |= 1ull << t1[j]; m2 |= 1ull << t2[j]; }
    if (__builtin_popcountll(m1) != 6 || __builtin_popcountll(m2) != 6) return false;
    uint64_t S = m1 | m2;
    if (__builtin_popcountll(S) > 12) return false;
    for (int q = 0; q < n && __builtin_popcountll(S) < tcp::kTileBits; ++q) S |= 1ull << q;
    std::memset(&a, 0, sizeof(a));
    int ns = 0, n1 = 0, n2 = 0;
    for (int q = 0; q < n; ++q) {
        if (!((S >> q) & 1)) continue;
        a.spos[ns++] = q;
        if (!((m1 >> q) & 1)) a.r1pos[n1++] = q;
        if (!((m2 >> q) & 1)) a.r2pos[n2++] = q;
    }
    for (int j = 0; j < 6; ++j) { a.t1pos[j] = t1[j]; a.t2pos[j] = t2[j]; }
    // where a qubit lands in the second product: bit j of t2 (< 8), or bit j of n2 (8 + j)
    auto to2 = [&](int q) -> uint8_t {
        for (int j = 0; j < 6; ++j) if (a.t2pos[j] == q) return (uint8_t)j;
        for (int j = 0; j < tcp::kRowBits; ++j) if (a.r2pos[j] == q) return (uint8_t)(8 + j);
        return 0xFF;
    };
    for (int j = 0; j < tcp::kRowBits; ++j) a.r1_to[j] = to2(a.r1pos[j]);
    for (int j = 0; j < 6; ++j) a.t1_to[j] = to2(a.t1pos[j]);
    auto in_s = [&](int q) -> uint8_t {
        for (int j = 0; j < tcp::kTileBits; ++j) if (a.spos[j] == q) return (uint8_t)j;
        return 0xFF;
    };
    for (int j = 0; j < 6; ++j) a.t2s[j] = in_s(a.t2pos[j]);
    for (int j = 0; j < tcp::kRowBits; ++j) a.r2s[j] = in_s(a.r2pos[j]);
    // The staging writes of a half-warp (8-byte accesses are served per half-warp) vary, per lane bit 0..3,
    // in tile bits: n2 bit 4 (which half of a thread's columns), then t2 bits 0..2 (lane bit 4, t2 bit 3,
    // only separates the half-warps). Tile bits 0..3 index bank groups directly; each higher one of these
    // four gets a unit vector the lower ones leave free, so the 16 lanes hit 16 different bank groups.
    const int vary[4] = {a.r2s[4], a.t2s[0], a.t2s[1], a.t2s[2]};
    unsigned used = 0;
    for (int v : vary) if (v < 4) used |= 1u << v;
    for (int v : vary) {
        if (v < 4) continue;
        int unit = -1;
        for (int u = 0; u < 4 && unit < 0; ++u) if (!((used >> u) & 1)) unit = u;
        if (unit >= 0) { a.fmask[v - 4] = (uint8_t)(1u << unit); used |= 1u << unit; }
    }
    a.ntiles = 1ull << (n - tcp::kTileBits);
    return true;
}

}  // namespace

bool tc_pair_supported(int n, const int* t1, int k1, const int* t2, int k2) {
    tcp::PairArgs a;
    return k1 == 6 && k2 == 6 && pair_geometry(n, t1, t2, a);
}

size_t tc_pair_operand_bytes() { return 4 * (size_t)tcp::kPlane; }

cudaError_t launch_tc_pair_prepare(const double* dU1, const double* dU2, void* dops, cudaStream_t s) {
    unsigned char* out = static_cast<unsigned char*>(dops);
    tcp::k_tcp_prepare<<<64, 256, 0, s>>>(dU1, out);
    tcp::k_tcp_prepare<<<64, 256, 0, s>>>(dU2, out + 2 * tcp::kPlane);
    return cudaGetLastError();
}

cudaError_t launch_tc_pair(void* psi, int n, const int* t1, const int* t2, const void* dops, unsigned* dev_err,
                           cudaStream_t s, const DevInfo& d, const uint64_t* from_basis) {
    tcp::PairArgs a;
    if (!pair_geometry(n, t1, t2, a)) return cudaErrorInvalidValue;
    if ((reinterpret_cast<uintptr_t>(dops) & 15) != 0) return cudaErrorInvalidValue;
    if (from_basis) { a.from_basis = 1; a.basis = *from_basis; }
    // operands, tables and barriers; at least 120 KiB, so that one CTA (one TMEM owner) runs per SM
    const size_t smem = std::max<size_t>((size_t)tcp::kOffTab + (64 + 512 + 16) * 8 + (64 + 128 + 16) * 4 + 8 * 8 + 16 + 1024,
                                         120 * 1024);
    cudaError_t e = cudaFuncSetAttribute(tcp::k_tc_pair, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.gridDim = dim3((unsigned)std::min<uint64_t>((uint64_t)d.num_sms, a.ntiles), 1, 1);
    cfg.blockDim = dim3(tcp::kThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, tcp::k_tc_pair, reinterpret_cast<float2*>(psi), a,
                              reinterpret_cast<const uint4*>(dops), dev_err);
}

}  // namespace qsim
