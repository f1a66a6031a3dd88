// k_tc7.cu -- a fused 7-qubit block on the tensor cores with FP16 split products (QSIM_PREC_FP16X3).
//
// Paper Sec. 2.1: fusion merges gates into one larger matrix; every fused block costs one read and one write
// of the state, so wider blocks mean fewer passes (the 30-qubit random brickwork of depth 40 needs 64
// blocks of 6 qubits but 49 of at most 7). Sec. 2.2 ties the useful fusion width to the arithmetic rate: at
// 7 qubits a block does 3072 tensor FLOP per amplitude in three FP16 products, 1.5 ms at 30 qubits at the
// FP16 rate, under the 2.5 ms it takes to stream the state once.
//
// Operands. A tile is 128 rows (the 7 lowest index bits outside the targets) by the 128 columns of the
// targets, and Y = X U^T per tile. The real form of U (256 x 256) would take 256 KiB of shared memory as two
// FP16 planes, more than a CTA has, so the real and imaginary parts of X are separate A operands (K = 128
// each). The output columns are cut in two halves h (columns 64h .. 64h + 63), each with an accumulator of
// 128 FP32 columns: [Im Y_h | Re Y_h]. B holds, per half, three 64-row blocks [Im U_h; Re U_h; -Im U_h]
// (U_h = rows 64h.. of U; 384 rows, 192 KiB as two planes), so that Re X multiplies the 128-row window
// starting at block 0 of its half and Im X the window starting at block 1, each an N = 128 MMA:
//     Im Y_h = Re X (Im U_h)^T + Im X (Re U_h)^T,   Re Y_h = Re X (Re U_h)^T + Im X (-Im U_h)^T.
// Scaling and split as in the 6-qubit FP16X3 block: amplitudes x 2^15, U x 2^14, each split into two FP16
// parts (here the leading 11 significant bits by Dekker's split, and the FP16 rounding of the remainder),
// products lo*hi + hi*lo + hi*hi, output x 2^-29.
//
// Tensor memory (512 columns, the whole of it): accumulator h at [128h, 128h + 128), A planes in [256, 512):
// plane p (0 hi, 1 lo), part (0 Re, 1 Im) at 256 + 128 p + 64 part, two FP16 values per column (even K in
// the low half). Per tile the MMAs of half 0 and of half 1 are committed separately, so that the drain of
// one half overlaps the MMAs of the other; the A planes are single-buffered, so the tensor cores wait only
// while a tile's A planes are written. Sequence of tile i (data warps, and the MMA issuer):
//   wait done1(i-1); write A(i); arrive full        issuer: wait full, MMAs of half 0, commit done0
//   drain half 1 of tile i-1; arrive free1          issuer: wait free1, MMAs of half 1, commit done1
//   load tile i+1 into registers (odd column groups before the half-1 drain, so that loads and stores of
//   different warps overlap); wait done0(i); drain half 0 of tile i, splitting tile i+1 into its packed
//   FP16 planes (in the registers it was loaded into) between the stores
// The loads and stores issue at the rate this SM's share of the HBM bandwidth drains them, so the data
// warps spend most of a tile in them; the MMAs of both halves run back to back while the warps drain half 1
// and load, and only the tensor-memory stores of A sit between one tile's MMAs and the next.
// The MMAs of a tile (3.6 us per SM at the measured FP16 rate) take less than the tile's share of the HBM
// time (5.9 us).
//
// Sixteen data warps (four per TMEM lane quadrant) and one warp whose lane 0 issues the MMAs (an issuing
// thread stalls until most of the MMAs it issued have run, so it has no other work), one CTA per SM
// (persistent over tiles); 17 warps leave 96 registers per thread. A thread owns one row of a tile and 16
// columns of each half; like the 6-qubit block its amplitudes move as 8-byte values, 16-byte pairs when
// qubit 0 is the first target, or 32-byte quads when qubits 0 and 1 are the first two. Every mbarrier wait is
// bounded (2 s); on expiry the kernel records DEVERR_TIMEOUT, waits once more (bounded) for its MMAs, frees
// its tensor memory and returns.
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "internal.h"
#include "tc_ptx.cuh"

namespace qsim {
namespace tc7 {

using namespace qsim::tc;

constexpr int K = 7, D = 1 << K;        // targets, complex columns of a tile
constexpr int H = D / 2;                // columns per output half
constexpr int kRowBits = 7;             // 128 rows per tile (MMA M = 128)
constexpr int NB = 3 * D;               // B rows: per half [Im U_h; Re U_h; -Im U_h]
constexpr int PB = NB * D * 2;          // bytes of one FP16 B plane (96 KiB)
constexpr int ATOM = NB * 128;          // one 128-byte K atom over all B rows
constexpr int kWarps = 16;                // data warps; warp 16 issues the MMAs
constexpr int kThreads = (kWarps + 1) * 32;
constexpr int CPH = H / 4;              // columns of each half per thread (4 warps per lane quadrant)
constexpr int CPT = 2 * CPH;            // complex columns per thread
constexpr uint32_t A0 = 2 * D;          // first A column in TMEM
constexpr uint32_t TCOLS = 512;
// kind::f16: FP32 accumulator, A and B FP16, K-major, N = 128, M = 128
constexpr uint32_t IDESC = (1u << 4) | ((uint32_t)(D >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
constexpr float kScaleX = 32768.0f;     // 2^15
constexpr double kScaleU = 16384.0;     // 2^14
constexpr float kOut = 1.0f / (32768.0f * 16384.0f);
constexpr int kBars = 5;                // full, free1, done0, done1, B loaded
constexpr size_t kSmem = 2 * (size_t)PB + sizeof(uint64_t) * D + 8 * kBars + 8 + 1024;

enum Mode { kRows = 0, kPairs = 1, kQuads = 2 };

struct Args {
    int nS;              // 14 index bits covered by a tile
    int spos[24];        // those bit positions, ascending
    int rpos[kRowBits];  // row bit j <-> index bit rpos[j]
    int tpos[K];         // column bit j <-> target j
    uint64_t ntiles;
    int from_basis;      // the input is |basis>, generated in registers instead of read
    uint64_t basis;
};

template <int MODE>
__global__ void __launch_bounds__(kThreads, 1)
k_tc7_block(float2* __restrict__ psi, const __grid_constant__ Args a, const uint4* __restrict__ bops,
            unsigned* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sb = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* sCol = reinterpret_cast<uint64_t*>(sb + 2 * PB);
    uint64_t* mbar = sCol + D;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + kBars);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int c = tid; c < D; c += kThreads) sCol[c] = deposit((uint64_t)c, a.tpos, K);
    if (tid == 0) {
        const int count[kBars] = {kWarps, kWarps, 1, 1, 1};
        for (int j = 0; j < kBars; ++j)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(mbar + j)), "r"(count[j]) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(tslot)), "r"(TCOLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tbase = *tslot;
    const uint32_t full = smem_u32(mbar + 0), free1 = smem_u32(mbar + 1), done0 = smem_u32(mbar + 2),
                   done1 = smem_u32(mbar + 3), bbar = smem_u32(mbar + 4);
    // programmatic dependent launch: the set-up above overlapped the previous kernel's tail
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (tid == 0) {
        constexpr uint32_t kChunk = 16384, kBytes = 2u * PB;
        static_assert(kBytes % kChunk == 0, "whole chunks");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bbar), "r"(kBytes) : "memory");
#pragma unroll 1
        for (uint32_t o = 0; o < kBytes; o += kChunk)
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         :: "r"(smem_u32(sb) + o), "l"(reinterpret_cast<const char*>(bops) + o), "r"(kChunk),
                            "r"(bbar) : "memory");
    }
    const uint32_t t0 = blockIdx.x, G = gridDim.x;  // (fewer than 2^32 tiles: checked by the host)
    const uint32_t m = t0 < a.ntiles ? (uint32_t)((a.ntiles - t0 + G - 1) / G) : 0u;  // tiles of this CTA
    auto tile = [&](uint32_t i) { return (uint64_t)t0 + (uint64_t)i * G; };

    // ---- MMA issue (lane 0 of warp 16) ----
    const uint64_t desc0 = sdesc_sw128(smem_u32(sb));
    const uint32_t dhi = (uint32_t)(desc0 >> 32);
    // The MMAs of output half h: products (A plane, B plane) lo*hi, hi*lo, hi*hi; Re X on the B window at
    // block 0 of the half, Im X on the window at block 1 (64 rows = 8 KiB further in every K atom); the first
    // MMA starts the half's accumulator.
    auto issue_half = [&](int h) {
        uint32_t dlo = (uint32_t)desc0, tb = tbase;
        asm volatile("" : "+r"(dlo), "+r"(tb));
        uint32_t acc = 0;
#pragma unroll
        for (int pr = 0; pr < 3; ++pr) {
            const int pa = pr == 0 ? 1 : 0, pb = pr == 1 ? 1 : 0;
#pragma unroll
            for (int part = 0; part < 2; ++part) {
                const uint32_t acol = tb + A0 + (uint32_t)(pa * D + part * (D / 2));
#pragma unroll
                for (int s = 0; s < D / 16; ++s) {
                    const uint32_t off = (uint32_t)(pb * PB + (s >> 2) * ATOM + (3 * H * h + H * part) * 128 + (s & 3) * 32);
                    mma_ts_lohi<true>(tb + (uint32_t)(D * h), acol + 8 * s, dlo + (off >> 4), dhi, IDESC, acc);
                    acc = 1;
                }
            }
        }
    };
    auto commit = [&](uint32_t bar) {
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(bar) : "memory");
    };
    bool b_ready = false;  // the MMA issuer has waited for B
    bool issued = false;   // MMAs issued; the last commit went to last_bar, phase last_par
    uint32_t last_bar = 0, last_par = 0;
    // ---- data movement (warps 0..15) ----
    const int quad = warp & 3, w4 = warp >> 2;
    const uint32_t tlane = (uint32_t)(quad * 32) << 16;
    float2* const prow = psi + deposit((uint64_t)(quad * 32 + lane), a.rpos, kRowBits);  // this thread's row
    // X[CPH * h + j] is column H h + CPH w4 + j. Column offsets are re-read from shared memory at each use
    // (one broadcast load) rather than held in 64-bit registers; the empty asm between accesses keeps those
    // reads next to their accesses.
    const volatile uint64_t* vCol = sCol + CPH * w4;
    auto col = [&](int x) { return vCol[(x / CPH) * H + x % CPH]; };

    auto load_tile = [&](float2 (&X)[CPT], uint64_t t) {
        const uint64_t b = insert_zeros(t, a.spos, a.nS);
        if (a.from_basis) {
            const uint64_t rb = b + deposit((uint64_t)(quad * 32 + lane), a.rpos, kRowBits);
#pragma unroll
            for (int x = 0; x < CPT; ++x) X[x] = make_float2(rb + col(x) == a.basis ? 1.0f : 0.0f, 0.0f);
        } else if constexpr (MODE == kQuads) {
#pragma unroll
            for (int x = 0; x < CPT; x += 4) {
                ld_v8(prow + b + col(x), X[x], X[x + 1], X[x + 2], X[x + 3]);
                asm volatile("" ::: "memory");
            }
        } else if constexpr (MODE == kPairs) {
#pragma unroll
            for (int x = 0; x < CPT; x += 2) {
                const float4 v = *reinterpret_cast<const float4*>(prow + b + col(x));
                X[x] = make_float2(v.x, v.y);
                X[x + 1] = make_float2(v.z, v.w);
                asm volatile("" ::: "memory");
            }
        } else {
#pragma unroll
            for (int x = 0; x < CPT; ++x) {
                X[x] = prow[b + col(x)];
                asm volatile("" ::: "memory");
            }
        }
    };
    // A planes of tile X, packed in place: the pair of columns (2q, 2q+1) of output half h's share, X[CPH h + 2q]
    // and X[CPH h + 2q + 1], becomes four 32-bit words (bits in the float2 fields): Re plane 0, Re plane 1, Im
    // plane 0, Im plane 1, each holding the two columns' FP16 values (2q in the low half). Plane 0 = the
    // scaled value's leading 11 significant bits, plane 1 = FP16 rounding of the remainder. Done before the wait for the
    // tensor memory they go to, between the stores of the drain that precedes it (which issue only as fast as
    // the memory system takes them).
    auto convert_pair = [&](float2 (&X)[CPT], int x) {
        {
            uint32_t w[4];
#pragma unroll
            for (int part = 0; part < 2; ++part) {
                const float e = (part ? X[x].y : X[x].x) * kScaleX, o = (part ? X[x + 1].y : X[x + 1].x) * kScaleX;
                // Dekker's split (Veltkamp's constant 2^13 + 1): the leading 11 significant bits, exact in FP16 for
                // scaled values from 2^-14 up, and the exact remainder, in FMA-pipe arithmetic (the _rn forms
                // are never contracted); only the packing to FP16 takes the conversion unit
                const float ce = __fmul_rn(e, 8193.0f), co = __fmul_rn(o, 8193.0f);
                const float he = __fsub_rn(ce, __fsub_rn(ce, e)), ho = __fsub_rn(co, __fsub_rn(co, o));
                uint32_t vh, vl;
                asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(vh) : "f"(ho), "f"(he));
                asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(vl) : "f"(__fsub_rn(o, ho)), "f"(__fsub_rn(e, he)));
                w[2 * part] = vh;
                w[2 * part + 1] = vl;
            }
            X[x] = make_float2(__uint_as_float(w[0]), __uint_as_float(w[1]));
            X[x + 1] = make_float2(__uint_as_float(w[2]), __uint_as_float(w[3]));
        }
    };
    auto convert = [&](float2 (&X)[CPT]) {
#pragma unroll
        for (int x = 0; x < CPT; x += 2) convert_pair(X, x);
    };
    auto store_a = [&](const float2 (&X)[CPT]) {
#pragma unroll
        for (int part = 0; part < 2; ++part)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t c = A0 + (uint32_t)(part * (D / 2) + (H * h + CPH * w4) / 2);
                uint32_t hi[CPH / 2], lo[CPH / 2];
#pragma unroll
                for (int q = 0; q < CPH / 2; ++q) {
                    const float2 v = X[CPH * h + 2 * q + part];
                    hi[q] = __float_as_uint(v.x);
                    lo[q] = __float_as_uint(v.y);
                }
                tmem_st<CPH / 2>(tbase + tlane + c, hi);
                tmem_st<CPH / 2>(tbase + tlane + D + c, lo);
            }
        wait_st();
    };
    // Half h of tile t's accumulator (Im Y at column 128 h + c', Re Y at 128 h + 64 + c'), scaled back and
    // stored in place; with cv, the pairs of X are converted (convert_pair), evenly between the stores.
    auto drain_half = [&](int h, uint64_t t, float2 (&X)[CPT], bool cv) {
        float2* const pt = prow + insert_zeros(t, a.spos, a.nS);
        constexpr int SPC = MODE == kQuads ? 2 : (MODE == kPairs ? 4 : 8);  // stores per chunk of 8 columns
        constexpr int PPS = (CPT / 2) / (SPC * (CPH / 8));                    // pairs converted per store
        auto after_store = [&](int k) {
            if (cv) {
#pragma unroll
                for (int p = 0; p < PPS; ++p) convert_pair(X, 2 * (k * PPS + p));
            }
        };
#pragma unroll
        for (int ch = 0; ch < CPH / 8; ++ch) {
            uint32_t re[8], im[8], v[16];
            const uint32_t c = (uint32_t)(D * h + CPH * w4 + 8 * ch);
            tmem_ld<8>(tbase + tlane + c, im);
            tmem_ld<8>(tbase + tlane + c + H, re);
            wait_ld();
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                v[2 * j] = __float_as_uint(__uint_as_float(re[j]) * kOut);
                v[2 * j + 1] = __float_as_uint(__uint_as_float(im[j]) * kOut);
            }
            const int x0 = CPH * h + 8 * ch;
            if constexpr (MODE == kQuads) {
#pragma unroll
                for (int j = 0; j < 8; j += 4) {
                    st_v8(pt + col(x0 + j), v + 2 * j);
                    asm volatile("" ::: "memory");
                    after_store(ch * SPC + j / 4);
                }
            } else if constexpr (MODE == kPairs) {
#pragma unroll
                for (int j = 0; j < 8; j += 2) {
                    *reinterpret_cast<float4*>(pt + col(x0 + j)) =
                        make_float4(__uint_as_float(v[2 * j]), __uint_as_float(v[2 * j + 1]),
                                    __uint_as_float(v[2 * j + 2]), __uint_as_float(v[2 * j + 3]));
                    asm volatile("" ::: "memory");
                    after_store(ch * SPC + j / 2);
                }
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    pt[col(x0 + j)] = make_float2(__uint_as_float(v[2 * j]), __uint_as_float(v[2 * j + 1]));
                    asm volatile("" ::: "memory");
                    after_store(ch * SPC + j);
                }
            }
        }
    };
    // one arrival per warp, after its TMEM accesses have completed
    auto arrive = [&](uint32_t bar) {
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(bar);
    };
    // warp-uniform bounded wait (the TMEM accesses that follow are .sync.aligned)
    auto wait = [&](uint32_t bar, uint32_t par) -> bool {
        const bool ok = !__any_sync(0xffffffffu, !mbar_wait_bounded(bar, par));
        fence_after();
        return ok;
    };

    bool bad = false;
    if (warp == kWarps) {
        // ---- MMA issuer: per tile, half 0 once every data warp has written the A planes, half 1 once every
        // data warp has drained half 1 of the previous tile ----
        if (lane == 0) {
            bad = !mbar_wait_bounded(bbar, 0);
            b_ready = true;
            if (bad) mbar_wait_bounded(bbar, 0);  // once more for the copy still in flight
            for (uint32_t i = 0; i < m && !bad; ++i) {
                const uint32_t pc = (uint32_t)(i & 1);
                for (int h = 0; h < 2 && !bad; ++h) {
                    if (!mbar_wait_bounded(h ? free1 : full, pc)) { bad = true; break; }
                    fence_after();
                    issue_half(h);
                    last_bar = h ? done1 : done0;
                    last_par = pc;
                    commit(last_bar);
                    issued = true;
                }
            }
            if (bad) {
                atomicOr(err, DEVERR_TIMEOUT);
                if (issued) mbar_wait_bounded(last_bar, last_par);  // the MMAs already issued
            }
        }
        __syncwarp();
    } else {
    float2 X[CPT];
    if (m > 0) {
        load_tile(X, t0);
        convert(X);
    }
    for (uint32_t i = 0; i < m; ++i) {
        const uint32_t pc = (uint32_t)(i & 1), pp = (uint32_t)((i - 1) & 1);
        if (i > 0 && !wait(done1, pp)) { bad = true; break; }  // A planes free, half 1 of tile i-1 final
        store_a(X);
        arrive(full);
        // warps of odd column groups load before draining half 1, the others after: loads and stores from
        // different warps overlap instead of every warp switching between them at once
        const bool early = (w4 & 1) != 0;
        if (early && i + 1 < m) load_tile(X, tile(i + 1));
        if (i > 0) drain_half(1, tile(i - 1), X, false);
        arrive(free1);
        if (!early && i + 1 < m) load_tile(X, tile(i + 1));  // in flight during the MMAs and the drain below
        if (!wait(done0, pc)) { bad = true; break; }
        drain_half(0, tile(i), X, i + 1 < m);      // converts tile i+1 between its stores
    }
    if (!bad && m > 0) {
        if (wait(done1, (uint32_t)((m - 1) & 1))) drain_half(1, tile(m - 1), X, false);
        else bad = true;
    }
    if (bad && lane == 0) atomicOr(err, DEVERR_TIMEOUT);
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tbase), "r"(TCOLS) : "memory");
    }
}

// B operand: row n = 192 h + 64 blk + i' holds, for output row i = 64 h + i' of U, Im U (blk 0), Re U (blk 1)
// or -Im U (blk 2) against input index c, scaled by 2^14 and split into two FP16 planes (value, residual), in
// the swizzled shared-memory byte layout.
__global__ void k_tc7_prepare(const double* __restrict__ U, unsigned char* __restrict__ out) {
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < NB * D; idx += gridDim.x * blockDim.x) {
        const int n = idx / D, c = idx % D;
        const int h = n / (3 * H), blk = (n % (3 * H)) / H, i = H * h + n % H;
        const double ur = U[2 * (i * D + c)], ui = U[2 * (i * D + c) + 1];
        const double w = kScaleU * (blk == 0 ? ui : (blk == 1 ? ur : -ui));
        const __half hv = __float2half_rn((float)w);
        const uint32_t off = sw128_offset(n, c, NB, 2);
        *reinterpret_cast<__half*>(out + off) = hv;
        *reinterpret_cast<__half*>(out + PB + off) = __float2half_rn((float)(w - (double)__half2float(hv)));
    }
}

}  // namespace tc7

size_t tc7_operand_bytes() { return 2 * (size_t)tc7::PB; }

cudaError_t launch_tc7_prepare(const double* dU, void* dB, cudaStream_t s) {
    const int blocks = (tc7::NB * tc7::D + 255) / 256;
    tc7::k_tc7_prepare<<<blocks, 256, 0, s>>>(dU, static_cast<unsigned char*>(dB));
    return cudaGetLastError();
}

cudaError_t launch_tc7_apply(void* psi, int n, const int* targets, const void* dB, unsigned* dev_err, cudaStream_t s,
                             const DevInfo& d, const uint64_t* from_basis) {
    if (n < tc7::K + tc7::kRowBits || n > 63 || (reinterpret_cast<uintptr_t>(dB) & 15) != 0 ||
        (reinterpret_cast<uintptr_t>(psi) & 15) != 0)
        return cudaErrorInvalidValue;
    tc7::Args a;
    std::memset(&a, 0, sizeof(a));
    uint64_t tmask = 0;
    for (int j = 0; j < tc7::K; ++j) {
        if (targets[j] < 0 || targets[j] >= n || ((tmask >> targets[j]) & 1)) return cudaErrorInvalidValue;
        a.tpos[j] = targets[j];
        tmask |= 1ull << targets[j];
    }
    int nr = 0;
    for (int q = 0; q < n && nr < tc7::kRowBits; ++q)
        if (!((tmask >> q) & 1)) a.rpos[nr++] = q;
    uint64_t smask = tmask;
    for (int j = 0; j < tc7::kRowBits; ++j) smask |= 1ull << a.rpos[j];
    for (int q = 0; q < n; ++q)
        if ((smask >> q) & 1) a.spos[a.nS++] = q;
    a.ntiles = 1ull << (n - a.nS);
    if (a.ntiles >> 32) return cudaErrorInvalidValue;  // 32-bit tile counters in the kernel
    if (from_basis) {
        a.from_basis = 1;
        a.basis = *from_basis;
    }
    const unsigned grid = (unsigned)std::min<uint64_t>((uint64_t)d.num_sms, a.ntiles);
    auto launch = [&](auto kern) -> cudaError_t {
        cudaError_t e = smem_optin(reinterpret_cast<const void*>(kern), (int)tc7::kSmem);
        if (e != cudaSuccess) return e;
        // programmatic dependent launch, as for the 6-qubit block (griddepcontrol.wait before any access)
        cudaLaunchConfig_t cfg{};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.gridDim = dim3(grid, 1, 1);
        cfg.blockDim = dim3(tc7::kThreads, 1, 1);
        cfg.dynamicSmemBytes = tc7::kSmem;
        cfg.stream = s;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, kern, reinterpret_cast<float2*>(psi), a, reinterpret_cast<const uint4*>(dB),
                                  dev_err);
    };
    if (a.tpos[0] == 0 && a.tpos[1] == 1 && (reinterpret_cast<uintptr_t>(psi) & 31) == 0)
        return launch(tc7::k_tc7_block<tc7::kQuads>);
    if (a.tpos[0] == 0) return launch(tc7::k_tc7_block<tc7::kPairs>);
    return launch(tc7::k_tc7_block<tc7::kRows>);
}

}  // namespace qsim
