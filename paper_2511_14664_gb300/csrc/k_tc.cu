// k_tc.cu -- a fused dense block on the 5th-generation tensor cores (tcgen05) with split precision.
//
// Paper Sec. 2.1: fusion merges gates into one larger matrix, which raises arithmetic intensity and moves
// the work from bandwidth-bound towards balanced; Sec. 2.2: the fusion level suited to Blackwell at FP32 is 5.
// For a block U (2^K x 2^K complex) on targets T, the amplitudes split into rows (the 7 lowest index bits
// outside T; a tile of 128 rows) and columns (the 2^K combinations of T). Per tile, Y = X U^T with X the
// [128 x 2^K] complex tile, computed as one real GEMM [128 x 2^(K+1)] . [2^(K+1) x 2^(K+1)] using the real
// form [[Ur, Ui], [-Ui, Ur]] of U. Complex64 accuracy is recovered from low-precision products by splitting
// both operands (Ootomo & Yokota 2022 for 3xTF32; Henry, Tang & Heinecke 2019 for BF16x3 / BF16x6), with
// FP32 accumulation in tensor memory.
//
// Data flow per CTA (one per SM, persistent over tiles). B planes (the split U, pre-swizzled in global
// memory) go to shared memory once, SWIZZLE_128B K-major. Every wait on an mbarrier is bounded (2 s); on
// expiry the kernel records DEVERR_TIMEOUT, waits once more (bounded) for its MMAs, frees its tensor memory
// and returns.
//   3xTF32 and BF16x3 (k_tc_block): warp-specialised. Eight data warps (two per TMEM lane quadrant) load
//   tiles into registers (one tile ahead at K = 6, two at K = 5), split them into the planes of the A
//   operand in TMEM and run the epilogue (tcgen05.ld of the finished accumulator, stores back in place); a
//   ninth warp issues the MMAs. Each A plane's products form a phase with its own barriers, so the split of
//   one plane overlaps the MMAs on another, and two TMEM accumulators let the epilogue of tile t-1 overlap
//   the MMAs of tile t. A thread owns one row of a tile (its TMEM lane); how its amplitudes move (Mode):
//   8-byte accesses, 16-byte pairs when qubit 0 is the first target, 32-byte quads (whole sectors) when
//   qubits 0 and 1 are the first two. When qubits 0..3 are the first four targets (3xTF32) four threads
//   share a row instead (line groups): each moves 32 bytes of the row's 128-byte line, and the tile goes to
//   and from TMEM in 16x256b fragments with B's columns permuted to match. When qubit 0 is not a target
//   but one of qubits 1..3 is (3xTF32, no epilogue) the 16x256b fragments carry pair rows: a thread's two
//   rows differ in qubit 0 and move as one 16-byte vector, and lanes l % 4 take the two lowest targets, so
//   every warp access covers whole lines whichever low qubits the block acts on. With a phase epilogue (EPI)
//   every output amplitude is multiplied by unit complex factors of its tile, row and column bits before it
//   is stored.
//   BF16x6 (k_tc_block_a2): 16 warps; two A buffers and one accumulator; one thread issues the MMAs.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "internal.h"
#include "tc_ptx.cuh"
#include "tmem_io.cuh"

namespace qsim {
namespace tc {

template <int PREC> struct Cfg;
template <> struct Cfg<QSIM_PREC_TF32X3> {
    static constexpr int planes = 2, esize = 4, nprod = 3;
    // small products first: lo*hi, hi*lo, hi*hi
    __host__ __device__ static constexpr int pa(int i) { return i == 0 ? 1 : 0; }
    __host__ __device__ static constexpr int pb(int i) { return i == 1 ? 1 : 0; }
};
template <> struct Cfg<QSIM_PREC_BF16X3> {
    static constexpr int planes = 2, esize = 2, nprod = 3;
    __host__ __device__ static constexpr int pa(int i) { return i == 0 ? 1 : 0; }
    __host__ __device__ static constexpr int pb(int i) { return i == 1 ? 1 : 0; }
};
// FP16 split products: amplitudes scaled by 2^15 (|a| <= 1 for a normalised state) and matrix entries by
// 2^14, each split into two FP16 parts (hardware conversion), three products, FP32 accumulation; the output
// is scaled back by 2^-29. 22 significant bits like 3xTF32, at the FP16 tensor rate and with half the
// tensor-memory traffic for A.
template <> struct Cfg<QSIM_PREC_FP16X3> {
    static constexpr int planes = 2, esize = 2, nprod = 3;
    __host__ __device__ static constexpr int pa(int i) { return i == 0 ? 1 : 0; }
    __host__ __device__ static constexpr int pb(int i) { return i == 1 ? 1 : 0; }
};
constexpr float kF16ScaleX = 32768.0f;              // 2^15
constexpr double kF16ScaleU = 16384.0;              // 2^14
constexpr float kF16Out = 1.0f / (32768.0f * 16384.0f);
template <> struct Cfg<QSIM_PREC_BF16X6> {
    static constexpr int planes = 3, esize = 2, nprod = 6;  // all products of planes i + j <= 2
    // (2,0) (1,1) (0,2) (1,0) (0,1) (0,0)
    __host__ __device__ static constexpr int pa(int i) { return i == 0 ? 2 : (i == 1 || i == 3) ? 1 : 0; }
    __host__ __device__ static constexpr int pb(int i) { return i == 2 ? 2 : (i == 1 || i == 4) ? 1 : 0; }
};

constexpr int kThreads = 512;
constexpr int kRowBits = 7;  // 128 rows per tile (MMA M = 128)

__host__ __device__ constexpr int plane_bytes(int K, int esize) { return (2 << K) * (2 << K) * esize; }
__host__ __device__ constexpr uint32_t pow2_at_least(uint32_t v) {
    uint32_t p = 32;
    while (p < v) p <<= 1;
    return p;
}

constexpr int kEpiGroups = kRowBits + 1 + 5;  // row bits, the half bit, up to 5 other column bits
constexpr int kEpiTile = 1 + kEpiGroups;     // factors per tile
constexpr int kBarBytes = 64;                 // shared memory for the mbarriers and the TMEM slot
constexpr int kEpiThrBytes = 2 * 128 * 6 * 8; // the epilogue's per-thread factors (float2)

struct Args {
    int nS;            // K + 7 index bits covered by a tile
    int spos[24];      // those bit positions, ascending (zeros inserted there to form a tile base)
    int rpos[kRowBits];// row bit j <-> index bit rpos[j]
    int tpos[8];       // column bit j <-> target j
    uint64_t ntiles;
    // Phase epilogue: every output amplitude x is multiplied by exp(i phi(x)), phi a quadratic form of its
    // index bits (a run of diagonal gates that follows the block). Terms on target bits alone are folded
    // into U; the rest come as unit complex factors. Bit groups: tile bits (outside the tile), row bits
    // 0..6, the column bit that selects a warp's half (target K-1, "H"), the other column bits (V).
    const float2* epi_tiles;              // [ntiles][14]: the tile's factors: tile-only terms, then the factor
                                          // of each row bit, H and each V bit given the tile's bits
    const float2* epi_thr;                // [2][128][6]: per (half, row): row / H-only terms, then each V bit's
                                          // factor given the row and H bits
    // from_basis: the input is the basis state |basis> (amplitude 1 there, 0 elsewhere), generated in
    // registers instead of read; the block writes every amplitude, so the state needs no prior set-up.
    int from_basis;
    uint64_t basis;
    int lines;                            // host side: run the line-group data path
};

// Warp-specialised block kernel, all precisions: warps 0..7 move data (tile loads, split into the A planes
// in TMEM, epilogue), warp 8 issues the MMAs. A tile is processed in one phase per A plane, smallest plane
// first; each phase has two mbarriers: full[p] (one arrival per data warp once its part of plane p is in
// TMEM) and empty[p] (tcgen05.commit after the MMAs that read plane p). The commit of the last phase (the
// hi plane) follows every MMA of the tile, so it also marks the tile's accumulator final.
constexpr int kDataWarps = 8;  // two per TMEM lane quadrant; 9 warps leave room for a two-tile prefetch
constexpr int kThreadsWS = (kDataWarps + 1) * 32;

// How the data warps move a tile between global memory and their registers (lane = row of the tile):
enum Mode {
    kRowsInLanes = 0,   // one 8-byte amplitude per access
    kPairsInLanes = 1,  // qubit 0 is target 0: columns 2i, 2i+1 move as one 16-byte vector
    kQuadsInLanes = 2,  // qubits 0 and 1 are targets 0 and 1: columns 4i..4i+3 move as one 32-byte vector, so
                        // each lane reads and writes whole 32-byte sectors
    kLineGroups = 3,    // qubits 0..3 are targets 0..3 (3xTF32, no epilogue): four lanes share a row and move
                        // its 16 adjacent amplitudes (one 128-byte line) with 32-byte accesses; the tile goes
                        // to and from TMEM with the 16x256b shape, so a warp access touches 8 whole lines
                        // instead of 32 partial ones
    kPairRows = 4,      // qubit 0 is not a target, one of 1..3 is (3xTF32, no epilogue): 16x256b fragments, a thread's two
                        // fragment rows differ in qubit 0 (row bit 3 is mapped to it) and move as one 16-byte
                        // vector per column; lanes l % 4 take the two lowest targets and l / 4 three more row
                        // qubits, so low targets no longer split a warp access over partly used lines
};

// kLineGroups column order: tile column slot s holds natural column index line_perm(s) (bits 0,1 and 2,3
// swapped), so that the slots a thread owns in the 16x256b fragment (s = 4j + lane % 4) are 4 adjacent
// amplitudes for j = 4m .. 4m + 3. The B operand is prepared in the same order.
__host__ __device__ constexpr int line_perm(int s) { return (s & ~15) | ((s & 3) << 2) | ((s >> 2) & 3); }

template <int K, int PREC, int MODE, bool EPI>
__global__ void __launch_bounds__(kThreadsWS, 1)
k_tc_block(float2* __restrict__ psi, const __grid_constant__ Args a, const uint4* __restrict__ bops,
           unsigned* __restrict__ err) {
    constexpr bool P0 = MODE == kPairsInLanes, Q0 = MODE == kQuadsInLanes, LG = MODE == kLineGroups,
                   PR = MODE == kPairRows;
    using C = Cfg<PREC>;
    constexpr bool BF16 = C::esize == 2;                   // any 16-bit operand type (packed re / im pairs)
    constexpr bool F16 = PREC == QSIM_PREC_FP16X3;         // FP16 with fixed scales
    constexpr int P = C::planes;
    constexpr int D = 1 << K, NR = 2 * D;
    constexpr int PB = plane_bytes(K, C::esize);
    constexpr int ATOM = NR * 128;                         // bytes of one 128-byte-wide K atom (all NR rows)
    constexpr int KSTEPS = NR * C::esize / 32;             // each MMA consumes 32 bytes of K
    constexpr int CPT = D / 2;                             // complex columns per thread (2 warps per quadrant)
    constexpr int QC = BF16 ? 16 : 8;                      // columns per tcgen05.st (16 32-bit values)
    constexpr int QE = 8;                                  // columns per tcgen05.ld of the FP32 accumulator
    constexpr int ACOLS = BF16 ? NR / 2 : NR;              // TMEM columns per A plane (BF16: re / im packed)
    constexpr int A0 = 2 * NR;                             // TMEM: D0 [0, NR), D1 [NR, 2 NR), A planes
    constexpr uint32_t TCOLS = pow2_at_least(A0 + P * ACOLS);
    constexpr uint32_t FMT = F16 ? 0u : (BF16 ? 1u : 2u);
    constexpr uint32_t IDESC = (1u << 4) | (FMT << 7) | (FMT << 10) | ((uint32_t)(NR >> 3) << 17) |
                               ((uint32_t)(128 >> 4) << 24);
    static_assert(CPT % QC == 0 && CPT % QE == 0, "whole chunks per thread");
    static_assert(TCOLS <= 512, "TMEM holds two accumulators and every A plane");
    static_assert(!(LG || PR) || (!BF16 && !EPI && CPT % 16 == 0), "16x256b paths: TF32 planes, no epilogue");
    constexpr int DEPTH = K >= 6 ? 1 : 2;                  // tiles of loads in flight (registers: CPT x 2 each)

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sb = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* sCol = reinterpret_cast<uint64_t*>(sb + P * PB);
    uint64_t* mbar = sCol + D;                             // empty[0..P), full[0..P), then B loaded
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2 * P + 1);
    // EPI: the per-thread factors (row / H term and V-bit coefficients of each (half, row)), transposed so
    // that a warp reads 32 consecutive entries: sTh[k * 256 + half * 128 + row]
    [[maybe_unused]] float2* sTh = reinterpret_cast<float2*>(reinterpret_cast<unsigned char*>(sCol + D) + kBarBytes);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quad = warp & 3;
    const int c0 = ((warp >> 2) & 1) * CPT;
    const int r = quad * 32 + lane;

    // Column offsets, barriers, TMEM. The B planes (already in the swizzled byte layout) come by bulk copies
    // issued after the barrier below; only the MMA issuer waits for them, so the data warps' first tile
    // loads overlap the copy.
    for (int c = tid; c < D; c += kThreadsWS) sCol[c] = deposit((uint64_t)(LG ? line_perm(c) : c), a.tpos, K);
    if constexpr (EPI) {  // plan data, written before the kernels that precede this one
        for (int i = tid; i < 2 * 128 * 6; i += kThreadsWS) sTh[(i % 6) * 256 + i / 6] = a.epi_thr[i];
    }
    if (tid == 0) {
        for (int j = 0; j < 2 * P + 1; ++j)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;"
                         :: "r"(smem_u32(mbar + j)), "r"(j < P || j == 2 * P ? 1 : kDataWarps) : "memory");
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
    const uint32_t bar0 = smem_u32(mbar);
    auto empty = [&](int p) { return bar0 + 8u * (uint32_t)p; };
    auto full = [&](int p) { return bar0 + 8u * (uint32_t)(P + p); };
    const uint32_t bbar = bar0 + 8u * (uint32_t)(2 * P);
    // Launched as a programmatic dependent of the kernel before it: everything above (offsets, barriers,
    // TMEM) overlapped that kernel's tail; from here on its writes are visible. The next block kernel may
    // be scheduled at once: it cannot share this SM (shared memory), so its CTAs start where ours finish.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (tid == 0) {
        constexpr uint32_t kChunk = 16384, kBytes = (uint32_t)(P * PB);
        static_assert(kBytes % kChunk == 0, "whole chunks");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bbar), "r"(kBytes) : "memory");
#pragma unroll 1
        for (uint32_t o = 0; o < kBytes; o += kChunk)
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         :: "r"(smem_u32(sb) + o), "l"(reinterpret_cast<const char*>(bops) + o), "r"(kChunk),
                            "r"(bbar) : "memory");
    }
    const uint64_t t0 = blockIdx.x, G = gridDim.x;
    const uint64_t m = t0 < a.ntiles ? (a.ntiles - t0 + G - 1) / G : 0;  // tiles of this CTA

    if (warp == kDataWarps) {
        // ---- MMA issuer (one thread) ----
        if (lane == 0) {
            const uint64_t desc0 = sdesc_sw128(smem_u32(sb));
            const uint32_t dhi = (uint32_t)(desc0 >> 32);
            // The products of A plane p in the order Cfg lists them; the first product of the tile starts the
            // accumulator. Descriptor offsets are compile-time constants added to the address field
            // (shared-memory addresses stay below 2^18 bytes, so the 14-bit field cannot carry). The base
            // goes through an empty asm so that the descriptors are formed at each use rather than held in
            // registers across the loop.
            auto issue = [&](int p, uint32_t dcol) {
                uint32_t dlo = (uint32_t)desc0, tb = tbase;
                asm volatile("" : "+r"(dlo), "+r"(tb));
                uint32_t acc = p == P - 1 ? 0u : 1u;
#pragma unroll
                for (int pr = 0; pr < C::nprod; ++pr) {
                    if (C::pa(pr) != p) continue;
                    const uint32_t acol = tb + A0 + p * ACOLS;
#pragma unroll
                    for (int s = 0; s < KSTEPS; ++s) {
                        const uint32_t off = (uint32_t)(C::pb(pr) * PB + (s >> 2) * ATOM + (s & 3) * 32);
                        mma_ts_lohi<BF16>(tb + dcol, acol + 8 * s, dlo + (off >> 4), dhi, IDESC, acc);
                        acc = 1;
                    }
                }
            };
            uint32_t last_bar = 0, last_par = 0;
            bool bad = !mbar_wait_bounded(bbar, 0);  // B in shared memory
            if (bad) mbar_wait_bounded(bbar, 0);     // once more for the copy still in flight
            for (uint64_t i = 0; i < m && !bad; ++i) {
                const uint32_t dcol = (i & 1) ? NR : 0, par = (uint32_t)(i & 1);
#pragma unroll
                for (int p = P - 1; p >= 0; --p) {
                    if (!mbar_wait_bounded(full(p), par)) { bad = true; break; }
                    fence_after();
                    issue(p, dcol);
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                                 :: "r"(empty(p)) : "memory");
                    last_bar = empty(p);
                    last_par = par;
                }
            }
            if (bad) {
                atomicOr(err, DEVERR_TIMEOUT);
                // the latest commit tracks every MMA issued before it: one more bounded wait on it
                if (last_bar) mbar_wait_bounded(last_bar, last_par);
            }
        }
        __syncwarp();
    } else {
        // ---- data warps ----
        const uint32_t tlane = (uint32_t)(quad * 32) << 16;
        const uint64_t rowoff = (LG || PR) ? 0 : deposit((uint64_t)r, a.rpos, kRowBits);
        // LG: this thread's rows quad * 32 + 8 rho + lane / 4 (rho = 0..3) and its slot lane % 4 of each 4
        [[maybe_unused]] uint64_t ro[4];
        [[maybe_unused]] const int li = lane & 3;
        if constexpr (LG) {
#pragma unroll
            for (int rho = 0; rho < 4; ++rho) ro[rho] = deposit((uint64_t)(quad * 32 + 8 * rho + (lane >> 2)), a.rpos, kRowBits);
        }
        // PR: rows quad * 32 + 16 pr + 8 e + lane / 4; row bit 3 (e) is qubit 0, so ro[pr] (e = 0) starts a
        // 16-byte pair of amplitudes
        if constexpr (PR) {
#pragma unroll
            for (int pr = 0; pr < 2; ++pr) ro[pr] = deposit((uint64_t)(quad * 32 + 16 * pr + (lane >> 2)), a.rpos, kRowBits);
        }
        constexpr int LPR = CPT / 4;  // LG: values per row in X (X[rho * LPR + j] is slot c0 + 4 j + lane % 4)
        // Column offsets are re-read from shared memory at each use (one broadcast load) instead of being
        // kept in 64-bit registers; the empty asm with a memory clobber between columns keeps the compiler
        // from batching those reads ahead of the accesses they address.
        const volatile uint64_t* vCol = sCol + c0;

        // Thread (r, columns c0..c0+CPT) of a tile. With P0 (qubit 0 is target 0) columns 2i and 2i+1 are
        // adjacent amplitudes and move as one 16-byte vector; otherwise lanes hold consecutive rows.
        auto load_tile = [&](float2 (&X)[CPT], uint64_t t) {
            const uint64_t b = insert_zeros(t, a.spos, a.nS) + rowoff;
            if constexpr (LG) {
#pragma unroll
                for (int rho = 0; rho < 4; ++rho)
#pragma unroll
                    for (int m = 0; m < CPT / 16; ++m) {
                        float2* x = X + rho * LPR + 4 * m;
                        const uint64_t o = b + ro[rho] + vCol[16 * m + li];  // 4 adjacent amplitudes from o
                        if (a.from_basis) {
#pragma unroll
                            for (int e = 0; e < 4; ++e) x[e] = make_float2(o + e == a.basis ? 1.0f : 0.0f, 0.0f);
                        } else {
                            ld_v8(psi + o, x[0], x[1], x[2], x[3]);
                        }
                        asm volatile("" ::: "memory");
                    }
            } else if constexpr (PR) {
                // X[pr * (CPT / 2) + 8 m + 2 jj + e]: slot c0 + 16 m + 4 jj + lane % 4, row bit 3 = e
#pragma unroll
                for (int pr = 0; pr < 2; ++pr)
#pragma unroll
                    for (int m = 0; m < CPT / 16; ++m)
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj) {
                            float2* x = X + pr * (CPT / 2) + 8 * m + 2 * jj;
                            const uint64_t o = b + ro[pr] + vCol[16 * m + 4 * jj + li];
                            if (a.from_basis) {
                                x[0] = make_float2(o == a.basis ? 1.0f : 0.0f, 0.0f);
                                x[1] = make_float2(o + 1 == a.basis ? 1.0f : 0.0f, 0.0f);
                            } else {
                                const float4 v = *reinterpret_cast<const float4*>(psi + o);
                                x[0] = make_float2(v.x, v.y);
                                x[1] = make_float2(v.z, v.w);
                            }
                            asm volatile("" ::: "memory");
                        }
            } else if (a.from_basis) {
#pragma unroll
                for (int j = 0; j < CPT; ++j) X[j] = make_float2(b + vCol[j] == a.basis ? 1.0f : 0.0f, 0.0f);
            } else if constexpr (Q0) {
#pragma unroll
                for (int j = 0; j < CPT; j += 4) {
                    ld_v8(psi + b + vCol[j], X[j], X[j + 1], X[j + 2], X[j + 3]);
                    asm volatile("" ::: "memory");
                }
            } else if constexpr (P0) {
#pragma unroll
                for (int j = 0; j < CPT; j += 2) {
                    const float4 v = *reinterpret_cast<const float4*>(psi + b + vCol[j]);
                    X[j] = make_float2(v.x, v.y);
                    X[j + 1] = make_float2(v.z, v.w);
                    asm volatile("" ::: "memory");
                }
            } else {
#pragma unroll
                for (int j = 0; j < CPT; ++j) {
                    X[j] = psi[b + vCol[j]];
                    asm volatile("" ::: "memory");
                }
            }
        };
        // Plane p of the split of x: TF32 hi = TF32(x), lo = TF32(x - hi); BF16 successive residuals rounded
        // to BF16 (p = 0, 1, 2). Every rounding is explicit: left to the tensor core, a residual's low bits
        // would be truncated towards zero.
        auto plane_of = [&](float x, int p) -> uint32_t {
            if constexpr (BF16) {
                uint32_t h = bf16_rne_bits(x);
                for (int q = 0; q < p; ++q) {
                    x -= bf16_bits_to_float(h);
                    h = bf16_rne_bits(x);
                }
                return h;
            } else {
                const uint32_t h = tf32_rna_alu(x);
                return p ? tf32_rna_alu(x - __uint_as_float(h)) : h;
            }
        };
        // Plane p of tile X into TMEM, then one arrival per warp on full[p].
        auto store_plane = [&](const float2 (&X)[CPT], int p) {
            if constexpr (LG) {
                // 16x256b: rows rho = 2 pr (TMEM lane quad * 32 + 16 pr + lane / 4) and 2 pr + 1 (8 lanes further);
                // repetition j' of chunk m holds slot c0 + 16 m + 4 j' + lane % 4 (re, im) for both rows
#pragma unroll
                for (int pr = 0; pr < 2; ++pr)
#pragma unroll
                    for (int m = 0; m < CPT / 16; ++m) {
                        uint32_t v[16];
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj) {
                            const float2 xe = X[(2 * pr) * LPR + 4 * m + jj], xo = X[(2 * pr + 1) * LPR + 4 * m + jj];
                            v[4 * jj] = plane_of(xe.x, p);
                            v[4 * jj + 1] = plane_of(xe.y, p);
                            v[4 * jj + 2] = plane_of(xo.x, p);
                            v[4 * jj + 3] = plane_of(xo.y, p);
                        }
                        tmem_st_16x256b_x4(tbase + tlane + ((uint32_t)(16 * pr) << 16) + A0 + p * ACOLS + 2 * (c0 + 16 * m), v);
                    }
            } else if constexpr (PR) {
                // 16x256b: repetition jj of chunk m holds slot c0 + 16 m + 4 jj + lane % 4 (re, im) for the
                // rows e = 0 (lane quad * 32 + 16 pr + lane / 4) and e = 1 (8 lanes further)
#pragma unroll
                for (int pr = 0; pr < 2; ++pr)
#pragma unroll
                    for (int m = 0; m < CPT / 16; ++m) {
                        uint32_t v[16];
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj) {
                            const float2 x0 = X[pr * (CPT / 2) + 8 * m + 2 * jj], x1 = X[pr * (CPT / 2) + 8 * m + 2 * jj + 1];
                            v[4 * jj] = plane_of(x0.x, p);
                            v[4 * jj + 1] = plane_of(x0.y, p);
                            v[4 * jj + 2] = plane_of(x1.x, p);
                            v[4 * jj + 3] = plane_of(x1.y, p);
                        }
                        tmem_st_16x256b_x4(tbase + tlane + ((uint32_t)(16 * pr) << 16) + A0 + p * ACOLS + 2 * (c0 + 16 * m), v);
                    }
            } else {
#pragma unroll
                for (int h = 0; h < CPT / QC; ++h) {
                    uint32_t v[16];
#pragma unroll
                    for (int j = 0; j < QC; ++j) {
                        const float2 x = X[h * QC + j];
                        if constexpr (F16) {
                            // (re, im) scaled; plane 0 = FP16 value, plane 1 = FP16 residual (re in the low half)
                            const float re = x.x * kF16ScaleX, im = x.y * kF16ScaleX;
                            uint32_t h;
                            asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(im), "f"(re));
                            if (p) {
                                const float2 hf = __half22float2(*reinterpret_cast<const __half2*>(&h));
                                asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(im - hf.y), "f"(re - hf.x));
                            }
                            v[j] = h;
                        } else if constexpr (BF16) {
                            v[j] = pack2(plane_of(x.x, p), plane_of(x.y, p));
                        } else {
                            v[2 * j] = plane_of(x.x, p);
                            v[2 * j + 1] = plane_of(x.y, p);
                        }
                    }
                    tmem_st<16>(tbase + tlane + A0 + p * ACOLS + (BF16 ? 1 : 2) * (c0 + h * QC), v);
                }
            }
            wait_st();
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(full(p));
        };
        // EPI: this thread's unit factors for tile t: E[0] for every amplitude (tile-only, row and H terms),
        // E[1 + v] for column bit v (its cross terms with the tile, row and H bits).
        constexpr int NV = K - 1;
        const int half = (warp >> 2) & 1;
        auto epi_factors = [&](uint64_t t, float2 (&E)[NV + 1]) {
            const float2* tf = a.epi_tiles + t * kEpiTile;
            const float2* th = sTh + half * 128 + r;  // th[k * 256]: factor k of this thread's (half, row)
            float2 e0 = cmul(tf[0], th[0]);
#pragma unroll
            for (int g = 0; g < kRowBits; ++g)
                if ((r >> g) & 1) e0 = cmul(e0, tf[1 + g]);
            if (half) e0 = cmul(e0, tf[1 + kRowBits]);
            E[0] = e0;
#pragma unroll
            for (int v = 0; v < NV; ++v) E[1 + v] = cmul(tf[2 + kRowBits + v], th[256 * (1 + v)]);
        };
        auto epilogue = [&](uint64_t t, uint32_t dcol) {
            const uint64_t b = insert_zeros(t, a.spos, a.nS) + rowoff;
            if constexpr (LG) {
#pragma unroll
                for (int pr = 0; pr < 2; ++pr)
#pragma unroll
                    for (int m = 0; m < CPT / 16; ++m) {
                        uint32_t v[16];
                        tmem_ld_16x256b_x4(tbase + tlane + ((uint32_t)(16 * pr) << 16) + dcol + 2 * (c0 + 16 * m), v);
                        wait_ld();
                        const uint64_t o = b + vCol[16 * m + li];
                        const uint32_t ve[8] = {v[0], v[1], v[4], v[5], v[8], v[9], v[12], v[13]};
                        const uint32_t vo[8] = {v[2], v[3], v[6], v[7], v[10], v[11], v[14], v[15]};
                        st_v8(psi + o + ro[2 * pr], ve);
                        asm volatile("" ::: "memory");
                        st_v8(psi + o + ro[2 * pr + 1], vo);
                        asm volatile("" ::: "memory");
                    }
            } else if constexpr (PR) {
#pragma unroll
                for (int pr = 0; pr < 2; ++pr)
#pragma unroll
                    for (int m = 0; m < CPT / 16; ++m) {
                        uint32_t v[16];
                        tmem_ld_16x256b_x4(tbase + tlane + ((uint32_t)(16 * pr) << 16) + dcol + 2 * (c0 + 16 * m), v);
                        wait_ld();
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj) {
                            // (re, im) of rows e = 0 and e = 1: two adjacent amplitudes
                            *reinterpret_cast<float4*>(psi + b + ro[pr] + vCol[16 * m + 4 * jj + li]) =
                                make_float4(__uint_as_float(v[4 * jj]), __uint_as_float(v[4 * jj + 1]),
                                            __uint_as_float(v[4 * jj + 2]), __uint_as_float(v[4 * jj + 3]));
                            asm volatile("" ::: "memory");
                        }
                    }
            } else {
                [[maybe_unused]] float2 E[NV + 1];
                if constexpr (EPI) epi_factors(t, E);
#pragma unroll
                for (int h = 0; h < CPT / QE; ++h) {
                    uint32_t v[2 * QE];
                    tmem_ld<2 * QE>(tbase + tlane + dcol + 2 * (c0 + h * QE), v);
                    wait_ld();
                    if constexpr (F16) {  // undo the operands' scales
#pragma unroll
                        for (int j = 0; j < 2 * QE; ++j) v[j] = __float_as_uint(__uint_as_float(v[j]) * kF16Out);
                    }
                    if constexpr (EPI) {
                        // factors of the chunk's 8 columns: column bits 0..2 vary inside it, bits 3.. are h
                        float2 f[QE];
                        f[0] = E[0];
#pragma unroll
                        for (int v2 = 3; v2 < NV; ++v2)
                            if ((h >> (v2 - 3)) & 1) f[0] = cmul(f[0], E[1 + v2]);
#pragma unroll
                        for (int e = 0; e < 3; ++e)
#pragma unroll
                            for (int q = 0; q < (1 << e); ++q) f[(1 << e) + q] = cmul(f[q], E[1 + e]);
#pragma unroll
                        for (int j = 0; j < QE; ++j) {
                            const float2 x = cmul(make_float2(__uint_as_float(v[2 * j]), __uint_as_float(v[2 * j + 1])), f[j]);
                            v[2 * j] = __float_as_uint(x.x);
                            v[2 * j + 1] = __float_as_uint(x.y);
                        }
                    }
                    if constexpr (Q0) {
#pragma unroll
                        for (int j = 0; j < QE; j += 4) {
                            st_v8(psi + b + vCol[h * QE + j], v + 2 * j);
                            asm volatile("" ::: "memory");
                        }
                    } else if constexpr (P0) {
#pragma unroll
                        for (int j = 0; j < QE; j += 2) {
                            *reinterpret_cast<float4*>(psi + b + vCol[h * QE + j]) =
                                make_float4(__uint_as_float(v[2 * j]), __uint_as_float(v[2 * j + 1]),
                                            __uint_as_float(v[2 * j + 2]), __uint_as_float(v[2 * j + 3]));
                            asm volatile("" ::: "memory");
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < QE; ++j) {
                            psi[b + vCol[h * QE + j]] =
                                make_float2(__uint_as_float(v[2 * j]), __uint_as_float(v[2 * j + 1]));
                            asm volatile("" ::: "memory");
                        }
                    }
                }
            }
        };
        // warp-uniform bounded wait (the TMEM accesses that follow are .sync.aligned)
        auto wait = [&](uint32_t bar, uint32_t par) -> bool {
            const bool ok = !__any_sync(0xffffffffu, !mbar_wait_bounded(bar, par));
            fence_after();
            return ok;
        };

        bool bad = false;
        float2 XA[CPT], XB[CPT];
        if (m > 0) load_tile(XA, t0);
        if (DEPTH == 2 && m > 1) load_tile(XB, t0 + G);
        // Tile i: per plane p (smallest first) wait for the MMAs of tile i-1 on plane p, store plane p of
        // tile i, arrive; the last wait (hi plane) also makes tile i-1 final. Then, with DEPTH 2, the
        // epilogue of tile i-1 and the loads of tile i+2 into the registers tile i used (tiles alternate
        // between the register sets XA and XB); with DEPTH 1, the loads of tile i+1 first, so that the
        // epilogue of tile i-1 covers part of their latency.
        auto step = [&](uint64_t i, float2 (&X)[CPT]) -> bool {
            const uint32_t pp = (uint32_t)((i - 1) & 1);
#pragma unroll
            for (int p = P - 1; p >= 0; --p) {
                if (i > 0 && !wait(empty(p), pp)) return false;
                store_plane(X, p);
            }
            if constexpr (DEPTH == 2) {
                if (i > 0) epilogue(t0 + (i - 1) * G, (i & 1) ? 0 : NR);
                if (i + 2 < m) load_tile(X, t0 + (i + 2) * G);
            } else {
                if (i + 1 < m) load_tile(X, t0 + (i + 1) * G);
                if (i > 0) epilogue(t0 + (i - 1) * G, (i & 1) ? 0 : NR);
            }
            return true;
        };
        uint64_t i = 0;
        if constexpr (DEPTH == 2) {
            for (; i + 1 < m; i += 2) {
                if (!step(i, XA) || !step(i + 1, XB)) { bad = true; break; }
            }
        }
        for (; !bad && i < m; ++i) {
            if (!step(i, XA)) bad = true;
        }
        if (!bad && m > 0) {
            if (wait(empty(0), (uint32_t)((m - 1) & 1))) epilogue(t0 + (m - 1) * G, ((m - 1) & 1) ? NR : 0);
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

// BF16 variants: their A planes take half the TMEM columns of TF32, so TMEM holds two A buffers and one
// accumulator. While the tensor cores run tile i from A[i&1], the warps split tile i+1 into A[(i+1)&1] and
// load tile i+2; after MMA(i) retires, D is drained into registers, MMA(i+1) is issued at once, and tile i's
// stores overlap it. The tensor cores idle only for the short drain of D.
template <int K, int PREC, bool P0>
__global__ void __launch_bounds__(kThreads, 1)
k_tc_block_a2(float2* __restrict__ psi, const __grid_constant__ Args a, const uint4* __restrict__ bops,
              unsigned* __restrict__ err) {
    using C = Cfg<PREC>;
    static_assert(C::esize == 2, "double-buffered A is for the BF16 precisions");
    constexpr int D = 1 << K, NR = 2 * D;
    constexpr int PB = plane_bytes(K, C::esize);
    constexpr int ATOM = NR * 128;
    constexpr int KSTEPS = NR * C::esize / 32;
    constexpr int CPT = D / 4;
    constexpr int ACOLS = NR / 2;                      // packed bf16 pairs
    constexpr int ABUF = C::planes * ACOLS;            // TMEM columns of one A buffer
    constexpr uint32_t TCOLS = pow2_at_least(NR + 2 * ABUF);
    constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NR >> 3) << 17) |
                               ((uint32_t)(128 >> 4) << 24);

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sb = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* sCol = reinterpret_cast<uint64_t*>(sb + C::planes * PB);
    uint64_t* mbar = sCol + D;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quad = warp & 3;
    const int c0 = (warp >> 2) * CPT;
    const int r = quad * 32 + lane;

    for (int i = tid; i < C::planes * PB / 16; i += kThreads) reinterpret_cast<uint4*>(sb)[i] = bops[i];
    for (int c = tid; c < D; c += kThreads) sCol[c] = deposit((uint64_t)c, a.tpos, K);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(mbar)), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(tslot)), "r"(TCOLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tbase = *tslot;
    const uint32_t tlane = (uint32_t)(quad * 32) << 16;
    const uint32_t mbar_addr = smem_u32(mbar);
    const uint32_t sB = smem_u32(sb);
    const uint64_t rowoff = deposit((uint64_t)r, a.rpos, kRowBits);

    float2 X[CPT];
    auto load_tile = [&](uint64_t t) {
        const uint64_t b = insert_zeros(t, a.spos, a.nS) + rowoff;
        if constexpr (P0) {
#pragma unroll
            for (int j = 0; j < CPT; j += 2) {
                const float4 v = *reinterpret_cast<const float4*>(psi + b + sCol[c0 + j]);
                X[j] = make_float2(v.x, v.y);
                X[j + 1] = make_float2(v.z, v.w);
            }
        } else {
#pragma unroll
            for (int j = 0; j < CPT; ++j) X[j] = psi[b + sCol[c0 + j]];
        }
    };
    auto split_into = [&](uint32_t abuf) {
        uint32_t p0[CPT], p1[CPT];
        [[maybe_unused]] uint32_t p2[CPT];
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
            const uint32_t hr = bf16_rne_bits(X[j].x), hm = bf16_rne_bits(X[j].y);
            const float rr = X[j].x - bf16_bits_to_float(hr), ri = X[j].y - bf16_bits_to_float(hm);
            const uint32_t mr = bf16_rne_bits(rr), mi = bf16_rne_bits(ri);
            p0[j] = pack2(hr, hm);
            p1[j] = pack2(mr, mi);
            if constexpr (C::planes == 3)
                p2[j] = pack2(bf16_rne_bits(rr - bf16_bits_to_float(mr)), bf16_rne_bits(ri - bf16_bits_to_float(mi)));
        }
        tmem_st<CPT>(tbase + tlane + abuf + 0 * ACOLS + c0, p0);
        tmem_st<CPT>(tbase + tlane + abuf + 1 * ACOLS + c0, p1);
        if constexpr (C::planes == 3) tmem_st<CPT>(tbase + tlane + abuf + 2 * ACOLS + c0, p2);
        wait_st();
    };
    auto issue = [&](uint32_t abuf) {  // thread 0 only
        fence_after();
        uint32_t acc = 0;
#pragma unroll
        for (int pr = 0; pr < C::nprod; ++pr) {
            const uint32_t acol = tbase + abuf + C::pa(pr) * ACOLS;
            const uint32_t bpl = sB + C::pb(pr) * PB;
#pragma unroll
            for (int s = 0; s < KSTEPS; ++s) {
                mma_ts<true>(tbase, acol + 8 * s, sdesc_sw128(bpl + (s >> 2) * ATOM + (s & 3) * 32), IDESC, acc);
                acc = 1;
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     :: "r"(mbar_addr) : "memory");
    };

    const uint64_t t0 = blockIdx.x, G = gridDim.x;
    const uint64_t m = t0 < a.ntiles ? (a.ntiles - t0 + G - 1) / G : 0;  // tiles of this CTA
    uint32_t phase = 0;
    bool bad = false;
    if (m > 0) {
        load_tile(t0);
        split_into(NR);
        if (m > 1) load_tile(t0 + G);
        fence_before();
        __syncthreads();
        if (tid == 0) issue(NR);
    }
    for (uint64_t i = 0; i < m; ++i) {
        const uint32_t anext = NR + (uint32_t)((i + 1) & 1) * ABUF;
        if (i + 1 < m) split_into(anext);          // A[(i+1)&1] was read by MMA(i-1), which has retired
        if (i + 2 < m) load_tile(t0 + (i + 2) * G);
        int to = 0;
        if (tid == 0) to = !mbar_wait_bounded(mbar_addr, phase);
        if (__syncthreads_or(to)) { bad = true; break; }
        phase ^= 1;
        fence_after();
        uint32_t v[2 * CPT];
        tmem_ld<2 * CPT>(tbase + tlane + 2 * c0, v);
        wait_ld();
        fence_before();
        __syncthreads();                            // D drained by every warp, A[(i+1)&1] written
        if (i + 1 < m && tid == 0) issue(anext);
        const uint64_t b = insert_zeros(t0 + i * G, a.spos, a.nS) + rowoff;
        if constexpr (P0) {
#pragma unroll
            for (int j = 0; j < CPT; j += 2)
                *reinterpret_cast<float4*>(psi + b + sCol[c0 + j]) =
                    make_float4(__uint_as_float(v[2 * j]), __uint_as_float(v[2 * j + 1]),
                                __uint_as_float(v[2 * j + 2]), __uint_as_float(v[2 * j + 3]));
        } else {
#pragma unroll
            for (int j = 0; j < CPT; ++j)
                psi[b + sCol[c0 + j]] = make_float2(__uint_as_float(v[2 * j]), __uint_as_float(v[2 * j + 1]));
        }
    }
    if (bad && tid == 0) {
        atomicOr(err, DEVERR_TIMEOUT);
        mbar_wait_bounded(mbar_addr, phase);
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tbase), "r"(TCOLS) : "memory");
    }
}

// B operand: Bt[n][kk] of the real form, Bt[2i][2c] = Re U_ic, Bt[2i][2c+1] = -Im U_ic, Bt[2i+1][2c] = Im U_ic,
// Bt[2i+1][2c+1] = Re U_ic, split into planes and written in the swizzled shared-memory byte layout (i, c taken
// through line_perm for the line-group data path).
// With rowphase (device, 2^K radians), row i of U is multiplied by exp(i rowphase[i]) first: the phase
// epilogue's terms on target bits alone.
template <int PREC>
__global__ void k_tc_prepare(const double* __restrict__ U, int K, const double* __restrict__ rowphase, int perm,
                             unsigned char* __restrict__ out) {
    using C = Cfg<PREC>;
    const int D = 1 << K, NR = 2 * D;
    const int PB = plane_bytes(K, C::esize);
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < NR * NR; idx += gridDim.x * blockDim.x) {
        const int n = idx / NR, kk = idx % NR;
        // perm: output and input slots in the line-group column order
        const int i = perm ? line_perm(n >> 1) : n >> 1, c = perm ? line_perm(kk >> 1) : kk >> 1;
        double ur = U[2 * (i * D + c)], ui = U[2 * (i * D + c) + 1];
        if (rowphase) {
            double sp, cp;
            sincos(rowphase[i], &sp, &cp);
            const double r2 = ur * cp - ui * sp;
            ui = ur * sp + ui * cp;
            ur = r2;
        }
        const double v = (n & 1) == 0 ? ((kk & 1) == 0 ? ur : -ui) : ((kk & 1) == 0 ? ui : ur);
        const uint32_t off = sw128_offset(n, kk, NR, C::esize);
        if constexpr (PREC == QSIM_PREC_FP16X3) {
            const double w = kF16ScaleU * v;
            const __half h = __float2half_rn((float)w);
            *reinterpret_cast<__half*>(out + off) = h;
            *reinterpret_cast<__half*>(out + PB + off) = __float2half_rn((float)(w - (double)__half2float(h)));
        } else if constexpr (C::esize == 4) {
            const uint32_t hi = tf32_rna((float)v);
            const float lo = (float)(v - (double)__uint_as_float(hi));
            *reinterpret_cast<uint32_t*>(out + off) = hi;
            *reinterpret_cast<uint32_t*>(out + PB + off) = tf32_rna(lo);
        } else {
            const __nv_bfloat16 h = __float2bfloat16_rn((float)v);
            const double r1 = v - (double)__bfloat162float(h);
            const __nv_bfloat16 m = __float2bfloat16_rn((float)r1);
            *reinterpret_cast<__nv_bfloat16*>(out + off) = h;
            *reinterpret_cast<__nv_bfloat16*>(out + PB + off) = m;
            if constexpr (C::planes == 3) {
                const double r2 = r1 - (double)__bfloat162float(m);
                *reinterpret_cast<__nv_bfloat16*>(out + 2 * PB + off) = __float2bfloat16_rn((float)r2);
            }
        }
    }
}

template <int PREC> constexpr int planes_of() { return Cfg<PREC>::planes; }
template <int PREC> constexpr int esize_of() { return Cfg<PREC>::esize; }

size_t smem_bytes(int K, int planes, int esize) {
    // B planes, column offsets, barriers and the TMEM slot, the epilogue's per-thread factors, alignment
    const size_t need = (size_t)planes * plane_bytes(K, esize) + sizeof(uint64_t) * (1 << K) + kBarBytes +
                        kEpiThrBytes + 1024;
    return std::max<size_t>(need, 120 * 1024);  // at most one CTA (and one TMEM owner) per SM
}

template <int K, int PREC, int MODE, bool EPI>
cudaError_t apply_p(void* psi, const Args& a, const void* dB, unsigned* err, cudaStream_t s, const DevInfo& d) {
    const size_t smem = smem_bytes(K, Cfg<PREC>::planes, Cfg<PREC>::esize);
    const unsigned grid = (unsigned)std::min<uint64_t>((uint64_t)d.num_sms, a.ntiles);
    auto launch = [&](auto kern, int threads, bool pdl) {
        cudaError_t e = smem_optin(reinterpret_cast<const void*>(kern), (int)smem);
        if (e != cudaSuccess) return e;
        if (!pdl) {
            kern<<<grid, threads, smem, s>>>(reinterpret_cast<float2*>(psi), a, reinterpret_cast<const uint4*>(dB), err);
            return cudaGetLastError();
        }
        // programmatic dependent launch: the prologue overlaps the tail of the kernel before (k_tc_block
        // waits for it with griddepcontrol.wait before it touches memory that kernel may write)
        cudaLaunchConfig_t cfg{};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.gridDim = dim3(grid, 1, 1);
        cfg.blockDim = dim3(threads, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, kern, reinterpret_cast<float2*>(psi), a, reinterpret_cast<const uint4*>(dB), err);
    };
    // BF16x6 (three A planes, the heaviest split) runs faster on 16 warps with two A buffers than on the
    // 8 data warps of the warp-specialised kernel (which alone has the 32-byte path)
    if constexpr (PREC == QSIM_PREC_BF16X6) {
        if constexpr (EPI) return cudaErrorInvalidValue;  // the 16-warp kernel has no phase epilogue
        else return launch(k_tc_block_a2<K, PREC, MODE != kRowsInLanes>, kThreads, false);
    } else {
        return launch(k_tc_block<K, PREC, MODE, EPI>, kThreadsWS, true);
    }
}

template <int K, int PREC, bool EPI>
cudaError_t apply_e(void* psi, const Args& a, const void* dB, unsigned* err, cudaStream_t s, const DevInfo& d) {
    if (a.lines) {
        if constexpr (PREC == QSIM_PREC_TF32X3 && !EPI) return apply_p<K, PREC, kLineGroups, EPI>(psi, a, dB, err, s, d);
        else return cudaErrorInvalidValue;
    }
    if constexpr (PREC == QSIM_PREC_TF32X3 && !EPI) {
        // Pair rows when qubit 0 is not a target but one of qubits 1..3 is (lanes on rows would split each
        // warp access over partly used lines; measured 2.6 vs 2.7-4.6 ms at 30 qubits). With targets from
        // qubit 4 up, lanes on rows stay faster (2.6 vs 2.9-3.1 ms): each of their accesses covers two
        // adjacent lines of one column rather than single lines of four columns.
        bool low = false;
        for (int j = 0; j < K; ++j) low = low || (a.tpos[j] >= 1 && a.tpos[j] <= 3);
        if (a.rpos[0] == 0 && low) {  // pair rows, with row bit 3 moved to qubit 0
            Args b = a;
            b.rpos[0] = a.rpos[1];
            b.rpos[1] = a.rpos[2];
            b.rpos[2] = a.rpos[3];
            b.rpos[3] = a.rpos[0];
            return apply_p<K, PREC, kPairRows, EPI>(psi, b, dB, err, s, d);
        }
    }
    if (a.tpos[0] == 0 && a.tpos[1] == 1 && PREC != QSIM_PREC_BF16X6 && (reinterpret_cast<uintptr_t>(psi) & 31) == 0)
        return apply_p<K, PREC, kQuadsInLanes, EPI>(psi, a, dB, err, s, d);
    if (a.tpos[0] == 0) return apply_p<K, PREC, kPairsInLanes, EPI>(psi, a, dB, err, s, d);
    return apply_p<K, PREC, kRowsInLanes, EPI>(psi, a, dB, err, s, d);
}

template <int K, int PREC>
cudaError_t apply_t(void* psi, const Args& a, const void* dB, unsigned* err, cudaStream_t s, const DevInfo& d) {
    if (a.epi_tiles) return apply_e<K, PREC, true>(psi, a, dB, err, s, d);
    return apply_e<K, PREC, false>(psi, a, dB, err, s, d);
}

}  // namespace tc

void tc_epi_pack(int n, int k, const int* targets, const PhaseForm& f, std::vector<unsigned char>& out,
                 TcEpiPacked& pk) {
    // group of each index bit as the kernel sees it: row bit j -> j, the half column bit (target k-1) -> 7,
    // column bit v < k-1 -> 8 + v, tile bits -> -1
    std::vector<int> grp(n, -1);
    uint64_t tmask = 0;
    for (int j = 0; j < k; ++j) tmask |= 1ull << targets[j];
    int nr = 0;
    for (int q = 0; q < n && nr < tc::kRowBits; ++q)
        if (!((tmask >> q) & 1)) grp[q] = nr++;
    grp[targets[k - 1]] = tc::kRowBits;
    for (int v = 0; v < k - 1; ++v) grp[targets[v]] = tc::kRowBits + 1 + v;
    auto colbit = [&](int g) { return g == tc::kRowBits ? k - 1 : g - tc::kRowBits - 1; };  // g >= 7: column bit
    auto bit = [](int g, int half, int r) { return g < tc::kRowBits ? (r >> g) & 1 : half; };
    std::vector<double> rowphase(1 << k, f.c);          // terms on target bits alone (and the constant)
    std::vector<uint32_t> tt_ab;
    std::vector<uint64_t> tt_l;
    std::vector<std::vector<std::pair<uint32_t, uint64_t>>> tb(tc::kEpiGroups);
    std::vector<double> thr(2 * 128 * 6, 0.0);          // radians: slot 0 row / H terms, 1 + v: V-bit coefficients
    auto thr_add = [&](int slot, double L, int g1, int g2) {  // conditions on row / H groups (g < 0: none)
        for (int half = 0; half < 2; ++half)
            for (int r = 0; r < 128; ++r)
                if ((g1 < 0 || bit(g1, half, r)) && (g2 < 0 || bit(g2, half, r))) thr[(half * 128 + r) * 6 + slot] += L;
    };
    auto rowphase_add = [&](double L, int c1, int c2) {  // column bits c1, c2 (c2 < 0: a single bit)
        for (int m = 0; m < (1 << k); ++m)
            if (((m >> c1) & 1) && (c2 < 0 || ((m >> c2) & 1))) rowphase[m] += L;
    };
    for (int a = 0; a < n; ++a) {
        if (f.h[a] == 0.0) continue;
        const int g = grp[a];
        if (g < 0) { tt_ab.push_back((uint32_t)a | ((uint32_t)a << 8)); tt_l.push_back(phase_turns(f.h[a])); }
        else if (g < tc::kRowBits) thr_add(0, f.h[a], g, -1);
        else rowphase_add(f.h[a], colbit(g), -1);
    }
    for (const auto& p : f.pairs) {
        const int ga = grp[p.a], gb = grp[p.b];
        if (ga < 0 && gb < 0) { tt_ab.push_back((uint32_t)p.a | ((uint32_t)p.b << 8)); tt_l.push_back(phase_turns(p.lam)); }
        else if (ga < 0) tb[gb].push_back({(uint32_t)p.a, phase_turns(p.lam)});
        else if (gb < 0) tb[ga].push_back({(uint32_t)p.b, phase_turns(p.lam)});
        else if (ga >= tc::kRowBits && gb >= tc::kRowBits) rowphase_add(p.lam, colbit(ga), colbit(gb));  // both targets
        else if (ga < tc::kRowBits && gb < tc::kRowBits) thr_add(0, p.lam, ga, gb);                      // both rows
        else {
            const int gr = ga < tc::kRowBits ? ga : gb, gc = ga < tc::kRowBits ? gb : ga;  // a row bit and a column bit
            if (gc == tc::kRowBits) thr_add(0, p.lam, gr, gc);                            // the H bit: per thread
            else thr_add(1 + gc - tc::kRowBits - 1, p.lam, gr, -1);                      // a V bit: its coefficient
        }
    }
    std::vector<uint32_t> tb_t;
    std::vector<uint64_t> tb_l;
    pk.off[0] = 0;
    for (int g = 0; g < tc::kEpiGroups; ++g) {
        for (const auto& t : tb[g]) { tb_t.push_back(t.first); tb_l.push_back(t.second); }
        pk.off[g + 1] = (int)tb_t.size();
    }
    pk.c = 0;  // the constant went into U with the target-only terms
    pk.ntt = (int)tt_ab.size();
    auto al = [](size_t v) { return (v + 15) & ~(size_t)15; };
    size_t off = 0;
    pk.off_rowphase = off; off = al(off + 8 * rowphase.size());
    pk.off_tt_ab = off; off = al(off + 4 * tt_ab.size());
    pk.off_tt_l = off;  off = al(off + 8 * tt_l.size());
    pk.off_tb_t = off;  off = al(off + 4 * tb_t.size());
    pk.off_tb_l = off;  off = al(off + 8 * tb_l.size());
    pk.off_thr = off;   off = al(off + 8 * thr.size());
    out.assign(off, 0);
    auto put = [&](size_t o, const void* src, size_t bytes) { if (bytes) std::memcpy(out.data() + o, src, bytes); };
    put(pk.off_rowphase, rowphase.data(), 8 * rowphase.size());
    put(pk.off_tt_ab, tt_ab.data(), 4 * tt_ab.size());
    put(pk.off_tt_l, tt_l.data(), 8 * tt_l.size());
    put(pk.off_tb_t, tb_t.data(), 4 * tb_t.size());
    put(pk.off_tb_l, tb_l.data(), 8 * tb_l.size());
    for (size_t i = 0; i < thr.size(); ++i) {
        const float v2[2] = {(float)std::cos(thr[i]), (float)std::sin(thr[i])};
        put(pk.off_thr + 8 * i, v2, 8);
    }
}

size_t tc_epi_scratch_bytes(int n, int k) {
    return sizeof(float2) * tc::kEpiTile * ((size_t)1 << (n - k - tc::kRowBits));
}

bool tc_supported(int k, int precision) {
    if (k == 7) return precision == QSIM_PREC_FP16X3;  // k_tc7.cu
    return (k == 5 || k == 6) &&
           (precision == QSIM_PREC_TF32X3 || precision == QSIM_PREC_BF16X3 || precision == QSIM_PREC_BF16X6 ||
            precision == QSIM_PREC_FP16X3);
}

size_t tc_operand_bytes(int k, int precision) {
    if (!tc_supported(k, precision)) return 0;
    if (k == 7) return tc7_operand_bytes();
    const int planes = precision == QSIM_PREC_BF16X6 ? 3 : 2;
    const int esize = precision == QSIM_PREC_TF32X3 ? 4 : 2;
    return (size_t)planes * tc::plane_bytes(k, esize);
}

bool tc_line_groups(int k, const int* targets, int precision, bool epi) {
    return precision == QSIM_PREC_TF32X3 && !epi && (k == 5 || k == 6) && targets[0] == 0 && targets[1] == 1 &&
           targets[2] == 2 && targets[3] == 3;
}

cudaError_t launch_tc_prepare(const double* dU, int k, int precision, bool lines, void* dB, cudaStream_t s,
                              const double* rowphase) {
    if (!tc_supported(k, precision)) return cudaErrorInvalidValue;
    if (lines && (precision != QSIM_PREC_TF32X3 || rowphase)) return cudaErrorInvalidValue;
    if (k == 7) return rowphase || lines ? cudaErrorInvalidValue : launch_tc7_prepare(dU, dB, s);
    unsigned char* out = static_cast<unsigned char*>(dB);
    const int blocks = ((2 << k) * (2 << k) + 255) / 256;
    const int perm = lines ? 1 : 0;
    switch (precision) {
        case QSIM_PREC_TF32X3: tc::k_tc_prepare<QSIM_PREC_TF32X3><<<blocks, 256, 0, s>>>(dU, k, rowphase, perm, out); break;
        case QSIM_PREC_BF16X3: tc::k_tc_prepare<QSIM_PREC_BF16X3><<<blocks, 256, 0, s>>>(dU, k, rowphase, perm, out); break;
        case QSIM_PREC_FP16X3: tc::k_tc_prepare<QSIM_PREC_FP16X3><<<blocks, 256, 0, s>>>(dU, k, rowphase, perm, out); break;
        default: tc::k_tc_prepare<QSIM_PREC_BF16X6><<<blocks, 256, 0, s>>>(dU, k, rowphase, perm, out); break;
    }
    return cudaGetLastError();
}

// The phase epilogue's per-tile factors (one thread per tile): exp(i * terms on tile bits alone) and, for each
// row bit, H and V bit, exp(i * its cross terms with the tile's bits).
__global__ void k_tc_epi_tiles(uint64_t ntiles, tc::Args a, TcEpiPacked pk, const unsigned char* __restrict__ tab,
                               float2* __restrict__ out) {
    const uint32_t* tt_ab = reinterpret_cast<const uint32_t*>(tab + pk.off_tt_ab);
    const uint64_t* tt_l = reinterpret_cast<const uint64_t*>(tab + pk.off_tt_l);
    const uint32_t* tb_t = reinterpret_cast<const uint32_t*>(tab + pk.off_tb_t);
    const uint64_t* tb_l = reinterpret_cast<const uint64_t*>(tab + pk.off_tb_l);
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t tb = insert_zeros(t, a.spos, a.nS);
        uint64_t s = pk.c;
        for (int i = 0; i < pk.ntt; ++i)
            if ((tb >> (tt_ab[i] & 0xFF)) & (tb >> (tt_ab[i] >> 8)) & 1) s += tt_l[i];
        float2* o = out + t * tc::kEpiTile;
        o[0] = unit_phase(0.0f, s);
        for (int g = 0; g < tc::kEpiGroups; ++g) {
            uint64_t k = 0;
            for (int i = pk.off[g]; i < pk.off[g + 1]; ++i)
                if ((tb >> tb_t[i]) & 1) k += tb_l[i];
            o[1 + g] = unit_phase(0.0f, k);
        }
    }
}

cudaError_t launch_tc_apply(void* psi, int n, int k, const int* targets, const void* dB, int precision,
                            unsigned* dev_err, cudaStream_t s, const DevInfo& d, const void* epi_tab,
                            const TcEpiPacked* epi, void* epi_scratch, const uint64_t* from_basis, bool lines) {
    if (!tc_supported(k, precision) || n < k + tc::kRowBits) return cudaErrorInvalidValue;
    if (lines && !tc_line_groups(k, targets, precision, epi != nullptr)) return cudaErrorInvalidValue;
    if ((reinterpret_cast<uintptr_t>(dB) & 15) != 0) return cudaErrorInvalidValue;
    if (epi && (!epi_tab || !epi_scratch || precision == QSIM_PREC_BF16X6)) return cudaErrorInvalidValue;
    if (k == 7) {  // FP16X3 only; no phase epilogue, no line groups
        if (epi || lines) return cudaErrorInvalidValue;
        return launch_tc7_apply(psi, n, targets, dB, dev_err, s, d, from_basis);
    }
    tc::Args a;
    std::memset(&a, 0, sizeof(a));

    uint64_t tmask = 0;
    for (int j = 0; j < k; ++j) { a.tpos[j] = targets[j]; tmask |= 1ull << targets[j]; }
    int nr = 0;
    for (int q = 0; q < n && nr < tc::kRowBits; ++q)
        if (!((tmask >> q) & 1)) a.rpos[nr++] = q;
    uint64_t smask = tmask;
    for (int j = 0; j < tc::kRowBits; ++j) smask |= 1ull << a.rpos[j];
    for (int q = 0; q < n; ++q)
        if ((smask >> q) & 1) a.spos[a.nS++] = q;
    a.ntiles = 1ull << (n - a.nS);
    a.lines = lines ? 1 : 0;
    if (from_basis) {
        if (precision == QSIM_PREC_BF16X6) return cudaErrorInvalidValue;  // the 16-warp kernel always reads
        a.from_basis = 1;
        a.basis = *from_basis;
    }
    if (epi) {
        // the tile factors go to the scratch (tc_epi_scratch_bytes), read by the block kernel that follows
        const unsigned char* b = static_cast<const unsigned char*>(epi_tab);
        float2* tiles = static_cast<float2*>(epi_scratch);
        const unsigned grid = grid_for((int64_t)a.ntiles, 256, d.num_sms, 4);
        k_tc_epi_tiles<<<grid, 256, 0, s>>>(a.ntiles, a, *epi, b, tiles);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        a.epi_tiles = tiles;
        a.epi_thr = reinterpret_cast<const float2*>(b + epi->off_thr);
    }
    switch (precision * 8 + k) {
        case QSIM_PREC_TF32X3 * 8 + 5: return tc::apply_t<5, QSIM_PREC_TF32X3>(psi, a, dB, dev_err, s, d);
        case QSIM_PREC_TF32X3 * 8 + 6: return tc::apply_t<6, QSIM_PREC_TF32X3>(psi, a, dB, dev_err, s, d);
        case QSIM_PREC_BF16X3 * 8 + 5: return tc::apply_t<5, QSIM_PREC_BF16X3>(psi, a, dB, dev_err, s, d);
        case QSIM_PREC_BF16X3 * 8 + 6: return tc::apply_t<6, QSIM_PREC_BF16X3>(psi, a, dB, dev_err, s, d);
        case QSIM_PREC_FP16X3 * 8 + 5: return tc::apply_t<5, QSIM_PREC_FP16X3>(psi, a, dB, dev_err, s, d);
        case QSIM_PREC_FP16X3 * 8 + 6: return tc::apply_t<6, QSIM_PREC_FP16X3>(psi, a, dB, dev_err, s, d);
        case QSIM_PREC_BF16X6 * 8 + 5: return tc::apply_t<5, QSIM_PREC_BF16X6>(psi, a, dB, dev_err, s, d);
        case QSIM_PREC_BF16X6 * 8 + 6: return tc::apply_t<6, QSIM_PREC_BF16X6>(psi, a, dB, dev_err, s, d);
    }
    return cudaErrorInvalidValue;
}

}  // namespace qsim
