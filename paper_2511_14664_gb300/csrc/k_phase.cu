// k_phase.cu -- one pass for any number of 1- and 2-qubit diagonal gates, on any qubits.
//
// Paper Sec. 2.1: a gate is an operator on the whole 2^n vector; diagonal gates (RZ, CZ, controlled phases,
// the RZZ of the TFIM Trotter step, Sec. 2.2) only multiply each amplitude by a phase, and they commute with
// each other. A run of them that the fusion planner can move together therefore costs one pass over the
// state, whatever qubits they touch. The combined phase of such a run is a quadratic form in the index bits,
//     phi(x) = c + sum_a h_a x_a + sum_{a<b} L_ab x_a x_b,
// because every 1- or 2-qubit diagonal unitary is exp(i (p0 + p1 x_a + p2 x_b + p3 x_a x_b)).
//
// Phases are 64-bit fixed-point turns (2^64 = one turn): sums wrap around exactly (mod 2 pi) and need no FP64
// arithmetic, which is scarce on GB300. A range is 1024 consecutive amplitudes: lanes are index bits 0..4
// (coalesced 256-byte accesses) and each lane's 32 amplitudes differ in bits 5..9. A warp owns a group of
// 16 consecutive ranges (bits 10..13): it reduces the terms on the group's fixed top bits once, into a
// constant and a coefficient for each bit below (warp shuffles), and folds in the 4 range bits from small
// shared-memory tables per range. Per lane this leaves
//     phi(lane, m) = s_lane + sum_e nu_e m_e + M(m)   (m = bits 5..9),
// evaluated as products of unit complex numbers in a depth-5 tree (no per-amplitude sin / cos).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace qsim {
namespace phase {

constexpr int kLowBits = 10;  // a warp's range: 2^10 amplitudes
constexpr int kLaneBits = 5;

// Index bits: 0..4 lane, 5..9 the lane's 32 amplitudes (mid), 10..10+nb-1 the range within a warp's group
// of 2^nb ranges (block), the rest fixed per group (top). Terms are split by the bit groups they touch.
constexpr int kBlockBits = 4;

struct Args {
    uint64_t c;
    int nb;                        // block bits (min(4, n - 10))
    int ntt;                       // terms on two top bits (a single top bit appears as a == b)
    int lt_off[kLowBits + kBlockBits + 1];  // terms (low or block bit j, top bit a): [lt_off[j], lt_off[j+1])
    const uint32_t* tt_ab;         // a | b << 8
    const uint64_t* tt_l;
    const uint32_t* lt_a;          // the top bit
    const uint64_t* lt_l;
    const uint64_t* small;         // ll_lane[32] | lm[32][5] | sb[16] | mb[16][10]  (see phase_pack)
    const void* tmid;              // [32] complex (state precision): exp(i * mid-mid terms of bits 5..9)
};
constexpr int kSmallWords = 32 + 32 * 5 + 16 + 16 * kLowBits;

template <typename R>
__global__ void __launch_bounds__(256) k_phase(typename Amp<R>::T* __restrict__ psi, int n, const Args a) {
    using T = typename Amp<R>::T;
    constexpr int M = 1 << (kLowBits - kLaneBits);  // 32 amplitudes per lane, in two halves of 16
    constexpr int H = M / 2;
    constexpr int NMU = kLowBits + kBlockBits;
    __shared__ uint64_t sm[kSmallWords];
    __shared__ uint64_t smu[8][NMU];                // per warp: coefficients of the low and block bits
    __shared__ T stmid[M];
    for (int i = threadIdx.x; i < kSmallWords; i += blockDim.x) sm[i] = a.small[i];
    if (threadIdx.x < M) stmid[threadIdx.x] = static_cast<const T*>(a.tmid)[threadIdx.x];
    __syncthreads();
    const uint64_t* ll_lane = sm;
    const uint64_t* lm = sm + 32;
    const uint64_t* sb = lm + 32 * 5;
    const uint64_t* mb = sb + 16;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint64_t* mu = smu[wib];
    const int gbits = kLowBits + a.nb;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    const uint64_t ngroups = 1ull << (n - gbits);
    for (uint64_t gp = (uint64_t)blockIdx.x * (blockDim.x >> 5) + wib; gp < ngroups; gp += warps) {
        const uint64_t gbase = gp << gbits;
        // terms on the group's fixed top bits: a constant and a coefficient for each low and block bit
        uint64_t s = 0;
        for (int i = lane; i < a.ntt; i += 32) {
            const uint32_t ab = a.tt_ab[i];
            if ((gbase >> (ab & 0xFF)) & (gbase >> (ab >> 8)) & 1) s += a.tt_l[i];
        }
        s = warp_sum64(s) + a.c;
        __syncwarp();  // the previous group's readers of mu are done
        for (int j = 0; j < NMU; ++j) {
            uint64_t t = 0;
            for (int i = a.lt_off[j] + lane; i < a.lt_off[j + 1]; i += 32)
                if ((gbase >> a.lt_a[i]) & 1) t += a.lt_l[i];
            t = warp_sum64(t);
            if (lane == 0) mu[j] = t;
        }
        __syncwarp();
        const uint64_t lane_c = ll_lane[lane] + s;
        for (int bv = 0; bv < (1 << a.nb); ++bv) {
            const uint64_t base = gbase | ((uint64_t)bv << kLowBits);
            const uint64_t* mbv = mb + bv * kLowBits;
            // this range's constant for the lane, with the block bits bv folded in
            uint64_t sl = lane_c + sb[bv];
            for (int k = 0; k < a.nb; ++k)
                if ((bv >> k) & 1) sl += mu[kLowBits + k];
#pragma unroll
            for (int j = 0; j < kLaneBits; ++j)
                if ((lane >> j) & 1) sl += mu[j] + mbv[j];
            auto coef = [&](int e) { return mu[kLaneBits + e] + mbv[kLaneBits + e] + lm[lane * (kLowBits - kLaneBits) + e]; };
            // factors of the first half (m < 16) by a depth-4 tree; the second half adds bit 9's factor
            T F[H];
            F[0] = unit_phase(R(0), sl);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const T B = unit_phase(R(0), coef(e));
#pragma unroll
                for (int m = 0; m < (1 << e); ++m) F[(1 << e) + m] = cmul(F[m], B);
            }
            const T B4 = unit_phase(R(0), coef(4));
            auto apply_half = [&](auto hc) {
                constexpr int half = decltype(hc)::value;
                T v[H];
#pragma unroll
                for (int m = 0; m < H; ++m) v[m] = psi[base + ((uint64_t)(half * H + m) << kLaneBits) + lane];
#pragma unroll
                for (int m = 0; m < H; ++m) {
                    const T f = half ? cmul(cmul(F[m], B4), stmid[H + m]) : cmul(F[m], stmid[m]);
                    psi[base + ((uint64_t)(half * H + m) << kLaneBits) + lane] = cmul(v[m], f);
                }
            };
            apply_half(std::integral_constant<int, 0>{});
            apply_half(std::integral_constant<int, 1>{});
        }
    }
}

}  // namespace phase

// ---- host: the quadratic form of a run of diagonal gates -------------------------------------------------------
uint64_t phase_turns(double phi) {
    double t = phi / 6.283185307179586476925286766559;
    t -= std::floor(t);
    if (!(t < 1.0)) t = 0.0;
    return (uint64_t)std::ldexp(t, 64);  // t < 1, so the value fits; 53 significant bits
}

bool phase_gate_ok(const qsim_gate& g) {
    return g.k >= 1 && g.k + g.nc <= 2;
}

bool phase_form_build(const qsim_gate* const* gates, int count, int n, PhaseForm& f) {
    f = PhaseForm{};
    f.h.assign(n, 0.0);
    std::map<std::pair<int, int>, double> lam;
    for (int i = 0; i < count; ++i) {
        const qsim_gate& g = *gates[i];
        if (!phase_gate_ok(g)) return false;
        const int D = 1 << g.k;
        double ph[4];
        for (int m = 0; m < D; ++m) ph[m] = std::atan2(g.matrix[2 * (m * D + m) + 1], g.matrix[2 * (m * D + m)]);
        if (g.nc == 0 && g.k == 1) {
            f.c += ph[0];
            f.h[g.targets[0]] += ph[1] - ph[0];
        } else if (g.nc == 0) {  // two targets: index m = x_t0 + 2 x_t1
            const int a = g.targets[0], b = g.targets[1];
            f.c += ph[0];
            f.h[a] += ph[1] - ph[0];
            f.h[b] += ph[2] - ph[0];
            lam[{std::min(a, b), std::max(a, b)}] += ph[3] - ph[2] - ph[1] + ph[0];
        } else {  // one control, one target: x_c (ph0 + (ph1 - ph0) x_t)
            const int c = g.controls[0], t = g.targets[0];
            f.h[c] += ph[0];
            lam[{std::min(c, t), std::max(c, t)}] += ph[1] - ph[0];
        }
    }
    for (const auto& kv : lam) f.pairs.push_back({kv.first.first, kv.first.second, kv.second});
    return true;
}

// Lay out the device tables of `f` in `out` (byte offsets relative to the start) and fill the launch counts.
void phase_pack(const PhaseForm& f, int dtype, std::vector<unsigned char>& out, PhasePacked& pk) {
    using namespace phase;
    const int n = (int)f.h.size();
    const int nb = std::max(0, std::min(kBlockBits, n - kLowBits));
    const int G = kLowBits + nb;  // bits below the top bits
    std::vector<uint32_t> tt_ab, lt_a;
    std::vector<uint64_t> tt_l, lt_l;
    std::vector<std::vector<std::pair<uint32_t, uint64_t>>> lt(kLowBits + kBlockBits);
    std::vector<uint64_t> hg(G, 0);  // single-bit terms of the low and block bits
    for (int a = 0; a < n; ++a) {
        if (f.h[a] == 0.0) continue;
        if (a >= G) { tt_ab.push_back((uint32_t)a | ((uint32_t)a << 8)); tt_l.push_back(phase_turns(f.h[a])); }
        else hg[a] = phase_turns(f.h[a]);
    }
    // pair terms by the groups of their bits (a < b)
    std::vector<uint64_t> small(kSmallWords, 0);
    uint64_t* ll_lane = small.data();
    uint64_t* lm = ll_lane + 32;
    uint64_t* sb = lm + 32 * 5;
    uint64_t* mb = sb + 16;
    double midmid[5][5] = {};
    uint64_t lanelane[5][5] = {};
    for (const auto& p : f.pairs) {
        const uint64_t L = phase_turns(p.lam);
        if (p.a >= G) { tt_ab.push_back((uint32_t)p.a | ((uint32_t)p.b << 8)); tt_l.push_back(L); }
        else if (p.b >= G) lt[p.a].push_back({(uint32_t)p.b, L});           // low/block x top
        else if (p.a >= kLowBits) {                                        // block x block
            for (int bv = 0; bv < (1 << nb); ++bv)
                if (((bv >> (p.a - kLowBits)) & 1) && ((bv >> (p.b - kLowBits)) & 1)) sb[bv] += L;
        } else if (p.b >= kLowBits) {                                      // low x block
            for (int bv = 0; bv < (1 << nb); ++bv)
                if ((bv >> (p.b - kLowBits)) & 1) mb[bv * kLowBits + p.a] += L;
        } else if (p.b < kLaneBits) lanelane[p.a][p.b] += L;              // lane x lane
        else if (p.a < kLaneBits) {                                        // lane x mid
            for (int l = 0; l < 32; ++l)
                if ((l >> p.a) & 1) lm[l * 5 + (p.b - kLaneBits)] += L;
        } else {
            midmid[p.a - kLaneBits][p.b - kLaneBits] += p.lam;             // mid x mid
        }
    }
    for (int bv = 0; bv < (1 << nb); ++bv)
        for (int k = 0; k < nb; ++k)
            if ((bv >> k) & 1) sb[bv] += hg[kLowBits + k];
    for (int l = 0; l < 32; ++l) {
        uint64_t v = 0;
        for (int j = 0; j < kLaneBits; ++j) {
            if (!((l >> j) & 1)) continue;
            v += hg[j];
            for (int k = j + 1; k < kLaneBits; ++k)
                if ((l >> k) & 1) v += lanelane[j][k];
        }
        ll_lane[l] = v;
        for (int e = 0; e < 5; ++e) lm[l * 5 + e] += hg[kLaneBits + e];
    }
    for (int j = 0; j < kLowBits + kBlockBits; ++j)
        for (const auto& t : lt[j]) { lt_a.push_back(t.first); lt_l.push_back(t.second); }
    pk.c = phase_turns(f.c);
    pk.nb = nb;
    pk.ntt = (int)tt_ab.size();
    pk.lt_off[0] = 0;
    for (int j = 0; j < kLowBits + kBlockBits; ++j) pk.lt_off[j + 1] = pk.lt_off[j] + (int)lt[j].size();
    // byte layout (16-byte aligned sections)
    auto al = [](size_t v) { return (v + 15) & ~(size_t)15; };
    size_t off = 0;
    pk.off_tt_ab = off; off = al(off + 4 * tt_ab.size());
    pk.off_tt_l = off;  off = al(off + 8 * tt_l.size());
    pk.off_lt_a = off;  off = al(off + 4 * lt_a.size());
    pk.off_lt_l = off;  off = al(off + 8 * lt_l.size());
    pk.off_small = off; off = al(off + 8 * small.size());
    pk.off_tmid = off;  off = al(off + (dtype == QSIM_C64 ? 8 : 16) * 32);
    out.assign(off, 0);
    auto put = [&](size_t o, const void* src, size_t bytes) { if (bytes) std::memcpy(out.data() + o, src, bytes); };
    put(pk.off_tt_ab, tt_ab.data(), 4 * tt_ab.size());
    put(pk.off_tt_l, tt_l.data(), 8 * tt_l.size());
    put(pk.off_lt_a, lt_a.data(), 4 * lt_a.size());
    put(pk.off_lt_l, lt_l.data(), 8 * lt_l.size());
    put(pk.off_small, small.data(), 8 * small.size());
    for (int m = 0; m < 32; ++m) {
        double ph = 0.0;
        for (int j = 0; j < 5; ++j)
            for (int k = j + 1; k < 5; ++k)
                if (((m >> j) & 1) && ((m >> k) & 1)) ph += midmid[j][k];
        const double re = std::cos(ph), im = std::sin(ph);
        if (dtype == QSIM_C64) {
            const float v[2] = {(float)re, (float)im};
            put(pk.off_tmid + 8 * m, v, 8);
        } else {
            const double v[2] = {re, im};
            put(pk.off_tmid + 16 * m, v, 16);
        }
    }
}

cudaError_t launch_phase(int dtype, void* psi, int n, const void* dtab, const PhasePacked& pk, cudaStream_t s,
                         const DevInfo& d) {
    if (n < phase::kLowBits || pk.nb != std::max(0, std::min(phase::kBlockBits, n - phase::kLowBits)))
        return cudaErrorInvalidValue;
    const unsigned char* b = static_cast<const unsigned char*>(dtab);
    phase::Args a;
    a.c = pk.c;
    a.nb = pk.nb;
    a.ntt = pk.ntt;
    for (int j = 0; j <= phase::kLowBits + phase::kBlockBits; ++j) a.lt_off[j] = pk.lt_off[j];
    a.tt_ab = reinterpret_cast<const uint32_t*>(b + pk.off_tt_ab);
    a.tt_l = reinterpret_cast<const uint64_t*>(b + pk.off_tt_l);
    a.lt_a = reinterpret_cast<const uint32_t*>(b + pk.off_lt_a);
    a.lt_l = reinterpret_cast<const uint64_t*>(b + pk.off_lt_l);
    a.small = reinterpret_cast<const uint64_t*>(b + pk.off_small);
    a.tmid = b + pk.off_tmid;
    const int64_t groups = (int64_t)1 << (n - phase::kLowBits - pk.nb);
    const unsigned grid = grid_for(groups * 32, 256, d.num_sms, 8);
    if (dtype == QSIM_C64) phase::k_phase<float><<<grid, 256, 0, s>>>(static_cast<float2*>(psi), n, a);
    else phase::k_phase<double><<<grid, 256, 0, s>>>(static_cast<double2*>(psi), n, a);
    return cudaGetLastError();
}

}  // namespace qsim
