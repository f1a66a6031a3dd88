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
// arithmetic, which is scarce on GB300. Each warp owns a range of 1024 consecutive amplitudes (index bits
// 10 and up fixed): lanes are index bits 0..4 (coalesced 256-byte accesses), and each lane's 32 amplitudes
// differ in bits 5..9. Per range the warp reduces the terms that involve the fixed high bits into
// s (a phase) and mu_j (a coefficient for each low bit j < 10); per lane this leaves
//     phi(lane, m) = s_lane + sum_e nu_e m_e + M(m)   (m = bits 5..9),
// evaluated as products of unit complex numbers in a depth-5 tree (no per-amplitude sin / cos).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>

#include "common.cuh"
#include "internal.h"

namespace qsim {
namespace phase {

constexpr int kLowBits = 10;  // a warp's range: 2^10 amplitudes
constexpr int kLaneBits = 5;

struct Args {
    uint64_t c;
    int nhh;                       // terms on two high bits (a single high bit appears as a == b)
    int lh_off[kLowBits + 1];      // terms (low bit j, high bit a) for j: [lh_off[j], lh_off[j+1])
    const uint32_t* hh_ab;         // a | b << 8
    const uint64_t* hh_l;
    const uint32_t* lh_a;          // the high bit
    const uint64_t* lh_l;
    const uint64_t* ll_lane;       // [32]: phase of the lane bits (bits 0..4) alone
    const uint64_t* lm;            // [32][5]: coefficient of bit 5+e given the lane bits (h and lane-mid terms)
    const void* tmid;              // [32] complex (state precision): exp(i * mid-mid terms of bits 5..9)
};

// exp(2 pi i t) for t = x / 2^64 turns.
__device__ __forceinline__ float2 unit_phase(float, uint64_t x) {
    // top 16 bits of the turn exactly in a float, the rest (under 2^-16 turns) by a short series
    const int32_t top = (int32_t)(x >> 32);
    const int32_t hi = top & (int32_t)0xFFFF0000;
    const float th = (float)hi * 0x1p-32f;
    const float tl = ((float)(top - hi) + (float)(uint32_t)x * 0x1p-32f) * 0x1p-32f;
    float sa, ca;
    sincospif(2.0f * th, &sa, &ca);
    const float b = tl * 6.28318530717958648f;
    const float sb = b - b * b * b * (1.0f / 6.0f), cb = 1.0f - 0.5f * b * b;
    return make_float2(ca * cb - sa * sb, sa * cb + ca * sb);
}
__device__ __forceinline__ double2 unit_phase(double, uint64_t x) {
    const double t = (double)(int64_t)x * 0x1p-64;
    double s, c;
    sincospi(2.0 * t, &s, &c);
    return make_double2(c, s);
}

template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
    V r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}

__device__ __forceinline__ uint64_t shfl_xor64(uint64_t v, int m) {
    const uint32_t lo = __shfl_xor_sync(0xffffffffu, (uint32_t)v, m);
    const uint32_t hi = __shfl_xor_sync(0xffffffffu, (uint32_t)(v >> 32), m);
    return ((uint64_t)hi << 32) | lo;
}
__device__ __forceinline__ uint64_t warp_sum64(uint64_t v) {
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) v += shfl_xor64(v, m);
    return v;
}

template <typename R>
__global__ void __launch_bounds__(256) k_phase(typename Amp<R>::T* __restrict__ psi, int n, const Args a) {
    using T = typename Amp<R>::T;
    constexpr int M = 1 << (kLowBits - kLaneBits);  // 32 amplitudes per lane
    const int lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    const uint64_t nr = 1ull << (n - kLowBits);
    const T* tmid = static_cast<const T*>(a.tmid);
    for (uint64_t rg = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); rg < nr; rg += warps) {
        const uint64_t base = rg << kLowBits;
        T v[M];
#pragma unroll
        for (int m = 0; m < M; ++m) v[m] = psi[base + ((uint64_t)m << kLaneBits) + lane];
        // terms on the fixed high bits
        uint64_t s = 0;
        for (int i = lane; i < a.nhh; i += 32) {
            const uint32_t ab = a.hh_ab[i];
            if ((base >> (ab & 0xFF)) & (base >> (ab >> 8)) & 1) s += a.hh_l[i];
        }
        s = warp_sum64(s) + a.c;
        uint64_t mu[kLowBits];
#pragma unroll
        for (int j = 0; j < kLowBits; ++j) {
            uint64_t t = 0;
            for (int i = a.lh_off[j] + lane; i < a.lh_off[j + 1]; i += 32)
                if ((base >> a.lh_a[i]) & 1) t += a.lh_l[i];
            mu[j] = warp_sum64(t);
        }
        // this lane's constant phase and the coefficients of bits 5..9
        uint64_t sl = s + a.ll_lane[lane];
#pragma unroll
        for (int j = 0; j < kLaneBits; ++j)
            if ((lane >> j) & 1) sl += mu[j];
        T F[M];
        F[0] = unit_phase(R(0), sl);
#pragma unroll
        for (int e = 0; e < kLowBits - kLaneBits; ++e) {
            const T B = unit_phase(R(0), mu[kLaneBits + e] + a.lm[lane * (kLowBits - kLaneBits) + e]);
#pragma unroll
            for (int m = 0; m < (1 << e); ++m) F[(1 << e) + m] = cmul(F[m], B);
        }
#pragma unroll
        for (int m = 0; m < M; ++m) psi[base + ((uint64_t)m << kLaneBits) + lane] = cmul(v[m], cmul(F[m], tmid[m]));
    }
}

}  // namespace phase

// ---- host: the quadratic form of a run of diagonal gates -------------------------------------------------------
namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;

uint64_t to_turns(double phi) {
    double t = phi / kTwoPi;
    t -= std::floor(t);
    if (!(t < 1.0)) t = 0.0;
    return (uint64_t)std::ldexp(t, 64);  // t < 1, so the value fits; 53 significant bits
}

}  // namespace

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
    std::vector<uint32_t> hh_ab, lh_a;
    std::vector<uint64_t> hh_l, lh_l;
    std::vector<std::vector<std::pair<uint32_t, uint64_t>>> lh(kLowBits);
    uint64_t c = to_turns(f.c);
    std::vector<uint64_t> hlow(kLowBits, 0);
    for (int a = 0; a < n; ++a) {
        if (f.h[a] == 0.0) continue;
        if (a >= kLowBits) { hh_ab.push_back((uint32_t)a | ((uint32_t)a << 8)); hh_l.push_back(to_turns(f.h[a])); }
        else hlow[a] = to_turns(f.h[a]);
    }
    // low-low terms: lane-lane, lane-mid, mid-mid
    std::vector<uint64_t> ll_lane(32, 0), lm(32 * 5, 0);
    double midmid[5][5] = {};
    uint64_t lanelane[5][5] = {};
    for (const auto& p : f.pairs) {
        if (p.a >= kLowBits) { hh_ab.push_back((uint32_t)p.a | ((uint32_t)p.b << 8)); hh_l.push_back(to_turns(p.lam)); }
        else if (p.b >= kLowBits) lh[p.a].push_back({(uint32_t)p.b, to_turns(p.lam)});
        else if (p.b < kLaneBits) lanelane[p.a][p.b] += to_turns(p.lam);
        else if (p.a < kLaneBits) {
            for (int l = 0; l < 32; ++l)
                if ((l >> p.a) & 1) lm[l * 5 + (p.b - kLaneBits)] += to_turns(p.lam);
        } else {
            midmid[p.a - kLaneBits][p.b - kLaneBits] += p.lam;
        }
    }
    for (int l = 0; l < 32; ++l) {
        uint64_t v = 0;
        for (int j = 0; j < kLaneBits; ++j) {
            if (!((l >> j) & 1)) continue;
            v += hlow[j];
            for (int k = j + 1; k < kLaneBits; ++k)
                if ((l >> k) & 1) v += lanelane[j][k];
        }
        ll_lane[l] = v;
        for (int e = 0; e < 5; ++e) lm[l * 5 + e] += hlow[kLaneBits + e];
    }
    for (int j = 0; j < kLowBits; ++j)
        for (const auto& t : lh[j]) { lh_a.push_back(t.first); lh_l.push_back(t.second); }
    pk.c = c;
    pk.nhh = (int)hh_ab.size();
    pk.lh_off[0] = 0;
    for (int j = 0; j < kLowBits; ++j) pk.lh_off[j + 1] = pk.lh_off[j] + (int)lh[j].size();
    // byte layout (16-byte aligned sections)
    auto al = [](size_t v) { return (v + 15) & ~(size_t)15; };
    size_t off = 0;
    pk.off_hh_ab = off; off = al(off + 4 * hh_ab.size());
    pk.off_hh_l = off;  off = al(off + 8 * hh_l.size());
    pk.off_lh_a = off;  off = al(off + 4 * lh_a.size());
    pk.off_lh_l = off;  off = al(off + 8 * lh_l.size());
    pk.off_ll = off;    off = al(off + 8 * 32);
    pk.off_lm = off;    off = al(off + 8 * 32 * 5);
    pk.off_tmid = off;  off = al(off + (dtype == QSIM_C64 ? 8 : 16) * 32);
    out.assign(off, 0);
    auto put = [&](size_t o, const void* src, size_t bytes) { if (bytes) std::memcpy(out.data() + o, src, bytes); };
    put(pk.off_hh_ab, hh_ab.data(), 4 * hh_ab.size());
    put(pk.off_hh_l, hh_l.data(), 8 * hh_l.size());
    put(pk.off_lh_a, lh_a.data(), 4 * lh_a.size());
    put(pk.off_lh_l, lh_l.data(), 8 * lh_l.size());
    put(pk.off_ll, ll_lane.data(), 8 * 32);
    put(pk.off_lm, lm.data(), 8 * 32 * 5);
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
    if (n < phase::kLowBits) return cudaErrorInvalidValue;
    const unsigned char* b = static_cast<const unsigned char*>(dtab);
    phase::Args a;
    a.c = pk.c;
    a.nhh = pk.nhh;
    for (int j = 0; j <= phase::kLowBits; ++j) a.lh_off[j] = pk.lh_off[j];
    a.hh_ab = reinterpret_cast<const uint32_t*>(b + pk.off_hh_ab);
    a.hh_l = reinterpret_cast<const uint64_t*>(b + pk.off_hh_l);
    a.lh_a = reinterpret_cast<const uint32_t*>(b + pk.off_lh_a);
    a.lh_l = reinterpret_cast<const uint64_t*>(b + pk.off_lh_l);
    a.ll_lane = reinterpret_cast<const uint64_t*>(b + pk.off_ll);
    a.lm = reinterpret_cast<const uint64_t*>(b + pk.off_lm);
    a.tmid = b + pk.off_tmid;
    const int64_t ranges = (int64_t)1 << (n - phase::kLowBits);
    const unsigned grid = grid_for(ranges * 32, 256, d.num_sms, 8);
    if (dtype == QSIM_C64) phase::k_phase<float><<<grid, 256, 0, s>>>(static_cast<float2*>(psi), n, a);
    else phase::k_phase<double><<<grid, 256, 0, s>>>(static_cast<double2*>(psi), n, a);
    return cudaGetLastError();
}

}  // namespace qsim
