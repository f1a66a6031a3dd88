// batch.cu -- many independent circuits in one persistent launch (paper Sec. 1: simulating many circuits,
// e.g. for iterative algorithms, is one reason for large GPU resources; Sec. 2.2 times circuits one by one).
//
// Each circuit is fused on the host (greedy, width k chosen per circuit width by a built-in tuner or given),
// every block is composed in FP64 on the device and stored as a complex64 matrix. One launch of k_batch then
// runs everything:
//   * a persistent grid of thread-block clusters (16 CTAs where the device co-schedules them, else 8);
//     each cluster claims the next large circuit
//     (n >= 14) from a device counter, keeps its state in the caller's workspace, applies the passes with
//     hardware cluster barriers between them, and reduces <Z_i>, <Z_i Z_{i+1}> across the cluster through
//     distributed shared memory;
//   * once the large queue is empty, every CTA claims small circuits (n <= 13) one at a time and runs each
//     entirely in its shared memory (64 KiB), with no global traffic for the state at all.
// There are no spin waits: the only waits are hardware barriers (__syncthreads, cluster barriers).
// With a tensor-core precision, circuits of at least batch_tc_min_n qubits (default 20) leave the persistent
// launch: one cluster streams a state at a fraction of the GPU's bandwidth (about 0.44 TB/s for a 16-CTA
// cluster on a 24-qubit state, where the whole GPU does 6.5), so each becomes a fused tensor-core plan
// (6-qubit blocks, or up to 7 with FP16X3) enqueued after the launch, its first block generating |0>, its <Z>
// values reduced on the device into the same output arrays. These plans run on eight worker streams forked
// from the caller's stream and joined back, so that one circuit's pipeline fill and drain overlap another's
// passes (the narrower circuits' kernels on a half or a quarter of the SMs, side by side). The whole enqueue
// is one CUDA graph when replayed.
#include <cooperative_groups.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <atomic>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "capi_state.h"
#include "common.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace qsim {
namespace batch {

constexpr int kThreads = 256;
constexpr int kKmax = 4;
constexpr int kSmallMax = 13;  // largest width kept in shared memory (2^13 x 8 B = 64 KiB)
constexpr size_t kWideStreams = 8;  // worker streams for the circuits run as tensor-core plans
constexpr int kHalfGridBelow = 24;     // wide circuits narrower than this run their plans on half the SMs,
constexpr int kQuarterGridBelow = 22;  // and narrower than this on a quarter of them

struct Pass {
    int k;
    int targets[kKmax];  // ascending; bit j of the matrix index <-> targets[j]
    int64_t mat_off;     // complex entries into the matrix pool
};
struct Circ {
    int n;
    int npass;
    int64_t first_pass;
    int64_t state_off;  // amplitudes into the workspace (large circuits only)
    int zi_off, zz_off;
};
struct Args {
    const Pass* passes;
    const Circ* circs;  // large circuits first, then small ones
    int nlarge, nsmall;
    const float2* mats;
    float2* ws;
    double* zi;
    double* zz;
    int* counters;  // [0] next large circuit, [1] next small circuit
};

struct Shared {
    float2 state[1 << kSmallMax];
    float2 U[1 << (2 * kKmax)];
    uint64_t off[1 << kKmax];  // gather offsets of the current pass
    ff seg[8][24];
    double segT, segS11;
    dd red[64];
    int claim;
};

// ---- dense pass: groups g0, g0 + stride, ... of psi (global or shared memory) ---------------------------
template <int K>
__device__ __noinline__ void apply_dense(float2* psi, int n, const int* tg, const float2* U, const uint64_t* off,
                                        uint64_t g0, uint64_t stride) {
    constexpr int D = 1 << K;
    const uint64_t G = 1ull << (n - K);
    if (tg[0] >= 1 && G >= 2) {
        // qubit 0 is not a target: groups 2h and 2h+1 are adjacent amplitudes, one 16-byte vector each
        for (uint64_t h = g0; h < G / 2; h += stride) {
            const uint64_t base = insert_zeros(2 * h, tg, K);
            float4 v[D];
#pragma unroll
            for (int m = 0; m < D; ++m) v[m] = *reinterpret_cast<const float4*>(psi + base + off[m]);
#pragma unroll
            for (int r = 0; r < D; ++r) {
                float r0 = 0.f, i0 = 0.f, r1 = 0.f, i1 = 0.f;
#pragma unroll
                for (int c = 0; c < D; ++c) {
                    const float2 u = U[r * D + c];
                    r0 = __fmaf_rn(u.x, v[c].x, r0); r0 = __fmaf_rn(-u.y, v[c].y, r0);
                    i0 = __fmaf_rn(u.x, v[c].y, i0); i0 = __fmaf_rn(u.y, v[c].x, i0);
                    r1 = __fmaf_rn(u.x, v[c].z, r1); r1 = __fmaf_rn(-u.y, v[c].w, r1);
                    i1 = __fmaf_rn(u.x, v[c].w, i1); i1 = __fmaf_rn(u.y, v[c].z, i1);
                }
                *reinterpret_cast<float4*>(psi + base + off[r]) = make_float4(r0, i0, r1, i1);
            }
        }
        return;
    }
    for (uint64_t g = g0; g < G; g += stride) {
        const uint64_t base = insert_zeros(g, tg, K);
        float2 v[D];
#pragma unroll
        for (int m = 0; m < D; ++m) v[m] = psi[base + off[m]];
#pragma unroll
        for (int r = 0; r < D; ++r) {
            float re = 0.f, im = 0.f;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const float2 u = U[r * D + c];
                re = __fmaf_rn(u.x, v[c].x, re);
                re = __fmaf_rn(-u.y, v[c].y, re);
                im = __fmaf_rn(u.x, v[c].y, im);
                im = __fmaf_rn(u.y, v[c].x, im);
            }
            psi[base + off[r]] = make_float2(re, im);
        }
    }
}

__device__ __noinline__ void apply_pass(float2* psi, int n, const Pass& P, const float2* U, const uint64_t* off,
                                       uint64_t g0, uint64_t stride) {
    switch (P.k) {
        case 1: apply_dense<1>(psi, n, P.targets, U, off, g0, stride); break;
        case 2: apply_dense<2>(psi, n, P.targets, U, off, g0, stride); break;
        case 3: apply_dense<3>(psi, n, P.targets, U, off, g0, stride); break;
        default: apply_dense<4>(psi, n, P.targets, U, off, g0, stride); break;
    }
}

// Load a pass's matrix and gather offsets into shared memory (the caller synchronises afterwards).
__device__ __forceinline__ void load_pass(const Args& a, const Pass& P, Shared& sh) {
    const int t = threadIdx.x;
    const int DD = 1 << (2 * P.k);
    for (int i = t; i < DD; i += kThreads) sh.U[i] = a.mats[P.mat_off + i];
    if (t < (1 << P.k)) {
        uint64_t o = 0;
        for (int j = 0; j < P.k; ++j) o |= (uint64_t)((t >> j) & 1) << P.targets[j];
        sh.off[t] = o;
    }
}

__device__ __forceinline__ ff p_of(const float2* psi, uint64_t i) {
    const float2 v = psi[i];
    return ff_abs2(v.x, v.y);
}

// One 4096-amplitude segment: the 24 quantities of index bits 0..11 (T, S_0..S_11, X_0..X_10; see
// k_reduce.cu for the thread layout), block-reduced. Thread q < 24 receives quantity q; the segment total
// and its S_11 part are left in sh.segT / sh.segS11.
__device__ __noinline__ double segment_stats(const float2* psi, uint64_t s, Shared& sh) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint64_t base = (s << 12) + 2 * t;
    ff P[8], Q[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const ff p0 = p_of(psi, base + 512 * j), p1 = p_of(psi, base + 512 * j + 1);
        Q[j] = p1;
        P[j] = ff_add(p0, p1);
    }
    ff T = P[0], S0 = Q[0];
#pragma unroll
    for (int j = 1; j < 8; ++j) { T = ff_add(T, P[j]); S0 = ff_add(S0, Q[j]); }
    const ff S9 = ff_add(ff_add(P[1], P[3]), ff_add(P[5], P[7]));
    const ff Z = {0.f, 0.f};
    ff c[24];
    c[0] = T;
    c[1] = S0;
#pragma unroll
    for (int i = 1; i <= 8; ++i) c[1 + i] = ((t >> (i - 1)) & 1) ? T : Z;
    c[10] = S9;
    c[11] = ff_add(ff_add(P[2], P[3]), ff_add(P[6], P[7]));
    c[12] = ff_add(ff_add(P[4], P[5]), ff_add(P[6], P[7]));
    c[13] = (t & 1) ? ff_add(T, ff_neg(S0)) : S0;
#pragma unroll
    for (int i = 1; i <= 7; ++i) c[13 + i] = (((t >> (i - 1)) ^ (t >> i)) & 1) ? T : Z;
    c[21] = ((t >> 7) & 1) ? ff_add(T, ff_neg(S9)) : S9;
    c[22] = ff_add(ff_add(P[1], P[2]), ff_add(P[5], P[6]));
    c[23] = ff_add(ff_add(P[2], P[3]), ff_add(P[4], P[5]));
#pragma unroll
    for (int q = 0; q < 24; ++q) {
        const ff v = warp_sum_ff(c[q]);
        if (lane == 0) sh.seg[warp][q] = v;
    }
    __syncthreads();
    double val = 0.0;
    if (t < 24) {
        ff v = sh.seg[0][t];
#pragma unroll
        for (int w = 1; w < 8; ++w) v = ff_add(v, sh.seg[w][t]);
        val = (double)v.hi + (double)v.lo;
        if (t == 0) sh.segT = val;
        if (t == 12) sh.segS11 = val;
    }
    __syncthreads();
    return val;
}

// Quantity layout of the partial sums red[0 .. 24 + 2 nh): [0, 24) bits 0..11 as in segment_stats; then
// S_{12..n-1} (nh values), X_11, X_{12..n-2} (nh - 1 values); nh = n - 12.
__device__ void zstats_segments(const float2* psi, int n, uint64_t s0, uint64_t sstride, Shared& sh) {
    const int t = threadIdx.x;
    const int nh = n - 12;
    const uint64_t nseg = 1ull << nh;
    dd acc = {0.0, 0.0};
    for (uint64_t s = s0; s < nseg; s += sstride) {
        const double v = segment_stats(psi, s, sh);
        if (t < 24) {
            acc = dd_add(acc, dd{v, 0.0});
        } else if (t < 24 + 2 * nh) {
            const int h = t - 24;
            const double T = sh.segT, S11 = sh.segS11;
            double add = 0.0;
            if (h < nh) add = ((s >> h) & 1) ? T : 0.0;
            else if (h == nh) add = (s & 1) ? T - S11 : S11;
            else { const int r = h - nh - 1; add = (((s >> r) ^ (s >> (r + 1))) & 1) ? T : 0.0; }
            acc = dd_add(acc, dd{add, 0.0});
        }
        __syncthreads();
    }
    if (t < 64) sh.red[t] = acc;
    __syncthreads();
}

// Small widths (n < 12): quantity q = 0 -> T, 1..n -> S_{q-1}, n+1..2n-1 -> X_{q-n-1}, one thread each.
__device__ __noinline__ void zstats_serial(const float2* psi, int n, Shared& sh) {
    const int q = threadIdx.x;
    if (q < 2 * n) {
        ff acc = {0.f, 0.f};
        const int N = 1 << n;
        for (int x = 0; x < N; ++x) {
            bool use;
            if (q == 0) use = true;
            else if (q <= n) use = (x >> (q - 1)) & 1;
            else { const int i = q - n - 1; use = ((x >> i) ^ (x >> (i + 1))) & 1; }
            if (use) acc = ff_add(acc, p_of(psi, x));
        }
        sh.red[q] = dd{(double)acc.hi + (double)acc.lo, 0.0};
    }
    __syncthreads();
}

__device__ __forceinline__ double dval(dd v) { return v.hi + v.lo; }

// Write <Z_i>, <Z_i Z_{i+1}> from the quantity vector red (layout of zstats_segments / zstats_serial),
// normalised by the state's squared norm T: the exact state of a circuit from |0...0> has norm 1, and
// dividing by T removes the FP32 drift of the norm from the reported values.
__device__ void write_z(const dd* red, int n, double* zi, double* zz) {
    const int t = threadIdx.x;
    if (n < 12) {
        const double T = dval(red[0]);
        if (t < n) zi[t] = (T - 2.0 * dval(red[1 + t])) / T;
        if (t < n - 1) zz[t] = (T - 2.0 * dval(red[n + 1 + t])) / T;
        return;
    }
    const int nh = n - 12;
    const double T = dval(red[0]);
    if (t < n) zi[t] = (T - 2.0 * dval(t < 12 ? red[1 + t] : red[24 + (t - 12)])) / T;
    if (t < n - 1) {
        const dd X = t <= 10 ? red[13 + t] : (t == 11 ? red[24 + nh] : red[24 + nh + 1 + (t - 12)]);
        zz[t] = (T - 2.0 * dval(X)) / T;
    }
}

__global__ void __launch_bounds__(kThreads, 2) k_batch(const __grid_constant__ Args a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Shared& sh = *reinterpret_cast<Shared*>(smem_raw);
    cg::cluster_group cl = cg::this_cluster();
    const unsigned rank = cl.block_rank(), CL = cl.num_blocks();
    const int t = threadIdx.x;

    // ---- large circuits: one cluster per circuit ------------------------------------------------------
    while (true) {
        if (rank == 0 && t == 0) sh.claim = atomicAdd(&a.counters[0], 1);
        cl.sync();
        const int idx = *cl.map_shared_rank(&sh.claim, 0);
        cl.sync();
        if (idx >= a.nlarge) break;
        const Circ c = a.circs[idx];
        float2* psi = a.ws + c.state_off;
        const uint64_t N = 1ull << c.n;
        const uint64_t gid = (uint64_t)rank * kThreads + t, gstride = (uint64_t)CL * kThreads;
        for (uint64_t i = gid; i < N; i += gstride) psi[i] = make_float2(i == 0 ? 1.f : 0.f, 0.f);
        cl.sync();
        for (int p = 0; p < c.npass; ++p) {
            const Pass P = a.passes[c.first_pass + p];
            load_pass(a, P, sh);
            __syncthreads();
            apply_pass(psi, c.n, P, sh.U, sh.off, gid, gstride);
            cl.sync();  // release / acquire at cluster scope: the next pass sees every CTA's stores
        }
        zstats_segments(psi, c.n, rank, CL, sh);
        cl.sync();
        if (rank == 0 && t < 24 + 2 * (c.n - 12)) {
            dd v = sh.red[t];
            for (unsigned r2 = 1; r2 < CL; ++r2) v = dd_add(v, cl.map_shared_rank(sh.red, r2)[t]);
            sh.red[t] = v;
        }
        cl.sync();
        if (rank == 0) write_z(sh.red, c.n, a.zi + c.zi_off, a.zz + c.zz_off);
    }

    // ---- small circuits: one CTA per circuit, the state in shared memory ---------------------------------
    while (true) {
        if (t == 0) sh.claim = atomicAdd(&a.counters[1], 1);
        __syncthreads();
        const int idx = sh.claim;
        __syncthreads();
        if (idx >= a.nsmall) break;
        const Circ c = a.circs[a.nlarge + idx];
        float2* psi = sh.state;
        const int N = 1 << c.n;
        for (int i = t; i < N; i += kThreads) psi[i] = make_float2(i == 0 ? 1.f : 0.f, 0.f);
        for (int p = 0; p < c.npass; ++p) {
            const Pass P = a.passes[c.first_pass + p];
            load_pass(a, P, sh);
            __syncthreads();
            apply_pass(psi, c.n, P, sh.U, sh.off, t, kThreads);
            __syncthreads();
        }
        if (c.n >= 12) zstats_segments(psi, c.n, 0, 1, sh);
        else zstats_serial(psi, c.n, sh);
        write_z(sh.red, c.n, a.zi + c.zi_off, a.zz + c.zz_off);
        __syncthreads();
    }
}

// ---- host side ----------------------------------------------------------------------------------------------
std::mutex g_tune_mu;
int g_tuned_k[QSIM_MAX_QUBITS + 1] = {0};
int g_tuned_tc_min_n[5] = {0, 0, 0, 0, 0};  // per tensor-core precision; 0 = not tuned (default 20)
bool g_cache_loaded = false;

int tuned_k(int n) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    return g_tuned_k[n] ? g_tuned_k[n] : kKmax;
}

int tuned_tc_min_n(int precision) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    const int v = (precision >= 1 && precision <= 4) ? g_tuned_tc_min_n[precision] : 0;
    return v ? v : 20;
}

// The tuning table as a small JSON object: fusion width per circuit width, and per tensor-core precision the
// smallest width that runs as a tensor-core plan.
std::string tune_json() {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    std::string o = "{\"format\": \"qsim-batch-tune-1\", \"k_by_width\": {";
    bool first = true;
    for (int n = 1; n <= QSIM_MAX_QUBITS; ++n)
        if (g_tuned_k[n]) {
            o += (first ? "\"" : ", \"") + std::to_string(n) + "\": " + std::to_string(g_tuned_k[n]);
            first = false;
        }
    o += "}, \"tc_min_n\": {";
    first = true;
    for (int p = 1; p <= 4; ++p)
        if (g_tuned_tc_min_n[p]) {
            o += (first ? "\"" : ", \"") + std::to_string(p) + "\": " + std::to_string(g_tuned_tc_min_n[p]);
            first = false;
        }
    return o + "}}\n";
}

// Read the "key": value integer pairs of the object that follows `name` in `text` (the format tune_json
// writes); false if the object is missing or malformed.
bool read_int_object(const std::string& text, const char* name, std::vector<std::pair<int, int>>& out) {
    const std::string key = std::string("\"") + name + "\"";
    size_t i = text.find(key);
    if (i == std::string::npos) return false;
    i = text.find('{', i + key.size());
    const size_t end = i == std::string::npos ? i : text.find('}', i);
    if (end == std::string::npos) return false;
    const std::string body = text.substr(i + 1, end - i - 1);
    size_t j = 0;
    while (true) {
        const size_t q0 = body.find('"', j);
        if (q0 == std::string::npos) return true;
        const size_t q1 = body.find('"', q0 + 1);
        const size_t colon = q1 == std::string::npos ? q1 : body.find(':', q1);
        if (colon == std::string::npos) return false;
        char* e1 = nullptr;
        char* e2 = nullptr;
        const long k = std::strtol(body.c_str() + q0 + 1, &e1, 10);
        const long v = std::strtol(body.c_str() + colon + 1, &e2, 10);
        if (e1 != body.c_str() + q1 || e2 == body.c_str() + colon + 1) return false;
        out.emplace_back((int)k, (int)v);
        j = (size_t)(e2 - body.c_str());
    }
}

int tune_load_file(const char* path) {
    FILE* f = std::fopen(path, "rb");
    if (!f) { set_error("cannot open tuning file %s", path); return QSIM_EINVAL; }
    std::string text;
    char buf[4096];
    size_t got;
    while ((got = std::fread(buf, 1, sizeof(buf), f)) > 0 && text.size() < (1u << 20)) text.append(buf, got);
    std::fclose(f);
    std::vector<std::pair<int, int>> ks, ts;
    if (text.find("qsim-batch-tune-1") == std::string::npos || !read_int_object(text, "k_by_width", ks) ||
        !read_int_object(text, "tc_min_n", ts)) {
        set_error("%s is not a batch tuning file", path);
        return QSIM_EINVAL;
    }
    for (const auto& kv : ks)
        if (kv.first < 1 || kv.first > QSIM_MAX_QUBITS || kv.second < 1 || kv.second > kKmax) {
            set_error("%s: fusion width %d for %d qubits out of range", path, kv.second, kv.first);
            return QSIM_EINVAL;
        }
    for (const auto& kv : ts)
        if (kv.first < 1 || kv.first > 4 || kv.second < 13 || kv.second > 27) {
            set_error("%s: tc_min_n %d for precision %d out of range", path, kv.second, kv.first);
            return QSIM_EINVAL;
        }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (const auto& kv : ks) g_tuned_k[kv.first] = kv.second;
    for (const auto& kv : ts) g_tuned_tc_min_n[kv.first] = kv.second;
    return QSIM_OK;
}

int tune_save_file(const char* path) {
    const std::string j = tune_json();
    FILE* f = std::fopen(path, "wb");
    if (!f) { set_error("cannot write tuning file %s", path); return QSIM_EINVAL; }
    const bool ok = std::fwrite(j.data(), 1, j.size(), f) == j.size();
    if (std::fclose(f) != 0 || !ok) { set_error("writing tuning file %s failed", path); return QSIM_EINVAL; }
    return QSIM_OK;
}

// QSIM_TUNE_CACHE names a tuning file: read once before the first batch plan, written after every tuning.
void tune_cache_autoload() {
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        if (g_cache_loaded) return;
        g_cache_loaded = true;
    }
    const char* p = std::getenv("QSIM_TUNE_CACHE");
    if (p && *p) {
        FILE* f = std::fopen(p, "rb");
        if (f) { std::fclose(f); tune_load_file(p); }
    }
}

void tune_cache_autosave() {
    const char* p = std::getenv("QSIM_TUNE_CACHE");
    if (p && *p) tune_save_file(p);
}

}  // namespace batch
}  // namespace qsim

struct qsim_batch {
    int count = 0;
    std::vector<int> widths;
    int nlarge = 0, nsmall = 0;
    void* dbuf = nullptr;
    qsim::batch::Args args{};
    size_t ws_need = 0;
    int total_zi = 0, total_zz = 0;
    int grid = 0;
    int cluster = 8;
    qsim_plan_info info{};
    cudaGraphExec_t gexec = nullptr;
    void* gws = nullptr;
    cudaStream_t gstream = nullptr;
    // wide circuits as tensor-core plans: plan, width, state offset (amplitudes), <Z> offsets
    std::vector<qsim_plan_h> wide_plans;
    std::vector<int> wide_n;
    std::vector<int64_t> wide_state_off;
    std::vector<int> wide_zi_off, wide_zz_off;
    unsigned* derr = nullptr;   // device error word of their tensor-core launches
    qsim::DevInfo dev;
    // The wide circuits are independent: they run on a few worker streams forked from the caller's stream
    // and joined back (one graph branch each), so that one circuit's pipeline fill and drain overlap
    // another's passes. Per worker: its stream, <Z> scratch (device buffers; hresult unused), join event.
    std::vector<cudaStream_t> wstreams;
    std::vector<qsim::ReduceScratch> reds;
    std::vector<cudaEvent_t> join_ev;
    cudaEvent_t fork_ev = nullptr;
    std::vector<int> wide_worker;  // worker of each wide circuit (longest first, to the least-loaded worker)
};

using namespace qsim;

namespace {

size_t small_state_bytes(int n) { return (size_t)8 << n; }

int validate_batch(const qsim_circuit* cs, int count) {
    if (!cs || count < 1) { set_error("need at least one circuit"); return QSIM_EINVAL; }
    for (int i = 0; i < count; ++i) {
        if (cs[i].n < 1 || cs[i].n > 26) { set_error("circuit %d: batched widths are 1..26", i); return QSIM_EINVAL; }
        if (cs[i].num_gates < 0 || (cs[i].num_gates > 0 && !cs[i].gates)) { set_error("circuit %d: bad gate list", i); return QSIM_EINVAL; }
    }
    return QSIM_OK;
}

// Run fn(i, t) for i in [0, count) on up to `threads` host threads (t = the thread's index, each thread with
// `device` current). The first failure (lowest i) is reported on the calling thread, with its message.
int parallel_for(int count, int threads, int device, const std::function<int(int, int)>& fn) {
    threads = std::max(1, std::min(threads, count));
    std::vector<int> rcs(count, QSIM_OK);
    std::vector<std::string> msgs(count);
    std::atomic<int> next{0};
    auto work = [&](int t) {
        if (t > 0) cudaSetDevice(device);
        for (int i = next++; i < count; i = next++) {
            rcs[i] = fn(i, t);
            if (rcs[i]) msgs[i] = qsim_last_error();
        }
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < threads; ++t) pool.emplace_back(work, t);
    work(0);
    for (auto& th : pool) th.join();
    for (int i = 0; i < count; ++i)
        if (rcs[i]) { set_error("%s", msgs[i].c_str()); return rcs[i]; }
    return QSIM_OK;
}

int host_threads(int work_items) {
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    return (int)std::min<unsigned>(std::min(hw, 16u), (unsigned)std::max(1, work_items / 4));
}

}  // namespace

extern "C" {

int qsim_batch_workspace_bytes(const qsim_circuit* cs, int count, size_t* out) {
    set_error("%s", "");
    if (!out) { set_error("NULL output"); return QSIM_EINVAL; }
    int rc = validate_batch(cs, count);
    if (rc) return rc;
    size_t b = 0;
    for (int i = 0; i < count; ++i)
        if (cs[i].n > batch::kSmallMax) b += (small_state_bytes(cs[i].n) + 255) & ~(size_t)255;
    *out = b;
    return QSIM_OK;
}

static int batch_launch(qsim_batch_h b, cudaStream_t s);
static int enqueue_wide(qsim_batch_h b, qsim_plan_h plan, size_t w, int k, void* dev_ws);

// Planning of a batch. With run_ws (the one-shot qsim_batch_run) the batch is also executed while it is
// planned: the persistent launch of the narrower circuits goes out as soon as they are planned, and each wide
// circuit's plan is enqueued on a worker stream as soon as it is made, so that the GPU runs the first
// tensor-core plans while the host still plans the others; the worker streams are joined back into `stream`
// before returning. (The running plans hold the SMs that the planning's own kernels need, so planning takes
// longer; measured on the 256-chain batch the overlap still wins: 124 ms from host circuits to host results
// against 130 ms planning first and 128 ms with only the persistent launch overlapped.)
static int batch_plan_create_impl(const qsim_circuit* cs, int count, const qsim_run_opts* opts_in, void* stream_v,
                                  qsim_batch_h* out, qsim_plan_info* info, void* run_ws) {
    set_error("%s", "");
    const auto t0 = std::chrono::steady_clock::now();
    if (!out) { set_error("NULL output"); return QSIM_EINVAL; }
    *out = nullptr;
    int rc = validate_batch(cs, count);
    if (rc) return rc;
    qsim_run_opts opts{};
    if (opts_in) opts = *opts_in;
    if (opts.max_fused < 0 || opts.max_fused > batch::kKmax) { set_error("batched fusion width must be 0 (tuned) or 1..%d", batch::kKmax); return QSIM_EINVAL; }
    if (opts.precision < QSIM_PREC_SIMT || opts.precision > QSIM_PREC_FP16X3) { set_error("unknown precision"); return QSIM_EINVAL; }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_v);
    // circuits this wide run as tensor-core plans (6-qubit blocks need n >= 13); 0 = the tuned threshold
    batch::tune_cache_autoload();
    const int tc_min_n = opts.precision == QSIM_PREC_SIMT ? 1000
                         : (opts.batch_tc_min_n > 0 ? std::max(13, opts.batch_tc_min_n) : batch::tuned_tc_min_n(opts.precision));
    std::vector<char> wide(count, 0);
    for (int ci = 0; ci < count; ++ci) wide[ci] = cs[ci].n >= tc_min_n;

    // ---- plan every circuit ---------------------------------------------------------------------------
    std::vector<ComposeBlock> cblocks;
    std::vector<ComposeGate> cgates;
    std::vector<double> pool;
    std::vector<batch::Pass> passes;
    std::vector<batch::Circ> circs(count);
    int64_t compose_out = 0;
    int64_t gates_total = 0;
    double bytes = 0.0;
    // validation and fusion of every circuit, on several host threads (circuits are independent)
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) { cudaGetLastError(); device = 0; }
    std::vector<std::vector<uint64_t>> gmasks(count);
    std::vector<std::vector<std::vector<int>>> cblk(count);
    rc = parallel_for(count, host_threads(count), device, [&](int ci, int) -> int {
        const qsim_circuit& c = cs[ci];
        const int n = c.n;
        std::vector<uint64_t>& gmask = gmasks[ci];
        gmask.resize(c.num_gates);
        std::vector<char> gdiag(c.num_gates);
        for (int i = 0; i < c.num_gates; ++i) {
            const qsim_gate& g = c.gates[i];
            const int vrc = validate_qubits(n, g.targets, g.k, g.controls, g.nc, batch::kKmax);
            if (vrc || g.k + g.nc > batch::kKmax) { set_error("circuit %d gate %d: batched gates act on at most %d qubits", ci, i, batch::kKmax); return QSIM_EINVAL; }
            if (!g.matrix || !is_unitary(g.matrix, g.k, 1e-8 * (1 << g.k))) { set_error("circuit %d gate %d: matrix missing or not unitary", ci, i); return QSIM_EINVAL; }
            uint64_t m = 0;
            for (int j = 0; j < g.k; ++j) m |= 1ull << g.targets[j];
            for (int j = 0; j < g.nc; ++j) m |= 1ull << g.controls[j];
            gmask[i] = m;
            gdiag[i] = is_diagonal(g.matrix, g.k);
        }
        if (!wide[ci]) {
            const int kmax = std::min(n, opts.max_fused ? opts.max_fused : batch::tuned_k(n));
            std::vector<uint64_t> key = {1 /* a batch circuit */, (uint64_t)n, (uint64_t)kmax, (uint64_t)c.num_gates};
            key.reserve(key.size() + 2 * (size_t)c.num_gates);
            for (int i = 0; i < c.num_gates; ++i) { key.push_back(gmask[i]); key.push_back((uint64_t)gdiag[i]); }
            if (!group_cache_get(key, cblk[ci])) {
                cblk[ci] = group_gates(gmask, gdiag, n, kmax);
                group_cache_put(key, cblk[ci]);
            }
        }
        return QSIM_OK;
    });
    if (rc) return rc;
    for (int ci = 0; ci < count; ++ci) {
        const qsim_circuit& c = cs[ci];
        const int n = c.n;
        const std::vector<uint64_t>& gmask = gmasks[ci];
        gates_total += c.num_gates;
        circs[ci].n = n;
        if (wide[ci]) { circs[ci].npass = 0; circs[ci].first_pass = (int64_t)passes.size(); continue; }
        const auto& blocks = cblk[ci];
        circs[ci].npass = (int)blocks.size();
        circs[ci].first_pass = (int64_t)passes.size();
        for (const auto& blk : blocks) {
            uint64_t Q = 0;
            for (int gi : blk) Q |= gmask[gi];
            int local[64], kb = 0;
            batch::Pass P{};
            for (int q = 0; q < n; ++q)
                if ((Q >> q) & 1) { local[q] = kb; P.targets[kb++] = q; }
            P.k = kb;
            P.mat_off = compose_out;
            ComposeBlock cb{kb, (int)cgates.size(), (int)blk.size(), compose_out};
            compose_out += (int64_t)1 << (2 * kb);
            for (int gi : blk) {
                const qsim_gate& g = c.gates[gi];
                ComposeGate cg_{};
                cg_.k = g.k;
                cg_.nc = g.nc;
                for (int j = 0; j < g.k; ++j) cg_.targets[j] = local[g.targets[j]];
                for (int j = 0; j < g.nc; ++j) cg_.controls[j] = local[g.controls[j]];
                cg_.mat_off = (int64_t)pool.size() / 2;
                pool.insert(pool.end(), g.matrix, g.matrix + (2 << (2 * g.k)));
                cgates.push_back(cg_);
            }
            cblocks.push_back(cb);
            passes.push_back(P);
            if (n > batch::kSmallMax) bytes += 16.0 * std::ldexp(1.0, n);
        }
    }

    // ---- order: large circuits (most work first), then small ones; workspace and output offsets ------------
    qsim_batch* b = new (std::nothrow) qsim_batch();
    if (!b) { set_error("out of host memory"); return QSIM_ENOMEM; }
    b->count = count;
    std::vector<int> order;
    for (int i = 0; i < count; ++i) b->widths.push_back(cs[i].n);
    int zio = 0, zzo = 0;
    for (int i = 0; i < count; ++i) {
        circs[i].zi_off = zio;
        circs[i].zz_off = zzo;
        zio += cs[i].n;
        zzo += std::max(0, cs[i].n - 1);
    }
    b->total_zi = zio;
    b->total_zz = zzo;
    std::vector<int> large, small, wides;
    for (int i = 0; i < count; ++i) (wide[i] ? wides : cs[i].n > batch::kSmallMax ? large : small).push_back(i);
    std::stable_sort(large.begin(), large.end(), [&](int x, int y) {
        return std::ldexp((double)circs[x].npass, circs[x].n) > std::ldexp((double)circs[y].npass, circs[y].n);
    });
    size_t wsoff = 0;
    std::vector<batch::Circ> ordered;
    for (int i : large) {
        circs[i].state_off = (int64_t)(wsoff / 8);
        wsoff += (small_state_bytes(circs[i].n) + 255) & ~(size_t)255;
        ordered.push_back(circs[i]);
    }
    for (int i : small) { circs[i].state_off = -1; ordered.push_back(circs[i]); }
    for (int i : wides) {
        b->wide_n.push_back(cs[i].n);
        b->wide_state_off.push_back((int64_t)(wsoff / 8));
        b->wide_zi_off.push_back(circs[i].zi_off);
        b->wide_zz_off.push_back(circs[i].zz_off);
        wsoff += (small_state_bytes(cs[i].n) + 255) & ~(size_t)255;
    }
    b->nlarge = (int)large.size();
    b->nsmall = (int)small.size();
    b->ws_need = wsoff;

    // ---- device buffer: [passes][circuits][float matrices][FP64 composed][pool][descriptors][counters][zi][zz]
    auto align = [](size_t v) { return (v + 255) & ~(size_t)255; };
    size_t o = 0;
    const size_t o_pass = o; o = align(o + sizeof(batch::Pass) * passes.size());
    const size_t o_circ = o; o = align(o + sizeof(batch::Circ) * ordered.size());
    const size_t o_mat = o; o = align(o + sizeof(float2) * compose_out);
    const size_t o_out = o; o = align(o + sizeof(double) * 2 * compose_out);
    const size_t o_pool = o; o = align(o + sizeof(double) * pool.size());
    const size_t o_cb = o; o = align(o + sizeof(ComposeBlock) * cblocks.size());
    const size_t o_cg = o; o = align(o + sizeof(ComposeGate) * cgates.size());
    const size_t o_cnt = o; o = align(o + sizeof(int) * 2);
    const size_t o_zi = o; o = align(o + sizeof(double) * zio);
    const size_t o_zz = o; o = align(o + sizeof(double) * std::max(1, zzo));
    cudaError_t e = cudaMalloc(&b->dbuf, o);
    if (e != cudaSuccess) { delete b; set_error("batch plan buffer of %zu bytes", o); return QSIM_ENOMEM; }
    char* base = static_cast<char*>(b->dbuf);
    e = cudaMemcpyAsync(base + o_pass, passes.data(), sizeof(batch::Pass) * passes.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_circ, ordered.data(), sizeof(batch::Circ) * ordered.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_pool, pool.data(), sizeof(double) * pool.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_cb, cblocks.data(), sizeof(ComposeBlock) * cblocks.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_cg, cgates.data(), sizeof(ComposeGate) * cgates.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host vectors are temporaries
    if (e == cudaSuccess)
        e = launch_compose(reinterpret_cast<ComposeBlock*>(base + o_cb), (int)cblocks.size(),
                           reinterpret_cast<ComposeGate*>(base + o_cg), reinterpret_cast<double*>(base + o_pool),
                           reinterpret_cast<double*>(base + o_out), batch::kKmax, s);
    if (e == cudaSuccess)
        e = launch_convert_matrix(QSIM_C64, reinterpret_cast<double*>(base + o_out), base + o_mat, 2 * compose_out, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(batch::k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(batch::Shared));
    // Cluster size: the widest circuits set the makespan, so prefer 16 CTAs (non-portable size, one CTA per
    // SM) when the device co-schedules enough of them, else 8.
    int nclusters = 0, clsize = 0;
    if (e == cudaSuccess && cudaFuncSetAttribute(batch::k_batch, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
        cudaGetLastError();
    for (int cl : {16, 8}) {
        if (e != cudaSuccess) break;
        cudaLaunchConfig_t cfg{};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cl;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(cl, 1, 1);
        cfg.blockDim = dim3(batch::kThreads, 1, 1);
        cfg.dynamicSmemBytes = sizeof(batch::Shared);
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int ncl = 0;
        if (cudaOccupancyMaxActiveClusters(&ncl, batch::k_batch, &cfg) != cudaSuccess) { cudaGetLastError(); ncl = 0; }
        if (ncl * cl >= 128) { nclusters = ncl; clsize = cl; break; }
        if (ncl * cl > nclusters * clsize) { nclusters = ncl; clsize = cl; }
    }
    if (e != cudaSuccess || nclusters < 1) {
        cudaFree(b->dbuf);
        delete b;
        return e != cudaSuccess ? cuda_fail(e, "batch plan preparation") : (set_error("no thread-block cluster fits"), QSIM_EUNSUPPORTED);
    }
    b->cluster = clsize;
    b->grid = nclusters * clsize;
    b->args.passes = reinterpret_cast<const batch::Pass*>(base + o_pass);
    b->args.circs = reinterpret_cast<const batch::Circ*>(base + o_circ);
    b->args.nlarge = b->nlarge;
    b->args.nsmall = b->nsmall;
    b->args.mats = reinterpret_cast<const float2*>(base + o_mat);
    b->args.zi = reinterpret_cast<double*>(base + o_zi);
    b->args.zz = reinterpret_cast<double*>(base + o_zz);
    b->args.counters = reinterpret_cast<int*>(base + o_cnt);

    qsim_plan_info& I = b->info;
    I.input_gates = gates_total;
    I.passes = (int64_t)passes.size();
    I.dense_blocks = (int64_t)passes.size();
    I.algorithmic_bytes = bytes;  // state traffic of the large circuits; small ones never leave shared memory
    // one-shot run: the wide circuits' planning streams are ordered after the caller's earlier work, not after
    // the persistent launch (pre_ev, recorded before it)
    cudaEvent_t pre_ev = nullptr;
    if (run_ws) {
        b->args.ws = static_cast<float2*>(run_ws);
        if (!wides.empty() && (cudaEventCreateWithFlags(&pre_ev, cudaEventDisableTiming) != cudaSuccess ||
                               cudaEventRecord(pre_ev, s) != cudaSuccess)) {
            if (pre_ev) cudaEventDestroy(pre_ev);
            qsim_batch_destroy(b);
            return cuda_fail(cudaGetLastError(), "batch ordering event");
        }
        if (b->nlarge + b->nsmall > 0 && (rc = batch_launch(b, s)) != QSIM_OK) {
            if (pre_ev) cudaEventDestroy(pre_ev);
            qsim_batch_destroy(b);
            return rc;
        }
    }

    // ---- wide circuits: fused tensor-core plans, <Z> scratch, device error word ---------------------------
    if (!wides.empty()) {
        auto fail = [&](int code) {
            if (pre_ev) cudaEventDestroy(pre_ev);
            pre_ev = nullptr;
            qsim_batch_destroy(b);
            return code;
        };
        int nmax = 0;
        for (int n : b->wide_n) nmax = std::max(nmax, n);
        int optin = 0;
        bool ok = cudaGetDevice(&b->dev.device) == cudaSuccess &&
                  cudaDeviceGetAttribute(&b->dev.num_sms, cudaDevAttrMultiProcessorCount, b->dev.device) == cudaSuccess &&
                  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->dev.device) == cudaSuccess;
        b->dev.smem_optin = (size_t)optin;
        const int nworkers = (int)std::min<size_t>(batch::kWideStreams, wides.size());
        b->reds.resize(nworkers);
        b->wstreams.assign(nworkers, nullptr);
        b->join_ev.assign(nworkers, nullptr);
        // k_zstats_warp partials (kZW per block, at most 8 blocks per SM) and the high-bit partials
        const size_t npart = (size_t)2 * 21 * 8 * std::max(1, b->dev.num_sms) + 8192;
        for (int k = 0; k < nworkers; ++k) {
            ok = ok && cudaMalloc(&b->reds[k].partials, sizeof(double) * npart) == cudaSuccess;
            ok = ok && cudaMalloc(&b->reds[k].seg, sizeof(double) * ((size_t)2 << (nmax - 10))) == cudaSuccess;
            ok = ok && cudaMalloc(&b->reds[k].result, sizeof(double) * 256) == cudaSuccess;
            ok = ok && cudaStreamCreateWithFlags(&b->wstreams[k], cudaStreamNonBlocking) == cudaSuccess;
            ok = ok && cudaEventCreateWithFlags(&b->join_ev[k], cudaEventDisableTiming) == cudaSuccess;
        }
        ok = ok && cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming) == cudaSuccess;
        ok = ok && cudaMalloc(&b->derr, sizeof(unsigned)) == cudaSuccess;
        ok = ok && cudaMemset(b->derr, 0, sizeof(unsigned)) == cudaSuccess;
        if (!ok) { set_error("batch: scratch and streams for the tensor-core plans"); return fail(QSIM_ENOMEM); }
        // one plan per wide circuit, made on several host threads, each thread on its own stream (a plan's
        // creation synchronises its stream); ordered after the caller's earlier work on `stream`
        const int nw = (int)wides.size();
        const int nth = host_threads(nw * 4);
        std::vector<cudaStream_t> pst(nth, nullptr);
        cudaEvent_t ord = pre_ev;
        if (!ord)
            ok = cudaEventCreateWithFlags(&ord, cudaEventDisableTiming) == cudaSuccess && cudaEventRecord(ord, s) == cudaSuccess;
        // planning streams at the highest priority: in a one-shot run their composition kernels are scheduled
        // ahead of the worker streams' passes of the plans already made
        int prio_lo = 0, prio_hi = 0;
        if (cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi) != cudaSuccess) { cudaGetLastError(); prio_hi = 0; }
        for (int t = 0; t < nth && ok; ++t)
            ok = cudaStreamCreateWithPriority(&pst[t], cudaStreamNonBlocking, prio_hi) == cudaSuccess &&
                 cudaStreamWaitEvent(pst[t], ord, 0) == cudaSuccess;
        std::vector<qsim_plan_h> wph(nw, nullptr);
        std::vector<qsim_plan_info> wpi(nw);
        // one-shot run: the worker streams start with the persistent launch (after the caller's earlier work,
        // pre_ev), their kernels taking the SMs it leaves; one host thread enqueues each plan as the planning
        // threads finish it (its passes and its <Z> readout) on the least-loaded worker stream, while the
        // planning threads go on planning
        std::mutex qmu;
        std::condition_variable qcv;
        std::deque<int> ready;
        bool planning_done = false;
        int enq_rc = QSIM_OK;
        std::string enq_msg;
        std::thread enq;
        if (run_ws && ok)
            for (int k = 0; k < nworkers && ok; ++k) ok = cudaStreamWaitEvent(b->wstreams[k], ord, 0) == cudaSuccess;
        if (run_ws && ok) {
            enq = std::thread([&, device]() {
                cudaSetDevice(device);
                std::vector<double> load(nworkers, 0.0);
                for (;;) {
                    int w = -1;
                    {
                        std::unique_lock<std::mutex> lk(qmu);
                        qcv.wait(lk, [&] { return !ready.empty() || planning_done; });
                        if (ready.empty()) break;
                        w = ready.front();
                        ready.pop_front();
                    }
                    if (enq_rc != QSIM_OK) continue;  // after an error: drain, enqueue nothing more
                    const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
                    load[k] += std::ldexp((double)wpi[w].passes, cs[wides[w]].n);
                    enq_rc = enqueue_wide(b, wph[w], (size_t)w, k, run_ws);
                    if (enq_rc != QSIM_OK) enq_msg = qsim_last_error();
                }
            });
        }
        const int prc = !ok ? QSIM_ENOMEM : parallel_for(nw, nth, device, [&](int w, int my_slot) -> int {
            qsim_run_opts po{};
            po.mode = QSIM_RUN_FUSED;
            // FP16X3: 7-qubit blocks where the planner finds them cheaper (nearest-neighbour chains)
            po.max_fused = opts.precision == QSIM_PREC_FP16X3 ? 7 : 6;
            po.precision = opts.precision;
            po.tc_min_k = 5;
            po.launch_per_pass = 1;  // plans run concurrently on worker streams inside a captured graph
            const int r = qsim_plan_create(&cs[wides[w]], QSIM_C64, &po, pst[my_slot], &wph[w], &wpi[w]);
            if (r == QSIM_OK && cudaStreamSynchronize(pst[my_slot]) != cudaSuccess)
                return cuda_fail(cudaGetLastError(), "tensor-core plan of a wide circuit");
            if (r == QSIM_OK && enq.joinable()) {
                std::lock_guard<std::mutex> lk(qmu);
                ready.push_back(w);
                qcv.notify_one();
            }
            return r;
        });
        if (enq.joinable()) {
            {
                std::lock_guard<std::mutex> lk(qmu);
                planning_done = true;
                qcv.notify_one();
            }
            enq.join();
            if (enq_rc != QSIM_OK) set_error("%s", enq_msg.c_str());
        }
        if (run_ws) {  // join every worker back into s, also after an error
            for (int k = 0; k < nworkers; ++k) {
                bool j = cudaEventRecord(b->join_ev[k], b->wstreams[k]) == cudaSuccess &&
                         cudaStreamWaitEvent(s, b->join_ev[k], 0) == cudaSuccess;
                ok = ok && j;
            }
        }
        for (cudaStream_t st : pst)
            if (st) cudaStreamDestroy(st);
        if (ord) cudaEventDestroy(ord);
        pre_ev = nullptr;  // it was ord
        for (qsim_plan_h ph : wph)
            if (ph) b->wide_plans.push_back(ph);
        if (!ok) { set_error("batch: streams for planning the tensor-core circuits"); return fail(QSIM_ENOMEM); }
        if (prc) return fail(prc);
        if (enq_rc) return fail(enq_rc);
        std::vector<double> wide_work;
        for (int w = 0; w < nw; ++w) {
            const int i = wides[w];
            const qsim_plan_info& pi = wpi[w];
            wide_work.push_back(std::ldexp((double)pi.passes, cs[i].n));
            I.passes += pi.passes;
            I.tc_blocks += pi.tc_blocks;
            I.dense_blocks += pi.dense_blocks;
            I.diag_blocks += pi.diag_blocks;
            I.algorithmic_bytes += pi.algorithmic_bytes;
            // the first block generates |0> (execute_from_basis) and only writes
            qsim_pass_info p0{};
            if (pi.passes > 0 && qsim_plan_pass_info(wph[w], 0, &p0) == QSIM_OK && p0.kind == QSIM_PASS_TC &&
                p0.precision != QSIM_PREC_BF16X6)
                I.algorithmic_bytes -= std::ldexp(8.0, cs[i].n);
        }
        // longest processing time first: each circuit, most work first, to the least-loaded worker
        std::vector<int> byw(wide_work.size());
        for (size_t w = 0; w < byw.size(); ++w) byw[w] = (int)w;
        std::stable_sort(byw.begin(), byw.end(), [&](int x, int y) { return wide_work[x] > wide_work[y]; });
        std::vector<double> load(nworkers, 0.0);
        b->wide_worker.assign(wide_work.size(), 0);
        for (int w : byw) {
            const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            b->wide_worker[w] = k;
            load[k] += wide_work[w];
        }
    }
    I.host_plan_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = I;
    *out = b;
    return QSIM_OK;
}

int qsim_batch_plan_create(const qsim_circuit* cs, int count, const qsim_run_opts* opts_in, void* stream_v,
                           qsim_batch_h* out, qsim_plan_info* info) {
    return batch_plan_create_impl(cs, count, opts_in, stream_v, out, info, nullptr);
}

// Wide circuit w (its plan) on worker stream k: the plan from |0> (its first block generates the basis
// state), then its <Z> values. Below 24 qubits (fewer than 7 tiles of a tensor-core pass per SM) the plan's
// kernels take half the SMs, below 22 a quarter: each CTA then has more tiles to pipeline, and other worker
// streams' kernels run on the rest (256-chain batch on 8 worker streams: 45.5 ms, against 49.2 ms with every
// kernel on all SMs and 4 streams; half the SMs below 24 alone 46.8 ms).
static int enqueue_wide(qsim_batch_h b, qsim_plan_h plan, size_t w, int k, void* dev_ws) {
    qsim_state st;
    st.n = b->wide_n[w];
    st.dtype = QSIM_C64;
    st.psi = static_cast<float2*>(dev_ws) + b->wide_state_off[w];
    st.bytes = small_state_bytes(st.n);
    st.stream = b->wstreams[k];
    st.dev = b->dev;
    if (b->wstreams.size() > 1 && st.n < batch::kHalfGridBelow)
        st.dev.num_sms = std::max(1, b->dev.num_sms / (st.n < batch::kQuarterGridBelow ? 4 : 2));
    st.derr = b->derr;
    int rc = qsim_plan_execute_from_basis(&st, plan, 0, -1);
    if (rc) return rc;
    cudaError_t e = run_zstats_device(QSIM_C64, st.psi, st.n, b->reds[k], st.stream, b->dev,
                                      b->args.zi + b->wide_zi_off[w], b->args.zz + b->wide_zz_off[w], true);
    return e == cudaSuccess ? QSIM_OK : cuda_fail(e, "batch <Z> of a tensor-core plan");
}

static int batch_enqueue(qsim_batch_h b, void* dev_ws, cudaStream_t s) {
    b->args.ws = static_cast<float2*>(dev_ws);
    if (b->nlarge + b->nsmall > 0) {
        const int rc = batch_launch(b, s);
        if (rc) return rc;
    }
    if (b->wide_plans.empty()) return QSIM_OK;
    // wide circuits on the worker streams (fork from s, join back into s): each plan from |0> (its first
    // block generates the basis state), then its <Z> values
    cudaError_t e = cudaEventRecord(b->fork_ev, s);
    for (size_t k = 0; e == cudaSuccess && k < b->wstreams.size(); ++k) e = cudaStreamWaitEvent(b->wstreams[k], b->fork_ev, 0);
    if (e != cudaSuccess) return cuda_fail(e, "batch fork");
    int rc = QSIM_OK;
    for (size_t w = 0; w < b->wide_plans.size() && rc == QSIM_OK; ++w)
        rc = enqueue_wide(b, b->wide_plans[w], w, b->wide_worker[w], dev_ws);
    // join every worker back into s, also after an error (a capture must end with all branches joined)
    for (size_t k = 0; k < b->wstreams.size(); ++k) {
        cudaError_t ej = cudaEventRecord(b->join_ev[k], b->wstreams[k]);
        if (ej == cudaSuccess) ej = cudaStreamWaitEvent(s, b->join_ev[k], 0);
        if (ej != cudaSuccess && rc == QSIM_OK) rc = cuda_fail(ej, "batch join");
    }
    return rc;
}

static int batch_launch(qsim_batch_h b, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(b->args.counters, 0, 2 * sizeof(int), s);
    if (e != cudaSuccess) return cuda_fail(e, "batch counters");
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = b->cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(b->grid, 1, 1);
    cfg.blockDim = dim3(batch::kThreads, 1, 1);
    cfg.dynamicSmemBytes = sizeof(batch::Shared);
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, batch::k_batch, b->args);
    return e == cudaSuccess ? QSIM_OK : cuda_fail(e, "batch launch");
}

int qsim_batch_execute(qsim_batch_h b, void* dev_ws, size_t ws_bytes, void* stream_v, int use_graph) {
    if (!b) { set_error("NULL batch plan"); return QSIM_EINVAL; }
    set_error("%s", "");
    if (b->ws_need && (!dev_ws || ws_bytes < b->ws_need)) { set_error("workspace of %zu bytes < %zu needed", ws_bytes, b->ws_need); return QSIM_ENOMEM; }
    if (dev_ws && (reinterpret_cast<uintptr_t>(dev_ws) & 255)) { set_error("workspace must be 256-byte aligned"); return QSIM_EINVAL; }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_v);
    if (!use_graph || s == nullptr) return batch_enqueue(b, dev_ws, s);
    if (b->gexec && b->gws == dev_ws && b->gstream == s) {
        cudaError_t e = cudaGraphLaunch(b->gexec, s);
        return e == cudaSuccess ? QSIM_OK : cuda_fail(e, "batch graph launch");
    }
    if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return cuda_fail(e, "begin capture");
    int rc = batch_enqueue(b, dev_ws, s);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s, &g);
    if (rc) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    e = cudaGraphInstantiate(&b->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { b->gexec = nullptr; return cuda_fail(e, "graph instantiate"); }
    b->gws = dev_ws;
    b->gstream = s;
    e = cudaGraphLaunch(b->gexec, s);
    return e == cudaSuccess ? QSIM_OK : cuda_fail(e, "batch graph launch");
}

int qsim_batch_results(qsim_batch_h b, void* stream_v, double* zi, double* zz) {
    if (!b || !zi || !zz) { set_error("NULL argument"); return QSIM_EINVAL; }
    set_error("%s", "");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_v);
    cudaError_t e = cudaMemcpyAsync(zi, b->args.zi, sizeof(double) * b->total_zi, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && b->total_zz > 0)
        e = cudaMemcpyAsync(zz, b->args.zz, sizeof(double) * b->total_zz, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "batch results");
    if (b->derr) {  // a bounded wait of a tensor-core launch expired
        qsim_state st;
        st.derr = b->derr;
        return check_device_error(&st);
    }
    return QSIM_OK;
}

int qsim_batch_destroy(qsim_batch_h b) {
    if (!b) return QSIM_OK;
    cudaDeviceSynchronize();
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    for (qsim_plan_h p : b->wide_plans) qsim_plan_destroy(p);
    for (auto& r : b->reds) {
        cudaFree(r.partials);
        cudaFree(r.seg);
        cudaFree(r.result);
    }
    for (cudaStream_t st : b->wstreams)
        if (st) cudaStreamDestroy(st);
    for (cudaEvent_t ev : b->join_ev)
        if (ev) cudaEventDestroy(ev);
    if (b->fork_ev) cudaEventDestroy(b->fork_ev);
    cudaFree(b->derr);
    cudaFree(b->dbuf);
    delete b;
    return QSIM_OK;
}

int qsim_batch_run(const qsim_circuit* cs, int count, const qsim_run_opts* opts, void* dev_ws, size_t ws_bytes,
                   void* stream, double* zi, double* zz, qsim_plan_info* info) {
    set_error("%s", "");
    if (!zi || !zz) { set_error("NULL argument"); return QSIM_EINVAL; }
    size_t need = 0;
    int rc = qsim_batch_workspace_bytes(cs, count, &need);
    if (rc) return rc;
    if (need && (!dev_ws || ws_bytes < need)) { set_error("workspace of %zu bytes < %zu needed", ws_bytes, need); return QSIM_ENOMEM; }
    if (dev_ws && (reinterpret_cast<uintptr_t>(dev_ws) & 255)) { set_error("workspace must be 256-byte aligned"); return QSIM_EINVAL; }
    // a workspace is needed to run while planning; a batch without one (every circuit in shared memory)
    // plans, then executes
    qsim_batch_h b = nullptr;
    void* run_ws = dev_ws ? dev_ws : nullptr;
    rc = batch_plan_create_impl(cs, count, opts, stream, &b, info, run_ws);
    if (rc) return rc;
    if (!run_ws) rc = qsim_batch_execute(b, dev_ws, ws_bytes, stream, 0);
    if (!rc) rc = qsim_batch_results(b, stream, zi, zz);
    qsim_batch_destroy(b);
    return rc;
}

// Built-in tuner: for every width present, time each fusion width k in 1..4 on the first circuit of that
// width (the median of three launches after a warm-up) and keep the fastest; later plans created with
// max_fused = 0 use it. The trial workspace is allocated here and released before returning.
int qsim_batch_autotune(const qsim_circuit* cs, int count, void* stream_v, int* chosen) {
    set_error("%s", "");
    int rc = validate_batch(cs, count);
    if (rc) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_v);
    batch::tune_cache_autoload();
    std::vector<int> seen(QSIM_MAX_QUBITS + 1, -1);
    for (int i = 0; i < count; ++i)
        if (seen[cs[i].n] < 0) seen[cs[i].n] = i;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int n = 1; n <= QSIM_MAX_QUBITS; ++n) {
        if (seen[n] < 0) continue;
        const qsim_circuit* c = &cs[seen[n]];
        size_t wsb = 0;
        qsim_batch_workspace_bytes(c, 1, &wsb);
        void* ws = nullptr;
        if (wsb && cudaMalloc(&ws, wsb) != cudaSuccess) { cudaGetLastError(); rc = QSIM_ENOMEM; set_error("tuning workspace"); break; }
        float best = 1e30f;
        int bestk = batch::kKmax;
        for (int k = 1; k <= std::min(n, batch::kKmax); ++k) {
            qsim_run_opts o{};
            o.mode = QSIM_RUN_FUSED;
            o.max_fused = k;
            qsim_batch_h b = nullptr;
            if (qsim_batch_plan_create(c, 1, &o, stream_v, &b, nullptr)) continue;
            float t[3];
            qsim_batch_execute(b, ws, wsb, stream_v, 0);  // warm-up
            for (int r = 0; r < 3; ++r) {
                cudaEventRecord(e0, s);
                qsim_batch_execute(b, ws, wsb, stream_v, 0);
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                cudaEventElapsedTime(&t[r], e0, e1);
            }
            std::sort(t, t + 3);
            if (t[1] < best) { best = t[1]; bestk = k; }
            qsim_batch_destroy(b);
        }
        if (ws) cudaFree(ws);
        std::lock_guard<std::mutex> lock(batch::g_tune_mu);
        batch::g_tuned_k[n] = bestk;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (chosen)
        for (int i = 0; i < count; ++i) chosen[i] = batch::tuned_k(cs[i].n);
    if (rc == QSIM_OK) batch::tune_cache_autosave();
    return rc;
}

int qsim_batch_autotune_threshold(const qsim_circuit* cs, int count, int precision, void* stream_v, int* best_min_n) {
    set_error("%s", "");
    int rc = validate_batch(cs, count);
    if (rc) return rc;
    if (precision < QSIM_PREC_TF32X3 || precision > QSIM_PREC_FP16X3) { set_error("a tensor-core precision is needed"); return QSIM_EINVAL; }
    batch::tune_cache_autoload();
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_v);
    size_t wsb = 0;
    if ((rc = qsim_batch_workspace_bytes(cs, count, &wsb)) != QSIM_OK) return rc;
    void* ws = nullptr;
    if (wsb && cudaMalloc(&ws, wsb) != cudaSuccess) { cudaGetLastError(); set_error("tuning workspace"); return QSIM_ENOMEM; }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int nmax = 0;
    for (int i = 0; i < count; ++i) nmax = std::max(nmax, cs[i].n);
    float best = 1e30f;
    int bestn = 0;
    // every candidate threshold, timed on the whole batch (median of three replays after a warm-up); a
    // threshold above the widest circuit keeps every circuit in the persistent launch
    for (int th : {14, 16, 18, 20, 22, 24, 27}) {
        if (th > nmax + 1 && th != 27) continue;
        qsim_run_opts o{};
        o.mode = QSIM_RUN_FUSED;
        o.precision = precision;
        o.batch_tc_min_n = th;
        qsim_batch_h b = nullptr;
        if ((rc = qsim_batch_plan_create(cs, count, &o, stream_v, &b, nullptr)) != QSIM_OK) break;
        float t[3] = {0, 0, 0};
        rc = qsim_batch_execute(b, ws, wsb, stream_v, 1);
        for (int r = 0; r < 3 && rc == QSIM_OK; ++r) {
            cudaEventRecord(e0, s);
            rc = qsim_batch_execute(b, ws, wsb, stream_v, 1);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&t[r], e0, e1);
        }
        qsim_batch_destroy(b);
        if (rc) break;
        std::sort(t, t + 3);
        if (t[1] < best) { best = t[1]; bestn = th; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (ws) cudaFree(ws);
    if (rc) return rc;
    {
        std::lock_guard<std::mutex> lock(batch::g_tune_mu);
        batch::g_tuned_tc_min_n[precision] = bestn;
    }
    if (best_min_n) *best_min_n = bestn;
    batch::tune_cache_autosave();
    return QSIM_OK;
}

int qsim_batch_tune_save(const char* path) {
    set_error("%s", "");
    if (!path) { set_error("NULL path"); return QSIM_EINVAL; }
    return batch::tune_save_file(path);
}

int qsim_batch_tune_load(const char* path) {
    set_error("%s", "");
    if (!path) { set_error("NULL path"); return QSIM_EINVAL; }
    return batch::tune_load_file(path);
}

}  // extern "C"
