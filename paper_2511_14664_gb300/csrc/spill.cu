// spill.cu -- states held in host memory and streamed through device windows (out-of-core execution).
//
// Paper Sec. 2.5: when a state outgrows GPU memory, host memory can supplement it, at a cost the paper puts
// at 4x or more per two extra qubits; Sec. 2.1: a state cut into 2^p pieces by its top p index bits needs no
// exchange for gates on the other (local) qubits, while a gate on one of the p global qubits needs the
// pieces that differ in that bit.
//
// Here the state lives in host memory (on a GB300 node, the Grace CPU's memory behind NVLink-C2C), cut into
// slices of 2^L amplitudes by its top n - L index bits. A circuit runs as a sequence of segments. A segment
// is a set of gates, dependencies kept, whose qubits include at most h of the global ones: its active set A
// (padded to h bits). For every value of the other global bits, the 2^h slices that differ only in the bits
// of A are copied into a device window of 2^(L+h) amplitudes, where global bit A[j] becomes window bit
// L + j; the segment's plan (made once by the ordinary planner for the (L+h)-qubit window: fused blocks on
// the tensor cores, phase passes, ...) runs on the window, which is then copied back. A segment thus moves
// the whole state over the host link once in and once out, however many gates it holds. Three windows
// rotate so that the copy in of window w+1, the passes on window w and the copy out of window w-1 overlap
// (both copy directions and the SMs work at once). The slices a segment writes are read by the next
// segment's windows, so segments are separated by the completion of all copies out.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <vector>

#include "capi_state.h"
#include "internal.h"

namespace qsim {
namespace {

struct SpillSeg {
    std::vector<int> gates;  // gate indices, ascending
    uint64_t used = 0;       // global qubits the gates touch
    std::vector<int> act;    // the h window slots: used global qubits first, then padding
};

// Greedy segmentation: scan the unplaced gates in order; a gate joins the segment when it shares no qubit
// with a gate skipped earlier in this scan (so every dependency is kept) and the union of the segment's
// global qubits stays within h; otherwise it is skipped and its qubits block later gates of the scan.
std::vector<SpillSeg> spill_segments(const qsim_circuit* c, int L, int h) {
    const int n = c->n, G = c->num_gates;
    const uint64_t gmask_all = n >= 64 ? ~0ull : ((1ull << n) - 1);
    const uint64_t global = gmask_all & ~((1ull << L) - 1);
    std::vector<uint64_t> qm(G);
    for (int i = 0; i < G; ++i) {
        uint64_t m = 0;
        for (int j = 0; j < c->gates[i].k; ++j) m |= 1ull << c->gates[i].targets[j];
        for (int j = 0; j < c->gates[i].nc; ++j) m |= 1ull << c->gates[i].controls[j];
        qm[i] = m;
    }
    std::vector<char> placed(G, 0);
    std::vector<SpillSeg> segs;
    for (int i = 0; i < G; ++i)  // callers check this first: such a gate could never join a segment
        if (__builtin_popcountll(qm[i] & global) > h) return segs;
    int first = 0;
    while (first < G) {
        SpillSeg sg;
        uint64_t blocked = 0;
        for (int i = first; i < G; ++i) {
            if (placed[i]) continue;
            const uint64_t gq = qm[i];
            const uint64_t u = sg.used | (gq & global);
            if ((gq & blocked) == 0 && __builtin_popcountll(u) <= h) {
                sg.gates.push_back(i);
                sg.used = u;
                placed[i] = 1;
            } else {
                blocked |= gq;
                if ((blocked & gmask_all) == gmask_all) break;
            }
        }
        for (int q = L; q < n; ++q)
            if ((sg.used >> q) & 1) sg.act.push_back(q);
        for (int q = L; q < n && (int)sg.act.size() < h; ++q)
            if (!((sg.used >> q) & 1)) sg.act.push_back(q);
        segs.push_back(std::move(sg));
        while (first < G && placed[first]) ++first;
    }
    return segs;
}

// Every gate must fit a window: at most h of its qubits global.
int spill_check_gates(const qsim_circuit* c, int L, int h) {
    for (int i = 0; i < c->num_gates; ++i) {
        const qsim_gate& g = c->gates[i];
        int ng = 0;
        for (int j = 0; j < g.k; ++j) ng += g.targets[j] >= L;
        for (int j = 0; j < g.nc; ++j) ng += g.controls[j] >= L;
        if (ng > h) {
            set_error("gate %d has %d qubits among the top %d index bits, more than the %d a window holds "
                      "(raise global_slots)", i, ng, c->n - L, h);
            return QSIM_EUNSUPPORTED;
        }
    }
    return QSIM_OK;
}

int spill_geometry(int n, int W, int slots, int* L, int* h) {
    if (W >= n) { *L = n; *h = 0; return QSIM_OK; }
    if (W < 14) { set_error("window_qubits %d below 14 (with n = %d > W)", W, n); return QSIM_EINVAL; }
    const int hh = slots > 0 ? slots : std::min(4, W - 12);
    if (hh < 1 || hh > 8 || W - hh < 10) { set_error("global_slots %d invalid for window_qubits %d", hh, W); return QSIM_EINVAL; }
    *L = W - hh;
    *h = hh;
    return QSIM_OK;
}

// Three device windows, their streams and events, and a handle per window.
struct Windows {
    int Wq = 0, dtype = 0;
    size_t amp = 8, bytes = 0;
    void* buf[3] = {nullptr, nullptr, nullptr};
    qsim_h hd[3] = {nullptr, nullptr, nullptr};
    cudaStream_t s_in = nullptr, s_comp = nullptr, s_out = nullptr;
    cudaEvent_t ev_in[3] = {}, ev_comp[3] = {}, ev_out[3] = {};
    int create(int Wq_, int dtype_) {
        Wq = Wq_;
        dtype = dtype_;
        amp = dtype == QSIM_C64 ? 8 : 16;
        bytes = amp << Wq;
        cudaError_t e = cudaStreamCreateWithFlags(&s_in, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s_comp, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s_out, cudaStreamNonBlocking);
        for (int i = 0; i < 3 && e == cudaSuccess; ++i) {
            e = cudaEventCreateWithFlags(&ev_in[i], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_comp[i], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_out[i], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return cuda_fail(e, "window streams");
        for (int i = 0; i < 3; ++i) {
            if (cudaMalloc(&buf[i], bytes) != cudaSuccess) {
                cudaGetLastError();
                set_error("cudaMalloc of a %zu-byte device window failed", bytes);
                return QSIM_ENOMEM;
            }
            const int rc = qsim_create(Wq, dtype, buf[i], bytes, s_comp, &hd[i]);
            if (rc) return rc;
        }
        return QSIM_OK;
    }
    ~Windows() {
        for (cudaStream_t s : {s_in, s_comp, s_out})
            if (s) cudaStreamSynchronize(s);
        for (int i = 0; i < 3; ++i) {
            if (hd[i]) qsim_destroy(hd[i]);
            if (buf[i]) cudaFree(buf[i]);
            for (cudaEvent_t ev : {ev_in[i], ev_comp[i], ev_out[i]})
                if (ev) cudaEventDestroy(ev);
        }
        for (cudaStream_t s : {s_in, s_comp, s_out})
            if (s) cudaStreamDestroy(s);
    }
};

uint64_t deposit_bits(uint64_t v, const std::vector<int>& pos) {
    uint64_t r = 0;
    for (size_t j = 0; j < pos.size(); ++j) r |= ((v >> j) & 1ull) << pos[j];
    return r;
}

}  // namespace
}  // namespace qsim

using namespace qsim;

extern "C" int qsim_spill_segments(const qsim_circuit* c, int window_qubits, int global_slots, int32_t* seg_of_gate,
                                   uint64_t* used_global, int64_t* nseg) {
    set_error("%s", "");
    if (!c || !nseg || (c->num_gates > 0 && (!c->gates || !seg_of_gate))) { set_error("NULL argument"); return QSIM_EINVAL; }
    if (c->n < 1 || c->n > QSIM_MAX_QUBITS) { set_error("n = %d outside 1..%d", c->n, QSIM_MAX_QUBITS); return QSIM_EINVAL; }
    for (int i = 0; i < c->num_gates; ++i) {
        const qsim_gate& g = c->gates[i];
        const int rc = validate_qubits(c->n, g.targets, g.k, g.controls, g.nc, QSIM_MAX_TARGETS);
        if (rc) { set_error("gate %d: invalid qubits", i); return rc; }
    }
    int L = 0, h = 0;
    int rc = spill_geometry(c->n, window_qubits, global_slots, &L, &h);
    if (rc) return rc;
    if ((rc = spill_check_gates(c, L, h)) != QSIM_OK) return rc;
    const auto segs = spill_segments(c, L, h);
    for (size_t s = 0; s < segs.size(); ++s) {
        for (int i : segs[s].gates) seg_of_gate[i] = (int32_t)s;
        if (used_global) used_global[s] = segs[s].used;
    }
    *nseg = (int64_t)segs.size();
    return QSIM_OK;
}

extern "C" int qsim_spill_run(void* host_state, const qsim_circuit* c, int dtype, const qsim_spill_opts* opts,
                              void* stream, qsim_spill_info* info) {
    set_error("%s", "");
    const auto t0 = std::chrono::steady_clock::now();
    if (!host_state || !c || !opts) { set_error("NULL argument"); return QSIM_EINVAL; }
    if (dtype != QSIM_C64 && dtype != QSIM_C128) { set_error("unknown dtype %d", dtype); return QSIM_EINVAL; }
    const int n = c->n;
    if (n < 1 || n > QSIM_MAX_QUBITS) { set_error("n = %d outside 1..%d", n, QSIM_MAX_QUBITS); return QSIM_EINVAL; }
    if (c->num_gates < 0 || (c->num_gates > 0 && !c->gates)) { set_error("bad gate list"); return QSIM_EINVAL; }
    int L = 0, h = 0;
    int rc = spill_geometry(n, opts->window_qubits, opts->global_slots, &L, &h);
    if (rc) return rc;
    for (int i = 0; i < c->num_gates; ++i) {
        const qsim_gate& g = c->gates[i];
        rc = validate_qubits(n, g.targets, g.k, g.controls, g.nc, QSIM_MAX_TARGETS);
        if (rc) { set_error("gate %d: invalid qubits", i); return rc; }
        if (!g.matrix) { set_error("gate %d: NULL matrix", i); return QSIM_EINVAL; }
    }
    if ((rc = spill_check_gates(c, L, h)) != QSIM_OK) return rc;
    const int Wq = L + h, g = n - L;
    const auto segs = spill_segments(c, L, h);

    Windows win;
    if ((rc = win.create(Wq, dtype)) != QSIM_OK) return rc;
    // order after the caller's earlier work on `stream`
    cudaStream_t caller = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t ev_caller = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&ev_caller, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev_caller, caller);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(win.s_in, ev_caller, 0);
    if (ev_caller) cudaEventDestroy(ev_caller);
    if (e != cudaSuccess) return cuda_fail(e, "ordering after the caller's stream");

    qsim_run_opts ro = opts->run;
    ro.use_graph = 0;
    ro.dry_run = 0;
    ro.local_qubits = 0;
    ro.launch_per_pass = 1;  // one plan runs on several windows at once (three streams)
    unsigned char* H = static_cast<unsigned char*>(host_state);
    const size_t slice_bytes = win.amp << L;
    std::vector<qsim_plan_h> plans;
    auto cleanup = [&](int r) {
        for (cudaStream_t s : {win.s_in, win.s_comp, win.s_out}) cudaStreamSynchronize(s);
        for (qsim_plan_h p : plans) qsim_plan_destroy(p);
        return r;
    };
    double plan_ms = 0.0;
    int64_t windows = 0, passes = 0;
    double host_bytes = 0.0;
    uint64_t wcount = 0;
    // every segment's plan first (plan creation allocates device memory, which would wait for the copies in
    // flight if it happened between segments)
    std::vector<int64_t> seg_passes;
    for (const SpillSeg& sg : segs) {
        // the segment's gates on the window: local qubit q stays q, global qubit act[j] becomes L + j
        std::vector<int> slot(n, -1);
        for (int q = 0; q < L; ++q) slot[q] = q;
        for (int j = 0; j < h; ++j) slot[sg.act[j]] = L + j;
        std::vector<qsim_gate> sub(sg.gates.size());
        for (size_t i = 0; i < sg.gates.size(); ++i) {
            sub[i] = c->gates[sg.gates[i]];
            for (int j = 0; j < sub[i].k; ++j) sub[i].targets[j] = slot[sub[i].targets[j]];
            for (int j = 0; j < sub[i].nc; ++j) sub[i].controls[j] = slot[sub[i].controls[j]];
        }
        const qsim_circuit sc{Wq, (int32_t)sub.size(), sub.data()};
        qsim_plan_h plan = nullptr;
        qsim_plan_info pi{};
        if ((rc = qsim_plan_create(&sc, dtype, &ro, win.s_comp, &plan, &pi)) != QSIM_OK) return cleanup(rc);
        plans.push_back(plan);
        seg_passes.push_back(pi.passes);
    }
    plan_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    for (size_t si = 0; si < segs.size(); ++si) {
        const SpillSeg& sg = segs[si];
        qsim_plan_h plan = plans[si];
        // the other global bits, as positions relative to L
        std::vector<int> other, actrel;
        for (int q = L; q < n; ++q)
            if (std::find(sg.act.begin(), sg.act.end(), q) == sg.act.end()) other.push_back(q - L);
        for (int j = 0; j < h; ++j) actrel.push_back(sg.act[j] - L);
        const uint64_t nwin = 1ull << (g - h);
        for (uint64_t w = 0; w < nwin; ++w, ++wcount) {
            const int b = (int)(wcount % 3);
            unsigned char* D = static_cast<unsigned char*>(win.buf[b]);
            const uint64_t base = deposit_bits(w, other);
            e = cudaStreamWaitEvent(win.s_in, win.ev_out[b], 0);  // the window's previous copy out is done
            for (uint64_t a = 0; a < (1ull << h) && e == cudaSuccess; ++a) {
                const uint64_t sl = base | deposit_bits(a, actrel);
                e = cudaMemcpyAsync(D + a * slice_bytes, H + sl * slice_bytes, slice_bytes, cudaMemcpyHostToDevice, win.s_in);
            }
            if (e == cudaSuccess) e = cudaEventRecord(win.ev_in[b], win.s_in);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(win.s_comp, win.ev_in[b], 0);
            if (e != cudaSuccess) return cleanup(cuda_fail(e, "window copy in"));
            if ((rc = qsim_plan_execute(win.hd[b], plan)) != QSIM_OK) return cleanup(rc);
            e = cudaEventRecord(win.ev_comp[b], win.s_comp);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(win.s_out, win.ev_comp[b], 0);
            for (uint64_t a = 0; a < (1ull << h) && e == cudaSuccess; ++a) {
                const uint64_t sl = base | deposit_bits(a, actrel);
                e = cudaMemcpyAsync(H + sl * slice_bytes, D + a * slice_bytes, slice_bytes, cudaMemcpyDeviceToHost, win.s_out);
            }
            if (e == cudaSuccess) e = cudaEventRecord(win.ev_out[b], win.s_out);
            if (e != cudaSuccess) return cleanup(cuda_fail(e, "window copy out"));
            ++windows;
            passes += seg_passes[si];
            host_bytes += 2.0 * (double)win.bytes;
        }
        // the next segment reads slices this one writes: wait for every copy out
        e = cudaStreamWaitEvent(win.s_in, win.ev_out[(wcount + 2) % 3], 0);
        if (e != cudaSuccess) return cleanup(cuda_fail(e, "segment barrier"));
    }
    for (cudaStream_t s : {win.s_in, win.s_comp, win.s_out}) {
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cleanup(cuda_fail(e, "out-of-core run"));
    }
    for (int i = 0; i < 3; ++i)
        if ((rc = qsim_synchronize(win.hd[i])) != QSIM_OK) return cleanup(rc);
    if (info) {
        info->segments = (int64_t)segs.size();
        info->windows = windows;
        info->passes = passes;
        info->host_bytes = host_bytes;
        info->elapsed_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        info->host_plan_ms = plan_ms;
        info->window_qubits = Wq;
        info->global_slots = h;
    }
    return cleanup(QSIM_OK);
}

extern "C" int qsim_spill_sample(const void* host_state, int n, int dtype, int window_qubits, uint64_t seed,
                                 int64_t shots, uint64_t* out, double* norm) {
    set_error("%s", "");
    if (!host_state || (!out && shots > 0)) { set_error("NULL argument"); return QSIM_EINVAL; }
    if (dtype != QSIM_C64 && dtype != QSIM_C128) { set_error("unknown dtype %d", dtype); return QSIM_EINVAL; }
    if (n < 1 || n > QSIM_MAX_QUBITS) { set_error("n = %d outside 1..%d", n, QSIM_MAX_QUBITS); return QSIM_EINVAL; }
    if (shots < 0 || shots > (1ll << 31)) { set_error("shots outside 0..2^31"); return QSIM_EINVAL; }
    if (window_qubits < 1) { set_error("window_qubits must be positive"); return QSIM_EINVAL; }
    const int Wq = std::min(window_qubits, n);
    const uint64_t nsl = 1ull << (n - Wq);
    Windows win;
    int rc = win.create(Wq, dtype);
    if (rc) return rc;
    const unsigned char* H = static_cast<const unsigned char*>(host_state);
    // pass 1: the squared norm of every slice (the copy of slice i+1 overlaps the sum over slice i)
    std::vector<double> tot(nsl, 0.0);
    cudaError_t e = cudaSuccess;
    auto copy_in = [&](uint64_t sl, int b) {
        cudaError_t x = cudaStreamWaitEvent(win.s_in, win.ev_comp[b], 0);
        if (x == cudaSuccess) x = cudaMemcpyAsync(win.buf[b], H + sl * win.bytes, win.bytes, cudaMemcpyHostToDevice, win.s_in);
        if (x == cudaSuccess) x = cudaEventRecord(win.ev_in[b], win.s_in);
        return x;
    };
    auto use = [&](int b) {  // the next work on window b waits for its copy in; its end is ev_comp[b]
        return cudaStreamWaitEvent(win.s_comp, win.ev_in[b], 0);
    };
    e = copy_in(0, 0);
    for (uint64_t sl = 0; sl < nsl && e == cudaSuccess; ++sl) {
        const int b = (int)(sl % 3);
        if (sl + 1 < nsl) e = copy_in(sl + 1, (int)((sl + 1) % 3));
        if (e == cudaSuccess) e = use(b);
        if (e != cudaSuccess) break;
        if ((rc = qsim_norm(win.hd[b], &tot[sl])) != QSIM_OK) return rc;
        e = cudaEventRecord(win.ev_comp[b], win.s_comp);
    }
    if (e != cudaSuccess) return cuda_fail(e, "slice sums");
    std::vector<double> cum(nsl + 1, 0.0);
    for (uint64_t s = 0; s < nsl; ++s) cum[s + 1] = cum[s] + tot[s];
    const double T = cum[nsl];
    if (norm) *norm = T;
    if (shots == 0) return QSIM_OK;
    if (!(T > 0.0)) { set_error("the state has zero norm"); return QSIM_EINVAL; }
    // uniforms (the library's SplitMix64 stream for `seed`, as qsim_sample), then the slice of each shot
    std::vector<double> u((size_t)shots);
    double* du = nullptr;
    if ((e = cudaMalloc(&du, sizeof(double) * shots)) != cudaSuccess) return cuda_fail(e, "uniform buffer");
    e = launch_uniforms(seed, shots, du, win.s_comp);
    if (e == cudaSuccess) e = cudaMemcpyAsync(u.data(), du, sizeof(double) * shots, cudaMemcpyDeviceToHost, win.s_comp);
    if (e == cudaSuccess) e = cudaStreamSynchronize(win.s_comp);
    cudaFree(du);
    if (e != cudaSuccess) return cuda_fail(e, "uniforms");
    std::vector<std::vector<int64_t>> by(nsl);
    std::vector<std::vector<double>> ul(nsl);
    for (int64_t i = 0; i < shots; ++i) {
        const double x = u[i] * T;
        uint64_t s = (uint64_t)(std::upper_bound(cum.begin() + 1, cum.end(), x) - (cum.begin() + 1));
        if (s >= nsl) s = nsl - 1;
        while (tot[s] <= 0.0 && s > 0) --s;  // never a slice of zero probability
        double v = (x - cum[s]) / tot[s];
        v = std::min(std::max(v, 0.0), 1.0 - 0x1.0p-53);
        by[s].push_back(i);
        ul[s].push_back(v);
    }
    // pass 2: sample inside every slice that received shots
    std::vector<uint64_t> loc;
    for (uint64_t s = 0; s < nsl; ++s) {
        if (by[s].empty()) continue;
        e = cudaMemcpyAsync(win.buf[0], H + s * win.bytes, win.bytes, cudaMemcpyHostToDevice, win.s_comp);
        if (e != cudaSuccess) return cuda_fail(e, "slice copy in");
        loc.assign(by[s].size(), 0);
        if ((rc = qsim_sample_uniforms(win.hd[0], ul[s].data(), (int64_t)ul[s].size(), loc.data())) != QSIM_OK) return rc;
        for (size_t j = 0; j < loc.size(); ++j) out[by[s][j]] = (s << Wq) | loc[j];
    }
    return QSIM_OK;
}
