// plan.cu -- circuit planning and execution.
//
// Fusion (paper Sec. 2.1: gate fusion groups gate applications into one larger matrix, raising arithmetic
// intensity; the best width depends on architecture and precision, Sec. 2.2 lists defaults 4/5/5): a greedy
// pass collects, starting from the earliest unplaced gate, every later gate that (a) is not blocked by an
// earlier unplaced gate sharing a qubit and (b) keeps the block within `max_fused` qubits. Diagonal gates
// commute with each other, so a diagonal gate is blocked only by earlier unplaced NON-diagonal gates.
// Each block becomes one device pass: a diagonal pass (only non-unit factors touched), a dense pass on CUDA
// cores (k <= 4 register gather, k = 5, 6 shared-memory tile) or a tensor-core pass (complex64, k >= tc_min_k).
// Block matrices are composed in FP64 on the device (k_compose.cu).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <unordered_map>
#include <utility>
#include <vector>

#include "capi_state.h"
#include "internal.h"

namespace qsim {

enum OpKind { OP_DENSE_SMALL = 0, OP_DIAG = 1, OP_DENSE_TILE = 2, OP_TC = 3, OP_SWAP = 4, OP_PHASE = 5,
              OP_MERGED = 6 /* a pass folded into the pass before it (phase epilogue, second block of a pair);
                               dropped from the plan */,
              OP_TC_PAIR = 7 /* two 6-qubit tensor-core blocks in one pass */ };

struct PlanOp {
    int kind = OP_DENSE_SMALL;
    int k = 0, nc = 0;
    int targets[QSIM_MAX_TARGETS] = {0};
    int controls[QSIM_MAX_CONTROLS] = {0};
    std::vector<double> mat;   // OP_DENSE_SMALL: 2^k x 2^k; OP_DIAG: 2^k diagonal entries (FP64, interleaved)
    std::vector<int> touch;    // OP_DIAG: patterns with a non-unit factor
    size_t dev_off = 0;        // OP_DENSE_TILE, OP_TC: byte offset of the operand in the plan buffer
    int precision = QSIM_PREC_SIMT;
    int compose_idx = -1;      // block index in the composition (-1: a single input gate)
    int64_t gates = 1;
    int nswap = 0;             // OP_SWAP: exchange qubit swap_a[i] with swap_b[i]
    int swap_a[8] = {0}, swap_b[8] = {0};
    PhasePacked phase;         // OP_PHASE: launch parameters; tables at dev_off
    std::vector<unsigned char> blob;  // OP_PHASE, OP_TC with a phase epilogue: the tables until uploaded
    PhaseForm form;            // OP_PHASE (and the epilogue it becomes): the combined phase
    bool has_epi = false;      // OP_TC: the output gets the phase of `form` (the pass that followed it)
    bool lines = false;        // OP_TC: line-group data path (B prepared in its column order)
    TcEpiPacked epi;           // OP_TC with has_epi: launch parameters; tables at epi_off
    size_t epi_off = 0;
    int targets2[6] = {0};     // OP_TC_PAIR: the second block's targets (the first block's are `targets`)
    int compose_idx2 = -1;     // OP_TC_PAIR: the second block's composition
};

struct PlanExtra {
    size_t epi_scratch_off = 0;  // per-tile factors of phase epilogues (shared: passes run in order)
};

}  // namespace qsim

struct qsim_plan {
    int n = 0;
    int dtype = QSIM_C64;
    std::vector<qsim::PlanOp> ops;
    void* dbuf = nullptr;
    size_t dbuf_bytes = 0;
    qsim_plan_info info{};
    bool use_graph = false;
    cudaGraphExec_t gexec = nullptr;
    const qsim_state* ghandle = nullptr;
    void* gpsi = nullptr;
    cudaStream_t gstream = nullptr;
    qsim::PlanExtra extra;
    bool dry = false;  // planned on the host only: no device buffer, cannot execute
    bool pooled = false;    // dbuf came from the library's memory pool
    bool small = false;     // a whole-plan execution is one resident launch (k_small.cu)
    size_t small_off = 0;   // its program in the plan buffer
};

namespace qsim {

static inline int popcnt(uint64_t v) { return __builtin_popcountll(v); }

// One block: scan the unplaced gates in order and absorb every gate that is not blocked by an earlier
// unplaced gate on a shared qubit (a diagonal gate is blocked only by non-diagonal ones) and that fits: with
// a fixed window W, gates whose qubits lie inside W; otherwise (W = 0) gates that keep the growing qubit set
// within kmax qubits (kmax - 1 once it touches a qubit in `narrow`), starting from `seed`.
// `und` lists the unplaced gates in circuit order.
static std::vector<int> build_block(const std::vector<uint64_t>& gmask, const std::vector<char>& gdiag,
                                    const std::vector<int>& und, int seed, uint64_t W, int kmax, uint64_t narrow) {
    auto lim = [&](uint64_t S) { return (S & narrow) ? kmax - 1 : kmax; };
    std::vector<int> blk;
    uint64_t Q = 0, bany = 0, bdiag = 0;
    if (seed >= 0) { blk.push_back(seed); Q = gmask[seed]; }
    for (const int i : und) {
        if (i == seed) continue;
        const uint64_t qs = gmask[i];
        const bool blocked = gdiag[i] ? (qs & bany) != 0 : (qs & (bany | bdiag)) != 0;
        const bool fits = W ? (qs & ~W) == 0 : popcnt(Q | qs) <= lim(Q | qs);
        if (!blocked && fits) {
            blk.push_back(i);
            Q |= qs;
        } else if (gdiag[i]) {
            bdiag |= qs;
        } else {
            bany |= qs;
        }
        // nothing further can join once every qubit a new gate could use is blocked by a non-diagonal gate
        const uint64_t usable = W ? W : (popcnt(Q) >= lim(Q) ? Q : ~0ull);
        if ((usable & ~bany) == 0) break;
    }
    std::sort(blk.begin(), blk.end());
    return blk;
}

// Window candidates kept across the steps of one grouping: a window's block depends only on the unplaced gates
// that touch it (gates elsewhere neither fit it nor block the qubits it uses), so it is rebuilt only after a
// block on one of its qubits was placed.
struct WinCache {
    std::vector<std::vector<int>> blk;
    std::vector<char> valid;
};

// Candidates for the next block (group_gates keeps the largest, or looks one step ahead):
// every window of kmax consecutive qubits (all available gates inside it), and, for every qubit, its
// earliest unplaced gate when no earlier unplaced gate blocks it, grown greedily. The plain greedy choice
// (seeded at the earliest unplaced gate) is one of the candidates. On nearest-neighbour circuits the
// windows tile the (qubit, time) plane in diamonds, about twice the gates per block of the plain greedy.
// Blocks that touch a qubit in `narrow` hold at most kmax - 1 qubits (a window over such a qubit is one
// qubit narrower).
static std::vector<std::vector<int>> candidates(const std::vector<uint64_t>& gmask, const std::vector<char>& gdiag,
                                                int n, int kmax, const std::vector<char>* gwide, int wide_factor,
                                                const std::vector<char>& done, int first, uint64_t narrow,
                                                bool* wide_won = nullptr, WinCache* wc = nullptr) {
    const int G = (int)gmask.size();
    std::vector<std::vector<int>> out;
    std::vector<int> wide;
    // the unplaced gates, in order: every candidate below scans a prefix of them
    std::vector<int> und;
    und.reserve(G - first);
    for (int i = first; i < G; ++i)
        if (!done[i]) und.push_back(i);
    if (gwide) {
        const uint64_t all = n >= 64 ? ~0ull : (1ull << n) - 1;
        uint64_t bany = 0;
        for (size_t u = 0; u < und.size() && bany != all; ++u) {
            const int i = und[u];
            if (gdiag[i] && (*gwide)[i] && (gmask[i] & bany) == 0) wide.push_back(i);
            else if (!gdiag[i]) bany |= gmask[i];
        }
    }
    if (popcnt(gmask[first]) > kmax && !(gwide && (*gwide)[first] && gdiag[first])) {
        out.push_back({first});  // wider than the fusion width: a block of its own
        return out;
    }
    size_t best = 0;
    const int wmax = std::min(kmax, n);
    if (wc && wc->valid.size() != (size_t)std::max(0, n - wmax + 1)) {
        wc->valid.assign(std::max(0, n - wmax + 1), 0);
        wc->blk.assign(wc->valid.size(), {});
    }
    for (int a0 = 0; a0 + wmax <= n; ++a0) {
        std::vector<int> blk;
        if (wc && wc->valid[a0]) {
            blk = wc->blk[a0];
        } else {
            uint64_t W = ((wmax == 64) ? ~0ull : ((1ull << wmax) - 1)) << a0;
            if (W & narrow) W &= ~(1ull << (a0 + wmax - 1));
            blk = build_block(gmask, gdiag, und, -1, W, kmax, narrow);
            if (wc) { wc->blk[a0] = blk; wc->valid[a0] = 1; }
        }
        best = std::max(best, blk.size());
        if (!blk.empty()) out.push_back(std::move(blk));
    }
    uint64_t seen = 0, bany = 0, bdiag = 0;
    for (size_t u = 0; u < und.size() && popcnt(seen) < n; ++u) {
        const int i = und[u];
        const uint64_t qs = gmask[i];
        const bool blocked = gdiag[i] ? (qs & bany) != 0 : (qs & (bany | bdiag)) != 0;
        if ((qs & ~seen) && !blocked && popcnt(qs) <= kmax) {
            auto blk = build_block(gmask, gdiag, und, i, 0, kmax, narrow);
            best = std::max(best, blk.size());
            if (!blk.empty()) out.push_back(std::move(blk));
        }
        seen |= qs;
        if (gdiag[i]) bdiag |= qs; else bany |= qs;
    }
    // A phase pass costs a full pass whatever it holds, and it only grows while dense blocks make progress
    // (each one frees the diagonal gates behind it): it wins against dense blocks of less than
    // 1 / wide_factor of its size.
    if (wide.size() > (size_t)wide_factor * best) {
        out.clear();
        out.push_back(std::move(wide));
        if (wide_won) *wide_won = true;
    }
    if (out.empty()) out.push_back({first});
    return out;
}

// Fusion into blocks of at most kmax qubits: at each step the largest candidate, or, with lookahead > 0,
// the candidate among the `lookahead` largest distinct ones whose size plus the size of the best block
// after it is largest (one step of look-ahead; slower planning, sometimes fewer blocks).
std::vector<std::vector<int>> group_gates(const std::vector<uint64_t>& gmask, const std::vector<char>& gdiag, int n,
                                          int kmax, const std::vector<char>* gwide, int wide_factor, int lookahead,
                                          uint64_t narrow, bool* wide_used) {
    const int G = (int)gmask.size();
    const int LA = lookahead;
    std::vector<std::vector<int>> blocks;
    std::vector<char> done(G, 0);
    int first = 0;
    auto next_first = [&](int f) { while (f < G && done[f]) ++f; return f; };
    WinCache wc;
    const int wmax = std::min(kmax, n);
    while (true) {
        first = next_first(first);
        if (first >= G) break;
        auto cands = candidates(gmask, gdiag, n, kmax, gwide, wide_factor, done, first, narrow, wide_used, &wc);
        size_t pick = 0;
        for (size_t c = 1; c < cands.size(); ++c)
            if (cands[c].size() > cands[pick].size()) pick = c;
        if (LA > 0 && cands.size() > 1) {
            // one step of look-ahead among the LA largest distinct candidates: size + best next size
            std::vector<size_t> order(cands.size());
            for (size_t c = 0; c < order.size(); ++c) order[c] = c;
            std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return cands[x].size() > cands[y].size(); });
            double best_score = -1;
            int tried = 0;
            for (size_t oi = 0; oi < order.size() && tried < LA; ++oi) {
                const auto& cb = cands[order[oi]];
                bool dup = false;
                for (size_t oj = 0; oj < oi && !dup; ++oj) dup = cands[order[oj]] == cb;
                if (dup) continue;
                ++tried;
                for (int g : cb) done[g] = 1;
                const int f2 = next_first(first);
                size_t nxt = 0;
                if (f2 < G) {
                    auto c2 = candidates(gmask, gdiag, n, kmax, gwide, wide_factor, done, f2, narrow);
                    for (const auto& b2 : c2) nxt = std::max(nxt, b2.size());
                }
                for (int g : cb) done[g] = 0;
                const double score = (double)cb.size() + (double)nxt;
                if (score > best_score) { best_score = score; pick = order[oi]; }
            }
        }
        std::vector<int> best = std::move(cands[pick]);
        uint64_t QB = 0;
        for (int i : best) { done[i] = 1; QB |= gmask[i]; }
        for (int a0 = 0; a0 < (int)wc.valid.size(); ++a0)
            if (((((wmax == 64) ? ~0ull : ((1ull << wmax) - 1)) << a0) & QB) != 0) wc.valid[a0] = 0;
        blocks.push_back(std::move(best));
    }
    return blocks;
}

// Fusion by beam search: keep the `beam` partial groupings (all with the same number of blocks) that have
// placed the most gates, extend each by every candidate of its next block, and stop at the first grouping
// that places every gate (so none with fewer blocks was pruned while it was still ahead). Partial groupings
// that placed the same set of gates are kept once (Zobrist hash of the placed set).
std::vector<std::vector<int>> group_gates_beam(const std::vector<uint64_t>& gmask, const std::vector<char>& gdiag,
                                               int n, int kmax, const std::vector<char>* gwide, int wide_factor,
                                               int beam, uint64_t narrow) {
    const int G = (int)gmask.size();
    if (G == 0) return {};
    std::vector<uint64_t> zob(G);
    uint64_t z = 0x243F6A8885A308D3ull;
    for (int i = 0; i < G; ++i) {  // SplitMix64 steps: a fixed, well-mixed 64-bit key per gate
        z += 0x9E3779B97F4A7C15ull;
        uint64_t x = z;
        x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
        x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
        zob[i] = x ^ (x >> 31);
    }
    struct State {
        std::vector<char> done;
        std::vector<std::vector<int>> blocks;
        int placed = 0, first = 0;
        uint64_t hash = 0;
    };
    struct Child {
        int parent;
        std::vector<int> blk;
        int placed, first;
        uint64_t hash;
    };
    std::vector<State> cur(1);
    cur[0].done.assign(G, 0);
    while (true) {
        for (const State& st : cur)
            if (st.placed == G) return st.blocks;
        std::vector<Child> kids;
        for (int pi = 0; pi < (int)cur.size(); ++pi) {
            State& st = cur[pi];
            auto cands = candidates(gmask, gdiag, n, kmax, gwide, wide_factor, st.done, st.first, narrow);
            for (size_t c = 0; c < cands.size(); ++c) {
                bool dup = false;
                for (size_t d = 0; d < c && !dup; ++d) dup = cands[d] == cands[c];
                if (dup) continue;
                uint64_t h = st.hash;
                for (int g : cands[c]) { h ^= zob[g]; st.done[g] = 1; }
                int f = st.first;
                while (f < G && st.done[f]) ++f;
                for (int g : cands[c]) st.done[g] = 0;
                kids.push_back({pi, std::move(cands[c]), st.placed, f, h});
                kids.back().placed += (int)kids.back().blk.size();
            }
        }
        // most gates placed first; among equals, the one whose earliest unplaced gate is latest
        std::stable_sort(kids.begin(), kids.end(), [](const Child& a, const Child& b) {
            return a.placed != b.placed ? a.placed > b.placed : a.first > b.first;
        });
        std::vector<State> nxt;
        std::vector<uint64_t> seen;
        for (const Child& k : kids) {
            if ((int)nxt.size() >= beam) break;
            if (std::find(seen.begin(), seen.end(), k.hash) != seen.end()) continue;
            seen.push_back(k.hash);
            State ns;
            ns.done = cur[k.parent].done;
            ns.blocks = cur[k.parent].blocks;
            for (int g : k.blk) ns.done[g] = 1;
            ns.blocks.push_back(k.blk);
            ns.placed = k.placed;
            ns.first = k.first;
            ns.hash = k.hash;
            nxt.push_back(std::move(ns));
        }
        cur.swap(nxt);
    }
}

// Groupings by gate structure. A grouping depends only on each gate's qubit set, whether it is diagonal and
// whether it may join a phase pass, and on the planning options -- not on the matrices -- so circuits that
// repeat a structure (a batch of chains of one width and depth, or one circuit planned again with new angles)
// are grouped once. Keys are kept whole (no reliance on the hash alone); at 1024 entries the cache starts
// over. qsim_plan_cache_clear empties it.
namespace {
struct GroupCache {
    std::mutex mu;
    std::unordered_map<uint64_t, std::vector<std::pair<std::vector<uint64_t>, std::vector<std::vector<int>>>>> map;
    size_t entries = 0;
};
GroupCache& group_cache() {
    static GroupCache c;
    return c;
}
uint64_t fnv1a(const std::vector<uint64_t>& w) {
    uint64_t h = 1469598103934665603ull;
    for (uint64_t v : w)
        for (int b = 0; b < 8; ++b) { h ^= (v >> (8 * b)) & 0xFF; h *= 1099511628211ull; }
    return h;
}
}  // namespace

bool group_cache_get(const std::vector<uint64_t>& key, std::vector<std::vector<int>>& out) {
    GroupCache& c = group_cache();
    std::lock_guard<std::mutex> lk(c.mu);
    auto it = c.map.find(fnv1a(key));
    if (it == c.map.end()) return false;
    for (const auto& e : it->second)
        if (e.first == key) { out = e.second; return true; }
    return false;
}

void group_cache_put(const std::vector<uint64_t>& key, const std::vector<std::vector<int>>& blocks) {
    GroupCache& c = group_cache();
    std::lock_guard<std::mutex> lk(c.mu);
    if (c.entries >= 1024) { c.map.clear(); c.entries = 0; }
    auto& bucket = c.map[fnv1a(key)];
    for (const auto& e : bucket)
        if (e.first == key) return;
    bucket.emplace_back(key, blocks);
    ++c.entries;
}

static double op_bytes(const PlanOp& op, int n, size_t amp) {
    if (op.kind == OP_SWAP) return 2.0 * amp * std::ldexp(1.0, n) * (1.0 - std::ldexp(1.0, -op.nswap));
    if (op.kind == OP_PHASE) return 2.0 * amp * std::ldexp(1.0, n);
    const double groups = std::ldexp(1.0, n - op.k - op.nc);
    if (op.kind == OP_DIAG) return 2.0 * amp * groups * (double)op.touch.size();
    return 2.0 * amp * groups * (double)(1 << op.k);
}

// Plan buffers come from a memory pool of the library's own (stream-ordered allocation): planning on several
// host threads at once, and one-shot runs that create and destroy a plan per call, then avoid the device-wide
// locking of cudaMalloc / cudaFree. Up to 256 MiB of freed plan buffers stay reserved in the pool for reuse.
static cudaMemPool_t plan_pool(int device) {
    static std::mutex mu;
    static std::vector<cudaMemPool_t> pools;
    static std::vector<char> tried;
    std::lock_guard<std::mutex> lk(mu);
    if (device < 0) return nullptr;
    if ((size_t)device >= pools.size()) {
        pools.resize(device + 1, nullptr);
        tried.resize(device + 1, 0);
    }
    if (!tried[device]) {  // one attempt per device; without a pool, plain cudaMalloc
        tried[device] = 1;
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        cudaMemPool_t mp = nullptr;
        if (cudaMemPoolCreate(&mp, &props) != cudaSuccess) { cudaGetLastError(); return nullptr; }
        uint64_t keep = 256ull << 20;
        cudaMemPoolSetAttribute(mp, cudaMemPoolAttrReleaseThreshold, &keep);
        pools[device] = mp;
    }
    return pools[device];
}

static cudaError_t plan_buffer_alloc(void** out, size_t bytes, cudaStream_t s, bool* pooled) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    cudaMemPool_t mp = plan_pool(dev);
    *pooled = mp != nullptr;
    if (!mp) return cudaMalloc(out, bytes);
    return cudaMallocFromPoolAsync(out, bytes, mp, s);
}

// Only once no work that uses the buffer can be in flight (the callers synchronise first).
static void plan_buffer_free(void* ptr, bool pooled) {
    if (!ptr) return;
    if (pooled) {
        cudaFreeAsync(ptr, cudaStreamLegacy);
        cudaStreamSynchronize(cudaStreamLegacy);  // returned to the pool before this call returns
    } else {
        cudaFree(ptr);
    }
}

static int enqueue_ops(qsim_state* h, const qsim_plan* p, size_t first = 0, size_t count = (size_t)-1,
                       const uint64_t* first_from_basis = nullptr) {
    cudaError_t e = cudaSuccess;
    const size_t last = std::min(p->ops.size(), count == (size_t)-1 ? p->ops.size() : first + count);
    if (p->small && first == 0 && last == p->ops.size()) {
        e = launch_small_run(h->dtype, h->psi, h->n, static_cast<char*>(p->dbuf) + p->small_off, (int)last, h->derr,
                             h->stream, h->dev, first_from_basis);
        if (e != cudaErrorCooperativeLaunchTooLarge) return e == cudaSuccess ? QSIM_OK : cuda_fail(e, "resident plan launch");
        // fewer SMs available than the device has (e.g. a share of them under MPS): launch per pass
        cudaGetLastError();
        e = cudaSuccess;
        if (first_from_basis) {
            e = launch_set_basis(h->dtype, h->psi, h->n, *first_from_basis, h->stream, h->dev);
            if (e != cudaSuccess) return cuda_fail(e, "plan pass launch");
            first_from_basis = nullptr;
        }
    }
    for (size_t oi = first; oi < last; ++oi) {
        const PlanOp& op = p->ops[oi];
        const uint64_t* fb = oi == first ? first_from_basis : nullptr;
        switch (op.kind) {
            case OP_DENSE_SMALL:
                e = launch_dense_small(h->dtype, h->psi, h->n, op.k, op.targets, op.nc, op.controls, op.mat.data(),
                                       h->stream, h->dev);
                break;
            case OP_DIAG:
                e = launch_diag(h->dtype, h->psi, h->n, op.k, op.targets, op.nc, op.controls, op.mat.data(), op.touch,
                                h->stream, h->dev);
                break;
            case OP_DENSE_TILE:
                e = launch_dense_tile(h->dtype, h->psi, h->n, op.k, op.targets, op.nc, op.controls,
                                      static_cast<char*>(p->dbuf) + op.dev_off, h->stream, h->dev);
                break;
            case OP_TC:
                e = launch_tc_apply(h->psi, h->n, op.k, op.targets, static_cast<char*>(p->dbuf) + op.dev_off,
                                    op.precision, h->derr, h->stream, h->dev,
                                    op.has_epi ? static_cast<char*>(p->dbuf) + op.epi_off : nullptr,
                                    op.has_epi ? &op.epi : nullptr,
                                    op.has_epi ? static_cast<char*>(p->dbuf) + p->extra.epi_scratch_off : nullptr,
                                    fb, op.lines);
                break;
            case OP_TC_PAIR:
                e = launch_tc_pair(h->psi, h->n, op.targets, op.targets2, static_cast<char*>(p->dbuf) + op.dev_off,
                                   h->derr, h->stream, h->dev, fb);
                break;
            case OP_MERGED:
                break;
            case OP_SWAP:
                e = launch_swap(h->dtype, h->psi, h->n, op.swap_a, op.swap_b, op.nswap, h->stream, h->dev, nullptr);
                break;
            case OP_PHASE:
                e = launch_phase(h->dtype, h->psi, h->n, static_cast<char*>(p->dbuf) + op.dev_off, op.phase, h->stream,
                                 h->dev);
                break;
        }
        if (e != cudaSuccess) return cuda_fail(e, "plan pass launch");
    }
    return QSIM_OK;
}

}  // namespace qsim

using namespace qsim;

extern "C" {

int qsim_plan_cache_clear(void) {
    GroupCache& c = group_cache();
    std::lock_guard<std::mutex> lk(c.mu);
    c.map.clear();
    c.entries = 0;
    return QSIM_OK;
}

int qsim_plan_create(const qsim_circuit* c, int dtype, const qsim_run_opts* opts_in, void* stream_v,
                     qsim_plan_h* out, qsim_plan_info* info) {
    set_error("%s", "");
    const auto t0 = std::chrono::steady_clock::now();
    if (!c || !out) { set_error("NULL argument"); return QSIM_EINVAL; }
    *out = nullptr;
    if (c->n < 1 || c->n > QSIM_MAX_QUBITS) { set_error("n = %d outside 1..%d", c->n, QSIM_MAX_QUBITS); return QSIM_EINVAL; }
    if (dtype != QSIM_C64 && dtype != QSIM_C128) { set_error("unknown dtype"); return QSIM_EINVAL; }
    if (c->num_gates < 0 || (c->num_gates > 0 && !c->gates)) { set_error("bad gate list"); return QSIM_EINVAL; }
    qsim_run_opts opts{};
    if (opts_in) opts = *opts_in;
    if (opts.mode != QSIM_RUN_PLAIN && opts.mode != QSIM_RUN_FUSED) { set_error("unknown mode"); return QSIM_EINVAL; }
    int kmax = opts.max_fused == 0 ? 5 : opts.max_fused;
    // 7-qubit blocks run on the tensor cores in FP16 split products (complex64); dry runs (host-only pass
    // counts) may also plan 7- and 8-qubit blocks at any precision, for sizing the fusion width
    if (opts.precision < QSIM_PREC_SIMT || opts.precision > QSIM_PREC_FP16X3) { set_error("unknown precision"); return QSIM_EINVAL; }
    const int kmax_ok = opts.dry_run ? 8 : (opts.precision == QSIM_PREC_FP16X3 && dtype == QSIM_C64 ? 7 : 6);
    if (kmax < 1 || kmax > kmax_ok) {
        set_error("max_fused must be 1..6 (7 with QSIM_PREC_FP16X3 on a complex64 state; 1..8 in a dry run)");
        return QSIM_EINVAL;
    }
    // FP16X3 with pair_blocks: consecutive 6-qubit blocks are paired into one pass where they fit a tile
    const bool pair_blocks = opts.precision == QSIM_PREC_FP16X3 && opts.pair_blocks != 0;
    const int tc_min = opts.tc_min_k == 0 ? 5 : opts.tc_min_k;
    const int n = c->n;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_v);
    const bool dry = opts.dry_run != 0;
    DevInfo dev;
    cudaError_t e = cudaSuccess;
    if (!dry) {
        e = cudaGetDevice(&dev.device);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&dev.num_sms, cudaDevAttrMultiProcessorCount, dev.device);
        if (e != cudaSuccess) return cuda_fail(e, "querying the device");
    }

    const int G = c->num_gates;
    std::vector<uint64_t> gmask(G);
    std::vector<char> gdiag(G);
    for (int i = 0; i < G; ++i) {
        const qsim_gate& g = c->gates[i];
        int rc = validate_qubits(n, g.targets, g.k, g.controls, g.nc, QSIM_MAX_TARGETS);
        if (rc) { set_error("gate %d: invalid qubits", i); return rc; }
        if (!g.matrix) { set_error("gate %d: NULL matrix", i); return QSIM_EINVAL; }
        if (!is_unitary(g.matrix, g.k, 1e-8 * (1 << g.k))) { set_error("gate %d: matrix is not unitary", i); return QSIM_EINVAL; }
        uint64_t m = 0;
        for (int j = 0; j < g.k; ++j) m |= 1ull << g.targets[j];
        for (int j = 0; j < g.nc; ++j) m |= 1ull << g.controls[j];
        gmask[i] = m;
        gdiag[i] = is_diagonal(g.matrix, g.k);
    }

    qsim_plan* p = new (std::nothrow) qsim_plan();
    if (!p) { set_error("out of host memory"); return QSIM_ENOMEM; }
    p->n = n;
    p->dtype = dtype;
    p->use_graph = opts.use_graph != 0;

    // ---- group gates into blocks -------------------------------------------------------------------------
    std::vector<std::vector<int>> blocks;
    // In fused plans, diagonal gates of one or two qubits may also gather in a phase pass of any width
    // (n >= 10). Not with global qubits: the phase tables name physical positions, which the reorder passes
    // would move.
    std::vector<char> gwide(G, 0);
    const bool remap_later = opts.local_qubits > 0 && opts.local_qubits < n;  // global qubits: targets remapped
    // 7-qubit tensor-core blocks need n >= 14 (a tile is 7 row bits x 7 targets); plans with global qubits
    // keep 6-qubit blocks
    if (!dry && kmax == 7 && (n < 14 || remap_later)) kmax = 6;
    const bool tc7 = kmax == 7 && opts.precision == QSIM_PREC_FP16X3 && dtype == QSIM_C64 && n >= 14;
    // 7-qubit blocks keep off qubits 0..2: on those the 7-qubit kernel moves partly used lines (4.0-5.5 ms at 30
    // qubits against 2.9-3.2 ms above them), while 6-qubit blocks there have the line-group and pair-rows paths
    const uint64_t narrow = tc7 ? 0x7ull : 0;
    const bool use_wide = opts.mode == QSIM_RUN_FUSED && n >= 10 && !remap_later;
    for (int i = 0; i < G; ++i) gwide[i] = use_wide && gdiag[i] && phase_gate_ok(c->gates[i]);
    // Estimated cost of a grouping in passes: a 7-qubit tensor-core block streams the state like any pass
    // but takes about 1.2 times as long (3.1-3.2 against 2.6 ms at 30 qubits); a phase pass counts 1, or 0.15
    // when it follows a dense block of at most 6 qubits (it becomes that block's epilogue, which only a
    // tensor-core precision has).
    auto cost = [&](const std::vector<std::vector<int>>& bl) {
        double cs = 0.0;
        bool prev_dense6 = false;
        for (const auto& b : bl) {
            uint64_t Q = 0;
            bool wide = use_wide, diag = true;
            for (int gi : b) { Q |= gmask[gi]; wide = wide && gwide[gi]; diag = diag && gdiag[gi]; }
            const int k = popcnt(Q);
            if (wide && k > 6) cs += (prev_dense6 && opts.precision != QSIM_PREC_SIMT) ? 0.15 : 1.0;
            else cs += (tc7 && k == 7 && !wide) ? 1.2 : 1.0;
            prev_dense6 = !diag && k <= 6;
        }
        return cs;
    };
    auto group_all = [&](int km, uint64_t nar) {
        std::vector<std::vector<int>> bl;
        bool have = false;
        // whether a phase pass should wait for more diagonal gates depends on the circuit, and so does
        // whether looking one block ahead pays: keep the cheapest grouping (the fewest blocks of each kind).
        // A grouping that never picked the phase candidate at factor f is also the grouping at 2f (every
        // step sees the same candidates, and the phase candidate loses by a wider margin), so the larger
        // factors are skipped then.
        for (int la = 0; la <= (opts.plan_effort > 0 ? 4 : 0); la += 4) {
            bool picked = true;
            for (int f = 1; f <= (use_wide ? 4 : 1) && picked; f *= 2) {
                picked = false;
                auto alt = group_gates(gmask, gdiag, n, km, use_wide ? &gwide : nullptr, f, la, nar, &picked);
                if (!have || cost(alt) < cost(bl)) { bl.swap(alt); have = true; }
            }
        }
        if (opts.plan_effort >= 2)
            for (int f = 1; f <= (use_wide ? 4 : 1); f *= 2) {
                auto alt = group_gates_beam(gmask, gdiag, n, km, use_wide ? &gwide : nullptr, f,
                                            opts.plan_effort >= 3 ? 32 : 8, nar);
                if (cost(alt) < cost(bl)) bl.swap(alt);
            }
        return bl;
    };
    if (opts.mode == QSIM_RUN_PLAIN) {
        for (int i = 0; i < G; ++i) blocks.push_back({i});
    } else {
        std::vector<uint64_t> key = {0 /* a plan */, (uint64_t)n, (uint64_t)kmax, narrow, (uint64_t)use_wide,
                                     (uint64_t)opts.plan_effort, (uint64_t)(opts.precision != QSIM_PREC_SIMT),
                                     (uint64_t)tc7, (uint64_t)G};
        key.reserve(key.size() + 2 * (size_t)G);
        for (int i = 0; i < G; ++i) {
            key.push_back(gmask[i]);
            key.push_back((uint64_t)gdiag[i] | ((uint64_t)gwide[i] << 1));
        }
        if (!group_cache_get(key, blocks)) {
            blocks = group_all(kmax, narrow);
            // 7-qubit blocks pay on nearest-neighbour circuits (whole windows of adjacent qubits), not always
            // (random target sets, the QFT's phase epilogues): the 6-qubit grouping is kept when it is cheaper
            if (tc7) {
                auto b6 = group_all(6, 0);
                if (cost(b6) <= cost(blocks)) blocks.swap(b6);
            }
            group_cache_put(key, blocks);
        }
    }
    // A diagonal block moves after a tensor-core block that follows it when they share no qubit (so they
    // commute), and neighbouring diagonal blocks merge (diagonal gates commute): a phase pass then follows
    // the tensor-core block and becomes its epilogue.
    if (use_wide && opts.precision != QSIM_PREC_SIMT && dtype == QSIM_C64) {
        auto qubits = [&](const std::vector<int>& blk) { uint64_t m = 0; for (int gi : blk) m |= gmask[gi]; return m; };
        auto all_wide = [&](const std::vector<int>& blk) {
            for (int gi : blk) if (!gwide[gi]) return false;
            return true;
        };
        auto tc_like = [&](const std::vector<int>& blk) {
            const int kb = popcnt(qubits(blk));
            bool diag = true;
            for (int gi : blk) diag = diag && gdiag[gi];
            return !diag && kb >= tc_min && kb <= 6 && tc_supported(kb, opts.precision) && n >= kb + 7 &&
                   !(blk.size() == 1 && c->gates[blk[0]].nc > 0);
        };
        for (bool changed = true; changed;) {
            changed = false;
            for (size_t i = 0; i + 1 < blocks.size(); ++i) {
                if (!all_wide(blocks[i])) continue;
                if (all_wide(blocks[i + 1])) {
                    blocks[i].insert(blocks[i].end(), blocks[i + 1].begin(), blocks[i + 1].end());
                    blocks.erase(blocks.begin() + (long)i + 1);
                    changed = true;
                } else if (tc_like(blocks[i + 1]) && (qubits(blocks[i]) & qubits(blocks[i + 1])) == 0) {
                    std::swap(blocks[i], blocks[i + 1]);
                    ++i;  // the diagonal block now sits at i + 1; look at what follows it on the next sweep
                    changed = true;
                }
            }
        }
    }

    // ---- decide each block's pass and lay out the device buffer --------------------------------------------
    const size_t amp = dtype == QSIM_C64 ? 8 : 16;
    std::vector<ComposeBlock> cblocks;
    std::vector<ComposeGate> cgates;
    std::vector<double> pool;  // gate matrices for composition (FP64 complex)
    int64_t compose_out = 0;   // complex entries
    int max_kb = 1;
    size_t dev_bytes = 0;
    auto align = [](size_t v) { return (v + 1023) & ~(size_t)1023; };
    struct Pending { int op; int kind; int kb; };  // device operand still to produce from a composed matrix
    std::vector<Pending> pending;
    std::vector<int> direct;  // ops whose gate matrix is uploaded as it is (single gates on 7-8 qubits)

    for (const auto& blk : blocks) {
        PlanOp op;
        op.gates = (int64_t)blk.size();
        uint64_t Qb = 0;
        bool wide_ok = use_wide;
        for (int gi : blk) { Qb |= gmask[gi]; wide_ok = wide_ok && gwide[gi]; }
        if (wide_ok && popcnt(Qb) > 6) {
            // a phase pass (wider than the diagonal kernel's 6 qubits): the quadratic form of every gate
            std::vector<const qsim_gate*> gp;
            for (int gi : blk) gp.push_back(&c->gates[gi]);
            if (!phase_form_build(gp.data(), (int)gp.size(), n, op.form)) { delete p; set_error("phase pass"); return QSIM_EINVAL; }
            op.kind = OP_PHASE;
            p->ops.push_back(std::move(op));
            continue;
        }
        if (blk.size() == 1) {
            const qsim_gate& g = c->gates[blk[0]];
            op.k = g.k;
            op.nc = g.nc;
            std::memcpy(op.targets, g.targets, sizeof(int) * g.k);
            std::memcpy(op.controls, g.controls, sizeof(int) * g.nc);
            const int D = 1 << g.k;
            if (g.k >= 7 && !(tc7 && g.k == 7 && g.nc == 0 && !gdiag[blk[0]])) {
                // 7 or 8 targets (diagonal or not; a dense 7-qubit gate without controls goes to the tensor
                // cores in a 7-qubit FP16X3 plan, below): its own CUDA-core pass; the matrix is uploaded as
                // given, in the state precision (no composition: one gate)
                op.kind = OP_DENSE_TILE;
                op.mat.assign(g.matrix, g.matrix + 2 * D * D);
                op.dev_off = dev_bytes;
                dev_bytes = align(dev_bytes + (amp << (2 * g.k)));
                direct.push_back((int)p->ops.size());
                p->ops.push_back(std::move(op));
                continue;
            }
            if (gdiag[blk[0]]) {
                op.kind = OP_DIAG;
                op.mat.resize(2 * D);
                for (int i = 0; i < D; ++i) {
                    op.mat[2 * i] = g.matrix[2 * (i * D + i)];
                    op.mat[2 * i + 1] = g.matrix[2 * (i * D + i) + 1];
                }
                op.touch = nonunit_patterns(op.mat.data(), g.k);
            } else if (g.k <= 4) {
                op.kind = OP_DENSE_SMALL;
                op.mat.assign(g.matrix, g.matrix + 2 * D * D);
            } else {
                // k = 5, 6 single gate: compose trivially (one gate) to reuse the device conversion path
                op.kind = OP_DENSE_TILE;
            }
            if (op.kind == OP_DIAG || op.kind == OP_DENSE_SMALL) {
                p->ops.push_back(std::move(op));
                continue;
            }
        }
        // multi-gate block (or a single wide gate): local qubit list Q ascending
        uint64_t Q = 0;
        bool all_diag = true;
        for (int gi : blk) { Q |= gmask[gi]; all_diag = all_diag && gdiag[gi]; }
        // A dense 4-qubit block costs 64 FMA an amplitude on CUDA cores (FMA-bound, ~70 % of the HBM rate);
        // in a tensor-core plan it takes the two highest idle qubits as extra targets (U x I) and runs as a
        // 6-qubit tensor-core block at the HBM rate.
        if (!all_diag && blk.size() > 1 && popcnt(Q) == 4 && dtype == QSIM_C64 && opts.precision != QSIM_PREC_SIMT &&
            tc_min <= 6 && tc_supported(6, opts.precision) && n >= 6 + 7) {
            for (int q = n - 1; q >= 0 && popcnt(Q) < 6; --q) Q |= 1ull << q;
        }
        int qs[64], kb = 0, local[64];
        for (int q = 0; q < n; ++q) if ((Q >> q) & 1) { local[q] = kb; qs[kb++] = q; }
        if (blk.size() == 1 && !all_diag) {
            // single k = 5/6 gate keeps its controls and target order
            const qsim_gate& g = c->gates[blk[0]];
            kb = g.k;
            for (int j = 0; j < g.k; ++j) { qs[j] = g.targets[j]; local[g.targets[j]] = j; }
        }
        ComposeBlock cb;
        cb.kb = kb;
        cb.first_gate = (int)cgates.size();
        cb.num_gates = (int)blk.size();
        cb.out_off = compose_out;
        compose_out += (int64_t)1 << (2 * kb);
        max_kb = std::max(max_kb, kb);
        for (int gi : blk) {
            const qsim_gate& g = c->gates[gi];
            ComposeGate cg;
            cg.k = g.k;
            cg.nc = (blk.size() == 1) ? 0 : g.nc;
            for (int j = 0; j < g.k; ++j) cg.targets[j] = local[g.targets[j]];
            for (int j = 0; j < cg.nc; ++j) cg.controls[j] = local[g.controls[j]];
            cg.mat_off = (int64_t)pool.size() / 2;
            pool.insert(pool.end(), g.matrix, g.matrix + (2 << (2 * g.k)));
            cgates.push_back(cg);
        }
        op.compose_idx = (int)cblocks.size();
        cblocks.push_back(cb);
        op.k = kb;
        op.nc = 0;
        for (int j = 0; j < kb; ++j) op.targets[j] = qs[j];
        if (blk.size() == 1) {
            const qsim_gate& g = c->gates[blk[0]];
            op.nc = g.nc;
            std::memcpy(op.controls, g.controls, sizeof(int) * g.nc);
        }
        if (all_diag && !(tc7 && kb == 7)) {  // (the diagonal kernel stops at 6 qubits)
            op.kind = OP_DIAG;
            // structural support: pattern m is touched if some gate's factor there is not exactly 1
            const int D = 1 << kb;
            for (int m = 0; m < D; ++m) {
                bool nonunit = false;
                for (int gi : blk) {
                    const qsim_gate& g = c->gates[gi];
                    bool ctl = true;
                    for (int j = 0; j < g.nc; ++j) ctl = ctl && ((m >> local[g.controls[j]]) & 1);
                    if (!ctl) continue;
                    int t = 0;
                    for (int j = 0; j < g.k; ++j) t |= ((m >> local[g.targets[j]]) & 1) << j;
                    const int Dg = 1 << g.k;
                    if (g.matrix[2 * (t * Dg + t)] != 1.0 || g.matrix[2 * (t * Dg + t) + 1] != 0.0) nonunit = true;
                }
                if (nonunit) op.touch.push_back(m);
            }
        } else if (dtype == QSIM_C64 && opts.precision != QSIM_PREC_SIMT && kb >= tc_min && op.nc == 0 &&
                   tc_supported(kb, opts.precision) && n >= kb + 7) {
            op.kind = OP_TC;
            op.precision = opts.precision;
            op.dev_off = dev_bytes;
            // an FP16X3 block may still become a 3xTF32 one below (its line-group / pair-rows path): room for
            // the larger operand
            const int room_prec = opts.precision == QSIM_PREC_FP16X3 ? QSIM_PREC_TF32X3 : opts.precision;
            dev_bytes = align(dev_bytes + std::max(tc_operand_bytes(kb, opts.precision), tc_operand_bytes(kb, room_prec)));
        } else if (kb <= 4) {
            op.kind = OP_DENSE_SMALL;
        } else {
            op.kind = OP_DENSE_TILE;
            op.dev_off = dev_bytes;
            dev_bytes = align(dev_bytes + (amp << (2 * kb)));
        }
        pending.push_back({(int)p->ops.size(), op.kind, kb});
        p->ops.push_back(std::move(op));
    }

    // ---- phase passes: one right after a tensor-core block becomes that block's epilogue (it multiplies
    // the block's output in registers instead of taking a pass of its own); the others keep their pass ----
    for (size_t oi = 0; oi < p->ops.size(); ++oi) {
        PlanOp& op = p->ops[oi];
        if (op.kind != OP_PHASE) continue;
        PlanOp* prev = oi > 0 ? &p->ops[oi - 1] : nullptr;
        if (prev && prev->kind == OP_TC && prev->k <= 6 && !prev->has_epi && prev->precision != QSIM_PREC_BF16X6) {
            prev->has_epi = true;
            prev->form = std::move(op.form);
            prev->gates += op.gates;
            op.kind = OP_MERGED;
            continue;
        }
        phase_pack(op.form, dtype, op.blob, op.phase);
        op.dev_off = dev_bytes;
        dev_bytes = align(dev_bytes + op.blob.size());
    }
    // ---- FP16X3: blocks whose targets give a 3xTF32 block its line-group or pair-rows data path (qubits 0..3
    // the first four targets; or qubit 0 idle and one of 1..3 a target) keep 3xTF32 -- those paths have no
    // FP16 form, and the 16-bit paths move such tiles over partly used lines ----
    if (opts.precision == QSIM_PREC_FP16X3) {
        for (PlanOp& op : p->ops) {
            if (op.kind != OP_TC || op.k > 6) continue;  // 7-qubit blocks exist in FP16X3 only
            bool q0 = false, low = false;
            for (int j = 0; j < op.k; ++j) { q0 = q0 || op.targets[j] == 0; low = low || (op.targets[j] >= 1 && op.targets[j] <= 3); }
            // (a block with a phase epilogue has neither path: it runs on lanes on rows and stays FP16)
            if ((!remap_later && tc_line_groups(op.k, op.targets, QSIM_PREC_TF32X3, op.has_epi)) || (!q0 && low && !op.has_epi))
                op.precision = QSIM_PREC_TF32X3;
        }
    }
    // ---- pairs: two consecutive 6-qubit tensor-core blocks without epilogue whose tile fits take one pass ----
    if (pair_blocks && !remap_later && dtype == QSIM_C64) {
        for (size_t oi = 0; oi < p->ops.size(); ++oi) {
            PlanOp& a = p->ops[oi];
            if (a.kind != OP_TC || a.has_epi || a.k != 6 || a.nc != 0) continue;
            size_t oj = oi + 1;
            while (oj < p->ops.size() && p->ops[oj].kind == OP_MERGED) ++oj;
            if (oj >= p->ops.size()) break;
            PlanOp& b = p->ops[oj];
            if (b.kind != OP_TC || b.has_epi || b.k != 6 || b.nc != 0 || !tc_pair_supported(n, a.targets, 6, b.targets, 6))
                continue;
            a.kind = OP_TC_PAIR;
            std::memcpy(a.targets2, b.targets, sizeof(a.targets2));
            a.compose_idx2 = b.compose_idx;
            a.gates += b.gates;
            a.precision = QSIM_PREC_FP16X3;
            a.dev_off = dev_bytes;
            dev_bytes = align(dev_bytes + tc_pair_operand_bytes());
            b.kind = OP_MERGED;
            oi = oj;
        }
    }
    size_t epi_scratch = 0;
    for (PlanOp& op : p->ops) {
        if (op.kind != OP_TC || !op.has_epi) continue;
        tc_epi_pack(n, op.k, op.targets, op.form, op.blob, op.epi);
        op.epi_off = dev_bytes;
        dev_bytes = align(dev_bytes + op.blob.size());
        epi_scratch = std::max(epi_scratch, tc_epi_scratch_bytes(n, op.k));
    }
    p->extra.epi_scratch_off = dev_bytes;
    dev_bytes = align(dev_bytes + epi_scratch);

    p->dry = dry;
    if (!dry) {
    // ---- device buffer: [operands][compose out][pool][block descriptors][gate descriptors] -------------------
    const size_t off_out = dev_bytes;
    const size_t off_pool = align(off_out + sizeof(double) * 2 * (size_t)compose_out);
    const size_t off_cb = align(off_pool + sizeof(double) * pool.size());
    const size_t off_cg = align(off_cb + sizeof(ComposeBlock) * cblocks.size());
    // a small state whose passes are all CUDA-core dense blocks, diagonals or phase passes runs them in one
    // resident launch
    bool small = !opts.launch_per_pass && n <= kSmallMaxQubits && !(opts.local_qubits > 0 && opts.local_qubits < n) &&
                 !p->ops.empty();
    for (const PlanOp& op : p->ops)
        small = small && ((op.kind == OP_DENSE_SMALL && op.k <= 4) || (op.kind == OP_DENSE_TILE && op.k == 5) ||
                          (op.kind == OP_DIAG && op.k <= 6) || op.kind == OP_PHASE);
    const size_t off_small = align(off_cg + sizeof(ComposeGate) * cgates.size());
    const size_t total = off_small + (small ? align(small_program_bytes(dtype, (int)p->ops.size())) : 0) + 1024;
    e = plan_buffer_alloc(&p->dbuf, total, s, &p->pooled);
    if (e != cudaSuccess) { delete p; set_error("plan buffer of %zu bytes", total); return QSIM_ENOMEM; }
    p->dbuf_bytes = total;
    char* base = static_cast<char*>(p->dbuf);
    int rc = QSIM_OK;
    // phase tables first: the row phases of an epilogue go into its block's operand below
    for (size_t oi = 0; rc == QSIM_OK && oi < p->ops.size(); ++oi) {
        PlanOp& op = p->ops[oi];
        if (op.kind != OP_PHASE && !(op.kind == OP_TC && op.has_epi)) continue;
        e = cudaMemcpyAsync(base + (op.kind == OP_PHASE ? op.dev_off : op.epi_off), op.blob.data(), op.blob.size(),
                            cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // pageable host source
        if (e != cudaSuccess) rc = cuda_fail(e, "plan preparation");
        op.blob.clear();
        op.blob.shrink_to_fit();
    }
    if (rc == QSIM_OK && !cblocks.empty()) {
        e = cudaMemcpyAsync(base + off_pool, pool.data(), sizeof(double) * pool.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(base + off_cb, cblocks.data(), sizeof(ComposeBlock) * cblocks.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(base + off_cg, cgates.data(), sizeof(ComposeGate) * cgates.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // host vectors are pageable temporaries
        if (e == cudaSuccess)
            e = launch_compose(reinterpret_cast<ComposeBlock*>(base + off_cb), (int)cblocks.size(),
                               reinterpret_cast<ComposeGate*>(base + off_cg), reinterpret_cast<double*>(base + off_pool),
                               reinterpret_cast<double*>(base + off_out), max_kb, s);
        // device operands and host copies of small composed matrices
        // composed matrices the host keeps (CUDA-core dense blocks and diagonals: they travel as launch
        // parameters or into a resident program): fetched below, in one copy where they lie close together
        std::vector<std::pair<size_t, size_t>> fetch;  // (op index, offset in doubles from the compose output)
        size_t lo = (size_t)-1, hi = 0, need = 0;
        for (const Pending& pd : pending) {
            if (e != cudaSuccess) break;
            PlanOp& op = p->ops[pd.op];
            if (op.kind == OP_TC_PAIR || op.kind == OP_MERGED) continue;  // pairs are prepared below
            const double* U = reinterpret_cast<double*>(base + off_out) + 2 * cblocks[op.compose_idx].out_off;
            const int D = 1 << pd.kb;
            if (pd.kind == OP_TC) {
                // decided on the targets as they are now: a plan with global qubits remaps them later, so it
                // keeps the row-per-thread paths
                op.lines = !remap_later && tc_line_groups(pd.kb, op.targets, op.precision, op.has_epi);
                e = launch_tc_prepare(U, pd.kb, op.precision, op.lines, base + op.dev_off, s,
                                      op.has_epi ? reinterpret_cast<const double*>(base + op.epi_off + op.epi.off_rowphase)
                                                 : nullptr);
            } else if (pd.kind == OP_DENSE_TILE && !(small && pd.kb == 5)) {
                e = launch_convert_matrix(dtype, U, base + op.dev_off, 2 * (int64_t)D * D, s);
            } else {
                // a 5-qubit block of a resident plan: its device matrix (for pass-range launches) and its FP64
                // matrix on the host (for the resident program), like the smaller blocks
                if (pd.kind == OP_DENSE_TILE) e = launch_convert_matrix(dtype, U, base + op.dev_off, 2 * (int64_t)D * D, s);
                op.mat.resize(2 * (size_t)D * D);
                const size_t o = 2 * (size_t)cblocks[op.compose_idx].out_off;
                fetch.emplace_back((size_t)pd.op, o);
                lo = std::min(lo, o);
                hi = std::max(hi, o + op.mat.size());
                need += op.mat.size();
            }
        }
        std::vector<double> stage;
        const bool one_copy = fetch.size() > 1 && hi - lo <= 4 * need + 8192;
        if (e == cudaSuccess && one_copy) {
            stage.resize(hi - lo);
            e = cudaMemcpyAsync(stage.data(), reinterpret_cast<double*>(base + off_out) + lo, sizeof(double) * stage.size(),
                                cudaMemcpyDeviceToHost, s);
        }
        for (size_t f = 0; e == cudaSuccess && !one_copy && f < fetch.size(); ++f) {
            PlanOp& op = p->ops[fetch[f].first];
            e = cudaMemcpyAsync(op.mat.data(), reinterpret_cast<double*>(base + off_out) + fetch[f].second,
                                sizeof(double) * op.mat.size(), cudaMemcpyDeviceToHost, s);
        }
        for (PlanOp& op : p->ops) {
            if (e != cudaSuccess) break;
            if (op.kind != OP_TC_PAIR) continue;
            const double* U1 = reinterpret_cast<double*>(base + off_out) + 2 * cblocks[op.compose_idx].out_off;
            const double* U2 = reinterpret_cast<double*>(base + off_out) + 2 * cblocks[op.compose_idx2].out_off;
            e = launch_tc_pair_prepare(U1, U2, base + op.dev_off, s);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess && one_copy)
            for (const auto& fo : fetch) {
                PlanOp& op = p->ops[fo.first];
                std::memcpy(op.mat.data(), stage.data() + (fo.second - lo), sizeof(double) * op.mat.size());
            }
        if (e == cudaSuccess) {
            for (const Pending& pd : pending) {
                PlanOp& op = p->ops[pd.op];
                if (op.kind == OP_DIAG) {  // keep the diagonal only
                    const int D = 1 << op.k;
                    std::vector<double> dg(2 * D);
                    for (int i = 0; i < D; ++i) { dg[2 * i] = op.mat[2 * (i * D + i)]; dg[2 * i + 1] = op.mat[2 * (i * D + i) + 1]; }
                    op.mat.swap(dg);
                }
            }
        }
        if (e != cudaSuccess) rc = cuda_fail(e, "plan preparation");
    }
    for (size_t di = 0; rc == QSIM_OK && di < direct.size(); ++di) {
        PlanOp& op = p->ops[direct[di]];
        const size_t cnt = (size_t)2 << (2 * op.k);
        std::vector<float> f;
        if (dtype == QSIM_C64) {
            f.resize(cnt);
            for (size_t i = 0; i < cnt; ++i) f[i] = (float)op.mat[i];
            e = cudaMemcpyAsync(base + op.dev_off, f.data(), cnt * sizeof(float), cudaMemcpyHostToDevice, s);
        } else {
            e = cudaMemcpyAsync(base + op.dev_off, op.mat.data(), cnt * sizeof(double), cudaMemcpyHostToDevice, s);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // pageable host sources
        if (e != cudaSuccess) rc = cuda_fail(e, "plan preparation");
        op.mat.clear();
        op.mat.shrink_to_fit();
    }
    if (rc == QSIM_OK && small) {
        std::vector<SmallOpDesc> sd(p->ops.size());
        for (size_t i = 0; i < p->ops.size(); ++i) {
            const PlanOp& op = p->ops[i];
            sd[i].diag = op.kind == OP_DIAG;
            sd[i].k = op.k;
            sd[i].nc = op.nc;
            sd[i].targets = op.targets;
            sd[i].controls = op.controls;
            sd[i].mat = op.mat.data();
            sd[i].touch = &op.touch;
            if (op.kind == OP_PHASE) sd[i].form = &op.form;
        }
        std::vector<unsigned char> prog(small_program_bytes(dtype, (int)p->ops.size()));
        if (small_program_build(dtype, sd, prog.data())) {
            e = cudaMemcpyAsync(base + off_small, prog.data(), prog.size(), cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // pageable host source
            if (e != cudaSuccess) rc = cuda_fail(e, "plan preparation");
            p->small = true;
            p->small_off = off_small;
        }
    }
    if (rc) { cudaStreamSynchronize(s); plan_buffer_free(p->dbuf, p->pooled); delete p; return rc; }
    }  // !dry

    // ---- global / local index bits: reorder before passes that touch a global qubit ------------------------
    if (opts.local_qubits > 0 && opts.local_qubits < n) {
        const int L = opts.local_qubits;
        std::vector<int> phys(n), logi(n);  // logical -> physical position and back
        std::vector<int64_t> last(n, -1);   // last pass that used each physical position
        for (int q = 0; q < n; ++q) phys[q] = logi[q] = q;
        std::vector<PlanOp> out_ops;
        int64_t clock = 0;
        // passes of at most 4 pairs: the direct exchange kernel's limit (more pairs take the slower
        // shared-memory path, so two direct passes cost less than one of 5..8 pairs)
        auto emit_swaps = [&](const std::vector<std::pair<int, int>>& pairs) {
            for (size_t i = 0; i < pairs.size(); i += 4) {
                PlanOp sw;
                sw.kind = OP_SWAP;
                sw.gates = 0;
                for (size_t j = i; j < pairs.size() && j < i + 4; ++j) {
                    sw.swap_a[sw.nswap] = pairs[j].first;
                    sw.swap_b[sw.nswap] = pairs[j].second;
                    ++sw.nswap;
                }
                out_ops.push_back(std::move(sw));
            }
            for (const auto& pr : pairs) {  // positions pr.first and pr.second exchange their logical qubits
                const int la = logi[pr.first], lb = logi[pr.second];
                logi[pr.first] = lb; logi[pr.second] = la;
                phys[la] = pr.second; phys[lb] = pr.first;
            }
        };
        auto op_qubits = [](const PlanOp& op) {
            std::vector<int> qs(op.targets, op.targets + op.k);
            qs.insert(qs.end(), op.controls, op.controls + op.nc);
            return qs;
        };
        for (size_t i = 0; i < p->ops.size(); ++i) {
            PlanOp& op = p->ops[i];
            bool needs = false;
            for (int q : op_qubits(op)) needs |= phys[q] >= L;
            if (needs) {
                // Look ahead: bring in, in one exchange, every global qubit needed by passes i..j, as long as
                // those passes' qubits all fit among the local positions and at most 4 pairs are exchanged
                // (pass i alone may need up to 8).
                // Beyond pass i, also stop before the protected set leaves fewer idle local positions >= 4 than
                // qubits to bring in: an exchange with a position below 4 moves runs shorter than 128 bytes
                // and takes the slower shared-memory path.
                uint64_t bring = 0, protect = 0;
                for (size_t j = i; j < p->ops.size(); ++j) {
                    uint64_t qj = 0, gj = 0;
                    for (int q : op_qubits(p->ops[j])) { qj |= 1ull << q; if (phys[q] >= L) gj |= 1ull << q; }
                    const uint64_t nb = bring | gj, np = protect | qj;
                    if (__builtin_popcountll(nb) > (j > i ? 4 : 8) || __builtin_popcountll(np) > L) break;
                    if (j > i) {
                        int idle_hi = 0;
                        for (int pp = 4; pp < L; ++pp) idle_hi += !((np >> logi[pp]) & 1);
                        if (idle_hi < __builtin_popcountll(nb)) break;
                    }
                    bring = nb;
                    protect = np;
                }
                // victims: local positions holding unprotected qubits; least recently used first, positions >= 4
                // before lower ones (large contiguous runs keep the exchange kernel streaming)
                std::vector<int> cand;
                for (int pp = 0; pp < L; ++pp) if (!((protect >> logi[pp]) & 1)) cand.push_back(pp);
                std::stable_sort(cand.begin(), cand.end(), [&](int x, int y) {
                    const bool lx = x < 4, ly = y < 4;
                    if (lx != ly) return ly;
                    return last[x] < last[y];
                });
                std::vector<int> glob;
                for (int q = 0; q < n; ++q) if ((bring >> q) & 1) glob.push_back(phys[q]);
                if (cand.size() < glob.size()) {
                    plan_buffer_free(p->dbuf, p->pooled);
                    delete p;
                    set_error("local_qubits = %d leaves too few idle local qubits for a %d-qubit pass", L, (int)op_qubits(op).size());
                    return QSIM_EINVAL;
                }
                std::vector<std::pair<int, int>> pairs;
                for (size_t g = 0; g < glob.size(); ++g) pairs.push_back({cand[g], glob[g]});
                emit_swaps(pairs);
            }
            for (int j = 0; j < op.k; ++j) { op.targets[j] = phys[op.targets[j]]; last[op.targets[j]] = clock; }
            for (int j = 0; j < op.nc; ++j) { op.controls[j] = phys[op.controls[j]]; last[op.controls[j]] = clock; }
            ++clock;
            out_ops.push_back(std::move(op));
        }
        // Restore the identity order. The positions form cycles under "the logical qubit at position c belongs
        // at position logi[c]"; a cycle (c_0 .. c_{k-1}), c_{i+1} = logi[c_i], is the product of two
        // reflections: exchanging c_i with c_{-i}, then c_i with c_{1-i} (indices mod k), moves the content of
        // every c_i to c_{i+1}. So two sets of disjoint exchanges restore any order; each set is emitted as
        // passes of at most 4 pairs (the direct exchange kernel's limit).
        {
            std::vector<std::pair<int, int>> inv1, inv2;
            std::vector<char> seen(n, 0);
            for (int c = 0; c < n; ++c) {
                if (seen[c] || logi[c] == c) { seen[c] = 1; continue; }
                std::vector<int> cyc;
                for (int x = c; !seen[x]; x = logi[x]) { seen[x] = 1; cyc.push_back(x); }
                const int k = (int)cyc.size();
                for (int a = 0; a < k; ++a) {
                    const int b1 = (k - a) % k, b2 = (1 - a + k) % k;
                    if (a < b1) inv1.push_back({cyc[a], cyc[b1]});
                    if (a < b2) inv2.push_back({cyc[a], cyc[b2]});
                }
            }
            // check on a copy: both sets applied in order leave every position holding its own qubit
            std::vector<int> chk = logi;
            for (const auto* inv : {&inv1, &inv2})
                for (const auto& pr : *inv) std::swap(chk[pr.first], chk[pr.second]);
            for (int q = 0; q < n; ++q)
                if (chk[q] != q) {
                    plan_buffer_free(p->dbuf, p->pooled);
                    delete p;
                    set_error("internal error: qubit order restore");
                    return QSIM_EINVAL;
                }
            for (const auto* inv : {&inv1, &inv2})
                for (size_t a = 0; a < inv->size(); a += 4) {
                    PlanOp sw;
                    sw.kind = OP_SWAP;
                    sw.gates = 0;
                    for (size_t b = a; b < inv->size() && b < a + 4; ++b) {
                        sw.swap_a[sw.nswap] = (*inv)[b].first;
                        sw.swap_b[sw.nswap] = (*inv)[b].second;
                        ++sw.nswap;
                    }
                    out_ops.push_back(std::move(sw));
                }
        }
        p->ops.swap(out_ops);
    }

    // drop the phase passes that became epilogues
    p->ops.erase(std::remove_if(p->ops.begin(), p->ops.end(), [](const PlanOp& op) { return op.kind == OP_MERGED; }),
                 p->ops.end());

    // ---- statistics ---------------------------------------------------------------------------------------
    qsim_plan_info& I = p->info;
    I.input_gates = G;
    for (const PlanOp& op : p->ops) {
        ++I.passes;
        if (op.kind == OP_DIAG || op.kind == OP_PHASE) ++I.diag_blocks;
        else if (op.kind == OP_TC) ++I.tc_blocks;
        else if (op.kind == OP_TC_PAIR) I.tc_blocks += 2;
        else if (op.kind == OP_SWAP) ++I.reorders;
        else ++I.dense_blocks;
        I.algorithmic_bytes += op_bytes(op, n, amp);
    }
    I.resident = p->small ? 1 : 0;
    I.host_plan_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = I;
    *out = p;
    return QSIM_OK;
}

int qsim_plan_execute(qsim_h h, qsim_plan_h p) {
    if (!h || !p) { set_error("NULL argument"); return QSIM_EINVAL; }
    set_error("%s", "");
    if (p->dry) { set_error("plan was created as a dry run"); return QSIM_EINVAL; }
    if (h->n != p->n || h->dtype != p->dtype) { set_error("plan was made for another n or dtype"); return QSIM_EINVAL; }
    if (!p->use_graph || h->stream == nullptr || p->small) return enqueue_ops(h, p);  // a resident plan is one launch
    if (p->gexec && p->ghandle == h && p->gpsi == h->psi && p->gstream == h->stream) {
        cudaError_t e = cudaGraphLaunch(p->gexec, h->stream);
        return e == cudaSuccess ? QSIM_OK : cuda_fail(e, "graph launch");
    }
    if (p->gexec) { cudaGraphExecDestroy(p->gexec); p->gexec = nullptr; }
    cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return cuda_fail(e, "begin capture");
    int rc = enqueue_ops(h, p);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(h->stream, &g);
    if (rc) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    e = cudaGraphInstantiate(&p->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { p->gexec = nullptr; return cuda_fail(e, "graph instantiate"); }
    p->ghandle = h;
    p->gpsi = h->psi;
    p->gstream = h->stream;
    e = cudaGraphLaunch(p->gexec, h->stream);
    return e == cudaSuccess ? QSIM_OK : cuda_fail(e, "graph launch");
}

int qsim_plan_num_passes(qsim_plan_h p, int64_t* out) {
    if (!p || !out) { set_error("NULL argument"); return QSIM_EINVAL; }
    *out = (int64_t)p->ops.size();
    return QSIM_OK;
}

int qsim_plan_pass_info(qsim_plan_h p, int64_t i, qsim_pass_info* out) {
    if (!p || !out) { set_error("NULL argument"); return QSIM_EINVAL; }
    if (i < 0 || i >= (int64_t)p->ops.size()) { set_error("pass index out of range"); return QSIM_EINVAL; }
    const PlanOp& op = p->ops[i];
    out->kind = op.kind;
    out->k = op.k;
    out->nc = op.nc;
    out->precision = op.precision;
    out->gates = op.gates;
    out->algorithmic_bytes = op_bytes(op, p->n, p->dtype == QSIM_C64 ? 8 : 16);
    std::memset(out->targets, 0, sizeof(out->targets));
    std::memset(out->controls, 0, sizeof(out->controls));
    for (int j = 0; j < op.k && j < QSIM_MAX_TARGETS; ++j) out->targets[j] = op.targets[j];
    for (int j = 0; j < op.nc && j < QSIM_MAX_CONTROLS; ++j) out->controls[j] = op.controls[j];
    if (op.kind == OP_SWAP) {  // the exchanged index-bit pairs: targets[i] <-> controls[i]
        out->k = out->nc = op.nswap;
        for (int j = 0; j < op.nswap && j < QSIM_MAX_TARGETS; ++j) {
            out->targets[j] = op.swap_a[j];
            out->controls[j] = op.swap_b[j];
        }
    }
    if (op.kind == OP_TC_PAIR) {  // the second block's targets in controls[]
        out->kind = QSIM_PASS_TC_PAIR;
        out->nc = 6;
        for (int j = 0; j < 6; ++j) out->controls[j] = op.targets2[j];
    }
    out->launches = op.kind == OP_TC && op.has_epi ? 2 : 1;
    out->reserved = 0;
    return QSIM_OK;
}

int qsim_plan_execute_range(qsim_h h, qsim_plan_h p, int64_t first, int64_t count) {
    if (!h || !p) { set_error("NULL argument"); return QSIM_EINVAL; }
    set_error("%s", "");
    if (p->dry) { set_error("plan was created as a dry run"); return QSIM_EINVAL; }
    if (h->n != p->n || h->dtype != p->dtype) { set_error("plan was made for another n or dtype"); return QSIM_EINVAL; }
    if (first < 0 || count < 0 || first + count > (int64_t)p->ops.size()) { set_error("pass range out of bounds"); return QSIM_EINVAL; }
    return enqueue_ops(h, p, (size_t)first, (size_t)count);
}

int qsim_plan_execute_from_basis(qsim_h h, qsim_plan_h p, uint64_t x, int64_t count) {
    if (!h || !p) { set_error("NULL argument"); return QSIM_EINVAL; }
    set_error("%s", "");
    if (p->dry) { set_error("plan was created as a dry run"); return QSIM_EINVAL; }
    if (h->n != p->n || h->dtype != p->dtype) { set_error("plan was made for another n or dtype"); return QSIM_EINVAL; }
    if (h->n < 64 && (x >> h->n) != 0) { set_error("basis index out of range"); return QSIM_EINVAL; }
    const int64_t nops = (int64_t)p->ops.size();
    if (count < 0) count = nops;
    if (count > nops) { set_error("pass range out of bounds"); return QSIM_EINVAL; }
    // a first tensor-core block (any precision but BF16x6; block pairs and 7-qubit blocks too) generates |x>
    // as its input and writes every amplitude
    if (count > 0 && ((p->ops[0].kind == OP_TC && p->ops[0].precision != QSIM_PREC_BF16X6) || p->ops[0].kind == OP_TC_PAIR))
        return enqueue_ops(h, p, 0, (size_t)count, &x);
    // a resident plan sets |x> itself, in the same launch
    if (p->small && count == nops) return enqueue_ops(h, p, 0, (size_t)count, &x);
    const int rc = qsim_set_basis(h, x);
    if (rc) return rc;
    return enqueue_ops(h, p, 0, (size_t)count);
}

int qsim_plan_destroy(qsim_plan_h p) {
    if (!p) return QSIM_OK;
    if (p->dry) { delete p; return QSIM_OK; }
    cudaDeviceSynchronize();
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    plan_buffer_free(p->dbuf, p->pooled);
    delete p;
    return QSIM_OK;
}

int qsim_run(qsim_h h, const qsim_circuit* c, const qsim_run_opts* opts, qsim_plan_info* info) {
    if (!h || !c) { set_error("NULL argument"); return QSIM_EINVAL; }
    if (c->n != h->n) { set_error("circuit has %d qubits, state has %d", c->n, h->n); return QSIM_EINVAL; }
    qsim_run_opts o{};
    if (opts) o = *opts;
    o.use_graph = 0;
    qsim_plan_h p = nullptr;
    int rc = qsim_plan_create(c, h->dtype, &o, h->stream, &p, info);
    if (rc) return rc;
    rc = qsim_plan_execute(h, p);
    cudaStreamSynchronize(h->stream);
    qsim_plan_destroy(p);
    return rc;
}

}  // extern "C"
