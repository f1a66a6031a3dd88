/*
 * oracle.c -- plain FP64 (complex128) state-vector simulator used as the correctness oracle.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library links, loads or calls this file; only the
 * test-suite, the smoke check and the benchmark's CPU-baseline leg use it. It shares no code, header
 * or table with the GPU path.
 *
 * Every routine is the plain definition of the quantity it computes, written for a reader to check by
 * eye against the paper (arXiv 2511.14664):
 *   - a state of n qubits is a vector of 2^n complex amplitudes (Sec. 2.1 "State-Vector Simulation");
 *   - a gate is the operator I (x) ... (x) U (x) ... (x) I applied to that vector (same passage), and a
 *     controlled gate acts only on the subspace where every control qubit is |1>;
 *   - measurement draws bitstrings with probability |amplitude|^2 (Sec. 2.1 "Measurement and Sampling");
 *   - expectation values <psi|P|psi> of Pauli strings (Sec. 2.5, sampling and expectation values).
 * Index convention: qubit q is bit q of the amplitude index; for targets (t_0..t_{k-1}) the matrix
 * row/column index is m = sum_j bit_{t_j} 2^j; matrices are row-major.
 *
 * The per-gate loop may run its independent groups on several threads (OpenMP); that changes no
 * arithmetic. All sums are serial, compensated (Neumaier) and in natural index order.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define ORACLE_KMAX 10

/* ---- helpers -------------------------------------------------------------------------------------- */

static int check_qubits(int n, int k, const int* targets, int nc, const int* controls) {
    if (n < 1 || n > 40 || k < 1 || k > ORACLE_KMAX || nc < 0 || k + nc > n) return -1;
    uint64_t seen = 0;
    for (int j = 0; j < k; ++j) {
        if (targets[j] < 0 || targets[j] >= n || (seen >> targets[j] & 1)) return -1;
        seen |= 1ull << targets[j];
    }
    for (int j = 0; j < nc; ++j) {
        if (controls[j] < 0 || controls[j] >= n || (seen >> controls[j] & 1)) return -1;
        seen |= 1ull << controls[j];
    }
    return 0;
}

/* Insert a zero bit at position p (all higher bits shift up by one). */
static inline uint64_t insert_zero(uint64_t v, int p) {
    uint64_t low = v & ((1ull << p) - 1);
    return ((v >> p) << (p + 1)) | low;
}

static int cmp_int(const void* a, const void* b) { return (*(const int*)a) - (*(const int*)b); }

/* Neumaier's improved Kahan summation: running sum s with compensation c. */
typedef struct { double s, c; } nsum;
static inline void nsum_add(nsum* a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}
static inline double nsum_get(const nsum* a) { return a->s + a->c; }

/* ---- gate application ---------------------------------------------------------------------------- */

/*
 * psi <- G psi, G = U on `targets` (in the given order), restricted to control bits all 1.
 * For every base index b of the 2^(n-k-nc) groups: insert zeros at all target and control positions,
 * set the control bits, gather v[m] = psi[b | sum_j bit_j(m) << t_j], compute w = U v, scatter w.
 * Returns 0, or -1 on invalid arguments (nothing applied).
 */
int oracle_apply_gate(int n, cplx* psi, int k, const int* targets, int nc, const int* controls,
                      const cplx* U) {
    if (!psi || !targets || !U || (nc > 0 && !controls)) return -1;
    if (check_qubits(n, k, targets, nc, controls)) return -1;
    int fixed[64];
    int nf = 0;
    uint64_t cmask = 0;
    for (int j = 0; j < k; ++j) fixed[nf++] = targets[j];
    for (int j = 0; j < nc; ++j) { fixed[nf++] = controls[j]; cmask |= 1ull << controls[j]; }
    qsort(fixed, (size_t)nf, sizeof(int), cmp_int);
    const int64_t ngroups = (int64_t)1 << (n - nf);
    const int dim = 1 << k;

    #pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < ngroups; ++g) {
        uint64_t base = (uint64_t)g;
        for (int i = 0; i < nf; ++i) base = insert_zero(base, fixed[i]);
        base |= cmask;
        uint64_t idx[1 << ORACLE_KMAX];
        cplx v[1 << ORACLE_KMAX];
        for (int m = 0; m < dim; ++m) {
            uint64_t off = 0;
            for (int j = 0; j < k; ++j) off |= (uint64_t)((m >> j) & 1) << targets[j];
            idx[m] = base | off;
            v[m] = psi[idx[m]];
        }
        for (int r = 0; r < dim; ++r) {
            cplx w = 0;
            for (int c = 0; c < dim; ++c) w += U[(size_t)r * dim + c] * v[c];
            psi[idx[r]] = w;
        }
    }
    return 0;
}

/*
 * Dense brute force (independent of oracle_apply_gate): build the full 2^n x 2^n operator of one gate
 * by explicit index mapping, G[y][x] = U[m(y)][m(x)] when x and y agree off the targets and all
 * controls of x are 1; G[x][x] = 1 when a control of x is 0; 0 otherwise. n <= 10.
 */
int oracle_dense_operator(int n, int k, const int* targets, int nc, const int* controls, const cplx* U,
                          cplx* G) {
    if (n > 10 || check_qubits(n, k, targets, nc, controls)) return -1;
    const uint64_t N = 1ull << n;
    uint64_t tmask = 0, cmask = 0;
    for (int j = 0; j < k; ++j) tmask |= 1ull << targets[j];
    for (int j = 0; j < nc; ++j) cmask |= 1ull << controls[j];
    const int dim = 1 << k;
    for (uint64_t y = 0; y < N; ++y)
        for (uint64_t x = 0; x < N; ++x) {
            cplx val = 0;
            if ((x & cmask) != cmask) {
                val = (x == y) ? 1.0 : 0.0;
            } else if ((x & ~tmask) == (y & ~tmask)) {
                int mx = 0, my = 0;
                for (int j = 0; j < k; ++j) {
                    mx |= (int)((x >> targets[j]) & 1) << j;
                    my |= (int)((y >> targets[j]) & 1) << j;
                }
                val = U[(size_t)my * dim + mx];
            }
            G[y * N + x] = val;
        }
    return 0;
}

/* psi <- G psi for a dense 2^n x 2^n operator (plain matrix-vector product). */
int oracle_dense_matvec(int n, const cplx* G, cplx* psi) {
    if (n > 12) return -1;
    const uint64_t N = 1ull << n;
    cplx* out = (cplx*)malloc(sizeof(cplx) * N);
    if (!out) return -1;
    for (uint64_t y = 0; y < N; ++y) {
        cplx s = 0;
        for (uint64_t x = 0; x < N; ++x) s += G[y * N + x] * psi[x];
        out[y] = s;
    }
    memcpy(psi, out, sizeof(cplx) * N);
    free(out);
    return 0;
}

/* ---- observables ----------------------------------------------------------------------------------- */

/* sum_x |psi_x|^2 (compensated). */
double oracle_norm2(int n, const cplx* psi) {
    nsum a = {0, 0};
    const uint64_t N = 1ull << n;
    for (uint64_t x = 0; x < N; ++x) {
        double re = creal(psi[x]), im = cimag(psi[x]);
        nsum_add(&a, re * re + im * im);
    }
    return nsum_get(&a);
}

/*
 * Marginal probabilities over `qubits` (nq <= 20): out[m] = sum over x with bit_{q_j}(x) = bit_j(m)
 * of |psi_x|^2, each bucket summed in natural order with compensation.
 */
int oracle_probs(int n, const cplx* psi, int nq, const int* qubits, double* out) {
    if (nq < 0 || nq > 20 || nq > n) return -1;
    for (int j = 0; j < nq; ++j) if (qubits[j] < 0 || qubits[j] >= n) return -1;
    const uint64_t M = 1ull << nq, N = 1ull << n;
    nsum* acc = (nsum*)calloc(M, sizeof(nsum));
    if (!acc) return -1;
    for (uint64_t x = 0; x < N; ++x) {
        uint64_t m = 0;
        for (int j = 0; j < nq; ++j) m |= ((x >> qubits[j]) & 1) << j;
        double re = creal(psi[x]), im = cimag(psi[x]);
        nsum_add(&acc[m], re * re + im * im);
    }
    for (uint64_t m = 0; m < M; ++m) out[m] = nsum_get(&acc[m]);
    free(acc);
    return 0;
}

/*
 * <psi| P |psi> for the Pauli string `paulis` (character q acts on qubit q; one of I, X, Y, Z).
 * P|x> = c(x) |x xor f>, with f the X/Y flip mask and c(x) the product over qubits of
 *   X: 1,  Y: +i if x_q = 0 else -i,  Z: +1 if x_q = 0 else -1.
 * Hence <psi|P|psi> = sum_x conj(psi_{x xor f}) c(x) psi_x. Real and imaginary parts are summed with
 * compensation; out[0] = real part, out[1] = imaginary part (zero for a Hermitian P up to rounding).
 */
int oracle_expect_pauli(int n, const cplx* psi, const char* paulis, double* out) {
    uint64_t f = 0;
    for (int q = 0; q < n; ++q) {
        char p = paulis[q];
        if (p != 'I' && p != 'X' && p != 'Y' && p != 'Z') return -1;
        if (p == 'X' || p == 'Y') f |= 1ull << q;
    }
    nsum re = {0, 0}, im = {0, 0};
    const uint64_t N = 1ull << n;
    for (uint64_t x = 0; x < N; ++x) {
        cplx c = 1.0;
        for (int q = 0; q < n; ++q) {
            int b = (int)((x >> q) & 1);
            if (paulis[q] == 'Y') c *= b ? -I : I;
            else if (paulis[q] == 'Z' && b) c = -c;
        }
        cplx t = conj(psi[x ^ f]) * c * psi[x];
        nsum_add(&re, creal(t));
        nsum_add(&im, cimag(t));
    }
    out[0] = nsum_get(&re);
    out[1] = nsum_get(&im);
    return 0;
}

/* <psi_a|psi_b> (compensated); out[0] = real, out[1] = imaginary. */
void oracle_inner(int n, const cplx* a, const cplx* b, double* out) {
    nsum re = {0, 0}, im = {0, 0};
    const uint64_t N = 1ull << n;
    for (uint64_t x = 0; x < N; ++x) {
        cplx t = conj(a[x]) * b[x];
        nsum_add(&re, creal(t));
        nsum_add(&im, cimag(t));
    }
    out[0] = nsum_get(&re);
    out[1] = nsum_get(&im);
}

/* ---- sampling -------------------------------------------------------------------------------------- */

/*
 * SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): the state advances by the golden-ratio increment
 * 0x9E3779B97F4A7C15 and each output is the state passed through the published 64-bit finaliser.
 * The i-th output of a generator seeded with `seed` is therefore mix(seed + (i + 1) * increment), which
 * makes the stream counter-addressable. A uniform in [0, 1) takes the top 53 bits.
 */
uint64_t oracle_splitmix64(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

void oracle_uniforms(uint64_t seed, int64_t count, double* out) {
    for (int64_t i = 0; i < count; ++i)
        out[i] = (double)(oracle_splitmix64(seed, (uint64_t)i) >> 11) * 0x1.0p-53;
}

/*
 * Inverse-CDF sampling (Sec. 2.1 "Measurement and Sampling"): with C(x) the inclusive prefix sum of
 * |psi_x|^2 in natural order and T = C(2^n - 1), each uniform u in [0, 1) yields
 * x = min{ x : C(x) > u T }. If rounding leaves no such x, the last x with nonzero probability is used.
 * The prefix sum is compensated. Returns 0 or -1.
 */
int oracle_sample(int n, const cplx* psi, int64_t shots, const double* uniforms, uint64_t* out) {
    if (n > 30) return -1;
    const uint64_t N = 1ull << n;
    double* cdf = (double*)malloc(sizeof(double) * N);
    if (!cdf) return -1;
    nsum a = {0, 0};
    uint64_t last_nz = 0;
    for (uint64_t x = 0; x < N; ++x) {
        double re = creal(psi[x]), im = cimag(psi[x]);
        double p = re * re + im * im;
        if (p > 0) last_nz = x;
        nsum_add(&a, p);
        cdf[x] = nsum_get(&a);
    }
    const double total = cdf[N - 1];
    for (int64_t s = 0; s < shots; ++s) {
        const double target = uniforms[s] * total;
        uint64_t lo = 0, hi = N; /* first x in [lo, hi) with cdf[x] > target */
        while (lo < hi) {
            uint64_t mid = lo + (hi - lo) / 2;
            if (cdf[mid] > target) hi = mid;
            else lo = mid + 1;
        }
        out[s] = (lo < N) ? lo : last_nz;
    }
    free(cdf);
    return 0;
}

/* Number of threads the per-gate loop uses (1 without OpenMP). */
int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_num_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}
