// k_compose.cu -- FP64 composition of fused gate blocks (paper Sec. 2.1: gate fusion groups several gate
// applications into one larger matrix).
//
// For a block on kb local qubits with gates G_1..G_g (each on a subset of those qubits, with controls),
// U = G_g ... G_1 is built column by column: start from the identity and apply every gate to all 2^kb
// columns at once, exactly like applying it to 2^kb small state vectors. The columns evolve independently,
// so a block's columns may be spread over several CTAs (grid y): each CTA holds W of them and ping-pongs
// them between two shared-memory buffers (W = 2^kb up to kb = 6, 2 x 64 KiB; W = 32 for kb = 7, 2 x 64 KiB).
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace qsim {

__global__ void __launch_bounds__(256) k_compose(const ComposeBlock* __restrict__ blocks,
                                                 const ComposeGate* __restrict__ gates,
                                                 const double* __restrict__ pool, double* __restrict__ out,
                                                 int cols_max) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const ComposeBlock b = blocks[blockIdx.x];
    const int D = 1 << b.kb, W = D < cols_max ? D : cols_max, E = D * W;
    const int c_lo = (int)blockIdx.y * W;  // this CTA's columns c_lo .. c_lo + W - 1, stored [row][column]
    if (c_lo >= D) return;
    double2* A = reinterpret_cast<double2*>(smem_raw);
    double2* B = A + E;
    for (int i = threadIdx.x; i < E; i += blockDim.x) A[i] = make_double2((i / W) == c_lo + (i % W) ? 1.0 : 0.0, 0.0);
    __syncthreads();
    for (int gi = 0; gi < b.num_gates; ++gi) {
        const ComposeGate g = gates[b.first_gate + gi];
        const double* G = pool + 2 * g.mat_off;
        const int dg = 1 << g.k;
        int tmask = 0, cmask = 0;
        for (int j = 0; j < g.k; ++j) tmask |= 1 << g.targets[j];
        for (int j = 0; j < g.nc; ++j) cmask |= 1 << g.controls[j];
        for (int i = threadIdx.x; i < E; i += blockDim.x) {
            const int r = i / W, c = i % W;
            if ((r & cmask) != cmask) {
                B[i] = A[i];
                continue;
            }
            int mr = 0;
            for (int j = 0; j < g.k; ++j) mr |= ((r >> g.targets[j]) & 1) << j;
            const int base = r & ~tmask;
            double re = 0.0, im = 0.0;
            for (int m = 0; m < dg; ++m) {
                int src = base;
                for (int j = 0; j < g.k; ++j) src |= ((m >> j) & 1) << g.targets[j];
                const double gr = G[2 * (mr * dg + m)], gim = G[2 * (mr * dg + m) + 1];
                const double2 a = A[src * W + c];
                re = __fma_rn(gr, a.x, re);
                re = __fma_rn(-gim, a.y, re);
                im = __fma_rn(gr, a.y, im);
                im = __fma_rn(gim, a.x, im);
            }
            B[i] = make_double2(re, im);
        }
        __syncthreads();
        double2* t = A; A = B; B = t;
    }
    double2* o = reinterpret_cast<double2*>(out) + b.out_off;
    for (int i = threadIdx.x; i < E; i += blockDim.x) o[(i / W) * D + c_lo + i % W] = A[i];
}

cudaError_t launch_compose(const ComposeBlock* dblocks, int nblocks, const ComposeGate* dgates,
                           const double* dpool, double* dout, int max_kb, cudaStream_t s) {
    if (nblocks == 0) return cudaSuccess;
    if (max_kb < 1 || max_kb > 7) return cudaErrorInvalidValue;
    const int Dm = 1 << max_kb, cols_max = max_kb <= 6 ? Dm : 32;
    const size_t smem = 2 * sizeof(double2) * (size_t)Dm * (size_t)cols_max;
    cudaError_t e = smem_optin(reinterpret_cast<const void*>(k_compose), (int)smem);
    if (e != cudaSuccess) return e;
    k_compose<<<dim3((unsigned)nblocks, (unsigned)(Dm / cols_max), 1), 256, smem, s>>>(dblocks, dgates, dpool, dout,
                                                                                   cols_max);
    return cudaGetLastError();
}

}  // namespace qsim
