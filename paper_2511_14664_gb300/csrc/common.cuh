// common.cuh -- device-side building blocks shared by the libqsim kernels.
//
// Amplitudes are interleaved complex: float2 (complex64) or double2 (complex128). Qubit q is bit q of the
// amplitude index. Index spaces are 64-bit throughout (a 34-qubit state has 2^34 amplitudes).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace qsim {

// ---- amplitude types ------------------------------------------------------------------------------------
template <typename R> struct Amp;
template <> struct Amp<float> { using T = float2; };
template <> struct Amp<double> { using T = double2; };

template <typename R> __device__ __forceinline__ typename Amp<R>::T make_amp(R re, R im);
template <> __device__ __forceinline__ float2 make_amp<float>(float re, float im) { return make_float2(re, im); }
template <> __device__ __forceinline__ double2 make_amp<double>(double re, double im) { return make_double2(re, im); }

// ---- index helpers ----------------------------------------------------------------------------------------
// Insert a zero bit at position p: bits >= p move up by one.
__host__ __device__ __forceinline__ uint64_t insert_zero(uint64_t v, int p) {
    const uint64_t low = v & ((1ull << p) - 1);
    return ((v >> p) << (p + 1)) | low;
}

// Insert zero bits at the sorted (ascending) positions pos[0..nf).
__host__ __device__ __forceinline__ uint64_t insert_zeros(uint64_t v, const int* pos, int nf) {
    for (int i = 0; i < nf; ++i) v = insert_zero(v, pos[i]);
    return v;
}

// Scatter the low bits of v to the positions listed in pos[0..nb) (bit j of v -> bit pos[j]).
__host__ __device__ __forceinline__ uint64_t deposit(uint64_t v, const int* pos, int nb) {
    uint64_t r = 0;
    for (int j = 0; j < nb; ++j) r |= ((v >> j) & 1ull) << pos[j];
    return r;
}

// ---- launch geometry ---------------------------------------------------------------------------------------
struct Geometry {
    int num_sms;
};

// Grid size for a grid-stride kernel: `per_sm` resident CTAs on every SM, never more CTAs than work.
__host__ __forceinline__ unsigned grid_for(int64_t work_items, int threads, int num_sms, int per_sm) {
    int64_t need = (work_items + threads - 1) / threads;
    int64_t cap = (int64_t)num_sms * per_sm;
    if (need < 1) need = 1;
    return (unsigned)(need < cap ? need : cap);
}

// ---- float-float ("double-single") compensated arithmetic --------------------------------------------------
// GB300's FP64 rate is a small fraction of its FP32 rate, so the bulk of every reduction accumulates
// unevaluated sums hi + lo of two floats (Knuth's TwoSum, Dekker's exact product via FMA), which carry
// about 48 significant bits, and only block-level partials are combined in FP64.
struct ff {
    float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ ff ff_renorm(float s, float e) {
    float hi = __fadd_rn(s, e);
    float lo = __fsub_rn(e, __fsub_rn(hi, s));
    return {hi, lo};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    return ff_renorm(s, e);
}

__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }

// Exact x*y as hi + lo.
__device__ __forceinline__ ff two_prod(float x, float y) {
    float p = __fmul_rn(x, y);
    float e = __fmaf_rn(x, y, -p);
    return {p, e};
}

// |z|^2 = re^2 + im^2 as a float-float (exact products, compensated sum).
__device__ __forceinline__ ff ff_abs2(float re, float im) { return ff_add(two_prod(re, re), two_prod(im, im)); }

__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

// ---- double-double (FP64 TwoSum) for block partials ---------------------------------------------------------
struct dd {
    double hi, lo;
};

__device__ __forceinline__ dd dd_add(dd a, dd b) {
    double s = __dadd_rn(a.hi, b.hi);
    double bb = __dsub_rn(s, a.hi);
    double e = __dadd_rn(__dsub_rn(a.hi, __dsub_rn(s, bb)), __dsub_rn(b.hi, bb));
    e = __dadd_rn(e, __dadd_rn(a.lo, b.lo));
    double hi = __dadd_rn(s, e);
    return {hi, __dsub_rn(e, __dsub_rn(hi, s))};
}

__device__ __forceinline__ ff shfl_xor_ff(ff v, int m) {
    return {__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m)};
}

__device__ __forceinline__ dd shfl_xor_dd(dd v, int m) {
    return {__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m)};
}

__device__ __forceinline__ ff warp_sum_ff(ff v) {
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) v = ff_add(v, shfl_xor_ff(v, m));
    return v;
}

__device__ __forceinline__ dd warp_sum_dd(dd v) {
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) v = dd_add(v, shfl_xor_dd(v, m));
    return v;
}

// ---- phases as 64-bit fixed-point turns ----------------------------------------------------------------------
// A phase stored as x / 2^64 turns adds with wraparound (mod 2 pi, exact). unit_phase returns exp(2 pi i x/2^64).
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

// ---- device error word -------------------------------------------------------------------------------------
// Kernels with bounded waits report expiry by OR-ing a code into a device word the host reads back.
enum : unsigned { DEVERR_TIMEOUT = 1u, DEVERR_BAD_ITEM = 2u, DEVERR_TMEM = 4u };

}  // namespace qsim
