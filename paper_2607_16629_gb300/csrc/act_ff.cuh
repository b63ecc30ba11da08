// Float-float ("double-float") arithmetic on the FP32 pipes: a value is the
// unevaluated sum hi + lo of two floats with |lo| <= ulp(hi) / 2, about 48
// significant bits.  Built from the error-free transformations
//   two_sum (Knuth, TAOCP Vol. 2, Sec. 4.2.2): a + b = s + e exactly;
//   fast_two_sum (Dekker, 1971), valid when |a| >= |b| or a == 0;
//   two_prod with a fused multiply-add: a b = p + e exactly, e = fma(a, b, -p).
// The chirplet phase needs more than FP32's 24 bits before its reduction
// mod 1 (it runs to hundreds of cycles), and the sums of a projection want
// more than FP32's accumulation; GB300 runs FP64 at a small fraction of its
// FP32 rate, so these kernels carry both in float-float instead.  Nothing
// here may be compiled with reassociating (fast-math) flags.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace act {

struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {
    const float s = a + b;
    return {s, b - (s - a)};
}

// The float pair nearest a double (hi = round(x), lo = round(x - hi)).
__device__ __forceinline__ ff ff_from_double(double x) {
    const float hi = (float)x;
    return {hi, (float)(x - (double)hi)};
}

__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ ff ff_add(ff a, ff b) {
    const ff s = ff_two_sum(a.hi, b.hi);
    const ff t = ff_two_sum(a.lo, b.lo);
    ff r = ff_fast_two_sum(s.hi, s.lo + t.hi);
    return ff_fast_two_sum(r.hi, r.lo + t.lo);
}

// a + b with one error-free sum of the high parts and the low parts added
// (error about 2^-47 (|a| + |b|); inputs need not be normalised).
__device__ __forceinline__ ff ff_add_sloppy(ff a, ff b) {
    const ff s = ff_two_sum(a.hi, b.hi);
    return ff_fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}

// a mod 1 to about [-1/2, 1/2]: hi - rint(hi) is exact; the pair is left
// unnormalised.
__device__ __forceinline__ ff ff_frac(ff a) { return {a.hi - rintf(a.hi), a.lo}; }

// a + b for a float b.
__device__ __forceinline__ ff ff_add_f(ff a, float b) {
    const ff s = ff_two_sum(a.hi, b);
    return ff_fast_two_sum(s.hi, s.lo + a.lo);
}

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return ff_fast_two_sum(p, e);
}

// Accumulator s += a * b with the product carried exactly (two_prod) and
// the sum in float-float; the low parts are gathered in s.lo.
__device__ __forceinline__ void ff_fma_acc(ff &s, float a, float b) {
    const float p = a * b;
    const float pe = fmaf(a, b, -p);
    const ff t = ff_two_sum(s.hi, p);
    s = ff_fast_two_sum(t.hi, t.lo + (s.lo + pe));
}

__device__ __forceinline__ ff ff_shfl_xor(ff v, int off) {
    return {__shfl_xor_sync(0xffffffffu, v.hi, off), __shfl_xor_sync(0xffffffffu, v.lo, off)};
}

__device__ __forceinline__ ff ff_warp_sum(ff v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = ff_add(v, ff_shfl_xor(v, off));
    return v;
}

// Per-atom constants of the chirplet sample (Eq. (1)): tc, 1 / fs, fc and
// the chirp rate c as float pairs, 1 / dt as a float pair for the envelope.
struct ChirpFF {
    ff tc, inv_fs, fc, c, inv_dt;
};

__device__ __forceinline__ ChirpFF chirp_ff(double tc, double inv_fs, double fc, double c, double inv_dt) {
    return {ff_from_double(tc), ff_from_double(inv_fs), ff_from_double(fc), ff_from_double(c),
            ff_from_double(inv_dt)};
}

// tau = d / fs for the sample offset d = n - tc (a float pair) and the phase
// (c tau + fc) tau reduced mod 1 (to about [-1/2, 1/2]) as an unnormalised
// pair.
__device__ __forceinline__ ff chirp_phase_of_offset(ff d, const ChirpFF &k, ff *tau_out) {
    const ff tau = ff_mul(d, k.inv_fs);
    *tau_out = tau;
    return ff_frac(ff_mul(ff_add(ff_mul(k.c, tau), k.fc), tau));
}

// The offset d = n - tc of sample n (exact while |n - tc| stays below 2^24
// and tc is a float pair), then its phase as above.  On a grid of
// whole-sample time centres d is the integer m = n - tc with a zero low
// part, so a template generated from m has the same bits.
__device__ __forceinline__ ff chirp_offset(int n, const ChirpFF &k) {
    const ff d = ff_two_sum((float)n, -k.tc.hi);
    return ff_fast_two_sum(d.hi, d.lo - k.tc.lo);
}

__device__ __forceinline__ ff chirp_phase_pair(int n, const ChirpFF &k, ff *tau_out) {
    return chirp_phase_of_offset(chirp_offset(n, k), k, tau_out);
}

// The same phase rounded once to FP32.
__device__ __forceinline__ float chirp_phase_ff(int n, const ChirpFF &k, ff *tau_out) {
    const ff p = chirp_phase_pair(n, k, tau_out);
    return p.hi + p.lo;
}

// The envelope argument x = tau / dt, rounded once to FP32.
__device__ __forceinline__ float chirp_x_ff(ff tau, const ChirpFF &k) {
    return fmaf(tau.hi, k.inv_dt.hi, fmaf(tau.hi, k.inv_dt.lo, tau.lo * k.inv_dt.hi));
}

// The unnormalised sample of Eq. (1) at offset d = n - tc with constants k:
// exp(-x^2 / 2) cos(2 pi phase) in FP32.  The dictionary and template
// generators both form their samples here.
__device__ __forceinline__ float chirp_sample_offset(ff d, const ChirpFF &k) {
    ff tau;
    const ff p = chirp_phase_of_offset(d, k, &tau);
    const float x = chirp_x_ff(tau, k);
    return expf(-0.5f * x * x) * cospif(2.0f * (p.hi + p.lo));
}

// Sample n of the chirplet with constants k (not normalised).
__device__ __forceinline__ float chirp_sample_ff(int n, const ChirpFF &k) {
    return chirp_sample_offset(chirp_offset(n, k), k);
}

// The constants of one warp lane's ChirpFF broadcast from lane src.
__device__ __forceinline__ ff ff_shfl(ff v, int src) {
    return {__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src)};
}

__device__ __forceinline__ ChirpFF chirp_ff_shfl(const ChirpFF &v, int src) {
    return {ff_shfl(v.tc, src), ff_shfl(v.inv_fs, src), ff_shfl(v.fc, src), ff_shfl(v.c, src),
            ff_shfl(v.inv_dt, src)};
}

}  // namespace act
