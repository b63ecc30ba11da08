// Pieces shared by the residual-update kernels (Eq. (4): c_k, r_{k+1} and
// |r_{k+1}|^2 per channel, the selected atom's parameters): the energy as a
// float-pair sum and the parameter decode spread over four lanes.  Both keep
// the serial tail of an update off the FP64 pipe, which on this GPU runs at a
// small fraction of the FP32 rate.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "act_ff.cuh"
#include "act_internal.cuh"

namespace act {

// v^2 added to a float-pair sum: the square split exactly by an FMA
// (two-product), then an error-free pair addition.
__device__ __forceinline__ void ff_add_square(ff &s, float v) {
    const float p = v * v;
    s = ff_add(s, ff{p, fmaf(v, v, -p)});
}

// Sum of float pairs over the block in a fixed order (the same bits on
// every run); every thread receives the total.  sh must hold 32 pairs.
__device__ __forceinline__ ff block_sum_ff(ff v, ff *sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = ff_warp_sum(v);
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    if (wid == 0) {
        ff t = lane < nw ? sh[lane] : ff{0.0f, 0.0f};
        t = ff_warp_sum(t);
        if (lane == 0) sh[0] = t;
    }
    __syncthreads();
    const ff r = sh[0];
    __syncthreads();
    return r;
}

// Lane a < 4 of the calling warp writes parameter a (tc, fc, logDt, c) of
// atom `flat` into *out, lane 0 also its flat index: the same values as
// decode_params (lo + i * step, one rounding per operation), with the index
// unravelled in 32 bits (selection keys carry 32-bit indices).
__device__ __forceinline__ void write_atom_lanes(const GridAxes &ax, uint32_t flat, act_atom *out) {
    const int a = threadIdx.x & 31;
    if (a >= 4) return;
    const uint32_t c3 = (uint32_t)ax.count[3], c2 = (uint32_t)ax.count[2], c1 = (uint32_t)ax.count[1];
    const uint32_t ic = flat % c3, r1 = flat / c3, il = r1 % c2, r2 = r1 / c2, ifc = r2 % c1, itc = r2 / c1;
    const uint32_t i = a == 0 ? itc : (a == 1 ? ifc : (a == 2 ? il : ic));
    const double v = axis_value(ax.lo[a], ax.step[a], (int64_t)i);
    if (a == 0) {
        out->tc = v;
        out->flat_index = (int64_t)flat;
    } else if (a == 1) {
        out->fc = v;
    } else if (a == 2) {
        out->logdt = v;
    } else {
        out->c = v;
    }
}

}  // namespace act
