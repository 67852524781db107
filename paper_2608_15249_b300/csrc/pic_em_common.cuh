// pic_em_common.cuh -- device helpers shared by the electromagnetic step's 2D
// (pic_em.cu) and 3D (pic_em3.cu) kernels: the fixed-point current scale and its
// rounding, staggered-lattice weights, the Boris push with gathered fields, the
// one-cell move with its Esirkepov shape factors, block diagnostics.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "pic_internal.cuh"

namespace apk {

constexpr int EM_THREADS = 256;
// Fixed point of the current: the Jx, Jy weights (|w| <= 1) at 2^22, rounded with the
// FMA magic number (exact for |w 2^22| <= 2^22, no float-to-int conversion, which
// would issue on the slow FP64 pipe); the Jz weights (weight times vz, unbounded) at
// the same scale, by the magic number below 2^22 and a rounding conversion above
// (both round to nearest, ties to even, so the two agree).
constexpr float J_SCALE = 4194304.0f;      // 2^22
constexpr float RND_MAGIC_F = 12582912.0f; // 1.5 * 2^23
constexpr int RND_MAGIC_I = 0x4B400000;

__device__ __forceinline__ int wrapi(int i, int n)
{
    return i < 0 ? i + n : (i >= n ? i - n : i);
}

// Weights of a staggered CIC lattice along one axis: the particle at c + f sees the
// lattice points (c + s) with s = 0 or 1/2; returns the lower lattice index and the
// fraction towards the upper one.
__device__ __forceinline__ void stagger(int c, float f, bool half, int n, int *i0, float *fr)
{
    if (!half) {
        *i0 = c;
        *fr = f;
    } else if (f >= 0.5f) {
        *i0 = c;
        *fr = f - 0.5f;
    } else {
        *i0 = wrapi(c - 1, n);
        *fr = f + 0.5f;
    }
}

// |v| <= 1: round(v 2^22) by the FMA magic number
__device__ __forceinline__ void add_fx_unit(unsigned long long *acc, float v)
{
    const int q = __float_as_int(fmaf(v, J_SCALE, RND_MAGIC_F)) - RND_MAGIC_I;
    if (q) atomicAdd(acc, (unsigned long long)(long long)q);
}

__device__ __forceinline__ void add_fx(unsigned long long *acc, float v)
{
    const float y = v * J_SCALE;  // exact (a power-of-two scale)
    const long long q = fabsf(y) < J_SCALE ? (long long)(__float_as_int(y + RND_MAGIC_F) - RND_MAGIC_I)
                                           : __float2ll_rn(y);
    if (q) atomicAdd(acc, (unsigned long long)q);
}

// Boris with the gathered fields: t = (q/m) B h / 2, s = 2 t / (1 + t^2).
__device__ __forceinline__ void em_boris(const float *v, const float *e, const float *b,
                                         const GridParams &g, float *vn)
{
    float t[3], s[3], vm[3];
    float tt = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        t[a] = g.qmh2 * b[a];
        tt += t[a] * t[a];
    }
    const float s_over_t = 2.0f / (1.0f + tt);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        s[a] = t[a] * s_over_t;
        vm[a] = v[a] + g.qmh2 * e[a];
    }
    const float w0 = vm[0] + (vm[1] * t[2] - vm[2] * t[1]);
    const float w1 = vm[1] + (vm[2] * t[0] - vm[0] * t[2]);
    const float w2 = vm[2] + (vm[0] * t[1] - vm[1] * t[0]);
    vn[0] = vm[0] + (w1 * s[2] - w2 * s[1]) + g.qmh2 * e[0];
    vn[1] = vm[1] + (w2 * s[0] - w0 * s[2]) + g.qmh2 * e[1];
    vn[2] = vm[2] + (w0 * s[1] - w1 * s[0]) + g.qmh2 * e[2];
}

// The move along one axis, at most one cell (the current stencil below assumes it):
// o = f + v dt / dx; returns false for a longer move.  sh is the cell shift, fr the
// new offset.  The old and new CIC supports (nodes c, c + 1 and c + sh, c + sh + 1)
// lie in the three lattice nodes from c + m, m = min(sh, 0); S0 and DS are the
// Esirkepov shape factors there: S0 at the old position, DS the change to the new.
__device__ __forceinline__ bool em_move_axis(float f, float vdtdx, int *sh, int *m, float *fr,
                                             float *S0, float *DS)
{
    const float o = f + vdtdx;
    bool ok = o > -1.0f && o < 2.0f;
    const bool hi = o >= 1.0f, lo = o < 0.0f;
    float r = hi ? o - 1.0f : (lo ? o + 1.0f : o);
    int s = hi ? 1 : (lo ? -1 : 0);
    if (r >= 1.0f) {  // o a tiny negative number: its fraction rounded up to 1
        r = 0.0f;
        s += 1;
    }
    *sh = s;
    *fr = r;
    const int mm = s < 0 ? -1 : 0;
    *m = mm;
    // Relative to node c + m the old position is f - m and the new one fr + sh - m,
    // both in [0, 2): the CIC weights (1 - x, x) sit on nodes 0, 1 when the position
    // is below 1, else on nodes 1, 2.
    const bool old_low = mm == 0, new_low = s == mm;
    const float g0 = 1.0f - f, g1 = 1.0f - r;
    S0[0] = old_low ? g0 : 0.0f;
    S0[1] = old_low ? f : g0;
    S0[2] = old_low ? 0.0f : f;
    DS[0] = (new_low ? g1 : 0.0f) - S0[0];
    DS[1] = (new_low ? r : g1) - S0[1];
    DS[2] = (new_low ? 0.0f : r) - S0[2];
    return ok;
}

// The current of the Ampere update, read from its fixed-point accumulator: component
// k at node id is f[k] times the accumulated weights (as FP32, no conversion
// instruction), plus the prescribed current when there is one.  The E update reads
// the three components of a node first and clears them (clear_j) after its own
// stores, so that no field load waits behind a store to the accumulator.
struct JTake {
    unsigned long long *acc;  // [3][cells]
    const float *ext;         // [3][cells] or null
    float f[3];
};

// The current of a step: the accumulator, the prescribed current, the factors.
JTake em_jtake(const EmBufs &em, double fx, double fy, double fz);

__device__ __forceinline__ void get_j(const JTake &t, int64_t cells, int64_t id, float *j)
{
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int64_t a = k * cells + id;
        j[k] = t.f[k] * i64_to_f32((long long)t.acc[a]);  // written below: no __ldg
        if (t.ext) j[k] += __ldg(t.ext + a);
    }
}

__device__ __forceinline__ void clear_j(const JTake &t, int64_t cells, int64_t id)
{
#pragma unroll
    for (int k = 0; k < 3; ++k) t.acc[k * cells + id] = 0ull;
}

// The four diagnostic sums of a block (time-centred 2 KE, momentum), in FP64, into
// diag_blocks[slot * 4 ..].
__device__ __forceinline__ void em_block_diag(float ke, const float *mom, double *diag_blocks,
                                              int slot)
{
    __shared__ double red[4][EM_THREADS / 32];
    const float vals[4] = {ke, mom[0], mom[1], mom[2]};
    const int w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        double x = vals[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0) red[k][w] = x;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double sum = 0.0;
        for (int j = 0; j < EM_THREADS / 32; ++j) sum += red[threadIdx.x][j];
        diag_blocks[(int64_t)slot * 4 + threadIdx.x] = sum;
    }
}

}  // namespace apk
