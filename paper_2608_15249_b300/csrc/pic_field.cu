// pic_field.cu -- grid side of the electrostatic PIC cycle: conversion of the
// int64 fixed-point charge to rho, the periodic Poisson solve
// -lap_h(phi) = rho - mean(rho) by Jacobi-preconditioned conjugate gradients
// (D_Poisson, Sec. 2.2; module D02 in Sec. 3.1), E = -grad_h(phi) by centred
// differences (D06), and the diagnostics reductions.
//
// Precision: CG vectors are FP32; every dot product is accumulated in FP64
// and reduced deterministically (fixed per-block order, then every block that
// needs the total re-reduces the block partials in the same fixed order, so
// all blocks see bit-identical scalars without an extra launch).
// The Jacobi preconditioner of the constant-coefficient Laplacian is the
// constant diagonal 2 sum_a 1/dx_a^2.
#include <math.h>

#include "pic_internal.cuh"

namespace apk {

constexpr int FT = 256;  // threads per block of the grid kernels

// Device scalar slots.
enum : int { SC_BNORM = 0, SC_RZ0 = 1, SC_RZ1 = 2, SC_RELRES = 3, SC_NSCAL = 8 };

int field_blocks(int64_t cells)
{
    const int sms = sm_count();
    int64_t need = (cells + FT - 1) / FT;
    int64_t cap = (int64_t)sms * 4;
    int64_t b = need < cap ? need : cap;
    return (int)(b < 1 ? 1 : b);
}

__device__ __forceinline__ double warp_sum(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

__device__ __forceinline__ long long warp_sum_ll(long long x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Sum over the block in a fixed order; result valid in every thread.
__device__ double block_sum(double x)
{
    __shared__ double red[FT / 32];
    __shared__ double total;
    x = warp_sum(x);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int j = 0; j < FT / 32; ++j) t += red[j];
        total = t;
    }
    __syncthreads();
    const double r = total;
    __syncthreads();
    return r;
}

__device__ long long block_sum_ll(long long x)
{
    __shared__ long long red[FT / 32];
    __shared__ long long total;
    x = warp_sum_ll(x);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int j = 0; j < FT / 32; ++j) t += red[j];
        total = t;
    }
    __syncthreads();
    const long long r = total;
    __syncthreads();
    return r;
}

// Sum of `n` block partials in a fixed order (identical in every block).
__device__ double reduce_partials(const double *__restrict__ part, int n)
{
    double s = 0.0;
    for (int j = threadIdx.x; j < n; j += FT) s += part[j];
    return block_sum(s);
}

// The periodic neighbours of node id along each of the D axes, as 32-bit node
// indices (cells < 2^31), for stencils whose axis loop is unrolled at compile time.
// The coordinates come from the multiply-high division (a runtime integer division
// would issue float conversions on this GPU's slow FP64 pipe).
template <int D>
struct Nbrs {
    int up[D], dn[D];
};

template <int D>
__device__ __forceinline__ Nbrs<D> neighbours(int id, const FieldBufs &f)
{
    int j[3] = {id, 0, 0};
    if (D >= 2) {
        const uint32_t u = (uint32_t)id;
        const uint32_t r = fdiv(u, f.div0);
        j[0] = (int)(u - r * (uint32_t)f.n[0]);
        if (D == 2) {
            j[1] = (int)r;
        } else {
            const uint32_t r2 = fdiv(r, f.div1);
            j[1] = (int)(r - r2 * (uint32_t)f.n[1]);
            j[2] = (int)r2;
        }
    }
    Nbrs<D> s;
    int st = 1;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const int na = f.n[a];
        s.up[a] = (j[a] + 1 == na) ? id - (na - 1) * st : id + st;
        s.dn[a] = (j[a] == 0) ? id + (na - 1) * st : id - st;
        st *= na;
    }
    return s;
}

// (-lap_h u)[id] on the periodic grid, the axes in order.
template <int D>
__device__ __forceinline__ float neg_lap_d(const float *__restrict__ u, int id, const Nbrs<D> &s,
                                           const float *idx2)
{
    const float c = u[id];
    float acc = 0.0f;
#pragma unroll
    for (int a = 0; a < D; ++a) acc += (2.0f * c - u[s.up[a]] - u[s.dn[a]]) * idx2[a];
    return acc;
}

// ---- charge conversion ----------------------------------------------------------------------

// b from the accumulator, its integer sum, and (clear non-null) the other
// accumulator zeroed for the next deposit.
__global__ void __launch_bounds__(FT)
    k_rho_convert(FieldBufs f, long long mean_q, float mean_r, float scale,
                  unsigned long long *__restrict__ clear)
{
    long long isum = 0;
    for (int64_t j = (int64_t)blockIdx.x * FT + threadIdx.x; j < f.cells;
         j += (int64_t)gridDim.x * FT) {
        const long long a = (long long)f.acc[j];
        if (clear) clear[j] = 0ull;
        isum += a;
        // acc - mean: the integer difference is exact, its float rounds once, then the
        // fraction of the mean and the scale (no cancellation of large terms)
        f.b[j] = scale * (i64_to_f32(a - mean_q) - mean_r);
    }
    const long long t = block_sum_ll(isum);
    if (threadIdx.x == 0) f.isum_part[blockIdx.x] = t;
}

cudaError_t launch_rho_convert(FieldBufs &f, long long mean_q, float mean_r, float scale,
                               unsigned long long *clear, cudaStream_t st)
{
    k_rho_convert<<<f.nblocks, FT, 0, st>>>(f, mean_q, mean_r, scale, clear);
    note_launch();
    return cudaGetLastError();
}

// ---- CG -------------------------------------------------------------------------------------

struct Lap {
    float idx2[3];  // 1 / dx_a^2
    float inv_diag; // 1 / (2 sum_a 1/dx_a^2)
};

static Lap make_lap(const FieldBufs &f)
{
    Lap L;
    double d = 0.0;
    for (int a = 0; a < 3; ++a) {
        L.idx2[a] = a < f.ndim ? (float)(1.0 / (f.dx[a] * f.dx[a])) : 0.0f;
        if (a < f.ndim) d += 2.0 / (f.dx[a] * f.dx[a]);
    }
    L.inv_diag = (float)(1.0 / d);
    return L;
}

// The periodic operator is singular (constants are its null space): FP32
// rounding leaves r with a small constant part that CG cannot remove, and once
// the rest has converged p would become nearly constant and p.Ap vanish.  So
// every direction update projects r onto zero mean (its sum comes with the
// r.r reduction; |r - m|^2 = r.r - N m^2), and a non-positive or non-finite
// p.Ap stops the iteration instead of dividing by it.

// ---- the whole CG solve in one cooperative launch ----------------------------------------------
//
// A CG loop of separate launches needs the host to read a done flag between blocks
// of launches.  k_cg_coop runs the Jacobi-PCG (FP32 vectors, FP64 dots, zero-mean
// projection of r, breakdown guard) as one cooperative launch of one block per SM:
// blocks meet at a grid barrier, every block re-reduces the block partials in the
// same fixed order (so all see bit-identical scalars and take the same decisions),
// and the convergence test never leaves the device.
//
// The iteration is the single-reduction (Chronopoulos-Gear) arrangement of the same
// PCG, so that it takes one grid barrier instead of two.  With z = M^-1 r, w = A z
// and s = A p carried by recurrences, both dots of an iteration, (r, z) and (w, z),
// come from one reduction:
//   p = z + beta p_old;  s = w + beta s_old;  x += alpha p;  r -= alpha s;
//   z = M^-1 r;  w = A z;  gamma' = (r, z);  delta = (w, z);
//   beta' = gamma' / gamma;  alpha' = gamma' / (delta - beta' gamma' / alpha),
// (first step: beta = 0, alpha = gamma / delta); in exact arithmetic it takes the
// same steps as the two-reduction form.  On this grid the Jacobi preconditioner is
// the scalar c = 1 / diag, and A annihilates constants, so with r projected onto zero
// mean (m = mean r, rb = r - m): z = c rb, w = c A r, gamma = c ((r, r) - N m^2) and
// delta = c^2 ((A r, r) - m sum A r) need only the sums (r, r), sum r, (A r, r) and
// sum A r of the unprojected r.  A node gets the new r at its neighbours, for its
// w, from their previous r, w and s (kept in ping-pong buffers), so the iteration
// has no second barrier.

// Threads per block of the cooperative solve.  Its iteration is bound by the
// latency of the block and grid reductions, which grow with the block: one block
// of 256 per SM measured 12.9 ms per 512^2 solve (786 iterations) against 15.0 ms
// with 128, 17.2 ms with 512 and 29.9 ms with 1024 (two or four blocks per SM were
// slower than one).
constexpr int CG_T = 256;
constexpr int GRID_WAIT_LIMIT = 1 << 22;  // polls of a grid barrier before giving up

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_add_release(unsigned *p, unsigned v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Barrier across the blocks of a cooperative launch (all co-resident).  *count
// (zero before the launch) only grows: barrier number g is passed once it reaches
// g * gridDim.x.  Each block's thread 0 arrives with a release add (its block's
// writes, ordered by the __syncthreads before it, are released) and polls
// with acquire loads, with a bound.  Returns false in every thread of the block if
// the bound ran out.
__device__ __forceinline__ bool grid_barrier(unsigned *count, unsigned &gen)
{
    __shared__ int s_ok;
    __syncthreads();
    ++gen;
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned target = gen * gridDim.x;
        red_add_release(count, 1u);
        int spins = 0;
        while (ld_acquire_u32(count) < target) {
            if (++spins > GRID_WAIT_LIMIT) {
                ok = 0;
                break;
            }
            __nanosleep(32);
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Fixed-order block sums of K values for CG_T threads (one pair of barriers for
// all K); the totals replace v[] in every thread.  Two calls with the same K must
// have a block barrier between them (in k_cg_coop, a grid barrier always does).
template <int K>
__device__ __forceinline__ void cg_block_sums(double (&v)[K])
{
    __shared__ double red[K][CG_T / 32];
    __shared__ double tot[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const double x = warp_sum(v[k]);
        if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = x;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        double t = 0.0;
        for (int j = 0; j < CG_T / 32; ++j) t += red[threadIdx.x][j];
        tot[threadIdx.x] = t;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = tot[k];
}

// Totals of K arrays of per-block partials (L2 loads: written by other blocks of
// this launch), the same fixed order in every block.
template <int K>
__device__ __forceinline__ void cg_reduce(double *const (&part)[K], double (&out)[K])
{
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = 0.0;
    for (int j = threadIdx.x; j < (int)gridDim.x; j += CG_T)
#pragma unroll
        for (int k = 0; k < K; ++k) out[k] += __ldcg(part[k] + j);
    cg_block_sums<K>(out);
}

struct CgCoop {
    const float *b;      // right-hand side
    float *x;            // solution, warm start on entry
    int maxit;           // iteration cap
    const int *it_used;  // iterations already spent (budget = maxit - *it_used), or null
    int *iters;          // iterations taken (out)
    int relres_slot;     // scal slot of the final relative residual
    int latch;           // latch EF_CG when the residual stays above rtol
};

template <int D>
__global__ void __launch_bounds__(CG_T, 1)
    k_cg_coop(FieldBufs f, Lap L, CgCoop c, double rtol, unsigned *bar, int *err)
{
    unsigned gen = 0u;
    const int stride = (int)gridDim.x * CG_T;
    const int first = (int)blockIdx.x * CG_T + (int)threadIdx.x;
    const int cells = (int)f.cells;
    // the vectors, unaliased (lets the loads of several nodes be in flight together)
    const float *__restrict__ bv = c.b;
    float *__restrict__ xv = c.x;
    float *__restrict__ pv = f.p;
    float *const R[2] = {f.r, f.r2}, *const W[2] = {f.q, f.w2}, *const S[2] = {f.p2, f.s2};
    const double N = (double)f.cells;
    const float cd = L.inv_diag;  // the Jacobi preconditioner (a scalar here)
    auto bail = [&]() {
        if (threadIdx.x == 0) atomicOr(err, EF_TIMEOUT);
    };
    // r = b - A x, and b.b
    double bb = 0.0;
    {
        float *__restrict__ r0 = R[0];
#pragma unroll 4
        for (int id = first; id < cells; id += stride) {
            const Nbrs<D> nb = neighbours<D>(id, f);
            const float bi = bv[id];
            r0[id] = bi - neg_lap_d<D>(xv, id, nb, L.idx2);
            bb += (double)bi * bi;
        }
    }
    if (!grid_barrier(bar, gen)) return bail();
    // w = c A r and the sums (r, r), sum r, (A r, r), sum A r, (b, b)
    {
        const float *__restrict__ r0 = R[0];
        float *__restrict__ w0 = W[0];
        double v[5] = {0.0, 0.0, 0.0, 0.0, bb};
#pragma unroll 4
        for (int id = first; id < cells; id += stride) {
            const Nbrs<D> nb = neighbours<D>(id, f);
            const float ri = r0[id];
            const float ar = neg_lap_d<D>(r0, id, nb, L.idx2);
            w0[id] = cd * ar;
            v[0] += (double)ri * ri;
            v[1] += ri;
            v[2] += (double)ri * ar;
            v[3] += ar;
        }
        cg_block_sums<5>(v);
        if (threadIdx.x == 0)
#pragma unroll
            for (int k = 0; k < 5; ++k) f.cgpart[0][k][blockIdx.x] = v[k];
    }
    if (!grid_barrier(bar, gen)) return bail();
    double m, rr, bn, gamma, delta;
    {
        double *const parts[5] = {f.cgpart[0][0], f.cgpart[0][1], f.cgpart[0][2],
                                  f.cgpart[0][3], f.cgpart[0][4]};
        double t[5];
        cg_reduce<5>(parts, t);
        m = t[1] / N;
        rr = fmax(t[0] - N * m * m, 0.0);
        bn = sqrt(t[4]);
        gamma = (double)cd * rr;
        delta = (double)cd * cd * (t[2] - m * t[3]);
    }
    double rel = bn > 0.0 ? sqrt(rr) / bn : 0.0;
    const int maxit = c.it_used ? max(c.maxit - *c.it_used, 1) : c.maxit;
    bool done = bn == 0.0 || rel <= rtol || maxit <= 0;
    double gamma_old = 0.0, alpha_old = 0.0;
    int it = 0;
    while (!done) {
        const double beta = it == 0 ? 0.0 : gamma / gamma_old;
        const double den = it == 0 ? delta : delta - beta * gamma / alpha_old;
        const double a64 = gamma / den;
        if (!(den > 0.0) || !isfinite(a64)) break;  // breakdown: keep x as it is
        // this iteration's buffers and the next (selected rather than indexed, so
        // that the arrays stay out of local memory)
        const bool odd = (it & 1) != 0;
        const float *__restrict__ ri = odd ? R[1] : R[0];
        const float *__restrict__ wi = odd ? W[1] : W[0];
        const float *__restrict__ so = odd ? S[1] : S[0];  // s of the previous iteration
        float *__restrict__ rn = odd ? R[0] : R[1];
        float *__restrict__ wn = odd ? W[0] : W[1];
        float *__restrict__ sn = odd ? S[0] : S[1];
        const float mf = (float)m, bf = (float)beta, af = (float)a64;
        const bool first_it = it == 0;
        // s and the new r at node k, from the previous r, w and s there
        auto s_at = [&](int k) { return first_it ? wi[k] : wi[k] + bf * so[k]; };
        auto r_at = [&](int k) { return (ri[k] - mf) - af * s_at(k); };
        double v[4] = {0.0, 0.0, 0.0, 0.0};  // (r, r), sum r, (A r, r), sum A r
#pragma unroll 4
        for (int id = first; id < cells; id += stride) {
            const Nbrs<D> nb = neighbours<D>(id, f);
            const float sc = s_at(id);
            const float rc = (ri[id] - mf) - af * sc;
            float pc = cd * (ri[id] - mf);
            if (!first_it) pc += bf * pv[id];
            pv[id] = pc;
            xv[id] += af * pc;
            sn[id] = sc;
            rn[id] = rc;
            float ar = 0.0f;
#pragma unroll
            for (int a = 0; a < D; ++a) ar += (2.0f * rc - r_at(nb.up[a]) - r_at(nb.dn[a])) * L.idx2[a];
            wn[id] = cd * ar;
            v[0] += (double)rc * rc;
            v[1] += rc;
            v[2] += (double)rc * ar;
            v[3] += ar;
        }
        // partials: set 1 in even iterations, set 0 in odd ones (the initial reduction
        // used set 0), so that no set is written while its last reduction is read
        double *const parts[4] = {odd ? f.cgpart[0][0] : f.cgpart[1][0],
                                  odd ? f.cgpart[0][1] : f.cgpart[1][1],
                                  odd ? f.cgpart[0][2] : f.cgpart[1][2],
                                  odd ? f.cgpart[0][3] : f.cgpart[1][3]};
        cg_block_sums<4>(v);
        if (threadIdx.x == 0)
#pragma unroll
            for (int k = 0; k < 4; ++k) parts[k][blockIdx.x] = v[k];
        if (!grid_barrier(bar, gen)) return bail();
        {
            double t[4];
            cg_reduce<4>(parts, t);
            m = t[1] / N;
            rr = fmax(t[0] - N * m * m, 0.0);
            gamma_old = gamma;
            alpha_old = a64;
            gamma = (double)cd * rr;
            delta = (double)cd * cd * (t[2] - m * t[3]);
        }
        rel = sqrt(rr) / bn;
        ++it;
        done = rel <= rtol || it >= maxit;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        f.scal[c.relres_slot] = rel;
        *c.iters = it;
        if (c.latch && rel > rtol) atomicOr(err, EF_CG);
    }
}

int cg_coop_blocks(int64_t cells)
{
    static std::atomic<int> per_sm{0};
    int c = per_sm.load(std::memory_order_relaxed);
    if (!c) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, k_cg_coop<3>, CG_T, 0) != cudaSuccess ||
            c < 1) {
            cudaGetLastError();
            c = 1;
        }
        per_sm.store(c, std::memory_order_relaxed);
    }
    // one block per SM (the barrier's cost grows with the blocks; two or four per SM
    // measured slower), never more than the co-resident capacity, the reduction
    // partials (field_blocks) or the work
    const int64_t need = (cells + CG_T - 1) / CG_T;
    int64_t b = (int64_t)sm_count();
    const int64_t cap = (int64_t)sm_count() * c;
    const int64_t parts = field_blocks(cells);
    b = b < cap ? b : cap;
    b = b < parts ? b : parts;
    b = b < need ? b : need;
    return (int)(b < 1 ? 1 : b);
}

cudaError_t launch_cg_solve(FieldBufs &f, const float *b, float *x, double rtol, int maxit,
                            const int *it_used, int *iters, int relres_slot, bool latch,
                            int *err, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(f.gbar, 0, 2 * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    Lap L = make_lap(f);
    CgCoop c;
    c.b = b;
    c.x = x;
    c.maxit = maxit;
    c.it_used = it_used;
    c.iters = iters;
    c.relres_slot = relres_slot;
    c.latch = latch ? 1 : 0;
    unsigned *bar = f.gbar;
    void *args[] = {&f, &L, &c, &rtol, &bar, &err};
    const int nb = cg_coop_blocks(f.cells);
    const void *fn = f.ndim == 1   ? (const void *)k_cg_coop<1>
                     : f.ndim == 2 ? (const void *)k_cg_coop<2>
                                   : (const void *)k_cg_coop<3>;
    e = cudaLaunchCooperativeKernel(fn, dim3(nb), dim3(CG_T), args, 0, st);
    note_launch();
    return e;
}

// ---- mixed-precision refinement -----------------------------------------------------------
//
// The FP32 CG above stalls near its rounding floor on large, smooth fields.  The
// solve is therefore an iterative refinement: the true residual of the FP32
// potential, rho - mean - A phi, is formed in FP64 from the FP64 charge density,
// rounded to FP32 as the right-hand side of a correction solve A x = r (FP32 CG,
// FP64 dots), and phi += x, until the FP64 residual meets the tolerance.

template <int D>
__device__ __forceinline__ double neg_lap64(const float *__restrict__ u, int id, const Nbrs<D> &s,
                                            const double *idx2)
{
    const double c = u[id];
    double acc = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a) acc += (2.0 * c - (double)u[s.up[a]] - (double)u[s.dn[a]]) * idx2[a];
    return acc;
}

template <int D>
__global__ void __launch_bounds__(FT)
    k_residual64(FieldBufs f, double i0, double i1, double i2, double scale, double bg,
                 double mean_total)
{
    const double idx2[3] = {i0, i1, i2};
    double rr = 0.0, bb = 0.0;
    const int cells = (int)f.cells;
    for (int id = (int)blockIdx.x * FT + (int)threadIdx.x; id < cells; id += (int)gridDim.x * FT) {
        const Nbrs<D> nb = neighbours<D>(id, f);
        const double rho = scale * (double)(long long)f.acc[id] + bg;
        const double bj = rho - mean_total;
        const double rj = bj - neg_lap64<D>(f.phi, id, nb, idx2);
        f.b[id] = (float)rj;
        rr += rj * rj;
        bb += bj * bj;
    }
    rr = block_sum(rr);
    bb = block_sum(bb);
    // the last block to finish reduces the partials (in block order, so the result
    // does not depend on which block that is) and re-arms the ticket
    __shared__ bool s_last;
    if (threadIdx.x == 0) {
        f.part[0][blockIdx.x] = rr;
        f.part[2][blockIdx.x] = bb;
        __threadfence();
        s_last = atomicAdd(f.ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // (L2 loads: the partials were written by other blocks of this launch)
    double s0 = 0.0, s2 = 0.0;
    for (int j = threadIdx.x; j < f.nblocks; j += FT) {
        s0 += __ldcg(f.part[0] + j);
        s2 += __ldcg(f.part[2] + j);
    }
    const double trr = block_sum(s0);
    const double tbb = block_sum(s2);
    if (threadIdx.x == 0) {
        const double bn = sqrt(tbb);
        f.scal[SCAL_BNORM64] = bn;
        f.scal[SCAL_TRUE_REL] = bn > 0.0 ? sqrt(trr) / bn : 0.0;
        *f.ticket = 0u;
    }
}

cudaError_t launch_residual64(FieldBufs &f, double scale, double bg, double mean_total,
                              cudaStream_t st)
{
    double i2[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < f.ndim; ++a) i2[a] = 1.0 / (f.dx[a] * f.dx[a]);
    if (f.ndim == 1)
        k_residual64<1><<<f.nblocks, FT, 0, st>>>(f, i2[0], i2[1], i2[2], scale, bg, mean_total);
    else if (f.ndim == 2)
        k_residual64<2><<<f.nblocks, FT, 0, st>>>(f, i2[0], i2[1], i2[2], scale, bg, mean_total);
    else
        k_residual64<3><<<f.nblocks, FT, 0, st>>>(f, i2[0], i2[1], i2[2], scale, bg, mean_total);
    note_launch();
    return cudaGetLastError();
}

__global__ void __launch_bounds__(FT) k_add_correction(FieldBufs f)
{
    for (int64_t id = (int64_t)blockIdx.x * FT + threadIdx.x; id < f.cells;
         id += (int64_t)gridDim.x * FT)
        f.phi[id] += f.x[id];
}

cudaError_t launch_add_correction(FieldBufs &f, cudaStream_t st)
{
    k_add_correction<<<f.nblocks, FT, 0, st>>>(f);
    note_launch();
    return cudaGetLastError();
}

// ---- E = -grad phi ---------------------------------------------------------------------------

template <int D>
__global__ void __launch_bounds__(FT) k_efield(FieldBufs f, float h0, float h1, float h2)
{
    const float h[3] = {h0, h1, h2};  // 1 / (2 dx_a)
    double fe = 0.0;
    const int cells = (int)f.cells;
    for (int id = (int)blockIdx.x * FT + (int)threadIdx.x; id < cells; id += (int)gridDim.x * FT) {
        const Nbrs<D> nb = neighbours<D>(id, f);
        float e[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int a = 0; a < D; ++a) {
            e[a] = -(f.phi[nb.up[a]] - f.phi[nb.dn[a]]) * h[a];
            fe += (double)e[a] * e[a];
        }
        // 1D and 2D: pairs (node x holds its own field and that of x + 1), so a node's
        // field goes to its own first half and to its lower x-neighbour's second half
        if (D == 1) {
            f.E[2 * id] = e[0];
            f.E[2 * nb.dn[0] + 1] = e[0];
        } else if (D == 2) {
            reinterpret_cast<float2 *>(f.E)[2 * id] = make_float2(e[0], e[1]);
            reinterpret_cast<float2 *>(f.E)[2 * nb.dn[0] + 1] = make_float2(e[0], e[1]);
        } else {
            reinterpret_cast<float4 *>(f.E)[id] = make_float4(e[0], e[1], e[2], 0.0f);
        }
    }
    fe = block_sum(fe);
    if (threadIdx.x == 0) f.fe_part[blockIdx.x] = fe;
}

cudaError_t launch_efield(FieldBufs &f, cudaStream_t st)
{
    float h[3] = {0.0f, 0.0f, 0.0f};
    for (int a = 0; a < f.ndim; ++a) h[a] = (float)(0.5 / f.dx[a]);
    if (f.ndim == 1) k_efield<1><<<f.nblocks, FT, 0, st>>>(f, h[0], h[1], h[2]);
    else if (f.ndim == 2) k_efield<2><<<f.nblocks, FT, 0, st>>>(f, h[0], h[1], h[2]);
    else k_efield<3><<<f.nblocks, FT, 0, st>>>(f, h[0], h[1], h[2]);
    note_launch();
    return cudaGetLastError();
}

// ---- diagnostics -----------------------------------------------------------------------------

// out: [0] sum (|v_old|^2 + |v_new|^2)/2, [1..3] sum v, [4] sum |E|^2, [5] relres,
// [6] iterations (as double);  acc_sum_out: sum of the accumulator.
__global__ void __launch_bounds__(FT)
    k_diag_finalize(const double *__restrict__ pblocks, int npb, FieldBufs f, double *out,
                    long long *acc_sum_out)
{
    for (int k = 0; k < 4; ++k) {
        double s = 0.0;
        if (pblocks)
            for (int j = threadIdx.x; j < npb; j += FT) s += pblocks[j * 4 + k];
        s = block_sum(s);
        if (threadIdx.x == 0 && pblocks) out[k] = s;
    }
    const double fe = reduce_partials(f.fe_part, f.nblocks);
    long long is = 0;
    for (int j = threadIdx.x; j < f.nblocks; j += FT) is += f.isum_part[j];
    is = block_sum_ll(is);
    if (threadIdx.x == 0) {
        out[4] = fe;
        out[5] = f.scal[SC_RELRES];
        out[6] = (double)*f.iters;
        *acc_sum_out = is;
    }
}

cudaError_t launch_diag_finalize(const DiagPartials &pd, bool have_particles, FieldBufs &f,
                                 double *out, long long *acc_sum_out, cudaStream_t st)
{
    k_diag_finalize<<<1, FT, 0, st>>>(have_particles ? pd.blocks : nullptr, pd.nblocks, f, out,
                                      acc_sum_out);
    note_launch();
    return cudaGetLastError();
}

// ---- read-back helpers -----------------------------------------------------------------------

__global__ void k_e_to_f64(FieldBufs f, double *__restrict__ out)
{
    for (int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; id < f.cells;
         id += (int64_t)gridDim.x * blockDim.x)
        for (int a = 0; a < f.ndim; ++a) out[a * f.cells + id] = f.E[id * f.Estride + a];
}

cudaError_t launch_e_to_f64(FieldBufs &f, double *out, cudaStream_t st)
{
    k_e_to_f64<<<f.nblocks, FT, 0, st>>>(f, out);
    note_launch();
    return cudaGetLastError();
}

__global__ void k_phi_to_f64(FieldBufs f, double *__restrict__ out)
{
    for (int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; id < f.cells;
         id += (int64_t)gridDim.x * blockDim.x)
        out[id] = f.phi[id];
}

cudaError_t launch_phi_to_f64(FieldBufs &f, double *out, cudaStream_t st)
{
    k_phi_to_f64<<<f.nblocks, FT, 0, st>>>(f, out);
    note_launch();
    return cudaGetLastError();
}

}  // namespace apk
