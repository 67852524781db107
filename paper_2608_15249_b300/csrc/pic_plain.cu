// pic_plain.cu -- the FP64 plain form of the PIC cycle: FP64 positions and
// velocities, FP64 field, one thread per particle, one 64-bit atomic per
// corner, no sort and no tiling.  It is the comparison form for the FP32
// cell + offset path (same cycle, Sec. 3.1, Listing 1; same readings), and the
// long-run reference of the precision study.
//
// Charge still goes through the int64 fixed-point accumulator (S = 40 by
// default, FP64 weights), so runs are reproducible and the total is exact.
#include <math.h>

#include "pic_internal.cuh"

namespace apk {

constexpr int PL_THREADS = 256;

__device__ __forceinline__ int upn(int c, int n) { return (c + 1 == n) ? 0 : c + 1; }

// c = floor(x / dx) (via x * (1/dx)), f = x/dx - c; a position that rounds onto
// c == n is node 0.
__device__ __forceinline__ void locate64(double x, double inv_dx, int n, int &c, double &f)
{
    const double u = x * inv_dx;
    const double fl = floor(u);
    c = (int)fl;
    f = u - fl;
    if (c >= n || c < 0) {
        c = 0;
        f = 0.0;
    }
}

template <int D, int NV>
__global__ void __launch_bounds__(PL_THREADS)
    k_plain_pass(GridParamsF64 g, ParticlesF64 p, const double *__restrict__ E,
                 unsigned long long *__restrict__ acc, int mode, double *__restrict__ diag_blocks,
                 int *__restrict__ err)
{
    const int64_t np = p.np;
    const int64_t cells = (int64_t)g.n[0] * g.n[1] * g.n[2];
    const double scale = ldexp(1.0, g.fx_bits);
    const long long one = 1ll << g.fx_bits;
    double ke = 0.0, mom[3] = {0.0, 0.0, 0.0};
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < np;
         i += (int64_t)gridDim.x * blockDim.x) {
        double x[3] = {0.0, 0.0, 0.0}, v[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int a = 0; a < D; ++a) x[a] = p.x[a * np + i];
#pragma unroll
        for (int a = 0; a < NV; ++a) v[a] = p.v[a * np + i];
        int c[3] = {0, 0, 0};
        double f[3] = {0.0, 0.0, 0.0};
        if (mode & 1) {  // gather + Boris by the step encoded in g.qmh2, t, s
#pragma unroll
            for (int a = 0; a < D; ++a) locate64(x[a], g.inv_dx[a], g.n[a], c[a], f[a]);
            double e[3] = {0.0, 0.0, 0.0};
#pragma unroll
            for (int k = 0; k < (1 << D); ++k) {
                double w = 1.0;
                int node = 0, stride = 1;
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    const int up = (k >> a) & 1;
                    w *= up ? f[a] : 1.0 - f[a];
                    node += (up ? upn(c[a], g.n[a]) : c[a]) * stride;
                    stride *= g.n[a];
                }
#pragma unroll
                for (int a = 0; a < D; ++a) e[a] += w * E[a * cells + node];
            }
            double vm[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) vm[a] = v[a] + g.qmh2 * (e[a] + g.E0[a]);
            if (g.magnetised) {
                const double w0 = vm[0] + (vm[1] * g.t[2] - vm[2] * g.t[1]);
                const double w1 = vm[1] + (vm[2] * g.t[0] - vm[0] * g.t[2]);
                const double w2 = vm[2] + (vm[0] * g.t[1] - vm[1] * g.t[0]);
                const double p0 = vm[0] + (w1 * g.s[2] - w2 * g.s[1]);
                const double p1 = vm[1] + (w2 * g.s[0] - w0 * g.s[2]);
                const double p2 = vm[2] + (w0 * g.s[1] - w1 * g.s[0]);
                vm[0] = p0;
                vm[1] = p1;
                vm[2] = p2;
            }
            double o2 = 0.0, n2 = 0.0;
#pragma unroll
            for (int a = 0; a < NV; ++a) {
                const double vn = vm[a] + g.qmh2 * (e[a] + g.E0[a]);
                if (!isfinite(vn)) bad = true;
                o2 += v[a] * v[a];
                n2 += vn * vn;
                mom[a] += vn;
                v[a] = vn;
                p.v[a * np + i] = vn;
            }
            ke += 0.5 * (o2 + n2);
        }
        if (mode & 2) {  // move + periodic wrap
#pragma unroll
            for (int a = 0; a < D; ++a) {
                double xa = x[a] + v[a] * g.dt;
                if (!isfinite(xa)) {
                    bad = true;
                    xa = x[a];
                }
                xa -= g.L[a] * floor(xa / g.L[a]);
                if (xa >= g.L[a] || xa < 0.0) xa = 0.0;
                x[a] = xa;
                p.x[a * np + i] = xa;
            }
        }
        if (mode & 4) {  // deposit at the (new) position
#pragma unroll
            for (int a = 0; a < D; ++a) locate64(x[a], g.inv_dx[a], g.n[a], c[a], f[a]);
            long long rest = one;
#pragma unroll
            for (int k = 0; k < (1 << D); ++k) {
                double w = 1.0;
                int node = 0, stride = 1;
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    const int up = (k >> a) & 1;
                    w *= up ? f[a] : 1.0 - f[a];
                    node += (up ? upn(c[a], g.n[a]) : c[a]) * stride;
                    stride *= g.n[a];
                }
                long long qk;
                if (k == (1 << D) - 1) {
                    qk = rest;
                } else {
                    qk = __double2ll_rn(w * scale);
                    rest -= qk;
                }
                atomicAdd(acc + node, (unsigned long long)qk);
            }
        }
    }
    if (bad) atomicOr(err, EF_NONFINITE);
    if ((mode & 8) && diag_blocks) {
        __shared__ double red[4][PL_THREADS / 32];
        double vals[4] = {ke, mom[0], mom[1], mom[2]};
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            double s = vals[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) red[k][w] = s;
        }
        __syncthreads();
        if (threadIdx.x < 4) {
            double s = 0.0;
            for (int j = 0; j < PL_THREADS / 32; ++j) s += red[threadIdx.x][j];
            diag_blocks[blockIdx.x * 4 + threadIdx.x] = s;
        }
    }
}

template <int D, int NV>
static void launch_plain_t(const GridParamsF64 &g, ParticlesF64 p, const double *E,
                           unsigned long long *acc, int mode, double *diag, int nb, int *err,
                           cudaStream_t st)
{
    k_plain_pass<D, NV><<<nb, PL_THREADS, 0, st>>>(g, p, E, acc, mode, diag, err);
    note_launch();
}

int plain_pass_blocks(int64_t np, int ndim)
{
    // one wave: 5 CTAs of 256 threads per SM (3 in 3D), 512 particles per CTA at least
    const int64_t need = (np + 511) / 512;
    const int64_t cap = (int64_t)sm_count() * (ndim == 3 ? 3 : 5);
    const int64_t b = need < cap ? need : cap;
    return (int)(b < 1 ? 1 : b);
}

cudaError_t launch_plain_pass(const GridParamsF64 &g, ParticlesF64 p, const double *E,
                              unsigned long long *acc, bool push, bool mv, bool deposit,
                              DiagPartials diag, int *err, cudaStream_t st)
{
    if (p.np == 0) return cudaSuccess;
    const int mode = (push ? 1 : 0) | (mv ? 2 : 0) | (deposit ? 4 : 0) |
                     (diag.blocks && push ? 8 : 0);
    const int nb = plain_pass_blocks(p.np, g.ndim);
    switch (g.ndim * 10 + p.nv) {
    case 11: launch_plain_t<1, 1>(g, p, E, acc, mode, diag.blocks, nb, err, st); break;
    case 12: launch_plain_t<1, 2>(g, p, E, acc, mode, diag.blocks, nb, err, st); break;
    case 13: launch_plain_t<1, 3>(g, p, E, acc, mode, diag.blocks, nb, err, st); break;
    case 22: launch_plain_t<2, 2>(g, p, E, acc, mode, diag.blocks, nb, err, st); break;
    case 23: launch_plain_t<2, 3>(g, p, E, acc, mode, diag.blocks, nb, err, st); break;
    case 33: launch_plain_t<3, 3>(g, p, E, acc, mode, diag.blocks, nb, err, st); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// x (count x ndim, row-major host layout) -> SoA FP64; v likewise.  Positions
// outside [0, L] latch EF_NONFINITE; x == L is 0.
__global__ void k_plain_load(GridParamsF64 g, const double *__restrict__ x,
                             const double *__restrict__ v, ParticlesF64 p, int64_t first,
                             int64_t count, int *err)
{
    bool bad = false;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = first + k;
        for (int a = 0; a < g.ndim; ++a) {
            double xa = x[k * g.ndim + a];
            if (!(xa >= 0.0 && xa <= g.L[a])) {
                bad = true;
                xa = 0.0;
            }
            if (xa == g.L[a]) xa = 0.0;
            p.x[a * p.np + i] = xa;
        }
        for (int a = 0; a < p.nv; ++a) {
            const double va = v[k * p.nv + a];
            if (!isfinite(va)) bad = true;
            p.v[a * p.np + i] = va;
        }
    }
    if (bad) atomicOr(err, EF_NONFINITE);
}

cudaError_t launch_plain_load(const GridParamsF64 &g, const double *x, const double *v,
                              ParticlesF64 p, int64_t first, int64_t count, int *err,
                              cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    int64_t nb = (count + 255) / 256;
    if (nb > 65535) nb = 65535;
    k_plain_load<<<(int)nb, 256, 0, st>>>(g, x, v, p, first, count, err);
    note_launch();
    return cudaGetLastError();
}

// ---- FP64 field: conversion, CG, E -----------------------------------------------------------

constexpr int PF = 256;

__device__ __forceinline__ double pwarp_sum(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

__device__ double pblock_sum(double x)
{
    __shared__ double red[PF / 32];
    __shared__ double total;
    x = pwarp_sum(x);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int j = 0; j < PF / 32; ++j) t += red[j];
        total = t;
    }
    __syncthreads();
    const double r = total;
    __syncthreads();
    return r;
}

__device__ long long pblock_sum_ll(long long x)
{
    __shared__ long long red[PF / 32];
    __shared__ long long total;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int j = 0; j < PF / 32; ++j) t += red[j];
        total = t;
    }
    __syncthreads();
    const long long r = total;
    __syncthreads();
    return r;
}

__device__ double preduce(const double *__restrict__ part, int n)
{
    double s = 0.0;
    for (int j = threadIdx.x; j < n; j += PF) s += part[j];
    return pblock_sum(s);
}

__device__ __forceinline__ void pcoords(int64_t id, const FieldBufsF64 &f, int *j)
{
    const uint32_t u = (uint32_t)id;
    const uint32_t r = fdiv(u, f.div0);
    j[0] = (int)(u - r * (uint32_t)f.n[0]);
    if (f.ndim >= 2) {
        const uint32_t r2 = fdiv(r, f.div1);
        j[1] = (int)(r - r2 * (uint32_t)f.n[1]);
        j[2] = (int)r2;
    } else {
        j[1] = 0;
        j[2] = 0;
    }
}

__device__ __forceinline__ double pneg_lap(const double *__restrict__ u, int64_t id, const int *j,
                                           const FieldBufsF64 &f, const double *idx2)
{
    const double c = u[id];
    double acc = 0.0;
    int64_t stride = 1;
    for (int a = 0; a < f.ndim; ++a) {
        const int na = f.n[a];
        const int64_t up = (j[a] + 1 == na) ? id - (int64_t)(na - 1) * stride : id + stride;
        const int64_t dn = (j[a] == 0) ? id + (int64_t)(na - 1) * stride : id - stride;
        acc += (2.0 * c - u[up] - u[dn]) * idx2[a];
        stride *= na;
    }
    return acc;
}

struct LapD {
    double idx2[3];
    double inv_diag;
};

static LapD make_lapd(const FieldBufsF64 &f)
{
    LapD L{};
    double d = 0.0;
    for (int a = 0; a < f.ndim; ++a) {
        L.idx2[a] = 1.0 / (f.dx[a] * f.dx[a]);
        d += 2.0 * L.idx2[a];
    }
    L.inv_diag = 1.0 / d;
    return L;
}

__global__ void __launch_bounds__(PF)
    k_plain_rho(FieldBufsF64 f, double scale, double bg, double mean_e)
{
    long long isum = 0;
    for (int64_t j = (int64_t)blockIdx.x * PF + threadIdx.x; j < f.cells;
         j += (int64_t)gridDim.x * PF) {
        const long long a = (long long)f.acc[j];
        isum += a;
        const double re = scale * (double)a;
        f.rho[j] = re + bg;
        f.b[j] = re - mean_e;
    }
    const long long t = pblock_sum_ll(isum);
    if (threadIdx.x == 0) f.isum_part[blockIdx.x] = t;
}

cudaError_t launch_plain_rho_convert(FieldBufsF64 &f, double scale, double bg, double mean_e,
                                     cudaStream_t st)
{
    k_plain_rho<<<f.nblocks, PF, 0, st>>>(f, scale, bg, mean_e);
    note_launch();
    return cudaGetLastError();
}

enum : int { PS_BNORM = 0, PS_RZ0 = 1, PS_RELRES = 3 };

// The periodic operator is singular (constants are its null space).  Rounding
// leaves r with a constant part that CG cannot remove; once the rest has
// converged, p would turn nearly constant, p.Ap would vanish and alpha blow up
// (a single-mode right-hand side, converged in one iteration, reaches that state
// at once).  So, as in the FP32 solve, r is projected onto zero mean at every
// direction update (its sum comes with the r.r reduction; |r - m|^2 = r.r - N m^2).
__global__ void __launch_bounds__(PF) k_plain_cg_init(FieldBufsF64 f, LapD L)
{
    double rr = 0.0, bb = 0.0, rs = 0.0;
    for (int64_t id = (int64_t)blockIdx.x * PF + threadIdx.x; id < f.cells;
         id += (int64_t)gridDim.x * PF) {
        int j[3];
        pcoords(id, f, j);
        const double ri = f.b[id] - pneg_lap(f.phi, id, j, f, L.idx2);
        f.r[id] = ri;
        rr += ri * ri;
        rs += ri;
        bb += f.b[id] * f.b[id];
    }
    rr = pblock_sum(rr);
    rs = pblock_sum(rs);
    bb = pblock_sum(bb);
    if (threadIdx.x == 0) {
        f.part[0][blockIdx.x] = rr;
        f.part[1][blockIdx.x] = rs;
        f.part[2][blockIdx.x] = bb;
    }
}

// r -= mean(r);  p = M^-1 r (after the initial residual's sums are reduced).
__global__ void __launch_bounds__(PF) k_plain_cg_init_dir(FieldBufsF64 f, LapD L)
{
    const double m = preduce(f.part[1], f.nblocks) / (double)f.cells;
    for (int64_t id = (int64_t)blockIdx.x * PF + threadIdx.x; id < f.cells;
         id += (int64_t)gridDim.x * PF) {
        const double ri = f.r[id] - m;
        f.r[id] = ri;
        f.p[id] = ri * L.inv_diag;
    }
}

__global__ void __launch_bounds__(PF) k_plain_cg_init_fin(FieldBufsF64 f, LapD L, double rtol)
{
    const double rr0 = preduce(f.part[0], f.nblocks);
    const double rs = preduce(f.part[1], f.nblocks);
    const double bb = preduce(f.part[2], f.nblocks);
    const double m = rs / (double)f.cells;
    const double rr = fmax(rr0 - (double)f.cells * m * m, 0.0);
    if (threadIdx.x == 0) {
        const double bn = sqrt(bb);
        f.scal[PS_BNORM] = bn;
        f.scal[PS_RZ0] = rr * L.inv_diag;
        const double rel = bn > 0.0 ? sqrt(rr) / bn : 0.0;
        f.scal[PS_RELRES] = rel;
        *f.iters = 0;
        *f.done = (bn == 0.0 || rel <= rtol) ? 1 : 0;
    }
}

__global__ void __launch_bounds__(PF) k_plain_cg_matvec(FieldBufsF64 f, LapD L)
{
    if (*f.done) return;
    double pq = 0.0;
    for (int64_t id = (int64_t)blockIdx.x * PF + threadIdx.x; id < f.cells;
         id += (int64_t)gridDim.x * PF) {
        int j[3];
        pcoords(id, f, j);
        const double qi = pneg_lap(f.p, id, j, f, L.idx2);
        f.q[id] = qi;
        pq += f.p[id] * qi;
    }
    pq = pblock_sum(pq);
    if (threadIdx.x == 0) f.part[0][blockIdx.x] = pq;
}

__global__ void __launch_bounds__(PF) k_plain_cg_update(FieldBufsF64 f, int it)
{
    if (*f.done) return;
    const double pq = preduce(f.part[0], f.nblocks);
    const double alpha = f.scal[PS_RZ0 + (it & 1)] / pq;
    if (!(pq > 0.0) || !isfinite(alpha)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) *f.done = 1;
        return;
    }
    double rr = 0.0, rs = 0.0;
    for (int64_t id = (int64_t)blockIdx.x * PF + threadIdx.x; id < f.cells;
         id += (int64_t)gridDim.x * PF) {
        f.phi[id] += alpha * f.p[id];
        const double ri = f.r[id] - alpha * f.q[id];
        f.r[id] = ri;
        rr += ri * ri;
        rs += ri;
    }
    rr = pblock_sum(rr);
    rs = pblock_sum(rs);
    if (threadIdx.x == 0) {
        f.part[1][blockIdx.x] = rr;
        f.part[2][blockIdx.x] = rs;
    }
}

__global__ void __launch_bounds__(PF)
    k_plain_cg_dir(FieldBufsF64 f, LapD L, int it, int maxit, double rtol)
{
    if (*f.done) return;
    const double rr0 = preduce(f.part[1], f.nblocks);
    const double m = preduce(f.part[2], f.nblocks) / (double)f.cells;
    const double rr = fmax(rr0 - (double)f.cells * m * m, 0.0);
    const double rz_new = rr * L.inv_diag;
    const double rz = f.scal[PS_RZ0 + (it & 1)];
    const double rel = sqrt(rr) / f.scal[PS_BNORM];
    const bool stop = rel <= rtol || it + 1 >= maxit;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        f.scal[PS_RZ0 + ((it + 1) & 1)] = rz_new;
        f.scal[PS_RELRES] = rel;
        *f.iters = it + 1;
        if (stop) *f.done = 1;
    }
    if (stop) return;
    const double beta = rz_new / rz;
    for (int64_t id = (int64_t)blockIdx.x * PF + threadIdx.x; id < f.cells;
         id += (int64_t)gridDim.x * PF) {
        const double ri = f.r[id] - m;
        f.r[id] = ri;
        f.p[id] = ri * L.inv_diag + beta * f.p[id];
    }
}

__global__ void k_plain_cg_finish(FieldBufsF64 f, double rtol, int *err)
{
    if (threadIdx.x == 0 && blockIdx.x == 0 && f.scal[PS_RELRES] > rtol) atomicOr(err, EF_CG);
}

cudaError_t launch_plain_cg_init(FieldBufsF64 &f, double rtol, cudaStream_t st)
{
    const LapD L = make_lapd(f);
    k_plain_cg_init<<<f.nblocks, PF, 0, st>>>(f, L);
    note_launch();
    k_plain_cg_init_dir<<<f.nblocks, PF, 0, st>>>(f, L);
    note_launch();
    k_plain_cg_init_fin<<<1, PF, 0, st>>>(f, L, rtol);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_plain_cg_iters(FieldBufsF64 &f, int first, int count, int maxit, double rtol,
                                  cudaStream_t st)
{
    const LapD L = make_lapd(f);
    for (int it = first; it < first + count && it < maxit; ++it) {
        k_plain_cg_matvec<<<f.nblocks, PF, 0, st>>>(f, L);
        note_launch();
        k_plain_cg_update<<<f.nblocks, PF, 0, st>>>(f, it);
        note_launch();
        k_plain_cg_dir<<<f.nblocks, PF, 0, st>>>(f, L, it, maxit, rtol);
        note_launch();
    }
    return cudaGetLastError();
}

cudaError_t launch_plain_cg_finish(FieldBufsF64 &f, double rtol, int *err, cudaStream_t st)
{
    k_plain_cg_finish<<<1, 32, 0, st>>>(f, rtol, err);
    note_launch();
    return cudaGetLastError();
}

__global__ void __launch_bounds__(PF) k_plain_efield(FieldBufsF64 f, double h0, double h1,
                                                     double h2)
{
    const double h[3] = {h0, h1, h2};
    double fe = 0.0;
    for (int64_t id = (int64_t)blockIdx.x * PF + threadIdx.x; id < f.cells;
         id += (int64_t)gridDim.x * PF) {
        int j[3];
        pcoords(id, f, j);
        int64_t stride = 1;
        for (int a = 0; a < f.ndim; ++a) {
            const int na = f.n[a];
            const int64_t up = (j[a] + 1 == na) ? id - (int64_t)(na - 1) * stride : id + stride;
            const int64_t dn = (j[a] == 0) ? id + (int64_t)(na - 1) * stride : id - stride;
            const double e = -(f.phi[up] - f.phi[dn]) * h[a];
            f.E[a * f.cells + id] = e;
            fe += e * e;
            stride *= na;
        }
    }
    fe = pblock_sum(fe);
    if (threadIdx.x == 0) f.fe_part[blockIdx.x] = fe;
}

cudaError_t launch_plain_efield(FieldBufsF64 &f, cudaStream_t st)
{
    double h[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < f.ndim; ++a) h[a] = 0.5 / f.dx[a];
    k_plain_efield<<<f.nblocks, PF, 0, st>>>(f, h[0], h[1], h[2]);
    note_launch();
    return cudaGetLastError();
}

__global__ void __launch_bounds__(PF)
    k_plain_diag(const double *__restrict__ pblocks, int npb, FieldBufsF64 f, double *out,
                 long long *acc_sum_out)
{
    for (int k = 0; k < 4; ++k) {
        double s = 0.0;
        if (pblocks)
            for (int j = threadIdx.x; j < npb; j += PF) s += pblocks[j * 4 + k];
        s = pblock_sum(s);
        if (threadIdx.x == 0 && pblocks) out[k] = s;
    }
    const double fe = preduce(f.fe_part, f.nblocks);
    long long is = 0;
    for (int j = threadIdx.x; j < f.nblocks; j += PF) is += f.isum_part[j];
    is = pblock_sum_ll(is);
    if (threadIdx.x == 0) {
        out[4] = fe;
        out[5] = f.scal[PS_RELRES];
        out[6] = (double)*f.iters;
        *acc_sum_out = is;
    }
}

cudaError_t launch_plain_diag_finalize(const DiagPartials &pd, bool have_particles,
                                       FieldBufsF64 &f, double *out, long long *acc_sum_out,
                                       cudaStream_t st)
{
    k_plain_diag<<<1, PF, 0, st>>>(have_particles ? pd.blocks : nullptr, pd.nblocks, f, out,
                                   acc_sum_out);
    note_launch();
    return cudaGetLastError();
}

}  // namespace apk
