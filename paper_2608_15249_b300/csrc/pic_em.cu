// pic_em.cu -- the electromagnetic step (E_Maxwell, Sec. 2.2: finite-difference
// time-domain updates on the Yee lattice) with its particle coupling, on a periodic
// 2D3V grid.
//
// Fields live at integer times on the Yee lattice, component-major [3][cells], with
// element (i, j) of a component at ((i + sx) dx, (j + sy) dy):
//   Ex (1/2, 0), Ey (0, 1/2), Ez (0, 0);  Bx (0, 1/2), By (1/2, 0), Bz (1/2, 1/2);
// the current J is staggered like E.  Units: eps0 = 1, mu0 = 1 / c^2.  A step:
//   particles: gather E^n, B^n (+ uniform B0) on each component's lattice (CIC),
//              Boris, move, Esirkepov current J^(n+1/2), charge at x^(n+1);
//   fields:    B -= (dt/2) curl E;  E += dt (c^2 curl B - J);  B -= (dt/2) curl E.
// The Esirkepov (2001) current makes rho^(n+1) - rho^n + dt div J = 0 hold exactly in
// exact arithmetic, so Gauss's law is kept by the field update.  Current and charge
// are accumulated in int64 fixed point (deterministic, order independent).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "pic_em_common.cuh"
#include "pic_internal.cuh"

namespace apk {

namespace {

// i mod n in [0, n) for any i (the remainder only off the fast path)
__device__ __forceinline__ int wrap_any(int i, int n)
{
    if ((unsigned)i < (unsigned)n) return i;
    i %= n;
    return i < 0 ? i + n : i;
}

__device__ __forceinline__ float lattice_cic(const float *__restrict__ F, int n0, int n1, int i0,
                                             float fx, int j0, float fy)
{
    const int i1 = i0 + 1 == n0 ? 0 : i0 + 1, j1 = j0 + 1 == n1 ? 0 : j0 + 1;
    return (1.0f - fy) * ((1.0f - fx) * __ldg(F + i0 + n0 * j0) + fx * __ldg(F + i1 + n0 * j0)) +
           fy * ((1.0f - fx) * __ldg(F + i0 + n0 * j1) + fx * __ldg(F + i1 + n0 * j1));
}

// Jz weight of lattice node (aq, bq) of the stencil, Esirkepov's 2D
//   W_z = S0x S0y + DSx S0y / 2 + S0x DSy / 2 + DSx DSy / 3,
// grouped as S0x (S0y + DSy / 2) + DSx (S0y / 2 + DSy / 3): the bracket of the first
// term is the Jx factor of the same row, and both brackets are shared along it.
__device__ __forceinline__ float esirkepov_wz(const float (&S0)[2][3], const float (&DS)[2][3],
                                              int aq, int bq)
{
    return fmaf(S0[0][aq], S0[1][bq] + 0.5f * DS[1][bq],
                DS[0][aq] * (0.5f * S0[1][bq] + DS[1][bq] * (1.0f / 3.0f)));
}

// One particle through the whole particle part of the step, reading the fields and
// adding the current and charge in global memory (the half push of the load, with
// MOVE false, and the particles of tiles too spread out for the shared-memory
// windows).  A particle that is not finite or moves more than a cell is left where it
// is and flagged.
template <bool MOVE>
__device__ __forceinline__ void em_particle_global(int64_t i, const GridParams &g, ParticlesF32 p,
                                                   const EmBufs &em,
                                                   unsigned long long *__restrict__ rho_acc,
                                                   float scale, int one, float &ke, float *mom,
                                                   bool &bad)
{
    const int n0 = g.n[0], n1 = g.n[1];
    const int64_t cells = (int64_t)n0 * n1;
    const int cell = p.cell[i];
    int c[2];
    c[1] = (int)fdiv((uint32_t)cell, g.div0);
    c[0] = cell - c[1] * n0;
    const float f[2] = {p.off[i], p.off[p.stride + i]};
    const float v[3] = {p.v[i], p.v[p.stride + i], p.v[2 * p.stride + i]};
    // staggered gathers
    int ix[2], iy[2];
    float fx[2], fy[2];
    stagger(c[0], f[0], false, n0, &ix[0], &fx[0]);
    stagger(c[0], f[0], true, n0, &ix[1], &fx[1]);
    stagger(c[1], f[1], false, n1, &iy[0], &fy[0]);
    stagger(c[1], f[1], true, n1, &iy[1], &fy[1]);
    float e[3], b[3];
    e[0] = lattice_cic(em.E, n0, n1, ix[1], fx[1], iy[0], fy[0]);
    e[1] = lattice_cic(em.E + cells, n0, n1, ix[0], fx[0], iy[1], fy[1]);
    e[2] = lattice_cic(em.E + 2 * cells, n0, n1, ix[0], fx[0], iy[0], fy[0]);
    b[0] = lattice_cic(em.B, n0, n1, ix[0], fx[0], iy[1], fy[1]) + em.B0[0];
    b[1] = lattice_cic(em.B + cells, n0, n1, ix[1], fx[1], iy[0], fy[0]) + em.B0[1];
    b[2] = lattice_cic(em.B + 2 * cells, n0, n1, ix[1], fx[1], iy[1], fy[1]) + em.B0[2];
#pragma unroll
    for (int a = 0; a < 3; ++a) e[a] += g.E0[a];
    float vn[3];
    em_boris(v, e, b, g, vn);
    bool finite = isfinite(vn[0]) && isfinite(vn[1]) && isfinite(vn[2]);
    float o2 = 0.0f, n2 = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        o2 += v[a] * v[a];
        n2 += vn[a] * vn[a];
        mom[a] += vn[a];
        p.v[a * p.stride + i] = vn[a];
    }
    ke += 0.5f * (o2 + n2);
    if constexpr (!MOVE) {
        if (!finite) bad = true;
    } else {
        int sh[2], m[2];
        float fn[2], S0[2][3], DS[2][3];
#pragma unroll
        for (int a = 0; a < 2; ++a)
            finite &= em_move_axis(f[a], vn[a] * g.dtdx[a], &sh[a], &m[a], &fn[a], S0[a], DS[a]);
        if (!finite) {
            bad = true;
            return;
        }
        const int cn[2] = {wrapi(c[0] + sh[0], n0), wrapi(c[1] + sh[1], n1)};
        const int base[2] = {c[0] + m[0], c[1] + m[1]};
        // Esirkepov current on the 3 x 3 stencil, in units of the weights (scaled at
        // conversion); Jx on the two x edges of each row, Jy on the two y edges of
        // each column (the third is zero: the shape changes sum to zero)
#pragma unroll
        for (int bq = 0; bq < 3; ++bq) {
            const int jj = wrapi(base[1] + bq, n1);
            float run = 0.0f;
#pragma unroll
            for (int aq = 0; aq < 2; ++aq) {
                run += DS[0][aq] * (S0[1][bq] + 0.5f * DS[1][bq]);
                add_fx_unit(em.J + wrapi(base[0] + aq, n0) + (int64_t)n0 * jj, run);
            }
        }
#pragma unroll
        for (int aq = 0; aq < 3; ++aq) {
            const int ii = wrapi(base[0] + aq, n0);
            float run = 0.0f;
#pragma unroll
            for (int bq = 0; bq < 2; ++bq) {
                run += DS[1][bq] * (S0[0][aq] + 0.5f * DS[0][aq]);
                add_fx_unit(em.J + cells + ii + (int64_t)n0 * wrapi(base[1] + bq, n1), run);
            }
        }
#pragma unroll
        for (int bq = 0; bq < 3; ++bq)
#pragma unroll
            for (int aq = 0; aq < 3; ++aq) {
                const float wz = esirkepov_wz(S0, DS, aq, bq);
                if (wz != 0.0f)
                    add_fx(em.J + 2 * cells + wrapi(base[0] + aq, n0) +
                               (int64_t)n0 * wrapi(base[1] + bq, n1),
                           vn[2] * wz);
            }
        // charge at the new position (int64 fixed point, exact total)
        const float wx[2] = {1.0f - fn[0], fn[0]}, wy[2] = {1.0f - fn[1], fn[1]};
        int qk[4], rest = one;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            qk[k] = __float_as_int(fmaf(wx[k & 1] * wy[k >> 1], scale, RND_MAGIC_F)) - RND_MAGIC_I;
            rest -= qk[k];
        }
        qk[3] = rest;
        const int x1 = cn[0] + 1 == n0 ? 0 : cn[0] + 1, y1 = cn[1] + 1 == n1 ? 0 : cn[1] + 1;
        const int64_t nodes[4] = {cn[0] + (int64_t)n0 * cn[1], x1 + (int64_t)n0 * cn[1],
                                  cn[0] + (int64_t)n0 * y1, x1 + (int64_t)n0 * y1};
#pragma unroll
        for (int k = 0; k < 4; ++k)
            atomicAdd(rho_acc + nodes[k], (unsigned long long)(long long)qk[k]);
        p.cell[i] = cn[0] + n0 * cn[1];
        p.off[i] = fn[0];
        p.off[p.stride + i] = fn[1];
    }
}

// The load's backward half push: every particle, global fields, no move.
__global__ void __launch_bounds__(EM_THREADS)
    k_em_half_push(GridParams g, ParticlesF32 p, EmBufs em, int *__restrict__ err)
{
    float ke = 0.0f, mom[3] = {0.0f, 0.0f, 0.0f};
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * EM_THREADS + threadIdx.x; i < p.np;
         i += (int64_t)gridDim.x * EM_THREADS)
        em_particle_global<false>(i, g, p, em, nullptr, 0.0f, 0, ke, mom, bad);
    if (bad) atomicOr(err, EF_NONFINITE);
}

// The particle part of a step, tile by tile (EMT_TILE consecutive particles, one per
// thread; persistent CTAs take tiles blockIdx.x, + gridDim.x, ...).  The particles
// of a tile were sorted by cell, so their old cells fill a small box; the stencils
// of the gather (cells c - 1 .. c + 1) and of the current and charge (c - 1 .. c + 2)
// then lie in the box widened by one cell below and two above.  When that window
// fits EMW_CAP nodes, the CTA copies the six field components of the window into
// shared memory, gathers from there, and accumulates Jx, Jy, Jz and the charge in
// int32 windows with shared atomics; every touched node then goes to the int64
// global accumulators once.  A tile whose window does not fit is flagged and left
// for k_em_spread.
//
// Overflow bounds of the int32 windows (256 particles per tile): |Jx|, |Jy| weights
// <= 1 and charge quanta <= 2^22 + 2 per particle and node give |sum| < 2^31; a Jz
// quantum at or above 2^22 (|vz W_z| >= 1) goes straight to global memory.
constexpr int EMT_TILE = EM_PASS_TILE;
constexpr int EMW_CAP = 1024;
static_assert(EMT_TILE == EM_THREADS, "one particle per thread");

__global__ void __launch_bounds__(EM_THREADS)
    k_em_tile(GridParams g, ParticlesF32 p, EmBufs em, unsigned long long *__restrict__ rho_acc,
              double *__restrict__ diag_blocks, int *__restrict__ err)
{
    __shared__ float s_f[6][EMW_CAP];  // Ex, Ey, Ez, Bx, By, Bz of the window
    __shared__ int s_j[4][EMW_CAP];    // Jx, Jy, Jz, charge quanta (zero between tiles)
    __shared__ int s_box[2][4];        // per tile parity: min d0, min d1, max d0, max d1
    const int n0 = g.n[0], n1 = g.n[1];
    const int64_t cells = (int64_t)n0 * n1;
    const int tid = threadIdx.x, lane = tid & 31;
    for (int k = tid; k < 4 * EMW_CAP; k += EM_THREADS) (&s_j[0][0])[k] = 0;
    if (tid < 8) (&s_box[0][0])[tid] = (tid & 3) < 2 ? 0x7fffffff : -0x7fffffff;
    __syncthreads();
    const float scale = ldexpf(1.0f, g.fx_bits);
    const int one = 1 << g.fx_bits;
    float ke = 0.0f, mom[3] = {0.0f, 0.0f, 0.0f};
    bool bad = false;
    const int64_t ntiles = (p.np + EMT_TILE - 1) / EMT_TILE;
    int par = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, par ^= 1) {
        // a warp's lanes take four rows of 32 of the tile (lane i: column i of row
        // (w + i mod 4) mod 8), so its window atomics spread over more nodes; lanes
        // of one row share cells, whose window reads are broadcasts
        const int64_t i = t * EMT_TILE + 32 * (((tid >> 5) + (lane & 3)) & 7) + lane;
        const bool valid = i < p.np;
        // reference cell: the tile's first particle's; d = old cell - reference,
        // unwrapped to [-n/2, n/2] per axis
        const int ref = p.cell[t * EMT_TILE];
        int rc[2];
        rc[1] = (int)fdiv((uint32_t)ref, g.div0);
        rc[0] = ref - rc[1] * n0;
        int c[2] = {0, 0}, d[2] = {0, 0};
        float f[2] = {0.0f, 0.0f}, v[3] = {0.0f, 0.0f, 0.0f};
        if (valid) {
            const int cell = p.cell[i];
            c[1] = (int)fdiv((uint32_t)cell, g.div0);
            c[0] = cell - c[1] * n0;
            f[0] = p.off[i];
            f[1] = p.off[p.stride + i];
#pragma unroll
            for (int a = 0; a < 3; ++a) v[a] = p.v[a * p.stride + i];
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                int dd = c[a] - rc[a];
                dd -= (2 * dd > g.n[a]) ? g.n[a] : 0;
                dd += (2 * dd < -g.n[a]) ? g.n[a] : 0;
                d[a] = dd;
            }
        }
        int *box = s_box[par];
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const int wl = __reduce_min_sync(0xffffffffu, valid ? d[a] : 0x7fffffff);
            const int wh = __reduce_max_sync(0xffffffffu, valid ? d[a] : -0x7fffffff);
            if (lane == 0) {
                atomicMin(&box[a], wl);
                atomicMax(&box[2 + a], wh);
            }
        }
        __syncthreads();
        const int lo0 = box[0], lo1 = box[1];
        const int W0 = box[2] - lo0 + 4, W1 = box[3] - lo1 + 4;
        if (W0 > EMW_CAP || W1 > EMW_CAP || W0 * W1 > EMW_CAP) {
            if (tid == 0) em.tile_flag[t] = 1;
            __syncthreads();  // every thread has read the box
            if (tid < 4) box[tid] = tid < 2 ? 0x7fffffff : -0x7fffffff;
            continue;
        }
        if (tid == 0) em.tile_flag[t] = 0;
        // local window node (lx, ly), index ly W0 + lx, is global node
        // (g0 + lx, g1 + ly) mod n; the fill and the flush walk it by rows (a warp per
        // row, lanes along x)
        const int g0 = rc[0] + lo0 - 1, g1 = rc[1] + lo1 - 1;
        const int warp = tid >> 5;
        auto global_node = [&](int l) -> int64_t {
            const int ly = l / W0, lx = l - ly * W0;
            return wrap_any(g0 + lx, n0) + (int64_t)n0 * wrap_any(g1 + ly, n1);
        };
        for (int ly = warp; ly < W1; ly += EM_THREADS / 32) {
            const int64_t row = (int64_t)n0 * wrap_any(g1 + ly, n1);
            for (int lx = lane; lx < W0; lx += 32) {
                const int64_t gid = row + wrap_any(g0 + lx, n0);
                const int l = ly * W0 + lx;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    s_f[k][l] = __ldg(em.E + k * cells + gid);
                    s_f[3 + k][l] = __ldg(em.B + k * cells + gid);
                }
            }
        }
        __syncthreads();
        if (valid) {
            // the old cell's local coordinates, and the staggered gathers from the window
            const int L0 = d[0] - lo0 + 1, L1 = d[1] - lo1 + 1;
            const bool hx = f[0] >= 0.5f, hy = f[1] >= 0.5f;
            const int ixh = hx ? L0 : L0 - 1, iyh = hy ? L1 : L1 - 1;
            const float fxh = hx ? f[0] - 0.5f : f[0] + 0.5f;
            const float fyh = hy ? f[1] - 0.5f : f[1] + 0.5f;
            auto cic = [&](int k, int ix, float fx, int iy, float fy) {
                const float *F = s_f[k] + ix + iy * W0;
                return (1.0f - fy) * ((1.0f - fx) * F[0] + fx * F[1]) +
                       fy * ((1.0f - fx) * F[W0] + fx * F[W0 + 1]);
            };
            float e[3], b[3];
            e[0] = cic(0, ixh, fxh, L1, f[1]);
            e[1] = cic(1, L0, f[0], iyh, fyh);
            e[2] = cic(2, L0, f[0], L1, f[1]);
            b[0] = cic(3, L0, f[0], iyh, fyh) + em.B0[0];
            b[1] = cic(4, ixh, fxh, L1, f[1]) + em.B0[1];
            b[2] = cic(5, ixh, fxh, iyh, fyh) + em.B0[2];
#pragma unroll
            for (int a = 0; a < 3; ++a) e[a] += g.E0[a];
            float vn[3];
            em_boris(v, e, b, g, vn);
            bool finite = isfinite(vn[0]) && isfinite(vn[1]) && isfinite(vn[2]);
            float o2 = 0.0f, n2 = 0.0f;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                o2 += v[a] * v[a];
                n2 += vn[a] * vn[a];
                mom[a] += vn[a];
                p.v[a * p.stride + i] = vn[a];
            }
            ke += 0.5f * (o2 + n2);
            int sh[2], m[2];
            float fn[2], S0[2][3], DS[2][3];
#pragma unroll
            for (int a = 0; a < 2; ++a)
                finite &= em_move_axis(f[a], vn[a] * g.dtdx[a], &sh[a], &m[a], &fn[a], S0[a],
                                       DS[a]);
            if (!finite) {
                bad = true;
            } else {
                // the stencil's lower corner (old cell + m) in window coordinates
                const int B0i = L0 + m[0], B1i = L1 + m[1];
#pragma unroll
                for (int bq = 0; bq < 3; ++bq) {
                    int *row = s_j[0] + (B1i + bq) * W0 + B0i;
                    float run = 0.0f;
#pragma unroll
                    for (int aq = 0; aq < 2; ++aq) {
                        run += DS[0][aq] * (S0[1][bq] + 0.5f * DS[1][bq]);
                        const int q = __float_as_int(fmaf(run, J_SCALE, RND_MAGIC_F)) - RND_MAGIC_I;
                        if (q) atomicAdd(row + aq, q);
                    }
                }
#pragma unroll
                for (int aq = 0; aq < 3; ++aq) {
                    int *col = s_j[1] + B1i * W0 + B0i + aq;
                    float run = 0.0f;
#pragma unroll
                    for (int bq = 0; bq < 2; ++bq) {
                        run += DS[1][bq] * (S0[0][aq] + 0.5f * DS[0][aq]);
                        const int q = __float_as_int(fmaf(run, J_SCALE, RND_MAGIC_F)) - RND_MAGIC_I;
                        if (q) atomicAdd(col + bq * W0, q);
                    }
                }
                const float vz_scaled = vn[2] * J_SCALE;  // exact: a power-of-two scale
#pragma unroll
                for (int bq = 0; bq < 3; ++bq)
#pragma unroll
                    for (int aq = 0; aq < 3; ++aq) {
                        const float y = vz_scaled * esirkepov_wz(S0, DS, aq, bq);
                        const int l = (B1i + bq) * W0 + B0i + aq;
                        if (fabsf(y) < J_SCALE) {
                            const int q = __float_as_int(y + RND_MAGIC_F) - RND_MAGIC_I;
                            if (q) atomicAdd(s_j[2] + l, q);
                        } else {
                            atomicAdd(em.J + 2 * cells + global_node(l),
                                      (unsigned long long)__float2ll_rn(y));
                        }
                    }
                // charge at the new position
                const float wx[2] = {1.0f - fn[0], fn[0]}, wy[2] = {1.0f - fn[1], fn[1]};
                int qk[4], rest = one;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    qk[k] = __float_as_int(fmaf(wx[k & 1] * wy[k >> 1], scale, RND_MAGIC_F)) -
                            RND_MAGIC_I;
                    rest -= qk[k];
                }
                qk[3] = rest;
                int *q0 = s_j[3] + (L1 + sh[1]) * W0 + L0 + sh[0];
                atomicAdd(q0, qk[0]);
                atomicAdd(q0 + 1, qk[1]);
                atomicAdd(q0 + W0, qk[2]);
                atomicAdd(q0 + W0 + 1, qk[3]);
                const int cn0 = wrapi(c[0] + sh[0], n0), cn1 = wrapi(c[1] + sh[1], n1);
                p.cell[i] = cn0 + n0 * cn1;
                p.off[i] = fn[0];
                p.off[p.stride + i] = fn[1];
            }
        }
        __syncthreads();
        // flush: every touched node once to the int64 accumulators, leaving zeros
        for (int ly = warp; ly < W1; ly += EM_THREADS / 32)
            for (int lx = lane; lx < W0; lx += 32) {
            const int l = ly * W0 + lx;
            const int qx = s_j[0][l], qy = s_j[1][l], qz = s_j[2][l], qr = s_j[3][l];
            if ((qx | qy | qz | qr) == 0) continue;
            const int64_t gid = wrap_any(g0 + lx, n0) + (int64_t)n0 * wrap_any(g1 + ly, n1);
            if (qx) {
                s_j[0][l] = 0;
                atomicAdd(em.J + gid, (unsigned long long)(long long)qx);
            }
            if (qy) {
                s_j[1][l] = 0;
                atomicAdd(em.J + cells + gid, (unsigned long long)(long long)qy);
            }
            if (qz) {
                s_j[2][l] = 0;
                atomicAdd(em.J + 2 * cells + gid, (unsigned long long)(long long)qz);
            }
            if (qr) {
                s_j[3][l] = 0;
                atomicAdd(rho_acc + gid, (unsigned long long)(long long)qr);
            }
            }
        // reset this parity's box (read by all before the barrier above); it is next
        // used two tiles on, after the next tile's barriers
        if (tid < 4) box[tid] = tid < 2 ? 0x7fffffff : -0x7fffffff;
    }
    if (bad) atomicOr(err, EF_NONFINITE);
    if (diag_blocks) em_block_diag(ke, mom, diag_blocks, blockIdx.x);
}

// The tiles that k_em_tile flagged, particle by particle through global memory.  A
// block reads the flags of EM_THREADS consecutive tiles at once (one per thread) and
// then takes the flagged ones in order; every block writes its diagnostic partials
// (slot gridDim.x + blockIdx.x).
__global__ void __launch_bounds__(EM_THREADS)
    k_em_spread(GridParams g, ParticlesF32 p, EmBufs em, unsigned long long *__restrict__ rho_acc,
                double *__restrict__ diag_blocks, int *__restrict__ err)
{
    __shared__ unsigned char s_flag[EM_THREADS];
    const float scale = ldexpf(1.0f, g.fx_bits);
    const int one = 1 << g.fx_bits;
    float ke = 0.0f, mom[3] = {0.0f, 0.0f, 0.0f};
    bool bad = false;
    const int64_t ntiles = (p.np + EMT_TILE - 1) / EMT_TILE;
    for (int64_t t0 = (int64_t)blockIdx.x * EM_THREADS; t0 < ntiles;
         t0 += (int64_t)gridDim.x * EM_THREADS) {
        const int64_t tt = t0 + threadIdx.x;
        const bool mine = tt < ntiles && em.tile_flag[tt];
        s_flag[threadIdx.x] = mine ? 1 : 0;
        if (!__syncthreads_or(mine)) continue;
        for (int q = 0; q < EM_THREADS; ++q) {
            if (!s_flag[q]) continue;
            const int64_t i = (t0 + q) * EMT_TILE + threadIdx.x;
            if (i < p.np) em_particle_global<true>(i, g, p, em, rho_acc, scale, one, ke, mom, bad);
        }
        __syncthreads();  // s_flag is rewritten for the next chunk
    }
    if (bad) atomicOr(err, EF_NONFINITE);
    if (diag_blocks) em_block_diag(ke, mom, diag_blocks, gridDim.x + blockIdx.x);
}

// Node coordinates of a flat index.
__device__ __forceinline__ void coords2(int64_t id, const GridParams &g, int *i, int *j)
{
    *j = (int)fdiv((uint32_t)id, g.div0);
    *i = (int)id - *j * g.n[0];
}

__global__ void __launch_bounds__(EM_THREADS)
    k_yee_b(GridParams g, const float *__restrict__ E, float *__restrict__ B, float hdx,
            float hdy)
{
    const int n0 = g.n[0], n1 = g.n[1];
    const int64_t cells = (int64_t)n0 * n1;
    for (int64_t id = (int64_t)blockIdx.x * EM_THREADS + threadIdx.x; id < cells;
         id += (int64_t)gridDim.x * EM_THREADS) {
        int i, j;
        coords2(id, g, &i, &j);
        const int64_t ip = (i + 1 == n0 ? 0 : i + 1) + (int64_t)n0 * j;
        const int64_t jp = i + (int64_t)n0 * (j + 1 == n1 ? 0 : j + 1);
        const float ez = E[2 * cells + id];
        B[id] -= hdy * (E[2 * cells + jp] - ez);
        B[cells + id] += hdx * (E[2 * cells + ip] - ez);
        B[2 * cells + id] -= hdx * (E[cells + ip] - E[cells + id]) - hdy * (E[jp] - E[id]);
    }
}

__global__ void __launch_bounds__(EM_THREADS)
    k_yee_e(GridParams g, const float *__restrict__ B, JTake jt, float *__restrict__ E,
            float c2dtdx, float c2dtdy, float dt)
{
    const int n0 = g.n[0], n1 = g.n[1];
    const int64_t cells = (int64_t)n0 * n1;
    for (int64_t id = (int64_t)blockIdx.x * EM_THREADS + threadIdx.x; id < cells;
         id += (int64_t)gridDim.x * EM_THREADS) {
        int i, j;
        coords2(id, g, &i, &j);
        const int64_t im = (i == 0 ? n0 - 1 : i - 1) + (int64_t)n0 * j;
        const int64_t jm = i + (int64_t)n0 * (j == 0 ? n1 - 1 : j - 1);
        const float bz = B[2 * cells + id];
        float J[3];
        get_j(jt, cells, id, J);
        E[id] += c2dtdy * (bz - B[2 * cells + jm]) - dt * J[0];
        E[cells + id] += -c2dtdx * (bz - B[2 * cells + im]) - dt * J[1];
        E[2 * cells + id] += c2dtdx * (B[cells + id] - B[cells + im]) -
                             c2dtdy * (B[id] - B[jm]) - dt * J[2];
        clear_j(jt, cells, id);
    }
}

// ---- convolutional PML on a non-periodic grid (Roden and Gedney) ----------------------------
// Values outside the grid count as zero; inside the layers every derivative d/da
// becomes (1/kappa_a) d/da + psi with psi <- b psi + c dF/da; the tangential E on the
// outer nodes is held at zero (a conducting wall behind the layer).

__device__ __forceinline__ float at_or_zero(const float *F, int n0, int n1, int i, int j)
{
    return (i < 0 || j < 0 || i >= n0 || j >= n1) ? 0.0f : F[i + (int64_t)n0 * j];
}

__global__ void __launch_bounds__(EM_THREADS)
    k_cpml_b(GridParams g, EmBufs em, float h, float idx, float idy)
{
    const int n0 = g.n[0], n1 = g.n[1];
    const int64_t cells = (int64_t)n0 * n1;
    const float *Ex = em.E, *Ey = em.E + cells, *Ez = em.E + 2 * cells;
    float *Bx = em.B, *By = em.B + cells, *Bz = em.B + 2 * cells;
    for (int64_t id = (int64_t)blockIdx.x * EM_THREADS + threadIdx.x; id < cells;
         id += (int64_t)gridDim.x * EM_THREADS) {
        int i, j;
        coords2(id, g, &i, &j);
        const float dyEz = (at_or_zero(Ez, n0, n1, i, j + 1) - Ez[id]) * idy;
        const float dxEz = (at_or_zero(Ez, n0, n1, i + 1, j) - Ez[id]) * idx;
        const float dxEy = (at_or_zero(Ey, n0, n1, i + 1, j) - Ey[id]) * idx;
        const float dyEx = (at_or_zero(Ex, n0, n1, i, j + 1) - Ex[id]) * idy;
        // outside the layer along an axis (b = 1, c = 0) psi stays zero: it is neither
        // read nor written there
        float p0 = 0.0f, p1 = 0.0f, p2 = 0.0f, p3 = 0.0f;
        if (em.pb[4][j] != 0.0f || em.pb[3][j] != 1.0f) {
            p0 = em.pb[3][j] * em.psib[0][id] + em.pb[4][j] * dyEz;
            p3 = em.pb[3][j] * em.psib[3][id] + em.pb[4][j] * dyEx;
            em.psib[0][id] = p0;
            em.psib[3][id] = p3;
        }
        if (em.pb[1][i] != 0.0f || em.pb[0][i] != 1.0f) {
            p1 = em.pb[0][i] * em.psib[1][id] + em.pb[1][i] * dxEz;
            p2 = em.pb[0][i] * em.psib[2][id] + em.pb[1][i] * dxEy;
            em.psib[1][id] = p1;
            em.psib[2][id] = p2;
        }
        Bx[id] -= h * (em.pb[5][j] * dyEz + p0);
        By[id] += h * (em.pb[2][i] * dxEz + p1);
        Bz[id] -= h * ((em.pb[2][i] * dxEy + p2) - (em.pb[5][j] * dyEx + p3));
    }
}

__global__ void __launch_bounds__(EM_THREADS)
    k_cpml_e(GridParams g, EmBufs em, JTake jt, float c2, float dt, float idx, float idy)
{
    const int n0 = g.n[0], n1 = g.n[1];
    const int64_t cells = (int64_t)n0 * n1;
    const float *Bx = em.B, *By = em.B + cells, *Bz = em.B + 2 * cells;
    float *Ex = em.E, *Ey = em.E + cells, *Ez = em.E + 2 * cells;
    for (int64_t id = (int64_t)blockIdx.x * EM_THREADS + threadIdx.x; id < cells;
         id += (int64_t)gridDim.x * EM_THREADS) {
        int i, j;
        coords2(id, g, &i, &j);
        const float dyBz = (Bz[id] - at_or_zero(Bz, n0, n1, i, j - 1)) * idy;
        const float dxBz = (Bz[id] - at_or_zero(Bz, n0, n1, i - 1, j)) * idx;
        const float dxBy = (By[id] - at_or_zero(By, n0, n1, i - 1, j)) * idx;
        const float dyBx = (Bx[id] - at_or_zero(Bx, n0, n1, i, j - 1)) * idy;
        float p0 = 0.0f, p1 = 0.0f, p2 = 0.0f, p3 = 0.0f;  // zero outside the layer
        if (em.pe[4][j] != 0.0f || em.pe[3][j] != 1.0f) {
            p0 = em.pe[3][j] * em.psie[0][id] + em.pe[4][j] * dyBz;
            p3 = em.pe[3][j] * em.psie[3][id] + em.pe[4][j] * dyBx;
            em.psie[0][id] = p0;
            em.psie[3][id] = p3;
        }
        if (em.pe[1][i] != 0.0f || em.pe[0][i] != 1.0f) {
            p1 = em.pe[0][i] * em.psie[1][id] + em.pe[1][i] * dxBz;
            p2 = em.pe[0][i] * em.psie[2][id] + em.pe[1][i] * dxBy;
            em.psie[1][id] = p1;
            em.psie[2][id] = p2;
        }
        const bool xb = i == 0 || i == n0 - 1, yb = j == 0 || j == n1 - 1;
        float J[3];
        get_j(jt, cells, id, J);
        const float ex = Ex[id] + dt * (c2 * (em.pe[5][j] * dyBz + p0) - J[0]);
        const float ey = Ey[id] + dt * (-c2 * (em.pe[2][i] * dxBz + p1) - J[1]);
        const float ez = Ez[id] + dt * (c2 * ((em.pe[2][i] * dxBy + p2) - (em.pe[5][j] * dyBx + p3)) -
                                        J[2]);
        Ex[id] = (yb || i == n0 - 1) ? 0.0f : ex;
        Ey[id] = (xb || j == n1 - 1) ? 0.0f : ey;
        Ez[id] = (xb || yb) ? 0.0f : ez;
        clear_j(jt, cells, id);
    }
}

// ---- particles in the non-periodic mode (absorbing layer and conducting walls) ------------
// Particles live in cells 0 .. n_a - 2 of each axis, between the walls on the outer
// nodes.  Gathers, current and charge take the periodic forms with the nodes outside
// the grid left out: a field there counts as zero and a contribution to it is
// dropped.  A particle whose move leaves the box deposits the current of its whole
// move and is then absorbed: its cell becomes -1 (every kernel skips it; the next sort
// moves it past the live particles, where it is dropped) and it is counted.

// Lower lattice index (possibly -1) and fraction on a non-periodic axis.
__device__ __forceinline__ void stagger_np(int c, float f, bool half, int *i0, float *fr)
{
    if (!half) {
        *i0 = c;
        *fr = f;
    } else if (f >= 0.5f) {
        *i0 = c;
        *fr = f - 0.5f;
    } else {
        *i0 = c - 1;
        *fr = f + 0.5f;
    }
}

__device__ __forceinline__ float lattice_cic_np(const float *__restrict__ F, int n0, int n1, int i0,
                                                float fx, int j0, float fy)
{
    return (1.0f - fy) * ((1.0f - fx) * at_or_zero(F, n0, n1, i0, j0) +
                          fx * at_or_zero(F, n0, n1, i0 + 1, j0)) +
           fy * ((1.0f - fx) * at_or_zero(F, n0, n1, i0, j0 + 1) +
                 fx * at_or_zero(F, n0, n1, i0 + 1, j0 + 1));
}

__device__ __forceinline__ bool inside(int n0, int n1, int i, int j)
{
    return i >= 0 && j >= 0 && i < n0 && j < n1;
}

template <bool MOVE>
__global__ void __launch_bounds__(EM_THREADS)
    k_em_np_push(GridParams g, ParticlesF32 p, EmBufs em, unsigned long long *__restrict__ rho_acc,
                 double *__restrict__ diag_blocks, int *__restrict__ err,
                 unsigned long long *__restrict__ n_absorbed)
{
    const int n0 = g.n[0], n1 = g.n[1];
    const int64_t cells = (int64_t)n0 * n1;
    const float scale = ldexpf(1.0f, g.fx_bits);
    const int one = 1 << g.fx_bits;
    float ke = 0.0f, mom[3] = {0.0f, 0.0f, 0.0f};
    bool bad = false;
    unsigned gone = 0;
    for (int64_t i = (int64_t)blockIdx.x * EM_THREADS + threadIdx.x; i < p.np;
         i += (int64_t)gridDim.x * EM_THREADS) {
        const int cell = p.cell[i];
        if (cell < 0) continue;  // absorbed in an earlier step
        int c[2];
        c[1] = (int)fdiv((uint32_t)cell, g.div0);
        c[0] = cell - c[1] * n0;
        const float f[2] = {p.off[i], p.off[p.stride + i]};
        const float v[3] = {p.v[i], p.v[p.stride + i], p.v[2 * p.stride + i]};
        int ix[2], iy[2];
        float fx[2], fy[2];
        stagger_np(c[0], f[0], false, &ix[0], &fx[0]);
        stagger_np(c[0], f[0], true, &ix[1], &fx[1]);
        stagger_np(c[1], f[1], false, &iy[0], &fy[0]);
        stagger_np(c[1], f[1], true, &iy[1], &fy[1]);
        float e[3], b[3];
        e[0] = lattice_cic_np(em.E, n0, n1, ix[1], fx[1], iy[0], fy[0]) + g.E0[0];
        e[1] = lattice_cic_np(em.E + cells, n0, n1, ix[0], fx[0], iy[1], fy[1]) + g.E0[1];
        e[2] = lattice_cic_np(em.E + 2 * cells, n0, n1, ix[0], fx[0], iy[0], fy[0]) + g.E0[2];
        b[0] = lattice_cic_np(em.B, n0, n1, ix[0], fx[0], iy[1], fy[1]) + em.B0[0];
        b[1] = lattice_cic_np(em.B + cells, n0, n1, ix[1], fx[1], iy[0], fy[0]) + em.B0[1];
        b[2] = lattice_cic_np(em.B + 2 * cells, n0, n1, ix[1], fx[1], iy[1], fy[1]) + em.B0[2];
        float vn[3];
        em_boris(v, e, b, g, vn);
        bool finite = isfinite(vn[0]) && isfinite(vn[1]) && isfinite(vn[2]);
        float o2 = 0.0f, n2 = 0.0f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            o2 += v[a] * v[a];
            n2 += vn[a] * vn[a];
            mom[a] += vn[a];
            p.v[a * p.stride + i] = vn[a];
        }
        ke += 0.5f * (o2 + n2);
        if constexpr (!MOVE) {
            if (!finite) bad = true;
        } else {
            int sh[2], m[2];
            float fn[2], S0[2][3], DS[2][3];
#pragma unroll
            for (int a = 0; a < 2; ++a)
                finite &= em_move_axis(f[a], vn[a] * g.dtdx[a], &sh[a], &m[a], &fn[a], S0[a], DS[a]);
            if (!finite) {
                bad = true;
                continue;
            }
            const int base[2] = {c[0] + m[0], c[1] + m[1]};
            // the Esirkepov current of the whole move, nodes outside the grid dropped
#pragma unroll
            for (int bq = 0; bq < 3; ++bq) {
                float run = 0.0f;
#pragma unroll
                for (int aq = 0; aq < 2; ++aq) {
                    run += DS[0][aq] * (S0[1][bq] + 0.5f * DS[1][bq]);
                    if (inside(n0, n1, base[0] + aq, base[1] + bq))
                        add_fx_unit(em.J + (base[0] + aq) + (int64_t)n0 * (base[1] + bq), run);
                }
            }
#pragma unroll
            for (int aq = 0; aq < 3; ++aq) {
                float run = 0.0f;
#pragma unroll
                for (int bq = 0; bq < 2; ++bq) {
                    run += DS[1][bq] * (S0[0][aq] + 0.5f * DS[0][aq]);
                    if (inside(n0, n1, base[0] + aq, base[1] + bq))
                        add_fx_unit(em.J + cells + (base[0] + aq) + (int64_t)n0 * (base[1] + bq),
                                    run);
                }
            }
#pragma unroll
            for (int bq = 0; bq < 3; ++bq)
#pragma unroll
                for (int aq = 0; aq < 3; ++aq) {
                    const float wz = esirkepov_wz(S0, DS, aq, bq);
                    if (wz != 0.0f && inside(n0, n1, base[0] + aq, base[1] + bq))
                        add_fx(em.J + 2 * cells + (base[0] + aq) + (int64_t)n0 * (base[1] + bq),
                               vn[2] * wz);
                }
            const int cn[2] = {c[0] + sh[0], c[1] + sh[1]};
            if (cn[0] < 0 || cn[1] < 0 || cn[0] > n0 - 2 || cn[1] > n1 - 2) {
                // left the box: absorbed (its current is in; no charge)
                p.cell[i] = -1;
                ++gone;
                continue;
            }
            // charge at the new position (all four nodes inside the grid)
            const float wx[2] = {1.0f - fn[0], fn[0]}, wy[2] = {1.0f - fn[1], fn[1]};
            int qk[4], rest = one;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                qk[k] = __float_as_int(fmaf(wx[k & 1] * wy[k >> 1], scale, RND_MAGIC_F)) -
                        RND_MAGIC_I;
                rest -= qk[k];
            }
            qk[3] = rest;
            const int64_t n00 = cn[0] + (int64_t)n0 * cn[1];
            atomicAdd(rho_acc + n00, (unsigned long long)(long long)qk[0]);
            atomicAdd(rho_acc + n00 + 1, (unsigned long long)(long long)qk[1]);
            atomicAdd(rho_acc + n00 + n0, (unsigned long long)(long long)qk[2]);
            atomicAdd(rho_acc + n00 + n0 + 1, (unsigned long long)(long long)qk[3]);
            p.cell[i] = (int)n00;
            p.off[i] = fn[0];
            p.off[p.stride + i] = fn[1];
        }
    }
    if (bad) atomicOr(err, EF_NONFINITE);
    gone = __reduce_add_sync(0xffffffffu, gone);
    if ((threadIdx.x & 31) == 0 && gone) atomicAdd(n_absorbed, (unsigned long long)gone);
    if (diag_blocks) em_block_diag(ke, mom, diag_blocks, blockIdx.x);
}

// Loaded positions must lie in the box between the walls: cells 0 .. n_a - 2.
__global__ void __launch_bounds__(EM_THREADS) k_em_np_check(GridParams g, ParticlesF32 p, int *err)
{
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * EM_THREADS + threadIdx.x; i < p.np;
         i += (int64_t)gridDim.x * EM_THREADS) {
        const int cell = p.cell[i];
        const int c1 = (int)fdiv((uint32_t)cell, g.div0);
        const int c0 = cell - c1 * g.n[0];
        bad |= c0 > g.n[0] - 2 || c1 > g.n[1] - 2;
    }
    if (bad) atomicOr(err, EF_NONFINITE);
}

// Initial field of the load: E = -grad phi by forward differences onto the staggered
// points (so that the discrete div E equals rho), Ez = 0.
__global__ void __launch_bounds__(EM_THREADS)
    k_em_e_from_phi(GridParams g, const float *__restrict__ phi, float *__restrict__ E,
                    float idx, float idy)
{
    const int n0 = g.n[0], n1 = g.n[1];
    const int64_t cells = (int64_t)n0 * n1;
    for (int64_t id = (int64_t)blockIdx.x * EM_THREADS + threadIdx.x; id < cells;
         id += (int64_t)gridDim.x * EM_THREADS) {
        int i, j;
        coords2(id, g, &i, &j);
        const int64_t ip = (i + 1 == n0 ? 0 : i + 1) + (int64_t)n0 * j;
        const int64_t jp = i + (int64_t)n0 * (j + 1 == n1 ? 0 : j + 1);
        E[id] = -(phi[ip] - phi[id]) * idx;
        E[cells + id] = -(phi[jp] - phi[id]) * idy;
        E[2 * cells + id] = 0.0f;
    }
}

// Per-block partials of sum (|E|^2 + c^2 |B|^2) over the nodes (electric plus
// magnetic field energy density, times 2).
__global__ void __launch_bounds__(EM_THREADS)
    k_em_energy(int64_t cells, const float *__restrict__ E, const float *__restrict__ B, float c2,
                double *__restrict__ part)
{
    double s = 0.0;
    for (int64_t id = (int64_t)blockIdx.x * EM_THREADS + threadIdx.x; id < cells;
         id += (int64_t)gridDim.x * EM_THREADS)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double e = E[k * cells + id], b = B[k * cells + id];
            s += e * e + (double)c2 * b * b;
        }
    __shared__ double red[EM_THREADS / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int j = 0; j < EM_THREADS / 32; ++j) t += red[j];
        part[blockIdx.x] = t;
    }
}

int em_blocks(int64_t n)
{
    const int sms = sm_count();
    const int64_t need = (n + EM_THREADS - 1) / EM_THREADS;
    const int64_t cap = (int64_t)sms * 8;
    const int64_t b = need < cap ? need : cap;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

// One resident wave of the tiled particle kernel: the CTAs of k_em_tile that fit an
// SM (occupancy calculator) times the SMs, fewer for small np.
int em_particle_blocks(int64_t np)
{
    static std::atomic<int> per_sm{0};
    int c = per_sm.load(std::memory_order_relaxed);
    if (!c) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, k_em_tile, EM_THREADS, 0) !=
                cudaSuccess ||
            c < 1) {
            cudaGetLastError();
            c = 1;
        }
        per_sm.store(c, std::memory_order_relaxed);
    }
    const int64_t need = (np + EMT_TILE - 1) / EMT_TILE;
    const int64_t cap = (int64_t)sm_count() * c;
    const int64_t b = need < cap ? need : cap;
    return (int)(b < 1 ? 1 : b);
}

cudaError_t launch_em_push(const GridParams &g, ParticlesF32 p, const EmBufs &em, bool move,
                           unsigned long long *rho_acc, double *diag_blocks, int nblocks,
                           int *err, cudaStream_t st)
{
    if (p.np == 0) return cudaSuccess;
    if (!move) {
        k_em_half_push<<<nblocks, EM_THREADS, 0, st>>>(g, p, em, err);
        note_launch();
        return cudaGetLastError();
    }
    // nblocks diagnostic slots: the first half for the tiled kernel, the second for
    // the spread-out tiles
    const int nb = nblocks / 2 > 0 ? nblocks / 2 : 1;
    k_em_tile<<<nb, EM_THREADS, 0, st>>>(g, p, em, rho_acc, diag_blocks, err);
    k_em_spread<<<nb, EM_THREADS, 0, st>>>(g, p, em, rho_acc, diag_blocks, err);
    note_launch(2);
    return cudaGetLastError();
}

JTake em_jtake(const EmBufs &em, double fx, double fy, double fz)
{
    JTake t;
    t.acc = em.J;
    t.ext = em.Jext;
    t.f[0] = (float)fx;
    t.f[1] = (float)fy;
    t.f[2] = (float)fz;
    return t;
}

cudaError_t launch_em_fields(const GridParams &g, const EmBufs &em, double dx, double dy,
                             double dt, double c, double qw, cudaStream_t st)
{
    const int64_t cells = (int64_t)g.n[0] * g.n[1];
    const int nb = em_blocks(cells);
    // J: the accumulated weights times -(qw / (dy dt)), -(qw / (dx dt)), qw / (dx dy),
    // each divided by the fixed-point scale, taken (and cleared) by the E update
    const JTake jt = em_jtake(em, -qw / (dy * dt) / J_SCALE, -qw / (dx * dt) / J_SCALE,
                              qw / (dx * dy) / J_SCALE);
    if (em.pb[0]) {
        // non-periodic grid with the absorbing layer
        const float idx = (float)(1.0 / dx), idy = (float)(1.0 / dy);
        k_cpml_b<<<nb, EM_THREADS, 0, st>>>(g, em, (float)(0.5 * dt), idx, idy);
        k_cpml_e<<<nb, EM_THREADS, 0, st>>>(g, em, jt, (float)(c * c), (float)dt, idx, idy);
        k_cpml_b<<<nb, EM_THREADS, 0, st>>>(g, em, (float)(0.5 * dt), idx, idy);
        note_launch(3);
        return cudaGetLastError();
    }
    const float hdx = (float)(0.5 * dt / dx), hdy = (float)(0.5 * dt / dy);
    k_yee_b<<<nb, EM_THREADS, 0, st>>>(g, em.E, em.B, hdx, hdy);
    k_yee_e<<<nb, EM_THREADS, 0, st>>>(g, em.B, jt, em.E, (float)(c * c * dt / dx),
                                       (float)(c * c * dt / dy), (float)dt);
    k_yee_b<<<nb, EM_THREADS, 0, st>>>(g, em.E, em.B, hdx, hdy);
    note_launch(3);
    return cudaGetLastError();
}

cudaError_t launch_em_e_from_phi(const GridParams &g, const float *phi, const EmBufs &em,
                                 double dx, double dy, cudaStream_t st)
{
    const int64_t cells = (int64_t)g.n[0] * g.n[1];
    k_em_e_from_phi<<<em_blocks(cells), EM_THREADS, 0, st>>>(g, phi, em.E, (float)(1.0 / dx),
                                                            (float)(1.0 / dy));
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_em_np_push(const GridParams &g, ParticlesF32 p, const EmBufs &em, bool move,
                              unsigned long long *rho_acc, double *diag_blocks, int nblocks,
                              int *err, unsigned long long *n_absorbed, cudaStream_t st)
{
    if (p.np == 0) return cudaSuccess;
    const int nb = nblocks > 0 ? nblocks : 1;  // every diagnostic slot is written
    if (move)
        k_em_np_push<true><<<nb, EM_THREADS, 0, st>>>(g, p, em, rho_acc, diag_blocks, err, n_absorbed);
    else
        k_em_np_push<false><<<nb, EM_THREADS, 0, st>>>(g, p, em, rho_acc, diag_blocks, err, n_absorbed);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_em_np_check(const GridParams &g, ParticlesF32 p, int *err, cudaStream_t st)
{
    if (p.np == 0) return cudaSuccess;
    k_em_np_check<<<em_blocks(p.np), EM_THREADS, 0, st>>>(g, p, err);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_em_energy(const EmBufs &em, int64_t cells, double c, double *part, int nblocks,
                             cudaStream_t st)
{
    k_em_energy<<<nblocks, EM_THREADS, 0, st>>>(cells, em.E, em.B, (float)(c * c), part);
    note_launch();
    return cudaGetLastError();
}

}  // namespace apk
