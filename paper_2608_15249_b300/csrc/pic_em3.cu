// pic_em3.cu -- the electromagnetic step (E_Maxwell, Sec. 2.2: finite-difference
// time-domain updates on the Yee lattice) with its particle coupling on a periodic
// 3D grid: the 3D form of pic_em.cu.
//
// Fields at integer times on the 3D Yee lattice, component-major [3][cells], element
// (i, j, k) of a component at ((i + sx) dx, (j + sy) dy, (k + sz) dz):
//   Ex (1/2, 0, 0), Ey (0, 1/2, 0), Ez (0, 0, 1/2);
//   Bx (0, 1/2, 1/2), By (1/2, 0, 1/2), Bz (1/2, 1/2, 0);
// J is staggered like E.  A step: gather E^n, B^n (+ uniform B0) by trilinear CIC on
// each component's lattice, Boris, move (under one cell per axis), the 3D Esirkepov
// current (2001) J^(n+1/2) and the charge at x^(n+1) in int64 fixed point; then
// B -= (dt/2) curl E;  E += dt (c^2 curl B - J);  B -= (dt/2) curl E.
//
// The particle kernel walks tiles of sorted particles, one per thread: fields are
// gathered from global memory (L2-resident), the current and charge of the particles
// inside the tile's fixed shared-memory window are summed there in int32 and flushed
// once per node; the tile's other particles are listed and a second kernel takes them
// through global memory.
#include <atomic>

#include "pic_em_common.cuh"
#include "pic_internal.cuh"

namespace apk {

namespace {

// The six components' lattice offsets: bit a set when component q sits half a cell
// up along axis a (q = Ex, Ey, Ez, Bx, By, Bz: 1, 2, 4, 6, 5, 3), packed 3 bits each.
constexpr unsigned HALF_BITS = 1u | (2u << 3) | (4u << 6) | (6u << 9) | (5u << 12) | (3u << 15);

__device__ __forceinline__ void decode3(int cell, const GridParams &g, int *c)
{
    const int c12 = (int)fdiv((uint32_t)cell, g.div0);
    c[0] = cell - c12 * g.n[0];
    const int c2 = (int)fdiv((uint32_t)c12, g.div1);
    c[1] = c12 - c2 * g.n[1];
    c[2] = c2;
}

__device__ __forceinline__ int64_t node3(const int *n, int i, int j, int k)
{
    return (int64_t)i + (int64_t)n[0] * ((int64_t)j + (int64_t)n[1] * k);
}

// The gather's lattice indices along one axis, as offsets (index times the axis
// stride): lower and upper (periodic) node and the fraction towards the upper one, on
// the integer lattice (h = 0) and on the half lattice (h = 1, nodes at c + 1/2).
struct Axis3 {
    int lo[2], hi[2];
    float fr[2];
};

__device__ __forceinline__ void axis3(int c, float f, int n, int stride, Axis3 &ax)
{
    const int up = c + 1 == n ? 0 : c + 1;
    const int dn = c == 0 ? n - 1 : c - 1;
    const bool upper = f >= 0.5f;
    ax.lo[0] = c * stride;
    ax.hi[0] = up * stride;
    ax.fr[0] = f;
    ax.lo[1] = (upper ? c : dn) * stride;
    ax.hi[1] = (upper ? up : c) * stride;
    ax.fr[1] = upper ? f - 0.5f : f + 0.5f;
}

// Trilinear CIC of component F on the lattice (hx, hy, hz).
__device__ __forceinline__ float cic3(const float *__restrict__ F, const Axis3 *ax, int hx, int hy,
                                      int hz)
{
    const float fx = ax[0].fr[hx];
    float s = 0.0f;
#pragma unroll
    for (int bk = 0; bk < 2; ++bk) {
        const float wz = bk ? ax[2].fr[hz] : 1.0f - ax[2].fr[hz];
        const int zo = bk ? ax[2].hi[hz] : ax[2].lo[hz];
#pragma unroll
        for (int bj = 0; bj < 2; ++bj) {
            const float wy = bj ? ax[1].fr[hy] : 1.0f - ax[1].fr[hy];
            const float *row = F + (zo + (bj ? ax[1].hi[hy] : ax[1].lo[hy]));
            s += wz * wy * ((1.0f - fx) * __ldg(row + ax[0].lo[hx]) + fx * __ldg(row + ax[0].hi[hx]));
        }
    }
    return s;
}

// E and B (without the external fields) at a particle in cell c, offsets f: each of
// the six components by trilinear CIC on its own lattice.
__device__ __forceinline__ void em3_gather(const int *c, const float *f, const int *n,
                                           const EmBufs &em, int64_t cells, float *e, float *b)
{
    Axis3 ax[3];
    axis3(c[0], f[0], n[0], 1, ax[0]);
    axis3(c[1], f[1], n[1], n[0], ax[1]);
    axis3(c[2], f[2], n[2], n[0] * n[1], ax[2]);
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const int hx = (HALF_BITS >> (3 * q)) & 1, hy = (HALF_BITS >> (3 * q + 1)) & 1,
                  hz = (HALF_BITS >> (3 * q + 2)) & 1;
        const float val = cic3((q < 3 ? em.E : em.B) + (q % 3) * cells, ax, hx, hy, hz);
        if (q < 3) e[q] = val;
        else b[q - 3] = val;
    }
}

// Weight of the 3D Esirkepov current along axis a at the transverse node (kb, kc) of
// the stencil: S0_b S0_c + DS_b S0_c / 2 + S0_b DS_c / 2 + DS_b DS_c / 3; the current
// on the a-edges is DS_a times it, summed along a (the third edge gets zero: the
// shape changes along a sum to zero); |J| <= 1 per node.
__device__ __forceinline__ float esirkepov_perp(const float (*S0)[3], const float (*DS)[3], int b1,
                                                int kb, int b2, int kc)
{
    return S0[b1][kb] * (S0[b2][kc] + 0.5f * DS[b2][kc]) +
           DS[b1][kb] * (0.5f * S0[b2][kc] + DS[b2][kc] * (1.0f / 3.0f));
}

// Current and charge of one moved particle straight to the global accumulators:
// the stencil's lower corner is old cell + m, the new cell cn; every index wraps.
__device__ __forceinline__ void em3_deposit_global(const int *n, int64_t cells, const int *c,
                                                   const int *m, const int *cn,
                                                   const float (*S0)[3], const float (*DS)[3],
                                                   const int *qk, unsigned long long *__restrict__ J,
                                                   unsigned long long *__restrict__ rho_acc)
{
    int base[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) base[a] = c[a] + m[a];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int b1 = (a + 1) % 3, b2 = (a + 2) % 3;
#pragma unroll
        for (int kc = 0; kc < 3; ++kc)
#pragma unroll
            for (int kb = 0; kb < 3; ++kb) {
                const float perp = esirkepov_perp(S0, DS, b1, kb, b2, kc);
                if (perp == 0.0f) continue;
                float run = 0.0f;
#pragma unroll
                for (int ka = 0; ka < 2; ++ka) {
                    run += DS[a][ka] * perp;
                    int idx[3];
                    idx[a] = wrapi(base[a] + ka, n[a]);
                    idx[b1] = wrapi(base[b1] + kb, n[b1]);
                    idx[b2] = wrapi(base[b2] + kc, n[b2]);
                    add_fx_unit(J + (int64_t)a * cells + node3(n, idx[0], idx[1], idx[2]), run);
                }
            }
    }
    const int up[3] = {cn[0] + 1 == n[0] ? 0 : cn[0] + 1, cn[1] + 1 == n[1] ? 0 : cn[1] + 1,
                       cn[2] + 1 == n[2] ? 0 : cn[2] + 1};
#pragma unroll
    for (int k = 0; k < 8; ++k)
        atomicAdd(rho_acc + node3(n, (k & 1) ? up[0] : cn[0], (k & 2) ? up[1] : cn[1],
                                  (k & 4) ? up[2] : cn[2]),
                  (unsigned long long)(long long)qk[k]);
}

// The charge quanta of a particle at offsets fn (int64 fixed point; the last corner
// takes the remainder, so every particle deposits exactly 2^S); corner k is
// (k & 1, k >> 1 & 1, k >> 2) from the new cell.
__device__ __forceinline__ void em3_charge_quanta(const float *fn, float scale, int one, int *qk)
{
    const float w[3][2] = {{1.0f - fn[0], fn[0]}, {1.0f - fn[1], fn[1]}, {1.0f - fn[2], fn[2]}};
    int rest = one;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        qk[k] = __float_as_int(fmaf(w[0][k & 1] * w[1][(k >> 1) & 1] * w[2][k >> 2], scale,
                                    RND_MAGIC_F)) -
                RND_MAGIC_I;
        rest -= qk[k];
    }
    qk[7] = rest;
}

// The load's backward half kick: gather and Boris of -dt/2, every particle,
// grid-stride; diagnostics per block into diag_blocks[blockIdx.x] when given.
__global__ void __launch_bounds__(EM_THREADS)
    k_em3_half(GridParams g, ParticlesF32 p, EmBufs em, double *__restrict__ diag_blocks,
               int *__restrict__ err)
{
    const int *n = g.n;
    const int64_t cells = (int64_t)n[0] * n[1] * n[2];
    float ke = 0.0f, mom[3] = {0.0f, 0.0f, 0.0f};
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * EM_THREADS + threadIdx.x; i < p.np;
         i += (int64_t)gridDim.x * EM_THREADS) {
        int c[3];
        decode3(p.cell[i], g, c);
        const float f[3] = {p.off[i], p.off[p.stride + i], p.off[2 * p.stride + i]};
        const float v[3] = {p.v[i], p.v[p.stride + i], p.v[2 * p.stride + i]};
        float e[3], b[3], vn[3];
        em3_gather(c, f, n, em, cells, e, b);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            e[a] += g.E0[a];
            b[a] += em.B0[a];
        }
        em_boris(v, e, b, g, vn);
        if (!(isfinite(vn[0]) && isfinite(vn[1]) && isfinite(vn[2]))) bad = true;
        float o2 = 0.0f, n2 = 0.0f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            o2 += v[a] * v[a];
            n2 += vn[a] * vn[a];
            mom[a] += vn[a];
            p.v[a * p.stride + i] = vn[a];
        }
        ke += 0.5f * (o2 + n2);
    }
    if (bad) atomicOr(err, EF_NONFINITE);
    if (diag_blocks) em_block_diag(ke, mom, diag_blocks, blockIdx.x);
}

// One particle through global memory: gather, Boris, the move, the current and the
// charge straight to the int64 accumulators (the particles that k_em3_tile leaves).
__device__ __forceinline__ void em3_particle_global(int64_t i, const GridParams &g, ParticlesF32 p,
                                                    const EmBufs &em,
                                                    unsigned long long *__restrict__ rho_acc,
                                                    float scale, int one, float &ke, float *mom,
                                                    bool &bad)
{
    const int *n = g.n;
    const int64_t cells = (int64_t)n[0] * n[1] * n[2];
    int c[3];
    decode3(p.cell[i], g, c);
    const float f[3] = {p.off[i], p.off[p.stride + i], p.off[2 * p.stride + i]};
    const float v[3] = {p.v[i], p.v[p.stride + i], p.v[2 * p.stride + i]};
    float e[3], b[3], vn[3];
    em3_gather(c, f, n, em, cells, e, b);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        e[a] += g.E0[a];
        b[a] += em.B0[a];
    }
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
    int sh[3], m[3];
    float fn[3], S0[3][3], DS[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
        finite &= em_move_axis(f[a], vn[a] * g.dtdx[a], &sh[a], &m[a], &fn[a], S0[a], DS[a]);
    if (!finite) {
        bad = true;
        return;
    }
    int cn[3], qk[8];
#pragma unroll
    for (int a = 0; a < 3; ++a) cn[a] = wrapi(c[a] + sh[a], n[a]);
    em3_charge_quanta(fn, scale, one, qk);
    em3_deposit_global(n, cells, c, m, cn, S0, DS, qk, em.J, rho_acc);
    p.cell[i] = (int)node3(n, cn[0], cn[1], cn[2]);
#pragma unroll
    for (int a = 0; a < 3; ++a) p.off[a * p.stride + i] = fn[a];
}

// ---- the tiled particle kernel -------------------------------------------------------------
//
// Persistent CTAs walk tiles of E3_TILE consecutive (sorted) particles, one per
// thread.  Each tile has a fixed deposit window of E3W_X x E3W_Y x E3W_Z nodes, placed
// E3W_L* nodes below the old cell of the tile's middle particle.  A particle whose old
// cell lies far enough inside that every node its step can touch (old cell - 1 to
// old cell + 2 per axis) is in the window: the CTA gathers E and B for it (global
// memory, L1/L2), pushes and moves it, and adds its current and charge quanta to int32
// windows in shared memory at constant offsets from one window index.  After the
// tile, every touched window node goes once to the int64 accumulators (64-bit
// atomics) and is cleared.  The other particles of the tile are listed, in tile
// order, at slots first..first + count of the spill list (count in tile_spill[t]), and
// k_em3_spill runs their whole step through global memory, with whole warps of them
// rather than single lanes beside the window path.  Sums are integers either way, so
// the result does not depend on which particles took which path.  With 4 x 4 x 4 sort
// bricks, nearly all particles of a tile fall in the window for the first ten or so
// steps after a sort at 8 particles per cell (thermal speed 0.1 cell per step).
constexpr int E3W_X = 16, E3W_Y = 16, E3W_Z = 12;  // window nodes per axis
constexpr int E3W_LX = 7, E3W_LY = 7, E3W_LZ = 5;  // window origin below the reference
constexpr int E3W_NODES = E3W_X * E3W_Y * E3W_Z;
constexpr int E3_TILE = EM_PASS_TILE;
constexpr size_t E3_SMEM = 4 * E3W_NODES * sizeof(int);
static_assert(E3_TILE == EM_THREADS, "one particle per thread");
static_assert(E3_TILE <= 65535, "per-tile spill counts are 16-bit");
// int32 window sums stay exact: per node, each of a tile's particles adds at most 2^22
// in magnitude to a current (|J weight| <= 1 at 2^22) and at most 2^22 + 4 to the
// charge (S <= 22; the remainder corner absorbs up to 7 roundings of 1/2)
static_assert((long long)E3_TILE * ((1 << 22) + 4) < (1ll << 31), "window sums fit int32");

__device__ __forceinline__ int wrap_far(int i, int n)
{
    if ((unsigned)i < (unsigned)n) return i;
    i %= n;
    return i < 0 ? i + n : i;
}

#ifndef AP_PIC_EM3_MIN_BLOCKS
#define AP_PIC_EM3_MIN_BLOCKS 3
#endif
// three CTAs per SM: 80 registers with no spills (two at 122 without the bound)
__global__ void __launch_bounds__(EM_THREADS, AP_PIC_EM3_MIN_BLOCKS)
    k_em3_tile(GridParams g, ParticlesF32 p, EmBufs em, int32_t *__restrict__ spill_list,
               unsigned long long *__restrict__ rho_acc, double *__restrict__ diag_blocks,
               int *__restrict__ err)
{
    extern __shared__ int s_win[];           // [4][E3W_NODES]: Jx, Jy, Jz, charge (zero between tiles)
    __shared__ int s_box[2][6];              // per tile parity: the window part's min x, y, z, max x, y, z
    __shared__ int s_wc[2][EM_THREADS / 32];  // per tile parity: listed particles per warp
    const int *n = g.n;
    const int64_t cells = (int64_t)n[0] * n[1] * n[2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int k = tid; k < 4 * E3W_NODES; k += EM_THREADS) s_win[k] = 0;
    if (tid < 12) (&s_box[0][0])[tid] = (tid % 6) < 3 ? 0x7fffffff : -0x7fffffff;
    __syncthreads();
    const float scale = ldexpf(1.0f, g.fx_bits);
    const int one = 1 << g.fx_bits;
    float ke = 0.0f, mom[3] = {0.0f, 0.0f, 0.0f};
    bool bad = false;
    const int64_t ntiles = (p.np + E3_TILE - 1) / E3_TILE;
    int par = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, par ^= 1) {
        const int64_t first = t * E3_TILE;
        const int64_t i = first + tid;
        const bool valid = i < p.np;
        int rc[3];
        decode3(p.cell[first + E3_TILE / 2 < p.np ? first + E3_TILE / 2 : p.np - 1], g, rc);
        bool inwin = false, moved = false;
        int c[3], m[3], sh[3], lc[3] = {0, 0, 0}, qk[8];
        float fn[3], S0[3][3], DS[3][3];
        if (valid) {
            decode3(p.cell[i], g, c);
            // the old cell relative to the reference, unwrapped to [-n/2, n/2]; in the
            // window when old cell - 1 .. old cell + 2 lie in it on every axis
            const int lo[3] = {E3W_LX, E3W_LY, E3W_LZ}, w[3] = {E3W_X, E3W_Y, E3W_Z};
            inwin = true;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                int dd = c[a] - rc[a];
                dd -= (2 * dd > n[a]) ? n[a] : 0;
                dd += (2 * dd < -n[a]) ? n[a] : 0;
                lc[a] = dd + lo[a];
                inwin &= lc[a] >= 1 && lc[a] <= w[a] - 3;
            }
        }
        const bool listed = valid && !inwin;
        const unsigned lmask = __ballot_sync(0xffffffffu, listed);
        if (lane == 0) s_wc[par][warp] = __popc(lmask);
        if (inwin) {
            const float f[3] = {p.off[i], p.off[p.stride + i], p.off[2 * p.stride + i]};
            const float v[3] = {p.v[i], p.v[p.stride + i], p.v[2 * p.stride + i]};
            float e[3], b[3], vn[3];
            em3_gather(c, f, n, em, cells, e, b);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                e[a] += g.E0[a];
                b[a] += em.B0[a];
            }
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
#pragma unroll
            for (int a = 0; a < 3; ++a)
                finite &= em_move_axis(f[a], vn[a] * g.dtdx[a], &sh[a], &m[a], &fn[a], S0[a], DS[a]);
            if (!finite) {
                bad = true;
            } else {
                moved = true;
                // the stencil's lower corner (old cell + m) in window coordinates: in
                // [0, w - 3] on every axis
#pragma unroll
                for (int a = 0; a < 3; ++a) lc[a] += m[a];
                em3_charge_quanta(fn, scale, one, qk);
            }
        }
        // the box of the window part of this tile, for the flush
        int *box = s_box[par];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int wl = __reduce_min_sync(0xffffffffu, moved ? lc[a] : 0x7fffffff);
            const int wh = __reduce_max_sync(0xffffffffu, moved ? lc[a] + 2 : -0x7fffffff);
            if (lane == 0 && wl != 0x7fffffff) {
                atomicMin(&box[a], wl);
                atomicMax(&box[3 + a], wh);
            }
        }
        __syncthreads();  // the previous tile's flush has left the window cleared
        // the other parity's box was last read by that flush: reset it for the next tile
        if (tid < 6) s_box[par ^ 1][tid] = tid < 3 ? 0x7fffffff : -0x7fffffff;
        // the listed particles, in tile order, for k_em3_spill (slot first + k < np:
        // at most the tile's particles are listed)
        if (listed) {
            int k = __popc(lmask & ((1u << lane) - 1u));
            for (int w = 0; w < warp; ++w) k += s_wc[par][w];
            spill_list[first + k] = (int32_t)i;
        }
        if (tid == 0) {
            int total = 0;
#pragma unroll
            for (int w = 0; w < EM_THREADS / 32; ++w) total += s_wc[par][w];
            em.tile_spill[t] = (unsigned short)total;
        }
        if (moved) {
            constexpr int st[3] = {1, E3W_X, E3W_X * E3W_Y};
            const int base = lc[0] + E3W_X * (lc[1] + E3W_Y * lc[2]);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const int b1 = (a + 1) % 3, b2 = (a + 2) % 3;
                int *J = s_win + a * E3W_NODES + base;
#pragma unroll
                for (int kc = 0; kc < 3; ++kc)
#pragma unroll
                    for (int kb = 0; kb < 3; ++kb) {
                        const float perp = esirkepov_perp(S0, DS, b1, kb, b2, kc);
                        float run = 0.0f;
#pragma unroll
                        for (int ka = 0; ka < 2; ++ka) {
                            run += DS[a][ka] * perp;
                            const int q = __float_as_int(fmaf(run, J_SCALE, RND_MAGIC_F)) - RND_MAGIC_I;
                            if (q) atomicAdd(J + ka * st[a] + kb * st[b1] + kc * st[b2], q);
                        }
                    }
            }
            // the new cell is the stencil's node sh - m (0 or 1) per axis
            int *R = s_win + 3 * E3W_NODES + base + (sh[0] - m[0]) +
                     E3W_X * ((sh[1] - m[1]) + E3W_Y * (sh[2] - m[2]));
#pragma unroll
            for (int k = 0; k < 8; ++k)
                atomicAdd(R + (k & 1) + ((k >> 1) & 1) * st[1] + (k >> 2) * st[2], qk[k]);
            int cn[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) cn[a] = wrapi(c[a] + sh[a], n[a]);
            p.cell[i] = (int)node3(n, cn[0], cn[1], cn[2]);
            p.off[i] = fn[0];
            p.off[p.stride + i] = fn[1];
            p.off[2 * p.stride + i] = fn[2];
        }
        __syncthreads();  // the window sums and the box are complete
        const int bx0 = box[0], by0 = box[1], bz0 = box[2];
        if (bx0 <= box[3]) {
            // every node of the box once: half a warp per (y, z) row, lanes along x
            const int nx = box[3] - bx0 + 1, ny = box[4] - by0 + 1, rows = ny * (box[5] - bz0 + 1);
            const int lx = bx0 + (tid & 15);
            const int gx = wrap_far(rc[0] - E3W_LX + lx, n[0]);
            for (int r = tid >> 4; r < rows; r += EM_THREADS / 16) {
                if ((tid & 15) >= nx) break;
                const int rz = r / ny, ly = by0 + (r - rz * ny), lz = bz0 + rz;
                const int l = lx + E3W_X * (ly + E3W_Y * lz);
                const int qx = s_win[l], qy = s_win[E3W_NODES + l], qz = s_win[2 * E3W_NODES + l],
                          qr = s_win[3 * E3W_NODES + l];
                if ((qx | qy | qz | qr) == 0) continue;
                const int64_t gid = gx + (int64_t)n[0] * (wrap_far(rc[1] - E3W_LY + ly, n[1]) +
                                                          (int64_t)n[1] * wrap_far(rc[2] - E3W_LZ + lz, n[2]));
                if (qx) {
                    s_win[l] = 0;
                    atomicAdd(em.J + gid, (unsigned long long)(long long)qx);
                }
                if (qy) {
                    s_win[E3W_NODES + l] = 0;
                    atomicAdd(em.J + cells + gid, (unsigned long long)(long long)qy);
                }
                if (qz) {
                    s_win[2 * E3W_NODES + l] = 0;
                    atomicAdd(em.J + 2 * cells + gid, (unsigned long long)(long long)qz);
                }
                if (qr) {
                    s_win[3 * E3W_NODES + l] = 0;
                    atomicAdd(rho_acc + gid, (unsigned long long)(long long)qr);
                }
            }
        }
    }
    if (bad) atomicOr(err, EF_NONFINITE);
    if (diag_blocks) em_block_diag(ke, mom, diag_blocks, blockIdx.x);
}

// The particles that k_em3_tile listed, through global memory.  Each warp takes a
// fixed, contiguous range of tiles and packs their lists into batches of 32 (one
// particle per lane): it reads 32 tiles' counts at once, scans them, and each lane
// finds the tile of its batch position by a binary search over the scan.  The
// assignment of particles to lanes is fixed, so the diagnostic partials are
// deterministic; every block writes its slot gridDim.x + blockIdx.x.
__global__ void __launch_bounds__(EM_THREADS)
    k_em3_spill(GridParams g, ParticlesF32 p, EmBufs em, const int32_t *__restrict__ spill_list,
                unsigned long long *__restrict__ rho_acc, double *__restrict__ diag_blocks,
                int *__restrict__ err)
{
    const float scale = ldexpf(1.0f, g.fx_bits);
    const int one = 1 << g.fx_bits;
    float ke = 0.0f, mom[3] = {0.0f, 0.0f, 0.0f};
    bool bad = false;
    const int lane = threadIdx.x & 31;
    const int64_t ntiles = (p.np + E3_TILE - 1) / E3_TILE;
    const int64_t warps = (int64_t)gridDim.x * (EM_THREADS / 32);
    const int64_t wid = (int64_t)blockIdx.x * (EM_THREADS / 32) + (threadIdx.x >> 5);
    const int64_t per = (ntiles + warps - 1) / warps;
    const int64_t t_end = (wid + 1) * per < ntiles ? (wid + 1) * per : ntiles;
    for (int64_t t0 = wid * per; t0 < t_end; t0 += 32) {
        // this lane's tile of the group of 32 and the exclusive scan of the counts
        const int64_t tt = t0 + lane;
        const int cnt = tt < t_end ? (int)em.tile_spill[tt] : 0;
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        const int excl = incl - cnt;
        for (int pos = lane; pos - lane < total; pos += 32) {
            // the tile q of position pos: the last q with excl[q] <= pos
            int q = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int e = __shfl_sync(0xffffffffu, excl, q + step);
                if (q + step < 32 && e <= pos) q += step;
            }
            const int eq = __shfl_sync(0xffffffffu, excl, q);
            if (pos < total) {
                const int64_t i = spill_list[(t0 + q) * E3_TILE + (pos - eq)];
                em3_particle_global(i, g, p, em, rho_acc, scale, one, ke, mom, bad);
            }
        }
    }
    if (bad) atomicOr(err, EF_NONFINITE);
    if (diag_blocks) em_block_diag(ke, mom, diag_blocks, gridDim.x + blockIdx.x);
}

__device__ __forceinline__ void coords3(int64_t id, const GridParams &g, int *c)
{
    decode3((int)id, g, c);
}

// Faraday: B -= h curl E, each component of curl E by forward differences at the B
// component's own position.
__global__ void __launch_bounds__(EM_THREADS)
    k_yee3_b(GridParams g, const float *__restrict__ E, float *__restrict__ B, float hx, float hy,
             float hz)
{
    const int *n = g.n;
    const int64_t cells = (int64_t)n[0] * n[1] * n[2];
    const float *Ex = E, *Ey = E + cells, *Ez = E + 2 * cells;
    for (int64_t id = (int64_t)blockIdx.x * EM_THREADS + threadIdx.x; id < cells;
         id += (int64_t)gridDim.x * EM_THREADS) {
        int c[3];
        coords3(id, g, c);
        const int64_t ip = node3(n, c[0] + 1 == n[0] ? 0 : c[0] + 1, c[1], c[2]);
        const int64_t jp = node3(n, c[0], c[1] + 1 == n[1] ? 0 : c[1] + 1, c[2]);
        const int64_t kp = node3(n, c[0], c[1], c[2] + 1 == n[2] ? 0 : c[2] + 1);
        const float ex = Ex[id], ey = Ey[id], ez = Ez[id];
        B[id] -= hy * (Ez[jp] - ez) - hz * (Ey[kp] - ey);
        B[cells + id] -= hz * (Ex[kp] - ex) - hx * (Ez[ip] - ez);
        B[2 * cells + id] -= hx * (Ey[ip] - ey) - hy * (Ex[jp] - ex);
    }
}

// Ampere: E += dt (c^2 curl B - J), curl B by backward differences at the E positions.
__global__ void __launch_bounds__(EM_THREADS)
    k_yee3_e(GridParams g, const float *__restrict__ B, JTake jt, float *__restrict__ E,
             float cx, float cy, float cz, float dt)
{
    const int *n = g.n;
    const int64_t cells = (int64_t)n[0] * n[1] * n[2];
    const float *Bx = B, *By = B + cells, *Bz = B + 2 * cells;
    for (int64_t id = (int64_t)blockIdx.x * EM_THREADS + threadIdx.x; id < cells;
         id += (int64_t)gridDim.x * EM_THREADS) {
        int c[3];
        coords3(id, g, c);
        const int64_t im = node3(n, c[0] == 0 ? n[0] - 1 : c[0] - 1, c[1], c[2]);
        const int64_t jm = node3(n, c[0], c[1] == 0 ? n[1] - 1 : c[1] - 1, c[2]);
        const int64_t km = node3(n, c[0], c[1], c[2] == 0 ? n[2] - 1 : c[2] - 1);
        const float bx = Bx[id], by = By[id], bz = Bz[id];
        float J[3];
        get_j(jt, cells, id, J);
        E[id] += cy * (bz - Bz[jm]) - cz * (by - By[km]) - dt * J[0];
        E[cells + id] += cz * (bx - Bx[km]) - cx * (bz - Bz[im]) - dt * J[1];
        E[2 * cells + id] += cx * (by - By[im]) - cy * (bx - Bx[jm]) - dt * J[2];
        clear_j(jt, cells, id);
    }
}

// The load's field: E_a = -(phi at the next node along a - phi) / dx_a, so the
// discrete div E equals rho; B is cleared by the caller.
__global__ void __launch_bounds__(EM_THREADS)
    k_em3_e_from_phi(GridParams g, const float *__restrict__ phi, float *__restrict__ E, float ix,
                     float iy, float iz)
{
    const int *n = g.n;
    const int64_t cells = (int64_t)n[0] * n[1] * n[2];
    for (int64_t id = (int64_t)blockIdx.x * EM_THREADS + threadIdx.x; id < cells;
         id += (int64_t)gridDim.x * EM_THREADS) {
        int c[3];
        coords3(id, g, c);
        const float p0 = phi[id];
        E[id] = -(phi[node3(n, c[0] + 1 == n[0] ? 0 : c[0] + 1, c[1], c[2])] - p0) * ix;
        E[cells + id] = -(phi[node3(n, c[0], c[1] + 1 == n[1] ? 0 : c[1] + 1, c[2])] - p0) * iy;
        E[2 * cells + id] = -(phi[node3(n, c[0], c[1], c[2] + 1 == n[2] ? 0 : c[2] + 1)] - p0) * iz;
    }
}

int em3_grid_blocks(int64_t n)
{
    const int64_t need = (n + EM_THREADS - 1) / EM_THREADS;
    const int64_t cap = (int64_t)sm_count() * 8;
    const int64_t b = need < cap ? need : cap;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

namespace {

// k_em3_tile takes E3_SMEM of dynamic shared memory, above the default limit: the
// attribute is set before each use (a host-side call, on the current device).
cudaError_t em3_tile_attribute()
{
    return cudaFuncSetAttribute(k_em3_tile, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)E3_SMEM);
}

}  // namespace

int em3_particle_blocks(int64_t np)
{
    static std::atomic<int> per_sm{0};
    int c = per_sm.load(std::memory_order_relaxed);
    if (!c) {
        if (em3_tile_attribute() != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, k_em3_tile, EM_THREADS, E3_SMEM) !=
                cudaSuccess ||
            c < 1) {
            cudaGetLastError();
            c = 1;
        }
        per_sm.store(c, std::memory_order_relaxed);
    }
    const int64_t need = (np + E3_TILE - 1) / E3_TILE;
    const int64_t cap = (int64_t)sm_count() * c;
    const int64_t b = need < cap ? need : cap;
    return (int)(b < 1 ? 1 : b);
}

cudaError_t launch_em3_push(const GridParams &g, ParticlesF32 p, const EmBufs &em, bool move,
                            unsigned long long *rho_acc, double *diag_blocks, int nblocks,
                            int *err, int32_t *spill_list, cudaStream_t st)
{
    if (p.np == 0) return cudaSuccess;
    if (!move) {
        // every diagnostic slot is written (blocks without particles write zeros)
        k_em3_half<<<nblocks > 0 ? nblocks : 1, EM_THREADS, 0, st>>>(g, p, em, diag_blocks, err);
        note_launch();
        return cudaGetLastError();
    }
    // nblocks diagnostic slots: the first half for the tiled kernel, the second for the
    // listed particles
    const int nb = nblocks / 2 > 0 ? nblocks / 2 : 1;
    const cudaError_t e = em3_tile_attribute();
    if (e != cudaSuccess) return e;
    k_em3_tile<<<nb, EM_THREADS, E3_SMEM, st>>>(g, p, em, spill_list, rho_acc, diag_blocks, err);
    k_em3_spill<<<nb, EM_THREADS, 0, st>>>(g, p, em, spill_list, rho_acc, diag_blocks, err);
    note_launch(2);
    return cudaGetLastError();
}

cudaError_t launch_em3_fields(const GridParams &g, const EmBufs &em, const double *dx, double dt,
                              double c, double qw, cudaStream_t st)
{
    const int64_t cells = (int64_t)g.n[0] * g.n[1] * g.n[2];
    const int nb = em3_grid_blocks(cells);
    // J_a = -(q w / (dx_b dx_c dt)) times the accumulated weights / 2^22, taken (and
    // cleared) by the E update
    const JTake jt = em_jtake(em, -qw / (dx[1] * dx[2] * dt) / J_SCALE,
                              -qw / (dx[2] * dx[0] * dt) / J_SCALE,
                              -qw / (dx[0] * dx[1] * dt) / J_SCALE);
    const float hx = (float)(0.5 * dt / dx[0]), hy = (float)(0.5 * dt / dx[1]),
                hz = (float)(0.5 * dt / dx[2]);
    const double c2dt = c * c * dt;
    k_yee3_b<<<nb, EM_THREADS, 0, st>>>(g, em.E, em.B, hx, hy, hz);
    k_yee3_e<<<nb, EM_THREADS, 0, st>>>(g, em.B, jt, em.E, (float)(c2dt / dx[0]),
                                        (float)(c2dt / dx[1]), (float)(c2dt / dx[2]), (float)dt);
    k_yee3_b<<<nb, EM_THREADS, 0, st>>>(g, em.E, em.B, hx, hy, hz);
    note_launch(3);
    return cudaGetLastError();
}

cudaError_t launch_em3_e_from_phi(const GridParams &g, const float *phi, const EmBufs &em,
                                  const double *dx, cudaStream_t st)
{
    const int64_t cells = (int64_t)g.n[0] * g.n[1] * g.n[2];
    k_em3_e_from_phi<<<em3_grid_blocks(cells), EM_THREADS, 0, st>>>(
        g, phi, em.E, (float)(1.0 / dx[0]), (float)(1.0 / dx[1]), (float)(1.0 / dx[2]));
    note_launch();
    return cudaGetLastError();
}

}  // namespace apk
