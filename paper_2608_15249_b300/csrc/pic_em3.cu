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
// The particle kernel takes one particle per thread and reads the fields and adds the
// current and charge in global memory (L2-resident fields; 64-bit atomics).
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

// Trilinear CIC of component F at lower lattice indices i0[3], fractions fr[3].
__device__ __forceinline__ float cic3(const float *__restrict__ F, const int *n, const int *i0,
                                      const float *fr)
{
    const int i1 = i0[0] + 1 == n[0] ? 0 : i0[0] + 1;
    const int j1 = i0[1] + 1 == n[1] ? 0 : i0[1] + 1;
    const int k1 = i0[2] + 1 == n[2] ? 0 : i0[2] + 1;
    const int ii[2] = {i0[0], i1}, jj[2] = {i0[1], j1}, kk[2] = {i0[2], k1};
    float s = 0.0f;
#pragma unroll
    for (int bk = 0; bk < 2; ++bk) {
        const float wz = bk ? fr[2] : 1.0f - fr[2];
#pragma unroll
        for (int bj = 0; bj < 2; ++bj) {
            const float wy = bj ? fr[1] : 1.0f - fr[1];
            const int64_t row = node3(n, 0, jj[bj], kk[bk]);
            s += wz * wy * ((1.0f - fr[0]) * __ldg(F + row + ii[0]) + fr[0] * __ldg(F + row + ii[1]));
        }
    }
    return s;
}

// One particle: gather, Boris, and (MOVE) the move, the Esirkepov current and the
// charge at the new position.  A particle that is not finite or moves more than a
// cell per axis is left where it is and flagged.
template <bool MOVE>
__device__ __forceinline__ void em3_particle(int64_t i, const GridParams &g, ParticlesF32 p,
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
    // lower lattice index and fraction per axis, on the integer and the half lattice
    int il[2][3];
    float fl[2][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        stagger(c[a], f[a], false, n[a], &il[0][a], &fl[0][a]);
        stagger(c[a], f[a], true, n[a], &il[1][a], &fl[1][a]);
    }
    float eb[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        int i0[3];
        float fr[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int h = (HALF_BITS >> (3 * q + a)) & 1;
            i0[a] = il[h][a];
            fr[a] = fl[h][a];
        }
        eb[q] = cic3((q < 3 ? em.E : em.B) + (q % 3) * cells, n, i0, fr);
    }
    float e[3], b[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        e[a] = eb[a] + g.E0[a];
        b[a] = eb[3 + a] + em.B0[a];
    }
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
        int sh[3], m[3];
        float fn[3], S0[3][3], DS[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
            finite &= em_move_axis(f[a], vn[a] * g.dtdx[a], &sh[a], &m[a], &fn[a], S0[a], DS[a]);
        if (!finite) {
            bad = true;
            return;
        }
        int cn[3], base[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cn[a] = wrapi(c[a] + sh[a], n[a]);
            base[a] = c[a] + m[a];
        }
        // Esirkepov current on the 3 x 3 x 3 stencil from c + m, in weights (scaled at
        // conversion): along axis a, for each node (kb, kc) of the two other axes,
        //   W_a = DS_a (S0_b S0_c + DS_b S0_c / 2 + S0_b DS_c / 2 + DS_b DS_c / 3),
        // and J_a on the two a-edges is its running sum (the third is zero: the shape
        // changes along a sum to zero); |W| <= 1 per node.
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int b1 = (a + 1) % 3, b2 = (a + 2) % 3;
#pragma unroll
            for (int kc = 0; kc < 3; ++kc)
#pragma unroll
                for (int kb = 0; kb < 3; ++kb) {
                    const float perp = S0[b1][kb] * (S0[b2][kc] + 0.5f * DS[b2][kc]) +
                                       DS[b1][kb] * (0.5f * S0[b2][kc] + DS[b2][kc] * (1.0f / 3.0f));
                    if (perp == 0.0f) continue;
                    float run = 0.0f;
#pragma unroll
                    for (int ka = 0; ka < 2; ++ka) {
                        run += DS[a][ka] * perp;
                        int idx[3];
                        idx[a] = wrapi(base[a] + ka, n[a]);
                        idx[b1] = wrapi(base[b1] + kb, n[b1]);
                        idx[b2] = wrapi(base[b2] + kc, n[b2]);
                        add_fx_unit(em.J + (int64_t)a * cells + node3(n, idx[0], idx[1], idx[2]),
                                    run);
                    }
                }
        }
        // charge at the new position (int64 fixed point; the last corner takes the
        // remainder, so every particle deposits exactly 2^S)
        const float w[3][2] = {{1.0f - fn[0], fn[0]}, {1.0f - fn[1], fn[1]}, {1.0f - fn[2], fn[2]}};
        int qk[8], rest = one;
#pragma unroll
        for (int k = 0; k < 7; ++k) {
            qk[k] = __float_as_int(fmaf(w[0][k & 1] * w[1][(k >> 1) & 1] * w[2][k >> 2], scale,
                                        RND_MAGIC_F)) -
                    RND_MAGIC_I;
            rest -= qk[k];
        }
        qk[7] = rest;
        const int up[3] = {cn[0] + 1 == n[0] ? 0 : cn[0] + 1, cn[1] + 1 == n[1] ? 0 : cn[1] + 1,
                           cn[2] + 1 == n[2] ? 0 : cn[2] + 1};
#pragma unroll
        for (int k = 0; k < 8; ++k)
            atomicAdd(rho_acc + node3(n, (k & 1) ? up[0] : cn[0], (k & 2) ? up[1] : cn[1],
                                      (k & 4) ? up[2] : cn[2]),
                      (unsigned long long)(long long)qk[k]);
        p.cell[i] = (int)node3(n, cn[0], cn[1], cn[2]);
#pragma unroll
        for (int a = 0; a < 3; ++a) p.off[a * p.stride + i] = fn[a];
    }
}

// Every particle, grid-stride, diagnostics per block into diag_blocks[blockIdx.x].
template <bool MOVE>
__global__ void __launch_bounds__(EM_THREADS)
    k_em3_push(GridParams g, ParticlesF32 p, EmBufs em, unsigned long long *__restrict__ rho_acc,
               double *__restrict__ diag_blocks, int *__restrict__ err)
{
    const float scale = ldexpf(1.0f, g.fx_bits);
    const int one = 1 << g.fx_bits;
    float ke = 0.0f, mom[3] = {0.0f, 0.0f, 0.0f};
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * EM_THREADS + threadIdx.x; i < p.np;
         i += (int64_t)gridDim.x * EM_THREADS)
        em3_particle<MOVE>(i, g, p, em, rho_acc, scale, one, ke, mom, bad);
    if (bad) atomicOr(err, EF_NONFINITE);
    if (diag_blocks) em_block_diag(ke, mom, diag_blocks, blockIdx.x);
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
    k_yee3_e(GridParams g, const float *__restrict__ B, const float *__restrict__ J,
             float *__restrict__ E, float cx, float cy, float cz, float dt)
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
        E[id] += cy * (bz - Bz[jm]) - cz * (by - By[km]) - dt * J[id];
        E[cells + id] += cz * (bx - Bx[km]) - cx * (bz - Bz[im]) - dt * J[cells + id];
        E[2 * cells + id] += cx * (by - By[im]) - cy * (bx - Bx[jm]) - dt * J[2 * cells + id];
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

cudaError_t launch_em3_push(const GridParams &g, ParticlesF32 p, const EmBufs &em, bool move,
                            unsigned long long *rho_acc, double *diag_blocks, int nblocks,
                            int *err, cudaStream_t st)
{
    if (p.np == 0) return cudaSuccess;
    // every diagnostic slot is written (blocks without particles write zeros)
    const int nb = nblocks > 0 ? nblocks : 1;
    if (move) k_em3_push<true><<<nb, EM_THREADS, 0, st>>>(g, p, em, rho_acc, diag_blocks, err);
    else k_em3_push<false><<<nb, EM_THREADS, 0, st>>>(g, p, em, rho_acc, diag_blocks, err);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_em3_fields(const GridParams &g, const EmBufs &em, const double *dx, double dt,
                              double c, double qw, cudaStream_t st)
{
    const int64_t cells = (int64_t)g.n[0] * g.n[1] * g.n[2];
    const int nb = em3_grid_blocks(cells);
    // J_a = -(q w / (dx_b dx_c dt)) times the accumulated weights / 2^22
    cudaError_t e = launch_em_j_convert(cells, em, -qw / (dx[1] * dx[2] * dt) / J_SCALE,
                                        -qw / (dx[2] * dx[0] * dt) / J_SCALE,
                                        -qw / (dx[0] * dx[1] * dt) / J_SCALE, st);
    if (e != cudaSuccess) return e;
    const float hx = (float)(0.5 * dt / dx[0]), hy = (float)(0.5 * dt / dx[1]),
                hz = (float)(0.5 * dt / dx[2]);
    const double c2dt = c * c * dt;
    k_yee3_b<<<nb, EM_THREADS, 0, st>>>(g, em.E, em.B, hx, hy, hz);
    k_yee3_e<<<nb, EM_THREADS, 0, st>>>(g, em.B, em.Jf, em.E, (float)(c2dt / dx[0]),
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
