// pic_particles.cu -- particle-side kernels of the electrostatic PIC cycle:
// load/convert, and the pass that gathers E (C01), advances v with the Boris
// scheme (A01), moves the particle with periodic wrap and deposits its charge
// (B01) -- the order of the paper's worked example (Sec. 3.1, Listing 1).
//
// Storage: int32 linear cell index, FP32 offsets in [0, 1) per axis (SoA,
// one array per axis), FP32 velocities (SoA).  E is stored interleaved per
// node (float, float2 or float4 for 1, 2, 3 dimensions) so a corner's field
// is one vector load.  Charge goes to an int64 fixed-point accumulator: each
// particle deposits exactly 2^S split over its 2^d corners (the last corner
// takes the remainder), so totals are exact and the sum is independent of
// the order of the atomics.
#include <math.h>

#include "pic_internal.cuh"

namespace apk {

constexpr int PP_THREADS = 256;

__device__ __forceinline__ void latch(int *flags, int bit) { atomicOr(flags, bit); }

template <int D>
__device__ __forceinline__ void decode_cell(int cell, const GridParams &g, int *c)
{
    if (D == 1) {
        c[0] = cell;
    } else if (D == 2) {
        const int c1 = (int)fdiv((uint32_t)cell, g.div0);
        c[0] = cell - c1 * g.n[0];
        c[1] = c1;
    } else {
        const int c12 = (int)fdiv((uint32_t)cell, g.div0);
        c[0] = cell - c12 * g.n[0];
        const int c2 = (int)fdiv((uint32_t)c12, g.div1);
        c[1] = c12 - c2 * g.n[1];
        c[2] = c2;
    }
}

template <int D>
__device__ __forceinline__ int encode_cell(const int *c, const int *n)
{
    if (D == 1) return c[0];
    if (D == 2) return c[0] + n[0] * c[1];
    return c[0] + n[0] * (c[1] + n[1] * c[2]);
}

// Upper neighbour on a periodic axis.
__device__ __forceinline__ int up(int c, int n) { return (c + 1 == n) ? 0 : c + 1; }

template <int D>
__device__ __forceinline__ void gather_E(const float *__restrict__ E, const int *c, const float *f,
                                         const int *n, float *e)
{
    if (D == 1) {
        const float w0 = 1.0f - f[0], w1 = f[0];
        e[0] = w0 * __ldg(E + c[0]) + w1 * __ldg(E + up(c[0], n[0]));
    } else if (D == 2) {
        const float2 *E2 = reinterpret_cast<const float2 *>(E);
        const int x0 = c[0], x1 = up(c[0], n[0]);
        const int y0 = c[1] * n[0], y1 = up(c[1], n[1]) * n[0];
        const float wx0 = 1.0f - f[0], wx1 = f[0], wy0 = 1.0f - f[1], wy1 = f[1];
        const float2 a = __ldg(E2 + x0 + y0), b = __ldg(E2 + x1 + y0);
        const float2 cc = __ldg(E2 + x0 + y1), d = __ldg(E2 + x1 + y1);
        e[0] = wy0 * (wx0 * a.x + wx1 * b.x) + wy1 * (wx0 * cc.x + wx1 * d.x);
        e[1] = wy0 * (wx0 * a.y + wx1 * b.y) + wy1 * (wx0 * cc.y + wx1 * d.y);
    } else {
        const float4 *E4 = reinterpret_cast<const float4 *>(E);
        const int nxy = n[0] * n[1];
        const int x[2] = {c[0], up(c[0], n[0])};
        const int y[2] = {c[1] * n[0], up(c[1], n[1]) * n[0]};
        const int z[2] = {c[2] * nxy, up(c[2], n[2]) * nxy};
        const float wx[2] = {1.0f - f[0], f[0]};
        const float wy[2] = {1.0f - f[1], f[1]};
        const float wz[2] = {1.0f - f[2], f[2]};
        e[0] = e[1] = e[2] = 0.0f;
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const float wyz = wy[j] * wz[k];
                const float4 a = __ldg(E4 + x[0] + y[j] + z[k]);
                const float4 b = __ldg(E4 + x[1] + y[j] + z[k]);
                e[0] += wyz * (wx[0] * a.x + wx[1] * b.x);
                e[1] += wyz * (wx[0] * a.y + wx[1] * b.y);
                e[2] += wyz * (wx[0] * a.z + wx[1] * b.z);
            }
    }
}

// Fixed-point CIC weights of one particle: corner k (bit a of k selects the
// upper node on axis a) gets round(W_k 2^S) for every corner but the last,
// which takes 2^S minus the others, so the particle deposits exactly 2^S.
// With S <= 25 every quantum, and a warp's sum of 32 of them, fits in int32.
template <int D>
__device__ __forceinline__ void cic_quanta(const float *f, float scale, int one, int *q)
{
    const float wx[2] = {1.0f - f[0], f[0]};
    if (D == 1) {
        q[0] = __float2int_rn(wx[0] * scale);
        q[1] = one - q[0];
    } else if (D == 2) {
        const float wy[2] = {1.0f - f[1], f[1]};
        q[0] = __float2int_rn(wx[0] * wy[0] * scale);
        q[1] = __float2int_rn(wx[1] * wy[0] * scale);
        q[2] = __float2int_rn(wx[0] * wy[1] * scale);
        q[3] = one - q[0] - q[1] - q[2];
    } else {
        const float wy[2] = {1.0f - f[1], f[1]};
        const float wz[2] = {1.0f - f[2], f[2]};
        int rest = one;
#pragma unroll
        for (int k = 0; k < 7; ++k) {
            q[k] = __float2int_rn(wx[k & 1] * wy[(k >> 1) & 1] * wz[k >> 2] * scale);
            rest -= q[k];
        }
        q[7] = rest;
    }
}

// Flat node index of corner k of cell c.
template <int D>
__device__ __forceinline__ void corner_nodes(const int *c, const int *n, int *node)
{
    const int x[2] = {c[0], up(c[0], n[0])};
    if (D == 1) {
        node[0] = x[0];
        node[1] = x[1];
    } else if (D == 2) {
        const int y[2] = {c[1] * n[0], up(c[1], n[1]) * n[0]};
#pragma unroll
        for (int k = 0; k < 4; ++k) node[k] = x[k & 1] + y[k >> 1];
    } else {
        const int nxy = n[0] * n[1];
        const int y[2] = {c[1] * n[0], up(c[1], n[1]) * n[0]};
        const int z[2] = {c[2] * nxy, up(c[2], n[2]) * nxy};
#pragma unroll
        for (int k = 0; k < 8; ++k) node[k] = x[k & 1] + y[(k >> 1) & 1] + z[k >> 2];
    }
}

// Warp-cooperative deposit.  Lanes hold consecutive particles of the sorted
// array, so runs of lanes share a cell (key).  A segmented inclusive scan over
// the lanes (five shuffle steps, fixed cost whatever the data) sums the first
// 2^d - 1 corner quanta of each run; the run's last corner is its particle
// count times 2^S minus those sums (the per-particle remainder rule, summed).
// The last lane of each run issues one 64-bit atomic per corner.  Lanes with
// key < 0 deposit nothing.  Integer sums make the result independent of how
// lanes group and of the order of the atomics.  Must be called by all lanes.
template <int D>
__device__ __forceinline__ void warp_deposit(unsigned long long *__restrict__ acc, int key,
                                             const int *node, const int *q, int one)
{
    constexpr int NC = 1 << D;
    const int lane = threadIdx.x & 31;
    const int kprev = __shfl_up_sync(0xffffffffu, key, 1);
    const bool head = lane == 0 || kprev != key;
    const unsigned heads = __ballot_sync(0xffffffffu, head);
    // first lane of this lane's run: the highest head at or below this lane
    const unsigned le = 0xffffffffu >> (31 - lane);
    const int seg = 31 - __clz(heads & le);
    int s[NC - 1];
#pragma unroll
    for (int k = 0; k < NC - 1; ++k) s[k] = q[k];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const bool take = lane - d >= seg;
#pragma unroll
        for (int k = 0; k < NC - 1; ++k) {
            const int y = __shfl_up_sync(0xffffffffu, s[k], d);
            if (take) s[k] += y;
        }
    }
    const bool tail = lane == 31 || ((heads >> (lane + 1)) & 1u);
    if (tail && key >= 0) {
        long long rest = (long long)(lane - seg + 1) * one;
#pragma unroll
        for (int k = 0; k < NC - 1; ++k) {
            rest -= s[k];
            atomicAdd(acc + node[k], (unsigned long long)(long long)s[k]);
        }
        atomicAdd(acc + node[NC - 1], (unsigned long long)rest);
    }
}

// Boris velocity advance in FP32 (A_Pusher, Sec. 2.2):
//   v- = v + qmh2 E;  w = v- + v- x t;  v+ = v- + w x s;  v = v+ + qmh2 E.
__device__ __forceinline__ void boris(float *v, const float *e, const GridParams &g)
{
    float vm[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) vm[a] = v[a] + g.qmh2 * e[a];
    if (g.magnetised) {
        const float w0 = vm[0] + (vm[1] * g.t[2] - vm[2] * g.t[1]);
        const float w1 = vm[1] + (vm[2] * g.t[0] - vm[0] * g.t[2]);
        const float w2 = vm[2] + (vm[0] * g.t[1] - vm[1] * g.t[0]);
        const float p0 = vm[0] + (w1 * g.s[2] - w2 * g.s[1]);
        const float p1 = vm[1] + (w2 * g.s[0] - w0 * g.s[2]);
        const float p2 = vm[2] + (w0 * g.s[1] - w1 * g.s[0]);
        vm[0] = p0;
        vm[1] = p1;
        vm[2] = p2;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) v[a] = vm[a] + g.qmh2 * e[a];
}

// Position update in cell units with periodic wrap (application code in
// Sec. 3.1): o = f + v dt/dx; shift = floor(o); f = o - shift (forced into
// [0, 1)); cell += shift mod n.  Returns false for a non-finite or absurd
// displacement (the particle is then left where it was).
template <int D>
__device__ __forceinline__ bool move(int *c, float *f, const float *v, const GridParams &g)
{
    float nf[3];
    int nc[3];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const float o = f[a] + v[a] * g.dtdx[a];
        if (!(fabsf(o) < 1.0e9f)) return false;  // also catches NaN / inf
        const float fl = floorf(o);
        float fr = o - fl;
        int s = (int)fl;
        if (fr >= 1.0f) {  // o a tiny negative number: o - floor(o) rounds up to 1
            fr = 0.0f;
            s += 1;
        }
        int ca = c[a] + s;
        if (ca < 0 || ca >= g.n[a]) {
            ca %= g.n[a];
            if (ca < 0) ca += g.n[a];
        }
        nc[a] = ca;
        nf[a] = fr;
    }
#pragma unroll
    for (int a = 0; a < D; ++a) {
        c[a] = nc[a];
        f[a] = nf[a];
    }
    return true;
}

__device__ __forceinline__ double warp_sum_d(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

enum : int { PASS_PUSH = 1, PASS_MOVE = 2, PASS_DEPOSIT = 4, PASS_DIAG = 8 };

template <int D, int NV>
__global__ void __launch_bounds__(PP_THREADS, D == 3 ? 3 : 4)
    k_particle_pass(GridParams g, ParticlesF32 p, const float *__restrict__ E,
                    unsigned long long *__restrict__ acc, int mode,
                    double *__restrict__ diag_blocks, int *__restrict__ err)
{
    const int64_t np = p.np;
    const float scale = ldexpf(1.0f, g.fx_bits);
    const int one = 1 << g.fx_bits;
    // FP32 running sums, folded into FP64 every 16 particles of this thread
    float ke = 0.0f, mom[3] = {0.0f, 0.0f, 0.0f};
    double dke = 0.0, dmom[3] = {0.0, 0.0, 0.0};
    int fold = 0;
    bool bad = false;
    // warp-uniform loop: lane i of a warp handles particle base + i
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = warp0 * 32; base < np; base += wstride * 32) {
        const int64_t i = base + lane;
        const bool valid = i < np;
        int c[3] = {0, 0, 0};
        float f[3] = {0.0f, 0.0f, 0.0f};
        float v[3] = {0.0f, 0.0f, 0.0f};
        bool ok = valid;
        if (valid) {
            decode_cell<D>(p.cell[i], g, c);
#pragma unroll
            for (int a = 0; a < D; ++a) f[a] = p.off[a * np + i];
            if (mode & (PASS_PUSH | PASS_MOVE)) {
#pragma unroll
                for (int a = 0; a < NV; ++a) v[a] = p.v[a * np + i];
            }
            if (mode & PASS_PUSH) {
                float e[3] = {0.0f, 0.0f, 0.0f};
                gather_E<D>(E, c, f, g.n, e);
#pragma unroll
                for (int a = 0; a < 3; ++a) e[a] += g.E0[a];
                float vn[3] = {v[0], v[1], v[2]};
                boris(vn, e, g);
                bool finite = true;
#pragma unroll
                for (int a = 0; a < NV; ++a) finite &= isfinite(vn[a]);
                if (!finite) bad = true;
                if (mode & PASS_DIAG) {
                    float o2 = 0.0f, n2 = 0.0f;
#pragma unroll
                    for (int a = 0; a < NV; ++a) {
                        o2 += v[a] * v[a];
                        n2 += vn[a] * vn[a];
                        mom[a] += vn[a];
                    }
                    ke += 0.5f * (o2 + n2);
                    if (++fold == 16) {
                        dke += ke;
                        ke = 0.0f;
#pragma unroll
                        for (int a = 0; a < 3; ++a) {
                            dmom[a] += mom[a];
                            mom[a] = 0.0f;
                        }
                        fold = 0;
                    }
                }
#pragma unroll
                for (int a = 0; a < NV; ++a) {
                    v[a] = vn[a];
                    p.v[a * np + i] = vn[a];
                }
            }
            if (mode & PASS_MOVE) {
                if (move<D>(c, f, v, g)) {
                    p.cell[i] = encode_cell<D>(c, g.n);
#pragma unroll
                    for (int a = 0; a < D; ++a) p.off[a * np + i] = f[a];
                } else {
                    bad = true;
                }
            }
        }
        if (mode & PASS_DEPOSIT) {
            int q[1 << D], node[1 << D];
            cic_quanta<D>(f, scale, one, q);
            corner_nodes<D>(c, g.n, node);
            warp_deposit<D>(acc, ok ? encode_cell<D>(c, g.n) : -1, node, q, one);
        }
    }
    if (bad) latch(err, EF_NONFINITE);
    if (mode & PASS_DIAG) {
        __shared__ double red[4][PP_THREADS / 32];
        double vals[4] = {dke + ke, dmom[0] + mom[0], dmom[1] + mom[1], dmom[2] + mom[2]};
        const int w = threadIdx.x >> 5;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const double s = warp_sum_d(vals[k]);
            if (lane == 0) red[k][w] = s;
        }
        __syncthreads();
        if (threadIdx.x < 4) {
            double s = 0.0;
            for (int j = 0; j < PP_THREADS / 32; ++j) s += red[threadIdx.x][j];
            diag_blocks[blockIdx.x * 4 + threadIdx.x] = s;
        }
    }
}

int particle_pass_blocks(int64_t np, int ndim)
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 148;
    }
    // one resident wave: 4 blocks of 256 per SM (3 in 3D, where the pass needs more
    // registers), each block striding over the particle array
    const int64_t need = (np + PP_THREADS - 1) / PP_THREADS;
    const int64_t cap = (int64_t)sms * (ndim == 3 ? 3 : 4);
    int64_t b = need < cap ? need : cap;
    return (int)(b < 1 ? 1 : b);
}

template <int D, int NV>
static void launch_pass_t(const GridParams &g, ParticlesF32 p, const float *E,
                          unsigned long long *acc, int mode, double *diag_blocks, int nblocks,
                          int *err, cudaStream_t st)
{
    k_particle_pass<D, NV><<<nblocks, PP_THREADS, 0, st>>>(g, p, E, acc, mode, diag_blocks, err);
    note_launch();
}

cudaError_t launch_particle_pass(const GridParams &g, ParticlesF32 p, const float *E,
                                 unsigned long long *acc, bool push, bool mv, bool deposit,
                                 DiagPartials diag, int *err, cudaStream_t st)
{
    if (p.np == 0) return cudaSuccess;
    const int mode = (push ? PASS_PUSH : 0) | (mv ? PASS_MOVE : 0) |
                     (deposit ? PASS_DEPOSIT : 0) | (diag.blocks && push ? PASS_DIAG : 0);
    const int nb = particle_pass_blocks(p.np, g.ndim);
    const int key = g.ndim * 10 + p.nv;
    switch (key) {
    case 11: launch_pass_t<1, 1>(g, p, E, acc, mode, diag.blocks, nb, err, st); break;
    case 12: launch_pass_t<1, 2>(g, p, E, acc, mode, diag.blocks, nb, err, st); break;
    case 13: launch_pass_t<1, 3>(g, p, E, acc, mode, diag.blocks, nb, err, st); break;
    case 22: launch_pass_t<2, 2>(g, p, E, acc, mode, diag.blocks, nb, err, st); break;
    case 23: launch_pass_t<2, 3>(g, p, E, acc, mode, diag.blocks, nb, err, st); break;
    case 33: launch_pass_t<3, 3>(g, p, E, acc, mode, diag.blocks, nb, err, st); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ---- load ------------------------------------------------------------------------------------

// x (count x ndim, row-major FP64) -> cell, offset; v (count x nv) -> FP32.
// Cell and offset are computed in FP64 exactly as c = floor(x / dx),
// f = x / dx - c; x / dx == n (x at L) is node 0; an offset that rounds to
// 1.0f in FP32 is clamped to the largest float below 1 so the cell index stays
// the FP64 one.  Anything outside [0, L] latches EF_NONFINITE.
__global__ void k_load_convert(GridParams g, double dx0, double dx1, double dx2,
                               const double *__restrict__ x, const double *__restrict__ v,
                               ParticlesF32 p, int64_t first, int64_t count, int *err)
{
    const double dx[3] = {dx0, dx1, dx2};
    const int D = g.ndim;
    bool bad = false;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = first + k;
        int c[3] = {0, 0, 0};
        for (int a = 0; a < D; ++a) {
            const double xa = x[k * D + a];
            const double u = xa / dx[a];
            const double fl = floor(u);
            double fa = u - fl;
            int ca;
            if (!(fl >= 0.0 && fl <= (double)g.n[a])) {  // outside [0, L] or NaN
                bad = true;
                ca = 0;
                fa = 0.0;
            } else {
                ca = (int)fl;
                if (ca == g.n[a]) {
                    ca = 0;
                    fa = 0.0;
                }
            }
            float ff = (float)fa;
            if (ff >= 1.0f) ff = 0x1.fffffep-1f;
            c[a] = ca;
            p.off[a * p.np + i] = ff;
        }
        int cell = c[0];
        if (D >= 2) cell += g.n[0] * c[1];
        if (D >= 3) cell += g.n[0] * g.n[1] * c[2];
        p.cell[i] = cell;
        for (int a = 0; a < p.nv; ++a) {
            const float va = (float)v[k * p.nv + a];
            if (!isfinite(va)) bad = true;
            p.v[a * p.np + i] = va;
        }
    }
    if (bad) latch(err, EF_NONFINITE);
}

cudaError_t launch_load_convert(const GridParams &g, const double *dx, const double *x,
                                const double *v, ParticlesF32 p, int64_t first, int64_t count,
                                int *err, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    int64_t nb = (count + 255) / 256;
    if (nb > 65535) nb = 65535;
    k_load_convert<<<(int)nb, 256, 0, st>>>(g, dx[0], dx[1], dx[2], x, v, p, first, count, err);
    note_launch();
    return cudaGetLastError();
}

// Exact FP32 state in host row-major layout (already copied to the device).
__global__ void k_load_state(GridParams g, const int32_t *__restrict__ cell,
                             const float *__restrict__ off, const float *__restrict__ v,
                             ParticlesF32 p, int *err)
{
    const int D = g.ndim;
    const int64_t cells = (int64_t)g.n[0] * (D >= 2 ? g.n[1] : 1) * (D >= 3 ? g.n[2] : 1);
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.np;
         i += (int64_t)gridDim.x * blockDim.x) {
        int c = cell[i];
        if (c < 0 || c >= cells) {
            bad = true;
            c = 0;
        }
        p.cell[i] = c;
        for (int a = 0; a < D; ++a) {
            float fa = off[i * D + a];
            if (!(fa >= 0.0f && fa < 1.0f)) {
                bad = true;
                fa = 0.0f;
            }
            p.off[a * p.np + i] = fa;
        }
        for (int a = 0; a < p.nv; ++a) {
            const float va = v[i * p.nv + a];
            if (!isfinite(va)) bad = true;
            p.v[a * p.np + i] = va;
        }
    }
    if (bad) latch(err, EF_NONFINITE);
}

cudaError_t launch_load_state(const GridParams &g, const int32_t *cell, const float *off,
                              const float *v, ParticlesF32 p, int *err, cudaStream_t st)
{
    if (p.np <= 0) return cudaSuccess;
    int64_t nb = (p.np + 255) / 256;
    if (nb > 65535) nb = 65535;
    k_load_state<<<(int)nb, 256, 0, st>>>(g, cell, off, v, p, err);
    note_launch();
    return cudaGetLastError();
}

// Positions (FP64, row-major np x ndim) = (cell_a + off_a) dx_a.
__global__ void k_positions_f64(GridParams g, double dx0, double dx1, double dx2, ParticlesF32 p,
                                double *__restrict__ x)
{
    const double dx[3] = {dx0, dx1, dx2};
    const int D = g.ndim;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.np;
         i += (int64_t)gridDim.x * blockDim.x) {
        int c[3] = {0, 0, 0};
        const int cell = p.cell[i];
        if (D == 1) decode_cell<1>(cell, g, c);
        else if (D == 2) decode_cell<2>(cell, g, c);
        else decode_cell<3>(cell, g, c);
        for (int a = 0; a < D; ++a)
            x[i * D + a] = ((double)c[a] + (double)p.off[a * p.np + i]) * dx[a];
    }
}

cudaError_t launch_positions_f64(const GridParams &g, const double *dx, ParticlesF32 p, double *x,
                                 cudaStream_t st)
{
    if (p.np <= 0) return cudaSuccess;
    int64_t nb = (p.np + 255) / 256;
    if (nb > 65535) nb = 65535;
    k_positions_f64<<<(int)nb, 256, 0, st>>>(g, dx[0], dx[1], dx[2], p, x);
    note_launch();
    return cudaGetLastError();
}

}  // namespace apk
