// pic_particles.cu -- particle-side kernels of the electrostatic PIC cycle:
// load/convert, and the pass that gathers E (C01), advances v with the Boris
// scheme (A01), moves the particle with periodic wrap and deposits its charge
// (B01) -- the order of the paper's worked example (Sec. 3.1, Listing 1).
//
// Storage: int32 linear cell index, FP32 offsets in [0, 1) per axis (SoA,
// one array per axis), FP32 velocities (SoA).  E is stored per node so that a
// gather takes few vector loads: in 1D and 2D each node holds its own field and
// its upper x-neighbour's (the periodic wrap already applied), so a row of two
// corners is one load (float2 in 1D, float4 in 2D); in 3D one float4 per node.
// (A batch's instances keep one field per node: its pass reads E without
// pairs.)  Charge goes to an int64 fixed-point accumulator: each particle
// deposits exactly 2^S split over its 2^d corners (the last corner takes the
// remainder), so totals are exact and the sum is independent of the order of
// the atomics.
#include <math.h>

#include <type_traits>

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

// CIC gather of E at a particle in cell c, offsets f.  PAIRS: the 1D / 2D pair
// layout (node x holds E(x) and E(x + 1)); otherwise one field per node.
template <int D, bool PAIRS = false>
__device__ __forceinline__ void gather_E(const float *__restrict__ E, const int *c, const float *f,
                                         const int *n, float *e)
{
    if (PAIRS && D == 1) {
        const float2 pr = __ldg(reinterpret_cast<const float2 *>(E) + c[0]);
        e[0] = (1.0f - f[0]) * pr.x + f[0] * pr.y;
        return;
    }
    if (PAIRS && D == 2) {
        const float4 *P = reinterpret_cast<const float4 *>(E);
        const int y0 = c[1] * n[0], y1 = up(c[1], n[1]) * n[0];
        const float4 r0 = __ldg(P + c[0] + y0), r1 = __ldg(P + c[0] + y1);
        const float wx0 = 1.0f - f[0], wx1 = f[0], wy0 = 1.0f - f[1], wy1 = f[1];
        e[0] = wy0 * (wx0 * r0.x + wx1 * r0.z) + wy1 * (wx0 * r1.x + wx1 * r1.z);
        e[1] = wy0 * (wx0 * r0.y + wx1 * r0.w) + wy1 * (wx0 * r1.y + wx1 * r1.w);
        return;
    }
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
// Rounding uses the FMA "magic number" idiom instead of a float-to-int
// conversion (conversions issue on the slow FP64 pipe of this GPU): for
// |x| <= 2^22, fma(w, 2^S, 1.5 * 2^23) rounds w 2^S to the nearest integer
// (ties to even) in the low mantissa bits, exactly once.  S <= 22 keeps every
// quantum in that range and a warp's sum of 32 of them inside int32.
constexpr float RND_MAGIC = 12582912.0f;     // 1.5 * 2^23
constexpr int RND_MAGIC_BITS = 0x4B400000;   // its bit pattern

__device__ __forceinline__ int round_fx(float w, float scale)
{
    return __float_as_int(fmaf(w, scale, RND_MAGIC)) - RND_MAGIC_BITS;
}

template <int D>
__device__ __forceinline__ void cic_quanta(const float *f, float scale, int one, int *q)
{
    const float wx[2] = {1.0f - f[0], f[0]};
    if (D == 1) {
        q[0] = round_fx(wx[0], scale);
        q[1] = one - q[0];
    } else if (D == 2) {
        const float wy[2] = {1.0f - f[1], f[1]};
        q[0] = round_fx(wx[0] * wy[0], scale);
        q[1] = round_fx(wx[1] * wy[0], scale);
        q[2] = round_fx(wx[0] * wy[1], scale);
        q[3] = one - q[0] - q[1] - q[2];
    } else {
        const float wy[2] = {1.0f - f[1], f[1]};
        const float wz[2] = {1.0f - f[2], f[2]};
        int rest = one;
#pragma unroll
        for (int k = 0; k < 7; ++k) {
            q[k] = round_fx(wx[k & 1] * wy[(k >> 1) & 1] * wz[k >> 2], scale);
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
// [0, 1)); cell += shift mod n.  A displacement under one cell (|v dt/dx| < 1,
// the usual case) takes shift from two compares and the fraction from one
// exact add, with no float-to-int conversion; larger ones take floorf.
// Returns false for an absurd displacement (the particle is then left as is).
template <int D>
__device__ __forceinline__ bool move(int *c, float *f, const float *v, const GridParams &g)
{
    float nf[3];
    int nc[3];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const float dsp = v[a] * g.dtdx[a];
        const float o = f[a] + dsp;
        float fr;
        int s;
        if (fabsf(dsp) < 1.0f) {
            // o in (-1, 2): o - 1 is exact on [1, 2); o + 1 may round up to 1
            const bool hi = o >= 1.0f, lo = o < 0.0f;
            fr = hi ? o - 1.0f : (lo ? o + 1.0f : o);
            s = hi ? 1 : (lo ? -1 : 0);
        } else {
            if (!(fabsf(dsp) < 1.0e6f)) return false;
            const float fl = floorf(o);
            fr = o - fl;
            s = (int)fl;
        }
        if (fr >= 1.0f) {  // o a tiny negative number: its fraction rounded up to 1
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

enum : int { PASS_PUSH = 1, PASS_MOVE = 2, PASS_DEPOSIT = 4, PASS_DIAG = 8, PASS_HC = 16 };

// Higuera-Cary advance (A_Pusher, Sec. 2.2) of the momentum per mass u = gamma v
// in FP32, with eps = qmh2 and tau = t (the Boris t vector, (q/m) B h / 2):
//   u- = u + eps E;  sigma = 1 + |u-|^2 / c^2 - |tau|^2;
//   gamma_bar^2 = (sigma + sqrt(sigma^2 + 4 (|tau|^2 + (u-.tau)^2 / c^2))) / 2;
//   t = tau / gamma_bar;  s = 1 / (1 + |t|^2);  u+ = s (u- + (u-.t) t + u- x t);
//   u = u+ + eps E + u+ x t.
// gamma_bar is the Lorentz factor of the mean momentum, so the turn is the
// implicit midpoint rotation; it keeps the relativistic E x B drift exact.
__device__ __forceinline__ void hc_push(float *u, const float *e, const GridParams &g)
{
    float um[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) um[a] = u[a] + g.qmh2 * e[a];
    if (!g.magnetised) {
        // tau = 0: the rotation is the identity (s = 1, t = 0), so u = u- + eps E; the
        // same numbers the general form gives, without its square roots and division
#pragma unroll
        for (int a = 0; a < 3; ++a) u[a] = um[a] + g.qmh2 * e[a];
        return;
    }
    const float tau2 = g.t[0] * g.t[0] + g.t[1] * g.t[1] + g.t[2] * g.t[2];
    const float um2 = um[0] * um[0] + um[1] * um[1] + um[2] * um[2];
    const float ustar = um[0] * g.t[0] + um[1] * g.t[1] + um[2] * g.t[2];
    const float sigma = 1.0f + um2 * g.inv_c2 - tau2;
    const float gbar2 =
        0.5f * (sigma + sqrtf(sigma * sigma + 4.0f * (tau2 + ustar * ustar * g.inv_c2)));
    const float ig = rsqrtf(gbar2);
    const float t[3] = {g.t[0] * ig, g.t[1] * ig, g.t[2] * ig};
    const float s = 1.0f / (1.0f + tau2 * ig * ig);
    const float ut = um[0] * t[0] + um[1] * t[1] + um[2] * t[2];
    const float up[3] = {s * (um[0] + ut * t[0] + (um[1] * t[2] - um[2] * t[1])),
                         s * (um[1] + ut * t[1] + (um[2] * t[0] - um[0] * t[2])),
                         s * (um[2] + ut * t[2] + (um[0] * t[1] - um[1] * t[0]))};
    u[0] = up[0] + g.qmh2 * e[0] + (up[1] * t[2] - up[2] * t[1]);
    u[1] = up[1] + g.qmh2 * e[1] + (up[2] * t[0] - up[0] * t[2]);
    u[2] = up[2] + g.qmh2 * e[2] + (up[0] * t[1] - up[1] * t[0]);
}

// 2 |u|^2 / (gamma + 1): twice the relativistic kinetic energy per mass,
// (gamma - 1) c^2, without cancellation.
template <int NV>
__device__ __forceinline__ float twice_ke_rel(const float *u, float inv_c2)
{
    float u2 = 0.0f;
#pragma unroll
    for (int a = 0; a < NV; ++a) u2 += u[a] * u[a];
    return 2.0f * u2 / (sqrtf(1.0f + u2 * inv_c2) + 1.0f);
}

// ---- TMA bulk-copy pipeline helpers (PTX) ---------------------------------------------------

template <int D>
__host__ __device__ constexpr int tile_of_dim() { return D == 3 ? PASS_TILE_3D : PASS_TILE; }
constexpr int TILE_MAX = PASS_TILE > PASS_TILE_3D ? PASS_TILE : PASS_TILE_3D;
static_assert(BATCH_TILE <= TILE_MAX, "the window bound covers every tile size");
constexpr int WIN_BITS = 11;        // a tile's shared-memory charge window: 2^11 nodes
constexpr int WIN_CAP = 1 << WIN_BITS;
constexpr int STAGES = 3;           // tiles in flight per CTA
constexpr int WAIT_LIMIT = 1 << 26;   // bounded mbarrier polling
// window words at or above WIN_NEG hold negative node totals (see the flush)
constexpr unsigned WIN_NEG = 0u - (unsigned)(4 * TILE_MAX);
static_assert((long long)TILE_MAX * (1ll << 22) < (long long)WIN_NEG,
              "a tile's node total must stay below the negative range of the window");

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Polls the barrier phase with an iteration cap; false if the cap ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity)
{
    for (int k = 0; k < WAIT_LIMIT; ++k)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// 1D bulk copy global -> shared, completing `bytes` of the barrier's transaction count.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                         uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// 1D bulk copy shared -> global (bulk-group completion).
__device__ __forceinline__ void bulk_s2g(void *dst, uint32_t src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(src),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// Waits until at most N committed bulk groups are still reading shared memory.
template <int N>
__device__ __forceinline__ void bulk_wait_read()
{
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Parameters of the tile being processed.
struct TileParams {
    GridParams g;
    const float *E;
    unsigned long long *acc;
};

// One instance: tiles of `tile` (the pass's tile size) consecutive particles of [0, np).
struct SingleSrc {
    static constexpr bool PER_TILE_DIAG = false;
    static constexpr int FIXED_TILE = 0;  // the tile size goes by the dimension
    static constexpr int NT = PP_THREADS;  // threads per CTA
    TileParams tp;
    int64_t np;
    int tile;
    __device__ int64_t ntiles() const { return (np + tile - 1) / tile; }
    __device__ int64_t start(int64_t t) const { return t * tile; }
    __device__ int count(int64_t t) const { return np - t * tile < tile ? (int)(np - t * tile) : tile; }
    __device__ void load_params(int64_t, TileParams *) const {}
    __device__ const TileParams &params(const TileParams &) const { return tp; }
};

// Many instances packed in one arena: tile t covers particles
// [tiles[t].start, + tiles[t].count) of instance tiles[t].inst; tiles of up to
// TILE_ particles, CTAs of NT_ threads (the batch's tuning picks the pair).
template <int TILE_, int NT_>
struct BatchSrcT {
    static constexpr bool PER_TILE_DIAG = true;
    static constexpr int FIXED_TILE = TILE_;
    static constexpr int NT = NT_;
    const BatchTile *tiles;
    const TileParams *inst;  // per instance: parameters, field and accumulator
    int64_t nt;
    __device__ int64_t ntiles() const { return nt; }
    __device__ int64_t start(int64_t t) const { return tiles[t].start; }
    __device__ int count(int64_t t) const { return tiles[t].count; }
    __device__ void load_params(int64_t t, TileParams *dst) const { *dst = inst[tiles[t].inst]; }
    __device__ const TileParams &params(const TileParams &s) const { return s; }
};

// The particle pass.  Persistent CTAs walk tiles of TILE consecutive particles
// (tile t for t = blockIdx.x, + gridDim.x, ...).  One thread streams each tile's
// record arrays (cell, offsets, velocities) into a shared-memory stage with TMA
// bulk copies, STAGES - 1 tiles ahead of the one being computed; the updated
// record is written back into the same stage and returned to global memory by
// TMA bulk stores, so no thread waits on its own loads or stores.  Each thread
// owns R = TILE / 256 particles of a tile and takes all R through each phase
// together (the field gathers are issued together).  The lanes of a warp hold
// particles spread over the whole tile (particle_of): sorted neighbours share a
// cell, and 32 lanes in one or two cells would serialise on the same few window
// words in every shared-memory atomic of the deposit.
// MODE (PASS_* bits) is a compile-time choice so each use carries only its work.
// Src supplies the tiles and the CTA size: one instance (SingleSrc, 256 threads)
// or the tiles of many independent instances packed in one particle arena
// (BatchSrcT, whose tiles each carry their instance's parameters, field and charge
// accumulator, prefetched one tile ahead by one thread).
template <int D, class Src>
__host__ __device__ constexpr int pass_tile()
{
    return Src::FIXED_TILE ? Src::FIXED_TILE : tile_of_dim<D>();
}

// The fixed charge window: FW2_X x FW2_Y nodes in 2D (FW3_X x FW3_Y x FW3_Z in 3D),
// x fastest, placed by a reference cell: the cells up to W / 2 - 1 away from it on
// each axis are inside.  The extents are compile-time constants, so the window
// index and its decode in the flush are a few multiply-adds, and no box of the
// tile's cells (nor the barrier that box needs) is computed.  Particles drift away
// from their sorted tiles over a sort cycle; those outside the window take global
// atomics.  Measured on 512^2 x 64 ppc and 128^3 x 64 ppc over 20-step sort cycles,
// these extents and groups of three tiles in 2D (single tiles in 3D) were the
// fastest tried: larger windows cost more in the flush, smaller ones in spills.
constexpr int TILE_GROUP = 3, TILE_GROUP_3D = 1;
constexpr int FW2_X = 40, FW2_Y = 20;
constexpr int FW3_X = 16, FW3_Y = 16, FW3_Z = 8;
template <int D>
__host__ __device__ constexpr bool fixed_window() { return D >= 2; }
template <int D>
__host__ __device__ constexpr int fw_ext(int a)
{
    return D == 2 ? (a == 0 ? FW2_X : FW2_Y) : (a == 0 ? FW3_X : (a == 1 ? FW3_Y : FW3_Z));
}
// window stride of axis a
template <int D>
__host__ __device__ constexpr int fw_stride(int a)
{
    return a == 0 ? 1 : (a == 1 ? fw_ext<D>(0) : fw_ext<D>(0) * fw_ext<D>(1));
}
template <int D>
__host__ __device__ constexpr int fw_total() { return fw_stride<D>(D - 1) * fw_ext<D>(D - 1); }
// window offset of corner k (bit a of k: the upper node on axis a)
template <int D>
__host__ __device__ constexpr int fw_corner(int k)
{
    return (k & 1) + (D > 1 ? ((k >> 1) & 1) * fw_stride<D>(1) : 0) +
           (D > 2 ? ((k >> 2) & 1) * fw_stride<D>(2) : 0);
}

// Words of the charge window: the fixed window, else the largest dynamic box.
template <int D>
__host__ __device__ constexpr int win_cap() { return fixed_window<D>() ? fw_total<D>() : WIN_CAP; }

// Tile groups (2D single instances): a CTA takes TILE_GROUP consecutive tiles of the
// sorted order, each depositing into a window of its own, and flushes the windows
// together after the last of them (one global atomic per node for the group, whose
// tiles share most of their nodes).  Separate 32-bit windows keep the per-tile bound
// of the window words; the flush sums them in 64 bits.
template <int D, class Src>
__host__ __device__ constexpr int tile_group()
{
    return Src::PER_TILE_DIAG ? 1 : (D == 2 ? TILE_GROUP : (D == 3 ? TILE_GROUP_3D : 1));
}
template <int D, class Src>
__host__ __device__ constexpr int win_words() { return win_cap<D>() * tile_group<D, Src>(); }

// Particle (index within the tile) of slot r of thread `tid`, for tiles of
// R * 32 NW particles (NW warps) seen as NW R rows of 32: lane i of warp w takes
// column i of row (w R + r + i) mod NW R.  For each column the pairs (w, r) cover
// every row once, so a warp's lanes are spread over the tile, while every
// shared-memory access of the record (one column per lane) stays free of bank
// conflicts.
template <int R, int NW>
__device__ __forceinline__ int particle_of(int r, int tid)
{
    const int lane = tid & 31;
    return 32 * (((tid >> 5) * R + r + lane) % (NW * R)) + lane;
}

// Resident CTAs per SM that the launch bounds ask for: a single instance's pass
// by its tile (3D: 4, 64 registers without spills, 4.7 % faster than 3 at 80
// registers on 128^3 x 64 ppc; 512-particle tiles: 5; 768: 4); a batch variant about
// 1,280 threads per SM (registers kept near 50).
template <int D, class Src>
__host__ __device__ constexpr int pass_min_blocks()
{
    return Src::PER_TILE_DIAG ? (1280 / Src::NT > 0 ? 1280 / Src::NT : 1)
                              : (D == 3 ? 4 : (pass_tile<D, Src>() == 512 ? 5 : 4));
}

template <int D, int NV, int MODE, class Src>
__global__ void __launch_bounds__(Src::NT, pass_min_blocks<D, Src>())
    k_particle_pass(Src src, ParticlesF32 p, double *__restrict__ diag_blocks,
                    int *__restrict__ err)
{
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int NT = Src::NT;
    constexpr int TILE = pass_tile<D, Src>();
    constexpr int R = TILE / NT;
    static_assert(R * NT == TILE, "a tile is R particles per thread");
    constexpr int NA_MAX = 1 + D + NV;
    constexpr bool PUSH = (MODE & PASS_PUSH) != 0, MOVE = (MODE & PASS_MOVE) != 0;
    constexpr bool DEPOSIT = (MODE & PASS_DEPOSIT) != 0, DIAG = (MODE & PASS_DIAG) != 0;
    constexpr bool HC = (MODE & PASS_HC) != 0;  // Higuera-Cary push, move at u / gamma
    constexpr bool NEED_V = PUSH || MOVE;
    constexpr int NA = 1 + D + (NEED_V ? NV : 0);
    constexpr bool WRITE = PUSH || MOVE;  // the record changes and goes back to global
    constexpr bool FIXED_WIN = fixed_window<D>();
    constexpr int G = tile_group<D, Src>();
    float *stage_base = reinterpret_cast<float *>(smem);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)STAGES * NA_MAX * TILE * 4);
    // the charge windows (int32 fixed point, kept zero between flushes: in 2D and 3D
    // one fixed window per tile of a group, in 1D one window sized by the tile's box)
    // and, in 1D, the tile's box of new cells (min, max of the unwrapped offset from
    // the tile's reference cell, per axis)
    unsigned *s_win = reinterpret_cast<unsigned *>(bars + STAGES);
    int *s_box = reinterpret_cast<int *>(s_win + win_words<D, Src>());
    // the current and the next tile's parameters (copied by one thread for a batch,
    // one tile ahead), the tile's reference cell, and per-warp diagnostic partials
    // of a batch tile
    __shared__ TileParams s_tp[2];
    __shared__ int s_ref_cell;
    __shared__ float s_diag[NT / 32][4];

    // groups of G consecutive tiles: group blockIdx.x + j gridDim.x for this CTA (the
    // last group of the grid short when G does not divide ntiles).  Interleaving the
    // groups across CTAs measured faster than a contiguous range of tiles per CTA,
    // which would balance the tail better.
    const int64_t ntiles = src.ntiles();
    const int64_t ngroups = (ntiles + G - 1) / G;
    int my_tiles = blockIdx.x < ngroups ? (int)((ngroups - 1 - blockIdx.x) / gridDim.x + 1) : 0;
    if (G > 1) {
        my_tiles *= G;
        if (my_tiles > 0 && (ngroups - 1) % gridDim.x == blockIdx.x)
            my_tiles -= (int)(G * ngroups - ntiles);
    }
    const int tid = threadIdx.x, lane = tid & 31;

    // stage s, array a (0: cell, 1..D: offsets, D+1..: velocities)
    auto stage_arr = [&](int st, int a) { return stage_base + ((size_t)st * NA_MAX + a) * TILE; };
    auto tile_of = [&](int k) {
        return G > 1 ? G * ((int64_t)blockIdx.x + (int64_t)(k / G) * gridDim.x) + k % G
                     : (int64_t)blockIdx.x + (int64_t)k * gridDim.x;
    };
    auto tile_bytes = [&](int64_t t) { return (uint32_t)(((src.count(t) + 3) / 4) * 16); };
    auto issue_load = [&](int k, int st) {
        const int64_t t = tile_of(k);
        const int64_t start = src.start(t);
        const uint32_t bytes = tile_bytes(t);
        const uint32_t bar = smem_addr(&bars[st]);
        mbar_expect_tx(bar, bytes * (uint32_t)NA);
        bulk_g2s(smem_addr(stage_arr(st, 0)), p.cell + start, bytes, bar);
#pragma unroll
        for (int a = 0; a < D; ++a)
            bulk_g2s(smem_addr(stage_arr(st, 1 + a)), p.off + a * p.stride + start, bytes, bar);
        if (NEED_V) {
#pragma unroll
            for (int a = 0; a < NV; ++a)
                bulk_g2s(smem_addr(stage_arr(st, 1 + D + a)), p.v + a * p.stride + start, bytes,
                         bar);
        }
    };
    auto issue_store = [&](int k, int st) {
        const int64_t t = tile_of(k);
        const int64_t start = src.start(t);
        const uint32_t bytes = tile_bytes(t);
        if (MOVE) {
            bulk_s2g(p.cell + start, smem_addr(stage_arr(st, 0)), bytes);
#pragma unroll
            for (int a = 0; a < D; ++a)
                bulk_s2g(p.off + a * p.stride + start, smem_addr(stage_arr(st, 1 + a)), bytes);
        }
        if (PUSH) {
#pragma unroll
            for (int a = 0; a < NV; ++a)
                bulk_s2g(p.v + a * p.stride + start, smem_addr(stage_arr(st, 1 + D + a)), bytes);
        }
        bulk_commit();
    };

    if (tid == 0) {
        for (int st = 0; st < STAGES; ++st) mbar_init(smem_addr(&bars[st]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (my_tiles > 0) src.load_params(tile_of(0), &s_tp[0]);
    }
    if (DEPOSIT) {
        for (int i = tid; i < win_words<D, Src>(); i += NT) s_win[i] = 0u;
        if (tid < 3) {
            s_box[tid] = 0x7fffffff;
            s_box[3 + tid] = -0x7fffffff;
        }
    }
    __syncthreads();
    if (tid == 0)
        for (int k = 0; k < STAGES - 1 && k < my_tiles; ++k) issue_load(k, k);

    // diagnostics: FP32 sums over this thread's particles (at most a few hundred, or
    // one batch tile), reduced across threads and blocks in FP64
    float ke = 0.0f, mom[3] = {0.0f, 0.0f, 0.0f};
    bool bad = false;

    for (int k = 0; k < my_tiles; ++k) {
        const int st = k % STAGES;
        const uint32_t parity = (uint32_t)((k / STAGES) & 1);
        const int64_t t = tile_of(k);
        // the next tile's parameters (its slot was last read by the previous tile,
        // finished at that tile's closing barrier); this tile's came one tile ago
        if (tid == 0 && k + 1 < my_tiles) src.load_params(tile_of(k + 1), &s_tp[(k + 1) & 1]);
        const bool ok_wait = mbar_wait_bounded(smem_addr(&bars[st]), parity);
        // the tile's reference cell (before the move: the cell of its first particle
        // for the box, of its middle one for the fixed window, of the last one of the
        // first tile of a group of several), kept before the barrier so that no
        // thread overwrites it first
        const int kg = k % G;  // the tile's place in its group
        if (tid == 0 && ok_wait && kg == 0) {
            const int cnt0 = src.count(t);
            const bool several = G > 1 && k + 1 < my_tiles;
            s_ref_cell = reinterpret_cast<const int32_t *>(stage_arr(st, 0))[
                several ? cnt0 - 1 : (FIXED_WIN ? (cnt0 - 1) / 2 : 0)];
        }
        if (__syncthreads_or(!ok_wait)) {
            // a copy did not land within the cap: report, drain what is in flight, stop
            if (tid == 0) {
                latch(err, EF_TIMEOUT);
                for (int kk = k; kk < my_tiles && kk < k + STAGES - 1; ++kk)
                    mbar_wait_bounded(smem_addr(&bars[kk % STAGES]),
                                      (uint32_t)((kk / STAGES) & 1));
                bulk_wait_all();
            }
            __syncthreads();
            return;
        }
        const TileParams &tp = src.params(s_tp[k & 1]);
        const GridParams &g = tp.g;
        const float *__restrict__ E = tp.E;
        unsigned long long *__restrict__ acc = tp.acc;
        const float scale = ldexpf(1.0f, g.fx_bits);
        const int one = 1 << g.fx_bits;
        const int cnt = src.count(t);
        int32_t *s_cell = reinterpret_cast<int32_t *>(stage_arr(st, 0));
        int ref[3] = {0, 0, 0};
        if (DEPOSIT) decode_cell<D>(s_ref_cell, g, ref);

        // phase A: read the record, decode the cell, issue the field gathers
        int c[R][3];
        float f[R][3], v[R][3], e[R][3];
        bool valid[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int j = particle_of<R, NT / 32>(r, tid);
            valid[r] = j < cnt;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                c[r][a] = 0;
                f[r][a] = 0.0f;
                v[r][a] = 0.0f;
                e[r][a] = 0.0f;
            }
            if (valid[r]) {
                decode_cell<D>(s_cell[j], g, c[r]);
#pragma unroll
                for (int a = 0; a < D; ++a) f[r][a] = stage_arr(st, 1 + a)[j];
                if (NEED_V) {
#pragma unroll
                    for (int a = 0; a < NV; ++a) v[r][a] = stage_arr(st, 1 + D + a)[j];
                }
                if (PUSH) gather_E<D, !Src::PER_TILE_DIAG>(E, c[r], f[r], g.n, e[r]);
            }
        }
        // phase B: push, move, write the record back into the stage
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (!valid[r]) continue;
            const int j = particle_of<R, NT / 32>(r, tid);
            bool finite = true;
            if (PUSH) {
#pragma unroll
                for (int a = 0; a < 3; ++a) e[r][a] += g.E0[a];
                float vn[3] = {v[r][0], v[r][1], v[r][2]};
                if (HC) hc_push(vn, e[r], g);
                else boris(vn, e[r], g);
#pragma unroll
                for (int a = 0; a < NV; ++a) finite &= isfinite(vn[a]);
                if (DIAG) {
                    float o2 = 0.0f, n2 = 0.0f;
                    if (HC) {
                        o2 = twice_ke_rel<NV>(v[r], g.inv_c2);
                        n2 = twice_ke_rel<NV>(vn, g.inv_c2);
                    } else {
#pragma unroll
                        for (int a = 0; a < NV; ++a) {
                            o2 += v[r][a] * v[r][a];
                            n2 += vn[a] * vn[a];
                        }
                    }
#pragma unroll
                    for (int a = 0; a < NV; ++a) mom[a] += vn[a];
                    ke += 0.5f * (o2 + n2);
                }
#pragma unroll
                for (int a = 0; a < NV; ++a) {
                    v[r][a] = vn[a];
                    stage_arr(st, 1 + D + a)[j] = vn[a];
                }
            }
            if (MOVE) {
                // dx/dt: v, or u / gamma for the relativistic pusher
                float w[3] = {v[r][0], v[r][1], v[r][2]};
                if (HC) {
                    float u2 = 0.0f;
#pragma unroll
                    for (int a = 0; a < NV; ++a) u2 += v[r][a] * v[r][a];
                    const float ig = rsqrtf(1.0f + u2 * g.inv_c2);
#pragma unroll
                    for (int a = 0; a < 3; ++a) w[a] *= ig;
                }
                if (finite && move<D>(c[r], f[r], w, g)) {
                    s_cell[j] = encode_cell<D>(c[r], g.n);
#pragma unroll
                    for (int a = 0; a < D; ++a) stage_arr(st, 1 + a)[j] = f[r][a];
                } else {
                    finite = false;
                }
            }
            if (!finite) bad = true;
        }
        // phase C: deposit at the (new) positions.  The tile's particles occupy a few
        // cells around its reference cell (they were sorted): corners inside the
        // shared-memory window are added there, and each touched node goes to the
        // global accumulator once per flush; other corners go to global memory.  In
        // 2D and 3D the window is fixed; in 1D it is the box of the tile's cells.
        if (DEPOSIT && FIXED_WIN) {
            // the fixed window: its origin (the node of window index 0) sits half the
            // window below the reference cell, wrapped into the grid; an axis shorter
            // than the window takes origin 0, so that every cell is inside and the
            // upper node of the last cell has a slot of its own (flushed to node 0)
            int org[3] = {0, 0, 0};
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const int W = fw_ext<D>(a);
                int o = ref[a] - (W / 2 - 1);
                o += o < 0 ? g.n[a] : 0;
                org[a] = g.n[a] >= W ? o : 0;
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (!valid[r]) continue;
                int q[1 << D];
                cic_quanta<D>(f[r], scale, one, q);
                unsigned base = 0u;
                bool in = true;
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    int d = c[r][a] - org[a];
                    d += d < 0 ? g.n[a] : 0;
                    in = in && d < fw_ext<D>(a) - 1;
                    base += (unsigned)d * (unsigned)fw_stride<D>(a);
                }
                if (in) {
                    unsigned *w = s_win + kg * fw_total<D>();
#pragma unroll
                    for (int kc = 0; kc < (1 << D); ++kc)
                        atomicAdd(&w[base + fw_corner<D>(kc)], (unsigned)q[kc]);
                } else {
                    int node[1 << D];
                    corner_nodes<D>(c[r], g.n, node);
#pragma unroll
                    for (int kc = 0; kc < (1 << D); ++kc)
                        atomicAdd(acc + node[kc], (unsigned long long)(long long)q[kc]);
                }
            }
            // flush as below, over the whole fixed window (with tile groups, after the
            // last tile of the group, or the CTA's last tile)
            const bool flush = kg == G - 1 || k + 1 == my_tiles;
            if (flush) __syncthreads();
            for (int i = tid; flush && i < fw_total<D>(); i += NT) {
                unsigned u[G];
                unsigned any = 0u;
#pragma unroll
                for (int h = 0; h < G; ++h) {
                    u[h] = s_win[h * fw_total<D>() + i];
                    any |= u[h];
                }
                if (any == 0u) continue;
                long long val = 0;
#pragma unroll
                for (int h = 0; h < G; ++h) {
                    s_win[h * fw_total<D>() + i] = 0u;
                    val += u[h] >= WIN_NEG ? (long long)u[h] - (1ll << 32) : (long long)u[h];
                }
                int node = 0, stride = 1;
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    int x = org[a] + (int)(((unsigned)i / fw_stride<D>(a)) % fw_ext<D>(a));
                    x -= x >= g.n[a] ? g.n[a] : 0;
                    node += x * stride;
                    stride *= g.n[a];
                }
                atomicAdd(acc + node, (unsigned long long)val);
            }
        } else if (DEPOSIT) {
            int q[R][1 << D], dd[R][3];
            int lo[3], hi[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                lo[a] = 0x7fffffff;
                hi[a] = -0x7fffffff;
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                cic_quanta<D>(f[r], scale, one, q[r]);
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    int d = c[r][a] - ref[a];  // unwrapped to [-n/2, n/2]
                    d -= (2 * d > g.n[a]) ? g.n[a] : 0;
                    d += (2 * d < -g.n[a]) ? g.n[a] : 0;
                    dd[r][a] = d;
                    if (valid[r]) {
                        lo[a] = min(lo[a], d);
                        hi[a] = max(hi[a], d);
                    }
                }
            }
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const int wl = __reduce_min_sync(0xffffffffu, lo[a]);
                const int wh = __reduce_max_sync(0xffffffffu, hi[a]);
                if (lane == 0) {
                    atomicMin(&s_box[a], wl);
                    atomicMax(&s_box[3 + a], wh);
                }
            }
            __syncthreads();
            // window extents rounded up to powers of two: index = sum of shifted offsets
            int sh[3] = {0, 0, 0}, bits[3] = {0, 0, 0}, blo[3] = {0, 0, 0};
            int tot_bits = 0;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                blo[a] = s_box[a];
                const int w = s_box[3 + a] - blo[a] + 2;  // cells lo..hi and the node above
                sh[a] = tot_bits;
                bits[a] = 32 - __clz(w - 1);              // ceil(log2 w)
                tot_bits += bits[a];
            }
            const bool use_win =
                tot_bits <= WIN_BITS && (1 << tot_bits) <= win_cap<D>() && s_box[3] >= s_box[0];
            if (use_win) {
                // shared-memory atomics into the window: corner k of a particle sits at
                // its cell's window index plus a per-tile offset
                int coff[1 << D];
#pragma unroll
                for (int kc = 0; kc < (1 << D); ++kc) {
                    coff[kc] = 0;
#pragma unroll
                    for (int a = 0; a < D; ++a) coff[kc] += ((kc >> a) & 1) << sh[a];
                }
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if (valid[r]) {
                        int base = 0;
#pragma unroll
                        for (int a = 0; a < D; ++a) base += (dd[r][a] - blo[a]) << sh[a];
#pragma unroll
                        for (int kc = 0; kc < (1 << D); ++kc)
                            atomicAdd(&s_win[base + coff[kc]], (unsigned)q[r][kc]);
                    }
            } else {
                // a box too large for the window (particles far from sorted order,
                // dilute plasmas): each corner straight to the global accumulator
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if (valid[r]) {
                        int node[1 << D];
                        corner_nodes<D>(c[r], g.n, node);
#pragma unroll
                        for (int kc = 0; kc < (1 << D); ++kc)
                            atomicAdd(acc + node[kc], (unsigned long long)(long long)q[r][kc]);
                    }
            }
            __syncthreads();
            if (use_win) {
                // flush: every touched node once to global memory, leaving the window zero.
                // A node's tile total lies in [-2 TILE, TILE * 2^S] with S <= 22 (a
                // particle's last corner quantum is at least -2), so its 32 bits
                // decode unambiguously: WIN_NEG and above are the negative totals.
                const int total = 1 << tot_bits;
                for (int i = tid; i < total; i += NT) {
                    const unsigned u = s_win[i];
                    if (u == 0u) continue;
                    s_win[i] = 0u;
                    const long long val =
                        u >= WIN_NEG ? (long long)u - (1ll << 32) : (long long)u;
                    int node = 0, stride = 1;
#pragma unroll
                    for (int a = 0; a < D; ++a) {
                        const int la = (i >> sh[a]) & ((1 << bits[a]) - 1);
                        int x = ref[a] + blo[a] + la;
                        x += x < 0 ? g.n[a] : 0;
                        x -= x >= g.n[a] ? g.n[a] : 0;
                        node += x * stride;
                        stride *= g.n[a];
                    }
                    atomicAdd(acc + node, (unsigned long long)val);
                }
            }
            if (tid < 3) {  // reset the box for the next tile (read by all before the sync)
                s_box[tid] = 0x7fffffff;
                s_box[3 + tid] = -0x7fffffff;
            }
        }
        if (DIAG && Src::PER_TILE_DIAG) {
            // this tile's sums, per warp, then per tile below (fixed order)
            float vals[4] = {ke, mom[0], mom[1], mom[2]};
#pragma unroll
            for (int kq = 0; kq < 4; ++kq) {
                float x = vals[kq];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                if (lane == 0) s_diag[tid >> 5][kq] = x;
            }
            ke = 0.0f;
            mom[0] = mom[1] = mom[2] = 0.0f;
        }
        // the stage is complete: make the generic-proxy writes visible to the bulk
        // copies, store it back, and refill the stage consumed one tile ago
        if (WRITE) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (DIAG && Src::PER_TILE_DIAG && tid < 4) {
            double sum = 0.0;
            for (int jw = 0; jw < NT / 32; ++jw) sum += (double)s_diag[jw][tid];
            diag_blocks[t * 4 + tid] = sum;
        }
        if (tid == 0) {
            if (WRITE) issue_store(k, st);
            const int kn = k + STAGES - 1;
            if (kn < my_tiles) {
                const int sn = kn % STAGES;  // the stage of tile k - 1 (free since then)
                if (WRITE && k >= 1) bulk_wait_read<1>();  // tile k - 1's store has read it
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue_load(kn, sn);
            }
        }
    }
    if (tid == 0 && WRITE) bulk_wait_all();
    if (bad) latch(err, EF_NONFINITE);
    if (DIAG && !Src::PER_TILE_DIAG) {
        __shared__ double red[4][NT / 32];
        double vals[4] = {ke, mom[0], mom[1], mom[2]};
        const int w = tid >> 5;
#pragma unroll
        for (int kq = 0; kq < 4; ++kq) {
            const double sum = warp_sum_d(vals[kq]);
            if (lane == 0) red[kq][w] = sum;
        }
        __syncthreads();
        if (tid < 4) {
            double sum = 0.0;
            for (int jw = 0; jw < NT / 32; ++jw) sum += red[tid][jw];
            diag_blocks[blockIdx.x * 4 + tid] = sum;
        }
    }
}

template <int D, int NV, class Src>
constexpr size_t pass_smem_bytes()
{
    return (size_t)STAGES * (1 + D + NV) * pass_tile<D, Src>() * 4 + STAGES * 8 +
           win_words<D, Src>() * 4 +
           8 * 4;
}

int sm_count()
{
    static std::atomic<int> sms{0};
    int n = sms.load(std::memory_order_relaxed);
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            n <= 0) {
            cudaGetLastError();
            n = 148;
        }
        sms.store(n, std::memory_order_relaxed);
    }
    return n;
}

// CTAs of the pass resident per SM, from the occupancy calculator for the fused
// pass with diagnostics (every mode of a (D, NV, Src) has the same dynamic shared
// memory, and the launch bounds give each at least this many).
template <int D, int NV, class Src = SingleSrc>
int pass_ctas_per_sm()
{
    static std::atomic<int> cached{0};
    int c = cached.load(std::memory_order_relaxed);
    if (c) return c;
    constexpr size_t smem = pass_smem_bytes<D, NV, Src>();
    auto k = k_particle_pass<D, NV, PASS_PUSH | PASS_MOVE | PASS_DEPOSIT | PASS_DIAG, Src>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, k, Src::NT, smem) != cudaSuccess ||
        c < 1) {
        cudaGetLastError();
        c = 1;
    }
    cached.store(c, std::memory_order_relaxed);
    return c;
}

int particle_pass_blocks(int64_t np, int ndim, int nv)
{
    int per_sm = 1;
    switch (ndim * 10 + nv) {
    case 11: per_sm = pass_ctas_per_sm<1, 1>(); break;
    case 12: per_sm = pass_ctas_per_sm<1, 2>(); break;
    case 13: per_sm = pass_ctas_per_sm<1, 3>(); break;
    case 22: per_sm = pass_ctas_per_sm<2, 2>(); break;
    case 23: per_sm = pass_ctas_per_sm<2, 3>(); break;
    default: per_sm = pass_ctas_per_sm<3, 3>(); break;
    }
    // one resident wave of persistent CTAs, each walking tiles of particles
    const int64_t tile = ndim == 3 ? PASS_TILE_3D : PASS_TILE;
    const int64_t need = (np + tile - 1) / tile;
    const int64_t cap = (int64_t)sm_count() * per_sm;
    const int64_t b = need < cap ? need : cap;
    return (int)(b < 1 ? 1 : b);
}

template <int D, int NV, int MODE, class Src>
static cudaError_t launch_pass_m(const Src &src, ParticlesF32 p, double *diag_blocks, int nblocks,
                                 int *err, cudaStream_t st)
{
    constexpr size_t smem = pass_smem_bytes<D, NV, Src>();
    static std::atomic<unsigned long long> configured{0};
    cudaError_t e = once_per_device(configured, [] {
        return cudaFuncSetAttribute(k_particle_pass<D, NV, MODE, Src>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
    if (e != cudaSuccess) return e;
    k_particle_pass<D, NV, MODE, Src><<<nblocks, Src::NT, smem, st>>>(src, p, diag_blocks, err);
    note_launch();
    return cudaGetLastError();
}

template <int D, int NV, class Src>
static cudaError_t launch_pass_t(const Src &src, ParticlesF32 p, int mode, double *diag_blocks,
                                 int nb, int *err, cudaStream_t st)
{
    constexpr int FUSED = PASS_PUSH | PASS_MOVE | PASS_DEPOSIT;
    constexpr int GP = PASS_PUSH | PASS_MOVE;
    if constexpr (std::is_same<Src, SingleSrc>::value) {
        // the relativistic pusher (single instances only)
        constexpr int H = PASS_HC;
        switch (mode) {
        case FUSED | H: return launch_pass_m<D, NV, FUSED | H>(src, p, diag_blocks, nb, err, st);
        case FUSED | PASS_DIAG | H:
            return launch_pass_m<D, NV, FUSED | PASS_DIAG | H>(src, p, diag_blocks, nb, err, st);
        case GP | H: return launch_pass_m<D, NV, GP | H>(src, p, diag_blocks, nb, err, st);
        case GP | PASS_DIAG | H:
            return launch_pass_m<D, NV, GP | PASS_DIAG | H>(src, p, diag_blocks, nb, err, st);
        case PASS_PUSH | H: return launch_pass_m<D, NV, PASS_PUSH | H>(src, p, diag_blocks, nb, err, st);
        default: break;
        }
    }
    switch (mode) {
    case FUSED: return launch_pass_m<D, NV, FUSED>(src, p, diag_blocks, nb, err, st);
    case FUSED | PASS_DIAG:
        return launch_pass_m<D, NV, FUSED | PASS_DIAG>(src, p, diag_blocks, nb, err, st);
    case GP: return launch_pass_m<D, NV, GP>(src, p, diag_blocks, nb, err, st);
    case GP | PASS_DIAG:
        return launch_pass_m<D, NV, GP | PASS_DIAG>(src, p, diag_blocks, nb, err, st);
    case PASS_DEPOSIT: return launch_pass_m<D, NV, PASS_DEPOSIT>(src, p, diag_blocks, nb, err, st);
    case PASS_PUSH: return launch_pass_m<D, NV, PASS_PUSH>(src, p, diag_blocks, nb, err, st);
    default: return cudaErrorInvalidValue;
    }
}

static int pass_mode(bool push, bool mv, bool deposit, bool diag)
{
    return (push ? PASS_PUSH : 0) | (mv ? PASS_MOVE : 0) | (deposit ? PASS_DEPOSIT : 0) |
           (diag && push && mv ? PASS_DIAG : 0);
}

cudaError_t launch_particle_pass(const GridParams &g, ParticlesF32 p, const float *E,
                                 unsigned long long *acc, bool push, bool mv, bool deposit,
                                 DiagPartials diag, int *err, cudaStream_t st)
{
    if (p.np == 0) return cudaSuccess;
    const int mode = pass_mode(push, mv, deposit, diag.blocks != nullptr) |
                     (push && g.pusher == AP_PIC_PUSHER_HIGUERA_CARY ? PASS_HC : 0);
    const int nb = particle_pass_blocks(p.np, g.ndim, p.nv);
    SingleSrc src;
    src.tp.g = g;
    src.tp.E = E;
    src.tp.acc = acc;
    src.np = p.np;
    src.tile = g.ndim == 3 ? PASS_TILE_3D : PASS_TILE;
    switch (g.ndim * 10 + p.nv) {
    case 11: return launch_pass_t<1, 1>(src, p, mode, diag.blocks, nb, err, st);
    case 12: return launch_pass_t<1, 2>(src, p, mode, diag.blocks, nb, err, st);
    case 13: return launch_pass_t<1, 3>(src, p, mode, diag.blocks, nb, err, st);
    case 22: return launch_pass_t<2, 2>(src, p, mode, diag.blocks, nb, err, st);
    case 23: return launch_pass_t<2, 3>(src, p, mode, diag.blocks, nb, err, st);
    case 33: return launch_pass_t<3, 3>(src, p, mode, diag.blocks, nb, err, st);
    default: return cudaErrorInvalidValue;
    }
}

// The batch pass's (threads per CTA, particles per thread) variants.
struct BatchVariant {
    int threads, per_thread;
};
constexpr BatchVariant BATCH_VARIANTS[] = {{256, 2}, {128, 2}, {128, 4}, {256, 1}, {256, 3},
                                           {512, 1}};
constexpr int N_BATCH_VARIANTS = (int)(sizeof(BATCH_VARIANTS) / sizeof(BATCH_VARIANTS[0]));

int batch_variant(int threads, int per_thread)
{
    for (int k = 0; k < N_BATCH_VARIANTS; ++k)
        if (BATCH_VARIANTS[k].threads == threads && BATCH_VARIANTS[k].per_thread == per_thread)
            return k;
    return -1;
}

int batch_variant_count() { return N_BATCH_VARIANTS; }

void batch_variant_shape(int variant, int *threads, int *per_thread)
{
    const BatchVariant v = BATCH_VARIANTS[variant >= 0 && variant < N_BATCH_VARIANTS ? variant : 0];
    *threads = v.threads;
    *per_thread = v.per_thread;
}

template <int NT, int PT>
static cudaError_t launch_batch_variant(int ndim, const BatchTile *tiles, int64_t ntiles,
                                        const void *inst_params, ParticlesF32 p, int mode,
                                        double *diag_tiles, int nblocks, int *err,
                                        cudaStream_t st)
{
    using Src = BatchSrcT<NT * PT, NT>;
    Src src;
    src.tiles = tiles;
    src.inst = static_cast<const TileParams *>(inst_params);
    src.nt = ntiles;
    // at most one resident wave, whatever the tuning asks for
    const int64_t wave = (int64_t)sm_count() *
                         (ndim == 1 ? pass_ctas_per_sm<1, 2, Src>() : pass_ctas_per_sm<2, 2, Src>());
    int64_t nb64 = nblocks < ntiles ? nblocks : ntiles;
    nb64 = nb64 < wave ? nb64 : wave;
    const int nb = (int)(nb64 < 1 ? 1 : nb64);
    switch (ndim * 10 + p.nv) {
    case 12: return launch_pass_t<1, 2>(src, p, mode, diag_tiles, nb, err, st);
    case 22: return launch_pass_t<2, 2>(src, p, mode, diag_tiles, nb, err, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_batch_pass(int ndim, int variant, const BatchTile *tiles, int64_t ntiles,
                              const void *inst_params, ParticlesF32 p, bool push, bool mv,
                              bool deposit, double *diag_tiles, int nblocks, int *err,
                              cudaStream_t st)
{
    if (ntiles == 0) return cudaSuccess;
    const int mode = pass_mode(push, mv, deposit, diag_tiles != nullptr);
    switch (variant) {
    case 0: return launch_batch_variant<256, 2>(ndim, tiles, ntiles, inst_params, p, mode,
                                               diag_tiles, nblocks, err, st);
    case 1: return launch_batch_variant<128, 2>(ndim, tiles, ntiles, inst_params, p, mode,
                                               diag_tiles, nblocks, err, st);
    case 2: return launch_batch_variant<128, 4>(ndim, tiles, ntiles, inst_params, p, mode,
                                               diag_tiles, nblocks, err, st);
    case 3: return launch_batch_variant<256, 1>(ndim, tiles, ntiles, inst_params, p, mode,
                                               diag_tiles, nblocks, err, st);
    case 4: return launch_batch_variant<256, 3>(ndim, tiles, ntiles, inst_params, p, mode,
                                               diag_tiles, nblocks, err, st);
    case 5: return launch_batch_variant<512, 1>(ndim, tiles, ntiles, inst_params, p, mode,
                                               diag_tiles, nblocks, err, st);
    default: return cudaErrorInvalidValue;
    }
}

size_t batch_tile_params_bytes() { return sizeof(TileParams); }

void make_tile_params(void *dst, const GridParams &g, const float *E, unsigned long long *acc)
{
    TileParams *t = static_cast<TileParams *>(dst);
    t->g = g;
    t->E = E;
    t->acc = acc;
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
            p.off[a * p.stride + i] = ff;
        }
        int cell = c[0];
        if (D >= 2) cell += g.n[0] * c[1];
        if (D >= 3) cell += g.n[0] * g.n[1] * c[2];
        p.cell[i] = cell;
        for (int a = 0; a < p.nv; ++a) {
            const float va = (float)v[k * p.nv + a];
            if (!isfinite(va)) bad = true;
            p.v[a * p.stride + i] = va;
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
            p.off[a * p.stride + i] = fa;
        }
        for (int a = 0; a < p.nv; ++a) {
            const float va = v[i * p.nv + a];
            if (!isfinite(va)) bad = true;
            p.v[a * p.stride + i] = va;
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
            x[i * D + a] = ((double)c[a] + (double)p.off[a * p.stride + i]) * dx[a];
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
