// pic_batch.cu -- many independent periodic PIC instances of uneven grid and
// particle counts advanced together (the serving form of the cycle of the
// paper's worked example, Sec. 3.1, Listing 1).
//
// Layout: one particle arena (the FP32 cell + offset SoA of every instance,
// each instance's range starting on a multiple of 64) and one grid arena per
// field array (each instance's nodes contiguous).  Work is split into
//   - particle tiles of <= 512 particles of one instance, walked by the shared
//     persistent particle pass (one launch per dimension class), and
//   - cell items of <= ITEM_CELLS nodes of one instance, walked by the grid
//     kernels below; per-instance sums (dot products, charge, energies) reduce
//     the partials of that instance's items in a fixed order, so every result
//     is deterministic.
// The field solve is the same Jacobi-preconditioned CG as the single instance
// (FP32 vectors, FP64 dots, null-space projection, breakdown guard), run for
// all instances in lockstep (an instance that has converged drops out of the
// launches), or the spectral solve of every instance in three passes of jobs.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "ap_pic.h"
#include "pic_internal.cuh"

using namespace apk;

namespace apk {

constexpr int BT = 256;  // threads per block of the batch grid kernels

// Per-instance grid description for the batch grid kernels.
struct BInst {
    int ndim;
    int n[2];
    FastDiv div0;
    int64_t node0;      // first node of the instance in the grid arenas
    int64_t cells;
    float idx2[2];      // 1 / dx_a^2
    double idx2d[2];
    float inv_diag;     // 1 / (2 sum 1/dx_a^2)
    float h[2];         // 1 / (2 dx_a)
    double scale;       // q w / dV / 2^S
    double bg;          // background density
    double mean_e;      // mean electron density (exact)
    long long mean_q;   // the accumulator's mean, np 2^S / cells: integer part
    float mean_r;       // and fraction
    float scale_f;      // scale in FP32
    int item0, nitems;  // this instance's cell items
    int tile0, ntiles;  // this instance's particle tiles (in its dimension class list)
    double dV;
};

struct CellItem {
    int inst;
    int count;
    int64_t start;      // first node (arena index)
};

struct BArena {
    unsigned long long *acc;  // charge (int64 fixed point); rho = scale acc + bg where read
    float *b, *phi, *r, *p, *q, *x;
    float2 *E;
};

__device__ __forceinline__ double bwarp_sum(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

__device__ double bblock_sum(double x)
{
    __shared__ double red[BT / 32];
    __shared__ double total;
    x = bwarp_sum(x);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int j = 0; j < BT / 32; ++j) t += red[j];
        total = t;
    }
    __syncthreads();
    const double r = total;
    __syncthreads();
    return r;
}

// An instance's done flag read once per block and broadcast, so that every thread
// of the block takes the same branch even while another block of the instance
// sets the flag in the same launch (the item loops below synchronise the block).
__device__ int block_flag(const int *p)
{
    __shared__ int s;
    __syncthreads();  // the previous broadcast has been read by every thread
    if (threadIdx.x == 0) s = *reinterpret_cast<const volatile int *>(p);
    __syncthreads();
    return s;
}

// Sum of instance `in`'s item partials (stride `stride` doubles per item, field
// `k`), in a fixed order; valid in every thread of the block.
__device__ double inst_sum(const double *__restrict__ part, int stride, int k, const BInst &in)
{
    double s = 0.0;
    for (int j = threadIdx.x; j < in.nitems; j += BT) s += part[(size_t)(in.item0 + j) * stride + k];
    return bblock_sum(s);
}

__device__ __forceinline__ void bcoords(int64_t local, const BInst &in, int *j)
{
    const uint32_t u = (uint32_t)local;
    if (in.ndim == 1) {
        j[0] = (int)u;
        j[1] = 0;
    } else {
        const uint32_t r = fdiv(u, in.div0);
        j[0] = (int)(u - r * (uint32_t)in.n[0]);
        j[1] = (int)r;
    }
}

// (-lap_h u) at arena node a = node0 + local.
__device__ __forceinline__ float bneg_lap(const float *__restrict__ u, const BInst &in, int64_t a,
                                          const int *j)
{
    const float c = u[a];
    float acc = 0.0f;
    int64_t stride = 1;
    for (int ax = 0; ax < in.ndim; ++ax) {
        const int na = in.n[ax];
        const int64_t up = (j[ax] + 1 == na) ? a - (int64_t)(na - 1) * stride : a + stride;
        const int64_t dn = (j[ax] == 0) ? a + (int64_t)(na - 1) * stride : a - stride;
        acc += (2.0f * c - u[up] - u[dn]) * in.idx2[ax];
        stride *= na;
    }
    return acc;
}

__device__ __forceinline__ double bneg_lap64(const float *__restrict__ u, const BInst &in,
                                             int64_t a, const int *j)
{
    const double c = u[a];
    double acc = 0.0;
    int64_t stride = 1;
    for (int ax = 0; ax < in.ndim; ++ax) {
        const int na = in.n[ax];
        const int64_t up = (j[ax] + 1 == na) ? a - (int64_t)(na - 1) * stride : a + stride;
        const int64_t dn = (j[ax] == 0) ? a + (int64_t)(na - 1) * stride : a - stride;
        acc += (2.0 * c - (double)u[up] - (double)u[dn]) * in.idx2d[ax];
        stride *= na;
    }
    return acc;
}

// Per-instance CG state (device).
struct BCG {
    double *part;     // [nitems][4]
    double *scal;     // [ninst][8]: 0 bnorm, 1-2 rz ping-pong, 3 relres
    int *done;        // [ninst]
    int *iters;       // [ninst]
};

#define ITEM_LOOP for (int it_ = blockIdx.x; it_ < nitems; it_ += gridDim.x)
// Over the items listed in act[0..nact) (every item when act is null): the CG
// iterations walk only the items of instances that have not converged.
#define ACT_LOOP                                                                               \
    for (int k_ = blockIdx.x, it_ = 0; k_ < nact && ((it_ = act ? act[k_] : k_), true);      \
         k_ += gridDim.x)

// b = scale (acc - mean(acc)) in FP32 per node, with no FP64 arithmetic (the exact
// mean split into an integer part and a fraction; see launch_rho_convert).
__global__ void __launch_bounds__(BT)
    k_b_convert(const CellItem *__restrict__ items, int nitems, const BInst *__restrict__ inst,
                BArena A)
{
    ITEM_LOOP
    {
        const CellItem ci = items[it_];
        const BInst in = inst[ci.inst];
        for (int k = threadIdx.x; k < ci.count; k += BT) {
            const int64_t a = ci.start + k;
            A.b[a] = in.scale_f * (i64_to_f32((long long)A.acc[a] - in.mean_q) - in.mean_r);
        }
    }
}

// CG on A x = rhs for every instance not yet done.  `x` and `rhs` select the
// solve (the potential, or the refinement's correction).
__global__ void __launch_bounds__(BT)
    k_b_cg_init(const CellItem *__restrict__ items, int nitems, const BInst *__restrict__ inst,
                BArena A, float *__restrict__ x, const float *__restrict__ rhs, BCG cg)
{
    ITEM_LOOP
    {
        const CellItem ci = items[it_];
        const BInst in = inst[ci.inst];
        double rr = 0.0, rs = 0.0, bb = 0.0;
        for (int k = threadIdx.x; k < ci.count; k += BT) {
            const int64_t a = ci.start + k;
            int j[2];
            bcoords(a - in.node0, in, j);
            const float bi = rhs[a];
            const float ri = bi - bneg_lap(x, in, a, j);
            A.r[a] = ri;
            A.p[a] = ri * in.inv_diag;
            rr += (double)ri * ri;
            rs += ri;
            bb += (double)bi * bi;
        }
        rr = bblock_sum(rr);
        rs = bblock_sum(rs);
        bb = bblock_sum(bb);
        if (threadIdx.x == 0) {
            cg.part[(size_t)it_ * 4 + 0] = rr;
            cg.part[(size_t)it_ * 4 + 1] = rs;
            cg.part[(size_t)it_ * 4 + 2] = bb;
        }
    }
}

__global__ void __launch_bounds__(BT)
    k_b_cg_init_fin(const BInst *__restrict__ inst, int ninst, BCG cg, double rtol)
{
    for (int i = blockIdx.x; i < ninst; i += gridDim.x) {
        const BInst in = inst[i];
        const double rr0 = inst_sum(cg.part, 4, 0, in);
        const double rs = inst_sum(cg.part, 4, 1, in);
        const double bb = inst_sum(cg.part, 4, 2, in);
        if (threadIdx.x == 0) {
            const double m = rs / (double)in.cells;
            const double rr = fmax(rr0 - (double)in.cells * m * m, 0.0);
            const double bn = sqrt(bb);
            cg.scal[i * 8 + 0] = bn;
            cg.scal[i * 8 + 1] = rr * (double)in.inv_diag;
            const double rel = bn > 0.0 ? sqrt(rr) / bn : 0.0;
            cg.scal[i * 8 + 3] = rel;
            cg.iters[i] = 0;
            cg.done[i] = (bn == 0.0 || rel <= rtol) ? 1 : 0;
        }
    }
}

__global__ void __launch_bounds__(BT)
    k_b_cg_matvec(const CellItem *__restrict__ items, const int *__restrict__ act, int nact, const BInst *__restrict__ inst,
                  BArena A, BCG cg)
{
    ACT_LOOP
    {
        const CellItem ci = items[it_];
        if (block_flag(cg.done + ci.inst)) continue;
        const BInst in = inst[ci.inst];
        double pq = 0.0;
        for (int k = threadIdx.x; k < ci.count; k += BT) {
            const int64_t a = ci.start + k;
            int j[2];
            bcoords(a - in.node0, in, j);
            const float qi = bneg_lap(A.p, in, a, j);
            A.q[a] = qi;
            pq += (double)A.p[a] * qi;
        }
        pq = bblock_sum(pq);
        if (threadIdx.x == 0) cg.part[(size_t)it_ * 4 + 3] = pq;
    }
}

__global__ void __launch_bounds__(BT)
    k_b_cg_update(const CellItem *__restrict__ items, const int *__restrict__ act, int nact, const BInst *__restrict__ inst,
                  BArena A, float *__restrict__ x, BCG cg, int it)
{
    ACT_LOOP
    {
        const CellItem ci = items[it_];
        if (block_flag(cg.done + ci.inst)) continue;
        const BInst in = inst[ci.inst];
        const double pq = inst_sum(cg.part, 4, 3, in);
        const double a64 = cg.scal[ci.inst * 8 + 1 + (it & 1)] / pq;
        if (!(pq > 0.0) || !isfinite(a64)) {  // breakdown: stop this instance
            if (threadIdx.x == 0) cg.done[ci.inst] = 2;
            continue;
        }
        const float alpha = (float)a64;
        double rr = 0.0, rs = 0.0;
        for (int k = threadIdx.x; k < ci.count; k += BT) {
            const int64_t a = ci.start + k;
            x[a] += alpha * A.p[a];
            const float ri = A.r[a] - alpha * A.q[a];
            A.r[a] = ri;
            rr += (double)ri * ri;
            rs += ri;
        }
        rr = bblock_sum(rr);
        rs = bblock_sum(rs);
        if (threadIdx.x == 0) {
            cg.part[(size_t)it_ * 4 + 0] = rr;
            cg.part[(size_t)it_ * 4 + 1] = rs;
        }
    }
}

__global__ void __launch_bounds__(BT)
    k_b_cg_dir(const CellItem *__restrict__ items, const int *__restrict__ act, int nact, const BInst *__restrict__ inst,
               BArena A, BCG cg, int it, int maxit, double rtol)
{
    ACT_LOOP
    {
        const CellItem ci = items[it_];
        if (block_flag(cg.done + ci.inst)) continue;
        const BInst in = inst[ci.inst];
        const double rr0 = inst_sum(cg.part, 4, 0, in);
        const double rs = inst_sum(cg.part, 4, 1, in);
        const double m = rs / (double)in.cells;
        const double rr = fmax(rr0 - (double)in.cells * m * m, 0.0);
        const double rz_new = rr * (double)in.inv_diag;
        const double rz = cg.scal[ci.inst * 8 + 1 + (it & 1)];
        const double rel = sqrt(rr) / cg.scal[ci.inst * 8 + 0];
        const bool stop = rel <= rtol || it + 1 >= maxit;
        if (it_ == in.item0 && threadIdx.x == 0) {
            cg.scal[ci.inst * 8 + 1 + ((it + 1) & 1)] = rz_new;
            cg.scal[ci.inst * 8 + 3] = rel;
            cg.iters[ci.inst] = it + 1;
        }
        if (stop) {
            // every block of this instance takes the same decision; the flag is read
            // by the next kernel only
            if (it_ == in.item0 && threadIdx.x == 0) cg.done[ci.inst] = 1;
            continue;
        }
        const float beta = (float)(rz_new / rz);
        const float mf = (float)m;
        for (int k = threadIdx.x; k < ci.count; k += BT) {
            const int64_t a = ci.start + k;
            const float ri = A.r[a] - mf;
            A.r[a] = ri;
            A.p[a] = ri * in.inv_diag + beta * A.p[a];
        }
    }
}

// Refinement right-hand side: r = (float)(rho - mean - A phi) in FP64.
__global__ void __launch_bounds__(BT)
    k_b_residual64(const CellItem *__restrict__ items, int nitems, const BInst *__restrict__ inst,
                   BArena A)
{
    ITEM_LOOP
    {
        const CellItem ci = items[it_];
        const BInst in = inst[ci.inst];
        const double mean_total = in.mean_e + in.bg;
        for (int k = threadIdx.x; k < ci.count; k += BT) {
            const int64_t a = ci.start + k;
            int j[2];
            bcoords(a - in.node0, in, j);
            const double rho = in.scale * (double)(long long)A.acc[a] + in.bg;
            A.b[a] = (float)((rho - mean_total) - bneg_lap64(A.phi, in, a, j));
        }
    }
}

__global__ void __launch_bounds__(BT)
    k_b_add_correction(const CellItem *__restrict__ items, int nitems, BArena A)
{
    ITEM_LOOP
    {
        const CellItem ci = items[it_];
        for (int k = threadIdx.x; k < ci.count; k += BT) A.phi[ci.start + k] += A.x[ci.start + k];
    }
}

__global__ void __launch_bounds__(BT)
    k_b_efield(const CellItem *__restrict__ items, int nitems, const BInst *__restrict__ inst,
               BArena A, double *__restrict__ fepart)
{
    ITEM_LOOP
    {
        const CellItem ci = items[it_];
        const BInst in = inst[ci.inst];
        double fe = 0.0;
        for (int k = threadIdx.x; k < ci.count; k += BT) {
            const int64_t a = ci.start + k;
            int j[2];
            bcoords(a - in.node0, in, j);
            float e[2] = {0.0f, 0.0f};
            int64_t stride = 1;
            for (int ax = 0; ax < in.ndim; ++ax) {
                const int na = in.n[ax];
                const int64_t up = (j[ax] + 1 == na) ? a - (int64_t)(na - 1) * stride : a + stride;
                const int64_t dn = (j[ax] == 0) ? a + (int64_t)(na - 1) * stride : a - stride;
                e[ax] = -(A.phi[up] - A.phi[dn]) * in.h[ax];
                fe += (double)e[ax] * e[ax];
                stride *= na;
            }
            // the particle pass reads ndim floats per node: 1D instances keep a packed
            // float field at the start of their (float2-sized) region
            if (in.ndim == 1)
                reinterpret_cast<float *>(A.E + in.node0)[a - in.node0] = e[0];
            else
                A.E[a] = make_float2(e[0], e[1]);
        }
        fe = bblock_sum(fe);
        if (threadIdx.x == 0) fepart[it_] = fe;
    }
}

// Per-instance diagnostics: [0] sum (|v-|^2 + |v+|^2)/2, [1..2] sum v, [3] sum |E|^2,
// [4] accumulator sum (exact: an int64 carried in a double only for sums < 2^53;
// the int64 value is also written to isum).
__global__ void __launch_bounds__(BT)
    k_b_diag(const BInst *__restrict__ inst, int ninst, const double *__restrict__ tdiag1,
             const double *__restrict__ tdiag2, const double *__restrict__ fepart,
             const long long *__restrict__ ipart_ll, double *__restrict__ out,
             long long *__restrict__ isum, int have_particles)
{
    for (int i = blockIdx.x; i < ninst; i += gridDim.x) {
        const BInst in = inst[i];
        const double *td = in.ndim == 1 ? tdiag1 : tdiag2;
        for (int k = 0; k < 3; ++k) {
            double s = 0.0;
            if (have_particles && td)
                for (int j = threadIdx.x; j < in.ntiles; j += BT) s += td[(size_t)(in.tile0 + j) * 4 + k];
            s = bblock_sum(s);
            if (threadIdx.x == 0 && have_particles) out[i * 8 + k] = s;
        }
        double fe = 0.0;
        for (int j = threadIdx.x; j < in.nitems; j += BT) fe += fepart[in.item0 + j];
        fe = bblock_sum(fe);
        if (threadIdx.x == 0) {
            out[i * 8 + 3] = fe;
            long long t = 0;
            for (int j = 0; j < in.nitems; ++j) t += ipart_ll[in.item0 + j];
            isum[i] = t;
        }
    }
}

// Exact int64 item sums of the accumulator (the FP64 partial of k_b_convert is
// only for the conversion; this one is integer).
__global__ void __launch_bounds__(BT)
    k_b_isum(const CellItem *__restrict__ items, int nitems, BArena A, long long *__restrict__ out)
{
    ITEM_LOOP
    {
        const CellItem ci = items[it_];
        long long s = 0;
        for (int k = threadIdx.x; k < ci.count; k += BT) s += (long long)A.acc[ci.start + k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        __shared__ long long red[BT / 32];
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            long long t = 0;
            for (int j = 0; j < BT / 32; ++j) t += red[j];
            out[it_] = t;
        }
        __syncthreads();
    }
}

// Sort keys of a batch: instance key base + the instance's brick-major key.
// Key tiles cover every slot of an instance's arena range, padding included;
// padding slots (local index >= np) take the instance's last key, so the global
// stable sort keeps every instance's particles, then its padding, in its range.
__global__ void __launch_bounds__(BT)
    k_b_keys(const BatchTile *__restrict__ tiles, int64_t ntiles, const int *__restrict__ kinfo,
             const int64_t *__restrict__ pbase, const int32_t *__restrict__ cell,
             uint32_t *__restrict__ keys)
{
    // kinfo per instance (8 ints): ndim, n0, b0, b1, nb0, key_base, padding key offset, np
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const BatchTile bt = tiles[t];
        const int *ki = kinfo + (size_t)bt.inst * 8;
        const int ndim = ki[0], n0 = ki[1], b0 = ki[2], b1 = ki[3], nb0 = ki[4];
        const uint32_t base = (uint32_t)ki[5];
        const uint32_t pad_key = base + (uint32_t)ki[6];
        const int64_t np_i = ki[7], first = pbase[bt.inst];
        const FastDiv dn0 = make_fastdiv((uint32_t)n0);
        const FastDiv db0 = make_fastdiv((uint32_t)b0), db1 = make_fastdiv((uint32_t)b1);
        for (int k = threadIdx.x; k < bt.count; k += BT) {
            const int64_t i = bt.start + k;
            if (i - first >= np_i) {
                keys[i] = pad_key;
                continue;
            }
            const uint32_t c = (uint32_t)cell[i];
            uint32_t c0 = c, c1 = 0;
            if (ndim == 2) {
                c1 = fdiv(c, dn0);
                c0 = c - c1 * (uint32_t)n0;
            }
            const uint32_t q0 = fdiv(c0, db0), q1 = fdiv(c1, db1);
            const uint32_t bid = q0 + (uint32_t)nb0 * q1;
            const uint32_t lid = (c0 - q0 * (uint32_t)b0) + (uint32_t)b0 * (c1 - q1 * (uint32_t)b1);
            keys[i] = base + bid * (uint32_t)(b0 * b1) + lid;
        }
    }
}

// ---- host launchers -------------------------------------------------------------------------

struct BatchGrid {
    CellItem *items;
    int nitems;
    BInst *inst;
    int ninst;
    BArena A;
    BCG cg;
    double *fepart;
    long long *ipart_ll;
    int nblocks;
    const int *act;  // items the CG iterations walk (null: all), nact of them
    int nact;
};

}  // namespace apk

// =============================================================================================
// host side
// =============================================================================================

namespace {

constexpr int B_TILE = BATCH_TILE;  // key tile of the sort (all slots of an instance)
constexpr int B_MIN_TILE = 256;     // smallest pass tile of the kernel variants
constexpr int64_t PAD = 64;      // instance ranges in the particle arena start on multiples of 64

int bitlen_u(uint64_t x)
{
    int b = 0;
    while (x) {
        ++b;
        x >>= 1;
    }
    return b;
}

}  // namespace

struct ap_pic_batch {
    int count = 0;
    std::vector<ap_pic_config> cfg;
    ap_pic_allocator alloc{};
    bool has_alloc = false;
    // All batch work runs on an own non-blocking stream (a graph cannot be captured
    // on the legacy default stream); it is fenced to the caller's stream with
    // events on entry and exit of every enqueuing call.
    cudaStream_t stream = nullptr;
    cudaStream_t user = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::string err;
    std::vector<std::pair<void *, size_t>> owned;
    ap_pic_batch_tuning tune{};

    // per instance (host)
    std::vector<int64_t> np, pbase, node0, cells;
    std::vector<int> fx_bits, key_base, nkeys;
    std::vector<GridParams> gp;
    std::vector<BInst> binst;
    int64_t slots = 0;        // particle arena length (with padding)
    int64_t total_nodes = 0;
    int key_bits = 0;
    bool loaded = false;
    int64_t step = 0;

    // particle arena + sort
    ParticlesF32 p{}, p_alt{};
    SortScratch sort{};
    std::vector<BatchTile> tiles1, tiles2, ktiles;  // 1D / 2D pass tiles, key tiles (all slots)
    int variant = 0;          // pass kernel variant (tune.pass_threads, tune.pass_per_thread)
    size_t tile_cap1 = 0, tile_cap2 = 0;  // device room for pass tiles (smallest tile size)
    int ptile = 0;            // particles per pass tile of the current tiles (0: none yet)
    BatchTile *d_tiles1 = nullptr, *d_tiles2 = nullptr, *d_ktiles = nullptr;
    int *d_kinfo = nullptr;
    int64_t *d_pbase = nullptr;
    void *d_tparams = nullptr;  // TileParams per instance
    double *d_tdiag1 = nullptr, *d_tdiag2 = nullptr;
    int perm_slot = -1;

    // grid
    std::vector<CellItem> items;
    BatchGrid G{};
    double *d_diag = nullptr;     // [count][8]
    long long *d_isum = nullptr;  // [count]
    int *d_err = nullptr;
    int *h_done = nullptr;   // pinned: per-instance CG done flags
    int *h_act = nullptr;    // pinned: the active item list, uploaded to d_act
    int *d_act = nullptr;
    int *h_err = nullptr;
    int pass_blocks = 0;
    int sms = 148;

    // per-step graphs (particle pass .. first CG block), one per particle-buffer
    // parity: a sort swaps the ping-pong buffers, whose addresses the graph holds
    cudaGraphExec_t graphs[2] = {nullptr, nullptr};
    int parity = 0;
    bool graph_diag = false;
    int graph_iters = 0;
    int64_t graph_launches = 0;  // kernels per replay (for the launch counter)

    int last_iters_max = 0;

    // spectral field solve (cfgs[0].solver == AP_PIC_SOLVER_FFT): three passes of
    // jobs (x forward of 2D grids and the whole 1D solves; y forward, scale and
    // inverse; x inverse), tables shared by instances of equal (n, dx)
    bool use_fft = false;
    FftGrid *d_fft_grids = nullptr;
    FftJob *d_fft_jobs[3] = {nullptr, nullptr, nullptr};
    int fft_njobs[3] = {0, 0, 0};
    size_t fft_smem[3] = {0, 0, 0};
    float2 *fft_Z = nullptr;
    const float2 *fft_tw = nullptr;
    int fft_log2M = 1;
};

namespace {

ap_pic_status bfail(ap_pic_batch *b, ap_pic_status st, const char *msg)
{
    if (b) b->err = msg;
    return st;
}

#define BCU(b, call)                                                                           \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            std::string m_ = std::string(#call) + ": " + cudaGetErrorString(e_);               \
            return bfail((b), AP_PIC_ERR_CUDA, m_.c_str());                                    \
        }                                                                                      \
    } while (0)

#define BTRY(expr)                                                                             \
    do {                                                                                       \
        ap_pic_status s_ = (expr);                                                             \
        if (s_ != AP_PIC_OK) return s_;                                                        \
    } while (0)

void *bdev_alloc(ap_pic_batch *b, size_t bytes)
{
    if (bytes == 0) bytes = 256;
    void *ptr = nullptr;
    if (b->has_alloc) ptr = b->alloc.alloc(bytes, b->alloc.ctx);
    else if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
        cudaGetLastError();
        ptr = nullptr;
    }
    if (ptr) b->owned.push_back({ptr, bytes});
    return ptr;
}

template <typename T>
ap_pic_status balloc(ap_pic_batch *b, T **out, size_t n)
{
    *out = static_cast<T *>(bdev_alloc(b, n * sizeof(T)));
    return *out ? AP_PIC_OK : bfail(b, AP_PIC_ERR_NOMEM, "device allocation failed");
}

void bfree_all(ap_pic_batch *b)
{
    for (auto &o : b->owned) {
        if (b->has_alloc) b->alloc.free(o.first, o.second, b->alloc.ctx);
        else cudaFree(o.first);
    }
    b->owned.clear();
}

// Pass tiles of at most `tile` particles, each within one instance, per dimension
// class; each instance's first tile and tile count go to its BInst.
void make_pass_tiles(ap_pic_batch *b, int tile)
{
    b->tiles1.clear();
    b->tiles2.clear();
    for (int i = 0; i < b->count; ++i) {
        std::vector<BatchTile> &tl = b->cfg[i].ndim == 1 ? b->tiles1 : b->tiles2;
        b->binst[i].tile0 = (int)tl.size();
        for (int64_t s = 0; s < b->np[i]; s += tile) {
            const int cnt = (int)(b->np[i] - s < tile ? b->np[i] - s : tile);
            tl.push_back(BatchTile{b->pbase[i] + s, cnt, i});
        }
        b->binst[i].ntiles = (int)tl.size() - b->binst[i].tile0;
    }
    b->ptile = tile;
}

// The pass tiles (and, once it exists, the device copy of the instance table) to
// the device; waits for the copies (the host lists may change again right after).
ap_pic_status upload_pass_tiles(ap_pic_batch *b)
{
    if (b->tiles1.size() > b->tile_cap1 || b->tiles2.size() > b->tile_cap2)
        return bfail(b, AP_PIC_ERR_STATE, "pass tiles exceed their device room");
    if (!b->tiles1.empty())
        BCU(b, cudaMemcpyAsync(b->d_tiles1, b->tiles1.data(), b->tiles1.size() * sizeof(BatchTile),
                               cudaMemcpyHostToDevice, b->stream));
    if (!b->tiles2.empty())
        BCU(b, cudaMemcpyAsync(b->d_tiles2, b->tiles2.data(), b->tiles2.size() * sizeof(BatchTile),
                               cudaMemcpyHostToDevice, b->stream));
    if (b->G.inst)
        BCU(b, cudaMemcpyAsync(b->G.inst, b->binst.data(), b->binst.size() * sizeof(BInst),
                               cudaMemcpyHostToDevice, b->stream));
    BCU(b, cudaStreamSynchronize(b->stream));
    return AP_PIC_OK;
}

void drop_graph(ap_pic_batch *b)
{
    for (auto &gx : b->graphs) {
        if (gx) cudaGraphExecDestroy(gx);
        gx = nullptr;
    }
}

GridParams make_gp(const ap_pic_config &c, int fx_bits, double step_h)
{
    GridParams g{};
    g.ndim = c.ndim;
    for (int a = 0; a < 3; ++a) {
        g.n[a] = a < c.ndim ? c.n[a] : 1;
        g.dtdx[a] = a < c.ndim ? (float)(c.dt / c.dx[a]) : 0.0f;
        g.E0[a] = (float)c.E0[a];
    }
    const double qm = c.q / c.m;
    g.qmh2 = (float)(qm * step_h * 0.5);
    g.magnetised = 0;
    g.fx_bits = fx_bits;
    g.div0 = make_fastdiv((uint32_t)g.n[0]);
    g.div1 = make_fastdiv((uint32_t)g.n[1]);
    return g;
}

// Per-instance tile parameters for a push by `factor` times each instance's dt.
ap_pic_status upload_tile_params(ap_pic_batch *b, double factor)
{
    const size_t tb = batch_tile_params_bytes();
    std::vector<unsigned char> host(tb * b->count);
    for (int i = 0; i < b->count; ++i) {
        const GridParams g = make_gp(b->cfg[i], b->fx_bits[i], factor * b->cfg[i].dt);
        make_tile_params(host.data() + tb * i, g,
                         reinterpret_cast<const float *>(b->G.A.E + b->node0[i]),
                         b->G.A.acc + b->node0[i]);
    }
    BCU(b, cudaMemcpyAsync(b->d_tparams, host.data(), host.size(), cudaMemcpyHostToDevice,
                           b->stream));
    return AP_PIC_OK;
}

// Tables and job lists of the spectral solve (grids already placed in the arenas).
ap_pic_status setup_fft(ap_pic_batch *b)
{
    static std::atomic<unsigned long long> configured{0};
    BCU(b, once_per_device(configured, [] { return fft_configure(); }));
    const int n = b->count;
    using Key = std::pair<int, double>;
    std::map<Key, size_t> at;  // float offset of the tables of an (n, dx) axis
    size_t total = 0;
    int log2M = 1;
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < b->cfg[i].ndim; ++a) {
            const Key key(b->cfg[i].n[a], b->cfg[i].dx[a]);
            if (at.count(key)) continue;
            at[key] = total;
            total += fft_axis_table_floats(key.first);
            const int l = fft_log2m(key.first);
            log2M = l > log2M ? l : log2M;
        }
    std::vector<float> host(total + fft_twiddle_floats(log2M), 0.0f);
    float *dev = nullptr;
    BTRY(balloc(b, &dev, host.size()));
    std::map<Key, FftAxis> axes;
    for (const auto &kv : at) {
        FftAxis ax{};
        fft_axis_tables(kv.first.first, kv.first.second, host.data() + kv.second,
                        dev + kv.second, &ax);
        axes[kv.first] = ax;
    }
    fft_twiddles(log2M, host.data() + total);
    b->fft_tw = reinterpret_cast<const float2 *>(dev + total);
    b->fft_log2M = log2M;
    // one grid per instance; jobs of W lines (W * m <= 4096 elements of shared memory)
    std::vector<FftGrid> grids((size_t)n);
    std::vector<FftJob> jobs[3];
    for (int k = 0; k < 3; ++k) b->fft_smem[k] = 0;
    for (int i = 0; i < n; ++i) {
        const ap_pic_config &c = b->cfg[i];
        FftGrid &g = grids[(size_t)i];
        g.node0 = b->node0[i];
        g.ndim = c.ndim;
        int64_t inner = 1;
        for (int a = 0; a < c.ndim; ++a) {
            g.ax[a] = axes[Key(c.n[a], c.dx[a])];
            g.ax[a].inner = inner;
            inner *= c.n[a];
        }
        g.div_n0 = make_fastdiv((uint32_t)c.n[0]);
        g.inv_cells = (float)(1.0 / (double)b->cells[i]);
        auto add = [&](int pass, int axis) {
            const int64_t lines = b->cells[i] / c.n[axis];
            const int log2m = g.ax[axis].log2m;
            // (Bluestein jobs of up to 4096 points; power-of-two jobs of up to 2048, whose
            // two Stockham buffers then take about as much shared memory)
            const bool blue = g.ax[axis].bluestein != 0;
            const int64_t cap = blue ? 4096 : 2048;
            int W = 32;
            while (W > 1 && (((int64_t)W << log2m) > cap || W / 2 >= lines)) W >>= 1;
            for (int64_t l0 = 0; l0 < lines; l0 += W)
                jobs[pass].push_back(
                    FftJob{i, axis, l0, (int)(lines - l0 < W ? lines - l0 : W), W});
            const size_t sm = fft_smem_bytes(W, log2m, blue);
            if (sm > b->fft_smem[pass]) b->fft_smem[pass] = sm;
        };
        add(0, 0);
        if (c.ndim == 2) {
            add(1, 1);
            add(2, 0);
        }
    }
    BTRY(balloc(b, &b->d_fft_grids, grids.size()));
    BCU(b, cudaMemcpyAsync(b->d_fft_grids, grids.data(), grids.size() * sizeof(FftGrid),
                           cudaMemcpyHostToDevice, b->stream));
    for (int k = 0; k < 3; ++k) {
        b->fft_njobs[k] = (int)jobs[k].size();
        BTRY(balloc(b, &b->d_fft_jobs[k], jobs[k].size() + 1));
        if (!jobs[k].empty())
            BCU(b, cudaMemcpyAsync(b->d_fft_jobs[k], jobs[k].data(),
                                   jobs[k].size() * sizeof(FftJob), cudaMemcpyHostToDevice,
                                   b->stream));
    }
    BCU(b, cudaMemcpyAsync(dev, host.data(), host.size() * sizeof(float), cudaMemcpyHostToDevice,
                           b->stream));
    BTRY(balloc(b, &b->fft_Z, (size_t)(b->total_nodes > 0 ? b->total_nodes : 1)));
    BCU(b, cudaStreamSynchronize(b->stream));  // the host tables go out of scope
    return AP_PIC_OK;
}

}  // namespace

extern "C" void ap_pic_batch_default_tuning(ap_pic_batch_tuning *t)
{
    if (!t) return;
    t->pass_ctas_per_sm = 4;
    t->item_cells = 2048;
    t->sort_every = 20;
    t->cg_iters_per_graph = 16;
    t->use_graph = 1;
    t->pass_threads = 256;
    t->pass_per_thread = 2;
}

extern "C" ap_pic_status ap_pic_batch_create(int count, const ap_pic_config *cfgs,
                                             const ap_pic_allocator *alloc, void *cuda_stream,
                                             ap_pic_batch **out)
{
    if (!out || !cfgs || count < 1) return AP_PIC_ERR_ARG;
    ap_pic_batch *b = new ap_pic_batch();
    *out = b;
    b->count = count;
    b->cfg.assign(cfgs, cfgs + count);
    if (alloc && alloc->alloc && alloc->free) {
        b->alloc = *alloc;
        b->has_alloc = true;
    }
    b->user = static_cast<cudaStream_t>(cuda_stream);
    BCU(b, cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
    BCU(b, cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming));
    BCU(b, cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming));
    ap_pic_batch_default_tuning(&b->tune);
    b->tune.sort_every = cfgs[0].sort_every;
    for (int i = 0; i < count; ++i) {
        ap_pic_config &c = b->cfg[i];
        if (c.ndim < 1 || c.ndim > 2)
            return bfail(b, AP_PIC_ERR_UNSUPPORTED, "batch instances must be 1D or 2D");
        if (c.nv != 2) return bfail(b, AP_PIC_ERR_UNSUPPORTED, "batch instances need nv = 2");
        if (c.precision != AP_PIC_FP32_CELLOFF || c.bc != AP_PIC_BC_PERIODIC)
            return bfail(b, AP_PIC_ERR_UNSUPPORTED, "batch: FP32 cell+offset, periodic only");
        if (c.B0[0] != 0.0 || c.B0[1] != 0.0 || c.B0[2] != 0.0)
            return bfail(b, AP_PIC_ERR_UNSUPPORTED, "batch instances: B0 must be 0");
        for (int a = 0; a < c.ndim; ++a)
            if (c.n[a] < 2 || !(c.dx[a] > 0.0)) return bfail(b, AP_PIC_ERR_ARG, "bad grid");
        for (int a = c.ndim; a < 3; ++a) {
            c.n[a] = 1;
            c.dx[a] = 1.0;
        }
        if (!(c.dt > 0.0) || !(c.m > 0.0) || !(c.weight > 0.0))
            return bfail(b, AP_PIC_ERR_ARG, "bad dt, m or weight");
        if (c.fx_bits == 0) c.fx_bits = 22;
        if (c.fx_bits < 8 || c.fx_bits > 22) return bfail(b, AP_PIC_ERR_ARG, "fx_bits in [8, 22]");
        if (c.pusher != AP_PIC_PUSHER_BORIS)
            return bfail(b, AP_PIC_ERR_UNSUPPORTED, "batch instances push with Boris only");
        if (b->cfg[0].solver == AP_PIC_SOLVER_FFT)
            for (int a = 0; a < c.ndim; ++a)
                if (!fft_length_ok(c.n[a]))
                    return bfail(b, AP_PIC_ERR_UNSUPPORTED, "FFT solver needs n <= 4096");
        for (int a = 0; a < c.ndim; ++a) {
            if (c.brick[a] == 0) c.brick[a] = c.ndim == 1 ? 64 : 8;
            if (c.brick[a] > c.n[a]) c.brick[a] = c.n[a];
        }
        for (int a = c.ndim; a < 3; ++a) c.brick[a] = 1;
    }
    if (b->cfg[0].solver != AP_PIC_SOLVER_CG && b->cfg[0].solver != AP_PIC_SOLVER_FFT)
        return bfail(b, AP_PIC_ERR_ARG, "unknown solver");
    b->use_fft = b->cfg[0].solver == AP_PIC_SOLVER_FFT;
    if (b->cfg[0].cg_rtol == 0.0) b->cfg[0].cg_rtol = 1e-6;
    if (b->cfg[0].cg_maxit == 0) b->cfg[0].cg_maxit = 20000;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    if (b->sms <= 0) b->sms = 148;
    BCU(b, cudaMallocHost(&b->h_done, sizeof(int) * (size_t)count));
    BCU(b, cudaMallocHost(&b->h_err, 64));
    return AP_PIC_OK;
}

extern "C" ap_pic_status ap_pic_batch_destroy(ap_pic_batch *b)
{
    if (!b) return AP_PIC_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graph(b);
    bfree_all(b);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->stream) cudaStreamDestroy(b->stream);
    if (b->h_done) cudaFreeHost(b->h_done);
    if (b->h_act) cudaFreeHost(b->h_act);
    if (b->h_err) cudaFreeHost(b->h_err);
    delete b;
    return AP_PIC_OK;
}

extern "C" const char *ap_pic_batch_last_error(const ap_pic_batch *b)
{
    return b ? b->err.c_str() : "";
}

extern "C" ap_pic_status ap_pic_batch_set_tuning(ap_pic_batch *b, const ap_pic_batch_tuning *t)
{
    if (!b || !t) return AP_PIC_ERR_ARG;
    if (t->pass_ctas_per_sm < 1 || t->pass_ctas_per_sm > 16 || t->item_cells < 256 ||
        t->item_cells > 65536 || t->item_cells % 256 || t->sort_every < 0 ||
        t->cg_iters_per_graph < 1 || t->cg_iters_per_graph > 256)
        return bfail(b, AP_PIC_ERR_ARG, "tuning out of range");
    const int variant = batch_variant(t->pass_threads, t->pass_per_thread);
    if (variant < 0)
        return bfail(b, AP_PIC_ERR_ARG,
                     "no particle-pass variant of that (pass_threads, pass_per_thread)");
    const bool relayout = b->loaded && t->item_cells != b->tune.item_cells;
    if (relayout) return bfail(b, AP_PIC_ERR_STATE, "item_cells must be set before loading");
    b->tune = *t;
    b->variant = variant;
    b->pass_blocks = b->sms * b->tune.pass_ctas_per_sm;
    drop_graph(b);
    const int tile = t->pass_threads * t->pass_per_thread;
    if (b->loaded && tile != b->ptile) {
        make_pass_tiles(b, tile);
        BTRY(upload_pass_tiles(b));
    }
    return AP_PIC_OK;
}

extern "C" ap_pic_status ap_pic_batch_get_tuning(const ap_pic_batch *b, ap_pic_batch_tuning *t)
{
    if (!b || !t) return AP_PIC_ERR_ARG;
    *t = b->tune;
    return AP_PIC_OK;
}

namespace {

// Orders the batch's stream after the caller's stream.
ap_pic_status enter(ap_pic_batch *b)
{
    BCU(b, cudaEventRecord(b->ev_in, b->user));
    BCU(b, cudaStreamWaitEvent(b->stream, b->ev_in, 0));
    return AP_PIC_OK;
}

// Orders the caller's stream after the batch's work.
ap_pic_status leave(ap_pic_batch *b)
{
    BCU(b, cudaEventRecord(b->ev_out, b->stream));
    BCU(b, cudaStreamWaitEvent(b->user, b->ev_out, 0));
    return AP_PIC_OK;
}

// Runs `body` between the two fences; the exit fence is recorded on failure too,
// so the caller's stream stays ordered after whatever the body enqueued.  The
// body's error wins over the fence's.
template <class F>
ap_pic_status fenced(ap_pic_batch *b, F &&body)
{
    BTRY(enter(b));
    const ap_pic_status s = body();
    const ap_pic_status l = leave(b);
    return s != AP_PIC_OK ? s : l;
}

ap_pic_status batch_sync_check(ap_pic_batch *b)
{
    BCU(b, cudaMemcpyAsync(b->h_err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    BCU(b, cudaStreamSynchronize(b->stream));
    if (*b->h_err & EF_NONFINITE)
        return bfail(b, AP_PIC_ERR_BOUNDS, "a particle was not finite or outside its box");
    if (*b->h_err & EF_TIMEOUT) return bfail(b, AP_PIC_ERR_CUDA, "a device wait hit its cap");
    if (*b->h_err & EF_CG) return bfail(b, AP_PIC_ERR_NOT_CONVERGED, "a field solve hit cg_maxit");
    return AP_PIC_OK;
}

// Enqueues a particle pass over both dimension classes.
ap_pic_status batch_pass(ap_pic_batch *b, bool push, bool mv, bool deposit, bool diag)
{
    if (!b->tiles1.empty())
        BCU(b, launch_batch_pass(1, b->variant, b->d_tiles1, (int64_t)b->tiles1.size(),
                                 b->d_tparams, b->p,
                                 push, mv, deposit, diag ? b->d_tdiag1 : nullptr, b->pass_blocks,
                                 b->d_err, b->stream));
    if (!b->tiles2.empty())
        BCU(b, launch_batch_pass(2, b->variant, b->d_tiles2, (int64_t)b->tiles2.size(),
                                 b->d_tparams, b->p,
                                 push, mv, deposit, diag ? b->d_tdiag2 : nullptr, b->pass_blocks,
                                 b->d_err, b->stream));
    return AP_PIC_OK;
}

int grid_blocks(const ap_pic_batch *b)
{
    const int cap = b->sms * 4;
    return (int)b->items.size() < cap ? (int)b->items.size() : cap;
}

ap_pic_status batch_convert(ap_pic_batch *b)
{
    BatchGrid &G = b->G;
    k_b_convert<<<grid_blocks(b), BT, 0, b->stream>>>(G.items, G.nitems, G.inst, G.A);
    note_launch();
    BCU(b, cudaGetLastError());
    return AP_PIC_OK;
}

// CG iterations [first, first + n) for the solve A x = rhs, over the active items.
void cg_iters(ap_pic_batch *b, float *x, int first, int n, int maxit, double rtol)
{
    BatchGrid &G = b->G;
    const int cap = b->sms * 4;
    const int nb = G.nact < cap ? G.nact : cap;
    if (nb == 0) return;
    for (int it = first; it < first + n && it < maxit; ++it) {
        k_b_cg_matvec<<<nb, BT, 0, b->stream>>>(G.items, G.act, G.nact, G.inst, G.A, G.cg);
        k_b_cg_update<<<nb, BT, 0, b->stream>>>(G.items, G.act, G.nact, G.inst, G.A, x, G.cg, it);
        k_b_cg_dir<<<nb, BT, 0, b->stream>>>(G.items, G.act, G.nact, G.inst, G.A, G.cg, it, maxit,
                                             rtol);
        note_launch(3);
    }
}

// Starts a solve on every item (the CG kernels then walk all items until the
// first host check narrows the list).
void cg_start(ap_pic_batch *b, float *x, const float *rhs, double rtol)
{
    BatchGrid &G = b->G;
    G.act = nullptr;
    G.nact = G.nitems;
    k_b_cg_init<<<grid_blocks(b), BT, 0, b->stream>>>(G.items, G.nitems, G.inst, G.A, x, rhs, G.cg);
    const int nbi = b->count < b->sms * 4 ? b->count : b->sms * 4;
    k_b_cg_init_fin<<<nbi, BT, 0, b->stream>>>(G.inst, G.ninst, G.cg, rtol);
    note_launch(2);
}

// Runs CG blocks until every instance is done.  Before each block the host reads
// the done flags and, when instances have finished, narrows the item list to
// those of the instances still iterating, so that the launches (sized to the
// list) cost nothing for converged instances.
ap_pic_status cg_finish(ap_pic_batch *b, float *x, int first, int maxit, double rtol)
{
    BatchGrid &G = b->G;
    int it = first;
    // the solve's first iterations (possibly replayed from a graph) walked every item
    G.act = nullptr;
    G.nact = G.nitems;
    int listed = b->count;  // instances in the current list
    while (true) {
        BCU(b, cudaMemcpyAsync(b->h_done, G.cg.done, sizeof(int) * (size_t)b->count,
                               cudaMemcpyDeviceToHost, b->stream));
        BCU(b, cudaStreamSynchronize(b->stream));
        int active = 0;
        for (int i = 0; i < b->count; ++i) active += b->h_done[i] ? 0 : 1;
        if (active == 0 || it >= maxit) break;
        if (active < listed) {
            int m = 0;
            for (int i = 0; i < b->count; ++i) {
                if (b->h_done[i]) continue;
                const BInst &in = b->binst[i];
                for (int j = 0; j < in.nitems; ++j) b->h_act[m++] = in.item0 + j;
            }
            BCU(b, cudaMemcpyAsync(b->d_act, b->h_act, sizeof(int) * (size_t)m,
                                   cudaMemcpyHostToDevice, b->stream));
            G.act = b->d_act;
            G.nact = m;
            listed = active;
        }
        const int n = b->tune.cg_iters_per_graph;
        cg_iters(b, x, it, n, maxit, rtol);
        it += n;
    }
    b->last_iters_max = it;
    return AP_PIC_OK;
}

ap_pic_status field_fft(ap_pic_batch *b);

// The part of a step that does not depend on host decisions: particle pass,
// charge conversion, start of the CG and its first block of iterations (with the
// spectral solve: the whole field update).
ap_pic_status step_front(ap_pic_batch *b, bool diag)
{
    BatchGrid &G = b->G;
    BCU(b, cudaMemsetAsync(G.A.acc, 0, (size_t)b->total_nodes * 8, b->stream));
    BTRY(batch_pass(b, true, true, true, diag));
    BTRY(batch_convert(b));
    if (b->use_fft) return field_fft(b);
    cg_start(b, G.A.phi, G.A.b, b->cfg[0].cg_rtol);
    cg_iters(b, G.A.phi, 0, b->tune.cg_iters_per_graph, b->cfg[0].cg_maxit, b->cfg[0].cg_rtol);
    return AP_PIC_OK;
}

// E from the potential, and the per-instance diagnostics.
ap_pic_status field_finish(ap_pic_batch *b)
{
    BatchGrid &G = b->G;
    const int nb = grid_blocks(b);
    k_b_efield<<<nb, BT, 0, b->stream>>>(G.items, G.nitems, G.inst, G.A, G.fepart);
    k_b_isum<<<nb, BT, 0, b->stream>>>(G.items, G.nitems, G.A, G.ipart_ll);
    const int nbi = b->count < b->sms * 4 ? b->count : b->sms * 4;
    k_b_diag<<<nbi, BT, 0, b->stream>>>(G.inst, G.ninst, b->d_tdiag1, b->d_tdiag2, G.fepart,
                                        G.ipart_ll, b->d_diag, b->d_isum, 1);
    note_launch(3);
    BCU(b, cudaGetLastError());
    return AP_PIC_OK;
}

// Finish the CG field: remaining CG blocks, one refinement pass, E, diagnostics.
ap_pic_status step_back(ap_pic_batch *b, int first_iter)
{
    BatchGrid &G = b->G;
    const double rtol = b->cfg[0].cg_rtol;
    const int maxit = b->cfg[0].cg_maxit;
    BTRY(cg_finish(b, G.A.phi, first_iter, maxit, rtol));
    // refinement: r = rho - mean - A phi (FP64) -> A x = r (FP32, to 1e-2) -> phi += x
    const int nb = grid_blocks(b);
    k_b_residual64<<<nb, BT, 0, b->stream>>>(G.items, G.nitems, G.inst, G.A);
    note_launch();
    BCU(b, cudaMemsetAsync(G.A.x, 0, (size_t)b->total_nodes * 4, b->stream));
    cg_start(b, G.A.x, G.A.b, 1e-2);
    cg_iters(b, G.A.x, 0, 8, maxit, 1e-2);
    BTRY(cg_finish(b, G.A.x, 8, maxit, 1e-2));
    k_b_add_correction<<<nb, BT, 0, b->stream>>>(G.items, G.nitems, G.A);
    note_launch();
    return field_finish(b);
}

// The spectral solve of every instance: x forward of the 2D grids (and the whole
// solve of the 1D ones), y forward / scale / inverse, x inverse.
ap_pic_status fft_solve(ap_pic_batch *b, const float *rhs, float *out)
{
    const int blocks = b->sms * 4;
    BCU(b, launch_fft_jobs(b->d_fft_jobs[0], b->fft_njobs[0], b->d_fft_grids, b->fft_Z, rhs,
                           nullptr, out, b->fft_tw, b->fft_log2M, FFT_FWD, b->fft_smem[0], blocks,
                           b->stream));
    BCU(b, launch_fft_jobs(b->d_fft_jobs[1], b->fft_njobs[1], b->d_fft_grids, b->fft_Z, nullptr,
                           nullptr, nullptr, b->fft_tw, b->fft_log2M, FFT_FWD_SCALE_INV,
                           b->fft_smem[1], blocks, b->stream));
    BCU(b, launch_fft_jobs(b->d_fft_jobs[2], b->fft_njobs[2], b->d_fft_grids, b->fft_Z, nullptr,
                           out, nullptr, b->fft_tw, b->fft_log2M, FFT_INV, b->fft_smem[2], blocks,
                           b->stream));
    return AP_PIC_OK;
}

// The spectral field of every instance: solve, the FP64-residual refinement
// (residual, solve, add), E and diagnostics.  No host decision, so it can be captured.
ap_pic_status field_fft(ap_pic_batch *b)
{
    BatchGrid &G = b->G;
    const int nb = grid_blocks(b);
    BTRY(fft_solve(b, G.A.b, G.A.phi));
    k_b_residual64<<<nb, BT, 0, b->stream>>>(G.items, G.nitems, G.inst, G.A);
    note_launch();
    BTRY(fft_solve(b, G.A.b, G.A.x));
    k_b_add_correction<<<nb, BT, 0, b->stream>>>(G.items, G.nitems, G.A);
    note_launch();
    return field_finish(b);
}

ap_pic_status batch_sort(ap_pic_batch *b)
{
    if (b->slots == 0) return AP_PIC_OK;
    k_b_keys<<<b->sms * 4, BT, 0, b->stream>>>(b->d_ktiles, (int64_t)b->ktiles.size(), b->d_kinfo,
                                               b->d_pbase, b->p.cell, b->sort.keys[0]);
    note_launch();
    BCU(b, cudaGetLastError());
    int slot = 0;
    BCU(b, launch_sort_keys(b->key_bits, b->slots, b->sort, &slot, b->stream));
    ParticlesF32 src = b->p;
    src.np = b->slots;
    ParticlesF32 dst = b->p_alt;
    dst.np = b->slots;
    BCU(b, launch_apply_perm(b->sort.idx[slot], src, dst, 2, b->stream));
    std::swap(b->p, b->p_alt);
    b->parity ^= 1;
    b->perm_slot = slot;
    return AP_PIC_OK;
}

// The upload and set-up of ap_pic_batch_load, inside its fences.
ap_pic_status load_body(ap_pic_batch *b, const int64_t *np, const double *const *x,
                        const double *const *v, unsigned flags)
{
    const int n = b->count;
    b->np.assign(np, np + n);
    b->pbase.resize(n);
    b->node0.resize(n);
    b->cells.resize(n);
    b->fx_bits.resize(n);
    b->key_base.resize(n);
    b->nkeys.resize(n);
    b->binst.resize(n);
    int64_t slots = 0, nodes = 0, keys = 0;
    for (int i = 0; i < n; ++i) {
        const ap_pic_config &c = b->cfg[i];
        if (np[i] < 0 || np[i] >= (int64_t(1) << 31)) return bfail(b, AP_PIC_ERR_ARG, "np");
        b->pbase[i] = slots;
        slots += (np[i] + PAD - 1) / PAD * PAD;
        b->node0[i] = nodes;
        b->cells[i] = (int64_t)c.n[0] * c.n[1];
        nodes += b->cells[i];
        const int cap = 62 - bitlen_u((uint64_t)(np[i] > 0 ? np[i] : 1));
        b->fx_bits[i] = c.fx_bits < cap ? c.fx_bits : cap;
        int64_t nk = 1;
        for (int a = 0; a < c.ndim; ++a)
            nk *= (int64_t)((c.n[a] + c.brick[a] - 1) / c.brick[a]) * c.brick[a];
        b->nkeys[i] = (int)(nk + 1);  // + one key for the instance's padding slots
        b->key_base[i] = (int)keys;
        keys += nk + 1;
        if (keys >= (int64_t(1) << 31)) return bfail(b, AP_PIC_ERR_ARG, "batch key range > 2^31");
    }
    b->slots = slots;
    b->total_nodes = nodes;
    b->key_bits = bitlen_u((uint64_t)(keys - 1));
    // particle arena
    const int64_t st = soa_stride(slots);
    ParticlesF32 *ps[2] = {&b->p, &b->p_alt};
    for (ParticlesF32 *q : ps) {
        BTRY(balloc(b, &q->cell, (size_t)st));
        BTRY(balloc(b, &q->off, (size_t)st * 2));
        BTRY(balloc(b, &q->v, (size_t)st * 2));
        BCU(b, cudaMemsetAsync(q->cell, 0, (size_t)st * 4, b->stream));
        BCU(b, cudaMemsetAsync(q->off, 0, (size_t)st * 8, b->stream));
        BCU(b, cudaMemsetAsync(q->v, 0, (size_t)st * 8, b->stream));
        q->np = slots;
        q->stride = st;
        q->nv = 2;
    }
    for (int k = 0; k < 2; ++k) {
        BTRY(balloc(b, &b->sort.keys[k], (size_t)(slots > 0 ? slots : 1)));
        BTRY(balloc(b, &b->sort.idx[k], (size_t)(slots > 0 ? slots : 1)));
    }
    const size_t hl = sort_hist_len(slots > 0 ? slots : 1);
    BTRY(balloc(b, &b->sort.hist, hl));
    b->sort.scan_tmp_len = sort_scan_tmp_len(hl);
    BTRY(balloc(b, &b->sort.scan_tmp, b->sort.scan_tmp_len));
    b->sort.capacity = slots;
    // tiles
    b->tiles1.clear();
    b->tiles2.clear();
    b->ktiles.clear();
    std::vector<int> kinfo(8 * n, 0);
    // pass tiles: capacity for the smallest tile of any variant, then the current one
    make_pass_tiles(b, B_MIN_TILE);
    const size_t cap1 = b->tiles1.size(), cap2 = b->tiles2.size();
    make_pass_tiles(b, b->tune.pass_threads * b->tune.pass_per_thread);
    for (int i = 0; i < n; ++i) {
        const ap_pic_config &c = b->cfg[i];
        const int64_t span = (np[i] + PAD - 1) / PAD * PAD;
        for (int64_t s = 0; s < span; s += B_TILE) {
            const int cnt = (int)(span - s < B_TILE ? span - s : B_TILE);
            b->ktiles.push_back(BatchTile{b->pbase[i] + s, cnt, i});
        }
        kinfo[8 * i + 0] = c.ndim;
        kinfo[8 * i + 1] = c.n[0];
        kinfo[8 * i + 2] = c.brick[0];
        kinfo[8 * i + 3] = c.ndim == 2 ? c.brick[1] : 1;
        kinfo[8 * i + 4] = (c.n[0] + c.brick[0] - 1) / c.brick[0];
        kinfo[8 * i + 5] = b->key_base[i];
        kinfo[8 * i + 6] = b->nkeys[i] - 1;  // the padding slots' key offset
        kinfo[8 * i + 7] = (int)np[i];       // local indices from here on are padding
    }
    auto upload = [&](auto &vec, auto **dptr) -> ap_pic_status {
        using T = typename std::remove_reference<decltype(vec)>::type::value_type;
        BTRY(balloc(b, dptr, vec.size() > 0 ? vec.size() : 1));
        if (!vec.empty())
            BCU(b, cudaMemcpyAsync(*dptr, vec.data(), vec.size() * sizeof(T),
                                   cudaMemcpyHostToDevice, b->stream));
        return AP_PIC_OK;
    };
    BTRY(balloc(b, &b->d_tiles1, cap1 > 0 ? cap1 : 1));
    BTRY(balloc(b, &b->d_tiles2, cap2 > 0 ? cap2 : 1));
    b->tile_cap1 = cap1;
    b->tile_cap2 = cap2;
    BTRY(upload_pass_tiles(b));
    BTRY(upload(b->ktiles, &b->d_ktiles));
    BTRY(upload(kinfo, &b->d_kinfo));
    BTRY(upload(b->pbase, &b->d_pbase));
    BTRY(balloc(b, &b->d_tdiag1, cap1 * 4 + 4));
    BTRY(balloc(b, &b->d_tdiag2, cap2 * 4 + 4));
    BCU(b, cudaMemsetAsync(b->d_tdiag1, 0, (cap1 * 4 + 4) * 8, b->stream));
    BCU(b, cudaMemsetAsync(b->d_tdiag2, 0, (cap2 * 4 + 4) * 8, b->stream));
    // cell items
    b->items.clear();
    const int ic = b->tune.item_cells;
    for (int i = 0; i < n; ++i) {
        b->binst[i].item0 = (int)b->items.size();
        for (int64_t s = 0; s < b->cells[i]; s += ic) {
            const int cnt = (int)(b->cells[i] - s < ic ? b->cells[i] - s : ic);
            b->items.push_back(CellItem{i, cnt, b->node0[i] + s});
        }
        b->binst[i].nitems = (int)b->items.size() - b->binst[i].item0;
    }
    // per-instance grid descriptions
    for (int i = 0; i < n; ++i) {
        const ap_pic_config &c = b->cfg[i];
        BInst &in = b->binst[i];
        in.ndim = c.ndim;
        in.n[0] = c.n[0];
        in.n[1] = c.ndim == 2 ? c.n[1] : 1;
        in.div0 = make_fastdiv((uint32_t)in.n[0]);
        in.node0 = b->node0[i];
        in.cells = b->cells[i];
        double d = 0.0, dV = 1.0;
        for (int a = 0; a < 2; ++a) {
            const bool on = a < c.ndim;
            in.idx2[a] = on ? (float)(1.0 / (c.dx[a] * c.dx[a])) : 0.0f;
            in.idx2d[a] = on ? 1.0 / (c.dx[a] * c.dx[a]) : 0.0;
            in.h[a] = on ? (float)(0.5 / c.dx[a]) : 0.0f;
            if (on) {
                d += 2.0 / (c.dx[a] * c.dx[a]);
                dV *= c.dx[a];
            }
        }
        in.inv_diag = (float)(1.0 / d);
        in.dV = dV;
        const double V = dV * (double)in.cells;
        in.scale = c.q * c.weight / dV * ldexp(1.0, -b->fx_bits[i]);
        in.mean_e = c.q * c.weight * (double)np[i] / V;
        in.bg = isnan(c.rho_background) ? -in.mean_e : c.rho_background;
        const unsigned long long M = (unsigned long long)np[i] << b->fx_bits[i];  // < 2^62
        const unsigned long long C = (unsigned long long)in.cells;
        in.mean_q = (long long)(M / C);
        in.mean_r = (float)((double)(M - (M / C) * C) / (double)C);
        in.scale_f = (float)in.scale;
    }
    BatchGrid &G = b->G;
    G.nitems = (int)b->items.size();
    G.ninst = n;
    BTRY(upload(b->items, &G.items));
    BTRY(upload(b->binst, &G.inst));
    const size_t nn = (size_t)(nodes > 0 ? nodes : 1);
    BTRY(balloc(b, &G.A.acc, nn));
    BTRY(balloc(b, &G.A.b, nn));
    BTRY(balloc(b, &G.A.phi, nn));
    BTRY(balloc(b, &G.A.r, nn));
    BTRY(balloc(b, &G.A.p, nn));
    BTRY(balloc(b, &G.A.q, nn));
    BTRY(balloc(b, &G.A.x, nn));
    BTRY(balloc(b, &G.A.E, nn));
    BCU(b, cudaMemsetAsync(G.A.phi, 0, nn * 4, b->stream));
    BCU(b, cudaMemsetAsync(G.A.E, 0, nn * 8, b->stream));
    BTRY(balloc(b, &G.cg.part, (size_t)G.nitems * 4 + 4));
    BTRY(balloc(b, &G.cg.scal, (size_t)n * 8));
    BTRY(balloc(b, &G.cg.done, (size_t)n));
    BTRY(balloc(b, &G.cg.iters, (size_t)n));
    BCU(b, cudaMemsetAsync(G.cg.scal, 0, (size_t)n * 64, b->stream));
    BCU(b, cudaMemsetAsync(G.cg.done, 0, (size_t)n * 4, b->stream));
    BCU(b, cudaMemsetAsync(G.cg.iters, 0, (size_t)n * 4, b->stream));
    if (b->use_fft) BTRY(setup_fft(b));
    BTRY(balloc(b, &b->d_act, (size_t)G.nitems + 1));
    if (b->h_act) cudaFreeHost(b->h_act);
    b->h_act = nullptr;
    BCU(b, cudaMallocHost(&b->h_act, sizeof(int) * ((size_t)G.nitems + 1)));
    G.act = nullptr;
    G.nact = G.nitems;
    BTRY(balloc(b, &G.fepart, (size_t)G.nitems + 1));
    BTRY(balloc(b, &G.ipart_ll, (size_t)G.nitems + 1));
    BTRY(balloc(b, &b->d_diag, (size_t)n * 8));
    BTRY(balloc(b, &b->d_isum, (size_t)n));
    BTRY(balloc(b, &b->d_err, 1));
    BCU(b, cudaMemsetAsync(b->d_diag, 0, (size_t)n * 64, b->stream));
    BCU(b, cudaMemsetAsync(b->d_err, 0, 4, b->stream));
    BTRY(balloc(b, reinterpret_cast<unsigned char **>(&b->d_tparams),
                batch_tile_params_bytes() * n));
    b->pass_blocks = b->sms * b->tune.pass_ctas_per_sm;
    // particles: host FP64 -> cell + FP32 offset, instance by instance
    int64_t maxnp = 1;
    for (int i = 0; i < n; ++i) maxnp = np[i] > maxnp ? np[i] : maxnp;
    double *dx_buf = nullptr, *dv_buf = nullptr;
    BTRY(balloc(b, &dx_buf, (size_t)maxnp * 2));
    BTRY(balloc(b, &dv_buf, (size_t)maxnp * 2));
    for (int i = 0; i < n; ++i) {
        if (np[i] == 0) continue;
        const ap_pic_config &c = b->cfg[i];
        BCU(b, cudaMemcpyAsync(dx_buf, x[i], (size_t)np[i] * c.ndim * 8, cudaMemcpyHostToDevice,
                               b->stream));
        BCU(b, cudaMemcpyAsync(dv_buf, v[i], (size_t)np[i] * 2 * 8, cudaMemcpyHostToDevice,
                               b->stream));
        ParticlesF32 sub = b->p;  // this instance's slice of the arena
        sub.cell += b->pbase[i];
        sub.off += b->pbase[i];
        sub.v += b->pbase[i];
        sub.np = np[i];
        const GridParams g = make_gp(c, b->fx_bits[i], c.dt);
        BCU(b, launch_load_convert(g, c.dx, dx_buf, dv_buf, sub, 0, np[i], b->d_err, b->stream));
        BCU(b, cudaStreamSynchronize(b->stream));  // the staging buffers are reused
    }
    BTRY(batch_sync_check(b));
    // sort, deposit, solve, half push (Listing 1's load)
    BTRY(batch_sort(b));
    BTRY(upload_tile_params(b, 1.0));
    BCU(b, cudaMemsetAsync(G.A.acc, 0, nn * 8, b->stream));
    BTRY(batch_pass(b, false, false, true, false));
    BTRY(batch_convert(b));
    if (b->use_fft) {
        BTRY(field_fft(b));
    } else {
        cg_start(b, G.A.phi, G.A.b, b->cfg[0].cg_rtol);
        BTRY(step_back(b, 0));
    }
    if (!(flags & AP_PIC_LOAD_NO_HALFPUSH)) {
        BTRY(upload_tile_params(b, -0.5));
        BTRY(batch_pass(b, true, false, false, false));
        BTRY(upload_tile_params(b, 1.0));
    }
    b->loaded = true;
    b->step = 0;
    return AP_PIC_OK;
}

}  // namespace

// Loads every instance: x[i] (np[i] x ndim_i) and v[i] (np[i] x 2), host FP64.
extern "C" ap_pic_status ap_pic_batch_load(ap_pic_batch *b, const int64_t *np,
                                           const double *const *x, const double *const *v,
                                           unsigned flags)
{
    if (!b || !np || !x || !v) return AP_PIC_ERR_ARG;
    if (b->loaded) return bfail(b, AP_PIC_ERR_STATE, "the batch is already loaded");
    BTRY(fenced(b, [&] { return load_body(b, np, x, v, flags); }));
    return batch_sync_check(b);
}

namespace {

// Captures the front of a step (particle pass .. first block of CG iterations)
// as a CUDA graph on first use; it is replayed every step.
ap_pic_status ensure_graph(ap_pic_batch *b)
{
    cudaGraphExec_t &gx = b->graphs[b->parity];
    if (gx) return AP_PIC_OK;
    const int64_t before = ap_pic_kernel_launches();
    cudaGraph_t g = nullptr;
    BCU(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    const ap_pic_status st = step_front(b, true);
    const cudaError_t ce = cudaStreamEndCapture(b->stream, &g);
    if (st != AP_PIC_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    BCU(b, ce);
    const cudaError_t ie = cudaGraphInstantiate(&gx, g, 0);
    cudaGraphDestroy(g);
    BCU(b, ie);
    // the capture recorded the kernels without running them
    b->graph_launches = ap_pic_kernel_launches() - before;
    note_launch(-(int)b->graph_launches);
    return AP_PIC_OK;
}

ap_pic_status need_loaded(ap_pic_batch *b, int i)
{
    if (!b) return AP_PIC_ERR_ARG;
    if (!b->loaded) return bfail(b, AP_PIC_ERR_STATE, "the batch is not loaded");
    if (i < 0 || i >= b->count) return bfail(b, AP_PIC_ERR_ARG, "instance index out of range");
    return AP_PIC_OK;
}

}  // namespace

extern "C" ap_pic_status ap_pic_batch_step(ap_pic_batch *b, int nsteps)
{
    BTRY(need_loaded(b, 0));
    if (nsteps < 0) return bfail(b, AP_PIC_ERR_ARG, "nsteps must be >= 0");
    return fenced(b, [&]() -> ap_pic_status {
        for (int s = 0; s < nsteps; ++s) {
            const int64_t k = b->step + 1;
            if (b->tune.use_graph) {
                BTRY(ensure_graph(b));
                BCU(b, cudaGraphLaunch(b->graphs[b->parity], b->stream));
                note_launch((int)b->graph_launches);
            } else {
                BTRY(step_front(b, true));
            }
            if (b->tune.sort_every > 0 && k % b->tune.sort_every == 0) BTRY(batch_sort(b));
            if (!b->use_fft) BTRY(step_back(b, b->tune.cg_iters_per_graph));
            b->step = k;
        }
        return AP_PIC_OK;
    });
}

// The parts of a step on their own (a step is push_deposit, a sort when due,
// solve_field); none of them advances the step counter.
extern "C" ap_pic_status ap_pic_batch_push_deposit(ap_pic_batch *b)
{
    BTRY(need_loaded(b, 0));
    return fenced(b, [&]() -> ap_pic_status {
        BCU(b, cudaMemsetAsync(b->G.A.acc, 0, (size_t)b->total_nodes * 8, b->stream));
        BTRY(batch_pass(b, true, true, true, true));
        return batch_convert(b);
    });
}

extern "C" ap_pic_status ap_pic_batch_sort(ap_pic_batch *b)
{
    BTRY(need_loaded(b, 0));
    return fenced(b, [&] { return batch_sort(b); });
}

extern "C" ap_pic_status ap_pic_batch_solve_field(ap_pic_batch *b)
{
    BTRY(need_loaded(b, 0));
    return fenced(b, [&]() -> ap_pic_status {
        BatchGrid &G = b->G;
        if (b->use_fft) return field_fft(b);
        const int first = b->tune.cg_iters_per_graph;
        cg_start(b, G.A.phi, G.A.b, b->cfg[0].cg_rtol);
        cg_iters(b, G.A.phi, 0, first, b->cfg[0].cg_maxit, b->cfg[0].cg_rtol);
        return step_back(b, first);
    });
}

extern "C" int64_t ap_pic_batch_num_particles(const ap_pic_batch *b, int i)
{
    return (b && b->loaded && i >= 0 && i < b->count) ? b->np[i] : 0;
}

extern "C" ap_pic_status ap_pic_batch_get_rho(ap_pic_batch *b, int i, double *out)
{
    BTRY(need_loaded(b, i));
    if (!out) return bfail(b, AP_PIC_ERR_ARG, "out is NULL");
    // rho = scale acc + bg, formed here in place from the int64 accumulator
    BCU(b, cudaMemcpyAsync(out, b->G.A.acc + b->node0[i], (size_t)b->cells[i] * 8,
                           cudaMemcpyDeviceToHost, b->stream));
    const ap_pic_status st = batch_sync_check(b);
    if (st != AP_PIC_OK) return st;
    const BInst &in = b->binst[i];
    for (int64_t j = 0; j < b->cells[i]; ++j) {
        int64_t a;
        memcpy(&a, &out[j], 8);
        out[j] = in.scale * (double)a + in.bg;
    }
    return AP_PIC_OK;
}

extern "C" ap_pic_status ap_pic_batch_get_E(ap_pic_batch *b, int i, double *out)
{
    BTRY(need_loaded(b, i));
    if (!out) return bfail(b, AP_PIC_ERR_ARG, "out is NULL");
    const int64_t c = b->cells[i];
    std::vector<float2> tmp((size_t)c);
    BCU(b, cudaMemcpyAsync(tmp.data(), b->G.A.E + b->node0[i], (size_t)c * 8,
                           cudaMemcpyDeviceToHost, b->stream));
    BTRY(batch_sync_check(b));
    if (b->cfg[i].ndim == 1) {  // packed floats at the start of the region
        const float *f = reinterpret_cast<const float *>(tmp.data());
        for (int64_t j = 0; j < c; ++j) out[j] = f[j];
    } else {
        for (int64_t j = 0; j < c; ++j) {
            out[j] = tmp[(size_t)j].x;
            out[c + j] = tmp[(size_t)j].y;
        }
    }
    return AP_PIC_OK;
}

extern "C" ap_pic_status ap_pic_batch_get_particles(ap_pic_batch *b, int i, int32_t *cell,
                                                    float *off, float *v, double *x)
{
    BTRY(need_loaded(b, i));
    const int64_t n = b->np[i], base = b->pbase[i], st = b->p.stride;
    const int nd = b->cfg[i].ndim;
    if (n == 0) return AP_PIC_OK;
    std::vector<int32_t> c((size_t)n);
    std::vector<float> o((size_t)n * nd), vv((size_t)n * 2);
    BCU(b, cudaMemcpyAsync(c.data(), b->p.cell + base, (size_t)n * 4, cudaMemcpyDeviceToHost,
                           b->stream));
    for (int a = 0; a < nd; ++a)
        BCU(b, cudaMemcpyAsync(o.data() + (size_t)a * n, b->p.off + a * st + base, (size_t)n * 4,
                               cudaMemcpyDeviceToHost, b->stream));
    for (int a = 0; a < 2; ++a)
        BCU(b, cudaMemcpyAsync(vv.data() + (size_t)a * n, b->p.v + a * st + base, (size_t)n * 4,
                               cudaMemcpyDeviceToHost, b->stream));
    BTRY(batch_sync_check(b));
    const ap_pic_config &cf = b->cfg[i];
    for (int64_t k = 0; k < n; ++k) {
        if (cell) cell[k] = c[(size_t)k];
        int cc[2] = {c[(size_t)k], 0};
        if (nd == 2) {
            cc[1] = c[(size_t)k] / cf.n[0];
            cc[0] = c[(size_t)k] - cc[1] * cf.n[0];
        }
        for (int a = 0; a < nd; ++a) {
            const float fa = o[(size_t)a * n + k];
            if (off) off[k * nd + a] = fa;
            if (x) x[k * nd + a] = ((double)cc[a] + (double)fa) * cf.dx[a];
        }
        if (v)
            for (int a = 0; a < 2; ++a) v[k * 2 + a] = vv[(size_t)a * n + k];
    }
    return AP_PIC_OK;
}

extern "C" ap_pic_status ap_pic_batch_get_perm(ap_pic_batch *b, int i, int64_t *perm)
{
    BTRY(need_loaded(b, i));
    if (!perm) return bfail(b, AP_PIC_ERR_ARG, "perm is NULL");
    if (b->perm_slot < 0) return bfail(b, AP_PIC_ERR_STATE, "no sort has run");
    const int64_t n = b->np[i], base = b->pbase[i];
    std::vector<uint32_t> tmp((size_t)n);
    if (n)
        BCU(b, cudaMemcpyAsync(tmp.data(), b->sort.idx[b->perm_slot] + base, (size_t)n * 4,
                               cudaMemcpyDeviceToHost, b->stream));
    BTRY(batch_sync_check(b));
    for (int64_t k = 0; k < n; ++k) perm[k] = (int64_t)tmp[(size_t)k] - base;
    return AP_PIC_OK;
}

extern "C" ap_pic_status ap_pic_batch_get_diag(ap_pic_batch *b, int i, ap_pic_diag *out)
{
    BTRY(need_loaded(b, i));
    if (!out) return bfail(b, AP_PIC_ERR_ARG, "out is NULL");
    double d[8];
    long long isum = 0;
    int iters = 0;
    double rel = 0.0;
    BCU(b, cudaMemcpyAsync(d, b->d_diag + (size_t)i * 8, sizeof d, cudaMemcpyDeviceToHost,
                           b->stream));
    BCU(b, cudaMemcpyAsync(&isum, b->d_isum + i, sizeof isum, cudaMemcpyDeviceToHost, b->stream));
    BCU(b, cudaMemcpyAsync(&iters, b->G.cg.iters + i, sizeof iters, cudaMemcpyDeviceToHost,
                           b->stream));
    BCU(b, cudaMemcpyAsync(&rel, b->G.cg.scal + (size_t)i * 8 + 3, sizeof rel,
                           cudaMemcpyDeviceToHost, b->stream));
    BTRY(batch_sync_check(b));
    const ap_pic_config &c = b->cfg[i];
    const double mw = c.m * c.weight;
    memset(out, 0, sizeof *out);
    out->step = b->step;
    out->t = (double)b->step * c.dt;
    out->np = b->np[i];
    out->fx_bits = b->fx_bits[i];
    out->charge_fx_sum = isum;
    out->total_charge = c.q * c.weight * ldexp((double)isum, -b->fx_bits[i]);
    out->kinetic = 0.5 * mw * d[0];
    out->momentum[0] = mw * d[1];
    out->momentum[1] = mw * d[2];
    out->field_energy = 0.5 * b->binst[i].dV * d[3];
    out->cg_iters = iters;
    out->cg_relres = rel;
    out->error_flags = *b->h_err;
    return AP_PIC_OK;
}

// ---- autotuner --------------------------------------------------------------------------------

namespace {

uint64_t shape_hash(const ap_pic_batch *b)
{
    uint64_t h = 1469598103934665603ull;  // FNV-1a, 64 bit
    auto mix = [&](uint64_t v) {
        for (int k = 0; k < 8; ++k) {
            h ^= (v >> (8 * k)) & 0xff;
            h *= 1099511628211ull;
        }
    };
    mix((uint64_t)b->count);
    for (int i = 0; i < b->count; ++i) {
        mix((uint64_t)b->cfg[i].ndim);
        mix((uint64_t)b->cfg[i].n[0]);
        mix((uint64_t)b->cfg[i].n[1]);
        mix((uint64_t)b->np[i]);
    }
    return h;
}

// Milliseconds per step of `steps` steps with the current tuning.
ap_pic_status time_steps(ap_pic_batch *b, int steps, double *ms)
{
    cudaEvent_t e0, e1;
    BCU(b, cudaEventCreate(&e0));
    BCU(b, cudaEventCreate(&e1));
    BCU(b, cudaEventRecord(e0, b->stream));
    const ap_pic_status st = ap_pic_batch_step(b, steps);
    BCU(b, cudaEventRecord(e1, b->stream));
    BCU(b, cudaEventSynchronize(e1));
    float t = 0.0f;
    cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = (double)t / steps;
    return st;
}

}  // namespace

extern "C" ap_pic_status ap_pic_batch_autotune(ap_pic_batch *b, int steps_per_trial,
                                               const char *cache_path)
{
    BTRY(need_loaded(b, 0));
    if (steps_per_trial < 1) return bfail(b, AP_PIC_ERR_ARG, "steps_per_trial must be >= 1");
    cudaDeviceProp prop;
    int dev = 0;
    cudaGetDevice(&dev);
    BCU(b, cudaGetDeviceProperties(&prop, dev));
    std::string gpu(prop.name);
    for (char &ch : gpu)
        if (ch == ' ') ch = '_';
    const uint64_t key = shape_hash(b);
    ap_pic_batch_tuning t = b->tune;
    if (cache_path) {
        FILE *f = fopen(cache_path, "r");
        if (f) {
            char name[256];
            unsigned long long k = 0;
            int c1, c2, c3, c4, c5;
            bool hit = false;
            while (fscanf(f, "%llx %255s %d %d %d %d %d", &k, name, &c1, &c2, &c3, &c4, &c5) ==
                   7) {
                if (k == key && gpu == name) {
                    t.pass_ctas_per_sm = c1;
                    t.cg_iters_per_graph = c2;
                    t.sort_every = c3;
                    t.pass_threads = c4;
                    t.pass_per_thread = c5;
                    hit = true;
                }
            }
            fclose(f);
            if (hit) return ap_pic_batch_set_tuning(b, &t);
        }
    }
    // Coordinate search: the pass kernel's shape (threads per CTA x particles per
    // thread), its CTAs per SM, the CG block length (CG solver only: the spectral
    // solve has no such block), then the sort cadence.
    const int ctas[] = {2, 3, 4, 6, 8};
    const int iters[] = {8, 16, 32};
    const int sorts[] = {10, 20, 40};
    auto trial = [&](ap_pic_batch_tuning cand, int steps, double *ms) -> ap_pic_status {
        BTRY(ap_pic_batch_set_tuning(b, &cand));
        BTRY(ap_pic_batch_step(b, 1));  // graph capture and warm-up
        return time_steps(b, steps, ms);
    };
    double best = 1e300;
    ap_pic_batch_tuning best_t = t;
    for (int v = 0; v < batch_variant_count(); ++v) {
        ap_pic_batch_tuning cand = best_t;
        batch_variant_shape(v, &cand.pass_threads, &cand.pass_per_thread);
        double ms = 0.0;
        BTRY(trial(cand, steps_per_trial, &ms));
        if (ms < best) {
            best = ms;
            best_t = cand;
        }
    }
    best = 1e300;
    for (int c : ctas) {
        ap_pic_batch_tuning cand = best_t;
        cand.pass_ctas_per_sm = c;
        double ms = 0.0;
        BTRY(trial(cand, steps_per_trial, &ms));
        if (ms < best) {
            best = ms;
            best_t = cand;
        }
    }
    if (!b->use_fft) {
        best = 1e300;
        for (int it : iters) {
            ap_pic_batch_tuning cand = best_t;
            cand.cg_iters_per_graph = it;
            double ms = 0.0;
            BTRY(trial(cand, steps_per_trial, &ms));
            if (ms < best) {
                best = ms;
                best_t = cand;
            }
        }
    }
    best = 1e300;
    for (int se : sorts) {
        ap_pic_batch_tuning cand = best_t;
        cand.sort_every = se;
        double ms = 0.0;
        // cover at least one sort so its cost is part of the per-step time
        BTRY(trial(cand, steps_per_trial > se ? steps_per_trial : se, &ms));
        if (ms < best) {
            best = ms;
            best_t = cand;
        }
    }
    BTRY(ap_pic_batch_set_tuning(b, &best_t));
    if (cache_path) {
        FILE *f = fopen(cache_path, "a");
        if (f) {
            fprintf(f, "%llx %s %d %d %d %d %d\n", (unsigned long long)key, gpu.c_str(),
                    best_t.pass_ctas_per_sm, best_t.cg_iters_per_graph, best_t.sort_every,
                    best_t.pass_threads, best_t.pass_per_thread);
            fclose(f);
        }
    }
    return AP_PIC_OK;
}
