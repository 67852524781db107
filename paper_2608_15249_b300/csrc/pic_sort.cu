// pic_sort.cu -- stable per-cell sort of the particles (a layout step: the
// paper does not name one; it keeps gather and deposit accesses local).
//
// Key: brick-major cell index.  The grid is tiled by bricks of b0 x b1 x b2
// cells (the last brick on an axis may be partial):
//   key = brick_id * (b0 b1 b2) + local_id,
//   brick_id = c0/b0 + nb0 (c1/b1 + nb1 c2/b2),   nb_a = ceil(n_a / b_a),
//   local_id = c0%b0 + b0 (c1%b1 + b1 c2%b2).
// Sort: least-significant-digit radix sort over (key, index) pairs with digits
// of up to 10 bits (as few passes as the key width allows: two 9-bit passes for
// an 18-bit key).  Each pass is stable (per-tile digit histograms, a device-wide
// exclusive scan in digit-major order, and a scatter whose in-tile ranks keep
// input order), so the result is the unique stable permutation.  The
// particle record is then gathered through the permutation.
#include <type_traits>

#include "pic_internal.cuh"

namespace apk {

constexpr int ST_THREADS = 256;
constexpr int ST_WARPS = ST_THREADS / 32;
constexpr int ST_ITEMS = 16;
constexpr int ST_TILE = ST_THREADS * ST_ITEMS;  // 4096 items per tile
static_assert(ST_TILE == SORT_TILE, "tile size shared with the scratch sizing");
constexpr int MAX_DIGIT_BITS = SORT_MAX_DIGIT_BITS;
constexpr int MAX_RADIX = SORT_MAX_RADIX;
constexpr int NO_DIGIT = -1;                    // marks an item past the end

static int64_t tiles_of(int64_t np) { return (np + ST_TILE - 1) / ST_TILE; }

size_t sort_hist_len(int64_t np) { return (size_t)MAX_RADIX * (size_t)tiles_of(np); }

// ---- keys ----------------------------------------------------------------------------------

// (Divisions by the grid and brick sizes use the multiply-high FastDiv: a
// runtime integer division compiles to float conversions, which issue on the
// slow FP64 pipe of this GPU.)
struct KeyParams {
    FastDiv dn0, dn1, db0, db1, db2;
    uint32_t nb0, nb1;
    uint32_t absorbed;  // key of a particle marked absorbed (negative cell): one past the
                        // last cell key, so the sort moves such particles to the end
};

template <int D>
__device__ __forceinline__ uint32_t brick_key(uint32_t c, const KeyParams &k)
{
    if ((int32_t)c < 0) return k.absorbed;
    uint32_t c0, c1 = 0, c2 = 0;
    if (D == 1) {
        c0 = c;
    } else if (D == 2) {
        c1 = fdiv(c, k.dn0);
        c0 = c - c1 * k.dn0.d;
    } else {
        const uint32_t c12 = fdiv(c, k.dn0);
        c0 = c - c12 * k.dn0.d;
        c2 = fdiv(c12, k.dn1);
        c1 = c12 - c2 * k.dn1.d;
    }
    const uint32_t b0 = k.db0.d, b1 = D >= 2 ? k.db1.d : 1u, b2 = D == 3 ? k.db2.d : 1u;
    const uint32_t q0 = fdiv(c0, k.db0);
    const uint32_t q1 = D >= 2 ? fdiv(c1, k.db1) : 0u, q2 = D == 3 ? fdiv(c2, k.db2) : 0u;
    const uint32_t bid = q0 + k.nb0 * (q1 + k.nb1 * q2);
    const uint32_t lid = (c0 - q0 * b0) + b0 * ((c1 - q1 * b1) + b1 * (c2 - q2 * b2));
    return bid * (b0 * b1 * b2) + lid;
}

// Four keys per thread and iteration (16-byte loads and stores when both arrays
// start on 16 bytes, as the library's own do; a caller's cell array may not, and
// then goes one key at a time), persistent grid.
template <int D>
__global__ void __launch_bounds__(256)
    k_keys(KeyParams kp, const int32_t *__restrict__ cell, int64_t np, uint32_t *__restrict__ keys)
{
    if ((reinterpret_cast<uintptr_t>(cell) | reinterpret_cast<uintptr_t>(keys)) & 15u) {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < np;
             i += (int64_t)gridDim.x * blockDim.x)
            keys[i] = brick_key<D>((uint32_t)cell[i], kp);
        return;
    }
    const int64_t nq = np / 4;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nq;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int4 c = __ldg(reinterpret_cast<const int4 *>(cell) + q);
        uint4 k;
        k.x = brick_key<D>((uint32_t)c.x, kp);
        k.y = brick_key<D>((uint32_t)c.y, kp);
        k.z = brick_key<D>((uint32_t)c.z, kp);
        k.w = brick_key<D>((uint32_t)c.w, kp);
        reinterpret_cast<uint4 *>(keys)[q] = k;
    }
    const int64_t t = 4 * nq + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < np) keys[t] = brick_key<D>((uint32_t)cell[t], kp);
}

// ---- per-tile digit histogram ----------------------------------------------------------------

// Thread t of a tile counts the 16 consecutive keys [16 t, 16 t + 16) of the tile
// (four 16-byte loads): runs of equal digits, which are long for the near-sorted
// keys of a re-sort, go to the shared histogram as one atomic each.
template <int RADIX>
__global__ void __launch_bounds__(ST_THREADS)
    k_hist(const uint32_t *__restrict__ keys, int64_t np, int shift, uint32_t *__restrict__ hist,
           int64_t ntiles)
{
    __shared__ uint32_t h[RADIX];
    for (int j = threadIdx.x; j < RADIX; j += ST_THREADS) h[j] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * ST_TILE + (int64_t)threadIdx.x * ST_ITEMS;
    uint32_t k[ST_ITEMS];
    int valid = ST_ITEMS;
    if (base + ST_ITEMS <= np) {
        const uint4 *src = reinterpret_cast<const uint4 *>(keys + base);
#pragma unroll
        for (int r = 0; r < ST_ITEMS / 4; ++r) {
            const uint4 q = __ldg(src + r);
            k[4 * r] = q.x;
            k[4 * r + 1] = q.y;
            k[4 * r + 2] = q.z;
            k[4 * r + 3] = q.w;
        }
    } else {
        valid = base < np ? (int)(np - base) : 0;
#pragma unroll
        for (int r = 0; r < ST_ITEMS; ++r) k[r] = r < valid ? keys[base + r] : 0u;
    }
    int run_d = -1;
    uint32_t run_n = 0;
#pragma unroll
    for (int r = 0; r < ST_ITEMS; ++r) {
        if (r >= valid) break;
        const int d = (int)((k[r] >> shift) & (RADIX - 1));
        if (d == run_d) {
            ++run_n;
        } else {
            if (run_n) atomicAdd(&h[run_d], run_n);
            run_d = d;
            run_n = 1;
        }
    }
    if (run_n) atomicAdd(&h[run_d], run_n);
    __syncthreads();
    for (int j = threadIdx.x; j < RADIX; j += ST_THREADS)
        hist[(int64_t)j * ntiles + blockIdx.x] = h[j];
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// ---- stable scatter --------------------------------------------------------------------------

// The lanes whose digit equals this lane's (NO_DIGIT lanes form their own group), from
// one ballot per digit bit: cheaper on this GPU than a lane match over many distinct
// values.
template <int RADIX>
__device__ __forceinline__ unsigned peer_mask(int d)
{
    const bool valid = d != NO_DIGIT;
    const unsigned vb = __ballot_sync(0xffffffffu, valid);
    unsigned m = valid ? vb : ~vb;
#pragma unroll
    for (int b = 0; (1 << b) < RADIX; ++b) {
        const bool bit = (d >> b) & 1;
        const unsigned bb = __ballot_sync(0xffffffffu, bit);
        m &= bit ? bb : ~bb;
    }
    return m;
}

// Warp w of a tile owns the contiguous items [w*512, (w+1)*512) of the tile and
// walks them in 16 rounds of 32, so (warp, round, lane) order is input order.  A
// round whose 32 digits are all equal (the usual case for the near-sorted keys of
// a re-sort) ranks by lane, against a running count of that digit kept in a
// register; other rounds rank against the warp's shared per-digit counts within
// groups of equal digits (peer_mask).  The ranked items are then placed in shared
// memory in the tile's own sorted order (digit runs one after another) and written
// out from there: consecutive threads write consecutive positions of each digit's
// run, so the global writes come in whole sectors instead of scattered words.
template <int RADIX, bool STAGED>
constexpr size_t scatter_smem_bytes()
{
    // per-warp digit counts; staged: the tile's keys and indices, per-digit local
    // starts and global deltas
    return STAGED ? ((size_t)ST_WARPS * RADIX + 2 * (size_t)ST_TILE + 2 * (size_t)RADIX) * 4
                  : (size_t)ST_WARPS * RADIX * 4;
}

template <int RADIX, bool STAGED>
__global__ void __launch_bounds__(ST_THREADS, 3)
    k_scatter(const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ idx_in, int64_t np,
              int shift, const uint32_t *__restrict__ offs, int64_t ntiles,
              uint32_t *__restrict__ keys_out, uint32_t *__restrict__ idx_out)
{
    extern __shared__ uint32_t sm_flat[];
    uint32_t *wcount_flat = sm_flat;                       // [ST_WARPS][RADIX]
    uint32_t *s_key = wcount_flat + ST_WARPS * RADIX;     // [ST_TILE], tile order (staged)
    uint32_t *s_idx = s_key + ST_TILE;                    // [ST_TILE]
    uint32_t *s_lstart = s_idx + ST_TILE;                 // [RADIX] digit run starts in the tile
    uint32_t *s_gdelta = s_lstart + RADIX;                // [RADIX] global start - local start
    auto wcount = [&](int w, int d) -> uint32_t & { return wcount_flat[w * RADIX + d]; };
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int j = threadIdx.x; j < ST_WARPS * RADIX; j += ST_THREADS) wcount_flat[j] = 0;
    __syncthreads();
    const int64_t tile0 = (int64_t)blockIdx.x * ST_TILE;
    const int64_t base = tile0 + (int64_t)w * (ST_ITEMS * 32);
    const int count = np - tile0 < ST_TILE ? (int)(np - tile0) : ST_TILE;
    const unsigned lt = (1u << lane) - 1u;
    uint32_t key[ST_ITEMS], rank[ST_ITEMS];
#pragma unroll
    for (int r = 0; r < ST_ITEMS; ++r) {
        const int64_t i = base + r * 32 + lane;
        key[r] = i < np ? keys_in[i] : 0u;
    }
    auto digit = [&](int r) {
        return base + r * 32 + lane < np ? (int)((key[r] >> shift) & (RADIX - 1)) : NO_DIGIT;
    };
    int cd = NO_DIGIT;  // the cached digit (warp-uniform) and its running count
    uint32_t cc = 0;
#pragma unroll
    for (int r = 0; r < ST_ITEMS; ++r) {
        const int d = digit(r);
        const int d0 = __shfl_sync(0xffffffffu, d, 0);
        if (__all_sync(0xffffffffu, d == d0) && d0 != NO_DIGIT) {
            if (d0 != cd) {
                if (cd != NO_DIGIT && lane == 0) wcount(w, cd) = cc;
                __syncwarp();
                cc = wcount(w, d0);
                cd = d0;
            }
            rank[r] = cc + (uint32_t)lane;
            cc += 32;
        } else {
            if (cd != NO_DIGIT && lane == 0) wcount(w, cd) = cc;
            cd = NO_DIGIT;
            __syncwarp();
            const unsigned m = peer_mask<RADIX>(d);
            uint32_t before = 0;
            if (d != NO_DIGIT) before = wcount(w, d);
            rank[r] = before + (uint32_t)__popc(m & lt);
            __syncwarp();
            if (d != NO_DIGIT && (m & lt) == 0) wcount(w, d) = before + (uint32_t)__popc(m);
            __syncwarp();
        }
    }
    if (cd != NO_DIGIT && lane == 0) wcount(w, cd) = cc;
    __syncthreads();
    if constexpr (!STAGED) {
        // each item straight to its global position (the digit runs of a pass whose
        // rounds are mostly uniform already come in long runs)
        for (int d = threadIdx.x; d < RADIX; d += ST_THREADS) {
            uint32_t run = offs[(int64_t)d * ntiles + blockIdx.x];
            for (int ww = 0; ww < ST_WARPS; ++ww) {
                const uint32_t t = wcount(ww, d);
                wcount(ww, d) = run;
                run += t;
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < ST_ITEMS; ++r) {
            const int d = digit(r);
            if (d == NO_DIGIT) continue;
            const int64_t i = base + r * 32 + lane;
            const uint32_t pos = wcount(w, d) + rank[r];
            if (keys_out) keys_out[pos] = key[r];
            idx_out[pos] = idx_in ? idx_in[i] : (uint32_t)i;
        }
    } else {
        // per digit: each warp's offset within the tile's run of that digit, and the run
        // length (kept in s_lstart until the scan below)
        for (int d = threadIdx.x; d < RADIX; d += ST_THREADS) {
            uint32_t run = 0;
            for (int ww = 0; ww < ST_WARPS; ++ww) {
                const uint32_t t = wcount(ww, d);
                wcount(ww, d) = run;
                run += t;
            }
            s_lstart[d] = run;
        }
        __syncthreads();
        // exclusive scan of the run lengths over the digits: RADIX / ST_THREADS (or one)
        // consecutive digits per thread, then a warp scan and the warps' totals
        {
            constexpr int PER = RADIX >= ST_THREADS ? RADIX / ST_THREADS : 1;
            const int d0 = threadIdx.x * PER;
            uint32_t v[PER], run = 0;
    #pragma unroll
            for (int k = 0; k < PER; ++k) {
                v[k] = d0 + k < RADIX ? s_lstart[d0 + k] : 0u;
                const uint32_t t = v[k];
                v[k] = run;
                run += t;
            }
            const uint32_t incl = warp_incl_scan(run);
            __shared__ uint32_t s_wsum[ST_WARPS];
            if (lane == 31) s_wsum[w] = incl;
            __syncthreads();
            uint32_t wbase = 0;
            for (int j = 0; j < w; ++j) wbase += s_wsum[j];
            const uint32_t excl = wbase + incl - run;
    #pragma unroll
            for (int k = 0; k < PER; ++k)
                if (d0 + k < RADIX) {
                    const uint32_t ls = v[k] + excl;
                    s_lstart[d0 + k] = ls;
                    s_gdelta[d0 + k] = offs[(int64_t)(d0 + k) * ntiles + blockIdx.x] - ls;
                }
        }
        __syncthreads();
        // the tile's items in its own sorted order
    #pragma unroll
        for (int r = 0; r < ST_ITEMS; ++r) {
            const int d = digit(r);
            if (d == NO_DIGIT) continue;
            const int64_t i = base + r * 32 + lane;
            const uint32_t lp = s_lstart[d] + wcount(w, d) + rank[r];
            s_key[lp] = key[r];
            s_idx[lp] = idx_in ? idx_in[i] : (uint32_t)i;
        }
        __syncthreads();
        // out in runs: local position q of digit d goes to global position gdelta[d] + q
        for (int q = threadIdx.x; q < count; q += ST_THREADS) {
            const uint32_t k = s_key[q];
            const uint32_t pos = s_gdelta[(k >> shift) & (RADIX - 1)] + (uint32_t)q;
            if (keys_out) keys_out[pos] = k;
            idx_out[pos] = s_idx[q];
        }
    }
}

// ---- device-wide exclusive scan of u32 (three phases, recursive on the partials) ------------

constexpr int SC_THREADS = 256;
constexpr int SC_ITEMS = 16;
constexpr int SC_TILE = SC_THREADS * SC_ITEMS;

size_t sort_scan_tmp_len(size_t n)
{
    size_t total = 0;
    while (n > (size_t)SC_TILE) {
        n = (n + SC_TILE - 1) / SC_TILE;
        total += n;
    }
    return total + 1;
}

// Exclusive scan of one tile held 16 consecutive items per thread; returns the
// tile total in *total (all threads).
__device__ void block_excl_scan(uint32_t (&v)[SC_ITEMS], uint32_t *total)
{
    __shared__ uint32_t wsum[SC_THREADS / 32];
    uint32_t run = 0;
#pragma unroll
    for (int k = 0; k < SC_ITEMS; ++k) {
        const uint32_t t = v[k];
        v[k] = run;
        run += t;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t incl = warp_incl_scan(run);
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    uint32_t wbase = 0, tot = 0;
    for (int j = 0; j < SC_THREADS / 32; ++j) {
        if (j < w) wbase += wsum[j];
        tot += wsum[j];
    }
    const uint32_t excl = wbase + incl - run;
#pragma unroll
    for (int k = 0; k < SC_ITEMS; ++k) v[k] += excl;
    *total = tot;
    __syncthreads();
}

__global__ void __launch_bounds__(SC_THREADS)
    k_scan_reduce(const uint32_t *__restrict__ in, size_t n, uint32_t *__restrict__ sums)
{
    const size_t base = (size_t)blockIdx.x * SC_TILE + (size_t)threadIdx.x * SC_ITEMS;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < SC_ITEMS; ++k)
        if (base + k < n) s += in[base + k];
    __shared__ uint32_t red[SC_THREADS / 32];
    s = warp_incl_scan(s);
    if ((threadIdx.x & 31) == 31) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int j = 0; j < SC_THREADS / 32; ++j) t += red[j];
        sums[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(SC_THREADS)
    k_scan_down(const uint32_t *__restrict__ in, size_t n, const uint32_t *__restrict__ block_off,
                uint32_t *__restrict__ out)
{
    const size_t base = (size_t)blockIdx.x * SC_TILE + (size_t)threadIdx.x * SC_ITEMS;
    uint32_t v[SC_ITEMS];
#pragma unroll
    for (int k = 0; k < SC_ITEMS; ++k) v[k] = (base + k < n) ? in[base + k] : 0u;
    uint32_t total;
    block_excl_scan(v, &total);
    const uint32_t off = block_off ? block_off[blockIdx.x] : 0u;
#pragma unroll
    for (int k = 0; k < SC_ITEMS; ++k)
        if (base + k < n) out[base + k] = v[k] + off;
}

cudaError_t launch_exclusive_scan_u32(const uint32_t *in, uint32_t *out, size_t n, uint32_t *tmp,
                                      cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const size_t nb = (n + SC_TILE - 1) / SC_TILE;
    if (nb == 1) {
        k_scan_down<<<1, SC_THREADS, 0, st>>>(in, n, nullptr, out);
        note_launch();
        return cudaGetLastError();
    }
    uint32_t *sums = tmp;
    uint32_t *rest = tmp + nb;
    k_scan_reduce<<<(unsigned)nb, SC_THREADS, 0, st>>>(in, n, sums);
    note_launch();
    cudaError_t e = launch_exclusive_scan_u32(sums, sums, nb, rest, st);
    if (e != cudaSuccess) return e;
    k_scan_down<<<(unsigned)nb, SC_THREADS, 0, st>>>(in, n, sums, out);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_sort_perm(const GridParams &g, const int brick[3], int key_bits,
                             const int32_t *cell, int64_t np, SortScratch &s, int *perm_slot,
                             cudaStream_t st)
{
    if (np <= 0) {
        *perm_slot = 0;
        return cudaSuccess;
    }
    const int b0 = brick[0], b1 = g.ndim >= 2 ? brick[1] : 1, b2 = g.ndim >= 3 ? brick[2] : 1;
    KeyParams kp;
    kp.dn0 = make_fastdiv((uint32_t)g.n[0]);
    kp.dn1 = make_fastdiv((uint32_t)g.n[1]);
    kp.db0 = make_fastdiv((uint32_t)b0);
    kp.db1 = make_fastdiv((uint32_t)b1);
    kp.db2 = make_fastdiv((uint32_t)b2);
    kp.nb0 = (uint32_t)((g.n[0] + b0 - 1) / b0);
    kp.nb1 = g.ndim >= 2 ? (uint32_t)((g.n[1] + b1 - 1) / b1) : 1u;
    {
        uint64_t nk = (uint64_t)kp.nb0 * b0;
        if (g.ndim >= 2) nk *= (uint64_t)kp.nb1 * b1;
        if (g.ndim >= 3) nk *= (uint64_t)((g.n[2] + b2 - 1) / b2) * b2;
        kp.absorbed = (uint32_t)nk;  // needs key_bits > bitlen(nk - 1) where it occurs
    }
    // a persistent grid of 8 CTAs per SM (fewer for small np)
    int64_t kb = (np / 4 + 255) / 256;
    const int64_t cap = (int64_t)sm_count() * 8;
    kb = kb < 1 ? 1 : (kb > cap ? cap : kb);
    if (g.ndim == 1) k_keys<1><<<(int)kb, 256, 0, st>>>(kp, cell, np, s.keys[0]);
    else if (g.ndim == 2) k_keys<2><<<(int)kb, 256, 0, st>>>(kp, cell, np, s.keys[0]);
    else k_keys<3><<<(int)kb, 256, 0, st>>>(kp, cell, np, s.keys[0]);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_sort_keys(key_bits, np, s, perm_slot, st);
}

template <int RADIX, bool STAGED>
static cudaError_t launch_scatter(const uint32_t *keys_in, const uint32_t *idx_in, int64_t np,
                                  int shift, const uint32_t *offs, int64_t ntiles,
                                  uint32_t *keys_out, uint32_t *idx_out, cudaStream_t st)
{
    constexpr size_t smem = scatter_smem_bytes<RADIX, STAGED>();
    static std::atomic<unsigned long long> configured{0};
    const cudaError_t e = once_per_device(configured, [] {
        return cudaFuncSetAttribute(k_scatter<RADIX, STAGED>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
    if (e != cudaSuccess) return e;
    k_scatter<RADIX, STAGED><<<(unsigned)ntiles, ST_THREADS, smem, st>>>(
        keys_in, idx_in, np, shift, offs, ntiles, keys_out, idx_out);
    return cudaSuccess;
}

cudaError_t launch_sort_keys(int key_bits, int64_t np, SortScratch &s, int *perm_slot,
                             cudaStream_t st)
{
    if (np <= 0) {
        *perm_slot = 0;
        return cudaSuccess;
    }
    cudaError_t e = cudaSuccess;
    const int64_t ntiles = tiles_of(np);
    const int passes = key_bits <= 0 ? 1 : (key_bits + MAX_DIGIT_BITS - 1) / MAX_DIGIT_BITS;
    const int dbits = key_bits <= 0 ? 8 : (key_bits + passes - 1) / passes;  // <= 10
    int cur = 0;
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = dbits * pass;
        const bool last = pass == passes - 1;
        const uint32_t *idx_in = pass == 0 ? nullptr : s.idx[cur];
        uint32_t *keys_out = last ? nullptr : s.keys[cur ^ 1];
        const size_t hist_len = ((size_t)1 << (dbits < 8 ? 8 : dbits)) * ntiles;
        auto run = [&](auto radix_tag) -> cudaError_t {
            constexpr int RADIX = decltype(radix_tag)::value;
            k_hist<RADIX><<<(unsigned)ntiles, ST_THREADS, 0, st>>>(s.keys[cur], np, shift, s.hist,
                                                                  ntiles);
            note_launch();
            cudaError_t e2 = launch_exclusive_scan_u32(s.hist, s.hist, hist_len, s.scan_tmp, st);
            if (e2 != cudaSuccess) return e2;
            // the last pass (high digits: long runs of equal digits in a re-sort)
            // writes directly; the others stage their output in shared memory
            e2 = last ? launch_scatter<RADIX, false>(s.keys[cur], idx_in, np, shift, s.hist,
                                                     ntiles, keys_out, s.idx[cur ^ 1], st)
                      : launch_scatter<RADIX, true>(s.keys[cur], idx_in, np, shift, s.hist,
                                                    ntiles, keys_out, s.idx[cur ^ 1], st);
            if (e2 != cudaSuccess) return e2;
            note_launch();
            return cudaGetLastError();
        };
        if (dbits <= 8) e = run(std::integral_constant<int, 256>{});
        else if (dbits == 9) e = run(std::integral_constant<int, 512>{});
        else e = run(std::integral_constant<int, 1024>{});
        if (e != cudaSuccess) return e;
        cur ^= 1;
    }
    *perm_slot = cur;
    return cudaSuccess;
}

// ---- gather the record through the permutation ----------------------------------------------

// dst[r] = src[perm[r]].  Each thread gathers 8 records, all loads issued before
// any store, so enough independent loads are in flight to cover the latency of
// the near-sorted gather (measured on the 16.8M-particle 2D re-sort: 2 records per
// thread 0.615 ms per sort, 4: 0.592, 8: 0.564, 12 and 16 past the register budget
// slower).
constexpr int APPLY_K = 8;

template <int D, int NV>
__global__ void __launch_bounds__(256) k_apply_perm(const uint32_t *__restrict__ perm,
                                                    ParticlesF32 src, ParticlesF32 dst)
{
    constexpr int K = APPLY_K;
    const int64_t np = src.np;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * K;
    for (int64_t base = ((int64_t)blockIdx.x * blockDim.x) * K + threadIdx.x; base < np;
         base += stride) {
        uint32_t j[K];
        bool ok[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int64_t r = base + (int64_t)k * blockDim.x;
            ok[k] = r < np;
            j[k] = ok[k] ? __ldg(perm + r) : 0u;
        }
        int32_t c[K];
        uint32_t id[K];
        float o[K][D], v[K][NV];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            c[k] = __ldg(src.cell + j[k]);
            id[k] = src.id ? __ldg(src.id + j[k]) : 0u;
#pragma unroll
            for (int a = 0; a < D; ++a) o[k][a] = __ldg(src.off + a * src.stride + j[k]);
#pragma unroll
            for (int a = 0; a < NV; ++a) v[k][a] = __ldg(src.v + a * src.stride + j[k]);
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (!ok[k]) continue;
            const int64_t r = base + (int64_t)k * blockDim.x;
            dst.cell[r] = c[k];
            if (src.id) dst.id[r] = id[k];
#pragma unroll
            for (int a = 0; a < D; ++a) dst.off[a * dst.stride + r] = o[k][a];
#pragma unroll
            for (int a = 0; a < NV; ++a) dst.v[a * dst.stride + r] = v[k][a];
        }
    }
}

cudaError_t launch_apply_perm(const uint32_t *perm, ParticlesF32 src, ParticlesF32 dst, int ndim,
                              cudaStream_t st)
{
    if (src.np <= 0) return cudaSuccess;
    int64_t nb = (src.np + 256 * APPLY_K - 1) / (256 * APPLY_K);
    if (nb > 65535) nb = 65535;
    switch (ndim * 10 + src.nv) {
    case 11: k_apply_perm<1, 1><<<(int)nb, 256, 0, st>>>(perm, src, dst); break;
    case 12: k_apply_perm<1, 2><<<(int)nb, 256, 0, st>>>(perm, src, dst); break;
    case 13: k_apply_perm<1, 3><<<(int)nb, 256, 0, st>>>(perm, src, dst); break;
    case 22: k_apply_perm<2, 2><<<(int)nb, 256, 0, st>>>(perm, src, dst); break;
    case 23: k_apply_perm<2, 3><<<(int)nb, 256, 0, st>>>(perm, src, dst); break;
    case 33: k_apply_perm<3, 3><<<(int)nb, 256, 0, st>>>(perm, src, dst); break;
    default: return cudaErrorInvalidValue;
    }
    note_launch();
    return cudaGetLastError();
}

}  // namespace apk
