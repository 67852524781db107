// pic_fft.cu -- spectral solve of the periodic discrete Poisson equation.
//
// The (2d+1)-point periodic Laplacian is diagonal in the discrete Fourier basis:
// -lap_h exp(i k.x) = K^2(k) exp(i k.x) with K^2 = sum_a (2 sin(pi k_a / n_a) / dx_a)^2,
// so -lap_h phi = b is solved exactly by phi_hat(k) = b_hat(k) / K^2(k) and
// phi_hat(0) = 0 (zero-mean potential, the same null-space choice as the CG).
// This is the faster replacement of the CG field solve (the Poisson step D02 of
// Sec. 2.2; the result is the same discrete potential the CG converges to).
//
// Layout: a complex FP32 work array Z[cells] in the grid's node order (x fastest).
// Each axis is transformed by one kernel over all lines along that axis; a CTA
// takes W lines (consecutive rows for the x axis, W adjacent columns otherwise, so
// that global accesses are W-wide segments), holds them in shared memory and
// transforms them there:
//   - power-of-two lengths: self-sorting (Stockham) mixed-radix passes, radix 8 and
//     a last radix 4 or 2, natural order in and out (see stockham below);
//   - other lengths: Bluestein's chirp-z form, X_k = w_k sum_j (x_j w_j) conj(w_{k-j})
//     with w_j = exp(-i pi j^2 / n), a cyclic convolution of power-of-two length
//     m >= 2n - 1 done with radix-2 stages: decimation in time (input scattered to
//     bit-reversed positions, natural-order output) for the forward transform and
//     decimation in frequency (natural input, bit-reversed output) for the inverse,
//     so no separate reordering pass is needed, and a precomputed filter.
// The last axis does forward transform, scaling by 1 / (N K^2) and inverse in one
// kernel; 1D is a single kernel, 2D three, 3D five.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <complex>
#include <vector>

#include "pic_internal.cuh"

namespace apk {

namespace {

constexpr int FFT_THREADS = 256;

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

__device__ __forceinline__ int brev(int j, int log2m) { return (int)(__brev((unsigned)j) >> (32 - log2m)); }

// Shared-memory layout of W lines of length m = 2^log2m: line t starts at t * ls and
// element i sits at i + (i >> ps), one padding slot per m / 32 elements, so the 32
// elements a warp scatters to bit-reversed positions (m / 32 apart) land in
// different banks.  Twiddles follow the lines, stage by stage: stage s (butterfly
// span 2h, h = 2^s) holds exp(-2 pi i k / 2h), k < h, at offset h - 1.
struct SLayout {
    int log2m, ps, ls;
    __device__ int at(int t, int i) const { return t * ls + i + (i >> ps); }
};

__device__ __forceinline__ SLayout slayout(int log2m)
{
    SLayout L;
    L.log2m = log2m;
    L.ps = log2m >= 5 ? log2m - 5 : 30;
    L.ls = (1 << log2m) + (log2m >= 5 ? 32 : 0);
    return L;
}

// W lines in bit-reversed order -> DFT (sign -1, or +1 when inverse) in natural order.
__device__ void dit(float2 *buf, int W, const SLayout &S, const float2 *tws, bool inverse)
{
    const int log2m = S.log2m, half = 1 << (log2m - 1);
    const int nb = W * half;
    for (int s = 0; s < log2m; ++s) {
        const int h = 1 << s;
        for (int b = threadIdx.x; b < nb; b += blockDim.x) {
            const int t = b >> (log2m - 1);
            const int bb = b & (half - 1);
            const int k = bb & (h - 1);
            const int i0 = ((bb >> s) << (s + 1)) + k;
            float2 w = tws[h - 1 + k];
            if (inverse) w.y = -w.y;
            const int a0 = S.at(t, i0), a1 = S.at(t, i0 + h);
            const float2 u = buf[a0], v = cmul(w, buf[a1]);
            buf[a0] = cadd(u, v);
            buf[a1] = csub(u, v);
        }
        __syncthreads();
    }
}

// Natural-order input -> DFT in bit-reversed order (decimation in frequency).
__device__ void dif(float2 *buf, int W, const SLayout &S, const float2 *tws, bool inverse)
{
    const int log2m = S.log2m, half = 1 << (log2m - 1);
    const int nb = W * half;
    for (int s = log2m - 1; s >= 0; --s) {
        const int h = 1 << s;
        for (int b = threadIdx.x; b < nb; b += blockDim.x) {
            const int t = b >> (log2m - 1);
            const int bb = b & (half - 1);
            const int k = bb & (h - 1);
            const int i0 = ((bb >> s) << (s + 1)) + k;
            float2 w = tws[h - 1 + k];
            if (inverse) w.y = -w.y;
            const int a0 = S.at(t, i0), a1 = S.at(t, i0 + h);
            const float2 u = buf[a0], v = buf[a1];
            buf[a0] = cadd(u, v);
            buf[a1] = cmul(csub(u, v), w);
        }
        __syncthreads();
    }
}

// ---- power-of-two lines: self-sorting (Stockham) mixed-radix passes ----------------------
// A length-m transform is a sequence of passes of radix R (8, and a last 2 or 4 when
// log2 m is not a multiple of 3).  Before a pass Ns is the product of the earlier
// radices; group j < m / R takes x[j + r m / R] (r < R), multiplies input r by
// exp(-+2 pi i (j mod Ns) r / (Ns R)), does an R-point DFT in registers, and writes
// output r to y[(j - j mod Ns) R + j mod Ns + r Ns].  Input and output are in natural
// order, so loads and stores need no bit reversal, and a 512-point line takes three
// passes (three barriers) instead of nine radix-2 stages.  Lines sit in shared
// memory with one padding slot per 8 elements (element i at i + i / 8), which breaks
// the 8-element stride of the first pass's writes across banks.

__device__ __forceinline__ int spad(int i) { return i + (i >> 3); }
__host__ __device__ inline int stockham_ls(int m) { return m + (m >> 3); }

// (a - b) times exp(-+2 pi i q / 8), q = 1, 2, 3
template <int Q>
__device__ __forceinline__ float2 rot8(float2 d, bool inverse)
{
    constexpr float c = 0.70710678118654752f;
    if (Q == 2) return inverse ? make_float2(-d.y, d.x) : make_float2(d.y, -d.x);
    if (Q == 1)
        return inverse ? make_float2(c * (d.x - d.y), c * (d.x + d.y))
                       : make_float2(c * (d.x + d.y), c * (d.y - d.x));
    return inverse ? make_float2(-c * (d.x + d.y), c * (d.x - d.y))
                   : make_float2(c * (d.y - d.x), -c * (d.x + d.y));
}

// In-register R-point DFT (sign -1, or +1 when inverse), natural order in and out:
// radix-2 decimation in frequency, then the bit-reversal permutation of registers.
template <int R>
__device__ __forceinline__ void dft_reg(float2 (&v)[8], bool inverse)
{
    if (R == 8) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const float2 a = v[r], b = v[r + 4];
            v[r] = cadd(a, b);
            const float2 d = csub(a, b);
            v[r + 4] = r == 0 ? d : (r == 1 ? rot8<1>(d, inverse)
                                            : (r == 2 ? rot8<2>(d, inverse) : rot8<3>(d, inverse)));
        }
    }
    if (R >= 4) {
#pragma unroll
        for (int h = 0; h < R; h += 4)
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const float2 a = v[h + r], b = v[h + r + 2];
                v[h + r] = cadd(a, b);
                const float2 d = csub(a, b);
                v[h + r + 2] = r == 0 ? d : rot8<2>(d, inverse);
            }
    }
#pragma unroll
    for (int h = 0; h < R; h += 2) {
        const float2 a = v[h], b = v[h + 1];
        v[h] = cadd(a, b);
        v[h + 1] = csub(a, b);
    }
    if (R == 8) {
        float2 t = v[1];  // output k sits at bit-reversed register brev3(k)
        v[1] = v[4];
        v[4] = t;
        t = v[3];
        v[3] = v[6];
        v[6] = t;
    } else if (R == 4) {
        const float2 t = v[1];
        v[1] = v[2];
        v[2] = t;
    }
}

// One pass over W lines (line stride ls) from src to dst; tw[i] = exp(-2 pi i i / M)
// for i < M / 2.
template <int LOG2R>
__device__ __forceinline__ void stockham_pass(const float2 *src, float2 *dst, int W, int log2m,
                                              int ls, int log2ns, bool inverse,
                                              const float2 *__restrict__ tw, int log2M)
{
    constexpr int R = 1 << LOG2R;
    const int lg = log2m - LOG2R;  // log2 of the groups per line
    const int G = W << lg;
    const int ns = 1 << log2ns;
    for (int q = threadIdx.x; q < G; q += blockDim.x) {
        const int t = q >> lg, j = q & ((1 << lg) - 1);
        const float2 *s = src + t * ls;
        float2 *d = dst + t * ls;
        const int k = j & (ns - 1);
        float2 v[8];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = s[spad(j + (r << lg))];
        if (log2ns > 0) {
            // exp(-2 pi i k r / (Ns R)) = exp(-2 pi i x / M), x = k r 2^sh < M; the table
            // holds the first half turn (M / 2 entries), and x + M / 2 is the negative
            const int sh = log2M - log2ns - LOG2R;
            const int half = 1 << (log2M - 1);
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const int x = (k * r) << sh;
                float2 w = __ldg(tw + (x & (half - 1)));
                if (x & half) {
                    w.x = -w.x;
                    w.y = -w.y;
                }
                if (inverse) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        dft_reg<R>(v, inverse);
        const int base = ((j - k) << LOG2R) + k;
#pragma unroll
        for (int r = 0; r < R; ++r) d[spad(base + (r << log2ns))] = v[r];
    }
}

// The whole transform of W lines held at a (natural order); returns the buffer (a
// or b) that holds the result, in natural order.
__device__ float2 *stockham(float2 *a, float2 *b, int W, int log2m, bool inverse,
                            const float2 *__restrict__ tw, int log2M)
{
    const int ls = stockham_ls(1 << log2m);
    int log2ns = 0;
    for (; log2ns + 3 <= log2m; log2ns += 3) {
        stockham_pass<3>(a, b, W, log2m, ls, log2ns, inverse, tw, log2M);
        __syncthreads();
        float2 *t = a;
        a = b;
        b = t;
    }
    if (log2m - log2ns == 2) {
        stockham_pass<2>(a, b, W, log2m, ls, log2ns, inverse, tw, log2M);
        __syncthreads();
        return b;
    }
    if (log2m - log2ns == 1) {
        stockham_pass<1>(a, b, W, log2m, ls, log2ns, inverse, tw, log2M);
        __syncthreads();
        return b;
    }
    return a;
}

// W lines along one axis of one grid.  Lines l in [0, inner * outer): inner index
// i = l % inner, outer index o = l / inner, element j at o * n * inner + i + j * inner
// (relative to the grid's first node).
struct LineJob {
    float2 *Z;             // the grid's complex work array
    const float *in_real;  // non-null: the input is this real array (first forward pass)
    float *out_real;       // non-null: write the real part here (last inverse pass)
    bool out_add;          // add the real part to out_real instead of storing it
    FftAxis ax;
    int64_t l0;            // first line
    int nl;                // lines of this job (<= W)
    int W;                 // lines per job (power of two, <= 32): shared-memory layout
    int mode;
    // scaling of the last axis: eigenvalues of the lower axes
    const float *lam0, *lam1;
    FastDiv div_n0;        // 3D: inner index i = k0 + n0 k1
    float inv_cells;
};

// 1 / (N K^2) for element k of the last axis of a line whose inner index is i.
__device__ __forceinline__ float spectral_scale(const LineJob &J, int k, int i)
{
    float K2 = J.ax.lam[k];
    if (J.lam0) {
        uint32_t k0 = (uint32_t)i;
        if (J.lam1) {
            const uint32_t k1 = fdiv((uint32_t)i, J.div_n0);
            k0 = (uint32_t)i - k1 * (uint32_t)J.div_n0.d;
            K2 += J.lam1[k1];
        }
        K2 += J.lam0[k0];
    }
    return K2 > 0.0f ? J.inv_cells / K2 : 0.0f;
}

// The transform of one job by the whole CTA (fsm: fft_smem_bytes(W, log2m)).
__device__ void fft_lines(const LineJob &J, const float2 *__restrict__ tw, int log2M, float2 *fsm)
{
    __shared__ int64_t s_base[32];  // first element of each of the job's lines
    __shared__ int s_inner[32];     // its inner index (the coordinates of the lower axes)
    const FftAxis &ax = J.ax;
    const int n = ax.n, log2m = ax.log2m, m = 1 << log2m, W = J.W, nl = J.nl;
    const SLayout S = slayout(log2m);
    float2 *buf = fsm;
    float2 *tws = fsm + (size_t)W * S.ls;
    // stage tables of the radix-2 path: entry h - 1 + k = exp(-2 pi i k / 2h) = tw[k M / 2h]
    for (int q = threadIdx.x; ax.bluestein && q < m - 1; q += blockDim.x) {
        const int s = 31 - __clz(q + 1), k = q + 1 - (1 << s);
        tws[q] = tw[(size_t)k << (log2M - 1 - s)];
    }
    const int64_t inner = ax.inner;
    if (threadIdx.x < nl) {
        const int64_t l = J.l0 + threadIdx.x;
        const int64_t o = l / inner, i = l - o * inner;
        s_base[threadIdx.x] = o * (int64_t)n * inner + i;
        s_inner[threadIdx.x] = (int)i;
    }
    __syncthreads();
    auto addr = [&](int t, int j) -> int64_t { return s_base[t] + (int64_t)j * inner; };
    // thread -> (line, element) so that consecutive threads touch consecutive addresses
    const bool rows = inner == 1;
    const int total = W * n;
    // (W is a power of two; so is n on the radix-2 path, where shifts replace the
    // divisions, which compile to slow float conversions on this GPU)
    const int log2W = 31 - __clz(W);
    const bool pow2 = n == m;
    auto coords = [&](int e, int *t, int *j) {
        if (rows) {
            *t = pow2 ? e >> log2m : e / n;
            *j = e - *t * n;
        } else {
            *t = e & (W - 1);
            *j = e >> log2W;
        }
    };
    const bool blue = ax.bluestein != 0;
    const bool inv_in = J.mode == FFT_INV;
    if (!blue) {
        // power of two: Stockham passes, natural order throughout
        const int lsS = stockham_ls(m);
        float2 *bufA = fsm, *bufB = fsm + (size_t)W * lsS;
        for (int e = threadIdx.x; e < total; e += blockDim.x) {
            int t, j;
            coords(e, &t, &j);
            if (t >= nl) continue;
            const int64_t a = addr(t, j);
            bufA[t * lsS + spad(j)] = J.in_real ? make_float2(J.in_real[a], 0.0f) : J.Z[a];
        }
        __syncthreads();
        float2 *res = stockham(bufA, bufB, W, log2m, inv_in, tw, log2M);
        if (J.mode == FFT_FWD_SCALE_INV) {
            for (int e = threadIdx.x; e < (W << log2m); e += blockDim.x) {
                const int t = e >> log2m, k = e & (m - 1);
                const float s = spectral_scale(J, k, s_inner[t < nl ? t : 0]);
                float2 &x = res[t * lsS + spad(k)];
                x.x *= s;
                x.y *= s;
            }
            __syncthreads();
            res = stockham(res, res == bufA ? bufB : bufA, W, log2m, true, tw, log2M);
        }
        for (int e = threadIdx.x; e < total; e += blockDim.x) {
            int t, j;
            coords(e, &t, &j);
            if (t >= nl) continue;
            const float2 v = res[t * lsS + spad(j)];
            const int64_t a = addr(t, j);
            if (J.out_real) {
                if (J.out_add) J.out_real[a] += v.x;
                else J.out_real[a] = v.x;
            } else {
                J.Z[a] = v;
            }
        }
        __syncthreads();  // the shared buffers are reused by the CTA's next job
        return;
    }
    // ---- load (scattered to bit-reversed positions, for the DIT) ----------------------------
    if (blue) {
        // zero the padding of Bluestein lines
        for (int e = threadIdx.x; e < W * S.ls; e += blockDim.x) buf[e] = make_float2(0.f, 0.f);
        __syncthreads();
    }
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        int t, j;
        coords(e, &t, &j);
        if (t >= nl) continue;
        const int64_t a = addr(t, j);
        float2 x = J.in_real ? make_float2(J.in_real[a], 0.0f) : J.Z[a];
        if (blue) {
            if (inv_in) x = cconj(x);
            x = cmul(x, ax.chirp[j]);
            buf[S.at(t, brev(j, log2m))] = x;
        } else if (inv_in) {
            buf[S.at(t, j)] = x;  // natural order for the DIF
        } else {
            buf[S.at(t, brev(j, log2m))] = x;
        }
    }
    __syncthreads();

    // ---- transform -----------------------------------------------------------------------------
    const float inv_m = 1.0f / (float)m;
    if (blue) {
        // forward DFT via the chirp-z convolution (an inverse is the conjugate of the
        // forward DFT of the conjugate input)
        dit(buf, W, S, tws, false);
        for (int e = threadIdx.x; e < (W << log2m); e += blockDim.x) {
            const int a = S.at(e >> log2m, e & (m - 1));
            buf[a] = cmul(buf[a], ax.bhat[e & (m - 1)]);
        }
        __syncthreads();
        dif(buf, W, S, tws, true);  // conv * m, bit-reversed
        if (J.mode == FFT_FWD_SCALE_INV) {
            // X_k = w_k c_k / m and Y_k = s_k X_k, then the inverse's input conj(Y_k) w_k,
            // all at position brev(k) of the line, which only this thread touches
            for (int e = threadIdx.x; e < (W << log2m); e += blockDim.x) {
                const int t = e >> log2m, p = e & (m - 1);
                const int k = brev(p, log2m);
                const int a = S.at(t, p);
                float2 v = make_float2(0.f, 0.f);
                if (k < n) {
                    const float2 w = ax.chirp[k];
                    float2 X = cmul(w, buf[a]);
                    const float s = inv_m * spectral_scale(J, k, s_inner[t < nl ? t : 0]);
                    X.x *= s;
                    X.y *= s;
                    v = cmul(cconj(X), w);
                }
                buf[a] = v;
            }
            __syncthreads();
            dit(buf, W, S, tws, false);
            for (int e = threadIdx.x; e < (W << log2m); e += blockDim.x) {
                const int a = S.at(e >> log2m, e & (m - 1));
                buf[a] = cmul(buf[a], ax.bhat[e & (m - 1)]);
            }
            __syncthreads();
            dif(buf, W, S, tws, true);
        }
    } else {
        if (J.mode == FFT_INV) {
            dif(buf, W, S, tws, true);  // bit-reversed result
        } else {
            dit(buf, W, S, tws, false);  // natural-order spectrum
            if (J.mode == FFT_FWD_SCALE_INV) {
                for (int e = threadIdx.x; e < (W << log2m); e += blockDim.x) {
                    const int t = e >> log2m, k = e & (m - 1);
                    const float s = spectral_scale(J, k, s_inner[t < nl ? t : 0]);
                    const int a = S.at(t, k);
                    buf[a].x *= s;
                    buf[a].y *= s;
                }
                __syncthreads();
                dif(buf, W, S, tws, true);
            }
        }
    }

    // ---- store ---------------------------------------------------------------------------------
    // natural order after a forward power-of-two pass; bit-reversed after a DIF
    const bool rev_out = blue || J.mode != FFT_FWD;
    const bool conj_out = blue && J.mode != FFT_FWD;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        int t, j;
        coords(e, &t, &j);
        if (t >= nl) continue;
        float2 v = buf[S.at(t, rev_out ? brev(j, log2m) : j)];
        if (blue) {
            v = cmul(ax.chirp[j], v);
            v.x *= inv_m;
            v.y *= inv_m;
            if (conj_out) v = cconj(v);
        }
        const int64_t a = addr(t, j);
        if (J.out_real) {
            if (J.out_add) J.out_real[a] += v.x;
            else J.out_real[a] = v.x;
        } else {
            J.Z[a] = v;
        }
    }
    __syncthreads();  // the shared buffers are reused by the CTA's next job
}

// One axis of one grid: CTA b takes lines [b W, b W + W).
__global__ void __launch_bounds__(FFT_THREADS) k_fft_axis(LineJob J, const float2 *__restrict__ tw,
                                                        int log2M, int64_t lines)
{
    extern __shared__ __align__(16) float2 fsm[];
    J.l0 = (int64_t)blockIdx.x * J.W;
    J.nl = (int)((lines - J.l0) < J.W ? (lines - J.l0) : J.W);
    fft_lines(J, tw, log2M, fsm);
}

// Many grids (a batch): CTAs walk a list of jobs, each W lines of one grid's axis.
__global__ void __launch_bounds__(FFT_THREADS)
    k_fft_jobs(const FftJob *__restrict__ jobs, int njobs, const FftGrid *__restrict__ grids,
               float2 *Z, const float *in_real, float *out_real, float *out_1d,
               const float2 *__restrict__ tw, int log2M, int mode)
{
    extern __shared__ __align__(16) float2 fsm[];
    for (int q = blockIdx.x; q < njobs; q += gridDim.x) {
        const FftJob jb = jobs[q];
        const FftGrid &G = grids[jb.grid];
        LineJob J;
        J.Z = Z + G.node0;
        J.in_real = in_real ? in_real + G.node0 : nullptr;
        float *out = G.ndim == 1 ? out_1d : out_real;
        J.out_real = out ? out + G.node0 : nullptr;
        J.out_add = false;
        J.ax = G.ax[jb.axis];
        J.l0 = jb.l0;
        J.nl = jb.nl;
        J.W = jb.W;
        J.mode = (G.ndim == 1) ? FFT_FWD_SCALE_INV : mode;
        J.lam0 = jb.axis >= 1 ? G.ax[0].lam : nullptr;
        J.lam1 = nullptr;
        J.div_n0 = G.div_n0;
        J.inv_cells = G.inv_cells;
        fft_lines(J, tw, log2M, fsm);
    }
}

// Host radix-2 FFT (double), used once per axis to build the Bluestein filter.
void host_fft(std::vector<std::complex<double>> &a)
{
    const size_t m = a.size();
    for (size_t i = 1, j = 0; i < m; ++i) {
        size_t bit = m >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(a[i], a[j]);
    }
    for (size_t len = 2; len <= m; len <<= 1) {
        const double ang = -2.0 * M_PI / (double)len;
        for (size_t i = 0; i < m; i += len)
            for (size_t k = 0; k < len / 2; ++k) {
                const std::complex<double> w(cos(ang * (double)k), sin(ang * (double)k));
                const std::complex<double> u = a[i + k], v = w * a[i + k + len / 2];
                a[i + k] = u + v;
                a[i + k + len / 2] = u - v;
            }
    }
}

int ilog2(int x)
{
    int l = 0;
    while ((1 << l) < x) ++l;
    return l;
}

}  // namespace

bool fft_length_ok(int n) { return n >= 1 && n <= FFT_MAX_N; }

int fft_log2m(int n) { return (n & (n - 1)) == 0 ? ilog2(n) : ilog2(2 * n - 1); }

size_t fft_axis_table_floats(int n)
{
    const bool pow2 = (n & (n - 1)) == 0;
    const int m = pow2 ? n : 1 << ilog2(2 * n - 1);
    // chirp (2n) + bhat (2m) floats (complex tables first, so they stay 8-byte
    // aligned), then lam (n), rounded up to an even count
    const size_t f = (pow2 ? 0 : 2 * (size_t)n + 2 * (size_t)m) + (size_t)n;
    return (f + 1) & ~(size_t)1;
}

// Fills the per-axis tables in host memory (`host` has fft_axis_table_floats(n)
// floats) and the axis descriptor with offsets relative to `dev` (the device copy).
void fft_axis_tables(int n, double dx, float *host, float *dev, FftAxis *ax)
{
    const bool pow2 = (n & (n - 1)) == 0;
    const int log2m = pow2 ? ilog2(n) : ilog2(2 * n - 1);
    const int m = 1 << log2m;
    ax->n = n;
    ax->log2m = log2m;
    ax->bluestein = pow2 ? 0 : 1;
    const size_t lam_at = pow2 ? 0 : 2 * (size_t)n + 2 * (size_t)m;
    float *lam = host + lam_at;
    for (int k = 0; k < n; ++k) {
        const double s = 2.0 * sin(M_PI * (double)k / (double)n) / dx;
        lam[k] = (float)(s * s);
    }
    ax->lam = dev + lam_at;
    ax->chirp = nullptr;
    ax->bhat = nullptr;
    if (pow2) return;
    float *chirp = host;
    float *bhat = chirp + 2 * (size_t)n;
    std::vector<std::complex<double>> w(n), b(m, 0.0);
    for (int j = 0; j < n; ++j) {
        // exp(-i pi j^2 / n), with j^2 reduced mod 2n so the angle stays exact
        const long long q = ((long long)j * j) % (2LL * n);
        const double ang = -M_PI * (double)q / (double)n;
        w[j] = std::complex<double>(cos(ang), sin(ang));
        chirp[2 * j] = (float)w[j].real();
        chirp[2 * j + 1] = (float)w[j].imag();
    }
    b[0] = std::conj(w[0]);
    for (int j = 1; j < n; ++j) b[j] = b[m - j] = std::conj(w[j]);
    host_fft(b);
    for (int k = 0; k < m; ++k) {
        bhat[2 * k] = (float)b[k].real();
        bhat[2 * k + 1] = (float)b[k].imag();
    }
    ax->chirp = reinterpret_cast<const float2 *>(dev);
    ax->bhat = reinterpret_cast<const float2 *>(dev + 2 * (size_t)n);
}

size_t fft_twiddle_floats(int log2M) { return (size_t)1 << log2M; }  // M / 2 complex

void fft_twiddles(int log2M, float *host)
{
    const int M = 1 << log2M;
    for (int t = 0; t < M / 2; ++t) {
        const double ang = -2.0 * M_PI * (double)t / (double)M;
        host[2 * t] = (float)cos(ang);
        host[2 * t + 1] = (float)sin(ang);
    }
}

// Lines per job: enough jobs to fill the GPU twice when the axis allows, at most
// 32 lines and `cap` elements of shared memory.
int lines_per_cta(int64_t lines, int log2m, int sms, int cap)
{
    int W = 32;
    while (W > 1 && (((int64_t)W << log2m) > cap || lines / W < 2 * (int64_t)sms)) W >>= 1;
    return W;
}

size_t fft_smem_bytes(int W, int log2m, bool bluestein)
{
    const size_t m = (size_t)1 << log2m;
    // Bluestein lines (radix-2 stages): W padded lines, then m - 1 stage twiddles
    if (bluestein) return ((size_t)W * (m + (log2m >= 5 ? 32 : 0)) + m) * sizeof(float2);
    // power-of-two lines (Stockham passes): two buffers of W padded lines
    return 2 * (size_t)W * (size_t)stockham_ls((int)m) * sizeof(float2);
}

cudaError_t fft_configure()
{
    // the larger of W * m <= 8192 elements (+ 32 padding slots per line, W <= 32) plus
    // m <= 8192 stage twiddles, and two Stockham buffers of 8192 + 1024 elements
    const int most = (int)(2 * (8192 + 1024) * sizeof(float2));
    cudaError_t e = cudaFuncSetAttribute(k_fft_axis, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         most);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_fft_jobs, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
}

cudaError_t launch_fft_poisson(const FftPlan &P, const float *b, float *phi, cudaStream_t st,
                               bool accumulate)
{
    const int d = P.ndim;
    auto run = [&](int a, int mode, const float *in, float *out) -> cudaError_t {
        LineJob J{};
        J.Z = P.Z;
        J.in_real = in;
        J.out_real = out;
        J.out_add = accumulate && out != nullptr;
        J.ax = P.ax[a];
        const int64_t lines = P.cells / J.ax.n;
        J.W = lines_per_cta(lines, J.ax.log2m, P.sms, 2048);
        J.mode = mode;
        J.lam0 = a >= 1 ? P.ax[0].lam : nullptr;
        J.lam1 = a >= 2 ? P.ax[1].lam : nullptr;
        J.div_n0 = make_fastdiv((uint32_t)P.ax[0].n);
        J.inv_cells = (float)(1.0 / (double)P.cells);
        const int64_t grid = (lines + J.W - 1) / J.W;
        k_fft_axis<<<(unsigned)grid, FFT_THREADS,
                     fft_smem_bytes(J.W, J.ax.log2m, J.ax.bluestein != 0), st>>>(
            J, P.tw, P.log2M, lines);
        note_launch();
        return cudaGetLastError();
    };
    cudaError_t e;
    if (d == 1) return run(0, FFT_FWD_SCALE_INV, b, phi);
    if ((e = run(0, FFT_FWD, b, nullptr)) != cudaSuccess) return e;
    for (int a = 1; a < d - 1; ++a)
        if ((e = run(a, FFT_FWD, nullptr, nullptr)) != cudaSuccess) return e;
    if ((e = run(d - 1, FFT_FWD_SCALE_INV, nullptr, nullptr)) != cudaSuccess) return e;
    for (int a = d - 2; a >= 1; --a)
        if ((e = run(a, FFT_INV, nullptr, nullptr)) != cudaSuccess) return e;
    return run(0, FFT_INV, nullptr, phi);
}

cudaError_t launch_fft_jobs(const FftJob *jobs, int njobs, const FftGrid *grids, float2 *Z,
                            const float *in_real, float *out_real, float *out_1d,
                            const float2 *tw, int log2M, int mode, size_t smem, int blocks,
                            cudaStream_t st)
{
    if (njobs == 0) return cudaSuccess;
    k_fft_jobs<<<blocks < njobs ? blocks : njobs, FFT_THREADS, smem, st>>>(
        jobs, njobs, grids, Z, in_real, out_real, out_1d, tw, log2M, mode);
    note_launch();
    return cudaGetLastError();
}

}  // namespace apk
