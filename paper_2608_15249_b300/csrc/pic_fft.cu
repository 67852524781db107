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
//   - power-of-two lengths: radix-2 decimation in time (input scattered to
//     bit-reversed positions, natural-order output) for the forward transform and
//     decimation in frequency (natural input, bit-reversed output) for the inverse,
//     so no separate reordering pass is needed;
//   - other lengths: Bluestein's chirp-z form, X_k = w_k sum_j (x_j w_j) conj(w_{k-j})
//     with w_j = exp(-i pi j^2 / n), a cyclic convolution of power-of-two length
//     m >= 2n - 1 done with the same two transforms and a precomputed filter.
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

// W lines of length m in shared memory (line t at buf + t * m), input in
// bit-reversed order -> DFT (sign -1, or +1 when inverse) in natural order.
// tws[t] = exp(-2 pi i t / m), t < m / 2.
__device__ void dit(float2 *buf, int W, int log2m, const float2 *tws, bool inverse)
{
    const int half = 1 << (log2m - 1);
    const int nb = W * half;
    for (int s = 0; s < log2m; ++s) {
        const int h = 1 << s;
        for (int b = threadIdx.x; b < nb; b += blockDim.x) {
            const int t = b >> (log2m - 1);
            const int bb = b & (half - 1);
            const int k = bb & (h - 1);
            const int i0 = ((bb >> s) << (s + 1)) + k;
            float2 *L = buf + ((size_t)t << log2m);
            float2 w = tws[k << (log2m - 1 - s)];
            if (inverse) w.y = -w.y;
            const float2 u = L[i0], v = cmul(w, L[i0 + h]);
            L[i0] = cadd(u, v);
            L[i0 + h] = csub(u, v);
        }
        __syncthreads();
    }
}

// Natural-order input -> DFT in bit-reversed order (decimation in frequency).
__device__ void dif(float2 *buf, int W, int log2m, const float2 *tws, bool inverse)
{
    const int half = 1 << (log2m - 1);
    const int nb = W * half;
    for (int s = log2m - 1; s >= 0; --s) {
        const int h = 1 << s;
        for (int b = threadIdx.x; b < nb; b += blockDim.x) {
            const int t = b >> (log2m - 1);
            const int bb = b & (half - 1);
            const int k = bb & (h - 1);
            const int i0 = ((bb >> s) << (s + 1)) + k;
            float2 *L = buf + ((size_t)t << log2m);
            float2 w = tws[k << (log2m - 1 - s)];
            if (inverse) w.y = -w.y;
            const float2 u = L[i0], v = L[i0 + h];
            L[i0] = cadd(u, v);
            L[i0 + h] = cmul(csub(u, v), w);
        }
        __syncthreads();
    }
}

enum : int { FFT_FWD = 0, FFT_INV = 1, FFT_FWD_SCALE_INV = 2 };

// One axis of the transform.  Lines l in [0, inner * outer): inner index i = l % inner,
// outer index o = l / inner, element j at o * n * inner + i + j * inner.
struct AxisArgs {
    FftAxis ax;
    const float2 *tw;    // exp(-2 pi i t / M), t < M / 2
    int log2M;
    int W;               // lines per CTA (power of two)
    int64_t lines;
    int mode;
    const float *in_real;  // non-null: the input is this real array (first forward pass)
    float *out_real;       // non-null: write Re * 1 into this array (last inverse pass)
    // scaling of the last axis: eigenvalues of the lower axes and their sizes
    const float *lam0, *lam1;
    FastDiv div_n0;        // coordinates of the inner index (3D: i = k0 + n0 k1)
    float inv_cells;
};

__global__ void __launch_bounds__(FFT_THREADS) k_fft_axis(float2 *__restrict__ Z, AxisArgs A)
{
    extern __shared__ __align__(16) float2 fsm[];
    __shared__ int64_t s_base[32];  // first element of each of the CTA's lines
    __shared__ int s_inner[32];     // its inner index (the coordinates of the lower axes)
    const FftAxis &ax = A.ax;
    const int n = ax.n, log2m = ax.log2m, m = 1 << log2m, W = A.W;
    float2 *buf = fsm;
    float2 *tws = fsm + ((size_t)W << log2m);
    for (int t = threadIdx.x; t < m / 2; t += blockDim.x) tws[t] = A.tw[(size_t)t << (A.log2M - log2m)];
    const int64_t l0 = (int64_t)blockIdx.x * W;
    const int nl = (int)((A.lines - l0) < W ? (A.lines - l0) : W);
    const int64_t inner = ax.inner;
    if (threadIdx.x < nl) {
        const int64_t l = l0 + threadIdx.x;
        const int64_t o = l / inner, i = l - o * inner;
        s_base[threadIdx.x] = o * (int64_t)n * inner + i;
        s_inner[threadIdx.x] = (int)i;
    }
    __syncthreads();
    auto addr = [&](int t, int j) -> int64_t { return s_base[t] + (int64_t)j * inner; };
    // thread -> (line, element) so that consecutive threads touch consecutive addresses
    const bool rows = inner == 1;
    const int total = W * n;
    auto coords = [&](int e, int *t, int *j) {
        if (rows) {
            *t = e / n;
            *j = e - *t * n;
        } else {
            *t = e & (W - 1);
            *j = e / W;
        }
    };
    const bool blue = ax.bluestein != 0;
    const bool inv_in = A.mode == FFT_INV;
    // ---- load (scattered to bit-reversed positions, for the DIT) ----------------------------
    if (blue) {
        // zero the padding of Bluestein lines
        for (int e = threadIdx.x; e < (W << log2m); e += blockDim.x) buf[e] = make_float2(0.f, 0.f);
        __syncthreads();
    }
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        int t, j;
        coords(e, &t, &j);
        if (t >= nl) continue;
        const int64_t a = addr(t, j);
        float2 x = A.in_real ? make_float2(A.in_real[a], 0.0f) : Z[a];
        if (blue) {
            if (inv_in) x = cconj(x);
            x = cmul(x, ax.chirp[j]);
            buf[((size_t)t << log2m) + brev(j, log2m)] = x;
        } else if (inv_in) {
            buf[((size_t)t << log2m) + j] = x;  // natural order for the DIF
        } else {
            buf[((size_t)t << log2m) + brev(j, log2m)] = x;
        }
    }
    __syncthreads();

    // ---- transform -----------------------------------------------------------------------------
    // After this block, line t holds its result at position pos(j) (natural or
    // bit-reversed), with a per-element factor applied on the way out.
    const float inv_m = 1.0f / (float)m;
    if (blue) {
        // forward DFT via the chirp-z convolution (an inverse is the conjugate of the
        // forward DFT of the conjugate input)
        dit(buf, W, log2m, tws, false);
        for (int e = threadIdx.x; e < (W << log2m); e += blockDim.x)
            buf[e] = cmul(buf[e], ax.bhat[e & (m - 1)]);
        __syncthreads();
        dif(buf, W, log2m, tws, true);  // conv * m, bit-reversed
        if (A.mode == FFT_FWD_SCALE_INV) {
            // X_k = w_k c_k / m; Y_k = s_k X_k; then the inverse input conj(Y_k) w_k in place
            for (int e = threadIdx.x; e < (W << log2m); e += blockDim.x) {
                const int t = e >> log2m, p = e & (m - 1);
                const int k = brev(p, log2m);
                float2 v = make_float2(0.f, 0.f);
                if (k < n) {
                    const float2 w = ax.chirp[k];
                    float2 X = cmul(w, buf[e]);
                    X.x *= inv_m;
                    X.y *= inv_m;
                    // element (t, k): its coordinates in the lower axes come from the line
                    const int i = s_inner[t < nl ? t : 0];
                    float K2 = ax.lam[k];
                    if (A.lam0) {
                        uint32_t k1 = 0, k0 = (uint32_t)i;
                        if (A.lam1) {
                            k1 = fdiv((uint32_t)i, A.div_n0);
                            k0 = (uint32_t)i - k1 * (uint32_t)A.div_n0.d;
                            K2 += A.lam1[k1];
                        }
                        K2 += A.lam0[k0];
                    }
                    const float s = K2 > 0.0f ? A.inv_cells / K2 : 0.0f;
                    X.x *= s;
                    X.y *= s;
                    v = cmul(cconj(X), w);
                }
                // position p of line t was read only by this thread; write it back
                buf[e] = make_float2(0.f, 0.f);
                if (k < n) buf[((size_t)t << log2m) + brev(k, log2m)] = v;
            }
            __syncthreads();
            dit(buf, W, log2m, tws, false);
            for (int e = threadIdx.x; e < (W << log2m); e += blockDim.x)
                buf[e] = cmul(buf[e], ax.bhat[e & (m - 1)]);
            __syncthreads();
            dif(buf, W, log2m, tws, true);
        }
    } else {
        if (A.mode == FFT_INV) {
            dif(buf, W, log2m, tws, true);  // bit-reversed result
        } else {
            dit(buf, W, log2m, tws, false);  // natural-order spectrum
            if (A.mode == FFT_FWD_SCALE_INV) {
                for (int e = threadIdx.x; e < (W << log2m); e += blockDim.x) {
                    const int t = e >> log2m, k = e & (m - 1);
                    const int i = s_inner[t < nl ? t : 0];
                    float K2 = ax.lam[k];
                    if (A.lam0) {
                        uint32_t k1 = 0, k0 = (uint32_t)i;
                        if (A.lam1) {
                            k1 = fdiv((uint32_t)i, A.div_n0);
                            k0 = (uint32_t)i - k1 * (uint32_t)A.div_n0.d;
                            K2 += A.lam1[k1];
                        }
                        K2 += A.lam0[k0];
                    }
                    const float s = K2 > 0.0f ? A.inv_cells / K2 : 0.0f;
                    buf[e].x *= s;
                    buf[e].y *= s;
                }
                __syncthreads();
                dif(buf, W, log2m, tws, true);
            }
        }
    }

    // ---- store ---------------------------------------------------------------------------------
    // natural order after a forward power-of-two pass; bit-reversed after a DIF
    const bool rev_out = blue || A.mode != FFT_FWD;
    const bool conj_out = blue && A.mode != FFT_FWD;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        int t, j;
        coords(e, &t, &j);
        if (t >= nl) continue;
        const size_t p = ((size_t)t << log2m) + (rev_out ? brev(j, log2m) : j);
        float2 v = buf[p];
        if (blue) {
            v = cmul(ax.chirp[j], v);
            v.x *= inv_m;
            v.y *= inv_m;
            if (conj_out) v = cconj(v);
        }
        const int64_t a = addr(t, j);
        if (A.out_real) A.out_real[a] = v.x;
        else Z[a] = v;
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

// Lines per CTA: enough CTAs to fill the GPU twice when the axis allows, at most
// 32 lines and 8192 elements of shared memory.
static int lines_per_cta(int64_t lines, int log2m, int sms)
{
    int W = 32;
    while (W > 1 && (((int64_t)W << log2m) > 8192 || lines / W < 2 * (int64_t)sms)) W >>= 1;
    return W;
}

static size_t axis_smem(int W, int log2m)
{
    return (((size_t)W << log2m) + ((size_t)1 << (log2m - 1))) * sizeof(float2);
}

cudaError_t fft_configure()
{
    // W * m <= 8192 elements plus m / 2 twiddles
    return cudaFuncSetAttribute(k_fft_axis, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)((8192 + 4096) * sizeof(float2)));
}

cudaError_t launch_fft_poisson(const FftPlan &P, const float *b, float *phi, cudaStream_t st)
{
    const int d = P.ndim;
    auto run = [&](int a, int mode, const float *in, float *out) -> cudaError_t {
        AxisArgs A{};
        A.ax = P.ax[a];
        A.tw = P.tw;
        A.log2M = P.log2M;
        A.lines = P.cells / A.ax.n;
        A.W = lines_per_cta(A.lines, A.ax.log2m, P.sms);
        A.mode = mode;
        A.in_real = in;
        A.out_real = out;
        A.lam0 = a >= 1 ? P.ax[0].lam : nullptr;
        A.lam1 = a >= 2 ? P.ax[1].lam : nullptr;
        A.div_n0 = make_fastdiv((uint32_t)P.ax[0].n);
        A.inv_cells = (float)(1.0 / (double)P.cells);
        const int64_t grid = (A.lines + A.W - 1) / A.W;
        k_fft_axis<<<(unsigned)grid, FFT_THREADS, axis_smem(A.W, A.ax.log2m), st>>>(P.Z, A);
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

}  // namespace apk
