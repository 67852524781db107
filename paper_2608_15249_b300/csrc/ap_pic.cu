// ap_pic.cu -- host side of the C ABI declared in include/ap_pic.h: instance
// state, device memory, and the order of the cycle of the paper's worked
// example (Sec. 3.1, Listing 1).
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <string>
#include <vector>

#include "ap_pic.h"
#include "pic_internal.cuh"

using namespace apk;

namespace {
std::atomic<long long> g_launches{0};
}

void apk::note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

namespace {

constexpr int DEFAULT_FX_BITS = 22;   // FP32 cell+offset form: near the FP32 weights' precision
constexpr int MAX_FX_BITS_F32 = 22;   // the FMA rounding idiom is exact up to 2^22
constexpr int DEFAULT_FX_BITS_F64 = 40;  // FP64 plain form: FP64 weights
constexpr int MAX_FX_BITS_F64 = 52;
constexpr double DEFAULT_CG_RTOL_F64 = 1e-10;
constexpr double DEFAULT_CG_RTOL = 1e-6;
constexpr int DEFAULT_CG_MAXIT = 20000;
constexpr int64_t LOAD_CHUNK = int64_t(1) << 23;  // particles per host->device load chunk

int bitlen(uint64_t x)
{
    int b = 0;
    while (x) {
        ++b;
        x >>= 1;
    }
    return b;
}

}  // namespace

struct ap_pic {
    ap_pic_config cfg;
    ap_pic_allocator alloc;
    bool has_alloc = false;
    cudaStream_t stream = nullptr;
    std::string err;
    std::vector<std::pair<void *, size_t>> owned;

    int ndim = 1, nv = 1;
    int64_t cells = 0;
    int64_t np = 0;
    int fx_bits = DEFAULT_FX_BITS;
    int brick[3] = {1, 1, 1};
    int key_bits = 0;
    double dV = 1.0, V = 1.0;
    int64_t step = 0;
    bool loaded = false;

    bool plain = false;            // AP_PIC_FP64_PLAIN
    ParticlesF64 p64{};
    FieldBufsF64 f64{};

    // particles (FP32 cell + offset form)
    ParticlesF32 p{};
    ParticlesF32 p_alt{};
    SortScratch sort{};
    int perm_slot = -1;

    // grid
    FieldBufs f{};
    DiagPartials dpart{};
    double *d_diag = nullptr;      // [8]
    long long *d_accsum = nullptr; // [1]
    int *d_err = nullptr;

    // pinned host mirrors
    int *h_done = nullptr;
    double *h_diag = nullptr;
    long long *h_accsum = nullptr;
    int *h_err = nullptr;
    int *h_iters = nullptr;

    // step graphs: with the spectral solve a step has no host decision, so each
    // (buffer parity, diagnostics, sort) variant is captured once and replayed on an
    // own non-blocking stream fenced to the caller's
    cudaStream_t gstream = nullptr;
    cudaEvent_t gev_in = nullptr, gev_out = nullptr;
    cudaGraphExec_t graphs[16] = {};
    int64_t graph_launches[16] = {};
    int graph_slot[16] = {};
    int parity = 0;  // flips with every sort (the ping-pong particle buffers)
    int acc_parity = 0;  // flips with every FP32 push_deposit (the two accumulators)

    // electromagnetic step (cfg.em)
    bool em = false;
    bool em_np = false;  // particles in the non-periodic mode (absorbing layer, walls)
    int64_t absorbed_total = 0;  // particles absorbed at the walls and dropped so far
    unsigned long long *d_absorbed = nullptr;  // particles absorbed since the last sort
    EmBufs emb{};
    float *jext = nullptr;  // storage of the prescribed current

    // null-collision Monte Carlo (ap_pic_set_collisions)
    bool mcc_on = false;
    MccParams mccp{};
    unsigned long long *d_mcc = nullptr;  // [3] counts of the last collision pass

    // spectral field solve (AP_PIC_SOLVER_FFT)
    bool use_fft = false;
    FftPlan fft{};
    bool relres_on_device = false;  // last_cg_relres is in f.scal[SCAL_TRUE_REL]
    bool cg_on_device = false;      // last CG iterations / residual are in f.iters, f.scal

    int last_cg_iters = 0;
    double last_cg_relres = 0.0;
    bool diag_valid = false;

    // stage timing: event pairs recorded on the stream, summed on request
    bool timing = false;
    struct Mark {
        int stage;
        cudaEvent_t a, b;
    };
    std::vector<Mark> marks;
    double stage_ms[AP_PIC_NSTAGES] = {0};
    int64_t stage_n[AP_PIC_NSTAGES] = {0};
};

// Records the start of a timed stage; returns the index of its mark (-1 when off).
static int stage_begin(ap_pic *h, int stage)
{
    if (!h->timing) return -1;
    ap_pic::Mark m{stage, nullptr, nullptr};
    if (cudaEventCreate(&m.a) != cudaSuccess || cudaEventCreate(&m.b) != cudaSuccess) return -1;
    cudaEventRecord(m.a, h->stream);
    h->marks.push_back(m);
    return (int)h->marks.size() - 1;
}

static void stage_end(ap_pic *h, int mark)
{
    if (mark < 0) return;
    cudaEventRecord(h->marks[(size_t)mark].b, h->stream);
}

static void drain_marks(ap_pic *h)
{
    if (h->marks.empty()) return;
    cudaStreamSynchronize(h->stream);
    for (auto &m : h->marks) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, m.a, m.b) == cudaSuccess) {
            h->stage_ms[m.stage] += ms;
            h->stage_n[m.stage] += 1;
        }
        cudaEventDestroy(m.a);
        cudaEventDestroy(m.b);
    }
    h->marks.clear();
}

// ---- small helpers ---------------------------------------------------------------------------

static ap_pic_status fail(ap_pic *h, ap_pic_status st, const char *fmt, ...)
{
    if (h) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        h->err = buf;
    }
    return st;
}

#define CU(h, call)                                                                            \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail((h), AP_PIC_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                                   \
    } while (0)

#define TRY(expr)                                                                              \
    do {                                                                                       \
        ap_pic_status s_ = (expr);                                                             \
        if (s_ != AP_PIC_OK) return s_;                                                        \
    } while (0)

static void *dev_alloc(ap_pic *h, size_t bytes)
{
    if (bytes == 0) bytes = 256;
    void *ptr = nullptr;
    if (h->has_alloc) {
        ptr = h->alloc.alloc(bytes, h->alloc.ctx);
    } else if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
        cudaGetLastError();
        ptr = nullptr;
    }
    if (ptr) h->owned.push_back({ptr, bytes});
    return ptr;
}

static void dev_free(ap_pic *h, void *ptr)
{
    if (!ptr) return;
    for (size_t i = 0; i < h->owned.size(); ++i) {
        if (h->owned[i].first == ptr) {
            const size_t bytes = h->owned[i].second;
            if (h->has_alloc) h->alloc.free(ptr, bytes, h->alloc.ctx);
            else cudaFree(ptr);
            h->owned.erase(h->owned.begin() + (long)i);
            return;
        }
    }
}

template <typename T>
static ap_pic_status alloc_n(ap_pic *h, T **out, size_t count)
{
    *out = static_cast<T *>(dev_alloc(h, count * sizeof(T)));
    if (!*out)
        return fail(h, AP_PIC_ERR_NOMEM, "device allocation of %zu bytes failed",
                    count * sizeof(T));
    return AP_PIC_OK;
}

static GridParams grid_params(const ap_pic *h, double step_h)
{
    GridParams g{};
    const ap_pic_config &c = h->cfg;
    g.ndim = h->ndim;
    for (int a = 0; a < 3; ++a) {
        g.n[a] = a < h->ndim ? c.n[a] : 1;
        g.dtdx[a] = a < h->ndim ? (float)(c.dt / c.dx[a]) : 0.0f;
        g.E0[a] = (float)c.E0[a];
    }
    const double qm = c.q / c.m;
    g.qmh2 = (float)(qm * step_h * 0.5);
    double t[3], tt = 0.0;
    for (int a = 0; a < 3; ++a) {
        t[a] = qm * c.B0[a] * step_h * 0.5;
        tt += t[a] * t[a];
    }
    for (int a = 0; a < 3; ++a) {
        g.t[a] = (float)t[a];
        g.s[a] = (float)(2.0 * t[a] / (1.0 + tt));
    }
    g.magnetised = (c.B0[0] != 0.0 || c.B0[1] != 0.0 || c.B0[2] != 0.0) ? 1 : 0;
    g.fx_bits = h->fx_bits;
    g.div0 = make_fastdiv((uint32_t)g.n[0]);
    g.div1 = make_fastdiv((uint32_t)g.n[1]);
    g.pusher = c.pusher;
    g.inv_c2 = c.c_light > 0.0 ? (float)(1.0 / (c.c_light * c.c_light)) : 0.0f;
    return g;
}

static GridParamsF64 grid_params_f64(const ap_pic *h, double step_h)
{
    GridParamsF64 g{};
    const ap_pic_config &c = h->cfg;
    g.ndim = h->ndim;
    for (int a = 0; a < 3; ++a) {
        g.n[a] = a < h->ndim ? c.n[a] : 1;
        g.dx[a] = c.dx[a];
        g.inv_dx[a] = 1.0 / c.dx[a];
        g.L[a] = g.n[a] * c.dx[a];
        g.E0[a] = c.E0[a];
    }
    g.dt = c.dt;
    const double qm = c.q / c.m;
    g.qmh2 = qm * step_h * 0.5;
    double tt = 0.0;
    for (int a = 0; a < 3; ++a) {
        g.t[a] = qm * c.B0[a] * step_h * 0.5;
        tt += g.t[a] * g.t[a];
    }
    for (int a = 0; a < 3; ++a) g.s[a] = 2.0 * g.t[a] / (1.0 + tt);
    g.magnetised = (c.B0[0] != 0.0 || c.B0[1] != 0.0 || c.B0[2] != 0.0) ? 1 : 0;
    g.fx_bits = h->fx_bits;
    return g;
}

// Reads the latched device error word (synchronises the stream).
static ap_pic_status sync_check(ap_pic *h)
{
    CU(h, cudaMemcpyAsync(h->h_err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
    const int e = *h->h_err;
    if (e & EF_NONFINITE)
        return fail(h, AP_PIC_ERR_BOUNDS,
                    "a particle position or velocity was not finite or outside the box");
    if (e & EF_OVERFLOW) return fail(h, AP_PIC_ERR_BOUNDS, "fixed-point charge overflow");
    if (e & EF_TIMEOUT)
        return fail(h, AP_PIC_ERR_CUDA, "a device wait hit its iteration cap; results are partial");
    if (e & EF_CG)
        return fail(h, AP_PIC_ERR_NOT_CONVERGED, "field solve stopped at cg_maxit = %d",
                    h->cfg.cg_maxit);
    return AP_PIC_OK;
}

// ---- configuration ---------------------------------------------------------------------------

extern "C" void ap_pic_config_default(ap_pic_config *c)
{
    if (!c) return;
    memset(c, 0, sizeof *c);
    c->ndim = 1;
    c->n[0] = 64;
    c->n[1] = c->n[2] = 1;
    c->dx[0] = c->dx[1] = c->dx[2] = 1.0;
    c->dt = 0.1;
    c->q = -1.0;
    c->m = 1.0;
    c->weight = 1.0;
    c->rho_background = NAN;
    c->bc = AP_PIC_BC_PERIODIC;
    c->precision = AP_PIC_FP32_CELLOFF;
    c->nv = 1;
    c->sort_every = 20;
    c->fx_bits = DEFAULT_FX_BITS;
    c->cg_rtol = DEFAULT_CG_RTOL;
    c->cg_maxit = DEFAULT_CG_MAXIT;
}

static ap_pic_status validate(ap_pic *h, ap_pic_config *c)
{
    if (c->ndim < 1 || c->ndim > 3) return fail(h, AP_PIC_ERR_ARG, "ndim must be 1, 2 or 3");
    int64_t cells = 1;
    for (int a = 0; a < c->ndim; ++a) {
        if (c->n[a] < 2) return fail(h, AP_PIC_ERR_ARG, "n[%d] must be >= 2", a);
        if (!(c->dx[a] > 0.0) || !isfinite(c->dx[a]))
            return fail(h, AP_PIC_ERR_ARG, "dx[%d] must be positive and finite", a);
        cells *= c->n[a];
    }
    if (cells > (int64_t(1) << 30))
        return fail(h, AP_PIC_ERR_ARG, "grid of %lld nodes exceeds 2^30", (long long)cells);
    for (int a = c->ndim; a < 3; ++a) {
        c->n[a] = 1;
        if (!(c->dx[a] > 0.0)) c->dx[a] = 1.0;
    }
    if (!(c->dt > 0.0) || !isfinite(c->dt)) return fail(h, AP_PIC_ERR_ARG, "dt must be > 0");
    if (!(c->m > 0.0) || !isfinite(c->q)) return fail(h, AP_PIC_ERR_ARG, "need m > 0, finite q");
    if (!(c->weight > 0.0)) return fail(h, AP_PIC_ERR_ARG, "weight must be > 0");
    if (c->bc != AP_PIC_BC_PERIODIC)
        return fail(h, AP_PIC_ERR_UNSUPPORTED, "only periodic boundaries are implemented");
    if (c->precision != AP_PIC_FP32_CELLOFF && c->precision != AP_PIC_FP64_PLAIN)
        return fail(h, AP_PIC_ERR_ARG, "unknown precision %d", c->precision);
    if (c->nv < c->ndim || c->nv > 3) return fail(h, AP_PIC_ERR_ARG, "need ndim <= nv <= 3");
    const bool mag = c->B0[0] != 0.0 || c->B0[1] != 0.0 || c->B0[2] != 0.0;
    if (mag && c->nv != 3) return fail(h, AP_PIC_ERR_ARG, "B0 != 0 needs nv = 3");
    for (int a = 0; a < 3; ++a)
        if (!isfinite(c->E0[a]) || !isfinite(c->B0[a]))
            return fail(h, AP_PIC_ERR_ARG, "E0 and B0 must be finite");
    if (c->sort_every < 0) return fail(h, AP_PIC_ERR_ARG, "sort_every must be >= 0");
    const bool plain = c->precision == AP_PIC_FP64_PLAIN;
    if (c->fx_bits == 0) c->fx_bits = plain ? DEFAULT_FX_BITS_F64 : DEFAULT_FX_BITS;
    const int fx_max = plain ? MAX_FX_BITS_F64 : MAX_FX_BITS_F32;
    if (c->fx_bits < 8 || c->fx_bits > fx_max)
        return fail(h, AP_PIC_ERR_ARG, "fx_bits must be in [8, %d] for this form", fx_max);
    if (c->cg_rtol == 0.0) c->cg_rtol = plain ? DEFAULT_CG_RTOL_F64 : DEFAULT_CG_RTOL;
    if (!(c->cg_rtol > 0.0)) return fail(h, AP_PIC_ERR_ARG, "cg_rtol must be > 0");
    if (c->cg_maxit == 0) c->cg_maxit = DEFAULT_CG_MAXIT;
    if (c->cg_maxit < 1) return fail(h, AP_PIC_ERR_ARG, "cg_maxit must be >= 1");
    if (c->diag_every < 0) return fail(h, AP_PIC_ERR_ARG, "diag_every must be >= 0");
    if (c->pusher != AP_PIC_PUSHER_BORIS && c->pusher != AP_PIC_PUSHER_HIGUERA_CARY)
        return fail(h, AP_PIC_ERR_ARG, "unknown pusher %d", c->pusher);
    if (!(c->c_light >= 0.0) || !isfinite(c->c_light))
        return fail(h, AP_PIC_ERR_ARG, "c_light must be >= 0 and finite (0: infinite)");
    if (c->pusher == AP_PIC_PUSHER_HIGUERA_CARY && plain)
        return fail(h, AP_PIC_ERR_UNSUPPORTED, "the FP64 plain form pushes with Boris only");
    if (c->solver != AP_PIC_SOLVER_CG && c->solver != AP_PIC_SOLVER_FFT)
        return fail(h, AP_PIC_ERR_ARG, "unknown solver %d", c->solver);
    if (c->em != 0 && c->em != 1) return fail(h, AP_PIC_ERR_ARG, "em must be 0 or 1");
    if (c->em) {
        if (c->ndim < 2 || c->nv != 3 || plain)
            return fail(h, AP_PIC_ERR_UNSUPPORTED,
                        "the electromagnetic step needs ndim = 2 or 3, nv = 3 and the FP32 form");
        if (c->pusher != AP_PIC_PUSHER_BORIS)
            return fail(h, AP_PIC_ERR_UNSUPPORTED, "the electromagnetic step pushes with Boris");
        if (!(c->c_light > 0.0))
            return fail(h, AP_PIC_ERR_ARG, "the electromagnetic step needs c_light > 0");
        double idx2 = 0.0;
        for (int a = 0; a < c->ndim; ++a) idx2 += 1.0 / (c->dx[a] * c->dx[a]);
        const double courant = c->c_light * c->dt * sqrt(idx2);
        if (!(courant < 1.0))
            return fail(h, AP_PIC_ERR_ARG, "Courant number c dt sqrt(sum 1/dx^2) = %.3f >= 1",
                        courant);
    }
    if (c->em_boundary != 0 && c->em_boundary != 1)
        return fail(h, AP_PIC_ERR_ARG, "em_boundary must be 0 or 1");
    if (c->em_boundary == 1) {
        if (!c->em) return fail(h, AP_PIC_ERR_ARG, "the absorbing layer needs em = 1");
        if (c->ndim != 2)
            return fail(h, AP_PIC_ERR_UNSUPPORTED, "the absorbing layer is built for 2D grids");
        if (c->pml_cells == 0) c->pml_cells = 12;
        if (c->pml_cells < 1 || 2 * c->pml_cells >= c->n[0] || 2 * c->pml_cells >= c->n[1])
            return fail(h, AP_PIC_ERR_ARG, "need 1 <= pml_cells and 2 pml_cells < n");
    }
    if (c->solver == AP_PIC_SOLVER_FFT) {
        if (plain)
            return fail(h, AP_PIC_ERR_UNSUPPORTED, "the FP64 plain form solves with the CG only");
        for (int a = 0; a < c->ndim; ++a)
            if (!fft_length_ok(c->n[a]))
                return fail(h, AP_PIC_ERR_UNSUPPORTED, "FFT solver needs n[%d] <= %d", a,
                            FFT_MAX_N);
    }
    if (c->diag_every == 0) c->diag_every = 1;
    // default sort brick: 64 cells in 1D, 8 x 8 in 2D, 8 x 8 x 8 in 3D, 4 x 4 x 4 in
    // the 3D electromagnetic step (its tiles of 256 particles then span few cells per
    // axis, which its fixed deposit window needs at low densities); capped by n
    for (int a = 0; a < 3; ++a) {
        if (a >= c->ndim) {
            c->brick[a] = 1;
            continue;
        }
        if (c->brick[a] == 0) c->brick[a] = c->ndim == 1 ? 64 : (c->ndim == 3 && c->em ? 4 : 8);
        if (c->brick[a] < 1) return fail(h, AP_PIC_ERR_ARG, "brick[%d] must be >= 1", a);
        if (c->brick[a] > c->n[a]) c->brick[a] = c->n[a];
    }
    return AP_PIC_OK;
}

// ---- create / destroy ------------------------------------------------------------------------

static ap_pic_status create_pinned(ap_pic *h)
{
    CU(h, cudaMallocHost(&h->h_done, 64));
    CU(h, cudaMallocHost(&h->h_diag, 64));
    CU(h, cudaMallocHost(&h->h_accsum, 64));
    CU(h, cudaMallocHost(&h->h_err, 64));
    CU(h, cudaMallocHost(&h->h_iters, 64));
    return AP_PIC_OK;
}

static ap_pic_status create_grid_f64(ap_pic *h)
{
    FieldBufsF64 &f = h->f64;
    f.ndim = h->ndim;
    f.cells = h->cells;
    for (int a = 0; a < 3; ++a) {
        f.n[a] = h->cfg.n[a];
        f.dx[a] = h->cfg.dx[a];
    }
    f.div0 = make_fastdiv((uint32_t)f.n[0]);
    f.div1 = make_fastdiv((uint32_t)f.n[1]);
    f.nblocks = field_blocks(h->cells);
    const size_t c = (size_t)h->cells;
    TRY(alloc_n(h, &f.acc, c));
    TRY(alloc_n(h, &f.rho, c));
    TRY(alloc_n(h, &f.b, c));
    TRY(alloc_n(h, &f.phi, c));
    TRY(alloc_n(h, &f.r, c));
    TRY(alloc_n(h, &f.p, c));
    TRY(alloc_n(h, &f.q, c));
    TRY(alloc_n(h, &f.E, c * h->ndim));
    for (int k = 0; k < 3; ++k) TRY(alloc_n(h, &f.part[k], (size_t)f.nblocks));
    TRY(alloc_n(h, &f.scal, 8));
    TRY(alloc_n(h, &f.done, 1));
    TRY(alloc_n(h, &f.iters, 1));
    TRY(alloc_n(h, &f.isum_part, (size_t)f.nblocks));
    TRY(alloc_n(h, &f.fe_part, (size_t)f.nblocks));
    TRY(alloc_n(h, &h->d_diag, 8));
    TRY(alloc_n(h, &h->d_accsum, 1));
    TRY(alloc_n(h, &h->d_err, 1));
    CU(h, cudaMemsetAsync(f.acc, 0, c * 8, h->stream));
    CU(h, cudaMemsetAsync(f.phi, 0, c * 8, h->stream));
    CU(h, cudaMemsetAsync(f.E, 0, c * h->ndim * 8, h->stream));
    CU(h, cudaMemsetAsync(f.isum_part, 0, (size_t)f.nblocks * 8, h->stream));
    CU(h, cudaMemsetAsync(f.fe_part, 0, (size_t)f.nblocks * 8, h->stream));
    CU(h, cudaMemsetAsync(f.scal, 0, 64, h->stream));
    CU(h, cudaMemsetAsync(f.iters, 0, 4, h->stream));
    CU(h, cudaMemsetAsync(f.done, 0, 4, h->stream));
    CU(h, cudaMemsetAsync(h->d_diag, 0, 64, h->stream));
    CU(h, cudaMemsetAsync(h->d_err, 0, 4, h->stream));
    return create_pinned(h);
}

// Tables of the spectral solve: per axis the Laplacian's Fourier eigenvalues (and
// for lengths other than powers of two the Bluestein chirp and filter), one
// twiddle table for the longest transform, and the complex work array.
static ap_pic_status create_fft(ap_pic *h)
{
    static std::atomic<unsigned long long> configured{0};
    CU(h, once_per_device(configured, [] { return fft_configure(); }));
    FftPlan &P = h->fft;
    P.ndim = h->ndim;
    P.cells = h->cells;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&P.sms, cudaDevAttrMultiProcessorCount, dev);
    if (P.sms <= 0) P.sms = 148;
    size_t total = 0;
    size_t off[3] = {0, 0, 0};
    P.log2M = 1;
    for (int a = 0; a < h->ndim; ++a) {
        off[a] = total;
        total += fft_axis_table_floats(h->cfg.n[a]);
        const int l = fft_log2m(h->cfg.n[a]);
        if (l > P.log2M) P.log2M = l;
    }
    std::vector<float> host(total + fft_twiddle_floats(P.log2M), 0.0f);
    float *dev_tab = nullptr;
    TRY(alloc_n(h, &dev_tab, host.size()));
    int64_t inner = 1;
    for (int a = 0; a < h->ndim; ++a) {
        fft_axis_tables(h->cfg.n[a], h->cfg.dx[a], host.data() + off[a], dev_tab + off[a],
                        &P.ax[a]);
        P.ax[a].inner = inner;
        inner *= h->cfg.n[a];
    }
    fft_twiddles(P.log2M, host.data() + total);
    P.tw = reinterpret_cast<const float2 *>(dev_tab + total);
    CU(h, cudaMemcpyAsync(dev_tab, host.data(), host.size() * sizeof(float),
                          cudaMemcpyHostToDevice, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
    TRY(alloc_n(h, &P.Z, (size_t)h->cells));
    h->use_fft = true;
    return AP_PIC_OK;
}

// Profiles of the convolutional PML along one axis of n nodes, at integer (shift 0)
// or half (shift 1/2) positions, for an update of step hstep: depth d = distance into
// the layer / its thickness, sigma = 0.8 (m + 1) c / dx d^m (m = 3), kappa = 1,
// alpha = 0; b = exp(-sigma hstep), c = b - 1 (sigma (b - 1) / (sigma kappa)), 1/kappa.
static void cpml_profile(int n, int npml, double dx, double hstep, double c, double shift,
                         float *b, float *cc, float *ik)
{
    const double sigma_max = 0.8 * 4.0 * c / dx;
    for (int i = 0; i < n; ++i) {
        const double x = i + shift;
        double depth = (double)npml - x;
        const double hi = x - (double)(n - 1 - npml);
        if (hi > depth) depth = hi;
        depth = depth > 0.0 ? depth / npml : 0.0;
        b[i] = 1.0f;
        cc[i] = 0.0f;
        ik[i] = 1.0f;
        if (depth <= 0.0) continue;
        const double sigma = sigma_max * depth * depth * depth;
        const double bb = exp(-sigma * hstep);
        b[i] = (float)bb;
        cc[i] = (float)(bb - 1.0);
    }
}

static ap_pic_status create_cpml(ap_pic *h)
{
    const int n0 = h->cfg.n[0], n1 = h->cfg.n[1], npml = h->cfg.pml_cells;
    const double c = h->cfg.c_light, dt = h->cfg.dt;
    std::vector<float> host(3 * (size_t)(n0 + n1) * 2);
    float *dev = nullptr;
    TRY(alloc_n(h, &dev, host.size()));
    // layout: for B (half positions, h = dt/2) then E (integer positions, h = dt):
    // bx cx ikx (n0 each), by cy iky (n1 each)
    size_t off = 0;
    for (int part = 0; part < 2; ++part) {
        const double shift = part == 0 ? 0.5 : 0.0, hs = part == 0 ? 0.5 * dt : dt;
        const float **dst = part == 0 ? h->emb.pb : h->emb.pe;
        float *b = host.data() + off;
        cpml_profile(n0, npml, h->cfg.dx[0], hs, c, shift, b, b + n0, b + 2 * n0);
        for (int k = 0; k < 3; ++k) dst[k] = dev + off + (size_t)k * n0;
        off += 3 * (size_t)n0;
        float *by = host.data() + off;
        cpml_profile(n1, npml, h->cfg.dx[1], hs, c, shift, by, by + n1, by + 2 * n1);
        for (int k = 0; k < 3; ++k) dst[3 + k] = dev + off + (size_t)k * n1;
        off += 3 * (size_t)n1;
    }
    CU(h, cudaMemcpyAsync(dev, host.data(), host.size() * 4, cudaMemcpyHostToDevice, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
    for (int k = 0; k < 4; ++k) {
        TRY(alloc_n(h, &h->emb.psib[k], (size_t)h->cells));
        TRY(alloc_n(h, &h->emb.psie[k], (size_t)h->cells));
        CU(h, cudaMemsetAsync(h->emb.psib[k], 0, (size_t)h->cells * 4, h->stream));
        CU(h, cudaMemsetAsync(h->emb.psie[k], 0, (size_t)h->cells * 4, h->stream));
    }
    return AP_PIC_OK;
}

static ap_pic_status create_grid(ap_pic *h)
{
    if (h->plain) return create_grid_f64(h);
    FieldBufs &f = h->f;
    f.ndim = h->ndim;
    f.cells = h->cells;
    for (int a = 0; a < 3; ++a) {
        f.n[a] = h->cfg.n[a];
        f.dx[a] = h->cfg.dx[a];
    }
    f.div0 = make_fastdiv((uint32_t)f.n[0]);
    f.div1 = make_fastdiv((uint32_t)f.n[1]);
    f.Estride = h->ndim == 3 ? 4 : 2 * h->ndim;
    f.nblocks = field_blocks(h->cells);
    const size_t c = (size_t)h->cells;
    TRY(alloc_n(h, &f.acc, c));
    TRY(alloc_n(h, &f.acc_spare, c));
    TRY(alloc_n(h, &f.b, c));
    TRY(alloc_n(h, &f.phi, c));
    TRY(alloc_n(h, &f.r, c));
    TRY(alloc_n(h, &f.p, c));
    TRY(alloc_n(h, &f.p2, c));
    TRY(alloc_n(h, &f.r2, c));
    TRY(alloc_n(h, &f.w2, c));
    TRY(alloc_n(h, &f.s2, c));
    TRY(alloc_n(h, &f.q, c));
    TRY(alloc_n(h, &f.x, c));
    TRY(alloc_n(h, &f.E, c * f.Estride));
    for (int k = 0; k < 3; ++k) TRY(alloc_n(h, &f.part[k], (size_t)f.nblocks));
    for (int j = 0; j < 2; ++j)
        for (int k = 0; k < 5; ++k) TRY(alloc_n(h, &f.cgpart[j][k], (size_t)f.nblocks));
    TRY(alloc_n(h, &f.ticket, 1));
    CU(h, cudaMemsetAsync(f.ticket, 0, 4, h->stream));
    TRY(alloc_n(h, &f.scal, 8));
    TRY(alloc_n(h, &f.done, 1));
    TRY(alloc_n(h, &f.iters, 2));
    TRY(alloc_n(h, &f.gbar, 2));
    CU(h, cudaMemsetAsync(f.gbar, 0, 8, h->stream));
    TRY(alloc_n(h, &f.isum_part, (size_t)f.nblocks));
    TRY(alloc_n(h, &f.fe_part, (size_t)f.nblocks));
    TRY(alloc_n(h, &h->d_diag, 8));
    TRY(alloc_n(h, &h->d_accsum, 1));
    TRY(alloc_n(h, &h->d_err, 1));
    CU(h, cudaMemsetAsync(f.acc, 0, c * 8, h->stream));
    CU(h, cudaMemsetAsync(f.acc_spare, 0, c * 8, h->stream));
    CU(h, cudaMemsetAsync(f.phi, 0, c * 4, h->stream));
    CU(h, cudaMemsetAsync(f.E, 0, c * f.Estride * 4, h->stream));
    CU(h, cudaMemsetAsync(f.isum_part, 0, (size_t)f.nblocks * 8, h->stream));
    CU(h, cudaMemsetAsync(f.fe_part, 0, (size_t)f.nblocks * 8, h->stream));
    CU(h, cudaMemsetAsync(f.scal, 0, 64, h->stream));
    CU(h, cudaMemsetAsync(f.iters, 0, 8, h->stream));
    CU(h, cudaMemsetAsync(f.done, 0, 4, h->stream));
    CU(h, cudaMemsetAsync(h->d_diag, 0, 64, h->stream));
    CU(h, cudaMemsetAsync(h->d_err, 0, 4, h->stream));
    TRY(alloc_n(h, &h->d_mcc, 3));
    CU(h, cudaMemsetAsync(h->d_mcc, 0, 24, h->stream));
    if (h->cfg.em) {
        h->em = true;
        h->em_np = h->cfg.em_boundary == 1;
        TRY(alloc_n(h, &h->d_absorbed, 1));
        CU(h, cudaMemsetAsync(h->d_absorbed, 0, 8, h->stream));
        TRY(alloc_n(h, &h->emb.E, c * 3));
        TRY(alloc_n(h, &h->emb.B, c * 3));
        TRY(alloc_n(h, &h->emb.J, c * 3));
        CU(h, cudaMemsetAsync(h->emb.E, 0, c * 12, h->stream));
        CU(h, cudaMemsetAsync(h->emb.B, 0, c * 12, h->stream));
        CU(h, cudaMemsetAsync(h->emb.J, 0, c * 24, h->stream));
        for (int a = 0; a < 3; ++a) h->emb.B0[a] = (float)h->cfg.B0[a];
        if (h->cfg.em_boundary == 1) TRY(create_cpml(h));
    }
    if (h->cfg.solver == AP_PIC_SOLVER_FFT) TRY(create_fft(h));
    return create_pinned(h);
}

static void free_particles(ap_pic *h)
{
    dev_free(h, h->p64.x);
    dev_free(h, h->p64.v);
    h->p64 = ParticlesF64{};
    dev_free(h, h->p.cell);
    dev_free(h, h->p.off);
    dev_free(h, h->p.v);
    dev_free(h, h->p_alt.cell);
    dev_free(h, h->p_alt.off);
    dev_free(h, h->p_alt.v);
    for (int k = 0; k < 2; ++k) {
        dev_free(h, h->sort.keys[k]);
        dev_free(h, h->sort.idx[k]);
    }
    dev_free(h, h->sort.hist);
    dev_free(h, h->sort.scan_tmp);
    dev_free(h, h->dpart.blocks);
    dev_free(h, h->emb.tile_flag);
    h->emb.tile_flag = nullptr;
    h->emb.tile_spill = nullptr;
    h->p = ParticlesF32{};
    h->p_alt = ParticlesF32{};
    h->sort = SortScratch{};
    h->dpart = DiagPartials{};
    h->np = 0;
    h->perm_slot = -1;
}

extern "C" ap_pic_status ap_pic_create(const ap_pic_config *cfg, const ap_pic_allocator *alloc,
                                       void *cuda_stream, ap_pic **out)
{
    if (!cfg || !out) return AP_PIC_ERR_ARG;
    *out = nullptr;
    ap_pic *h = new ap_pic();
    h->cfg = *cfg;
    ap_pic_status st = validate(h, &h->cfg);
    if (st != AP_PIC_OK) {
        // the handle carries the message; hand it back so ap_pic_last_error works
        *out = h;
        return st;
    }
    if (alloc && alloc->alloc && alloc->free) {
        h->alloc = *alloc;
        h->has_alloc = true;
    }
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    h->ndim = h->cfg.ndim;
    h->nv = h->cfg.nv;
    h->plain = h->cfg.precision == AP_PIC_FP64_PLAIN;
    h->cells = 1;
    h->dV = 1.0;
    for (int a = 0; a < h->ndim; ++a) {
        h->cells *= h->cfg.n[a];
        h->dV *= h->cfg.dx[a];
    }
    h->V = h->dV * (double)h->cells;
    for (int a = 0; a < 3; ++a) h->brick[a] = h->cfg.brick[a];
    int64_t nkeys = 1;
    for (int a = 0; a < h->ndim; ++a)
        nkeys *= (int64_t)((h->cfg.n[a] + h->brick[a] - 1) / h->brick[a]) * h->brick[a];
    // (the non-periodic mode keeps one key past the cells for absorbed particles)
    h->key_bits = bitlen((uint64_t)(h->cfg.em && h->cfg.em_boundary == 1 ? nkeys : nkeys - 1));
    if (nkeys > (int64_t(1) << 32)) {
        *out = h;
        return fail(h, AP_PIC_ERR_ARG, "sort key range exceeds 32 bits");
    }
    st = create_grid(h);
    *out = h;
    return st;
}

extern "C" ap_pic_status ap_pic_get_config(const ap_pic *h, ap_pic_config *out)
{
    if (!h || !out) return AP_PIC_ERR_ARG;
    *out = h->cfg;
    out->fx_bits = h->fx_bits;
    return AP_PIC_OK;
}

static void drop_graphs(ap_pic *h);

extern "C" ap_pic_status ap_pic_destroy(ap_pic *h)
{
    if (!h) return AP_PIC_OK;
    drain_marks(h);
    if (!h->owned.empty()) cudaStreamSynchronize(h->stream);
    while (!h->owned.empty()) dev_free(h, h->owned.back().first);
    if (h->h_done) cudaFreeHost(h->h_done);
    if (h->h_diag) cudaFreeHost(h->h_diag);
    if (h->h_accsum) cudaFreeHost(h->h_accsum);
    if (h->h_err) cudaFreeHost(h->h_err);
    if (h->h_iters) cudaFreeHost(h->h_iters);
    drop_graphs(h);
    if (h->gev_in) cudaEventDestroy(h->gev_in);
    if (h->gev_out) cudaEventDestroy(h->gev_out);
    if (h->gstream) cudaStreamDestroy(h->gstream);
    delete h;
    return AP_PIC_OK;
}

// ---- particle storage ------------------------------------------------------------------------

// Captured step graphs hold the particle buffers, the particle count and the
// fixed-point scale of the load they were captured under: a new load drops them
// (after any replay still in flight).
static void drop_graphs(ap_pic *h)
{
    bool any = false;
    for (auto &gx : h->graphs) any = any || gx != nullptr;
    if (!any) return;
    if (h->gstream) cudaStreamSynchronize(h->gstream);
    for (auto &gx : h->graphs)
        if (gx) {
            cudaGraphExecDestroy(gx);
            gx = nullptr;
        }
}

static ap_pic_status alloc_particles(ap_pic *h, int64_t np)
{
    drop_graphs(h);
    free_particles(h);
    h->np = np;
    const size_t n = (size_t)(np > 0 ? np : 1);
    // fixed-point scale: S <= 62 - bitlen(np) keeps |sum| < 2^62 whatever the clustering
    const int cap = 62 - bitlen((uint64_t)(np > 0 ? np : 1));
    h->fx_bits = h->cfg.fx_bits < cap ? h->cfg.fx_bits : cap;
    h->dpart.nblocks = h->plain ? plain_pass_blocks(np > 0 ? np : 1, h->ndim)
                       : h->em  ? 2 * (h->ndim == 3 ? em3_particle_blocks(np > 0 ? np : 1)
                                                     : em_particle_blocks(np > 0 ? np : 1))
                                : particle_pass_blocks(np > 0 ? np : 1, h->ndim, h->nv);
    TRY(alloc_n(h, &h->dpart.blocks, (size_t)h->dpart.nblocks * 4));
    CU(h, cudaMemsetAsync(h->dpart.blocks, 0, (size_t)h->dpart.nblocks * 32, h->stream));
    if (h->em) {
        // a flag (2D) or a 16-bit count (3D) per particle tile
        const size_t tiles = (size_t)((np + EM_PASS_TILE - 1) / EM_PASS_TILE) + 1;
        TRY(alloc_n(h, &h->emb.tile_flag, 2 * tiles));
        CU(h, cudaMemsetAsync(h->emb.tile_flag, 0, 2 * tiles, h->stream));
        h->emb.tile_spill = reinterpret_cast<unsigned short *>(h->emb.tile_flag);
    }
    if (h->plain) {
        TRY(alloc_n(h, &h->p64.x, n * h->ndim));
        TRY(alloc_n(h, &h->p64.v, n * h->nv));
        h->p64.np = np;
        h->p64.nv = h->nv;
        return AP_PIC_OK;
    }
    const size_t st = (size_t)soa_stride(np);
    ParticlesF32 *ps[2] = {&h->p, &h->p_alt};
    for (ParticlesF32 *q : ps) {
        TRY(alloc_n(h, &q->cell, st));
        TRY(alloc_n(h, &q->off, st * h->ndim));
        TRY(alloc_n(h, &q->v, st * h->nv));
        CU(h, cudaMemsetAsync(q->cell, 0, st * 4, h->stream));
        CU(h, cudaMemsetAsync(q->off, 0, st * h->ndim * 4, h->stream));
        CU(h, cudaMemsetAsync(q->v, 0, st * h->nv * 4, h->stream));
        q->np = np;
        q->stride = (int64_t)st;
        q->nv = h->nv;
        q->id = nullptr;
        if (h->mcc_on) TRY(alloc_n(h, &q->id, st));
    }
    for (int k = 0; k < 2; ++k) {
        TRY(alloc_n(h, &h->sort.keys[k], n));
        TRY(alloc_n(h, &h->sort.idx[k], n));
    }
    const size_t hl = sort_hist_len(np > 0 ? np : 1);
    TRY(alloc_n(h, &h->sort.hist, hl));
    h->sort.scan_tmp_len = sort_scan_tmp_len(hl);
    TRY(alloc_n(h, &h->sort.scan_tmp, h->sort.scan_tmp_len));
    h->sort.capacity = np;
    return AP_PIC_OK;
}

// ---- the cycle's stages ----------------------------------------------------------------------

static double bg_density(const ap_pic *h)
{
    const double c = h->cfg.rho_background;
    return isnan(c) ? -h->cfg.q * h->cfg.weight * (double)h->np / h->V : c;
}

// rho_e = q w / dV * acc / 2^S: the charge density per unit of the accumulator.
static double rho_scale(const ap_pic *h)
{
    return h->cfg.q * h->cfg.weight / h->dV * ldexp(1.0, -h->fx_bits);
}

// rho from the accumulator: rho_e = q w / dV * acc / 2^S;  b = rho_e - mean(rho_e)
// (mean exact: every particle deposits 2^S, so mean(rho_e) = q w np / V).
static ap_pic_status convert_rho(ap_pic *h, unsigned long long *clear = nullptr)
{
    const double scale = rho_scale(h);
    const double mean_e = h->cfg.q * h->cfg.weight * (double)h->np / h->V;
    const int mk = stage_begin(h, AP_PIC_STAGE_RHO);
    if (h->plain) {
        CU(h, launch_plain_rho_convert(h->f64, scale, bg_density(h), mean_e, h->stream));
    } else {
        // the accumulator's mean, np 2^S / cells, as an integer part and a fraction
        const unsigned long long M = (unsigned long long)h->np << h->fx_bits;  // < 2^62
        const unsigned long long C = (unsigned long long)h->cells;
        const unsigned long long q = M / C;
        CU(h, launch_rho_convert(h->f, (long long)q, (float)((double)(M - q * C) / (double)C),
                                 (float)scale, clear, h->stream));
    }
    stage_end(h, mk);
    return AP_PIC_OK;
}

static ap_pic_status deposit_only(ap_pic *h)
{
    if (h->plain) {
        CU(h, cudaMemsetAsync(h->f64.acc, 0, (size_t)h->cells * 8, h->stream));
        const GridParamsF64 g = grid_params_f64(h, h->cfg.dt);
        CU(h, launch_plain_pass(g, h->p64, h->f64.E, h->f64.acc, false, false, true,
                                DiagPartials{}, h->d_err, h->stream));
        return convert_rho(h);
    }
    CU(h, cudaMemsetAsync(h->f.acc, 0, (size_t)h->cells * 8, h->stream));
    const GridParams g = grid_params(h, h->cfg.dt);
    CU(h, launch_particle_pass(g, h->p, h->f.E, h->f.acc, false, false, true, DiagPartials{},
                               h->d_err, h->stream));
    return convert_rho(h);
}

// CG iterations on `fb` until its device done flag is set or maxit; host checks
// the flag after each block of iterations.  Returns the iterations taken.
template <class LaunchIters>
static ap_pic_status cg_loop(ap_pic *h, int *d_done, int maxit, LaunchIters launch_iters)
{
    int it = 0, chunk = 8;
    while (true) {
        CU(h, cudaMemcpyAsync(h->h_done, d_done, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        CU(h, cudaStreamSynchronize(h->stream));
        if (*h->h_done || it >= maxit) break;
        CU(h, launch_iters(it, chunk));
        it += chunk;
        if (chunk < 64) chunk *= 2;
    }
    return AP_PIC_OK;
}

static ap_pic_status read_scalar(ap_pic *h, const double *d, double *out)
{
    CU(h, cudaMemcpyAsync(h->h_diag + 7, d, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
    *out = h->h_diag[7];
    return AP_PIC_OK;
}

static ap_pic_status read_iters(ap_pic *h, const int *d, int *out)
{
    CU(h, cudaMemcpyAsync(h->h_iters, d, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
    *out = *h->h_iters;
    return AP_PIC_OK;
}

// FP64 plain form: one FP64 Jacobi-PCG solve.
static ap_pic_status solve_field_f64(ap_pic *h)
{
    const double rtol = h->cfg.cg_rtol;
    const int maxit = h->cfg.cg_maxit;
    const int mk = stage_begin(h, AP_PIC_STAGE_FIELD);
    CU(h, launch_plain_cg_init(h->f64, rtol, h->stream));
    TRY(cg_loop(h, h->f64.done, maxit, [&](int it, int n) {
        return launch_plain_cg_iters(h->f64, it, n, maxit, rtol, h->stream);
    }));
    CU(h, launch_plain_cg_finish(h->f64, rtol, h->d_err, h->stream));
    CU(h, launch_plain_efield(h->f64, h->stream));
    stage_end(h, mk);
    TRY(read_iters(h, h->f64.iters, &h->last_cg_iters));
    TRY(read_scalar(h, h->f64.scal + 3, &h->last_cg_relres));
    if (h->last_cg_relres > rtol)
        return fail(h, AP_PIC_ERR_NOT_CONVERGED,
                    "field solve stopped at %d iterations, relative residual %.3e > %.3e",
                    h->last_cg_iters, h->last_cg_relres, rtol);
    return AP_PIC_OK;
}

// FP32 form: FP32-vector Jacobi-PCG with FP64 dots, warm-started from the previous
// potential and stopped on its (recursive) relative residual; then one refinement
// pass: the true residual rho - mean - A phi in FP64, a short FP32 correction solve
// A x = r, phi += x.  The refinement removes the smooth-mode error that the FP32
// recursion cannot see.  (The true residual itself cannot serve as the stopping
// test: the rounding of an FP32 potential, amplified by the Laplacian, floors it.)
static ap_pic_status solve_field_fft(ap_pic *h)
{
    const double mean_total = h->cfg.q * h->cfg.weight * (double)h->np / h->V + bg_density(h);
    FieldBufs &f = h->f;
    const int mk = stage_begin(h, AP_PIC_STAGE_FIELD);
    CU(h, launch_fft_poisson(h->fft, f.b, f.phi, h->stream));
    // refinement pass: the FP64 residual of the FP32 solve, solved again and added to
    // phi by the transform's last pass
    CU(h, launch_residual64(f, rho_scale(h), bg_density(h), mean_total, h->stream));
    CU(h, launch_fft_poisson(h->fft, f.b, f.phi, h->stream, true));
    CU(h, launch_efield(f, h->stream));
    stage_end(h, mk);
    h->last_cg_iters = 0;
    h->relres_on_device = true;  // the first solve's true residual, read with the diagnostics
    h->cg_on_device = false;
    return AP_PIC_OK;
}

// FP32 form: FP32-vector Jacobi-PCG with FP64 dots, warm-started from the previous
// potential and stopped on its (recursive) relative residual, run as one
// cooperative launch that tests convergence on the device; then one refinement
// pass: the true residual rho - mean - A phi in FP64, a short FP32 correction
// solve A x = r (its cap: what the first solve left of cg_maxit), phi += x.  No
// host round trip: a solve that stops at its cap latches EF_CG, reported as
// AP_PIC_ERR_NOT_CONVERGED by the next synchronising call, and the iterations and
// residual are read with the diagnostics.
static ap_pic_status solve_field(ap_pic *h)
{
    if (h->plain) return solve_field_f64(h);
    if (h->use_fft) return solve_field_fft(h);
    constexpr double REFINE_RTOL = 1e-2;
    const double rtol = h->cfg.cg_rtol;
    const int maxit = h->cfg.cg_maxit;
    const double mean_total = h->cfg.q * h->cfg.weight * (double)h->np / h->V + bg_density(h);
    FieldBufs &f = h->f;
    const int mk = stage_begin(h, AP_PIC_STAGE_FIELD);
    CU(h, launch_cg_solve(f, f.b, f.phi, rtol, maxit, nullptr, f.iters, SCAL_CG_REL, true,
                          h->d_err, h->stream));
    // refinement pass
    CU(h, launch_residual64(f, rho_scale(h), bg_density(h), mean_total, h->stream));
    CU(h, cudaMemsetAsync(f.x, 0, (size_t)h->cells * 4, h->stream));
    CU(h, launch_cg_solve(f, f.b, f.x, REFINE_RTOL, maxit, f.iters, f.iters + 1, SCAL_CG_REL2,
                          false, h->d_err, h->stream));
    CU(h, launch_add_correction(f, h->stream));
    CU(h, launch_efield(f, h->stream));
    stage_end(h, mk);
    h->relres_on_device = false;
    h->cg_on_device = true;
    return AP_PIC_OK;
}

static ap_pic_status sort_particles(ap_pic *h)
{
    if (h->np == 0 || h->plain) return AP_PIC_OK;
    const GridParams g = grid_params(h, h->cfg.dt);
    int slot = 0;
    const int mk = stage_begin(h, AP_PIC_STAGE_SORT);
    CU(h, launch_sort_perm(g, h->brick, h->key_bits, h->p.cell, h->np, h->sort, &slot, h->stream));
    CU(h, launch_apply_perm(h->sort.idx[slot], h->p, h->p_alt, h->ndim, h->stream));
    stage_end(h, mk);
    h->parity ^= 1;
    ParticlesF32 t = h->p;
    h->p = h->p_alt;
    h->p_alt = t;
    h->perm_slot = slot;
    if (h->em_np) {
        // the sort moved the particles absorbed since the last one past the live ones
        // (their key follows every cell's): drop them
        unsigned long long gone = 0;
        CU(h, cudaMemcpyAsync(h->h_accsum + 4, h->d_absorbed, 8, cudaMemcpyDeviceToHost,
                              h->stream));
        CU(h, cudaStreamSynchronize(h->stream));
        gone = (unsigned long long)h->h_accsum[4];
        CU(h, cudaMemsetAsync(h->d_absorbed, 0, 8, h->stream));
        if (gone > (unsigned long long)h->np)
            return fail(h, AP_PIC_ERR_STATE, "absorbed count exceeds the particles");
        h->np -= (int64_t)gone;
        h->absorbed_total += (int64_t)gone;
        h->p.np = h->p_alt.np = h->np;
    }
    return AP_PIC_OK;
}

static ap_pic_status finalize_diag(ap_pic *h, bool have_particles)
{
    const int mk = stage_begin(h, AP_PIC_STAGE_DIAG);
    if (h->plain)
        CU(h, launch_plain_diag_finalize(h->dpart, have_particles, h->f64, h->d_diag, h->d_accsum,
                                         h->stream));
    else
        CU(h, launch_diag_finalize(h->dpart, have_particles, h->f, h->d_diag, h->d_accsum,
                                   h->stream));
    stage_end(h, mk);
    h->diag_valid = true;
    return AP_PIC_OK;
}

// Field update after particles moved: deposit -> rho -> Poisson -> E (D06).
static ap_pic_status field_update(ap_pic *h)
{
    TRY(deposit_only(h));
    return solve_field(h);
}

static ap_pic_status half_push(ap_pic *h)
{
    if (h->plain) {
        const GridParamsF64 g = grid_params_f64(h, -0.5 * h->cfg.dt);
        CU(h, launch_plain_pass(g, h->p64, h->f64.E, h->f64.acc, true, false, false,
                                DiagPartials{}, h->d_err, h->stream));
        return AP_PIC_OK;
    }
    const GridParams g = grid_params(h, -0.5 * h->cfg.dt);
    if (h->em) {
        if (h->em_np)
            CU(h, launch_em_np_push(g, h->p, h->emb, false, nullptr, nullptr, h->dpart.nblocks,
                                    h->d_err, h->d_absorbed, h->stream));
        else if (h->ndim == 3)
            CU(h, launch_em3_push(g, h->p, h->emb, false, nullptr, nullptr, h->dpart.nblocks,
                                  h->d_err, nullptr, h->stream));
        else
            CU(h, launch_em_push(g, h->p, h->emb, false, nullptr, nullptr, h->dpart.nblocks,
                                 h->d_err, h->stream));
        return AP_PIC_OK;
    }
    CU(h, launch_particle_pass(g, h->p, h->f.E, h->f.acc, true, false, false, DiagPartials{},
                               h->d_err, h->stream));
    return AP_PIC_OK;
}

static ap_pic_status after_load(ap_pic *h, unsigned flags)
{
    if (h->em_np) {
        const GridParams g = grid_params(h, h->cfg.dt);
        CU(h, launch_em_np_check(g, h->p, h->d_err, h->stream));
    }
    TRY(sync_check(h));
    TRY(sort_particles(h));
    if (h->em_np) {
        // the non-periodic mode starts from zero fields (no Poisson solve): only the
        // charge of the loaded particles, for the diagnostics
        TRY(deposit_only(h));
        CU(h, cudaMemsetAsync(h->emb.E, 0, (size_t)h->cells * 12, h->stream));
        CU(h, cudaMemsetAsync(h->emb.B, 0, (size_t)h->cells * 12, h->stream));
        CU(h, launch_em_energy(h->emb, h->cells, h->cfg.c_light, h->f.fe_part, h->f.nblocks,
                               h->stream));
    } else {
        TRY(field_update(h));
    }
    if (h->em && !h->em_np) {
        // the electrostatic field of the loaded charge on the Yee lattice, B = 0
        const GridParams g = grid_params(h, h->cfg.dt);
        if (h->ndim == 3)
            CU(h, launch_em3_e_from_phi(g, h->f.phi, h->emb, h->cfg.dx, h->stream));
        else
            CU(h, launch_em_e_from_phi(g, h->f.phi, h->emb, h->cfg.dx[0], h->cfg.dx[1], h->stream));
        CU(h, cudaMemsetAsync(h->emb.B, 0, (size_t)h->cells * 12, h->stream));
        CU(h, launch_em_energy(h->emb, h->cells, h->cfg.c_light, h->f.fe_part, h->f.nblocks,
                               h->stream));
    }
    TRY(finalize_diag(h, false));
    if (!(flags & AP_PIC_LOAD_NO_HALFPUSH)) TRY(half_push(h));
    h->step = 0;
    h->loaded = true;
    return sync_check(h);
}

extern "C" ap_pic_status ap_pic_load(ap_pic *h, int64_t np, const double *x, const double *v,
                                     unsigned flags)
{
    if (!h) return AP_PIC_ERR_ARG;
    if (np < 0 || np >= (int64_t(1) << 31)) return fail(h, AP_PIC_ERR_ARG, "np out of range");
    if (np > 0 && (!x || !v)) return fail(h, AP_PIC_ERR_ARG, "x and v are required");
    TRY(alloc_particles(h, np));
    const int64_t chunk = np < LOAD_CHUNK ? (np > 0 ? np : 1) : LOAD_CHUNK;
    double *dx_buf = nullptr, *dv_buf = nullptr;
    TRY(alloc_n(h, &dx_buf, (size_t)chunk * h->ndim));
    TRY(alloc_n(h, &dv_buf, (size_t)chunk * h->nv));
    const GridParams g = grid_params(h, h->cfg.dt);
    const GridParamsF64 g64 = grid_params_f64(h, h->cfg.dt);
    for (int64_t first = 0; first < np; first += chunk) {
        const int64_t cnt = np - first < chunk ? np - first : chunk;
        CU(h, cudaMemcpyAsync(dx_buf, x + first * h->ndim, (size_t)cnt * h->ndim * 8,
                              cudaMemcpyHostToDevice, h->stream));
        CU(h, cudaMemcpyAsync(dv_buf, v + first * h->nv, (size_t)cnt * h->nv * 8,
                              cudaMemcpyHostToDevice, h->stream));
        if (h->plain)
            CU(h, launch_plain_load(g64, dx_buf, dv_buf, h->p64, first, cnt, h->d_err, h->stream));
        else
            CU(h, launch_load_convert(g, h->cfg.dx, dx_buf, dv_buf, h->p, first, cnt, h->d_err,
                                      h->stream));
    }
    if (h->mcc_on) CU(h, launch_iota(h->p.id, np, h->stream));  // ids: the load order
    CU(h, cudaStreamSynchronize(h->stream));
    dev_free(h, dx_buf);
    dev_free(h, dv_buf);
    if (h->plain) CU(h, cudaMemsetAsync(h->f64.phi, 0, (size_t)h->cells * 8, h->stream));
    else CU(h, cudaMemsetAsync(h->f.phi, 0, (size_t)h->cells * 4, h->stream));
    return after_load(h, flags);
}

extern "C" ap_pic_status ap_pic_load_state(ap_pic *h, int64_t np, const int32_t *cell,
                                           const float *off, const float *v, unsigned flags)
{
    if (!h) return AP_PIC_ERR_ARG;
    if (np < 0 || np >= (int64_t(1) << 31)) return fail(h, AP_PIC_ERR_ARG, "np out of range");
    if (np > 0 && (!cell || !off || !v)) return fail(h, AP_PIC_ERR_ARG, "cell, off, v required");
    if (h->plain)
        return fail(h, AP_PIC_ERR_UNSUPPORTED, "ap_pic_load_state needs the FP32 cell+offset form");
    TRY(alloc_particles(h, np));
    if (np > 0) {
        // the alternate buffers double as staging for the row-major host layout
        CU(h, cudaMemcpyAsync(h->p_alt.cell, cell, (size_t)np * 4, cudaMemcpyHostToDevice,
                              h->stream));
        CU(h, cudaMemcpyAsync(h->p_alt.off, off, (size_t)np * h->ndim * 4, cudaMemcpyHostToDevice,
                              h->stream));
        CU(h, cudaMemcpyAsync(h->p_alt.v, v, (size_t)np * h->nv * 4, cudaMemcpyHostToDevice,
                              h->stream));
        const GridParams g = grid_params(h, h->cfg.dt);
        CU(h, launch_load_state(g, h->p_alt.cell, h->p_alt.off, h->p_alt.v, h->p, h->d_err,
                                h->stream));
        if (h->mcc_on) CU(h, launch_iota(h->p.id, np, h->stream));
    }
    CU(h, cudaMemsetAsync(h->f.phi, 0, (size_t)h->cells * 4, h->stream));
    return after_load(h, flags);
}

static ap_pic_status need_loaded(ap_pic *h)
{
    if (!h) return AP_PIC_ERR_ARG;
    if (!h->loaded) return fail(h, AP_PIC_ERR_STATE, "no particles loaded");
    return AP_PIC_OK;
}

extern "C" ap_pic_status ap_pic_gather_push(ap_pic *h)
{
    TRY(need_loaded(h));
    if (h->em) return fail(h, AP_PIC_ERR_UNSUPPORTED, "em = 1: use ap_pic_step");
    if (h->plain) {
        const GridParamsF64 g = grid_params_f64(h, h->cfg.dt);
        CU(h, launch_plain_pass(g, h->p64, h->f64.E, h->f64.acc, true, true, false, h->dpart,
                                h->d_err, h->stream));
        return AP_PIC_OK;
    }
    const GridParams g = grid_params(h, h->cfg.dt);
    CU(h, launch_particle_pass(g, h->p, h->f.E, h->f.acc, true, true, false, h->dpart, h->d_err,
                               h->stream));
    return AP_PIC_OK;
}

extern "C" ap_pic_status ap_pic_deposit(ap_pic *h)
{
    TRY(need_loaded(h));
    if (h->em) return fail(h, AP_PIC_ERR_UNSUPPORTED, "em = 1: use ap_pic_step");
    return deposit_only(h);
}

// The two FP32-form accumulators trade places (see push_deposit).
static void swap_acc(ap_pic *h)
{
    unsigned long long *t = h->f.acc;
    h->f.acc = h->f.acc_spare;
    h->f.acc_spare = t;
    h->acc_parity ^= 1;
}

static ap_pic_status push_deposit(ap_pic *h, bool diag)
{
    if (h->plain) {
        CU(h, cudaMemsetAsync(h->f64.acc, 0, (size_t)h->cells * 8, h->stream));
        const GridParamsF64 g = grid_params_f64(h, h->cfg.dt);
        const int mk = stage_begin(h, AP_PIC_STAGE_PUSH_DEPOSIT);
        CU(h, launch_plain_pass(g, h->p64, h->f64.E, h->f64.acc, true, true, true,
                                diag ? h->dpart : DiagPartials{}, h->d_err, h->stream));
        stage_end(h, mk);
        return convert_rho(h);
    }
    // deposit into the spare accumulator (zero), make it the current one, and convert
    // it while clearing the previous one: no memset per step
    const GridParams g = grid_params(h, h->cfg.dt);
    const int mk = stage_begin(h, AP_PIC_STAGE_PUSH_DEPOSIT);
    CU(h, launch_particle_pass(g, h->p, h->f.E, h->f.acc_spare, true, true, true,
                               diag ? h->dpart : DiagPartials{}, h->d_err, h->stream));
    stage_end(h, mk);
    swap_acc(h);
    return convert_rho(h, h->f.acc_spare);
}

extern "C" ap_pic_status ap_pic_push_deposit(ap_pic *h)
{
    TRY(need_loaded(h));
    if (h->em) return fail(h, AP_PIC_ERR_UNSUPPORTED, "em = 1: use ap_pic_step");
    return push_deposit(h, true);
}

extern "C" ap_pic_status ap_pic_solve_field(ap_pic *h)
{
    TRY(need_loaded(h));
    if (h->em) return fail(h, AP_PIC_ERR_UNSUPPORTED, "em = 1: use ap_pic_step");
    return solve_field(h);
}

extern "C" ap_pic_status ap_pic_sort(ap_pic *h)
{
    TRY(need_loaded(h));
    return sort_particles(h);
}

// One electromagnetic step: particles (gather, push, move, current, charge), then
// the field update; the diagnostics' field energy is electric plus magnetic.
static ap_pic_status em_step(ap_pic *h, bool diag)
{
    CU(h, cudaMemsetAsync(h->f.acc, 0, (size_t)h->cells * 8, h->stream));
    const GridParams g = grid_params(h, h->cfg.dt);
    const int mk = stage_begin(h, AP_PIC_STAGE_PUSH_DEPOSIT);
    if (h->em_np)
        CU(h, launch_em_np_push(g, h->p, h->emb, true, h->f.acc, diag ? h->dpart.blocks : nullptr,
                                h->dpart.nblocks, h->d_err, h->d_absorbed, h->stream));
    else if (h->ndim == 3)
        // the sort's destination buffer is free between sorts: its cell array holds
        // the list of particles the tiled kernel leaves to the global-memory kernel
        CU(h, launch_em3_push(g, h->p, h->emb, true, h->f.acc, diag ? h->dpart.blocks : nullptr,
                              h->dpart.nblocks, h->d_err, h->p_alt.cell, h->stream));
    else
        CU(h, launch_em_push(g, h->p, h->emb, true, h->f.acc, diag ? h->dpart.blocks : nullptr,
                             h->dpart.nblocks, h->d_err, h->stream));
    stage_end(h, mk);
    TRY(convert_rho(h));
    const int mf = stage_begin(h, AP_PIC_STAGE_FIELD);
    if (h->ndim == 3)
        CU(h, launch_em3_fields(g, h->emb, h->cfg.dx, h->cfg.dt, h->cfg.c_light,
                                h->cfg.q * h->cfg.weight, h->stream));
    else
        CU(h, launch_em_fields(g, h->emb, h->cfg.dx[0], h->cfg.dx[1], h->cfg.dt, h->cfg.c_light,
                               h->cfg.q * h->cfg.weight, h->stream));
    if (diag)
        CU(h, launch_em_energy(h->emb, h->cells, h->cfg.c_light, h->f.fe_part, h->f.nblocks,
                               h->stream));
    stage_end(h, mf);
    return AP_PIC_OK;
}

extern "C" ap_pic_status ap_pic_set_collisions(ap_pic *h, const ap_pic_mcc *c)
{
    if (!h) return AP_PIC_ERR_ARG;
    if (h->loaded || h->np > 0)
        return fail(h, AP_PIC_ERR_STATE, "set collisions before loading particles");
    if (!c) {
        h->mcc_on = false;
        return AP_PIC_OK;
    }
    if (h->plain) return fail(h, AP_PIC_ERR_UNSUPPORTED, "collisions need the FP32 form");
    if (h->nv != 3) return fail(h, AP_PIC_ERR_ARG, "collisions need nv = 3");
    if (h->em) return fail(h, AP_PIC_ERR_UNSUPPORTED, "collisions with the electromagnetic step");
    if (h->cfg.pusher != AP_PIC_PUSHER_BORIS)
        return fail(h, AP_PIC_ERR_UNSUPPORTED, "collisions need the Boris pusher");
    const double vals[5] = {c->density, c->sigma_el, c->sigma_exc, c->eps_exc, c->mass_ratio};
    for (double x : vals)
        if (!(x >= 0.0) || !isfinite(x))
            return fail(h, AP_PIC_ERR_ARG, "collision parameters must be >= 0 and finite");
    if (c->mass_ratio > 0.25) return fail(h, AP_PIC_ERR_ARG, "mass_ratio must be <= 0.25");
    if (!(c->vmax > 0.0) || !isfinite(c->vmax)) return fail(h, AP_PIC_ERR_ARG, "vmax must be > 0");
    h->mccp = make_mcc_params(c->density, c->sigma_el, c->sigma_exc, c->eps_exc, c->mass_ratio,
                              c->vmax, h->cfg.m, h->cfg.dt, c->seed);
    h->mcc_on = true;
    return AP_PIC_OK;
}

extern "C" ap_pic_status ap_pic_collide(ap_pic *h)
{
    TRY(need_loaded(h));
    if (!h->mcc_on) return fail(h, AP_PIC_ERR_STATE, "collisions are not enabled");
    CU(h, launch_mcc(h->p, h->mccp, (uint64_t)(h->step + 1), h->d_mcc, h->stream));
    return AP_PIC_OK;
}

// A step can replay a graph when it holds no host decision and no per-step value:
// the FP32 form (either solver: the CG tests convergence on the device), no
// collisions (their draws take the step number), not the electromagnetic step,
// stage timing off.
static bool step_graphable(const ap_pic *h)
{
    return !h->plain && !h->mcc_on && !h->em && !h->timing;
}

// One step through its captured graph (captured on first use of its variant).
static ap_pic_status graph_step(ap_pic *h, bool diag, bool sort)
{
    if (!h->gstream) {
        CU(h, cudaStreamCreateWithFlags(&h->gstream, cudaStreamNonBlocking));
        CU(h, cudaEventCreateWithFlags(&h->gev_in, cudaEventDisableTiming));
        CU(h, cudaEventCreateWithFlags(&h->gev_out, cudaEventDisableTiming));
    }
    const int key = h->acc_parity * 8 + h->parity * 4 + (diag ? 2 : 0) + (sort ? 1 : 0);
    // fence: the graph stream after the caller's work
    CU(h, cudaEventRecord(h->gev_in, h->stream));
    CU(h, cudaStreamWaitEvent(h->gstream, h->gev_in, 0));
    if (!h->graphs[key]) {
        cudaStream_t user = h->stream;
        h->stream = h->gstream;
        const int64_t before = ap_pic_kernel_launches();
        cudaGraph_t graph = nullptr;
        ap_pic_status st = AP_PIC_OK;
        cudaError_t ce = cudaStreamBeginCapture(h->gstream, cudaStreamCaptureModeThreadLocal);
        if (ce == cudaSuccess) {
            st = push_deposit(h, diag);
            if (st == AP_PIC_OK && sort) st = sort_particles(h);
            if (st == AP_PIC_OK) st = solve_field(h);
            if (st == AP_PIC_OK && diag) st = finalize_diag(h, true);
            ce = cudaStreamEndCapture(h->gstream, &graph);
        }
        h->stream = user;
        if (st != AP_PIC_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        CU(h, ce);
        const cudaError_t ie = cudaGraphInstantiate(&h->graphs[key], graph, 0);
        cudaGraphDestroy(graph);
        CU(h, ie);
        // the capture recorded the launches without running them; the host state
        // (the accumulators' and a sort's buffer swaps) is already that of after the step
        h->graph_launches[key] = ap_pic_kernel_launches() - before;
        note_launch(-(int)h->graph_launches[key]);
        h->graph_slot[key] = h->perm_slot;
    } else {
        // replay: the host side of the swaps
        swap_acc(h);
        if (sort) {
            h->parity ^= 1;
            ParticlesF32 t = h->p;
            h->p = h->p_alt;
            h->p_alt = t;
            h->perm_slot = h->graph_slot[key];
        }
    }
    CU(h, cudaGraphLaunch(h->graphs[key], h->gstream));
    note_launch((int)h->graph_launches[key]);
    CU(h, cudaEventRecord(h->gev_out, h->gstream));
    CU(h, cudaStreamWaitEvent(h->stream, h->gev_out, 0));
    return AP_PIC_OK;
}

extern "C" ap_pic_status ap_pic_step(ap_pic *h, int nsteps)
{
    TRY(need_loaded(h));
    if (nsteps < 0) return fail(h, AP_PIC_ERR_ARG, "nsteps must be >= 0");
    for (int s = 0; s < nsteps; ++s) {
        const int64_t k = h->step + 1;
        const bool diag = (k % h->cfg.diag_every) == 0;
        if (h->em) {
            TRY(em_step(h, diag));
            if (h->cfg.sort_every > 0 && k % h->cfg.sort_every == 0) TRY(sort_particles(h));
            if (diag) TRY(finalize_diag(h, true));
            h->step = k;
            continue;
        }
        if (step_graphable(h)) {
            TRY(graph_step(h, diag, h->cfg.sort_every > 0 && k % h->cfg.sort_every == 0));
            h->step = k;
            continue;
        }
        TRY(push_deposit(h, diag));
        if (h->mcc_on) CU(h, launch_mcc(h->p, h->mccp, (uint64_t)k, h->d_mcc, h->stream));
        if (h->cfg.sort_every > 0 && k % h->cfg.sort_every == 0) TRY(sort_particles(h));
        TRY(solve_field(h));
        if (diag) TRY(finalize_diag(h, true));
        h->step = k;
    }
    return AP_PIC_OK;
}

// ---- read-back -------------------------------------------------------------------------------

extern "C" ap_pic_status ap_pic_get_rho(ap_pic *h, double *out)
{
    if (!h || !out) return AP_PIC_ERR_ARG;
    if (h->plain) {
        CU(h, cudaMemcpyAsync(out, h->f64.rho, (size_t)h->cells * 8, cudaMemcpyDeviceToHost,
                              h->stream));
        return sync_check(h);
    }
    // the FP32 form keeps the charge as the int64 accumulator: rho = scale acc + bg,
    // formed here in place (the same FP64 arithmetic as the device's residual)
    CU(h, cudaMemcpyAsync(out, h->f.acc, (size_t)h->cells * 8, cudaMemcpyDeviceToHost,
                          h->stream));
    const ap_pic_status st = sync_check(h);
    if (st != AP_PIC_OK) return st;
    const double scale = rho_scale(h), bg = bg_density(h);
    for (int64_t j = 0; j < h->cells; ++j) {
        int64_t a;
        memcpy(&a, &out[j], 8);
        out[j] = scale * (double)a + bg;
    }
    return AP_PIC_OK;
}

extern "C" ap_pic_status ap_pic_get_rho_fx(ap_pic *h, int64_t *out)
{
    if (!h || !out) return AP_PIC_ERR_ARG;
    CU(h, cudaMemcpyAsync(out, h->plain ? h->f64.acc : h->f.acc, (size_t)h->cells * 8,
                          cudaMemcpyDeviceToHost, h->stream));
    return sync_check(h);
}

// A [3][cells] FP32 device array as FP64 on the host.
static ap_pic_status copy3_f32(ap_pic *h, const float *src, double *out)
{
    std::vector<float> tmp((size_t)h->cells * 3);
    CU(h, cudaMemcpyAsync(tmp.data(), src, tmp.size() * 4, cudaMemcpyDeviceToHost, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
    for (size_t i = 0; i < tmp.size(); ++i) out[i] = tmp[i];
    return sync_check(h);
}

extern "C" ap_pic_status ap_pic_set_current(ap_pic *h, const double *J)
{
    if (!h) return AP_PIC_ERR_ARG;
    if (!h->em) return fail(h, AP_PIC_ERR_STATE, "a prescribed current needs em = 1");
    if (!J) {
        h->emb.Jext = nullptr;
        return AP_PIC_OK;
    }
    if (!h->jext) TRY(alloc_n(h, &h->jext, (size_t)h->cells * 3));
    std::vector<float> tmp((size_t)h->cells * 3);
    for (size_t i = 0; i < tmp.size(); ++i) tmp[i] = (float)J[i];
    CU(h, cudaMemcpyAsync(h->jext, tmp.data(), tmp.size() * 4, cudaMemcpyHostToDevice, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));  // tmp goes out of scope
    h->emb.Jext = h->jext;
    return AP_PIC_OK;
}

extern "C" ap_pic_status ap_pic_get_B(ap_pic *h, double *out)
{
    if (!h || !out) return AP_PIC_ERR_ARG;
    if (!h->em) return fail(h, AP_PIC_ERR_STATE, "no magnetic field: em = 0");
    return copy3_f32(h, h->emb.B, out);
}

extern "C" ap_pic_status ap_pic_get_E(ap_pic *h, double *out)
{
    if (!h || !out) return AP_PIC_ERR_ARG;
    if (h->em) return copy3_f32(h, h->emb.E, out);
    if (h->plain) {
        CU(h, cudaMemcpyAsync(out, h->f64.E, (size_t)h->cells * h->ndim * 8,
                              cudaMemcpyDeviceToHost, h->stream));
        return sync_check(h);
    }
    double *tmp = nullptr;
    TRY(alloc_n(h, &tmp, (size_t)h->cells * h->ndim));
    CU(h, launch_e_to_f64(h->f, tmp, h->stream));
    CU(h, cudaMemcpyAsync(out, tmp, (size_t)h->cells * h->ndim * 8, cudaMemcpyDeviceToHost,
                          h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
    dev_free(h, tmp);
    return sync_check(h);
}

extern "C" ap_pic_status ap_pic_get_phi(ap_pic *h, double *out)
{
    if (!h || !out) return AP_PIC_ERR_ARG;
    if (h->plain) {
        CU(h, cudaMemcpyAsync(out, h->f64.phi, (size_t)h->cells * 8, cudaMemcpyDeviceToHost,
                              h->stream));
        CU(h, cudaStreamSynchronize(h->stream));
    } else {
        double *tmp = nullptr;
        TRY(alloc_n(h, &tmp, (size_t)h->cells));
        CU(h, launch_phi_to_f64(h->f, tmp, h->stream));
        CU(h, cudaMemcpyAsync(out, tmp, (size_t)h->cells * 8, cudaMemcpyDeviceToHost, h->stream));
        CU(h, cudaStreamSynchronize(h->stream));
        dev_free(h, tmp);
    }
    // phi is defined up to a constant; report the zero-mean representative
    double mean = 0.0;
    for (int64_t i = 0; i < h->cells; ++i) mean += out[i];
    mean /= (double)h->cells;
    for (int64_t i = 0; i < h->cells; ++i) out[i] -= mean;
    return sync_check(h);
}

// FP64 plain form: positions and velocities are stored; cell and offset are
// derived on the host with the same floor rule as the device.
static ap_pic_status get_particles_plain(ap_pic *h, int32_t *cell, float *off, float *v, double *x)
{
    const int64_t np = h->np;
    std::vector<double> xs((size_t)np * h->ndim), vs;
    CU(h, cudaMemcpyAsync(xs.data(), h->p64.x, xs.size() * 8, cudaMemcpyDeviceToHost, h->stream));
    if (v) {
        vs.resize((size_t)np * h->nv);
        CU(h, cudaMemcpyAsync(vs.data(), h->p64.v, vs.size() * 8, cudaMemcpyDeviceToHost,
                              h->stream));
    }
    CU(h, cudaStreamSynchronize(h->stream));
    for (int64_t i = 0; i < np; ++i) {
        int64_t lin = 0, stride = 1;
        for (int a = 0; a < h->ndim; ++a) {
            const double xa = xs[(size_t)a * np + i];
            const double u = xa * (1.0 / h->cfg.dx[a]);
            double fl = floor(u);
            double fa = u - fl;
            int ca = (int)fl;
            if (ca >= h->cfg.n[a] || ca < 0) {
                ca = 0;
                fa = 0.0;
            }
            lin += ca * stride;
            stride *= h->cfg.n[a];
            if (x) x[i * h->ndim + a] = xa;
            if (off) off[i * h->ndim + a] = (float)fa < 1.0f ? (float)fa : 0x1.fffffep-1f;
        }
        if (cell) cell[i] = (int32_t)lin;
        if (v)
            for (int a = 0; a < h->nv; ++a) v[i * h->nv + a] = (float)vs[(size_t)a * np + i];
    }
    return sync_check(h);
}

extern "C" ap_pic_status ap_pic_get_particles(ap_pic *h, int32_t *cell, float *off, float *v,
                                              double *x)
{
    TRY(need_loaded(h));
    const int64_t np = h->np;
    if (np == 0) return AP_PIC_OK;
    if (h->plain) return get_particles_plain(h, cell, off, v, x);
    if (cell)
        CU(h, cudaMemcpyAsync(cell, h->p.cell, (size_t)np * 4, cudaMemcpyDeviceToHost, h->stream));
    std::vector<float> tmp;
    if (off) {
        tmp.resize((size_t)h->p.stride * h->ndim);
        CU(h, cudaMemcpyAsync(tmp.data(), h->p.off, tmp.size() * 4, cudaMemcpyDeviceToHost,
                              h->stream));
        CU(h, cudaStreamSynchronize(h->stream));
        for (int64_t i = 0; i < np; ++i)
            for (int a = 0; a < h->ndim; ++a)
                off[i * h->ndim + a] = tmp[(size_t)a * h->p.stride + i];
    }
    if (v) {
        tmp.resize((size_t)h->p.stride * h->nv);
        CU(h, cudaMemcpyAsync(tmp.data(), h->p.v, tmp.size() * 4, cudaMemcpyDeviceToHost,
                              h->stream));
        CU(h, cudaStreamSynchronize(h->stream));
        for (int64_t i = 0; i < np; ++i)
            for (int a = 0; a < h->nv; ++a) v[i * h->nv + a] = tmp[(size_t)a * h->p.stride + i];
    }
    if (x) {
        double *dxp = nullptr;
        TRY(alloc_n(h, &dxp, (size_t)np * h->ndim));
        const GridParams g = grid_params(h, h->cfg.dt);
        CU(h, launch_positions_f64(g, h->cfg.dx, h->p, dxp, h->stream));
        CU(h, cudaMemcpyAsync(x, dxp, (size_t)np * h->ndim * 8, cudaMemcpyDeviceToHost,
                              h->stream));
        CU(h, cudaStreamSynchronize(h->stream));
        dev_free(h, dxp);
    }
    return sync_check(h);
}

extern "C" ap_pic_status ap_pic_get_velocities_f64(ap_pic *h, double *v)
{
    TRY(need_loaded(h));
    if (!v) return fail(h, AP_PIC_ERR_ARG, "v is NULL");
    if (!h->plain)
        return fail(h, AP_PIC_ERR_UNSUPPORTED, "only the FP64 plain form stores FP64 velocities");
    std::vector<double> vs((size_t)h->np * h->nv);
    if (h->np)
        CU(h, cudaMemcpyAsync(vs.data(), h->p64.v, vs.size() * 8, cudaMemcpyDeviceToHost,
                              h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
    for (int64_t i = 0; i < h->np; ++i)
        for (int a = 0; a < h->nv; ++a) v[i * h->nv + a] = vs[(size_t)a * h->np + i];
    return sync_check(h);
}

extern "C" ap_pic_status ap_pic_get_perm(ap_pic *h, int64_t *perm)
{
    TRY(need_loaded(h));
    if (!perm) return fail(h, AP_PIC_ERR_ARG, "perm is NULL");
    if (h->perm_slot < 0) return fail(h, AP_PIC_ERR_STATE, "no sort has run");
    std::vector<uint32_t> tmp((size_t)h->np);
    if (h->np)
        CU(h, cudaMemcpyAsync(tmp.data(), h->sort.idx[h->perm_slot], (size_t)h->np * 4,
                              cudaMemcpyDeviceToHost, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
    for (int64_t i = 0; i < h->np; ++i) perm[i] = tmp[(size_t)i];
    return sync_check(h);
}

extern "C" ap_pic_status ap_pic_get_diag(ap_pic *h, ap_pic_diag *out)
{
    if (!h || !out) return AP_PIC_ERR_ARG;
    memset(out, 0, sizeof *out);
    CU(h, cudaMemcpyAsync(h->h_diag, h->d_diag, 7 * sizeof(double), cudaMemcpyDeviceToHost,
                          h->stream));
    CU(h, cudaMemcpyAsync(h->h_accsum, h->d_accsum, sizeof(long long), cudaMemcpyDeviceToHost,
                          h->stream));
    CU(h, cudaMemcpyAsync(h->h_err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    if (h->d_mcc)
        CU(h, cudaMemcpyAsync(h->h_accsum + 1, h->d_mcc, 3 * sizeof(long long),
                              cudaMemcpyDeviceToHost, h->stream));
    if (h->relres_on_device)
        CU(h, cudaMemcpyAsync(h->h_diag + 7, h->f.scal + SCAL_TRUE_REL, sizeof(double),
                              cudaMemcpyDeviceToHost, h->stream));
    if (h->cg_on_device) {
        CU(h, cudaMemcpyAsync(h->h_diag + 7, h->f.scal + SCAL_CG_REL, sizeof(double),
                              cudaMemcpyDeviceToHost, h->stream));
        CU(h, cudaMemcpyAsync(h->h_iters, h->f.iters, 2 * sizeof(int), cudaMemcpyDeviceToHost,
                              h->stream));
    }
    CU(h, cudaStreamSynchronize(h->stream));
    if (h->relres_on_device) h->last_cg_relres = h->h_diag[7];
    if (h->cg_on_device) {
        h->last_cg_relres = h->h_diag[7];
        h->last_cg_iters = h->h_iters[0] + h->h_iters[1];
    }
    const double mw = h->cfg.m * h->cfg.weight;
    out->step = h->step;
    out->t = (double)h->step * h->cfg.dt;
    out->np = h->np;
    out->fx_bits = h->fx_bits;
    out->charge_fx_sum = *h->h_accsum;
    out->total_charge = h->cfg.q * h->cfg.weight * ldexp((double)*h->h_accsum, -h->fx_bits);
    out->kinetic = 0.5 * mw * h->h_diag[0];
    for (int a = 0; a < 3; ++a) out->momentum[a] = mw * h->h_diag[1 + a];
    out->field_energy = 0.5 * h->dV * h->h_diag[4];
    out->cg_iters = h->last_cg_iters;
    out->cg_relres = h->last_cg_relres;
    out->error_flags = *h->h_err;
    for (int k = 0; k < 3; ++k) out->mcc_counts[k] = h->d_mcc ? h->h_accsum[1 + k] : 0;
    return AP_PIC_OK;
}

extern "C" ap_pic_status ap_pic_set_timing(ap_pic *h, int enable)
{
    if (!h) return AP_PIC_ERR_ARG;
    drain_marks(h);
    for (int k = 0; k < AP_PIC_NSTAGES; ++k) {
        h->stage_ms[k] = 0.0;
        h->stage_n[k] = 0;
    }
    h->timing = enable != 0;
    return AP_PIC_OK;
}

extern "C" ap_pic_status ap_pic_get_timing(ap_pic *h, double *ms, int64_t *count)
{
    if (!h) return AP_PIC_ERR_ARG;
    drain_marks(h);
    for (int k = 0; k < AP_PIC_NSTAGES; ++k) {
        if (ms) ms[k] = h->stage_ms[k];
        if (count) count[k] = h->stage_n[k];
    }
    return AP_PIC_OK;
}

extern "C" int64_t ap_pic_kernel_launches(void) { return g_launches.load(); }

extern "C" int64_t ap_pic_num_particles(const ap_pic *h) { return h ? h->np : 0; }

extern "C" const char *ap_pic_last_error(const ap_pic *h) { return h ? h->err.c_str() : ""; }

extern "C" const char *ap_pic_version(void) { return "ap_pic 0.1 (sm_103a)"; }
