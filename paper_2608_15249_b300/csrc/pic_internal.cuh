// pic_internal.cuh -- shared declarations of the CUDA translation units of the
// electrostatic PIC library (device-side parameter blocks, launcher
// prototypes).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>

#include "ap_pic.h"

namespace apk {

// Counts kernel launches (process-wide); every launcher calls it once per kernel.
void note_launch(int n = 1);

// Runs the set-up `f` (a kernel attribute, which is per device) once for the
// current device, marking it in `done` (one bit per device); thread-safe.
template <class F>
inline cudaError_t once_per_device(std::atomic<unsigned long long> &done, F &&f)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
    static std::mutex m;
    std::lock_guard<std::mutex> lock(m);
    if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
    e = f();
    if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_release);
    return e;
}

// Division by a loop-invariant divisor d >= 2 through a multiply-high
// (Granlund and Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994, the round-up variant for unsigned operands):
//   l = ceil(log2 d),  m = floor(2^32 (2^l - d) / d) + 1,
//   q = (t + ((x - t) >> 1)) >> (l - 1),  t = umulhi(m, x),   valid for x < 2^31.
struct FastDiv {
    uint32_t d, m;
    int l;
};

#ifdef __CUDACC__
__host__ __device__
#endif
inline FastDiv make_fastdiv(uint32_t d)
{
    FastDiv f{d, 0u, 0};
    if (d < 2) return f;
    int l = 0;
    while ((uint64_t(1) << l) < d) ++l;
    f.l = l;
    f.m = (uint32_t)(((uint64_t(1) << 32) * ((uint64_t(1) << l) - d)) / d + 1);
    return f;
}

#ifdef __CUDACC__
__device__ __forceinline__ uint32_t fdiv(uint32_t x, const FastDiv &f)
{
    if (f.d == 1) return x;
    const uint32_t t = __umulhi(f.m, x);
    return (t + ((x - t) >> 1)) >> (f.l - 1);
}
#endif

// Everything a particle kernel needs about the grid and the push, by value.
struct GridParams {
    int ndim;
    int n[3];          // nodes per axis (unused axes 1)
    FastDiv div0, div1; // division by n[0] and n[1] (cell index decode)
    float dtdx[3];     // dt / dx_a in FP32 (position update in cell units)
    float qmh2;        // (q/m) h / 2 for the step h of this launch
    float E0[3];       // uniform external field
    float t[3];        // Boris t = (q/m) B0 h / 2
    float s[3];        // Boris s = 2 t / (1 + |t|^2)
    int fx_bits;       // S
    int magnetised;    // B0 != 0
    int pusher;        // AP_PIC_PUSHER_*
    float inv_c2;      // 1 / c^2 of the Higuera-Cary pusher (0: non-relativistic)
};

// Error bits latched in the device word (same values as AP_PIC_EFLAG_*).
enum : int { EF_NONFINITE = 1, EF_CG = 2, EF_OVERFLOW = 4, EF_TIMEOUT = 8 };

// ---- particle kernels (pic_particles.cu) --------------------------------------------------
struct ParticlesF32 {
    int32_t *cell;     // [stride] (np used)
    float *off;        // [ndim][stride]
    float *v;          // [nv][stride]
    int64_t np;
    int64_t stride;    // np rounded up to a multiple of 64: every component array starts
                       // 256-byte aligned and may be read (TMA) up to a multiple of 16 bytes
    int nv;
    uint32_t *id;      // [stride] particle ids (load order), only with collisions; else null
};

// An int64 as FP32 with no conversion instruction (those issue on this GPU's slow FP64
// pipe): the magnitude (below 2^62) in three 22-bit parts, each of which becomes a
// float exactly by the magic-number trick (bits of 1.5 * 2^23 plus the integer, less
// 1.5 * 2^23, exact below 2^22); the parts, all of one sign, are summed with two
// roundings, then the sign is applied.
__device__ __forceinline__ float i64_to_f32(long long a)
{
    const unsigned long long m = a < 0 ? 0ull - (unsigned long long)a : (unsigned long long)a;
    const int lo = (int)(m & 0x3FFFFF), mid = (int)((m >> 22) & 0x3FFFFF), hi = (int)(m >> 44);
    const float flo = __int_as_float(0x4B400000 + lo) - 12582912.0f;
    const float fmid = __int_as_float(0x4B400000 + mid) - 12582912.0f;
    const float fhi = __int_as_float(0x4B400000 + hi) - 12582912.0f;
    const float v = fmaf(fhi, 17592186044416.0f, fmaf(fmid, 4194304.0f, flo));  // 2^44, 2^22
    return a < 0 ? -v : v;
}

// Component stride for np particles.
inline int64_t soa_stride(int64_t np) { return ((np > 0 ? np : 1) + 63) / 64 * 64; }

struct DiagPartials {
    double *blocks;    // [nblocks][4]: kinetic, momentum x, y, z
    int nblocks;
};

// Converts host-layout FP64 positions/velocities (row-major, one chunk) into
// cell + FP32 offset + FP32 velocity storage at [first, first + count).
cudaError_t launch_load_convert(const GridParams &g, const double *dx, const double *x,
                                const double *v, ParticlesF32 p, int64_t first, int64_t count,
                                int *err_flags, cudaStream_t st);

// Copies an exact FP32 state (row-major host layout already on the device).
cudaError_t launch_load_state(const GridParams &g, const int32_t *cell, const float *off,
                              const float *v, ParticlesF32 p, int *err_flags, cudaStream_t st);

// One pass over the particles: optional gather+Boris push (step h encoded in g),
// optional move, optional deposit into acc, optional diagnostics partials.
cudaError_t launch_particle_pass(const GridParams &g, ParticlesF32 p, const float *E,
                                 unsigned long long *acc, bool push, bool move, bool deposit,
                                 DiagPartials diag, int *err_flags, cudaStream_t st);

// A tile of a batch: particles [start, start + count) of the arena, all of
// instance `inst` (count <= 512; start a multiple of 4).
struct BatchTile {
    int64_t start;
    int count;
    int inst;
};

// The particle pass over the tiles of many instances (one dimension class: ndim
// 1 or 2 with nv = 2), in kernel variant `variant` (batch_variant: CTA threads and
// particles per thread; tiles of at most threads * per_thread particles).
// inst_params: device array of per-instance tile parameters (make_tile_params);
// diag_tiles: [ntiles][4] per-tile sums or NULL.
cudaError_t launch_batch_pass(int ndim, int variant, const BatchTile *tiles, int64_t ntiles,
                              const void *inst_params, ParticlesF32 p, bool push, bool mv,
                              bool deposit, double *diag_tiles, int nblocks, int *err,
                              cudaStream_t st);
// Variant index of (threads per CTA, particles per thread), or -1 if there is none.
int batch_variant(int threads, int per_thread);
int batch_variant_count();
void batch_variant_shape(int variant, int *threads, int *per_thread);
size_t batch_tile_params_bytes();
void make_tile_params(void *dst, const GridParams &g, const float *E, unsigned long long *acc);

// Particles per tile of the particle pass in 1D and 2D (3 per thread of a
// 256-thread CTA; the batch packs its instances in tiles of the same size), and in
// 3D (2 per thread: the 3D pass needs more registers per particle).
constexpr int PASS_TILE = 768;
constexpr int PASS_TILE_3D = 512;
// The batch's tiles (one instance each, most of them small): 2 per thread, where the
// lighter per-thread state lets 5 CTAs share an SM.
constexpr int BATCH_TILE = 512;

// Number of blocks the particle pass uses for np particles with nv velocity
// components: one resident wave (the CTAs of the pass that fit an SM, times the
// SMs), fewer for small np.  Fixed for a handle, so the diagnostics reduction
// order is deterministic.
int particle_pass_blocks(int64_t np, int ndim, int nv);

// The same for the FP64 plain pass.
int plain_pass_blocks(int64_t np, int ndim);

// SMs of the current device (cached on first use).
int sm_count();

// Reconstruct positions (FP64) from cell + offset for host read-back.
cudaError_t launch_positions_f64(const GridParams &g, const double *dx, ParticlesF32 p,
                                 double *x, cudaStream_t st);

// ---- FP64 plain form (pic_plain.cu) --------------------------------------------------------
struct ParticlesF64 {
    double *x;         // [ndim][np]
    double *v;         // [nv][np]
    int64_t np;
    int nv;
};

struct GridParamsF64 {
    int ndim;
    int n[3];
    double dx[3];
    double inv_dx[3];
    double L[3];
    double dt;
    double qmh2;
    double E0[3], t[3], s[3];
    int fx_bits;
    int magnetised;
};

cudaError_t launch_plain_load(const GridParamsF64 &g, const double *x, const double *v,
                              ParticlesF64 p, int64_t first, int64_t count, int *err_flags,
                              cudaStream_t st);
cudaError_t launch_plain_pass(const GridParamsF64 &g, ParticlesF64 p, const double *E,
                              unsigned long long *acc, bool push, bool move, bool deposit,
                              DiagPartials diag, int *err_flags, cudaStream_t st);

// ---- sort (pic_sort.cu) ---------------------------------------------------------------------
constexpr int SORT_TILE = 4096;             // items per radix tile
constexpr int SORT_MAX_DIGIT_BITS = 10;     // widest radix digit
constexpr int SORT_MAX_RADIX = 1 << SORT_MAX_DIGIT_BITS;

struct SortScratch {
    uint32_t *keys[2];
    uint32_t *idx[2];
    uint32_t *hist;        // 256 * ntiles
    uint32_t *scan_tmp;    // scan partials
    size_t scan_tmp_len;
    int64_t capacity;      // particles
};

size_t sort_hist_len(int64_t np);
size_t sort_scan_tmp_len(size_t n);

// Computes keys, sorts (stable LSD radix, digits of up to 10 bits) and leaves the
// final permutation in s.idx[*perm_slot].
cudaError_t launch_sort_perm(const GridParams &g, const int brick[3], int key_bits,
                             const int32_t *cell, int64_t np, SortScratch &s, int *perm_slot,
                             cudaStream_t st);
// The radix passes alone, on keys already in s.keys[0] (key_bits wide).
cudaError_t launch_sort_keys(int key_bits, int64_t np, SortScratch &s, int *perm_slot,
                             cudaStream_t st);
// dst[r] = src[perm[r]] for the SoA particle record.
cudaError_t launch_apply_perm(const uint32_t *perm, ParticlesF32 src, ParticlesF32 dst,
                              int ndim, cudaStream_t st);
cudaError_t launch_exclusive_scan_u32(const uint32_t *in, uint32_t *out, size_t n, uint32_t *tmp,
                                      cudaStream_t st);

// ---- field (pic_field.cu) -------------------------------------------------------------------
struct FieldBufs {
    int ndim;
    int n[3];
    FastDiv div0, div1;        // division by n[0], n[1] (node coordinates)
    int64_t cells;
    double dx[3];
    unsigned long long *acc;   // int64 fixed point: the latest deposit
    unsigned long long *acc_spare;  // the other accumulator, zero between steps (the
                               // step deposits into it, converts it while clearing the
                               // previous one, and the two trade places)
    float *b;                  // rho - mean(rho), FP32 (rho itself, in FP64, is formed
                               // from acc where it is read)
    float *phi, *r, *p, *q;    // CG vectors
    float *p2;                 // the cooperative CG's second buffers: r2 of r, q and w2
    float *r2, *w2, *s2;       // of w = c A r, p2 and s2 of s = A p (ping-pong, see
                               // k_cg_coop)
    unsigned *gbar;            // grid barrier of the cooperative solve (count, generation)
    float *x;                  // correction of the refinement step
    float *E;                  // interleaved, Estride floats per node: 1D and 2D the
                               // node's field and its upper x-neighbour's (2, 4),
                               // 3D (Ex, Ey, Ez, 0)
    int Estride;
    double *part[3];           // reduction partials (ping-pong + spare), nblocks each
    double *cgpart[2][5];      // the cooperative CG's partials: two sets, for alternate
                               // reductions (a block may write the next reduction's
                               // partials while another still reads this one's)
    int nblocks;
    double *scal;              // device scalars, see pic_field.cu
    int *done;                 // CG done flag
    int *iters;                // CG iteration count
    long long *isum_part;      // int64 partials for the accumulator sum
    double *fe_part;           // field-energy partials
    unsigned *ticket;          // blocks of k_residual64 finished (zero between launches)
};

int field_blocks(int64_t cells);

// b = scale (acc - mean(acc)) in FP32, with mean(acc) = mean_q + mean_r (its integer
// part and fraction: every particle deposits exactly 2^S, so the mean is known before
// the deposit), formed without FP64 arithmetic; partial sums of acc.  rho itself,
// scale acc + bg in FP64, is formed where it is read (the refinement's residual, the
// read-back).
cudaError_t launch_rho_convert(FieldBufs &f, long long mean_q, float mean_r, float scale,
                               unsigned long long *clear, cudaStream_t st);
// The whole Jacobi-PCG solve of A x = b (warm start x) as one cooperative launch,
// convergence tested on the device: iterations to *iters, final relative residual
// to scal[relres_slot]; the cap is maxit - *it_used when it_used is given; latch:
// EF_CG when the residual stays above rtol.  A grid barrier that gives up latches
// EF_TIMEOUT.
cudaError_t launch_cg_solve(FieldBufs &f, const float *b, float *x, double rtol, int maxit,
                            const int *it_used, int *iters, int relres_slot, bool latch,
                            int *err_flags, cudaStream_t st);
// Refinement: b = (float)(rho - mean - A phi) computed in FP64 with rho = scale acc +
// bg, and its relative norm |rho - mean - A phi| / |rho - mean| into scal[SCAL_TRUE_REL].
cudaError_t launch_residual64(FieldBufs &f, double scale, double bg, double mean_total,
                              cudaStream_t st);
// phi += x
cudaError_t launch_add_correction(FieldBufs &f, cudaStream_t st);
enum : int { SCAL_TRUE_REL = 4, SCAL_BNORM64 = 5, SCAL_CG_REL = 3, SCAL_CG_REL2 = 6 };
cudaError_t launch_efield(FieldBufs &f, cudaStream_t st);

// ---- electromagnetic step (pic_em.cu) -----------------------------------------------------------
struct EmBufs {
    float *E, *B;              // [3][cells] Yee-staggered fields at integer time
    unsigned long long *J;     // [3][cells] fixed-point current weights (2^22 per unit)
    float *Jext;               // [3][cells] prescribed current added each step, or null
    float B0[3];               // uniform external B added to the gathered one
    // convolutional PML (non-periodic grid), null when periodic:
    // profiles b, c, 1/kappa per axis, at half positions for the B half steps
    // (pb[0..2] along x, pb[3..5] along y) and integer positions for the E step (pe)
    const float *pb[6], *pe[6];
    float *psib[4], *psie[4];  // Bx_y, By_x, Bz_x, Bz_y;  Ex_y, Ey_x, Ez_x, Ez_y
    // per particle tile of the step kernel: 1 when its particles were too spread out
    // for the shared-memory windows (handled particle by particle), else 0
    unsigned char *tile_flag;
    // 3D: per particle tile, the number of its particles left to the global-memory
    // kernel (the same allocation as tile_flag, two bytes per tile)
    unsigned short *tile_spill;
};
// Particles per tile of the electromagnetic step kernel (one per thread).
constexpr int EM_PASS_TILE = 256;
// Blocks of one resident wave of the step kernel; the handle keeps twice as many
// diagnostic slots (the tiled kernel's and the spread-out tiles').
int em_particle_blocks(int64_t np);
// Gather, Boris with the gathered B, and (move) the move, Esirkepov current and the
// charge at the new positions (into rho_acc).
cudaError_t launch_em_push(const GridParams &g, ParticlesF32 p, const EmBufs &em, bool move,
                           unsigned long long *rho_acc, double *diag_blocks, int nblocks,
                           int *err, cudaStream_t st);
// J from its accumulator (cleared), then B -= (dt/2) curl E; E += dt (c^2 curl B - J);
// B -= (dt/2) curl E.
// Particles in the non-periodic mode (absorbing layer, conducting walls): gather
// with fields outside the grid zero, Boris, and with move the move, the Esirkepov
// current (contributions outside the grid dropped), the charge of the particles
// still in the box; a particle that leaves the box gets cell -1 and is counted in
// *n_absorbed.  The check latches EF_NONFINITE for a loaded particle outside the box.
cudaError_t launch_em_np_push(const GridParams &g, ParticlesF32 p, const EmBufs &em, bool move,
                              unsigned long long *rho_acc, double *diag_blocks, int nblocks,
                              int *err, unsigned long long *n_absorbed, cudaStream_t st);
cudaError_t launch_em_np_check(const GridParams &g, ParticlesF32 p, int *err, cudaStream_t st);
// The 3D electromagnetic step (pic_em3.cu): particles (gather E, B on the 3D Yee
// lattice, Boris, and with move the move, the 3D Esirkepov current and the charge),
// the field update, and the load's E from phi.
// Blocks of one resident wave of the 3D tiled particle kernel; the handle keeps twice
// as many diagnostic slots (the tiled kernel's and the listed particles' kernel's).
int em3_particle_blocks(int64_t np);
// spill_list: np int32 slots of scratch (free between sorts), for the particles the
// tiled kernel leaves to the global-memory kernel.
cudaError_t launch_em3_push(const GridParams &g, ParticlesF32 p, const EmBufs &em, bool move,
                            unsigned long long *rho_acc, double *diag_blocks, int nblocks,
                            int *err, int32_t *spill_list, cudaStream_t st);
cudaError_t launch_em3_fields(const GridParams &g, const EmBufs &em, const double *dx, double dt,
                              double c, double qw, cudaStream_t st);
cudaError_t launch_em3_e_from_phi(const GridParams &g, const float *phi, const EmBufs &em,
                                  const double *dx, cudaStream_t st);
cudaError_t launch_em_fields(const GridParams &g, const EmBufs &em, double dx, double dy,
                             double dt, double c, double qw, cudaStream_t st);
cudaError_t launch_em_e_from_phi(const GridParams &g, const float *phi, const EmBufs &em,
                                 double dx, double dy, cudaStream_t st);
cudaError_t launch_em_energy(const EmBufs &em, int64_t cells, double c, double *part, int nblocks,
                             cudaStream_t st);

// ---- null-collision Monte Carlo (pic_mcc.cu) ---------------------------------------------------
struct MccParams {
    uint64_t seed;
    uint32_t thr;          // candidate iff draw 0 < thr = round((1 - exp(-nu' dt)) 2^24)
    float ng_sig_el, ng_sig_exc;  // n_g sigma_j: nu_j = n_g sigma_j |v|
    float nu_max;          // nu' = n_g (sigma_el + sigma_exc) vmax
    float eps_exc;         // excitation threshold energy
    float two_eps_over_m;  // 2 eps_exc / m
    float two_mass_ratio;  // 2 m / M
    float half_m;          // m / 2
};
MccParams make_mcc_params(double density, double sigma_el, double sigma_exc, double eps_exc,
                          double mass_ratio, double vmax, double m, double dt, uint64_t seed);
// One null-collision pass over the particles (nv = 3, ids set) for time step `step`;
// counts[0..2] = elastic, excitation, candidates above the bound (zeroed first).
cudaError_t launch_mcc(ParticlesF32 p, const MccParams &c, uint64_t step,
                       unsigned long long *counts, cudaStream_t st);
cudaError_t launch_iota(uint32_t *id, int64_t np, cudaStream_t st);

// ---- spectral Poisson solve (pic_fft.cu) ------------------------------------------------------
constexpr int FFT_MAX_N = 4096;  // longest axis (power-of-two or Bluestein length <= 8192)
struct FftAxis {
    int n;                 // nodes on the axis
    int log2m;             // transform length m = 2^log2m in shared memory
    int bluestein;         // 1: n is not a power of two (chirp-z form, m >= 2n - 1)
    const float *lam;      // (2 sin(pi k / n) / dx)^2, k < n
    const float2 *chirp;   // exp(-i pi j^2 / n), j < n
    const float2 *bhat;    // length-m DFT of the chirp filter
    int64_t inner;         // stride of the axis (product of the lower axes' n)
};
struct FftPlan {
    int ndim;
    int64_t cells;
    FftAxis ax[3];
    float2 *Z;             // complex work array [cells]
    const float2 *tw;      // exp(-2 pi i t / M), t < M / 2
    int log2M;             // M: the longest transform length
    int sms;
};
enum : int { FFT_FWD = 0, FFT_INV = 1, FFT_FWD_SCALE_INV = 2 };
// A grid of a batch for the spectral solve, and a job: W lines of one of its axes.
struct FftGrid {
    int64_t node0;         // first node in the batch's grid arenas
    int ndim;
    FftAxis ax[2];
    FastDiv div_n0;
    float inv_cells;
};
struct FftJob {
    int grid, axis;
    int64_t l0;
    int nl, W;
};
int lines_per_cta(int64_t lines, int log2m, int sms, int cap);
size_t fft_smem_bytes(int W, int log2m, bool bluestein);
// Runs `jobs` (one pass of a batch's transform: every job in the same mode, except
// that 1D grids always take the fused forward / scale / inverse form and write their
// real result to out_1d).
cudaError_t launch_fft_jobs(const FftJob *jobs, int njobs, const FftGrid *grids, float2 *Z,
                            const float *in_real, float *out_real, float *out_1d,
                            const float2 *tw, int log2M, int mode, size_t smem, int blocks,
                            cudaStream_t st);
bool fft_length_ok(int n);
int fft_log2m(int n);  // log2 of the transform length of an axis of n nodes
size_t fft_axis_table_floats(int n);
void fft_axis_tables(int n, double dx, float *host, float *dev, FftAxis *ax);
size_t fft_twiddle_floats(int log2M);
void fft_twiddles(int log2M, float *host);
cudaError_t fft_configure();
// phi = the zero-mean solution of -lap_h phi = b (b's mean is ignored).
// phi = the zero-mean solution of -lap_h phi = b, or phi += it when accumulate.
cudaError_t launch_fft_poisson(const FftPlan &P, const float *b, float *phi, cudaStream_t st,
                               bool accumulate = false);
// Finalise diagnostics: reduce particle partials, accumulator sum, field energy
// into out[0..7] = {kinetic, px, py, pz, field_energy, acc_sum (as bits), -, -}.
cudaError_t launch_diag_finalize(const DiagPartials &pd, bool have_particles, FieldBufs &f,
                                 double *out, long long *acc_sum_out, cudaStream_t st);
cudaError_t launch_e_to_f64(FieldBufs &f, double *out, cudaStream_t st);
cudaError_t launch_phi_to_f64(FieldBufs &f, double *out, cudaStream_t st);

// ---- FP64 plain field path (pic_plain.cu) ---------------------------------------------------
struct FieldBufsF64 {
    int ndim;
    int n[3];
    FastDiv div0, div1;
    int64_t cells;
    double dx[3];
    unsigned long long *acc;
    double *rho, *b, *phi, *r, *p, *q, *E;   // E component-major [ndim][cells]
    double *part[3];
    int nblocks;
    double *scal;
    int *done, *iters;
    long long *isum_part;
    double *fe_part;
};
cudaError_t launch_plain_rho_convert(FieldBufsF64 &f, double scale, double bg, double mean_e,
                                     cudaStream_t st);
cudaError_t launch_plain_cg_init(FieldBufsF64 &f, double rtol, cudaStream_t st);
cudaError_t launch_plain_cg_iters(FieldBufsF64 &f, int first, int count, int maxit, double rtol,
                                  cudaStream_t st);
cudaError_t launch_plain_cg_finish(FieldBufsF64 &f, double rtol, int *err_flags, cudaStream_t st);
cudaError_t launch_plain_efield(FieldBufsF64 &f, cudaStream_t st);
cudaError_t launch_plain_diag_finalize(const DiagPartials &pd, bool have_particles,
                                       FieldBufsF64 &f, double *out, long long *acc_sum_out,
                                       cudaStream_t st);

}  // namespace apk
