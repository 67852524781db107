/*
 * ap_pic.h -- C ABI of the B300 electrostatic particle-in-cell hot path.
 *
 * The library advances one (or a batch of) periodic electrostatic PIC
 * instance(s) on one CUDA device.  The cycle is the one of the AlgoPlasma
 * paper's worked example (Sec. 3.1, Listing 1):
 *
 *   load:  initialise particles (I01) -> update the field -> initial half push
 *   step:  push velocities (C01 gather + A01 Boris) -> move + periodic wrap
 *          -> update the field (B01 deposit -> D02 Poisson -> D05/D06 E)
 *
 * Physics conventions (Debye units, eps0 = 1):
 *   - node-centred periodic grid: node j_a sits at x = j_a dx_a, L_a = n_a dx_a;
 *     flat node index j0 + n0 (j1 + n1 j2) (axis 0 fastest);
 *   - linear (cloud-in-cell) weights for both deposit and gather;
 *   - -lap_h(phi) = rho - mean(rho) with the (2 ndim + 1)-point Laplacian,
 *     phi of zero mean, E = -grad_h(phi) by centred differences;
 *   - Boris velocity advance (Sec. 2.2, A_Pusher); with B0 = 0 it is the
 *     leapfrog kick;  the initial half push is a Boris step of -dt/2.
 *
 * Storage (precision AP_PIC_FP32_CELLOFF): each particle is an int32 linear
 * cell index plus FP32 in-cell offsets in [0, 1) per axis and FP32
 * velocities; charge is accumulated as int64 fixed point (2^S per particle,
 * exactly), so the deposit is run-to-run deterministic and conserves the
 * total charge bit for bit.  AP_PIC_FP64_PLAIN keeps FP64 positions and
 * velocities instead (comparison form).
 *
 * Conventions for every call:
 *   - Return value: AP_PIC_OK or a negative ap_pic_status; no call aborts or
 *     exits.  ap_pic_last_error() gives a one-line reason.
 *   - Asynchrony: compute calls are enqueued on the handle's stream and return
 *     without waiting; calls that copy into host buffers (ap_pic_get_*)
 *     synchronise the stream first.
 *   - Device-detected errors (non-finite particle state, a CG solve that did
 *     not converge) are latched on the device and reported by the next
 *     synchronising call; once latched they stay until ap_pic_destroy.
 *   - Ownership: the caller owns every host buffer it passes; the library owns
 *     all device memory, obtained through the optional allocator (NULL:
 *     cudaMalloc / cudaFree).
 *   - Threading: a handle may be used by one host thread at a time.
 */
#ifndef AP_PIC_H
#define AP_PIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    AP_PIC_OK = 0,
    AP_PIC_ERR_ARG = -1,           /* invalid argument or configuration        */
    AP_PIC_ERR_UNSUPPORTED = -2,   /* valid but not implemented (e.g. bc)      */
    AP_PIC_ERR_NOMEM = -3,         /* device allocation failed                 */
    AP_PIC_ERR_CUDA = -4,          /* a CUDA runtime call failed               */
    AP_PIC_ERR_NOT_CONVERGED = -5, /* field solve hit cg_maxit                 */
    AP_PIC_ERR_BOUNDS = -6,        /* non-finite or out-of-range particle      */
    AP_PIC_ERR_STATE = -7,         /* call out of order (e.g. step before load) */
    AP_PIC_ERR_TOO_LARGE = -8      /* size beyond a fixed capacity              */
} ap_pic_status;

enum { AP_PIC_BC_PERIODIC = 0 };

enum {
    AP_PIC_FP32_CELLOFF = 0,  /* int32 cell + FP32 offsets/velocities (default)   */
    AP_PIC_FP64_PLAIN = 1     /* FP64 positions/velocities, no sort, no tiling     */
};

/* Field solver of the FP32 form (the FP64 plain form always uses the CG). */
enum {
    AP_PIC_SOLVER_CG = 0,   /* Jacobi-preconditioned CG (D02, Sec. 2.2), default        */
    AP_PIC_SOLVER_FFT = 1   /* spectral solve of the same discrete equation: phi_hat =
                               rho_hat / K^2 with K^2 the Fourier symbol of the (2d+1)-
                               point Laplacian; exact, no iteration.  Every n[a] must be
                               <= AP_PIC_FFT_MAX_N (other lengths than powers of two use
                               Bluestein's chirp-z form)                               */
};
#define AP_PIC_FFT_MAX_N 4096

/* Particle pusher (A_Pusher, Sec. 2.2, which lists the Boris and Higuera-Cary
 * pushers).  With AP_PIC_PUSHER_HIGUERA_CARY the stored (and loaded) velocities
 * are the momenta per mass u = gamma v, positions advance with u / gamma, and the
 * kinetic energy is m w sum (gamma - 1) c^2; the FP32 form only. */
enum {
    AP_PIC_PUSHER_BORIS = 0,          /* Boris / leapfrog (A01), default          */
    AP_PIC_PUSHER_HIGUERA_CARY = 1    /* relativistic, volume-preserving, exact
                                         E x B drift                            */
};

/* ap_pic_load flags */
enum { AP_PIC_LOAD_NO_HALFPUSH = 1u };

typedef struct {
    int ndim;              /* 1, 2 or 3 spatial dimensions                        */
    int n[3];              /* nodes (= cells) per axis; unused axes ignored        */
    double dx[3];          /* node spacing per axis (> 0)                          */
    double dt;             /* time step                                            */
    double q, m;           /* species charge and mass (electrons: -1, 1)           */
    double weight;         /* physical particles per macro-particle (> 0)          */
    double rho_background; /* uniform immobile charge density; NaN: neutralise the
                              loaded particles exactly (-q w np / V)              */
    double E0[3], B0[3];   /* uniform external fields; B0 enters the Boris turn    */
    int bc;                /* AP_PIC_BC_PERIODIC only                              */
    int precision;         /* AP_PIC_FP32_CELLOFF or AP_PIC_FP64_PLAIN             */
    int nv;                /* stored velocity components, ndim <= nv <= 3; nv must
                              be 3 when B0 != 0                                    */
    int sort_every;        /* ap_pic_step sorts by cell every this many steps (0:
                              never); ignored by AP_PIC_FP64_PLAIN                 */
    int fx_bits;           /* fixed-point fraction bits S of the charge accumulator:
                              each particle deposits exactly 2^S.  FP32 form: 0 means
                              22, which is also the maximum (its FP32 weights are
                              rounded to 2^-S without a float-to-int conversion,
                              exact up to 2^22).  FP64 plain form: 0 means 40, at
                              most 52.  Always capped at 62 - bitlen(np) so the
                              int64 sum cannot overflow                            */
    double cg_rtol;        /* field-solve relative residual target (0: 1e-6)      */
    int cg_maxit;          /* field-solve iteration cap (0: 20000)                 */
    int brick[3];          /* sort brick in cells per axis (0: library default:
                              64 in 1D, 8 per axis in 2D and 3D, 4 per axis in the 3D
                              electromagnetic step, whose particle kernel's fixed
                              deposit windows need compact tiles)                     */
    int diag_every;        /* diagnostics every this many steps (0: every step)    */
    int solver;            /* AP_PIC_SOLVER_CG (default) or AP_PIC_SOLVER_FFT; both
                              end with one FP64-residual refinement pass           */
    int pusher;            /* AP_PIC_PUSHER_BORIS (default) or _HIGUERA_CARY        */
    double c_light;        /* speed of light in the run's units, for the Higuera-
                              Cary pusher (0: infinite, the non-relativistic limit)
                              and the electromagnetic step (required there)         */
    int em;                /* 0: electrostatic (default); 1: the electromagnetic step
                              (E_Maxwell, Sec. 2.2): periodic 2D3V or 3D Yee grid, E
                              and B at integer times (B split in two half steps
                              around the E update), Esirkepov charge-conserving
                              current, Boris with the gathered B (+ B0).  The load's E
                              is the Poisson field of the loaded charge, B = 0.
                              Needs ndim = 2 or 3, nv = 3, the FP32 form, the Boris
                              pusher and c dt sqrt(sum_a 1/dx_a^2) < 1 (and moves
                              under one cell per step); ap_pic_step advances it
                              (the gather_push / deposit / push_deposit /
                              solve_field calls do not apply), ap_pic_get_E then
                              returns the 3 staggered components and ap_pic_get_B
                              the magnetic field                                  */
    int em_boundary;       /* with em = 1: 0 periodic (default); 1 (2D only) a
                              convolutional PML (Roden and Gedney, the CPML of
                              E_Maxwell) of pml_cells cells on every side, backed by
                              a conducting wall: a non-periodic grid, with or
                              without particles (a prescribed current may drive it:
                              ap_pic_set_current).  Graded profiles, depth d in
                              [0, 1]: sigma = 0.8 (m + 1) c / dx d^3, kappa = 1,
                              alpha = 0.  Particles live in [0, (n0 - 1) dx) x
                              [0, (n1 - 1) dy) (a load outside it is
                              AP_PIC_ERR_BOUNDS); fields start at zero (no Poisson
                              solve); gathers, current and charge leave out the
                              nodes outside the grid; a particle that leaves the box
                              deposits the current of its whole move and is
                              absorbed: marked (cell -1) until the next sort, which
                              drops it (np decreases).  rho's background is
                              rho_background (NaN: the neutralising density of the
                              particles present)                                   */
    int pml_cells;         /* PML thickness in cells (0: 12); 2 pml_cells < n[a]    */
} ap_pic_config;

typedef struct {
    /* Returns device memory of `bytes` bytes (>= 256-byte aligned) or NULL. */
    void *(*alloc)(size_t bytes, void *ctx);
    void (*free)(void *ptr, size_t bytes, void *ctx);
    void *ctx;
} ap_pic_allocator;

typedef struct {
    int64_t step;           /* steps taken since load                            */
    double t;               /* simulated time = step * dt                        */
    int64_t np;             /* particles                                         */
    int fx_bits;            /* S in use                                          */
    int64_t charge_fx_sum;  /* sum of the int64 accumulator; np * 2^S when exact  */
    double total_charge;    /* q w (charge_fx_sum / 2^S)                          */
    double kinetic;         /* (1/2) m w sum |v|^2, time-centred at the last push
                               (mean of the two half-step energies)               */
    double field_energy;    /* (1/2) dV sum_j |E_j|^2 of the current field        */
    double momentum[3];     /* m w sum v after the last push                      */
    int cg_iters;           /* iterations of the last field solve                 */
    double cg_relres;       /* its final relative residual                        */
    int error_flags;        /* latched device error bits (AP_PIC_EFLAG_*)         */
    int64_t mcc_counts[3];  /* collisions of the last collision pass: elastic,
                               excitation, and candidates whose frequency exceeded
                               the null-collision bound (0 without collisions)      */
} ap_pic_diag;

enum {
    AP_PIC_EFLAG_NONFINITE = 1,     /* a particle's offset or velocity was not finite */
    AP_PIC_EFLAG_CG = 2,            /* a field solve stopped at cg_maxit              */
    AP_PIC_EFLAG_OVERFLOW = 4,      /* a particle count exceeded the fixed-point range */
    AP_PIC_EFLAG_TIMEOUT = 8        /* a bounded device wait gave up (the pass stopped) */
};

typedef struct ap_pic ap_pic;

/* Fills *cfg with defaults (1D, 64 nodes, dx = 1, dt = 0.1, electrons, w = 1,
 * neutralising background, periodic, FP32 cell+offset, nv = 1, sort every 20). */
void ap_pic_config_default(ap_pic_config *cfg);

/* Creates an instance on the current CUDA device.  `cuda_stream` is a
 * cudaStream_t (NULL: the legacy default stream).  `alloc` may be NULL.
 * The grid arrays are allocated here; particle arrays at ap_pic_load. */
ap_pic_status ap_pic_create(const ap_pic_config *cfg, const ap_pic_allocator *alloc,
                            void *cuda_stream, ap_pic **out);

/* The instance's configuration after validation, with every default resolved
 * (fx_bits is the value in use once particles are loaded). */
ap_pic_status ap_pic_get_config(const ap_pic *h, ap_pic_config *out);

/* Frees every device allocation and the handle (NULL is accepted). */
ap_pic_status ap_pic_destroy(ap_pic *h);

/* I01 + field update + initial half push (Sec. 3.1, Listing 1).
 * x: host FP64, np x ndim row-major, each coordinate in [0, L_a) (a value equal
 * to L_a is taken as 0; anything else outside is AP_PIC_ERR_BOUNDS).
 * v: host FP64, np x nv row-major.  The call copies x and v to the device,
 * converts them to the instance's storage, sorts by cell (FP32 form),
 * deposits, solves for E and, unless AP_PIC_LOAD_NO_HALFPUSH, moves v back
 * half a step (Boris with -dt/2).  Synchronises the stream. */
ap_pic_status ap_pic_load(ap_pic *h, int64_t np, const double *x, const double *v,
                          unsigned flags);

/* Loads an exact FP32 state (checkpoint restore): cell[np] linear cell
 * indices, off (np x ndim, row-major, each in [0, 1)), v (np x nv).  Host
 * buffers.  Then deposits and solves as ap_pic_load (no half push unless
 * flags lacks AP_PIC_LOAD_NO_HALFPUSH).  FP32_CELLOFF only. */
ap_pic_status ap_pic_load_state(ap_pic *h, int64_t np, const int32_t *cell, const float *off,
                                const float *v, unsigned flags);

/* C01 + A01 + position update (Sec. 3.1): gathers E at each particle, advances
 * v by a Boris step of dt and x by v dt with periodic wrap.  Does not deposit. */
ap_pic_status ap_pic_gather_push(ap_pic *h);

/* B01 (Sec. 2.2, Sec. 3.1): deposits the charge of the current positions into
 * the int64 fixed-point accumulator and converts it to rho (FP64, with the
 * background). */
ap_pic_status ap_pic_deposit(ap_pic *h);

/* The fused hot path: ap_pic_gather_push followed by ap_pic_deposit in one
 * pass over the particles (identical results, bit for bit). */
ap_pic_status ap_pic_push_deposit(ap_pic *h);

/* D02 + D05/D06 (Sec. 2.2, Sec. 3.1): solves -lap_h(phi) = rho - mean(rho) by
 * Jacobi-preconditioned CG (FP32 vectors, FP64 dot products, warm start from
 * the previous phi) and sets E = -grad_h(phi).  Synchronises the stream once
 * per block of iterations to test convergence. */
ap_pic_status ap_pic_solve_field(ap_pic *h);

/* Per-cell sort: stable reorder of the particle arrays by the brick-major
 * cell key (ties keep their order).  FP32_CELLOFF only; a no-op for FP64_PLAIN. */
ap_pic_status ap_pic_sort(ap_pic *h);

/* Capacity (particles) of ap_pic_sort_perm_noalloc. */
#define AP_PIC_NOALLOC_MAX_NP (1 << 20)

/* The per-cell sort permutation without allocating device memory.
 * The paper has no counterpart: this exists for callers that may not call
 * cudaMalloc -- a host framework that owns all of the device's memory through
 * its own pool, or a hot loop that cannot afford the device-wide
 * synchronisation of cudaMalloc/cudaFree.
 * Computes the same stable brick-major permutation as ap_pic_sort: perm[r] =
 * index in `cell` of the particle of rank r (ties keep input order).
 *   ndim, n[3], brick[3]: grid and sort brick as in ap_pic_config (brick 0:
 *       the library default of an electrostatic handle; bricks are capped by n);
 *   np: particles, 0 <= np <= AP_PIC_NOALLOC_MAX_NP, else AP_PIC_ERR_TOO_LARGE
 *       with no device work;
 *   cell: device, np int32 linear cell indices in [0, cells);
 *   perm: device, np int32 (output); both caller-owned;
 *   cuda_stream: cudaStream_t (NULL: legacy default stream); the call is
 *       asynchronous on it.
 * Scratch is one fixed array of ~17 MiB in device global memory, held by
 * every GPU that loads the library until the process exits.  The first call
 * on a device (with that device current) looks up the array's device address
 * and keeps it for the life of the process, so it must come before any stream
 * capture, and the entry point must not be called on a device again after
 * cudaDeviceReset there (the reset unloads the array; the kept address would
 * be stale).  All calls share the array and each overwrites it: calls that
 * overlap on the GPU race, so the caller must order them (one stream per
 * device, or explicit synchronisation). */
ap_pic_status ap_pic_sort_perm_noalloc(int ndim, const int n[3], const int brick[3], int64_t np,
                                       const int32_t *cell, int32_t *perm, void *cuda_stream);

/* nsteps full cycles: push+deposit (fused), sort when due, field solve,
 * diagnostics when due. */
ap_pic_status ap_pic_step(ap_pic *h, int nsteps);

/* Host copies (each synchronises the stream).
 * rho: cells doubles (total charge density incl. background).
 * E:   ndim x cells doubles, component-major.
 * phi: cells doubles. */
ap_pic_status ap_pic_get_rho(ap_pic *h, double *rho);
ap_pic_status ap_pic_get_E(ap_pic *h, double *E);
ap_pic_status ap_pic_get_phi(ap_pic *h, double *phi);
/* The raw int64 fixed-point accumulator of the last deposit (cells entries). */
ap_pic_status ap_pic_get_rho_fx(ap_pic *h, int64_t *acc);

/* Particle state in storage order; any pointer may be NULL.
 * cell: np int32; off: np x ndim float; v: np x nv float;
 * x: np x ndim double, reconstructed as (cell_a + off_a) dx_a (FP64_PLAIN:
 * the stored position; cell/off/v then come from it). */
ap_pic_status ap_pic_get_particles(ap_pic *h, int32_t *cell, float *off, float *v, double *x);
/* FP64 velocities of the FP64_PLAIN form (np x nv). */
ap_pic_status ap_pic_get_velocities_f64(ap_pic *h, double *v);

/* Permutation applied by the most recent sort: perm[r] = storage position,
 * before that sort, of the particle now at position r (np int64). */
ap_pic_status ap_pic_get_perm(ap_pic *h, int64_t *perm);

ap_pic_status ap_pic_get_diag(ap_pic *h, ap_pic_diag *out);

/* Stage timing with CUDA events recorded on the handle's stream.
 * ap_pic_set_timing(h, 1) starts recording an event pair around every stage
 * launched afterwards (and clears the totals); ap_pic_get_timing synchronises
 * and returns, per stage, the summed milliseconds and the number of timed
 * occurrences.  Arrays have AP_PIC_NSTAGES entries. */
enum {
    AP_PIC_STAGE_PUSH_DEPOSIT = 0, /* the particle pass (gather, push, move, deposit) */
    AP_PIC_STAGE_RHO = 1,          /* fixed point -> rho conversion                  */
    AP_PIC_STAGE_SORT = 2,         /* keys, radix passes, record gather              */
    AP_PIC_STAGE_FIELD = 3,        /* CG iterations and E                            */
    AP_PIC_STAGE_DIAG = 4,         /* diagnostics reduction                          */
    AP_PIC_NSTAGES = 8
};
ap_pic_status ap_pic_set_timing(ap_pic *h, int enable);
ap_pic_status ap_pic_get_timing(ap_pic *h, double *ms, int64_t *count);

/* Kernels this library has launched in the process so far (all handles). */
int64_t ap_pic_kernel_launches(void);

/* ---- null-collision Monte Carlo (G_collision, Sec. 2.2) --------------------------------
 * Electrons against a uniform neutral background of density `density`, with
 * constant cross sections: isotropic elastic scattering (energy loss
 * 2 (m/M) (1 - cos chi) of E) and excitation above `eps_exc` (loses eps_exc, then
 * scatters isotropically).  The null-collision method bounds the total frequency by
 * nu' = density (sigma_el + sigma_exc) vmax: a fraction 1 - exp(-nu' dt) of the
 * particles are candidates each step, and a candidate of speed v takes process j
 * with probability density sigma_j v / nu' (else a null collision); candidates
 * faster than vmax are counted in ap_pic_diag.mcc_counts[2].  Random draws come from
 * a counter-based generator keyed by (seed, step, particle id, draw): the output
 * function of SplitMix64 on seed + (counter + 1) 0x9E3779B97F4A7C15, counter =
 * step 2^34 + id 4 + draw, top 24 bits; particle ids are the load order and follow
 * the sort.  FP32 cell + offset form, nv = 3, Boris pusher. */
typedef struct {
    double density;     /* neutral density n_g (>= 0)                                */
    double sigma_el;    /* elastic cross section (>= 0)                              */
    double sigma_exc;   /* excitation cross section above eps_exc (>= 0)             */
    double eps_exc;     /* excitation threshold energy (>= 0)                        */
    double mass_ratio;  /* m / M of electron and neutral, in [0, 0.25]               */
    double vmax;        /* speed bound of the null-collision frequency (> 0)         */
    uint64_t seed;      /* generator key                                             */
} ap_pic_mcc;

/* Enables (c non-NULL) or disables collisions; before ap_pic_load (the ids are
 * allocated at load).  ap_pic_step then runs one collision pass after each
 * particle pass, drawing with the step number being completed (1 for the first). */
ap_pic_status ap_pic_set_collisions(ap_pic *h, const ap_pic_mcc *c);
/* One collision pass now, drawing with step number (steps taken + 1). */
ap_pic_status ap_pic_collide(ap_pic *h);

/* ---- batch: many independent instances advanced together ----------------------------
 * The serving form of the same cycle: `count` periodic instances of uneven grid
 * and particle counts (each 1D or 2D, nv = 2, B0 = 0, FP32 cell + offset form)
 * share one particle arena and one set of grid arenas.  Each step runs one
 * persistent particle pass per dimension class over the tiles of every
 * instance, the charge conversion, and the field solve of every instance:
 * with cfgs[0].solver = AP_PIC_SOLVER_CG in lockstep (same Jacobi-PCG and
 * refinement as a single instance; an instance that has converged drops out),
 * with AP_PIC_SOLVER_FFT the spectral solve of every instance in three passes.
 * The front of the step (particle pass to the first block of CG iterations, or
 * the whole field update with the spectral solve) is captured once as a CUDA
 * graph and replayed.  Instance i of a batch computes what a single instance with cfgs[i]
 * computes, within the single instance's tolerance. */
typedef struct ap_pic_batch ap_pic_batch;

typedef struct {
    int pass_ctas_per_sm;   /* CTAs per SM of the persistent particle pass (1..16;
                               at most one resident wave is launched)               */
    int item_cells;         /* nodes per work item of the grid kernels (multiple of
                               256, 256..65536; set before loading)                  */
    int sort_every;         /* steps between sorts (0: never)                         */
    int cg_iters_per_graph; /* CG iterations in each replayed block (1..256)          */
    int use_graph;          /* 1: capture and replay the step front as a CUDA graph   */
    int pass_threads;       /* threads per CTA of the particle pass: 128, 256 or 512  */
    int pass_per_thread;    /* particles per thread of the pass (tiles of
                               threads x per_thread particles): with 128 threads 2
                               or 4, with 256 threads 1, 2 or 3, with 512 threads 1 */
} ap_pic_batch_tuning;

void ap_pic_batch_default_tuning(ap_pic_batch_tuning *t);

/* cfgs: `count` configurations (validated as for ap_pic_create, plus the batch
 * limits above; solver, cg_rtol and cg_maxit are taken from cfgs[0]).  Allocates no
 * device memory yet (that happens at ap_pic_batch_load).  The batch enqueues its
 * work on a stream of its own, ordered after `cuda_stream` on entry to each call
 * and making `cuda_stream` wait for it on exit. */
ap_pic_status ap_pic_batch_create(int count, const ap_pic_config *cfgs,
                                  const ap_pic_allocator *alloc, void *cuda_stream,
                                  ap_pic_batch **out);
ap_pic_status ap_pic_batch_destroy(ap_pic_batch *b);

/* Loads every instance at once: np[i] particles, x[i] host FP64 (np[i] x ndim_i),
 * v[i] host FP64 (np[i] x 2); then sorts, deposits, solves and (unless
 * AP_PIC_LOAD_NO_HALFPUSH) applies the initial half push, as ap_pic_load. */
ap_pic_status ap_pic_batch_load(ap_pic_batch *b, const int64_t *np, const double *const *x,
                                const double *const *v, unsigned flags);

/* nsteps cycles of every instance (sort every tuning.sort_every steps). */
ap_pic_status ap_pic_batch_step(ap_pic_batch *b, int nsteps);

/* The parts of a step, for timing them apart (a step is push_deposit, a sort
 * when due, then solve_field; none of these advances the step counter):
 *   push_deposit: one particle pass of every instance (gather, push, move,
 *                 deposit, Sec. 3.1 steps of Listing 1) and the charge conversion;
 *   sort:         the stable sort of every instance's particles by brick-major key;
 *   solve_field:  the Jacobi-PCG solve of every instance, its refinement pass, E
 *                 and the diagnostics.
 * Stream-ordered and asynchronous like ap_pic_batch_step; errors latched on the
 * device surface at the next read-back. */
ap_pic_status ap_pic_batch_push_deposit(ap_pic_batch *b);
ap_pic_status ap_pic_batch_sort(ap_pic_batch *b);
ap_pic_status ap_pic_batch_solve_field(ap_pic_batch *b);

ap_pic_status ap_pic_batch_set_tuning(ap_pic_batch *b, const ap_pic_batch_tuning *t);
ap_pic_status ap_pic_batch_get_tuning(const ap_pic_batch *b, ap_pic_batch_tuning *t);

/* Picks the particle pass's shape (pass_threads x pass_per_thread),
 * pass_ctas_per_sm, cg_iters_per_graph (CG solver only) and sort_every for this
 * batch by a coordinate search, timing `steps_per_trial` steps of each candidate
 * (the batch advances while it is tuned).  With a non-NULL cache_path, a result stored there for the same
 * batch shape and GPU is reused, and a new one is written back. */
ap_pic_status ap_pic_batch_autotune(ap_pic_batch *b, int steps_per_trial, const char *cache_path);

/* Per-instance read-back (host buffers; each synchronises), as the single-instance
 * calls of the same names. */
ap_pic_status ap_pic_batch_get_rho(ap_pic_batch *b, int i, double *rho);
ap_pic_status ap_pic_batch_get_E(ap_pic_batch *b, int i, double *E);
ap_pic_status ap_pic_batch_get_particles(ap_pic_batch *b, int i, int32_t *cell, float *off,
                                         float *v, double *x);
ap_pic_status ap_pic_batch_get_perm(ap_pic_batch *b, int i, int64_t *perm);
ap_pic_status ap_pic_batch_get_diag(ap_pic_batch *b, int i, ap_pic_diag *out);
int64_t ap_pic_batch_num_particles(const ap_pic_batch *b, int i);
const char *ap_pic_batch_last_error(const ap_pic_batch *b);

/* A prescribed current density (3 x cells doubles, staggered like E) added to the
 * particles' current in every following electromagnetic step (em = 1), until set
 * again; NULL clears it. */
ap_pic_status ap_pic_set_current(ap_pic *h, const double *J);

/* The magnetic field of the electromagnetic step (em = 1): 3 x cells doubles,
 * component-major, Bx at (i, j+1/2), By at (i+1/2, j), Bz at (i+1/2, j+1/2). */
ap_pic_status ap_pic_get_B(ap_pic *h, double *out);

/* Number of particles loaded (0 before ap_pic_load). */
int64_t ap_pic_num_particles(const ap_pic *h);

/* Last error message of the handle ("" if none); valid until the next call. */
const char *ap_pic_last_error(const ap_pic *h);

/* Library version string. */
const char *ap_pic_version(void);

#ifdef __cplusplus
}
#endif

#endif /* AP_PIC_H */
