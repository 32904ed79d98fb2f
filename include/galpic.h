/*
 * galpic.h - C ABI of the Galilean-PSATD particle-in-cell step (GB300, sm_103a).
 *
 * Method: Kirchen et al., "Stable discrete representation of relativistically
 * drifting plasmas" (arXiv:1608.00215). The particle-in-cell equations are
 * written in Galilean coordinates x' = x - v_gal t (the coordinate transform
 * and the transformed equations of motion and Maxwell equations at the start
 * of the method section); the spectral fields advance with the Galilean-PSATD
 * update (the update equations and the coefficient block C, S, nu, theta,
 * chi1, chi2, chi3 that follows them); one step deposits J at (n+1/2)dt and
 * rho at (n+1)dt, transforms them to Fourier space, updates E and B,
 * transforms back, interpolates to the particles and advances them (the
 * paragraph that follows the update equations).
 *
 * Conventions used by every call:
 *   - Grid: nx*ny*nz collocated nodes, periodic; real arrays are row-major
 *     [nx][ny][nz] (z contiguous). Spectral arrays are the R2C half spectrum
 *     [nx][ny][nz/2+1] of interleaved complex numbers (re, im).
 *   - Forward transform exp(-i k.x), inverse with 1/N; Nyquist planes of
 *     even axes are held at zero.
 *   - A particle sits at ((i + f_x) dx, (j + f_y) dy, (l + f_z) dz) with the
 *     linear cell index cell = (i*ny + j)*nz + l (int32) and offsets
 *     f in [0, 1); u = gamma v is the momentum per mass.
 *   - precision 32: offsets, momenta, grids and spectra are float; the
 *     coefficient tables are built in double and rounded to float.
 *     precision 64: everything is double.
 *   - Streams are cudaStream_t values passed as void* (NULL = legacy default
 *     stream). Every call is asynchronous on its stream unless it says
 *     otherwise.
 *   - Memory: the caller allocates ONE device workspace of pic_footprint()
 *     bytes and owns it; the library carves every grid, spectrum, table and
 *     particle array out of it and never calls cudaMalloc for them. The
 *     library owns only its cuFFT plans, one private stream, a CUDA graph
 *     and the small host handle (freed by pic_destroy).
 *   - Errors: every int-returning call returns PIC_OK (0) or a negative
 *     PIC_E* code and leaves a message for pic_last_error() (thread-local).
 *     Conditions that the device detects (non-finite field energy) are
 *     recorded in a device status word and reported by pic_status(). No
 *     call aborts the process.
 */
#ifndef GALPIC_H
#define GALPIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PIC_OK 0
#define PIC_EINVAL (-1)     /* invalid argument or configuration            */
#define PIC_ENOMEM (-2)     /* workspace smaller than pic_footprint()        */
#define PIC_ECUDA (-3)      /* a CUDA runtime call failed                    */
#define PIC_ETIMEOUT (-4)   /* a bounded device wait gave up                 */
#define PIC_ENONFINITE (-5) /* a diagnostic saw a NaN or infinity            */
#define PIC_EBOUNDS (-6)    /* an index left its buffer (checked build)      */
#define PIC_ECUFFT (-7)     /* a cuFFT call failed                           */

#define PIC_MAX_SPECIES 8

/* Status bits of the device status word (pic_status). */
#define PIC_STATUS_NONFINITE 1  /* a diagnostic saw a NaN or infinity                  */
#define PIC_STATUS_BADINPUT 2   /* loaded particles had a cell outside [0, N) or an
                                   offset outside [0, 1); they were clamped to cell 0 /
                                   offset 0 so that every kernel stays in bounds         */
#define PIC_STATUS_BOUNDS 4     /* checked build (libgalpic_checked.so, compiled with
                                   PIC_CHECKED): a particle, grid, tile or staging index
                                   was outside its buffer's logical range; the access was
                                   skipped. Never set by the ordinary build, which does
                                   not test indices                                      */

typedef struct pic_sim pic_sim;

/* Problem statement of one run (the paper's grid, time step and v_gal). */
typedef struct {
    double dx, dy, dz;          /* cell size                                          */
    double dt;                  /* time step                                          */
    double vgal[3];             /* Galilean frame velocity, |v_gal| < c               */
    double c;                   /* speed of light                                     */
    double eps0;                /* vacuum permittivity (mu0 = 1/(eps0 c^2))           */
    double rho_bg;              /* uniform background charge density that is static
                                   on the moving grid: adds rho_bg to rho and
                                   rho_bg*v_gal to J                                   */
    double beta_init[3];        /* drift velocity / c of the initial field            */
    int32_t nx, ny, nz;         /* grid nodes per axis, each >= 2                     */
    int32_t shape_order;        /* particle shape: B-spline of order 1, 2 or 3        */
    int32_t precision;          /* 32 or 64                                           */
    int32_t current_correction; /* 1: enforce the discrete Galilean continuity
                                   equation per mode on J before the update           */
    int32_t init_fields;        /* 0: E = B = 0; 1: field of rho^0 moving rigidly at
                                   beta_init*c (boosted Coulomb, satisfies Gauss)     */
    int32_t tile_margin;        /* 0 or 1: cells of shared-memory tile kept around each
                                   8x8x8 bin for particles that left it since the last
                                   sort (0: smaller tiles, any particle outside its bin
                                   takes the global-memory path and counts toward the
                                   re-sort threshold; 1: particles up to one cell out
                                   still use the tile)                                 */
    int32_t deposit;            /* deposit strategy. FP32 quadratic/cubic passes:
                                   0: grouped by cell, J and rho in separate group
                                   passes (many particles per cell), 1: by stencil row
                                   (few particles per cell), 2: grouped by cell, J and
                                   rho in one group pass, 3: by stencil row with the
                                   row's nodes in registers (z starts unrolled).
                                   Linear passes (FP32 or FP64): 0: grouped by cell, J
                                   and rho together, 4: one thread per cell, the cell's
                                   2x2x2 stencil accumulated in registers (particles at
                                   rest on the grid). Other combinations use 0; FP64
                                   quadratic/cubic passes always use 0. pic_tune picks. */
    int32_t stencil_order;      /* 0: spectral derivatives i k (the paper's solver);
                                   even p in [2, 128]: finite-order spectral stencil,
                                   every k_d of the update (curl, |k|, k.v_gal, current
                                   correction, initial field) replaced by the symbol of
                                   the centred difference of order p on the collocated
                                   grid, [k_d] = (2/d) sum_{l<=p/2} a_l sin(l k_d d)
                                   (the arbitrary-order solvers the paper's conclusion
                                   names for domain decomposition); 0 on Nyquist planes */
    int32_t deterministic;      /* 0: the deposit sums in floating point through
                                   atomics, so its rounding depends on the order in
                                   which threads add (results agree to rounding, not
                                   bit for bit); 1: every deposited value
                                   q w v S(x_node - x)/dV and q w S/dV is rounded to an
                                   integer multiple of delta = 2^e and summed as a 64-bit
                                   integer, e being the smallest integer with
                                   max(1, c) sum_s |q_s w_s| n_s / dV < 2^(62 + e) (no
                                   node's sum can overflow); integer sums do not depend on the
                                   order, so J, rho and every later stage are bitwise
                                   reproducible: a run gives the same bits alone, next
                                   to other runs, and continued from a checkpoint
                                   (pic_get / pic_set / pic_get_particles). The
                                   particle order inside a cell may still differ after a
                                   re-sort; the particles as a set do not. Uses the
                                   grouped deposit (pic_config.deposit is ignored) and
                                   4*N int64 of extra workspace. delta is far below FP32
                                   rounding; in FP64 runs a node's error is about delta
                                   times the square root of its number of contributions */
} pic_config;

/* One particle species. Particles are either generated on the device on a
 * regular lattice with seeded jitter (ppc[0] > 0) or copied from caller
 * arrays (host or device memory) at pic_init. */
typedef struct {
    double q;                   /* charge of one physical particle                    */
    double m;                   /* mass of one physical particle                      */
    double w;                   /* macro weight (physical particles per macro)        */
    double jitter;              /* generated: uniform jitter half-width in cells      */
    double u0[3];               /* generated: initial momentum per mass               */
    int64_t n;                  /* number of macro particles                          */
    uint64_t seed;              /* generated: random seed                             */
    int32_t ppc[3];             /* generated: lattice particles per cell per axis;
                                   n must equal nx*ny*nz*ppc[0]*ppc[1]*ppc[2]          */
    int32_t species_id;         /* generated: enters the random key (seed ^ id<<56)   */
    const int32_t* cell;        /* copied: linear cell index, n entries               */
    const void* off[3];         /* copied: offsets in [0,1), float or double          */
    const void* u[3];           /* copied: momentum per mass, float or double         */
} pic_species;

/* Buffers that pic_get / pic_set address. */
enum pic_buffer {
    PIC_BUF_E = 0,        /* real E^n, 3*N values (x, y, z planes)                      */
    PIC_BUF_B = 1,        /* real B^n, 3*N                                             */
    PIC_BUF_J = 2,        /* real J of the last particle pass, 3*N                       */
    PIC_BUF_RHO = 3,      /* real rho of the last particle pass, N                       */
    PIC_BUF_E_HAT = 4,    /* spectral E^n, 3*M complex                                 */
    PIC_BUF_B_HAT = 5,    /* spectral B^n, 3*M complex                                 */
    PIC_BUF_RHO_HAT = 6,  /* spectral rho^n, M complex                                  */
    PIC_BUF_SRC_HAT = 7,  /* spectra of the last sources (Jx, Jy, Jz, rho), 4*M complex  */
    PIC_BUF_TABLES = 8,   /* per-mode factors T1, T2, T3, T4, A5, A6, 6*M complex        */
    PIC_BUF_STATUS = 9    /* the device status word (int32, PIC_STATUS_* bits); reading it
                             with pic_get does not clear it and does not synchronise     */
};

/* Library version string. */
const char* pic_version(void);

/* Message of the last failed call on this thread ("" if none). */
const char* pic_last_error(void);

/* Bytes of device workspace that pic_init needs for this configuration.
 * Needs a CUDA device (it sizes the cuFFT work area). Returns PIC_EINVAL for
 * an invalid configuration. */
int pic_footprint(const pic_config* cfg, const pic_species* species, int nspecies,
                  size_t* bytes_out);

/* Create a run: validate, carve the caller-owned device workspace (at least
 * pic_footprint() bytes, 256-byte aligned), build the FP64 coefficient
 * tables, load or generate the particles and sort them into cell bins,
 * deposit rho^0, and set the initial fields. Enqueued on `stream`. When any
 * species is copied from caller arrays, the call then synchronises that stream
 * and returns PIC_EINVAL (and no run) if the particles were out of range
 * (PIC_STATUS_BADINPUT). The species array is read during the call only.
 * cuFFT plans are created once per grid shape and precision and shared by all
 * runs of that shape for the life of the process. */
int pic_init(const pic_config* cfg, const pic_species* species, int nspecies,
             void* workspace, size_t ws_bytes, void* stream, pic_sim** out);

/* Release the run's host handle, private stream, CUDA graph and events. The
 * workspace stays the caller's, and so do the shared cuFFT plans. The caller
 * must have completed (or synchronised) the work it enqueued for this run on its
 * own streams; the call does not synchronise the device. */
int pic_destroy(pic_sim* sim);

/* Deposit rho and J = sum q w v S / dV at the current positions x^n with the
 * current momenta into the real source grids (J, RHO buffers); the shape
 * factor of the paper's "deposited to the grid nodes". */
int pic_deposit(pic_sim* sim, void* stream);

/* The particle half of a step: gather E^n, B^n at x^n (interpolation to the
 * particles), relativistic Boris push u^{n-1/2} -> u^{n+1/2}, half Galilean
 * drift x' += (v - v_gal) dt/2, deposit J^{n+1/2}, second half drift, deposit
 * rho^{n+1}. Re-sorts the particles into cell bins first when the previous
 * pass left too many outside their bin. */
int pic_gather_push(pic_sim* sim, void* stream);

/* The field half of a step: forward R2C FFT of Jx, Jy, Jz, rho^{n+1};
 * optional current correction; Galilean-PSATD update of spectral E, B;
 * Nyquist zeroing; rho^n <- rho^{n+1}; inverse C2R FFT to the real E, B. */
int pic_field_update(pic_sim* sim, void* stream);

/* nsteps full steps (pic_gather_push then pic_field_update), replayed from a
 * CUDA graph captured on the first call. */
int pic_step(pic_sim* sim, int nsteps, void* stream);

/* Serving many runs: several runs of one grid shape advanced in shared launches (the
 * continuous-batching pattern of many small independent runs, which one GPU only keeps
 * busy when their work goes out together). Each step of every run goes through one launch
 * per stage for all of them: the re-sort check (per species slot), the particle pass (one
 * CTA per run and bin), one batched forward transform over all runs' sources, one k-space
 * update (one block row per run), one batched inverse transform; one such step of the set
 * is captured once as a CUDA graph (cached for this workspace and set of runs) and
 * replayed nsteps times. Each run's arithmetic is its single-run step's: results equal
 * pic_step's to rounding; in deterministic mode bitwise (those runs' transforms then use
 * their single-run cuFFT plans, one per run, since a batched plan may round differently).
 *   sims:      nsims (1 .. 4096) distinct runs with equal nx, ny, nz, precision, shape
 *              order, tile margin, deposit strategy (as chosen by pic_config.deposit or
 *              pic_tune), species count and deterministic mode; other parameters (cell
 *              size, dt, v_gal, c, species, stencil order, ...) may differ.
 *   workspace: caller-owned device memory, 256-byte aligned, of at least
 *              pic_many_footprint(sims[0], nsims) bytes: one slot per run (rounded up to a
 *              power of two) for the sources, their spectra, the inverse-transform input
 *              and the real E, B, plus the parameter tables and the FFT work area. Runs
 *              keep their state in their own workspaces; the call copies their real E, B
 *              in at the start and E, B, the sources and source spectra back at the end.
 *              Two calls that overlap on the GPU must not share a workspace.
 * Asynchronous on `stream`. The first call for a new set of runs (or a changed strategy)
 * creates the batched cuFFT plans for its slot count (shared for the life of the process)
 * and captures the step; pic_destroy forgets the captured steps of a destroyed run.
 * Errors: PIC_EINVAL (bad arguments, runs that cannot share launches), PIC_ENOMEM
 * (workspace too small), PIC_ECUDA, PIC_ECUFFT. */
int pic_many_footprint(const pic_sim* sim, int capacity, size_t* bytes_out);
int pic_step_many(pic_sim** sims, int nsims, int nsteps, void* workspace, size_t ws_bytes, void* stream);

/* Several plasmas, each on its own Galilean grid, sharing E and B (the
 * generalisation proposed in the paper's conclusion for counter-streaming
 * plasmas: separate grids in different Galilean coordinates, only the
 * electromagnetic field shared, by superposition). Each run's spectral state
 * holds the part of the field its own plasma drives, advanced by the
 * Galilean-PSATD update with its own v_gal; the grids coincide at t = 0, so
 * node x' of run j sits at x' + v_gal,j t. Every step pushes each run's
 * particles with the TOTAL field on its own nodes: the other runs' parts moved
 * onto its grid by the exact Fourier shift exp(i k.(v_gal,j - v_gal,i) t)
 * (spectral k, whatever the stencil order), added before its inverse FFT.
 *   sims:   nsims (1..16) distinct runs with equal nx, ny, nz, dx, dy, dz, dt,
 *           c, eps0 and precision, all at the same step count; the caller keeps
 *           ownership.
 *   nsteps: steps to take (>= 0; 0 only forms the total fields).
 * On return every run's real E, B (PIC_BUF_E, PIC_BUF_B) is the total field at
 * the new step; its spectral E, B stay its own part. Once coupled, runs should
 * only be stepped through this call (pic_step would advance one part alone and
 * gather only that part). Not graph-captured: each step enqueues each run's
 * particle pass, forward FFT and k-space update, then per run and per other run
 * two small kernels (shift phases, shifted add) and its inverse FFT.
 * Errors: PIC_EINVAL for a bad array, a repeated run, mismatched grids or step
 * counts; otherwise as pic_step. */
int pic_step_coupled(pic_sim** sims, int nsims, int nsteps, void* stream);

/* Domain decomposition of the field update along z, all subdomains on this GPU (the
 * paper's conclusion names decomposition with arbitrary-order spectral solvers as the route
 * to many processors). Each step: the ordinary particle pass (global deposit), then each of
 * the ndomains subdomains takes its nz/ndomains cells plus `guard` cells on either side
 * (periodic) of the real E, B, J, rho^{n+1} and rho^n as a periodic window, applies the
 * Galilean-PSATD update there with the window's own finite-order-stencil wavenumbers (the
 * Nyquist planes of a window are updated like any mode), and keeps its own cells. All
 * windows go through one gather kernel, one batched R2C, one k-space launch, one batched C2R
 * and one scatter kernel. The real E, B are the state between steps; rho^n is the last
 * deposit's rho (PIC_BUF_RHO). At the end of the call the run's spectral E, B, rho^n and
 * source spectra are refreshed as the forward transforms of the real state (whose inverse
 * transform gives the real state back), so that pic_step can continue from it.
 *   ndomains: >= 1, divides nz; guard: >= 0 cells; with ndomains > 1 the run must have
 *             current_correction = 0 (its 1/k^2 reaches the whole grid) and a finite
 *             stencil_order (the spectral solver's update has unbounded reach).
 *   workspace: caller-owned device memory, 256-byte aligned, of at least
 *             pic_decomposed_footprint() bytes (windows, their spectra, the window factors,
 *             the FFT work area). The window factors are rebuilt at every call (FP64).
 * The batched window plans are created on first use per window shape and kept for the life
 * of the process. Asynchronous on `stream`. Errors: PIC_EINVAL, PIC_ENOMEM, PIC_ECUDA,
 * PIC_ECUFFT. */
int pic_decomposed_footprint(const pic_sim* sim, int ndomains, int guard, size_t* bytes_out);
int pic_step_decomposed(pic_sim* sim, int ndomains, int guard, int nsteps, void* workspace, size_t ws_bytes,
                        void* stream);

/* Field energy W = (eps0/2) sum (|E|^2 + c^2 |B|^2) dV of the real E^n, B^n,
 * written as one double to the DEVICE address out_dev. Sets
 * PIC_STATUS_NONFINITE in the status word if any field value is not finite.
 * Precision 64 squares and sums in FP64. Precision 32 forms each node's |E|^2
 * and |B|^2 in FP32 (finite while every component is below 1.8e19) and sums the
 * nodes in FP64. The same holds for pic_field_energy_noalloc. */
int pic_diag_energy(pic_sim* sim, double* out_dev, void* stream);

/* Copy a buffer out to dst (host or device, `bytes` must equal its size). */
int pic_get(pic_sim* sim, int which, void* dst, size_t bytes, void* stream);

/* Copy the line of real field component `component` (0..5 = Ex, Ey, Ez, Bx, By, Bz) at
 * grid column (ix, iy), all nz nodes along z, to dst (host or device, nz reals of the
 * run's precision), e.g. the on-axis Ez that the boosted-frame wakefield runs record
 * every step. Asynchronous on `stream`. Errors: PIC_EINVAL (NULL pointers, component
 * or column out of range), PIC_ECUDA. */
int pic_get_line(pic_sim* sim, int component, int ix, int iy, void* dst, void* stream);

/* Overwrite the spectral E^n, B^n or rho^n (PIC_BUF_E_HAT, _B_HAT, _RHO_HAT)
 * from src (host or device). Setting E_HAT or B_HAT recomputes the real E, B. */
int pic_set(pic_sim* sim, int which, const void* src, size_t bytes, void* stream);

/* Autotuner: times the particle pass of this run for each tile margin (0, 1) and,
 * for FP32 quadratic/cubic runs, each deposit strategy (pic_config.deposit), on the
 * run's own particles and fields, keeps the fastest for all later steps (the step
 * graph is re-captured) and writes it to chosen[0] (margin) and chosen[1]
 * (strategy); chosen may be NULL. Each candidate takes three real, complete steps
 * (one to settle, two timed), so the run advances by 6 or 18 steps, exactly as
 * pic_step would advance it. Candidates are tried margin 0 then 1, strategy 0, 1, 2;
 * a later one replaces the best so far only when it is at least 2 % faster. Synchronises `stream`. Errors: PIC_EINVAL, PIC_ECUDA,
 * PIC_ECUFFT (the run keeps its previous choice). */
int pic_tune(pic_sim* sim, int32_t chosen[2], void* stream);

/* Re-sort policy. Particles are kept sorted by bin so that a CTA finds them in its
 * shared-memory tile; a particle outside the tile takes a slower global-memory path
 * (correct at any distance). The pass counts particles outside their bin and
 * outside their tile; the next pass re-sorts first when the first count exceeds
 * home_miss_threshold or the second exceeds far_threshold (defaults: 1/32 and
 * 1/1024 of all particles). A negative value keeps that threshold. Asynchronous on
 * `stream`. Errors: PIC_EINVAL (NULL sim), PIC_ECUDA. */
int pic_sort_policy(pic_sim* sim, int64_t home_miss_threshold, int64_t far_threshold, void* stream);

/* Add external real-space fields to E^n and B^n, e.g. the laser pulse of the
 * boosted-frame wakefield runs (laser-plasma acceleration section of the paper).
 * fields: 6 * nx*ny*nz reals of the run's precision (host or device), components
 * Ex, Ey, Ez, Bx, By, Bz, each [nx][ny][nz] with z fastest; read, not kept. They
 * are transformed with the forward FFT of the step, added to the spectral E, B
 * (Nyquist modes stay zero) and the real E, B are recomputed. Particles, rho^n
 * and the current are not touched. Errors: PIC_EINVAL for NULL arguments,
 * PIC_ECUDA / PIC_ECUFFT from the copy or transforms. */
int pic_add_fields(pic_sim* sim, const void* fields, void* stream);

/* Copy one species' particles out (in the library's current order, which is
 * sorted by cell bin) to caller arrays (host or device). Any pointer may be
 * NULL to skip that array. */
int pic_get_particles(pic_sim* sim, int species, int32_t* cell, void* off[3], void* u[3],
                      void* stream);

/* Replace one species' particles (n must match) and re-sort them into bins.
 * Out-of-range input is clamped and flagged with PIC_STATUS_BADINPUT. */
int pic_set_particles(pic_sim* sim, int species, const int32_t* cell, const void* const off[3],
                      const void* const u[3], void* stream);

/* Re-sort every species into its cell bins now (the order pic_get_particles
 * returns is then stable until a later pass finds too many particles outside
 * their bins). */
int pic_sort(pic_sim* sim, void* stream);

/* Synchronising: read the device status word (PIC_STATUS_* bits) and clear
 * it. Returns PIC_EBOUNDS if the bounds bit was set (checked build), else
 * PIC_ENONFINITE if the non-finite bit was set, else PIC_OK. */
int pic_status(pic_sim* sim, int32_t* status_out);

/* Synchronising: read the run's counters: [0] steps taken, [1] particle
 * re-sorts performed, [2] particles outside their bin after the last pass,
 * [3] particles handled by the out-of-tile path in the last pass, [4] the
 * library's own kernel launches enqueued so far (graph replays included;
 * cuFFT's kernels and memsets not counted), [5] reserved (0). */
int pic_counters(pic_sim* sim, int64_t out[6]);

/* Stage timing (tracing). While enabled, the uncaptured calls pic_gather_push,
 * pic_field_update and pic_diag_energy record a CUDA event pair around each
 * stage on their stream: 0 particle re-sort check, 1 particle pass (gather,
 * push, deposit), 2 forward FFT, 3 k-space update, 4 inverse FFT, 5 energy.
 * pic_step replays a graph and records nothing. Enabling clears old records. */
int pic_profile(pic_sim* sim, int enable);

/* Synchronising: per stage, the summed milliseconds and the number of
 * recorded intervals since the last read (or enable); clears the records. */
int pic_profile_read(pic_sim* sim, double ms[8], int64_t count[8]);

/* Grid sizes of a run: N = nx*ny*nz and M = nx*ny*(nz/2+1). */
int pic_sizes(pic_sim* sim, int64_t* n_cells, int64_t* n_modes);

/* Field energy W = (eps0/2) sum (|E|^2 + c^2 |B|^2) dV of caller-provided fields,
 * computed without allocating any device memory. The paper has no counterpart;
 * this is a convenience for callers that cannot call cudaMalloc: plain host code
 * with no device allocator of its own, processes whose device memory is already
 * reserved by another allocator's pool, and code paths that must not allocate or
 * synchronise (allocation can block on other streams).
 *   fields:    DEVICE pointer to 6*n_cells values, E then B, each component a
 *              contiguous [n_cells] array (the layout of PIC_BUF_E followed by
 *              PIC_BUF_B), float (precision 32) or double (precision 64).
 *   n_cells:   1 .. 2^30; anything else returns PIC_EINVAL with a message.
 *   out_dev:   DEVICE address of one double that receives W.
 * The per-block partial sums live in one fixed array inside the library (16 KiB
 * of partial sums plus a status word, present on every device that loads the
 * library until the process exits). Every call shares that array: calls whose
 * kernels overlap on the GPU (different streams, or different threads on one
 * device) race and give wrong results; serialise them. The first call on a
 * device looks up the array's device address (once per device, with that device
 * current) and should come before any stream capture on that device. Non-finite
 * field values make W non-finite. Asynchronous on `stream`. */
int pic_field_energy_noalloc(const void* fields, int64_t n_cells, int precision, double eps0, double c,
                             double dV, double* out_dev, void* stream);

/* ---- Quasi-cylindrical geometry ---------------------------------------------------------
 *
 * The paper runs its boosted-frame results in a quasi-cylindrical spectral code (the
 * implementation paragraph after the update equations): fields are azimuthal modes
 * F(r, theta, z) = F_0 + 2 Re sum_{m=1}^{M-1} F_m(r, z) e^{i m theta} on radial nodes
 * r_j = (j + 1/2) dr (j < nr) and axial nodes z_l = l dz (l < nz, periodic, Galilean
 * coordinate). The paper prints no formulas for this geometry; the readings are:
 *   - Spectral state of mode m: the Cartesian amplitudes at phi = 0, for a vector
 *     F_x + i F_y = -i H_{m+1}[F_r + i F_theta], F_x - i F_y = i H_{m-1}[F_r - i F_theta],
 *     F_z = H_m[F_z]; scalars H_m[g]; H_n the discrete Hankel transform of order n on the
 *     spectral nodes k_i = alpha_i / R (alpha_i the zeros of J_b, b = max(m - 1, 0),
 *     R = nr dr; inverse transform f(r_j) = sum_i w_i J_n(k_i r_j) F_i with
 *     w_i = 2 / (R^2 J_{b+1}(alpha_i)^2); forward transform: that matrix's inverse for
 *     |n| <= 1, the midpoint quadrature sum_j f(r_j) J_n(k_i r_j) r_j dr of the Hankel
 *     integral for |n| >= 2), times the FFT along z (forward e^{-i k_z z}); the Nyquist
 *     plane of an even nz is held at zero.
 *   - Field update: the Galilean-PSATD update (v_gal along z) at k = (k_r, 0, k_z) on
 *     these amplitudes, with FP64-built factors, current correction optional.
 *   - Particles: Cartesian positions (x, y, z) and momenta u = gamma v, Boris push and
 *     Galilean drift as in the Cartesian step; linear shapes in r and z; mode deposits
 *     sum q w S_r S_z e^{-i m theta} / V_j with V_j = 2 pi r_j dr dz; the node below the
 *     axis folds onto node 0 with factor (-1)^m (scalars, z components) or (-1)^(m+1)
 *     (r, theta components). Every particle must satisfy r < (nr - 1/2) dr.
 * Memory follows the Cartesian API: one caller-owned device workspace of
 * pic_cyl_footprint() bytes; the handle owns its cuFFT plans and host struct. */
typedef struct pic_cyl pic_cyl;

typedef struct {
    double dr, dz;        /* radial and axial spacing */
    double dt;
    double vgal;          /* Galilean velocity along z */
    double c, eps0;
    double beta_init;     /* initial fields: the boosted-Coulomb field of rho^0 moving at
                             beta_init c along z (0: electrostatic field of rho^0) */
    int32_t nr, nz;       /* 2 <= nr <= 1024, nz >= 2 */
    int32_t nmodes;       /* azimuthal modes kept, 1 .. 4 */
    int32_t precision;    /* 32 or 64 (transform matrices and factors built in FP64) */
    int32_t current_correction;
    int32_t pad_;
} pic_cyl_config;

typedef struct {
    double q, m;          /* charge and mass of one physical particle */
    int64_t n;            /* macro-particles, 0 .. 2^31 - 1 */
    const void* w;        /* n macro weights (reals of the run's precision; host or device) */
    const void* x[3];     /* n positions x, y, z (z in [0, nz dz)) */
    const void* u[3];     /* n momenta per mass u_x, u_y, u_z */
} pic_cyl_species;

enum pic_cyl_buffer {
    PIC_CYL_EB_HAT = 0,   /* spectral E, B: [M][6][nr][nz] complex (E_x, E_y, E_z, B_x, B_y, B_z) */
    PIC_CYL_RHO_HAT = 1,  /* spectral rho^n: [M][nr][nz] complex */
    PIC_CYL_FIELDS = 2,   /* real-space mode fields: [M][6][nr][nz] complex (E_r, E_theta, E_z,
                             B_r, B_theta, B_z) */
    PIC_CYL_SOURCES = 3,  /* last deposits: [M][4][nr][nz] complex (J_r, J_theta, J_z at
                             (n+1/2) dt, rho at (n+1) dt) */
    PIC_CYL_K = 4,        /* wavenumbers of each mode: [M][nr + 1 + nz] double: k_r, 0, k_z */
    PIC_CYL_STATUS = 5    /* the device status word (int32, PIC_STATUS_* bits) */
};

/* Workspace bytes of a quasi-cylindrical run (creates and destroys its cuFFT plans).
 * Errors: PIC_EINVAL (configuration out of range), PIC_ECUFFT. */
int pic_cyl_footprint(const pic_cyl_config* cfg, const pic_cyl_species* species, int nspecies,
                      size_t* bytes_out);

/* Create a run in `workspace` (device, 256-byte aligned, >= pic_cyl_footprint()):
 * copies the particles, builds the Bessel zeros, transform matrices (FP64; Gauss-Jordan
 * inverses for the orders |n| <= 1) and update factors on the GPU, deposits rho^0 and sets the initial fields.
 * Synchronises `stream`. Errors: PIC_EINVAL (also when a particle lies outside the
 * radial extent or a transform matrix is singular), PIC_ENOMEM, PIC_ECUDA, PIC_ECUFFT. */
int pic_cyl_init(const pic_cyl_config* cfg, const pic_cyl_species* species, int nspecies,
                 void* workspace, size_t ws_bytes, void* stream, pic_cyl** out);

/* Advance nsteps steps: gather at x^n, Boris push, half drift, J^{n+1/2}, half drift,
 * rho^{n+1}; forward transforms; Galilean-PSATD update of every mode; inverse
 * transforms. A particle that leaves the radial extent sets PIC_STATUS_BADINPUT and
 * is not deposited. Asynchronous on `stream`. */
int pic_cyl_step(pic_cyl* run, int nsteps, void* stream);

/* Copy a PIC_CYL_* buffer to dst (host or device); `bytes` must equal its size. */
int pic_cyl_get(pic_cyl* run, int which, void* dst, size_t bytes, void* stream);

/* Copy species k's positions and momenta out, in input order (any pointer may be NULL).
 * The run keeps its particles sorted by (r, z) bin in one of two buffers; this call reads
 * which one on `stream` (synchronising it) and restores the input order on the device. */
int pic_cyl_get_particles(pic_cyl* run, int species, void* x[3], void* u[3], void* stream);

/* Field energy W = (eps0/2) sum_m (1 for m = 0, else 2) sum_{j,l} (|E_m|^2 + c^2 |B_m|^2) V_j
 * of the real mode fields, one double written to the DEVICE address out_dev. */
int pic_cyl_energy(pic_cyl* run, double* out_dev, void* stream);

/* Stage timing (tracing). While enabled, pic_cyl_step records a CUDA event pair around
 * each stage on its stream and waits for it at the end of every step (and for the radial
 * products inside the transforms): 0 particle kernel (with the deposit arrays' clear),
 * 1 sources to spectral space, 2 k-space update, 3 fields to real space, 4 the radial
 * matrix products (inside stages 1 and 3). Enabling clears old records. */
int pic_cyl_profile(pic_cyl* run, int enable);

/* Per stage, the summed milliseconds and the number of recorded intervals since the last
 * read (or enable); clears the records. */
int pic_cyl_profile_read(pic_cyl* run, double ms[5], int64_t count[5]);

int pic_cyl_destroy(pic_cyl* run);

#ifdef __cplusplus
}
#endif

#endif /* GALPIC_H */
