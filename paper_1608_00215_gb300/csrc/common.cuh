// Internal definitions shared by the galpic CUDA sources (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "galpic.h"

namespace galpic {

// ---------------------------------------------------------------------------
// Error plumbing
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);

#define GP_CUDA(call)                                                                 \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess)                                                        \
            return ::galpic::fail(PIC_ECUDA, std::string(#call) + ": " +              \
                                                 cudaGetErrorString(e_));             \
    } while (0)

#define GP_CUFFT(call)                                                                \
    do {                                                                              \
        cufftResult r_ = (call);                                                      \
        if (r_ != CUFFT_SUCCESS)                                                      \
            return ::galpic::fail(PIC_ECUFFT, std::string(#call) + ": cufft error " + \
                                                  std::to_string((int)r_));           \
    } while (0)

#define GP_CHECK(expr)                                                                \
    do {                                                                              \
        int rc_ = (expr);                                                             \
        if (rc_ != PIC_OK) return rc_;                                                \
    } while (0)

// ---------------------------------------------------------------------------
// Complex helpers for float2 / double2
// ---------------------------------------------------------------------------
template <typename T> struct cplx;
template <> struct cplx<float> { typedef float2 type; };
template <> struct cplx<double> { typedef double2 type; };

template <typename C> __host__ __device__ __forceinline__ C mk(double re, double im) {
    C r; r.x = (decltype(r.x))re; r.y = (decltype(r.y))im; return r;
}
template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
    C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <typename C, typename T> __host__ __device__ __forceinline__ C cscale(C a, T s) { a.x *= s; a.y *= s; return a; }
template <typename C> __host__ __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }
template <typename C> __host__ __device__ __forceinline__ C ctimesi(C a) { C r; r.x = -a.y; r.y = a.x; return r; }
__host__ __device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    double d = b.x * b.x + b.y * b.y;
    double2 r; r.x = (a.x * b.x + a.y * b.y) / d; r.y = (a.y * b.x - a.x * b.y) / d; return r;
}

// ---------------------------------------------------------------------------
// Counters in device memory (uint64 each)
// ---------------------------------------------------------------------------
enum {
    CNT_FORCE_SORT = 0,   // nonzero: re-sort before the next particle pass
    CNT_SORTS = 1,        // re-sorts performed
    CNT_HOME_MISS = 2,    // particles outside their bin after the last pass
    CNT_FAR = 3,          // particles that took the out-of-tile path in the last pass
    CNT_THRESHOLD = 4,    // re-sort when HOME_MISS exceeds this
    CNT_FAR_THRESHOLD = 5,   // re-sort when FAR exceeds this
    CNT_COUNT = 8
};

// Decision shared by every re-sort kernel: identical for all of them because
// none of them writes the words it reads (the final kernel clears FORCE last).
// Particles outside their tile are handled correctly by the global-memory path at
// any distance, so a re-sort is only a matter of speed.
__device__ __forceinline__ bool sort_needed(const unsigned long long* cnt) {
    return cnt[CNT_FORCE_SORT] != 0ull || cnt[CNT_FAR] > cnt[CNT_FAR_THRESHOLD] ||
           cnt[CNT_HOME_MISS] > cnt[CNT_THRESHOLD];
}

// ---------------------------------------------------------------------------
// Checked build (PIC_CHECKED): index tests that record a violation in the device status
// word and let the caller skip the access. The ordinary build compiles them away.
// ---------------------------------------------------------------------------
#ifdef PIC_CHECKED
__device__ __forceinline__ bool index_ok(int64_t i, int64_t n, int32_t* status) {
    if (i >= 0 && i < n) return true;
    atomicOr(status, PIC_STATUS_BOUNDS);
    return false;
}
#define PIC_INDEX_OK(i, n, status) ::galpic::index_ok((int64_t)(i), (int64_t)(n), (status))
#else
#define PIC_INDEX_OK(i, n, status) true
#endif

// ---------------------------------------------------------------------------
// splitmix64 (Vigna): output function applied to a counter
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// ---------------------------------------------------------------------------
// Internal run handle
// ---------------------------------------------------------------------------
struct SpeciesDev {
    double q, m, w;
    int64_t n;
    int32_t* cell;
    void* off[3];
    void* u[3];
    int32_t* bin_start;   // nbins + 1
    int32_t* cell_start;  // nbins * BX*BY*BZ + 1: first particle of each cell key as of the last sort
};

struct Layout {
    size_t total;
    size_t off_species[PIC_MAX_SPECIES][9];   // cell, off x/y/z, u x/y/z, bin_start, cell_start
    size_t off_tmp[8];                        // cell, off x/y/z, u x/y/z, rank
    size_t off_key_cnt, off_tile_sum;
    size_t off_S64, off_desc;
    size_t off_F, off_S, off_EBh, off_EBs, off_Sh, off_Rn, off_Tab, off_K, off_Kt, off_Ph;
    size_t off_fftwork;
    size_t off_epart;
    size_t off_cnt, off_status;
    size_t fft_bytes;
};

struct Dims {
    int nx, ny, nz, nzh;
    int64_t N, M;
    int BX, BY, BZ, nbx, nby, nbz, nbins;
    int margin;
};

struct PlanEntry;

}  // namespace galpic

struct pic_sim {
    pic_config cfg;
    int nspecies;
    galpic::SpeciesDev sp[PIC_MAX_SPECIES];
    galpic::Dims d;
    galpic::Layout L;
    char* ws;
    size_t ws_bytes;
    void* F;     // real E (3N) then B (3N)
    void* S;     // real Jx, Jy, Jz, rho (4N)
    long long* S64;   // deterministic mode: the sources in 64-bit fixed point (4N), else NULL
    char* desc;       // deterministic mode: the run's pass and k-space parameter tables (device)
    int fix_exp;      // deterministic mode: delta = 2^fix_exp (units of the fixed-point sources)
    void* EBh;   // spectral master E, B (6M complex)
    void* EBs;   // C2R input: master / N (6M complex)
    void* Sh;    // spectra of Jx, Jy, Jz, rho^{n+1} (4M complex)
    void* Rn;    // spectral rho^n (M complex)
    void* Tab;   // per-mode factors T1..T4, A5, A6 (6M complex)
    double* K;   // wavenumbers per axis (spectral or modified), kx[nx], ky[ny], kz[nzh], FP64
    void* Kt;    // the same in the run's precision
    void* Ph;    // per-axis shift phases of a coupled step (nx + ny + nzh complex)
    void* fftwork;
    double* epart;
    int energy_blocks;
    int32_t* tmp_cell;
    void* tmp_off[3];
    void* tmp_u[3];
    int32_t* tmp_rank;
    int32_t* key_cnt;     // sort: particles per cell key
    int32_t* tile_sum;    // sort: scan partial sums
    unsigned long long* cnt;
    int32_t* status;
    cufftHandle plan_r2c, plan_c2r;   // shared by runs of the same shape (not owned)
    galpic::PlanEntry* plans;
    cudaStream_t priv;
    cudaGraphExec_t graph;
    bool graph_ok;
    int64_t steps;
    int64_t launches;        // own kernel launches enqueued (incl. graph replays)
    int64_t graph_kernels;   // own kernels in one captured step
    bool capturing;
    bool profiling;
    int inject;   // checked build only: a deliberate tile-index offset for the checker's own test
    struct Rec { int stage; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> event_pool;
};

namespace galpic {

// Launchers implemented in the .cu files (all enqueue on `st`).
int launch_build_tables(pic_sim* s, cudaStream_t st);
int launch_kspace_update(pic_sim* s, cudaStream_t st);
int launch_init_fields(pic_sim* s, cudaStream_t st);
int launch_master_to_scratch(pic_sim* s, cudaStream_t st);
// Adds src's spectral master, moved onto dst's grid at time t and scaled by 1/N, to
// dst's inverse-transform copy (two kernels: per-axis phases, then the add).
int launch_add_shifted(pic_sim* dst, const pic_sim* src, double t, cudaStream_t st);
// Adds six spectra (`add`, [6][M] complex) to the spectral master, Nyquist modes excluded.
int launch_add_spectra(pic_sim* s, const void* add, cudaStream_t st);
int launch_energy(pic_sim* s, double* out_dev, cudaStream_t st);
// Energy kernels on caller-given fields (real [6][N]) and partial-sum storage.
int launch_energy_on(const void* F, int64_t N, int precision, double* part, int nb, int32_t* status,
                     double se_scale, double sb_scale, double* out_dev, cudaStream_t st);
int launch_generate(pic_sim* s, int species, const pic_species* spec, cudaStream_t st);
int launch_sort(pic_sim* s, cudaStream_t st);
int launch_sanitize(pic_sim* s, int species, cudaStream_t st);
int launch_particle_pass(pic_sim* s, int mode, cudaStream_t st);
// Deterministic mode: real sources S = delta * S64 (4N values).
int launch_fixed_to_real(pic_sim* s, cudaStream_t st);
int launch_pass_fp32(pic_sim* s, int mode, cudaStream_t st);   // pass_fp32.cu
int launch_pass_fp64(pic_sim* s, int mode, cudaStream_t st);   // pass_fp64.cu

// Shared launches over several runs of one shape class (pic_step_many, many.cu).
// Particle pass: parameter blocks (one per run, F, S, S64 redirected to a staging area)
// and the launch over all of them; the variant code says which runs can share it.
size_t pass_desc_bytes_fp32();
size_t pass_desc_bytes_fp64();
void fill_pass_desc_fp32(const pic_sim* s, void* out, const void* F, void* S, long long* S64);
void fill_pass_desc_fp64(const pic_sim* s, void* out, const void* F, void* S, long long* S64);
int launch_pass_many_fp32(pic_sim* s0, const void* descs, int nruns, cudaStream_t st);
int launch_pass_many_fp64(pic_sim* s0, const void* descs, int nruns, cudaStream_t st);
int pass_variant_of(const pic_sim* s);
// K-space update: parameter blocks (EBs, Sh redirected) and the launch over them.
size_t kspace_desc_bytes(int precision);
void fill_kspace_desc(const pic_sim* s, void* out, void* EBs, const void* Sh);
int launch_kspace_many(const pic_sim* s0, const void* descs, int nruns, cudaStream_t st);
// Re-sort check of every run for one species slot: descriptor blocks and the kernels.
size_t sort_desc_bytes(int precision);
void fill_sort_desc(const pic_sim* s, int species, void* out);
int launch_sort_many(const pic_sim* s0, const void* descs, int nruns, int64_t nmax, cudaStream_t st);
// After the re-sort checks of every species: per run, a performed re-sort is counted and
// the request cleared, and the stray counts are cleared for the next pass.
int launch_sort_finish_many(unsigned long long* const* cnts_dev, int nruns, cudaStream_t st);
// Copies of `n` (dst, src, bytes) triples listed in device memory, one launch.
struct CopyDesc {
    void* dst;
    const void* src;
    size_t bytes;
};
int launch_copy_many(const CopyDesc* descs_dev, int n, size_t max_bytes, cudaStream_t st);
// Forget the captured shared-launch steps that involve a run (called by pic_destroy).
void many_forget(pic_sim* s);

// Decomposed field update (decomp.cu): wavenumbers and factors of the window grid
// (nx, ny, nz_w), and the k-space update of nwin windows (descriptors in device memory;
// the Nyquist planes of a window are updated like any mode).
int launch_window_tables(const pic_sim* s, int nz_w, double* K, void* Kt, void* tab, cudaStream_t st);
void fill_window_kspace_desc(const pic_sim* s, void* out, int nz_w, void* spec, void* ebs, const void* Kt,
                             const void* tab);
int launch_kspace_windows(const pic_sim* s, const void* descs, int nwin, int64_t M_w, cudaStream_t st);
// The mutex that serialises the set-stream / set-work-area / execute sequence of a run's
// shared single-run cuFFT plans (api.cu).
std::mutex* plan_mutex(pic_sim* s);
// Quasi-cylindrical modes (cyl.cu): factors at k = (k_r, 0, k_z) from K = [k_r (nr), 0,
// k_z (nz)], the k-space parameters of one mode, and the k-space launch over n modes.
int launch_cyl_tables(int precision, int nr, int nz, const double* K, void* tab, double dt, double vgal, double c,
                      double eps0, int cc, cudaStream_t st);
void fill_cyl_kspace_desc(int precision, void* out, int nr, int nz, void* EBh, const void* Sh, void* Rn,
                          void* scratch, const void* tab, const void* Kt, double c, int cc);
int launch_kspace_descs(int precision, const void* descs, int n, int64_t M, cudaStream_t st);
// Pieces of the single-run step that the decomposed step reuses (api.cu).
int gather_push_stage(pic_sim* s, cudaStream_t st);
int r2c_on(pic_sim* s, void* in, void* out, cudaStream_t st);
// Deterministic mode over a staging area: real sources from fixed-point sums, run r of
// nruns at S64 + r n (its unit 2^e[r], e in device memory).
int launch_fixed_to_real_many(const long long* S64, void* S, int64_t n, const int* e_dev, int nruns,
                              int precision, cudaStream_t st);

enum { PASS_STEP = 0, PASS_DEPOSIT = 1 };
enum { STAGE_SORT = 0, STAGE_PARTICLES = 1, STAGE_R2C = 2, STAGE_KSPACE = 3, STAGE_C2R = 4,
       STAGE_ENERGY = 5, STAGE_COUNT = 8 };

// Shared-memory bytes of one particle-pass CTA.
size_t tile_bytes(const pic_config& c, const Dims& d, int mode);
// Number of cell keys of the sort (bins x cells per bin) and of scan tiles.
int64_t sort_keys(const Dims& d);
int64_t sort_tiles(const Dims& d);

}  // namespace galpic
