// C ABI of the Galilean-PSATD step (include/galpic.h): validation, workspace
// layout, cuFFT plans, stage sequencing and CUDA-graph replay.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "common.cuh"

namespace galpic {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

// cuFFT plans, shared by every run of the same grid shape and precision on a device
// for the life of the process (plan creation allocates and synchronises). A run
// keeps its own work area in its workspace; the entry's mutex serialises the
// set-stream / set-work-area / execute sequence of runs that share a plan.
struct PlanEntry {
    cufftHandle r2c = 0, c2r = 0;
    size_t work = 0;
    std::mutex mu;
};

namespace {

constexpr size_t ALIGN = 256;
// Deterministic runs step through the same table-driven kernels as shared launches
// (pic_step_many), so that a run's bits do not depend on which path advanced it: its pass
// parameters at offset 0 and its k-space parameters at DESC_KSPACE of this region.
constexpr size_t DESC_KSPACE = 2048, DESC_BYTES = 4096;

size_t align_up(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

int validate(const pic_config* c, const pic_species* sp, int ns) {
    if (!c) return fail(PIC_EINVAL, "config is NULL");
    if (c->nx < 2 || c->ny < 2 || c->nz < 2) return fail(PIC_EINVAL, "grid needs >= 2 nodes per axis");
    if ((int64_t)c->nx * c->ny * c->nz > (int64_t)1 << 30)
        return fail(PIC_EINVAL, "grid larger than 2^30 nodes");
    if (c->shape_order < 1 || c->shape_order > 3) return fail(PIC_EINVAL, "shape_order must be 1, 2 or 3");
    if (c->precision != 32 && c->precision != 64) return fail(PIC_EINVAL, "precision must be 32 or 64");
    if (!(c->dx > 0 && c->dy > 0 && c->dz > 0 && c->dt > 0 && c->c > 0 && c->eps0 > 0))
        return fail(PIC_EINVAL, "dx, dy, dz, dt, c and eps0 must be positive");
    double v2 = c->vgal[0] * c->vgal[0] + c->vgal[1] * c->vgal[1] + c->vgal[2] * c->vgal[2];
    if (!(v2 < c->c * c->c)) return fail(PIC_EINVAL, "|v_gal| must be below c");
    double b2 = c->beta_init[0] * c->beta_init[0] + c->beta_init[1] * c->beta_init[1] +
                c->beta_init[2] * c->beta_init[2];
    if (c->init_fields == 1 && !(b2 < 1.0)) return fail(PIC_EINVAL, "|beta_init| must be below 1");
    if (c->init_fields != 0 && c->init_fields != 1) return fail(PIC_EINVAL, "init_fields must be 0 or 1");
    if (c->tile_margin != 0 && c->tile_margin != 1) return fail(PIC_EINVAL, "tile_margin must be 0 or 1");
    if (c->deposit < 0 || c->deposit > 4) return fail(PIC_EINVAL, "deposit must be 0 .. 4");
    if (c->stencil_order < 0 || c->stencil_order > 128 || (c->stencil_order & 1))
        return fail(PIC_EINVAL, "stencil_order must be 0 or an even number in [2, 128]");
    if (c->deterministic != 0 && c->deterministic != 1) return fail(PIC_EINVAL, "deterministic must be 0 or 1");
    if (ns < 0 || ns > PIC_MAX_SPECIES) return fail(PIC_EINVAL, "nspecies out of range");
    if (ns > 0 && !sp) return fail(PIC_EINVAL, "species array is NULL");
    int64_t ncell = (int64_t)c->nx * c->ny * c->nz;
    for (int k = 0; k < ns; ++k) {
        const pic_species& s = sp[k];
        if (s.n < 0 || s.n > INT32_MAX) return fail(PIC_EINVAL, "species n out of range [0, 2^31)");
        if (!(s.m > 0)) return fail(PIC_EINVAL, "species mass must be positive");
        if (s.ppc[0] > 0) {
            if (s.ppc[1] < 1 || s.ppc[2] < 1) return fail(PIC_EINVAL, "ppc must be >= 1 per axis");
            if (s.n != ncell * s.ppc[0] * s.ppc[1] * s.ppc[2])
                return fail(PIC_EINVAL, "generated species: n must equal cells * ppc");
        } else if (s.n > 0) {
            if (!s.cell || !s.off[0] || !s.off[1] || !s.off[2] || !s.u[0] || !s.u[1] || !s.u[2])
                return fail(PIC_EINVAL, "copied species: every particle array must be given");
        }
    }
    return PIC_OK;
}

Dims make_dims(const pic_config& c) {
    Dims d;
    d.nx = c.nx;
    d.ny = c.ny;
    d.nz = c.nz;
    d.nzh = c.nz / 2 + 1;
    d.N = (int64_t)c.nx * c.ny * c.nz;
    d.M = (int64_t)c.nx * c.ny * d.nzh;
    d.BX = d.BY = d.BZ = 8;
    d.nbx = (c.nx + d.BX - 1) / d.BX;
    d.nby = (c.ny + d.BY - 1) / d.BY;
    d.nbz = (c.nz + d.BZ - 1) / d.BZ;
    d.nbins = d.nbx * d.nby * d.nbz;
    d.margin = c.tile_margin;
    return d;
}

int energy_blocks_for(int64_t N) {
    int64_t b = (N + 2047) / 2048;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 1216));
}

std::mutex g_plan_mu;
std::map<std::tuple<int, int, int, int, int>, std::unique_ptr<PlanEntry>> g_plans;

int make_plans(const pic_config& c, const Dims& d, cufftHandle* r2c, cufftHandle* c2r,
               size_t* work);

int shared_plans(const pic_config& c, const Dims& d, PlanEntry** out) {
    int dev = 0;
    GP_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_plan_mu);
    auto key = std::make_tuple(dev, c.nx, c.ny, c.nz, c.precision);
    auto it = g_plans.find(key);
    if (it == g_plans.end()) {
        std::unique_ptr<PlanEntry> e(new PlanEntry());
        int rc = make_plans(c, d, &e->r2c, &e->c2r, &e->work);
        if (rc != PIC_OK) {
            if (e->r2c) cufftDestroy(e->r2c);
            if (e->c2r) cufftDestroy(e->c2r);
            return rc;
        }
        it = g_plans.emplace(key, std::move(e)).first;
    }
    *out = it->second.get();
    return PIC_OK;
}

int make_plans(const pic_config& c, const Dims& d, cufftHandle* r2c, cufftHandle* c2r,
               size_t* work) {
    long long n[3] = {c.nx, c.ny, c.nz};
    long long rn[3] = {c.nx, c.ny, c.nz};
    long long cn[3] = {c.nx, c.ny, d.nzh};
    size_t w1 = 0, w2 = 0;
    GP_CUFFT(cufftCreate(r2c));
    GP_CUFFT(cufftCreate(c2r));
    GP_CUFFT(cufftSetAutoAllocation(*r2c, 0));
    GP_CUFFT(cufftSetAutoAllocation(*c2r, 0));
    bool dbl = c.precision == 64;
    GP_CUFFT(cufftMakePlanMany64(*r2c, 3, n, rn, 1, d.N, cn, 1, d.M, dbl ? CUFFT_D2Z : CUFFT_R2C, 4, &w1));
    GP_CUFFT(cufftMakePlanMany64(*c2r, 3, n, cn, 1, d.M, rn, 1, d.N, dbl ? CUFFT_Z2D : CUFFT_C2R, 6, &w2));
    *work = std::max(w1, w2);
    return PIC_OK;
}

void make_layout(const pic_config& c, const Dims& d, const int64_t* n, int ns, size_t fft_bytes,
                 Layout& L) {
    const size_t T = c.precision == 64 ? 8 : 4;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align_up(o + bytes);
        return at;
    };
    int64_t nmax = 0;
    for (int k = 0; k < ns; ++k) {
        nmax = std::max(nmax, n[k]);
        L.off_species[k][0] = take(n[k] * 4);
        for (int q = 1; q <= 6; ++q) L.off_species[k][q] = take(n[k] * T);
        L.off_species[k][7] = take((d.nbins + 1) * 4);
        L.off_species[k][8] = take((sort_keys(d) + 1) * 4);
    }
    L.off_tmp[0] = take(nmax * 4);
    for (int q = 1; q <= 6; ++q) L.off_tmp[q] = take(nmax * T);
    L.off_tmp[7] = take(nmax * 4);
    L.off_key_cnt = take(sort_keys(d) * 4);
    L.off_tile_sum = take(sort_tiles(d) * 4);
    L.off_S64 = take(c.deterministic ? 4 * d.N * 8 : 0);
    L.off_desc = take(c.deterministic ? DESC_BYTES : 0);
    L.off_F = take(6 * d.N * T);
    L.off_S = take(4 * d.N * T);
    L.off_EBh = take(6 * d.M * 2 * T);
    L.off_EBs = take(6 * d.M * 2 * T);
    L.off_Sh = take(4 * d.M * 2 * T);
    L.off_Rn = take(d.M * 2 * T);
    L.off_Tab = take(6 * d.M * 2 * T);
    L.off_K = take((size_t)(d.nx + d.ny + d.nzh) * 8);
    L.off_Kt = take((size_t)(d.nx + d.ny + d.nzh) * T);
    L.off_Ph = take((size_t)(d.nx + d.ny + d.nzh) * 2 * T);
    L.off_fftwork = take(std::max<size_t>(fft_bytes, 1));
    L.off_epart = take(2 * energy_blocks_for(d.N) * sizeof(double));
    L.off_cnt = take(CNT_COUNT * sizeof(unsigned long long));
    L.off_status = take(sizeof(int32_t));
    L.fft_bytes = fft_bytes;
    L.total = o;
}

int check_tile_fits(const pic_config& c, const Dims& d) {
    int dev = 0, optin = 0;
    GP_CUDA(cudaGetDevice(&dev));
    GP_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    size_t need = tile_bytes(c, d, PASS_STEP);
    if (need > (size_t)optin)
        return fail(PIC_EINVAL, "particle tile needs " + std::to_string(need) +
                                    " bytes of shared memory, device allows " + std::to_string(optin));
    return PIC_OK;
}

int exec_r2c(pic_sim* s, cudaStream_t st) {
    std::lock_guard<std::mutex> lk(s->plans->mu);
    GP_CUFFT(cufftSetWorkArea(s->plan_r2c, s->fftwork));
    GP_CUFFT(cufftSetStream(s->plan_r2c, st));
    if (s->cfg.precision == 64)
        GP_CUFFT(cufftExecD2Z(s->plan_r2c, (cufftDoubleReal*)s->S, (cufftDoubleComplex*)s->Sh));
    else
        GP_CUFFT(cufftExecR2C(s->plan_r2c, (cufftReal*)s->S, (cufftComplex*)s->Sh));
    return PIC_OK;
}

// Forward transform of four real grids at `in` ([4][N]) into `out` ([4][M]).
int exec_r2c_on(pic_sim* s, void* in, void* out, cudaStream_t st) {
    std::lock_guard<std::mutex> lk(s->plans->mu);
    GP_CUFFT(cufftSetWorkArea(s->plan_r2c, s->fftwork));
    GP_CUFFT(cufftSetStream(s->plan_r2c, st));
    if (s->cfg.precision == 64)
        GP_CUFFT(cufftExecD2Z(s->plan_r2c, (cufftDoubleReal*)in, (cufftDoubleComplex*)out));
    else
        GP_CUFFT(cufftExecR2C(s->plan_r2c, (cufftReal*)in, (cufftComplex*)out));
    return PIC_OK;
}

int exec_c2r(pic_sim* s, cudaStream_t st) {
    std::lock_guard<std::mutex> lk(s->plans->mu);
    GP_CUFFT(cufftSetWorkArea(s->plan_c2r, s->fftwork));
    GP_CUFFT(cufftSetStream(s->plan_c2r, st));
    if (s->cfg.precision == 64)
        GP_CUFFT(cufftExecZ2D(s->plan_c2r, (cufftDoubleComplex*)s->EBs, (cufftDoubleReal*)s->F));
    else
        GP_CUFFT(cufftExecC2R(s->plan_c2r, (cufftComplex*)s->EBs, (cufftReal*)s->F));
    return PIC_OK;
}

size_t real_bytes(const pic_sim* s) { return s->cfg.precision == 64 ? 8 : 4; }

// Own kernel launches: counted per enqueue, or per captured step while capturing.
void count_launches(pic_sim* s, int64_t n) {
    if (s->capturing)
        s->graph_kernels += n;
    else
        s->launches += n;
}

int sort_kernel_count(const pic_sim* s) {
    int n = 1;
    for (int k = 0; k < s->nspecies; ++k)
        if (s->sp[k].n > 0) n += 7;
    return n;
}

cudaEvent_t take_event(pic_sim* s) {
    if (!s->event_pool.empty()) {
        cudaEvent_t e = s->event_pool.back();
        s->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Records a CUDA event pair around one stage when profiling (never inside a capture).
struct StageTimer {
    pic_sim* s;
    int stage;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    StageTimer(pic_sim* s_, int stage_, cudaStream_t st_) : s(s_), stage(stage_), st(st_) {
        if (s->profiling && !s->capturing) {
            a = take_event(s);
            if (a && cudaEventRecord(a, st) != cudaSuccess) a = nullptr;
        }
    }
    ~StageTimer() {
        if (!a) return;
        cudaEvent_t b = take_event(s);
        if (b && cudaEventRecord(b, st) == cudaSuccess)
            s->recs.push_back({stage, a, b});
        else
            s->event_pool.push_back(a);
    }
};

int set_force_sort(pic_sim* s, cudaStream_t st) {
    static const unsigned long long one = 1ull;
    GP_CUDA(cudaMemcpyAsync(s->cnt + CNT_FORCE_SORT, &one, sizeof(one), cudaMemcpyHostToDevice, st));
    return PIC_OK;
}

int sort_particles(pic_sim* s, cudaStream_t st) {
    StageTimer t(s, STAGE_SORT, st);
    count_launches(s, sort_kernel_count(s));
    return launch_sort(s, st);
}

int deposit_sources(pic_sim* s, int mode, cudaStream_t st) {
    if (s->S64) {   // deterministic mode: integer sums, then the real sources from them
        GP_CUDA(cudaMemsetAsync(s->S64, 0, 4 * s->d.N * sizeof(long long), st));
        StageTimer t(s, STAGE_PARTICLES, st);
        count_launches(s, 2);
        if (mode == PASS_STEP)
            GP_CHECK(s->cfg.precision == 64 ? launch_pass_many_fp64(s, s->desc, 1, st)
                                            : launch_pass_many_fp32(s, s->desc, 1, st));
        else
            GP_CHECK(launch_particle_pass(s, mode, st));
        return launch_fixed_to_real(s, st);
    }
    GP_CUDA(cudaMemsetAsync(s->S, 0, 4 * s->d.N * real_bytes(s), st));
    StageTimer t(s, STAGE_PARTICLES, st);
    count_launches(s, 1);
    return launch_particle_pass(s, mode, st);
}

// Deterministic mode: the fixed-point unit delta = 2^e, e the smallest integer with
// max(1, c) sum_s |q_s w_s| n_s / dV < 2^(62 + e): a node's sum of deposited values is at
// most that sum in magnitude, so its integer sum stays below 2^62 plus half a unit per
// term (fewer than 2^40 terms), inside int64; partial sums may wrap, the total cannot.
int fixed_point_exponent(const pic_config& c, const pic_species* sp, int ns) {
    double B = 0.0;
    const double dV = c.dx * c.dy * c.dz;
    for (int k = 0; k < ns; ++k) B += fabs(sp[k].q * sp[k].w) * (double)sp[k].n / dV;
    B *= std::max(1.0, c.c);
    int e = -62;
    if (B > 0.0 && std::isfinite(B)) {
        int E = 0;
        frexp(B, &E);    // B = m 2^E, 1/2 <= m < 1, so B < 2^E
        e = E - 62;
    }
    // 1/delta must stay finite in the run's precision
    return std::max(e, c.precision == 32 ? -120 : -1000);
}

int gather_push(pic_sim* s, cudaStream_t st) {
    GP_CHECK(sort_particles(s, st));
    GP_CUDA(cudaMemsetAsync(s->cnt + CNT_HOME_MISS, 0, 2 * sizeof(unsigned long long), st));
    return deposit_sources(s, PASS_STEP, st);
}

// Forward transform of the sources and the k-space update (master spectrum and its
// scaled copy for the inverse transform).
int field_update_spectral(pic_sim* s, cudaStream_t st) {
    {
        StageTimer t(s, STAGE_R2C, st);
        GP_CHECK(exec_r2c(s, st));
    }
    StageTimer t(s, STAGE_KSPACE, st);
    count_launches(s, 1);
    if (s->desc) return launch_kspace_many(s, s->desc + DESC_KSPACE, 1, st);
    return launch_kspace_update(s, st);
}

int field_update(pic_sim* s, cudaStream_t st) {
    GP_CHECK(field_update_spectral(s, st));
    StageTimer t(s, STAGE_C2R, st);
    return exec_c2r(s, st);
}

// Coupled runs: for every run, its inverse-transform copy (its own master / N when
// `rescale`, else as the k-space update left it) plus the other runs' masters moved
// onto its grid at the common time, then the inverse transform: the gathered field
// of every run is the total field.
int couple_fields(pic_sim** sims, int n, bool rescale, cudaStream_t st) {
    const double t = (double)sims[0]->steps * sims[0]->cfg.dt;
    for (int j = 0; j < n; ++j) {
        pic_sim* s = sims[j];
        if (rescale) {
            count_launches(s, 1);
            GP_CHECK(launch_master_to_scratch(s, st));
        }
        for (int i = 0; i < n; ++i) {
            if (i == j) continue;
            count_launches(s, 2);
            GP_CHECK(launch_add_shifted(s, sims[i], t, st));
        }
        StageTimer tm(s, STAGE_C2R, st);
        GP_CHECK(exec_c2r(s, st));
    }
    return PIC_OK;
}

int check_coupled(pic_sim** sims, int n) {
    if (!sims || n < 1 || n > 16) return fail(PIC_EINVAL, "coupled runs: need 1 to 16 sims");
    for (int j = 0; j < n; ++j) {
        if (!sims[j]) return fail(PIC_EINVAL, "sims[" + std::to_string(j) + "] is NULL");
        for (int i = 0; i < j; ++i)
            if (sims[i] == sims[j]) return fail(PIC_EINVAL, "a sim appears twice in a coupled step");
        const pic_config &a = sims[0]->cfg, &b = sims[j]->cfg;
        if (a.nx != b.nx || a.ny != b.ny || a.nz != b.nz || a.dx != b.dx || a.dy != b.dy || a.dz != b.dz ||
            a.dt != b.dt || a.c != b.c || a.eps0 != b.eps0 || a.precision != b.precision)
            return fail(PIC_EINVAL, "coupled runs must share grid, cell size, dt, c, eps0 and precision");
        if (sims[j]->steps != sims[0]->steps) return fail(PIC_EINVAL, "coupled runs must be at the same step");
    }
    return PIC_OK;
}

int capture_step(pic_sim* s) {
    cudaGraph_t g = nullptr;
    GP_CUDA(cudaStreamBeginCapture(s->priv, cudaStreamCaptureModeThreadLocal));
    s->capturing = true;
    s->graph_kernels = 0;
    int rc = gather_push(s, s->priv);
    if (rc == PIC_OK) rc = field_update(s, s->priv);
    s->capturing = false;
    cudaError_t e = cudaStreamEndCapture(s->priv, &g);
    if (rc != PIC_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(PIC_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&s->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(PIC_ECUDA, std::string("instantiate: ") + cudaGetErrorString(e));
    s->graph_ok = true;
    return PIC_OK;
}

}  // namespace

int gather_push_stage(pic_sim* s, cudaStream_t st) { return gather_push(s, st); }

std::mutex* plan_mutex(pic_sim* s) { return &s->plans->mu; }

int r2c_on(pic_sim* s, void* in, void* out, cudaStream_t st) { return exec_r2c_on(s, in, out, st); }

}  // namespace galpic

using namespace galpic;

extern "C" {

#ifdef PIC_CHECKED
const char* pic_version(void) { return "galpic 0.2 (Galilean-PSATD PIC, sm_103a, checked build)"; }
#else
const char* pic_version(void) { return "galpic 0.2 (Galilean-PSATD PIC, sm_103a)"; }
#endif

const char* pic_last_error(void) { return g_err.c_str(); }

int pic_footprint(const pic_config* cfg, const pic_species* species, int nspecies, size_t* bytes_out) {
    GP_CHECK(validate(cfg, species, nspecies));
    if (!bytes_out) return fail(PIC_EINVAL, "bytes_out is NULL");
    Dims d = make_dims(*cfg);
    PlanEntry* pe = nullptr;
    GP_CHECK(shared_plans(*cfg, d, &pe));
    size_t work = pe->work;
    int64_t n[PIC_MAX_SPECIES];
    for (int k = 0; k < nspecies; ++k) n[k] = species[k].n;
    Layout L;
    make_layout(*cfg, d, n, nspecies, work, L);
    *bytes_out = L.total;
    return PIC_OK;
}

int pic_init(const pic_config* cfg, const pic_species* species, int nspecies, void* workspace,
             size_t ws_bytes, void* stream, pic_sim** out) {
    GP_CHECK(validate(cfg, species, nspecies));
    if (!out) return fail(PIC_EINVAL, "out is NULL");
    *out = nullptr;
    if (!workspace) return fail(PIC_EINVAL, "workspace is NULL");
    if ((uintptr_t)workspace % ALIGN) return fail(PIC_EINVAL, "workspace must be 256-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    pic_sim* s = new (std::nothrow) pic_sim();
    if (!s) return fail(PIC_ENOMEM, "host allocation failed");
    s->cfg = *cfg;
    s->nspecies = nspecies;
    s->d = make_dims(*cfg);
    int rc = check_tile_fits(*cfg, s->d);
    size_t work = 0;
    if (rc == PIC_OK) rc = shared_plans(*cfg, s->d, &s->plans);
    if (rc == PIC_OK) {
        s->plan_r2c = s->plans->r2c;
        s->plan_c2r = s->plans->c2r;
        work = s->plans->work;
    }
    if (rc != PIC_OK) {
        pic_destroy(s);
        return rc;
    }
    int64_t n[PIC_MAX_SPECIES];
    for (int k = 0; k < nspecies; ++k) n[k] = species[k].n;
    make_layout(*cfg, s->d, n, nspecies, work, s->L);
    if (ws_bytes < s->L.total) {
        size_t need = s->L.total;
        pic_destroy(s);
        return fail(PIC_ENOMEM, "workspace has " + std::to_string(ws_bytes) + " bytes, needs " +
                                    std::to_string(need));
    }
    char* w = (char*)workspace;
    const Layout& L = s->L;
    s->ws = w;
    s->ws_bytes = ws_bytes;
    for (int k = 0; k < nspecies; ++k) {
        SpeciesDev& sp = s->sp[k];
        sp.q = species[k].q;
        sp.m = species[k].m;
        sp.w = species[k].w;
        sp.n = species[k].n;
        sp.cell = (int32_t*)(w + L.off_species[k][0]);
        for (int dd = 0; dd < 3; ++dd) {
            sp.off[dd] = w + L.off_species[k][1 + dd];
            sp.u[dd] = w + L.off_species[k][4 + dd];
        }
        sp.bin_start = (int32_t*)(w + L.off_species[k][7]);
        sp.cell_start = (int32_t*)(w + L.off_species[k][8]);
    }
    s->tmp_cell = (int32_t*)(w + L.off_tmp[0]);
    for (int dd = 0; dd < 3; ++dd) {
        s->tmp_off[dd] = w + L.off_tmp[1 + dd];
        s->tmp_u[dd] = w + L.off_tmp[4 + dd];
    }
    s->tmp_rank = (int32_t*)(w + L.off_tmp[7]);
    s->key_cnt = (int32_t*)(w + L.off_key_cnt);
    s->tile_sum = (int32_t*)(w + L.off_tile_sum);
    s->F = w + L.off_F;
    s->S = w + L.off_S;
    s->S64 = cfg->deterministic ? (long long*)(w + L.off_S64) : nullptr;
    s->desc = cfg->deterministic ? (char*)(w + L.off_desc) : nullptr;
#ifdef PIC_CHECKED
    // the checker's own test: GALPIC_CHECKED_INJECT=gather shifts the gather's tile index
    // by one tile (still inside the CTA's shared memory) so that its bound test must fire
    {
        const char* inj = getenv("GALPIC_CHECKED_INJECT");
        const int TEc = 8 + (cfg->shape_order == 1 ? 2 : 4) - 1 + 2 * cfg->tile_margin;
        s->inject = (inj && strcmp(inj, "gather") == 0) ? TEc * TEc * TEc : 0;
    }
#endif
    s->fix_exp = fixed_point_exponent(*cfg, species, nspecies);
    s->EBh = w + L.off_EBh;
    s->EBs = w + L.off_EBs;
    s->Sh = w + L.off_Sh;
    s->Rn = w + L.off_Rn;
    s->Tab = w + L.off_Tab;
    s->K = (double*)(w + L.off_K);
    s->Kt = w + L.off_Kt;
    s->Ph = w + L.off_Ph;
    s->fftwork = w + L.off_fftwork;
    s->epart = (double*)(w + L.off_epart);
    s->energy_blocks = energy_blocks_for(s->d.N);
    s->cnt = (unsigned long long*)(w + L.off_cnt);
    s->status = (int32_t*)(w + L.off_status);

#define INIT_TRY(expr)              \
    do {                            \
        int rc_ = (expr);           \
        if (rc_ != PIC_OK) {        \
            std::string m_ = g_err; \
            pic_destroy(s);         \
            g_err = m_;             \
            return rc_;             \
        }                           \
    } while (0)

    {
        cudaError_t e = cudaStreamCreateWithFlags(&s->priv, cudaStreamNonBlocking);
        INIT_TRY(e == cudaSuccess ? PIC_OK : fail(PIC_ECUDA, cudaGetErrorString(e)));
    }
    INIT_TRY(cudaMemsetAsync(s->cnt, 0, CNT_COUNT * sizeof(unsigned long long), st) == cudaSuccess
                 ? PIC_OK : fail(PIC_ECUDA, "memset counters"));
    INIT_TRY(cudaMemsetAsync(s->status, 0, sizeof(int32_t), st) == cudaSuccess
                 ? PIC_OK : fail(PIC_ECUDA, "memset status"));
    {
        int64_t ntot = 0;
        for (int k = 0; k < nspecies; ++k) ntot += n[k];
        // re-sort when more than 1/32 of the particles left their bin or more than
        // 1/1024 left their tile (a pageable source is staged before the copy returns)
        static thread_local unsigned long long thr[2];
        thr[0] = (unsigned long long)std::max<int64_t>(0, ntot / 32);
        thr[1] = (unsigned long long)std::max<int64_t>(0, ntot / 1024);
        INIT_TRY(cudaMemcpyAsync(s->cnt + CNT_THRESHOLD, thr, sizeof(thr), cudaMemcpyHostToDevice,
                                 st) == cudaSuccess ? PIC_OK : fail(PIC_ECUDA, "threshold"));
    }
    const size_t Tb = real_bytes(s);
    // The k-space tables depend on the configuration alone: they are built on the run's
    // private stream while the particles are copied (or generated) and sorted on `st`,
    // which waits for them before the initial fields.
    struct EventPair {
        cudaEvent_t a = nullptr, b = nullptr;
        ~EventPair() {
            if (a) cudaEventDestroy(a);
            if (b) cudaEventDestroy(b);
        }
    } tev;
    INIT_TRY(cudaEventCreateWithFlags(&tev.a, cudaEventDisableTiming) == cudaSuccess &&
                     cudaEventCreateWithFlags(&tev.b, cudaEventDisableTiming) == cudaSuccess &&
                     cudaEventRecord(tev.a, st) == cudaSuccess && cudaStreamWaitEvent(s->priv, tev.a, 0) == cudaSuccess
                 ? PIC_OK : fail(PIC_ECUDA, "table stream events"));
    count_launches(s, 2);   // wavenumbers, tables
    INIT_TRY(launch_build_tables(s, s->priv));
    INIT_TRY(cudaEventRecord(tev.b, s->priv) == cudaSuccess ? PIC_OK : fail(PIC_ECUDA, "table event"));
    for (int k = 0; k < nspecies; ++k) {
        // every bin range starts empty (a species with no particles is never sorted)
        INIT_TRY(cudaMemsetAsync(s->sp[k].bin_start, 0, (s->d.nbins + 1) * sizeof(int32_t), st) ==
                         cudaSuccess ? PIC_OK : fail(PIC_ECUDA, "memset bin_start"));
        INIT_TRY(cudaMemsetAsync(s->sp[k].cell_start, 0, (sort_keys(s->d) + 1) * sizeof(int32_t), st) ==
                         cudaSuccess ? PIC_OK : fail(PIC_ECUDA, "memset cell_start"));
    }
    for (int k = 0; k < nspecies; ++k) {
        const pic_species& spec = species[k];
        SpeciesDev& sp = s->sp[k];
        if (sp.n == 0) continue;
        count_launches(s, 1);   // generator or sanitizer
        if (spec.ppc[0] > 0) {
            INIT_TRY(launch_generate(s, k, &spec, st));
        } else {
            cudaError_t e = cudaMemcpyAsync(sp.cell, spec.cell, sp.n * 4, cudaMemcpyDefault, st);
            for (int dd = 0; dd < 3 && e == cudaSuccess; ++dd) {
                e = cudaMemcpyAsync(sp.off[dd], spec.off[dd], sp.n * Tb, cudaMemcpyDefault, st);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(sp.u[dd], spec.u[dd], sp.n * Tb, cudaMemcpyDefault, st);
            }
            INIT_TRY(e == cudaSuccess ? PIC_OK : fail(PIC_ECUDA, std::string("particle copy: ") +
                                                                     cudaGetErrorString(e)));
            INIT_TRY(launch_sanitize(s, k, st));
        }
    }
    INIT_TRY(set_force_sort(s, st));
    INIT_TRY(sort_particles(s, st));
    INIT_TRY(cudaStreamWaitEvent(st, tev.b, 0) == cudaSuccess ? PIC_OK : fail(PIC_ECUDA, "table wait"));
    count_launches(s, 2);   // initial fields, scaled copy
    INIT_TRY(deposit_sources(s, PASS_DEPOSIT, st));
    INIT_TRY(exec_r2c(s, st));
    INIT_TRY(launch_init_fields(s, st));
    INIT_TRY(launch_master_to_scratch(s, st));
    INIT_TRY(exec_c2r(s, st));
    bool copied = false;
    for (int k = 0; k < nspecies; ++k) copied |= species[k].n > 0 && species[k].ppc[0] <= 0;
    if (copied) {   // report bad caller input now (the generator never produces any)
        int32_t stv = 0;
        cudaError_t e = cudaStreamSynchronize(st);
        if (e == cudaSuccess) e = cudaMemcpy(&stv, s->status, sizeof(stv), cudaMemcpyDeviceToHost);
        INIT_TRY(e == cudaSuccess ? PIC_OK : fail(PIC_ECUDA, std::string("init: ") + cudaGetErrorString(e)));
        INIT_TRY((stv & PIC_STATUS_BADINPUT) == 0
                     ? PIC_OK : fail(PIC_EINVAL, "particle input: a cell outside [0, N) or an offset outside [0, 1)"));
    }
    if (s->desc) {   // the run's parameter tables (pageable source: staged before the call returns)
        const size_t pb = s->cfg.precision == 64 ? pass_desc_bytes_fp64() : pass_desc_bytes_fp32();
        INIT_TRY(pb <= DESC_KSPACE && kspace_desc_bytes(s->cfg.precision) <= DESC_BYTES - DESC_KSPACE
                     ? PIC_OK : fail(PIC_EINVAL, "parameter tables larger than their region"));
        std::vector<char> host(DESC_BYTES, 0);
        if (s->cfg.precision == 64)
            fill_pass_desc_fp64(s, host.data(), nullptr, nullptr, nullptr);
        else
            fill_pass_desc_fp32(s, host.data(), nullptr, nullptr, nullptr);
        fill_kspace_desc(s, host.data() + DESC_KSPACE, nullptr, nullptr);
        INIT_TRY(cudaMemcpyAsync(s->desc, host.data(), DESC_BYTES, cudaMemcpyHostToDevice, st) == cudaSuccess
                     ? PIC_OK : fail(PIC_ECUDA, "parameter tables"));
    }
#undef INIT_TRY
    *out = s;
    return PIC_OK;
}

int pic_destroy(pic_sim* s) {
    if (!s) return PIC_OK;
    // Only the run's own graph, private stream and events are released here; the
    // caller has finished (or synchronised) the work it enqueued on its streams.
    if (s->priv) cudaStreamSynchronize(s->priv);
    many_forget(s);
    if (s->graph_ok) cudaGraphExecDestroy(s->graph);
    for (auto& r : s->recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : s->event_pool) cudaEventDestroy(e);
    if (s->priv) cudaStreamDestroy(s->priv);
    delete s;
    return PIC_OK;
}

int pic_deposit(pic_sim* s, void* stream) {
    if (!s) return fail(PIC_EINVAL, "sim is NULL");
    return deposit_sources(s, PASS_DEPOSIT, (cudaStream_t)stream);
}

int pic_gather_push(pic_sim* s, void* stream) {
    if (!s) return fail(PIC_EINVAL, "sim is NULL");
    return gather_push(s, (cudaStream_t)stream);
}

int pic_field_update(pic_sim* s, void* stream) {
    if (!s) return fail(PIC_EINVAL, "sim is NULL");
    return field_update(s, (cudaStream_t)stream);
}

int pic_step(pic_sim* s, int nsteps, void* stream) {
    if (!s) return fail(PIC_EINVAL, "sim is NULL");
    if (nsteps < 0) return fail(PIC_EINVAL, "nsteps < 0");
    if (!s->graph_ok) GP_CHECK(capture_step(s));
    cudaStream_t st = (cudaStream_t)stream;
    for (int i = 0; i < nsteps; ++i) GP_CUDA(cudaGraphLaunch(s->graph, st));
    s->steps += nsteps;
    s->launches += (int64_t)nsteps * s->graph_kernels;
    return PIC_OK;
}

int pic_step_coupled(pic_sim** sims, int nsims, int nsteps, void* stream) {
    GP_CHECK(check_coupled(sims, nsims));
    if (nsteps < 0) return fail(PIC_EINVAL, "nsteps < 0");
    cudaStream_t st = (cudaStream_t)stream;
    GP_CHECK(couple_fields(sims, nsims, true, st));   // total fields at the current step
    for (int i = 0; i < nsteps; ++i) {
        for (int k = 0; k < nsims; ++k) GP_CHECK(gather_push(sims[k], st));
        for (int k = 0; k < nsims; ++k) {
            GP_CHECK(field_update_spectral(sims[k], st));
            sims[k]->steps += 1;
        }
        GP_CHECK(couple_fields(sims, nsims, false, st));
    }
    return PIC_OK;
}

int pic_diag_energy(pic_sim* s, double* out_dev, void* stream) {
    if (!s || !out_dev) return fail(PIC_EINVAL, "sim or out_dev is NULL");
    StageTimer t(s, STAGE_ENERGY, (cudaStream_t)stream);
    count_launches(s, 2);
    return launch_energy(s, out_dev, (cudaStream_t)stream);
}

static int buffer_of(pic_sim* s, int which, char** ptr, size_t* bytes) {
    const size_t T = real_bytes(s);
    const int64_t N = s->d.N, M = s->d.M;
    switch (which) {
        case PIC_BUF_E: *ptr = (char*)s->F; *bytes = 3 * N * T; break;
        case PIC_BUF_B: *ptr = (char*)s->F + 3 * N * T; *bytes = 3 * N * T; break;
        case PIC_BUF_J: *ptr = (char*)s->S; *bytes = 3 * N * T; break;
        case PIC_BUF_RHO: *ptr = (char*)s->S + 3 * N * T; *bytes = N * T; break;
        case PIC_BUF_E_HAT: *ptr = (char*)s->EBh; *bytes = 3 * M * 2 * T; break;
        case PIC_BUF_B_HAT: *ptr = (char*)s->EBh + 3 * M * 2 * T; *bytes = 3 * M * 2 * T; break;
        case PIC_BUF_RHO_HAT: *ptr = (char*)s->Rn; *bytes = M * 2 * T; break;
        case PIC_BUF_SRC_HAT: *ptr = (char*)s->Sh; *bytes = 4 * M * 2 * T; break;
        case PIC_BUF_TABLES: *ptr = (char*)s->Tab; *bytes = 6 * M * 2 * T; break;
        case PIC_BUF_STATUS: *ptr = (char*)s->status; *bytes = sizeof(int32_t); break;
        default: return fail(PIC_EINVAL, "unknown buffer id " + std::to_string(which));
    }
    return PIC_OK;
}

int pic_get(pic_sim* s, int which, void* dst, size_t bytes, void* stream) {
    if (!s || !dst) return fail(PIC_EINVAL, "sim or dst is NULL");
    char* p;
    size_t n;
    GP_CHECK(buffer_of(s, which, &p, &n));
    if (bytes != n) return fail(PIC_EINVAL, "buffer has " + std::to_string(n) + " bytes, got " +
                                                std::to_string(bytes));
    GP_CUDA(cudaMemcpyAsync(dst, p, n, cudaMemcpyDefault, (cudaStream_t)stream));
    return PIC_OK;
}

int pic_get_line(pic_sim* s, int component, int ix, int iy, void* dst, void* stream) {
    if (!s || !dst) return fail(PIC_EINVAL, "sim or dst is NULL");
    if (component < 0 || component > 5) return fail(PIC_EINVAL, "component must be 0..5 (Ex..Bz)");
    if (ix < 0 || ix >= s->d.nx || iy < 0 || iy >= s->d.ny) return fail(PIC_EINVAL, "line outside the grid");
    const size_t T = real_bytes(s);
    const char* src = (const char*)s->F + ((size_t)component * s->d.N + ((size_t)ix * s->d.ny + iy) * s->d.nz) * T;
    GP_CUDA(cudaMemcpyAsync(dst, src, (size_t)s->d.nz * T, cudaMemcpyDefault, (cudaStream_t)stream));
    return PIC_OK;
}

int pic_set(pic_sim* s, int which, const void* src, size_t bytes, void* stream) {
    if (!s || !src) return fail(PIC_EINVAL, "sim or src is NULL");
    if (which != PIC_BUF_E_HAT && which != PIC_BUF_B_HAT && which != PIC_BUF_RHO_HAT)
        return fail(PIC_EINVAL, "only E_HAT, B_HAT and RHO_HAT can be set");
    char* p;
    size_t n;
    GP_CHECK(buffer_of(s, which, &p, &n));
    if (bytes != n) return fail(PIC_EINVAL, "buffer has " + std::to_string(n) + " bytes, got " +
                                                std::to_string(bytes));
    cudaStream_t st = (cudaStream_t)stream;
    GP_CUDA(cudaMemcpyAsync(p, src, n, cudaMemcpyDefault, st));
    if (which != PIC_BUF_RHO_HAT) {
        count_launches(s, 1);
        GP_CHECK(launch_master_to_scratch(s, st));
        GP_CHECK(exec_c2r(s, st));
    }
    return PIC_OK;
}

int pic_tune(pic_sim* s, int32_t chosen[2], void* stream) {
    if (!s) return fail(PIC_EINVAL, "sim is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    struct Ev {
        cudaEvent_t e = nullptr;
        ~Ev() { if (e) cudaEventDestroy(e); }
    } a, b;
    GP_CUDA(cudaEventCreate(&a.e));
    GP_CUDA(cudaEventCreate(&b.e));
    // candidate deposit strategies: FP32 quadratic/cubic 0..3, linear 0 and 4 (one thread
    // per cell), deterministic runs their single fixed-point deposit
    int cand[4] = {0, 0, 0, 0};
    int nstrat = 1;
    if (!s->cfg.deterministic) {
        if (s->cfg.precision == 32 && s->cfg.shape_order >= 2) {
            nstrat = 4;
            for (int k = 0; k < 4; ++k) cand[k] = k;
        } else if (s->cfg.shape_order == 1) {
            nstrat = 2;
            cand[1] = 4;
        }
    }
    const int keep_m = s->d.margin, keep_d = s->cfg.deposit;
    int best_m = keep_m, best_d = keep_d;
    float tbest = 0.f;
    bool first = true;
    for (int m = 0; m < 2; ++m)
        for (int ki = 0; ki < nstrat; ++ki) {
            const int k = cand[ki];
            s->d.margin = m;
            s->cfg.deposit = k;
            // one full step to settle (a re-sort may be due), then two timed ones;
            // only the particle pass (with its re-sort) is timed
            int rc = gather_push(s, st);
            if (rc == PIC_OK) rc = field_update(s, st);
            float ms = 0.f;
            for (int r = 0; r < 2 && rc == PIC_OK; ++r) {
                float t = 0.f;
                if (cudaEventRecord(a.e, st) != cudaSuccess) rc = fail(PIC_ECUDA, "event");
                if (rc == PIC_OK) rc = gather_push(s, st);
                if (rc == PIC_OK && cudaEventRecord(b.e, st) != cudaSuccess) rc = fail(PIC_ECUDA, "event");
                if (rc == PIC_OK) rc = field_update(s, st);
                if (rc == PIC_OK && (cudaEventSynchronize(b.e) != cudaSuccess ||
                                     cudaEventElapsedTime(&t, a.e, b.e) != cudaSuccess))
                    rc = fail(PIC_ECUDA, "tuning timing");
                ms += t;
            }
            if (rc != PIC_OK) {
                s->d.margin = keep_m;
                s->cfg.deposit = keep_d;
                return rc;
            }
            s->steps += 3;
            // a later candidate must be clearly faster (2 %): timing noise does not flip
            // the choice between near-equal candidates, and the earlier (simpler) one stays
            if (first || ms < 0.98f * tbest) {
                tbest = ms;
                best_m = m;
                best_d = k;
                first = false;
            }
        }
    s->d.margin = best_m;
    s->cfg.tile_margin = best_m;
    s->cfg.deposit = best_d;
    if (s->graph_ok) {   // the captured step uses the previous choice
        cudaGraphExecDestroy(s->graph);
        s->graph_ok = false;
    }
    if (chosen) {
        chosen[0] = best_m;
        chosen[1] = best_d;
    }
    return PIC_OK;
}

int pic_sort_policy(pic_sim* s, int64_t home_miss_threshold, int64_t far_threshold, void* stream) {
    if (!s) return fail(PIC_EINVAL, "sim is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    static thread_local unsigned long long v[2];
    if (home_miss_threshold >= 0) {
        v[0] = (unsigned long long)home_miss_threshold;
        GP_CUDA(cudaMemcpyAsync(s->cnt + CNT_THRESHOLD, &v[0], sizeof(v[0]), cudaMemcpyHostToDevice, st));
    }
    if (far_threshold >= 0) {
        v[1] = (unsigned long long)far_threshold;
        GP_CUDA(cudaMemcpyAsync(s->cnt + CNT_FAR_THRESHOLD, &v[1], sizeof(v[1]), cudaMemcpyHostToDevice, st));
    }
    return PIC_OK;   // pageable sources are staged before the copies return
}

int pic_add_fields(pic_sim* s, const void* fields, void* stream) {
    if (!s || !fields) return fail(PIC_EINVAL, "sim or fields is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t T = real_bytes(s);
    const int64_t N = s->d.N, M = s->d.M;
    // the real field grids are recomputed below, so they serve as the transform input
    GP_CUDA(cudaMemcpyAsync(s->F, fields, 6 * N * T, cudaMemcpyDefault, st));
    char* out = (char*)s->EBs;
    GP_CHECK(exec_r2c_on(s, s->F, out, st));                                          // Ex Ey Ez Bx
    GP_CHECK(exec_r2c_on(s, (char*)s->F + 2 * N * T, out + 2 * M * 2 * T, st));      // Ez Bx By Bz
    count_launches(s, 2);
    GP_CHECK(launch_add_spectra(s, s->EBs, st));
    GP_CHECK(launch_master_to_scratch(s, st));
    GP_CHECK(exec_c2r(s, st));
    return PIC_OK;
}

int pic_get_particles(pic_sim* s, int k, int32_t* cell, void* off[3], void* u[3], void* stream) {
    if (!s || k < 0 || k >= s->nspecies) return fail(PIC_EINVAL, "bad sim or species index");
    cudaStream_t st = (cudaStream_t)stream;
    const SpeciesDev& sp = s->sp[k];
    const size_t T = real_bytes(s);
    if (cell) GP_CUDA(cudaMemcpyAsync(cell, sp.cell, sp.n * 4, cudaMemcpyDefault, st));
    for (int d = 0; d < 3; ++d) {
        if (off && off[d]) GP_CUDA(cudaMemcpyAsync(off[d], sp.off[d], sp.n * T, cudaMemcpyDefault, st));
        if (u && u[d]) GP_CUDA(cudaMemcpyAsync(u[d], sp.u[d], sp.n * T, cudaMemcpyDefault, st));
    }
    return PIC_OK;
}

int pic_set_particles(pic_sim* s, int k, const int32_t* cell, const void* const off[3],
                      const void* const u[3], void* stream) {
    if (!s || k < 0 || k >= s->nspecies) return fail(PIC_EINVAL, "bad sim or species index");
    if (!cell || !off || !u) return fail(PIC_EINVAL, "particle arrays are NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const SpeciesDev& sp = s->sp[k];
    const size_t T = real_bytes(s);
    GP_CUDA(cudaMemcpyAsync(sp.cell, cell, sp.n * 4, cudaMemcpyDefault, st));
    for (int d = 0; d < 3; ++d) {
        if (!off[d] || !u[d]) return fail(PIC_EINVAL, "particle arrays are NULL");
        GP_CUDA(cudaMemcpyAsync(sp.off[d], off[d], sp.n * T, cudaMemcpyDefault, st));
        GP_CUDA(cudaMemcpyAsync(sp.u[d], u[d], sp.n * T, cudaMemcpyDefault, st));
    }
    count_launches(s, 1);
    GP_CHECK(launch_sanitize(s, k, st));
    GP_CHECK(set_force_sort(s, st));
    return sort_particles(s, st);
}

int pic_sort(pic_sim* s, void* stream) {
    if (!s) return fail(PIC_EINVAL, "sim is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    GP_CHECK(set_force_sort(s, st));
    return sort_particles(s, st);
}

int pic_status(pic_sim* s, int32_t* status_out) {
    if (!s) return fail(PIC_EINVAL, "sim is NULL");
    GP_CUDA(cudaDeviceSynchronize());
    int32_t v = 0;
    GP_CUDA(cudaMemcpy(&v, s->status, sizeof(v), cudaMemcpyDeviceToHost));
    GP_CUDA(cudaMemset(s->status, 0, sizeof(v)));
    if (status_out) *status_out = v;
    if (v & PIC_STATUS_BOUNDS) return fail(PIC_EBOUNDS, "an index left its buffer's range (checked build)");
    if (v & PIC_STATUS_NONFINITE) return fail(PIC_ENONFINITE, "non-finite field value seen");
    return PIC_OK;
}

int pic_counters(pic_sim* s, int64_t out[6]) {
    if (!s || !out) return fail(PIC_EINVAL, "sim or out is NULL");
    GP_CUDA(cudaDeviceSynchronize());
    unsigned long long c[CNT_COUNT];
    GP_CUDA(cudaMemcpy(c, s->cnt, sizeof(c), cudaMemcpyDeviceToHost));
    out[0] = s->steps;
    out[1] = (int64_t)c[CNT_SORTS];
    out[2] = (int64_t)c[CNT_HOME_MISS];
    out[3] = (int64_t)c[CNT_FAR];
    out[4] = s->launches;
    out[5] = 0;
    return PIC_OK;
}

int pic_profile(pic_sim* s, int enable) {
    if (!s) return fail(PIC_EINVAL, "sim is NULL");
    GP_CUDA(cudaDeviceSynchronize());
    for (auto& r : s->recs) {
        s->event_pool.push_back(r.a);
        s->event_pool.push_back(r.b);
    }
    s->recs.clear();
    s->profiling = enable != 0;
    return PIC_OK;
}

int pic_profile_read(pic_sim* s, double ms[8], int64_t count[8]) {
    if (!s || !ms || !count) return fail(PIC_EINVAL, "sim, ms or count is NULL");
    for (int i = 0; i < STAGE_COUNT; ++i) {
        ms[i] = 0.0;
        count[i] = 0;
    }
    for (auto& r : s->recs) {
        GP_CUDA(cudaEventSynchronize(r.b));
        float t = 0.f;
        GP_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
        ms[r.stage] += t;
        count[r.stage] += 1;
        s->event_pool.push_back(r.a);
        s->event_pool.push_back(r.b);
    }
    s->recs.clear();
    return PIC_OK;
}

int pic_sizes(pic_sim* s, int64_t* n_cells, int64_t* n_modes) {
    if (!s) return fail(PIC_EINVAL, "sim is NULL");
    if (n_cells) *n_cells = s->d.N;
    if (n_modes) *n_modes = s->d.M;
    return PIC_OK;
}

}  // extern "C"
