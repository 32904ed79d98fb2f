// Domain decomposition of the field update along z on one GPU: pic_decomposed_footprint,
// pic_step_decomposed.
//
// The paper's conclusion names domain decomposition with arbitrary-order (finite) spectral
// stencils as the way to many processors: each subdomain transforms only its cells plus
// guard cells, and a finite stencil keeps the update's reach short. Here the P subdomains
// of one run are all on this GPU: every step, after the ordinary particle pass (global
// deposit), a gather kernel copies each window (the subdomain's nz/P cells plus `guard`
// cells on either side, periodic) of the real E, B, J, rho^{n+1} and rho^n into one
// buffer; one batched R2C transforms all windows, one launch applies the Galilean-PSATD
// update on every window's modes (the window's own wavenumbers; no current correction,
// whose 1/k^2 reaches the whole grid; the Nyquist planes of a window are updated like
// any mode, since the window's wrap makes them large); one batched C2R brings E, B back;
// and a scatter kernel keeps each window's own cells. The real E, B are the state
// between steps. At the end of a call the run's spectral E, B, rho^n and source spectra
// are refreshed as the forward transforms of the real state (inverse-transforming them
// gives the real state back), so pic_step can continue from it.
#include <string.h>

#include <algorithm>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "common.cuh"

namespace galpic {
namespace {

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

constexpr int NWIN_COMP = 11;   // E (3), B (3), J (3), rho^{n+1}, rho^n

struct DecompLayout {
    int nl, ext, nzh;
    int64_t Nw, Mw;
    size_t win_real, win_spec, ebs, out_real, rho_real, K, Kt, tab, desc, work, total;
};

DecompLayout decomp_layout(const pic_sim* s, int P, int g, size_t fft_work) {
    DecompLayout L;
    const size_t T = s->cfg.precision == 64 ? 8 : 4;
    L.nl = s->d.nz / P;
    L.ext = L.nl + 2 * g;
    L.nzh = L.ext / 2 + 1;
    L.Nw = (int64_t)s->d.nx * s->d.ny * L.ext;
    L.Mw = (int64_t)s->d.nx * s->d.ny * L.nzh;
    size_t o = 0;
    auto take = [&](size_t b) {
        size_t at = o;
        o = up256(o + b);
        return at;
    };
    L.win_real = take((size_t)P * NWIN_COMP * L.Nw * T);
    L.win_spec = take((size_t)P * NWIN_COMP * L.Mw * 2 * T);
    L.ebs = take((size_t)P * 6 * L.Mw * 2 * T);
    L.out_real = take((size_t)P * 6 * L.Nw * T);
    L.rho_real = take((size_t)s->d.N * T);
    L.K = take((size_t)(s->d.nx + s->d.ny + L.nzh) * 8);
    L.Kt = take((size_t)(s->d.nx + s->d.ny + L.nzh) * T);
    L.tab = take((size_t)6 * L.Mw * 2 * T);
    L.desc = take((size_t)P * kspace_desc_bytes(s->cfg.precision));
    L.work = take(std::max<size_t>(fft_work, 1));
    L.total = o;
    return L;
}

struct DecompPlan {
    cufftHandle r2c = 0, c2r = 0;
    size_t work = 0;
    std::mutex mu;
};

std::mutex g_mu;
std::map<std::tuple<int, int, int, int, int, int>, std::unique_ptr<DecompPlan>> g_plans;

// Batched plans over the windows: R2C of 11 P window grids, C2R of 6 P.
int decomp_plan(const pic_sim* s, int P, int ext, DecompPlan** out) {
    int dev = 0;
    GP_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_mu);
    auto key = std::make_tuple(dev, s->d.nx, s->d.ny, ext, s->cfg.precision, P);
    auto it = g_plans.find(key);
    if (it == g_plans.end()) {
        std::unique_ptr<DecompPlan> e(new DecompPlan());
        const long long nzh = ext / 2 + 1;
        long long n[3] = {s->d.nx, s->d.ny, ext};
        long long cn[3] = {s->d.nx, s->d.ny, nzh};
        const long long Nw = (long long)s->d.nx * s->d.ny * ext, Mw = (long long)s->d.nx * s->d.ny * nzh;
        const bool dbl = s->cfg.precision == 64;
        size_t w1 = 0, w2 = 0;
        auto bad = [&](cufftResult r, const char* what) {
            if (e->r2c) cufftDestroy(e->r2c);
            if (e->c2r) cufftDestroy(e->c2r);
            return fail(PIC_ECUFFT, std::string(what) + ": cufft error " + std::to_string((int)r));
        };
        cufftResult r;
        if ((r = cufftCreate(&e->r2c)) != CUFFT_SUCCESS) return bad(r, "create");
        if ((r = cufftCreate(&e->c2r)) != CUFFT_SUCCESS) return bad(r, "create");
        if ((r = cufftSetAutoAllocation(e->r2c, 0)) != CUFFT_SUCCESS) return bad(r, "auto allocation");
        if ((r = cufftSetAutoAllocation(e->c2r, 0)) != CUFFT_SUCCESS) return bad(r, "auto allocation");
        if ((r = cufftMakePlanMany64(e->r2c, 3, n, n, 1, Nw, cn, 1, Mw, dbl ? CUFFT_D2Z : CUFFT_R2C,
                                     (long long)NWIN_COMP * P, &w1)) != CUFFT_SUCCESS)
            return bad(r, "window R2C plan");
        if ((r = cufftMakePlanMany64(e->c2r, 3, n, cn, 1, Mw, n, 1, Nw, dbl ? CUFFT_Z2D : CUFFT_C2R, 6LL * P,
                                     &w2)) != CUFFT_SUCCESS)
            return bad(r, "window C2R plan");
        e->work = std::max(w1, w2);
        it = g_plans.emplace(key, std::move(e)).first;
    }
    *out = it->second.get();
    return PIC_OK;
}

// Window buffer [P][11][nx][ny][ext] from the global real grids: window w covers the
// global z nodes (w nl - g + j) mod nz, j = 0 .. ext-1.
template <typename T>
__global__ void gather_windows_kernel(T* __restrict__ win, const T* __restrict__ F, const T* __restrict__ S,
                                      const T* __restrict__ rho0, int P, int nxy, int nz, int nl, int g, int ext) {
    const int64_t per = (int64_t)nxy * ext;
    const int64_t total = (int64_t)P * NWIN_COMP * per;
    const int64_t N = (int64_t)nxy * nz;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(i % ext);
        const int64_t r = i / ext;
        const int xy = (int)(r % nxy);
        const int64_t r2 = r / nxy;
        const int q = (int)(r2 % NWIN_COMP);
        const int w = (int)(r2 / NWIN_COMP);
        int z = w * nl - g + j;
        z %= nz;
        if (z < 0) z += nz;
        const int64_t at = (int64_t)xy * nz + z;
        T v;
        if (q < 6)
            v = F[q * N + at];                 // E, B
        else if (q < 10)
            v = S[(q - 6) * N + at];           // J, rho^{n+1}
        else
            v = rho0[at];                      // rho^n
        win[i] = v;
    }
}

// Each window's own cells of E, B ([P][6][nx][ny][ext], C2R output) back to the global grid.
template <typename T>
__global__ void scatter_windows_kernel(T* __restrict__ F, const T* __restrict__ out, int P, int nxy, int nz, int nl,
                                       int g, int ext) {
    const int64_t N = (int64_t)nxy * nz;
    const int64_t total = 6 * N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int z = (int)(i % nz);
        const int64_t r = i / nz;
        const int xy = (int)(r % nxy);
        const int q = (int)(r / nxy);
        const int w = z / nl;
        const int j = z - w * nl + g;
        F[i] = out[(((int64_t)w * 6 + q) * nxy + xy) * ext + j];
    }
}

int grid_for(int64_t n, int block) {
    int64_t gsz = (n + block - 1) / block;
    gsz = std::min<int64_t>(gsz, 152 * 16);
    return (int)std::max<int64_t>(1, gsz);
}

int check_decomp(const pic_sim* s, int P, int g) {
    if (!s) return fail(PIC_EINVAL, "sim is NULL");
    if (P < 1 || P > s->d.nz) return fail(PIC_EINVAL, "ndomains must be in [1, nz]");
    if (s->d.nz % P) return fail(PIC_EINVAL, "nz must be a multiple of ndomains");
    if (g < 0) return fail(PIC_EINVAL, "guard must be >= 0");
    if (s->d.nz / P + 2 * g < 2) return fail(PIC_EINVAL, "a window needs at least 2 nodes along z");
    if (s->cfg.current_correction && P > 1)
        return fail(PIC_EINVAL, "decomposed runs go without the current correction (its 1/k^2 is not local): "
                                "set current_correction = 0");
    if (s->cfg.stencil_order == 0 && P > 1)
        return fail(PIC_EINVAL, "decomposition needs a finite-order stencil (stencil_order >= 2): the spectral "
                                "solver's update reaches the whole window");
    return PIC_OK;
}

}  // namespace
}  // namespace galpic

using namespace galpic;

extern "C" {

int pic_decomposed_footprint(const pic_sim* sim, int ndomains, int guard, size_t* bytes_out) {
    GP_CHECK(check_decomp(sim, ndomains, guard));
    if (!bytes_out) return fail(PIC_EINVAL, "bytes_out is NULL");
    DecompPlan* dp = nullptr;
    GP_CHECK(decomp_plan(sim, ndomains, sim->d.nz / ndomains + 2 * guard, &dp));
    *bytes_out = decomp_layout(sim, ndomains, guard, dp->work).total;
    return PIC_OK;
}

int pic_step_decomposed(pic_sim* s, int ndomains, int guard, int nsteps, void* workspace, size_t ws_bytes,
                        void* stream) {
    GP_CHECK(check_decomp(s, ndomains, guard));
    if (nsteps < 0) return fail(PIC_EINVAL, "nsteps < 0");
    if (!workspace) return fail(PIC_EINVAL, "workspace is NULL");
    if ((uintptr_t)workspace % 256) return fail(PIC_EINVAL, "workspace must be 256-byte aligned");
    const int P = ndomains, g = guard;
    DecompPlan* dp = nullptr;
    GP_CHECK(decomp_plan(s, P, s->d.nz / P + 2 * g, &dp));
    const DecompLayout L = decomp_layout(s, P, g, dp->work);
    if (ws_bytes < L.total)
        return fail(PIC_ENOMEM, "decomposed workspace has " + std::to_string(ws_bytes) + " bytes, needs " +
                                    std::to_string(L.total));
    if (nsteps == 0) return PIC_OK;
    char* ws = (char*)workspace;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t T = s->cfg.precision == 64 ? 8 : 4;
    const int64_t N = s->d.N;
    const int nxy = s->d.nx * s->d.ny;

    // window factors, window k-space descriptors, and rho^n real from the last deposit
    GP_CHECK(launch_window_tables(s, L.ext, (double*)(ws + L.K), ws + L.Kt, ws + L.tab, st));
    {
        std::vector<char> host((size_t)P * kspace_desc_bytes(s->cfg.precision));
        const size_t db = kspace_desc_bytes(s->cfg.precision);
        for (int w = 0; w < P; ++w)
            fill_window_kspace_desc(s, host.data() + w * db, L.ext,
                                    ws + L.win_spec + (size_t)w * NWIN_COMP * L.Mw * 2 * T,
                                    ws + L.ebs + (size_t)w * 6 * L.Mw * 2 * T, ws + L.Kt, ws + L.tab);
        GP_CUDA(cudaMemcpyAsync(ws + L.desc, host.data(), host.size(), cudaMemcpyHostToDevice, st));
    }
    GP_CUDA(cudaMemcpyAsync(ws + L.rho_real, (char*)s->S + 3 * N * T, N * T, cudaMemcpyDeviceToDevice, st));
    s->launches += 2;
    for (int n = 0; n < nsteps; ++n) {
        GP_CHECK(gather_push_stage(s, st));
        const int64_t nwin = (int64_t)P * NWIN_COMP * L.Nw;
        if (s->cfg.precision == 64)
            gather_windows_kernel<double><<<grid_for(nwin, 256), 256, 0, st>>>(
                (double*)(ws + L.win_real), (const double*)s->F, (const double*)s->S,
                (const double*)(ws + L.rho_real), P, nxy, s->d.nz, L.nl, g, L.ext);
        else
            gather_windows_kernel<float><<<grid_for(nwin, 256), 256, 0, st>>>(
                (float*)(ws + L.win_real), (const float*)s->F, (const float*)s->S, (const float*)(ws + L.rho_real),
                P, nxy, s->d.nz, L.nl, g, L.ext);
        GP_CUDA(cudaGetLastError());
        {
            std::lock_guard<std::mutex> lk(dp->mu);
            GP_CUFFT(cufftSetWorkArea(dp->r2c, ws + L.work));
            GP_CUFFT(cufftSetStream(dp->r2c, st));
            if (s->cfg.precision == 64)
                GP_CUFFT(cufftExecD2Z(dp->r2c, (cufftDoubleReal*)(ws + L.win_real),
                                      (cufftDoubleComplex*)(ws + L.win_spec)));
            else
                GP_CUFFT(cufftExecR2C(dp->r2c, (cufftReal*)(ws + L.win_real), (cufftComplex*)(ws + L.win_spec)));
        }
        GP_CHECK(launch_kspace_windows(s, ws + L.desc, P, L.Mw, st));
        {
            std::lock_guard<std::mutex> lk(dp->mu);
            GP_CUFFT(cufftSetWorkArea(dp->c2r, ws + L.work));
            GP_CUFFT(cufftSetStream(dp->c2r, st));
            if (s->cfg.precision == 64)
                GP_CUFFT(cufftExecZ2D(dp->c2r, (cufftDoubleComplex*)(ws + L.ebs), (cufftDoubleReal*)(ws + L.out_real)));
            else
                GP_CUFFT(cufftExecC2R(dp->c2r, (cufftComplex*)(ws + L.ebs), (cufftReal*)(ws + L.out_real)));
        }
        if (s->cfg.precision == 64)
            scatter_windows_kernel<double><<<grid_for(6 * N, 256), 256, 0, st>>>(
                (double*)s->F, (const double*)(ws + L.out_real), P, nxy, s->d.nz, L.nl, g, L.ext);
        else
            scatter_windows_kernel<float><<<grid_for(6 * N, 256), 256, 0, st>>>(
                (float*)s->F, (const float*)(ws + L.out_real), P, nxy, s->d.nz, L.nl, g, L.ext);
        GP_CUDA(cudaGetLastError());
        GP_CUDA(cudaMemcpyAsync(ws + L.rho_real, (char*)s->S + 3 * N * T, N * T, cudaMemcpyDeviceToDevice, st));
        s->steps += 1;
        s->launches += 3;
    }
    // the spectral state as the transform of the real one, so that pic_step continues
    const int64_t M = s->d.M;
    GP_CHECK(r2c_on(s, s->F, s->EBh, st));                                                  // Ex Ey Ez Bx
    GP_CHECK(r2c_on(s, (char*)s->F + 2 * N * T, (char*)s->EBh + 2 * M * 2 * T, st));      // Ez Bx By Bz
    GP_CHECK(r2c_on(s, s->S, s->Sh, st));                                                   // sources
    GP_CUDA(cudaMemcpyAsync(s->Rn, (char*)s->Sh + 3 * M * 2 * T, M * 2 * T, cudaMemcpyDeviceToDevice, st));
    return PIC_OK;
}

}  // extern "C"
