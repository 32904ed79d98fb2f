// Quasi-cylindrical Galilean-PSATD particle-in-cell step on the GPU (pic_cyl_*).
//
// The paper runs its boosted-frame results in a quasi-cylindrical spectral code (the
// implementation paragraph after the update equations). Fields are kept as azimuthal modes
// m = 0 .. M-1 on the (r, z) grid, F = F_0 + 2 Re sum_{m>=1} F_m e^{i m theta}, and in
// spectral space as the Cartesian amplitudes at phi = 0 of each mode: for a vector,
//   F_x + i F_y = -i H_{m+1}[F_r + i F_theta],  F_x - i F_y = i H_{m-1}[F_r - i F_theta],
//   F_z = H_m[F_z],  scalars H_m[g],
// with discrete Hankel transforms H_n along r (radial nodes r_j = (j + 1/2) dr; spectral
// nodes k_i = alpha_{b,i}/R, the zeros of J_b, b = max(m - 1, 0), Fourier-Bessel weights
// w_i = 2/(R^2 J_{b+1}(alpha_{b,i})^2); the inverse transform of order n is the synthesis
// f(r_j) = sum_i w_i J_n(k_i r_j) F_i; the forward transform is that matrix's exact inverse
// for |n| <= 1 and the midpoint quadrature F_i = sum_j f(r_j) J_n(k_i r_j) r_j dr of the
// Hankel integral for |n| >= 2, whose synthesis matrices have rows ~ (k r)^|n| at the axis
// and whose inverses would amplify the irregular part of particle deposits there) and a
// complex FFT along z. The Galilean-PSATD update, with v_gal along z, commutes with
// rotations about z, so on these amplitudes it is the Cartesian update at
// k = (k_r, 0, k_z): the k-space kernel of the Cartesian path runs it, on per-mode factors
// built by the Cartesian table builder at those k.
//
// Particles keep Cartesian positions and momenta (Boris push and Galilean drift as in the
// Cartesian step); deposits and gathers use linear shapes in r and z with the mode phases
// e^{-i m theta}, the annulus volumes V_j = 2 pi r_j dr dz, and the fold of the node below
// the axis (r = -dr/2 is the point dr/2 at theta + pi): factor (-1)^m for scalars and z
// components, (-1)^(m+1) for r and theta components.
//
// Set-up (FP64 on the GPU, once per run): the Bessel zeros by Newton's method on CUDA's
// jn, the synthesis matrices of orders m-1, m, m+1, the forward matrices (Gauss-Jordan
// inverses with partial pivoting for |n| <= 1, quadrature weights for |n| >= 2), the
// per-mode factors. Per step: the inverse
// transforms of spectral E, B to real mode fields (tiled real-by-complex matrix products
// along r for every mode and component in one launch, one batched complex FFT along z),
// the particle kernel, the forward transforms of J and rho, the k-space update of every
// mode in one launch.
#include <math.h>

#include <cmath>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "common.cuh"

struct pic_cyl {
    pic_cyl_config cfg;
    int nspecies;
    struct Sp {
        double q, m;
        int64_t n;
        void *w, *x[3], *u[3];   // buffer 0 of the particle arrays
        void* alt[7];            // buffer 1 (w, x, u); the device state says which is current
        int32_t *pid, *pid_alt;  // input index of each particle (buffers 0 and 1)
        int32_t* starts;         // per bin: first particle (nbins + 1), from the last sort
        void* state;             // CylSortState in device memory
    } sp[PIC_MAX_SPECIES];
    int32_t *key, *rank;         // per particle of the largest species: bin and rank in bin
    int32_t* counts;             // per bin: particles (during a sort)
    int nbz = 0, nbins = 0;
    int64_t G;          // nr * nz
    char* ws;
    // device arrays (carved from the caller's workspace)
    double* alpha;      // [M][nr] zeros of J_b of each mode's base order
    double* Kd;         // [M][nr + 1 + nz] k_r, 0, k_z (FP64)
    void* Kt;           // the same in the run's precision
    void* syn;          // [M][3][nr][nr] synthesis matrices of orders m+1, m-1, m (run precision)
    void* fwd;          // [M][3][nr][nr] their inverses
    double* tmp64;      // [3][2][nr][nr] FP64 scratch of the set-up (matrices and inverses)
    void* tab;          // [M][6][G] complex factors
    void* EBh;          // [M][6][G] spectral E, B
    void* Sh;           // [M][4][G] spectra of J, rho^{n+1}
    void* Rn;           // [M][G] spectral rho^n
    void* Fr;           // [M][6][G] real-space mode fields E_r, E_t, E_z, B_r, B_t, B_z
    void* Dr;           // [M][4][G] real-space mode deposits J_r, J_t, J_z, rho
    void* W1;           // [M][6][G] transform work
    void* W2;           // [M][6][G] transform work
    void* scratch;      // [M][6][G] k-space copy output (unused values)
    void* kdesc;        // [M] k-space parameter blocks
    void* gdesc;        // matrix-product batch tables: [2][3][GDESC_MAX] pointers (A, X, Y)
                        // of the inverse (fields) and forward (sources) transforms
    double* wsum;       // energy partial sums
    int32_t* status;
    void* fftwork;
    cufftHandle plan6 = 0, plan4 = 0;   // C2C along z: M*6*nr and M*4*nr rows
    int64_t steps = 0;
    // stage timing (pic_cyl_profile): 0 particles, 1 sources to spectral space, 2 k-space
    // update, 3 fields to real space, 4 the radial products inside stages 1 and 3
    bool prof = false;
    cudaEvent_t ev[5][2] = {};
    double prof_ms[5] = {};
    int64_t prof_n[5] = {};
};

namespace galpic {
namespace {

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

struct CylLayout {
    size_t alpha, Kd, Kt, syn, fwd, tmp64, tab, EBh, Sh, Rn, Fr, Dr, W1, W2, scratch, kdesc, gdesc, wsum, status,
        sp[PIC_MAX_SPECIES][7], alt[PIC_MAX_SPECIES][7], pid[PIC_MAX_SPECIES][2], starts[PIC_MAX_SPECIES],
        state[PIC_MAX_SPECIES], key, rank, counts, fftwork, total;
};

// Particle bins of the sorted deposit: CBR x CBZ cells in (r, z); the deposit tile of a bin
// reaches CPAD cells past it on every side.
constexpr int CBR = 8, CBZ = 16, CPAD = 2, CTR = CBR + 2 * CPAD, CTZ = CBZ + 2 * CPAD;
int cyl_nbz(int nz) { return (nz + CBZ - 1) / CBZ; }
int cyl_nbins(int nr, int nz) { return ((nr + CBR - 1) / CBR) * cyl_nbz(nz); }

constexpr int GDESC_MAX = 64;   // matrix-product batches per launch: M * 6

CylLayout cyl_layout(const pic_cyl_config& c, const int64_t* n, int ns, size_t fft_work) {
    CylLayout L;
    const size_t T = c.precision == 64 ? 8 : 4, C = 2 * T;
    const size_t M = c.nmodes, nr = c.nr, G = (size_t)c.nr * c.nz;
    size_t o = 0;
    auto take = [&](size_t b) {
        size_t at = o;
        o = up256(o + b);
        return at;
    };
    L.alpha = take(M * nr * 8);
    L.Kd = take(M * (nr + 1 + c.nz) * 8);
    L.Kt = take(M * (nr + 1 + c.nz) * T);
    L.syn = take(M * 3 * nr * nr * T);
    L.fwd = take(M * 3 * nr * nr * T);
    L.tmp64 = take(3 * 2 * nr * nr * 8);
    L.tab = take(M * 6 * G * C);
    L.EBh = take(M * 6 * G * C);
    L.Sh = take(M * 4 * G * C);
    L.Rn = take(M * G * C);
    L.Fr = take(M * 6 * G * C);
    L.Dr = take(M * 4 * G * C);
    L.W1 = take(M * 6 * G * C);
    L.W2 = take(M * 6 * G * C);
    L.scratch = take(M * 6 * G * C);
    L.kdesc = take(M * 256 * 8);
    L.gdesc = take(2 * 3 * GDESC_MAX * sizeof(void*));
    L.wsum = take(1024 * 8);
    L.status = take(8);
    int64_t nmax = 0;
    for (int k = 0; k < ns; ++k) {
        for (int q = 0; q < 7; ++q) L.sp[k][q] = take(n[k] * T);
        for (int q = 0; q < 7; ++q) L.alt[k][q] = take(n[k] * T);
        L.pid[k][0] = take(n[k] * 4);
        L.pid[k][1] = take(n[k] * 4);
        nmax = std::max(nmax, n[k]);
    }
    const size_t nb = cyl_nbins(c.nr, c.nz);
    for (int k = 0; k < ns; ++k) {
        L.starts[k] = take((nb + 1) * 4);
        L.state[k] = take(32);
    }
    L.key = take(nmax * 4);
    L.rank = take(nmax * 4);
    L.counts = take(nb * 4);
    L.fftwork = take(std::max<size_t>(fft_work, 1));
    L.total = o;
    return L;
}

int validate_cyl(const pic_cyl_config* c, const pic_cyl_species* sp, int ns) {
    if (!c) return fail(PIC_EINVAL, "config is NULL");
    if (c->nr < 2 || c->nr > 1024 || c->nz < 2) return fail(PIC_EINVAL, "need 2 <= nr <= 1024 and nz >= 2");
    if (c->nmodes < 1 || c->nmodes > 4) return fail(PIC_EINVAL, "nmodes must be 1 .. 4");
    if (c->precision != 32 && c->precision != 64) return fail(PIC_EINVAL, "precision must be 32 or 64");
    if (!(c->dr > 0 && c->dz > 0 && c->dt > 0 && c->c > 0 && c->eps0 > 0))
        return fail(PIC_EINVAL, "dr, dz, dt, c and eps0 must be positive");
    if (!(fabs(c->vgal) < c->c)) return fail(PIC_EINVAL, "|v_gal| must be below c");
    if (!(fabs(c->beta_init) < 1.0)) return fail(PIC_EINVAL, "|beta_init| must be below 1");
    if (ns < 0 || ns > PIC_MAX_SPECIES) return fail(PIC_EINVAL, "nspecies out of range");
    for (int k = 0; k < ns; ++k) {
        if (sp[k].n < 0 || sp[k].n > INT32_MAX) return fail(PIC_EINVAL, "species n out of range");
        if (!(sp[k].m > 0)) return fail(PIC_EINVAL, "species mass must be positive");
        if (sp[k].n > 0 && (!sp[k].w || !sp[k].x[0] || !sp[k].x[1] || !sp[k].x[2] || !sp[k].u[0] ||
                            !sp[k].u[1] || !sp[k].u[2]))
            return fail(PIC_EINVAL, "every particle array must be given");
    }
    return PIC_OK;
}

// ---- set-up kernels (FP64) ---------------------------------------------------------------

// J_n of a signed integer order (J_{-n} = (-1)^n J_n).
__device__ __forceinline__ double besselj(int n, double x) {
    if (n >= 0) return jn(n, x);
    return (n & 1) ? -jn(-n, x) : jn(-n, x);
}

// The first nr positive zeros of J_b by Newton's method on CUDA's jn, from McMahon's
// asymptotic expansion (i + 1 + b/2 - 1/4) pi - (mu - 1)/(8 beta) - ..., mu = 4 b^2,
// and, for the first zero of b >= 1, b + 1.8557571 b^(1/3) + 1.033150 b^(-1/3).
__global__ void bessel_zeros_kernel(double* alpha, int b, int nr) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nr) return;
    const double beta = (i + 1 + 0.5 * b - 0.25) * M_PI;
    const double mu = 4.0 * b * b;
    double x = beta - (mu - 1.0) / (8.0 * beta) - 4.0 * (mu - 1.0) * (7.0 * mu - 31.0) / (3.0 * pow(8.0 * beta, 3.0));
    if (i == 0 && b >= 1) x = b + 1.8557571 * cbrt((double)b) + 1.033150 / cbrt((double)b);
    for (int it = 0; it < 60; ++it) {
        const double f = besselj(b, x);
        const double df = 0.5 * (besselj(b - 1, x) - besselj(b + 1, x));
        const double dx = f / df;
        x -= dx;
        if (fabs(dx) <= 1e-15 * x) break;
    }
    alpha[i] = x;
}

// A[j][i] = w_i J_n(k_i r_j), w_i = 2/(R^2 J_{b+1}(alpha_i)^2), k_i = alpha_i/R.
__global__ void synthesis_kernel(double* A, const double* alpha, int b, int n, int nr, double dr) {
    const double R = nr * dr;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nr * nr; t += gridDim.x * blockDim.x) {
        const int j = t / nr, i = t - j * nr;
        const double a = alpha[i];
        const double jb1 = besselj(b + 1, a);
        const double w = 2.0 / (R * R * jb1 * jb1);
        A[t] = w * besselj(n, a / R * (j + 0.5) * dr);
    }
}

// T[i][j] = r_j dr J_n(k_i r_j): the midpoint quadrature of int_0^R f(r) J_n(k_i r) r dr.
__global__ void hankel_quadrature_kernel(double* T, const double* alpha, int n, int nr, double dr) {
    const double R = nr * dr;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nr * nr; t += gridDim.x * blockDim.x) {
        const int i = t / nr, j = t - i * nr;
        const double r = (j + 0.5) * dr;
        T[t] = r * dr * besselj(n, alpha[i] / R * r);
    }
}

// Gauss-Jordan inverse (FP64, partial pivoting) of the nr x nr matrices at
// base + 2 b nr^2, one CTA per matrix b whose bit is set in `need` (the others return): the
// matrix is reduced in place and its inverse is written to the following nr^2 doubles. A
// zero pivot sets PIC_STATUS_NONFINITE.
__global__ void __launch_bounds__(1024) gauss_jordan_kernel(double* base, int nr, unsigned need, int32_t* status) {
    if (!((need >> blockIdx.x) & 1u)) return;
    double* A = base + (size_t)blockIdx.x * 2 * nr * nr;
    double* B = A + (size_t)nr * nr;
    __shared__ double sv[32];
    __shared__ int si[32];
    __shared__ int piv;
    for (int t = threadIdx.x; t < nr * nr; t += blockDim.x) B[t] = (t / nr == t % nr) ? 1.0 : 0.0;
    __syncthreads();
    for (int k = 0; k < nr; ++k) {
        // pivot: the largest |A[r][k]|, r >= k
        double best = -1.0;
        int bi = k;
        for (int r = k + threadIdx.x; r < nr; r += blockDim.x) {
            const double v = fabs(A[r * nr + k]);
            if (v > best) {
                best = v;
                bi = r;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_down_sync(0xffffffffu, best, o);
            const int oi = __shfl_down_sync(0xffffffffu, bi, o);
            if (ov > best) {
                best = ov;
                bi = oi;
            }
        }
        if ((threadIdx.x & 31) == 0) {
            sv[threadIdx.x >> 5] = best;
            si[threadIdx.x >> 5] = bi;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double b2 = -1.0;
            int i2 = k;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
                if (sv[w] > b2) {
                    b2 = sv[w];
                    i2 = si[w];
                }
            piv = i2;
            if (!(b2 > 0.0)) atomicOr(status, PIC_STATUS_NONFINITE);
        }
        __syncthreads();
        const int p = piv;
        if (p != k)
            for (int c = threadIdx.x; c < nr; c += blockDim.x) {
                double t = A[k * nr + c];
                A[k * nr + c] = A[p * nr + c];
                A[p * nr + c] = t;
                t = B[k * nr + c];
                B[k * nr + c] = B[p * nr + c];
                B[p * nr + c] = t;
            }
        __syncthreads();
        const double d = A[k * nr + k];
        __syncthreads();
        for (int c = threadIdx.x; c < nr; c += blockDim.x) {
            A[k * nr + c] /= d;
            B[k * nr + c] /= d;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < nr * nr; t += blockDim.x) {
            const int r = t / nr, c = t - r * nr;
            if (r == k) continue;
            const double f = A[r * nr + k];
            if (c != k) A[r * nr + c] -= f * A[k * nr + c];
            B[r * nr + c] -= f * B[k * nr + c];
        }
        __syncthreads();
        for (int r = threadIdx.x; r < nr; r += blockDim.x)
            if (r != k) A[r * nr + k] = 0.0;
        __syncthreads();
    }
}

template <typename T>
__global__ void to_precision_kernel(T* dst, const double* src, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (T)src[i];
}

// K of mode m: k_r = alpha/R (nr), 0, k_z = 2 pi s/(nz dz) with s the signed FFT index (nz).
template <typename T>
__global__ void cyl_wavenumbers_kernel(double* Kd, T* Kt, const double* alpha, int nr, int nz, double R, double dz) {
    const int tot = nr + 1 + nz;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += gridDim.x * blockDim.x) {
        double k;
        if (i < nr)
            k = alpha[i] / R;
        else if (i == nr)
            k = 0.0;
        else {
            const int q = i - nr - 1;
            const int s = q < (nz + 1) / 2 ? q : q - nz;
            k = 2.0 * M_PI * ((double)s / ((double)nz * dz));
        }
        Kd[i] = k;
        Kt[i] = (T)k;
    }
}

// ---- transforms --------------------------------------------------------------------------

// Y_b = A_b X_b for batches b (blockIdx.z): A_b real nr x nr, X_b and Y_b complex nr x nz
// (z contiguous). 64 x 64 output tiles (rows i, columns z) of 256 threads, each thread 4
// rows x 4 columns (rows ty + 16 r, columns tx + 16 c); A (transposed) and X staged in
// shared memory 16 values of j at a time, so that a thread's 8 loads per j feed 32 FMAs.
constexpr int RM_T = 64, RM_K = 16;
template <typename T>
__global__ void __launch_bounds__(256) radial_matmul_kernel(const T* const* __restrict__ As,
                                                            const typename cplx<T>::type* const* __restrict__ Xs,
                                                            typename cplx<T>::type* const* __restrict__ Ys, int nr,
                                                            int nz) {
    typedef typename cplx<T>::type C;
    __shared__ T sA[RM_K][RM_T + 1];   // [j][i]
    __shared__ C sX[RM_K][RM_T];       // [j][z]
    const T* A = As[blockIdx.z];
    const C* X = Xs[blockIdx.z];
    C* Y = Ys[blockIdx.z];
    const int i0 = blockIdx.y * RM_T, z0 = blockIdx.x * RM_T;
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    C acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = mk<C>(0.0, 0.0);
    for (int j0 = 0; j0 < nr; j0 += RM_K) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int idx = t + 256 * e;
            const int ia = idx >> 4, ka = idx & 15;       // A: row ia, column j0 + ka
            sA[ka][ia] = (i0 + ia < nr && j0 + ka < nr) ? A[(int64_t)(i0 + ia) * nr + j0 + ka] : (T)0;
            const int kx = idx >> 6, zx = idx & 63;       // X: row j0 + kx, column z0 + zx
            sX[kx][zx] = (j0 + kx < nr && z0 + zx < nz) ? X[(int64_t)(j0 + kx) * nz + z0 + zx] : mk<C>(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < RM_K; ++k) {
            T av[4];
            C xv[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) av[r] = sA[k][ty + 16 * r];
#pragma unroll
            for (int c = 0; c < 4; ++c) xv[c] = sX[k][tx + 16 * c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    acc[r][c].x = fma(av[r], xv[c].x, acc[r][c].x);
                    acc[r][c].y = fma(av[r], xv[c].y, acc[r][c].y);
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int i = i0 + ty + 16 * r;
        if (i >= nr) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int z = z0 + tx + 16 * c;
            if (z < nz) Y[(int64_t)i * nz + z] = acc[r][c];
        }
    }
}

// Spectral E, B of every mode -> the inverse-transform inputs: for each field F (E, B) the
// rows i (F_x + i F_y), -i (F_x - i F_y), F_z (orders m+1, m-1, m).
template <typename C>
__global__ void spectral_to_pq_kernel(C* __restrict__ W, const C* __restrict__ EBh, int M, int64_t G) {
    const int64_t tot = (int64_t)M * 2 * G;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = t % G;
        const int64_t r = t / G;   // m * 2 + field
        const C* F = EBh + (r * 3) * G;
        C* O = W + (r * 3) * G;
        const C fx = F[g], fy = F[G + g], fz = F[2 * G + g];
        const C P = cadd(fx, ctimesi(fy)), Q = csub(fx, ctimesi(fy));
        O[g] = ctimesi(P);                  // i P
        O[G + g] = cscale(ctimesi(Q), -1);  // -i Q
        O[2 * G + g] = fz;
    }
}

// After the inverse transforms (X1 = order m+1 row, X2 = order m-1, X3 = order m; z
// transform unnormalised): F_r = (X1 + X2)/2, F_theta = (X1 - X2)/(2i), F_z = X3, / nz.
template <typename C, typename T>
__global__ void pq_to_polar_kernel(C* __restrict__ Fr, const C* __restrict__ W, int M, int64_t G, T inv_nz) {
    const int64_t tot = (int64_t)M * 2 * G;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = t % G;
        const int64_t r = t / G;
        const C* X = W + (r * 3) * G;
        C* O = Fr + (r * 3) * G;
        const C x1 = X[g], x2 = X[G + g], x3 = X[2 * G + g];
        const C s = cadd(x1, x2), d = csub(x1, x2);
        O[g] = cscale(s, (T)0.5 * inv_nz);
        O[G + g] = cscale(mk<C>(d.y, -d.x), (T)0.5 * inv_nz);   // d/(2i) = -i d/2
        O[2 * G + g] = cscale(x3, inv_nz);
    }
}

// Real-space mode deposits J_r, J_t, J_z, rho -> the forward-transform inputs
// J_r + i J_t (order m+1), J_r - i J_t (m-1), J_z (m), rho (m).
template <typename C>
__global__ void polar_to_cd_kernel(C* __restrict__ W, const C* __restrict__ Dr, int M, int64_t G) {
    const int64_t tot = (int64_t)M * G;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = t % G;
        const int64_t m = t / G;
        const C* D = Dr + m * 4 * G;
        C* O = W + m * 4 * G;
        const C jr = D[g], jt = D[G + g];
        O[g] = cadd(jr, ctimesi(jt));
        O[G + g] = csub(jr, ctimesi(jt));
        O[2 * G + g] = D[2 * G + g];
        O[3 * G + g] = D[3 * G + g];
    }
}

// After the forward transforms (Y1 = H_{m+1}(C), Y2 = H_{m-1}(D)): P = -i Y1, Q = i Y2,
// J_x = (P + Q)/2, J_y = (P - Q)/(2i); J_z and rho as they are.
template <typename C>
__global__ void cd_to_spectral_kernel(C* __restrict__ Sh, const C* __restrict__ W, int M, int64_t G) {
    const int64_t tot = (int64_t)M * G;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = t % G;
        const int64_t m = t / G;
        const C* Y = W + m * 4 * G;
        C* O = Sh + m * 4 * G;
        const C P = cscale(ctimesi(Y[g]), -1), Q = ctimesi(Y[G + g]);
        const C s = cadd(P, Q), d = csub(P, Q);
        O[g] = cscale(s, 0.5);
        O[G + g] = cscale(mk<C>(d.y, -d.x), 0.5);
        O[2 * G + g] = Y[2 * G + g];
        O[3 * G + g] = Y[3 * G + g];
    }
}

// Boosted-Coulomb field of each mode's rho^0 moving at beta c along z (the Cartesian
// formula at k = (k_r, 0, k_z)): E = -i (k - (k.beta) beta) rho / (eps0 (k^2 - (k.beta)^2)),
// B = beta x E / c; zero at k = 0 and on the z-Nyquist plane; rho^n <- rho^0 (Nyquist 0).
template <typename C>
__global__ void cyl_init_fields_kernel(C* EBh, C* Rn, const C* Sh, const double* Kd, int M, int nr, int nz,
                                       double beta, double c, double eps0) {
    const int64_t G = (int64_t)nr * nz;
    const int64_t tot = (int64_t)M * G;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = t % G;
        const int m = (int)(t / G);
        const int i = (int)(g / nz), l = (int)(g % nz);
        const double* K = Kd + (int64_t)m * (nr + 1 + nz);
        const double kr = K[i], kz = K[nr + 1 + l];
        const C rho = Sh[((int64_t)m * 4 + 3) * G + g];
        const bool nyq = (nz % 2 == 0) && l == nz / 2;
        const double kb = kz * beta;
        const double den = eps0 * (kr * kr + kz * kz - kb * kb);
        double2 E[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
        if (!nyq && den != 0.0) {
            const double rr = (double)rho.x, ri = (double)rho.y;
            const double kk[3] = {kr, 0.0, kz - kb * beta};
            for (int d = 0; d < 3; ++d) E[d] = make_double2(kk[d] * ri / den, -kk[d] * rr / den);
        }
        C* O = EBh + (int64_t)m * 6 * G;
        O[0 * G + g] = mk<C>(E[0].x, E[0].y);
        O[1 * G + g] = mk<C>(E[1].x, E[1].y);
        O[2 * G + g] = mk<C>(E[2].x, E[2].y);
        // B = beta x E / c with beta along z: (-beta E_y, beta E_x, 0) / c
        O[3 * G + g] = mk<C>(-beta * E[1].x / c, -beta * E[1].y / c);
        O[4 * G + g] = mk<C>(beta * E[0].x / c, beta * E[0].y / c);
        O[5 * G + g] = mk<C>(0.0, 0.0);
        Rn[(int64_t)m * G + g] = nyq ? mk<C>(0.0, 0.0) : rho;
    }
}

// ---- particles -----------------------------------------------------------------------------

// Re-sort bookkeeping of one species, in device memory: the passes count the particles that
// end a step outside their bin, the next step sorts only when they exceed a threshold (or a
// sort is forced), and the sort flips which buffer is current.
struct CylSortState {
    int sel;                    // current buffer: 0 (w, x, u, pid) or 1 (alt, pid_alt)
    int force;                  // sort at the next step whatever the count
    int need;                   // this step sorts
    int pad;
    unsigned long long moved;   // particles outside their bin after the last pass
};

template <typename T>
struct CylPassK {
    typedef typename cplx<T>::type C;
    const C* F;   // [M][6][nr][nz] E_r, E_t, E_z, B_r, B_t, B_z
    C* D;         // [M][4][nr][nz] J_r, J_t, J_z, rho
    T* buf[2][7]; // the two particle buffers: w, x, y, z, ux, uy, uz
    CylSortState* state;
    int64_t n;
    T q, qdt2m, inv_c2, hdt, vgal, dr, dz, Lz, c2pi_drdz;
    int nr, nz, M;
    int32_t* status;
};

// Divisions and reciprocal square roots of the particle pass: FP32 runs take the fast
// division and the hardware reciprocal square root (CUDA's __fdividef and rsqrtf, within
// 2 ulp, against the FP32 mode's 1e-4 tolerance to the FP64 oracle) instead of the
// correctly rounded sequences and their special-case branches; FP64 runs keep the
// correctly rounded forms.
__device__ __forceinline__ float cyl_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double cyl_div(double a, double b) { return a / b; }
__device__ __forceinline__ float cyl_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double cyl_rsqrt(double x) { return 1.0 / sqrt(x); }

// Radius and direction of (x, y): r, cos(theta), sin(theta) (theta = 0 on the axis).
template <typename T>
__device__ __forceinline__ void cyl_polar(T x, T y, T& r, T& cs, T& sn) {
    const T rr = x * x + y * y;
    if constexpr (sizeof(T) == 4) {
        const T ir = rr > (T)0 ? cyl_rsqrt(rr) : (T)0;
        r = rr * ir;
        cs = rr > (T)0 ? x * ir : (T)1;
        sn = y * ir;
    } else {
        r = sqrt(rr);
        cs = r > (T)0 ? x / r : (T)1;
        sn = r > (T)0 ? y / r : (T)0;
    }
}

// Linear radial stencil of a particle at radius r: nodes j0 (folded onto 0 below the axis)
// and j0 + 1, weights 1 - f and f. Returns false (and flags) outside the radial extent.
template <typename T>
__device__ __forceinline__ bool radial_stencil(const CylPassK<T>& p, T r, int& j0, int& j1, T& w0, T& w1,
                                               bool& ghost) {
    if (!(r < ((T)p.nr - (T)0.5) * p.dr)) {
        atomicOr(p.status, PIC_STATUS_BADINPUT);
        return false;
    }
    const T u = cyl_div(r, p.dr) - (T)0.5;
    const T fl = floor(u);
    int j = (int)fl;
    T f = u - fl;
    if (j > p.nr - 2) {   // r just below the limit can round to u = nr - 1
        j = p.nr - 2;
        f = (T)1;
    }
    ghost = j < 0;
    j0 = ghost ? 0 : j;
    j1 = j + 1;
    w0 = (T)1 - f;
    w1 = f;
    return true;
}

template <typename T>
__device__ __forceinline__ void axial_stencil(const CylPassK<T>& p, T z, int& l0, int& l1, T& w0, T& w1) {
    const T u = cyl_div(z, p.dz);
    const T fl = floor(u);
    int l = (int)fl;
    const T f = u - fl;
    l %= p.nz;
    if (l < 0) l += p.nz;
    l0 = l;
    l1 = l + 1 == p.nz ? 0 : l + 1;
    w0 = (T)1 - f;
    w1 = f;
}

// Real E and B (Cartesian) at (x, y, z) from the mode fields: from the bin's field tile
// ftile ([M][6][CTR][CTZ] complex, rows tj0 .., columns tl0 .. modulo nz) when the stencil
// lies inside it, else from global memory.
template <typename T>
__device__ void cyl_gather(const CylPassK<T>& p, const typename cplx<T>::type* ftile, int tj0, int tl0, T x, T y,
                           T z, T* E, T* B, bool& ok) {
    typedef typename cplx<T>::type C;
    T r, cs, sn;
    cyl_polar(x, y, r, cs, sn);
    int j0, j1, l0, l1;
    T wr0, wr1, wz0, wz1;
    bool ghost;
    ok = radial_stencil(p, r, j0, j1, wr0, wr1, ghost);
    T Fr[6] = {0, 0, 0, 0, 0, 0};
    if (ok) {
        axial_stencil(p, z, l0, l1, wz0, wz1);
        const int64_t G = (int64_t)p.nr * p.nz;
        int tc0 = l0 - tl0, tc1 = l1 - tl0;
        if (tc0 < 0) tc0 += p.nz;
        if (tc1 < 0) tc1 += p.nz;
        const int tr0 = j0 - tj0, tr1 = j1 - tj0;
        const bool intile = ftile && tr0 >= 0 && tr1 < CTR && tc0 < CTZ && tc1 < CTZ;
        C ph = mk<C>(1.0, 0.0);            // e^{i m theta}
        const C rot = mk<C>(cs, sn);
        for (int m = 0; m < p.M; ++m) {
            const T sflip = (m & 1) ? (T)-1 : (T)1;   // (-1)^m: scalars, z components
            const T vflip = -sflip;                    // (-1)^(m+1): r and theta components
            for (int q = 0; q < 6; ++q) {
                const T fac = ghost ? ((q == 2 || q == 5) ? sflip : vflip) : (T)1;
                const T a0 = wr0 * fac, a1 = wr1;
                C v = mk<C>(0.0, 0.0);
                C f00, f01, f10, f11;
                if (intile) {
                    const C* F = ftile + ((int64_t)m * 6 + q) * CTR * CTZ;
                    f00 = F[tr0 * CTZ + tc0];
                    f01 = F[tr0 * CTZ + tc1];
                    f10 = F[tr1 * CTZ + tc0];
                    f11 = F[tr1 * CTZ + tc1];
                } else {
                    const C* F = p.F + ((int64_t)m * 6 + q) * G;
                    f00 = F[(int64_t)j0 * p.nz + l0];
                    f01 = F[(int64_t)j0 * p.nz + l1];
                    f10 = F[(int64_t)j1 * p.nz + l0];
                    f11 = F[(int64_t)j1 * p.nz + l1];
                }
                v.x = a0 * (wz0 * f00.x + wz1 * f01.x) + a1 * (wz0 * f10.x + wz1 * f11.x);
                v.y = a0 * (wz0 * f00.y + wz1 * f01.y) + a1 * (wz0 * f10.y + wz1 * f11.y);
                Fr[q] += (m == 0) ? v.x : (T)2 * (v.x * ph.x - v.y * ph.y);
            }
            ph = cmul(ph, rot);
        }
    }
    E[0] = Fr[0] * cs - Fr[1] * sn;
    E[1] = Fr[0] * sn + Fr[1] * cs;
    E[2] = Fr[2];
    B[0] = Fr[3] * cs - Fr[4] * sn;
    B[1] = Fr[3] * sn + Fr[4] * cs;
    B[2] = Fr[5];
}

// Add values val[0..nq) (component offsets q0 ..) at (x, y, z) to the mode deposits:
// sum val S_r S_z e^{-i m theta} / V_j, fold factors by component kind. Nodes inside the
// bin's shared-memory tile (rows tj0 .. tj0 + CTR - 1, columns tl0 .. tl0 + CTZ - 1 modulo
// nz; layout [M][4][CTR][CTZ] complex) are added there, the others to global memory. With
// itile (FP32 runs) the tile holds 32-bit fixed point, value * scale rounded: native
// integer atomics instead of the compare-and-swap loops of shared float atomics.
template <typename T>
__device__ void cyl_deposit(const CylPassK<T>& p, T* tile, int tj0, int tl0, T x, T y, T z, int q0, int nq,
                            const T* val, int* itile = nullptr, T scale = (T)1) {
    typedef typename cplx<T>::type C;
    T r, cs, sn;
    cyl_polar(x, y, r, cs, sn);
    int j0, j1, l0, l1;
    T wr0, wr1, wz0, wz1;
    bool ghost;
    if (!radial_stencil(p, r, j0, j1, wr0, wr1, ghost)) return;
    axial_stencil(p, z, l0, l1, wz0, wz1);
    const int64_t G = (int64_t)p.nr * p.nz;
    const T iv0 = cyl_div((T)1, p.c2pi_drdz * ((T)j0 + (T)0.5)), iv1 = cyl_div((T)1, p.c2pi_drdz * ((T)j1 + (T)0.5));
    // tile coordinates of the four nodes (-1: outside the tile)
    auto tcol = [&](int l) {
        int d = l - tl0;
        if (d < 0) d += p.nz;
        if (d >= p.nz) d -= p.nz;
        return d < CTZ ? d : -1;
    };
    const int tr0 = (j0 - tj0 >= 0 && j0 - tj0 < CTR) ? j0 - tj0 : -1;
    const int tr1 = (j1 - tj0 >= 0 && j1 - tj0 < CTR) ? j1 - tj0 : -1;
    const int tc0 = tcol(l0), tc1 = tcol(l1);
    auto add = [&](int m, int q, int jj, int ll, int tr, int tc, T re, T im) {
        if (itile && tr >= 0 && tc >= 0) {
            int* t = itile + 2 * (((m * 4 + q) * CTR + tr) * CTZ + tc);
            atomicAdd(t, __float2int_rn((float)(re * scale)));
            atomicAdd(t + 1, __float2int_rn((float)(im * scale)));
        } else if (tile && tr >= 0 && tc >= 0) {
            T* t = tile + 2 * ((((int64_t)m * 4 + q) * CTR + tr) * CTZ + tc);
            atomicAdd(t, re);
            atomicAdd(t + 1, im);
        } else {
            T* d = reinterpret_cast<T*>(p.D + ((int64_t)m * 4 + q) * G + (int64_t)jj * p.nz + ll);
            atomicAdd(d, re);
            atomicAdd(d + 1, im);
        }
    };
    C ph = mk<C>(1.0, 0.0);                // e^{-i m theta}
    const C rot = mk<C>(cs, -sn);
    for (int m = 0; m < p.M; ++m) {
        const T sflip = (m & 1) ? (T)-1 : (T)1;
        const T vflip = -sflip;
        for (int k = 0; k < nq; ++k) {
            const int q = q0 + k;
            const T fac = ghost ? ((q >= 2) ? sflip : vflip) : (T)1;   // J_z, rho: scalars
            const T a0 = val[k] * wr0 * fac * iv0, a1 = val[k] * wr1 * iv1;
            const T c00 = a0 * wz0, c01 = a0 * wz1, c10 = a1 * wz0, c11 = a1 * wz1;
            add(m, q, j0, l0, tr0, tc0, c00 * ph.x, c00 * ph.y);
            add(m, q, j0, l1, tr0, tc1, c01 * ph.x, c01 * ph.y);
            add(m, q, j1, l0, tr1, tc0, c10 * ph.x, c10 * ph.y);
            add(m, q, j1, l1, tr1, tc1, c11 * ph.x, c11 * ph.y);
        }
        ph = cmul(ph, rot);
    }
}

template <typename T>
__device__ __forceinline__ T wrap_len(T z, T L) {
    // a half drift moves a particle far less than L: one add or subtract, fmod otherwise
    if (z < (T)0) z += L;
    else if (z >= L) z -= L;
    if (!(z >= (T)0 && z < L)) {
        z = fmod(z, L);
        if (z < (T)0) z += L;
        if (z >= L) z -= L;
    }
    return z;
}

// Bin of a particle at (x, y, z): its radial cell floor(r / dr) (beyond the extent, which
// is flagged elsewhere: the last row) and its axial cell, periodic.
template <typename T>
__device__ __forceinline__ int cyl_bin_of(T x, T y, T z, T inv_dr, T inv_dz, int nr, int nz, int nbz) {
    const T r = sqrt(x * x + y * y);
    const T u = r * inv_dr, v = floor(z * inv_dz);
    const int jc = (u >= (T)0 && u < (T)nr) ? (int)u : nr - 1;
    int lc = (v >= (T)-nz && v < (T)(2 * nz)) ? (int)v : 0;
    if (lc < 0) lc += nz;
    if (lc >= nz) lc -= nz;
    return (jc / CBR) * nbz + lc / CBZ;
}

// One CTA per (r, z) bin of CBR x CBZ cells, its particles (sorted by bin) one per thread.
// step: gather at x^n, Boris, half drift, J^{n+1/2}, half drift, rho^{n+1}; deposit only
// (step = 0): rho at the current positions. The deposits of the bin's particles are summed
// in a shared-memory tile reaching CPAD cells past the bin, which is then added to the
// global mode arrays once; a particle whose stencil leaves the tile adds there directly.
// (Summing the tile in 64-bit fixed point instead was slower: 6.1 against 4.8 ms per step
// for 16.7M particles.)
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1)
    cyl_particle_kernel(CylPassK<T> p, const int32_t* __restrict__ starts, int nbz, int step) {
    typedef typename cplx<T>::type C;
    extern __shared__ __align__(16) unsigned char cyl_smem[];
    const int nt = p.M * 4 * CTR * CTZ;
    T* tile = reinterpret_cast<T*>(cyl_smem);
    C* ftile = reinterpret_cast<C*>(cyl_smem + (size_t)2 * nt * sizeof(T));   // [M][6][CTR][CTZ]
    const int bin = blockIdx.x;
    const int tj0 = (bin / nbz) * CBR - CPAD, tl0 = (bin % nbz) * CBZ - CPAD;
    const int sel = p.state->sel;   // the current particle buffer
    const T* const pw = p.buf[sel][0];
    T* const px = p.buf[sel][1];
    T* const py = p.buf[sel][2];
    T* const pz = p.buf[sel][3];
    T* const pux = p.buf[sel][4];
    T* const puy = p.buf[sel][5];
    T* const puz = p.buf[sel][6];
    const T inv_dr = (T)1 / p.dr, inv_dz = (T)1 / p.dz;
    unsigned moved = 0;
    for (int t = threadIdx.x; t < 2 * nt; t += blockDim.x) tile[t] = (T)0;
    if (step) {   // the bin's mode fields (nodes outside 0 .. nr - 1 are never read)
        const int64_t G = (int64_t)p.nr * p.nz;
        for (int t = threadIdx.x; t < p.M * 6 * CTR * CTZ; t += blockDim.x) {
            const int tc = t % CTZ, tr = (t / CTZ) % CTR, mq = t / (CTZ * CTR);
            const int jj = tj0 + tr;
            int ll = tl0 + tc;
            if (ll < 0) ll += p.nz;
            if (ll >= p.nz) ll -= p.nz;
            ftile[t] = (jj >= 0 && jj < p.nr && ll >= 0 && ll < p.nz) ? p.F[(int64_t)mq * G + (int64_t)jj * p.nz + ll]
                                                                     : mk<C>(0.0, 0.0);
        }
    }
    const int beg = starts[bin], end = starts[bin + 1];
    // FP32: the tile sums in 32-bit fixed point. No node of the bin's deposit exceeds
    // S = max(1, c) sum |q w| / V (V the smallest annulus of the tile), so with 2 S < 2^E
    // the scale 2^(30 - E) keeps every sum inside 31 bits.
    __shared__ float s_abs[8];
    int* itile = nullptr;
    T scale = (T)1;
    if constexpr (sizeof(T) == 4) {
        float a = 0.f;
        for (int i = beg + threadIdx.x; i < end; i += blockDim.x) a += fabsf((float)(p.q * pw[i]));
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if ((threadIdx.x & 31) == 0) s_abs[threadIdx.x >> 5] = a;
        __syncthreads();
        float sum = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += s_abs[w];
        const float vmin = (float)p.c2pi_drdz * ((float)max(tj0, 0) + 0.5f);
        const float bound = 2.f * fmaxf(1.f, sqrtf(1.f / (float)p.inv_c2)) * sum / vmin;
        int E = 0;
        if (bound > 0.f && bound < 3.0e38f) frexpf(bound, &E);
        scale = (T)ldexpf(1.f, 30 - E);
        itile = reinterpret_cast<int*>(tile);
    }
    __syncthreads();
    for (int i = beg + threadIdx.x; i < end; i += blockDim.x) {
        T x = px[i], y = py[i], z = pz[i];
        T ux = pux[i], uy = puy[i], uz = puz[i];
        const T qw = p.q * pw[i];
        if (!step) {
            const T val[1] = {qw};
            cyl_deposit(p, tile, tj0, tl0, x, y, z, 3, 1, val, itile, scale);
            continue;
        }
        T E[3], B[3];
        bool ok;
        cyl_gather(p, ftile, tj0, tl0, x, y, z, E, B, ok);
        const T a = p.qdt2m;
        const T umx = ux + a * E[0], umy = uy + a * E[1], umz = uz + a * E[2];
        const T igm = cyl_rsqrt((T)1 + (umx * umx + umy * umy + umz * umz) * p.inv_c2);
        const T tx = a * B[0] * igm, ty = a * B[1] * igm, tz = a * B[2] * igm;
        const T s2 = cyl_div((T)2, (T)1 + tx * tx + ty * ty + tz * tz);
        const T sx = s2 * tx, sy = s2 * ty, sz = s2 * tz;
        const T upx = umx + (umy * tz - umz * ty);
        const T upy = umy + (umz * tx - umx * tz);
        const T upz = umz + (umx * ty - umy * tx);
        ux = umx + (upy * sz - upz * sy) + a * E[0];
        uy = umy + (upz * sx - upx * sz) + a * E[1];
        uz = umz + (upx * sy - upy * sx) + a * E[2];
        const T igam = cyl_rsqrt((T)1 + (ux * ux + uy * uy + uz * uz) * p.inv_c2);
        const T vx = ux * igam, vy = uy * igam, vz = uz * igam;
        x += vx * p.hdt;
        y += vy * p.hdt;
        z = wrap_len(z + (vz - p.vgal) * p.hdt, p.Lz);
        {
            T r, cs, sn;
            cyl_polar(x, y, r, cs, sn);
            const T val[3] = {qw * (vx * cs + vy * sn), qw * (-vx * sn + vy * cs), qw * vz};
            cyl_deposit(p, tile, tj0, tl0, x, y, z, 0, 3, val, itile, scale);
        }
        x += vx * p.hdt;
        y += vy * p.hdt;
        z = wrap_len(z + (vz - p.vgal) * p.hdt, p.Lz);
        const T val[1] = {qw};
        cyl_deposit(p, tile, tj0, tl0, x, y, z, 3, 1, val, itile, scale);
        px[i] = x;
        py[i] = y;
        pz[i] = z;
        pux[i] = ux;
        puy[i] = uy;
        puz[i] = uz;
        moved += cyl_bin_of(x, y, z, inv_dr, inv_dz, p.nr, p.nz, nbz) != bin;
    }
    for (int o = 16; o > 0; o >>= 1) moved += __shfl_down_sync(0xffffffffu, moved, o);
    if ((threadIdx.x & 31) == 0 && moved) atomicAdd(&p.state->moved, (unsigned long long)moved);
    __syncthreads();
    const int64_t G = (int64_t)p.nr * p.nz;
    for (int t = threadIdx.x; t < nt; t += blockDim.x) {
        T re, im;
        if (itile) {
            if (itile[2 * t] == 0 && itile[2 * t + 1] == 0) continue;
            re = (T)itile[2 * t] / scale;
            im = (T)itile[2 * t + 1] / scale;
        } else {
            re = tile[2 * t];
            im = tile[2 * t + 1];
            if (re == (T)0 && im == (T)0) continue;
        }
        const int tc = t % CTZ, tr = (t / CTZ) % CTR, mq = t / (CTZ * CTR);
        const int jj = tj0 + tr;
        int ll = tl0 + tc;
        if (ll < 0) ll += p.nz;
        if (ll >= p.nz) ll -= p.nz;
        if (jj < 0 || jj >= p.nr || ll < 0 || ll >= p.nz) continue;   // never written
        T* d = reinterpret_cast<T*>(p.D + (int64_t)mq * G + (int64_t)jj * p.nz + ll);
        atomicAdd(d, re);
        atomicAdd(d + 1, im);
    }
}

// ---- sorting particles into (r, z) bins (counting sort; order inside a bin follows the
// atomic ranks) -------------------------------------------------------------------------

template <typename T>
__global__ void cyl_key_kernel(const CylSortState* __restrict__ sst, const T* x0, const T* y0, const T* z0,
                               const T* x1, const T* y1, const T* z1, int64_t n, T inv_dr, T inv_dz, int nr, int nz,
                               int nbz, int32_t* key, int32_t* rank, int32_t* counts) {
    if (!sst->need) return;
    const bool b = sst->sel != 0;
    const T* x = b ? x1 : x0;
    const T* y = b ? y1 : y0;
    const T* z = b ? z1 : z0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int k = cyl_bin_of(x[i], y[i], z[i], inv_dr, inv_dz, nr, nz, nbz);
        key[i] = k;
        // particles arrive nearly sorted (last step's order), so neighbouring lanes share
        // bins: one atomic per bin and warp, ranks from the lanes' order
        const unsigned act = __activemask();
        const unsigned peers = __match_any_sync(act, k);
        const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(&counts[k], __popc(peers));
        base = __shfl_sync(peers, base, leader);
        rank[i] = base + __popc(peers & ((1u << lane) - 1u));
    }
}

// Whether this step re-sorts species' particles: when a sort is forced or more than
// `threshold` particles ended the last pass outside their bins. Clears the count.
__global__ void cyl_sort_decide_kernel(CylSortState* sst, unsigned long long threshold) {
    sst->need = sst->force || sst->moved > threshold;
    sst->force = 0;
    sst->moved = 0;
}

// After a sort, the other buffer is current.
__global__ void cyl_sort_flip_kernel(CylSortState* sst) {
    if (sst->need) sst->sel ^= 1;
}

// Exclusive scan of the bin counts (one CTA of 1024 threads, each a contiguous segment).
__global__ void __launch_bounds__(1024) cyl_scan_kernel(const CylSortState* __restrict__ sst,
                                                        const int32_t* __restrict__ counts, int32_t* starts,
                                                        int nbins) {
    if (!sst->need) return;
    __shared__ int32_t part[1024];
    const int per = (nbins + 1023) / 1024;
    const int a = threadIdx.x * per, e = min(a + per, nbins);
    int sum = 0;
    for (int i = a; i < e; ++i) sum += counts[i];
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int run = part[threadIdx.x] - sum;
    for (int i = a; i < e; ++i) {
        starts[i] = run;
        run += counts[i];
    }
    if (threadIdx.x == 1023) starts[nbins] = part[1023];
}

struct CylArrays {
    void* a[7];      // w, x, y, z, ux, uy, uz
    int32_t* pid;
};

// Particle buffer b (0 or 1) of a species.
CylArrays cyl_buffer(const pic_cyl::Sp& sp, int b) {
    CylArrays a;
    void* b0[7] = {sp.w, sp.x[0], sp.x[1], sp.x[2], sp.u[0], sp.u[1], sp.u[2]};
    for (int q = 0; q < 7; ++q) a.a[q] = b ? sp.alt[q] : b0[q];
    a.pid = b ? sp.pid_alt : sp.pid;
    return a;
}

template <typename T>
__global__ void cyl_scatter_kernel(const CylSortState* __restrict__ sst, CylArrays b0, CylArrays b1, int64_t n,
                                   const int32_t* __restrict__ key, const int32_t* __restrict__ rank,
                                   const int32_t* __restrict__ starts) {
    if (!sst->need) return;
    const CylArrays& src = sst->sel ? b1 : b0;
    const CylArrays& dst = sst->sel ? b0 : b1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = (int64_t)starts[key[i]] + rank[i];
#pragma unroll
        for (int q = 0; q < 7; ++q) reinterpret_cast<T*>(dst.a[q])[o] = reinterpret_cast<const T*>(src.a[q])[i];
        dst.pid[o] = src.pid[i];
    }
}

__global__ void cyl_iota_kernel(int32_t* pid, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        pid[i] = (int32_t)i;
}

// dst[pid[i]] = src[i]: a species array back in input order.
template <typename T>
__global__ void cyl_unpermute_kernel(const T* __restrict__ src, const int32_t* __restrict__ pid, T* dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[pid[i]] = src[i];
}

// W = (eps0/2) sum_m (1 or 2) sum_{j,l} (|E|^2 + c^2 |B|^2) V_j over the real mode fields.
template <typename C>
__global__ void __launch_bounds__(256) cyl_energy_kernel(const C* F, int M, int nr, int nz, double* part) {
    const int64_t G = (int64_t)nr * nz;
    double se = 0.0, sb = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)M * G;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int m = (int)(t / G);
        const int64_t g = t - (int64_t)m * G;
        const int j = (int)(g / nz);
        const double wm = (m == 0 ? 1.0 : 2.0) * (j + 0.5);   // times 2 pi dr^2 dz below
        for (int q = 0; q < 3; ++q) {
            const C e = F[((int64_t)m * 6 + q) * G + g], b = F[((int64_t)m * 6 + 3 + q) * G + g];
            se += wm * ((double)e.x * e.x + (double)e.y * e.y);
            sb += wm * ((double)b.x * b.x + (double)b.y * b.y);
        }
    }
    __shared__ double s_e[8], s_b[8];
    for (int o = 16; o > 0; o >>= 1) {
        se += __shfl_down_sync(0xffffffffu, se, o);
        sb += __shfl_down_sync(0xffffffffu, sb, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s_e[threadIdx.x >> 5] = se;
        s_b[threadIdx.x >> 5] = sb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < 8; ++w) {
            a += s_e[w];
            b += s_b[w];
        }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
}

__global__ void cyl_energy_final_kernel(const double* part, int nb, double se_scale, double sb_scale, double* out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double a = 0.0, b = 0.0;
    for (int i = 0; i < nb; ++i) {
        a += part[2 * i];
        b += part[2 * i + 1];
    }
    *out = se_scale * a + sb_scale * b;
}

int gridn(int64_t n) {
    int64_t g = (n + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 16));
}

// Matrix of mode m and order slot o (0: m+1, 1: m-1, 2: m), synthesis or forward.
const void* mat(const pic_cyl* s, bool fwd, int m, int o) {
    const size_t T = s->cfg.precision == 64 ? 8 : 4;
    const size_t nr = s->cfg.nr;
    return (const char*)(fwd ? s->fwd : s->syn) + (((size_t)m * 3 + o) * nr * nr) * T;
}

// The two batch tables of the radial products, written once at set-up: set 0, the inverse
// transforms of E, B (mode m, field f, order slot o at batch m*6 + f*3 + o, W1 -> W2); set
// 1, the forward transforms of the sources (mode m, row q at batch m*4 + q, W1 -> W2; rows
// J_r + i J_t, J_r - i J_t, J_z, rho take orders m+1, m-1, m, m).
std::vector<const void*> radial_tables(const pic_cyl* s) {
    const int M = s->cfg.nmodes;
    const size_t G = (size_t)s->G, C = s->cfg.precision == 64 ? 16 : 8;
    std::vector<const void*> h(2 * 3 * GDESC_MAX, nullptr);
    auto put = [&](int set, int b, const void* A, size_t row) {
        const void** t = h.data() + (size_t)set * 3 * GDESC_MAX;
        t[b] = A;
        t[GDESC_MAX + b] = (const char*)s->W1 + row;
        t[2 * GDESC_MAX + b] = (const char*)s->W2 + row;
    };
    for (int m = 0; m < M; ++m)
        for (int f = 0; f < 2; ++f)
            for (int o = 0; o < 3; ++o) {
                const int b = m * 6 + f * 3 + o;
                put(0, b, mat(s, false, m, o), (size_t)b * G * C);
            }
    const int slot[4] = {0, 1, 2, 2};
    for (int m = 0; m < M; ++m)
        for (int q = 0; q < 4; ++q) {
            const int b = m * 4 + q;
            put(1, b, mat(s, true, m, slot[q]), (size_t)b * G * C);
        }
    return h;
}

// One launch of the radial products of table `set` (nb batches).
int radial_products(pic_cyl* s, int set, int nb, cudaStream_t st) {
    void** d = (void**)s->gdesc + (size_t)set * 3 * GDESC_MAX;
    const dim3 grid((s->cfg.nz + RM_T - 1) / RM_T, (s->cfg.nr + RM_T - 1) / RM_T, nb), block(256);
    if (s->cfg.precision == 64)
        radial_matmul_kernel<double><<<grid, block, 0, st>>>((const double* const*)d,
                                                             (const double2* const*)(d + GDESC_MAX),
                                                             (double2* const*)(d + 2 * GDESC_MAX), s->cfg.nr,
                                                             s->cfg.nz);
    else
        radial_matmul_kernel<float><<<grid, block, 0, st>>>((const float* const*)d,
                                                            (const float2* const*)(d + GDESC_MAX),
                                                            (float2* const*)(d + 2 * GDESC_MAX), s->cfg.nr,
                                                            s->cfg.nz);
    GP_CUDA(cudaGetLastError());
    return PIC_OK;
}

// Stage timing: an event pair around stage q when profiling is on; the pair is read (and
// the stream waited for) at the end of the step.
void prof_mark(pic_cyl* s, int q, int end, cudaStream_t st) {
    if (s->prof) cudaEventRecord(s->ev[q][end], st);
}

int exec_z(pic_cyl* s, cufftHandle plan, void* data, int dir, cudaStream_t st) {
    GP_CUFFT(cufftSetStream(plan, st));
    GP_CUFFT(cufftSetWorkArea(plan, s->fftwork));
    if (s->cfg.precision == 64)
        GP_CUFFT(cufftExecZ2Z(plan, (cufftDoubleComplex*)data, (cufftDoubleComplex*)data, dir));
    else
        GP_CUFFT(cufftExecC2C(plan, (cufftComplex*)data, (cufftComplex*)data, dir));
    return PIC_OK;
}

// Spectral E, B -> real mode fields Fr.
int fields_to_real(pic_cyl* s, cudaStream_t st) {
    const int M = s->cfg.nmodes;
    const int64_t G = s->G;
    if (s->cfg.precision == 64)
        spectral_to_pq_kernel<double2><<<gridn(M * 2 * G), 256, 0, st>>>((double2*)s->W1, (const double2*)s->EBh, M, G);
    else
        spectral_to_pq_kernel<float2><<<gridn(M * 2 * G), 256, 0, st>>>((float2*)s->W1, (const float2*)s->EBh, M, G);
    GP_CUDA(cudaGetLastError());
    prof_mark(s, 4, 0, st);
    GP_CHECK(radial_products(s, 0, M * 6, st));
    prof_mark(s, 4, 1, st);
    if (s->prof) {
        float a = 0.f;
        GP_CUDA(cudaEventSynchronize(s->ev[4][1]));
        GP_CUDA(cudaEventElapsedTime(&a, s->ev[4][0], s->ev[4][1]));
        s->prof_ms[4] += a;
        s->prof_n[4] += 1;
    }
    GP_CHECK(exec_z(s, s->plan6, s->W2, CUFFT_INVERSE, st));
    if (s->cfg.precision == 64)
        pq_to_polar_kernel<double2, double><<<gridn(M * 2 * G), 256, 0, st>>>((double2*)s->Fr, (const double2*)s->W2, M,
                                                                            G, 1.0 / s->cfg.nz);
    else
        pq_to_polar_kernel<float2, float><<<gridn(M * 2 * G), 256, 0, st>>>((float2*)s->Fr, (const float2*)s->W2, M,
                                                                          G, 1.0f / s->cfg.nz);
    GP_CUDA(cudaGetLastError());
    return PIC_OK;
}

// Real mode deposits Dr -> source spectra Sh (J_x, J_y, J_z, rho^{n+1} of every mode).
int sources_to_spectral(pic_cyl* s, cudaStream_t st) {
    const int M = s->cfg.nmodes;
    const int64_t G = s->G;
    if (s->cfg.precision == 64)
        polar_to_cd_kernel<double2><<<gridn(M * G), 256, 0, st>>>((double2*)s->W1, (const double2*)s->Dr, M, G);
    else
        polar_to_cd_kernel<float2><<<gridn(M * G), 256, 0, st>>>((float2*)s->W1, (const float2*)s->Dr, M, G);
    GP_CUDA(cudaGetLastError());
    GP_CHECK(exec_z(s, s->plan4, s->W1, CUFFT_FORWARD, st));
    prof_mark(s, 4, 0, st);
    GP_CHECK(radial_products(s, 1, M * 4, st));
    prof_mark(s, 4, 1, st);
    if (s->prof) {
        float a = 0.f;
        GP_CUDA(cudaEventSynchronize(s->ev[4][1]));
        GP_CUDA(cudaEventElapsedTime(&a, s->ev[4][0], s->ev[4][1]));
        s->prof_ms[4] += a;
        s->prof_n[4] += 1;
    }
    if (s->cfg.precision == 64)
        cd_to_spectral_kernel<double2><<<gridn(M * G), 256, 0, st>>>((double2*)s->Sh, (const double2*)s->W2, M, G);
    else
        cd_to_spectral_kernel<float2><<<gridn(M * G), 256, 0, st>>>((float2*)s->Sh, (const float2*)s->W2, M, G);
    GP_CUDA(cudaGetLastError());
    return PIC_OK;
}

template <typename T>
CylPassK<T> passk(pic_cyl* s, int k) {
    typedef typename cplx<T>::type C;
    CylPassK<T> p;
    memset(&p, 0, sizeof(p));
    const pic_cyl_config& c = s->cfg;
    p.F = (const C*)s->Fr;
    p.D = (C*)s->Dr;
    for (int b = 0; b < 2; ++b) {
        const CylArrays a = cyl_buffer(s->sp[k], b);
        for (int q = 0; q < 7; ++q) p.buf[b][q] = (T*)a.a[q];
    }
    p.state = (CylSortState*)s->sp[k].state;
    p.n = s->sp[k].n;
    p.q = (T)s->sp[k].q;
    p.qdt2m = (T)(s->sp[k].q * c.dt / (2.0 * s->sp[k].m));
    p.inv_c2 = (T)(1.0 / (c.c * c.c));
    p.hdt = (T)(0.5 * c.dt);
    p.vgal = (T)c.vgal;
    p.dr = (T)c.dr;
    p.dz = (T)c.dz;
    p.Lz = (T)(c.nz * c.dz);
    p.c2pi_drdz = (T)(2.0 * M_PI * c.dr * c.dr * c.dz);
    p.nr = c.nr;
    p.nz = c.nz;
    p.M = c.nmodes;
    p.status = s->status;
    return p;
}

// Counting sort of species k into the (r, z) bins, when the device decides that it is due
// (more than 1/64 of the particles outside their bins after the last pass, or forced): keys
// and ranks, bin starts, scatter of every array (and the input indices) into the other
// buffer, which then becomes current. Otherwise every kernel of it returns at once.
template <typename T>
int sort_species(pic_cyl* s, int k, cudaStream_t st) {
    pic_cyl::Sp& sp = s->sp[k];
    const int64_t n = sp.n;
    CylSortState* sst = (CylSortState*)sp.state;
    const CylArrays b0 = cyl_buffer(sp, 0), b1 = cyl_buffer(sp, 1);
    cyl_sort_decide_kernel<<<1, 1, 0, st>>>(sst, (unsigned long long)(n / 64));
    GP_CUDA(cudaMemsetAsync(s->counts, 0, (size_t)s->nbins * 4, st));
    cyl_key_kernel<T><<<gridn(n), 256, 0, st>>>(sst, (const T*)b0.a[1], (const T*)b0.a[2], (const T*)b0.a[3],
                                                (const T*)b1.a[1], (const T*)b1.a[2], (const T*)b1.a[3], n,
                                                (T)(1.0 / s->cfg.dr), (T)(1.0 / s->cfg.dz), s->cfg.nr, s->cfg.nz,
                                                s->nbz, s->key, s->rank, s->counts);
    cyl_scan_kernel<<<1, 1024, 0, st>>>(sst, s->counts, sp.starts, s->nbins);
    cyl_scatter_kernel<T><<<gridn(n), 256, 0, st>>>(sst, b0, b1, n, s->key, s->rank, sp.starts);
    cyl_sort_flip_kernel<<<1, 1, 0, st>>>(sst);
    GP_CUDA(cudaGetLastError());
    return PIC_OK;
}

template <typename T>
int particles_t(pic_cyl* s, int step, cudaStream_t st) {
    const size_t tile = (size_t)s->cfg.nmodes * CTR * CTZ * (4 * 2 * sizeof(T) + 6 * 2 * sizeof(T));
    GP_CUDA(cudaFuncSetAttribute(cyl_particle_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tile));
    for (int k = 0; k < s->nspecies; ++k) {
        if (s->sp[k].n == 0) continue;
        GP_CHECK(sort_species<T>(s, k, st));
        cyl_particle_kernel<T><<<s->nbins, 256, tile, st>>>(passk<T>(s, k), s->sp[k].starts, s->nbz, step);
        GP_CUDA(cudaGetLastError());
    }
    return PIC_OK;
}

int particles(pic_cyl* s, int step, cudaStream_t st) {
    const size_t C = s->cfg.precision == 64 ? 16 : 8;
    GP_CUDA(cudaMemsetAsync(s->Dr, 0, (size_t)s->cfg.nmodes * 4 * s->G * C, st));
    return s->cfg.precision == 64 ? particles_t<double>(s, step, st) : particles_t<float>(s, step, st);
}

int make_plans(pic_cyl* s, size_t* work) {
    int n[1] = {s->cfg.nz};
    size_t w6 = 0, w4 = 0;
    const cufftType t = s->cfg.precision == 64 ? CUFFT_Z2Z : CUFFT_C2C;
    GP_CUFFT(cufftCreate(&s->plan6));
    GP_CUFFT(cufftCreate(&s->plan4));
    GP_CUFFT(cufftSetAutoAllocation(s->plan6, 0));
    GP_CUFFT(cufftSetAutoAllocation(s->plan4, 0));
    GP_CUFFT(cufftMakePlanMany(s->plan6, 1, n, n, 1, s->cfg.nz, n, 1, s->cfg.nz, t,
                               s->cfg.nmodes * 6 * s->cfg.nr, &w6));
    GP_CUFFT(cufftMakePlanMany(s->plan4, 1, n, n, 1, s->cfg.nz, n, 1, s->cfg.nz, t,
                               s->cfg.nmodes * 4 * s->cfg.nr, &w4));
    *work = std::max(w6, w4);
    return PIC_OK;
}

}  // namespace
}  // namespace galpic

using namespace galpic;

extern "C" {

int pic_cyl_footprint(const pic_cyl_config* cfg, const pic_cyl_species* species, int nspecies, size_t* bytes_out) {
    GP_CHECK(validate_cyl(cfg, species, nspecies));
    if (!bytes_out) return fail(PIC_EINVAL, "bytes_out is NULL");
    pic_cyl tmp;
    tmp.cfg = *cfg;
    size_t work = 0;
    const int rc = make_plans(&tmp, &work);
    if (tmp.plan6) cufftDestroy(tmp.plan6);
    if (tmp.plan4) cufftDestroy(tmp.plan4);
    GP_CHECK(rc);
    int64_t n[PIC_MAX_SPECIES];
    for (int k = 0; k < nspecies; ++k) n[k] = species[k].n;
    *bytes_out = cyl_layout(*cfg, n, nspecies, work).total;
    return PIC_OK;
}

int pic_cyl_destroy(pic_cyl* s) {
    if (!s) return PIC_OK;
    for (int q = 0; q < 5; ++q)
        for (int e = 0; e < 2; ++e)
            if (s->ev[q][e]) cudaEventDestroy(s->ev[q][e]);
    if (s->plan6) cufftDestroy(s->plan6);
    if (s->plan4) cufftDestroy(s->plan4);
    delete s;
    return PIC_OK;
}

int pic_cyl_init(const pic_cyl_config* cfg, const pic_cyl_species* species, int nspecies, void* workspace,
                 size_t ws_bytes, void* stream, pic_cyl** out) {
    GP_CHECK(validate_cyl(cfg, species, nspecies));
    if (!out || !workspace) return fail(PIC_EINVAL, "out or workspace is NULL");
    if ((uintptr_t)workspace % 256) return fail(PIC_EINVAL, "workspace must be 256-byte aligned");
    *out = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    pic_cyl* s = new (std::nothrow) pic_cyl();
    if (!s) return fail(PIC_ENOMEM, "host allocation failed");
    s->cfg = *cfg;
    s->nspecies = nspecies;
    s->G = (int64_t)cfg->nr * cfg->nz;
    size_t work = 0;
    int rc = make_plans(s, &work);
    if (rc != PIC_OK) {
        pic_cyl_destroy(s);
        return rc;
    }
    int64_t n[PIC_MAX_SPECIES];
    for (int k = 0; k < nspecies; ++k) n[k] = species[k].n;
    const CylLayout L = cyl_layout(*cfg, n, nspecies, work);
    if (ws_bytes < L.total) {
        pic_cyl_destroy(s);
        return fail(PIC_ENOMEM, "cylindrical workspace too small: " + std::to_string(L.total) + " bytes needed");
    }
    char* w = (char*)workspace;
    s->ws = w;
    s->alpha = (double*)(w + L.alpha);
    s->Kd = (double*)(w + L.Kd);
    s->Kt = w + L.Kt;
    s->syn = w + L.syn;
    s->fwd = w + L.fwd;
    s->tmp64 = (double*)(w + L.tmp64);
    s->tab = w + L.tab;
    s->EBh = w + L.EBh;
    s->Sh = w + L.Sh;
    s->Rn = w + L.Rn;
    s->Fr = w + L.Fr;
    s->Dr = w + L.Dr;
    s->W1 = w + L.W1;
    s->W2 = w + L.W2;
    s->scratch = w + L.scratch;
    s->kdesc = w + L.kdesc;
    s->gdesc = w + L.gdesc;
    s->wsum = (double*)(w + L.wsum);
    s->status = (int32_t*)(w + L.status);
    s->fftwork = w + L.fftwork;
    const size_t T = cfg->precision == 64 ? 8 : 4;
    const int nr = cfg->nr, nz = cfg->nz, M = cfg->nmodes;
    for (int k = 0; k < nspecies; ++k) {
        s->sp[k].q = species[k].q;
        s->sp[k].m = species[k].m;
        s->sp[k].n = species[k].n;
        s->sp[k].w = w + L.sp[k][0];
        for (int d = 0; d < 3; ++d) {
            s->sp[k].x[d] = w + L.sp[k][1 + d];
            s->sp[k].u[d] = w + L.sp[k][4 + d];
        }
        for (int q = 0; q < 7; ++q) s->sp[k].alt[q] = w + L.alt[k][q];
        s->sp[k].pid = (int32_t*)(w + L.pid[k][0]);
        s->sp[k].pid_alt = (int32_t*)(w + L.pid[k][1]);
    }
    s->key = (int32_t*)(w + L.key);
    s->rank = (int32_t*)(w + L.rank);
    s->counts = (int32_t*)(w + L.counts);
    for (int k = 0; k < nspecies; ++k) {
        s->sp[k].starts = (int32_t*)(w + L.starts[k]);
        s->sp[k].state = w + L.state[k];
    }
    s->nbz = cyl_nbz(cfg->nz);
    s->nbins = cyl_nbins(cfg->nr, cfg->nz);
#define CYL_TRY(expr)           \
    do {                        \
        int rc_ = (expr);       \
        if (rc_ != PIC_OK) {    \
            pic_cyl_destroy(s); \
            return rc_;         \
        }                       \
    } while (0)
#define CYL_CUDA(call) CYL_TRY((call) == cudaSuccess ? PIC_OK : fail(PIC_ECUDA, #call))
    CYL_CUDA(cudaMemsetAsync(s->status, 0, sizeof(int32_t), st));
    // particles
    for (int k = 0; k < nspecies; ++k) {
        const size_t b = (size_t)species[k].n * T;
        if (!b) continue;
        CYL_CUDA(cudaMemcpyAsync(s->sp[k].w, species[k].w, b, cudaMemcpyDefault, st));
        cyl_iota_kernel<<<gridn(species[k].n), 256, 0, st>>>(s->sp[k].pid, species[k].n);
        const CylSortState init = {0, 1, 0, 0, 0ull};   // buffer 0 current, first step sorts
        CYL_CUDA(cudaMemcpyAsync(s->sp[k].state, &init, sizeof(init), cudaMemcpyHostToDevice, st));
        for (int d = 0; d < 3; ++d) {
            CYL_CUDA(cudaMemcpyAsync(s->sp[k].x[d], species[k].x[d], b, cudaMemcpyDefault, st));
            CYL_CUDA(cudaMemcpyAsync(s->sp[k].u[d], species[k].u[d], b, cudaMemcpyDefault, st));
        }
    }
    // Hankel transforms of every mode: orders m+1, m-1, m on the zeros of J_b, b = max(m-1, 0);
    // the three synthesis matrices of a mode are inverted side by side (one CTA each)
    const size_t NN = (size_t)nr * nr;
    for (int m = 0; m < M; ++m) {
        const int b = std::max(m - 1, 0);
        bessel_zeros_kernel<<<(nr + 127) / 128, 128, 0, st>>>(s->alpha + (size_t)m * nr, b, nr);
        const int orders[3] = {m + 1, m - 1, m};
        for (int o = 0; o < 3; ++o) {
            double* A64 = s->tmp64 + (size_t)o * 2 * NN;
            synthesis_kernel<<<gridn((int64_t)NN), 256, 0, st>>>(A64, s->alpha + (size_t)m * nr, b, orders[o], nr,
                                                                 cfg->dr);
            char* syn = (char*)s->syn + (((size_t)m * 3 + o) * NN) * T;
            if (cfg->precision == 64)
                to_precision_kernel<double><<<gridn((int64_t)NN), 256, 0, st>>>((double*)syn, A64, (int64_t)NN);
            else
                to_precision_kernel<float><<<gridn((int64_t)NN), 256, 0, st>>>((float*)syn, A64, (int64_t)NN);
        }
        unsigned need = 0;
        for (int o = 0; o < 3; ++o)
            if (std::abs(orders[o]) <= 1) need |= 1u << o;
        gauss_jordan_kernel<<<3, 1024, 0, st>>>(s->tmp64, nr, need, s->status);
        for (int o = 0; o < 3; ++o) {
            double* inv = s->tmp64 + ((size_t)o * 2 + 1) * NN;
            if (!((need >> o) & 1u))
                hankel_quadrature_kernel<<<gridn((int64_t)NN), 256, 0, st>>>(inv, s->alpha + (size_t)m * nr, orders[o],
                                                                             nr, cfg->dr);
            char* fwd = (char*)s->fwd + (((size_t)m * 3 + o) * NN) * T;
            if (cfg->precision == 64)
                to_precision_kernel<double><<<gridn((int64_t)NN), 256, 0, st>>>((double*)fwd, inv, (int64_t)NN);
            else
                to_precision_kernel<float><<<gridn((int64_t)NN), 256, 0, st>>>((float*)fwd, inv, (int64_t)NN);
        }
        double* Kd = s->Kd + (size_t)m * (nr + 1 + nz);
        char* Kt = (char*)s->Kt + (size_t)m * (nr + 1 + nz) * T;
        if (cfg->precision == 64)
            cyl_wavenumbers_kernel<double><<<gridn(nr + 1 + nz), 256, 0, st>>>(Kd, (double*)Kt, s->alpha + (size_t)m * nr,
                                                                              nr, nz, nr * cfg->dr, cfg->dz);
        else
            cyl_wavenumbers_kernel<float><<<gridn(nr + 1 + nz), 256, 0, st>>>(Kd, (float*)Kt, s->alpha + (size_t)m * nr,
                                                                             nr, nz, nr * cfg->dr, cfg->dz);
        CYL_CUDA(cudaGetLastError());
        CYL_TRY(launch_cyl_tables(cfg->precision, nr, nz, Kd, (char*)s->tab + (size_t)m * 6 * s->G * 2 * T, cfg->dt,
                                  cfg->vgal, cfg->c, cfg->eps0, cfg->current_correction, st));
    }
    // k-space parameter blocks of every mode
    {
        const size_t kb = kspace_desc_bytes(cfg->precision);
        std::vector<char> host((size_t)M * kb, 0);
        for (int m = 0; m < M; ++m) {
            const size_t C = 2 * T;
            fill_cyl_kspace_desc(cfg->precision, host.data() + m * kb, nr, nz, (char*)s->EBh + (size_t)m * 6 * s->G * C,
                                 (char*)s->Sh + (size_t)m * 4 * s->G * C, (char*)s->Rn + (size_t)m * s->G * C,
                                 (char*)s->scratch + (size_t)m * 6 * s->G * C,
                                 (char*)s->tab + (size_t)m * 6 * s->G * C, (char*)s->Kt + (size_t)m * (nr + 1 + nz) * T,
                                 cfg->c, cfg->current_correction);
        }
        CYL_CUDA(cudaMemcpyAsync(s->kdesc, host.data(), host.size(), cudaMemcpyHostToDevice, st));
        const std::vector<const void*> rt = radial_tables(s);
        CYL_CUDA(cudaMemcpyAsync(s->gdesc, rt.data(), rt.size() * sizeof(void*), cudaMemcpyHostToDevice, st));
    }
    // initial state: rho^0, its spectra, the boosted-Coulomb field, the real mode fields
    CYL_TRY(particles(s, 0, st));
    CYL_TRY(sources_to_spectral(s, st));
    if (cfg->precision == 64)
        cyl_init_fields_kernel<double2><<<gridn(M * s->G), 256, 0, st>>>(
            (double2*)s->EBh, (double2*)s->Rn, (const double2*)s->Sh, s->Kd, M, nr, nz, cfg->beta_init, cfg->c,
            cfg->eps0);
    else
        cyl_init_fields_kernel<float2><<<gridn(M * s->G), 256, 0, st>>>(
            (float2*)s->EBh, (float2*)s->Rn, (const float2*)s->Sh, s->Kd, M, nr, nz, cfg->beta_init, cfg->c,
            cfg->eps0);
    CYL_CUDA(cudaGetLastError());
    CYL_TRY(fields_to_real(s, st));
    // report set-up failures (a singular transform matrix) and particles outside the radius
    int32_t stv = 0;
    CYL_CUDA(cudaStreamSynchronize(st));
    CYL_CUDA(cudaMemcpy(&stv, s->status, sizeof(stv), cudaMemcpyDeviceToHost));
    if (stv) {
        pic_cyl_destroy(s);
        return fail(PIC_EINVAL, (stv & PIC_STATUS_NONFINITE) ? "singular Hankel transform matrix"
                                                             : "a particle lies outside the radial extent");
    }
#undef CYL_CUDA
#undef CYL_TRY
    *out = s;
    return PIC_OK;
}

int pic_cyl_step(pic_cyl* s, int nsteps, void* stream) {
    if (!s) return fail(PIC_EINVAL, "cyl run is NULL");
    if (nsteps < 0) return fail(PIC_EINVAL, "nsteps < 0");
    cudaStream_t st = (cudaStream_t)stream;
    for (int i = 0; i < nsteps; ++i) {
        prof_mark(s, 0, 0, st);
        GP_CHECK(particles(s, 1, st));
        prof_mark(s, 0, 1, st);
        prof_mark(s, 1, 0, st);
        GP_CHECK(sources_to_spectral(s, st));
        prof_mark(s, 1, 1, st);
        prof_mark(s, 2, 0, st);
        GP_CHECK(launch_kspace_descs(s->cfg.precision, s->kdesc, s->cfg.nmodes, s->G, st));
        prof_mark(s, 2, 1, st);
        prof_mark(s, 3, 0, st);
        GP_CHECK(fields_to_real(s, st));
        prof_mark(s, 3, 1, st);
        if (s->prof) {
            GP_CUDA(cudaEventSynchronize(s->ev[3][1]));
            for (int q = 0; q < 4; ++q) {
                float a = 0.f;
                GP_CUDA(cudaEventElapsedTime(&a, s->ev[q][0], s->ev[q][1]));
                s->prof_ms[q] += a;
                s->prof_n[q] += 1;
            }
        }
        s->steps += 1;
    }
    return PIC_OK;
}

int pic_cyl_profile(pic_cyl* s, int enable) {
    if (!s) return fail(PIC_EINVAL, "cyl run is NULL");
    if (enable && !s->ev[0][0])
        for (int q = 0; q < 5; ++q)
            for (int e = 0; e < 2; ++e) GP_CUDA(cudaEventCreate(&s->ev[q][e]));
    s->prof = enable != 0;
    for (int q = 0; q < 5; ++q) {
        s->prof_ms[q] = 0.0;
        s->prof_n[q] = 0;
    }
    return PIC_OK;
}

int pic_cyl_profile_read(pic_cyl* s, double ms[5], int64_t count[5]) {
    if (!s || !ms || !count) return fail(PIC_EINVAL, "NULL argument");
    for (int q = 0; q < 5; ++q) {
        ms[q] = s->prof_ms[q];
        count[q] = s->prof_n[q];
        s->prof_ms[q] = 0.0;
        s->prof_n[q] = 0;
    }
    return PIC_OK;
}

int pic_cyl_get(pic_cyl* s, int which, void* dst, size_t bytes, void* stream) {
    if (!s || !dst) return fail(PIC_EINVAL, "cyl run or dst is NULL");
    const size_t T = s->cfg.precision == 64 ? 8 : 4, C = 2 * T, M = s->cfg.nmodes, G = (size_t)s->G;
    const char* src = nullptr;
    size_t n = 0;
    switch (which) {
        case PIC_CYL_EB_HAT: src = (const char*)s->EBh; n = M * 6 * G * C; break;   // E, B of each mode
        case PIC_CYL_RHO_HAT: src = (const char*)s->Rn; n = M * G * C; break;
        case PIC_CYL_FIELDS: src = (const char*)s->Fr; n = M * 6 * G * C; break;
        case PIC_CYL_SOURCES: src = (const char*)s->Dr; n = M * 4 * G * C; break;
        case PIC_CYL_K: src = (const char*)s->Kd; n = M * (s->cfg.nr + 1 + s->cfg.nz) * 8; break;
        case PIC_CYL_STATUS: src = (const char*)s->status; n = 4; break;
        default: return fail(PIC_EINVAL, "unknown cylindrical buffer " + std::to_string(which));
    }
    if (bytes != n) return fail(PIC_EINVAL, "buffer has " + std::to_string(n) + " bytes, got " + std::to_string(bytes));
    GP_CUDA(cudaMemcpyAsync(dst, src, n, cudaMemcpyDefault, (cudaStream_t)stream));
    return PIC_OK;
}

int pic_cyl_get_particles(pic_cyl* s, int k, void* x[3], void* u[3], void* stream) {
    if (!s || k < 0 || k >= s->nspecies || !x || !u) return fail(PIC_EINVAL, "bad cyl run, species or arrays");
    // the run keeps its particles sorted by bin, in one of two buffers (the device state
    // says which): each array goes back to input order through the other buffer, then out
    cudaStream_t st = (cudaStream_t)stream;
    const pic_cyl::Sp& sp = s->sp[k];
    const int64_t n = sp.n;
    if (n == 0) return PIC_OK;
    CylSortState h;
    GP_CUDA(cudaMemcpyAsync(&h, sp.state, sizeof(h), cudaMemcpyDeviceToHost, st));
    GP_CUDA(cudaStreamSynchronize(st));
    const CylArrays cur = cyl_buffer(sp, h.sel), other = cyl_buffer(sp, h.sel ^ 1);
    const size_t b = (size_t)n * (s->cfg.precision == 64 ? 8 : 4);
    for (int d = 0; d < 6; ++d) {
        void* dst = d < 3 ? x[d] : u[d - 3];
        if (!dst) continue;
        const void* src = cur.a[1 + d];
        void* tmp = other.a[1 + d];
        if (s->cfg.precision == 64)
            cyl_unpermute_kernel<double><<<gridn(n), 256, 0, st>>>((const double*)src, cur.pid, (double*)tmp, n);
        else
            cyl_unpermute_kernel<float><<<gridn(n), 256, 0, st>>>((const float*)src, cur.pid, (float*)tmp, n);
        GP_CUDA(cudaGetLastError());
        GP_CUDA(cudaMemcpyAsync(dst, tmp, b, cudaMemcpyDefault, st));
    }
    return PIC_OK;
}

int pic_cyl_energy(pic_cyl* s, double* out_dev, void* stream) {
    if (!s || !out_dev) return fail(PIC_EINVAL, "cyl run or out_dev is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const int nb = 512;
    if (s->cfg.precision == 64)
        cyl_energy_kernel<double2><<<nb, 256, 0, st>>>((const double2*)s->Fr, s->cfg.nmodes, s->cfg.nr, s->cfg.nz,
                                                       s->wsum);
    else
        cyl_energy_kernel<float2><<<nb, 256, 0, st>>>((const float2*)s->Fr, s->cfg.nmodes, s->cfg.nr, s->cfg.nz,
                                                      s->wsum);
    GP_CUDA(cudaGetLastError());
    const double vol = 2.0 * M_PI * s->cfg.dr * s->cfg.dr * s->cfg.dz;
    cyl_energy_final_kernel<<<1, 32, 0, st>>>(s->wsum, nb, 0.5 * s->cfg.eps0 * vol,
                                              0.5 * s->cfg.eps0 * vol * s->cfg.c * s->cfg.c, out_dev);
    GP_CUDA(cudaGetLastError());
    return PIC_OK;
}

}  // extern "C"
