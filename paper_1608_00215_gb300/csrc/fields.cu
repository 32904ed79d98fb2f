// Spectral-side kernels of the Galilean-PSATD step:
//   * build_tables   - per-mode factors of the update, built in FP64 (once per run);
//   * kspace_update  - current correction + Galilean-PSATD update + Nyquist zeroing
//                      + rho^n <- rho^{n+1} + copy of the result for the inverse FFT;
//   * init_fields    - boosted-Coulomb field of rho^0 (or zero fields);
//   * energy         - field energy W = (eps0/2) sum (|E|^2 + c^2 |B|^2) dV.
#include <math.h>
#include <string.h>

#include <algorithm>

#include <vector>

#include "common.cuh"

namespace galpic {

namespace {

constexpr int GL_N = 16;

struct GaussLegendre {
    double x[GL_N];
    double w[GL_N];
};

// Nodes and weights of the GL_N-point Gauss-Legendre rule on [-1, 1]: the roots
// of the Legendre polynomial P_n found by Newton's method from the Chebyshev-like
// guesses cos(pi (i + 3/4)/(n + 1/2)), with P_n and P_n' from the three-term
// recurrence (j+1) P_{j+1} = (2j+1) x P_j - j P_{j-1}; weight 2/((1-x^2) P_n'(x)^2).
GaussLegendre gauss_legendre() {
    GaussLegendre g;
    const int n = GL_N;
    for (int i = 0; i < n; ++i) {
        double x = cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int j = 1; j < n; ++j) {
                double p2 = ((2.0 * j + 1.0) * x * p1 - j * p0) / (j + 1.0);
                p0 = p1;
                p1 = p2;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        g.x[i] = x;
        g.w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    return g;
}

__device__ __forceinline__ int signed_index(int i, int n) { return i < (n + 1) / 2 ? i : i - n; }

__device__ __forceinline__ double sinc_d(double a, double sa) { return a == 0.0 ? 1.0 : sa / a; }

// Weights of the centred difference of even order p (at most 128):
// f'(x) ~ (1/d) sum_{l=1}^{p/2} a_l (f(x + l d) - f(x - l d)).
struct StencilWeights {
    int m;            // p / 2; 0 = spectral (no stencil)
    double a[64];
};

// a_l = (-1)^(l+1) (m!)^2 / (l (m-l)! (m+l)!), evaluated as the running product
// prod_{j<=l} (m - j + 1)/(m + j) so that no factorial overflows.
StencilWeights stencil_weights(int p) {
    StencilWeights w;
    w.m = p / 2;
    double r = 1.0;
    for (int l = 1; l <= w.m; ++l) {
        r *= (double)(w.m - l + 1) / (double)(w.m + l);
        w.a[l - 1] = (l & 1 ? r : -r) / l;
    }
    return w;
}

// Wavenumbers of the three axes in FFT order, kx[nx], ky[ny], kz[nzh] (half axis),
// one thread per entry, FP64: spectral 2 pi s/(n d) for the signed index s, or the
// symbol of the centred difference (2/d) sum_l a_l sin(2 pi l s / n), with the phase
// l s reduced modulo n in integers and sin(pi x) taken by sinpi; 0 on the Nyquist
// entry of an even axis for a finite stencil. Written in FP64 and in T.
template <typename T>
__global__ void wavenumbers_kernel(double* __restrict__ K, T* __restrict__ Kt, int nx, int ny, int nzh,
                                   int nz, double dx, double dy, double dz, StencilWeights w) {
    const int total = nx + ny + nzh;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        int n, s;
        double d;
        if (i < nx) {
            n = nx, d = dx, s = signed_index(i, nx);
        } else if (i < nx + ny) {
            n = ny, d = dy, s = signed_index(i - nx, ny);
        } else {
            n = nz, d = dz, s = i - nx - ny;
        }
        double k;
        if (w.m == 0) {
            k = 2.0 * M_PI * ((double)s * (1.0 / ((double)n * d)));
        } else if ((n & 1) == 0 && (s == n / 2 || s == -n / 2)) {
            k = 0.0;
        } else {
            double acc = 0.0;
            for (int l = 1; l <= w.m; ++l) {
                const long long r = ((long long)l * s) % n;   // sign of s, |r| < n
                acc += w.a[l - 1] * sinpi(2.0 * (double)r / (double)n);
            }
            k = 2.0 * acc / d;
        }
        K[i] = k;
        Kt[i] = (T)k;
    }
}

// Per-mode factors, FP64 throughout.
//
// With phi = c k dt, nu = k.v_gal/(c k), theta = exp(i nu phi/2) and
// E1(x) = (exp(ix) - 1)/(ix) = exp(ix/2) sinc(x/2), the paper's
//   chi1 = (theta* - C theta + i nu theta S)/(1 - nu^2),
//   chi2 = (chi1 - theta (1 - C))/(theta* - theta),
//   chi3 = (chi1 - theta* (1 - C))/(theta* - theta)
// are evaluated from the equivalent integrals (analytic in nu, no 0/0):
//   theta chi1 = Is = int_0^phi exp(i nu t) sin t dt,
//   chi2 = int_0^phi exp(i nu t) (phi - t) E1(nu (phi - t)) sin t dt / (phi E1(nu phi)),
//   chi3 = -int_0^phi t E1(nu t) sin t dt / (phi E1(nu phi)),
// by composite Gauss-Legendre quadrature (panels of length <= 3, 16 nodes each: the
// integrands are entire with frequencies |nu| + 1 <= 2, so the rule's error on a
// panel is of order 3^32/32! ~ 1e-20 relative).
// Stored factors (E update: E' = T1 E + c^2 T2 (i k x B) + T4 J' + k (A5 rho^{n+1}
// + A6 rho^n), B update: B' = T1 B - T2 (i k x E) + T3 (i k x J)):
//   T1 = theta^2 C, T2 = theta^2 S/(c k), T3 = Is/(eps0 c^2 k^2),
//   T4 = (i nu Is - theta^2 S)/(eps0 c k),
//   without current correction (J' = J): A5 = -i chi2/(eps0 k^2), A6 = i theta^2 chi3/(eps0 k^2);
//   with current correction (J' = transverse part of J; the longitudinal part is
//   fixed by the continuity equation): A5 = -i/(eps0 k^2), A6 = i theta^2 C/(eps0 k^2),
//   which is the paper's update applied to the corrected current, simplified
//   exactly (Gauss's law is then carried from rho^n to rho^{n+1} per mode).
// k = 0: T1 = 1, T2 = dt, T4 = -dt/eps0, T3 = A5 = A6 = 0 (B unchanged, E -= dt J/eps0).
// The factors depend on k only through |k| and k.v_gal, so with v_gal,x = 0 (fx = 1)
// the modes kx and -kx share them, and likewise along y: the kernel then evaluates
// one representative mx <= nx/2 (my <= ny/2) and writes its mirrors too.
template <typename C>
__global__ void build_tables_kernel(C* __restrict__ tab, const double* __restrict__ K, int nx, int ny,
                                    int nz, int nzh, int64_t M, double dt, double vx, double vy,
                                    double vz, double c, double eps0, int cc, GaussLegendre gl, int fx,
                                    int fy) {
    const int X = fx ? nx / 2 + 1 : nx, Y = fy ? ny / 2 + 1 : ny;
    const int64_t Mrep = (int64_t)X * Y * nzh;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < Mrep;
         q += (int64_t)gridDim.x * blockDim.x) {
        int mz = (int)(q % nzh);
        int64_t r = q / nzh;
        int my = (int)(r % Y);
        int mx = (int)(r / Y);
        const int64_t m = ((int64_t)mx * ny + my) * nzh + mz;
        const double kx = K[mx], ky = K[nx + my], kz = K[nx + ny + mz];
        double k2 = kx * kx + ky * ky + kz * kz;
        double2 T1, T2, T3, T4, A5, A6;
        if (k2 == 0.0) {
            T1 = make_double2(1.0, 0.0);
            T2 = make_double2(dt, 0.0);
            T3 = make_double2(0.0, 0.0);
            T4 = make_double2(-dt / eps0, 0.0);
            A5 = make_double2(0.0, 0.0);
            A6 = make_double2(0.0, 0.0);
        } else {
            double k = sqrt(k2);
            double phi = c * k * dt;
            double kv = kx * vx + ky * vy + kz * vz;
            double nu = kv / (c * k);
            double S, Cc;
            sincos(phi, &S, &Cc);
            double xh = 0.5 * kv * dt;   // = nu phi / 2
            double sh, ch;
            sincos(xh, &sh, &ch);
            double2 th = make_double2(ch, sh);
            double2 Is = make_double2(0.0, 0.0), I2 = Is, I3 = Is;
            int npan = (int)ceil(phi / 3.0);
            if (npan < 1) npan = 1;
            double h = phi / npan;
            for (int p = 0; p < npan; ++p) {
                double a0 = h * p;
                for (int j = 0; j < GL_N; ++j) {
                    double t = a0 + 0.5 * h * (gl.x[j] + 1.0);
                    double wt = 0.5 * h * gl.w[j];
                    double st = sin(t);
                    double a = 0.5 * nu * t;
                    double sa, ca;
                    sincos(a, &sa, &ca);
                    double2 eh = make_double2(ca, sa);                 // exp(i nu t/2)
                    double2 et = cmul(eh, eh);                        // exp(i nu t)
                    double2 e1t = cscale(eh, sinc_d(a, sa));          // E1(nu t)
                    double b = 0.5 * nu * (phi - t);
                    double sb, cb;
                    sincos(b, &sb, &cb);
                    double2 e1g = cscale(make_double2(cb, sb), sinc_d(b, sb));   // E1(nu (phi - t))
                    Is = cadd(Is, cscale(et, wt * st));
                    I2 = cadd(I2, cscale(cmul(et, e1g), wt * st * (phi - t)));
                    I3 = cadd(I3, cscale(e1t, wt * st * t));
                }
            }
            double2 e1phi = cscale(th, sinc_d(xh, sh));              // E1(nu phi)
            double2 den = cscale(e1phi, phi);
            double2 chi2 = cdiv(I2, den);
            double2 chi3 = cscale(cdiv(I3, den), -1.0);
            double2 th2 = cmul(th, th);
            T1 = cscale(th2, Cc);
            T2 = cscale(th2, S / (c * k));
            T3 = cscale(Is, 1.0 / (eps0 * c * c * k2));
            T4 = cscale(csub(cscale(ctimesi(Is), nu), cscale(th2, S)), 1.0 / (eps0 * c * k));
            if (cc) {
                A5 = make_double2(0.0, -1.0 / (eps0 * k2));
                A6 = cscale(ctimesi(th2), Cc / (eps0 * k2));
            } else {
                A5 = cscale(ctimesi(chi2), -1.0 / (eps0 * k2));
                A6 = cscale(ctimesi(cmul(th2, chi3)), 1.0 / (eps0 * k2));
            }
        }
        const C v[6] = {mk<C>(T1.x, T1.y), mk<C>(T2.x, T2.y), mk<C>(T3.x, T3.y),
                        mk<C>(T4.x, T4.y), mk<C>(A5.x, A5.y), mk<C>(A6.x, A6.y)};
        const bool mirx = fx && mx != 0 && 2 * mx != nx, miry = fy && my != 0 && 2 * my != ny;
        const int64_t mxx = ((int64_t)(nx - mx) * ny + my) * nzh + mz;
        const int64_t myy = ((int64_t)mx * ny + (ny - my)) * nzh + mz;
        const int64_t mxy = ((int64_t)(nx - mx) * ny + (ny - my)) * nzh + mz;
#pragma unroll
        for (int t = 0; t < 6; ++t) {
            tab[t * M + m] = v[t];
            if (mirx) tab[t * M + mxx] = v[t];
            if (miry) tab[t * M + myy] = v[t];
            if (mirx && miry) tab[t * M + mxy] = v[t];
        }
    }
}

template <typename T>
struct KParams {
    typedef typename cplx<T>::type C;
    C* EBh;          // master E (3M) then B (3M), updated in place
    C* EBs;          // copy of the result / N for the inverse FFT
    const C* Sh;     // spectra of Jx, Jy, Jz, rho^{n+1}
    C* Rn;           // rho^n, replaced by rho^{n+1}
    const C* tab;    // T1, T2, T3, T4, A5, A6
    int64_t M;
    int nx, ny, nz, nzh;
    const T* kx;      // wavenumbers per axis: kx[nx], ky[ny], kz[nzh]
    const T* ky;
    const T* kz;
    T c2;             // c^2
    T invN;
    T bg[3];          // N rho_bg v_gal: background current at k = 0
    int cc;
    int nyq_mask;     // Nyquist planes held at zero: bit 0 x, bit 1 y, bit 2 z (7 for a run;
                      // 0 for decomposed windows; 4 for quasi-cylindrical modes, whose first
                      // axis is the radial spectrum)
};

__device__ __forceinline__ bool is_nyquist(int mx, int my, int mz, int nx, int ny, int nz) {
    return ((nx & 1) == 0 && mx == nx / 2) || ((ny & 1) == 0 && my == ny / 2) ||
           ((nz & 1) == 0 && mz == nz / 2);
}

__device__ __forceinline__ bool is_nyquist_masked(int mx, int my, int mz, int nx, int ny, int nz, int mask) {
    return ((mask & 1) && (nx & 1) == 0 && mx == nx / 2) || ((mask & 2) && (ny & 1) == 0 && my == ny / 2) ||
           ((mask & 4) && (nz & 1) == 0 && mz == nz / 2);
}

// One thread per mode: reads E, B, J, rho^{n+1}, rho^n and the six factors;
// writes E, B (master and scaled copy) and rho^n. Every array is read or
// written once, coalesced; this kernel is bound by HBM bandwidth.
template <typename T>
__device__ __forceinline__ void kspace_update_body(const KParams<T>& p) {
    typedef typename cplx<T>::type C;
    const int64_t M = p.M;
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < M;
         m += (int64_t)gridDim.x * blockDim.x) {
        int mz = (int)(m % p.nzh);
        int64_t r = m / p.nzh;
        int my = (int)(r % p.ny);
        int mx = (int)(r / p.ny);
        if (is_nyquist_masked(mx, my, mz, p.nx, p.ny, p.nz, p.nyq_mask)) {
            C z = mk<C>(0.0, 0.0);
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                p.EBh[q * M + m] = z;
                p.EBs[q * M + m] = z;
            }
            p.Rn[m] = z;
            continue;
        }
        const T kx = p.kx[mx], ky = p.ky[my], kz = p.kz[mz];
        C Ex = p.EBh[0 * M + m], Ey = p.EBh[1 * M + m], Ez = p.EBh[2 * M + m];
        C Bx = p.EBh[3 * M + m], By = p.EBh[4 * M + m], Bz = p.EBh[5 * M + m];
        C Jx = p.Sh[0 * M + m], Jy = p.Sh[1 * M + m], Jz = p.Sh[2 * M + m];
        C r1 = p.Sh[3 * M + m];
        C r0 = p.Rn[m];
        C T1 = p.tab[0 * M + m], T2 = p.tab[1 * M + m], T3 = p.tab[2 * M + m];
        C T4 = p.tab[3 * M + m], A5 = p.tab[4 * M + m], A6 = p.tab[5 * M + m];
        if (m == 0) {
            Jx.x += p.bg[0];
            Jy.x += p.bg[1];
            Jz.x += p.bg[2];
        }
        T k2 = kx * kx + ky * ky + kz * kz;
        if (p.cc && k2 > (T)0) {
            // keep only the transverse part of J; the longitudinal part enters
            // through A5, A6 (continuity equation)
            T ik2 = (T)1 / k2;
            C g = cscale(cadd(cadd(cscale(Jx, kx), cscale(Jy, ky)), cscale(Jz, kz)), ik2);
            Jx = csub(Jx, cscale(g, kx));
            Jy = csub(Jy, cscale(g, ky));
            Jz = csub(Jz, cscale(g, kz));
        }
        // i k x F
        C kEx = ctimesi(csub(cscale(Ez, ky), cscale(Ey, kz)));
        C kEy = ctimesi(csub(cscale(Ex, kz), cscale(Ez, kx)));
        C kEz = ctimesi(csub(cscale(Ey, kx), cscale(Ex, ky)));
        C kBx = ctimesi(csub(cscale(Bz, ky), cscale(By, kz)));
        C kBy = ctimesi(csub(cscale(Bx, kz), cscale(Bz, kx)));
        C kBz = ctimesi(csub(cscale(By, kx), cscale(Bx, ky)));
        C kJx = ctimesi(csub(cscale(Jz, ky), cscale(Jy, kz)));
        C kJy = ctimesi(csub(cscale(Jx, kz), cscale(Jz, kx)));
        C kJz = ctimesi(csub(cscale(Jy, kx), cscale(Jx, ky)));
        C T2c = cscale(T2, p.c2);
        C src = cadd(cmul(A5, r1), cmul(A6, r0));
        C nEx = cadd(cadd(cmul(T1, Ex), cmul(T2c, kBx)), cadd(cmul(T4, Jx), cscale(src, kx)));
        C nEy = cadd(cadd(cmul(T1, Ey), cmul(T2c, kBy)), cadd(cmul(T4, Jy), cscale(src, ky)));
        C nEz = cadd(cadd(cmul(T1, Ez), cmul(T2c, kBz)), cadd(cmul(T4, Jz), cscale(src, kz)));
        C nBx = cadd(csub(cmul(T1, Bx), cmul(T2, kEx)), cmul(T3, kJx));
        C nBy = cadd(csub(cmul(T1, By), cmul(T2, kEy)), cmul(T3, kJy));
        C nBz = cadd(csub(cmul(T1, Bz), cmul(T2, kEz)), cmul(T3, kJz));
        p.EBh[0 * M + m] = nEx;
        p.EBh[1 * M + m] = nEy;
        p.EBh[2 * M + m] = nEz;
        p.EBh[3 * M + m] = nBx;
        p.EBh[4 * M + m] = nBy;
        p.EBh[5 * M + m] = nBz;
        p.EBs[0 * M + m] = cscale(nEx, p.invN);
        p.EBs[1 * M + m] = cscale(nEy, p.invN);
        p.EBs[2 * M + m] = cscale(nEz, p.invN);
        p.EBs[3 * M + m] = cscale(nBx, p.invN);
        p.EBs[4 * M + m] = cscale(nBy, p.invN);
        p.EBs[5 * M + m] = cscale(nBz, p.invN);
        p.Rn[m] = r1;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) kspace_update_kernel(KParams<T> p) {
    kspace_update_body<T>(p);
}

// The k-space update of several runs of one grid shape in one launch: blockIdx.y picks
// the run, whose parameters are copied from a device table into shared memory.
template <typename T>
__global__ void __launch_bounds__(256) kspace_update_many_kernel(const KParams<T>* __restrict__ descs) {
    __shared__ __align__(16) KParams<T> P;
    static_assert(sizeof(KParams<T>) % 4 == 0, "KParams is copied as 32-bit words");
    const int* a = reinterpret_cast<const int*>(descs + blockIdx.y);
    int* d = reinterpret_cast<int*>(&P);
    for (int i = threadIdx.x; i < (int)(sizeof(KParams<T>) / 4); i += blockDim.x) d[i] = a[i];
    __syncthreads();
    kspace_update_body<T>(P);
}

// Initial spectral state from rho^0 (fourth source spectrum). FP64 arithmetic.
//   init 1: E = -i (k - (k.beta) beta) rho / (eps0 (k^2 - (k.beta)^2)), B = beta x E / c;
//   init 0: E = B = 0.  k = 0 and Nyquist modes: E = B = 0; rho^n = rho^0 (0 on Nyquist).
template <typename C>
__global__ void init_fields_kernel(C* EBh, C* Rn, const C* Sh, int64_t M, int nx, int ny, int nz,
                                   int nzh, const double* __restrict__ K, double bx, double by,
                                   double bz, double c, double eps0, int mode) {
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < M;
         m += (int64_t)gridDim.x * blockDim.x) {
        int mz = (int)(m % nzh);
        int64_t r = m / nzh;
        int my = (int)(r % ny);
        int mx = (int)(r / ny);
        C rho = Sh[3 * M + m];
        double2 E[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
        double2 B[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
        bool nyq = is_nyquist(mx, my, mz, nx, ny, nz);
        const double kx = K[mx], ky = K[nx + my], kz = K[nx + ny + mz];
        double k2 = kx * kx + ky * ky + kz * kz;
        if (mode == 1 && !nyq && k2 > 0.0) {
            double kb = kx * bx + ky * by + kz * bz;
            double den = eps0 * (k2 - kb * kb);
            double2 rr = make_double2((double)rho.x, (double)rho.y);
            double kk[3] = {kx - kb * bx, ky - kb * by, kz - kb * bz};
            for (int d = 0; d < 3; ++d) {
                // -i * kk[d] * rho / den
                E[d] = make_double2(kk[d] * rr.y / den, -kk[d] * rr.x / den);
            }
            double bv[3] = {bx, by, bz};
            for (int d = 0; d < 3; ++d) {
                int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
                B[d] = cscale(csub(cscale(E[d2], bv[d1]), cscale(E[d1], bv[d2])), 1.0 / c);
            }
        }
        for (int d = 0; d < 3; ++d) {
            EBh[d * M + m] = mk<C>(E[d].x, E[d].y);
            EBh[(3 + d) * M + m] = mk<C>(B[d].x, B[d].y);
        }
        Rn[m] = nyq ? mk<C>(0.0, 0.0) : rho;
    }
}

// Spectral master += added spectra (six components), Nyquist modes left at zero.
template <typename C>
__global__ void add_spectra_kernel(C* EBh, const C* add, int64_t M, int nx, int ny, int nz, int nzh) {
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < M;
         m += (int64_t)gridDim.x * blockDim.x) {
        const int mz = (int)(m % nzh);
        const int64_t r = m / nzh;
        const int my = (int)(r % ny);
        const int mx = (int)(r / ny);
        if (is_nyquist(mx, my, mz, nx, ny, nz)) continue;
#pragma unroll
        for (int q = 0; q < 6; ++q) EBh[q * M + m] = cadd(EBh[q * M + m], add[q * M + m]);
    }
}

// Per-axis phases of the shift that carries a field from one Galilean grid to
// another moving (dvx, dvy, dvz) faster: exp(i k_d dv_d t) with the spectral k_d =
// 2 pi s/(n d), entries ph[nx + ny + nzh] in FFT order. FP64: the phase in turns,
// s dv t/(n d), is reduced to its fractional part before sincospi, so that long
// runs (large t) keep full accuracy.
template <typename C>
__global__ void shift_phases_kernel(C* __restrict__ ph, int nx, int ny, int nzh, int nz, double dx,
                                    double dy, double dz, double dvx, double dvy, double dvz, double t) {
    const int total = nx + ny + nzh;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        int n, s;
        double d, dv;
        if (i < nx) {
            n = nx, d = dx, dv = dvx, s = signed_index(i, nx);
        } else if (i < nx + ny) {
            n = ny, d = dy, dv = dvy, s = signed_index(i - nx, ny);
        } else {
            n = nz, d = dz, dv = dvz, s = i - nx - ny;
        }
        double turns = (double)s * (dv * t / ((double)n * d));
        turns -= rint(turns);
        double sn, cs;
        sincospi(2.0 * turns, &sn, &cs);
        ph[i] = mk<C>(cs, sn);
    }
}

// EBs_dst += (1/N) exp(i k.(v_dst - v_src) t) EBh_src for the six components: the
// part of the field carried by another grid, moved onto this grid's nodes and
// added to the copy that the inverse transform turns into the gathered field.
// Reads 12 and writes 6 complex per mode; HBM-bound like the k-space update.
template <typename C, typename T>
__global__ void add_shifted_kernel(C* __restrict__ EBs, const C* __restrict__ EBh_src,
                                   const C* __restrict__ ph, int64_t M, int nx, int ny, int nz, int nzh,
                                   T invN) {
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < M;
         m += (int64_t)gridDim.x * blockDim.x) {
        const int mz = (int)(m % nzh);
        const int64_t r = m / nzh;
        const int my = (int)(r % ny);
        const int mx = (int)(r / ny);
        if (is_nyquist(mx, my, mz, nx, ny, nz)) continue;
        const C p = cscale(cmul(cmul(ph[mx], ph[nx + my]), ph[nx + ny + mz]), invN);
#pragma unroll
        for (int q = 0; q < 6; ++q) EBs[q * M + m] = cadd(EBs[q * M + m], cmul(p, EBh_src[q * M + m]));
    }
}

template <typename C, typename T>
__global__ void scale_copy_kernel(C* dst, const C* src, int64_t n, T s) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = cscale(src[i], s);
}

// Field energy, pass 1: per-block sums of E^2 and B^2 (FP64) into `part`, and
// the non-finite flag. Pass 2 adds the partial sums in a fixed order, so the
// result does not depend on scheduling.
// FP32 fields: a node's |E|^2 and |B|^2 are formed in FP32 (three squares, relative
// error a few 2^-24, finite while every component is below 1.8e19) and only the sums
// over nodes run in FP64; this GPU's FP64 rate is low enough that squaring each
// component in FP64 made the kernel several times slower than its memory traffic.
template <typename T>
__global__ void __launch_bounds__(256) energy_partial_kernel(const T* __restrict__ F, int64_t N,
                                                             double* __restrict__ part,
                                                             int32_t* status) {
    double se = 0.0, sb = 0.0;
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        if constexpr (sizeof(T) == 4) {
            const float e0 = F[i], e1 = F[N + i], e2 = F[2 * N + i];
            const float b0 = F[3 * N + i], b1 = F[4 * N + i], b2 = F[5 * N + i];
            se += (double)fmaf(e0, e0, fmaf(e1, e1, e2 * e2));
            sb += (double)fmaf(b0, b0, fmaf(b1, b1, b2 * b2));
            bad |= !(isfinite(e0) && isfinite(e1) && isfinite(e2) && isfinite(b0) && isfinite(b1) &&
                     isfinite(b2));
        } else {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                double v = (double)F[q * N + i];
                double w = (double)F[(3 + q) * N + i];
                se += v * v;
                sb += w * w;
                bad |= !isfinite(v) || !isfinite(w);
            }
        }
    }
    __shared__ double s_e[8], s_b[8];
    for (int o = 16; o > 0; o >>= 1) {
        se += __shfl_down_sync(0xffffffffu, se, o);
        sb += __shfl_down_sync(0xffffffffu, sb, o);
    }
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        s_e[warp] = se;
        s_b[warp] = sb;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, PIC_STATUS_NONFINITE);
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += s_e[w];
            b += s_b[w];
        }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
}

__global__ void energy_final_kernel(const double* __restrict__ part, int nb, double se_scale,
                                    double sb_scale, double* out) {
    __shared__ double s_e[256], s_b[256];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        a += part[2 * i];
        b += part[2 * i + 1];
    }
    s_e[threadIdx.x] = a;
    s_b[threadIdx.x] = b;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            s_e[threadIdx.x] += s_e[threadIdx.x + s];
            s_b[threadIdx.x] += s_b[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = se_scale * s_e[0] + sb_scale * s_b[0];
}

int grid_for(int64_t n, int block) {
    int64_t g = (n + block - 1) / block;
    int64_t cap = 152 * 16;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

int launch_build_tables(pic_sim* s, cudaStream_t st) {
    const pic_config& c = s->cfg;
    GaussLegendre gl = gauss_legendre();
    const int fx = c.vgal[0] == 0.0, fy = c.vgal[1] == 0.0;
    const int64_t rep = (int64_t)(fx ? s->d.nx / 2 + 1 : s->d.nx) * (fy ? s->d.ny / 2 + 1 : s->d.ny) * s->d.nzh;
    // wavenumbers first: the tables, the initial field and every k-space update read them
    const StencilWeights sw = stencil_weights(c.stencil_order);
    const int nk = s->d.nx + s->d.ny + s->d.nzh;
    if (c.precision == 64)
        wavenumbers_kernel<double><<<(nk + 127) / 128, 128, 0, st>>>(
            s->K, (double*)s->Kt, s->d.nx, s->d.ny, s->d.nzh, s->d.nz, c.dx, c.dy, c.dz, sw);
    else
        wavenumbers_kernel<float><<<(nk + 127) / 128, 128, 0, st>>>(
            s->K, (float*)s->Kt, s->d.nx, s->d.ny, s->d.nzh, s->d.nz, c.dx, c.dy, c.dz, sw);
    GP_CUDA(cudaGetLastError());
    int grid = grid_for(rep, 128);
    if (c.precision == 64)
        build_tables_kernel<double2><<<grid, 128, 0, st>>>(
            (double2*)s->Tab, s->K, s->d.nx, s->d.ny, s->d.nz, s->d.nzh, s->d.M, c.dt,
            c.vgal[0], c.vgal[1], c.vgal[2], c.c, c.eps0, c.current_correction, gl, fx, fy);
    else
        build_tables_kernel<float2><<<grid, 128, 0, st>>>(
            (float2*)s->Tab, s->K, s->d.nx, s->d.ny, s->d.nz, s->d.nzh, s->d.M, c.dt,
            c.vgal[0], c.vgal[1], c.vgal[2], c.c, c.eps0, c.current_correction, gl, fx, fy);
    GP_CUDA(cudaGetLastError());
    return PIC_OK;
}

template <typename T>
static void fill_kparams(const pic_sim* s, KParams<T>& p, void* EBs, const void* Sh) {
    typedef typename cplx<T>::type C;
    const pic_config& c = s->cfg;
    memset(&p, 0, sizeof(p));
    p.EBh = (C*)s->EBh;
    p.EBs = (C*)(EBs ? EBs : s->EBs);
    p.Sh = (const C*)(Sh ? Sh : s->Sh);
    p.Rn = (C*)s->Rn;
    p.tab = (const C*)s->Tab;
    p.M = s->d.M;
    p.nx = s->d.nx;
    p.ny = s->d.ny;
    p.nz = s->d.nz;
    p.nzh = s->d.nzh;
    p.kx = (const T*)s->Kt;
    p.ky = p.kx + s->d.nx;
    p.kz = p.ky + s->d.ny;
    p.c2 = (T)(c.c * c.c);
    p.invN = (T)(1.0 / (double)s->d.N);
    for (int d = 0; d < 3; ++d) p.bg[d] = (T)((double)s->d.N * c.rho_bg * c.vgal[d]);
    p.cc = c.current_correction;
    p.nyq_mask = 7;
}

template <typename T>
static int kspace_typed(pic_sim* s, cudaStream_t st) {
    KParams<T> p;
    fill_kparams<T>(s, p, nullptr, nullptr);
    kspace_update_kernel<T><<<grid_for(s->d.M, 256), 256, 0, st>>>(p);
    GP_CUDA(cudaGetLastError());
    return PIC_OK;
}

int launch_kspace_update(pic_sim* s, cudaStream_t st) {
    return s->cfg.precision == 64 ? kspace_typed<double>(s, st) : kspace_typed<float>(s, st);
}

// Wavenumbers and per-mode factors of a grid that has the run's nx, ny, cell sizes,
// units, v_gal and stencil order but nz_w nodes along z (the windows of a decomposed
// field update): K (FP64) and Kt (run precision) hold nx + ny + nz_w/2 + 1 entries, tab
// 6 nx ny (nz_w/2 + 1) complex factors.
int launch_window_tables(const pic_sim* s, int nz_w, double* K, void* Kt, void* tab, cudaStream_t st) {
    const pic_config& c = s->cfg;
    const int nx = s->d.nx, ny = s->d.ny, nzh = nz_w / 2 + 1;
    const int64_t M = (int64_t)nx * ny * nzh;
    const StencilWeights sw = stencil_weights(c.stencil_order);
    const int nk = nx + ny + nzh;
    if (c.precision == 64)
        wavenumbers_kernel<double><<<(nk + 127) / 128, 128, 0, st>>>(K, (double*)Kt, nx, ny, nzh, nz_w, c.dx, c.dy,
                                                                     c.dz, sw);
    else
        wavenumbers_kernel<float><<<(nk + 127) / 128, 128, 0, st>>>(K, (float*)Kt, nx, ny, nzh, nz_w, c.dx, c.dy,
                                                                    c.dz, sw);
    GP_CUDA(cudaGetLastError());
    GaussLegendre gl = gauss_legendre();
    const int fx = c.vgal[0] == 0.0, fy = c.vgal[1] == 0.0;
    const int64_t rep = (int64_t)(fx ? nx / 2 + 1 : nx) * (fy ? ny / 2 + 1 : ny) * nzh;
    const int grid = grid_for(rep, 128);
    if (c.precision == 64)
        build_tables_kernel<double2><<<grid, 128, 0, st>>>((double2*)tab, K, nx, ny, nz_w, nzh, M, c.dt, c.vgal[0],
                                                           c.vgal[1], c.vgal[2], c.c, c.eps0, c.current_correction,
                                                           gl, fx, fy);
    else
        build_tables_kernel<float2><<<grid, 128, 0, st>>>((float2*)tab, K, nx, ny, nz_w, nzh, M, c.dt, c.vgal[0],
                                                          c.vgal[1], c.vgal[2], c.c, c.eps0, c.current_correction,
                                                          gl, fx, fy);
    GP_CUDA(cudaGetLastError());
    return PIC_OK;
}

template <typename T>
static void fill_window_kparams(const pic_sim* s, KParams<T>& p, int nz_w, void* spec, void* ebs, const void* Kt,
                                const void* tab) {
    typedef typename cplx<T>::type C;
    const pic_config& c = s->cfg;
    const int nzh = nz_w / 2 + 1;
    const int64_t M = (int64_t)s->d.nx * s->d.ny * nzh, N = (int64_t)s->d.nx * s->d.ny * nz_w;
    memset(&p, 0, sizeof(p));
    p.EBh = (C*)spec;                 // window spectra: E (3), B (3), J (3), rho^{n+1}, rho^n
    p.Sh = (const C*)spec + 6 * M;
    p.Rn = (C*)spec + 10 * M;
    p.EBs = (C*)ebs;
    p.tab = (const C*)tab;
    p.M = M;
    p.nx = s->d.nx;
    p.ny = s->d.ny;
    p.nz = nz_w;
    p.nzh = nzh;
    p.kx = (const T*)Kt;
    p.ky = p.kx + s->d.nx;
    p.kz = p.ky + s->d.ny;
    p.c2 = (T)(c.c * c.c);
    p.invN = (T)(1.0 / (double)N);
    for (int d = 0; d < 3; ++d) p.bg[d] = (T)((double)N * c.rho_bg * c.vgal[d]);
    p.cc = c.current_correction;
    p.nyq_mask = 0;
}

void fill_window_kspace_desc(const pic_sim* s, void* out, int nz_w, void* spec, void* ebs, const void* Kt,
                             const void* tab) {
    if (s->cfg.precision == 64)
        fill_window_kparams<double>(s, *static_cast<KParams<double>*>(out), nz_w, spec, ebs, Kt, tab);
    else
        fill_window_kparams<float>(s, *static_cast<KParams<float>*>(out), nz_w, spec, ebs, Kt, tab);
}

int launch_kspace_windows(const pic_sim* s, const void* descs, int nwin, int64_t M_w, cudaStream_t st) {
    const int gx = std::max(1, grid_for(M_w, 256) / std::max(1, std::min(nwin, 16)));
    if (s->cfg.precision == 64)
        kspace_update_many_kernel<double><<<dim3(gx, nwin), 256, 0, st>>>((const KParams<double>*)descs);
    else
        kspace_update_many_kernel<float><<<dim3(gx, nwin), 256, 0, st>>>((const KParams<float>*)descs);
    GP_CUDA(cudaGetLastError());
    return PIC_OK;
}

// Quasi-cylindrical modes: per-mode factors at k = (k_r, 0, k_z) (no mirror symmetry along
// the radial spectrum) and the k-space parameters of one mode's arrays.
int launch_cyl_tables(int precision, int nr, int nz, const double* K, void* tab, double dt, double vgal, double c,
                      double eps0, int cc, cudaStream_t st) {
    GaussLegendre gl = gauss_legendre();
    const int64_t M = (int64_t)nr * nz;
    const int grid = grid_for(M, 128);
    if (precision == 64)
        build_tables_kernel<double2><<<grid, 128, 0, st>>>((double2*)tab, K, nr, 1, nz, nz, M, dt, 0.0, 0.0, vgal, c,
                                                           eps0, cc, gl, 0, 0);
    else
        build_tables_kernel<float2><<<grid, 128, 0, st>>>((float2*)tab, K, nr, 1, nz, nz, M, dt, 0.0, 0.0, vgal, c,
                                                          eps0, cc, gl, 0, 0);
    GP_CUDA(cudaGetLastError());
    return PIC_OK;
}

template <typename T>
static void fill_cyl_kparams(KParams<T>& p, int nr, int nz, void* EBh, const void* Sh, void* Rn, void* scratch,
                             const void* tab, const void* Kt, double c, int cc) {
    typedef typename cplx<T>::type C;
    memset(&p, 0, sizeof(p));
    p.EBh = (C*)EBh;
    p.EBs = (C*)scratch;
    p.Sh = (const C*)Sh;
    p.Rn = (C*)Rn;
    p.tab = (const C*)tab;
    p.M = (int64_t)nr * nz;
    p.nx = nr;
    p.ny = 1;
    p.nz = nz;
    p.nzh = nz;
    p.kx = (const T*)Kt;
    p.ky = p.kx + nr;
    p.kz = p.ky + 1;
    p.c2 = (T)(c * c);
    p.invN = (T)1;
    p.cc = cc;
    p.nyq_mask = 4;
}

void fill_cyl_kspace_desc(int precision, void* out, int nr, int nz, void* EBh, const void* Sh, void* Rn,
                          void* scratch, const void* tab, const void* Kt, double c, int cc) {
    if (precision == 64)
        fill_cyl_kparams<double>(*static_cast<KParams<double>*>(out), nr, nz, EBh, Sh, Rn, scratch, tab, Kt, c, cc);
    else
        fill_cyl_kparams<float>(*static_cast<KParams<float>*>(out), nr, nz, EBh, Sh, Rn, scratch, tab, Kt, c, cc);
}

int launch_kspace_descs(int precision, const void* descs, int n, int64_t M, cudaStream_t st) {
    const int gx = std::max(1, grid_for(M, 256) / std::max(1, std::min(n, 16)));
    if (precision == 64)
        kspace_update_many_kernel<double><<<dim3(gx, n), 256, 0, st>>>((const KParams<double>*)descs);
    else
        kspace_update_many_kernel<float><<<dim3(gx, n), 256, 0, st>>>((const KParams<float>*)descs);
    GP_CUDA(cudaGetLastError());
    return PIC_OK;
}

size_t kspace_desc_bytes(int precision) {
    return precision == 64 ? sizeof(KParams<double>) : sizeof(KParams<float>);
}

void fill_kspace_desc(const pic_sim* s, void* out, void* EBs, const void* Sh) {
    if (s->cfg.precision == 64)
        fill_kparams<double>(s, *static_cast<KParams<double>*>(out), EBs, Sh);
    else
        fill_kparams<float>(s, *static_cast<KParams<float>*>(out), EBs, Sh);
}

int launch_kspace_many(const pic_sim* s0, const void* descs, int nruns, cudaStream_t st) {
    // every run has the same mode count; the grid-stride loop covers it per run
    const int gx = std::max(1, grid_for(s0->d.M, 256) / std::max(1, std::min(nruns, 16)));
    const dim3 grid(gx, nruns);
    if (s0->cfg.precision == 64)
        kspace_update_many_kernel<double><<<grid, 256, 0, st>>>((const KParams<double>*)descs);
    else
        kspace_update_many_kernel<float><<<grid, 256, 0, st>>>((const KParams<float>*)descs);
    GP_CUDA(cudaGetLastError());
    return PIC_OK;
}

int launch_init_fields(pic_sim* s, cudaStream_t st) {
    const pic_config& c = s->cfg;
    int grid = grid_for(s->d.M, 256);
    if (c.precision == 64)
        init_fields_kernel<double2><<<grid, 256, 0, st>>>(
            (double2*)s->EBh, (double2*)s->Rn, (const double2*)s->Sh, s->d.M, s->d.nx, s->d.ny,
            s->d.nz, s->d.nzh, s->K, c.beta_init[0], c.beta_init[1], c.beta_init[2], c.c,
            c.eps0, c.init_fields);
    else
        init_fields_kernel<float2><<<grid, 256, 0, st>>>(
            (float2*)s->EBh, (float2*)s->Rn, (const float2*)s->Sh, s->d.M, s->d.nx, s->d.ny,
            s->d.nz, s->d.nzh, s->K, c.beta_init[0], c.beta_init[1], c.beta_init[2], c.c,
            c.eps0, c.init_fields);
    GP_CUDA(cudaGetLastError());
    return PIC_OK;
}

int launch_add_spectra(pic_sim* s, const void* add, cudaStream_t st) {
    int grid = grid_for(s->d.M, 256);
    if (s->cfg.precision == 64)
        add_spectra_kernel<double2><<<grid, 256, 0, st>>>((double2*)s->EBh, (const double2*)add, s->d.M,
                                                          s->d.nx, s->d.ny, s->d.nz, s->d.nzh);
    else
        add_spectra_kernel<float2><<<grid, 256, 0, st>>>((float2*)s->EBh, (const float2*)add, s->d.M,
                                                         s->d.nx, s->d.ny, s->d.nz, s->d.nzh);
    GP_CUDA(cudaGetLastError());
    return PIC_OK;
}

int launch_add_shifted(pic_sim* dst, const pic_sim* src, double t, cudaStream_t st) {
    const pic_config& c = dst->cfg;
    const double dv[3] = {c.vgal[0] - src->cfg.vgal[0], c.vgal[1] - src->cfg.vgal[1],
                          c.vgal[2] - src->cfg.vgal[2]};
    const int nk = dst->d.nx + dst->d.ny + dst->d.nzh;
    const int grid = grid_for(dst->d.M, 256);
    const double invN = 1.0 / (double)dst->d.N;
    if (c.precision == 64) {
        shift_phases_kernel<double2><<<(nk + 127) / 128, 128, 0, st>>>(
            (double2*)dst->Ph, dst->d.nx, dst->d.ny, dst->d.nzh, dst->d.nz, c.dx, c.dy, c.dz, dv[0], dv[1],
            dv[2], t);
        add_shifted_kernel<double2, double><<<grid, 256, 0, st>>>(
            (double2*)dst->EBs, (const double2*)src->EBh, (const double2*)dst->Ph, dst->d.M, dst->d.nx,
            dst->d.ny, dst->d.nz, dst->d.nzh, invN);
    } else {
        shift_phases_kernel<float2><<<(nk + 127) / 128, 128, 0, st>>>(
            (float2*)dst->Ph, dst->d.nx, dst->d.ny, dst->d.nzh, dst->d.nz, c.dx, c.dy, c.dz, dv[0], dv[1],
            dv[2], t);
        add_shifted_kernel<float2, float><<<grid, 256, 0, st>>>(
            (float2*)dst->EBs, (const float2*)src->EBh, (const float2*)dst->Ph, dst->d.M, dst->d.nx,
            dst->d.ny, dst->d.nz, dst->d.nzh, (float)invN);
    }
    GP_CUDA(cudaGetLastError());
    return PIC_OK;
}

int launch_master_to_scratch(pic_sim* s, cudaStream_t st) {
    int64_t n = 6 * s->d.M;
    int grid = grid_for(n, 256);
    double invN = 1.0 / (double)s->d.N;
    if (s->cfg.precision == 64)
        scale_copy_kernel<double2, double><<<grid, 256, 0, st>>>((double2*)s->EBs,
                                                                 (const double2*)s->EBh, n, invN);
    else
        scale_copy_kernel<float2, float><<<grid, 256, 0, st>>>((float2*)s->EBs,
                                                               (const float2*)s->EBh, n, (float)invN);
    GP_CUDA(cudaGetLastError());
    return PIC_OK;
}

int launch_energy_on(const void* F, int64_t N, int precision, double* part, int nb, int32_t* status,
                     double se_scale, double sb_scale, double* out_dev, cudaStream_t st) {
    if (precision == 64)
        energy_partial_kernel<double><<<nb, 256, 0, st>>>((const double*)F, N, part, status);
    else
        energy_partial_kernel<float><<<nb, 256, 0, st>>>((const float*)F, N, part, status);
    GP_CUDA(cudaGetLastError());
    energy_final_kernel<<<1, 256, 0, st>>>(part, nb, se_scale, sb_scale, out_dev);
    GP_CUDA(cudaGetLastError());
    return PIC_OK;
}

int launch_energy(pic_sim* s, double* out_dev, cudaStream_t st) {
    const pic_config& c = s->cfg;
    double dV = c.dx * c.dy * c.dz;
    int nb = s->energy_blocks;
    if (c.precision == 64)
        energy_partial_kernel<double><<<nb, 256, 0, st>>>((const double*)s->F, s->d.N, s->epart,
                                                          s->status);
    else
        energy_partial_kernel<float><<<nb, 256, 0, st>>>((const float*)s->F, s->d.N, s->epart,
                                                         s->status);
    GP_CUDA(cudaGetLastError());
    energy_final_kernel<<<1, 256, 0, st>>>(s->epart, nb, 0.5 * c.eps0 * dV,
                                           0.5 * c.eps0 * dV * c.c * c.c, out_dev);
    GP_CUDA(cudaGetLastError());
    return PIC_OK;
}

}  // namespace galpic
