// Particle-side kernels of the Galilean-PSATD step:
//   * generate       - regular lattice plus seeded jitter (splitmix64 counters);
//   * sort           - counting sort of each species into bins of BX*BY*BZ cells,
//                      executed only when the device counters ask for it;
//   * particle pass  - one CTA per bin: the bin's field tile (plus halo) is staged
//                      in shared memory, each particle gathers E and B, takes the
//                      relativistic Boris push and the Galilean drift in two halves,
//                      and deposits J^{n+1/2} and rho^{n+1} into a shared-memory
//                      tile, which is added to the global grids once per CTA.
//                      Particles whose stencil leaves the tile (they moved far from
//                      their bin since the last sort) use global memory directly.
#include <math.h>

#include "common.cuh"

namespace galpic {

namespace {

__device__ __forceinline__ int wrapi(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

// Shape factors of order 1, 2, 3 (B-splines) for a particle at cell i with offset
// f in [0, 1): node i + J0 + a gets weight w[a], a = 0 .. NW-1.
template <int ORDER> struct Shape;

template <> struct Shape<1> {
    static constexpr int NW = 2, J0 = 0;
    template <typename T> __device__ static void w(T f, T* w) {
        w[0] = (T)1 - f;
        w[1] = f;
    }
};

template <> struct Shape<2> {
    static constexpr int NW = 4, J0 = -1;
    // nearest node n = i + (f >= 1/2), d = f - (f >= 1/2):
    // W(n-1) = (1/2 - d)^2/2, W(n) = 3/4 - d^2, W(n+1) = (1/2 + d)^2/2
    template <typename T> __device__ static void w(T f, T* w) {
        bool up = f >= (T)0.5;
        T d = up ? f - (T)1 : f;
        T a = (T)0.5 * ((T)0.5 - d) * ((T)0.5 - d);
        T b = (T)0.75 - d * d;
        T c = (T)0.5 * ((T)0.5 + d) * ((T)0.5 + d);
        w[0] = up ? (T)0 : a;
        w[1] = up ? a : b;
        w[2] = up ? b : c;
        w[3] = up ? c : (T)0;
    }
};

template <> struct Shape<3> {
    static constexpr int NW = 4, J0 = -1;
    // cubic B-spline at node distances 1+f, f, 1-f, 2-f
    template <typename T> __device__ static void w(T f, T* w) {
        T g = (T)1 - f;
        T f2 = f * f, g2 = g * g;
        w[0] = g2 * g * (T)(1.0 / 6.0);
        w[1] = (T)(2.0 / 3.0) - f2 + (T)0.5 * f2 * f;
        w[2] = (T)(2.0 / 3.0) - g2 + (T)0.5 * g2 * g;
        w[3] = f2 * f * (T)(1.0 / 6.0);
    }
};

template <typename T>
struct SpeciesK {
    int32_t* cell;
    T* off[3];
    T* u[3];
    const int32_t* bin_start;
    T qw_dv;   // q w / dV
    T qdt2m;   // q dt / (2 m)
};

template <typename T>
struct PassK {
    const T* F;     // real E (3N) then B (3N)
    T* S;           // real Jx, Jy, Jz, rho (4N)
    int64_t N;
    int nx, ny, nz;
    int BX, BY, BZ, nbx, nby, nbz;
    int RX, RY, RZ, R;   // shared tile extent (nodes)
    int margin;
    T inv_c2;
    T hd[3];             // dt / (2 d) per axis
    T vgal[3];
    int nspecies;
    SpeciesK<T> sp[PIC_MAX_SPECIES];
    unsigned long long* cnt;
};

// Move (i, f) by d cells along an axis of n cells: offset back to [0, 1), periodic.
template <typename T>
__device__ __forceinline__ void drift_axis(int& i, T& f, T d, int n) {
    f += d;
    T s = floor(f);
    f -= s;
    int si = (int)s;
    if (f >= (T)1) {
        f -= (T)1;
        si += 1;
    }
    i = wrapi(i + si, n);
}

// Tile index of the first stencil node of a particle in cell i along one axis
// (tile node t holds global node o + t with o = bin origin + J0 - margin, so the
// stencil start i + J0 sits at t = i - bin origin + margin, taken modulo the
// periodic axis length n); -1 if the tile does not hold the whole stencil.
template <int ORDER>
__device__ __forceinline__ int tile_start(int rel, int n, int extent) {
    int r = wrapi(rel, n);
    return (r + Shape<ORDER>::NW <= extent) ? r : -1;
}

template <typename T, int ORDER, int MODE>
__global__ void __launch_bounds__(256) particle_pass_kernel(PassK<T> p) {
    typedef Shape<ORDER> SH;
    constexpr int NW = SH::NW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sF = reinterpret_cast<T*>(smem_raw);              // 6 * R (STEP only)
    T* sD = sF + (MODE == PASS_STEP ? 6 * p.R : 0);       // 4 * R

    const int b = blockIdx.x;
    const int bz = b % p.nbz, by = (b / p.nbz) % p.nby, bx = b / (p.nbz * p.nby);
    const int x0 = bx * p.BX, y0 = by * p.BY, z0 = bz * p.BZ;
    // tile origin (global node of tile index 0) and the stencil origin of a
    // particle in the bin's first cell
    const int ox = x0 + SH::J0 - p.margin, oy = y0 + SH::J0 - p.margin, oz = z0 + SH::J0 - p.margin;
    const int R = p.R;
    const int64_t N = p.N;

    for (int idx = threadIdx.x; idx < R; idx += blockDim.x) {
        int rz = idx % p.RZ, ry = (idx / p.RZ) % p.RY, rx = idx / (p.RZ * p.RY);
        if (MODE == PASS_STEP) {
            int64_t g = ((int64_t)wrapi(ox + rx, p.nx) * p.ny + wrapi(oy + ry, p.ny)) * p.nz +
                        wrapi(oz + rz, p.nz);
#pragma unroll
            for (int q = 0; q < 6; ++q) sF[q * R + idx] = p.F[q * N + g];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) sD[q * R + idx] = (T)0;
    }
    __syncthreads();

    unsigned long long miss = 0, far = 0;
    for (int s = 0; s < p.nspecies; ++s) {
        const SpeciesK<T> sp = p.sp[s];
        const int beg = sp.bin_start[b], end = sp.bin_start[b + 1];
        for (int i = beg + threadIdx.x; i < end; i += blockDim.x) {
            int c = sp.cell[i];
            int ix = c / (p.ny * p.nz);
            int rem = c - ix * (p.ny * p.nz);
            int iy = rem / p.nz;
            int iz = rem - iy * p.nz;
            T fx = sp.off[0][i], fy = sp.off[1][i], fz = sp.off[2][i];
            T ux = sp.u[0][i], uy = sp.u[1][i], uz = sp.u[2][i];
            T wx[4], wy[4], wz[4];
            T vx, vy, vz;
            if (MODE == PASS_STEP) {
                // ---- gather E^n, B^n at x^n
                SH::w(fx, wx);
                SH::w(fy, wy);
                SH::w(fz, wz);
                T E[3] = {0, 0, 0}, B[3] = {0, 0, 0};
                int rx = tile_start<ORDER>(ix - x0 + p.margin, p.nx, p.RX);
                int ry = tile_start<ORDER>(iy - y0 + p.margin, p.ny, p.RY);
                int rz = tile_start<ORDER>(iz - z0 + p.margin, p.nz, p.RZ);
                if (rx >= 0 && ry >= 0 && rz >= 0) {
#pragma unroll
                    for (int a = 0; a < NW; ++a)
#pragma unroll
                        for (int bb = 0; bb < NW; ++bb) {
                            T wxy = wx[a] * wy[bb];
                            int base = ((rx + a) * p.RY + (ry + bb)) * p.RZ + rz;
#pragma unroll
                            for (int cc = 0; cc < NW; ++cc) {
                                T w = wxy * wz[cc];
                                int q0 = base + cc;
                                E[0] += w * sF[0 * R + q0];
                                E[1] += w * sF[1 * R + q0];
                                E[2] += w * sF[2 * R + q0];
                                B[0] += w * sF[3 * R + q0];
                                B[1] += w * sF[4 * R + q0];
                                B[2] += w * sF[5 * R + q0];
                            }
                        }
                } else {
                    far++;
#pragma unroll
                    for (int a = 0; a < NW; ++a)
#pragma unroll
                        for (int bb = 0; bb < NW; ++bb) {
                            T wxy = wx[a] * wy[bb];
                            int64_t base = ((int64_t)wrapi(ix + SH::J0 + a, p.nx) * p.ny +
                                            wrapi(iy + SH::J0 + bb, p.ny)) * p.nz;
#pragma unroll
                            for (int cc = 0; cc < NW; ++cc) {
                                T w = wxy * wz[cc];
                                int64_t g = base + wrapi(iz + SH::J0 + cc, p.nz);
                                E[0] += w * p.F[0 * N + g];
                                E[1] += w * p.F[1 * N + g];
                                E[2] += w * p.F[2 * N + g];
                                B[0] += w * p.F[3 * N + g];
                                B[1] += w * p.F[4 * N + g];
                                B[2] += w * p.F[5 * N + g];
                            }
                        }
                }
                // ---- relativistic Boris push u^{n-1/2} -> u^{n+1/2}
                const T a = sp.qdt2m;
                T umx = ux + a * E[0], umy = uy + a * E[1], umz = uz + a * E[2];
                T gm = sqrt((T)1 + (umx * umx + umy * umy + umz * umz) * p.inv_c2);
                T tx = a * B[0] / gm, ty = a * B[1] / gm, tz = a * B[2] / gm;
                T s2 = (T)2 / ((T)1 + tx * tx + ty * ty + tz * tz);
                T sx = s2 * tx, sy = s2 * ty, sz = s2 * tz;
                T upx = umx + (umy * tz - umz * ty);
                T upy = umy + (umz * tx - umx * tz);
                T upz = umz + (umx * ty - umy * tx);
                ux = umx + (upy * sz - upz * sy) + a * E[0];
                uy = umy + (upz * sx - upx * sz) + a * E[1];
                uz = umz + (upx * sy - upy * sx) + a * E[2];
            }
            T gam = sqrt((T)1 + (ux * ux + uy * uy + uz * uz) * p.inv_c2);
            vx = ux / gam;
            vy = uy / gam;
            vz = uz / gam;
            // deposit passes: J (3 values) at x^{n+1/2} then rho at x^{n+1} (STEP),
            // or J and rho at the current x (DEPOSIT)
#pragma unroll
            for (int phase = 0; phase < 2; ++phase) {
                if (MODE == PASS_STEP) {
                    drift_axis(ix, fx, (vx - p.vgal[0]) * p.hd[0], p.nx);
                    drift_axis(iy, fy, (vy - p.vgal[1]) * p.hd[1], p.ny);
                    drift_axis(iz, fz, (vz - p.vgal[2]) * p.hd[2], p.nz);
                }
                if (MODE == PASS_STEP || phase == 0) {
                    SH::w(fx, wx);
                    SH::w(fy, wy);
                    SH::w(fz, wz);
                }
                // quantities deposited in this phase: Jx, Jy, Jz, then rho
                const int q_lo = phase == 0 ? 0 : 3;
                const int q_hi = phase == 0 ? 3 : 4;
                T val[3];
                if (phase == 0) {
                    val[0] = sp.qw_dv * vx;
                    val[1] = sp.qw_dv * vy;
                    val[2] = sp.qw_dv * vz;
                } else {
                    val[0] = sp.qw_dv;
                }
                int rx = tile_start<ORDER>(ix - x0 + p.margin, p.nx, p.RX);
                int ry = tile_start<ORDER>(iy - y0 + p.margin, p.ny, p.RY);
                int rz = tile_start<ORDER>(iz - z0 + p.margin, p.nz, p.RZ);
                if (rx >= 0 && ry >= 0 && rz >= 0) {
#pragma unroll
                    for (int a = 0; a < NW; ++a)
#pragma unroll
                        for (int bb = 0; bb < NW; ++bb) {
                            T wxy = wx[a] * wy[bb];
                            int base = ((rx + a) * p.RY + (ry + bb)) * p.RZ + rz;
#pragma unroll
                            for (int cc = 0; cc < NW; ++cc) {
                                T w = wxy * wz[cc];
                                for (int q = q_lo; q < q_hi; ++q)
                                    atomicAdd(&sD[q * R + base + cc], w * val[q - q_lo]);
                            }
                        }
                } else {
                    if (phase == 1) far++;
#pragma unroll
                    for (int a = 0; a < NW; ++a)
#pragma unroll
                        for (int bb = 0; bb < NW; ++bb) {
                            T wxy = wx[a] * wy[bb];
                            int64_t base = ((int64_t)wrapi(ix + SH::J0 + a, p.nx) * p.ny +
                                            wrapi(iy + SH::J0 + bb, p.ny)) * p.nz;
#pragma unroll
                            for (int cc = 0; cc < NW; ++cc) {
                                T w = wxy * wz[cc];
                                int64_t g = base + wrapi(iz + SH::J0 + cc, p.nz);
                                for (int q = q_lo; q < q_hi; ++q)
                                    atomicAdd(&p.S[q * N + g], w * val[q - q_lo]);
                            }
                        }
                }
            }
            if (MODE == PASS_STEP) {
                sp.cell[i] = (ix * p.ny + iy) * p.nz + iz;
                sp.off[0][i] = fx;
                sp.off[1][i] = fy;
                sp.off[2][i] = fz;
                sp.u[0][i] = ux;
                sp.u[1][i] = uy;
                sp.u[2][i] = uz;
                if (ix / p.BX != bx || iy / p.BY != by || iz / p.BZ != bz) miss++;
            }
        }
    }
    __syncthreads();

    // add the tile to the global source grids
    for (int idx = threadIdx.x; idx < R; idx += blockDim.x) {
        int rz = idx % p.RZ, ry = (idx / p.RZ) % p.RY, rx = idx / (p.RZ * p.RY);
        int64_t g = ((int64_t)wrapi(ox + rx, p.nx) * p.ny + wrapi(oy + ry, p.ny)) * p.nz +
                    wrapi(oz + rz, p.nz);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            T v = sD[q * R + idx];
            if (v != (T)0) atomicAdd(&p.S[q * N + g], v);
        }
    }

    if (MODE == PASS_STEP) {
        // warp-aggregated counters
        for (int o = 16; o > 0; o >>= 1) {
            miss += __shfl_down_sync(0xffffffffu, miss, o);
            far += __shfl_down_sync(0xffffffffu, far, o);
        }
        if ((threadIdx.x & 31) == 0) {
            if (miss) atomicAdd(&p.cnt[CNT_HOME_MISS], miss);
            if (far) atomicAdd(&p.cnt[CNT_FAR], far);
        }
    }
}

// ---------------------------------------------------------------------------
// Lattice generator
// ---------------------------------------------------------------------------
template <typename T>
__global__ void generate_kernel(int32_t* cell, T* ox, T* oy, T* oz, T* ux, T* uy, T* uz, int64_t n,
                                int nx, int ny, int nz, int px, int py, int pz, double jitter,
                                uint64_t key, double u0x, double u0y, double u0z) {
    const int64_t ppc = (int64_t)px * py * pz;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        int64_t c0 = p / ppc;
        int64_t slot = p - c0 * ppc;
        int la = (int)(slot / (py * pz));
        int lb = (int)((slot / pz) % py);
        int lc = (int)(slot % pz);
        int ii[3] = {(int)(c0 / ((int64_t)ny * nz)), (int)((c0 / nz) % ny), (int)(c0 % nz)};
        int ls[3] = {la, lb, lc};
        int np[3] = {px, py, pz};
        int ng[3] = {nx, ny, nz};
        T fo[3];
        for (int axis = 0; axis < 3; ++axis) {
            uint64_t z = splitmix64(key ^ ((uint64_t)p * 3ull + (uint64_t)axis));
            double r = (double)(z >> 11) * 0x1.0p-53;
            // same operation order as the host generator, without FMA contraction,
            // so that both produce bit-identical offsets
            double f = __dadd_rn(__ddiv_rn(ls[axis] + 0.5, (double)np[axis]),
                                 __dmul_rn(jitter, __dsub_rn(2.0 * r, 1.0)));
            double s = floor(f);
            f -= s;
            int i = ii[axis] + (int)s;
            if (f >= 1.0) {
                f -= 1.0;
                i += 1;
            }
            T ft = (T)f;
            if (ft >= (T)1) {   // rounding to float can reach 1
                ft = (T)0;
                i += 1;
            }
            ii[axis] = wrapi(i, ng[axis]);
            fo[axis] = ft;
        }
        cell[p] = (ii[0] * ny + ii[1]) * nz + ii[2];
        ox[p] = fo[0];
        oy[p] = fo[1];
        oz[p] = fo[2];
        ux[p] = (T)u0x;
        uy[p] = (T)u0y;
        uz[p] = (T)u0z;
    }
}

// Loaded particles: clamp a cell outside [0, N) to 0 and an offset outside
// [0, 1) (or not finite) to 0, and flag PIC_STATUS_BADINPUT, so that no kernel
// indexes out of bounds on bad input.
template <typename T>
__global__ void sanitize_kernel(int32_t* cell, T* ox, T* oy, T* oz, int64_t n, int64_t N,
                                int32_t* status) {
    bool any = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int c = cell[i];
        if (c < 0 || (int64_t)c >= N) {
            cell[i] = 0;
            any = true;
        }
        T* o[3] = {ox, oy, oz};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            T f = o[d][i];
            if (!(f >= (T)0 && f < (T)1)) {
                o[d][i] = (T)0;
                any = true;
            }
        }
    }
    if (any) atomicOr(status, PIC_STATUS_BADINPUT);
}

// ---------------------------------------------------------------------------
// Bin sort (runs only when sort_needed(cnt))
// ---------------------------------------------------------------------------
struct BinGeom {
    int ny, nz, BX, BY, BZ, nby, nbz;
    __device__ __forceinline__ int bin_of(int c) const {
        int ix = c / (ny * nz);
        int rem = c - ix * (ny * nz);
        int iy = rem / nz;
        int iz = rem - iy * nz;
        return ((ix / BX) * nby + iy / BY) * nbz + iz / BZ;
    }
};

__global__ void sort_zero_kernel(int32_t* bin_cnt, int nb, const unsigned long long* cnt) {
    if (!sort_needed(cnt)) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += gridDim.x * blockDim.x)
        bin_cnt[i] = 0;
}

__global__ void sort_count_kernel(const int32_t* __restrict__ cell, int64_t n, int32_t* rank,
                                  int32_t* bin_cnt, BinGeom g, const unsigned long long* cnt) {
    if (!sort_needed(cnt)) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        rank[i] = atomicAdd(&bin_cnt[g.bin_of(cell[i])], 1);
}

// Exclusive scan of the bin counts into bin_start[0 .. nb]; one block of 1024.
__global__ void __launch_bounds__(1024) sort_scan_kernel(const int32_t* bin_cnt, int32_t* bin_start,
                                                         int nb, const unsigned long long* cnt) {
    if (!sort_needed(cnt)) return;
    __shared__ int32_t part[1024];
    const int per = (nb + 1023) / 1024;
    const int lo = threadIdx.x * per;
    const int hi = min(nb, lo + per);
    int32_t s = 0;
    for (int i = lo; i < hi; ++i) s += bin_cnt[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        int32_t v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int32_t run = part[threadIdx.x] - s;
    for (int i = lo; i < hi; ++i) {
        bin_start[i] = run;
        run += bin_cnt[i];
    }
    if (threadIdx.x == 1023) bin_start[nb] = part[1023];
}

template <typename T>
struct Ptr6 {
    T* p[6];
};

template <typename T>
__global__ void sort_scatter_kernel(const int32_t* __restrict__ cell, Ptr6<T> src, int64_t n,
                                    const int32_t* __restrict__ rank,
                                    const int32_t* __restrict__ bin_start, int32_t* tcell,
                                    Ptr6<T> dst, BinGeom g, const unsigned long long* cnt) {
    if (!sort_needed(cnt)) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int c = cell[i];
        int64_t j = (int64_t)bin_start[g.bin_of(c)] + rank[i];
        tcell[j] = c;
#pragma unroll
        for (int q = 0; q < 6; ++q) dst.p[q][j] = src.p[q][i];
    }
}

template <typename T>
__global__ void sort_copyback_kernel(int32_t* cell, Ptr6<T> dst, int64_t n,
                                     const int32_t* __restrict__ tcell, Ptr6<T> src,
                                     const unsigned long long* cnt) {
    if (!sort_needed(cnt)) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        cell[i] = tcell[i];
#pragma unroll
        for (int q = 0; q < 6; ++q) dst.p[q][i] = src.p[q][i];
    }
}

// After a re-sort every particle is in its bin again: clear the request and the
// stray counts of the previous pass.
__global__ void sort_finish_kernel(unsigned long long* cnt) {
    if (sort_needed(cnt)) {
        cnt[CNT_FORCE_SORT] = 0ull;
        cnt[CNT_HOME_MISS] = 0ull;
        cnt[CNT_FAR] = 0ull;
        cnt[CNT_SORTS] += 1ull;
    }
}

int grid_for(int64_t n, int block) {
    int64_t g = (n + block - 1) / block;
    int64_t cap = 152 * 16;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

template <typename T>
int sort_typed(pic_sim* s, cudaStream_t st) {
    BinGeom g{s->d.ny, s->d.nz, s->d.BX, s->d.BY, s->d.BZ, s->d.nby, s->d.nbz};
    Ptr6<T> tmp;
    for (int d = 0; d < 3; ++d) {
        tmp.p[d] = (T*)s->tmp_off[d];
        tmp.p[3 + d] = (T*)s->tmp_u[d];
    }
    for (int k = 0; k < s->nspecies; ++k) {
        SpeciesDev& sp = s->sp[k];
        if (sp.n == 0) continue;
        sort_zero_kernel<<<grid_for(s->d.nbins, 256), 256, 0, st>>>(s->bin_cnt, s->d.nbins, s->cnt);
        sort_count_kernel<<<grid_for(sp.n, 256), 256, 0, st>>>(sp.cell, sp.n, s->tmp_rank,
                                                               s->bin_cnt, g, s->cnt);
        sort_scan_kernel<<<1, 1024, 0, st>>>(s->bin_cnt, sp.bin_start, s->d.nbins, s->cnt);
        Ptr6<T> own;
        for (int d = 0; d < 3; ++d) {
            own.p[d] = (T*)sp.off[d];
            own.p[3 + d] = (T*)sp.u[d];
        }
        sort_scatter_kernel<T><<<grid_for(sp.n, 256), 256, 0, st>>>(
            sp.cell, own, sp.n, s->tmp_rank, sp.bin_start, s->tmp_cell, tmp, g, s->cnt);
        sort_copyback_kernel<T><<<grid_for(sp.n, 256), 256, 0, st>>>(sp.cell, own, sp.n,
                                                                     s->tmp_cell, tmp, s->cnt);
    }
    sort_finish_kernel<<<1, 1, 0, st>>>(s->cnt);
    GP_CUDA(cudaGetLastError());
    return PIC_OK;
}

template <typename T, int ORDER, int MODE>
int pass_launch(pic_sim* s, cudaStream_t st) {
    const pic_config& c = s->cfg;
    PassK<T> p;
    p.F = (const T*)s->F;
    p.S = (T*)s->S;
    p.N = s->d.N;
    p.nx = s->d.nx;
    p.ny = s->d.ny;
    p.nz = s->d.nz;
    p.BX = s->d.BX;
    p.BY = s->d.BY;
    p.BZ = s->d.BZ;
    p.nbx = s->d.nbx;
    p.nby = s->d.nby;
    p.nbz = s->d.nbz;
    p.margin = s->d.margin;
    const int span = Shape<ORDER>::NW - 1 + 2 * s->d.margin;
    p.RX = s->d.BX + span;
    p.RY = s->d.BY + span;
    p.RZ = s->d.BZ + span;
    p.R = p.RX * p.RY * p.RZ;
    p.inv_c2 = (T)(1.0 / (c.c * c.c));
    p.hd[0] = (T)(0.5 * c.dt / c.dx);
    p.hd[1] = (T)(0.5 * c.dt / c.dy);
    p.hd[2] = (T)(0.5 * c.dt / c.dz);
    for (int d = 0; d < 3; ++d) p.vgal[d] = (T)c.vgal[d];
    p.nspecies = s->nspecies;
    const double dV = c.dx * c.dy * c.dz;
    for (int k = 0; k < s->nspecies; ++k) {
        const SpeciesDev& sp = s->sp[k];
        p.sp[k].cell = sp.cell;
        for (int d = 0; d < 3; ++d) {
            p.sp[k].off[d] = (T*)sp.off[d];
            p.sp[k].u[d] = (T*)sp.u[d];
        }
        p.sp[k].bin_start = sp.bin_start;
        p.sp[k].qw_dv = (T)(sp.q * sp.w / dV);
        p.sp[k].qdt2m = (T)(sp.q * c.dt / (2.0 * sp.m));
    }
    p.cnt = s->cnt;
    size_t smem = (size_t)(MODE == PASS_STEP ? 10 : 4) * p.R * sizeof(T);
    auto kern = particle_pass_kernel<T, ORDER, MODE>;
    GP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<s->d.nbins, 256, smem, st>>>(p);
    GP_CUDA(cudaGetLastError());
    return PIC_OK;
}

template <typename T, int MODE>
int pass_order(pic_sim* s, cudaStream_t st) {
    switch (s->cfg.shape_order) {
        case 1: return pass_launch<T, 1, MODE>(s, st);
        case 2: return pass_launch<T, 2, MODE>(s, st);
        default: return pass_launch<T, 3, MODE>(s, st);
    }
}

}  // namespace

size_t tile_bytes(const pic_config& c, const Dims& d, int mode) {
    int nw = c.shape_order == 1 ? 2 : 4;
    int span = nw - 1 + 2 * d.margin;
    size_t R = (size_t)(d.BX + span) * (d.BY + span) * (d.BZ + span);
    return (mode == PASS_STEP ? 10 : 4) * R * (c.precision == 64 ? 8 : 4);
}

int launch_particle_pass(pic_sim* s, int mode, cudaStream_t st) {
    if (s->cfg.precision == 64)
        return mode == PASS_STEP ? pass_order<double, PASS_STEP>(s, st)
                                 : pass_order<double, PASS_DEPOSIT>(s, st);
    return mode == PASS_STEP ? pass_order<float, PASS_STEP>(s, st)
                             : pass_order<float, PASS_DEPOSIT>(s, st);
}

int launch_sanitize(pic_sim* s, int k, cudaStream_t st) {
    const SpeciesDev& sp = s->sp[k];
    if (sp.n == 0) return PIC_OK;
    int grid = grid_for(sp.n, 256);
    if (s->cfg.precision == 64)
        sanitize_kernel<double><<<grid, 256, 0, st>>>(sp.cell, (double*)sp.off[0], (double*)sp.off[1],
                                                      (double*)sp.off[2], sp.n, s->d.N, s->status);
    else
        sanitize_kernel<float><<<grid, 256, 0, st>>>(sp.cell, (float*)sp.off[0], (float*)sp.off[1],
                                                     (float*)sp.off[2], sp.n, s->d.N, s->status);
    GP_CUDA(cudaGetLastError());
    return PIC_OK;
}

int launch_sort(pic_sim* s, cudaStream_t st) {
    return s->cfg.precision == 64 ? sort_typed<double>(s, st) : sort_typed<float>(s, st);
}

int launch_generate(pic_sim* s, int k, const pic_species* spec, cudaStream_t st) {
    const SpeciesDev& sp = s->sp[k];
    uint64_t key = spec->seed ^ ((uint64_t)spec->species_id << 56);
    int grid = grid_for(sp.n, 256);
    if (s->cfg.precision == 64)
        generate_kernel<double><<<grid, 256, 0, st>>>(
            sp.cell, (double*)sp.off[0], (double*)sp.off[1], (double*)sp.off[2], (double*)sp.u[0],
            (double*)sp.u[1], (double*)sp.u[2], sp.n, s->d.nx, s->d.ny, s->d.nz, spec->ppc[0],
            spec->ppc[1], spec->ppc[2], spec->jitter, key, spec->u0[0], spec->u0[1], spec->u0[2]);
    else
        generate_kernel<float><<<grid, 256, 0, st>>>(
            sp.cell, (float*)sp.off[0], (float*)sp.off[1], (float*)sp.off[2], (float*)sp.u[0],
            (float*)sp.u[1], (float*)sp.u[2], sp.n, s->d.nx, s->d.ny, s->d.nz, spec->ppc[0],
            spec->ppc[1], spec->ppc[2], spec->jitter, key, spec->u0[0], spec->u0[1], spec->u0[2]);
    GP_CUDA(cudaGetLastError());
    return PIC_OK;
}

}  // namespace galpic
