// The particle pass of the Galilean-PSATD step (templates; instantiated by
// pass_fp32.cu and pass_fp64.cu, one translation unit per precision so that they
// compile in parallel). One CTA per bin: the bin's E, B tile (plus stencil halo and
// a margin) is staged in shared memory as component pairs; each particle gathers E
// and B with packed FP32x2 FMAs, takes the relativistic Boris push and the Galilean
// drift in two halves, and deposits J^{n+1/2} and rho^{n+1}. The deposit is reduced
// inside the warp first (grouped by cell, or by stencil row for few particles per
// cell), then added to the shared tile, and the tile to the global grids once per
// CTA. Particles whose stencil leaves the tile use global memory directly.
#pragma once

#include <math.h>
#include <string.h>

#include "common.cuh"

namespace galpic {

namespace {

constexpr int PASS_THREADS = 256;
constexpr int PASS_WARPS = PASS_THREADS / 32;

__device__ __forceinline__ int wrapi(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

// Periodic wrap for an index that is at most one period outside [0, n) (the
// common case); anything further goes through the modulo.
__device__ __forceinline__ int wrap_near(int i, int n) {
    if (i < 0)
        i += n;
    else if (i >= n)
        i -= n;
    return (i >= 0 && i < n) ? i : wrapi(i, n);
}

// Periodic wrap on the out-of-tile paths: the near form for 4x4x4 stencils; the
// modulo for 2x2x2 ones, whose kernels then fit their register budget without spills.
template <int NW>
__device__ __forceinline__ int wrapf(int i, int n) { return NW == 2 ? wrapi(i, n) : wrap_near(i, n); }

// Division of a non-negative int32 by a fixed divisor d >= 1 with one 64-bit
// multiply and a shift: q = (x * M) >> s with s = 31 + ceil(log2 d) and
// M = ceil(2^s / d) < 2^32. For x < 2^31 the rounding error of M adds less than
// x/2^s < 2^-ceil(log2 d) <= 1/d to x/d, which never carries past the next integer.
struct FastDiv {
    uint32_t d, M;
    int s;
    __host__ void init(uint32_t dd) {
        d = dd;
        int L = 0;
        while ((1ull << L) < dd) ++L;
        s = 31 + L;
        M = (uint32_t)(((1ull << s) + dd - 1) / dd);
    }
    __device__ __forceinline__ int div(int x) const {
        return (int)(((unsigned long long)(unsigned)x * M) >> s);
    }
};

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

// Packed pair FMA: d = a * b + c per component. FP32 uses the paired FP32 FMA of
// sm_100-class GPUs (one instruction for two IEEE round-to-nearest FMAs).
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) {
    unsigned long long ra = *reinterpret_cast<unsigned long long*>(&a);
    unsigned long long rb = *reinterpret_cast<unsigned long long*>(&b);
    unsigned long long rc = *reinterpret_cast<unsigned long long*>(&c);
    unsigned long long rd;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(rd) : "l"(ra), "l"(rb), "l"(rc));
    return *reinterpret_cast<float2*>(&rd);
}
__device__ __forceinline__ double2 pfma(double2 a, double2 b, double2 c) {
    return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ float2 pmul(float2 a, float2 b) {
    unsigned long long ra = *reinterpret_cast<unsigned long long*>(&a);
    unsigned long long rb = *reinterpret_cast<unsigned long long*>(&b);
    unsigned long long rd;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    return *reinterpret_cast<float2*>(&rd);
}
__device__ __forceinline__ double2 pmul(double2 a, double2 b) {
    return make_double2(a.x * b.x, a.y * b.y);
}

// 1/sqrt(x) and a/b of the Boris push: FP32 runs take the hardware reciprocal square root
// and the fast division (CUDA's rsqrtf and __fdividef, within 2 ulp, against a 1e-5 FP32
// step tolerance) instead of the correctly rounded sequences with their special-case
// branches; FP64 runs keep the correctly rounded forms.
__device__ __forceinline__ float boris_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double boris_rsqrt(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float boris_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double boris_div(double a, double b) { return a / b; }

// Relativistic Boris push u^{n-1/2} -> u^{n+1/2} of momentum per mass u with a = q dt / 2m.
template <typename T>
__device__ __forceinline__ void boris_push(const T a, const T* E, const T* B, const T inv_c2, T& ux, T& uy, T& uz) {
    const T umx = ux + a * E[0], umy = uy + a * E[1], umz = uz + a * E[2];
    const T igm = boris_rsqrt((T)1 + (umx * umx + umy * umy + umz * umz) * inv_c2);
    const T tx = a * B[0] * igm, ty = a * B[1] * igm, tz = a * B[2] * igm;
    const T s2 = boris_div((T)2, (T)1 + tx * tx + ty * ty + tz * tz);
    const T sx = s2 * tx, sy = s2 * ty, sz = s2 * tz;
    const T upx = umx + (umy * tz - umz * ty);
    const T upy = umy + (umz * tx - umx * tz);
    const T upz = umz + (umx * ty - umy * tx);
    ux = umx + (upy * sz - upz * sy) + a * E[0];
    uy = umy + (upz * sx - upx * sz) + a * E[1];
    uz = umz + (upx * sy - upy * sx) + a * E[2];
}

template <typename T> struct Pair;
template <> struct Pair<float> {
    typedef float2 type;
    __device__ static float2 make(float a, float b) { return make_float2(a, b); }
};
template <> struct Pair<double> {
    typedef double2 type;
    __device__ static double2 make(double a, double b) { return make_double2(a, b); }
};

// E, B tile in shared memory as three component pairs per node:
// P0 = (Ex, Ey), P1 = (Ez, Bx), P2 = (By, Bz).
// float: one float4 (P0, P1) and one float2 (P2) per node; double: three double2.
template <typename T> struct FieldTile;
template <> struct FieldTile<float> {
    float4* q;
    float2* r;
    __device__ void init(unsigned char* base, int R) {
        q = reinterpret_cast<float4*>(base);
        r = reinterpret_cast<float2*>(base + 16 * (size_t)R);
    }
    __device__ void store(int idx, const float* v) {
        q[idx] = make_float4(v[0], v[1], v[2], v[3]);
        r[idx] = make_float2(v[4], v[5]);
    }
    __device__ void load(int idx, float2& p0, float2& p1, float2& p2) const {
        float4 a = q[idx];
        p0 = make_float2(a.x, a.y);
        p1 = make_float2(a.z, a.w);
        p2 = r[idx];
    }
    static constexpr size_t bytes_per_node = 24;
};
template <> struct FieldTile<double> {
    double2 *a, *b, *c;
    __device__ void init(unsigned char* base, int R) {
        a = reinterpret_cast<double2*>(base);
        b = a + R;
        c = b + R;
    }
    __device__ void store(int idx, const double* v) {
        a[idx] = make_double2(v[0], v[1]);
        b[idx] = make_double2(v[2], v[3]);
        c[idx] = make_double2(v[4], v[5]);
    }
    __device__ void load(int idx, double2& p0, double2& p1, double2& p2) const {
        p0 = a[idx];
        p1 = b[idx];
        p2 = c[idx];
    }
    static constexpr size_t bytes_per_node = 48;
};

__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) / 16 * 16; }

// Per-warp staging area of the grouped deposit, transposed: one row per staged
// quantity, indexed by lane. Rows 0..2 hold the velocity (J phase), then NW rows of
// x weights wx[a], NW rows of y weights wy[b] and NW rows of z weights wz[c].
// A group of lanes that share a stencil is summed two members at a time: the values
// of lanes m and m+1 of one row are one aligned pair, loaded in one instruction and
// fed to the packed FP32x2 multiply/FMA. The row stride RS = 34 elements keeps pairs
// aligned and puts consecutive rows two banks apart, so the up-to-16 distinct rows a
// warp reads at one lane index hit distinct banks; a lane's stores to its own column
// are contiguous across the warp.
// Linear stencils (NW = 2) add a flag row and rows of the x^{n+1} (rho) weights for
// the combined J and rho deposit.
template <typename T, int NW> struct Stage {
    static constexpr int RS = 34;
    T* base;
    __device__ T* row(int r) const { return base + r * RS; }
    __device__ T* vrow(int q) const { return row(q); }
    __device__ T* xrow(int a) const { return row(3 + a); }
    __device__ T* yrow(int b) const { return row(3 + NW + b); }
    __device__ T* zrow(int c) const { return row(3 + 2 * NW + c); }
    __device__ T* frow() const { return row(3 + 3 * NW); }
    __device__ T* xRrow(int a) const { return row(4 + 3 * NW + a); }
    __device__ T* yRrow(int b) const { return row(4 + 4 * NW + b); }
    __device__ T* zRrow(int c) const { return row(4 + 5 * NW + c); }
};

// Per-warp staging area of the row deposit (FP32, quadratic/cubic): one block of 52
// floats per lane (member) m at m * 52, in two halves h = 0 (the lanes that own Jx,
// Jy) and h = 1 (Jz, rho), each of pairs ready for the packed multiply/FMA:
//   XV[h][a]: h = 0 (wxJ[a] qw vx, wxJ[a] qw vy), h = 1 (wxJ[a] qw vz, wxR[a] qw);
//   Y[h][b]:  h = 0 (wyJ[b], wyJ[b]),             h = 1 (wyJ[b], wyR[b]);
//   Z[h][c]:  h = 0 (wzJ[c], wzJ[c]),             h = 1 (wzJ[c], wzR[c]);
// J is the stencil at x^{n+1/2}, R the one at x^{n+1}. The 208-byte stride puts
// the eight lanes of a quarter-warp 16-byte store on distinct banks.
struct RowStage {
    static constexpr int MEMBER = 52;
    static constexpr int XV = 0, Y = 16, Z = 32;
    static constexpr size_t BYTES = 32 * MEMBER * sizeof(float);
};

// Deposit strategies: grouped by cell, J and rho in separate group passes (all
// passes; linear passes always combine them), by stencil row (FP32, NW = 4), grouped
// by cell with J and rho in one group pass (FP32, NW = 4), or grouped by cell in 64-bit
// fixed point (deterministic mode, all shapes and precisions).
enum { DEP_GROUP = 0, DEP_ROW = 1, DEP_JR = 2, DEP_ROWU = 3, DEP_CELL = 4, DEP_FIXED = 8 };

// Rows of the grouped staging area: velocity, x, y, z weights; the combined J and rho
// pass adds a flag row and the x^{n+1} weights.
__host__ __device__ constexpr int stage_rows(int NW, bool jr) { return jr ? 4 + 6 * NW : 3 + 3 * NW; }

// Per-warp particle staging of the one-thread-per-cell pass: CELL_CHUNK particles of one
// species (cell, three offsets, three momenta), loaded and stored coalesced. A warp's 32
// cells hold 256 particles of a species at 8 per cell, which one chunk then covers, so
// that every lane has its cell's particles in the same chunk. Entry j sits at slot
// j + j/32 of each array: lanes then read their cells' particles (strides of a few
// entries, 8 for the bench plasma) from distinct banks instead of 8-way conflicts.
constexpr int CELL_CHUNK = 256;
constexpr int CELL_STRIDE = CELL_CHUNK + CELL_CHUNK / 32;
__host__ __device__ __forceinline__ int cell_slot(int j) { return j + (j >> 5); }

// Asynchronous copy of one 4- or 8-byte element from global to shared memory (cp.async):
// the data goes to shared memory without passing through registers, so a lane can have
// all of its chunk's loads in flight at once. async_wait_all waits for the calling
// thread's copies; a __syncwarp after it publishes them to the warp.
template <int BYTES>
__device__ __forceinline__ void async_copy(void* dst_smem, const void* src) {
    static_assert(BYTES == 4 || BYTES == 8, "cp.async.ca copies 4, 8 or 16 bytes");
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__host__ __device__ constexpr size_t stage_bytes(int NW, size_t T, int dep) {
    return dep == DEP_CELL ? align16((size_t)CELL_STRIDE * (4 + 6 * T))
           : (T == 4 && NW == 4 && (dep == DEP_ROW || dep == DEP_ROWU))
               ? RowStage::BYTES
               : align16((size_t)stage_rows(NW, NW == 2 || dep == DEP_JR) * 34 * T);
}

// Shared-memory layout of one particle-pass CTA (bytes), shared with the host.
struct PassSmem {
    size_t tile, dep, stage, total;
    __host__ __device__ PassSmem(int R, int NW, size_t T, bool step, int strategy) {
        size_t tb = step ? (T == 4 ? FieldTile<float>::bytes_per_node : FieldTile<double>::bytes_per_node) : 0;
        tile = 0;
        dep = align16(tb * (size_t)R);
        // the deposit tile holds four components per node, 64-bit integers in fixed point
        stage = align16(dep + 4 * (size_t)R * (strategy == DEP_FIXED ? 8 : T));
        total = align16(stage + (size_t)PASS_WARPS * stage_bytes(NW, T, strategy));
    }
};

// Bins are BIN^3 cells; the shared tile of a bin covers its cells' stencils plus
// MARGIN cells on every side, so particles that moved up to MARGIN cells out of
// their bin since the last sort still use the tile.
constexpr int BIN = 8;
template <int NW, int MARGIN> struct TileGeom {
    static constexpr int E = BIN + NW - 1 + 2 * MARGIN;   // tile extent per axis (nodes)
    static constexpr int R = E * E * E;
};

template <typename T>
struct SpeciesK {
    int32_t* cell;
    T* off[3];
    T* u[3];
    const int32_t* bin_start;
    const int32_t* cell_start;   // first particle of each cell key (bin-major) as of the last sort
    int32_t n;   // particles of the species (the checked build tests indices against it)
    T qw_dv;   // q w / dV
    T qdt2m;   // q dt / (2 m)
};

template <typename T>
struct PassK {
    const T* F;     // real E (3N) then B (3N)
    T* S;           // real Jx, Jy, Jz, rho (4N)
    long long* S64;   // deterministic mode: the same sources in fixed point (units of delta)
    T inv_delta;      // deterministic mode: 1/delta = 2^-e, a power of two
    int64_t N;
    int nx, ny, nz;
    FastDiv div_nynz, div_nz;
    int nbx, nby, nbz;
    T inv_c2;
    T hd[3];             // dt / (2 d) per axis
    T vgal[3];
    int nspecies;
    SpeciesK<T> sp[PIC_MAX_SPECIES];
    unsigned long long* cnt;
    int32_t* status;   // device status word (checked build: PIC_STATUS_BOUNDS)
    int inject;        // checked build only: tile-index offset of the checker's own test
};

// Move (i, f) by d cells along an axis of n cells: offset back to [0, 1), periodic.
// Returns the cell shift (before the periodic wrap).
template <typename T>
__device__ __forceinline__ int drift_axis(int& i, T& f, T d, int n) {
    f += d;
    T s = floor(f);
    f -= s;
    int si = (int)s;
    if (f >= (T)1) {
        f -= (T)1;
        si += 1;
    }
    i = wrap_near(i + si, n);
    return si;
}

// Tile coordinates: tile node t holds global node (o + t) mod n with
// o = bin origin + J0 - margin, so the stencil of a particle in cell i starts at tile
// index r = i - bin origin + margin; the pass tracks r through the drifts without
// wrapping it (r + shift stays congruent to the new cell's index modulo n). The
// stencil lies in the tile iff 0 <= r <= extent - NW; otherwise the particle takes
// the global-memory path.
template <int NW, int TE>
__device__ __forceinline__ bool in_tile(int r) {
    return (unsigned)r <= (unsigned)(TE - NW);
}

// Element i of a small register array without dynamic indexing (the array stays in
// registers).
template <typename T, int NW>
__device__ __forceinline__ T pick(const T* w, int i) {
    T r = w[0];
#pragma unroll
    for (int k = 1; k < NW; ++k) r = (i == k) ? w[k] : r;
    return r;
}

// Direct deposit of Q values at one particle's stencil into the global grids
// (particles outside the tile, a rare path). For 4x4x4 stencils a rolled loop over
// the nodes keeps it from holding registers the in-tile path needs; 2x2x2 stencils
// are unrolled.
template <typename T, int NW, int J0>
__device__ void deposit_global(const PassK<T>& p, int ix, int iy, int iz, const T* wx, const T* wy,
                               const T* wz, int q0, int Q, const T* val) {
    if constexpr (NW == 2) {
#pragma unroll
        for (int a = 0; a < NW; ++a)
#pragma unroll
            for (int b = 0; b < NW; ++b) {
                const T wxy = wx[a] * wy[b];
                const int64_t base =
                    ((int64_t)wrapi(ix + J0 + a, p.nx) * p.ny + wrapi(iy + J0 + b, p.ny)) * p.nz;
#pragma unroll
                for (int c = 0; c < NW; ++c) {
                    const T w = wxy * wz[c];
                    const int64_t g = base + wrapi(iz + J0 + c, p.nz);
                    if (!PIC_INDEX_OK(g, p.N, p.status)) continue;
                    for (int q = 0; q < Q; ++q) atomicAdd(&p.S[(q0 + q) * p.N + g], w * val[q]);
                }
            }
        return;
    }
    const T v0 = val[0], v1 = Q > 1 ? val[1] : (T)0, v2 = Q > 2 ? val[2] : (T)0;
#pragma unroll 1
    for (int n = 0; n < NW * NW * NW; ++n) {
        const int a = n / (NW * NW), b = (n / NW) % NW, c = n % NW;
        const T w = pick<T, NW>(wx, a) * pick<T, NW>(wy, b) * pick<T, NW>(wz, c);
        const int64_t g = ((int64_t)wrap_near(ix + J0 + a, p.nx) * p.ny + wrap_near(iy + J0 + b, p.ny)) * p.nz +
                          wrap_near(iz + J0 + c, p.nz);
        if (!PIC_INDEX_OK(g, p.N, p.status)) continue;
        T* dst = p.S + q0 * p.N + g;
        atomicAdd(dst, w * v0);
        if (Q > 1) {
            atomicAdd(dst + p.N, w * v1);
            atomicAdd(dst + 2 * p.N, w * v2);
        }
    }
}

// Adds K values to K distinct shared-memory words. Shared-memory floating-point
// atomics are compare-and-swap loops on this GPU; issuing all K reads, then all K
// compare-and-swaps, and retrying only the ones that lost a race keeps K round trips
// in flight at once instead of K dependent ones.
__device__ __forceinline__ unsigned as_bits(float x) { return __float_as_uint(x); }
__device__ __forceinline__ unsigned long long as_bits(double x) { return (unsigned long long)__double_as_longlong(x); }
__device__ __forceinline__ float from_bits(unsigned x) { return __uint_as_float(x); }
__device__ __forceinline__ double from_bits(unsigned long long x) { return __longlong_as_double((long long)x); }

template <typename T, int K>
__device__ __forceinline__ void smem_add_batch(T* const (&addr)[K], const T (&val)[K]) {
    typedef decltype(as_bits((T)0)) U;
    U old[K];
    bool done[K];
#pragma unroll
    for (int k = 0; k < K; ++k) old[k] = as_bits(*reinterpret_cast<volatile T*>(addr[k]));
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const U prev = atomicCAS(reinterpret_cast<U*>(addr[k]), old[k], as_bits(from_bits(old[k]) + val[k]));
        done[k] = prev == old[k];
        old[k] = prev;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        while (!done[k]) {   // lost a race with another warp: retry (lock-free, always progresses)
            const U prev = atomicCAS(reinterpret_cast<U*>(addr[k]), old[k], as_bits(from_bits(old[k]) + val[k]));
            done[k] = prev == old[k];
            old[k] = prev;
        }
    }
}

// ---- deterministic mode: 64-bit fixed point ---------------------------------
// A deposited value x (already multiplied by 1/delta) becomes the integer nearest to
// it; integer additions are associative, so the sums below do not depend on the
// order of members, groups, warps or CTAs. The weight product is formed in one order,
// wx * (wy * wz) * value, on the tile path and on the out-of-tile path alike, so a
// particle contributes the same integers whichever path it takes.
template <typename T> __device__ __forceinline__ long long to_fixed(T x);
template <> __device__ __forceinline__ long long to_fixed<float>(float x) { return __float2ll_rn(x); }
template <> __device__ __forceinline__ long long to_fixed<double>(double x) { return __double2ll_rn(x); }

template <typename T>
__device__ __forceinline__ long long fixed_contrib(T wx, T wy, T wz, T v) {
    return to_fixed<T>(wx * (wy * wz) * v);
}

__device__ __forceinline__ void add_fixed(long long* p, long long v) {
    atomicAdd(reinterpret_cast<unsigned long long*>(p), (unsigned long long)v);
}

// Out-of-tile deposit in fixed point: Q values (already scaled by q w/(dV delta)) at
// one particle's stencil, straight into the global integer grids.
template <typename T, int NW, int J0>
__device__ void deposit_global_fixed(const PassK<T>& p, int ix, int iy, int iz, const T* wx, const T* wy,
                                     const T* wz, int q0, int Q, const T* val) {
#pragma unroll 1
    for (int n = 0; n < NW * NW * NW; ++n) {
        const int a = n / (NW * NW), b = (n / NW) % NW, c = n % NW;
        const T xa = pick<T, NW>(wx, a), yb = pick<T, NW>(wy, b), zc = pick<T, NW>(wz, c);
        const int64_t g = ((int64_t)wrapi(ix + J0 + a, p.nx) * p.ny + wrapi(iy + J0 + b, p.ny)) * p.nz +
                          wrapi(iz + J0 + c, p.nz);
        if (!PIC_INDEX_OK(g, p.N, p.status)) continue;
        for (int q = 0; q < Q; ++q) {
            const long long v = fixed_contrib<T>(xa, yb, zc, val[q]);
            if (v) add_fixed(p.S64 + (int64_t)(q0 + q) * p.N + g, v);
        }
    }
}

template <typename T>
__device__ __forceinline__ typename Pair<T>::type ld2(const T* p) {
    return *reinterpret_cast<const typename Pair<T>::type*>(p);
}

// Grouped deposit of one warp. `member`: this lane staged its weights (and, for J,
// its velocity) and its stencil starts at tile node `key` (tile linear index).
// Q = 3 (J, components q0 = 0..2) or 1 (rho, q0 = 3); every deposited value is
// qw * (weight product) * (velocity component or 1). For each group of lanes with
// one key, the lanes take (node, component) roles, sum over the group's members
// (two at a time when the group is a contiguous run of lanes, the normal case for
// cell-sorted particles) and add each role's sum to the shared tile once.
// Every lane of the warp must call this (warp-collective).
// PREMUL: the members' staged values already carry their charge factor (the J rows
// hold q w v / dV, and for rho, row 0 holds q w / dV), so members of different
// species can share a group; qw is then 1.
template <typename T, int NW, int Q, int TE, bool PREMUL = false>
__device__ void group_deposit(T* sD, const Stage<T, NW>& stg, bool member, int key, int lane, T qw) {
    typedef typename Pair<T>::type P2;
    constexpr int q0 = (Q == 3) ? 0 : 3;
    constexpr int R = TE * TE * TE;
    const P2 one = Pair<T>::make((T)1, (T)1);
    const P2 zero = Pair<T>::make((T)0, (T)0);
    unsigned pending = __ballot_sync(0xffffffffu, member);
    while (pending) {
        const int leader = __ffs(pending) - 1;
        const int gkey = __shfl_sync(0xffffffffu, key, leader);
        const unsigned grp = __ballot_sync(0xffffffffu, member && key == gkey);
        pending &= ~grp;
        const int lo = __ffs(grp) - 1;
        const int len = __popc(grp);
        const bool run = (grp >> lo) == (len == 32 ? 0xffffffffu : ((1u << len) - 1u));   // warp-uniform
        if (NW == 4) {
            // lane -> y-z node (b, c) = (bc >> 2, bc & 3), bc = lane & 15, and x nodes h, h + 2
            const int bc = lane & 15, h = lane >> 4, b = bc >> 2, c = bc & 3;
            const T* xh = stg.xrow(h);
            const T* xh2 = stg.xrow(h + 2);
            const T* yb = stg.yrow(b);
            const T* zc = stg.zrow(c);
            P2 A[Q], A2[Q];   // (even, odd member) partial sums for x nodes h and h + 2
#pragma unroll
            for (int q = 0; q < Q; ++q) A[q] = A2[q] = zero;
            auto single = [&](int m) {
                const T wyz = yb[m] * zc[m];
                const T w0 = xh[m] * wyz, w1 = xh2[m] * wyz;
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const T v = (Q == 3) ? stg.vrow(q)[m] : (PREMUL ? stg.vrow(0)[m] : (T)1);
                    A[q].x = fma(w0, v, A[q].x);
                    A2[q].x = fma(w1, v, A2[q].x);
                }
            };
            auto pair = [&](int m) {
                const P2 wyz = pmul(ld2(yb + m), ld2(zc + m));
                const P2 w0 = pmul(ld2(xh + m), wyz);
                const P2 w1 = pmul(ld2(xh2 + m), wyz);
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const P2 v = (Q == 3) ? ld2(stg.vrow(q) + m) : (PREMUL ? ld2(stg.vrow(0) + m) : one);
                    A[q] = pfma(w0, v, A[q]);
                    A2[q] = pfma(w1, v, A2[q]);
                }
            };
            if (run) {
                int m = lo;
                const int me = lo + len;
                if (m & 1) single(m++);
                for (; m + 1 < me; m += 2) pair(m);
                if (m < me) single(m);
            } else {
                // several runs of consecutive lanes (e.g. one cell's particles of two
                // species in the two half-warps): pairs within each run
                unsigned g = grp;
                while (g) {
                    const int r0 = __ffs(g) - 1;
                    const unsigned inv = ~(g >> r0);
                    const int rl = inv ? __ffs(inv) - 1 : 32 - r0;
                    int m = r0;
                    const int me = r0 + rl;
                    if (m & 1) single(m++);
                    for (; m + 1 < me; m += 2) pair(m);
                    if (m < me) single(m);
                    g &= rl == 32 ? 0u : ~(((1u << rl) - 1u) << r0);
                }
            }
            const int n0 = gkey + (h * TE + b) * TE + c;
            const int n1 = n0 + 2 * TE * TE;
            T* addr[2 * Q];
            T val[2 * Q];
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                addr[2 * q] = &sD[(q0 + q) * R + n0];
                addr[2 * q + 1] = &sD[(q0 + q) * R + n1];
                val[2 * q] = (A[q].x + A[q].y) * qw;
                val[2 * q + 1] = (A2[q].x + A2[q].y) * qw;
            }
            smem_add_batch<T, 2 * Q>(addr, val);
        } else {
            // NW == 2: lane -> (component q = lane / 8, node j = lane % 8)
            if (lane < 8 * Q) {
                const int q = lane >> 3, j = lane & 7;
                const int ax = j >> 2, by = (j >> 1) & 1, cz = j & 1;
                const T* xa = stg.xrow(ax);
                const T* yb = stg.yrow(by);
                const T* zc = stg.zrow(cz);
                const T* vq = stg.vrow(Q == 3 ? q : 0);
                P2 A = zero;
                if (run) {
                    int m = lo;
                    const int me = lo + len;
                    if (m & 1) {
                        A.x = fma(xa[m] * yb[m] * zc[m], (Q == 3) ? vq[m] : (T)1, A.x);
                        ++m;
                    }
                    for (; m + 1 < me; m += 2) {
                        const P2 w = pmul(pmul(ld2(xa + m), ld2(yb + m)), ld2(zc + m));
                        A = pfma(w, (Q == 3) ? ld2(vq + m) : one, A);
                    }
                    if (m < me) A.x = fma(xa[m] * yb[m] * zc[m], (Q == 3) ? vq[m] : (T)1, A.x);
                } else {
                    unsigned g = grp;
                    while (g) {
                        const int m = __ffs(g) - 1;
                        g &= g - 1;
                        A.x = fma(xa[m] * yb[m] * zc[m], (Q == 3) ? vq[m] : (T)1, A.x);
                    }
                }
                T* addr[1] = {&sD[(q0 + q) * R + gkey + (ax * TE + by) * TE + cz]};
                const T val[1] = {(A.x + A.y) * qw};
                smem_add_batch<T, 1>(addr, val);
            }
        }
    }
}

// Grouped deposit of one warp in fixed point (deterministic mode), for every shape and
// precision. Roles as in group_deposit; the staged value rows hold the members' values
// already multiplied by q w/(dV delta) (J: rows 0..2 = that times v; rho: row 0). Each
// member's contribution is rounded to an integer before it is summed, and each role's
// integer sum is added to the integer tile. Every lane of the warp must call this.
template <typename T, int NW, int Q, int TE>
__device__ void group_deposit_fixed(long long* sD, const Stage<T, NW>& stg, bool member, int key, int lane) {
    constexpr int q0 = (Q == 3) ? 0 : 3;
    constexpr int R = TE * TE * TE;
    unsigned pending = __ballot_sync(0xffffffffu, member);
    while (pending) {
        const int leader = __ffs(pending) - 1;
        const int gkey = __shfl_sync(0xffffffffu, key, leader);
        const unsigned grp = __ballot_sync(0xffffffffu, member && key == gkey);
        pending &= ~grp;
        if (NW == 4) {
            // lane -> y-z node (b, c) = (bc >> 2, bc & 3), bc = lane & 15, and x nodes h, h + 2
            const int bc = lane & 15, h = lane >> 4, b = bc >> 2, c = bc & 3;
            const T* xh = stg.xrow(h);
            const T* xh2 = stg.xrow(h + 2);
            const T* yb = stg.yrow(b);
            const T* zc = stg.zrow(c);
            long long A[Q], A2[Q];
#pragma unroll
            for (int q = 0; q < Q; ++q) A[q] = A2[q] = 0;
            unsigned g = grp;
            while (g) {
                const int m = __ffs(g) - 1;
                g &= g - 1;
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const T v = stg.vrow(Q == 3 ? q : 0)[m];
                    A[q] += fixed_contrib<T>(xh[m], yb[m], zc[m], v);
                    A2[q] += fixed_contrib<T>(xh2[m], yb[m], zc[m], v);
                }
            }
            const int n0 = gkey + (h * TE + b) * TE + c;
            const int n1 = n0 + 2 * TE * TE;
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                if (A[q]) add_fixed(&sD[(q0 + q) * R + n0], A[q]);
                if (A2[q]) add_fixed(&sD[(q0 + q) * R + n1], A2[q]);
            }
        } else {
            // NW == 2: lane -> (component q = lane / 8, node j = lane % 8)
            if (lane < 8 * Q) {
                const int q = lane >> 3, j = lane & 7;
                const int ax = j >> 2, by = (j >> 1) & 1, cz = j & 1;
                const T* xa = stg.xrow(ax);
                const T* yb = stg.yrow(by);
                const T* zc = stg.zrow(cz);
                const T* vq = stg.vrow(Q == 3 ? q : 0);
                long long A = 0;
                unsigned g = grp;
                while (g) {
                    const int m = __ffs(g) - 1;
                    g &= g - 1;
                    A += fixed_contrib<T>(xa[m], yb[m], zc[m], vq[m]);
                }
                if (A) add_fixed(&sD[(q0 + q) * R + gkey + (ax * TE + by) * TE + cz], A);
            }
        }
    }
}

// Combined J and rho deposit of one warp for linear stencils (NW = 2). Members are
// grouped by the start `key` of their J stencil; lane q * 8 + j takes component q
// (Jx, Jy, Jz, rho) at node j = (a, b, c) of the 2x2x2 stencil, so every lane works
// on every group. The rho lanes read the x^{n+1} weights and, as the value, the
// member's flag: 1 when its rho stencil starts at its J stencil's node (the normal
// case), 0 otherwise (that member's rho goes through a separate rho-only pass).
// Every lane of the warp must call this (warp-collective).
template <typename T, int TE>
__device__ void group_deposit_jr(T* sD, const Stage<T, 2>& stg, bool member, int key, int lane, T qw) {
    typedef typename Pair<T>::type P2;
    constexpr int R = TE * TE * TE;
    const int q = lane >> 3, j = lane & 7;
    const int ax = j >> 2, by = (j >> 1) & 1, cz = j & 1;
    const bool rho = q == 3;
    const T* xa = rho ? stg.xRrow(ax) : stg.xrow(ax);
    const T* yb = rho ? stg.yRrow(by) : stg.yrow(by);
    const T* zc = rho ? stg.zRrow(cz) : stg.zrow(cz);
    const T* vq = rho ? stg.frow() : stg.vrow(q);
    T* const dst = sD + q * R + (ax * TE + by) * TE + cz;
    unsigned pending = __ballot_sync(0xffffffffu, member);
    while (pending) {
        const int leader = __ffs(pending) - 1;
        const int gkey = __shfl_sync(0xffffffffu, key, leader);
        const unsigned grp = __ballot_sync(0xffffffffu, member && key == gkey);
        pending &= ~grp;
        const int lo = __ffs(grp) - 1;
        const int len = __popc(grp);
        const bool run = (grp >> lo) == (len == 32 ? 0xffffffffu : ((1u << len) - 1u));   // warp-uniform
        P2 A = Pair<T>::make((T)0, (T)0);
        if (run) {
            int m = lo;
            const int me = lo + len;
            if (m & 1) {
                A.x = fma(xa[m] * yb[m] * zc[m], vq[m], A.x);
                ++m;
            }
            for (; m + 1 < me; m += 2) {
                const P2 w = pmul(pmul(ld2(xa + m), ld2(yb + m)), ld2(zc + m));
                A = pfma(w, ld2(vq + m), A);
            }
            if (m < me) A.x = fma(xa[m] * yb[m] * zc[m], vq[m], A.x);
        } else {
            unsigned g = grp;
            while (g) {
                const int m = __ffs(g) - 1;
                g &= g - 1;
                A.x = fma(xa[m] * yb[m] * zc[m], vq[m], A.x);
            }
        }
        T* addr[1] = {dst + gkey};
        const T val[1] = {(A.x + A.y) * qw};
        smem_add_batch<T, 1>(addr, val);
    }
}

// Combined J and rho deposit of one warp for 4x4x4 stencils (strategy DEP_JR). Members
// are grouped by the start `key` of their J stencil; lane (b, c, h) = ((lane & 15) >> 2,
// lane & 3, lane >> 4) sums the y-z node (b, c) at x nodes h and h + 2 for Jx, Jy, Jz
// (x^{n+1/2} weights, velocity rows) and rho (x^{n+1} weights, flag row: the member's
// value when its rho stencil starts at its J stencil's node, 0 otherwise; those members'
// rho goes through a rho-only pass). One group loop and one batch of eight
// compare-and-swaps serve both. PREMUL as for group_deposit.
// Every lane of the warp must call this (warp-collective).
template <typename T, int TE>
__device__ void group_deposit_jr4(T* sD, const Stage<T, 4>& stg, bool member, int key, int lane, T qw) {
    typedef typename Pair<T>::type P2;
    constexpr int R = TE * TE * TE;
    const P2 zero = Pair<T>::make((T)0, (T)0);
    const int bc = lane & 15, h = lane >> 4, b = bc >> 2, c = bc & 3;
    const T* xh = stg.xrow(h);
    const T* xh2 = stg.xrow(h + 2);
    const T* yb = stg.yrow(b);
    const T* zc = stg.zrow(c);
    const T* xRh = stg.xRrow(h);
    const T* xRh2 = stg.xRrow(h + 2);
    const T* yRb = stg.yRrow(b);
    const T* zRc = stg.zRrow(c);
    const T* fr = stg.frow();
    unsigned pending = __ballot_sync(0xffffffffu, member);
    while (pending) {
        const int leader = __ffs(pending) - 1;
        const int gkey = __shfl_sync(0xffffffffu, key, leader);
        const unsigned grp = __ballot_sync(0xffffffffu, member && key == gkey);
        pending &= ~grp;
        P2 A[3], A2[3], Rr = zero, Rr2 = zero;
#pragma unroll
        for (int q = 0; q < 3; ++q) A[q] = A2[q] = zero;
        auto single = [&](int m) {
            const T wyz = yb[m] * zc[m];
            const T w0 = xh[m] * wyz, w1 = xh2[m] * wyz;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const T v = stg.vrow(q)[m];
                A[q].x = fma(w0, v, A[q].x);
                A2[q].x = fma(w1, v, A2[q].x);
            }
            const T rz = yRb[m] * zRc[m] * fr[m];
            Rr.x = fma(xRh[m], rz, Rr.x);
            Rr2.x = fma(xRh2[m], rz, Rr2.x);
        };
        auto pair = [&](int m) {
            const P2 wyz = pmul(ld2(yb + m), ld2(zc + m));
            const P2 w0 = pmul(ld2(xh + m), wyz);
            const P2 w1 = pmul(ld2(xh2 + m), wyz);
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const P2 v = ld2(stg.vrow(q) + m);
                A[q] = pfma(w0, v, A[q]);
                A2[q] = pfma(w1, v, A2[q]);
            }
            const P2 rz = pmul(pmul(ld2(yRb + m), ld2(zRc + m)), ld2(fr + m));
            Rr = pfma(ld2(xRh + m), rz, Rr);
            Rr2 = pfma(ld2(xRh2 + m), rz, Rr2);
        };
        // runs of consecutive lanes (one per cell and species), pairs within each
        unsigned g = grp;
        while (g) {
            const int r0 = __ffs(g) - 1;
            const unsigned inv = ~(g >> r0);
            const int rl = inv ? __ffs(inv) - 1 : 32 - r0;
            int m = r0;
            const int me = r0 + rl;
            if (m & 1) single(m++);
            for (; m + 1 < me; m += 2) pair(m);
            if (m < me) single(m);
            g &= rl == 32 ? 0u : ~(((1u << rl) - 1u) << r0);
        }
        const int n0 = gkey + (h * TE + b) * TE + c;
        const int n1 = n0 + 2 * TE * TE;
        T* addr[8];
        T val[8];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            addr[2 * q] = &sD[q * R + n0];
            addr[2 * q + 1] = &sD[q * R + n1];
            val[2 * q] = (A[q].x + A[q].y) * qw;
            val[2 * q + 1] = (A2[q].x + A2[q].y) * qw;
        }
        addr[6] = &sD[3 * R + n0];
        addr[7] = &sD[3 * R + n1];
        val[6] = (Rr.x + Rr.y) * qw;
        val[7] = (Rr2.x + Rr2.y) * qw;
        smem_add_batch<T, 8>(addr, val);
    }
}

// Stage this lane's weights (and, for J, its velocity) in its column of the rows.
template <typename T, int NW>
__device__ __forceinline__ void stage_record(const Stage<T, NW>& stg, int lane, const T* wx, const T* wy,
                                             const T* wz, const T* vel) {
    if (vel) {
#pragma unroll
        for (int q = 0; q < 3; ++q) stg.vrow(q)[lane] = vel[q];
    }
#pragma unroll
    for (int a = 0; a < NW; ++a) {
        stg.xrow(a)[lane] = wx[a];
        stg.yrow(a)[lane] = wy[a];
        stg.zrow(a)[lane] = wz[a];
    }
}

// Stage this lane's block of the row deposit (see RowStage).
__device__ __forceinline__ void row_record(float* blk, const float* wxJ, const float* wyJ, const float* wzJ,
                                           const float* wxR, const float* wyR, const float* wzR,
                                           float qvx, float qvy, float qvz, float qw) {
    float4* q = reinterpret_cast<float4*>(blk);
#pragma unroll
    for (int a = 0; a < 4; a += 2) {
        q[a / 2] = make_float4(wxJ[a] * qvx, wxJ[a] * qvy, wxJ[a + 1] * qvx, wxJ[a + 1] * qvy);
        q[2 + a / 2] = make_float4(wxJ[a] * qvz, wxR[a] * qw, wxJ[a + 1] * qvz, wxR[a + 1] * qw);
        q[4 + a / 2] = make_float4(wyJ[a], wyJ[a], wyJ[a + 1], wyJ[a + 1]);
        q[6 + a / 2] = make_float4(wyJ[a], wyR[a], wyJ[a + 1], wyR[a + 1]);
        q[8 + a / 2] = make_float4(wzJ[a], wzJ[a], wzJ[a + 1], wzJ[a + 1]);
        q[10 + a / 2] = make_float4(wzJ[a], wzR[a], wzJ[a + 1], wzR[a + 1]);
    }
}

// Adds v to the float at p, whose value was `old` when read: compare-and-swap,
// retried while another warp changed it in between (shared-memory float atomics are
// compare-and-swap loops on this GPU; lock-free, always progresses).
__device__ __forceinline__ void cas_add_retry(unsigned* p, unsigned old, unsigned prev, float v) {
    while (prev != old) {
        old = prev;
        prev = atomicCAS(p, old, __float_as_uint(__uint_as_float(old) + v));
    }
}

// Row deposit of one warp (FP32, NW = 4, tile extent TE): the strategy for few
// particles per cell. Members are grouped by the (x, y) start of their stencil in
// the tile (`row` = rx * TE + ry), so the particles of a whole row of cells form
// one group. For a row, lane (h, a, b) = (lane >> 4, (lane >> 2) & 3, lane & 3)
// owns the tile nodes (rx + a, ry + b, z) for every z and two components, (Jx, Jy)
// for h = 0 and (Jz, rho) for h = 1. The row is walked along z: at stencil start j
// the members starting there add their staged x-weight-times-value pair times
// y-weight pair times z-weight pair c to a window of four packed register pairs
// (nodes j .. j + 3; one packed multiply, four packed FMAs each); node j is then
// complete and goes to the shared tile, and the window shifts by one node. The walk
// is one rolled loop, so its code is small. J (stencil at x^{n+1/2}) and rho (at
// x^{n+1}) of a particle normally start at the same node; where they do not, the
// particle joins two (row, j) groups with the other part zeroed. mJ / mR: this
// lane's J / rho stencil lies in the tile; zJ / zR: its z start. Every lane of the
// warp must call this (warp-collective).
template <int TE>
__device__ void row_deposit(float* sD, const float* stg, bool mJ, int rowJ, int zJ, bool mR, int rowR, int zR,
                            int lane) {
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int R = TE * TE * TE;
    constexpr int M = RowStage::MEMBER;
    const int h = lane >> 4, a = (lane >> 2) & 3, b = lane & 3;
    const bool hi = h != 0;
    const float* sx = stg + RowStage::XV + 8 * h + 2 * a;
    const float* sy = stg + RowStage::Y + 8 * h + 2 * b;
    const float* sz = stg + RowStage::Z + 8 * h;
    unsigned pendJ = __ballot_sync(FULL, mJ), pendR = __ballot_sync(FULL, mR);
    while (pendJ | pendR) {
        const int leader = __ffs(pendJ ? pendJ : pendR) - 1;
        const int cur = __shfl_sync(FULL, pendJ ? rowJ : rowR, leader);
        const bool inJ = mJ && rowJ == cur, inR = mR && rowR == cur;
        const unsigned gJ = __ballot_sync(FULL, inJ), gR = __ballot_sync(FULL, inR);
        pendJ &= ~gJ;
        pendR &= ~gR;
        // stencil starts present in this row, and the nodes they touch
        const unsigned zs = __reduce_or_sync(FULL, (inJ ? 1u << zJ : 0u) | (inR ? 1u << zR : 0u));
        const unsigned touched = zs | (zs << 1) | (zs << 2) | (zs << 3);
        const int jlo = __ffs(zs) - 1, jend = 31 - __clz(zs) + 3;
        const int node0 = (cur + a * TE + b) * TE;
        unsigned* const p0 = reinterpret_cast<unsigned*>(sD + (2 * h) * R + node0);
        unsigned* const p1 = reinterpret_cast<unsigned*>(sD + (2 * h + 1) * R + node0);
        float2 w0 = make_float2(0.f, 0.f), w1 = w0, w2 = w0, w3 = w0;
        auto coef = [&](int m) { return pmul(ld2(sx + m * M), ld2(sy + m * M)); };
        auto add = [&](int m, float2 c) {
            const float4 z01 = *reinterpret_cast<const float4*>(sz + m * M);
            const float4 z23 = *reinterpret_cast<const float4*>(sz + m * M + 4);
            w0 = pfma(c, make_float2(z01.x, z01.y), w0);
            w1 = pfma(c, make_float2(z01.z, z01.w), w1);
            w2 = pfma(c, make_float2(z23.x, z23.y), w2);
            w3 = pfma(c, make_float2(z23.z, z23.w), w3);
        };
#pragma unroll 1
        for (int j = jlo; j <= jend; ++j) {   // warp-uniform bounds
            const bool flush = (touched >> j) & 1u;
            unsigned o0 = 0u, o1 = 0u;
            if (flush) {   // read node j's old values before the adds, to overlap the latency
                o0 = *reinterpret_cast<volatile unsigned*>(p0 + j);
                o1 = *reinterpret_cast<volatile unsigned*>(p1 + j);
            }
            if ((zs >> j) & 1u) {
                const unsigned sJ = __ballot_sync(FULL, inJ && zJ == j);
                const unsigned sR = __ballot_sync(FULL, inR && zR == j);
                // members whose J and rho both start here, two at a time; cell-sorted
                // particles make them one run of consecutive lanes
                unsigned mm = sJ & sR;
                if (mm) {
                    const int lo = __ffs(mm) - 1, len = __popc(mm);
                    if ((mm >> lo) == (len == 32 ? FULL : ((1u << len) - 1u))) {
                        int m = lo;
                        const int me = lo + len;
                        for (; m + 1 < me; m += 2) {
                            const float2 c1 = coef(m), c2 = coef(m + 1);
                            add(m, c1);
                            add(m + 1, c2);
                        }
                        if (m < me) add(m, coef(m));
                    } else {
                        while (mm) {
                            const int m = __ffs(mm) - 1;
                            mm &= mm - 1;
                            add(m, coef(m));
                        }
                    }
                }
                // members with only one of J, rho starting here: zero the other part
                unsigned rr = (sJ | sR) & ~(sJ & sR);
                while (rr) {
                    const int k = __ffs(rr) - 1;
                    rr &= rr - 1;
                    const float fJ = ((sJ >> k) & 1u) ? 1.f : 0.f, fR = ((sR >> k) & 1u) ? 1.f : 0.f;
                    add(k, pmul(coef(k), make_float2(fJ, hi ? fR : fJ)));
                }
            }
            if (flush) {   // node j is complete: add it to the tile
                const unsigned q0 = atomicCAS(p0 + j, o0, __float_as_uint(__uint_as_float(o0) + w0.x));
                const unsigned q1 = atomicCAS(p1 + j, o1, __float_as_uint(__uint_as_float(o1) + w0.y));
                cas_add_retry(p0 + j, o0, q0, w0.x);
                cas_add_retry(p1 + j, o1, q1, w0.y);
            }
            w0 = w1;
            w1 = w2;
            w2 = w3;
            w3 = make_float2(0.f, 0.f);
        }
    }
}

// Row deposit with the z starts unrolled (FP32, NW = 4, tile extent TE): the same
// grouping and lane roles as row_deposit, but the row's nodes are register pairs
// acc[0 .. TE-1] indexed at compile time. For each stencil start j (unrolled) the
// members whose J and rho both start at (row, j) add into acc[j .. j+3]; the touched
// nodes are then added to the shared tile once each. Members whose J and rho start at
// different nodes (or only one of them in this row) add their parts straight to the
// shared tile by compare-and-swap (rare: a particle crossing a cell boundary between
// x^{n+1/2} and x^{n+1}). Every lane of the warp must call this.
template <int TE>
__device__ void row_deposit_unrolled(float* sD, const float* stg, bool mJ, int rowJ, int zJ, bool mR, int rowR,
                                     int zR, int lane) {
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int R = TE * TE * TE;
    constexpr int M = RowStage::MEMBER;
    constexpr int J = TE - 3;   // stencil starts 0 .. TE-4
    const int h = lane >> 4, a = (lane >> 2) & 3, b = lane & 3;
    const bool hi = h != 0;
    const float* sx = stg + RowStage::XV + 8 * h + 2 * a;
    const float* sy = stg + RowStage::Y + 8 * h + 2 * b;
    const float* sz = stg + RowStage::Z + 8 * h;
    unsigned pendJ = __ballot_sync(FULL, mJ), pendR = __ballot_sync(FULL, mR);
    while (pendJ | pendR) {
        const int leader = __ffs(pendJ ? pendJ : pendR) - 1;
        const int cur = __shfl_sync(FULL, pendJ ? rowJ : rowR, leader);
        const bool inJ = mJ && rowJ == cur, inR = mR && rowR == cur;
        const unsigned gJ = __ballot_sync(FULL, inJ), gR = __ballot_sync(FULL, inR);
        pendJ &= ~gJ;
        pendR &= ~gR;
        const bool both = inJ && inR && zJ == zR;
        const unsigned gB = __ballot_sync(FULL, both);
        const int node0 = (cur + a * TE + b) * TE;
        float* const p0 = sD + (2 * h) * R + node0;
        float* const p1 = sD + (2 * h + 1) * R + node0;
        float2 acc[TE];
#pragma unroll
        for (int j = 0; j < TE; ++j) acc[j] = make_float2(0.f, 0.f);
        unsigned touched = 0u;
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const unsigned mm = __ballot_sync(FULL, both && zJ == j);
            if (!mm) continue;   // warp-uniform
            touched |= 0xfu << j;
            const int lo = __ffs(mm) - 1, len = __popc(mm);
            auto add = [&](int m) {
                const float2 c = pmul(ld2(sx + m * M), ld2(sy + m * M));
                const float4 z01 = *reinterpret_cast<const float4*>(sz + m * M);
                const float4 z23 = *reinterpret_cast<const float4*>(sz + m * M + 4);
                acc[j] = pfma(c, make_float2(z01.x, z01.y), acc[j]);
                acc[j + 1] = pfma(c, make_float2(z01.z, z01.w), acc[j + 1]);
                acc[j + 2] = pfma(c, make_float2(z23.x, z23.y), acc[j + 2]);
                acc[j + 3] = pfma(c, make_float2(z23.z, z23.w), acc[j + 3]);
            };
            if ((mm >> lo) == (len == 32 ? FULL : ((1u << len) - 1u))) {   // one run of lanes
#pragma unroll 1
                for (int m = lo; m < lo + len; ++m) add(m);
            } else {
                unsigned g = mm;
#pragma unroll 1
                while (g) {
                    const int m = __ffs(g) - 1;
                    g &= g - 1;
                    add(m);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < TE; ++j) {
            if ((touched >> j) & 1u) {   // warp-uniform
                atomicAdd(p0 + j, acc[j].x);
                atomicAdd(p1 + j, acc[j].y);
            }
        }
        // members whose J and rho parts do not start together in this row
        unsigned rest = (gJ | gR) & ~gB;
        while (rest) {
            const int k = __ffs(rest) - 1;
            rest &= rest - 1;
            const int kzJ = __shfl_sync(FULL, zJ, k), kzR = __shfl_sync(FULL, zR, k);
            const bool kJ = (gJ >> k) & 1u, kR = (gR >> k) & 1u;
            const float2 ck = pmul(ld2(sx + k * M), ld2(sy + k * M));
            const float4 z01 = *reinterpret_cast<const float4*>(sz + k * M);
            const float4 z23 = *reinterpret_cast<const float4*>(sz + k * M + 4);
            const float zc[8] = {z01.x, z01.y, z01.z, z01.w, z23.x, z23.y, z23.z, z23.w};
            // J part (both components of h = 0; the first of h = 1) at kzJ
            if (kJ) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    atomicAdd(p0 + kzJ + c, ck.x * zc[2 * c]);
                    if (!hi) atomicAdd(p1 + kzJ + c, ck.y * zc[2 * c + 1]);
                }
            }
            // rho part (the second component of h = 1) at kzR
            if (kR && hi) {
#pragma unroll
                for (int c = 0; c < 4; ++c) atomicAdd(p1 + kzR + c, ck.y * zc[2 * c + 1]);
            }
        }
    }
}

template <typename T, int ORDER, int MODE, int MARGIN, int DEP, bool MIX>
__device__ __forceinline__ void particle_pass_body(const PassK<T>& p, const int b) {
    typedef Shape<ORDER> SH;
    typedef typename Pair<T>::type P2;
    constexpr int NW = SH::NW;
    constexpr int TE = TileGeom<NW, MARGIN>::E;
    constexpr int R = TileGeom<NW, MARGIN>::R;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const PassSmem L(R, NW, sizeof(T), MODE == PASS_STEP, DEP);
    static_assert(DEP == DEP_GROUP || DEP == DEP_FIXED || (sizeof(T) == 4 && NW == 4),
                  "row deposit: FP32, NW = 4 only");
    static_assert(!MIX || (NW == 4 && (DEP == DEP_GROUP || DEP == DEP_JR)),
                  "mixed-species groups: NW = 4, grouped deposits");
    static_assert(DEP != DEP_JR || (sizeof(T) == 4 && NW == 4), "combined J and rho groups: FP32, NW = 4 only");
    static_assert(DEP != DEP_FIXED || !MIX, "fixed-point deposit: one species at a time");
    constexpr bool FIX = DEP == DEP_FIXED;
    FieldTile<T> tile;
    tile.init(smem_raw + L.tile, R);
    T* sD = reinterpret_cast<T*>(smem_raw + L.dep);
    long long* const sD64 = reinterpret_cast<long long*>(smem_raw + L.dep);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    Stage<T, NW> stg;
    stg.base = reinterpret_cast<T*>(smem_raw + L.stage + warp * stage_bytes(NW, sizeof(T), DEP));
    float* const rstg = reinterpret_cast<float*>(stg.base);

    const int bz = b % p.nbz, by = (b / p.nbz) % p.nby, bx = b / (p.nbz * p.nby);
    const int x0 = bx * BIN, y0 = by * BIN, z0 = bz * BIN;
    // global node of tile index 0 along each axis
    const int ox = x0 + SH::J0 - MARGIN, oy = y0 + SH::J0 - MARGIN, oz = z0 + SH::J0 - MARGIN;
    const int64_t N = p.N;

    for (int idx = threadIdx.x; idx < R; idx += blockDim.x) {
        const int rx = idx / (TE * TE);
        const int rem = idx - rx * (TE * TE);
        const int ry = rem / TE;
        const int rz = rem - ry * TE;
        if (MODE == PASS_STEP) {
            int64_t g = ((int64_t)wrap_near(ox + rx, p.nx) * p.ny + wrap_near(oy + ry, p.ny)) * p.nz +
                        wrap_near(oz + rz, p.nz);
            T v[6];
#pragma unroll
            for (int q = 0; q < 6; ++q) v[q] = p.F[q * N + g];
            tile.store(idx, v);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if constexpr (FIX)
                sD64[q * R + idx] = 0;
            else
                sD[q * R + idx] = (T)0;
        }
    }
    __syncthreads();

    unsigned long long miss = 0, far = 0;
    // MIX (two species, cell-sorted alike): half-warps take 16 particles of each
    // species from the same place in their bin ranges, so the particles of one cell of
    // both species form one deposit group. Otherwise one species at a time.
    constexpr int STRIDE = MIX ? PASS_THREADS / 2 : PASS_THREADS;
    const int local = MIX ? (int)((threadIdx.x >> 5) * 16 + (threadIdx.x & 15)) : (int)threadIdx.x;
    for (int s = 0; s < (MIX ? 1 : p.nspecies); ++s) {
        const int hs = MIX ? (int)((threadIdx.x >> 4) & 1) : s;
        const SpeciesK<T> sp = p.sp[hs];
        int beg = sp.bin_start[b], end = sp.bin_start[b + 1];
        // checked build: a bin range outside the species' particles is flagged and emptied
        if (!(PIC_INDEX_OK(beg, (int64_t)sp.n + 1, p.status) && PIC_INDEX_OK(end, (int64_t)sp.n + 1, p.status) &&
              PIC_INDEX_OK(end - beg, (int64_t)sp.n + 1, p.status)))
            beg = end = 0;
        int span = end - beg;
        if constexpr (MIX)
            span = max(p.sp[0].bin_start[b + 1] - p.sp[0].bin_start[b],
                       p.sp[1].bin_start[b + 1] - p.sp[1].bin_start[b]);
        // the next chunk's particle is loaded while the current one is processed
        int c_n = 0;
        T f_n[3] = {0, 0, 0}, u_n[3] = {0, 0, 0};
        if (beg + local < end) {
            const int j = beg + local;
            c_n = sp.cell[j];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                f_n[d] = sp.off[d][j];
                u_n[d] = sp.u[d][j];
            }
        }
        for (int off0 = 0; off0 < span; off0 += STRIDE) {
            const int i = beg + off0 + local;
            // checked build: a cell index outside the grid is flagged and the particle skipped
            const bool valid = i < end && PIC_INDEX_OK(c_n, N, p.status);
            int ix = 0, iy = 0, iz = 0, rx = -1, ry = -1, rz = -1;
            T fx = f_n[0], fy = f_n[1], fz = f_n[2], ux = u_n[0], uy = u_n[1], uz = u_n[2];
            const int c = c_n;
            if (i + STRIDE < end) {
                const int j = i + STRIDE;
                c_n = sp.cell[j];
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    f_n[d] = sp.off[d][j];
                    u_n[d] = sp.u[d][j];
                }
            }
            T wx[4], wy[4], wz[4];
            T vx = 0, vy = 0, vz = 0;
            if (valid) {
                ix = p.div_nynz.div(c);
                const int rem = c - ix * (p.ny * p.nz);
                iy = p.div_nz.div(rem);
                iz = rem - iy * p.nz;
                rx = ix - x0 + MARGIN;
                ry = iy - y0 + MARGIN;
                rz = iz - z0 + MARGIN;
                if (MODE == PASS_STEP) {
                    // ---- gather E^n, B^n at x^n
                    SH::w(fx, wx);
                    SH::w(fy, wy);
                    SH::w(fz, wz);
                    T E[3], B[3];
                    if (in_tile<NW, TE>(rx) && in_tile<NW, TE>(ry) && in_tile<NW, TE>(rz)) {
                        // two interleaved accumulator sets (even / odd z node) for ILP
                        P2 a0 = Pair<T>::make(0, 0), a1 = a0, a2 = a0, c0 = a0, c1 = a0, c2 = a0;
                        P2 wzp[NW];
#pragma unroll
                        for (int cc = 0; cc < NW; ++cc) wzp[cc] = Pair<T>::make(wz[cc], wz[cc]);
                        // one runtime base index; every node is a compile-time offset from it
                        int base0 = (rx * TE + ry) * TE + rz;
#ifdef PIC_CHECKED
                        base0 += p.inject;
                        if (!PIC_INDEX_OK(base0, R - (NW - 1) * (TE * TE + TE + 1), p.status)) base0 = 0;
#endif
#pragma unroll
                        for (int a = 0; a < NW; ++a)
#pragma unroll
                            for (int bb = 0; bb < NW; ++bb) {
                                const T wxy = wx[a] * wy[bb];
                                const P2 wxyp = Pair<T>::make(wxy, wxy);
                                const int base_t = base0 + (a * TE + bb) * TE;
#pragma unroll
                                for (int cc = 0; cc < NW; ++cc) {
                                    const P2 w2 = pmul(wxyp, wzp[cc]);
                                    P2 f0, f1, f2;
                                    tile.load(base_t + cc, f0, f1, f2);
                                    if (cc & 1) {
                                        c0 = pfma(w2, f0, c0);
                                        c1 = pfma(w2, f1, c1);
                                        c2 = pfma(w2, f2, c2);
                                    } else {
                                        a0 = pfma(w2, f0, a0);
                                        a1 = pfma(w2, f1, a1);
                                        a2 = pfma(w2, f2, a2);
                                    }
                                }
                            }
                        E[0] = a0.x + c0.x; E[1] = a0.y + c0.y; E[2] = a1.x + c1.x;
                        B[0] = a1.y + c1.y; B[1] = a2.x + c2.x; B[2] = a2.y + c2.y;
                    } else {
                        far++;
                        for (int q = 0; q < 3; ++q) E[q] = B[q] = (T)0;
#pragma unroll
                        for (int a = 0; a < NW; ++a)
#pragma unroll
                            for (int bb = 0; bb < NW; ++bb) {
                                const T wxy = wx[a] * wy[bb];
                                const int64_t gb = ((int64_t)wrapf<NW>(ix + SH::J0 + a, p.nx) * p.ny +
                                                    wrapf<NW>(iy + SH::J0 + bb, p.ny)) * p.nz;
#pragma unroll
                                for (int cc = 0; cc < NW; ++cc) {
                                    const T w = wxy * wz[cc];
                                    const int64_t g = gb + wrapf<NW>(iz + SH::J0 + cc, p.nz);
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
                    const T umx = ux + a * E[0], umy = uy + a * E[1], umz = uz + a * E[2];
                    const T igm = boris_rsqrt((T)1 + (umx * umx + umy * umy + umz * umz) * p.inv_c2);
                    const T tx = a * B[0] * igm, ty = a * B[1] * igm, tz = a * B[2] * igm;
                    const T s2 = boris_div((T)2, (T)1 + tx * tx + ty * ty + tz * tz);
                    const T sx = s2 * tx, sy = s2 * ty, sz = s2 * tz;
                    const T upx = umx + (umy * tz - umz * ty);
                    const T upy = umy + (umz * tx - umx * tz);
                    const T upz = umz + (umx * ty - umy * tx);
                    ux = umx + (upy * sz - upz * sy) + a * E[0];
                    uy = umy + (upz * sx - upx * sz) + a * E[1];
                    uz = umz + (upx * sy - upy * sx) + a * E[2];
                }
                const T igam = boris_rsqrt((T)1 + (ux * ux + uy * uy + uz * uz) * p.inv_c2);
                vx = ux * igam;
                vy = uy * igam;
                vz = uz * igam;
            }
            // ---- deposit J (phase 0: at x^{n+1/2} with v^{n+1/2}) and rho (phase 1:
            // at x^{n+1}); DEPOSIT mode: both at the current x
            if constexpr (!FIX && (NW == 2 || DEP == DEP_JR)) {
                // both stencils first, then one combined J and rho group pass
                // (group_deposit_jr / group_deposit_jr4)
                bool mJ = false, mR = false, same = false;
                int keyJ = 0, keyR = 0;
                T wxR[NW], wyR[NW], wzR[NW];
                if (valid) {
                    if (MODE == PASS_STEP) {
                        rx += drift_axis(ix, fx, (vx - p.vgal[0]) * p.hd[0], p.nx);
                        ry += drift_axis(iy, fy, (vy - p.vgal[1]) * p.hd[1], p.ny);
                        rz += drift_axis(iz, fz, (vz - p.vgal[2]) * p.hd[2], p.nz);
                    }
                    SH::w(fx, wx);
                    SH::w(fy, wy);
                    SH::w(fz, wz);
                    mJ = in_tile<NW, TE>(rx) && in_tile<NW, TE>(ry) && in_tile<NW, TE>(rz) &&
                         PIC_INDEX_OK((rx * TE + ry) * TE + rz, R - (NW - 1) * (TE * TE + TE + 1), p.status);
                    if (mJ) {
                        keyJ = (rx * TE + ry) * TE + rz;
                    } else {
                        const T val[3] = {sp.qw_dv * vx, sp.qw_dv * vy, sp.qw_dv * vz};
                        deposit_global<T, NW, SH::J0>(p, ix, iy, iz, wx, wy, wz, 0, 3, val);
                    }
                    if (MODE == PASS_STEP) {
                        rx += drift_axis(ix, fx, (vx - p.vgal[0]) * p.hd[0], p.nx);
                        ry += drift_axis(iy, fy, (vy - p.vgal[1]) * p.hd[1], p.ny);
                        rz += drift_axis(iz, fz, (vz - p.vgal[2]) * p.hd[2], p.nz);
                        SH::w(fx, wxR);
                        SH::w(fy, wyR);
                        SH::w(fz, wzR);
                    } else {
#pragma unroll
                        for (int q = 0; q < NW; ++q) {
                            wxR[q] = wx[q];
                            wyR[q] = wy[q];
                            wzR[q] = wz[q];
                        }
                    }
                    mR = in_tile<NW, TE>(rx) && in_tile<NW, TE>(ry) && in_tile<NW, TE>(rz) &&
                         PIC_INDEX_OK((rx * TE + ry) * TE + rz, R - (NW - 1) * (TE * TE + TE + 1), p.status);
                    if (mR) {
                        keyR = (rx * TE + ry) * TE + rz;
                    } else {
                        far++;
                        const T val[1] = {sp.qw_dv};
                        deposit_global<T, NW, SH::J0>(p, ix, iy, iz, wxR, wyR, wzR, 3, 1, val);
                    }
                    same = mJ && mR && keyR == keyJ;
                    if (mJ) {
                        // MIX: values carry q w / dV (members of both species)
                        const T qs = MIX ? sp.qw_dv : (T)1;
                        const T vel[3] = {qs * vx, qs * vy, qs * vz};
                        stage_record<T, NW>(stg, lane, wx, wy, wz, vel);
                        stg.frow()[lane] = same ? qs : (T)0;
#pragma unroll
                        for (int a = 0; a < NW; ++a) {
                            stg.xRrow(a)[lane] = wxR[a];
                            stg.yRrow(a)[lane] = wyR[a];
                            stg.zRrow(a)[lane] = wzR[a];
                        }
                    }
                }
                __syncwarp();
                if constexpr (NW == 2)
                    group_deposit_jr<T, TE>(sD, stg, mJ, keyJ, lane, MIX ? (T)1 : sp.qw_dv);
                else
                    group_deposit_jr4<T, TE>(sD, stg, mJ, keyJ, lane, MIX ? (T)1 : sp.qw_dv);
                __syncwarp();
                // rho of members whose rho stencil starts elsewhere
                const bool restR = mR && !same;
                if (__any_sync(0xffffffffu, restR)) {
                    if (restR) {
                        stage_record<T, NW>(stg, lane, wxR, wyR, wzR, nullptr);
                        if constexpr (MIX) stg.vrow(0)[lane] = sp.qw_dv;
                    }
                    __syncwarp();
                    group_deposit<T, NW, 1, TE, MIX>(sD, stg, restR, keyR, lane, MIX ? (T)1 : sp.qw_dv);
                    __syncwarp();
                }
            } else if constexpr (DEP == DEP_ROW || DEP == DEP_ROWU) {
                // few particles per cell: both stencils first, then one pass by stencil row
                bool mJ = false, mR = false;
                int rowJ = 0, zJ = 0, rowR = 0, zR = 0;
                if (valid) {
                    if (MODE == PASS_STEP) {
                        rx += drift_axis(ix, fx, (vx - p.vgal[0]) * p.hd[0], p.nx);
                        ry += drift_axis(iy, fy, (vy - p.vgal[1]) * p.hd[1], p.ny);
                        rz += drift_axis(iz, fz, (vz - p.vgal[2]) * p.hd[2], p.nz);
                    }
                    SH::w(fx, wx);
                    SH::w(fy, wy);
                    SH::w(fz, wz);
                    const T qvx = sp.qw_dv * vx, qvy = sp.qw_dv * vy, qvz = sp.qw_dv * vz;
                    mJ = in_tile<NW, TE>(rx) && in_tile<NW, TE>(ry) && in_tile<NW, TE>(rz) &&
                         PIC_INDEX_OK((rx * TE + ry) * TE + rz, R - (NW - 1) * (TE * TE + TE + 1), p.status);
                    if (mJ) {
                        rowJ = rx * TE + ry;
                        zJ = rz;
                    } else {
                        const T val[3] = {qvx, qvy, qvz};
                        deposit_global<T, NW, SH::J0>(p, ix, iy, iz, wx, wy, wz, 0, 3, val);
                    }
                    T wxR[NW], wyR[NW], wzR[NW];
                    if (MODE == PASS_STEP) {
                        rx += drift_axis(ix, fx, (vx - p.vgal[0]) * p.hd[0], p.nx);
                        ry += drift_axis(iy, fy, (vy - p.vgal[1]) * p.hd[1], p.ny);
                        rz += drift_axis(iz, fz, (vz - p.vgal[2]) * p.hd[2], p.nz);
                        SH::w(fx, wxR);
                        SH::w(fy, wyR);
                        SH::w(fz, wzR);
                    } else {
#pragma unroll
                        for (int q = 0; q < NW; ++q) {
                            wxR[q] = wx[q];
                            wyR[q] = wy[q];
                            wzR[q] = wz[q];
                        }
                    }
                    mR = in_tile<NW, TE>(rx) && in_tile<NW, TE>(ry) && in_tile<NW, TE>(rz) &&
                         PIC_INDEX_OK((rx * TE + ry) * TE + rz, R - (NW - 1) * (TE * TE + TE + 1), p.status);
                    if (mR) {
                        rowR = rx * TE + ry;
                        zR = rz;
                    } else {
                        far++;
                        const T val[1] = {sp.qw_dv};
                        deposit_global<T, NW, SH::J0>(p, ix, iy, iz, wxR, wyR, wzR, 3, 1, val);
                    }
                    if (mJ || mR)
                        row_record(rstg + lane * RowStage::MEMBER, (const float*)wx, (const float*)wy,
                                   (const float*)wz, (const float*)wxR, (const float*)wyR, (const float*)wzR,
                                   (float)qvx, (float)qvy, (float)qvz, (float)sp.qw_dv);
                }
                __syncwarp();
                if constexpr (DEP == DEP_ROWU)
                    row_deposit_unrolled<TE>(reinterpret_cast<float*>(sD), rstg, mJ, rowJ, zJ, mR, rowR, zR, lane);
                else
                    row_deposit<TE>(reinterpret_cast<float*>(sD), rstg, mJ, rowJ, zJ, mR, rowR, zR, lane);
                __syncwarp();
            } else
#pragma unroll
            for (int phase = 0; phase < 2; ++phase) {
                bool member = false;
                int key = 0;
                if (valid) {
                    if (MODE == PASS_STEP) {
                        rx += drift_axis(ix, fx, (vx - p.vgal[0]) * p.hd[0], p.nx);
                        ry += drift_axis(iy, fy, (vy - p.vgal[1]) * p.hd[1], p.ny);
                        rz += drift_axis(iz, fz, (vz - p.vgal[2]) * p.hd[2], p.nz);
                    }
                    if (MODE == PASS_STEP || phase == 0) {
                        SH::w(fx, wx);
                        SH::w(fy, wy);
                        SH::w(fz, wz);
                    }
                    T val[3];
                    if (phase == 0) {
                        val[0] = sp.qw_dv * vx;
                        val[1] = sp.qw_dv * vy;
                        val[2] = sp.qw_dv * vz;
                    } else {
                        val[0] = sp.qw_dv;
                        val[1] = val[2] = (T)0;
                    }
                    if constexpr (FIX) {   // values carry q w / (dV delta)
                        const T qs = sp.qw_dv * p.inv_delta;
                        if (phase == 0) {
                            val[0] = qs * vx;
                            val[1] = qs * vy;
                            val[2] = qs * vz;
                        } else {
                            val[0] = qs;
                        }
                    }
                    if (in_tile<NW, TE>(rx) && in_tile<NW, TE>(ry) && in_tile<NW, TE>(rz) &&
                        PIC_INDEX_OK((rx * TE + ry) * TE + rz, R - (NW - 1) * (TE * TE + TE + 1), p.status)) {
                        member = true;
                        key = (rx * TE + ry) * TE + rz;
                        if constexpr (FIX) {
                            stage_record<T, NW>(stg, lane, wx, wy, wz, phase == 0 ? val : nullptr);
                            if (phase == 1) stg.vrow(0)[lane] = val[0];
                        } else if constexpr (MIX) {   // values carry q w / dV (members of both species)
                            const T qvel[3] = {sp.qw_dv * vx, sp.qw_dv * vy, sp.qw_dv * vz};
                            stage_record<T, NW>(stg, lane, wx, wy, wz, phase == 0 ? qvel : nullptr);
                            if (phase == 1) stg.vrow(0)[lane] = sp.qw_dv;
                        } else {
                            const T vel[3] = {vx, vy, vz};
                            stage_record<T, NW>(stg, lane, wx, wy, wz, phase == 0 ? vel : nullptr);
                        }
                    } else {
                        if (phase == 1) far++;
                        if constexpr (FIX) {
                            if (phase == 0)
                                deposit_global_fixed<T, NW, SH::J0>(p, ix, iy, iz, wx, wy, wz, 0, 3, val);
                            else
                                deposit_global_fixed<T, NW, SH::J0>(p, ix, iy, iz, wx, wy, wz, 3, 1, val);
                        } else {
                            if (phase == 0)
                                deposit_global<T, NW, SH::J0>(p, ix, iy, iz, wx, wy, wz, 0, 3, val);
                            else
                                deposit_global<T, NW, SH::J0>(p, ix, iy, iz, wx, wy, wz, 3, 1, val);
                        }
                    }
                }
                __syncwarp();
                if constexpr (FIX) {
                    if (phase == 0)
                        group_deposit_fixed<T, NW, 3, TE>(sD64, stg, member, key, lane);
                    else
                        group_deposit_fixed<T, NW, 1, TE>(sD64, stg, member, key, lane);
                } else {
                    if (phase == 0)
                        group_deposit<T, NW, 3, TE, MIX>(sD, stg, member, key, lane, MIX ? (T)1 : sp.qw_dv);
                    else
                        group_deposit<T, NW, 1, TE, MIX>(sD, stg, member, key, lane, MIX ? (T)1 : sp.qw_dv);
                }
                __syncwarp();
            }
            if (valid && MODE == PASS_STEP) {
                sp.cell[i] = (ix * p.ny + iy) * p.nz + iz;
                sp.off[0][i] = fx;
                sp.off[1][i] = fy;
                sp.off[2][i] = fz;
                sp.u[0][i] = ux;
                sp.u[1][i] = uy;
                sp.u[2][i] = uz;
                if (ix < x0 || ix >= x0 + BIN || iy < y0 || iy >= y0 + BIN || iz < z0 || iz >= z0 + BIN)
                    miss++;
            }
        }
    }
    __syncthreads();

    // add the tile to the global source grids
    for (int idx = threadIdx.x; idx < R; idx += blockDim.x) {
        const int rx = idx / (TE * TE);
        const int rem = idx - rx * (TE * TE);
        const int ry = rem / TE;
        const int rz = rem - ry * TE;
        int64_t g = ((int64_t)wrap_near(ox + rx, p.nx) * p.ny + wrap_near(oy + ry, p.ny)) * p.nz +
                    wrap_near(oz + rz, p.nz);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if constexpr (FIX) {
                const long long v = sD64[q * R + idx];
                if (v) add_fixed(p.S64 + q * N + g, v);
            } else {
                T v = sD[q * R + idx];
                if (v != (T)0) atomicAdd(&p.S[q * N + g], v);
            }
        }
    }

    if (MODE == PASS_STEP) {
        for (int o = 16; o > 0; o >>= 1) {
            miss += __shfl_down_sync(0xffffffffu, miss, o);
            far += __shfl_down_sync(0xffffffffu, far, o);
        }
        if (lane == 0) {
            if (miss) atomicAdd(&p.cnt[CNT_HOME_MISS], miss);
            if (far) atomicAdd(&p.cnt[CNT_FAR], far);
        }
    }
}

// ---- linear shapes: one thread per cell -----------------------------------------
// Particles are sorted by cell (cell_start ranges of the last sort). A thread takes one
// cell of the bin and walks that cell's particles of every species. A particle still in
// the cell gathers E, B from the cell's eight tile nodes (compile-time offsets from one
// base), and its J^{n+1/2} and rho^{n+1}, when their stencils still start at the cell,
// add into 32 register accumulators (8 nodes x Jx, Jy, Jz, rho) that go to the shared
// tile once per cell. A particle that has left the cell since the sort, or whose J or
// rho stencil starts elsewhere, uses the tile at its own position (per-node shared
// atomics) or, outside the tile, global memory.
constexpr int CELL_THREADS = 256;

// 2x2x2 gather from the tile at base index `base` (node (a, b, c) at base + (a TE + b) TE + c).
template <typename T, int TE>
__device__ __forceinline__ void gather2(const FieldTile<T>& tile, int base, const T* wx, const T* wy,
                                        const T* wz, T* E, T* B) {
    typedef typename Pair<T>::type P2;
    P2 a0 = Pair<T>::make(0, 0), a1 = a0, a2 = a0;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const T wxy = wx[a] * wy[b];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const T w = wxy * wz[c];
                const P2 w2 = Pair<T>::make(w, w);
                P2 f0, f1, f2;
                tile.load(base + (a * TE + b) * TE + c, f0, f1, f2);
                a0 = pfma(w2, f0, a0);
                a1 = pfma(w2, f1, a1);
                a2 = pfma(w2, f2, a2);
            }
        }
    E[0] = a0.x; E[1] = a0.y; E[2] = a1.x;
    B[0] = a1.y; B[1] = a2.x; B[2] = a2.y;
}

// Per-node shared-memory atomics of Q values at a 2x2x2 stencil in the tile.
template <typename T, int TE>
__device__ __forceinline__ void tile_atomic2(T* sD, int base, const T* wx, const T* wy, const T* wz, int q0,
                                             int Q, const T* val) {
    constexpr int R = TE * TE * TE;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const T w = wx[a] * wy[b] * wz[c];
                const int idx = base + (a * TE + b) * TE + c;
                for (int q = 0; q < Q; ++q) atomicAdd(&sD[(q0 + q) * R + idx], w * val[q]);
            }
}

// Tile coordinate of cell i along an axis whose bin starts at o (tile node 0 = o - MARGIN):
// the periodic image of i nearest to the bin, so that a particle that crossed the
// periodic boundary next to the bin still finds its nodes in the tile.
__device__ __forceinline__ int tile_coord(int i, int o, int n, int margin) {
    int d = i - o;
    if (2 * d > n) d -= n;
    else if (2 * d < -n) d += n;
    return d + margin;
}

template <typename T, int MODE, int MARGIN>
__device__ __forceinline__ void cell_pass_body(const PassK<T>& p, const int b) {
    typedef typename Pair<T>::type P2;
    typedef Shape<1> SH;
    constexpr int NW = 2;
    constexpr int TE = TileGeom<NW, MARGIN>::E;
    constexpr int R = TileGeom<NW, MARGIN>::R;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const PassSmem L(R, NW, sizeof(T), MODE == PASS_STEP, DEP_CELL);
    FieldTile<T> tile;
    tile.init(smem_raw + L.tile, R);
    T* sD = reinterpret_cast<T*>(smem_raw + L.dep);
    const int lane = threadIdx.x & 31;
    const int bz = b % p.nbz, by = (b / p.nbz) % p.nby, bx = b / (p.nbz * p.nby);
    const int x0 = bx * BIN, y0 = by * BIN, z0 = bz * BIN;
    const int ox = x0 - MARGIN, oy = y0 - MARGIN, oz = z0 - MARGIN;
    const int64_t N = p.N;
    // the step's scalars, read once (the shared-launch kernels keep the run's parameters in
    // shared memory, which would otherwise be read at every use)
    const T inv_c2 = p.inv_c2;
    const T vg[3] = {p.vgal[0], p.vgal[1], p.vgal[2]}, hd[3] = {p.hd[0], p.hd[1], p.hd[2]};
    for (int idx = threadIdx.x; idx < R; idx += blockDim.x) {
        const int rx = idx / (TE * TE);
        const int rem = idx - rx * (TE * TE);
        const int ry = rem / TE;
        const int rz = rem - ry * TE;
        if (MODE == PASS_STEP) {
            int64_t g = ((int64_t)wrap_near(ox + rx, p.nx) * p.ny + wrap_near(oy + ry, p.ny)) * p.nz +
                        wrap_near(oz + rz, p.nz);
            T v[6];
#pragma unroll
            for (int q = 0; q < 6; ++q) v[q] = p.F[q * N + g];
            tile.store(idx, v);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) sD[q * R + idx] = (T)0;
    }
    __syncthreads();

    unsigned long long miss = 0, far = 0;
    const int warp = threadIdx.x >> 5;
    // this warp's particle staging: cell[CELL_STRIDE] then off x, y, z and u x, y, z, entry j
    // of a chunk at slot cell_slot(j)
    unsigned char* const wst = smem_raw + L.stage + (size_t)warp * stage_bytes(NW, sizeof(T), DEP_CELL);
    int32_t* const st_cell = reinterpret_cast<int32_t*>(wst);
    T* const st_v = reinterpret_cast<T*>(wst + CELL_STRIDE * 4);   // [6][CELL_STRIDE]
    // warp w takes the 32 consecutive cells (keys) 32 w .. 32 w + 31, then 256 + 32 w ..;
    // lane t the cell 32 w + t of each group: the group's particles are one contiguous
    // range per species, staged CELL_CHUNK at a time
    for (int g0 = 32 * warp; g0 < BIN * BIN * BIN; g0 += CELL_THREADS) {
        const int lc = g0 + lane;
        const int lx = lc >> 6, ly = (lc >> 3) & 7, lz = lc & 7;
        const int hx = x0 + lx, hy = y0 + ly, hz = z0 + lz;
        const int key = b * (BIN * BIN * BIN) + lc;
        // cells past the grid's edge in a partial bin hold no particles (empty ranges)
        const int home = (hx * p.ny + hy) * p.nz + hz;
        const int hrx = lx + MARGIN, hry = ly + MARGIN, hrz = lz + MARGIN;
        const int hbase = (hrx * TE + hry) * TE + hrz;
        P2 aJ[8];
        T aZ[8], aR[8];
#pragma unroll
        for (int n = 0; n < 8; ++n) {
            aJ[n] = Pair<T>::make(0, 0);
            aZ[n] = aR[n] = (T)0;
        }
        for (int s = 0; s < p.nspecies; ++s) {
            const SpeciesK<T>& sp = p.sp[s];
            const T qdt2m = sp.qdt2m, qw_dv = sp.qw_dv;
            int beg = sp.cell_start[key], end = sp.cell_start[key + 1];
            // checked build: a cell range outside the species' particles is flagged and emptied
            if (!(PIC_INDEX_OK(beg, (int64_t)sp.n + 1, p.status) && PIC_INDEX_OK(end, (int64_t)sp.n + 1, p.status) &&
                  PIC_INDEX_OK(end - beg, (int64_t)sp.n + 1, p.status)))
                beg = end = 0;
            int A = __shfl_sync(0xffffffffu, beg, 0), Bend = __shfl_sync(0xffffffffu, end, 31);
            if (!PIC_INDEX_OK(Bend - A, (int64_t)sp.n + 1, p.status)) A = Bend = 0;
            for (int lo = A; lo < Bend; lo += CELL_CHUNK) {
                const int hi = min(lo + CELL_CHUNK, Bend);
                bool moved = false;   // a particle of this lane changed cell in this chunk
                // stage in, coalesced, every load of the chunk in flight at once
                for (int j = lane; j < hi - lo; j += 32) {
                    const int q = cell_slot(j);
                    async_copy<4>(&st_cell[q], &sp.cell[lo + j]);
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        async_copy<sizeof(T)>(&st_v[d * CELL_STRIDE + q], &sp.off[d][lo + j]);
                        async_copy<sizeof(T)>(&st_v[(3 + d) * CELL_STRIDE + q], &sp.u[d][lo + j]);
                    }
                }
                async_wait_all();
                __syncwarp();
                const int i0 = max(beg, lo), i1 = min(end, hi);
                // one particle at staging slot j from its loaded values; `pushed`: E, B were
                // gathered at its home cell and u pushed already
                auto one = [&](const int j, const int c, T fx, T fy, T fz, T ux, T uy, T uz, const bool pushed) {
                    if (!PIC_INDEX_OK(c, N, p.status)) return;
                    int ix = hx, iy = hy, iz = hz, rx = hrx, ry = hry, rz = hrz;
                    if (c != home) {   // moved since the sort
                        ix = p.div_nynz.div(c);
                        const int rem = c - ix * (p.ny * p.nz);
                        iy = p.div_nz.div(rem);
                        iz = rem - iy * p.nz;
                        rx = tile_coord(ix, x0, p.nx, MARGIN);
                        ry = tile_coord(iy, y0, p.ny, MARGIN);
                        rz = tile_coord(iz, z0, p.nz, MARGIN);
                    }
                    T wx[2], wy[2], wz[2];
                    if (MODE == PASS_STEP && !pushed) {
                        // ---- gather E^n, B^n at x^n
                        SH::w(fx, wx);
                        SH::w(fy, wy);
                        SH::w(fz, wz);
                        T E[3], B[3];
                        int gbase = hbase;
#ifdef PIC_CHECKED
                        gbase += p.inject;
                        if (!PIC_INDEX_OK(gbase, R - (TE * TE + TE + 1), p.status)) gbase = 0;
#endif
                        if (c == home) {
                            gather2<T, TE>(tile, gbase, wx, wy, wz, E, B);
                        } else if (in_tile<NW, TE>(rx) && in_tile<NW, TE>(ry) && in_tile<NW, TE>(rz)) {
                            gather2<T, TE>(tile, (rx * TE + ry) * TE + rz, wx, wy, wz, E, B);
                        } else {
                            far++;
                            for (int q = 0; q < 3; ++q) E[q] = B[q] = (T)0;
    #pragma unroll
                            for (int a = 0; a < 2; ++a)
    #pragma unroll
                                for (int bb = 0; bb < 2; ++bb) {
                                    const T wxy = wx[a] * wy[bb];
                                    const int64_t gb =
                                        ((int64_t)wrapi(ix + a, p.nx) * p.ny + wrapi(iy + bb, p.ny)) * p.nz;
    #pragma unroll
                                    for (int cc = 0; cc < 2; ++cc) {
                                        const T w = wxy * wz[cc];
                                        const int64_t g = gb + wrapi(iz + cc, p.nz);
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
                        boris_push(qdt2m, E, B, inv_c2, ux, uy, uz);
                    }
                    const T igam = boris_rsqrt((T)1 + (ux * ux + uy * uy + uz * uz) * inv_c2);
                    const T vx = ux * igam, vy = uy * igam, vz = uz * igam;
                    // ---- J^{n+1/2} at x^{n+1/2} with v^{n+1/2} (DEPOSIT mode: at x with v)
                    if (MODE == PASS_STEP) {
                        rx += drift_axis(ix, fx, (vx - vg[0]) * hd[0], p.nx);
                        ry += drift_axis(iy, fy, (vy - vg[1]) * hd[1], p.ny);
                        rz += drift_axis(iz, fz, (vz - vg[2]) * hd[2], p.nz);
                        SH::w(fx, wx);
                        SH::w(fy, wy);
                        SH::w(fz, wz);
                    } else {
                        SH::w(fx, wx);
                        SH::w(fy, wy);
                        SH::w(fz, wz);
                    }
                    const T qv[3] = {qw_dv * vx, qw_dv * vy, qw_dv * vz};
                    if (rx == hrx && ry == hry && rz == hrz) {
                        const P2 qxy = Pair<T>::make(qv[0], qv[1]);
    #pragma unroll
                        for (int a = 0; a < 2; ++a)
    #pragma unroll
                            for (int bb = 0; bb < 2; ++bb) {
                                const T wxy = wx[a] * wy[bb];
    #pragma unroll
                                for (int cc = 0; cc < 2; ++cc) {
                                    const T w = wxy * wz[cc];
                                    const int n = (a * 2 + bb) * 2 + cc;
                                    aJ[n] = pfma(Pair<T>::make(w, w), qxy, aJ[n]);
                                    aZ[n] = fma(w, qv[2], aZ[n]);
                                }
                            }
                    } else if (in_tile<NW, TE>(rx) && in_tile<NW, TE>(ry) && in_tile<NW, TE>(rz)) {
                        tile_atomic2<T, TE>(sD, (rx * TE + ry) * TE + rz, wx, wy, wz, 0, 3, qv);
                    } else {
                        deposit_global<T, NW, 0>(p, ix, iy, iz, wx, wy, wz, 0, 3, qv);
                    }
                    // ---- rho^{n+1} at x^{n+1} (DEPOSIT mode: at x)
                    if (MODE == PASS_STEP) {
                        rx += drift_axis(ix, fx, (vx - vg[0]) * hd[0], p.nx);
                        ry += drift_axis(iy, fy, (vy - vg[1]) * hd[1], p.ny);
                        rz += drift_axis(iz, fz, (vz - vg[2]) * hd[2], p.nz);
                        SH::w(fx, wx);
                        SH::w(fy, wy);
                        SH::w(fz, wz);
                    }
                    const T qr[1] = {qw_dv};
                    if (rx == hrx && ry == hry && rz == hrz) {
    #pragma unroll
                        for (int a = 0; a < 2; ++a)
    #pragma unroll
                            for (int bb = 0; bb < 2; ++bb) {
                                const T wxy = wx[a] * wy[bb];
    #pragma unroll
                                for (int cc = 0; cc < 2; ++cc)
                                    aR[(a * 2 + bb) * 2 + cc] = fma(wxy * wz[cc], qr[0], aR[(a * 2 + bb) * 2 + cc]);
                            }
                    } else if (in_tile<NW, TE>(rx) && in_tile<NW, TE>(ry) && in_tile<NW, TE>(rz)) {
                        tile_atomic2<T, TE>(sD, (rx * TE + ry) * TE + rz, wx, wy, wz, 3, 1, qr);
                    } else {
                        far++;
                        deposit_global<T, NW, 0>(p, ix, iy, iz, wx, wy, wz, 3, 1, qr);
                    }
                    if (MODE == PASS_STEP) {
                        const int nc = (ix * p.ny + iy) * p.nz + iz;
                        moved = moved || nc != c;
                        st_cell[j] = nc;
                        st_v[0 * CELL_STRIDE + j] = fx;
                        st_v[1 * CELL_STRIDE + j] = fy;
                        st_v[2 * CELL_STRIDE + j] = fz;
                        st_v[3 * CELL_STRIDE + j] = ux;
                        st_v[4 * CELL_STRIDE + j] = uy;
                        st_v[5 * CELL_STRIDE + j] = uz;
                        if (ix < x0 || ix >= x0 + BIN || iy < y0 || iy >= y0 + BIN || iz < z0 || iz >= z0 + BIN)
                            miss++;
                    }
                };
                auto load = [&](const int j, T* f, T* u) {
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        f[d] = st_v[d * CELL_STRIDE + j];
                        u[d] = st_v[(3 + d) * CELL_STRIDE + j];
                    }
                };
                if (MODE != PASS_STEP || sizeof(T) != 4) {   // FP64: one at a time (registers)
                    for (int i = i0; i < i1; ++i) {
                        const int j0 = i - lo;
                        if (!PIC_INDEX_OK(j0, CELL_CHUNK, p.status)) break;
                        const int j = cell_slot(j0);
                        T f[3], u[3];
                        load(j, f, u);
                        one(j, st_cell[j], f[0], f[1], f[2], u[0], u[1], u[2], false);
                    }
                } else {
                    // Particles two at a time: a pair at rest in the home cell through both
                    // half drifts (the common case on a Galilean grid) runs as two independent
                    // instruction streams; any other particle takes the general path. The
                    // second member of an odd tail repeats the first with zero charge and is
                    // not stored. Per accumulator the additions come in particle order, as
                    // one at a time.
                    for (int i = i0; i < i1; i += 2) {
                        const bool has1 = i + 1 < i1;
                        const int ja0 = i - lo, jb0 = (has1 ? i + 1 : i) - lo;
                        if (!(PIC_INDEX_OK(ja0, CELL_CHUNK, p.status) && PIC_INDEX_OK(jb0, CELL_CHUNK, p.status))) break;
                        const int j[2] = {cell_slot(ja0), cell_slot(jb0)};
                        const int c[2] = {st_cell[j[0]], st_cell[j[1]]};
                        T f[2][3], u[2][3];
                        load(j[0], f[0], u[0]);
                        load(j[1], f[1], u[1]);
                        if (c[0] != home || c[1] != home) {
                            one(j[0], c[0], f[0][0], f[0][1], f[0][2], u[0][0], u[0][1], u[0][2], false);
                            if (has1) one(j[1], c[1], f[1][0], f[1][1], f[1][2], u[1][0], u[1][1], u[1][2], false);
                            continue;
                        }
                        int gbase = hbase;
#ifdef PIC_CHECKED
                        gbase += p.inject;
                        if (!PIC_INDEX_OK(gbase, R - (TE * TE + TE + 1), p.status)) gbase = 0;
#endif
                        T g1[2][3], g2[2][3];
                        bool stay = true;
#pragma unroll
                        for (int k = 0; k < 2; ++k) {
                            T wx[2], wy[2], wz[2], E[3], B[3];
                            SH::w(f[k][0], wx);
                            SH::w(f[k][1], wy);
                            SH::w(f[k][2], wz);
                            gather2<T, TE>(tile, gbase, wx, wy, wz, E, B);
                            boris_push(qdt2m, E, B, inv_c2, u[k][0], u[k][1], u[k][2]);
                            const T igam = boris_rsqrt((T)1 + (u[k][0] * u[k][0] + u[k][1] * u[k][1] +
                                                                u[k][2] * u[k][2]) * inv_c2);
#pragma unroll
                            for (int d = 0; d < 3; ++d) {
                                const T dd = (u[k][d] * igam - vg[d]) * hd[d];
                                g1[k][d] = f[k][d] + dd;
                                g2[k][d] = g1[k][d] + dd;
                                stay = stay && g1[k][d] >= (T)0 && g1[k][d] < (T)1 && g2[k][d] >= (T)0 &&
                                       g2[k][d] < (T)1;
                            }
                        }
                        if (!stay) {
                            one(j[0], c[0], f[0][0], f[0][1], f[0][2], u[0][0], u[0][1], u[0][2], true);
                            if (has1) one(j[1], c[1], f[1][0], f[1][1], f[1][2], u[1][0], u[1][1], u[1][2], true);
                            continue;
                        }
#pragma unroll
                        for (int k = 0; k < 2; ++k) {
                            const T qk = (k == 0 || has1) ? qw_dv : (T)0;
                            const T igam = boris_rsqrt((T)1 + (u[k][0] * u[k][0] + u[k][1] * u[k][1] +
                                                                u[k][2] * u[k][2]) * inv_c2);
                            const T qv[3] = {qk * (u[k][0] * igam), qk * (u[k][1] * igam), qk * (u[k][2] * igam)};
                            T wx[2], wy[2], wz[2];
                            SH::w(g1[k][0], wx);
                            SH::w(g1[k][1], wy);
                            SH::w(g1[k][2], wz);
                            const P2 qxy = Pair<T>::make(qv[0], qv[1]);
#pragma unroll
                            for (int a = 0; a < 2; ++a)
#pragma unroll
                                for (int bb = 0; bb < 2; ++bb) {
                                    const T wxy = wx[a] * wy[bb];
#pragma unroll
                                    for (int cc = 0; cc < 2; ++cc) {
                                        const T w = wxy * wz[cc];
                                        const int n = (a * 2 + bb) * 2 + cc;
                                        aJ[n] = pfma(Pair<T>::make(w, w), qxy, aJ[n]);
                                        aZ[n] = fma(w, qv[2], aZ[n]);
                                    }
                                }
                        }
#pragma unroll
                        for (int k = 0; k < 2; ++k) {
                            const T qk = (k == 0 || has1) ? qw_dv : (T)0;
                            T wx[2], wy[2], wz[2];
                            SH::w(g2[k][0], wx);
                            SH::w(g2[k][1], wy);
                            SH::w(g2[k][2], wz);
#pragma unroll
                            for (int a = 0; a < 2; ++a)
#pragma unroll
                                for (int bb = 0; bb < 2; ++bb) {
                                    const T wxy = wx[a] * wy[bb];
#pragma unroll
                                    for (int cc = 0; cc < 2; ++cc)
                                        aR[(a * 2 + bb) * 2 + cc] = fma(wxy * wz[cc], qk, aR[(a * 2 + bb) * 2 + cc]);
                                }
                        }
#pragma unroll
                        for (int k = 0; k < 2; ++k) {
                            if (k == 1 && !has1) break;
#pragma unroll
                            for (int d = 0; d < 3; ++d) {
                                st_v[d * CELL_STRIDE + j[k]] = g2[k][d];
                                st_v[(3 + d) * CELL_STRIDE + j[k]] = u[k][d];
                            }
                        }
                    }
                }
                __syncwarp();
                if (MODE == PASS_STEP) {   // stage out, coalesced; the cells only if one changed
                    const bool any_moved = __any_sync(0xffffffffu, moved);
                    for (int j = lane; j < hi - lo; j += 32) {
                        const int q = cell_slot(j);
                        if (any_moved) sp.cell[lo + j] = st_cell[q];
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            sp.off[d][lo + j] = st_v[d * CELL_STRIDE + q];
                            sp.u[d][lo + j] = st_v[(3 + d) * CELL_STRIDE + q];
                        }
                    }
                }
                __syncwarp();
            }
        }
        // the cell's accumulated nodes, once (neighbouring lanes are neighbouring cells along
        // z, so one node index per instruction never makes two lanes meet)
#pragma unroll
        for (int n = 0; n < 8; ++n) {
            const int a = n >> 2, bb = (n >> 1) & 1, cc = n & 1;
            const int idx = hbase + (a * TE + bb) * TE + cc;
            if (aJ[n].x != (T)0) atomicAdd(&sD[0 * R + idx], aJ[n].x);
            if (aJ[n].y != (T)0) atomicAdd(&sD[1 * R + idx], aJ[n].y);
            if (aZ[n] != (T)0) atomicAdd(&sD[2 * R + idx], aZ[n]);
            if (aR[n] != (T)0) atomicAdd(&sD[3 * R + idx], aR[n]);
        }
    }
    __syncthreads();

    // add the tile to the global source grids
    for (int idx = threadIdx.x; idx < R; idx += blockDim.x) {
        const int rx = idx / (TE * TE);
        const int rem = idx - rx * (TE * TE);
        const int ry = rem / TE;
        const int rz = rem - ry * TE;
        int64_t g = ((int64_t)wrap_near(ox + rx, p.nx) * p.ny + wrap_near(oy + ry, p.ny)) * p.nz +
                    wrap_near(oz + rz, p.nz);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            T v = sD[q * R + idx];
            if (v != (T)0) atomicAdd(&p.S[q * N + g], v);
        }
    }
    if (MODE == PASS_STEP) {
        for (int o = 16; o > 0; o >>= 1) {
            miss += __shfl_down_sync(0xffffffffu, miss, o);
            far += __shfl_down_sync(0xffffffffu, far, o);
        }
        if (lane == 0) {
            if (miss) atomicAdd(&p.cnt[CNT_HOME_MISS], miss);
            if (far) atomicAdd(&p.cnt[CNT_FAR], far);
        }
    }
}

template <typename T, int MODE, int MARGIN>
__global__ void __launch_bounds__(CELL_THREADS, 2) cell_pass_kernel(PassK<T> p) {
    cell_pass_body<T, MODE, MARGIN>(p, blockIdx.x);
}

// One CTA per bin. FP32 linear passes and FP32 grouped quadratic/cubic steps at tile
// margin 0 fit three CTAs per SM by shared memory and have their registers held to
// that; row-deposit and combined J and rho passes are held to two; the others are left
// to the compiler.
template <typename T, int ORDER, int MODE, int MARGIN, int DEP, bool MIX>
__global__ void __launch_bounds__(PASS_THREADS) particle_pass_kernel(PassK<T> p) {
    particle_pass_body<T, ORDER, MODE, MARGIN, DEP, MIX>(p, blockIdx.x);
}

template <typename T, int ORDER, int MODE, int MARGIN, int DEP, bool MIX>
__global__ void __launch_bounds__(PASS_THREADS, 3) particle_pass_kernel_3(PassK<T> p) {
    particle_pass_body<T, ORDER, MODE, MARGIN, DEP, MIX>(p, blockIdx.x);
}

template <typename T, int ORDER, int MODE, int MARGIN, int DEP, bool MIX>
__global__ void __launch_bounds__(PASS_THREADS, 2) particle_pass_kernel_2(PassK<T> p) {
    particle_pass_body<T, ORDER, MODE, MARGIN, DEP, MIX>(p, blockIdx.x);
}

// Parameters of a run's particle pass. F, S and S64 default to the run's own grids;
// shared launches over several runs point them at a staging area instead.
template <typename T>
void fill_passk(const pic_sim* s, PassK<T>& p, const void* F = nullptr, void* S = nullptr,
                long long* S64 = nullptr) {
    const pic_config& c = s->cfg;
    memset(&p, 0, sizeof(p));
    p.F = (const T*)(F ? F : s->F);
    p.S = (T*)(S ? S : s->S);
    p.S64 = S64 ? S64 : s->S64;
    p.inv_delta = (T)ldexp(1.0, -s->fix_exp);
    p.N = s->d.N;
    p.nx = s->d.nx;
    p.ny = s->d.ny;
    p.nz = s->d.nz;
    p.nbx = s->d.nbx;
    p.nby = s->d.nby;
    p.nbz = s->d.nbz;
    p.div_nynz.init((uint32_t)(s->d.ny * s->d.nz));
    p.div_nz.init((uint32_t)s->d.nz);
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
        p.sp[k].cell_start = sp.cell_start;
        p.sp[k].n = (int32_t)sp.n;
        p.sp[k].qw_dv = (T)(sp.q * sp.w / dV);
        p.sp[k].qdt2m = (T)(sp.q * c.dt / (2.0 * sp.m));
    }
    p.cnt = s->cnt;
    p.status = s->status;
    p.inject = s->inject;
}

// Shared launches over several runs of one shape class: one CTA per (run, bin), the run's
// parameters copied from a table in device memory into shared memory first.
template <typename T>
__device__ __forceinline__ void load_passk(PassK<T>& dst, const PassK<T>* src) {
    static_assert(sizeof(PassK<T>) % 4 == 0, "PassK is copied as 32-bit words");
    const int* a = reinterpret_cast<const int*>(src);
    int* d = reinterpret_cast<int*>(&dst);
    for (int i = threadIdx.x; i < (int)(sizeof(PassK<T>) / 4); i += blockDim.x) d[i] = a[i];
}

template <typename T, int ORDER, int MODE, int MARGIN, int DEP, bool MIX, int MINB>
__global__ void __launch_bounds__(PASS_THREADS, MINB)
    particle_pass_many_kernel(const PassK<T>* __restrict__ descs, int nbins) {
    __shared__ __align__(16) PassK<T> P;
    const int run = blockIdx.x / nbins;
    load_passk(P, descs + run);
    __syncthreads();
    particle_pass_body<T, ORDER, MODE, MARGIN, DEP, MIX>(P, blockIdx.x - run * nbins);
}

template <typename T, int MODE, int MARGIN>
__global__ void __launch_bounds__(CELL_THREADS, 2) cell_pass_many_kernel(const PassK<T>* __restrict__ descs,
                                                                        int nbins) {
    __shared__ __align__(16) PassK<T> P;
    const int run = blockIdx.x / nbins;
    load_passk(P, descs + run);
    __syncthreads();
    cell_pass_body<T, MODE, MARGIN>(P, blockIdx.x - run * nbins);
}

// A shared launch: `descs` (device) holds `nruns` parameter blocks.
struct ManyLaunch {
    const void* descs;
    int nruns;
};

template <typename T, int ORDER, int MODE, int MARGIN, int DEP, bool MIX = false>
int pass_launch(pic_sim* s, cudaStream_t st, const ManyLaunch* many) {
    const PassSmem L(TileGeom<Shape<ORDER>::NW, MARGIN>::R, Shape<ORDER>::NW, sizeof(T), MODE == PASS_STEP, DEP);
    // FP32 grouped quadratic/cubic steps at tile margin 0 (70 KB of shared memory) run
    // three CTAs per SM: registers held to 80 (a few spill) and the largest shared
    // memory carve-out; measured 48.1 against 51.2 ms at two CTAs on the 256x256x512
    // cubic plasma.
    constexpr bool three = sizeof(T) == 4 && ORDER >= 2 && MARGIN == 0 && DEP == DEP_GROUP &&
                           MODE == PASS_STEP;
    constexpr int MINB = (DEP == DEP_CELL) ? 2
                         : (sizeof(T) == 4 && (ORDER == 1 || three) && DEP != DEP_FIXED) ? 3
                         : (DEP == DEP_ROW || DEP == DEP_ROWU || DEP == DEP_JR) ? 2 : 1;
    const int threads = DEP == DEP_CELL ? CELL_THREADS : PASS_THREADS;
    if (many) {
        void (*kern)(const PassK<T>*, int);
        if constexpr (DEP == DEP_CELL)
            kern = cell_pass_many_kernel<T, MODE, MARGIN>;
        else
            kern = particle_pass_many_kernel<T, ORDER, MODE, MARGIN, DEP, MIX, MINB>;
        GP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total));
        if constexpr (three)
            GP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
        kern<<<(unsigned)s->d.nbins * (unsigned)many->nruns, threads, L.total, st>>>(
            (const PassK<T>*)many->descs, s->d.nbins);
        GP_CUDA(cudaGetLastError());
        return PIC_OK;
    }
    PassK<T> p;
    fill_passk<T>(s, p);
    void (*kern)(PassK<T>);
    if constexpr (DEP == DEP_CELL) {
        static_assert(ORDER == 1, "one thread per cell: linear shapes only");
        kern = cell_pass_kernel<T, MODE, MARGIN>;
    } else if constexpr (MINB == 3)
        kern = particle_pass_kernel_3<T, ORDER, MODE, MARGIN, DEP, MIX>;
    else if constexpr (MINB == 2)
        kern = particle_pass_kernel_2<T, ORDER, MODE, MARGIN, DEP, MIX>;
    else
        kern = particle_pass_kernel<T, ORDER, MODE, MARGIN, DEP, MIX>;
    GP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total));
    if constexpr (three)
        GP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    kern<<<s->d.nbins, threads, L.total, st>>>(p);
    GP_CUDA(cudaGetLastError());
    return PIC_OK;
}

// Deposit variant a run's pass uses (strategy, and whether two equal species share groups):
// runs advanced by one shared launch must agree on it.
inline int pass_variant(const pic_sim* s) {
    const bool mix = s->nspecies == 2 && s->sp[0].n == s->sp[1].n;
    if (s->cfg.deterministic) return DEP_FIXED;
    if (s->cfg.shape_order == 1) return s->cfg.deposit == DEP_CELL ? DEP_CELL : DEP_GROUP;
    if (s->cfg.precision != 32) return DEP_GROUP;
    if (s->cfg.deposit == DEP_ROW || s->cfg.deposit == DEP_ROWU) return s->cfg.deposit;
    const int d = s->cfg.deposit == DEP_JR ? DEP_JR : DEP_GROUP;
    return d + (mix ? 16 : 0);
}

template <typename T, int ORDER, int MODE, int MARGIN>
int pass_strategy(pic_sim* s, cudaStream_t st, const ManyLaunch* many) {
    if (s->cfg.deterministic) return pass_launch<T, ORDER, MODE, MARGIN, DEP_FIXED>(s, st, many);
    if constexpr (sizeof(T) == 4) {
        if (s->cfg.deposit == DEP_ROW) return pass_launch<T, ORDER, MODE, MARGIN, DEP_ROW>(s, st, many);
        if (s->cfg.deposit == DEP_ROWU) return pass_launch<T, ORDER, MODE, MARGIN, DEP_ROWU>(s, st, many);
        // two species of equal size (the neutral plasmas): one group per cell for both
        const bool mix = MODE == PASS_STEP && s->nspecies == 2 && s->sp[0].n == s->sp[1].n;
        if (s->cfg.deposit == DEP_JR) {
            if constexpr (MODE == PASS_STEP) {
                if (mix) return pass_launch<T, ORDER, MODE, MARGIN, DEP_JR, true>(s, st, many);
                return pass_launch<T, ORDER, MODE, MARGIN, DEP_JR>(s, st, many);
            }
        }
        if constexpr (MODE == PASS_STEP) {
            if (mix) return pass_launch<T, ORDER, MODE, MARGIN, DEP_GROUP, true>(s, st, many);
        }
    }
    return pass_launch<T, ORDER, MODE, MARGIN, DEP_GROUP>(s, st, many);
}

template <typename T, int MODE, int MARGIN>
int pass_order(pic_sim* s, cudaStream_t st, const ManyLaunch* many) {
    switch (s->cfg.shape_order) {
        case 1:
            if (s->cfg.deterministic) return pass_launch<T, 1, MODE, MARGIN, DEP_FIXED>(s, st, many);
            if (s->cfg.deposit == DEP_CELL) return pass_launch<T, 1, MODE, MARGIN, DEP_CELL>(s, st, many);
            return pass_launch<T, 1, MODE, MARGIN, DEP_GROUP>(s, st, many);
        case 2: return pass_strategy<T, 2, MODE, MARGIN>(s, st, many);
        default: return pass_strategy<T, 3, MODE, MARGIN>(s, st, many);
    }
}

template <typename T, int MODE>
int pass_margin(pic_sim* s, cudaStream_t st, const ManyLaunch* many = nullptr) {
    return s->d.margin == 0 ? pass_order<T, MODE, 0>(s, st, many) : pass_order<T, MODE, 1>(s, st, many);
}

}  // namespace

}  // namespace galpic
