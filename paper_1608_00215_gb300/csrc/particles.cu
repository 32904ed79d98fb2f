// Particle-side kernels of the Galilean-PSATD step other than the pass itself:
//   * generate       - regular lattice plus seeded jitter (splitmix64 counters);
//   * sanitize       - clamp out-of-range loaded particles and flag them;
//   * sort           - counting sort of each species by cell, cells numbered bin by
//                      bin (bins of BX*BY*BZ cells), executed only when the device
//                      counters ask for it. Particles of one cell are contiguous, and
//                      the cells of a bin form one contiguous range.
// The particle pass is in pass.cuh (instantiated by pass_fp32.cu, pass_fp64.cu).
#include <algorithm>

#include "pass.cuh"

namespace galpic {

namespace {

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
// Cell sort (runs only when sort_needed(cnt)). Key of a cell: its bin times
// BX*BY*BZ plus its index inside the bin, so every bin is one key range.
// ---------------------------------------------------------------------------
struct BinGeom {
    int ny, nz, BX, BY, BZ, nby, nbz;
    __device__ __forceinline__ int key_of(int c) const {
        int ix = c / (ny * nz);
        int rem = c - ix * (ny * nz);
        int iy = rem / nz;
        int iz = rem - iy * nz;
        int b = ((ix / BX) * nby + iy / BY) * nbz + iz / BZ;
        int l = ((ix % BX) * BY + iy % BY) * BZ + iz % BZ;
        return b * (BX * BY * BZ) + l;
    }
};

constexpr int SCAN_THREADS = 1024, SCAN_ITEMS = 8, SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ void sort_zero_body(int32_t* key_cnt, int64_t K, const unsigned long long* cnt) {
    if (!sort_needed(cnt)) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < K;
         i += (int64_t)gridDim.x * blockDim.x)
        key_cnt[i] = 0;
}

__device__ __forceinline__ void sort_count_body(const int32_t* __restrict__ cell, int64_t n, int32_t* rank,
                                                int32_t* key_cnt, BinGeom g, const unsigned long long* cnt,
                                                int64_t K, int32_t* status) {
    if (!sort_needed(cnt)) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int key = g.key_of(cell[i]);
        if (!PIC_INDEX_OK(key, K, status)) continue;
        rank[i] = atomicAdd(&key_cnt[key], 1);
    }
}

// Block-wide exclusive scan of one value per thread (1024 threads); returns the
// thread's exclusive prefix and writes the block total to *total.
__device__ int32_t block_exclusive_scan(int32_t v, int32_t* sh, int32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int32_t w = sh[lane];
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        sh[lane] = w;
    }
    __syncthreads();
    int32_t before = (warp > 0 ? sh[warp - 1] : 0) + x - v;
    if (total) *total = sh[31];
    __syncthreads();
    return before;
}

// pass A: per-tile sums of the key counts
__device__ __forceinline__ void scan_tiles_body(const int32_t* key_cnt, int64_t K, int32_t* tile_sum,
                                                const unsigned long long* cnt) {
    if (!sort_needed(cnt)) return;
    __shared__ int32_t sh[32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    int32_t s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j)
        if (base + j < K) s += key_cnt[base + j];
    int32_t tot;
    block_exclusive_scan(s, sh, &tot);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = tot;
}

// pass B: exclusive scan of the tile sums (one block)
__device__ __forceinline__ void scan_sums_body(int32_t* tile_sum, int nt, const unsigned long long* cnt) {
    if (!sort_needed(cnt)) return;
    __shared__ int32_t sh[32];
    const int per = (nt + SCAN_THREADS - 1) / SCAN_THREADS;
    const int lo = threadIdx.x * per, hi = min(nt, lo + per);
    int32_t s = 0;
    for (int i = lo; i < hi; ++i) s += tile_sum[i];
    int32_t run = block_exclusive_scan(s, sh, nullptr);
    for (int i = lo; i < hi; ++i) {
        int32_t v = tile_sum[i];
        tile_sum[i] = run;
        run += v;
    }
}

// pass C: exclusive key starts (cell_start, with cell_start[K] = n); the start of every
// bin's first key goes to bin_start
__device__ __forceinline__ void scan_write_body(const int32_t* key_cnt, int64_t K, const int32_t* tile_sum,
                                                int32_t* cell_start, int32_t* bin_start, int bxyz, int nbins,
                                                int64_t n, const unsigned long long* cnt) {
    if (!sort_needed(cnt)) return;
    __shared__ int32_t sh[32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    int32_t v[SCAN_ITEMS];
    int32_t s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        v[j] = (base + j < K) ? key_cnt[base + j] : 0;
        s += v[j];
    }
    int32_t run = block_exclusive_scan(s, sh, nullptr) + tile_sum[blockIdx.x];
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        const int64_t k = base + j;
        if (k < K) {
            cell_start[k] = run;
            if (k % bxyz == 0) bin_start[k / bxyz] = run;
        }
        run += v[j];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        bin_start[nbins] = (int32_t)n;
        cell_start[K] = (int32_t)n;
    }
}

template <typename T>
struct Ptr6 {
    T* p[6];
};

template <typename T>
__device__ __forceinline__ void sort_scatter_body(const int32_t* __restrict__ cell, Ptr6<T> src, int64_t n,
                                                  const int32_t* __restrict__ rank,
                                                  const int32_t* __restrict__ cell_start, int32_t* tcell,
                                                  Ptr6<T> dst, BinGeom g, const unsigned long long* cnt,
                                                  int32_t* status) {
    if (!sort_needed(cnt)) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int c = cell[i];
        int64_t j = (int64_t)cell_start[g.key_of(c)] + rank[i];
        if (!PIC_INDEX_OK(j, n, status)) continue;
        tcell[j] = c;
#pragma unroll
        for (int q = 0; q < 6; ++q) dst.p[q][j] = src.p[q][i];
    }
}

template <typename T>
__device__ __forceinline__ void sort_copyback_body(int32_t* cell, Ptr6<T> dst, int64_t n,
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

__global__ void sort_zero_kernel(int32_t* key_cnt, int64_t K, const unsigned long long* cnt) {
    sort_zero_body(key_cnt, K, cnt);
}
__global__ void sort_count_kernel(const int32_t* __restrict__ cell, int64_t n, int32_t* rank, int32_t* key_cnt,
                                  BinGeom g, const unsigned long long* cnt, int64_t K, int32_t* status) {
    sort_count_body(cell, n, rank, key_cnt, g, cnt, K, status);
}
__global__ void __launch_bounds__(SCAN_THREADS) scan_tiles_kernel(const int32_t* key_cnt, int64_t K,
                                                                  int32_t* tile_sum,
                                                                  const unsigned long long* cnt) {
    scan_tiles_body(key_cnt, K, tile_sum, cnt);
}
__global__ void __launch_bounds__(SCAN_THREADS) scan_sums_kernel(int32_t* tile_sum, int nt,
                                                                 const unsigned long long* cnt) {
    scan_sums_body(tile_sum, nt, cnt);
}
__global__ void __launch_bounds__(SCAN_THREADS) scan_write_kernel(const int32_t* key_cnt, int64_t K,
                                                                  const int32_t* tile_sum, int32_t* cell_start,
                                                                  int32_t* bin_start, int bxyz, int nbins,
                                                                  int64_t n, const unsigned long long* cnt) {
    scan_write_body(key_cnt, K, tile_sum, cell_start, bin_start, bxyz, nbins, n, cnt);
}
template <typename T>
__global__ void sort_scatter_kernel(const int32_t* __restrict__ cell, Ptr6<T> src, int64_t n,
                                    const int32_t* __restrict__ rank, const int32_t* __restrict__ cell_start,
                                    int32_t* tcell, Ptr6<T> dst, BinGeom g, const unsigned long long* cnt,
                                    int32_t* status) {
    sort_scatter_body<T>(cell, src, n, rank, cell_start, tcell, dst, g, cnt, status);
}
template <typename T>
__global__ void sort_copyback_kernel(int32_t* cell, Ptr6<T> dst, int64_t n, const int32_t* __restrict__ tcell,
                                     Ptr6<T> src, const unsigned long long* cnt) {
    sort_copyback_body<T>(cell, dst, n, tcell, src, cnt);
}

// ---- re-sort checks of several runs in shared launches (pic_step_many) ----------
// One descriptor per run for one species slot; blockIdx.y picks the run. Every run of
// a shared launch has the same grid (K, tiles, bin geometry); particle counts differ.
template <typename T>
struct SortDesc {
    int32_t* cell;
    Ptr6<T> own, tmp;
    int32_t* tcell;
    int32_t* rank;
    int32_t* key_cnt;
    int32_t* tile_sum;
    int32_t* bin_start;
    int32_t* cell_start;
    const unsigned long long* cnt;
    int32_t* status;
    int64_t n, K;
    BinGeom g;
    int nt, bxyz, nbins, pad;
};

template <typename T>
__global__ void sort_zero_many(const SortDesc<T>* __restrict__ d) {
    const SortDesc<T>& r = d[blockIdx.y];
    sort_zero_body(r.key_cnt, r.K, r.cnt);
}
template <typename T>
__global__ void sort_count_many(const SortDesc<T>* __restrict__ d) {
    const SortDesc<T>& r = d[blockIdx.y];
    sort_count_body(r.cell, r.n, r.rank, r.key_cnt, r.g, r.cnt, r.K, r.status);
}
template <typename T>
__global__ void __launch_bounds__(SCAN_THREADS) scan_tiles_many(const SortDesc<T>* __restrict__ d) {
    const SortDesc<T>& r = d[blockIdx.y];
    scan_tiles_body(r.key_cnt, r.K, r.tile_sum, r.cnt);
}
template <typename T>
__global__ void __launch_bounds__(SCAN_THREADS) scan_sums_many(const SortDesc<T>* __restrict__ d) {
    const SortDesc<T>& r = d[blockIdx.y];
    scan_sums_body(r.tile_sum, r.nt, r.cnt);
}
template <typename T>
__global__ void __launch_bounds__(SCAN_THREADS) scan_write_many(const SortDesc<T>* __restrict__ d) {
    const SortDesc<T>& r = d[blockIdx.y];
    scan_write_body(r.key_cnt, r.K, r.tile_sum, r.cell_start, r.bin_start, r.bxyz, r.nbins, r.n, r.cnt);
}
template <typename T>
__global__ void sort_scatter_many(const SortDesc<T>* __restrict__ d) {
    const SortDesc<T>& r = d[blockIdx.y];
    sort_scatter_body<T>(r.cell, r.own, r.n, r.rank, r.cell_start, r.tcell, r.tmp, r.g, r.cnt, r.status);
}
template <typename T>
__global__ void sort_copyback_many(const SortDesc<T>* __restrict__ d) {
    const SortDesc<T>& r = d[blockIdx.y];
    sort_copyback_body<T>(r.cell, r.own, r.n, r.tcell, r.tmp, r.cnt);
}

// Per run (one thread each): count a performed re-sort and clear its request, then clear
// the stray counts that the coming pass accumulates.
__global__ void sort_finish_many_kernel(unsigned long long* const* __restrict__ cnts, int nruns) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nruns) return;
    unsigned long long* cnt = cnts[r];
    if (sort_needed(cnt)) {
        cnt[CNT_FORCE_SORT] = 0ull;
        cnt[CNT_SORTS] += 1ull;
    }
    cnt[CNT_HOME_MISS] = 0ull;
    cnt[CNT_FAR] = 0ull;
}

// Copies listed in device memory: blockIdx.y picks the copy; 16-byte words when both
// addresses and the length allow it, else 4-byte words (every buffer holds 4- or 8-byte
// values, so its address and length are multiples of 4).
__global__ void copy_many_kernel(const CopyDesc* __restrict__ d) {
    const CopyDesc c = d[blockIdx.y];
    const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
    if ((((uintptr_t)c.dst | (uintptr_t)c.src | (uintptr_t)c.bytes) & 15) == 0) {
        const int64_t n = (int64_t)(c.bytes / 16);
        const uint4* src = (const uint4*)c.src;
        uint4* dst = (uint4*)c.dst;
        for (int64_t i = i0; i < n; i += stride) dst[i] = src[i];
    } else {
        const int64_t n = (int64_t)(c.bytes / 4);
        const uint32_t* src = (const uint32_t*)c.src;
        uint32_t* dst = (uint32_t*)c.dst;
        for (int64_t i = i0; i < n; i += stride) dst[i] = src[i];
    }
}

template <typename T>
__global__ void fixed_to_real_many_kernel(const long long* __restrict__ S64, T* __restrict__ S, int64_t n,
                                          const int* __restrict__ e) {
    const int r = blockIdx.y;
    const long long* a = S64 + (int64_t)r * n;
    T* b = S + (int64_t)r * n;
    const int er = e[r];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (T)ldexp((double)a[i], er);
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

// Deterministic mode: real sources from their fixed-point sums, S = delta * S64 (the
// integer to FP64, exact scaling by the power of two delta, then the run's precision).
template <typename T>
__global__ void fixed_to_real_kernel(const long long* __restrict__ S64, T* __restrict__ S, int64_t n, int e) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        S[i] = (T)ldexp((double)S64[i], e);
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
    const int bxyz = s->d.BX * s->d.BY * s->d.BZ;
    const int64_t K = (int64_t)s->d.nbins * bxyz;
    const int nt = (int)((K + SCAN_TILE - 1) / SCAN_TILE);
    Ptr6<T> tmp;
    for (int d = 0; d < 3; ++d) {
        tmp.p[d] = (T*)s->tmp_off[d];
        tmp.p[3 + d] = (T*)s->tmp_u[d];
    }
    for (int k = 0; k < s->nspecies; ++k) {
        SpeciesDev& sp = s->sp[k];
        if (sp.n == 0) continue;
        sort_zero_kernel<<<grid_for(K, 256), 256, 0, st>>>(s->key_cnt, K, s->cnt);
        sort_count_kernel<<<grid_for(sp.n, 256), 256, 0, st>>>(sp.cell, sp.n, s->tmp_rank,
                                                               s->key_cnt, g, s->cnt, K, s->status);
        scan_tiles_kernel<<<nt, SCAN_THREADS, 0, st>>>(s->key_cnt, K, s->tile_sum, s->cnt);
        scan_sums_kernel<<<1, SCAN_THREADS, 0, st>>>(s->tile_sum, nt, s->cnt);
        scan_write_kernel<<<nt, SCAN_THREADS, 0, st>>>(s->key_cnt, K, s->tile_sum, sp.cell_start,
                                                       sp.bin_start, bxyz, s->d.nbins, sp.n, s->cnt);
        Ptr6<T> own;
        for (int d = 0; d < 3; ++d) {
            own.p[d] = (T*)sp.off[d];
            own.p[3 + d] = (T*)sp.u[d];
        }
        sort_scatter_kernel<T><<<grid_for(sp.n, 256), 256, 0, st>>>(
            sp.cell, own, sp.n, s->tmp_rank, sp.cell_start, s->tmp_cell, tmp, g, s->cnt, s->status);
        sort_copyback_kernel<T><<<grid_for(sp.n, 256), 256, 0, st>>>(sp.cell, own, sp.n,
                                                                     s->tmp_cell, tmp, s->cnt);
    }
    sort_finish_kernel<<<1, 1, 0, st>>>(s->cnt);
    GP_CUDA(cudaGetLastError());
    return PIC_OK;
}

}  // namespace

size_t tile_bytes(const pic_config& c, const Dims& d, int mode) {
    int nw = c.shape_order == 1 ? 2 : 4;
    int e = BIN + nw - 1 + 2 * d.margin;
    const int dep = c.deterministic ? DEP_FIXED
                    : (c.deposit == DEP_CELL && c.shape_order != 1) ? DEP_GROUP : c.deposit;
    return PassSmem(e * e * e, nw, c.precision == 64 ? 8 : 4, mode == PASS_STEP, dep).total;
}

int64_t sort_keys(const Dims& d) { return (int64_t)d.nbins * d.BX * d.BY * d.BZ; }

int64_t sort_tiles(const Dims& d) { return (sort_keys(d) + SCAN_TILE - 1) / SCAN_TILE; }

int launch_particle_pass(pic_sim* s, int mode, cudaStream_t st) {
    return s->cfg.precision == 64 ? launch_pass_fp64(s, mode, st) : launch_pass_fp32(s, mode, st);
}

size_t sort_desc_bytes(int precision) {
    return precision == 64 ? sizeof(SortDesc<double>) : sizeof(SortDesc<float>);
}

template <typename T>
static void fill_sort_desc_t(const pic_sim* s, int k, SortDesc<T>& r) {
    memset(&r, 0, sizeof(r));
    const SpeciesDev& sp = s->sp[k];
    r.cell = sp.cell;
    for (int d = 0; d < 3; ++d) {
        r.own.p[d] = (T*)sp.off[d];
        r.own.p[3 + d] = (T*)sp.u[d];
        r.tmp.p[d] = (T*)s->tmp_off[d];
        r.tmp.p[3 + d] = (T*)s->tmp_u[d];
    }
    r.tcell = s->tmp_cell;
    r.rank = s->tmp_rank;
    r.key_cnt = s->key_cnt;
    r.tile_sum = s->tile_sum;
    r.bin_start = sp.bin_start;
    r.cell_start = sp.cell_start;
    r.cnt = s->cnt;
    r.status = s->status;
    r.n = sp.n;
    r.K = sort_keys(s->d);
    r.g = BinGeom{s->d.ny, s->d.nz, s->d.BX, s->d.BY, s->d.BZ, s->d.nby, s->d.nbz};
    r.nt = (int)sort_tiles(s->d);
    r.bxyz = s->d.BX * s->d.BY * s->d.BZ;
    r.nbins = s->d.nbins;
}

void fill_sort_desc(const pic_sim* s, int k, void* out) {
    if (s->cfg.precision == 64)
        fill_sort_desc_t<double>(s, k, *static_cast<SortDesc<double>*>(out));
    else
        fill_sort_desc_t<float>(s, k, *static_cast<SortDesc<float>*>(out));
}

template <typename T>
static int sort_many_t(const pic_sim* s0, const SortDesc<T>* d, int nruns, int64_t nmax, cudaStream_t st) {
    const int64_t K = sort_keys(s0->d);
    const int nt = (int)sort_tiles(s0->d);
    const int gk = std::max(1, grid_for(K, 256) / std::max(1, std::min(nruns, 8)));
    const int gn = std::max(1, grid_for(nmax, 256) / std::max(1, std::min(nruns, 8)));
    sort_zero_many<T><<<dim3(gk, nruns), 256, 0, st>>>(d);
    sort_count_many<T><<<dim3(gn, nruns), 256, 0, st>>>(d);
    scan_tiles_many<T><<<dim3(nt, nruns), SCAN_THREADS, 0, st>>>(d);
    scan_sums_many<T><<<dim3(1, nruns), SCAN_THREADS, 0, st>>>(d);
    scan_write_many<T><<<dim3(nt, nruns), SCAN_THREADS, 0, st>>>(d);
    sort_scatter_many<T><<<dim3(gn, nruns), 256, 0, st>>>(d);
    sort_copyback_many<T><<<dim3(gn, nruns), 256, 0, st>>>(d);
    GP_CUDA(cudaGetLastError());
    return PIC_OK;
}

int launch_sort_many(const pic_sim* s0, const void* descs, int nruns, int64_t nmax, cudaStream_t st) {
    if (s0->cfg.precision == 64) return sort_many_t<double>(s0, (const SortDesc<double>*)descs, nruns, nmax, st);
    return sort_many_t<float>(s0, (const SortDesc<float>*)descs, nruns, nmax, st);
}

int launch_sort_finish_many(unsigned long long* const* cnts_dev, int nruns, cudaStream_t st) {
    sort_finish_many_kernel<<<(nruns + 127) / 128, 128, 0, st>>>(cnts_dev, nruns);
    GP_CUDA(cudaGetLastError());
    return PIC_OK;
}

int launch_copy_many(const CopyDesc* descs_dev, int n, size_t max_bytes, cudaStream_t st) {
    if (n <= 0) return PIC_OK;
    const int g = std::max(1, grid_for((int64_t)(max_bytes / 16), 256) / std::max(1, std::min(n, 16)));
    copy_many_kernel<<<dim3(g, n), 256, 0, st>>>(descs_dev);
    GP_CUDA(cudaGetLastError());
    return PIC_OK;
}

int launch_fixed_to_real_many(const long long* S64, void* S, int64_t n, const int* e_dev, int nruns,
                              int precision, cudaStream_t st) {
    const int g = std::max(1, grid_for(n, 256) / std::max(1, std::min(nruns, 16)));
    if (precision == 64)
        fixed_to_real_many_kernel<double><<<dim3(g, nruns), 256, 0, st>>>(S64, (double*)S, n, e_dev);
    else
        fixed_to_real_many_kernel<float><<<dim3(g, nruns), 256, 0, st>>>(S64, (float*)S, n, e_dev);
    GP_CUDA(cudaGetLastError());
    return PIC_OK;
}

int launch_fixed_to_real(pic_sim* s, cudaStream_t st) {
    const int64_t n = 4 * s->d.N;
    if (s->cfg.precision == 64)
        fixed_to_real_kernel<double><<<grid_for(n, 256), 256, 0, st>>>(s->S64, (double*)s->S, n, s->fix_exp);
    else
        fixed_to_real_kernel<float><<<grid_for(n, 256), 256, 0, st>>>(s->S64, (float*)s->S, n, s->fix_exp);
    GP_CUDA(cudaGetLastError());
    return PIC_OK;
}

int launch_sort(pic_sim* s, cudaStream_t st) {
    return s->cfg.precision == 64 ? sort_typed<double>(s, st) : sort_typed<float>(s, st);
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
