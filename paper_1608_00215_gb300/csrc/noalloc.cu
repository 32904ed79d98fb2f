// Field energy of caller-provided fields without any device allocation.
//
// The two-pass energy reduction needs room for one partial sum per block. The run
// API takes that room from the run's workspace; this entry point instead uses a
// fixed array in the library's own device memory (statically sized, present on
// every device that loads the library until the process exits), so it can be
// called by code that has no device allocator or must not allocate.
#include <mutex>

#include "common.cuh"

namespace galpic {
namespace {

// Partial-sum blocks; inputs of any size up to the cell limit are covered by
// grid-stride loops over at most this many blocks.
constexpr int NOALLOC_BLOCKS = 1024;
constexpr size_t NOALLOC_PART_BYTES = 2 * NOALLOC_BLOCKS * sizeof(double);   // 16 KiB
constexpr int64_t NOALLOC_MAX_CELLS = (int64_t)1 << 30;

// [0, 16 KiB): per-block sums of E^2 and B^2; then one int32 word that receives the
// shared energy launcher's non-finite flag. Nothing reads that word (a non-finite field
// makes W itself non-finite, which is what callers see), so it is never cleared.
static __device__ __align__(256) unsigned char g_energy_scratch[NOALLOC_PART_BYTES + 256];

// Device address of g_energy_scratch per device ordinal (the symbol's name is only a
// host-side stand-in in host code).
constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_addr[MAX_DEVICES];

int scratch_address(void** out) {
    int dev = 0;
    GP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MAX_DEVICES) return fail(PIC_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_energy_scratch);
        if (e != cudaSuccess || !p)
            return fail(PIC_ECUDA, std::string("cudaGetSymbolAddress(energy scratch): ") +
                                       cudaGetErrorString(e));
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return PIC_OK;
}

}  // namespace
}  // namespace galpic

using namespace galpic;

extern "C" int pic_field_energy_noalloc(const void* fields, int64_t n_cells, int precision, double eps0,
                                        double c, double dV, double* out_dev, void* stream) {
    if (!fields || !out_dev) return fail(PIC_EINVAL, "fields or out_dev is NULL");
    if (precision != 32 && precision != 64) return fail(PIC_EINVAL, "precision must be 32 or 64");
    if (n_cells < 1 || n_cells > NOALLOC_MAX_CELLS)
        return fail(PIC_EINVAL, "n_cells must be in [1, 2^30] for the allocation-free energy, got " +
                                    std::to_string(n_cells));
    if (!(eps0 > 0 && c > 0 && dV > 0)) return fail(PIC_EINVAL, "eps0, c and dV must be positive");
    void* scratch = nullptr;
    GP_CHECK(scratch_address(&scratch));
    cudaStream_t st = (cudaStream_t)stream;
    double* part = (double*)scratch;
    int32_t* status = (int32_t*)((char*)scratch + NOALLOC_PART_BYTES);
    int64_t nb = (n_cells + 2047) / 2048;
    if (nb > NOALLOC_BLOCKS) nb = NOALLOC_BLOCKS;
    return launch_energy_on(fields, n_cells, precision, part, (int)nb, status, 0.5 * eps0 * dV,
                            0.5 * eps0 * dV * c * c, out_dev, st);
}
