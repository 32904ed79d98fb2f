// double entry points of the particle pass (pass.cuh); the kernels of each tile margin are
// instantiated in pass_fp64_m0.cu and pass_fp64_m1.cu, which compile in parallel.
#include "pass.cuh"

namespace galpic {

int pass_fp64_margin0(pic_sim* s, int mode, cudaStream_t st, const void* descs, int nruns);
int pass_fp64_margin1(pic_sim* s, int mode, cudaStream_t st, const void* descs, int nruns);

static int dispatch(pic_sim* s, int mode, cudaStream_t st, const void* descs, int nruns) {
    return s->d.margin == 0 ? pass_fp64_margin0(s, mode, st, descs, nruns)
                            : pass_fp64_margin1(s, mode, st, descs, nruns);
}

int launch_pass_fp64(pic_sim* s, int mode, cudaStream_t st) { return dispatch(s, mode, st, nullptr, 0); }

size_t pass_desc_bytes_fp64() { return sizeof(PassK<double>); }

void fill_pass_desc_fp64(const pic_sim* s, void* out, const void* F, void* S, long long* S64) {
    fill_passk<double>(s, *static_cast<PassK<double>*>(out), F, S, S64);
}

int launch_pass_many_fp64(pic_sim* s0, const void* descs, int nruns, cudaStream_t st) {
    return dispatch(s0, PASS_STEP, st, descs, nruns);
}

}  // namespace galpic
