// double instantiations of the particle pass (pass.cuh).
#include "pass.cuh"

namespace galpic {

int launch_pass_fp64(pic_sim* s, int mode, cudaStream_t st) {
    return mode == PASS_STEP ? pass_margin<double, PASS_STEP>(s, st) : pass_margin<double, PASS_DEPOSIT>(s, st);
}

size_t pass_desc_bytes_fp64() { return sizeof(PassK<double>); }

void fill_pass_desc_fp64(const pic_sim* s, void* out, const void* F, void* S, long long* S64) {
    fill_passk<double>(s, *static_cast<PassK<double>*>(out), F, S, S64);
}

int launch_pass_many_fp64(pic_sim* s0, const void* descs, int nruns, cudaStream_t st) {
    const ManyLaunch m{descs, nruns};
    return pass_margin<double, PASS_STEP>(s0, st, &m);
}

}  // namespace galpic
