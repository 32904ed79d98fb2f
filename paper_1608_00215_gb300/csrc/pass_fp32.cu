// float instantiations of the particle pass (pass.cuh).
#include "pass.cuh"

namespace galpic {

int launch_pass_fp32(pic_sim* s, int mode, cudaStream_t st) {
    return mode == PASS_STEP ? pass_margin<float, PASS_STEP>(s, st) : pass_margin<float, PASS_DEPOSIT>(s, st);
}

size_t pass_desc_bytes_fp32() { return sizeof(PassK<float>); }

void fill_pass_desc_fp32(const pic_sim* s, void* out, const void* F, void* S, long long* S64) {
    fill_passk<float>(s, *static_cast<PassK<float>*>(out), F, S, S64);
}

int launch_pass_many_fp32(pic_sim* s0, const void* descs, int nruns, cudaStream_t st) {
    const ManyLaunch m{descs, nruns};
    return pass_margin<float, PASS_STEP>(s0, st, &m);
}

int pass_variant_of(const pic_sim* s) { return pass_variant(s); }

}  // namespace galpic
