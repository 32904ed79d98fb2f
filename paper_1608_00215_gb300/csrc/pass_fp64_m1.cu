// double particle-pass kernels at tile margin 1 (pass.cuh).
#include "pass.cuh"

namespace galpic {

int pass_fp64_margin1(pic_sim* s, int mode, cudaStream_t st, const void* descs, int nruns) {
    const ManyLaunch m{descs, nruns};
    const ManyLaunch* many = descs ? &m : nullptr;
    return mode == PASS_STEP ? pass_order<double, PASS_STEP, 1>(s, st, many)
                             : pass_order<double, PASS_DEPOSIT, 1>(s, st, nullptr);
}

}  // namespace galpic
